"""GPU parity of the exact-segment-integration density variant
(LV_FLAG_EXACT_SEGMENT: a sample's density is the mean of the trilinear field
over the chord) against the oracle's same variant: images, w_max, gradients,
the FP64 re-render, and the full-size workload on sampled crops.  Tolerances
as for the midpoint reading (per-pixel FP32 sensitivity bound; w_max argmax
within the oracle's near-max set; every gradient element within 1e-4 relative
plus the oracle's FP32 floor)."""
import numpy as np
import pytest
import torch

from gpu_helpers import dequantized, gpu_forward, np_
from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth
from test_gpu_render import _loss_grads, cam_far, cam_near, compare_images, compare_wmax, grad_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    return synth.scene_tiny()


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_segment_forward_parity(ora, tiny, tile):
    cams = [cam_near(100, 70, az=80.0), cam_far(64, 48, az=200.0)]
    scene, ctx, vox = gpu_forward(tiny, cams, tile=tile, exact_segment=True)
    r = ora.render(tiny, cams, segment=True)
    compare_images(r, ctx)
    compare_wmax(ora, tiny, cams, r, ctx, segment=True)
    # and it is a different model from the midpoint reading on this scene
    m = ora.render(tiny, cams)
    assert np.abs(m["rgb"] - r["rgb"]).max() > 1e-3


@pytest.mark.parametrize("cfg", ["fp32", "mixed"])
def test_segment_backward_parity(ora, tiny, cfg):
    dd, sd = (torch.float32, torch.float32) if cfg == "fp32" else (torch.float16, torch.bfloat16)
    cams = [cam_near(80, 60)]
    scene, ctx, vox = gpu_forward(tiny, cams, density_dtype=dd, sh_dtype=sd, exact_segment=True)
    ref_scene = dequantized(tiny, dd, sd)
    r = ora.render(ref_scene, cams, segment=True)
    gC, gD, gT = _loss_grads(ctx.n_pix, 4, r["near_stop"])
    d_dens, d_sh = ctx.backward(vox, torch.from_numpy(gC).cuda(), torch.from_numpy(gD).cuda(),
                                torch.from_numpy(gT).cuda())
    torch.cuda.synchronize()
    grad_parity(ora, ref_scene, cams, d_dens, d_sh, gC, gD, gT, segment=True)


def test_segment_fp64_rerender(ora, tiny):
    cams = [cam_near(64, 64)]
    scene, ctx, vox = gpu_forward(tiny, cams, exact_segment=True)
    px = torch.arange(ctx.n_pix, dtype=torch.int64, device="cuda")
    rgb = torch.zeros((ctx.n_pix, 3), dtype=torch.float64, device="cuda")
    T = torch.zeros(ctx.n_pix, dtype=torch.float64, device="cuda")
    L.lv_render_pixels_f64(vox, ctx.cams_arr, ctx.n_views, ctx.opts, ctx.workspace, ctx.pair_capacity, px, rgb, T)
    torch.cuda.synchronize()
    r = ora.render(tiny, cams, segment=True)
    assert np.abs(np_(rgb) - r["rgb"]).max() < 1e-10
    assert np.abs(np_(T) - r["T"]).max() < 1e-10


def test_segment_full_size_crops(ora):
    # the 2M-voxel bench scene and view: the variant's GPU image on three crops against the oracle
    sc = synth.scene_360()
    cam = synth.orbit_camera(1237, 822, 60.0, 3.0, 37.0, 15.0)
    scene, ctx, vox = gpu_forward(sc, [cam], exact_segment=True)
    rgb, T, depth = np_(ctx.rgb), np_(ctx.T), np_(ctx.depth)
    for (x0, y0) in ((600, 400), (100, 700), (1150, 60)):
        crop = [x0, y0, x0 + 24, y0 + 24]
        r = ora.render(sc, [cam], crop=crop, segment=True)
        mask = np.zeros(ctx.n_pix, bool)
        yy, xx = np.mgrid[y0:y0 + 24, x0:x0 + 24]
        mask[(yy * 1237 + xx).ravel()] = True
        compare_images(r, ctx, rgb=rgb, T=T, depth=depth, mask=mask)
