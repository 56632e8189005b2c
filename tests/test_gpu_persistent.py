"""The persistent scheduling of the composites (LV_FLAG_PERSISTENT: resident
warps take (tile, strip) items from a global counter) against the default
one-block-per-tile launch and the oracle.  Per pixel both run the same
arithmetic in the same order, so images, transmittance, contribution counts
and w_max are bit-identical; gradients differ only in the order of FP32
atomic additions (1e-4 of the largest, as every gradient)."""
import numpy as np
import pytest
import torch

from gpu_helpers import np_
from paper_2511_02510_gb300 import synth
from paper_2511_02510_gb300.raster import RasterContext
from test_gpu_render import GRAD_TOL, _grad_err, cam_far, cam_near, compare_images

pytestmark = pytest.mark.gpu


def run(sc, cams, tile, persistent, g=None, exact_segment=False, persistent_sms=0, batch=32):
    from gpu_helpers import to_scene
    scene = to_scene(sc)
    ctx = RasterContext(cams, scene.n, tile=tile, persistent=persistent, exact_segment=exact_segment,
                        persistent_sms=persistent_sms, batch=batch)
    vox = scene.voxels()
    ctx.fit_capacity(vox)
    ctx.reset_stats()
    ctx.forward(vox)
    out = {k: np_(getattr(ctx, k)).copy() for k in ("rgb", "T", "depth", "n_contrib", "wmax_packed")}
    if g is not None:
        dd, ds = ctx.backward(vox, torch.from_numpy(g).cuda())
        torch.cuda.synchronize()
        out["dd"], out["ds"] = np_(dd), np_(ds)
    ctx.check()
    return out, ctx


@pytest.mark.parametrize("tile,seg", [(8, False), (16, False), (32, False), (16, True)])
def test_persistent_equals_default_and_oracle(ora, tile, seg):
    sc = synth.scene_tiny()
    cams = [cam_near(100, 70, az=80.0), cam_far(64, 48, az=200.0)]
    P = sum(c["width"] * c["height"] for c in cams)
    g = np.random.default_rng(tile).normal(size=(P, 3)).astype(np.float32)
    a, _ = run(sc, cams, tile, False, g, seg)
    b, ctx = run(sc, cams, tile, True, g, seg)
    for k in ("rgb", "T", "depth", "n_contrib", "wmax_packed"):
        np.testing.assert_array_equal(a[k], b[k])
    assert _grad_err(b["dd"], a["dd"]) < GRAD_TOL and _grad_err(b["ds"], a["ds"]) < GRAD_TOL
    compare_images(ora.render(sc, cams, segment=seg), ctx)


def test_persistent_full_size_view():
    sc = synth.scene_360()
    cam = synth.orbit_camera(1237, 822, 60.0, 3.0, 37.0, 15.0)
    g = np.random.default_rng(0).normal(size=(1237 * 822, 3)).astype(np.float32) * 1e-3
    a, _ = run(sc, [cam], 16, False, g)
    b, _ = run(sc, [cam], 16, True, g)
    for k in ("rgb", "T", "depth", "n_contrib", "wmax_packed"):
        np.testing.assert_array_equal(a[k], b[k])
    assert _grad_err(b["dd"], a["dd"]) < GRAD_TOL and _grad_err(b["ds"], a["ds"]) < GRAD_TOL


@pytest.mark.parametrize("sms", [1, 7, 120])
def test_persistent_on_fewer_sms(sms):
    """persistent_sms only sizes the resident grid: the same bits on any SM count."""
    sc = synth.scene_tiny()
    cams = [cam_near(100, 70, az=80.0), cam_far(64, 48, az=200.0)]
    P = sum(c["width"] * c["height"] for c in cams)
    g = np.random.default_rng(sms).normal(size=(P, 3)).astype(np.float32)
    a, _ = run(sc, cams, 32, True, g)
    b, _ = run(sc, cams, 32, True, g, persistent_sms=sms)
    for k in ("rgb", "T", "depth", "n_contrib", "wmax_packed"):
        np.testing.assert_array_equal(a[k], b[k])
    assert _grad_err(b["dd"], a["dd"]) < GRAD_TOL and _grad_err(b["ds"], a["ds"]) < GRAD_TOL


@pytest.mark.parametrize("tile,persistent,seg", [(8, False, False), (16, True, False), (32, True, False),
                                                 (16, False, True)])
def test_batches_give_the_same_bits(ora, tile, persistent, seg):
    """The batch (list entries a warp stages per round) only groups the loads: every batch gives the
    bits of batch 32, and the oracle's image."""
    sc = synth.scene_tiny()
    cams = [cam_near(100, 70, az=80.0), cam_far(64, 48, az=200.0)]
    P = sum(c["width"] * c["height"] for c in cams)
    g = np.random.default_rng(tile).normal(size=(P, 3)).astype(np.float32)
    a, _ = run(sc, cams, tile, persistent, g, seg, batch=32)
    for batch in (64, 128) if tile < 32 else (64,):
        b, ctx = run(sc, cams, tile, persistent, g, seg, batch=batch)
        for k in ("rgb", "T", "depth", "n_contrib", "wmax_packed"):
            np.testing.assert_array_equal(a[k], b[k])
        assert _grad_err(b["dd"], a["dd"]) < 1e-5 and _grad_err(b["ds"], a["ds"]) < 1e-5
    compare_images(ora.render(sc, cams, segment=seg), ctx)
