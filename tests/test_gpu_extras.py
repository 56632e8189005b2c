"""GPU checks beyond the core parity tests: FP64 finite differences on the GPU,
the autograd wrapper, the tile autotuner and CUDA-graph capture."""
import numpy as np
import pytest
import torch

from gpu_helpers import gpu_forward, np_, to_scene
from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth
from paper_2511_02510_gb300.raster import CapturedStep, RasterContext, autotune_tile, rasterize

pytestmark = pytest.mark.gpu


def cam_near(W=64, H=64, az=30.0):
    return synth.orbit_camera(W, H, 60.0, 1.6, az, 25.0, target=(0.5, 0.4, 0.5))


def f64_render(scene, ctx, pixels):
    rgb = torch.zeros((pixels.numel(), 3), dtype=torch.float64, device="cuda")
    T = torch.zeros(pixels.numel(), dtype=torch.float64, device="cuda")
    L.lv_render_pixels_f64(scene.voxels(), ctx.cams_arr, ctx.n_views, ctx.opts, ctx.workspace, ctx.pair_capacity,
                           pixels, rgb, T)
    torch.cuda.synchronize()
    return rgb, T


def test_fp64_rerender_matches_oracle(ora):
    sc = synth.scene_tiny()
    cams = [cam_near()]
    scene, ctx, vox = gpu_forward(sc, cams)
    px = torch.arange(ctx.n_pix, dtype=torch.int64, device="cuda")
    rgb, T = f64_render(scene, ctx, px)
    r = ora.render(sc, cams)
    # same FP64 arithmetic on both sides: agreement far below any FP32 tolerance
    assert np.abs(np_(rgb) - r["rgb"]).max() < 1e-10
    assert np.abs(np_(T) - r["T"]).max() < 1e-10


def test_fp64_gpu_finite_differences_of_backward():
    # Central differences of the FP64 GPU re-render against the FP32 analytic backward.
    sc = synth.scene_tiny()
    cams = [cam_near(48, 48)]
    scene, ctx, vox = gpu_forward(sc, cams)
    rng = np.random.default_rng(21)
    g = torch.from_numpy(rng.normal(size=(ctx.n_pix, 3))).cuda()
    d_dens, d_sh = ctx.backward(vox, g.float())
    torch.cuda.synchronize()
    w, a = ctx.unpack_wmax()
    hit = np.where(np_(a) >= 0)[0]
    px = torch.arange(ctx.n_pix, dtype=torch.int64, device="cuda")

    def loss():
        rgb, _ = f64_render(scene, ctx, px)
        return float((rgb * g).sum())

    gd, gs = np_(d_dens), np_(d_sh)
    scale_d, scale_s = np.abs(gd).max(), np.abs(gs).max()
    ok = total = 0
    for v in rng.choice(hit, size=10, replace=False):
        for kind, idx in (("density", int(rng.integers(8))), ("sh", int(rng.integers(48)))):
            arr = scene.density if kind == "density" else scene.sh
            x0 = float(arr[v, idx])
            h = 1e-3 * max(1.0, abs(x0))
            vals = []
            for sgn in (1, -1):
                arr[v, idx] = x0 + sgn * h
                actual = float(arr[v, idx]) - x0
                vals.append((actual, loss()))
            arr[v, idx] = x0
            fd = (vals[0][1] - vals[1][1]) / (vals[0][0] - vals[1][0])
            an = float((gd if kind == "density" else gs)[v, idx])
            scale = scale_d if kind == "density" else scale_s
            total += 1
            if abs(fd - an) <= 1e-4 * scale + 1e-3 * abs(fd):
                ok += 1
    # kinks (ReLU, colour clamp, stop rule) inside the step can spoil a few differences
    assert ok >= total - 3, (ok, total)


def test_autograd_function_matches_direct_backward():
    sc = synth.scene_tiny()
    cams = [cam_near()]
    scene = to_scene(sc)
    ctx = RasterContext(cams, scene.n)
    ctx.fit_capacity(scene.voxels())
    density = scene.density.clone().requires_grad_(True)
    sh = scene.sh.clone().requires_grad_(True)
    rng = np.random.default_rng(3)
    gC = torch.from_numpy(rng.normal(size=(ctx.n_pix, 3)).astype(np.float32)).cuda()
    gT = torch.from_numpy(rng.normal(size=ctx.n_pix).astype(np.float32)).cuda()
    ctx.reset_stats()
    rgb, depth, T = rasterize(density, sh, scene, ctx)
    ((rgb * gC).sum() + (T * gT).sum()).backward()
    dd, ds = ctx.backward(scene.voxels(), gC, None, gT)
    torch.cuda.synchronize()
    assert torch.allclose(density.grad, dd, rtol=1e-5, atol=1e-7 * float(dd.abs().max()))
    assert torch.allclose(sh.grad, ds, rtol=1e-5, atol=1e-7 * float(ds.abs().max()))


def test_autotune_picks_a_valid_tile(tmp_path):
    sc = synth.scene_tiny()
    scene = to_scene(sc)
    cams = [cam_near(160, 120)]
    path = str(tmp_path / "tune.json")
    best, times = autotune_tile(scene, cams, steps=2, cache_path=path)
    assert best in (8, 16, 32) and set(times) == {8, 16, 32}
    assert best == min(times, key=times.get)
    again, times2 = autotune_tile(scene, cams, steps=2, cache_path=path)   # served from the cache
    assert again == best and times2 == times


def test_captured_step_replays_the_same_result():
    sc = synth.scene_tiny()
    cams = [cam_near(96, 80)]
    scene = to_scene(sc)
    ctx = RasterContext(cams, scene.n)
    vox = scene.voxels()
    ctx.fit_capacity(vox)
    g = torch.full((ctx.n_pix, 3), 1e-2, device="cuda")
    dd = torch.empty((scene.n, 8), device="cuda")
    ds = torch.empty((scene.n, 48), device="cuda")

    def step():
        ctx.reset_stats()
        ctx.forward(vox)
        ctx.backward(vox, g, d_density=dd, d_sh=ds)

    step()
    torch.cuda.synchronize()
    rgb0, dd0, wm0 = ctx.rgb.clone(), dd.clone(), ctx.wmax_packed.clone()
    graph = CapturedStep(step)
    ctx.rgb.zero_()
    dd.zero_()
    graph()
    torch.cuda.synchronize()
    assert torch.equal(ctx.rgb, rgb0)
    assert torch.equal(ctx.wmax_packed, wm0)
    assert torch.allclose(dd, dd0, rtol=1e-5, atol=1e-7 * float(dd0.abs().max()))
