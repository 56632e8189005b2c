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


def test_fp64_gpu_finite_differences_of_backward(ora):
    # Central differences of the FP64 GPU re-render (the finite-difference checker) of
    # L = sum(g . rgb), per corner density and SH coefficient:
    #  - against the oracle's FP64 reverse pass: 1e-6 relative (both are FP64; the step's
    #    truncation and rounding are far below that);
    #  - against the FP32 GPU backward: 1e-4 relative plus the oracle's FP32 floor of that element.
    # Entries whose step could cross a kink (sigma_raw = 0, the colour clamp, a stop decision) are
    # found from the oracle's per-sample trace (fd_margins) and skipped; every other entry must pass.
    sc = synth.scene_tiny()
    cams = [cam_near(48, 48)]
    scene, ctx, vox = gpu_forward(sc, cams)
    r = ora.render(sc, cams)
    rng = np.random.default_rng(21)
    g64 = rng.normal(size=(ctx.n_pix, 3))
    g64[r["near_stop"] != 0] = 0
    g = torch.from_numpy(g64).cuda()
    d_dens, d_sh = ctx.backward(vox, g.float())
    torch.cuda.synchronize()
    ref = ora.render_backward(sc, cams, g64)
    bnd = ora.backward_bounds(sc, cams, g64)
    marg = ora.fd_margins(sc, cams)
    px = torch.arange(ctx.n_pix, dtype=torch.int64, device="cuda")

    def loss():
        rgb, _ = f64_render(scene, ctx, px)
        return float((rgb * g).sum())

    gd, gs = np_(d_dens), np_(d_sh)
    hit = np.where(np.isfinite(marg["m_sigma"]))[0]
    checked = skipped = 0
    worst = {"fd_vs_oracle": 0.0, "fd_vs_gpu_over_tol": 0.0}
    for v in rng.choice(hit, size=24, replace=False):
        for kind in ("density", "sh"):
            if kind == "density":
                idx = int(rng.integers(8))
                arr, x0 = scene.density, float(scene.density[v, idx])
            else:
                idx = int(rng.integers(48))
                arr, x0 = scene.sh, float(scene.sh[v, idx])
            h = 1e-4 * max(1.0, abs(x0))
            margin = min(marg["m_sigma"][v], marg["m_stop"][v]) if kind == "density" else \
                marg["m_color"][v, idx % 3] / 1.2
            if not margin > 20 * h:
                skipped += 1
                continue
            vals = []
            for sgn in (1, -1):
                arr[v, idx] = x0 + sgn * h
                actual = float(arr[v, idx]) - x0
                vals.append((actual, loss()))
            arr[v, idx] = x0
            fd = (vals[0][1] - vals[1][1]) / (vals[0][0] - vals[1][0])
            if kind == "density":
                an64, an32, e = ref["d_density"][v, idx], gd[v, idx], bnd["e_density"][v, idx]
            else:
                an64, an32, e = ref["d_sh"][v, idx], gs[v, idx], bnd["e_sh"][v, idx]
            checked += 1
            assert abs(fd - an64) <= 1e-6 * abs(an64) + 1e-9, (kind, v, idx, fd, an64)
            tol = 1e-4 * abs(fd) + e
            assert abs(fd - an32) <= tol, (kind, v, idx, fd, an32, e)
            worst["fd_vs_oracle"] = max(worst["fd_vs_oracle"], abs(fd - an64) / max(abs(an64), 1e-30))
            worst["fd_vs_gpu_over_tol"] = max(worst["fd_vs_gpu_over_tol"], abs(fd - an32) / tol)
    print(f"FD checker: {checked} entries checked, {skipped} skipped at kinks, worst {worst}")
    assert checked >= 36


def test_autograd_function_matches_oracle(ora):
    # Gradients returned by the torch.autograd.Function (rgb, depth and T losses) against the
    # oracle's reverse pass of Eq. 2-4, element by element (tests/parity.py: check_grads).
    from test_gpu_render import _loss_grads, grad_parity
    sc = synth.scene_tiny()
    cams = [cam_near(72, 56), cam_near(40, 48, az=170.0)]
    scene = to_scene(sc)
    ctx = RasterContext(cams, scene.n)
    ctx.fit_capacity(scene.voxels())
    density = scene.density.clone().requires_grad_(True)
    sh = scene.sh.clone().requires_grad_(True)
    r = ora.render(sc, cams)
    gC, gD, gT = _loss_grads(ctx.n_pix, 12, r["near_stop"])
    ctx.reset_stats()
    rgb, depth, T = rasterize(density, sh, scene, ctx)
    ok = r["near_stop"] == 0
    assert np.abs(np_(rgb)[ok] - r["rgb"][ok]).max() <= 1e-5 + r["bound_rgb"][ok].max()
    loss = (rgb * torch.from_numpy(gC).cuda()).sum() + (depth * torch.from_numpy(gD).cuda()).sum() + \
        (T * torch.from_numpy(gT).cuda()).sum()
    loss.backward()
    torch.cuda.synchronize()
    grad_parity(ora, sc, cams, density.grad, sh.grad, gC, gD, gT)


def test_autograd_refuses_a_stale_context():
    # A second forward on the same context overwrites the sorted lists the first pass's backward needs.
    sc = synth.scene_tiny()
    cams = [cam_near()]
    scene = to_scene(sc)
    ctx = RasterContext(cams, scene.n)
    ctx.fit_capacity(scene.voxels())
    density = scene.density.clone().requires_grad_(True)
    sh = scene.sh.clone().requires_grad_(True)
    rgb1, _, _ = rasterize(density, sh, scene, ctx)
    rgb2, _, _ = rasterize(density, sh, scene, ctx)
    with pytest.raises(RuntimeError, match="another forward"):
        rgb1.sum().backward()
    rgb2.sum().backward()          # the latest pass still has its lists
    assert density.grad is not None and torch.isfinite(density.grad).all()


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
