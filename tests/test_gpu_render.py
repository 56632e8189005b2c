"""GPU parity of the rasterizer (forward, w_max, statistics, pair lists,
backward) against the CPU oracle, through the C ABI.

Tolerances (from the arithmetic; tests/parity.py states the rules):
 - images: within 1e-5 max-abs of the FP64 oracle, plus the oracle's per-pixel
   FP32 sensitivity bound (a chord's length moves with sub-ulp shifts of the
   ray at grazing incidence and at large distances); pixels whose bound is
   below 1e-6 must meet 1e-5 outright, and the mean error stays below 2e-6;
 - w_max: for every voxel, the oracle's argmax unless the oracle's near-max set
   shows FP32 rounding can reorder the top weights (then a member of that
   set, with that member's weight);
 - integer outputs (pair lists, tile ranges, seen, FP32-pinned statistics):
   bit-exact;
 - gradients: every element within 1e-4 of the oracle's, relative, plus the
   oracle's FP32 floor of that element (rounding of the reverse pass, the
   order of the atomic sums, FP32 geometry); relative L2 error within 1e-5.
"""

import numpy as np
import pytest
import torch

from gpu_helpers import dequantized, gpu_forward, gpu_pairs, np_
from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth
from parity import check_grads, check_wmax

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5
GRAD_TOL = 1e-4
U32 = 2.0 ** -24


def cam_far(W=128, H=128, az=30.0):
    return synth.orbit_camera(W, H, 60.0, 3.0, az, 20.0, target=(0.5, 0.5, 0.5))


def cam_near(W=128, H=128, az=30.0, el=25.0, r=1.6):
    return synth.orbit_camera(W, H, 60.0, r, az, el, target=(0.5, 0.4, 0.5))


@pytest.fixture(scope="module")
def tiny():
    return synth.scene_tiny()


def compare_images(ora_r, ctx, tol=IMG_TOL, rgb=None, T=None, depth=None, mask=None):
    ok = ora_r["near_stop"] == 0
    if mask is not None:
        ok &= mask
    assert ok.sum() > 0.99 * (mask.sum() if mask is not None else ok.size)
    rgb = np_(ctx.rgb) if rgb is None else rgb
    T = np_(ctx.T) if T is None else T
    depth = np_(ctx.depth) if depth is None else depth
    e_rgb = np.abs(rgb - ora_r["rgb"]).max(axis=1)
    e_T = np.abs(T - ora_r["T"])
    e_d = np.abs(depth - ora_r["depth"])
    dscale = max(1.0, float(np.abs(ora_r["depth"]).max()))
    # every pixel within 1e-5 plus its FP32 sensitivity bound
    assert np.all(e_rgb[ok] <= tol + ora_r["bound_rgb"][ok]), (e_rgb - ora_r["bound_rgb"])[ok].max()
    assert np.all(e_T[ok] <= tol + ora_r["bound_T"][ok]), (e_T - ora_r["bound_T"])[ok].max()
    assert np.all(e_d[ok] <= tol * dscale + ora_r["bound_depth"][ok])
    # well-conditioned pixels meet 1e-5 outright, and the typical error is far below it
    well = ok & (ora_r["bound_rgb"] < 1e-6) & (ora_r["bound_T"] < 1e-6)
    if well.any():
        assert e_rgb[well].max() < tol and e_T[well].max() < tol
    assert e_rgb[ok].mean() < 0.2 * tol and e_T[ok].mean() < 0.2 * tol
    return float(e_rgb[ok].max()), float(e_T[ok].max())


def image_report(ora_r, ctx, mask=None, tol=IMG_TOL):
    """How many checked pixels needed their FP32 sensitivity bound (error above 1e-5), and the
    largest bound among the checked pixels."""
    ok = ora_r["near_stop"] == 0
    if mask is not None:
        ok &= mask
    e_rgb = np.abs(np_(ctx.rgb) - ora_r["rgb"]).max(axis=1)
    e_T = np.abs(np_(ctx.T) - ora_r["T"])
    need = ok & ((e_rgb > tol) | (e_T > tol))
    return {"pixels": int(ok.sum()), "needed_bound": int(need.sum()),
            "max_bound_rgb": float(ora_r["bound_rgb"][ok].max(initial=0.0)),
            "max_bound_T": float(ora_r["bound_T"][ok].max(initial=0.0)),
            "max_err_rgb": float(e_rgb[ok].max(initial=0.0)), "max_err_T": float(e_T[ok].max(initial=0.0))}


def compare_wmax(ora, sc, cams, ora_r, ctx, segment=False):
    """Every voxel's w_max and argmax against the oracle's (tests/parity.py: check_wmax)."""
    w, a = ctx.unpack_wmax()
    ws = ora.wmax_sets(sc, cams, segment=segment)
    rep = check_wmax(np_(w), np_(a), ws, ora_r["near_stop"])
    print("w_max:", rep)
    return rep


def grad_parity(ora, sc, cams, d_dens, d_sh, gC, gD=None, gT=None, crop=None, segment=False, times=1):
    """Per-element gradient parity (tests/parity.py: check_grads) of d_dens / d_sh against
    `times` x the oracle's gradients of sum(gC.rgb + gD depth + gT T)."""
    f = lambda x: None if x is None else np.asarray(x, np.float64)
    ref = ora.render_backward(sc, cams, f(gC), f(gD), f(gT), crop=crop, segment=segment)
    e = ora.backward_bounds(sc, cams, f(gC), f(gD), f(gT), crop=crop, segment=segment)
    reps = {}
    for k, g, ek, ak in (("d_density", d_dens, "e_density", "a_density"), ("d_sh", d_sh, "e_sh", "a_sh")):
        r = times * ref[k]
        # a sum of `times` passes: each pass within its floor, plus one rounding per added pass
        reps[k] = check_grads(k, np_(g) if torch.is_tensor(g) else g, r, times * e[ek] + (times - 1) * U32 * np.abs(r),
                              times * e[ak] + (times - 1) * U32 * np.abs(r))
    print("gradients:", reps)
    return reps


@pytest.mark.parametrize("which", ["far", "near"])
def test_forward_parity_tiny(ora, tiny, which):
    cams = [cam_far()] if which == "far" else [cam_near()]
    scene, ctx, vox = gpu_forward(tiny, cams)
    r = ora.render(tiny, cams)
    compare_images(r, ctx)
    compare_wmax(ora, tiny, cams, r, ctx)


@pytest.mark.parametrize("radius,az,W", [(1.2, 30.0, 48), (1.3, 50.0, 40)])
def test_wmax_ties_on_a_saturated_voxel(ora, radius, az, W):
    # One voxel so dense that every ray crossing it with optical depth above 18 gets alpha = 1.0 exactly
    # in FP32 (1 - e^-18 rounds to 1), all at T = 1: those weights tie exactly, and the argmax of Eq. 5
    # must take the smallest pixel id among them.  The oracle's FP64 weights do not tie (its argmax is the
    # longest chord), so the expected pixel comes from the per-ray optical depths of its trace; no ray
    # with a smaller id may sit where FP32 saturation is uncertain (16 < x <= 18).
    sc = synth.constant_voxel_scene([[0.5, 0.5, 0.5]], 0.2, [1e4], [(1, 1, 1)])
    cam = synth.orbit_camera(W, W, 60.0, radius, az, 25.0, target=(0.5, 0.4, 0.5))
    x = {}
    for y in range(W):
        for xx in range(W):
            tr = ora.trace_pixel(sc, cam, xx, y, sh_degree=0)
            if tr["n"] > 0:
                x[y * W + xx] = 1e4 * tr["l"][0]
    sat = min(p for p, v in x.items() if v > 18.0)
    assert all(p > sat for p, v in x.items() if 16.0 < v <= 18.0)
    scene, ctx, vox = gpu_forward(sc, [cam], sh_degree=0)
    w, a = ctx.unpack_wmax()
    assert float(w[0]) == 1.0 and int(a[0]) == sat


def test_pairs_and_stats_bit_exact(ora, tiny):
    cams = [cam_near(), cam_near(96, 72, az=150.0), cam_far(70, 50, az=250.0)]
    scene, ctx, vox = gpu_forward(tiny, cams)
    keys, vox_ids, ranges, pairs = gpu_pairs(ctx, scene.n)
    ref = ora.pairs(tiny, cams, ts=16)
    assert pairs == ref["n_pairs"]
    np.testing.assert_array_equal(keys, ref["keys"])
    np.testing.assert_array_equal(vox_ids, ref["vals"])
    np.testing.assert_array_equal(ranges, ref["ranges"])
    np.testing.assert_array_equal(np_(ctx.seen), ref["seen"])
    np.testing.assert_array_equal(np_(ctx.z_min).view(np.uint32), ref["z_min"].view(np.uint32))
    np.testing.assert_array_equal(np_(ctx.delta_min).view(np.uint32), ref["delta_min"].view(np.uint32))


@pytest.mark.parametrize("tile,batch", [(8, 64), (16, 128), (32, 32), (32, 64), (8, 128), (16, 32)])
def test_forward_tiles_batches_ragged(ora, tiny, tile, batch):
    cams = [cam_near(100, 70, az=80.0), cam_near(37, 53, az=200.0, el=40.0)]
    scene, ctx, vox = gpu_forward(tiny, cams, tile=tile, batch=batch)
    r = ora.render(tiny, cams)
    compare_images(r, ctx)
    keys, vox_ids, ranges, pairs = gpu_pairs(ctx, scene.n)
    ref = ora.pairs(tiny, cams, ts=tile)
    np.testing.assert_array_equal(keys, ref["keys"])
    np.testing.assert_array_equal(vox_ids, ref["vals"])


def test_mixed_precision_storage(ora, tiny):
    cams = [cam_near(), cam_near(64, 48, az=300.0)]
    scene, ctx, vox = gpu_forward(tiny, cams, density_dtype=torch.float16, sh_dtype=torch.bfloat16)
    ref_scene = dequantized(tiny, torch.float16, torch.bfloat16)
    r = ora.render(ref_scene, cams)
    e_rgb, e_T = compare_images(r, ctx)
    compare_wmax(ora, ref_scene, cams, r, ctx)
    w, _ = ctx.unpack_wmax()
    hit = r["w_arg"] >= 0
    print("mixed-precision storage, tiny scene: rgb", e_rgb, "T", e_T, "w_max",
          float(np.abs(np_(w)[hit] - r["w_max"][hit]).max()))


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_sh_degrees(ora, tiny, deg):
    cams = [cam_near(64, 64)]
    scene, ctx, vox = gpu_forward(tiny, cams, sh_degree=deg)
    r = ora.render(tiny, cams, sh_degree=deg)
    compare_images(r, ctx)


def _loss_grads(P, seed, near_stop):
    rng = np.random.default_rng(seed)
    gC = rng.normal(size=(P, 3)).astype(np.float32)
    gD = (0.1 * rng.normal(size=P)).astype(np.float32)
    gT = rng.normal(size=P).astype(np.float32)
    # pixels whose stop decision is within rounding of t_stop are excluded
    gC[near_stop == 1] = 0
    gD[near_stop == 1] = 0
    gT[near_stop == 1] = 0
    return gC, gD, gT


def _grad_err(g, ref):
    """Largest error relative to the largest magnitude (for GPU-against-GPU comparisons, where the
    two sides differ only in the order of their atomic sums)."""
    scale = np.abs(ref).max()
    return np.abs(g - ref).max() / max(scale, 1e-30)


@pytest.mark.parametrize("cfg", ["near16", "multi8", "mixed32"])
def test_backward_parity(ora, tiny, cfg):
    if cfg == "near16":
        cams, tile, dd, sd = [cam_near()], 16, torch.float32, torch.float32
    elif cfg == "multi8":
        cams, tile, dd, sd = [cam_near(80, 60), cam_far(64, 64, az=120.0)], 8, torch.float32, torch.float32
    else:
        cams, tile, dd, sd = [cam_near(90, 90, az=250.0)], 32, torch.float16, torch.bfloat16
    scene, ctx, vox = gpu_forward(tiny, cams, tile=tile, density_dtype=dd, sh_dtype=sd)
    ref_scene = dequantized(tiny, dd, sd)
    r = ora.render(ref_scene, cams)
    P = ctx.n_pix
    gC, gD, gT = _loss_grads(P, 3, r["near_stop"])
    d_dens, d_sh = ctx.backward(vox, torch.from_numpy(gC).cuda(), torch.from_numpy(gD).cuda(),
                                torch.from_numpy(gT).cuda())
    torch.cuda.synchronize()
    grad_parity(ora, ref_scene, cams, d_dens, d_sh, gC, gD, gT)
    # accumulate = True adds onto existing gradients
    d2, s2 = ctx.backward(vox, torch.from_numpy(gC).cuda(), torch.from_numpy(gD).cuda(), torch.from_numpy(gT).cuda(),
                          d_density=d_dens.clone(), d_sh=d_sh.clone(), accumulate=True)
    torch.cuda.synchronize()
    grad_parity(ora, ref_scene, cams, d2, s2, gC, gD, gT, times=2)


def test_backward_matches_fd_of_gpu_forward(tiny):
    # Central differences of the GPU forward itself (FP32, larger steps) agree with the GPU backward.
    cams = [cam_near(48, 48)]
    scene, ctx, vox = gpu_forward(tiny, cams)
    rng = np.random.default_rng(9)
    P = ctx.n_pix
    gC = torch.from_numpy(rng.normal(size=(P, 3)).astype(np.float32)).cuda()
    d_dens, d_sh = ctx.backward(vox, gC)
    w, a = ctx.unpack_wmax()
    hit = np.where(np_(a) >= 0)[0]
    pick = rng.choice(hit, size=8, replace=False)

    def loss():
        ctx.forward(scene.voxels(), stats=False)
        return float((ctx.rgb.double() * gC.double()).sum())

    n_ok = 0
    for v in pick:
        i = int(rng.integers(8))
        x0 = float(scene.density[v, i])
        h = 1e-2
        scene.density[v, i] = x0 + h
        lp = loss()
        scene.density[v, i] = x0 - h
        lm = loss()
        scene.density[v, i] = x0
        fd = (lp - lm) / (2 * h)
        an = float(d_dens[v, i])
        if abs(fd - an) <= 2e-2 * max(abs(fd), abs(an), 1e-3):
            n_ok += 1
    assert n_ok >= 6


def test_empty_and_culled(ora):
    empty = synth.constant_voxel_scene(np.zeros((0, 3)), 0.1, np.zeros(0), np.zeros((0, 3)))
    cams = [cam_near(40, 30)]
    scene, ctx, vox = gpu_forward(empty, cams, pair_capacity=16)
    assert np.all(np_(ctx.rgb) == 0) and np.all(np_(ctx.T) == 1)
    # everything behind the camera
    sc = synth.constant_voxel_scene([[0.5, 0.5, 0.5]], 0.2, [3.0], [(1, 1, 1)])
    cam = synth.look_at_camera([0.5, 0.5, 2.0], [0.5, 0.5, 5.0], 32, 32, 60.0)
    scene, ctx, vox = gpu_forward(sc, [cam], pair_capacity=16)
    assert np.all(np_(ctx.T) == 1) and int(np_(ctx.seen)[0]) == 0
    # a voxel straddling the near plane covers the whole image and still matches the oracle
    cam = synth.look_at_camera([0.5, 0.5, 0.45], [0.5, 0.5, 5.0], 24, 20, 60.0)
    scene, ctx, vox = gpu_forward(sc, [cam])
    r = ora.render(sc, [cam])
    compare_images(r, ctx)


def test_capacity_overflow_reported(tiny):
    from gpu_helpers import to_scene
    from paper_2511_02510_gb300.raster import RasterContext
    cams = [cam_near()]
    scene = to_scene(tiny)
    ctx = RasterContext(cams, scene.n, pair_capacity=100)           # far too small
    vox = scene.voxels()
    opts = L.make_opts(16, 32, 1e-4, sync_check=True)
    with pytest.raises(L.LvError) as ei:
        L.lv_rasterize_forward(vox, ctx.cams_arr, 1, opts, ctx.fwd_struct(), ctx.workspace, 100, None)
    assert ei.value.status == L.LV_ERR_CAPACITY
    pairs, _ = ctx.counters()
    assert pairs > 100


def test_invalid_arguments_rejected(tiny):
    cams = [cam_near()]
    scene, ctx, vox = gpu_forward(tiny, cams)
    bad = L.make_opts(12, 256)
    with pytest.raises(L.LvError) as ei:
        L.lv_rasterize_forward(vox, ctx.cams_arr, 1, bad, ctx.fwd_struct(), ctx.workspace, ctx.pair_capacity)
    assert ei.value.status == L.LV_ERR_INVALID_ARG
    small = ctx.workspace[:1024]
    with pytest.raises(L.LvError) as ei:
        L.lv_rasterize_forward(vox, ctx.cams_arr, 1, ctx.opts, ctx.fwd_struct(), small, ctx.pair_capacity)
    assert ei.value.status == L.LV_ERR_WORKSPACE


def test_deterministic_integer_outputs(tiny):
    cams = [cam_near(), cam_near(72, 40, az=10.0)]
    a = gpu_forward(tiny, cams)[1]
    ka, va, ra, _ = gpu_pairs(a, tiny["geom"].shape[0])
    wa = np_(a.wmax_packed).copy()
    b = gpu_forward(tiny, cams)[1]
    kb, vb, rb, _ = gpu_pairs(b, tiny["geom"].shape[0])
    np.testing.assert_array_equal(ka, kb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(wa, np_(b.wmax_packed))
    np.testing.assert_array_equal(np_(a.n_contrib), np_(b.n_contrib))


@pytest.fixture(scope="module")
def full360(ora):
    """The 2M-voxel 360 scene and its 1237x822 view, with the oracle's whole-view render and w_max sets."""
    sc = synth.scene_360()
    cam = synth.orbit_camera(1237, 822, 60.0, 3.0, 37.0, 15.0)
    return sc, cam, ora.render(sc, [cam]), ora.wmax_sets(sc, [cam])


@pytest.mark.slow
@pytest.mark.parametrize("tile,persistent", [(16, False), (32, True)])
def test_full_size_360_whole_view(ora, full360, tile, persistent):
    # The 2M-voxel 1237x822 workload at full size, in the default launch and in the bench's tuned one
    # (tile 32, persistent warps): every pixel against the oracle's whole-view render, every voxel's
    # w_max and argmax, the FP32-pinned statistics bit for bit, and per-element gradients of a loss
    # on a 64x48 crop.
    sc, cam, r, ws = full360
    scene, ctx, vox = gpu_forward(sc, [cam], tile=tile)
    if persistent:
        from paper_2511_02510_gb300.raster import RasterContext
        ctx = RasterContext([cam], scene.n, tile=tile, persistent=True)
        ctx.fit_capacity(vox)
        ctx.reset_stats()
        ctx.forward(vox)
        ctx.check()
    compare_images(r, ctx)
    print("full-size images:", image_report(r, ctx))
    w, a = ctx.unpack_wmax()
    print("full-size w_max:", check_wmax(np_(w), np_(a), ws, r["near_stop"]))
    ref = ora.pairs(sc, [cam], ts=tile)
    np.testing.assert_array_equal(np_(ctx.seen), ref["seen"])
    np.testing.assert_array_equal(np_(ctx.z_min).view(np.uint32), ref["z_min"].view(np.uint32))
    np.testing.assert_array_equal(np_(ctx.delta_min).view(np.uint32), ref["delta_min"].view(np.uint32))
    # every pair list of the whole view, front to back (tile 32: lists of up to 11142 pairs)
    keys, vox_ids, ranges, pairs = gpu_pairs(ctx, scene.n)
    assert pairs == ref["n_pairs"]
    np.testing.assert_array_equal(keys, ref["keys"])
    np.testing.assert_array_equal(vox_ids, ref["vals"])
    np.testing.assert_array_equal(ranges, ref["ranges"])
    x0, y0 = 580, 380
    crop = [x0, y0, x0 + 64, y0 + 48]
    m = np.zeros((822, 1237), bool)
    m[y0:y0 + 48, x0:x0 + 64] = True
    gC, gD, gT = _loss_grads(ctx.n_pix, 7, r["near_stop"])
    gC[~m.ravel()], gD[~m.ravel()], gT[~m.ravel()] = 0, 0, 0
    d_dens, d_sh = ctx.backward(vox, torch.from_numpy(gC).cuda(), torch.from_numpy(gD).cuda(),
                                torch.from_numpy(gT).cuda())
    torch.cuda.synchronize()
    grad_parity(ora, sc, [cam], d_dens, d_sh, gC, gD, gT, crop=crop)


def test_max_views_and_limits(ora, tiny):
    # LV_MAX_VIEWS small views in one launch match the oracle; one more is refused, as is a batch of
    # 128 with 32x32 tiles (more shared memory than a block has)
    cams = [synth.orbit_camera(24 + (i % 5) * 4, 18 + (i % 3) * 6, 60.0, 1.6, 360.0 * i / 64, 20.0 + (i % 7),
                               target=(0.5, 0.4, 0.5)) for i in range(L.LV_MAX_VIEWS)]
    scene, ctx, vox = gpu_forward(tiny, cams)
    r = ora.render(tiny, cams)
    compare_images(r, ctx)
    keys, vox_ids, ranges, pairs = gpu_pairs(ctx, scene.n)
    ref = ora.pairs(tiny, cams, ts=16)
    np.testing.assert_array_equal(keys, ref["keys"])
    np.testing.assert_array_equal(vox_ids, ref["vals"])
    too_many = L.make_cameras(cams + [cams[0]])
    assert L.lv_forward_workspace_size(scene.n, too_many, L.LV_MAX_VIEWS + 1, ctx.opts, 1024) == 0
    bad = L.make_opts(32, 128)
    with pytest.raises(L.LvError) as ei:
        L.lv_rasterize_forward(vox, ctx.cams_arr, ctx.n_views, bad, ctx.fwd_struct(), ctx.workspace,
                               ctx.pair_capacity)
    assert ei.value.status == L.LV_ERR_UNSUPPORTED
