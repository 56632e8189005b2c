"""GPU parity of depth-quantile pruning, priority subdivision and the
LF-weighted loss against the CPU oracle, through the C ABI.

Pruning and subdivision take integer decisions from FP32 values; both sides
compute them in FP32 with the same operation order from the same FP32 inputs,
so masks, EMA values, states, selections and child arrays must match bit for
bit.  The loss is compared with the FP64 oracle at 1e-5 relative (FP32
per-pixel terms, FP64 sums).
"""

import numpy as np
import pytest
import torch

from gpu_helpers import gpu_forward, np_
from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth

pytestmark = pytest.mark.gpu


def cu(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


def prune_params(n_bins=16, q_ppm=50000, alpha=0.1, m_low=0.3, m_high=0.7, cap_ppm=10000):
    p = L.lv_prune_params()
    p.n_bins, p.q_ppm, p.ema_alpha, p.m_low, p.m_high, p.cap_ppm = n_bins, q_ppm, alpha, m_low, m_high, cap_ppm
    p.lo_ppm, p.hi_ppm = 50000, 950000
    return p


def gpu_prune(w, seen, z, m, s, **kw):
    p = prune_params(**kw)
    n = len(w)
    ws = torch.empty(L.lv_prune_workspace_size(n, p), dtype=torch.uint8, device="cuda")
    mt, st = cu(m), cu(s)
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    npr = torch.zeros(1, dtype=torch.int64, device="cuda")
    L.lv_prune_depth_quantile(cu(w), cu(seen), cu(z), mt, st, p, mask, npr, ws)
    torch.cuda.synchronize()
    return np_(mask), int(npr.item()), np_(mt), np_(st)


def check_prune(ora, w, seen, z, m, s, **kw):
    gm, gn, gmm, gs = gpu_prune(w, seen, z, m, s, **kw)
    names = {"n_bins": "n_bins", "q_ppm": "q_ppm", "alpha": "ema_alpha", "m_low": "m_low", "m_high": "m_high",
             "cap_ppm": "cap_ppm"}
    r = ora.prune(w, seen, z, m, s, **{names[k]: v for k, v in kw.items()})
    np.testing.assert_array_equal(gm, r["mask"])
    assert gn == r["n_pruned"]
    np.testing.assert_array_equal(gmm.view(np.uint32), r["m"].view(np.uint32))
    np.testing.assert_array_equal(gs, r["s"])
    return r


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_prune_random_bit_exact(ora, seed):
    rng = np.random.default_rng(seed)
    n = [5000, 20000, 777, 100000][seed]
    w = rng.uniform(0, 1, n).astype(np.float32)
    w[rng.integers(0, n, n // 10)] = np.float32(0.125)          # ties
    z = rng.gamma(2.0, 2.0, n).astype(np.float32)
    seen = (rng.uniform(size=n) < 0.85).astype(np.uint8)
    m = rng.uniform(0.2, 1.0, n).astype(np.float32)
    s = (rng.uniform(size=n) < 0.7).astype(np.uint8)
    kw = [dict(), dict(q_ppm=300000, cap_ppm=50000), dict(n_bins=1, q_ppm=500000, cap_ppm=1000000),
          dict(n_bins=64, q_ppm=999999, cap_ppm=0)][seed]
    r = check_prune(ora, w, seen, z, m, s, **kw)
    if seed == 0:
        assert r["n_pruned"] > 0


def test_prune_multistep_hysteresis(ora):
    # Several consecutive steps: m and s evolve identically on both sides.
    rng = np.random.default_rng(7)
    n = 4000
    z = rng.uniform(1, 10, n).astype(np.float32)
    seen = np.ones(n, np.uint8)
    m = np.ones(n, np.float32)
    s = np.ones(n, np.uint8)
    for step in range(14):
        w = rng.uniform(0, 1, n).astype(np.float32)
        w[:50] = np.float32(0.0)                           # a group that always votes out
        gm, gn, gmm, gs = gpu_prune(w, seen, z, m, s, cap_ppm=5000)
        r = ora.prune(w, seen, z, m, s, cap_ppm=5000)
        np.testing.assert_array_equal(gm, r["mask"])
        np.testing.assert_array_equal(gmm.view(np.uint32), r["m"].view(np.uint32))
        np.testing.assert_array_equal(gs, r["s"])
        m, s = r["m"], r["s"]
    assert np.all(s[:50] == 0)


def test_prune_degenerate(ora):
    n = 300
    check_prune(ora, np.full(n, 0.5, np.float32), np.ones(n, np.uint8), np.full(n, 2.0, np.float32),
                np.ones(n, np.float32), np.ones(n, np.uint8), cap_ppm=1000000)
    check_prune(ora, np.full(n, 0.5, np.float32), np.zeros(n, np.uint8), np.full(n, 2.0, np.float32),
                np.full(n, 0.1, np.float32), np.zeros(n, np.uint8))
    check_prune(ora, np.zeros(1, np.float32), np.ones(1, np.uint8), np.ones(1, np.float32),
                np.full(1, 0.31, np.float32), np.ones(1, np.uint8), cap_ppm=1000000)


def test_prune_from_rendered_statistics(ora):
    # The integer path end to end: render (w_max, z_min, seen on the GPU), then prune on both sides.
    sc = synth.scene_tiny()
    cams = [synth.orbit_camera(96, 96, 60.0, 1.6, a, 25.0, target=(0.5, 0.4, 0.5)) for a in (20.0, 140.0, 260.0)]
    scene, ctx, vox = gpu_forward(sc, cams)
    w, _ = ctx.unpack_wmax()
    torch.cuda.synchronize()
    w, z, seen = np_(w), np_(ctx.z_min), np_(ctx.seen)
    n = len(w)
    r = check_prune(ora, w, seen, z, np.full(n, 0.32, np.float32), np.ones(n, np.uint8), cap_ppm=20000)
    assert r["n_pruned"] > 0


# ------------------------------------------------------------------ subdivision
def sub_params(kappa=1.0, beta=0.2, top_ppm=50000, l_max=16, budget=1 << 62):
    p = L.lv_subdiv_params()
    p.kappa, p.beta, p.top_ppm, p.l_max, p.budget = kappa, beta, top_ppm, l_max, budget
    p.lo_ppm, p.hi_ppm = 50000, 950000
    return p


def gpu_subdivide(sc, delta, z, u, seen, pm=None, density_dtype=torch.float32, sh_dtype=torch.float32, aux=(),
                  capacity=None, **kw):
    p = sub_params(**kw)
    n = sc["geom"].shape[0]
    geom, level = cu(sc["geom"]), cu(sc["level"])
    dens, sh = cu(sc["density"], density_dtype), cu(sc["sh"], sh_dtype)
    vin = L.make_voxels(geom, dens, sh, level)
    cap = capacity if capacity is not None else n + 7 * n
    og = torch.zeros((cap, 4), dtype=torch.float32, device="cuda")
    ol = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    od = torch.zeros((cap, 8), dtype=density_dtype, device="cuda")
    osh = torch.zeros((cap, 48), dtype=sh_dtype, device="cuda")
    vout = L.make_voxels(og, od, osh, ol)
    vout.n = cap
    auxs, keep = [], []
    for arr, fill in aux:
        ti = cu(arr)
        to = torch.zeros((cap,) + tuple(ti.shape[1:]), dtype=ti.dtype, device="cuda")
        a = L.lv_aux_array()
        a.in_, a.out = ti.data_ptr(), to.data_ptr()
        a.width = 1 if ti.dim() == 1 else ti.shape[1]
        a.elem_bytes = ti.element_size()
        a.fill = int(np.array([fill], arr.dtype).view({1: np.uint8, 2: np.uint16, 4: np.uint32}[arr.dtype.itemsize])[0])
        auxs.append(a)
        keep.append((ti, to))
    sel = torch.zeros(n, dtype=torch.uint8, device="cuda")
    nn = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(L.lv_subdivide_workspace_size(n, p), dtype=torch.uint8, device="cuda")
    L.lv_subdivide_priority(vin, cu(delta), cu(z), cu(u), cu(seen), None if pm is None else cu(pm), p, auxs, vout,
                            sel, nn, ws, status)
    torch.cuda.synchronize()
    m = int(nn.item())
    return {"geom": np_(og)[:m], "level": np_(ol)[:m], "density": od[:m].cpu(), "sh": osh[:m].cpu(),
            "selected": np_(sel), "n_new": m, "status": int(status.item()), "aux": [np_(t)[:m] for _, t in keep]}


def rand_scene(n, seed):
    rng = np.random.default_rng(seed)
    sc = synth.constant_voxel_scene(rng.uniform(-1, 1, (n, 3)), rng.uniform(0.01, 0.2, n), np.ones(n),
                                    np.ones((n, 3)) * 0.5)
    sc["density"] = rng.normal(2, 1, (n, 8)).astype(np.float32)
    sc["sh"] = rng.normal(0, 1, (n, 48)).astype(np.float32)
    sc["level"] = rng.integers(3, 17, n).astype(np.uint8)
    return sc


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_subdivide_bit_exact(ora, seed):
    n = [3000, 20000, 500][seed]
    sc = rand_scene(n, 100 + seed)
    rng = np.random.default_rng(seed)
    delta = rng.uniform(0.0, 0.2, n).astype(np.float32)
    z = rng.uniform(1, 20, n).astype(np.float32)
    u = rng.uniform(0, 1, n).astype(np.float32)
    u[: n // 8] = np.float32(0.5)
    seen = (rng.uniform(size=n) < 0.8).astype(np.uint8)
    pm = (rng.uniform(size=n) < 0.1).astype(np.uint8) if seed != 2 else None
    adam_m = rng.normal(size=(n, 8)).astype(np.float32)
    ema = rng.uniform(size=n).astype(np.float32)
    st = (rng.uniform(size=n) < 0.5).astype(np.uint8)
    kw = [dict(), dict(top_ppm=200000, beta=0.3), dict(top_ppm=1000000, budget=n + 7 * 40)][seed]
    aux = [(adam_m, 0.0), (ema, 1.0), (st, 1)]
    g = gpu_subdivide(sc, delta, z, u, seen, pm, aux=aux, **kw)
    r = ora.subdivide(sc, delta, z, u, seen, prune_mask=pm, aux=aux, **kw)
    assert g["status"] == 0
    assert g["n_new"] == r["n_new"] and r["k"] > 0
    np.testing.assert_array_equal(g["selected"], r["selected"])
    np.testing.assert_array_equal(g["geom"].view(np.uint32), r["geom"].view(np.uint32))
    np.testing.assert_array_equal(g["level"], r["level"])
    np.testing.assert_array_equal(g["density"].numpy().view(np.uint32), r["density"].view(np.uint32))
    np.testing.assert_array_equal(g["sh"].numpy(), r["sh"])
    for a, b in zip(g["aux"], r["aux"]):
        np.testing.assert_array_equal(a, b)


def test_subdivide_mixed_precision_storage(ora):
    n = 4000
    sc = rand_scene(n, 7)
    rng = np.random.default_rng(8)
    delta = rng.uniform(0.0, 0.2, n).astype(np.float32)
    z = rng.uniform(1, 20, n).astype(np.float32)
    u = rng.uniform(0, 1, n).astype(np.float32)
    seen = np.ones(n, np.uint8)
    g = gpu_subdivide(sc, delta, z, u, seen, density_dtype=torch.float16, sh_dtype=torch.bfloat16)
    ref = dict(sc)
    ref["density"] = torch.as_tensor(sc["density"]).half().float().numpy()
    ref["sh"] = torch.as_tensor(sc["sh"]).bfloat16().float().numpy()
    r = ora.subdivide(ref, delta, z, u, seen)
    assert g["n_new"] == r["n_new"]
    np.testing.assert_array_equal(g["density"].numpy().view(np.uint16),
                                  r["density"].astype(np.float16).view(np.uint16))
    np.testing.assert_array_equal(g["sh"].float().numpy(), r["sh"])


def test_subdivide_capacity_and_budget(ora):
    n = 1000
    sc = rand_scene(n, 3)
    sc["level"][:] = 4
    ones = np.ones(n, np.float32)
    g = gpu_subdivide(sc, np.zeros(n, np.float32), ones, np.arange(n, dtype=np.float32), np.ones(n, np.uint8),
                      top_ppm=100000, capacity=n + 10)
    assert g["status"] == L.LV_ERR_CAPACITY and g["n_new"] == n + 7 * 100
    g = gpu_subdivide(sc, np.zeros(n, np.float32), ones, ones, np.ones(n, np.uint8), top_ppm=1000000, budget=n)
    assert g["n_new"] == n and g["selected"].sum() == 0


def test_prune_then_subdivide_step(ora):
    # One adaptation step on rendered statistics: prune, then subdivide the survivors.
    sc = synth.scene_tiny()
    cams = [synth.orbit_camera(96, 96, 60.0, 1.6, a, 25.0, target=(0.5, 0.4, 0.5)) for a in (60.0, 200.0)]
    scene, ctx, vox = gpu_forward(sc, cams)
    w, _ = ctx.unpack_wmax()
    torch.cuda.synchronize()
    w, z, dl, seen = np_(w), np_(ctx.z_min), np_(ctx.delta_min), np_(ctx.seen)
    n = len(w)
    mask, npr, m, s = gpu_prune(w, seen, z, np.full(n, 0.32, np.float32), np.ones(n, np.uint8), cap_ppm=20000)
    g = gpu_subdivide(sc, dl, z, w, seen, pm=mask, top_ppm=50000, l_max=8)
    r = ora.subdivide(sc, dl, z, w, seen, prune_mask=mask, top_ppm=50000, l_max=8)
    assert npr > 0 and r["k"] > 0
    assert g["n_new"] == r["n_new"]
    np.testing.assert_array_equal(g["selected"], r["selected"])
    np.testing.assert_array_equal(g["geom"].view(np.uint32), r["geom"].view(np.uint32))
    np.testing.assert_array_equal(g["density"].numpy().view(np.uint32), r["density"].view(np.uint32))


# ------------------------------------------------------------------ LF loss
def lf_params(eps=1e-3, gamma_max=0.6, t0=300.0, t1=600.0, pctl=990000):
    p = L.lv_lf_params()
    p.eps, p.gamma_max, p.t0, p.t1, p.pctl_ppm = eps, gamma_max, t0, t1, pctl
    return p


def gpu_lf(rgb, gt, sizes, t, **kw):
    p = lf_params(**kw)
    W = [s[0] for s in sizes]
    H = [s[1] for s in sizes]
    ws = torch.empty(L.lv_lf_workspace_size(W, H), dtype=torch.uint8, device="cuda")
    loss = torch.zeros(len(sizes), dtype=torch.float32, device="cuda")
    g = torch.zeros((rgb.shape[0], 3), dtype=torch.float32, device="cuda")
    L.lv_lf_weighted_loss(cu(rgb), cu(gt), W, H, t, p, loss, g, ws)
    torch.cuda.synchronize()
    return np_(loss), np_(g), L.lv_lf_gamma(t, p)


@pytest.mark.parametrize("t", [0.0, 450.0, 1000.0])
def test_lf_loss_parity(ora, t):
    sizes = [(128, 96), (77, 45), (200, 130)]
    P = sum(w * h for w, h in sizes)
    rng = np.random.default_rng(int(t))
    gt = np.concatenate([synth.smooth_image(w, h, seed=i) for i, (w, h) in enumerate(sizes)])
    rgb = np.clip(gt + rng.normal(0, 0.1, gt.shape), 0, 1).astype(np.float32)
    loss, grad, gamma = gpu_lf(rgb, gt, sizes, t)
    assert abs(gamma - ora.lf_gamma(t, 300.0, 600.0, 0.6)) < 1e-7
    r = ora.lf_loss(rgb.astype(np.float64), gt.astype(np.float64), sizes, gamma=gamma)
    np.testing.assert_allclose(loss, r["loss"], rtol=1e-5)
    scale = np.abs(r["dL_drgb"]).max()
    assert np.abs(grad - r["dL_drgb"]).max() <= 1e-5 * scale


def test_lf_loss_random_target_full_gamma(ora):
    sizes = [(160, 120)]
    rng = np.random.default_rng(5)
    gt = synth.random_image(160, 120, seed=5)
    rgb = rng.uniform(size=gt.shape).astype(np.float32)
    loss, grad, gamma = gpu_lf(rgb, gt, sizes, 50.0, gamma_max=1.0, t0=15.0, t1=30.0)
    assert gamma == 1.0
    r = ora.lf_loss(rgb.astype(np.float64), gt.astype(np.float64), sizes, gamma=1.0)
    np.testing.assert_allclose(loss, r["loss"], rtol=1e-5)
    assert np.abs(grad - r["dL_drgb"]).max() <= 1e-5 * np.abs(r["dL_drgb"]).max()


def test_lf_loss_constant_target():
    sizes = [(33, 17)]
    rng = np.random.default_rng(1)
    gt = np.full((33 * 17, 3), 0.25, np.float32)
    rgb = rng.uniform(size=gt.shape).astype(np.float32)
    loss, grad, _ = gpu_lf(rgb, gt, sizes, 1e9)
    mse = np.mean((rgb.astype(np.float64) - gt) ** 2)
    assert abs(loss[0] - mse) <= 1e-6 * mse


def test_lf_split_calls_match_fused_across_streams(ora):
    """lv_lf_weights on a side stream, then lv_lf_loss_from_weights on the main
    stream after an event: the same bits as the one-call loss.  Tiny views put
    view boundaries inside and between 4-pixel groups."""
    sizes = [(2, 3), (1, 1), (3, 1), (77, 45), (128, 96)]
    W = [s[0] for s in sizes]
    H = [s[1] for s in sizes]
    P = sum(w * h for w, h in sizes)
    rng = np.random.default_rng(11)
    gt = np.concatenate([synth.smooth_image(w, h, seed=i) for i, (w, h) in enumerate(sizes)])
    rgb = np.clip(gt + rng.normal(0, 0.1, gt.shape), 0, 1).astype(np.float32)
    loss_a, grad_a, gamma = gpu_lf(rgb, gt, sizes, 450.0)
    p = lf_params()
    ws = torch.empty(L.lv_lf_workspace_size(W, H), dtype=torch.uint8, device="cuda")
    loss = torch.zeros(len(sizes), dtype=torch.float32, device="cuda")
    g = torch.zeros((P, 3), dtype=torch.float32, device="cuda")
    gt_d, rgb_d = cu(gt), cu(rgb)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        L.lv_lf_weights(gt_d, W, H, 450.0, p, ws)
    torch.cuda.current_stream().wait_stream(side)
    L.lv_lf_loss_from_weights(rgb_d, gt_d, W, H, loss, g, ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(np_(loss), loss_a)
    np.testing.assert_array_equal(np_(g), grad_a)
    r = ora.lf_loss(rgb.astype(np.float64), gt.astype(np.float64), sizes, gamma=gamma)
    np.testing.assert_allclose(loss_a, r["loss"], rtol=1e-5)
    assert np.abs(grad_a - r["dL_drgb"]).max() <= 1e-5 * np.abs(r["dL_drgb"]).max()


def test_prune_halves_match_one_call_across_streams(ora):
    """lv_prune_bins on a side stream, lv_prune_finish after an event: the
    same bits as lv_prune_depth_quantile (masks, EMA, states, count)."""
    n = 20000
    rng = np.random.default_rng(21)
    w = rng.uniform(0, 1, n).astype(np.float32)
    w[: n // 10] = np.float32(0.25)
    seen = (rng.uniform(size=n) < 0.9).astype(np.uint8)
    z = rng.uniform(0.5, 20, n).astype(np.float32)
    m0 = rng.uniform(size=n).astype(np.float32)
    s0 = (rng.uniform(size=n) < 0.5).astype(np.uint8)
    ref_mask, ref_n, ref_m, ref_s = gpu_prune(w, seen, z, m0, s0)
    r = ora.prune(w, seen, z, m0, s0)
    np.testing.assert_array_equal(ref_mask, r["mask"])
    p = prune_params()
    ws = torch.empty(L.lv_prune_workspace_size(n, p), dtype=torch.uint8, device="cuda")
    m, s = cu(m0), cu(s0)
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    npr = torch.zeros(1, dtype=torch.int64, device="cuda")
    seen_d, z_d, w_d = cu(seen), cu(z), cu(w)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        L.lv_prune_bins(seen_d, z_d, p, ws)
    torch.cuda.current_stream().wait_stream(side)
    L.lv_prune_finish(w_d, seen_d, z_d, m, s, p, mask, npr, ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(np_(mask), ref_mask)
    np.testing.assert_array_equal(np_(m).view(np.uint32), ref_m.view(np.uint32))
    np.testing.assert_array_equal(np_(s), ref_s)
    assert int(npr.item()) == ref_n
