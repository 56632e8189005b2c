"""GPU parity of the pruning guards (annealed / relaxed q_b, keep-halo, running
depth percentiles), the running percentiles of subdivision, the per-pixel
edge map of the LF loss and the per-voxel edge gather, against the oracle.

Integer decisions and FP32 state (m, s, masks, percentile state) are compared
bit for bit; the edge map (FP32 on the GPU, FP64 in the oracle) to 1e-5
(a few FP32 roundings of a Sobel sum, divided by its 99th percentile).
"""
import numpy as np
import pytest
import torch

from gpu_helpers import np_
from paper_2511_02510_gb300 import litevoxel as L
from test_gpu_adapt import cu, prune_params

pytestmark = pytest.mark.gpu


def inputs(seed, n):
    rng = np.random.default_rng(seed)
    w = rng.uniform(0, 1, n).astype(np.float32)
    w[rng.integers(0, n, n // 10)] = np.float32(0.125)          # ties
    z = rng.gamma(2.0, 2.0, n).astype(np.float32)
    seen = (rng.uniform(size=n) < 0.85).astype(np.uint8)
    m = rng.uniform(0.2, 1.0, n).astype(np.float32)
    s = (rng.uniform(size=n) < 0.7).astype(np.uint8)
    geom = np.zeros((n, 4), np.float32)
    geom[:, :3] = rng.uniform(-1, 1, (n, 3))
    geom[:, 3] = rng.uniform(0.01, 0.2, n)
    delta = rng.uniform(0.02, 0.2, n).astype(np.float32)
    delta[: n // 50] = geom[: n // 50, 3]                      # h == delta: the strict test's edge
    edge = rng.uniform(0, 1, n).astype(np.float32)
    edge[: n // 40] = np.float32(0.5)
    return w, z, seen, m, s, geom, delta, edge


def gpu_prune_guarded(w, seen, z, m, s, q_ppm=50000, cap_ppm=10000, n_bins=16, anneal_ppm=None, relax_ppm=0,
                      geom=None, delta=None, halo_small=0.0, edge=None, halo_w=0.0, halo_edge=0.0, pct_ema=0.0,
                      pct_state=None):
    p = prune_params(n_bins=n_bins, q_ppm=q_ppm, cap_ppm=cap_ppm)
    keep = []
    if anneal_ppm is not None:
        p.anneal, p.anneal_ppm, p.relax_ppm = 1, int(anneal_ppm), int(relax_ppm)
    if geom is not None:
        keep += [cu(geom), cu(delta)]
        p.geom, p.delta, p.halo_small = keep[-2].data_ptr(), keep[-1].data_ptr(), halo_small
    if edge is not None:
        keep.append(cu(edge))
        p.edge, p.halo_w, p.halo_edge = keep[-1].data_ptr(), halo_w, halo_edge
    st_t = None
    if pct_state is not None:
        st_t = cu(pct_state)
        p.pct_ema, p.pct_state = pct_ema, st_t.data_ptr()
    n = len(w)
    ws = torch.empty(L.lv_prune_workspace_size(n, p), dtype=torch.uint8, device="cuda")
    mt, stt = cu(m), cu(s)
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    npr = torch.zeros(1, dtype=torch.int64, device="cuda")
    L.lv_prune_depth_quantile(cu(w), cu(seen), cu(z), mt, stt, p, mask, npr, ws)
    torch.cuda.synchronize()
    return {"mask": np_(mask), "n_pruned": int(npr.item()), "m": np_(mt), "s": np_(stt),
            "pct_state": None if st_t is None else np_(st_t)}


def same(g, r):
    np.testing.assert_array_equal(g["mask"], r["mask"])
    assert g["n_pruned"] == r["n_pruned"]
    np.testing.assert_array_equal(g["m"].view(np.uint32), r["m"].view(np.uint32))
    np.testing.assert_array_equal(g["s"], r["s"])


@pytest.mark.parametrize("cfg", [
    dict(anneal_ppm=1000000, relax_ppm=250000),
    dict(anneal_ppm=370000, relax_ppm=0, q_ppm=400000),
    dict(anneal_ppm=0),
    dict(anneal_ppm=820000, relax_ppm=1000000, n_bins=7, cap_ppm=1000000),
])
def test_prune_annealed_quantiles_bit_exact(ora, cfg):
    w, z, seen, m, s, *_ = inputs(1, 30000)
    g = gpu_prune_guarded(w, seen, z, m, s, **cfg)
    r = ora.prune(w, seen, z, m, s, **cfg)
    same(g, r)


@pytest.mark.parametrize("which", ["size", "edge", "both"])
def test_prune_keep_halo_bit_exact(ora, which):
    w, z, seen, m, s, geom, delta, edge = inputs(2, 40000)
    kw = dict(cap_ppm=20000)
    if which in ("size", "both"):
        kw.update(geom=geom, delta=delta, halo_small=1.0)
    if which in ("edge", "both"):
        kw.update(edge=edge, halo_w=0.0 if which == "edge" else 0.3, halo_edge=0.5)
    g = gpu_prune_guarded(w, seen, z, m, s, **kw)
    r = ora.prune(w, seen, z, m, s, **kw)
    same(g, r)
    base = ora.prune(w, seen, z, m, s, cap_ppm=20000)
    assert r["n_pruned"] > 0 and not np.array_equal(r["mask"], base["mask"])


def test_prune_running_percentiles_over_steps(ora):
    # several adaptation steps with drifting depths: the percentile state, m and s evolve identically
    w, z, seen, m, s, *_ = inputs(3, 20000)
    rng = np.random.default_rng(33)
    st_g = np.full(2, np.nan, np.float32)
    st_o = np.full(2, np.nan, np.float32)
    for step in range(6):
        zz = (z * np.float32(1.0 + 0.1 * step)).astype(np.float32)
        ww = rng.uniform(0, 1, len(w)).astype(np.float32)
        g = gpu_prune_guarded(ww, seen, zz, m, s, pct_ema=0.3, pct_state=st_g, anneal_ppm=600000 + 50000 * step,
                              relax_ppm=200000)
        r = ora.prune(ww, seen, zz, m, s, pct_ema=0.3, pct_state=st_o, anneal_ppm=600000 + 50000 * step,
                      relax_ppm=200000)
        same(g, r)
        np.testing.assert_array_equal(g["pct_state"].view(np.uint32), st_o.view(np.uint32))
        st_g = g["pct_state"]
        m, s = r["m"], r["s"]


def test_prune_running_state_untouched_without_seen_voxels(ora):
    w, z, seen, m, s, *_ = inputs(4, 1000)
    st = np.array([1.0, 2.0], np.float32)
    g = gpu_prune_guarded(w, np.zeros_like(seen), z, m, s, pct_ema=0.5, pct_state=st)
    assert g["n_pruned"] == 0 and list(g["pct_state"]) == [1.0, 2.0]


def gpu_subdivide_select(sc, delta, z, u, seen, pct_ema, pct_state, **kw):
    from test_gpu_adapt import sub_params
    p = sub_params(**kw)
    st_t = cu(pct_state)
    p.pct_ema, p.pct_state = pct_ema, st_t.data_ptr()
    n = sc["geom"].shape[0]
    arrays = [cu(sc["geom"]), cu(sc["density"]), cu(sc["sh"]), cu(sc["level"])]  # alive through the call
    vin = L.make_voxels(*arrays)
    sel = torch.zeros(n, dtype=torch.uint8, device="cuda")
    nn = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(L.lv_subdivide_workspace_size(n, p), dtype=torch.uint8, device="cuda")
    L.lv_subdivide_select(vin, cu(delta), cu(z), cu(u), cu(seen), None, p, 8 * n, sel, nn, ws)
    torch.cuda.synchronize()
    return np_(sel), int(nn.item()), np_(st_t)


def test_subdivide_running_percentiles_bit_exact(ora):
    from test_oracle_adapt import _scene_rand
    n = 30000
    sc = _scene_rand(n, 41)
    rng = np.random.default_rng(42)
    delta = rng.uniform(0.0, 0.2, n).astype(np.float32)
    z = rng.uniform(0.5, 20, n).astype(np.float32)
    u = rng.uniform(0, 1, n).astype(np.float32)
    seen = (rng.uniform(size=n) < 0.8).astype(np.uint8)
    st_g = np.array([3.0, 11.0], np.float32)
    st_o = st_g.copy()
    for step in range(3):
        zz = (z + np.float32(step)).astype(np.float32)
        sel_g, n_new_g, st_g = gpu_subdivide_select(sc, delta, zz, u, seen, 0.25, st_g, beta=0.3)
        r = ora.subdivide(sc, delta, zz, u, seen, beta=0.3, pct_ema=0.25, pct_state=st_o)
        np.testing.assert_array_equal(sel_g, r["selected"])
        assert n_new_g == r["n_new"]
        np.testing.assert_array_equal(st_g.view(np.uint32), st_o.view(np.uint32))


def test_lf_edge_map_and_gather(ora):
    rng = np.random.default_rng(5)
    sizes = [(97, 61), (64, 64)]
    P = sum(w * h for w, h in sizes)
    gt = rng.uniform(0, 1, (P, 3)).astype(np.float32)
    gt[:97 * 61] = np.repeat(np.linspace(0, 1, 97 * 61, dtype=np.float32)[:, None], 3, 1)
    rgb = rng.uniform(0, 1, (P, 3)).astype(np.float32)
    p = L.lv_lf_params()
    p.eps, p.gamma_max, p.t0, p.t1, p.pctl_ppm = 1e-3, 0.6, 300.0, 600.0, 990000
    W = [s[0] for s in sizes]
    H = [s[1] for s in sizes]
    ws = torch.empty(L.lv_lf_workspace_size(W, H), dtype=torch.uint8, device="cuda")
    loss0 = torch.zeros(2, device="cuda")
    loss1 = torch.zeros(2, device="cuda")
    rgb_t, gt_t = cu(rgb), cu(gt)
    L.lv_lf_weighted_loss(rgb_t, gt_t, W, H, 450.0, p, loss0, None, ws)
    edge_map = torch.full((P,), -1.0, device="cuda")
    p.edge_out = edge_map.data_ptr()
    L.lv_lf_weighted_loss(rgb_t, gt_t, W, H, 450.0, p, loss1, None, ws)
    torch.cuda.synchronize()
    assert torch.equal(loss0, loss1)                               # the extra output changes nothing
    r = ora.lf_loss(rgb, gt, sizes, ora.lf_gamma(450.0, 300.0, 600.0, 0.6))
    np.testing.assert_allclose(np_(edge_map), r["s"], atol=1e-5, rtol=0)
    # per-voxel gather at the w_max argmax pixel, -1 and out-of-range ids give 0
    n = 5000
    arg = rng.integers(-1, P + 3, n).astype(np.int64)
    out = torch.empty(n, device="cuda")
    L.lv_gather_edge(cu(arg), edge_map, out)
    torch.cuda.synchronize()
    em = np_(edge_map)
    expect = np.where((arg >= 0) & (arg < P), em[np.clip(arg, 0, P - 1)], 0.0).astype(np.float32)
    np.testing.assert_array_equal(np_(out), expect)


def test_guard_parameter_validation():
    n = 100
    p = prune_params()
    p.anneal, p.anneal_ppm = 1, 1000001
    ws = torch.empty(L.lv_prune_workspace_size(n, p), dtype=torch.uint8, device="cuda")
    args = (cu(np.zeros(n, np.float32)), cu(np.ones(n, np.uint8)), cu(np.ones(n, np.float32)),
            cu(np.ones(n, np.float32)), cu(np.ones(n, np.uint8)))
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LvError):
        L.lv_prune_depth_quantile(*args, p, mask, None, ws)
    p = prune_params()
    p.pct_ema = 1.5
    with pytest.raises(L.LvError):
        L.lv_prune_depth_quantile(*args, p, mask, None, ws)
