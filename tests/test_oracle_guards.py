"""Pins for the oracle's pruning guards beyond guards i/iii (Sec. IV-C): the
annealed, near/far-relaxed per-bin quantile q_b, the keep-halo protection
(guard ii) and the running depth percentiles of Eq. 14.

Expected values come from closed forms, brute-force selection with numpy's
sort, exact FP32 identities (0.5 p + 0.5 p = p) and comparisons with the
guard-free rule on inputs where the guard cannot act.
"""
import math

import numpy as np
import pytest


# --------------------------------------------------------------------- q_b schedule

def test_q_bin_closed_forms(ora):
    q, nb = 50000, 16
    # no annealing progress and no relaxation: q itself; a = 0: nothing
    assert all(ora.prune_q_bin(q, 1000000, 0, b, nb) == q for b in range(nb))
    assert all(ora.prune_q_bin(q, 0, 500000, b, nb) == 0 for b in range(nb))
    # a = 1/2: floor(q / 2)
    assert ora.prune_q_bin(12345, 500000, 0, 3, nb) == 6172
    # full relaxation: |2 c_b - 1| = |2b + 1 - nb| / nb; the two end bins get q / nb,
    # the two centre bins q (nb - 1) / nb (floors)
    assert ora.prune_q_bin(q, 1000000, 1000000, 0, nb) == q // nb
    assert ora.prune_q_bin(q, 1000000, 1000000, nb - 1, nb) == q // nb
    assert ora.prune_q_bin(q, 1000000, 1000000, nb // 2, nb) == q * (nb - 1) // nb
    # odd bin count: the centre bin is not relaxed at all
    assert ora.prune_q_bin(q, 1000000, 1000000, 3, 7) == q


def test_q_bin_symmetric_and_peaked(ora):
    for nb in (1, 2, 5, 16, 64):
        vals = [ora.prune_q_bin(999999, 734567, 300000, b, nb) for b in range(nb)]
        assert vals == vals[::-1]                               # near/far symmetric
        half = vals[: (nb + 1) // 2]
        assert all(x <= y for x, y in zip(half, half[1:]))     # relaxation strongest at the ends
        assert max(vals) <= 999999 * 734567 // 1000000


def test_anneal_schedule(ora):
    from paper_2511_02510_gb300 import litevoxel as L
    assert ora.anneal_ppm(0, 100, 300) == 0
    assert ora.anneal_ppm(100, 100, 300) == 0
    assert ora.anneal_ppm(200, 100, 300) == 500000
    assert ora.anneal_ppm(300, 100, 300) == 1000000
    assert ora.anneal_ppm(1e9, 100, 300) == 1000000
    assert ora.anneal_ppm(5, 10, 10) == 1000000               # degenerate ramp: fully on
    # the library's host helper computes the same integers
    L.load()
    rng = np.random.default_rng(0)
    for t in rng.uniform(-50, 450, 200):
        assert L.lv_prune_anneal_ppm(t, 100.0, 300.0) == ora.anneal_ppm(t, 100.0, 300.0)


# --------------------------------------------------------------------- annealed quantiles

def _prune_inputs(seed, n=4000):
    rng = np.random.default_rng(seed)
    w = rng.uniform(0, 1, n).astype(np.float32)
    w[rng.integers(0, n, n // 10)] = np.float32(0.25)          # ties
    z = rng.gamma(2.0, 2.0, n).astype(np.float32)
    seen = (rng.uniform(size=n) < 0.9).astype(np.uint8)
    m = rng.uniform(0.2, 1.0, n).astype(np.float32)
    s = (rng.uniform(size=n) < 0.7).astype(np.uint8)
    return w, z, seen, m, s


@pytest.mark.parametrize("seed,anneal,relax", [(0, 1000000, 200000), (1, 400000, 0), (2, 650000, 1000000)])
def test_annealed_thresholds_brute_force(ora, seed, anneal, relax):
    # tau_b: nearest-rank q_b-quantile of w_max in each bin, with q_b from the schedule
    w, z, seen, m, s = _prune_inputs(seed)
    q = 300000
    r = ora.prune(w, seen, z, m, s, q_ppm=q, cap_ppm=1000000, anneal_ppm=anneal, relax_ppm=relax)
    p5, p95 = r["p_lo"], r["p_hi"]
    zt = np.clip((z.astype(np.float64) - p5) / (p95 - p5), 0, 1)
    b = np.minimum(15, np.floor(16 * zt)).astype(int)
    sc16 = 16 * zt[seen == 1]
    checked = 0
    for bb in range(16):
        sel = (seen == 1) & (b == bb)
        # skip bins whose membership could differ by FP32 rounding at an interior bin edge
        near = [j for j in (bb, bb + 1) if 1 <= j <= 15]
        if sel.sum() == 0 or any((np.abs(sc16 - j) < 1e-5).any() for j in near):
            continue
        qb = ora.prune_q_bin(q, anneal, relax, bb, 16)
        vals = np.sort(w[sel])
        k = max(1, -(-qb * len(vals) // 1000000))
        assert r["tau"][bb] == vals[k - 1]
        checked += 1
    assert checked >= 8


def test_zero_quantile_sets_no_threshold(ora):
    # a = 0 (start of the schedule): q_b = 0 in every bin, so every seen voxel votes in (x = 1):
    # the EMA moves every seen voxel up by the same rule, unseen voxels keep m
    w, z, seen, m, s = _prune_inputs(4)
    r0 = ora.prune(w, seen, z, m, s, anneal_ppm=0, cap_ppm=1000000)
    a, oma = np.float32(0.1), np.float32(0.9)
    expect = (oma * m + a * np.float32(1.0)).astype(np.float32)
    np.testing.assert_array_equal(r0["m"][seen == 1], expect[seen == 1])
    np.testing.assert_array_equal(r0["m"][seen == 0], m[seen == 0])
    # an in-vote turns a voxel out only when its EMA is still below m_low
    flipped = (s == 1) & (r0["s"] == 0)
    assert np.all(r0["m"][flipped] < np.float32(0.3))


# --------------------------------------------------------------------- keep-halo (guard ii)

def test_keep_halo_size_test_protects_everything(ora):
    # halo_small huge: every voxel is small against its footprint -> nothing pruned,
    # while the EMA and the hysteresis state evolve exactly as without the guard
    w, z, seen, m, s = _prune_inputs(5)
    n = len(w)
    geom = np.zeros((n, 4), np.float32)
    geom[:, 3] = 0.01
    delta = np.full(n, 1.0, np.float32)
    base = ora.prune(w, seen, z, m, s, cap_ppm=1000000)
    g = ora.prune(w, seen, z, m, s, cap_ppm=1000000, geom=geom, delta=delta, halo_small=1.0)
    assert base["n_pruned"] > 0 and g["n_pruned"] == 0
    np.testing.assert_array_equal(g["m"], base["m"])
    np.testing.assert_array_equal(g["s"], base["s"])


def test_keep_halo_size_test_threshold(ora):
    # protection iff h < halo_small * delta (strict), checked voxel by voxel with the cap off
    w, z, seen, m, s = _prune_inputs(6)
    n = len(w)
    rng = np.random.default_rng(60)
    geom = np.zeros((n, 4), np.float32)
    geom[:, 3] = rng.uniform(0.01, 0.2, n).astype(np.float32)
    delta = rng.uniform(0.05, 0.2, n).astype(np.float32)
    delta[:20] = geom[:20, 3]                                   # h == 1 * delta: not protected
    base = ora.prune(w, seen, z, m, s, cap_ppm=1000000)
    g = ora.prune(w, seen, z, m, s, cap_ppm=1000000, geom=geom, delta=delta, halo_small=1.0)
    prot = geom[:, 3] < delta
    np.testing.assert_array_equal(g["mask"], base["mask"] & (~prot).astype(np.uint8))
    assert (base["mask"] & prot).sum() > 0 and (g["mask"] > 0).sum() > 0


def test_keep_halo_edge_test(ora):
    # protection iff w_max >= halo_w and edge >= halo_edge
    w, z, seen, m, s = _prune_inputs(7)
    n = len(w)
    rng = np.random.default_rng(70)
    edge = rng.uniform(0, 1, n).astype(np.float32)
    edge[:30] = np.float32(0.5)                                 # exactly at the edge threshold
    base = ora.prune(w, seen, z, m, s, cap_ppm=1000000)
    g = ora.prune(w, seen, z, m, s, cap_ppm=1000000, edge=edge, halo_w=0.0, halo_edge=0.5)
    prot = (w >= 0.0) & (edge >= np.float32(0.5))
    np.testing.assert_array_equal(g["mask"], base["mask"] & (~prot).astype(np.uint8))
    # a weight threshold above every w_max disables the edge test
    g2 = ora.prune(w, seen, z, m, s, cap_ppm=1000000, edge=edge, halo_w=2.0, halo_edge=0.0)
    np.testing.assert_array_equal(g2["mask"], base["mask"])


def test_keep_halo_cap_counts_only_candidates(ora):
    # guard iii applies to the unprotected candidates: the cap smallest (w, id) among them
    n = 1000
    rng = np.random.default_rng(8)
    w = rng.uniform(0.01, 1, n).astype(np.float32)
    seen = np.ones(n, np.uint8)
    z = np.ones(n, np.float32)
    m = np.full(n, 0.1, np.float32)
    s = np.zeros(n, np.uint8)
    edge = np.zeros(n, np.float32)
    order = np.lexsort((np.arange(n), w))
    edge[order[:4]] = 1.0                                       # protect the 4 smallest
    r = ora.prune(w, seen, z, m, s, cap_ppm=8000, edge=edge, halo_w=0.0, halo_edge=0.5)
    expect = np.zeros(n, np.uint8)
    expect[order[4:12]] = 1
    np.testing.assert_array_equal(r["mask"], expect)


# --------------------------------------------------------------------- running percentiles

def test_running_percentiles_first_call_and_rate_one(ora):
    w, z, seen, m, s = _prune_inputs(9)
    base = ora.prune(w, seen, z, m, s, cap_ppm=1000000)
    st = np.full(2, np.nan, np.float32)
    r = ora.prune(w, seen, z, m, s, cap_ppm=1000000, pct_ema=0.3, pct_state=st)
    assert st[0] == base["p_lo"] and st[1] == base["p_hi"]     # NaN state takes the step's value
    for k in ("mask", "m", "s", "tau"):
        np.testing.assert_array_equal(r[k], base[k])
    st = np.array([0.1, 99.0], np.float32)
    r = ora.prune(w, seen, z, m, s, cap_ppm=1000000, pct_ema=1.0, pct_state=st)
    assert st[0] == base["p_lo"] and st[1] == base["p_hi"]     # rate 1: the step's value
    np.testing.assert_array_equal(r["tau"], base["tau"])


def test_running_percentiles_half_rate_identity(ora):
    # 0.5 p + 0.5 p == p exactly in FP32, so a state equal to the step's percentiles is a fixed point
    w, z, seen, m, s = _prune_inputs(10)
    base = ora.prune(w, seen, z, m, s, cap_ppm=1000000)
    st = np.array([base["p_lo"], base["p_hi"]], np.float32)
    r = ora.prune(w, seen, z, m, s, cap_ppm=1000000, pct_ema=0.5, pct_state=st)
    assert st[0] == base["p_lo"] and st[1] == base["p_hi"]
    np.testing.assert_array_equal(r["tau"], base["tau"])
    # and a state below the step's values pulls the percentiles down by half the gap (exact halves)
    st = np.array([base["p_lo"] - 1.0, base["p_hi"] - 2.0], np.float32)
    r = ora.prune(w, seen, z, m, s, cap_ppm=1000000, pct_ema=0.5, pct_state=st)
    assert abs(float(st[0]) - (float(base["p_lo"]) - 0.5)) < 1e-5
    assert abs(float(st[1]) - (float(base["p_hi"]) - 1.0)) < 1e-5
    assert r["p_lo"] == st[0] and r["p_hi"] == st[1]


def test_running_percentiles_converge(ora):
    # with the same data every call the state approaches the step's percentiles geometrically
    w, z, seen, m, s = _prune_inputs(11)
    base = ora.prune(w, seen, z, m, s)
    st = np.array([0.0, 100.0], np.float32)
    gaps = []
    for _ in range(40):
        ora.prune(w, seen, z, m, s, pct_ema=0.2, pct_state=st)
        gaps.append(abs(float(st[1]) - float(base["p_hi"])))
    assert gaps[-1] < 1e-3 * gaps[0]
    assert all(b <= a + 1e-6 for a, b in zip(gaps, gaps[1:]))


def test_running_percentiles_untouched_without_seen_voxels(ora):
    w, z, seen, m, s = _prune_inputs(12)
    st = np.array([1.0, 2.0], np.float32)
    ora.prune(w, np.zeros_like(seen), z, m, s, pct_ema=0.5, pct_state=st)
    assert st[0] == 1.0 and st[1] == 2.0


def test_subdivide_running_percentiles(ora):
    from test_oracle_adapt import _scene_rand
    n = 1500
    sc = _scene_rand(n, 21)
    rng = np.random.default_rng(22)
    delta = rng.uniform(0.0, 0.2, n).astype(np.float32)
    z = rng.uniform(0.5, 20, n).astype(np.float32)
    u = rng.uniform(0, 1, n).astype(np.float32)
    seen = (rng.uniform(size=n) < 0.8).astype(np.uint8)
    base = ora.subdivide(sc, delta, z, u, seen, beta=0.3)
    st = np.full(2, np.nan, np.float32)
    r = ora.subdivide(sc, delta, z, u, seen, beta=0.3, pct_ema=0.25, pct_state=st)
    np.testing.assert_array_equal(r["selected"], base["selected"])
    zs = np.sort(z[seen == 1])
    assert st[0] == zs[math.ceil(0.05 * len(zs)) - 1] and st[1] == zs[math.ceil(0.95 * len(zs)) - 1]
    # a state at the step's values and rate 1/2: unchanged selection (exact fixed point)
    r = ora.subdivide(sc, delta, z, u, seen, beta=0.3, pct_ema=0.5, pct_state=st)
    np.testing.assert_array_equal(r["selected"], base["selected"])
    # a far-off state changes z~ and so the far bias: the selection moves
    st2 = np.array([float(zs[-1]), float(zs[-1]) + 50.0], np.float32)
    r2 = ora.subdivide(sc, delta, z, u, seen, beta=3.0, pct_ema=0.01, pct_state=st2)
    b3 = ora.subdivide(sc, delta, z, u, seen, beta=3.0)
    assert not np.array_equal(r2["selected"], b3["selected"])
