"""Pins for the oracle's binning, pruning (Eq. 11-12, guards i/iii), subdivision
(Eq. 13-16) and LF-weighted loss (Eq. 7-10, 18).

Expected values come from hand traces, brute-force selection with numpy's
sort, closed forms, or the stored fixtures under tests/golden/.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2511_02510_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------- binning

def _ray(cam, x, y):
    R = np.asarray(cam["w2c"], np.float64).reshape(3, 4)[:, :3]
    t = np.asarray(cam["w2c"], np.float64).reshape(3, 4)[:, 3]
    o = -R.T @ t
    d = R.T @ np.array([(x + 0.5 - cam["cx"]) / cam["fx"], (y + 0.5 - cam["cy"]) / cam["fy"], 1.0])
    return o, d / np.linalg.norm(d)


def _hits(o, d, c, h):
    """Which boxes does the ray cross with positive length?  (dense sampling of the inside predicate)"""
    ts = np.linspace(0.0, 6.0, 3001)
    pts = o[None] + ts[:, None] * d[None]
    inside = np.all(np.abs(pts[:, None, :] - c[None, :, :]) < h[None, :, None], axis=2)
    return inside.any(axis=0)


def test_pairs_cover_every_hit_pixel(ora):
    # The FP32 tile rectangle (1-pixel margin) must contain every pixel whose ray crosses the voxel.
    rng = np.random.default_rng(3)
    n = 40
    centers = rng.uniform(-0.6, 0.6, (n, 3))
    half = rng.uniform(0.02, 0.15, n)
    sc = synth.constant_voxel_scene(centers, half, np.ones(n), np.ones((n, 3)) * 0.5)
    cam = synth.look_at_camera([0.2, 0.3, -2.5], [0, 0, 0], 40, 36, 55.0)
    ts = 8
    pr = ora.pairs(sc, [cam], ts=ts)
    tiles_x = (40 + ts - 1) // ts
    cover = {}
    for k, v in zip(pr["keys"], pr["vals"]):
        cover.setdefault(int(v), set()).add(int(k >> np.uint64(32)))
    g = sc["geom"].astype(np.float64)
    checked = 0
    for y in range(36):
        for x in range(40):
            o, d = _ray(cam, x, y)
            tile = (y // ts) * tiles_x + x // ts
            for i in np.where(_hits(o, d, g[:, :3], g[:, 3]))[0]:
                assert tile in cover.get(int(i), set()), (i, x, y)
                checked += 1
    assert checked > 200


def test_pairs_sorted_and_depth_ordered(ora):
    sc = synth.scene_tiny()
    cams = [synth.orbit_camera(64, 48, 60.0, 1.6, a, 25.0, target=(0.5, 0.4, 0.5)) for a in (10.0, 140.0)]
    pr = ora.pairs(sc, cams, ts=16)
    keys, vals = pr["keys"], pr["vals"]
    assert pr["n_pairs"] > 1000
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) or np.all(keys[1:] >= keys[:-1])
    tile = (keys >> np.uint64(32)).astype(np.int64)
    # within a tile, the depth key follows the FP64 camera depth of the voxel centre
    R0 = np.asarray(cams[0]["w2c"], np.float64).reshape(3, 4)
    R1 = np.asarray(cams[1]["w2c"], np.float64).reshape(3, 4)
    g = sc["geom"].astype(np.float64)
    tiles0 = ((64 + 15) // 16) * ((48 + 15) // 16)
    for a in range(len(keys) - 1):
        if tile[a] != tile[a + 1]:
            continue
        R = R0 if tile[a] < tiles0 else R1
        za = R[2, :3] @ g[vals[a], :3] + R[2, 3]
        zb = R[2, :3] @ g[vals[a + 1], :3] + R[2, 3]
        assert za <= zb + 1e-6
        if keys[a] == keys[a + 1]:
            assert vals[a] < vals[a + 1]
    # tile ranges partition the list
    rng = pr["ranges"]
    nonempty = rng[:, 1] > rng[:, 0]
    assert rng[nonempty, 1].max() == len(keys)
    for t in np.where(nonempty)[0]:
        assert np.all(tile[rng[t, 0]:rng[t, 1]] == t)
    assert (rng[nonempty, 1] - rng[nonempty, 0]).sum() == len(keys)


def test_pairs_statistics(ora):
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(64, 64, 60.0, 1.6, 10.0, 25.0, target=(0.5, 0.4, 0.5))
    pr = ora.pairs(sc, [cam])
    seen = pr["seen"].astype(bool)
    assert seen.sum() > 100
    R = np.asarray(cam["w2c"], np.float64).reshape(3, 4)
    z = sc["geom"][:, :3].astype(np.float64) @ R[2, :3] + R[2, 3]
    np.testing.assert_allclose(pr["z_min"][seen], np.maximum(z[seen], 0.05), rtol=1e-6)
    np.testing.assert_allclose(pr["delta_min"][seen], np.maximum(z[seen], 0.05) / cam["fx"], rtol=1e-6)
    assert np.all(np.isinf(pr["z_min"][~seen]))


def test_footprint_floor_at_the_near_plane(ora):
    # delta_v is the ray spacing at the voxel's depth, and no seen voxel sits closer than the near plane:
    # every footprint is at least z_near / f_x, and a voxel whose centre lies in front of the near plane
    # (seen through its far part) gets exactly that floor, with z_min = z_near.
    rng = np.random.default_rng(8)
    n = 200
    centers = np.c_[rng.uniform(-0.5, 0.5, n), rng.uniform(-0.4, 0.4, n), rng.uniform(-0.2, 1.5, n)]
    sc = synth.constant_voxel_scene(centers, rng.uniform(0.05, 0.4, n), np.ones(n), np.ones((n, 3)) * 0.5)
    cam = {"width": 48, "height": 40, "fx": 30.0, "fy": 30.0, "cx": 24.0, "cy": 20.0,
           "w2c": [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], "z_near": 0.3}
    pr = ora.pairs(sc, [cam], ts=8)
    seen = pr["seen"].astype(bool)
    floor_ = np.float32(np.float32(0.3) / np.float32(30.0))
    behind = seen & (sc["geom"][:, 2] < np.float32(0.3))
    assert seen.sum() > 50 and behind.sum() > 5
    assert np.all(pr["delta_min"][seen] >= floor_) and np.all(pr["z_min"][seen] >= np.float32(0.3))
    assert np.all(pr["delta_min"][behind] == floor_) and np.all(pr["z_min"][behind] == np.float32(0.3))


# --------------------------------------------------------------------- pruning

def test_ema_hysteresis_hand_trace(ora):
    # Stored hand trace (tests/golden/ema_hysteresis_trace.json): with m0 = 1 and alpha = 0.1,
    # voxel 0 always votes "out" (its w_max is the bin minimum) and flips to out at step 12.
    spec = json.load(open(os.path.join(GOLDEN, "ema_hysteresis_trace.json")))
    n = 20
    w = np.linspace(0.1, 1.0, n).astype(np.float32)       # voxel 0 is the unique minimum
    seen = np.ones(n, np.uint8)
    z = np.ones(n, np.float32)                            # one depth bin
    m = np.ones(n, np.float32)
    s = np.ones(n, np.uint8)
    states = []
    for step in range(spec["steps"]):
        r = ora.prune(w, seen, z, m, s, n_bins=16, q_ppm=50000, ema_alpha=0.1, m_low=0.3, m_high=0.7,
                      cap_ppm=1000000)
        m, s = r["m"], r["s"]
        states.append(int(s[0]))
        assert abs(float(m[0]) - spec["m_voxel0"][step]) < 1e-6
    assert states == spec["state_voxel0"]
    assert int(np.argmax(np.array(states) == 0)) + 1 == spec["first_out_step"]


def test_hysteresis_band_holds_state(ora):
    # m inside [m_low, m_high] keeps the previous state (guard i).
    w = np.array([0.1, 0.5, 0.9], np.float32)
    seen = np.ones(3, np.uint8)
    z = np.ones(3, np.float32)
    m = np.array([0.5, 0.5, 0.5], np.float32)
    s_in = np.array([1, 1, 1], np.uint8)
    s_out = np.array([0, 0, 0], np.uint8)
    r1 = ora.prune(w, seen, z, m, s_in, q_ppm=330000, cap_ppm=1000000)   # k = ceil(0.99) = 1
    r2 = ora.prune(w, seen, z, m, s_out, q_ppm=330000, cap_ppm=1000000)
    # voxel 0 votes out (w <= tau = 0.1): m = 0.45; voxels 1, 2 vote in: m = 0.55 -> all stay
    np.testing.assert_allclose(r1["m"], [0.45, 0.55, 0.55], rtol=1e-6)
    assert list(r1["s"]) == [1, 1, 1] and list(r2["s"]) == [0, 0, 0]
    assert r1["n_pruned"] == 0 and r2["n_pruned"] == 3
    # the band is closed: m landing exactly on m_low or m_high (exact in FP32 with alpha = 1/2) keeps the state
    m_edge = np.array([0.6, 0.4, 0.4], np.float32)             # 0.6 / 2 = 0.3 ; 0.4 / 2 + 1/2 = 0.7
    r3 = ora.prune(w, seen, z, m_edge, s_in, q_ppm=330000, cap_ppm=1000000, ema_alpha=0.5)
    r4 = ora.prune(w, seen, z, m_edge, s_out, q_ppm=330000, cap_ppm=1000000, ema_alpha=0.5)
    assert r3["m"][0] == np.float32(0.3) and r3["m"][1] == np.float32(0.7)
    assert list(r3["s"]) == [1, 1, 1] and list(r4["s"]) == [0, 0, 0]


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_quantile_thresholds_brute_force(ora, seed):
    # tau_b is the nearest-rank q-quantile of w_max within each depth bin (Eq. 11-12),
    # recomputed here with numpy's sort over the bins implied by Eq. 14.
    rng = np.random.default_rng(seed)
    n = 3000
    w = rng.uniform(0, 1, n).astype(np.float32)
    w[rng.integers(0, n, 300)] = np.float32(0.25)          # ties
    z = rng.gamma(2.0, 2.0, n).astype(np.float32)
    seen = (rng.uniform(size=n) < 0.9).astype(np.uint8)
    m = np.ones(n, np.float32)
    s = np.ones(n, np.uint8)
    q = [50000, 200000, 500000, 999999][seed]
    r = ora.prune(w, seen, z, m, s, n_bins=16, q_ppm=q, cap_ppm=1000000)
    zs = np.sort(z[seen == 1])
    ns = len(zs)
    p5 = zs[max(1, math.ceil(0.05 * ns)) - 1]
    p95 = zs[max(1, math.ceil(0.95 * ns)) - 1]
    assert r["p_lo"] == p5 and r["p_hi"] == p95
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
        checked += 1
        vals = np.sort(w[sel])
        k = max(1, -(-q * len(vals) // 1000000))
        assert r["tau"][bb] == vals[k - 1]
        # inside score: x = [w > tau_b]; from m = 1: m' = 0.9 + 0.1 x
        x = (w[sel] > vals[k - 1]).astype(np.float64)
        np.testing.assert_allclose(r["m"][sel], 0.9 + 0.1 * x, rtol=1e-6)
    assert checked >= 8
    assert np.all(r["m"][seen == 0] == 1.0)


def test_cap_prunes_smallest(ora):
    # Guard iii: more out-state candidates than the cap -> the cap smallest (w_max, id) go.
    rng = np.random.default_rng(5)
    n = 1000
    w = rng.uniform(0.01, 1, n).astype(np.float32)
    w[10:20] = np.float32(0.001)                       # ties at the bottom, broken by id
    seen = np.ones(n, np.uint8)
    z = np.ones(n, np.float32)
    m = np.full(n, 0.1, np.float32)                     # everyone is already "out"
    s = np.zeros(n, np.uint8)
    w[0:5] = np.float32(0.001)
    r = ora.prune(w, seen, z, m, s, cap_ppm=8000)       # cap = 8
    assert r["n_pruned"] == 8
    order = np.lexsort((np.arange(n), w))
    expect = np.zeros(n, np.uint8)
    expect[order[:8]] = 1
    np.testing.assert_array_equal(r["mask"], expect)
    assert set(np.where(r["mask"])[0]) == {0, 1, 2, 3, 4, 10, 11, 12}
    # the cap is a fraction of all voxels, not of those seen this step: with 300 unseen voxels it stays 8
    seen[600:900] = 0
    r = ora.prune(w, seen, z, m, s, cap_ppm=8000)
    assert r["n_pruned"] == 8
    assert set(np.where(r["mask"])[0]) == {0, 1, 2, 3, 4, 10, 11, 12}
    # "at most" the fraction: 0.85 % of 1000 voxels prunes 8, never 9
    assert ora.prune(w, seen, z, m, s, cap_ppm=8500)["n_pruned"] == 8


def test_prune_degenerate_cases(ora):
    n = 50
    w = np.full(n, 0.5, np.float32)
    z = np.full(n, 3.0, np.float32)                    # p95 == p5 -> z~ = 0, one bin
    seen = np.ones(n, np.uint8)
    r = ora.prune(w, seen, z, np.ones(n, np.float32), np.ones(n, np.uint8), cap_ppm=1000000)
    assert r["tau"][0] == np.float32(0.5)
    np.testing.assert_allclose(r["m"], 0.9, rtol=1e-6)  # all tied at tau -> all vote out
    r = ora.prune(w, np.zeros(n, np.uint8), z, np.ones(n, np.float32), np.zeros(n, np.uint8))
    assert r["n_pruned"] == 0 and np.all(r["m"] == 1.0)  # nothing seen: nothing changes


# --------------------------------------------------------------------- subdivision

def _scene_rand(n, seed):
    rng = np.random.default_rng(seed)
    sc = synth.constant_voxel_scene(rng.uniform(-1, 1, (n, 3)), rng.uniform(0.01, 0.2, n), np.ones(n),
                                    np.ones((n, 3)) * 0.5)
    sc["density"] = rng.normal(2, 1, (n, 8)).astype(np.float32)
    sc["sh"] = rng.normal(0, 1, (n, 48)).astype(np.float32)
    sc["level"] = rng.integers(3, 17, n).astype(np.uint8)
    return sc


def test_subdivide_selection_brute_force(ora):
    n = 2000
    sc = _scene_rand(n, 11)
    rng = np.random.default_rng(12)
    delta = rng.uniform(0.0, 0.2, n).astype(np.float32)
    z = rng.uniform(1, 20, n).astype(np.float32)
    u = rng.uniform(0, 1, n).astype(np.float32)
    u[:200] = np.float32(0.5)                           # ties broken by id
    seen = (rng.uniform(size=n) < 0.8).astype(np.uint8)
    pm = (rng.uniform(size=n) < 0.1).astype(np.uint8)
    r = ora.subdivide(sc, delta, z, u, seen, prune_mask=pm, kappa=1.0, beta=0.2, top_ppm=50000, l_max=16)
    alive = pm == 0
    fl = alive & (seen == 1)
    zs = np.sort(z[fl])
    p5, p95 = zs[math.ceil(0.05 * len(zs)) - 1], zs[math.ceil(0.95 * len(zs)) - 1]
    zt = np.clip((z.astype(np.float64) - p5) / (p95 - p5), 0, 1)
    pri = u.astype(np.float64) * (1 + 0.2 * zt)
    elig = fl & (sc["level"] < 16) & (sc["geom"][:, 3].astype(np.float64) > delta.astype(np.float64))
    k = min(int(0.05 * alive.sum()), int(elig.sum()))
    assert r["k"] == k
    ids = np.where(elig)[0]
    order = ids[np.lexsort((ids, -pri[ids]))]
    # FP32 rounding can swap near-equal priorities; compare where the gap is clear
    thr = pri[order[k - 1]]
    clear = np.abs(pri - thr) > 1e-5
    sel = r["selected"].astype(bool)
    assert sel.sum() == k
    assert np.all(sel[order[:k]][clear[order[:k]]])
    assert not np.any(sel[clear & ~np.isin(np.arange(n), order[:k])])
    assert r["n_new"] == alive.sum() + 7 * k


def test_subdivide_children_geometry_and_fields(ora):
    # Children tile the parent exactly and inherit its trilinear field; linear fields are reproduced.
    sc = synth.constant_voxel_scene([[0.25, -0.5, 1.0]], 0.5, [0.0], [(0.2, 0.4, 0.6)])
    a, b = np.array([1.5, -2.0, 0.5]), 0.75
    corners = np.array([[(i & 1) * 2 - 1, ((i >> 1) & 1) * 2 - 1, ((i >> 2) & 1) * 2 - 1] for i in range(8)], float)
    sc["density"][0] = ((corners * 0.5 + sc["geom"][0, :3]) @ a + b).astype(np.float32)
    sc["level"][:] = 4
    aux_m = np.array([[0.3] * 8], np.float32)
    aux_e = np.array([0.42], np.float32)
    aux_s = np.array([0], np.uint8)
    aux_h = np.array([[7, 9, 11]], np.uint16)            # 2-byte elements: FP16 moments, for example
    r = ora.subdivide(sc, np.zeros(1, np.float32), np.ones(1, np.float32), np.ones(1, np.float32),
                      np.ones(1, np.uint8), top_ppm=1000000,
                      aux=[(aux_m, 0.0), (aux_e, 1.0), (aux_s, 1), (aux_h, 0x3C00)])
    assert r["n_new"] == 8
    g = r["geom"]
    np.testing.assert_array_equal(g[:, 3], 0.25)
    assert np.all(r["level"] == 5)
    for i in range(8):
        off = np.array([(i & 1) * 2 - 1, ((i >> 1) & 1) * 2 - 1, ((i >> 2) & 1) * 2 - 1]) * 0.25
        np.testing.assert_array_equal(g[i, :3], sc["geom"][0, :3] + off)
        cc = corners * 0.25 + g[i, :3]
        np.testing.assert_allclose(r["density"][i], cc @ a + b, atol=1e-5)
    assert np.all(r["sh"] == sc["sh"][0])
    assert np.all(r["aux"][0] == 0) and np.all(r["aux"][1] == 1.0) and np.all(r["aux"][2] == 1)
    assert r["aux"][3].shape == (8, 3) and np.all(r["aux"][3] == 0x3C00)   # each child element takes the fill
    # volumes add up
    assert abs((8 * g[:, 3] ** 3).sum() - 8 * 0.5 ** 3) < 1e-12


def test_subdivide_budget_and_output_order(ora):
    n = 100
    sc = _scene_rand(n, 21)
    sc["level"][:] = 5
    u = np.arange(n, dtype=np.float32)[::-1].copy()     # voxel 0 has the highest priority
    pm = np.zeros(n, np.uint8)
    pm[[3, 7]] = 1
    r = ora.subdivide(sc, np.zeros(n, np.float32), np.ones(n, np.float32), u, np.ones(n, np.uint8),
                      prune_mask=pm, top_ppm=1000000, budget=98 + 21, aux=[(np.arange(n, dtype=np.float32), -1.0)])
    # alive = 98; budget allows floor(21 / 7) = 3 splits: voxels 0, 1, 2
    assert r["k"] == 3
    assert list(np.where(r["selected"])[0]) == [0, 1, 2]
    surv = [i for i in range(n) if i not in (0, 1, 2, 3, 7)]
    np.testing.assert_array_equal(r["aux"][0][:len(surv)], np.array(surv, np.float32))
    assert np.all(r["aux"][0][len(surv):] == -1.0)
    np.testing.assert_array_equal(r["geom"][:len(surv)], sc["geom"][surv])
    assert r["n_new"] == len(surv) + 24
    # budget already reached -> nothing is split
    r = ora.subdivide(sc, np.zeros(n, np.float32), np.ones(n, np.float32), u, np.ones(n, np.uint8),
                      top_ppm=1000000, budget=50)
    assert r["k"] == 0 and r["n_new"] == n


def test_subdivide_eligibility(ora):
    # Eq. 13: h > kappa * delta and level < l_max; unseen voxels are not eligible.
    sc = synth.constant_voxel_scene(np.zeros((4, 3)), [0.1, 0.1, 0.1, 0.1], np.ones(4), np.ones((4, 3)))
    sc["level"][:] = [3, 16, 3, 3]
    delta = np.array([0.05, 0.05, 0.2, 0.05], np.float32)
    seen = np.array([1, 1, 1, 0], np.uint8)
    r = ora.subdivide(sc, delta, np.ones(4, np.float32), np.ones(4, np.float32), seen, top_ppm=1000000,
                      kappa=1.0, l_max=16)
    assert list(r["selected"]) == [1, 0, 0, 0]
    # the inequality is strict: h = kappa * delta exactly (kappa a power of two) is not eligible
    for kappa in (1.0, 2.0, 0.5):
        d = np.array([0.1 / kappa, 0.1 / kappa * 0.999, 0.1 / kappa * 1.001, 0.05 / kappa], np.float32)
        assert np.float32(kappa) * d[0] == sc["geom"][0, 3]
        r = ora.subdivide(sc, d, np.ones(4, np.float32), np.ones(4, np.float32), np.ones(4, np.uint8),
                          top_ppm=1000000, kappa=kappa, l_max=17)
        assert list(r["selected"]) == [0, 1, 0, 1]


def test_subdivide_equal_priorities_take_the_smallest_ids(ora):
    # With every priority equal, the budgeted top-k is the k eligible voxels with the smallest ids.
    n = 100
    sc = _scene_rand(n, 31)
    sc["level"][:] = 4
    sc["level"][[2, 5, 11]] = 16                        # at l_max: not eligible
    r = ora.subdivide(sc, np.zeros(n, np.float32), np.full(n, 3.0, np.float32), np.full(n, 0.25, np.float32),
                      np.ones(n, np.uint8), top_ppm=100000, l_max=16)
    assert r["k"] == 10
    assert list(np.where(r["selected"])[0]) == [0, 1, 3, 4, 6, 7, 8, 9, 10, 12]


def test_compact_is_subdivision_without_splits(ora):
    """Compaction (removing pruned voxels) equals the C subdivision with no
    split allowed and prune_mask = !keep, for the voxel and auxiliary arrays."""
    n = 300
    sc = _scene_rand(n, 5)
    rng = np.random.default_rng(5)
    keep = (rng.uniform(size=n) < 0.7).astype(np.uint8)
    aux = [rng.normal(size=(n, 8)).astype(np.float32), rng.integers(0, 255, size=n).astype(np.uint8),
           rng.integers(0, 60000, size=(n, 3)).astype(np.uint16)]
    c = ora.compact(sc, keep, aux)
    r = ora.subdivide(sc, np.zeros(n, np.float32), np.ones(n, np.float32), np.ones(n, np.float32),
                      np.ones(n, np.uint8), prune_mask=1 - keep, top_ppm=0, aux=[(a, 0) for a in aux])
    assert r["k"] == 0 and c["n_new"] == r["n_new"] == int(keep.sum())
    for name in ("geom", "level", "density", "sh"):
        np.testing.assert_array_equal(c[name], r[name])
    for x, y in zip(c["aux"], r["aux"]):
        np.testing.assert_array_equal(x, y)
    # order: the i-th kept row is the i-th index with keep set
    np.testing.assert_array_equal(c["geom"], np.asarray(sc["geom"])[np.flatnonzero(keep)])
    # degenerate masks
    assert ora.compact(sc, np.zeros(n, np.uint8))["n_new"] == 0
    np.testing.assert_array_equal(ora.compact(sc, np.ones(n, np.uint8))["sh"], sc["sh"])


# --------------------------------------------------------------------- LF loss

def test_gamma_schedule(ora):
    spec = json.load(open(os.path.join(GOLDEN, "gamma_schedule.json")))
    for t, g in zip(spec["t"], spec["gamma"]):
        assert abs(ora.lf_gamma(t, spec["t0"], spec["t1"], spec["gamma_max"]) - g) < 1e-12


def test_lf_gamma_zero_is_mse(ora):
    rng = np.random.default_rng(0)
    W, H = 17, 11
    rgb = rng.uniform(size=(W * H, 3))
    gt = rng.uniform(size=(W * H, 3))
    r = ora.lf_loss(rgb, gt, [(W, H)], gamma=0.0)
    np.testing.assert_allclose(r["loss"][0], np.mean((rgb - gt) ** 2), rtol=1e-12)
    np.testing.assert_allclose(r["dL_drgb"], 2 * (rgb - gt) / (3 * W * H), rtol=1e-12)


def test_lf_constant_target_is_mse(ora):
    rng = np.random.default_rng(1)
    W, H = 9, 13
    rgb = rng.uniform(size=(W * H, 3))
    gt = np.full((W * H, 3), 0.3)
    r = ora.lf_loss(rgb, gt, [(W, H)], gamma=0.6)
    assert np.all(r["s"] == 0)
    np.testing.assert_allclose(r["w_tilde"], 1.0, rtol=1e-12)
    np.testing.assert_allclose(r["loss"][0], np.mean((rgb - gt) ** 2), rtol=1e-12)


def test_lf_sobel_ramp_and_weights(ora):
    # Y = a x^2: interior Sobel gx = 4 * (Y(x+1) - Y(x-1)) = 16 a x, gy = 0.
    W, H, a = 30, 8, 0.001
    xs = np.tile(np.arange(W, dtype=np.float64), H)
    gt = np.repeat((a * xs ** 2)[:, None], 3, axis=1)
    rgb = gt + 0.1
    r = ora.lf_loss(rgb, gt, [(W, H)], gamma=0.6, eps=1e-3, pctl_ppm=990000)
    s = r["s"].reshape(H, W)
    mag = np.zeros((H, W))
    mag[:, 1:W - 1] = 16 * a * np.arange(1, W - 1)
    mag[:, 0] = 4 * a * 1.0                             # replicate border: Y(1) - Y(0)
    mag[:, W - 1] = 4 * a * ((W - 1) ** 2 - (W - 2) ** 2)
    srt = np.sort(mag.ravel())
    p99 = srt[math.ceil(0.99 * W * H) - 1]
    np.testing.assert_allclose(s, np.clip(mag / p99, 0, 1), rtol=1e-9, atol=1e-12)
    w = (1e-3 + 1 - np.clip(mag / p99, 0, 1)) ** 0.6
    np.testing.assert_allclose(r["w_tilde"].reshape(H, W), w / w.mean(), rtol=1e-9)
    assert abs(r["w_tilde"].mean() - 1.0) < 1e-12
    # flat pixels weigh more than edges once gamma > 0
    assert np.all(r["w_tilde"].reshape(H, W)[:, 1] > r["w_tilde"].reshape(H, W)[:, W // 2])


@pytest.mark.parametrize("W,H,pctl", [(23, 17, 990000), (8, 5, 900000), (1, 7, 500000)])
def test_lf_edge_map_against_scipy(ora, W, H, pctl):
    # s = clip(|Sobel Y| / P, 0, 1) with Y the channel mean, scipy's Sobel with a replicated border, and P the
    # nearest-rank percentile (numpy's "inverted_cdf"); then w~ = (eps + 1 - s)^gamma / mean (Eq. 7-8).
    from scipy import ndimage
    gt = synth.random_image(W, H, seed=W + H).astype(np.float64)
    Y = gt.reshape(H, W, 3).mean(axis=2)
    mag = np.hypot(ndimage.sobel(Y, axis=1, mode="nearest"), ndimage.sobel(Y, axis=0, mode="nearest"))
    P = np.percentile(mag.ravel(), pctl / 1e4, method="inverted_cdf")
    s = np.clip(mag / P, 0, 1) if P > 0 else np.zeros_like(mag)
    r = ora.lf_loss(gt + 0.05, gt, [(W, H)], gamma=0.7, eps=1e-3, pctl_ppm=pctl)
    np.testing.assert_allclose(r["s"].reshape(H, W), s, rtol=1e-12, atol=1e-14)
    w = (1e-3 + 1 - s) ** 0.7
    np.testing.assert_allclose(r["w_tilde"].reshape(H, W), w / w.mean(), rtol=1e-12)


def test_lf_gradient_central_differences(ora):
    rng = np.random.default_rng(2)
    W, H = 7, 6
    rgb = rng.uniform(size=(W * H, 3))
    gt = synth.smooth_image(W, H, seed=3).astype(np.float64)
    r = ora.lf_loss(rgb, gt, [(W, H)], gamma=0.8)
    for _ in range(10):
        p, c = int(rng.integers(W * H)), int(rng.integers(3))
        e = 1e-6
        a = rgb.copy(); a[p, c] += e
        b = rgb.copy(); b[p, c] -= e
        fd = (ora.lf_loss(a, gt, [(W, H)], gamma=0.8)["loss"][0] - ora.lf_loss(b, gt, [(W, H)], gamma=0.8)["loss"][0]) / (2 * e)
        assert abs(fd - r["dL_drgb"][p, c]) < 1e-8


def test_lf_per_view_independence(ora):
    rng = np.random.default_rng(4)
    sizes = [(8, 6), (5, 9)]
    P = sum(w * h for w, h in sizes)
    rgb = rng.uniform(size=(P, 3))
    gt = rng.uniform(size=(P, 3))
    both = ora.lf_loss(rgb, gt, sizes, gamma=0.5)
    a = ora.lf_loss(rgb[:48], gt[:48], [sizes[0]], gamma=0.5)
    b = ora.lf_loss(rgb[48:], gt[48:], [sizes[1]], gamma=0.5)
    np.testing.assert_allclose(both["loss"], [a["loss"][0], b["loss"][0]], rtol=1e-14)


def test_pairs_of_two_views(ora):
    # Binning two views at once: the second view's tiles follow the first view's, every pair of a single-view
    # list appears with its tile id shifted by that offset, and the statistics are the per-view minima (z_min,
    # delta_min) and the union (seen).
    sc = synth.scene_tiny()
    a = synth.orbit_camera(40, 28, 60.0, 1.6, 30.0, 25.0, target=(0.5, 0.4, 0.5))
    b = synth.orbit_camera(24, 36, 50.0, 1.8, 140.0, 10.0, target=(0.5, 0.4, 0.5))
    pa, pb, both = ora.pairs(sc, [a], ts=8), ora.pairs(sc, [b], ts=8), ora.pairs(sc, [a, b], ts=8)
    ta = ((40 + 7) // 8) * ((28 + 7) // 8)
    shift = np.uint64(ta) << np.uint64(32)
    keys = np.concatenate([pa["keys"], pb["keys"] + shift])
    vals = np.concatenate([pa["vals"], pb["vals"]])
    order = np.lexsort((vals, keys))
    np.testing.assert_array_equal(both["keys"], keys[order])
    np.testing.assert_array_equal(both["vals"], vals[order])
    np.testing.assert_array_equal(both["z_min"], np.minimum(pa["z_min"], pb["z_min"]))
    np.testing.assert_array_equal(both["delta_min"], np.minimum(pa["delta_min"], pb["delta_min"]))
    np.testing.assert_array_equal(both["seen"], pa["seen"] | pb["seen"])
    assert (pa["z_min"] < pb["z_min"]).sum() > 10 and (pb["z_min"] < pa["z_min"]).sum() > 10


def test_seen_means_at_least_one_pair(ora):
    # A voxel is seen when it covers at least one tile of some view: exactly the voxels with a pair.  Many
    # voxels of this scene lie beside the narrow view (in front of the camera, not culled, but off screen).
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(40, 30, 25.0, 1.2, 60.0, 20.0, target=(0.45, 0.35, 0.5))
    pr = ora.pairs(sc, [cam], ts=8)
    has_pair = np.isin(np.arange(sc["geom"].shape[0]), pr["vals"])
    np.testing.assert_array_equal(pr["seen"].astype(bool), has_pair)
    np.testing.assert_array_equal(np.isfinite(pr["z_min"]), has_pair)
    M = np.asarray(cam["w2c"], np.float64).reshape(3, 4)
    z = sc["geom"][:, :3].astype(np.float64) @ M[2, :3] + M[2, 3]
    assert ((z > 0.2) & ~has_pair).sum() > 100 and has_pair.sum() > 100


def test_depth_keys_order_negative_centre_depths(ora):
    # A large voxel whose centre lies behind the camera (negative depth) but whose far part is beyond the near
    # plane comes first in its tiles: the depth key orders negative depths below positive ones.
    cam = {"width": 32, "height": 32, "fx": 20.0, "fy": 20.0, "cx": 16.0, "cy": 16.0,
           "w2c": [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], "z_near": 0.05}
    centers = [[0.0, 0.0, -0.3], [0.05, 0.02, 0.8], [-0.1, 0.05, 1.6], [0.02, -0.03, -0.1]]
    sc = synth.constant_voxel_scene(centers, [0.5, 0.1, 0.2, 0.25], np.ones(4), np.ones((4, 3)) * 0.5)
    pr = ora.pairs(sc, [cam], ts=8)
    zc = np.array([c[2] for c in centers])
    tile = (pr["keys"] >> np.uint64(32)).astype(np.int64)
    multi = 0
    for t in np.unique(tile):
        ids = pr["vals"][tile == t].astype(np.int64)
        np.testing.assert_array_equal(ids, ids[np.argsort(zc[ids], kind="stable")])
        multi += len(ids) >= 3 and (zc[ids] < 0).sum() == 2
    assert multi > 0                               # some tile holds both negative-depth voxels and a positive one
