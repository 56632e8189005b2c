"""Pins for the oracle's FP32 error bounds and finite-difference kink margins.

These functions change no result of the method: they tell a parity test how
far an FP32 evaluation may legitimately land from the FP64 oracle (the w_max
argmax ambiguity of Eq. 5, per-element gradient floors of the reverse pass of
Eq. 2-4) and where a central difference would straddle a kink.  Each pin checks
them against something other than their own formulas: brute force over traced
pixels, one-ulp FP32 perturbations of the inputs re-rendered in FP64, float32
summation of per-pixel contributions in random orders, and finite differences.
No GPU is used.
"""
import numpy as np
import pytest

from paper_2511_02510_gb300 import synth


def cam_near(W=32, H=32, az=30.0):
    return synth.orbit_camera(W, H, 60.0, 1.6, az, 25.0, target=(0.5, 0.4, 0.5))


@pytest.fixture(scope="module")
def tiny():
    return synth.scene_tiny()


def perturbed(sc, cam, rng):
    """The scene and camera with every FP32 position and camera entry moved by one ulp, random signs."""
    sc2 = {k: np.array(v, copy=True) for k, v in sc.items()}
    g = sc2["geom"]
    sgn = rng.choice([-1.0, 1.0], size=g[:, :3].shape).astype(np.float32)
    g[:, :3] = np.nextafter(g[:, :3], g[:, :3] + sgn * np.float32(1e30))
    cam2 = dict(cam)
    w = np.asarray(cam["w2c"], np.float32)
    w = np.nextafter(w, w + rng.choice([-1.0, 1.0], size=w.shape).astype(np.float32) * np.float32(1e30))
    cam2["w2c"] = w.tolist()
    return sc2, cam2


def set_lookup(ws, v, pix):
    """Index of entry (v, pix) in the sorted near-max set, or -1."""
    key = ws["set_v"] * (1 << 32) + ws["set_pix"]
    q = np.asarray(v, np.int64) * (1 << 32) + np.asarray(pix, np.int64)
    i = np.searchsorted(key, q)
    i = np.minimum(i, len(key) - 1)
    return np.where(key[i] == q, i, -1)


def test_wmax_sets_agree_with_render(ora, tiny):
    cams = [cam_near(40, 30), cam_near(24, 36, az=140.0)]
    r = ora.render(tiny, cams)
    ws = ora.wmax_sets(tiny, cams)
    np.testing.assert_array_equal(ws["a1"], r["w_arg"])
    np.testing.assert_array_equal(ws["w1"], r["w_max"])
    hit = ws["a1"] >= 0
    assert hit.sum() > 100
    assert np.all(ws["e1"][hit] > 0) and np.all(ws["w2"][hit] <= ws["w1"][hit])
    # the maximum itself is in its near-max set, and every entry can reach the maximum's lower bound
    assert np.all(set_lookup(ws, np.where(hit)[0], ws["a1"][hit]) >= 0)
    v = ws["set_v"]
    assert np.all(ws["set_w"] + ws["set_e"] >= ws["w1"][v] - ws["e1"][v])


def test_wmax_top2_and_set_by_brute_force(ora, tiny):
    # Every pixel traced on its own: the largest and second-largest weight of each voxel over
    # all rays (the tie rule of Eq. 5's argmax: smallest pixel id), and every sample whose weight
    # reaches w1 - e1 belongs to the near-max set.
    cam = cam_near(24, 20, az=75.0)
    ws = ora.wmax_sets(tiny, [cam])
    n = tiny["geom"].shape[0]
    best = np.full(n, -1.0)
    arg = np.full(n, -1, np.int64)
    second = np.full(n, -1.0)
    samples = []
    for y in range(cam["height"]):
        for x in range(cam["width"]):
            tr = ora.trace_pixel(tiny, cam, x, y)
            p = y * cam["width"] + x
            for vid, w in zip(tr["ids"], tr["w"]):
                samples.append((int(vid), p, float(w)))
                if arg[vid] < 0 or w > best[vid]:
                    if arg[vid] >= 0:
                        second[vid] = max(second[vid], best[vid])
                    best[vid], arg[vid] = w, p
                else:
                    second[vid] = max(second[vid], w)
    np.testing.assert_array_equal(ws["a1"], arg)
    np.testing.assert_array_equal(ws["w1"], np.where(arg >= 0, best, 0.0))
    np.testing.assert_array_equal(ws["w2"], second)
    sv = np.array([s[0] for s in samples])
    sp = np.array([s[1] for s in samples])
    sw = np.array([s[2] for s in samples])
    near = sw >= ws["w1"][sv] - ws["e1"][sv]
    assert np.all(set_lookup(ws, sv[near], sp[near]) >= 0)
    # the set's weights of real samples are the traced weights
    idx = set_lookup(ws, sv, sp)
    found = idx >= 0
    np.testing.assert_array_equal(ws["set_w"][idx[found]], sw[found])


@pytest.mark.parametrize("az", [30.0, 200.0])
def test_wmax_bound_covers_fp32_perturbations(ora, tiny, az):
    # One-ulp FP32 perturbations of every voxel position and camera entry, re-rendered in FP64:
    # the perturbed maximum stays within [w1 - e1, the largest w + e of the near-max set], its
    # argmax lands in the near-max set, and every voxel with a certain hit is still hit.
    cam = cam_near(40, 40, az)
    ws = ora.wmax_sets(tiny, [cam])
    r0 = ora.render(tiny, [cam])
    n = tiny["geom"].shape[0]
    top = np.zeros(n)
    np.maximum.at(top, ws["set_v"], ws["set_w"] + ws["set_e"])
    rng = np.random.default_rng(11)
    moved = 0
    for trial in range(3):
        sc2, cam2 = perturbed(tiny, cam, rng)
        r1 = ora.render(sc2, [cam2])
        stop_px = np.where((r0["near_stop"] | r1["near_stop"]) != 0)[0]
        # voxels whose maximum may come from beyond an ambiguous stop are checked by the stop rule instead
        hit1 = r1["w_arg"] >= 0
        ok = hit1 & ~np.isin(r1["w_arg"], stop_px) & ~np.isin(ws["a1"], stop_px)
        w1 = r1["w_max"]
        assert np.all(w1[ok] >= ws["w1"][ok] - ws["e1"][ok])
        assert np.all(w1[ok] <= top[ok])
        assert np.all(set_lookup(ws, np.where(ok)[0], r1["w_arg"][ok]) >= 0)
        cert = ws["n_certain"] > 0
        assert np.all(hit1[cert])
        moved += int(np.sum(w1[ok] != ws["w1"][ok]))
    assert moved > 0   # the perturbations did move the weights


def test_backward_geometric_bound_covers_fp32_perturbations(ora, tiny):
    # The geometric part of the gradient floor (full minus arithmetic) covers what one-ulp FP32
    # perturbations of the voxel positions and of the camera do to the FP64 gradients.
    cam = cam_near(40, 40, 250.0)
    P = 40 * 40
    rng = np.random.default_rng(5)
    gC = rng.normal(size=(P, 3))
    gD = 0.1 * rng.normal(size=P)
    gT = rng.normal(size=P)
    r0 = ora.render(tiny, [cam])
    sc2, cam2 = perturbed(tiny, cam, rng)
    r1 = ora.render(sc2, [cam2])
    stop = (r0["near_stop"] | r1["near_stop"]) != 0
    gC[stop], gD[stop], gT[stop] = 0, 0, 0
    b0 = ora.render_backward(tiny, [cam], gC, gD, gT)
    b1 = ora.render_backward(sc2, [cam2], gC, gD, gT)
    e = ora.backward_bounds(tiny, [cam], gC, gD, gT)
    for k, ek, ak in (("d_density", "e_density", "a_density"), ("d_sh", "e_sh", "a_sh")):
        geo = e[ek] - e[ak]
        diff = np.abs(b1[k] - b0[k])
        assert np.all(geo >= 0) and np.all(e[ak] >= 0)
        assert np.all(diff <= geo + 1e-15), (k, (diff - geo).max())
        assert diff.max() > 0


def test_backward_arithmetic_bound_covers_float32_summation(ora, tiny):
    # The per-element gradient is a sum of per-pixel contributions (the reverse pass of Eq. 2-4 summed
    # over rays).  Each pixel's contribution, taken from the oracle with a one-pixel crop, rounded to
    # FP32 and summed in FP32 in random orders, stays within the arithmetic floor of the total.
    cam = cam_near(16, 16, 60.0)
    P = 16 * 16
    rng = np.random.default_rng(8)
    gC = rng.normal(size=(P, 3))
    tot = ora.render_backward(tiny, [cam], gC)
    e = ora.backward_bounds(tiny, [cam], gC)
    parts = []
    for y in range(16):
        for x in range(16):
            parts.append(ora.render_backward(tiny, [cam], gC, crop=[x, y, x + 1, y + 1])["d_density"])
    parts = np.stack(parts)
    np.testing.assert_allclose(parts.sum(0), tot["d_density"], rtol=1e-12, atol=1e-15)
    p32 = parts.astype(np.float32)
    worst = np.zeros_like(tot["d_density"])
    for trial in range(4):
        order = rng.permutation(P)
        acc = np.zeros(tot["d_density"].shape, np.float32)
        for i in order:
            acc = acc + p32[i]
        worst = np.maximum(worst, np.abs(acc.astype(np.float64) - tot["d_density"]))
    assert np.all(worst <= e["a_density"] + 1e-15), (worst - e["a_density"]).max()
    nz = np.abs(tot["d_density"]) > 0
    assert worst[nz].max() > 0


def test_fd_margins_find_kinks(ora, tiny):
    # Away from the margins a central difference of the FP64 render agrees with the reverse pass
    # to high accuracy; a voxel whose density is moved onto the clamp max(0, .) reports a margin
    # below the step, and the difference across it disagrees.
    cam = cam_near(24, 24, 110.0)
    P = 24 * 24
    rng = np.random.default_rng(2)
    g = rng.normal(size=(P, 3))
    m = ora.fd_margins(tiny, [cam])
    b = ora.render_backward(tiny, [cam], g)
    h = 1e-4

    def loss(sc):
        return float((ora.render(sc, [cam])["rgb"] * g).sum())

    safe = np.where((m["m_sigma"] > 50 * h) & (m["m_stop"] > 50 * h) & np.isfinite(m["m_sigma"]))[0]
    assert len(safe) > 50
    for v in rng.choice(safe, size=6, replace=False):
        i = int(rng.integers(8))
        sc = {k: np.array(a, copy=True) for k, a in tiny.items()}
        x0 = sc["density"][v, i]
        sc["density"][v, i] = np.float32(x0 + h)
        hp = float(sc["density"][v, i]) - float(x0)
        lp = loss(sc)
        sc["density"][v, i] = np.float32(x0 - h)
        hm = float(sc["density"][v, i]) - float(x0)
        lm = loss(sc)
        fd = (lp - lm) / (hp - hm)
        an = b["d_density"][v, i]
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (v, i, fd, an)
    # plant a kink: all corners of a sampled voxel at +-h/4 around zero put its sigma_raw inside the step
    v = int(safe[0])
    sc = {k: np.array(a, copy=True) for k, a in tiny.items()}
    sc["density"][v] = np.float32(h / 4) * np.array([1, -1, 1, -1, -1, 1, -1, 1], np.float32)
    m2 = ora.fd_margins(sc, [cam])
    assert m2["m_sigma"][v] < h
    # the colour margin is the pre-clamp colour: a DC term of -0.5 / Y_0 puts a channel at the clamp
    sc = {k: np.array(a, copy=True) for k, a in tiny.items()}
    sc["sh"][v, 0:3] = np.float32(-0.5 / 0.28209479177387814)
    sc["sh"][v, 3:] = 0
    m3 = ora.fd_margins(sc, [cam])
    assert np.all(m3["m_color"][v] < 1e-6)
