"""Pins for the oracle's renderer (Eq. 1-5) and its backward pass.

Each test checks the oracle against something other than itself: a closed
form, an invariant of Eq. 2-4, a brute-force construction, or finite
differences.  No GPU is used.
"""
import math

import numpy as np
import pytest

from paper_2511_02510_gb300 import synth


def axis_camera(W=3, H=3, f=2.0, eye=(0.0, 0.0, 0.0)):
    """Camera at ``eye`` looking down +z with identity rotation; the centre pixel ray is exactly +z."""
    e = np.asarray(eye, np.float64)
    w2c = [1, 0, 0, -e[0], 0, 1, 0, -e[1], 0, 0, 1, -e[2]]
    return {"width": W, "height": H, "fx": f, "fy": f, "cx": W / 2.0, "cy": H / 2.0, "w2c": w2c, "z_near": 0.05}


def ray_of(cam, x, y):
    R = np.asarray(cam["w2c"], np.float64).reshape(3, 4)[:, :3]
    t = np.asarray(cam["w2c"], np.float64).reshape(3, 4)[:, 3]
    o = -R.T @ t
    dc = np.array([(x + 0.5 - cam["cx"]) / cam["fx"], (y + 0.5 - cam["cy"]) / cam["fy"], 1.0])
    d = R.T @ dc
    return o, d / np.linalg.norm(d)


def chord_by_bisection(o, d, center, h, t_max=100.0, steps=200000):
    """Entry/exit of a ray through an axis-aligned box by dense sampling + bisection.

    Independent of any slab formula: it only evaluates the point-in-box predicate.
    """
    inside = lambda t: bool(np.all(np.abs(o + t * d - center) <= h))
    ts = np.linspace(0.0, t_max, steps)
    pts = o[None, :] + ts[:, None] * d[None, :]
    ins = np.all(np.abs(pts - center[None, :]) <= h, axis=1)
    if not ins.any():
        return None
    i0 = int(np.argmax(ins))
    i1 = len(ins) - 1 - int(np.argmax(ins[::-1]))

    def bis(a, b, want_in_at_b):
        for _ in range(80):
            m = 0.5 * (a + b)
            if inside(m) == want_in_at_b:
                b = m
            else:
                a = m
        return 0.5 * (a + b)

    t_in = 0.0 if i0 == 0 else bis(ts[i0 - 1], ts[i0], True)
    t_out = bis(ts[min(i1 + 1, len(ts) - 1)], ts[i1], True)
    return t_in, t_out


def test_single_voxel_axis_aligned(ora):
    # Centre pixel ray is +z; voxel of half-size 0.5 at z=5: chord l = 2h = 1 exactly.
    cam = axis_camera()
    c = 2.0
    col = (0.25, 0.5, 0.75)
    sc = synth.constant_voxel_scene([[0.0, 0.0, 5.0]], 0.5, [c], [col])
    r = ora.render(sc, [cam], sh_degree=0)
    p = 1 * 3 + 1
    alpha = 1.0 - math.exp(-c * 1.0)
    np.testing.assert_allclose(r["T"][p], 1.0 - alpha, rtol=0, atol=1e-6)  # colour stored as FP32 SH
    np.testing.assert_allclose(r["rgb"][p], alpha * np.asarray(col), rtol=0, atol=1e-6)
    np.testing.assert_allclose(r["depth"][p], alpha * 5.0, rtol=1e-12)
    assert r["n_hit"][p] == 1
    assert r["w_arg"][0] >= 0
    np.testing.assert_allclose(r["w_max"][0], alpha, rtol=1e-12)


@pytest.mark.parametrize("seed,aspect", [(0, 1.0), (1, 1.0), (2, 1.0), (3, 1.37), (0, 0.71)])
def test_single_voxel_oblique_chord(ora, seed, aspect):
    # alpha = 1 - exp(-sigma * l) with l measured by bisection on the inside predicate;
    # aspect != 1: non-square pixels (fy = aspect * fx).
    rng = np.random.default_rng(seed)
    center = rng.uniform(-0.3, 0.3, 3)
    h = 0.4
    cam = synth.look_at_camera(rng.uniform(-1, 1, 3) + np.array([0, 0, -4.0]), center + rng.uniform(-.1, .1, 3),
                               16, 16, 40.0)
    cam["fy"] = float(np.float32(cam["fx"] * aspect))
    c = 1.7
    sc = synth.constant_voxel_scene([center], h, [c], [(1.0, 1.0, 1.0)])
    r = ora.render(sc, [cam], sh_degree=0)
    hits = 0
    for y in range(16):
        for x in range(16):
            o, d = ray_of(cam, x, y)
            ch = chord_by_bisection(o, d, center.astype(np.float32).astype(np.float64), np.float64(np.float32(h)),
                                    t_max=8.0, steps=4001)
            p = y * 16 + x
            if ch is None:
                assert r["n_hit"][p] == 0 and r["T"][p] == 1.0
                continue
            hits += 1
            l = ch[1] - ch[0]
            alpha = 1.0 - math.exp(-np.float32(c) * l)
            assert abs(r["T"][p] - (1.0 - alpha)) < 1e-9
            assert abs(r["depth"][p] - alpha * 0.5 * (ch[0] + ch[1])) < 1e-8
            assert abs(r["rgb"][p][0] - alpha) < 1e-6
    assert hits > 20


def test_linear_density_field(ora):
    # Corners sampled from sigma(x) = a.x + b; trilinear reproduces it, so the
    # midpoint density is a.p_mid + b with p_mid from the bisected chord.
    center = np.array([0.1, -0.05, 0.0])
    h = 0.5
    a = np.array([0.8, -0.6, 1.1])
    b = 3.0
    corners = np.array([[(i & 1) * 2 - 1, ((i >> 1) & 1) * 2 - 1, ((i >> 2) & 1) * 2 - 1] for i in range(8)], float)
    dens = (corners * h + center) @ a + b
    sc = synth.constant_voxel_scene([center], h, [0.0], [(1, 1, 1)])
    sc["density"][0] = dens.astype(np.float32)
    cam = synth.look_at_camera([0.7, 0.4, -3.5], center, 12, 12, 35.0)
    r = ora.render(sc, [cam], sh_degree=0)
    checked = 0
    for y in range(12):
        for x in range(12):
            o, d = ray_of(cam, x, y)
            ch = chord_by_bisection(o, d, center.astype(np.float32).astype(np.float64), h, t_max=7.0, steps=3001)
            if ch is None:
                continue
            pm = o + 0.5 * (ch[0] + ch[1]) * d
            # the corners were sampled from field(p) = p . a + b
            sigma = max(0.0, float(pm @ a + b))
            alpha = 1.0 - math.exp(-sigma * (ch[1] - ch[0]))
            assert abs(r["T"][y * 12 + x] - (1 - alpha)) < 2e-6
            checked += 1
    assert checked > 10


def test_stacked_voxels_product(ora):
    # Three voxels on the centre ray: T = prod (1 - alpha_k), C = sum T_{k-1} alpha_k c_k in depth order.
    cam = axis_camera()
    zs = [7.0, 4.0, 5.5]          # deliberately not in id order
    dens = [0.7, 1.3, 0.4]
    cols = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    sc = synth.constant_voxel_scene([[0, 0, z] for z in zs], 0.25, dens, cols)
    r = ora.render(sc, [cam], sh_degree=0)
    order = np.argsort(zs)
    T = 1.0
    C = np.zeros(3)
    D = 0.0
    for k in order:
        al = 1.0 - math.exp(-float(np.float32(dens[k])) * 0.5)   # densities are stored as FP32
        C += T * al * np.asarray(cols[k], float)
        D += T * al * zs[k]
        T *= 1.0 - al
    p = 4
    assert abs(r["T"][p] - T) < 1e-12
    np.testing.assert_allclose(r["rgb"][p], C, atol=1e-6)
    assert abs(r["depth"][p] - D) < 1e-6
    assert r["n_hit"][p] == 3


def test_white_scene_partition_of_unity(ora):
    # With every colour = 1, Eq. 2-4 telescope: sum_k w_k + T_final = 1 for every ray.
    sc = synth.scene_tiny()
    sc["sh"][:] = 0.0
    sc["sh"][:, 0:3] = np.float32(0.5 / (0.5 / math.sqrt(math.pi)))
    cam = synth.orbit_camera(48, 48, 60.0, 1.6, 30.0, 25.0, target=(0.5, 0.4, 0.5))
    r = ora.render(sc, [cam])
    s = r["rgb"][:, 0] + r["T"]
    np.testing.assert_allclose(s, 1.0, atol=1e-6)
    assert (r["n_hit"] > 0).mean() > 0.2
    assert np.all(r["w_max"] <= 1.0) and np.all(r["w_max"] >= 0.0)


def test_transmittance_monotone_and_weights(ora):
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(32, 32, 60.0, 1.6, 200.0, 35.0, target=(0.5, 0.4, 0.5))
    n_checked = 0
    for (x, y) in [(16, 16), (10, 20), (20, 8), (5, 5), (28, 30)]:
        tr = ora.trace_pixel(sc, cam, x, y)
        if tr["n"] == 0:
            continue
        T = np.concatenate([[1.0], tr["T_after"]])
        assert np.all(np.diff(T) <= 1e-15)
        # w_k = T_{k-1} - T_k  (Eq. 2-3)
        np.testing.assert_allclose(tr["w"], T[:-1] - T[1:], atol=1e-15)
        n_checked += 1
    assert n_checked >= 3


def test_empty_scene(ora):
    sc = synth.constant_voxel_scene(np.zeros((0, 3)), 0.1, np.zeros(0), np.zeros((0, 3)))
    cam = axis_camera(8, 8)
    r = ora.render(sc, [cam])
    assert np.all(r["rgb"] == 0) and np.all(r["T"] == 1) and np.all(r["n_hit"] == 0)


def test_early_stop_rule(ora):
    # The sample that crosses t_stop is included; nothing behind it is processed.
    cam = axis_camera()
    sc = synth.constant_voxel_scene([[0, 0, 4.0], [0, 0, 6.0]], 0.5, [20.0, 1.0], [(1, 1, 1), (1, 1, 1)])
    r = ora.render(sc, [cam], sh_degree=0)
    p = 4
    assert r["n_hit"][p] == 1
    assert abs(r["T"][p] - math.exp(-20.0)) < 1e-15
    assert r["w_arg"][1] == -1 or r["w_arg"][1] != p
    # a t_stop below T keeps marching
    r2 = ora.render(sc, [cam], sh_degree=0, t_stop=1e-12)
    assert r2["n_hit"][p] == 2


def test_stop_count_at_the_threshold(ora):
    # Six equal voxels on the centre ray, each of chord 0.5: T after k samples is exp(-k sigma / 2).
    # sigma puts T_4 between t_stop / 2 and t_stop, so the ray stops after exactly four samples.
    t_stop = 1e-4
    sigma = float(np.float32(-math.log(0.75 * t_stop) / 2.0))
    T = [math.exp(-k * 0.5 * sigma) for k in range(7)]
    assert T[3] > t_stop and 0.5 * t_stop < T[4] < t_stop
    cam = axis_camera()
    sc = synth.constant_voxel_scene([[0, 0, z] for z in (2.0, 3.0, 4.0, 5.0, 6.0, 7.0)], 0.25, [sigma] * 6,
                                    [(1, 1, 1)] * 6)
    r = ora.render(sc, [cam], sh_degree=0, t_stop=t_stop)
    assert r["n_hit"][4] == 4
    assert abs(r["T"][4] - T[4]) < 1e-15
    assert list(r["w_arg"][4:] >= 0) == [False, False]      # the voxels behind the stop are never reached
    # a threshold just below T_4 takes one more sample, and one just above T_3 stops after three
    assert ora.render(sc, [cam], sh_degree=0, t_stop=0.99 * T[4])["n_hit"][4] == 5
    assert ora.render(sc, [cam], sh_degree=0, t_stop=1.01 * T[3])["n_hit"][4] == 3


def test_w_max_ties_go_to_the_smallest_pixel(ora):
    # A voxel so dense that alpha rounds to exactly 1 on every ray with a chord above 0.01: w = 1 ties on all
    # of them, and the argmax is the smallest pixel id whose ray crosses it (chords by bisection).
    W, H = 12, 10
    cam = axis_camera(W, H, 8.0)
    center, h = np.array([0.9, 0.35, 6.0]), 1.5
    sc = synth.constant_voxel_scene([center], h, [1.0e4], [(1, 1, 1)])
    r = ora.render(sc, [cam], sh_degree=0)
    c32, h32 = center.astype(np.float32).astype(np.float64), float(np.float32(h))
    chords = []
    for y in range(H):
        for x in range(W):
            o, d = ray_of(cam, x, y)
            ch = chord_by_bisection(o, d, c32, h32, t_max=12.0, steps=6001)
            chords.append(0.0 if ch is None else ch[1] - ch[0])
    chords = np.array(chords)
    first = int(np.argmax(chords > 0.01))
    assert first > 0 and np.all(chords[:first] == 0.0)      # no grazing ray before it: the tie is well defined
    assert (chords > 0.01).sum() > 10
    assert r["w_max"][0] == 1.0
    assert r["w_arg"][0] == first


def test_culling_near_plane(ora):
    # A voxel entirely in front of z_near is culled even though the ray (t >= 0) crosses it.
    cam = axis_camera()
    cam["z_near"] = 0.5
    sc = synth.constant_voxel_scene([[0, 0, 0.2]], 0.1, [5.0], [(1, 1, 1)])
    r = ora.render(sc, [cam], sh_degree=0)
    assert np.all(r["T"] == 1.0)
    cam["z_near"] = 0.05
    r = ora.render(sc, [cam], sh_degree=0)
    assert r["T"][4] < 1.0


def test_binned_equals_brute_force(ora):
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(40, 40, 60.0, 1.7, 60.0, 20.0, target=(0.5, 0.4, 0.5))
    a = ora.render(sc, [cam])
    b = ora.render(sc, [cam], brute=True)
    for k in ("rgb", "depth", "T", "n_hit", "w_max", "w_arg"):
        np.testing.assert_array_equal(a[k], b[k])


def test_w_max_brute_force(ora):
    # Eq. 5: the max over every ray of T_{k-1} alpha, recomputed from per-pixel traces.
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(20, 20, 50.0, 1.5, 120.0, 30.0, target=(0.5, 0.4, 0.5))
    r = ora.render(sc, [cam])
    best = {}
    for y in range(20):
        for x in range(20):
            tr = ora.trace_pixel(sc, cam, x, y)
            for i, w in zip(tr["ids"], tr["w"]):
                g = y * 20 + x
                if int(i) not in best or w > best[int(i)][0]:
                    best[int(i)] = (w, g)
    assert len(best) > 20
    for i, (w, g) in best.items():
        assert r["w_max"][i] == w
        assert r["w_arg"][i] == g
    untouched = np.setdiff1d(np.arange(len(r["w_arg"])), list(best.keys()))
    assert np.all(r["w_arg"][untouched] == -1)


def test_sh_orthonormal(ora):
    # Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 products exactly.
    xs, ws = np.polynomial.legendre.leggauss(16)
    nphi = 32
    G = np.zeros((16, 16))
    for ct, wt in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for j in range(nphi):
            ph = 2 * math.pi * j / nphi
            Y = ora.sh_basis([st * math.cos(ph), st * math.sin(ph), ct])
            G += np.outer(Y, Y) * wt * (2 * math.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_subdivision_invariance_of_render(ora):
    # A constant-density, constant-colour voxel split into 8 children renders the same image:
    # the children's chords partition the parent's chord.
    cam = synth.look_at_camera([0.6, 0.5, -3.0], [0, 0, 0], 24, 24, 40.0)
    sc = synth.constant_voxel_scene([[0.0, 0.0, 0.0]], 0.5, [2.5], [(0.3, 0.6, 0.9)])
    r0 = ora.render(sc, [cam], sh_degree=0)
    u = np.ones(1, np.float32)
    sub = ora.subdivide(sc, delta=np.zeros(1, np.float32), z=np.ones(1, np.float32), u=u,
                        seen=np.ones(1, np.uint8), top_ppm=1000000, kappa=1.0)
    assert sub["n_new"] == 8
    r1 = ora.render(sub, [cam], sh_degree=0)
    np.testing.assert_allclose(r1["T"], r0["T"], atol=1e-12)
    np.testing.assert_allclose(r1["rgb"], r0["rgb"], atol=1e-6)


def _loss(ora, sc, cam, gC, gD, gT, t_stop):
    r = ora.render(sc, [cam], t_stop=t_stop)
    return float((r["rgb"] * gC).sum() + (r["depth"] * gD).sum() + (r["T"] * gT).sum())


def test_backward_matches_central_differences(ora):
    # Central FP64 differences of L = sum(g_C.rgb + g_D depth + g_T T) against the reverse pass.
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(24, 24, 45.0, 1.4, 75.0, 30.0, target=(0.5, 0.3, 0.5))
    rng = np.random.default_rng(7)
    P = 24 * 24
    gC = rng.normal(size=(P, 3))
    gD = rng.normal(size=P) * 0.1
    gT = rng.normal(size=P)
    t_stop = 1e-4
    r = ora.render(sc, [cam], t_stop=t_stop)
    bw = ora.render_backward(sc, [cam], gC, gD, gT, t_stop=t_stop)
    hit = np.where(r["w_arg"] >= 0)[0]
    assert len(hit) > 30
    pick = rng.choice(hit, size=12, replace=False)
    checked = 0
    for v in pick:
        for kind, idx in (("density", int(rng.integers(8))), ("sh", int(rng.integers(48)))):
            arr = sc[kind]
            x0 = float(arr[v, idx])
            eps = 1e-3 * max(1.0, abs(x0))
            vals = []
            for s_ in (+1, -1, +2, -2):
                sc2 = {k: np.array(a, copy=True) for k, a in sc.items()}
                sc2[kind][v, idx] = np.float32(x0 + s_ * eps)
                actual = float(sc2[kind][v, idx]) - x0
                vals.append((actual, _loss(ora, sc2, cam, gC, gD, gT, t_stop)))
            (hp, lp), (hm, lm), (hp2, lp2), (hm2, lm2) = vals
            fd1 = (lp - lm) / (hp - hm)
            fd2 = (lp2 - lm2) / (hp2 - hm2)
            an = bw["d_density" if kind == "density" else "d_sh"][v, idx]
            scale = max(1e-6, abs(fd1), abs(an))
            if abs(fd1 - fd2) > 1e-3 * scale:
                continue            # a kink (ReLU, clamp or early stop) lies within the step
            assert abs(fd1 - an) <= 1e-4 * scale + 1e-9, (kind, v, idx, fd1, an)
            checked += 1
    assert checked >= 16


def test_backward_through_the_clamps(ora):
    # sigma = max(0, trilinear) and c = max(0, SH + 0.5): a voxel whose corners are all negative has zero density
    # gradient, and a colour channel clamped at 0 has zero SH gradient -- both by finite differences (the loss
    # does not move) and in the reverse pass; the unclamped channels of the same voxel still match.
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(24, 24, 45.0, 1.4, 75.0, 30.0, target=(0.5, 0.3, 0.5))
    r0 = ora.render(sc, [cam])
    vis = np.where(r0["w_arg"] >= 0)[0]
    rng = np.random.default_rng(3)
    dark, dim = (int(v) for v in rng.choice(vis, size=2, replace=False))
    sc["density"][dark] = -np.abs(sc["density"][dark]) - np.float32(0.5)
    sc["sh"][dim, 0::3] = 0.0
    sc["sh"][dim, 0] = np.float32(-4.0)                   # red: 0.5 - 4 Y_0 < 0 in every direction
    P = 24 * 24
    gC = rng.normal(size=(P, 3))
    gT = rng.normal(size=P)
    r = ora.render(sc, [cam])
    assert r["w_arg"][dim] >= 0                            # the dimmed voxel is still seen
    bw = ora.render_backward(sc, [cam], gC, None, gT)

    def loss(kind, v, idx, e):
        sc2 = {k: np.array(a, copy=True) for k, a in sc.items()}
        sc2[kind][v, idx] = np.float32(sc2[kind][v, idx] + e)
        rr = ora.render(sc2, [cam])
        return float((rr["rgb"] * gC).sum() + (rr["T"] * gT).sum()), float(sc2[kind][v, idx]) - float(sc[kind][v, idx])

    for i in range(8):
        assert bw["d_density"][dark, i] == 0.0
        assert loss("density", dark, i, 1e-2)[0] == loss("density", dark, i, -1e-2)[0]
    for j in range(16):
        assert bw["d_sh"][dim, 3 * j] == 0.0
    assert loss("sh", dim, 0, 1e-2)[0] == loss("sh", dim, 0, -1e-2)[0]
    lp, hp = loss("sh", dim, 1, 1e-3)
    lm, hm = loss("sh", dim, 1, -1e-3)
    fd = (lp - lm) / (hp - hm)
    assert abs(fd) > 1e-6 and abs(fd - bw["d_sh"][dim, 1]) <= 1e-4 * abs(fd)


def test_fp32_sensitivity_bound_covers_ulp_perturbations(ora):
    # The per-pixel bound must cover what one-ulp FP32 perturbations of the voxel
    # positions and of the camera actually do to the FP64 image.
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(40, 40, 60.0, 1.6, 200.0, 40.0, target=(0.5, 0.4, 0.5))
    r0 = ora.render(sc, [cam])
    rng = np.random.default_rng(4)
    for trial in range(3):
        sc2 = {k: np.array(v, copy=True) for k, v in sc.items()}
        g = sc2["geom"]
        sgn = rng.choice([-1.0, 1.0], size=g[:, :3].shape).astype(np.float32)
        g[:, :3] = np.nextafter(g[:, :3], g[:, :3] + sgn * np.float32(1e30))
        cam2 = dict(cam)
        w = np.asarray(cam["w2c"], np.float32)
        w = np.nextafter(w, w + rng.choice([-1.0, 1.0], size=w.shape).astype(np.float32) * np.float32(1e30))
        cam2["w2c"] = w.tolist()
        r1 = ora.render(sc2, [cam2])
        ok = (r0["near_stop"] == 0) & (r1["near_stop"] == 0)
        d_rgb = np.abs(r1["rgb"] - r0["rgb"]).max(axis=1)
        d_T = np.abs(r1["T"] - r0["T"])
        assert np.all(d_rgb[ok] <= r0["bound_rgb"][ok] + 1e-12), (trial, (d_rgb - r0["bound_rgb"])[ok].max())
        assert np.all(d_T[ok] <= r0["bound_T"][ok] + 1e-12)
        assert d_rgb[ok].max() > 0            # the perturbation did change the image


def test_near_plane_clips_the_chord(ora):
    # A voxel crossing the near plane contributes only its part beyond it:
    # on the axis ray the chord runs from z_near to the far face.
    cam = axis_camera()
    cam["z_near"] = 0.5
    sc = synth.constant_voxel_scene([[0.0, 0.0, 0.6]], 0.3, [2.0], [(1, 1, 1)])
    r = ora.render(sc, [cam], sh_degree=0)
    l = 0.9 - 0.5
    assert abs(r["T"][4] - math.exp(-2.0 * l)) < 1e-7   # z_near and h are FP32 values
    assert r["n_hit"][4] == 1


def test_near_plane_straddler_tiles_cover_hits(ora):
    # The clipped FP32 rectangle of voxels crossing the near plane still covers every
    # pixel whose ray meets the voxel beyond the plane (dense sampling of the inside predicate).
    rng = np.random.default_rng(12)
    n = 30
    centers = np.c_[rng.uniform(-0.4, 0.4, n), rng.uniform(-0.3, 0.3, n), rng.uniform(0.1, 0.5, n)]
    half = rng.uniform(0.05, 0.25, n)
    sc = synth.constant_voxel_scene(centers, half, np.ones(n), np.ones((n, 3)) * 0.5)
    cam = axis_camera(48, 40, 30.0)
    cam["z_near"] = 0.3
    pr = ora.pairs(sc, [cam], ts=8)
    tiles_x = (48 + 7) // 8
    cover = {}
    for k, v in zip(pr["keys"], pr["vals"]):
        cover.setdefault(int(v), set()).add(int(k >> np.uint64(32)))
    g = sc["geom"].astype(np.float64)
    checked, straddlers = 0, set()
    for i in range(n):
        if g[i, 2] - g[i, 3] < 0.3 < g[i, 2] + g[i, 3]:
            straddlers.add(i)
    for y in range(40):
        for x in range(48):
            o, d = ray_of(cam, x, y)
            t = np.linspace(0.3 / d[2], 3.0, 2701)            # beyond the near plane only
            pts = o[None] + t[:, None] * d[None]
            inside = np.all(np.abs(pts[:, None, :] - g[None, :, :3]) < g[None, :, 3:4], axis=2).any(axis=0)
            tile = (y // 8) * tiles_x + x // 8
            for i in np.where(inside)[0]:
                assert tile in cover.get(int(i), set()), (i, x, y)
                checked += int(i) in straddlers
    assert checked > 50
    # and a straddler no longer covers the whole image
    assert any(len(cover.get(i, ())) < ((48 + 7) // 8) * ((40 + 7) // 8) for i in straddlers)


@pytest.mark.parametrize("rotated", [False, True])
def test_straddler_tiles_are_tight(ora, rotated):
    # The FP32 tile rectangle of each voxel is that of the exact footprint of its part beyond the near plane,
    # widened by the 1-pixel margin: the footprint's bounding box comes from the vertices of the clipped box
    # in camera space (scipy's half-space intersection; a ratio of linear functions peaks at a vertex), and
    # the rectangle's edges must sit on the tiles of that box +- 1 pixel, within 5e-3 pixel of rounding.
    # The rotated camera sees the boxes' edges obliquely, so edges of every direction cross the near plane.
    from scipy.spatial import HalfspaceIntersection
    rng = np.random.default_rng(21)
    n, ts, W, H, z_near = 60, 8, 48, 40, 0.3
    if rotated:
        cam = synth.look_at_camera([0.35, -0.25, -0.6], [0.05, 0.1, 0.5], W, H, 77.0, z_near=z_near)
    else:
        cam = axis_camera(W, H, 30.0)
        cam["z_near"] = z_near
    M = np.asarray(cam["w2c"], np.float64).reshape(3, 4)
    R, t = M[:, :3], M[:, 3]
    cc = np.c_[rng.uniform(-0.5, 0.5, n), rng.uniform(-0.4, 0.4, n), rng.uniform(0.1, 1.2, n)]
    centers = (cc - t) @ R                               # camera-space centres mapped to the world
    half = rng.uniform(0.05, 0.3, n)
    sc = synth.constant_voxel_scene(centers, half, np.ones(n), np.ones((n, 3)) * 0.5)
    pr = ora.pairs(sc, [cam], ts=ts)
    tiles_x, tiles_y = (W + ts - 1) // ts, (H + ts - 1) // ts
    rect = {}
    for k, v in zip(pr["keys"], pr["vals"]):
        tile = int(k >> np.uint64(32))
        tx, ty = tile % tiles_x, tile // tiles_x
        a = rect.setdefault(int(v), [tx, ty, tx, ty])
        a[:] = [min(a[0], tx), min(a[1], ty), max(a[2], tx), max(a[3], ty)]
    M = np.asarray(np.float32(cam["w2c"]), np.float64).reshape(3, 4)  # the FP32 camera both sides use
    R, t = M[:, :3], M[:, 3]
    g = sc["geom"].astype(np.float64)
    zn = float(np.float32(z_near))
    eps = 5e-3
    lo = lambda a, e, m: min(max(math.floor((a - 1 + e) / ts), 0), m)
    hi = lambda a, e, m: min(max(math.ceil((a + 1 + e) / ts), 0), m)
    checked = straddling = 0
    for i in range(n):
        c, h = g[i, :3], g[i, 3]
        corners = np.array([[c[0] + sx * h, c[1] + sy * h, c[2] + sz * h]
                            for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]) @ R.T + t
        zc = corners[:, 2]
        if zc.max() < zn + 1e-3:
            if zc.max() < zn - 1e-3:
                assert i not in rect                 # wholly in front of the near plane: culled
            continue
        # world box a.x <= b as camera-space rows (R a, -(R a).t - b), plus z_cam >= z_near
        rows = []
        for ax in range(3):
            for sgn in (-1.0, 1.0):
                a = np.zeros(3)
                a[ax] = sgn
                b = sgn * c[ax] + h
                ra = R @ a
                rows.append(np.r_[ra, -ra @ t - b])
        rows.append([0.0, 0.0, -1.0, zn])
        far = corners[int(np.argmax(zc))]
        inner = 0.97 * far + 0.03 * (np.asarray(c) @ R.T + t)
        vx = HalfspaceIntersection(np.asarray(rows), inner).intersections
        u = cam["fx"] * vx[:, 0] / vx[:, 2] + cam["cx"]
        v = cam["fy"] * vx[:, 1] / vx[:, 2] + cam["cy"]
        want = [(lo(u.min(), -eps, tiles_x), lo(u.min(), eps, tiles_x)),
                (lo(v.min(), -eps, tiles_y), lo(v.min(), eps, tiles_y)),
                (hi(u.max(), -eps, tiles_x), hi(u.max(), eps, tiles_x)),
                (hi(v.max(), -eps, tiles_y), hi(v.max(), eps, tiles_y))]
        if want[0][1] >= want[2][0] or want[1][1] >= want[3][0]:
            continue                                  # off screen or empty: no pairs expected either way
        got = rect[i][:2] + [rect[i][2] + 1, rect[i][3] + 1]
        for e, (a, b) in zip(got, want):
            assert a <= e <= b, (i, got, want)
        checked += 1
        straddling += zc.min() < zn
    assert checked > 30 and straddling > 5


def _two_views():
    sc = synth.scene_tiny()
    a = synth.orbit_camera(40, 28, 60.0, 1.6, 30.0, 25.0, target=(0.5, 0.4, 0.5))
    b = synth.orbit_camera(24, 36, 50.0, 1.8, 140.0, 10.0, target=(0.5, 0.4, 0.5))
    return sc, a, b


def test_views_render_independently(ora):
    # Views are independent: rendering two at once gives each view's image in view-major order, and
    # w_max accumulates over both -- the larger of the two, at the global id (offset + local id) of its pixel.
    sc, a, b = _two_views()
    both = ora.render(sc, [a, b])
    ra, rb = ora.render(sc, [a]), ora.render(sc, [b])
    na = 40 * 28
    for k in ("rgb", "depth", "T", "n_hit"):
        np.testing.assert_array_equal(both[k][:na], ra[k])
        np.testing.assert_array_equal(both[k][na:], rb[k])
    wa, wb = ra["w_max"], rb["w_max"]
    ga = ra["w_arg"]
    gb = np.where(rb["w_arg"] >= 0, rb["w_arg"] + na, -1)
    take_b = (wb > wa) | ((ga < 0) & (gb >= 0))
    np.testing.assert_array_equal(both["w_max"], np.where(take_b, wb, wa))
    np.testing.assert_array_equal(both["w_arg"], np.where(take_b, gb, ga))
    assert take_b.sum() > 10 and (~take_b & (ga >= 0)).sum() > 10       # both views contribute maxima


def test_views_backward_add_up(ora):
    # The gradient of a loss over two views is the sum of the two single-view gradients.
    sc, a, b = _two_views()
    na, nb = 40 * 28, 24 * 36
    rng = np.random.default_rng(11)
    gC, gT = rng.normal(size=(na + nb, 3)), rng.normal(size=na + nb)
    both = ora.render_backward(sc, [a, b], gC, None, gT)
    sa = ora.render_backward(sc, [a], gC[:na], None, gT[:na])
    sb = ora.render_backward(sc, [b], gC[na:], None, gT[na:])
    for k in ("d_density", "d_sh"):
        ref = sa[k] + sb[k]
        np.testing.assert_allclose(both[k], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert np.abs(sa[k]).max() > 0 and np.abs(sb[k]).max() > 0


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_sh_colour_uses_every_coefficient_of_the_degree(ora, degree):
    # c = max(0, 0.5 + sum_{j < (degree+1)^2} sh_j Y_j(dir)), dir from the camera centre to the voxel centre:
    # a voxel whose only nonzero coefficient is the last one of its degree shows 0.5 + sh Y_last(dir), and
    # coefficients beyond the degree are ignored.  Y comes from the basis pinned by orthonormality.
    cam = synth.look_at_camera([2.5, -0.4, -1.5], [0.15, 0.1, 0.05], 9, 9, 40.0)
    center = np.array([0.15, 0.1, 0.05])
    sc = synth.constant_voxel_scene([center], 0.6, [50.0], [(0.5, 0.5, 0.5)])   # opaque: rgb ~ colour
    last = (degree + 1) ** 2 - 1
    sc["sh"][0, :] = 0.0
    sc["sh"][0, 3 * last:3 * last + 3] = np.float32([0.9, -0.7, 0.4])
    if last + 1 < 16:
        sc["sh"][0, 3 * (last + 1):] = np.float32(5.0)                   # beyond the degree: unused
    r = ora.render(sc, [cam], sh_degree=degree)
    o, _ = ray_of(cam, 4, 4)
    c32 = center.astype(np.float32).astype(np.float64)
    direction = (c32 - o) / np.linalg.norm(c32 - o)
    Y = ora.sh_basis(direction)[last]
    col = np.maximum(0.0, 0.5 + np.float32([0.9, -0.7, 0.4]).astype(np.float64) * Y)
    p = 4 * 9 + 4
    alpha = 1.0 - r["T"][p]
    assert alpha > 0.999
    np.testing.assert_allclose(r["rgb"][p], alpha * col, rtol=0, atol=1e-7)
    assert abs(Y) > 0.05                                  # the test direction does exercise the coefficient


def test_near_plane_clips_oblique_chords(ora):
    # Off the axis the chord starts where the ray's camera depth reaches z_near, at t = z_near / d_z.
    cam = axis_camera(11, 9, 4.0)
    cam["z_near"] = 0.5
    center, h, sigma = np.array([0.1, -0.05, 0.62]), 0.3, 2.0
    sc = synth.constant_voxel_scene([center], h, [sigma], [(1, 1, 1)])
    r = ora.render(sc, [cam], sh_degree=0)
    c32, h32 = center.astype(np.float32).astype(np.float64), float(np.float32(h))
    zn = float(np.float32(0.5))
    checked = 0
    for y in range(9):
        for x in range(11):
            o, d = ray_of(cam, x, y)
            ch = chord_by_bisection(o, d, c32, h32, t_max=3.0, steps=30001)
            p = y * 11 + x
            if ch is None:
                continue
            t0 = max(ch[0], zn / d[2])
            l = max(0.0, ch[1] - t0)
            assert abs(r["T"][p] - math.exp(-float(np.float32(sigma)) * l)) < 1e-6, (x, y)
            checked += abs(d[2] - 1.0) > 1e-3 and l > 0
    assert checked > 15


def test_samples_are_ordered_by_centre_depth(ora):
    # Eq. 2 composites front to back in the order of the voxels' camera-space centre depth (ties by id),
    # whatever order the rays enter them: every traced pixel's samples come sorted by that depth.
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(32, 32, 60.0, 1.6, 200.0, 35.0, target=(0.5, 0.4, 0.5))
    M = np.asarray(cam["w2c"], np.float64).reshape(3, 4)
    zc = sc["geom"][:, :3].astype(np.float64) @ M[2, :3] + M[2, 3]
    traced = 0
    for (x, y) in [(16, 16), (10, 20), (20, 8), (5, 5), (28, 30), (12, 3), (3, 25)]:
        tr = ora.trace_pixel(sc, cam, x, y, t_stop=1e-12)
        ids = np.asarray(tr["ids"], np.int64)
        if len(ids) < 2:
            continue
        np.testing.assert_array_equal(ids, ids[np.lexsort((ids, zc[ids]))])
        traced += len(ids) >= 4
    assert traced >= 3
