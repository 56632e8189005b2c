"""Pins for the oracle's exact-segment-integration variant (the density-model
variant in which a sample's density is the mean of the trilinear field over
the chord rather than its value at the chord midpoint).

Expected values: equality with the midpoint reading where the field is
constant or linear along the chord (the mean then equals the midpoint value),
brute-force quadrature of the trilinear field along chords found by bisection
of the inside predicate, and central finite differences of the backward.
"""
import math

import numpy as np

from paper_2511_02510_gb300 import synth
from test_oracle_render import chord_by_bisection, ray_of


def trilinear(dens, center, h, p):
    """The trilinear interpolant of 8 corner values (corner c = x + 2y + 4z) at point p."""
    u = np.clip((p - (center - h)) / (2 * h), 0.0, 1.0)
    f = 0.0
    for c in range(8):
        w = (u[0] if c & 1 else 1 - u[0]) * (u[1] if c & 2 else 1 - u[1]) * (u[2] if c & 4 else 1 - u[2])
        f += w * dens[c]
    return f


def test_constant_and_linear_fields_equal_the_midpoint_reading(ora):
    # a constant field and a linear field have mean = midpoint value on every chord
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(40, 32, 50.0, 1.5, 40.0, 20.0, target=(0.5, 0.4, 0.5))
    const = {k: np.array(v, copy=True) for k, v in sc.items()}
    const["density"][:] = const["density"].mean(axis=1, keepdims=True)
    a = ora.render(const, [cam])
    b = ora.render(const, [cam], segment=True)
    np.testing.assert_allclose(b["rgb"], a["rgb"], atol=1e-12)
    np.testing.assert_allclose(b["T"], a["T"], atol=1e-12)
    lin = {k: np.array(v, copy=True) for k, v in sc.items()}
    g = lin["geom"].astype(np.float64)
    corners = np.array([[(c & 1) * 2 - 1, ((c >> 1) & 1) * 2 - 1, ((c >> 2) & 1) * 2 - 1] for c in range(8)], float)
    k = np.array([3.0, -2.0, 5.0])
    pts = g[:, None, :3] + corners[None] * g[:, None, 3:4]
    lin["density"] = (pts @ k + 4.0).astype(np.float32)
    a = ora.render(lin, [cam])
    b = ora.render(lin, [cam], segment=True)
    np.testing.assert_allclose(b["T"], a["T"], atol=1e-9)


def test_mean_density_by_quadrature(ora):
    # one voxel with arbitrary positive corners: the sample's optical depth is l times the mean of the
    # trilinear field over the chord, checked against a 20k-point midpoint-rule quadrature
    rng = np.random.default_rng(4)
    center = np.array([0.05, -0.1, 0.02])
    h = 0.45
    dens = rng.uniform(0.2, 3.0, 8)
    sc = synth.constant_voxel_scene([center], h, [0.0], [(1, 1, 1)])
    sc["density"][0] = dens.astype(np.float32)
    d32 = sc["density"][0].astype(np.float64)
    c32 = sc["geom"][0, :3].astype(np.float64)
    h32 = float(sc["geom"][0, 3])
    cam = synth.look_at_camera([0.6, 0.5, -3.2], center, 10, 10, 38.0)
    mid = ora.render(sc, [cam], sh_degree=0)
    seg = ora.render(sc, [cam], sh_degree=0, segment=True)
    checked = differs = 0
    for y in range(10):
        for x in range(10):
            o, d = ray_of(cam, x, y)
            ch = chord_by_bisection(o, d, c32, h32, t_max=7.0, steps=3001)
            if ch is None or ch[1] - ch[0] < 1e-3:
                continue
            t0, t1 = ch
            n = 20000
            ts = t0 + (np.arange(n) + 0.5) * (t1 - t0) / n
            tau = sum(trilinear(d32, c32, h32, o + t * d) for t in ts) * (t1 - t0) / n
            assert abs(-math.log(seg["T"][y * 10 + x]) - tau) < 1e-6 * max(1.0, tau)
            differs += abs(seg["T"][y * 10 + x] - mid["T"][y * 10 + x]) > 1e-6
            checked += 1
    assert checked > 15 and differs > 5     # the variant is not the midpoint reading on a curved field


def test_segment_backward_matches_central_differences(ora):
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(20, 20, 45.0, 1.4, 75.0, 30.0, target=(0.5, 0.3, 0.5))
    rng = np.random.default_rng(9)
    P = 20 * 20
    gC = rng.normal(size=(P, 3))
    gT = rng.normal(size=P)
    r = ora.render(sc, [cam], segment=True)
    bw = ora.render_backward(sc, [cam], gC, None, gT, segment=True)
    hit = np.where(r["w_arg"] >= 0)[0]
    checked = 0
    for v in rng.choice(hit, size=12, replace=False):
        idx = int(rng.integers(8))
        x0 = float(sc["density"][v, idx])
        eps = 1e-3 * max(1.0, abs(x0))
        vals = []
        for s_ in (+1, -1, +2, -2):
            sc2 = {k: np.array(a, copy=True) for k, a in sc.items()}
            sc2["density"][v, idx] = np.float32(x0 + s_ * eps)
            rr = ora.render(sc2, [cam], segment=True)
            vals.append((float(sc2["density"][v, idx]) - x0, float((rr["rgb"] * gC).sum() + (rr["T"] * gT).sum())))
        (hp, lp), (hm, lm), (hp2, lp2), (hm2, lm2) = vals
        fd1, fd2 = (lp - lm) / (hp - hm), (lp2 - lm2) / (hp2 - hm2)
        an = bw["d_density"][v, idx]
        scale = max(1e-6, abs(fd1), abs(an))
        if abs(fd1 - fd2) > 1e-3 * scale:
            continue
        assert abs(fd1 - an) <= 1e-4 * scale + 1e-9, (v, idx, fd1, an)
        checked += 1
    assert checked >= 8
