"""Pins for the training-step oracle (oracle/train_aux.py): the transmittance
concentration and density TV terms of Eq. 17 and the Adam update.

Expected values are closed forms (constant and linear fields, T in {0, 1/2,
1}, the first Adam step), central finite differences of the losses, and a
hand-traced two-step Adam sequence.
"""
import math

import numpy as np

from oracle import train_aux as TA


def test_edges_are_the_cube_edges():
    assert len(TA.EDGES) == 12 and len(set(TA.EDGES)) == 12
    for i, j in TA.EDGES:
        assert bin(i ^ j).count("1") == 1 and i < j
    deg = np.bincount(np.array(TA.EDGES).ravel(), minlength=8)
    assert np.all(deg == 3)


def test_tc_closed_forms():
    loss, g = TA.transmittance_concentration([0.0, 1.0, 0.0, 1.0], 2.0)
    assert loss == 0.0
    np.testing.assert_allclose(g, [0.5, -0.5, 0.5, -0.5])        # 2 * (1 - 2T) / 4
    loss, g = TA.transmittance_concentration([0.5, 0.5], 1.0)
    assert loss == 0.25 and np.all(g == 0.0)


def test_tc_gradient_finite_differences():
    rng = np.random.default_rng(0)
    T = rng.uniform(0, 1, 50)
    _, g = TA.transmittance_concentration(T, 0.7)
    h = 1e-6
    for i in range(0, 50, 7):
        e = np.zeros(50)
        e[i] = h
        fd = (TA.transmittance_concentration(T + e, 0.7)[0] - TA.transmittance_concentration(T - e, 0.7)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7


def test_tv_constant_and_linear_fields():
    d = np.full((5, 8), 3.25)
    loss, g = TA.density_tv(d, 1.0)
    assert loss == 0.0 and np.all(g == 0.0)
    # corners of a linear field a.x on a cube of edge e: every edge along axis k differs by e a_k,
    # four edges per axis -> L_v = 4 e^2 |a|^2
    a = np.array([0.3, -1.2, 2.0])
    e = 0.5
    corners = np.array([[(c & 1) * e, ((c >> 1) & 1) * e, ((c >> 2) & 1) * e] for c in range(8)])
    d = (corners @ a)[None, :].repeat(3, 0)
    loss, _ = TA.density_tv(d, 2.0)
    assert math.isclose(loss, 2.0 * 4 * e * e * float(a @ a), rel_tol=1e-12)


def test_tv_gradient_finite_differences():
    rng = np.random.default_rng(1)
    d = rng.normal(size=(6, 8))
    _, g = TA.density_tv(d, 0.3)
    h = 1e-6
    for v in range(6):
        for c in range(8):
            e = np.zeros_like(d)
            e[v, c] = h
            fd = (TA.density_tv(d + e, 0.3)[0] - TA.density_tv(d - e, 0.3)[0]) / (2 * h)
            assert abs(fd - g[v, c]) < 1e-7


def test_adam_first_step_is_a_signed_step():
    # from m = v = 0 at t = 1: m^ = g and v^ = g^2, so the step is lr g / (|g| + eps)
    g = np.array([2.0, -0.5, 0.0, 1e-3])
    p, m, v = TA.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 0.01, 0.9, 0.999, 1e-8, 1)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_adam_two_step_trace():
    # g = 1 then g = 3, b1 = 0.5, b2 = 0.75, eps = 0, lr = 1:
    # t=1: m = .5, v = .25, m^ = 1, v^ = 1 -> p = -1
    # t=2: m = .25 + 1.5 = 1.75, v = .1875 + 2.25 = 2.4375, m^ = 1.75 / .75, v^ = 2.4375 / .4375
    p, m, v = TA.adam(np.zeros(1), np.ones(1), np.zeros(1), np.zeros(1), 1.0, 0.5, 0.75, 0.0, 1)
    assert p[0] == -1.0 and m[0] == 0.5 and v[0] == 0.25
    p, m, v = TA.adam(p, np.full(1, 3.0), m, v, 1.0, 0.5, 0.75, 0.0, 2)
    assert m[0] == 1.75 and v[0] == 2.4375
    assert math.isclose(p[0], -1.0 - (1.75 / 0.75) / math.sqrt(2.4375 / 0.4375), rel_tol=1e-14)


def test_adam_voxels_tv_enters_the_density_gradient():
    rng = np.random.default_rng(2)
    n = 10
    dens = rng.normal(size=(n, 8))
    sh = rng.normal(size=(n, 48))
    z8, z48 = np.zeros((n, 8)), np.zeros((n, 48))
    # zero photometric gradient: the density moves against the TV gradient only, SH stays
    out = TA.adam_voxels(dens, sh, z8, z48, z8, z8, z48, z48, 0.1, 0.1, 0.9, 0.999, 1e-8, 1, tv_weight=1.0)
    _, g_tv = TA.density_tv(dens, 1.0)
    np.testing.assert_allclose(out["density"], dens - 0.1 * g_tv / (np.abs(g_tv) + 1e-8), rtol=1e-12)
    np.testing.assert_array_equal(out["sh"], sh)
    # the update lowers the TV energy
    assert TA.density_tv(out["density"], 1.0)[0] < TA.density_tv(dens, 1.0)[0]
