"""The parity checkers of tests/parity.py have teeth: the oracle's own FP64
results, rounded to FP32, pass them, and plausible mistakes planted in a copy
of those results (a wrong argmax, a tie broken the other way on distinct
weights, a dropped hit, a gradient off by 1e-3 on 1 % of elements) fail them.
CPU only; the oracle stands in for the GPU result."""
import numpy as np
import pytest

from paper_2511_02510_gb300 import synth
from parity import check_grads, check_wmax, set_lookup


@pytest.fixture(scope="module")
def case(ora):
    sc = synth.scene_tiny()
    cams = [synth.orbit_camera(48, 40, 60.0, 1.6, 30.0, 25.0, target=(0.5, 0.4, 0.5)),
            synth.orbit_camera(32, 32, 60.0, 1.6, 160.0, 30.0, target=(0.5, 0.4, 0.5))]
    r = ora.render(sc, cams)
    ws = ora.wmax_sets(sc, cams)
    rng = np.random.default_rng(4)
    P = r["rgb"].shape[0]
    gC = rng.normal(size=(P, 3))
    gC[r["near_stop"] != 0] = 0
    b = ora.render_backward(sc, cams, gC)
    e = ora.backward_bounds(sc, cams, gC)
    return sc, cams, r, ws, b, e


def test_oracle_rounded_to_fp32_passes(case):
    sc, cams, r, ws, b, e = case
    rep = check_wmax(ws["w1"].astype(np.float32), ws["a1"], ws, r["near_stop"])
    assert rep["argmax_equal"] == rep["hit_oracle"] > 100
    for k, ek, ak in (("d_density", "e_density", "a_density"), ("d_sh", "e_sh", "a_sh")):
        check_grads(k, b[k].astype(np.float32), b[k], e[ek], e[ak])


def test_wrong_argmax_is_caught(case):
    sc, cams, r, ws, b, e = case
    a = ws["a1"].copy()
    hit = np.where(a >= 0)[0]
    # a voxel whose set holds only its maximum, moved to a pixel outside the set
    single = [v for v in hit if np.sum(ws["set_v"] == v) == 1]
    v = single[0]
    other = a[v] + 1 if set_lookup(ws, v, a[v] + 1) < 0 else a[v] - 1
    a[v] = other
    with pytest.raises(AssertionError):
        check_wmax(ws["w1"].astype(np.float32), a, ws, r["near_stop"])


def test_argmax_within_the_set_passes_and_weight_must_match(case):
    sc, cams, r, ws, b, e = case
    multi = [v for v in np.unique(ws["set_v"]) if np.sum(ws["set_v"] == v) > 1 and ws["a1"][v] >= 0]
    if not multi:
        pytest.skip("no voxel with more than one near-max ray in this view")
    v = multi[0]
    i = np.where((ws["set_v"] == v) & (ws["set_pix"] != ws["a1"][v]))[0][0]
    a = ws["a1"].copy()
    w = ws["w1"].astype(np.float32).copy()
    a[v], w[v] = ws["set_pix"][i], np.float32(ws["set_w"][i])
    check_wmax(w, a, ws, r["near_stop"])
    w[v] = np.float32(ws["set_w"][i] + ws["set_e"][i] + 1e-3)
    with pytest.raises(AssertionError):
        check_wmax(w, a, ws, r["near_stop"])


def test_dropped_certain_hit_is_caught(case):
    sc, cams, r, ws, b, e = case
    v = int(np.where((ws["n_certain"] > 0) & (ws["w1"] > 1e-3))[0][0])
    a = ws["a1"].copy()
    w = ws["w1"].astype(np.float32).copy()
    a[v], w[v] = -1, 0.0
    with pytest.raises(AssertionError):
        check_wmax(w, a, ws, r["near_stop"])


def test_gradient_mistakes_are_caught(case):
    sc, cams, r, ws, b, e = case
    g = b["d_density"].copy()
    rng = np.random.default_rng(0)
    nz = np.argwhere(np.abs(g) > 1e-3 * np.abs(g).max())
    pick = nz[rng.choice(len(nz), size=max(1, len(nz) // 100), replace=False)]
    g[pick[:, 0], pick[:, 1]] *= 1.0 + 1e-3
    with pytest.raises(AssertionError):
        check_grads("d_density", g, b["d_density"], e["e_density"], e["a_density"])
    # one element wildly off, however small
    g = b["d_sh"].copy()
    small = np.argwhere((np.abs(g) > 0) & (np.abs(g) < 1e-3 * np.abs(g).max()))[0]
    g[small[0], small[1]] *= -1.0
    with pytest.raises(AssertionError):
        check_grads("d_sh", g, b["d_sh"], e["e_sh"], e["a_sh"])
