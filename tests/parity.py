"""Parity checks of FP32 results against the FP64 oracle (numpy only).

check_wmax: w_max and its argmax (Eq. 5) for every voxel.  The argmax must be
the oracle's pixel unless the oracle's own near-max set says FP32 rounding can
reorder the top weights: then the picked pixel must belong to that set (its
oracle weight within FP32 error of the maximum), and the picked weight must
match that pixel's oracle weight.  Hit/miss flips must be explained by the
oracle: a missed voxel may have no certain hit, a voxel the oracle misses may
be picked only on a near miss of the set.  Pixels whose stop decision FP32
rounding can change (near_stop) may add or drop samples below t_stop.

check_grads: every gradient element within 1e-4 of its oracle value, relative,
plus the oracle's FP32 floor of that element; the relative L2 error of the
whole array within 1e-5; elements that needed the floor are counted.
"""
import numpy as np

W_TOL = 1e-5           # absolute tolerance of a weight, as for images
GRAD_REL = 1e-4        # per-element relative tolerance of gradients
GRAD_L2 = 1e-5         # relative L2 error of a whole gradient array


def set_lookup(ws, v, pix):
    """Index of entry (v, pix) in the oracle's sorted near-max set, or -1."""
    key = ws["set_v"] * (1 << 32) + ws["set_pix"]
    q = np.asarray(v, np.int64) * (1 << 32) + np.asarray(pix, np.int64)
    if len(key) == 0:
        return np.full(q.shape, -1, np.int64)
    i = np.minimum(np.searchsorted(key, q), len(key) - 1)
    return np.where(key[i] == q, i, -1)


def check_wmax(w_gpu, a_gpu, ws, near_stop, t_stop=1e-4):
    """Assert the w_max rules above for every voxel; returns a report dict.

    w_gpu / a_gpu: the FP32 w_max and argmax pixel (-1: never hit) under test;
    ws: oracle.wmax_sets of the same scene and views; near_stop: oracle.render's flag per pixel."""
    w = np.asarray(w_gpu, np.float64)
    a = np.asarray(a_gpu, np.int64)
    w1, a1, e1 = ws["w1"], ws["a1"], ws["e1"]
    n = len(w1)
    stop = np.asarray(near_stop) != 0
    at_stop = lambda p: (p >= 0) & stop[np.maximum(p, 0)]
    same = a == a1
    bad_value = same & (a1 >= 0) & ~(np.abs(w - w1) <= W_TOL + e1)
    assert not bad_value.any(), ("w_max value", np.where(bad_value)[0][:10])
    # a different pick: a member of the near-max set with a matching weight, or a sample beyond an
    # ambiguous stop (its weight below t_stop, and the oracle's maximum too)
    diff = ~same & (a >= 0)
    idx = set_lookup(ws, np.where(diff)[0], a[diff])
    vd = np.where(diff)[0]
    member = idx >= 0
    ok_member = member & (np.abs(w[vd] - np.where(member, ws["set_w"][idx], 0.0)) <=
                          W_TOL + np.where(member, ws["set_e"][idx], 0.0))
    beyond_stop = (~member & (at_stop(a[vd]) | at_stop(a1[vd])) & (w[vd] <= 1.01 * t_stop) &
                   (w1[vd] - e1[vd] <= 1.01 * t_stop))
    bad_pick = ~(ok_member | beyond_stop)
    assert not bad_pick.any(), ("w_max argmax outside the oracle's near-max set", vd[bad_pick][:10],
                                a[vd[bad_pick][:10]], a1[vd[bad_pick][:10]])
    # missed by the FP32 pass, hit by the oracle: no certain hit, and a maximum within its rounding
    # (or beyond an ambiguous stop)
    miss = (a < 0) & (a1 >= 0)
    ok_miss = (ws["n_certain"] == 0) & ((w1 <= 2.0 * e1 + W_TOL) | (at_stop(a1) & (w1 <= 1.01 * t_stop)))
    assert not (miss & ~ok_miss).any(), ("voxel hit by the oracle missed", np.where(miss & ~ok_miss)[0][:10])
    gap = np.where(ws["w2"] >= 0, w1 - ws["w2"], np.inf)
    return {"voxels": n, "hit_oracle": int((a1 >= 0).sum()), "hit_gpu": int((a >= 0).sum()),
            "argmax_equal": int((same & (a1 >= 0)).sum()), "argmax_in_near_max_set": int(ok_member.sum()),
            "argmax_beyond_ambiguous_stop": int((beyond_stop & ~ok_member).sum()),
            "gpu_miss_oracle_hit": int(miss.sum()), "gpu_hit_oracle_miss": int(((a >= 0) & (a1 < 0)).sum()),
            "ambiguous_top2": int(((a1 >= 0) & (gap <= e1 + ws["e2"])).sum()),
            "max_w_err": float(np.abs(w - w1)[same & (a1 >= 0)].max(initial=0.0))}


def check_grads(name, g, ref, e_full, e_arith, rel=GRAD_REL, l2=GRAD_L2):
    """Assert |g - ref| <= rel |ref| + e_full for every element and the relative L2 error <= l2;
    returns a report (how many elements needed the arithmetic floor, the geometric one, and the
    max-normalised error)."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(g - ref)
    tol = rel * np.abs(ref) + e_full
    bad = err > tol
    assert not bad.any(), (name, int(bad.sum()), np.argwhere(bad)[:5].tolist(), float((err - tol).max()))
    nr = float(np.linalg.norm(ref))
    l2_err = float(np.linalg.norm(g - ref)) / max(nr, 1e-300)
    assert l2_err <= l2, (name, "relative L2 error", l2_err)
    nz = np.abs(ref) > 0
    return {"elements": int(ref.size), "nonzero": int(nz.sum()),
            "within_rel_alone": int((err <= rel * np.abs(ref)).sum()),
            "needed_arith_floor": int(((err > rel * np.abs(ref)) & (err <= rel * np.abs(ref) + e_arith)).sum()),
            "needed_geometric_floor": int((err > rel * np.abs(ref) + e_arith).sum()),
            "max_floor_over_ref": float((e_full[nz] / np.abs(ref[nz])).max(initial=0.0)),
            "rel_l2": l2_err, "max_normalised": float(err.max() / max(np.abs(ref).max(), 1e-300))}
