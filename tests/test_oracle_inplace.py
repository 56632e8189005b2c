"""Pins of the in-place topology change (oracle/inplace.py): hand-traced
placements in the growing and the shrinking case, and on random scenes the
properties the placement promises -- untouched rows keep their bytes and
index, a split parent's row holds its first child, pruned rows hold new
children, the output is dense and holds exactly the rows of the
out-of-place subdivision."""
import numpy as np
import pytest

from oracle import inplace as IP
from paper_2511_02510_gb300 import synth


def test_placement_when_the_array_grows():
    # 5 rows, row 1 pruned, row 3 split: child 0 stays at 3, child 1 fills the hole at 1, children 2..7
    # are appended at 5..10.  Output rows: survivors 0, 2, 4, then the 8 children of 3.
    dest, n_new = IP.placement(5, [1], [3])
    assert n_new == 11
    assert list(dest) == [0, 2, 4, 3, 1, 5, 6, 7, 8, 9, 10]


def test_placement_when_the_array_shrinks():
    # 12 rows, rows 0..8 pruned, row 11 split: n' = 12 - 9 + 7 = 10.  Child 0 at 11, children 1..7 at 0..6;
    # rows 7 and 8 stay empty below n', so the occupied rows 10 (a survivor) and 11 (child 0) move there.
    dest, n_new = IP.placement(12, list(range(9)), [11])
    assert n_new == 10
    assert list(dest) == [9, 7, 8, 0, 1, 2, 3, 4, 5, 6]
    # no split at all: plain compaction from the tail
    dest, n_new = IP.placement(6, [1, 3], [])
    assert n_new == 4 and list(dest) == [0, 2, 1, 3]      # survivors 0, 2, 4, 5 -> rows 0, 2, 1, 3


def test_placement_degenerate_cases():
    dest, n_new = IP.placement(0, [], [])
    assert n_new == 0 and len(dest) == 0
    dest, n_new = IP.placement(4, [], [])
    assert n_new == 4 and list(dest) == [0, 1, 2, 3]
    dest, n_new = IP.placement(3, [0, 1, 2], [])
    assert n_new == 0 and len(dest) == 0
    dest, n_new = IP.placement(2, [], [0, 1])            # everything split: 16 rows
    assert n_new == 16 and sorted(dest) == list(range(16)) and list(dest[:1]) == [0] and dest[8] == 1


def _scene(n, seed):
    rng = np.random.default_rng(seed)
    sc = synth.constant_voxel_scene(rng.uniform(-1, 1, (n, 3)), rng.uniform(0.05, 0.2, n), np.ones(n),
                                    np.ones((n, 3)) * 0.5)
    sc["density"] = rng.normal(2, 1, (n, 8)).astype(np.float32)
    sc["sh"] = rng.normal(0, 1, (n, 48)).astype(np.float32)
    sc["level"] = rng.integers(3, 12, n).astype(np.uint8)
    return sc, rng


@pytest.mark.parametrize("seed,p_prune,top_ppm", [(0, 0.02, 50000), (1, 0.3, 20000), (2, 0.0, 100000),
                                                  (3, 0.5, 0)])
def test_inplace_properties(ora, seed, p_prune, top_ppm):
    n = 500
    sc, rng = _scene(n, seed)
    pm = (rng.uniform(size=n) < p_prune).astype(np.uint8)
    aux = [rng.normal(size=(n, 8)).astype(np.float32)]
    args = (np.zeros(n, np.float32), rng.uniform(1, 10, n).astype(np.float32), rng.uniform(size=n).astype(np.float32),
            np.ones(n, np.uint8))
    ref = ora.subdivide(sc, *args, prune_mask=pm, top_ppm=top_ppm, aux=[(a, 0.0) for a in aux])
    out = IP.subdivide_inplace(sc, *args, prune_mask=pm, top_ppm=top_ppm, aux=[(a, 0.0) for a in aux])
    n_new, k, h = ref["n_new"], ref["k"], int(pm.sum())
    assert out["n_new"] == n_new == n - h + 7 * k
    # dense, and the same rows as the out-of-place form
    assert sorted(out["dest"]) == list(range(n_new))
    key = lambda g, d: sorted(map(bytes, np.concatenate([g.view(np.uint8), d.view(np.uint8)], axis=1)))
    assert key(out["geom"], out["density"]) == key(ref["geom"], ref["density"])
    parents = np.flatnonzero(ref["selected"])
    gone = pm.astype(bool)
    if 7 * k >= h:
        # growing: untouched rows keep their index and bytes, the parent's row holds child 0 (all minus
        # offsets, half the size), and the pruned rows hold children (one level finer)
        keep = np.flatnonzero(~gone & ~ref["selected"].astype(bool))
        for name in ("geom", "level", "density", "sh"):
            np.testing.assert_array_equal(out[name][keep], np.asarray(sc[name])[keep])
        np.testing.assert_array_equal(out["aux"][0][keep], aux[0][keep])
        g = sc["geom"][parents]
        np.testing.assert_array_equal(out["geom"][parents, :3], g[:, :3] - g[:, 3:4] * np.float32(0.5))
        np.testing.assert_array_equal(out["geom"][parents, 3], g[:, 3] * np.float32(0.5))
        holes = np.flatnonzero(gone)
        np.testing.assert_array_equal(out["level"][holes], sc["level"][np.repeat(parents, 7)[:h]] + 1)
        assert np.all(out["aux"][0][np.r_[parents, holes]] == 0.0)     # children start from zero moments
    else:
        # shrinking: every row below n' is occupied, and at most h - 7k rows moved
        moved = [i for i, d in zip(np.flatnonzero(~gone & ~ref["selected"].astype(bool)), out["dest"]) if i != d]
        assert len(moved) <= h - 7 * k
