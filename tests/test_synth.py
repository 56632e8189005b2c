"""The seeded synthetic inputs have the shapes and structure the benchmark and
the parity tests are quoted on (the recipe of the design notes): voxel counts,
level ranges and half-sizes of the scenes, value ranges of densities and SH,
the view-size ladder of the batched views, camera geometry, and determinism
by seed.  CPU only."""
import math

import numpy as np

from paper_2511_02510_gb300 import synth


def check_octree(sc, root_edge, root_min):
    g, lvl = sc["geom"], sc["level"]
    # every voxel is a cell of its level: half-size = root / 2^(level + 1), centre on that level's grid
    half = root_edge / 2.0 ** (lvl.astype(np.float64) + 1)
    np.testing.assert_array_equal(g[:, 3], half.astype(np.float32))
    cell = (g[:, :3].astype(np.float64) - np.asarray(root_min) - half[:, None]) / (2 * half[:, None])
    np.testing.assert_allclose(cell, np.rint(cell), atol=1e-3)
    assert sc["density"].shape == (g.shape[0], 8) and sc["sh"].shape == (g.shape[0], 48)
    assert sc["density"].dtype == np.float32 and sc["sh"].dtype == np.float32


def test_tiny_scene_recipe():
    sc = synth.scene_tiny()
    assert sc["geom"].shape[0] == 4043
    assert set(np.unique(sc["level"])) == {4, 5, 6}
    check_octree(sc, 1.0, (0.0, 0.0, 0.0))
    sh = sc["sh"].reshape(-1, 16, 3)
    assert sh[:, 0].min() >= 0.0 and sh[:, 0].max() < 1.0           # SH DC ~ U(0, 1)
    assert abs(sh[:, 1:].std() - 0.05) < 0.005                        # higher bands ~ N(0, 0.05)
    d = sc["density"]
    assert d.max() < 10.0 + 6 * 0.1 and d.min() > -6 * 0.1            # peak 10 sigmoid + N(0, 0.1)


def test_scenes_are_deterministic_by_seed():
    a, b, c = synth.scene_tiny(0), synth.scene_tiny(0), synth.scene_tiny(1)
    for k in ("geom", "level", "density", "sh"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["geom"].shape != c["geom"].shape or not np.array_equal(a["geom"], c["geom"])
    np.testing.assert_array_equal(synth.random_image(17, 9, seed=3), synth.random_image(17, 9, seed=3))


def test_bench_scene_recipe():
    sc = synth.scene_360()
    n = sc["geom"].shape[0]
    assert n == 1976376
    counts = np.bincount(sc["level"], minlength=13)
    assert counts[:6].sum() == 0 and counts[6:].sum() == n            # levels 6-12
    check_octree(sc, 32.0, (-16.0, -16.0, -16.0))
    r = np.linalg.norm(sc["geom"][:, :3].astype(np.float64), axis=1)
    assert r.max() < 16.0 * math.sqrt(3)
    assert np.all(r[sc["level"] >= 9] < 3.0)                          # the fine levels are the foreground
    assert (r > 11.0).sum() > 10000                                   # background shell beyond r ~ 12


def test_batched_view_ladder():
    cams = synth.uneven_views()
    sizes = [(c["width"], c["height"]) for c in cams]
    assert len(sizes) == 16 and sizes[0] == (640, 480) and sizes[-1] == (1600, 1060)
    assert all(w % 2 == 0 and h % 2 == 0 for w, h in sizes)
    assert all(a[0] < b[0] and a[1] < b[1] for a, b in zip(sizes, sizes[1:]))


def test_orbit_camera_geometry():
    cam = synth.orbit_camera(1237, 822, 60.0, 3.0, 37.0, 15.0)
    M = np.asarray(cam["w2c"], np.float64).reshape(3, 4)
    R, t = M[:, :3], M[:, 3]
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)        # a rotation
    eye = -R.T @ t
    assert abs(np.linalg.norm(eye) - 3.0) < 1e-5                      # radius 3 about the origin
    assert abs(math.degrees(math.asin(abs(eye[1]) / 3.0)) - 15.0) < 1e-3   # elevation 15 degrees
    np.testing.assert_allclose(R[2] @ (-eye) / 3.0, 1.0, atol=1e-6)   # looks at the target
    assert abs(cam["fx"] - 1237 / 2 / math.tan(math.radians(30))) < 1e-2   # fov_x 60 degrees
    assert cam["cx"] == 1237 / 2 and cam["cy"] == 822 / 2
