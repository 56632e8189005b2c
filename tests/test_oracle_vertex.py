"""Pins for the shared grid-vertex oracle (oracle/vertex.py): vertex counts
and sharing on regular blocks and across a level change (closed forms), a
linear field that vertices reproduce on every voxel, and finite differences
of the render through shared vertices against the scattered corner
gradients."""
import itertools

import numpy as np

from oracle import vertex as VX
from paper_2511_02510_gb300 import synth


def block(k, h, origin=(0.0, 0.0, 0.0)):
    o = np.asarray(origin, np.float64)
    centres = [o + (2 * np.array(ijk) + 1) * h for ijk in itertools.product(range(k), repeat=3)]
    return synth.constant_voxel_scene(centres, h, np.ones(len(centres)), np.ones((len(centres), 3)) * 0.5)


def test_regular_block_counts_and_sharing():
    k, h = 3, 0.125
    sc = block(k, h)
    vidx, nv = VX.vertex_index(sc["geom"], h)
    assert nv == (k + 1) ** 3
    uses = np.bincount(vidx.ravel(), minlength=nv)
    assert uses.max() == 8 and uses.min() == 1                  # interior vertices in 8 voxels, cube corners in 1
    assert (uses == 8).sum() == (k - 1) ** 3
    # face neighbours share exactly 4 vertices, edge neighbours 2, corner neighbours 1
    g = sc["geom"][:, :3]
    for a in range(len(g)):
        for b in range(a + 1, len(g)):
            d = np.round(np.abs(g[a] - g[b]) / (2 * h)).astype(int)
            if d.max() > 1:
                continue
            shared = len(set(vidx[a]) & set(vidx[b]))
            assert shared == {1: 4, 2: 2, 3: 1}[int(d.sum())]


def test_vertex_ids_are_ranks_in_z_y_x_order():
    # On a 2 x 2 x 2 block the vertices form a 3 x 3 x 3 grid; ids are the ranks of the points ordered by
    # z, then y, then x: grid point (i, j, k) has id i + 3 j + 9 k.  Corner c of a voxel is at bits
    # (c & 1, c & 2, c & 4) = (+x, +y, +z).
    h = 0.25
    sc = block(2, h)
    vidx, nv = VX.vertex_index(sc["geom"], h)
    assert nv == 27
    for v, (a, b, c) in enumerate(itertools.product(range(2), repeat=3)):
        # block() lays voxels out with the last index fastest: voxel v sits at grid cell (a, b, c) = (x, y, z)
        for corner in range(8):
            i, j, k = a + (corner & 1), b + ((corner >> 1) & 1), c + ((corner >> 2) & 1)
            assert vidx[v, corner] == i + 3 * j + 9 * k, (v, corner)


def test_level_change_shares_coincident_corners():
    # a coarse voxel (h = 1/4) beside a face of four fine voxels (h = 1/8): the coarse face's 4 corners
    # coincide with fine corners; the fine face's centre and edge midpoints are fine-only
    coarse = synth.constant_voxel_scene([[0.25, 0.25, 0.25]], 0.25, [1.0], [(1, 1, 1)])
    fine_c = [[0.5 + 0.125, 0.125 + 0.25 * j, 0.125 + 0.25 * i] for i in range(2) for j in range(2)]
    fine = synth.constant_voxel_scene(fine_c, 0.125, np.ones(4), np.ones((4, 3)))
    geom = np.concatenate([coarse["geom"], fine["geom"]])
    vidx, nv = VX.vertex_index(geom, 0.125)
    assert len(set(vidx[0]) & set(vidx[1:].ravel())) == 4
    # 8 coarse + the fine block's 3x3x2 = 18 vertices, 4 of them shared
    assert nv == 8 + 18 - 4


def test_linear_field_on_vertices():
    rng = np.random.default_rng(0)
    sc = synth.scene_tiny()
    unit = float(sc["geom"][:, 3].min())
    vidx, nv = VX.vertex_index(sc["geom"], unit)
    a, b = rng.normal(size=3), 1.5
    pts = np.zeros((nv, 3))
    q = VX.corner_points(sc["geom"], unit) * unit
    pts[vidx.ravel()] = q.reshape(-1, 3)
    vals = pts @ a + b
    corners = VX.gather(vidx, vals)
    np.testing.assert_allclose(corners, q @ a + b, atol=1e-12)
    # shared vertices really are shared: corners at one point agree across voxels
    assert nv < 8 * sc["geom"].shape[0]


def test_vertex_gradient_is_the_scattered_corner_gradient(ora):
    sc = synth.scene_tiny()
    unit = float(sc["geom"][:, 3].min())
    vidx, nv = VX.vertex_index(sc["geom"], unit)
    rng = np.random.default_rng(1)
    vals = rng.uniform(0.5, 12.0, nv)
    cam = synth.orbit_camera(20, 20, 45.0, 1.4, 75.0, 30.0, target=(0.5, 0.3, 0.5))
    gC = rng.normal(size=(400, 3))

    def loss(v):
        s2 = dict(sc)
        s2["density"] = VX.gather(vidx, v).astype(np.float32)
        return float((ora.render(s2, [cam])["rgb"] * gC).sum())

    s2 = dict(sc)
    s2["density"] = VX.gather(vidx, vals).astype(np.float32)
    bw = ora.render_backward(s2, [cam], gC)
    gv = VX.scatter_add(vidx, bw["d_density"], nv)
    hit = np.where(np.abs(gv) > 1e-3 * np.abs(gv).max())[0]
    checked = 0
    for j in rng.choice(hit, size=min(10, len(hit)), replace=False):
        eps = 1e-3 * max(1.0, abs(vals[j]))
        vp, vm = vals.copy(), vals.copy()
        vp[j] = np.float32(vals[j] + eps)
        vm[j] = np.float32(vals[j] - eps)
        fd = (loss(vp) - loss(vm)) / (float(np.float32(vp[j])) - float(np.float32(vm[j])))
        if abs(fd - gv[j]) <= 1e-4 * max(abs(fd), abs(gv[j])) + 1e-9:
            checked += 1
    assert checked >= 8
