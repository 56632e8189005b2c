"""CPU oracle for the shared grid-vertex density variant: the corner ->
vertex numbering and the gather / scatter between vertex values and
per-voxel corners.  Plain numpy.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product
package.

Definition: corner c (= x + 2y + 4z) of voxel v lies at centre +- h per
axis; two corners are the same vertex when they are the same point of the
finest grid (coordinates in units of the finest half-size).  Vertex ids are
the ranks of the distinct points ordered by (z, y, x).  With the vertex
variant a voxel's corner densities are the values of its 8 vertices, and the
gradient of a vertex value is the sum of the gradients of the corners that
read it.
"""
from __future__ import annotations

import numpy as np

COORD_BITS = 21
COORD_OFF = 1 << (COORD_BITS - 1)


def corner_points(geom, unit):
    """Integer finest-grid coordinates [n, 8, 3] of every voxel corner."""
    g = np.asarray(geom, np.float64).reshape(-1, 4)
    sign = np.array([[1 if c & 1 else -1, 1 if c & 2 else -1, 1 if c & 4 else -1] for c in range(8)], np.float64)
    p = g[:, None, :3] + sign[None] * g[:, None, 3:4]
    x = p / unit
    r = np.rint(x)
    if np.any(np.abs(x - r) > 1e-3) or np.any(r < -COORD_OFF) or np.any(r >= COORD_OFF):
        raise ValueError("corners are not on the finest grid")
    return r.astype(np.int64)


def vertex_index(geom, unit):
    """(vidx [n, 8] int64, n_vert)."""
    q = corner_points(geom, unit) + COORD_OFF
    keys = q[..., 0] | (q[..., 1] << COORD_BITS) | (q[..., 2] << (2 * COORD_BITS))
    uniq, inv = np.unique(keys.ravel(), return_inverse=True)
    return inv.reshape(-1, 8), int(uniq.size)


def gather(vidx, values):
    return np.asarray(values, np.float64)[np.asarray(vidx)]


def scatter_add(vidx, corners, n_vert):
    out = np.zeros(n_vert, np.float64)
    np.add.at(out, np.asarray(vidx).ravel(), np.asarray(corners, np.float64).ravel())
    return out
