"""CPU oracle of the in-place topology change: subdivision (Sec. IV-D,
Eq. 13-16) and removal of pruned voxels (Sec. IV-C) that rewrite the voxel
arrays where they are, instead of writing survivors and children to new
arrays.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product
package.

The selection, the children's values and the auxiliary fills are those of
``oracle.subdivide`` (used here as a step); only where each row ends up
differs.  Placement (n rows in, h of them pruned, k parents split):

  1. a split parent's row becomes its child 0;
  2. the other children -- children 1..7 of each split parent, parents in id
     order -- fill the pruned rows in increasing index order, and once those
     are used up, rows n, n + 1, ... (appended);
  3. if fewer children than pruned rows exist (7k < h), the array shrinks to
     n' = n - h + 7k: the rows at index >= n' that are still occupied move, in
     increasing index order, into the rows below n' that are still empty, in
     increasing index order.

Every other row keeps its index.  The result holds the same rows as
``oracle.subdivide``'s output (survivors in id order, then children), in
another order; n' is the same.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def placement(n: int, pruned, parents):
    """Destination of every row of ``oracle.subdivide``'s output, and n'.

    ``pruned``: sorted indices of the removed rows; ``parents``: sorted
    indices of the split parents.  Returns (dest, n_new) where dest[j] is
    the in-place index of output row j: the survivors first (in id order),
    then 8 children per parent (parent order, child index order).
    """
    pruned = np.asarray(pruned, np.int64)
    parents = np.asarray(parents, np.int64)
    h, k = len(pruned), len(parents)
    n_new = n - h + 7 * k
    gone = np.zeros(n, bool)
    gone[pruned] = True
    split = np.zeros(n, bool)
    split[parents] = True
    survivors = np.flatnonzero(~gone & ~split)           # output rows 0 .. len(survivors) - 1
    # step 1 and 2: where each child goes
    child_dest = np.empty((k, 8), np.int64)
    child_dest[:, 0] = parents
    others = 7 * k
    slots = np.concatenate([pruned[:min(h, others)], n + np.arange(max(0, others - h))])
    child_dest[:, 1:] = slots.reshape(k, 7) if k else np.zeros((0, 7), np.int64)
    # step 3: close the gaps from the tail when the array shrinks
    occupied = np.zeros(max(n, n_new), bool)
    occupied[survivors] = True
    occupied[child_dest.ravel()] = True
    move_from = np.flatnonzero(occupied[n_new:]) + n_new
    move_to = np.flatnonzero(~occupied[:n_new])
    assert len(move_from) == len(move_to)
    moved = dict(zip(move_from.tolist(), move_to.tolist()))
    remap = lambda i: moved.get(int(i), int(i))
    dest = [remap(i) for i in survivors] + [remap(i) for i in child_dest.ravel()]
    return np.asarray(dest, np.int64), n_new


def subdivide_inplace(scene: dict, delta, z, u, seen, prune_mask=None, aux=None, **params) -> dict:
    """The in-place form of ``oracle.subdivide``: same arguments and outputs
    (``geom``, ``level``, ``density``, ``sh``, ``aux``, ``selected``, ``k``,
    ``n_new``), with the rows placed as the module docstring states."""
    n = int(np.asarray(scene["geom"]).shape[0])
    r = O.subdivide(scene, delta, z, u, seen, prune_mask=prune_mask, aux=aux, **params)
    pruned = np.flatnonzero(np.asarray(prune_mask).astype(bool)) if prune_mask is not None else np.zeros(0, np.int64)
    parents = np.flatnonzero(r["selected"])
    dest, n_new = placement(n, pruned, parents)
    assert n_new == r["n_new"]
    out = dict(r)
    for name in ("geom", "level", "density", "sh"):
        a = np.zeros_like(r[name])
        a[dest] = r[name]
        out[name] = a
    out["aux"] = []
    for a_ref in r["aux"]:
        a = np.zeros_like(a_ref)
        a[dest] = a_ref
        out["aux"].append(a)
    out["dest"] = dest
    return out
