"""Data-parallel training over views: one process per GPU, each rendering its own
views of the same replicated voxel state, then one exchange step.

Every rank runs the forward (Eq. 1-5), its loss and the backward (reverse of
Eq. 2-4) on its own views through the library.  The exchange then gives every
rank what one call over all the views would have produced:

  - d_density [n, 8] and d_sh [n, 48]: summed (each view's loss is its own mean,
    so the gradient of the total loss is the sum over views);
  - packed w_max [n] (Eq. 5): the maximum.  The packed word is
    (f32 bits of w << 32) | (0xffffffff - pixel id); with disjoint pixel ids per
    rank (``pixel_id_bases`` and ``lv_raster_opts.pixel_id_base``) the maximum
    keeps the larger weight and, on equal weights, the smaller global pixel id:
    the argmax and tie rule of one call over all views.  w >= 0, so the high
    word stays below 2^31 and the signed 64-bit maximum orders the words as the
    unsigned one does;
  - z_min and delta_min [n]: the minimum; seen [n]: the maximum (logical or).

Pruning (Eq. 11-12) and subdivision (Eq. 13-16) are deterministic functions of
these reduced arrays and of the replicated state, so every rank then takes the
same decisions with no further exchange.  The collectives are those of the
process group's backend: NCCL for GPU tensors, gloo for host tensors.  No data
passes between GPUs any other way.
"""
from __future__ import annotations


def pixel_id_bases(pixels_per_rank) -> list:
    """Global id of each rank's first pixel: the pixels of the ranks before it, in rank order
    (views numbered rank-major, as one call over all ranks' views would number them)."""
    out, acc = [], 0
    for p in pixels_per_rank:
        out.append(acc)
        acc += int(p)
    if acc > 0xfffffffe:
        raise ValueError("more than 2^32 - 1 pixels over all ranks")
    return out


def allreduce_step(d_density, d_sh, wmax_packed, z_min, delta_min, seen, group=None):
    """The exchange step of one data-parallel training step, in place on every rank.

    d_density, d_sh: float gradients (summed); wmax_packed: int64 view of the packed
    w_max words (maximum); z_min, delta_min: float (minimum); seen: uint8 (maximum).
    Any argument may be None (that array is not exchanged)."""
    import torch.distributed as dist
    ops = ((d_density, dist.ReduceOp.SUM), (d_sh, dist.ReduceOp.SUM), (wmax_packed, dist.ReduceOp.MAX),
           (z_min, dist.ReduceOp.MIN), (delta_min, dist.ReduceOp.MIN), (seen, dist.ReduceOp.MAX))
    for t, op in ops:
        if t is not None:
            dist.all_reduce(t, op=op, group=group)
