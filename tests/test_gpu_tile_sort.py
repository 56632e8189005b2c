"""Per-tile depth order of the pair lists against the oracle, bit for bit, on
lists of every length class the forward handles: up to 256 pairs (one warp),
up to 4096 (one block), longer lists sorted in chunks of 4096 and merged (two
or three chunks by merging through shared memory, more by binary searches of
the other chunks), key spans that take 3 and 4 digit passes, ties in the depth key
(broken by voxel id), and a one-tile view (no sort by tile runs).  The oracle
sorts (tile, depth key) pairs stably in voxel-id order."""
import numpy as np
import pytest

from gpu_helpers import gpu_forward, gpu_pairs
from paper_2511_02510_gb300 import synth

pytestmark = pytest.mark.gpu


def column_scene(counts, depth_ranges, seed):
    """A (32 * len(counts)) x 32 view looking along +z from (0.5, 0.5, -1) and,
    for each tile t, counts[t] small voxels near the line of sight through the
    tile's centre at camera depths log-uniform in depth_ranges[t]; a fifth of
    them in groups of about 8 sharing one depth (equal depth keys); voxel ids
    shuffled."""
    rng = np.random.default_rng(seed)
    cam = synth.look_at_camera((0.5, 0.5, -1.0), (0.5, 0.5, 1.0), 32 * len(counts), 32, 60.0, z_near=1e-3)
    fx, cx, cy = cam["fx"], cam["cx"], cam["cy"]
    cents = []
    for t, (m, (d0, d1)) in enumerate(zip(counts, depth_ranges)):
        d = np.exp(rng.uniform(np.log(d0), np.log(d1), m))
        tied = np.flatnonzero(rng.random(m) < 0.2)
        d[tied] = d[tied[rng.integers(0, max(1, len(tied) // 8), len(tied))]]
        u = 32.0 * t + 16.0 + rng.uniform(-6.0, 6.0, m)  # pixel column inside tile t
        v = 16.0 + rng.uniform(-6.0, 6.0, m)
        x = 0.5 - (u - cx) * d / fx                     # the camera's x and y axes are world -x, -y
        y = 0.5 - (v - cy) * d / fx
        cents.append(np.stack([x, y, d - 1.0], 1))      # camera depth = world z + 1
    c = np.concatenate(cents)
    c = c[rng.permutation(len(c))]
    half = 1e-3 * (c[:, 2] + 1.0)                       # about 0.06 pixel wide
    return synth.constant_voxel_scene(c, half, 2.0, np.full((len(c), 3), 0.5)), cam


def compare(ora, sc, cam):
    scene, ctx, vox = gpu_forward(sc, [cam], tile=32)
    keys, vox_ids, ranges, pairs = gpu_pairs(ctx, scene.n)
    ref = ora.pairs(sc, [cam], ts=32)
    assert pairs == ref["n_pairs"]
    np.testing.assert_array_equal(keys, ref["keys"])
    np.testing.assert_array_equal(vox_ids, ref["vals"])
    np.testing.assert_array_equal(ranges, ref["ranges"])
    return ref


def span_bits(ref, t):
    a, b = ref["ranges"][t]
    dk = (ref["keys"][a:b] & 0xffffffff).astype(np.int64)
    return int(dk.max() - dk.min()).bit_length(), len(np.unique(dk)) < len(dk)


@pytest.mark.parametrize("far,passes,longest", [(5000.0, 4, 20000), (40.0, 3, 11000)])
def test_long_tile_lists_bit_exact(ora, far, passes, longest):
    # tile 0: 20000 pairs (5 chunks: merged by binary searches) or 11000 (3 chunks: two merges in
    # shared memory), tile 1: 7000 (2 chunks), tile 2: 900 (one block), tile 3: 200 (one warp).  Depths
    # 0.01..5000 span 28 bits of key (4 passes of 9 bits), 0.5..40 span 26 bits (3 passes)
    sc, cam = column_scene([longest, 7000, 900, 200],
                           [(0.01 if passes == 4 else 0.5, far), (0.5, 30.0), (0.3, 3.0), (0.2, 9.0)], 3)
    ref = compare(ora, sc, cam)
    lens = (ref["ranges"][:, 1] - ref["ranges"][:, 0]).astype(np.int64)
    assert lens[0] == longest and lens[1] == 7000 and lens[2] == 900 and lens[3] == 200
    bits, ties = span_bits(ref, 0)
    assert (bits + 8) // 9 == passes and ties
    assert all(span_bits(ref, t)[1] for t in (1, 2, 3))


def test_one_tile_view_bit_exact(ora):
    sc, cam = column_scene([3000], [(0.05, 20.0)], 5)
    ref = compare(ora, sc, cam)
    assert ref["n_pairs"] == 3000 and ref["ranges"].shape == (1, 2) and span_bits(ref, 0)[1]
