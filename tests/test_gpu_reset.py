"""lv_reset_stats: one launch starts a new statistics window (w_max 0,
z_min and delta_min +inf, seen 0), on aligned arrays, on views that start at
an odd element, at ragged lengths, and with arrays left out."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import np_
from paper_2511_02510_gb300 import litevoxel as L

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,off", [(1, 0), (4097, 0), (4097, 1), (100003, 3)])
def test_reset_stats(n, off):
    w = torch.full((n + off,), 7, dtype=torch.int64, device="cuda")[off:]
    z = torch.full((n + off,), 2.0, device="cuda")[off:]
    d = torch.full((n + off,), 3.0, device="cuda")[off:]
    s = torch.full((n + off,), 1, dtype=torch.uint8, device="cuda")[off:]
    L.lv_reset_stats(w, z, d, s)
    torch.cuda.synchronize()
    assert np.all(np_(w) == 0) and np.all(np_(s) == 0)
    assert np.all(np.isposinf(np_(z))) and np.all(np.isposinf(np_(d)))


def test_reset_stats_subset():
    n = 1000
    z = torch.zeros(n, device="cuda")
    s = torch.ones(n, dtype=torch.uint8, device="cuda")
    L.lv_reset_stats(None, z, None, s)
    torch.cuda.synchronize()
    assert np.all(np.isposinf(np_(z))) and np.all(np_(s) == 0)
    assert math.isinf(float(z[-1]))
