"""The allocation-free LF loss entry point (for callers that cannot allocate
device memory themselves) gives the same result as the workspace version.

Collected last on purpose: a failure here leaves every other test already run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the tolerance of the LF-loss parity tests (FP64 sums in a different order)


def _params(gamma_max=0.6, t0=300.0, t1=600.0):
    p = L.lv_lf_params()
    p.eps, p.gamma_max, p.t0, p.t1, p.pctl_ppm = 1e-3, gamma_max, t0, t1, 990000
    return p


def _inputs(sizes, seed):
    gt = np.concatenate([synth.smooth_image(w, h, seed=seed + i) for i, (w, h) in enumerate(sizes)])
    rng = np.random.default_rng(seed)
    rgb = np.clip(gt + rng.normal(0, 0.1, gt.shape), 0, 1).astype(np.float32)
    return torch.from_numpy(rgb).cuda(), torch.from_numpy(gt).cuda()


def _with_workspace(rgb, gt, sizes, t, p):
    W, H = [s[0] for s in sizes], [s[1] for s in sizes]
    ws = torch.empty(L.lv_lf_workspace_size(W, H), dtype=torch.uint8, device="cuda")
    loss = torch.zeros(len(sizes), dtype=torch.float32, device="cuda")
    g = torch.zeros_like(rgb)
    L.lv_lf_weighted_loss(rgb, gt, W, H, t, p, loss, g, ws)
    return loss, g


def _no_alloc(rgb, gt, sizes, t, p):
    W, H = [s[0] for s in sizes], [s[1] for s in sizes]
    loss = torch.full((len(sizes),), -1.0, dtype=torch.float32, device="cuda")
    g = torch.full_like(rgb, -1.0)
    L.lv_lf_weighted_loss_noalloc(rgb, gt, W, H, t, p, loss, g)
    return loss, g


def test_no_alloc_matches_workspace_version_on_consecutive_calls():
    calls = [([(1237, 822)], 450.0, 11), ([(320, 240), (97, 61), (640, 480)], 1000.0, 12)]
    for sizes, t, seed in calls:
        rgb, gt = _inputs(sizes, seed)
        p = _params()
        la, ga = _with_workspace(rgb, gt, sizes, t, p)
        lb, gb = _no_alloc(rgb, gt, sizes, t, p)
        torch.cuda.synchronize()
        la, ga, lb, gb = (x.cpu().numpy() for x in (la, ga, lb, gb))
        np.testing.assert_allclose(lb, la, rtol=TOL)
        assert np.abs(gb - ga).max() <= TOL * np.abs(ga).max()


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    rgb = torch.zeros((1, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(L.LvError) as ei:
        L.lv_lf_weighted_loss_noalloc(rgb, rgb, [2048], [1024], 0.0, _params(), torch.zeros(1, device="cuda"), None)
    assert ei.value.status == L.LV_ERR_INVALID_ARG
    assert "scratch" in L.last_error()
