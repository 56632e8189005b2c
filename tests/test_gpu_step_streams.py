"""The benchmark step on three streams (LF weights beside the forward, pruning
and the subdivision selection beside the backward) computes what the one-stream
step computes: the same bits for every output that has a fixed summation order,
and the same gradients up to the order of the FP32 atomic sums."""
import pytest
import torch

import bench
from paper_2511_02510_gb300 import synth

pytestmark = pytest.mark.gpu


def test_three_stream_step_matches_one_stream():
    wl = bench.Workload(synth.scene_tiny(), bench.camera_for(0), synth.random_image(bench.W_IMG, bench.H_IMG, seed=3))
    for _ in range(2):
        wl.step()
    torch.cuda.synchronize()
    ema0, st0 = wl.ema.clone(), wl.state.clone()

    def outputs():
        n_new = int(wl.n_new.item())
        exact = [wl.loss, wl.dL, wl.w_max, wl.w_arg, wl.pmask, wl.selected, wl.n_new, wl.n_pruned, wl.ema, wl.state,
                 wl.o_geom[:n_new], wl.o_dens[:n_new], wl.o_sh[:n_new]] + [a[:n_new] for a in wl.aux_out]
        return [t.clone() for t in exact], wl.d_dens.clone(), wl.d_sh.clone()

    wl.step()
    torch.cuda.synchronize()
    a, a_dd, a_dsh = outputs()
    wl.ema.copy_(ema0)
    wl.state.copy_(st0)
    wl.step_concurrent()
    torch.cuda.synchronize()
    b, b_dd, b_dsh = outputs()
    assert int(wl.n_new.item()) > 0 and int(wl.selected.sum().item()) > 0
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    for x, y in ((a_dd, b_dd), (a_dsh, b_dsh)):
        scale = float(x.abs().max())
        assert scale > 0 and float((x - y).abs().max()) <= 1e-5 * scale
