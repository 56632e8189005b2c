"""The benchmark step on four streams (LF weights beside the forward, the LF
loss's gradient fused into the backward composite, pruning and the subdivision
selection beside the backward, the in-place topology change after both with
the SH backward beside it)
computes what the one-stream step computes: the same bits for every output
that has a fixed summation order (dL/drgb, the rewritten voxel rows and
auxiliary arrays included), the same loss up to the order of its sums, and the
same gradients up to the order of the FP32 atomic sums.  Both steps start from the same state; the restore that the timed bench
adds at the end of a step is left out, so the rewritten rows can be compared."""
import pytest
import torch

import bench
from paper_2511_02510_gb300 import synth

pytestmark = pytest.mark.gpu


def test_four_stream_step_matches_one_stream():
    wl = bench.Workload(synth.scene_tiny(), bench.camera_for(0), synth.random_image(bench.W_IMG, bench.H_IMG, seed=3))
    state = wl.cap_arrays + wl.aux_arrays          # EMA and hysteresis state are the last two aux arrays
    start = [t.clone() for t in state]

    def reset():
        for t, t0 in zip(state, start):
            t.copy_(t0)

    def outputs():
        n_new = int(wl.n_new.item())
        exact = [wl.dL, wl.w_max, wl.w_arg, wl.pmask, wl.selected, wl.n_new, wl.n_pruned]
        exact += [t[:n_new] for t in state]
        return [t.clone() for t in exact], wl.d_dens.clone(), wl.d_sh.clone(), float(wl.loss[0])

    wl.step()
    torch.cuda.synchronize()
    a, a_dd, a_dsh, a_loss = outputs()
    reset()
    wl.step_concurrent()
    torch.cuda.synchronize()
    b, b_dd, b_dsh, b_loss = outputs()
    assert int(wl.n_new.item()) > wl.n and int(wl.selected.sum().item()) > 0 and int(wl.n_pruned.item()) > 0
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert a_loss > 0 and abs(a_loss - b_loss) <= 2e-6 * a_loss
    for x, y in ((a_dd, b_dd), (a_dsh, b_dsh)):
        scale = float(x.abs().max())
        assert scale > 0 and float((x - y).abs().max()) <= 1e-5 * scale
