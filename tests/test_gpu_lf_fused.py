"""The LF-weighted loss fused into the backward composite (Sec. IV-B, Eq. 8 and
18) against the separate loss call on the same rendered image: dL/drgb bit for
bit, the density and SH gradients up to the order of the FP32 atomic sums, the
per-view loss within FP32 summation order (the fused backward sums per warp and
block, the loss kernel per thread and block), for one-block-per-tile and
persistent schedules and several views; the sums start from zero again after
lv_lf_loss_finish; bad fused-loss arguments are refused on the host."""
import numpy as np
import pytest
import torch

from gpu_helpers import gpu_forward
from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth
from paper_2511_02510_gb300.raster import RasterContext

pytestmark = pytest.mark.gpu


def lf_params():
    p = L.lv_lf_params()
    p.eps, p.t0, p.t1, p.gamma_max, p.pctl_ppm = 1e-3, 0.0, 900.0, 2.0, 990000
    return p


@pytest.mark.parametrize("tile,persistent", [(16, False), (32, True), (8, False)])
def test_fused_loss_matches_the_loss_call(tile, persistent):
    sc = synth.scene_tiny()
    cams = [synth.orbit_camera(120, 90, 60.0, 1.6, 30.0, 25.0, target=(0.5, 0.4, 0.5)),
            synth.orbit_camera(77, 101, 60.0, 1.7, 160.0, 30.0, target=(0.5, 0.4, 0.5))]
    widths, heights = [c["width"] for c in cams], [c["height"] for c in cams]
    scene, ctx0, vox = gpu_forward(sc, cams)
    ctx = RasterContext(cams, scene.n, tile=tile, persistent=persistent)
    ctx.fit_capacity(vox)
    gt = torch.from_numpy(np.concatenate([synth.smooth_image(w, h, seed=5 + i).reshape(-1, 3)
                                          for i, (w, h) in enumerate(zip(widths, heights))])).float().cuda()
    P = gt.shape[0]
    p = lf_params()
    ws_a = torch.empty(L.lv_lf_workspace_size(widths, heights), dtype=torch.uint8, device="cuda")
    ws_b = torch.empty_like(ws_a)
    loss_a = torch.zeros(2, device="cuda")
    dl_a = torch.zeros(P, 3, device="cuda")
    ctx.reset_stats()
    ctx.forward(vox)
    L.lv_lf_weighted_loss(ctx.rgb, gt, widths, heights, 450.0, p, loss_a, dl_a, ws_a)
    dd_a, ds_a = ctx.backward(vox, dl_a)
    dd_a, ds_a = dd_a.clone(), ds_a.clone()
    for rep in range(2):  # the second round checks that lv_lf_loss_finish cleared the sums
        loss_b = torch.zeros(2, device="cuda")
        dl_b = torch.full((P, 3), float("nan"), device="cuda")
        L.lv_lf_weights(gt, widths, heights, 450.0, p, ws_b)
        dd_b, ds_b = ctx.backward(vox, None, lf=(gt, ws_b, dl_b))
        L.lv_lf_loss_finish(widths, heights, loss_b, ws_b)
        ctx.check()
        assert torch.equal(dl_b, dl_a)
        for x, y in ((dd_a, dd_b), (ds_a, ds_b)):
            scale = float(x.abs().max())
            assert scale > 0 and float((x - y).abs().max()) <= 1e-5 * scale
        la, lb = loss_a.cpu().numpy().astype(np.float64), loss_b.cpu().numpy().astype(np.float64)
        assert np.all(la > 0) and np.all(np.abs(la - lb) <= 2e-6 * la)
        if rep == 0:  # the loss again from the same sums: finish cleared them
            L.lv_lf_loss_finish(widths, heights, loss_b, ws_b)
            assert float(loss_b.abs().max()) == 0.0


def test_fused_loss_argument_checks():
    sc = synth.scene_tiny()
    cams = [synth.orbit_camera(64, 48, 60.0, 1.6, 30.0, 25.0, target=(0.5, 0.4, 0.5))]
    scene, ctx, vox = gpu_forward(sc, cams)
    gt = torch.zeros(64 * 48, 3, device="cuda")
    ws = torch.empty(L.lv_lf_workspace_size([64], [48]), dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LvError) as ei:  # neither dL_drgb nor the fused loss
        ctx.backward(vox, None)
    assert ei.value.status == L.LV_ERR_INVALID_ARG
    with pytest.raises(L.LvError) as ei:  # lf_gt missing
        ctx.backward(vox, None, lf=(None, ws, None))
    assert ei.value.status == L.LV_ERR_INVALID_ARG
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LvError) as ei:  # workspace too small for the views
        ctx.backward(vox, None, lf=(gt, small, None))
    assert ei.value.status == L.LV_ERR_WORKSPACE
