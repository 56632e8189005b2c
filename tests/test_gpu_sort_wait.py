"""The radix sort's look-back wait is bounded: a tile whose predecessor never
publishes its counts gives up, reports LV_ERR_TIMEOUT and returns, and the
GPU keeps working (a full forward pass afterwards is exact)."""
import time

import pytest
import torch

from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth
from paper_2511_02510_gb300.raster import RasterContext
from test_gpu_render import compare_images

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit", [1, 1000])
def test_lookback_wait_gives_up(limit):
    ws = torch.empty(L.lv_debug_sort_timeout_workspace_size(), dtype=torch.uint8, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    L.lv_debug_sort_timeout(limit, ws, st)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 5.0
    assert int(st.item()) == L.LV_ERR_TIMEOUT


def test_gpu_usable_after_timeout(ora):
    ws = torch.empty(L.lv_debug_sort_timeout_workspace_size(), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.lv_debug_sort_timeout(100, ws, st)
    torch.cuda.synchronize()
    assert int(st.item()) == L.LV_ERR_TIMEOUT
    sc = synth.scene_tiny()
    cams = [synth.orbit_camera(96, 80, 60.0, 3.0, 20.0, 15.0)]
    arrays = [torch.as_tensor(sc[k]).cuda() for k in ("geom", "density", "sh")]  # kept alive for the calls
    vox = L.make_voxels(*arrays)
    ctx = RasterContext(cams, vox.n)
    ctx.fit_capacity(vox)
    ctx.forward(vox)
    ctx.check()
    compare_images(ora.render(sc, cams), ctx)


def test_bad_arguments():
    ws = torch.empty(L.lv_debug_sort_timeout_workspace_size(), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    for lim in (0, (1 << 20) + 1):
        with pytest.raises(L.LvError):
            L.lv_debug_sort_timeout(lim, ws, st)
