"""The C-ABI autotuner (lv_autotune): every (tile, schedule, batch) candidate is
timed on the caller's scene, the fastest is returned, the choice is cached,
candidates that overflow the pair capacity are skipped, and the chosen
options render the same image as the defaults."""
import numpy as np
import pytest
import torch

from gpu_helpers import np_
from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth
from paper_2511_02510_gb300.raster import RasterContext

pytestmark = pytest.mark.gpu


def _setup():
    sc = synth.scene_tiny()
    arrays = [torch.as_tensor(sc[k]).cuda() for k in ("geom", "density", "sh")]
    vox = L.make_voxels(*arrays)
    cams = [synth.orbit_camera(128, 96, 60.0, 3.0, 20.0, 15.0), synth.orbit_camera(200, 130, 60.0, 3.0, 140.0, 25.0)]
    return sc, arrays, vox, cams


def test_autotune_picks_the_fastest_and_caches(tmp_path):
    sc, arrays, vox, cams = _setup()
    cams_arr = L.make_cameras(cams)
    base = L.make_opts()
    cap = 400000
    ws = torch.empty(L.lv_autotune_workspace_size(vox.n, cams_arr, len(cams), base, cap), dtype=torch.uint8,
                     device="cuda")
    path = str(tmp_path / "tune.txt")
    best, ms = L.lv_autotune(vox, cams_arr, len(cams), base, cap, 3, ws, path)
    assert best.tile in (8, 16, 32) and best.batch in (32, 64, 128)
    # every candidate timed except batch 128 with tile 32 (refused)
    refused = [6 * 2 + 3 * p + 2 for p in (0, 1)]
    assert all(m > 0 for i, m in enumerate(ms) if i not in refused) and all(ms[i] == -1 for i in refused)
    idx = [8, 16, 32].index(best.tile) * 6 + (3 if best.flags & L.LV_FLAG_PERSISTENT else 0) + \
        [32, 64, 128].index(best.batch)
    assert ms[idx] == min(m for m in ms if m > 0)
    # cache hit: same choice, nothing timed
    best2, ms2 = L.lv_autotune(vox, cams_arr, len(cams), base, cap, 3, ws, path)
    assert best2.tile == best.tile and best2.flags == best.flags and best2.batch == best.batch
    assert all(m == -1 for m in ms2)
    assert open(path).read().count("\n") == 1
    # the chosen options give the image of the default ones
    imgs = []
    for o in (base, best):
        ctx = RasterContext(cams, vox.n, tile=o.tile, batch=o.batch, persistent=bool(o.flags & L.LV_FLAG_PERSISTENT))
        ctx.fit_capacity(vox)
        ctx.forward(vox)
        ctx.check()
        imgs.append(np_(ctx.rgb).copy())
    assert np.abs(imgs[0] - imgs[1]).max() < 1e-5


def test_autotune_skips_candidates_over_capacity():
    sc, arrays, vox, cams = _setup()
    cams_arr = L.make_cameras(cams)
    base = L.make_opts()
    ws = torch.empty(L.lv_autotune_workspace_size(vox.n, cams_arr, len(cams), base, 1), dtype=torch.uint8,
                     device="cuda")
    with pytest.raises(L.LvError):
        L.lv_autotune(vox, cams_arr, len(cams), base, 1, 2, ws)
