"""The GPU side of data-parallel training over views: two calls that each
render one view, with disjoint pixel-id bases (lv_raster_opts.pixel_id_base),
reduced as the exchange step reduces them (maximum of the packed w_max,
minimum of z_min and delta_min, maximum of seen, sum of the gradients), equal
one call over both views: bit for bit for the statistics and the packed w_max
(Eq. 5's argmax and tie rule included), within the per-element gradient
tolerance of the oracle parity tests for the sums."""
import numpy as np
import pytest
import torch

from gpu_helpers import np_, to_scene
from paper_2511_02510_gb300 import dp
from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth
from paper_2511_02510_gb300.raster import RasterContext
from parity import check_grads

pytestmark = pytest.mark.gpu


def cams():
    return [synth.orbit_camera(96, 72, 60.0, 1.6, 30.0, 25.0, target=(0.5, 0.4, 0.5)),
            synth.orbit_camera(80, 64, 60.0, 1.6, 150.0, 30.0, target=(0.5, 0.4, 0.5))]


def render(scene, cs, base, g, tile=16):
    ctx = RasterContext(cs, scene.n, tile=tile)
    ctx.opts.pixel_id_base = base
    vox = scene.voxels()
    ctx.fit_capacity(vox)
    ctx.reset_stats()
    ctx.forward(vox)
    dd, ds = ctx.backward(vox, g)
    torch.cuda.synchronize()
    ctx.check()
    return ctx, dd, ds


@pytest.mark.parametrize("tile", [16, 32])
def test_two_calls_with_pixel_bases_equal_one_call(ora, tile):
    sc = synth.scene_tiny()
    scene = to_scene(sc)
    cs = cams()
    sizes = [c["width"] * c["height"] for c in cs]
    bases = dp.pixel_id_bases(sizes)
    gn = np.random.default_rng(5).normal(size=(sum(sizes), 3)).astype(np.float32)
    gn[ora.render(sc, cs)["near_stop"] != 0] = 0      # stop decisions within rounding are excluded
    g = torch.from_numpy(gn).cuda()
    whole, dd, ds = render(scene, cs, 0, g, tile)
    parts = [render(scene, [cs[v]], bases[v], g[bases[v]:bases[v] + sizes[v]].contiguous(), tile) for v in range(2)]
    wm = torch.maximum(parts[0][0].wmax_packed, parts[1][0].wmax_packed)
    np.testing.assert_array_equal(np_(wm), np_(whole.wmax_packed))
    np.testing.assert_array_equal(np_(torch.minimum(parts[0][0].z_min, parts[1][0].z_min)).view(np.uint32),
                                  np_(whole.z_min).view(np.uint32))
    np.testing.assert_array_equal(np_(torch.minimum(parts[0][0].delta_min, parts[1][0].delta_min)).view(np.uint32),
                                  np_(whole.delta_min).view(np.uint32))
    np.testing.assert_array_equal(np_(torch.maximum(parts[0][0].seen, parts[1][0].seen)), np_(whole.seen))
    # the image of each view is the one call's image of that view, bit for bit
    for v in range(2):
        np.testing.assert_array_equal(np_(parts[v][0].rgb), np_(whole.rgb)[bases[v]:bases[v] + sizes[v]])
    # gradient sums against the oracle's two-view gradients
    g64 = np_(g).astype(np.float64)
    ref = ora.render_backward(sc, cs, g64)
    e = ora.backward_bounds(sc, cs, g64)
    u = 2.0 ** -24
    for k, i, ek, ak in (("d_density", 1, "e_density", "a_density"), ("d_sh", 2, "e_sh", "a_sh")):
        summed = np_(parts[0][i]) + np_(parts[1][i])
        check_grads(k, summed, ref[k], e[ek] + u * np.abs(ref[k]), e[ak] + u * np.abs(ref[k]))


def test_pixel_id_base_is_checked():
    sc = synth.scene_tiny()
    scene = to_scene(sc)
    cs = cams()
    ctx = RasterContext(cs[:1], scene.n)
    bad = L.make_opts(16, pixel_id_base=(1 << 32) - 100)
    with pytest.raises(L.LvError) as ei:
        L.lv_rasterize_forward(scene.voxels(), ctx.cams_arr, 1, bad, ctx.fwd_struct(), ctx.workspace,
                               ctx.pair_capacity)
    assert ei.value.status == L.LV_ERR_INVALID_ARG
