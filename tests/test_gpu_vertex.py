"""GPU parity of the shared grid-vertex density variant against the oracle:
the vertex numbering bit for bit, gather and scatter exactly, and the
rasterizer reading vertex densities (images, the per-corner gradient turned
into the vertex gradient, the FP64 re-render).  Tolerances as for the
per-voxel corners; the scattered vertex gradient sums FP32 atomics in any
order (1e-4 of the largest gradient, like every gradient)."""
import numpy as np
import pytest
import torch

from gpu_helpers import np_
from oracle import vertex as VX
from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth
from paper_2511_02510_gb300.raster import RasterContext
from parity import check_grads
from test_gpu_render import _loss_grads, cam_near, compare_images

pytestmark = pytest.mark.gpu


def gpu_index(geom_np, unit):
    geom = torch.as_tensor(geom_np).cuda()
    vidx = torch.empty((geom.shape[0], 8), dtype=torch.int32, device="cuda")
    nv = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.lv_build_vertex_index(geom, unit, vidx, nv, st)
    torch.cuda.synchronize()
    return vidx, int(nv.item()), int(st.item())


@pytest.mark.parametrize("which", ["tiny", "360"])
def test_vertex_index_bit_exact(which):
    sc = synth.scene_tiny() if which == "tiny" else synth.scene_360()
    unit = float(sc["geom"][:, 3].min())
    vidx, nv, st = gpu_index(sc["geom"], unit)
    ref, nref = VX.vertex_index(sc["geom"], unit)
    assert st == 0 and nv == nref
    np.testing.assert_array_equal(np_(vidx).astype(np.int64), ref)


def test_misaligned_corners_report():
    sc = synth.constant_voxel_scene([[0.1, 0.2, 0.3]], 0.25, [1.0], [(1, 1, 1)])
    _, _, st = gpu_index(sc["geom"], 0.25)          # 0.1 +- 0.25 is not a multiple of 0.25
    assert st == L.LV_ERR_INVALID_ARG


def test_gather_and_scatter_exact():
    sc = synth.scene_tiny()
    unit = float(sc["geom"][:, 3].min())
    vidx, nv, _ = gpu_index(sc["geom"], unit)
    rng = np.random.default_rng(0)
    vals = rng.normal(size=nv).astype(np.float32)
    corners = torch.empty((sc["geom"].shape[0], 8), device="cuda")
    L.lv_vertex_gather(vidx, torch.as_tensor(vals).cuda(), corners)
    ref_vidx = np_(vidx).astype(np.int64)
    np.testing.assert_array_equal(np_(corners), vals[ref_vidx])
    # integer-valued corner data: FP32 atomic sums are exact in any order
    cint = rng.integers(-50, 50, size=(sc["geom"].shape[0], 8)).astype(np.float32)
    s = torch.zeros(nv, device="cuda")
    cnt = torch.zeros(nv, device="cuda")
    L.lv_vertex_scatter_add(vidx, torch.as_tensor(cint).cuda(), s, cnt)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(np_(s), VX.scatter_add(ref_vidx, cint, nv).astype(np.float32))
    np.testing.assert_array_equal(np_(cnt), np.bincount(ref_vidx.ravel(), minlength=nv).astype(np.float32))


def test_vertex_render_forward_backward(ora):
    sc = synth.scene_tiny()
    unit = float(sc["geom"][:, 3].min())
    vidx, nv, _ = gpu_index(sc["geom"], unit)
    ref_vidx = np_(vidx).astype(np.int64)
    # vertex values: the average of the corners that meet there (as a caller converts a scene)
    vsum = VX.scatter_add(ref_vidx, sc["density"], nv)
    vcnt = np.bincount(ref_vidx.ravel(), minlength=nv)
    vals = (vsum / vcnt).astype(np.float32)
    cams = [cam_near(90, 70), cam_near(64, 64, az=200.0)]
    geom = torch.as_tensor(sc["geom"]).cuda()
    dens_v = torch.as_tensor(vals).cuda()
    sh = torch.as_tensor(sc["sh"]).cuda()
    vox = L.make_voxels(geom, dens_v, sh, vidx=vidx)
    vox.n = sc["geom"].shape[0]
    ctx = RasterContext(cams, vox.n)
    ctx.fit_capacity(vox)
    ctx.reset_stats()
    ctx.forward(vox)
    ctx.check()
    ref_sc = dict(sc)
    ref_sc["density"] = vals[ref_vidx]
    r = ora.render(ref_sc, cams)
    compare_images(r, ctx)
    # backward: per-corner gradient from the rasterizer, vertex gradient by scatter
    gC, gD, gT = _loss_grads(ctx.n_pix, 5, r["near_stop"])
    d_corner, _ = ctx.backward(vox, torch.from_numpy(gC).cuda(), torch.from_numpy(gD).cuda(),
                               torch.from_numpy(gT).cuda())
    gv = torch.zeros(nv, device="cuda")
    L.lv_vertex_scatter_add(vidx, d_corner, gv)
    torch.cuda.synchronize()
    f64 = lambda x: x.astype(np.float64)
    bw = ora.render_backward(ref_sc, cams, f64(gC), f64(gD), f64(gT))
    eb = ora.backward_bounds(ref_sc, cams, f64(gC), f64(gD), f64(gT))
    # a vertex sums the corners that share it: their floors add, plus the order of that sum
    cnt = np.bincount(ref_vidx.ravel(), minlength=nv).astype(np.float64)
    ref_v = VX.scatter_add(ref_vidx, bw["d_density"], nv)
    abs_v = VX.scatter_add(ref_vidx, np.abs(bw["d_density"]), nv)
    e_v = VX.scatter_add(ref_vidx, eb["e_density"], nv) + 2.0 ** -24 * (cnt + 1) * abs_v
    a_v = VX.scatter_add(ref_vidx, eb["a_density"], nv) + 2.0 ** -24 * (cnt + 1) * abs_v
    print("vertex gradients:", check_grads("d_vertex", np_(gv), ref_v, e_v, a_v))
    # FP64 re-render reads the vertices too
    px = torch.arange(ctx.n_pix, dtype=torch.int64, device="cuda")
    rgb = torch.zeros((ctx.n_pix, 3), dtype=torch.float64, device="cuda")
    L.lv_render_pixels_f64(vox, ctx.cams_arr, ctx.n_views, ctx.opts, ctx.workspace, ctx.pair_capacity, px, rgb, None)
    torch.cuda.synchronize()
    assert np.abs(np_(rgb) - r["rgb"]).max() < 1e-10


def test_subdivide_rejects_vertex_densities():
    sc = synth.scene_tiny()
    unit = float(sc["geom"][:, 3].min())
    vidx, nv, _ = gpu_index(sc["geom"], unit)
    geom = torch.as_tensor(sc["geom"]).cuda()
    vox = L.make_voxels(geom, torch.zeros(nv, device="cuda"), torch.as_tensor(sc["sh"]).cuda(),
                        torch.as_tensor(sc["level"]).cuda(), vidx=vidx)
    p = L.lv_subdiv_params()
    p.kappa, p.beta, p.top_ppm, p.l_max, p.budget, p.lo_ppm, p.hi_ppm = 1.0, 0.2, 50000, 16, 1 << 40, 50000, 950000
    n = sc["geom"].shape[0]
    ws = torch.empty(L.lv_subdivide_workspace_size(n, p), dtype=torch.uint8, device="cuda")
    one = torch.ones(n, device="cuda")
    with pytest.raises(L.LvError):
        L.lv_subdivide_select(vox, one, one, one, torch.ones(n, dtype=torch.uint8, device="cuda"), None, p, 8 * n,
                              torch.zeros(n, dtype=torch.uint8, device="cuda"),
                              torch.zeros(1, dtype=torch.int64, device="cuda"), ws)


def test_vertex_calls_with_no_voxels():
    geom = torch.zeros((0, 4), device="cuda")
    vidx = torch.zeros((0, 8), dtype=torch.int32, device="cuda")
    nv = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    L.lv_build_vertex_index(geom, 0.5, vidx, nv)
    torch.cuda.synchronize()
    assert int(nv.item()) == 0
    L.lv_vertex_gather(vidx, torch.zeros(1, device="cuda"), torch.zeros((0, 8), device="cuda"))
    L.lv_vertex_scatter_add(vidx, torch.zeros((0, 8), device="cuda"), torch.zeros(1, device="cuda"))
