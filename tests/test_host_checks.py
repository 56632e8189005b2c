"""Host-side argument checks of the C ABI, run without a GPU.

Every entry point validates its pointers, sizes, dtypes and options on the
host before it touches the device: a bad call returns LV_ERR_INVALID_ARG (or
LV_ERR_UNSUPPORTED / LV_ERR_WORKSPACE), leaves a message in lv_last_error and
launches no kernel.  The device addresses below are never dereferenced by a
check, so any 256-byte-aligned integer stands in for one.

The module runs only where no CUDA device is present: there a call that got
past its checks by mistake fails at its first CUDA call instead of launching
a kernel on the stand-in addresses.
"""
import ctypes as C
import math

import pytest
import torch

from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth

pytestmark = pytest.mark.skipif(torch.cuda.is_available(),
                                reason="stand-in device addresses are only safe without a CUDA device")

ADDR = 1 << 24          # a 256-byte-aligned stand-in for a device pointer
TINY_WS = 64            # smaller than any workspace the library asks for


@pytest.fixture(scope="module")
def lib():
    from paper_2511_02510_gb300 import build as B
    B.build()
    return L.load()


def cams_of(*sizes):
    return L.make_cameras([synth.orbit_camera(w, h, 60.0, 3.0, 0.0, 10.0) for w, h in sizes])


def voxels(n=100, **kw):
    v = L.lv_voxels(n=n, geom=ADDR, level=ADDR, density=ADDR, density_dtype=L.LV_F32, sh=ADDR,
                    sh_dtype=L.LV_F32, sh_degree=3, vidx=None)
    for k, x in kw.items():
        setattr(v, k, x)
    return v


def fwd_out(**kw):
    o = L.lv_fwd_out(rgb=ADDR, T=ADDR, n_contrib=ADDR)
    for k, x in kw.items():
        setattr(o, k, x)
    return o


def opts(**kw):
    o = L.make_opts()
    for k, x in kw.items():
        setattr(o, k, x)
    return o


def expect(lib, code, fn, *args):
    """fn(*args) returns `code`, leaves a message and launches nothing."""
    before = lib.lv_launch_count()
    got = fn(*args)
    assert got == code, (L.STATUS_NAMES.get(got, got), L.last_error())
    assert L.last_error(), "no message for a failed call"
    assert lib.lv_launch_count() == before


# ------------------------------------------------------------------ forward / backward
FORWARD_CASES = {
    "null voxels": dict(vox=None),
    "no view": dict(n_views=0),
    "65 views": dict(n_views=65),
    "negative voxel count": dict(vox=voxels(n=-1)),
    "null geometry": dict(vox=voxels(geom=None)),
    "BF16 densities": dict(vox=voxels(density_dtype=L.LV_BF16)),
    "FP16 SH": dict(vox=voxels(sh_dtype=L.LV_F16)),
    "SH degree 4": dict(vox=voxels(sh_degree=4)),
    "misaligned vertex index": dict(vox=voxels(vidx=ADDR + 4)),
    "tile 12": dict(opts=opts(tile=12)),
    "batch 100": dict(opts=opts(batch=100)),
    "batch 256": dict(opts=opts(batch=256)),
    "negative pixel id base": dict(opts=opts(pixel_id_base=-1)),
    "pixel ids past 2^32 - 1": dict(opts=opts(pixel_id_base=(1 << 32) - 1000)),
    "t_stop 1": dict(opts=opts(t_stop=1.0)),
    "t_stop NaN": dict(opts=opts(t_stop=math.nan)),
    "negative persistent_sms": dict(opts=opts(persistent_sms=-1)),
    "empty view": dict(cams=cams_of((0, 96))),
    "view of 32769 columns": dict(cams=cams_of((32769, 4))),
    "no rgb output": dict(out=fwd_out(rgb=None)),
    "no T output": dict(out=fwd_out(T=None)),
    "null workspace": dict(ws=None),
    "misaligned workspace": dict(ws=ADDR + 16),
    "negative pair capacity": dict(cap=-1),
    "pair capacity above 2^32 - 1": dict(cap=1 << 32),
}


def forward_args(vox="default", cams=None, n_views=1, opts_=None, out=None, ws=ADDR, ws_bytes=1 << 40, cap=1000,
                 **kw):
    o = kw.get("opts", opts_) or opts()
    v = voxels() if isinstance(vox, str) else vox
    return (None if v is None else C.byref(v), cams if cams is not None else cams_of((128, 96)), n_views,
            C.byref(o), C.byref(out or fwd_out()), ws, ws_bytes, cap, None, None)


@pytest.mark.parametrize("case", sorted(FORWARD_CASES))
def test_forward_rejects(lib, case):
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_rasterize_forward, *forward_args(**FORWARD_CASES[case]))


def test_forward_unsupported_and_workspace(lib):
    expect(lib, L.LV_ERR_UNSUPPORTED, lib.lv_rasterize_forward, *forward_args(opts=opts(tile=32, batch=128)))
    expect(lib, L.LV_ERR_WORKSPACE, lib.lv_rasterize_forward, *forward_args(ws_bytes=TINY_WS))


def test_camera_intrinsics_checked(lib):
    for field in ("fx", "fy", "z_near"):
        cams = cams_of((128, 96))
        setattr(cams[0], field, 0.0)
        expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_rasterize_forward, *forward_args(cams=cams))


def test_backward_rejects(lib):
    cams, o = cams_of((128, 96)), opts()
    v = voxels()
    def bwd(fwd, ws=ADDR, ws_bytes=1 << 40, dL=ADDR, dd=ADDR):
        return (C.byref(v), cams, 1, C.byref(o), None if fwd is None else C.byref(fwd), ws, ws_bytes, 1000, dL,
                None, None, dd, ADDR, 0, None, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_rasterize_backward, *bwd(None))
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_rasterize_backward, *bwd(fwd_out(T=None)))
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_rasterize_backward, *bwd(fwd_out(n_contrib=None)))
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_rasterize_backward, *bwd(fwd_out(), dL=None))
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_rasterize_backward, *bwd(fwd_out(), dd=None))
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_rasterize_backward, *bwd(fwd_out(), ws=ADDR + 8))
    expect(lib, L.LV_ERR_WORKSPACE, lib.lv_rasterize_backward, *bwd(fwd_out(), ws_bytes=TINY_WS))
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_sh_backward, C.byref(v), cams, 1, C.byref(o), ADDR, 1 << 40, 1000,
           None, 0, None)
    expect(lib, L.LV_ERR_WORKSPACE, lib.lv_sh_backward, C.byref(v), cams, 1, C.byref(o), ADDR, TINY_WS, 1000,
           ADDR, 0, None)


def test_statistics_calls_reject(lib):
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_reset_stats, -1, None, None, None, None, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_unpack_wmax, None, 10, ADDR, None, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_unpack_wmax, ADDR, -1, ADDR, None, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_check_status, None, None)
    out2 = (C.c_int64 * 2)()
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_workspace_counters, ADDR, 8, out2, None)


def test_workspace_queries_refuse_bad_configurations(lib):
    cams = cams_of((128, 96))
    assert lib.lv_forward_workspace_size(1000, cams, 1, C.byref(opts()), 0) > 0
    assert lib.lv_forward_workspace_size(1000, cams, 0, C.byref(opts()), 0) == 0
    assert lib.lv_forward_workspace_size(1000, cams, 65, C.byref(opts()), 0) == 0
    assert lib.lv_forward_workspace_size(-1, cams, 1, C.byref(opts()), 0) == 0
    assert lib.lv_forward_workspace_size(1000, cams, 1, C.byref(opts(tile=12)), 0) == 0
    assert lib.lv_compact_workspace_size(-1) == 0
    assert lib.lv_vertex_index_workspace_size(-1) == 0
    assert lib.lv_autotune_workspace_size(1000, cams, 0, C.byref(opts()), 1000) == 0
    # the autotuner's scratch holds the largest of the three tile sizes' forward workspaces
    fwd_max = max(lib.lv_forward_workspace_size(1000, cams, 1, C.byref(opts(tile=t)), 1000) for t in (8, 16, 32))
    assert lib.lv_autotune_workspace_size(1000, cams, 1, C.byref(opts()), 1000) > fwd_max


def test_workspace_sizes_grow_with_the_problem(lib):
    cams1, cams2 = cams_of((128, 96)), cams_of((128, 96), (200, 150))
    o = C.byref(opts())
    assert lib.lv_forward_workspace_size(2000, cams1, 1, o, 0) > lib.lv_forward_workspace_size(1000, cams1, 1, o, 0)
    assert lib.lv_forward_workspace_size(1000, cams2, 2, o, 0) > lib.lv_forward_workspace_size(1000, cams1, 1, o, 0)
    assert lib.lv_compact_workspace_size(10 ** 6) > lib.lv_compact_workspace_size(1000)
    assert lib.lv_vertex_index_workspace_size(10 ** 6) > lib.lv_vertex_index_workspace_size(1000)
    w = (C.c_int32 * 2)(128, 200)
    h = (C.c_int32 * 2)(96, 150)
    assert lib.lv_lf_workspace_size(w, h, 2) > lib.lv_lf_workspace_size(w, h, 1) > 0


# ------------------------------------------------------------------ pruning / subdivision / compaction
def prune_params(**kw):
    p = L.lv_prune_params(n_bins=16, q_ppm=50000, ema_alpha=0.1, m_low=0.3, m_high=0.7, cap_ppm=10000,
                          lo_ppm=50000, hi_ppm=950000)
    for k, x in kw.items():
        setattr(p, k, x)
    return p


PRUNE_CASES = {
    "no bin": dict(n_bins=0),
    "q above 1e6 ppm": dict(q_ppm=1000001),
    "negative cap": dict(cap_ppm=-1),
    "hi percentile above 1e6": dict(hi_ppm=1000001),
    "EMA rate 2": dict(ema_alpha=2.0),
    "EMA rate NaN": dict(ema_alpha=math.nan),
    "anneal above 1e6": dict(anneal=1, anneal_ppm=2000000),
    "relax below 0": dict(anneal=1, relax_ppm=-1),
    "running rate 1.5": dict(pct_ema=1.5),
    "negative halo size": dict(halo_small=-1.0),
    "NaN halo weight": dict(halo_w=math.nan),
}


@pytest.mark.parametrize("case", sorted(PRUNE_CASES))
def test_prune_rejects(lib, case):
    p = prune_params(**PRUNE_CASES[case])
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_prune_depth_quantile, 100, ADDR, ADDR, ADDR, ADDR, ADDR, C.byref(p),
           ADDR, ADDR, ADDR, 1 << 40, None, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_prune_bins, 100, ADDR, ADDR, C.byref(p), ADDR, 1 << 40, None)


def test_prune_arrays_and_workspace(lib):
    p = prune_params()
    args = [100, ADDR, ADDR, ADDR, ADDR, ADDR, C.byref(p), ADDR, ADDR, ADDR, 1 << 40, None, None]
    for i in (1, 2, 3, 4, 5, 7):        # w_max, seen, z, ema_m, state, prune_mask
        a = list(args)
        a[i] = None
        expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_prune_depth_quantile, *a)
    a = list(args)
    a[9] = ADDR + 64
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_prune_depth_quantile, *a)
    a = list(args)
    a[10] = TINY_WS
    expect(lib, L.LV_ERR_WORKSPACE, lib.lv_prune_depth_quantile, *a)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_prune_depth_quantile, -1, *args[1:])
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_prune_finish, 100, None, ADDR, ADDR, ADDR, ADDR, C.byref(p), ADDR,
           ADDR, ADDR, 1 << 40, None, None)


def subdiv_params(**kw):
    p = L.lv_subdiv_params(kappa=1.0, beta=0.2, top_ppm=50000, l_max=16, budget=10 ** 6, lo_ppm=50000,
                           hi_ppm=950000)
    for k, x in kw.items():
        setattr(p, k, x)
    return p


def subdivide(lib, vin=None, vout=None, p=None, aux=None, n_aux=0, ws=ADDR, ws_bytes=1 << 40, arrays=ADDR):
    vin = vin or voxels()
    vout = vout or voxels(n=1000)
    p = p or subdiv_params()
    return lib.lv_subdivide_priority(C.byref(vin), arrays, arrays, arrays, arrays, None, C.byref(p), aux, n_aux,
                                     C.byref(vout), arrays, arrays, ws, ws_bytes, None, None)


def test_subdivide_rejects(lib):
    expect(lib, L.LV_ERR_UNSUPPORTED, subdivide, lib, voxels(vidx=ADDR))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, voxels(density_dtype=L.LV_BF16))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, voxels(sh_dtype=L.LV_F16))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, voxels(n=-1))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, voxels(level=None))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, None, voxels(n=1000, density_dtype=L.LV_F16))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, None, voxels(n=-1))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, None, None, subdiv_params(top_ppm=-1))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, None, None, subdiv_params(lo_ppm=2000000))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, None, None, subdiv_params(pct_ema=-0.5))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, None, None, None, None, 17)   # LV_MAX_AUX + 1
    aux = (L.lv_aux_array * 1)(L.lv_aux_array(in_=ADDR, out=ADDR, width=8, elem_bytes=3, fill=0))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, None, None, None, aux, 1)
    aux = (L.lv_aux_array * 1)(L.lv_aux_array(in_=ADDR, out=ADDR, width=0, elem_bytes=4, fill=0))
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, None, None, None, aux, 1)
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, None, None, None, None, 0, ADDR + 128)
    expect(lib, L.LV_ERR_WORKSPACE, subdivide, lib, None, None, None, None, 0, ADDR, TINY_WS)
    expect(lib, L.LV_ERR_INVALID_ARG, subdivide, lib, None, None, None, None, 0, ADDR, 1 << 40, None)


def test_compact_rejects(lib):
    def compact(vin=None, keep=ADDR, n_aux=0, ws=ADDR, ws_bytes=1 << 40, vout="default"):
        vin = vin or voxels()
        vo = voxels(n=1000) if isinstance(vout, str) else vout
        return lib.lv_compact(C.byref(vin), keep, None, n_aux, None if vo is None else C.byref(vo), None, ws,
                              ws_bytes, None, None)
    expect(lib, L.LV_ERR_UNSUPPORTED, compact, voxels(vidx=ADDR))
    expect(lib, L.LV_ERR_INVALID_ARG, compact, None, None)
    expect(lib, L.LV_ERR_INVALID_ARG, compact, None, ADDR, 1)            # one aux array, none given
    expect(lib, L.LV_ERR_INVALID_ARG, compact, None, ADDR, 0, ADDR, 1 << 40, None)
    expect(lib, L.LV_ERR_INVALID_ARG, compact, None, ADDR, 0, ADDR + 32)
    expect(lib, L.LV_ERR_WORKSPACE, compact, None, ADDR, 0, ADDR, TINY_WS)


# ------------------------------------------------------------------ loss, training step, vertices
def lf_params(**kw):
    p = L.lv_lf_params(eps=1e-3, gamma_max=1.0, t0=300.0, t1=600.0, pctl_ppm=990000, edge_out=None)
    for k, x in kw.items():
        setattr(p, k, x)
    return p


def test_lf_loss_rejects(lib):
    w = (C.c_int32 * 1)(128)
    h = (C.c_int32 * 1)(96)
    def loss(p=None, widths=w, heights=h, n_views=1, ws=ADDR, ws_bytes=1 << 40, rgb=ADDR):
        return lib.lv_lf_weighted_loss(rgb, ADDR, widths, heights, n_views, 450.0, C.byref(p or lf_params()),
                                       ADDR, ADDR, ws, ws_bytes, None)
    expect(lib, L.LV_ERR_INVALID_ARG, loss, lf_params(eps=0.0))
    expect(lib, L.LV_ERR_INVALID_ARG, loss, lf_params(t1=300.0))
    expect(lib, L.LV_ERR_INVALID_ARG, loss, lf_params(gamma_max=-1.0))
    expect(lib, L.LV_ERR_INVALID_ARG, loss, lf_params(pctl_ppm=1000001))
    expect(lib, L.LV_ERR_INVALID_ARG, loss, None, (C.c_int32 * 1)(0))
    expect(lib, L.LV_ERR_INVALID_ARG, loss, None, w, h, 0)
    expect(lib, L.LV_ERR_INVALID_ARG, loss, None, w, h, 1, ADDR + 4)
    expect(lib, L.LV_ERR_WORKSPACE, loss, None, w, h, 1, ADDR, TINY_WS)
    expect(lib, L.LV_ERR_INVALID_ARG, loss, None, w, h, 1, ADDR, 1 << 40, None)
    assert lib.lv_lf_workspace_size((C.c_int32 * 1)(0), h, 1) == 0


def test_training_step_rejects(lib):
    ap = L.lv_adam_params(lr_density=1e-2, lr_sh=1e-3, beta1=0.9, beta2=0.999, eps=1e-15, step=1, tv_weight=0.0)
    def adam(n=100, p=ap, dens_dt=L.LV_F32, sh_dt=L.LV_F32, grad=ADDR, ws=ADDR, ws_bytes=1 << 40):
        return lib.lv_adam_voxels(n, ADDR, dens_dt, ADDR, sh_dt, grad, ADDR, ADDR, ADDR, ADDR, ADDR,
                                  None if p is None else C.byref(p), ADDR, ws, ws_bytes, None)
    expect(lib, L.LV_ERR_INVALID_ARG, adam, -1)
    expect(lib, L.LV_ERR_INVALID_ARG, adam, 100, None)
    expect(lib, L.LV_ERR_INVALID_ARG, adam, 100, ap, L.LV_BF16)
    expect(lib, L.LV_ERR_INVALID_ARG, adam, 100, ap, L.LV_F32, L.LV_F16)
    expect(lib, L.LV_ERR_INVALID_ARG, adam, 100, ap, L.LV_F32, L.LV_F32, None)
    expect(lib, L.LV_ERR_INVALID_ARG, adam, 100, ap, L.LV_F32, L.LV_F32, ADDR + 4)
    bad = L.lv_adam_params(lr_density=1e-2, lr_sh=1e-3, beta1=1.5, beta2=0.999, eps=1e-15, step=1)
    expect(lib, L.LV_ERR_INVALID_ARG, adam, 100, bad)
    expect(lib, L.LV_ERR_WORKSPACE, adam, 100, ap, L.LV_F32, L.LV_F32, ADDR, ADDR, TINY_WS)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_adam_array, 10, ADDR, 7, ADDR, ADDR, ADDR, 1.0, C.byref(ap), None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_adam_array, 10, None, L.LV_F32, ADDR, ADDR, ADDR, 1.0, C.byref(ap),
           None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_transmittance_loss, ADDR, -1, 1.0, ADDR, None, 0, ADDR, 1 << 40, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_transmittance_loss, ADDR, 10, 1.0, None, None, 0, ADDR, 1 << 40, None)
    expect(lib, L.LV_ERR_WORKSPACE, lib.lv_transmittance_loss, ADDR, 10, 1.0, ADDR, None, 0, ADDR, 8, None)


def test_vertex_calls_reject(lib):
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_vertex_gather, ADDR, 10, ADDR, L.LV_BF16, ADDR, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_vertex_gather, None, 10, ADDR, L.LV_F32, ADDR, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_vertex_scatter_add, ADDR + 4, 10, ADDR, ADDR, None, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_vertex_scatter_add, ADDR, -1, ADDR, ADDR, None, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_build_vertex_index, ADDR, 10, 0.0, ADDR, ADDR, ADDR, 1 << 40, None,
           None)
    expect(lib, L.LV_ERR_WORKSPACE, lib.lv_build_vertex_index, ADDR, 10, 0.01, ADDR, ADDR, ADDR, TINY_WS, None,
           None)


# ------------------------------------------------------------------ autotuner cache
def test_autotune_reads_its_cache_without_running(lib, tmp_path):
    """A cache hit returns the stored tile, schedule and batch before any launch; the last matching line wins
    and lines with another key, a tile that is not 8/16/32, a batch that is not 32/64/128 (or 128 with tile
    32) or too few fields are skipped; a line without a batch means 32.  Without a device the key's GPU name
    is "gpu"."""
    cams = cams_of((128, 96), (64, 48))
    key = "gpu|100|128x96|64x48|f0"
    path = tmp_path / "tune.txt"
    path.write_text(f"{key} 8 0 64\n"
                    f"{key.replace('|100|', '|101|')} 32 1 32\n"
                    f"{key} 16 1 128\n"
                    f"{key} 12 0 32\n"
                    f"{key} 32 1 128\n"
                    f"{key} 8 0 256\n"
                    f"{key} 32\n")
    best = L.lv_raster_opts()
    ms = (C.c_float * 18)()
    v = voxels(n=100)
    expect_ok = lib.lv_autotune(C.byref(v), cams, 2, C.byref(opts()), 1000, 3, C.byref(best), ms,
                                str(path).encode(), None, 0, None)
    assert expect_ok == L.LV_OK, L.last_error()
    assert best.tile == 16 and best.flags & L.LV_FLAG_PERSISTENT and best.batch == 128
    assert list(ms) == [-1.0] * 18
    path.write_text(f"{key} 32 0\n")                 # the cache format without a batch
    assert lib.lv_autotune(C.byref(v), cams, 2, C.byref(opts()), 1000, 3, C.byref(best), ms, str(path).encode(),
                           None, 0, None) == L.LV_OK
    assert best.tile == 32 and best.batch == 32 and not best.flags & L.LV_FLAG_PERSISTENT
    # flags other than the schedule are part of the key: an exact-segment request misses the cache and, with no
    # workspace, is refused before anything runs
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_autotune, C.byref(v), cams, 2,
           C.byref(opts(flags=L.LV_FLAG_EXACT_SEGMENT)), 1000, 3, C.byref(best), ms, str(path).encode(), None, 0,
           None)


def test_autotune_rejects(lib):
    cams = cams_of((128, 96))
    best = L.lv_raster_opts()
    v = voxels()
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_autotune, C.byref(v), cams, 0, C.byref(opts()), 1000, 3, C.byref(best),
           None, None, ADDR, 1 << 40, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_autotune, C.byref(v), cams, 1, C.byref(opts()), 1000, 0, C.byref(best),
           None, None, ADDR, 1 << 40, None)
    expect(lib, L.LV_ERR_INVALID_ARG, lib.lv_autotune, C.byref(v), cams, 1, C.byref(opts()), 1000, 3, None, None,
           None, ADDR, 1 << 40, None)


def test_rows_scatter_argument_checks():
    arr = (L.lv_rows * 17)()
    assert L.load().lv_rows_scatter(arr, 17, None) == L.LV_ERR_INVALID_ARG
    arr[0].m, arr[0].row_bytes = 5, 0  # a row of no bytes
    arr[0].dst = arr[0].src = ADDR
    assert L.load().lv_rows_scatter(arr, 1, None) == L.LV_ERR_INVALID_ARG
    arr[0].row_bytes, arr[0].src = 4, None  # no source
    assert L.load().lv_rows_scatter(arr, 1, None) == L.LV_ERR_INVALID_ARG
    assert L.load().lv_rows_scatter(arr, 0, None) == L.LV_OK
