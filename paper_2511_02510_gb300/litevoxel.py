"""Python binding of ``liblitevoxel.so`` (the C ABI in include/litevoxel.h).

Argument marshalling only: every function forwards torch CUDA tensors'
device pointers and the current CUDA stream to the library; all arithmetic
runs in the library's CUDA kernels.  There is no CPU fallback: if the
library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblitevoxel.so")

LV_OK, LV_ERR_INVALID_ARG, LV_ERR_WORKSPACE, LV_ERR_CAPACITY, LV_ERR_CUDA, LV_ERR_TIMEOUT, LV_ERR_UNSUPPORTED = range(7)
LV_F32, LV_F16, LV_BF16 = 0, 1, 2
LV_FLAG_SYNC_CHECK = 1
LV_FLAG_EXACT_SEGMENT = 2
LV_FLAG_PERSISTENT = 4
LV_MAX_VIEWS = 64
STATUS_NAMES = {0: "LV_OK", 1: "LV_ERR_INVALID_ARG", 2: "LV_ERR_WORKSPACE", 3: "LV_ERR_CAPACITY", 4: "LV_ERR_CUDA",
                5: "LV_ERR_TIMEOUT", 6: "LV_ERR_UNSUPPORTED"}


class LvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# ------------------------------------------------------------------ structs
class lv_voxels(C.Structure):
    _fields_ = [("n", C.c_int64), ("geom", C.c_void_p), ("level", C.c_void_p), ("density", C.c_void_p),
                ("density_dtype", C.c_int32), ("sh", C.c_void_p), ("sh_dtype", C.c_int32), ("sh_degree", C.c_int32),
                ("vidx", C.c_void_p)]


class lv_camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("w2c", C.c_float * 12), ("z_near", C.c_float)]


class lv_raster_opts(C.Structure):
    _fields_ = [("tile", C.c_int32), ("batch", C.c_int32), ("t_stop", C.c_float),
                ("flags", C.c_uint32), ("persistent_sms", C.c_int32), ("pixel_id_base", C.c_int64)]


class lv_fwd_out(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("T", C.c_void_p), ("n_contrib", C.c_void_p),
                ("wmax_packed", C.c_void_p), ("z_min", C.c_void_p), ("delta_min", C.c_void_p), ("seen", C.c_void_p),
                ("n_samples", C.c_void_p), ("stats_event", C.c_void_p), ("composite_event", C.c_void_p),
                ("lf_gt", C.c_void_p), ("lf_workspace", C.c_void_p), ("lf_ws_bytes", C.c_size_t),
                ("lf_dL", C.c_void_p), ("lf_wait_event", C.c_void_p)]


class lv_prune_params(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("q_ppm", C.c_int32), ("ema_alpha", C.c_float), ("m_low", C.c_float),
                ("m_high", C.c_float), ("cap_ppm", C.c_int32), ("lo_ppm", C.c_int32), ("hi_ppm", C.c_int32),
                ("anneal", C.c_int32), ("anneal_ppm", C.c_int32), ("relax_ppm", C.c_int32),
                ("halo_small", C.c_float), ("halo_w", C.c_float), ("halo_edge", C.c_float),
                ("geom", C.c_void_p), ("delta", C.c_void_p), ("edge", C.c_void_p),
                ("pct_ema", C.c_float), ("pct_state", C.c_void_p)]


class lv_subdiv_params(C.Structure):
    _fields_ = [("kappa", C.c_float), ("beta", C.c_float), ("top_ppm", C.c_int32), ("l_max", C.c_int32),
                ("budget", C.c_int64), ("lo_ppm", C.c_int32), ("hi_ppm", C.c_int32),
                ("pct_ema", C.c_float), ("pct_state", C.c_void_p)]


class lv_rows(C.Structure):
    _fields_ = [("dst", C.c_void_p), ("src", C.c_void_p), ("row_bytes", C.c_int64), ("idx", C.c_void_p),
                ("m", C.c_int64)]


class lv_aux_array(C.Structure):
    _fields_ = [("in_", C.c_void_p), ("out", C.c_void_p), ("width", C.c_int32), ("elem_bytes", C.c_int32),
                ("fill", C.c_uint32)]


class lv_adam_params(C.Structure):
    _fields_ = [("lr_density", C.c_float), ("lr_sh", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("step", C.c_int64), ("tv_weight", C.c_float)]


class lv_lf_params(C.Structure):
    _fields_ = [("eps", C.c_float), ("gamma_max", C.c_float), ("t0", C.c_float), ("t1", C.c_float),
                ("pctl_ppm", C.c_int32), ("edge_out", C.c_void_p)]


# ------------------------------------------------------------------ loading
_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_P, _I64, _I32, _F, _SZ = C.c_void_p, C.c_int64, C.c_int32, C.c_float, C.c_size_t
_PV = C.POINTER(lv_voxels)
_PC = C.POINTER(lv_camera)
_PO = C.POINTER(lv_raster_opts)
_PF = C.POINTER(lv_fwd_out)
SIGNATURES = {
    "lv_forward_workspace_size": (_SZ, [_I64, _PC, C.c_int, _PO, _I64]),
    "lv_rasterize_forward": (C.c_int, [_PV, _PC, C.c_int, _PO, _PF, _P, _SZ, _I64, _P, _P]),
    "lv_workspace_counters": (C.c_int, [_P, _SZ, C.POINTER(C.c_int64), _P]),
    "lv_rasterize_backward": (C.c_int, [_PV, _PC, C.c_int, _PO, _PF, _P, _SZ, _I64, _P, _P, _P, _P, _P, C.c_int, _P,
                                        _P]),
    "lv_sh_backward": (C.c_int, [_PV, _PC, C.c_int, _PO, _P, _SZ, _I64, _P, C.c_int, _P]),
    "lv_unpack_wmax": (C.c_int, [_P, _I64, _P, _P, _P]),
    "lv_gather_edge": (C.c_int, [_P, _I64, _P, _I64, _P, _P]),
    "lv_train_workspace_size": (_SZ, []),
    "lv_adam_array": (C.c_int, [_I64, _P, C.c_int, _P, _P, _P, _F, C.POINTER(lv_adam_params), _P]),
    "lv_vertex_index_workspace_size": (_SZ, [_I64]),
    "lv_build_vertex_index": (C.c_int, [_P, _I64, C.c_double, _P, _P, _P, _SZ, _P, _P]),
    "lv_vertex_gather": (C.c_int, [_P, _I64, _P, C.c_int, _P, _P]),
    "lv_vertex_scatter_add": (C.c_int, [_P, _I64, _P, _P, _P, _P]),
    "lv_transmittance_loss": (C.c_int, [_P, _I64, _F, _P, _P, C.c_int, _P, _SZ, _P]),
    "lv_adam_voxels": (C.c_int, [_I64, _P, C.c_int, _P, C.c_int, _P, _P, _P, _P, _P, _P,
                                 C.POINTER(lv_adam_params), _P, _P, _SZ, _P]),
    "lv_prune_anneal_ppm": (_I32, [C.c_double, C.c_double, C.c_double]),
    "lv_debug_pairs": (C.c_int, [_I64, _PC, C.c_int, _PO, _P, _SZ, _I64, _P, _P, _P, _P]),
    "lv_debug_sort_timeout_workspace_size": (_SZ, []),
    "lv_debug_sort_timeout": (C.c_int, [C.c_int32, _P, _SZ, _P, _P]),
    "lv_render_pixels_f64": (C.c_int, [_PV, _PC, C.c_int, _PO, _P, _SZ, _I64, _P, _I64, _P, _P, _P]),
    "lv_prune_workspace_size": (_SZ, [_I64, C.POINTER(lv_prune_params)]),
    "lv_prune_bins": (C.c_int, [_I64, _P, _P, C.POINTER(lv_prune_params), _P, _SZ, _P]),
    "lv_prune_finish": (C.c_int, [_I64, _P, _P, _P, _P, _P, C.POINTER(lv_prune_params), _P, _P, _P, _SZ, _P,
                                  _P]),
    "lv_prune_depth_quantile": (C.c_int, [_I64, _P, _P, _P, _P, _P, C.POINTER(lv_prune_params), _P, _P, _P, _SZ, _P,
                                          _P]),
    "lv_subdivide_workspace_size": (_SZ, [_I64, C.POINTER(lv_subdiv_params)]),
    "lv_subdivide_priority": (C.c_int, [_PV, _P, _P, _P, _P, _P, C.POINTER(lv_subdiv_params),
                                        C.POINTER(lv_aux_array), C.c_int, _PV, _P, _P, _P, _SZ, _P, _P]),
    "lv_subdivide_select": (C.c_int, [_PV, _P, _P, _P, _P, _P, C.POINTER(lv_subdiv_params), _I64, _P, _P, _P, _SZ,
                                      _P, _P]),
    "lv_subdivide_apply": (C.c_int, [_PV, C.POINTER(lv_subdiv_params), C.POINTER(lv_aux_array), C.c_int, _PV, _P,
                                     _SZ, _P]),
    "lv_rows_scatter": (C.c_int, [_P, C.c_int, _P]),
    "lv_subdivide_apply_inplace": (C.c_int, [_PV, C.c_int64, C.POINTER(lv_subdiv_params), C.POINTER(lv_aux_array),
                                             C.c_int, _P, _SZ, _P]),
    "lv_compact_workspace_size": (_SZ, [_I64]),
    "lv_compact": (C.c_int, [_PV, _P, C.POINTER(lv_aux_array), C.c_int, _PV, _P, _P, _SZ, _P, _P]),
    "lv_check_status": (C.c_int, [_P, _P]),
    "lv_reset_stats": (C.c_int, [_I64, _P, _P, _P, _P, _P]),
    "lv_autotune_workspace_size": (_SZ, [_I64, _PC, C.c_int, _PO, _I64]),
    "lv_autotune": (C.c_int, [_PV, _PC, C.c_int, _PO, _I64, C.c_int, _PO, C.POINTER(C.c_float), C.c_char_p, _P, _SZ,
                              _P]),
    "lv_lf_gamma": (_F, [_F, C.POINTER(lv_lf_params)]),
    "lv_lf_workspace_size": (_SZ, [_P, _P, C.c_int]),
    "lv_lf_weighted_loss": (C.c_int, [_P, _P, _P, _P, C.c_int, _F, C.POINTER(lv_lf_params), _P, _P, _P, _SZ, _P]),
    "lv_lf_weighted_loss_noalloc": (C.c_int, [_P, _P, _P, _P, C.c_int, _F, C.POINTER(lv_lf_params), _P, _P, _P]),
    "lv_lf_weights": (C.c_int, [_P, _P, _P, C.c_int, _F, C.POINTER(lv_lf_params), _P, _SZ, _P]),
    "lv_lf_loss_from_weights": (C.c_int, [_P, _P, _P, _P, C.c_int, _P, _P, _P, _SZ, _P]),
    "lv_lf_loss_finish": (C.c_int, [_P, _P, C.c_int, _P, _P, _SZ, _P]),
    "lv_last_error": (C.c_char_p, []),
    "lv_version": (C.c_int32, []),
    "lv_launch_count": (C.c_int64, []),
}


def load():
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2511_02510_gb300.build.build()")
            lib = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name, None)
                if fn is None:
                    continue          # a missing export raises when it is called
                fn.restype = res
                fn.argtypes = args
            _lib = lib
        return _lib


def last_error() -> str:
    return load().lv_last_error().decode()


def launch_count() -> int:
    return int(load().lv_launch_count())


def _check(status: int, what: str):
    if status != LV_OK:
        raise LvError(status, f"{what}: {last_error()}")


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# ------------------------------------------------------------------ marshalling helpers
_DT = {torch.float32: LV_F32, torch.float16: LV_F16, torch.bfloat16: LV_BF16}


def make_voxels(geom, density, sh, level=None, sh_degree=3, vidx=None) -> lv_voxels:
    """vidx (int32 [n, 8]) selects the shared grid-vertex variant: density is then the vertex array."""
    v = lv_voxels()
    v.vidx = _ptr(vidx)
    v.n = int(geom.shape[0])
    v.geom = _ptr(geom)
    v.level = _ptr(level)
    v.density = _ptr(density)
    v.density_dtype = _DT[density.dtype]
    v.sh = _ptr(sh)
    v.sh_dtype = _DT[sh.dtype]
    v.sh_degree = int(sh_degree)
    return v


def make_cameras(cams) -> C.Array:
    arr = (lv_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].width, arr[i].height = int(c["width"]), int(c["height"])
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = c["fx"], c["fy"], c["cx"], c["cy"]
        for k in range(12):
            arr[i].w2c[k] = float(c["w2c"][k])
        arr[i].z_near = c["z_near"]
    return arr


def make_opts(tile=16, batch=32, t_stop=1e-4, sync_check=False, exact_segment=False,
              persistent=False, persistent_sms=0, pixel_id_base=0) -> lv_raster_opts:
    o = lv_raster_opts()
    o.tile, o.batch, o.t_stop = tile, batch, t_stop
    o.persistent_sms = int(persistent_sms)
    o.pixel_id_base = int(pixel_id_base)
    o.flags = ((LV_FLAG_SYNC_CHECK if sync_check else 0) | (LV_FLAG_EXACT_SEGMENT if exact_segment else 0) |
               (LV_FLAG_PERSISTENT if persistent else 0))
    return o


def make_fwd_out(rgb, T, n_contrib, depth=None, wmax_packed=None, z_min=None, delta_min=None, seen=None,
                 n_samples=None, stats_event=None, composite_event=None, lf=None) -> lv_fwd_out:
    """stats_event: a torch.cuda.Event (recorded once before, so that it exists) that the forward
    records as soon as the per-voxel statistics are final; composite_event: one it records right
    before launching the composite.  lf: (gt, lf workspace, dL or None[, event]) to fuse the
    LF-weighted loss into the backward called with this struct and dL_drgb = None (after
    lv_lf_weights on that workspace, or after the event that follows it on another stream;
    lv_lf_loss_finish writes the loss after the backward)."""
    o = lv_fwd_out()
    o.rgb, o.depth, o.T, o.n_contrib = _ptr(rgb), _ptr(depth), _ptr(T), _ptr(n_contrib)
    o.wmax_packed, o.z_min, o.delta_min, o.seen = _ptr(wmax_packed), _ptr(z_min), _ptr(delta_min), _ptr(seen)
    o.n_samples = _ptr(n_samples)
    o.stats_event = stats_event.cuda_event if stats_event is not None else None
    o.composite_event = composite_event.cuda_event if composite_event is not None else None
    if lf is not None:
        gt, ws, dL = lf[:3]
        o.lf_gt, o.lf_workspace, o.lf_dL = _ptr(gt), _ptr(ws), _ptr(dL)
        o.lf_ws_bytes = ws.numel() * ws.element_size()
        o.lf_wait_event = lf[3].cuda_event if len(lf) > 3 and lf[3] is not None else None
    return o


# ------------------------------------------------------------------ C-ABI calls (same names)
def lv_forward_workspace_size(n, cams_arr, n_views, opts, pair_capacity) -> int:
    return int(load().lv_forward_workspace_size(n, cams_arr, n_views, C.byref(opts), pair_capacity))


def lv_rasterize_forward(vox, cams_arr, n_views, opts, out, workspace, pair_capacity, d_status=None):
    _check(load().lv_rasterize_forward(C.byref(vox), cams_arr, n_views, C.byref(opts), C.byref(out), _ptr(workspace),
                                       workspace.numel() * workspace.element_size(), pair_capacity, _ptr(d_status),
                                       _stream()), "lv_rasterize_forward")


def lv_workspace_counters(workspace):
    out = (C.c_int64 * 2)()
    _check(load().lv_workspace_counters(_ptr(workspace), workspace.numel() * workspace.element_size(), out,
                                        _stream()), "lv_workspace_counters")
    return int(out[0]), int(out[1])


def lv_rasterize_backward(vox, cams_arr, n_views, opts, fwd, workspace, pair_capacity, dL_drgb, dL_ddepth, dL_dT,
                          d_density, d_sh, accumulate=False, d_status=None):
    _check(load().lv_rasterize_backward(C.byref(vox), cams_arr, n_views, C.byref(opts), C.byref(fwd),
                                        _ptr(workspace), workspace.numel() * workspace.element_size(), pair_capacity,
                                        _ptr(dL_drgb), _ptr(dL_ddepth), _ptr(dL_dT), _ptr(d_density), _ptr(d_sh),
                                        int(bool(accumulate)), _ptr(d_status), _stream()), "lv_rasterize_backward")


def lv_sh_backward(vox, cams_arr, n_views, opts, workspace, pair_capacity, d_sh, accumulate=False):
    _check(load().lv_sh_backward(C.byref(vox), cams_arr, n_views, C.byref(opts), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), pair_capacity, _ptr(d_sh),
                                 int(bool(accumulate)), _stream()), "lv_sh_backward")


def lv_unpack_wmax(packed, w_max, argmax=None):
    _check(load().lv_unpack_wmax(_ptr(packed), int(packed.numel()), _ptr(w_max), _ptr(argmax), _stream()),
           "lv_unpack_wmax")


def lv_gather_edge(argmax, edge_map, edge):
    _check(load().lv_gather_edge(_ptr(argmax), int(argmax.numel()), _ptr(edge_map), int(edge_map.numel()),
                                 _ptr(edge), _stream()), "lv_gather_edge")


def lv_adam_array(param, grad, m, v, lr, params):
    _check(load().lv_adam_array(int(param.numel()), _ptr(param), _DT[param.dtype], _ptr(grad), _ptr(m), _ptr(v),
                                float(lr), C.byref(params), _stream()), "lv_adam_array")


def lv_build_vertex_index(geom, unit, vidx, n_vert, d_status=None):
    """Vertex ids [n, 8] (int32 tensor, written) and the vertex count (int64 device tensor)."""
    n = int(geom.shape[0])
    ws = torch.empty(max(int(load().lv_vertex_index_workspace_size(n)), 256), dtype=torch.uint8, device=geom.device)
    _check(load().lv_build_vertex_index(_ptr(geom), n, float(unit), _ptr(vidx), _ptr(n_vert), _ptr(ws),
                                        ws.numel(), _ptr(d_status), _stream()), "lv_build_vertex_index")


def lv_vertex_gather(vidx, vertex_values, corners):
    _check(load().lv_vertex_gather(_ptr(vidx), int(vidx.shape[0]), _ptr(vertex_values), _DT[vertex_values.dtype],
                                   _ptr(corners), _stream()), "lv_vertex_gather")


def lv_vertex_scatter_add(vidx, corners, vertex_sum, vertex_count=None):
    _check(load().lv_vertex_scatter_add(_ptr(vidx), int(vidx.shape[0]), _ptr(corners), _ptr(vertex_sum),
                                        _ptr(vertex_count), _stream()), "lv_vertex_scatter_add")


def lv_train_workspace_size():
    return int(load().lv_train_workspace_size())


def lv_transmittance_loss(T, weight, loss, dL_dT, workspace, accumulate=False):
    _check(load().lv_transmittance_loss(_ptr(T), int(T.numel()), float(weight), _ptr(loss), _ptr(dL_dT),
                                        int(bool(accumulate)), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), _stream()),
           "lv_transmittance_loss")


def lv_adam_voxels(density, sh, d_density, d_sh, m_density, v_density, m_sh, v_sh, params, workspace,
                   tv_loss=None):
    """One Adam step (with the density TV gradient) on density [n, 8] and sh [n, 48], in place."""
    _check(load().lv_adam_voxels(int(density.shape[0]), _ptr(density), _DT[density.dtype], _ptr(sh),
                                 _DT[sh.dtype] if sh is not None else LV_F32, _ptr(d_density), _ptr(d_sh),
                                 _ptr(m_density), _ptr(v_density), _ptr(m_sh), _ptr(v_sh), C.byref(params),
                                 _ptr(tv_loss), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                 _stream()), "lv_adam_voxels")


def lv_prune_anneal_ppm(t, t0, t1):
    return int(load().lv_prune_anneal_ppm(float(t), float(t0), float(t1)))


def lv_debug_sort_timeout(spin_limit, workspace, status):
    """One sort pass whose look-back wait can never end: it must give up and report LV_ERR_TIMEOUT."""
    _check(load().lv_debug_sort_timeout(int(spin_limit), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                        _ptr(status), _stream()), "lv_debug_sort_timeout")


def lv_debug_sort_timeout_workspace_size() -> int:
    return int(load().lv_debug_sort_timeout_workspace_size())


def lv_debug_pairs(n, cams_arr, n_views, opts, workspace, pair_capacity, keys=None, voxel=None, ranges=None):
    _check(load().lv_debug_pairs(n, cams_arr, n_views, C.byref(opts), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), pair_capacity, _ptr(keys), _ptr(voxel),
                                 _ptr(ranges), _stream()), "lv_debug_pairs")


def lv_render_pixels_f64(vox, cams_arr, n_views, opts, workspace, pair_capacity, pixels, rgb, T=None):
    _check(load().lv_render_pixels_f64(C.byref(vox), cams_arr, n_views, C.byref(opts), _ptr(workspace),
                                       workspace.numel() * workspace.element_size(), pair_capacity, _ptr(pixels),
                                       int(pixels.numel()), _ptr(rgb), _ptr(T), _stream()), "lv_render_pixels_f64")


def lv_prune_workspace_size(n, params) -> int:
    return int(load().lv_prune_workspace_size(n, C.byref(params)))


def lv_prune_depth_quantile(w_max, seen, z, ema_m, state, params, prune_mask, n_pruned, workspace, d_status=None):
    _check(load().lv_prune_depth_quantile(int(w_max.numel()), _ptr(w_max), _ptr(seen), _ptr(z), _ptr(ema_m),
                                          _ptr(state), C.byref(params), _ptr(prune_mask), _ptr(n_pruned),
                                          _ptr(workspace), workspace.numel() * workspace.element_size(),
                                          _ptr(d_status), _stream()), "lv_prune_depth_quantile")


def lv_prune_bins(seen, z, params, workspace):
    """First half of lv_prune_depth_quantile: percentiles of z over the seen voxels and depth bins."""
    _check(load().lv_prune_bins(int(z.numel()), _ptr(seen), _ptr(z), C.byref(params), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream()), "lv_prune_bins")


def lv_prune_finish(w_max, seen, z, ema_m, state, params, prune_mask, n_pruned, workspace, d_status=None):
    """Second half: per-bin quantiles of w_max, guards, cap; the workspace lv_prune_bins filled."""
    _check(load().lv_prune_finish(int(w_max.numel()), _ptr(w_max), _ptr(seen), _ptr(z), _ptr(ema_m), _ptr(state),
                                  C.byref(params), _ptr(prune_mask), _ptr(n_pruned), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _ptr(d_status), _stream()),
           "lv_prune_finish")


def lv_subdivide_workspace_size(n, params) -> int:
    return int(load().lv_subdivide_workspace_size(n, C.byref(params)))


def lv_subdivide_priority(vin, delta, z, u, seen, prune_mask, params, aux, vout, selected, n_new, workspace,
                          d_status=None):
    aux_arr = (lv_aux_array * max(1, len(aux)))(*aux)
    _check(load().lv_subdivide_priority(C.byref(vin), _ptr(delta), _ptr(z), _ptr(u), _ptr(seen), _ptr(prune_mask),
                                        C.byref(params), aux_arr, len(aux), C.byref(vout), _ptr(selected),
                                        _ptr(n_new), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                        _ptr(d_status), _stream()), "lv_subdivide_priority")


def lv_subdivide_select(vin, delta, z, u, seen, prune_mask, params, out_capacity, selected, n_new, workspace,
                        d_status=None):
    _check(load().lv_subdivide_select(C.byref(vin), _ptr(delta), _ptr(z), _ptr(u), _ptr(seen), _ptr(prune_mask),
                                      C.byref(params), int(out_capacity), _ptr(selected), _ptr(n_new),
                                      _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(d_status),
                                      _stream()), "lv_subdivide_select")


def lv_subdivide_apply(vin, params, aux, vout, workspace):
    aux_arr = (lv_aux_array * max(1, len(aux)))(*aux)
    _check(load().lv_subdivide_apply(C.byref(vin), C.byref(params), aux_arr, len(aux), C.byref(vout),
                                     _ptr(workspace), workspace.numel() * workspace.element_size(), _stream()),
           "lv_subdivide_apply")


def lv_subdivide_apply_inplace(vox, capacity, params, aux, workspace):
    """The topology change written where the rows are (after lv_subdivide_select with
    out_capacity = capacity); vox's arrays hold `capacity` rows, aux arrays are updated in place."""
    aux_arr = (lv_aux_array * max(1, len(aux)))(*aux)
    _check(load().lv_subdivide_apply_inplace(C.byref(vox), int(capacity), C.byref(params), aux_arr, len(aux),
                                             _ptr(workspace), workspace.numel() * workspace.element_size(), _stream()),
           "lv_subdivide_apply_inplace")


def lv_compact_workspace_size(n) -> int:
    return int(load().lv_compact_workspace_size(int(n)))


def lv_compact(vin, keep, aux, vout, n_new, workspace, d_status=None):
    """Rows with keep != 0, in id order, into vout and every auxiliary array."""
    aux_arr = (lv_aux_array * max(1, len(aux)))(*aux)
    _check(load().lv_compact(C.byref(vin), _ptr(keep), aux_arr, len(aux), C.byref(vout), _ptr(n_new), _ptr(workspace),
                             workspace.numel() * workspace.element_size(), _ptr(d_status), _stream()), "lv_compact")


def lv_autotune_workspace_size(n, cams_arr, n_views, base, pair_capacity) -> int:
    return int(load().lv_autotune_workspace_size(int(n), cams_arr, n_views, C.byref(base), int(pair_capacity)))


def lv_autotune(vox, cams_arr, n_views, base, pair_capacity, reps, workspace, cache_path=None):
    """Time every (tile, schedule, batch) candidate; returns (best lv_raster_opts, [18] ms per candidate at
    6 tile + 3 schedule + batch, -1 = skipped)."""
    best = lv_raster_opts()
    ms = (C.c_float * 18)()
    path = cache_path.encode() if cache_path else None
    _check(load().lv_autotune(C.byref(vox), cams_arr, n_views, C.byref(base), int(pair_capacity), int(reps),
                              C.byref(best), ms, path, _ptr(workspace), workspace.numel() * workspace.element_size(),
                              _stream()), "lv_autotune")
    return best, [float(x) for x in ms]


def lv_reset_stats(wmax_packed, z_min, delta_min, seen):
    """One launch: w_max 0, z_min and delta_min +inf, seen 0."""
    n = next(t.numel() for t in (wmax_packed, z_min, delta_min, seen) if t is not None)
    _check(load().lv_reset_stats(int(n), _ptr(wmax_packed), _ptr(z_min), _ptr(delta_min), _ptr(seen), _stream()),
           "lv_reset_stats")


def lv_check_status(d_status) -> int:
    """Synchronise the current stream and return the device status word as an lv_status code."""
    return int(load().lv_check_status(_ptr(d_status), _stream()))


def lv_lf_gamma(t, params) -> float:
    return float(load().lv_lf_gamma(float(t), C.byref(params)))


def lv_lf_workspace_size(widths, heights) -> int:
    w = (C.c_int32 * len(widths))(*widths)
    h = (C.c_int32 * len(heights))(*heights)
    return int(load().lv_lf_workspace_size(w, h, len(widths)))


def lv_lf_weighted_loss(rgb, gt, widths, heights, t, params, loss, dL_drgb, workspace):
    w = (C.c_int32 * len(widths))(*widths)
    h = (C.c_int32 * len(heights))(*heights)
    _check(load().lv_lf_weighted_loss(_ptr(rgb), _ptr(gt), w, h, len(widths), float(t), C.byref(params), _ptr(loss),
                                      _ptr(dL_drgb), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                      _stream()), "lv_lf_weighted_loss")


def lv_lf_weights(gt, widths, heights, t, params, workspace):
    """Eq. 7-9 weight map of the ground truth into the workspace (first half of lv_lf_weighted_loss)."""
    w = (C.c_int32 * len(widths))(*widths)
    h = (C.c_int32 * len(heights))(*heights)
    _check(load().lv_lf_weights(_ptr(gt), w, h, len(widths), float(t), C.byref(params), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream()), "lv_lf_weights")


def lv_lf_loss_from_weights(rgb, gt, widths, heights, loss, dL_drgb, workspace):
    """Loss and dL/drgb from the weight map lv_lf_weights left in the workspace (second half)."""
    w = (C.c_int32 * len(widths))(*widths)
    h = (C.c_int32 * len(heights))(*heights)
    _check(load().lv_lf_loss_from_weights(_ptr(rgb), _ptr(gt), w, h, len(widths), _ptr(loss), _ptr(dL_drgb),
                                          _ptr(workspace), workspace.numel() * workspace.element_size(), _stream()),
           "lv_lf_loss_from_weights")


def lv_lf_loss_finish(widths, heights, loss, workspace):
    """Per-view losses of a forward that fused the LF loss (make_fwd_out(lf=...)); clears the sums."""
    w = (C.c_int32 * len(widths))(*widths)
    h = (C.c_int32 * len(heights))(*heights)
    _check(load().lv_lf_loss_finish(w, h, len(widths), _ptr(loss), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), _stream()), "lv_lf_loss_finish")


LV_LF_NOALLOC_SCRATCH_BYTES = 16 << 20


def lv_lf_weighted_loss_noalloc(rgb, gt, widths, heights, t, params, loss, dL_drgb):
    """Allocation-free LF loss: the library's fixed scratch array replaces the workspace."""
    w = (C.c_int32 * len(widths))(*widths)
    h = (C.c_int32 * len(heights))(*heights)
    _check(load().lv_lf_weighted_loss_noalloc(_ptr(rgb), _ptr(gt), w, h, len(widths), float(t), C.byref(params),
                                              _ptr(loss), _ptr(dL_drgb), _stream()), "lv_lf_weighted_loss_noalloc")


def lv_rows_scatter(items):
    """items: (dst, src, idx) per array, torch tensors whose first dimension is the row: dst[idx[j]] =
    src[j] (idx an int64 device tensor), or dst[:len(src)] = src when idx is None.  One launch."""
    arr = (lv_rows * max(1, len(items)))()
    for i, (dst, src, idx) in enumerate(items):
        arr[i].dst, arr[i].src = _ptr(dst), _ptr(src)
        arr[i].row_bytes = (src[0].numel() if src.dim() > 1 else 1) * src.element_size()
        arr[i].idx = _ptr(idx) if idx is not None else None
        arr[i].m = src.shape[0]
    _check(load().lv_rows_scatter(arr, len(items), _stream()), "lv_rows_scatter")
