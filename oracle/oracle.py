"""ctypes front end of the CPU oracle (``lv_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.

Every function takes and returns numpy arrays.  FP64 for rendering and the
loss; FP32 for the integer-deciding binning, pruning and subdivision (both
sides of a parity test take those decisions in FP32 with the same operation
order, from the same FP32 inputs).  The functions cite the paper passage they
follow in ``lv_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lv_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblv_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction). Returns the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OraCam(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("w2c", C.c_float * 12), ("z_near", C.c_float)]


def _cams(cams) -> C.Array:
    arr = (OraCam * len(cams))()
    for i, c in enumerate(cams):
        arr[i].width, arr[i].height = int(c["width"]), int(c["height"])
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = c["fx"], c["fy"], c["cx"], c["cy"]
        for k in range(12):
            arr[i].w2c[k] = float(c["w2c"][k])
        arr[i].z_near = c["z_near"]
    return arr


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            P = C.c_void_p
            I64, I32, D, F = C.c_int64, C.c_int, C.c_double, C.c_float
            _lib.ora_pairs.argtypes = [I64, P, I32, P, I32, I64, P, P, P, P, P, P, P]
            _lib.ora_render.argtypes = [I64, P, P, P, I32, I32, P, D, I32, P, P, P, P, P, P, P, P, P, I32]
            _lib.ora_render_backward.argtypes = [I64, P, P, P, I32, I32, P, D, P, P, P, P, P, P, I32]
            _lib.ora_trace_pixel.argtypes = [I64, P, P, P, I32, P, D, I32, I32, I64, P, P, P, P, P, I32]
            _lib.ora_prune.argtypes = [I64, P, P, P, P, P, I32, I64, F, F, F, F, I64, I64, I64, P, P, P, P,
                                       I32, I64, I64, P, P, F, P, F, F, F, F, P]
            _lib.ora_prune_q_bin.argtypes = [I64, I64, I64, I32, I32]
            _lib.ora_prune_q_bin.restype = I64
            _lib.ora_subdivide.argtypes = [I64, P, P, P, P, P, P, P, P, P, F, F, I64, I64, I32, I64, I64, I64,
                                           P, P, P, P, P, P, P, I32, P, P, P, P, P, F, F, P]
            _lib.ora_lf_loss.argtypes = [I32, P, P, P, P, D, D, I64, P, P, P, P]
            _lib.ora_lf_gamma.argtypes = [D, D, D, D]
            _lib.ora_lf_gamma.restype = D
            _lib.ora_sh_basis.argtypes = [P, P]
            _lib.ora_wmax_sets.argtypes = [I64, P, P, P, I32, I32, P, D, I32, P, P, P, P, P, P, P, P, P, P, P]
            _lib.ora_backward_bounds.argtypes = [I64, P, P, P, I32, I32, P, D, P, P, P, P, P, P, I32, I32]
            _lib.ora_fd_margins.argtypes = [I64, P, P, P, I32, I32, P, D, I32, P, P, P]
            _lib.ora_free.argtypes = [P]
            _lib.ora_num_threads.restype = C.c_int
        return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().ora_num_threads())


def tiles_of(cam, ts=16):
    return (cam["width"] + ts - 1) // ts, (cam["height"] + ts - 1) // ts


def sh_basis(direction) -> np.ndarray:
    d = _c(direction, np.float64)
    Y = np.zeros(16, np.float64)
    lib().ora_sh_basis(_p(d), _p(Y))
    return Y


def pairs(scene: dict, cams: list, ts: int = 16, cap: int | None = None) -> dict:
    """FP32 binning: sorted (tile << 32 | depth key, voxel id) pairs, tile ranges, z_min, delta_min, seen."""
    geom = _c(scene["geom"], np.float32)
    n = geom.shape[0]
    tiles = sum(tx * ty for tx, ty in (tiles_of(c, ts) for c in cams))
    if cap is None:
        cap = 0
        np_ = C.c_int64(0)
        z = np.full(n, np.inf, np.float32)
        dl = np.full(n, np.inf, np.float32)
        sn = np.zeros(n, np.uint8)
        rng = np.zeros(2 * tiles, np.uint32)
        lib().ora_pairs(n, _p(geom), len(cams), _cams(cams), ts, 0, None, None, C.byref(np_), _p(rng),
                        _p(z), _p(dl), _p(sn))
        cap = np_.value
    keys = np.zeros(max(cap, 1), np.uint64)
    vals = np.zeros(max(cap, 1), np.uint32)
    z = np.full(n, np.inf, np.float32)
    dl = np.full(n, np.inf, np.float32)
    sn = np.zeros(n, np.uint8)
    rng = np.zeros(2 * tiles, np.uint32)
    np_ = C.c_int64(0)
    rc = lib().ora_pairs(n, _p(geom), len(cams), _cams(cams), ts, cap, _p(keys), _p(vals), C.byref(np_),
                         _p(rng), _p(z), _p(dl), _p(sn))
    if rc != 0:
        raise RuntimeError("pair capacity exceeded")
    m = np_.value
    return {"keys": keys[:m], "vals": vals[:m], "ranges": rng.reshape(-1, 2), "z_min": z, "delta_min": dl,
            "seen": sn, "n_pairs": m}


def _npix(cams):
    return sum(int(c["width"]) * int(c["height"]) for c in cams)


def render(scene: dict, cams: list, t_stop: float = 1e-4, sh_degree: int = 3, brute: bool = False,
           crop=None, segment: bool = False) -> dict:
    """FP64 forward render (Eq. 1-5) of all views; outputs over all views' pixels.

    segment: the exact-segment-integration variant (sample density = mean of
    the trilinear field over the chord) instead of the chord-midpoint value.

    bound_rgb / bound_depth / bound_T: admissible FP32-vs-FP64 difference of
    each pixel from the sensitivity of its samples to FP32 geometry rounding;
    near_stop: pixels whose stop decision such rounding can change.
    """
    geom = _c(scene["geom"], np.float32)
    dens = _c(scene["density"], np.float32)
    sh = _c(scene["sh"], np.float32)
    n = geom.shape[0]
    P = _npix(cams)
    rgb = np.zeros((P, 3), np.float64)
    depth = np.zeros(P, np.float64)
    T = np.ones(P, np.float64)
    nh = np.zeros(P, np.int32)
    ns = np.zeros(P, np.uint8)
    wm = np.zeros(n, np.float64)
    wa = np.full(n, -1, np.int64)
    bnd = np.zeros((P, 3), np.float64)
    cr = None if crop is None else _c(np.asarray(crop).reshape(-1, 4), np.int32)
    lib().ora_render(n, _p(geom), _p(dens), _p(sh), sh_degree, len(cams), _cams(cams), t_stop, int(brute),
                     _p(cr), _p(rgb), _p(depth), _p(T), _p(nh), _p(ns), _p(wm), _p(wa), _p(bnd), int(segment))
    return {"rgb": rgb, "depth": depth, "T": T, "n_hit": nh, "near_stop": ns, "w_max": wm, "w_arg": wa,
            "bound_rgb": bnd[:, 0], "bound_depth": bnd[:, 1], "bound_T": bnd[:, 2]}


def render_backward(scene: dict, cams: list, dL_drgb, dL_ddepth=None, dL_dT=None, t_stop: float = 1e-4,
                    sh_degree: int = 3, crop=None, segment: bool = False) -> dict:
    """FP64 gradients of sum(g_C . rgb + g_D depth + g_T T) w.r.t. corner densities and SH."""
    geom = _c(scene["geom"], np.float32)
    dens = _c(scene["density"], np.float32)
    sh = _c(scene["sh"], np.float32)
    n = geom.shape[0]
    gC = _c(dL_drgb, np.float64)
    gD = None if dL_ddepth is None else _c(dL_ddepth, np.float64)
    gT = None if dL_dT is None else _c(dL_dT, np.float64)
    dd = np.zeros((n, 8), np.float64)
    ds = np.zeros((n, 48), np.float64)
    cr = None if crop is None else _c(np.asarray(crop).reshape(-1, 4), np.int32)
    lib().ora_render_backward(n, _p(geom), _p(dens), _p(sh), sh_degree, len(cams), _cams(cams), t_stop, _p(cr),
                              _p(gC), _p(gD), _p(gT), _p(dd), _p(ds), int(segment))
    return {"d_density": dd, "d_sh": ds}


def trace_pixel(scene: dict, cam: dict, x: int, y: int, t_stop: float = 1e-4, sh_degree: int = 3,
                max_out: int = 4096, segment: bool = False) -> dict:
    geom = _c(scene["geom"], np.float32)
    dens = _c(scene["density"], np.float32)
    sh = _c(scene["sh"], np.float32)
    n = geom.shape[0]
    ids = np.zeros(max_out, np.uint32)
    w = np.zeros(max_out, np.float64)
    Ta = np.zeros(max_out, np.float64)
    ll = np.zeros(max_out, np.float64)
    k = C.c_int64(0)
    lib().ora_trace_pixel(n, _p(geom), _p(dens), _p(sh), sh_degree, _cams([cam]), t_stop, x, y, max_out,
                          _p(ids), _p(w), _p(Ta), _p(ll), C.byref(k), int(segment))
    m = min(k.value, max_out)
    return {"ids": ids[:m], "w": w[:m], "T_after": Ta[:m], "l": ll[:m], "n": k.value}


def wmax_sets(scene: dict, cams: list, t_stop: float = 1e-4, sh_degree: int = 3, segment: bool = False) -> dict:
    """w_max (Eq. 5) with the FP32 ambiguity of its argmax, for the parity test.

    Per voxel: w1 / a1 / e1 (FP64 maximum weight, its global pixel id or -1, the
    FP32 error bound of that weight), w2 / e2 (largest weight on any other ray,
    -1 if none), n_certain (samples that any FP32 pass must hit).  The near-max
    set: every (voxel, pixel) sample or near miss whose weight can reach
    w1 - e1, as arrays sorted by (voxel, pixel): set_v, set_pix, set_w, set_e.
    """
    geom = _c(scene["geom"], np.float32)
    dens = _c(scene["density"], np.float32)
    sh = _c(scene["sh"], np.float32)
    n = geom.shape[0]
    w1 = np.zeros(n, np.float64)
    a1 = np.full(n, -1, np.int64)
    e1 = np.zeros(n, np.float64)
    w2 = np.zeros(n, np.float64)
    e2 = np.zeros(n, np.float64)
    nc = np.zeros(n, np.int32)
    ns = C.c_int64(0)
    pv, pp, pw, pe = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
    lib().ora_wmax_sets(n, _p(geom), _p(dens), _p(sh), sh_degree, len(cams), _cams(cams), t_stop, int(segment),
                        _p(w1), _p(a1), _p(e1), _p(w2), _p(e2), _p(nc), C.byref(ns), C.byref(pv), C.byref(pp),
                        C.byref(pw), C.byref(pe))
    m = ns.value

    def take(ptr, ctype, dtype):
        out = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ctype)), shape=(max(m, 1),))[:m].astype(dtype, copy=True)
        lib().ora_free(ptr)
        return out

    sv = take(pv, C.c_int64, np.int64)
    sp = take(pp, C.c_int64, np.int64)
    sw = take(pw, C.c_double, np.float64)
    se = take(pe, C.c_double, np.float64)
    order = np.lexsort((sp, sv))
    return {"w1": w1, "a1": a1, "e1": e1, "w2": w2, "e2": e2, "n_certain": nc, "set_v": sv[order],
            "set_pix": sp[order], "set_w": sw[order], "set_e": se[order]}


def backward_bounds(scene: dict, cams: list, dL_drgb, dL_ddepth=None, dL_dT=None, t_stop: float = 1e-4,
                    sh_degree: int = 3, crop=None, segment: bool = False) -> dict:
    """Absolute FP32 error floors of render_backward's gradients (same arguments):
    e_density [n, 8] and e_sh [n, 48]; an FP32 evaluation g of a gradient whose
    FP64 value is ref stays within |g - ref| <= e under the error model of
    lv_oracle.c (geometry rounding, arithmetic, atomic summation order).
    a_density / a_sh: the same bound without the geometric terms (exact chords
    and hit decisions): arithmetic and summation order only."""
    geom = _c(scene["geom"], np.float32)
    dens = _c(scene["density"], np.float32)
    sh = _c(scene["sh"], np.float32)
    n = geom.shape[0]
    gC = _c(dL_drgb, np.float64)
    gD = None if dL_ddepth is None else _c(dL_ddepth, np.float64)
    gT = None if dL_dT is None else _c(dL_dT, np.float64)
    ed = np.zeros((n, 8), np.float64)
    es = np.zeros((n, 48), np.float64)
    cr = None if crop is None else _c(np.asarray(crop).reshape(-1, 4), np.int32)
    ad = np.zeros((n, 8), np.float64)
    as_ = np.zeros((n, 48), np.float64)
    for e_d, e_s, arith in ((ed, es, 0), (ad, as_, 1)):
        lib().ora_backward_bounds(n, _p(geom), _p(dens), _p(sh), sh_degree, len(cams), _cams(cams), t_stop, _p(cr),
                                  _p(gC), _p(gD), _p(gT), _p(e_d), _p(e_s), int(segment), arith)
    return {"e_density": ed, "e_sh": es, "a_density": ad, "a_sh": as_}


def fd_margins(scene: dict, cams: list, t_stop: float = 1e-4, sh_degree: int = 3, segment: bool = False) -> dict:
    """Kink margins of the render for finite differences: per voxel the smallest
    |sigma_raw| of its samples (m_sigma), the smallest corner step that can move a
    stop decision of a ray through it (m_stop), and per channel the smallest
    |pre-clamp colour| over the views that sample it (m_color [n, 3]); inf if
    never sampled."""
    geom = _c(scene["geom"], np.float32)
    dens = _c(scene["density"], np.float32)
    sh = _c(scene["sh"], np.float32)
    n = geom.shape[0]
    ms = np.zeros(n, np.float64)
    mt = np.zeros(n, np.float64)
    mc = np.zeros((n, 3), np.float64)
    lib().ora_fd_margins(n, _p(geom), _p(dens), _p(sh), sh_degree, len(cams), _cams(cams), t_stop, int(segment),
                         _p(ms), _p(mt), _p(mc))
    return {"m_sigma": ms, "m_stop": mt, "m_color": mc}


def prune(w_max, seen, z, m, s, n_bins=16, q_ppm=50000, ema_alpha=0.1, m_low=0.3, m_high=0.7, cap_ppm=10000,
          lo_ppm=50000, hi_ppm=950000, anneal_ppm=None, relax_ppm=0, geom=None, delta=None, halo_small=0.0,
          edge=None, halo_w=0.0, halo_edge=0.0, pct_ema=0.0, pct_state=None) -> dict:
    """Depth-quantile pruning (Eq. 11-12, guards i-iii). m, s are returned updated (copies).

    anneal_ppm: the q_b schedule value a(t) in ppm (None: q_b = q in every bin);
    relax_ppm: near/far relaxation; geom/delta/halo_small and edge/halo_w/halo_edge:
    keep-halo tests (guard ii); pct_ema/pct_state: running percentiles (state is a
    float32[2] updated in place, NaN = uninitialised)."""
    w_max = _c(w_max, np.float32)
    seen = _c(seen, np.uint8)
    z = _c(z, np.float32)
    m = _c(m, np.float32).copy()
    s = _c(s, np.uint8).copy()
    n = w_max.shape[0]
    mask = np.zeros(n, np.uint8)
    tau = np.zeros(n_bins, np.float32)
    pct = np.zeros(2, np.float32)
    npr = C.c_int64(0)
    a = np.float32(ema_alpha)
    oma = np.float32(np.float32(1.0) - a)
    r = np.float32(pct_ema)
    omr = np.float32(np.float32(1.0) - r)
    g = None if geom is None else _c(geom, np.float32)
    d = None if delta is None else _c(delta, np.float32)
    e = None if edge is None else _c(edge, np.float32)
    if pct_state is not None:
        assert pct_state.dtype == np.float32 and pct_state.flags.c_contiguous and pct_state.size == 2
    lib().ora_prune(n, _p(w_max), _p(seen), _p(z), _p(m), _p(s), n_bins, q_ppm, float(a), float(oma),
                    float(np.float32(m_low)), float(np.float32(m_high)), cap_ppm, lo_ppm, hi_ppm, _p(mask),
                    C.byref(npr), _p(tau), _p(pct), 0 if anneal_ppm is None else 1,
                    0 if anneal_ppm is None else int(anneal_ppm), int(relax_ppm), _p(g), _p(d),
                    float(np.float32(halo_small)), _p(e), float(np.float32(halo_w)), float(np.float32(halo_edge)),
                    float(r), float(omr), _p(pct_state))
    return {"mask": mask, "n_pruned": npr.value, "m": m, "s": s, "tau": tau, "p_lo": pct[0], "p_hi": pct[1]}


def prune_q_bin(q_ppm, anneal_ppm, relax_ppm, b, n_bins) -> int:
    """The annealed, near/far-relaxed per-bin quantile q_b in ppm."""
    return int(lib().ora_prune_q_bin(int(q_ppm), int(anneal_ppm), int(relax_ppm), int(b), int(n_bins)))


def anneal_ppm(t, t0, t1) -> int:
    """a(t) = clip((t - t0) / (t1 - t0), 0, 1) in ppm (floor), 1e6 when t1 <= t0."""
    if t1 <= t0:
        return 1000000
    x = (float(t) - float(t0)) / (float(t1) - float(t0))
    return int(math.floor(1e6 * min(max(x, 0.0), 1.0)))


def subdivide(scene: dict, delta, z, u, seen, prune_mask=None, kappa=1.0, beta=0.2, top_ppm=50000,
              budget=1 << 62, l_max=16, lo_ppm=50000, hi_ppm=950000, aux=None, pct_ema=0.0,
              pct_state=None) -> dict:
    """Priority-driven subdivision (Eq. 13-16, budgeted top-k, child init).

    aux: list of (array [n, width] or [n], fill_value) copied for survivors and
    filled for children (optimizer moments: fill 0; EMA m: fill 1; state s: fill 1).
    """
    geom = _c(scene["geom"], np.float32)
    level = _c(scene["level"], np.uint8)
    dens = _c(scene["density"], np.float32)
    sh = _c(scene["sh"], np.float32)
    n = geom.shape[0]
    delta = _c(delta, np.float32)
    z = _c(z, np.float32)
    u = _c(u, np.float32)
    seen = _c(seen, np.uint8)
    pm = None if prune_mask is None else _c(prune_mask, np.uint8)
    alive = n if pm is None else int(n - pm.astype(np.int64).sum())
    k_max = min(top_ppm * alive // 1000000, (budget - alive) // 7 if budget > alive else 0)
    cap = alive + 7 * max(0, k_max)
    out = {"geom": np.zeros((cap, 4), np.float32), "level": np.zeros(cap, np.uint8),
           "density": np.zeros((cap, 8), np.float32), "sh": np.zeros((cap, 48), np.float32)}
    aux = aux or []
    aux_in, aux_out, widths, nbytes, fills, keep = [], [], [], [], [], []
    for arr, fill in aux:
        a = np.ascontiguousarray(arr)
        w = 1 if a.ndim == 1 else a.shape[1]
        o = np.zeros((cap,) + a.shape[1:], a.dtype)
        keep.append((a, o))
        aux_in.append(a.ctypes.data)
        aux_out.append(o.ctypes.data)
        widths.append(w)
        nbytes.append(a.dtype.itemsize)
        fills.append(int(np.array([fill], a.dtype).view({1: np.uint8, 2: np.uint16, 4: np.uint32}[a.dtype.itemsize])[0]))
    na = len(aux)
    ain = (C.c_void_p * max(na, 1))(*aux_in)
    aout = (C.c_void_p * max(na, 1))(*aux_out)
    aw = (C.c_int32 * max(na, 1))(*widths)
    ab = (C.c_int32 * max(na, 1))(*nbytes)
    af = (C.c_uint32 * max(na, 1))(*fills)
    sel = np.zeros(n, np.uint8)
    nn = C.c_int64(0)
    kk = C.c_int64(0)
    rc = lib().ora_subdivide(n, _p(geom), _p(level), _p(dens), _p(sh), _p(delta), _p(z), _p(u), _p(seen), _p(pm),
                             float(np.float32(kappa)), float(np.float32(beta)), top_ppm, budget, l_max, lo_ppm,
                             hi_ppm, cap, _p(out["geom"]), _p(out["level"]), _p(out["density"]), _p(out["sh"]),
                             _p(sel), C.byref(nn), C.byref(kk), na, ain, aout, aw, ab, af,
                             float(np.float32(pct_ema)), float(np.float32(np.float32(1.0) - np.float32(pct_ema))),
                             _p(pct_state))
    if rc != 0:
        raise RuntimeError("subdivide capacity")
    m = nn.value
    res = {k: v[:m] for k, v in out.items()}
    res["selected"] = sel
    res["n_new"] = m
    res["k"] = kk.value
    res["aux"] = [o[:m] for (_, o) in keep]
    return res


def compact(scene: dict, keep, aux=None) -> dict:
    """Removal of the voxels a step prunes (Sec. IV-C) without a split: the
    rows with keep != 0, in id order, of the voxel arrays and of every
    auxiliary array (optimizer moments, EMA state) -- the survivors part of
    the topology change that subdivide() writes."""
    k = np.asarray(keep).astype(bool)
    res = {name: np.ascontiguousarray(np.asarray(scene[name])[k]) for name in ("geom", "level", "density", "sh")}
    res["aux"] = [np.ascontiguousarray(np.asarray(a)[k]) for a in (aux or [])]
    res["n_new"] = int(k.sum())
    return res


def lf_gamma(t, t0, t1, gamma_max) -> float:
    return float(lib().ora_lf_gamma(float(t), float(t0), float(t1), float(gamma_max)))


def lf_loss(rgb, gt, sizes, gamma, eps=1e-3, pctl_ppm=990000) -> dict:
    """LF-weighted loss (Eq. 7-10, 18) per view; sizes = [(W, H), ...]."""
    rgb = _c(rgb, np.float64).reshape(-1, 3)
    gt = _c(gt, np.float64).reshape(-1, 3)
    nv = len(sizes)
    W = np.array([s[0] for s in sizes], np.int32)
    H = np.array([s[1] for s in sizes], np.int32)
    P = int((W.astype(np.int64) * H).sum())
    loss = np.zeros(nv, np.float64)
    g = np.zeros((P, 3), np.float64)
    s = np.zeros(P, np.float64)
    w = np.zeros(P, np.float64)
    lib().ora_lf_loss(nv, _p(W), _p(H), _p(rgb), _p(gt), float(gamma), float(eps), int(pctl_ppm), _p(loss), _p(g),
                      _p(s), _p(w))
    return {"loss": loss, "dL_drgb": g, "s": s, "w_tilde": w}
