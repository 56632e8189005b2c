"""High-level rasterizer API over the C ABI: workspace management, forward,
backward and a torch.autograd.Function.

Everything numeric runs in liblitevoxel.so; this module only allocates
caller-owned device buffers (through torch) and forwards pointers.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import litevoxel as L


class RasterContext:
    """Workspace and outputs for one camera set and a voxel count.

    exact_segment selects the density-model variant in which a sample's
    density is the mean of the trilinear field over the chord; persistent
    runs the composites as resident warps on a work counter.

    The pair capacity (sorted (tile, voxel) pairs) is sized once, with
    headroom, by :meth:`fit_capacity`; a later forward that overflows it
    reports LV_ERR_CAPACITY (checked by :meth:`check`).
    """

    def __init__(self, cams, n_voxels, tile=16, batch=32, t_stop=1e-4, pair_capacity=None, device="cuda",
                 exact_segment=False, persistent=False, persistent_sms=0):
        self.cams = list(cams)
        self.n_views = len(self.cams)
        self.cams_arr = L.make_cameras(self.cams)
        self.opts = L.make_opts(tile, batch, t_stop, exact_segment=exact_segment, persistent=persistent,
                                persistent_sms=persistent_sms)
        self.device = torch.device(device)
        self.n = int(n_voxels)
        self.sizes = [(int(c["width"]), int(c["height"])) for c in self.cams]
        self.n_pix = sum(w * h for w, h in self.sizes)
        self.pair_capacity = int(pair_capacity) if pair_capacity is not None else max(1024, 4 * self.n * self.n_views)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        # forward passes launched so far: the workspace, T and n_contrib belong to the latest one
        self.generation = 0
        self._alloc_outputs()
        self._alloc_workspace()

    # ---------------------------------------------------------------- buffers
    def _alloc_outputs(self):
        d, P, n = self.device, self.n_pix, self.n
        self.rgb = torch.empty((P, 3), dtype=torch.float32, device=d)
        self.depth = torch.empty(P, dtype=torch.float32, device=d)
        self.T = torch.empty(P, dtype=torch.float32, device=d)
        self.n_contrib = torch.empty(P, dtype=torch.int32, device=d)
        self.n_samples = torch.empty(P, dtype=torch.int32, device=d)
        self.wmax_packed = torch.zeros(n, dtype=torch.int64, device=d)
        self.z_min = torch.full((n,), math.inf, dtype=torch.float32, device=d)
        self.delta_min = torch.full((n,), math.inf, dtype=torch.float32, device=d)
        self.seen = torch.zeros(n, dtype=torch.uint8, device=d)

    def _alloc_workspace(self):
        nb = L.lv_forward_workspace_size(self.n, self.cams_arr, self.n_views, self.opts, self.pair_capacity)
        if nb == 0:
            raise ValueError("invalid rasterizer configuration")
        self.workspace = torch.empty(nb, dtype=torch.uint8, device=self.device)

    def set_pair_capacity(self, cap):
        self.pair_capacity = int(cap)
        self.workspace = None
        self._alloc_workspace()

    def reset_stats(self):
        """Zero w_max and reset z_min / delta_min / seen before a new accumulation window."""
        L.lv_reset_stats(self.wmax_packed, self.z_min, self.delta_min, self.seen)

    def fwd_struct(self, stats=True, stats_event=None, composite_event=None, lf=None):
        return L.make_fwd_out(self.rgb, self.T, self.n_contrib, self.depth,
                              self.wmax_packed if stats else None, self.z_min if stats else None,
                              self.delta_min if stats else None, self.seen if stats else None,
                              self.n_samples if stats else None, stats_event, composite_event, lf)

    # ---------------------------------------------------------------- calls
    def forward(self, vox: L.lv_voxels, stats=True, stats_event=None, composite_event=None):
        """Launch the forward pass (asynchronous).  Returns (rgb, depth, T).  stats_event (a
        torch.cuda.Event recorded once before) is recorded when the voxel statistics are final;
        composite_event right before the composite is launched."""
        L.lv_rasterize_forward(vox, self.cams_arr, self.n_views, self.opts,
                               self.fwd_struct(stats, stats_event, composite_event),
                               self.workspace, self.pair_capacity, self.status)
        self.generation += 1
        return self.rgb, self.depth, self.T

    def backward(self, vox: L.lv_voxels, dL_drgb, dL_ddepth=None, dL_dT=None, d_density=None, d_sh=None,
                 accumulate=False, lf=None):
        """dL_drgb = None with lf = (gt, LF workspace, dL output or None[, event]): the backward
        computes the LF-weighted loss's gradient itself (lv_lf_weights first on that workspace,
        lv_lf_loss_finish after for the loss)."""
        if d_density is None:
            d_density = torch.empty((self.n, 8), dtype=torch.float32, device=self.device)
        if d_sh is None:
            d_sh = torch.empty((self.n, 48), dtype=torch.float32, device=self.device)
        L.lv_rasterize_backward(vox, self.cams_arr, self.n_views, self.opts, self.fwd_struct(False, lf=lf),
                                self.workspace, self.pair_capacity,
                                None if dL_drgb is None else dL_drgb.contiguous(),
                                None if dL_ddepth is None else dL_ddepth.contiguous(),
                                None if dL_dT is None else dL_dT.contiguous(), d_density, d_sh, accumulate,
                                self.status)
        return d_density, d_sh

    def counters(self):
        """(pairs emitted by the last forward, visible slots); synchronises."""
        return L.lv_workspace_counters(self.workspace)

    def check(self):
        """Synchronise and raise if a kernel reported an error (e.g. pair capacity)."""
        st = int(self.status.item())
        if st != 0:
            self.status.zero_()
            raise L.LvError(st, "device-side status")

    def fit_capacity(self, vox: L.lv_voxels, headroom=1.25):
        """Run one forward, grow the pair capacity if needed (with headroom) and re-run."""
        self.status.zero_()
        self.forward(vox, stats=False)
        pairs, _ = self.counters()
        need = int(pairs * headroom) + 1024
        if pairs > self.pair_capacity or need > 2 * self.pair_capacity:
            self.set_pair_capacity(max(need, 1024))
            self.status.zero_()
            self.forward(vox, stats=False)
        self.status.zero_()
        return pairs

    def unpack_wmax(self):
        w = torch.empty(self.n, dtype=torch.float32, device=self.device)
        a = torch.empty(self.n, dtype=torch.int64, device=self.device)
        L.lv_unpack_wmax(self.wmax_packed, w, a)
        return w, a


class Scene:
    """Voxel arrays on the device (structure of arrays)."""

    def __init__(self, geom, level, density, sh, sh_degree=3):
        self.geom, self.level, self.density, self.sh, self.sh_degree = geom, level, density, sh, sh_degree

    @staticmethod
    def from_numpy(arrs, device="cuda", density_dtype=torch.float32, sh_dtype=torch.float32, sh_degree=3):
        return Scene(torch.as_tensor(arrs["geom"]).to(device).contiguous(),
                     torch.as_tensor(arrs["level"]).to(device).contiguous(),
                     torch.as_tensor(arrs["density"]).to(device=device, dtype=density_dtype).contiguous(),
                     torch.as_tensor(arrs["sh"]).to(device=device, dtype=sh_dtype).contiguous(), sh_degree)

    @property
    def n(self):
        return int(self.geom.shape[0])

    def voxels(self) -> L.lv_voxels:
        return L.make_voxels(self.geom, self.density, self.sh, self.level, self.sh_degree)


class _RasterFn(torch.autograd.Function):
    """rgb, depth, T = raster(density, sh); the backward re-walks the sorted
    lists back to front (no per-sample storage), using only the context's
    workspace, T and n_contrib.  Those belong to the context's latest forward
    pass, so a backward whose context has run another forward since raises
    instead of returning the other pass's gradients."""

    @staticmethod
    def forward(ctx, density, sh, scene, rctx):
        vox = L.make_voxels(scene.geom, density, sh, scene.level, scene.sh_degree)
        rgb, depth, T = rctx.forward(vox, stats=True)
        ctx.scene, ctx.rctx, ctx.vox_keep = scene, rctx, (density, sh)
        ctx.generation = rctx.generation
        return rgb.clone(), depth.clone(), T.clone()

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_T):
        if ctx.rctx.generation != ctx.generation:
            raise RuntimeError("rasterize: the RasterContext ran another forward pass after this one; its "
                               "workspace no longer holds this pass's sorted lists (use one context per "
                               "pending backward)")
        density, sh = ctx.vox_keep
        vox = L.make_voxels(ctx.scene.geom, density, sh, ctx.scene.level, ctx.scene.sh_degree)
        g_rgb = torch.zeros_like(ctx.rctx.rgb) if g_rgb is None else g_rgb.float().contiguous()
        dd, ds = ctx.rctx.backward(vox, g_rgb, None if g_depth is None else g_depth.float().contiguous(),
                                   None if g_T is None else g_T.float().contiguous())
        return dd.to(density.dtype), ds.to(sh.dtype), None, None


def rasterize(density, sh, scene: Scene, rctx: RasterContext):
    """Differentiable forward: returns (rgb [P,3], depth [P], T [P])."""
    return _RasterFn.apply(density, sh, scene, rctx)


class CapturedStep:
    """A step function captured once into a CUDA graph and replayed.

    ``fn`` must only launch work on the current stream (the library's calls
    and torch tensor ops do) and must have run once before capture, so that
    one-time set-up (kernel attributes) happens outside the capture.
    """

    def __init__(self, fn, warmup=1):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            fn()
        torch.cuda.synchronize()

    def __call__(self):
        self.graph.replay()


def autotune_tile(scene: Scene, cams, tiles=(8, 16, 32), steps=5, cache_path=None, t_stop=1e-4,
                  schedules=(False, True)):
    """Pick the tile size and composite scheduling (one block per tile, or persistent warps on a
    work counter) with the fastest forward + backward for this scene and camera set.

    Each candidate is timed with CUDA events over ``steps`` forward + backward passes after one
    warm-up.  With ``cache_path`` the choice is stored in a JSON file keyed by the GPU name, voxel
    count and view sizes, and reused.  Returns (best_tile, {tile: ms}) where each tile's time is
    that of its faster schedule; ``autotune_tile.last_persistent`` holds the chosen schedule.
    """
    key = "|".join([torch.cuda.get_device_name(), str(scene.n)] +
                   [f"{int(c['width'])}x{int(c['height'])}" for c in cams])
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            autotune_tile.last_persistent = bool(cache[key].get("persistent", False))
            return int(cache[key]["tile"]), {int(k): v for k, v in cache[key]["ms"].items()}
    vox = scene.voxels()
    times, sched = {}, {}
    for ts in tiles:
        for per in schedules:
            ctx = RasterContext(cams, scene.n, tile=ts, t_stop=t_stop, persistent=per)
            ctx.fit_capacity(vox)
            g = torch.full((ctx.n_pix, 3), 1e-3, device=ctx.device)
            dd = torch.empty((scene.n, 8), device=ctx.device)
            ds = torch.empty((scene.n, 48), device=ctx.device)
            ctx.forward(vox)
            ctx.backward(vox, g, d_density=dd, d_sh=ds)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                ctx.forward(vox)
                ctx.backward(vox, g, d_density=dd, d_sh=ds)
            e1.record()
            torch.cuda.synchronize()
            ctx.check()
            ms = e0.elapsed_time(e1) / steps
            if ts not in times or ms < times[ts]:
                times[ts], sched[ts] = ms, per
            del ctx
    best = min(times, key=times.get)
    autotune_tile.last_persistent = sched[best]
    if cache_path:
        cache[key] = {"tile": best, "persistent": sched[best], "ms": times}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, times


autotune_tile.last_persistent = False
