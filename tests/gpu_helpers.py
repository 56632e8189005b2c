"""Shared helpers for the GPU parity tests (CUDA library vs CPU oracle)."""
import numpy as np
import torch

from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300.raster import RasterContext, Scene


def to_scene(sc, density_dtype=torch.float32, sh_dtype=torch.float32, sh_degree=3):
    return Scene.from_numpy(sc, "cuda", density_dtype, sh_dtype, sh_degree)


def dequantized(sc, density_dtype=torch.float32, sh_dtype=torch.float32):
    """The FP32 arrays the kernels actually see after loading reduced-precision storage."""
    out = dict(sc)
    out["density"] = torch.as_tensor(sc["density"]).to(density_dtype).float().numpy()
    out["sh"] = torch.as_tensor(sc["sh"]).to(sh_dtype).float().numpy()
    return out


def gpu_forward(sc, cams, tile=16, batch=32, t_stop=1e-4, density_dtype=torch.float32, sh_dtype=torch.float32,
                sh_degree=3, pair_capacity=None, exact_segment=False):
    scene = to_scene(sc, density_dtype, sh_dtype, sh_degree)
    ctx = RasterContext(cams, scene.n, tile=tile, batch=batch, t_stop=t_stop, pair_capacity=pair_capacity,
                        exact_segment=exact_segment)
    vox = scene.voxels()
    if pair_capacity is None:
        ctx.fit_capacity(vox)
    ctx.reset_stats()
    ctx.forward(vox)
    ctx.check()
    return scene, ctx, vox


def gpu_pairs(ctx, n):
    pairs, _ = ctx.counters()
    m = min(pairs, ctx.pair_capacity)
    keys = torch.zeros(max(m, 1), dtype=torch.int64, device="cuda")
    vox = torch.zeros(max(m, 1), dtype=torch.int32, device="cuda")
    tiles = sum(((w + ctx.opts.tile - 1) // ctx.opts.tile) * ((h + ctx.opts.tile - 1) // ctx.opts.tile)
                for w, h in ctx.sizes)
    rng = torch.zeros(2 * tiles, dtype=torch.int32, device="cuda")
    L.lv_debug_pairs(n, ctx.cams_arr, ctx.n_views, ctx.opts, ctx.workspace, ctx.pair_capacity, keys, vox, rng)
    torch.cuda.synchronize()
    return (keys.cpu().numpy()[:m].view(np.uint64), vox.cpu().numpy()[:m].view(np.uint32),
            rng.cpu().numpy().view(np.uint32).reshape(-1, 2), pairs)


def np_(t):
    return t.detach().cpu().numpy()
