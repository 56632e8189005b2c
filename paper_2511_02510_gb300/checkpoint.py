"""Checkpoint and resume of a training state.

The library keeps no state between calls: everything a run needs to resume
lives in caller-owned arrays -- the voxel structure of arrays (centre and
half-size, level, corner densities, SH), the per-voxel pruning state (EMA m
and hysteresis state s of Sec. IV-C guard i), the optimizer moments refreshed
at each topology change (Sec. IV-D), the running depth percentiles of Eq. 14
and the step count.  ``save`` writes host copies of them with ``torch.save``
(dtypes kept, FP16 corners and BF16 SH included) through a temporary file
that is renamed into place, so a crash mid-write leaves the previous
checkpoint intact; ``load`` checks the shapes and puts the arrays on a device.
"""
from __future__ import annotations

import os

import torch

from .raster import Scene

FORMAT = 1
SCENE_ARRAYS = ("geom", "level", "density", "sh")


def save(path: str, scene: Scene, state: dict | None = None, step: int = 0, meta: dict | None = None) -> None:
    """Write ``scene``, the named ``state`` tensors, the step count and ``meta``
    (plain str / int / float / bool values) to ``path``."""
    n = scene.n
    _check_scene({k: getattr(scene, k) for k in SCENE_ARRAYS}, n)
    blob = {
        "format": FORMAT,
        "n": n,
        "sh_degree": int(scene.sh_degree),
        "step": int(step),
        "scene": {k: getattr(scene, k).detach().to("cpu", copy=True).contiguous() for k in SCENE_ARRAYS},
        "state": {k: v.detach().to("cpu", copy=True).contiguous() for k, v in (state or {}).items()},
        "meta": dict(meta or {}),
    }
    tmp = f"{path}.tmp{os.getpid()}"
    torch.save(blob, tmp)
    os.replace(tmp, path)


def load(path: str, device="cuda"):
    """Read a checkpoint; returns (scene, state, step, meta) with every tensor on ``device``."""
    blob = torch.load(path, map_location="cpu", weights_only=True)
    if blob.get("format") != FORMAT:
        raise ValueError(f"{path}: checkpoint format {blob.get('format')!r}, expected {FORMAT}")
    n = int(blob["n"])
    arrays = blob["scene"]
    _check_scene(arrays, n)
    scene = Scene(*(arrays[k].to(device).contiguous() for k in SCENE_ARRAYS), sh_degree=int(blob["sh_degree"]))
    state = {k: v.to(device).contiguous() for k, v in blob["state"].items()}
    return scene, state, int(blob["step"]), dict(blob["meta"])


def _check_scene(arrays: dict, n: int) -> None:
    want = {"geom": (n, 4), "level": (n,), "density": (n, 8), "sh": (n, 48)}
    for k, shape in want.items():
        if tuple(arrays[k].shape) != shape:
            raise ValueError(f"{k}: shape {tuple(arrays[k].shape)}, expected {shape}")
