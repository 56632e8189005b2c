"""Seeded synthetic inputs: sparse-voxel octrees, pinhole cameras and target images.

This module only *generates data*.  It holds none of the rasterizer's arithmetic
(projection, compositing, adaptation, loss): both the CUDA library and the CPU
oracle consume what it produces, and neither depends on anything else here.

The scenes stand in for the paper's Mip-NeRF 360 and Tanks & Temples captures
(Sec. V), which are not available: an analytic signed-distance field (three
spheres and a ground plane, plus an inward-facing background shell for the
360-degree scenes) is voxelised into a leaves-only octree whose cells are
refined near the surface (Sec. III, "Sparse Voxel/Octree Indexing").  Each voxel
carries 8 corner densities ``10*sigmoid(-SDF/0.05) + N(0, 0.1)`` and degree-3
SH colour (DC ~ U(0,1), higher bands ~ N(0, 0.05)).

Layouts (all little-endian, C-contiguous numpy arrays):
  geom    float32 [N, 4]   center x, y, z and half-size h
  level   uint8   [N]      octree depth below the root cube (edge = root / 2**level)
  density float32 [N, 8]   corner i at (x +- h, y +- h, z +- h), bit0 = x, bit1 = y, bit2 = z
  sh      float32 [N, 48]  [coefficient 0..15][r, g, b]
Cameras are dicts with width, height, fx, fy, cx, cy, w2c (3x4 row-major
[R | t], x_cam = R x_world + t, OpenCV axes: x right, y down, z forward) and z_near.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "SceneSpec", "make_scene", "scene_tiny", "scene_360", "scene_tt", "scene_stress",
    "look_at_camera", "orbit_camera", "uneven_views", "random_image", "smooth_image",
    "constant_voxel_scene",
]


@dataclass
class SceneSpec:
    """Recipe for one synthetic octree scene."""
    seed: int = 0
    root_min: tuple = (0.0, 0.0, 0.0)
    root_edge: float = 1.0
    l_min: int = 4
    l_max_fg: int = 6
    l_max_bg: int = 6
    band: float = 0.5          # finest-level cells are kept when |SDF(center)| < band * edge
    halo: float = 1.0          # coarse leaves are kept when |SDF| < (0.87 + halo) * edge
    fg_center: tuple = (0.5, 0.5, 0.5)
    fg_scale: float = 1.0      # unit-cube foreground is mapped to fg_center + fg_scale * (p - 0.5)
    fg_box_half: float = 0.5   # foreground clipped to this half-extent around fg_center (unit-cube units)
    shell: tuple | None = None  # (r_in, r_out) background shell around fg_center, or None
    fine_near_spheres: float | None = None  # if set, only cells this close (unit-cube units) to a
                                            # sphere surface may reach l_max_fg; others stop at l_max_bg
    sigmoid_scale: float = 0.05
    density_peak: float = 10.0
    density_noise: float = 0.1
    sh_noise: float = 0.05


def _shapes(seed: int):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0.25, 0.75, size=(3, 3))
    radii = rng.uniform(0.08, 0.18, size=3)
    return centers, radii


def _sdf_factory(spec: SceneSpec):
    centers, radii = _shapes(spec.seed)
    fc = np.asarray(spec.fg_center, dtype=np.float64)
    s = float(spec.fg_scale)

    def sphere_dist(p: np.ndarray) -> np.ndarray:
        q = (p - fc) / s + 0.5
        d = np.full(q.shape[:-1], np.inf)
        for c, r in zip(centers, radii):
            d = np.minimum(d, np.abs(np.linalg.norm(q - c, axis=-1) - r))
        return d

    def sdf(p: np.ndarray) -> np.ndarray:
        # foreground in unit-cube coordinates
        q = (p - fc) / s + 0.5
        d = q[..., 1] - 0.15                       # ground plane y = 0.15 (solid below)
        for c, r in zip(centers, radii):
            d = np.minimum(d, np.linalg.norm(q - c, axis=-1) - r)
        box = np.max(np.abs(q - 0.5), axis=-1) - spec.fg_box_half
        d = np.maximum(d, box) * s                 # clip to the foreground box, back to world units
        if spec.shell is not None:
            r = np.linalg.norm(p - fc, axis=-1)
            r_in, _ = spec.shell
            d = np.minimum(d, r_in - r)           # solid outside r_in (seen from inside)
        return d

    sdf.sphere_dist = sphere_dist
    return sdf


def _build_octree(spec: SceneSpec, sdf):
    """Leaves-only octree: refine cells near the surface, keep a coarse halo."""
    rmin = np.asarray(spec.root_min, dtype=np.float64)
    fc = np.asarray(spec.fg_center, dtype=np.float64)
    n0 = 1 << spec.l_min
    g = np.arange(n0, dtype=np.int64)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    leaves_ijk, leaves_lvl = [], []
    level = spec.l_min
    fg_reach = spec.fg_scale * (spec.fg_box_half + 0.1)
    while cells.shape[0]:
        edge = spec.root_edge / (1 << level)
        centers = rmin + (cells + 0.5) * edge
        d = np.abs(sdf(centers))
        in_fg = np.max(np.abs(centers - fc), axis=-1) < fg_reach
        if spec.fine_near_spheres is not None:
            in_fg &= sdf.sphere_dist(centers) < spec.fine_near_spheres
        cap = np.where(in_fg, spec.l_max_fg, spec.l_max_bg)
        straddle = d < 0.87 * edge                  # the cell may contain the surface
        if spec.shell is not None:                  # nothing beyond the outer shell radius
            straddle &= np.linalg.norm(centers - fc, axis=-1) < spec.shell[1]
        refine = straddle & (level < cap)
        keep = ((level >= cap) & (d < spec.band * edge)) | \
               ((level < cap) & (~straddle) & (d < (0.87 + spec.halo) * edge))
        if spec.shell is not None:
            keep &= np.linalg.norm(centers - fc, axis=-1) < spec.shell[1]
        leaves_ijk.append(cells[keep])
        leaves_lvl.append(np.full(int(keep.sum()), level, dtype=np.uint8))
        par = cells[refine]
        if par.shape[0] == 0:
            break
        offs = np.array([[(i >> 0) & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)], dtype=np.int64)
        cells = (2 * par[:, None, :] + offs[None, :, :]).reshape(-1, 3)
        level += 1
    ijk = np.concatenate(leaves_ijk) if leaves_ijk else np.zeros((0, 3), np.int64)
    lvl = np.concatenate(leaves_lvl) if leaves_lvl else np.zeros((0,), np.uint8)
    edge = spec.root_edge / (2.0 ** lvl.astype(np.float64))
    centers = rmin + (ijk + 0.5) * edge[:, None]
    return centers, edge * 0.5, lvl


def make_scene(spec: SceneSpec, chunk: int = 1 << 20) -> dict:
    """Generate the voxel arrays for ``spec`` (deterministic in ``spec.seed``)."""
    sdf = _sdf_factory(spec)
    centers, half, lvl = _build_octree(spec, sdf)
    n = centers.shape[0]
    rng = np.random.default_rng(spec.seed + 1000)
    geom = np.empty((n, 4), np.float32)
    geom[:, :3] = centers
    geom[:, 3] = half
    dens = np.empty((n, 8), np.float32)
    offs = np.array([[(i & 1) * 2 - 1, ((i >> 1) & 1) * 2 - 1, ((i >> 2) & 1) * 2 - 1] for i in range(8)],
                    dtype=np.float64)
    for s0 in range(0, n, chunk):
        s1 = min(n, s0 + chunk)
        c = geom[s0:s1, :3].astype(np.float64)
        h = geom[s0:s1, 3].astype(np.float64)
        pts = c[:, None, :] + offs[None, :, :] * h[:, None, None]
        d = sdf(pts)
        val = spec.density_peak / (1.0 + np.exp(np.clip(d / spec.sigmoid_scale, -60, 60)))
        val += rng.normal(0.0, spec.density_noise, size=val.shape)
        dens[s0:s1] = val.astype(np.float32)
    sh = np.empty((n, 48), np.float32)
    sh[:, 0:3] = rng.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)
    sh[:, 3:] = rng.normal(0.0, spec.sh_noise, size=(n, 45)).astype(np.float32)
    return {"geom": geom, "level": lvl.astype(np.uint8), "density": dens, "sh": sh}


def scene_tiny(seed: int = 0) -> dict:
    """~4k voxels in the unit cube, levels 4-6 (spheres + plane)."""
    spec = SceneSpec(seed=seed, root_min=(0, 0, 0), root_edge=1.0, l_min=4, l_max_fg=6, l_max_bg=5,
                     band=0.4, halo=0.2, fg_center=(0.5, 0.5, 0.5), fg_scale=1.0, fg_box_half=0.5,
                     fine_near_spheres=0.03)
    return make_scene(spec)


def _spec_360(seed: int, band: float, halo: float) -> SceneSpec:
    return SceneSpec(seed=seed, root_min=(-16, -16, -16), root_edge=32.0, l_min=6, l_max_fg=12, l_max_bg=8,
                     band=band, halo=halo, fg_center=(0.0, 0.0, 0.0), fg_scale=2.5, fg_box_half=0.5,
                     shell=(12.0, 16.0))


def _opaque_peak(spec: SceneSpec, tau_finest: float = 2.5) -> float:
    """Peak density giving optical depth ``tau_finest`` across one finest-level voxel."""
    return tau_finest / (spec.root_edge / (1 << spec.l_max_fg))


def scene_360(seed: int = 0, band: float = 2.0, halo: float = 1.0, opaque: bool = True) -> dict:
    """Mip-NeRF-360-shaped scene: ~2M voxels, levels 6-12, coarse background shell r in [12, 16].

    opaque=True scales the peak corner density so that a finest-level voxel
    inside a solid has optical depth 2.5 (surfaces stop rays within a few
    voxels, as in a trained scene); opaque=False keeps the peak of 10 per unit
    length of the unit-cube recipe (semi-transparent objects).
    """
    spec = _spec_360(seed, band, halo)
    if opaque:
        spec.density_peak = _opaque_peak(spec)
    return make_scene(spec)


def scene_tt(seed: int = 0, band: float = 1.5, halo: float = 0.85, opaque: bool = True, clean: bool = False) -> dict:
    """Tanks-and-Temples-shaped scene: ~6M voxels, levels 6-13, wider foreground extent.

    clean=True leaves the N(0, 0.1) noise out of the corner densities (the same
    random draws are still taken, so the SH coefficients are those of the noisy
    scene): the noise-free scene whose render is the PSNR target."""
    spec = SceneSpec(seed=seed, root_min=(-16, -16, -16), root_edge=32.0, l_min=6, l_max_fg=13, l_max_bg=8,
                     band=band, halo=halo, fg_center=(0.0, 0.0, 0.0), fg_scale=3.0, fg_box_half=0.5,
                     shell=(12.0, 16.0))
    if opaque:
        spec.density_peak = _opaque_peak(spec)
    if clean:
        spec.density_noise = 0.0
    return make_scene(spec)


def scene_stress(seed: int = 0, band: float = 1.5, halo: float = 0.85, opaque: bool = True) -> dict:
    """Growth-budget stress scene: ~10M voxels, levels 6-13."""
    spec = SceneSpec(seed=seed, root_min=(-16, -16, -16), root_edge=32.0, l_min=6, l_max_fg=13, l_max_bg=8,
                     band=band, halo=halo, fg_center=(0.0, 0.0, 0.0), fg_scale=3.5, fg_box_half=0.5,
                     shell=(12.0, 16.0))
    if opaque:
        spec.density_peak = _opaque_peak(spec)
    return make_scene(spec)


def constant_voxel_scene(centers, half, dens, rgb) -> dict:
    """Hand-placed voxels with constant corner density and degree-0 colour ``rgb``.

    The DC coefficient is chosen so that the decoded colour equals ``rgb``
    for the standard real-SH normalisation Y_0 = 1 / (2 sqrt(pi)).
    """
    centers = np.asarray(centers, np.float32).reshape(-1, 3)
    n = centers.shape[0]
    geom = np.empty((n, 4), np.float32)
    geom[:, :3] = centers
    geom[:, 3] = np.broadcast_to(np.asarray(half, np.float32), (n,))
    density = np.empty((n, 8), np.float32)
    density[:] = np.asarray(dens, np.float32).reshape(n, 1) if np.ndim(dens) else dens
    sh = np.zeros((n, 48), np.float32)
    y0 = 0.5 / math.sqrt(math.pi)
    sh[:, 0:3] = ((np.asarray(rgb, np.float64).reshape(-1, 3) - 0.5) / y0).astype(np.float32)
    return {"geom": geom, "level": np.zeros(n, np.uint8), "density": density, "sh": sh}


def look_at_camera(eye, target, width, height, fov_x_deg, z_near=0.05, up=(0.0, 1.0, 0.0)) -> dict:
    """Pinhole camera at ``eye`` looking at ``target`` (OpenCV axes, principal point at the centre)."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    upv = np.asarray(up, np.float64)
    down = -(upv - np.dot(upv, fwd) * fwd)
    down /= np.linalg.norm(down)
    right = np.cross(down, fwd)
    R = np.stack([right, down, fwd])
    t = -R @ eye
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    w2c = np.concatenate([R, t[:, None]], axis=1).astype(np.float32)
    return {"width": int(width), "height": int(height), "fx": float(np.float32(fx)), "fy": float(np.float32(fx)),
            "cx": float(width) * 0.5, "cy": float(height) * 0.5, "w2c": w2c.reshape(-1).tolist(),
            "z_near": float(z_near)}


def orbit_camera(width, height, fov_x_deg, radius, azimuth_deg, elevation_deg, target=(0.0, 0.0, 0.0),
                 z_near=0.05) -> dict:
    """Camera on a sphere of ``radius`` around ``target`` (y is up)."""
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    tgt = np.asarray(target, np.float64)
    eye = tgt + radius * np.array([math.cos(el) * math.sin(az), math.sin(el), math.cos(el) * math.cos(az)])
    return look_at_camera(eye, tgt, width, height, fov_x_deg, z_near)


def uneven_views(n_views=16, seed=2, radius=3.0, fov_x_deg=60.0, target=(0.0, 0.0, 0.0),
                 w0=640, w1=1600, h0=480, h1=1060) -> list:
    """``n_views`` orbit cameras with sizes ramping from w0 x h0 to w1 x h1 (rounded to even)."""
    rng = np.random.default_rng(seed)
    cams = []
    for i in range(n_views):
        f = i / max(1, n_views - 1)
        w = int(round((w0 + (w1 - w0) * f) / 2.0)) * 2
        h = int(round((h0 + (h1 - h0) * f) / 2.0)) * 2
        yaw = rng.uniform(0.0, 360.0)
        elev = rng.uniform(5.0, 30.0)
        cams.append(orbit_camera(w, h, fov_x_deg, radius, yaw, elev, target))
    return cams


def random_image(width, height, seed=1) -> np.ndarray:
    """U(0,1) RGB target image, float32 [H*W, 3]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(height * width, 3)).astype(np.float32)


def smooth_image(width, height, seed=1, blobs=12) -> np.ndarray:
    """Piecewise-smooth RGB image (flat regions separated by edges), float32 [H*W, 3]."""
    rng = np.random.default_rng(seed)
    ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
    img = np.zeros((height, width, 3))
    img[:] = rng.uniform(0.2, 0.8, size=3)
    for _ in range(blobs):
        cx, cy = rng.uniform(0, width), rng.uniform(0, height)
        r = rng.uniform(0.05, 0.3) * min(width, height)
        mask = (xs - cx) ** 2 + (ys - cy) ** 2 < r * r
        img[mask] = rng.uniform(0.0, 1.0, size=3)
    img += 0.05 * (xs / max(1, width - 1))[..., None]
    return np.clip(img, 0, 1).reshape(-1, 3).astype(np.float32)
