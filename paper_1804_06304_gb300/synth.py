"""Seeded synthetic volumes shaped like the paper's microscopy workloads.

Input generation only: this module holds none of the snakuscule arithmetic, and
both the CUDA path's tests/benchmarks and the FP64 oracle read its outputs.  The
paper's own images (DAPI rat-brain slice, mouse-hippocampus confocal stacks and the
Cell Tracking Challenge sets of Tables I-II) are not available; these generators
stand in for them with bright round nuclei on a darker background:

* ``small_3d``   64x64x32 uint8, 20 balls of radius 4-6 (min separation 8),
                 intensity 200 on 30, Gaussian noise sigma 15.
* ``large_2d``   4096x4096 uint8, ~12k disks of radius 5-10 (overlap allowed),
                 200 on 30, Gaussian blur sigma 1.5, Poisson noise.
* ``brain_3d``   1024x1024x256 uint16 (spacing 1:1:2), ~100k rotated ellipsoids
                 with semi-axes 3-8, log-normal brightness around 2000, background
                 300 plus a 600 ramp along x, Gaussian noise sigma 50; an FP16 copy.
* ``batch_3d``   64 uint8 volumes from 64^3 to 512x512x128 (log-uniform voxel
                 count), one nucleus per 2000 voxels, radius 3-8.
* ``tile_stream`` uint16 tiles from 128^3 to 1024x1024x64 (log-uniform voxel
                 count) with Poisson arrival times; nuclei as in ``brain_3d``.

Arrays are indexed [z, y, x] (3D) or [y, x] (2D), x fastest in memory.  Nucleus
centres are physical coordinates (index * spacing) in x, y, z order.  Every
generator takes a seed and uses numpy's PCG64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Synth:
    name: str
    volume: np.ndarray            # [z, y, x] or [y, x]
    spacing: tuple                # physical voxel size along x, y, z
    centres: np.ndarray           # (n, 3) physical x, y, z of each nucleus
    radii: np.ndarray             # (n,) radius (ellipsoids: mean semi-axis)
    contrast: float               # typical foreground - background, stored units
    seed: int
    volume_f16: np.ndarray | None = None

    @property
    def ndim(self) -> int:
        return self.volume.ndim

    @property
    def shape_xyz(self) -> tuple:
        return tuple(self.volume.shape[::-1])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _paint_balls(label: np.ndarray, centres_idx: np.ndarray, radii_idx: np.ndarray) -> None:
    """Mark voxels whose centre lies inside each ball (index units, per-axis radii)."""
    nd = label.ndim
    shape_xyz = label.shape[::-1]
    for c, r in zip(centres_idx, radii_idx):
        lo = [max(0, int(math.floor(c[a] - r[a]))) for a in range(nd)]
        hi = [min(shape_xyz[a] - 1, int(math.ceil(c[a] + r[a]))) for a in range(nd)]
        if any(h < l for l, h in zip(lo, hi)):
            continue
        axes = [np.arange(lo[a], hi[a] + 1) for a in range(nd)]
        if nd == 3:
            z, y, x = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
            inside = ((x - c[0]) / r[0]) ** 2 + ((y - c[1]) / r[1]) ** 2 + ((z - c[2]) / r[2]) ** 2 < 1.0
            label[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] |= inside
        else:
            y, x = np.meshgrid(axes[1], axes[0], indexing="ij")
            inside = ((x - c[0]) / r[0]) ** 2 + ((y - c[1]) / r[1]) ** 2 < 1.0
            label[lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] |= inside


def sphere_volume(shape_xyz, centre, radius, inside=200.0, outside=30.0, noise=0.0, seed=0,
                  dtype=np.uint8) -> np.ndarray:
    """One ball (or disk) on a flat background; voxel-centre-inside rule."""
    nd = len(shape_xyz)
    label = np.zeros(tuple(shape_xyz[::-1]), dtype=bool)
    _paint_balls(label, np.array([centre], dtype=np.float64), np.array([[radius] * nd], dtype=np.float64))
    vol = np.where(label, inside, outside).astype(np.float64)
    if noise > 0:
        vol += _rng(seed).normal(0.0, noise, size=vol.shape)
    if np.issubdtype(dtype, np.integer):
        info = np.iinfo(dtype)
        vol = np.clip(np.rint(vol), info.min, info.max)
    return vol.astype(dtype)


def _uniform_centres(rng, n, shape_xyz, min_sep=0.0, max_tries=10_000):
    lo = np.zeros(len(shape_xyz))
    hi = np.array(shape_xyz, dtype=np.float64) - 1.0
    out = []
    tries = 0
    while len(out) < n and tries < max_tries:
        tries += 1
        c = rng.uniform(lo, hi)
        if min_sep > 0 and out and np.min(np.linalg.norm(np.array(out) - c, axis=1)) < min_sep:
            continue
        out.append(c)
    return np.array(out)


def small_3d(seed: int = 0) -> Synth:
    """64x64x32 uint8, 20 balls radius U[4,6], min separation 8, 200 on 30, noise 15."""
    rng = _rng(seed)
    shape = (64, 64, 32)
    centres = _uniform_centres(rng, 20, shape, min_sep=8.0)
    radii = rng.uniform(4.0, 6.0, size=len(centres))
    label = np.zeros(shape[::-1], dtype=bool)
    _paint_balls(label, centres, np.repeat(radii[:, None], 3, axis=1))
    vol = np.where(label, 200.0, 30.0) + rng.normal(0.0, 15.0, size=label.shape)
    vol = np.clip(np.rint(vol), 0, 255).astype(np.uint8)
    return Synth("small-3d 64x64x32 u8", vol, (1.0, 1.0, 1.0), centres, radii, 170.0, seed)


def large_2d(seed: int = 1, shape=(4096, 4096), n_nuclei: int = 12_000) -> Synth:
    """4096x4096 uint8, ~12k disks radius U[5,10], blur sigma 1.5, Poisson noise."""
    from scipy.ndimage import gaussian_filter

    rng = _rng(seed)
    centres = rng.uniform((0.0, 0.0), (shape[0] - 1.0, shape[1] - 1.0), size=(n_nuclei, 2))
    radii = rng.uniform(5.0, 10.0, size=n_nuclei)
    label = np.zeros(shape[::-1], dtype=bool)
    _paint_balls(label, centres, np.repeat(radii[:, None], 2, axis=1))
    img = np.where(label, np.float32(200.0), np.float32(30.0)).astype(np.float32)
    img = gaussian_filter(img, sigma=1.5, mode="nearest")
    img = rng.poisson(np.maximum(img, 0.0)).astype(np.float64)
    img = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    c3 = np.concatenate([centres, np.zeros((n_nuclei, 1))], axis=1)
    return Synth(f"large-2d {shape[0]}x{shape[1]} u8", img, (1.0, 1.0, 1.0), c3, radii, 170.0, seed)


def _random_rotations(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], axis=1)


def _render_brain(rng, shape_xyz, spacing, n_nuclei, dtype=np.uint16, with_f16=True):
    """Ellipsoidal nuclei, log-normal brightness, ramp background, Gaussian noise."""
    sp = np.array(spacing, dtype=np.float64)
    ext = (np.array(shape_xyz) - 1) * sp
    centres = rng.uniform(np.zeros(3), ext, size=(n_nuclei, 3))
    axes = rng.uniform(3.0, 8.0, size=(n_nuclei, 3))
    rots = _random_rotations(rng, n_nuclei)
    bright = rng.lognormal(math.log(2000.0), 0.4, size=n_nuclei)
    nx, ny, nz = shape_xyz
    fg = np.zeros((nz, ny, nx), dtype=np.float32)
    for c, a, Rm, b in zip(centres, axes, rots, bright):
        rmax = a.max()
        lo = np.maximum(np.floor((c - rmax) / sp).astype(int), 0)
        hi = np.minimum(np.ceil((c + rmax) / sp).astype(int), np.array(shape_xyz) - 1)
        if np.any(hi < lo):
            continue
        z, y, x = np.meshgrid(np.arange(lo[2], hi[2] + 1), np.arange(lo[1], hi[1] + 1),
                              np.arange(lo[0], hi[0] + 1), indexing="ij")
        d = np.stack([x * sp[0] - c[0], y * sp[1] - c[1], z * sp[2] - c[2]], -1) @ Rm
        inside = ((d / a) ** 2).sum(-1) < 1.0
        blk = fg[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
        np.maximum(blk, np.where(inside, np.float32(b), np.float32(0.0)), out=blk)
    ramp = (300.0 + 600.0 * np.arange(nx, dtype=np.float32) / max(nx - 1, 1)).astype(np.float32)
    vol = np.empty((nz, ny, nx), dtype=dtype)
    vol16 = np.empty((nz, ny, nx), dtype=np.float16) if with_f16 else None
    for z0 in range(0, nz, 16):
        z1 = min(nz, z0 + 16)
        slab = np.where(fg[z0:z1] > 0, fg[z0:z1], ramp[None, None, :])
        slab = slab + rng.normal(0.0, 50.0, size=slab.shape).astype(np.float32)
        slab = np.clip(np.rint(slab), 0, 65535)
        vol[z0:z1] = slab.astype(dtype)
        if with_f16:
            vol16[z0:z1] = vol[z0:z1].astype(np.float16)
    return vol, vol16, centres, axes.mean(axis=1)


def brain_3d(seed: int = 2, shape=(1024, 1024, 256), n_nuclei: int = 100_000, with_f16: bool = True) -> Synth:
    """Brain-like uint16 volume (x, y, z) with spacing 1:1:2 and an FP16 copy."""
    rng = _rng(seed)
    spacing = (1.0, 1.0, 2.0)
    vol, vol16, centres, radii = _render_brain(rng, shape, spacing, n_nuclei, with_f16=with_f16)
    return Synth(f"brain-3d {shape[0]}x{shape[1]}x{shape[2]} u16", vol, spacing, centres, radii, 1700.0, seed,
                 volume_f16=vol16)


def batch_3d(seed: int = 3, count: int = 64, max_scale: float = 1.0) -> list:
    """Uneven uint8 volumes: X=Y=64*8^t, Z=64*2^t with t ~ U[0,1] (optionally scaled
    down by ``max_scale``), one nucleus per 2000 voxels, radius U[3,8], 200 on 30,
    Gaussian noise 15."""
    rng = _rng(seed)
    out = []
    for i in range(count):
        t = rng.uniform(0.0, 1.0) * max_scale
        X = int(round(64 * 8 ** t))
        Z = int(round(64 * 2 ** t))
        shape = (X, X, Z)
        n = rng.poisson(X * X * Z / 2000.0)
        centres = rng.uniform(np.zeros(3), np.array(shape) - 1.0, size=(n, 3))
        radii = rng.uniform(3.0, 8.0, size=n)
        label = np.zeros(shape[::-1], dtype=bool)
        _paint_balls(label, centres, np.repeat(radii[:, None], 3, axis=1))
        vol = np.where(label, 200.0, 30.0) + rng.normal(0.0, 15.0, size=label.shape)
        vol = np.clip(np.rint(vol), 0, 255).astype(np.uint8)
        out.append(Synth(f"batch-3d[{i}] {X}x{X}x{Z} u8", vol, (1.0, 1.0, 1.0), centres, radii, 170.0, seed))
    return out


def tile_stream(seed: int = 4, count: int = 32, rate_hz: float = 10.0, max_scale: float = 1.0):
    """Tiles X=Y=128*8^t, Z=128*2^-t (t ~ U[0,1], optionally scaled by ``max_scale``)
    with brain_3d's nucleus model (isotropic spacing), arriving as a Poisson process
    of rate ``rate_hz``.  Returns [(arrival_s, Synth)]."""
    rng = _rng(seed)
    t_arr = np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
    out = []
    for i in range(count):
        t = rng.uniform(0.0, 1.0) * max_scale
        X = int(round(128 * 8 ** t))
        Z = int(round(128 * 2 ** (-t)))
        shape = (X, X, Z)
        n = max(1, int(X * X * Z / 2700))
        vol, _, centres, radii = _render_brain(rng, shape, (1.0, 1.0, 1.0), n, with_f16=False)
        out.append((float(t_arr[i]), Synth(f"tile[{i}] {X}x{X}x{Z} u16", vol, (1.0, 1.0, 1.0), centres, radii,
                                           1700.0, seed)))
    return out
