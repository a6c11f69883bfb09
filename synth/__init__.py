"""Seeded synthetic inputs for the ray caster: HI-like spectral cubes, cameras
and transfer-function tables.

This module only draws inputs. It holds none of the rendering arithmetic, so
both the CUDA path and the FP64 oracle can consume what it produces: the cube
is generated once and the same stored bytes are handed to each side.

Cubes stand in for the HIPASS survey cubes the paper renders (Section 5,
Table of datasets): a 21-cm spectral cube is mostly Gaussian noise with compact
sources.  Axis order is the FITS order: x = RA (fastest), y = Dec, z = frequency.

Random parameters come from splitmix64 (Steele, Lea & Flood 2014), written
out here so that the draws are identical on every machine.  The noise field
comes from ``torch.randn`` with a seeded generator on the device that holds
the cube (CPU and CUDA streams differ; the bytes are shared afterwards, never
regenerated).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator (Steele, Lea & Flood, OOPSLA 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1)) if hi > lo else lo


# --------------------------------------------------------------------------
# Source catalogue (host-side parameter draws)
# --------------------------------------------------------------------------

@dataclass
class Blob:
    amp: float
    sigma: float
    cx: float
    cy: float
    cz: float


@dataclass
class Disk:
    """Rotating-disk HI source: Gaussian spatial profile (sigma = radius/2,
    truncated at 2 radii) times a Gaussian spectral line whose centre is
    shifted along z by a linear velocity gradient along an in-plane axis."""
    amp: float
    radius: float
    width: float
    cx: float
    cy: float
    cz: float
    phi: float        # in-plane axis of the velocity gradient
    grad: float       # channels of line shift per voxel of projected offset


@dataclass
class Catalogue:
    blobs: list = field(default_factory=list)
    disks: list = field(default_factory=list)


def draw_catalogue(dims, n_blobs: int, n_disks: int, seed: int) -> Catalogue:
    nx, ny, nz = dims
    rng = SplitMix64(seed)
    cat = Catalogue()
    for _ in range(n_blobs):
        cat.blobs.append(Blob(amp=rng.uniform(5.0, 50.0), sigma=rng.uniform(2.0, 8.0),
                              cx=rng.uniform(0.0, nx - 1.0), cy=rng.uniform(0.0, ny - 1.0),
                              cz=rng.uniform(0.0, nz - 1.0)))
    for _ in range(n_disks):
        radius = rng.uniform(4.0, 20.0)
        width = rng.uniform(3.0, 10.0)
        span = rng.uniform(2.0, 4.0)          # shift at one radius, in line widths
        cat.disks.append(Disk(amp=rng.uniform(5.0, 50.0), radius=radius, width=width,
                              cx=rng.uniform(0.0, nx - 1.0), cy=rng.uniform(0.0, ny - 1.0),
                              cz=rng.uniform(0.0, nz - 1.0), phi=rng.uniform(0.0, 2.0 * math.pi),
                              grad=span * width / radius))
    return cat


# --------------------------------------------------------------------------
# Cube synthesis (torch, on any device)
# --------------------------------------------------------------------------

def _axis(lo, hi, n, device, torch):
    a = max(0, int(math.floor(lo)))
    b = min(n - 1, int(math.ceil(hi)))
    return a, b, torch.arange(a, b + 1, device=device, dtype=torch.float32)


def hi_cube(dims, n_blobs: int, n_disks: int, seed: int, device="cpu", noise_sigma: float = 1.0,
            out=None):
    """Float32 HI-like cube, shape (nz, ny, nx) (x fastest in memory).

    i.i.d. N(0, noise_sigma^2) noise plus ``n_blobs`` 3D Gaussian blobs
    (amplitude U[5,50], sigma U[2,8] voxels, centres uniform; truncated at
    4 sigma) and ``n_disks`` rotating-disk sources (see :class:`Disk`).
    """
    import torch
    nx, ny, nz = (int(d) for d in dims)
    cat = draw_catalogue((nx, ny, nz), n_blobs, n_disks, seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    if out is None:
        cube = torch.randn((nz, ny, nx), generator=gen, device=device, dtype=torch.float32)
    else:
        cube = out
        cube.normal_(generator=gen)
    if noise_sigma != 1.0:
        cube.mul_(noise_sigma)
    for b in cat.blobs:
        r = 4.0 * b.sigma
        x0, x1, xs = _axis(b.cx - r, b.cx + r, nx, device, torch)
        y0, y1, ys = _axis(b.cy - r, b.cy + r, ny, device, torch)
        z0, z1, zs = _axis(b.cz - r, b.cz + r, nz, device, torch)
        inv = -0.5 / (b.sigma * b.sigma)
        gx = torch.exp((xs - b.cx) ** 2 * inv)
        gy = torch.exp((ys - b.cy) ** 2 * inv)
        gz = torch.exp((zs - b.cz) ** 2 * inv) * b.amp
        cube[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] += gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    for d in cat.disks:
        r = 2.0 * d.radius
        x0, x1, xs = _axis(d.cx - r, d.cx + r, nx, device, torch)
        y0, y1, ys = _axis(d.cy - r, d.cy + r, ny, device, torch)
        zr = 4.0 * d.width + d.grad * r
        z0, z1, zs = _axis(d.cz - zr, d.cz + zr, nz, device, torch)
        sig = 0.5 * d.radius
        dx = (xs - d.cx)[None, :]
        dy = (ys - d.cy)[:, None]
        spatial = torch.exp(-(dx * dx + dy * dy) / (2.0 * sig * sig)) * d.amp          # (y, x)
        shift = d.grad * (dx * math.cos(d.phi) + dy * math.sin(d.phi))                 # (y, x)
        dz = zs[:, None, None] - d.cz - shift[None, :, :]
        line = torch.exp(-(dz * dz) / (2.0 * d.width * d.width))
        cube[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] += line * spatial[None, :, :]
    return cube


# --------------------------------------------------------------------------
# Transfer functions
# --------------------------------------------------------------------------

TF_VMIN, TF_VMAX = -3.0, 50.0


def tf_ramp(K: int = 256, alpha_max: float = 0.1, knee: float = 2.0, vmin: float = TF_VMIN,
            vmax: float = TF_VMAX) -> np.ndarray:
    """Linear-ramp table over [vmin, vmax] (K x 4 float32, straight RGBA).

    Entry i stands for v_i = vmin + (vmax-vmin) i/(K-1); with t = i/(K-1) the
    colour is (t, t^2, 1-t) and the opacity rises linearly from 0 at ``knee`` to
    ``alpha_max`` at vmax (zero below the knee) -- our reading of the paper's
    "linear increasing opacity" sample rendering (Section 5).
    """
    i = np.arange(K, dtype=np.float64)
    t = i / (K - 1)
    v = vmin + (vmax - vmin) * t
    tf = np.empty((K, 4), dtype=np.float64)
    tf[:, 0] = t
    tf[:, 1] = t * t
    tf[:, 2] = 1.0 - t
    tf[:, 3] = np.where(v < knee, 0.0, alpha_max * (v - knee) / (vmax - knee))
    return tf.astype(np.float32)


def tf_random_pwl(seed: int, K: int = 256, alpha_max: float = 0.15) -> np.ndarray:
    """Random piecewise-linear K-entry table with 4-8 knots per channel."""
    rng = SplitMix64(seed)
    nk = rng.randint(4, 8)
    xs = np.linspace(0.0, 1.0, nk)
    out = np.empty((K, 4), dtype=np.float64)
    grid = np.linspace(0.0, 1.0, K)
    for ch in range(4):
        ys = np.array([rng.uniform() for _ in range(nk)])
        if ch == 3:
            ys = ys * alpha_max
            ys[0] = 0.0
        out[:, ch] = np.interp(grid, xs, ys)
    return out.astype(np.float32)


# --------------------------------------------------------------------------
# Cameras (plain dicts; both sides build their own structs from them)
# --------------------------------------------------------------------------

def camera_ortho(eye, forward, up, ortho_height, width, height):
    return dict(kind=0, eye=tuple(map(float, eye)), forward=tuple(map(float, forward)),
                up=tuple(map(float, up)), fov_y_deg=0.0, ortho_height=float(ortho_height),
                width=int(width), height=int(height))


def camera_persp(eye, forward, up, fov_y_deg, width, height):
    return dict(kind=1, eye=tuple(map(float, eye)), forward=tuple(map(float, forward)),
                up=tuple(map(float, up)), fov_y_deg=float(fov_y_deg), ortho_height=0.0,
                width=int(width), height=int(height))


def orbit_cameras(dims, n_views: int, fov_y_deg: float, width: int, height: int,
                  start_deg: float = 0.0, spacing=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0)):
    """Perspective views orbiting the cube about +y (the paper rotates the
    cube about Y, Section 5).  The eye distance makes the bounding sphere fit
    the vertical field of view."""
    ext = [(d - 1) * s for d, s in zip(dims, spacing)]
    centre = [o + e / 2.0 for o, e in zip(origin, ext)]
    radius = 0.5 * math.sqrt(sum(e * e for e in ext))
    dist = radius / math.sin(math.radians(fov_y_deg) / 2.0)
    cams = []
    for v in range(n_views):
        th = math.radians(start_deg + 360.0 * v / n_views)
        fwd = (-math.sin(th), 0.0, math.cos(th))
        eye = tuple(c - dist * f for c, f in zip(centre, fwd))
        cams.append(camera_persp(eye, fwd, (0.0, 1.0, 0.0), fov_y_deg, width, height))
    return cams


def camera_random_persp(dims, seed: int, width: int, height: int, fov_y_deg: float = 40.0):
    """Perspective camera at a random azimuth and elevation looking at the
    cube centre from a distance that fits its bounding sphere."""
    rng = SplitMix64(seed)
    az = rng.uniform(0.0, 2.0 * math.pi)
    el = rng.uniform(-0.6, 0.6)
    ext = [d - 1.0 for d in dims]
    centre = [e / 2.0 for e in ext]
    radius = 0.5 * math.sqrt(sum(e * e for e in ext))
    dist = radius / math.sin(math.radians(fov_y_deg) / 2.0)
    fwd = (-math.cos(el) * math.sin(az), -math.sin(el), math.cos(el) * math.cos(az))
    eye = tuple(c - dist * f for c, f in zip(centre, fwd))
    return camera_persp(eye, fwd, (0.0, 1.0, 0.0), fov_y_deg, width, height)


# --------------------------------------------------------------------------
# Workload presets (sizes of the five benchmark configurations)
# --------------------------------------------------------------------------

def preset_plain_128():
    """128^3 f32, 20 blobs, ortho along +z, 256^2, step 0.5, no early termination."""
    dims = (128, 128, 128)
    c = 63.5
    cam = camera_ortho((c, c, c - 200.0), (0, 0, 1), (0, 1, 0), 127.0, 256, 256)
    return dict(dims=dims, n_blobs=20, n_disks=0, seed=1, cameras=[cam], step=0.5, ert=2.0)


def preset_scale_1024(n_views: int = 8):
    """1024^3 f32, 2000 blobs + 200 disks, 8 perspective orbit views at 1080p,
    step 1 voxel, early termination at alpha >= 0.99."""
    dims = (1024, 1024, 1024)
    return dict(dims=dims, n_blobs=2000, n_disks=200, seed=2,
                cameras=orbit_cameras(dims, n_views, 40.0, 1920, 1080), step=1.0, ert=0.99)


def preset_diff_512(n_views: int = 4):
    """512^3 f32, 1024^2 images from 4 views, step 0.5, no early termination."""
    dims = (512, 512, 512)
    n_blobs = int(round(20 * (512 / 128) ** 3))
    return dict(dims=dims, n_blobs=n_blobs, n_disks=0, seed=5,
                cameras=orbit_cameras(dims, n_views, 40.0, 1024, 1024, start_deg=20.0),
                step=0.5, ert=2.0)


def batch_dims(seed: int = 4, n: int = 64):
    """Uneven cube sizes: each axis from {64, 96, ..., 512}, z up to 1024."""
    rng = SplitMix64(seed)
    xy_choices = list(range(64, 513, 32))
    z_choices = list(range(64, 1025, 32))
    out = []
    for _ in range(n):
        out.append((xy_choices[rng.randint(0, len(xy_choices) - 1)],
                    xy_choices[rng.randint(0, len(xy_choices) - 1)],
                    z_choices[rng.randint(0, len(z_choices) - 1)]))
    return out


def batch_image_size(seed: int):
    rng = SplitMix64(seed)
    s = rng.randint(512, 1024)
    return s, s
