"""Seeded synthetic inputs for the Eikonal solver (shared by tests and bench).

This module holds only input synthesis: grids, sources, level sets and speed
fields.  It contains none of the fast marching arithmetic, so both the CUDA
library's callers and the CPU oracle's tests can use it.

The paper measures on analytic cases only (Sec. 5.1: a sphere, a plane, point
sources with analytic speed functions, Eq. (8)-(11)); there is no dataset.
The recipes below are those analytic cases, plus the seeded random ones the
workload table asks for (random spheres, random Fourier speed, uneven batches).

Geometry (a reading of Sec. 2.1): the domain is the box [0, n*h]^3 with psi at
cell centres x_i = (i + 1/2) h.  For the cubic grids h = 1/n (unit cube); for
non-cubic grids h = 1 / max(nx, ny, nz).

Random parameters are drawn with ``numpy.random.default_rng(seed)`` in a fixed
order so that every consumer sees the same problem.  Fields are evaluated in
float64 with numpy, or, when ``device`` is given, with torch on that device
(used only for grids too large for a quick host evaluation).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def spacing(shape):
    """Cell size h for a (nz, ny, nx) grid: 1 / max extent (unit cube when
    the grid is cubic)."""
    return 1.0 / float(max(shape))


def _axes(shape, h, device=None):
    """Cell-centre coordinates; h is one cell size or (dx, dy, dz)."""
    nz, ny, nx = shape
    hx, hy, hz = (h, h, h) if np.isscalar(h) else (float(v) for v in h)
    if device is None:
        x = (np.arange(nx, dtype=np.float64) + 0.5) * hx
        y = (np.arange(ny, dtype=np.float64) + 0.5) * hy
        z = (np.arange(nz, dtype=np.float64) + 0.5) * hz
        return x[None, None, :], y[None, :, None], z[:, None, None]
    import torch
    x = (torch.arange(nx, dtype=torch.float64, device=device) + 0.5) * hx
    y = (torch.arange(ny, dtype=torch.float64, device=device) + 0.5) * hy
    z = (torch.arange(nz, dtype=torch.float64, device=device) + 0.5) * hz
    return x.view(1, 1, nx), y.view(1, ny, 1), z.view(nz, 1, 1)


def _lib(device):
    if device is None:
        return np
    import torch
    return torch


# --------------------------------------------------------------------------
# level sets
# --------------------------------------------------------------------------

@dataclass
class Spheres:
    centres: np.ndarray  # (k, 3) as (x, y, z)
    radii: np.ndarray    # (k,)


def draw_spheres(rng, count, lo=0.15, hi=0.85, rmin=0.05, rmax=0.15):
    """Sphere centres uniform in [lo, hi]^3 and radii uniform in [rmin, rmax]."""
    c = rng.uniform(lo, hi, size=(count, 3))
    r = rng.uniform(rmin, rmax, size=count)
    return Spheres(c, r)


def spheres_phi0(shape, spheres: Spheres, h=None, modulate=True, device=None):
    """phi0 = min_k (|x - c_k| - r_k), times (1 + 0.3 sin5x sin5y sin5z) when
    ``modulate`` (the reinitialisation workload's perturbed level set)."""
    h = spacing(shape) if h is None else h
    x, y, z = _axes(shape, h, device)
    L = _lib(device)
    phi = None
    for (cx, cy, cz), r in zip(spheres.centres, spheres.radii):
        d = L.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) - r
        phi = d if phi is None else L.minimum(phi, d)
    if modulate:
        phi = phi * (1.0 + 0.3 * L.sin(5.0 * x) * L.sin(5.0 * y) * L.sin(5.0 * z))
    return phi


def sphere_phi0(shape, centre=(0.5, 0.5, 0.5), radius=0.3, h=None, device=None):
    """Signed distance to one sphere: |x - c| - r (negative inside; Sec. 5.1
    case 1 uses the same sign convention)."""
    h = spacing(shape) if h is None else h
    x, y, z = _axes(shape, h, device)
    L = _lib(device)
    cx, cy, cz = centre
    return L.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) - radius


def plane_phi0(shape, normal, offset, h=None):
    """phi0 = (n . x - offset) / |n| for a plane with normal n."""
    h = spacing(shape) if h is None else h
    x, y, z = _axes(shape, h)
    nx_, ny_, nz_ = normal
    s = math.sqrt(nx_ * nx_ + ny_ * ny_ + nz_ * nz_)
    return (nx_ * x + ny_ * y + nz_ * z - offset) / s


# --------------------------------------------------------------------------
# speed fields
# --------------------------------------------------------------------------

@dataclass
class FourierModes:
    kappa: np.ndarray   # (m,) integer wavenumbers
    u: np.ndarray       # (m, 3) unit directions
    phase: np.ndarray   # (m,)
    amp: float


def draw_fourier_modes(rng, n_modes=16, kmin=1, kmax=8):
    """g(x) = sum_m sqrt(2/m) cos(2 pi kappa_m u_m . x + phi_m): integer
    kappa uniform in [kmin, kmax], u uniform on the sphere, phi uniform in
    [0, 2 pi); unit variance."""
    kappa = rng.integers(kmin, kmax + 1, size=n_modes)
    v = rng.normal(size=(n_modes, 3))
    u = v / np.linalg.norm(v, axis=1, keepdims=True)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    return FourierModes(kappa, u, phase, math.sqrt(2.0 / n_modes))


def fourier_speed(shape, modes: FourierModes, h=None, device=None):
    """F = exp(0.5 g(x)) with g the random Fourier field."""
    h = spacing(shape) if h is None else h
    x, y, z = _axes(shape, h, device)
    L = _lib(device)
    g = 0.0
    for kap, (ux, uy, uz), ph in zip(modes.kappa, modes.u, modes.phase):
        arg = 2.0 * np.pi * float(kap) * (ux * x + uy * y + uz * z) + ph
        g = g + modes.amp * L.cos(arg)
    return L.exp(0.5 * g)


def paper_speed(shape, case, h=None):
    """Speed functions of Sec. 5.1 on the [-0.5, 0.5]^3 cube of the paper
    (Eq. (8)-(10)); case in {3, 4, 5, 6}: case 6 is F = 1 with F = 0 inside
    four concentric spherical shells of width 1/24 (radii 0.15, 0.25, 0.35,
    0.45), each with a cylindrical gap around the z axis (Eq. (11))."""
    h = spacing(shape) if h is None else h
    x, y, z = _axes(shape, h)
    x, y, z = x - 0.5, y - 0.5, z - 0.5
    if case == 3:
        return np.ones(shape)
    if case == 4:
        return 1.0 + 0.5 * np.sin(20 * np.pi * x) * np.sin(20 * np.pi * y) * np.sin(20 * np.pi * z)
    if case == 5:
        return 1.0 - 0.99 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)
    if case == 6:
        w = 1.0 / 24.0
        R = np.sqrt(x * x + y * y + z * z)
        r = np.sqrt(x * x + y * y)
        wall = np.zeros(np.broadcast(x, y, z).shape, dtype=bool)
        for r0, gap, below in ((0.15, 0.05, True), (0.25, 0.10, False), (0.35, 0.10, True),
                               (0.45, 0.10, False)):
            shell = (R > r0) & (R < r0 + w)
            hole = (r < gap) & ((z < 0) if below else (z > 0))
            wall |= shell & ~hole
        return np.where(wall, 0.0, 1.0)
    raise ValueError(case)


# --------------------------------------------------------------------------
# cells
# --------------------------------------------------------------------------

def random_cells(rng, shape, count, exclude=()):
    """``count`` distinct random cells (i, j, k), none of them in exclude."""
    nz, ny, nx = shape
    ex = {tuple(int(v) for v in c) for c in exclude}
    out = []
    while len(out) < count:
        c = (int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz)))
        if c in ex:
            continue
        ex.add(c)
        out.append(c)
    return np.asarray(out, dtype=np.int64).reshape(-1, 3)


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------

@dataclass
class Problem:
    """One Eikonal problem: either point sources or a level set phi0."""
    name: str
    shape: tuple          # (nz, ny, nx)
    h: float
    sources: np.ndarray | None = None     # (k, 3) cells (i, j, k)
    phi0: object = None                   # (nz, ny, nx) float64 (numpy or torch)
    speed: object = None                  # None -> speed_const
    speed_const: float = 1.0
    receivers: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_points(self):
        nz, ny, nx = self.shape
        return nx * ny * nz


def point_source(n=64):
    """n^3 unit cube, F = 1, one source at cell (n/2, n/2, n/2) (Sec. 5.1
    case 3 / Eq. (8))."""
    shape = (n, n, n)
    c = n // 2
    return Problem(f"point_source_{n}", shape, 1.0 / n,
                   sources=np.array([[c, c, c]], np.int64))


def random_spheres(n=256, count=32, seed=2, device=None, shape=None):
    """Reinitialisation of ``count`` seeded random spheres with the
    sin-modulated level set, on an n^3 unit cube (or ``shape``)."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n) if shape is None else tuple(shape)
    sph = draw_spheres(rng, count)
    h = spacing(shape)
    phi = spheres_phi0(shape, sph, h=h, device=device)
    return Problem(f"spheres{count}_{shape[2]}x{shape[1]}x{shape[0]}", shape, h,
                   phi0=phi, meta={"spheres": sph, "seed": seed})


def fourier_sources(n=512, n_sources=8, n_receivers=64, seed=3, device=None):
    """Heterogeneous speed F = exp(0.5 g) with 16 random Fourier modes and
    ``n_sources`` random point sources; ``n_receivers`` random receiver cells
    (distinct from the sources).  The physical modes depend only on the seed,
    so a smaller n gives the same field on a coarser grid."""
    rng = np.random.default_rng(seed)
    modes = draw_fourier_modes(rng)
    shape = (n, n, n)
    src = random_cells(rng, shape, n_sources)
    rec = random_cells(rng, shape, n_receivers, exclude=src)
    h = 1.0 / n
    F = fourier_speed(shape, modes, h=h, device=device)
    return Problem(f"fourier_{n}", shape, h, sources=src, speed=F,
                   receivers=rec, meta={"modes": modes, "seed": seed})


def single_sphere(n=1024, radius=0.3, device=None):
    """Signed distance to one sphere of radius 0.3 at the centre of the unit
    cube (Sec. 5.1 case 1 with the unit-cube geometry)."""
    shape = (n, n, n)
    return Problem(f"sphere_{n}", shape, 1.0 / n,
                   phi0=sphere_phi0(shape, radius=radius, device=device))


def batch_shapes(n_grids=256, lo=32, hi=192, seed=4):
    """Grid shapes for the batched workload: each axis uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    dims = rng.integers(lo, hi + 1, size=(n_grids, 3))
    counts = rng.integers(1, 9, size=n_grids)
    return dims, counts, rng


def batch(n_grids=256, lo=32, hi=192, seed=4, device=None):
    """Independent reinitialisation problems of uneven sizes: per grid 1-8
    random spheres with the modulated level set, h = 1 / max extent.  The
    sphere law of the 32-sphere workload is applied to each grid's own box
    (extents e = (nx, ny, nz) h): centres uniform in [0.15, 0.85] e per
    axis, radii uniform in [0.05, 0.15] min(e), so every grid has a front."""
    dims, counts, rng = batch_shapes(n_grids, lo, hi, seed)
    out = []
    for g in range(n_grids):
        nx, ny, nz = (int(v) for v in dims[g])
        shape = (nz, ny, nx)
        h = spacing(shape)
        ext = np.array([nx, ny, nz], dtype=np.float64) * h
        unit = draw_spheres(rng, int(counts[g]))
        sph = Spheres(unit.centres * ext[None, :], unit.radii * float(ext.min()))
        out.append(Problem(f"batch{g}", shape, h,
                           phi0=spheres_phi0(shape, sph, h=h, device=device),
                           meta={"spheres": sph}))
    return out
