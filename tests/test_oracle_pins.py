"""Pins for the CPU oracle: each check comes from the mathematics or the paper,
not from re-running the oracle's own formula.

* closed-form values of the upwind scheme on tiny grids (derived by hand from
  Eq. (2)-(3): exact along axes, the 2-D and 3-D diagonal roots)
* the discrete Eq. (2) residual, re-evaluated in numpy with all six final
  neighbours, vanishes at every accepted cell
* an independent Gauss-Seidel fast sweeping solve (sorted Godunov update)
  reaches the same discrete solution
* acceptance order is non-decreasing in |psi| per side (Sec. 2.2, heap order)
* a planar interface is reproduced exactly; front cells of oblique planes get
  the exact distance (the linear-interpolation reading of Algorithm 8)
* first-order convergence to the exact distance (Appendix, Eq. (12))
* the narrow band stops at width_band (Algorithm 5 / Algorithm 12)
* adjoint vs central finite differences, adjoint vs tangent (dot product)
* cells of size dx * dy * dz (Sec. 2.1, Algorithm 11's h_i): per-axis roots
  against np.roots, axis planes exact with each axis's own cell size, closed
  forms near a point source, exact front cells of an oblique plane, the
  weighted residual and weighted fast sweeping, transposing two axes with
  their cell sizes, the adjoint against finite differences
"""
import math

import numpy as np
import pytest

from paper_1502_07303_gb300 import workloads as wl

SQ2, SQ3 = math.sqrt(2.0), math.sqrt(3.0)


# --------------------------------------------------------------------------
# helpers written independently of the oracle
# --------------------------------------------------------------------------

def eq2_residual(T, h, F):
    """|grad psi| F - 1 with the Godunov operator of Eq. (2): per axis
    max(D-, -D+, 0) over |psi|, missing neighbours contribute nothing."""
    A = np.abs(T)
    s = np.zeros_like(A)
    for ax in range(3):
        pad = [(0, 0)] * 3
        pad[ax] = (1, 1)
        P = np.pad(A, pad, constant_values=np.inf)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -2)
        hi[ax] = slice(2, None)
        Dm = (A - P[tuple(lo)]) / h
        Dp = (P[tuple(hi)] - A) / h
        with np.errstate(invalid="ignore"):
            term = np.maximum(np.maximum(Dm, -Dp), 0.0)
        term = np.nan_to_num(term, nan=0.0, posinf=0.0)
        s += term * term
    return np.sqrt(s) * F - 1.0


def godunov3(a, sh):
    a = sorted(a)
    S = sum(a)
    Q = sum(v * v for v in a)
    return (S + math.sqrt(S * S - 3 * (Q - sh * sh))) / 3


def godunov2(a1, a2, sh):
    return 0.5 * (a1 + a2 + math.sqrt(2 * sh * sh - (a1 - a2) ** 2))


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def test_closed_forms_unit_speed(oracle):
    r = oracle.solve_sources((6, 6, 6), [(0, 0, 0)], 1.0)
    T = r["T"]  # indexed [k, j, i]
    for k in range(6):
        assert T[0, 0, k] == float(k)
        assert T[0, k, 0] == float(k)
        assert T[k, 0, 0] == float(k)
    d2 = 1 + 1 / SQ2
    assert abs(T[0, 1, 1] - d2) < 1e-15
    assert abs(T[1, 0, 1] - d2) < 1e-15
    assert abs(T[1, 1, 0] - d2) < 1e-15
    d3 = d2 + 1 / SQ3
    assert abs(T[1, 1, 1] - d3) < 1e-15
    t210 = ((1 + 1 / SQ2) + 2 + math.sqrt(2 - (1 - 1 / SQ2) ** 2)) / 2
    assert abs(T[0, 1, 2] - t210) < 1e-15
    assert abs(T[0, 2, 1] - t210) < 1e-15
    assert abs(T[1, 0, 2] - t210) < 1e-15
    # (2,2,0): 2-D root on two equal neighbours
    assert abs(T[0, 2, 2] - (t210 + 1 / SQ2)) < 1e-14
    # (2,1,1): 3-D root on (d3, t210, t210)
    assert abs(T[1, 1, 2] - godunov3([d3, t210, t210], 1.0)) < 1e-14


def test_closed_forms_scaled(oracle):
    h, F = 0.25, 2.0
    r = oracle.solve_sources((5, 5, 5), [(2, 2, 2)], h, speed=F)
    T = r["T"]
    for d in range(-2, 3):
        assert abs(T[2, 2, 2 + d] - abs(d) * h / F) < 1e-15
        assert abs(T[2, 2 + d, 2] - abs(d) * h / F) < 1e-15
    sh = h / F
    assert abs(T[2, 3, 3] - (sh + sh / SQ2)) < 1e-15
    assert abs(T[3, 3, 3] - (sh + sh / SQ2 + sh / SQ3)) < 1e-15


def test_local_solve_cases(oracle):
    inf = np.inf
    h = 0.5
    # one known neighbour: 1-D root psi + h/F
    v = oracle.local_solve([0.3, inf, inf, inf, inf, inf], [1, 0, 0, 0, 0, 0], inf, h, 2.0)
    assert abs(v - (0.3 + h / 2.0)) < 1e-15
    # the smaller of the two neighbours on an axis is used
    v = oracle.local_solve([0.7, 0.3, inf, inf, inf, inf], [1, 1, 0, 0, 0, 0], inf, h, 1.0)
    assert abs(v - 0.8) < 1e-15
    # 2-D root
    v = oracle.local_solve([1.0, inf, 1.2, inf, inf, inf], [1, 0, 1, 0, 0, 0], inf, 1.0, 1.0)
    assert abs(v - godunov2(1.0, 1.2, 1.0)) < 1e-14
    # non-causal 2-D set falls back to 1-D
    v = oracle.local_solve([1.0, inf, 5.0, inf, inf, inf], [1, 0, 1, 0, 0, 0], inf, 1.0, 1.0)
    assert v == 2.0
    # neighbours that are not KNOWN are ignored
    v = oracle.local_solve([1.0, inf, 1.0, inf, inf, inf], [1, 0, 0, 0, 0, 0], inf, 1.0, 1.0)
    assert v == 2.0
    # the upwind filter |psi_n| < |psi_cell| drops larger neighbours
    v = oracle.local_solve([1.0, inf, 1.5, inf, inf, inf], [1, 0, 1, 0, 0, 0], 1.4, 1.0, 1.0)
    assert v == 2.0
    # 3-D root
    v = oracle.local_solve([1.0, inf, 1.1, inf, 1.2, inf], [1, 0, 1, 0, 1, 0], inf, 1.0, 1.0)
    assert abs(v - godunov3([1.0, 1.1, 1.2], 1.0)) < 1e-14
    # nothing known: +inf
    v = oracle.local_solve([1.0] * 6, [0] * 6, inf, 1.0, 1.0)
    assert v == inf


# --------------------------------------------------------------------------
# discrete equation, fast sweeping, acceptance order
# --------------------------------------------------------------------------

def _rand_problem(seed, shape):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    h = 1.0 / max(shape)
    F = np.exp(0.6 * rng.standard_normal(shape))
    # smooth it a little so the speed is not pure noise
    for ax in range(3):
        F = 0.5 * F + 0.25 * (np.roll(F, 1, ax) + np.roll(F, -1, ax))
    nsrc = int(rng.integers(1, 5))
    src = wl.random_cells(rng, shape, nsrc)
    return h, F, src


@pytest.mark.parametrize("seed,shape", [(1, (8, 8, 8)), (2, (9, 13, 7)),
                                        (3, (16, 12, 20)), (4, (24, 24, 24))])
def test_residual_and_fast_sweep_sources(oracle, seed, shape):
    h, F, src = _rand_problem(seed, shape)
    r = oracle.solve_sources(shape, src, h, speed=F, record=True)
    T, G = r["T"], r["G"]
    assert np.all(np.isfinite(T))
    assert np.all((G == oracle.KNOWN_NEW) | (G == oracle.KNOWN_FIX))
    res = eq2_residual(T, h, F)
    mask = G == oracle.KNOWN_NEW
    assert np.max(np.abs(res[mask])) < 1e-10
    fixed = (G == oracle.KNOWN_FIX).astype(np.uint8)
    A, rounds = oracle.fast_sweep(np.abs(T) * fixed, fixed, h, speed=F)
    assert rounds < 10000
    assert np.max(np.abs(A - np.abs(T))) <= 1e-13 * np.max(np.abs(T))
    # acceptance order non-decreasing, each cell once
    order = r["order"]
    vals = np.abs(T.ravel()[order])
    assert np.all(np.diff(vals) >= 0)
    assert len(np.unique(order)) == len(order) == int(mask.sum())


@pytest.mark.parametrize("seed,shape", [(5, (12, 12, 12)), (6, (20, 14, 17))])
def test_two_sided_reinit(oracle, seed, shape):
    rng = np.random.default_rng(seed)
    sph = wl.draw_spheres(rng, 3, rmin=0.12, rmax=0.3)
    h = wl.spacing(shape)
    phi = wl.spheres_phi0(shape, sph, h=h)
    r = oracle.solve_reinit(phi, h, record=True)
    T, G = r["T"], r["G"]
    assert np.all(np.isfinite(T))
    # sign of the solution is the sign of phi0 (sgn(0) = +1)
    assert np.all((T >= 0) == (phi >= 0))
    # every edge with a sign change has KNOWN_FIX at both ends
    for ax in range(3):
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        a[ax] = slice(0, -1)
        b[ax] = slice(1, None)
        change = (phi[tuple(a)] >= 0) != (phi[tuple(b)] >= 0)
        assert np.all(G[tuple(a)][change] == oracle.KNOWN_FIX)
        assert np.all(G[tuple(b)][change] == oracle.KNOWN_FIX)
    res = eq2_residual(T, h, 1.0)
    assert np.max(np.abs(res[G == oracle.KNOWN_NEW])) < 1e-10
    fixed = (G == oracle.KNOWN_FIX).astype(np.uint8)
    A, _ = oracle.fast_sweep(np.abs(T), fixed, h)
    assert np.max(np.abs(A - np.abs(T))) <= 1e-13 * np.max(np.abs(T))
    # per side: non-decreasing |psi| in pop order
    order = r["order"]
    for sgn in (-1, 1):
        sel = order[np.sign(T.ravel()[order]) == sgn]
        assert np.all(np.diff(np.abs(T.ravel()[sel])) >= 0)


def test_translation_invariance(oracle):
    """Eq. (2) involves only differences of psi: raising every FIX value by a
    constant C must raise the whole solution by C.  With C of a few hundred
    cells the check also rejects a root formula whose rounding grows with
    |psi| (the unshifted form loses about 3 (psi F/h)^2 ulp)."""
    shape = (20, 18, 22)
    h, F, src = _rand_problem(13, shape)
    T0, G0 = oracle.init_sources(shape, src)
    r0 = oracle.march(T0, G0, h, speed=F)
    C = 700.0 * h
    TC = np.where(G0 == oracle.KNOWN_FIX, C, T0)
    rC = oracle.march(TC, G0, h, speed=F)
    diff = np.abs((rC["T"] - C) - r0["T"])
    assert np.max(diff) <= 1e-13 * (C + np.max(r0["T"])), np.max(diff)


def test_planted_mistake_is_caught(oracle):
    """A wrong sign in the discriminant of a 2-D root changes the value the
    residual check sees: the pins above would fail for such an oracle."""
    r = oracle.solve_sources((6, 6, 6), [(0, 0, 0)], 1.0)
    T = r["T"].copy()
    T[0, 1, 1] = (2 - math.sqrt(4 + 8)) / 2 + 2  # planted wrong root
    res = eq2_residual(T, 1.0, 1.0)
    assert abs(res[0, 1, 1]) > 1e-3


# --------------------------------------------------------------------------
# interfaces
# --------------------------------------------------------------------------

def test_axis_plane_exact(oracle):
    shape = (10, 11, 24)
    h = 1.0 / 24
    x0 = 0.4123
    phi = wl.plane_phi0(shape, (1.0, 0.0, 0.0), x0, h=h)
    phi = np.broadcast_to(phi, shape).copy()
    r = oracle.solve_reinit(phi, h)
    assert np.max(np.abs(r["T"] - phi)) < 1e-14


@pytest.mark.parametrize("normal", [(1.0, 1.0, 0.0), (1.0, 1.0, 1.0), (1.0, 2.0, 0.0)])
def test_oblique_plane_front_exact(oracle, normal):
    shape = (16, 16, 16)
    h = 1.0 / 16
    n = np.asarray(normal) / np.linalg.norm(normal)
    phi = wl.plane_phi0(shape, normal, 0.513 * n.sum(), h=h)
    phi = np.broadcast_to(phi, shape).copy()
    T, G = oracle.init_reinit(phi, h)
    fix = G == oracle.KNOWN_FIX
    assert fix.sum() > 0
    # a front cell gets the exact distance when the plane crosses every axis
    # whose normal component is non-zero within one cell of it
    k = len([c for c in normal if c != 0])
    nz_axes = [a for a, c in enumerate(normal) if c != 0]
    ok = np.zeros(shape, bool)
    ok[1:-1, 1:-1, 1:-1] = True
    sign = phi >= 0
    full = ok & fix
    for a in nz_axes:
        ax = 2 - a  # numpy axis of spatial axis a
        cross = np.zeros(shape, bool)
        for d in (-1, 1):
            cross |= np.roll(sign, d, ax) != sign
        full &= cross
    assert full.sum() > 0
    assert np.max(np.abs(T[full] - phi[full])) < 1e-14
    if k == 2 and normal[1] == normal[0]:
        # 45 degree plane x + y = c (c ~ 10.6 cells): each positive cell
        # depends on the cells with smaller x and y down to the plane, each
        # negative cell on those with larger x and y up to it; for x, y index
        # <= 10 neither cone reaches a domain face, so the march is exact
        r = oracle.march(T, G, h)
        inner = np.zeros(shape, bool)
        inner[:, :11, :11] = True
        assert np.max(np.abs(r["T"][inner] - phi[inner])) < 1e-13


def test_narrow_band_width(oracle):
    shape = (20, 20, 20)
    h, F, src = _rand_problem(11, shape)
    full = oracle.solve_sources(shape, src, h, speed=F)
    W = 0.5 * np.max(full["T"])
    band = oracle.solve_sources(shape, src, h, speed=F, width=W)
    acc = band["G"] == oracle.KNOWN_NEW
    inside = full["T"] <= W
    margin = np.abs(full["T"] - W) > 1e-12
    assert np.array_equal(acc[margin], (inside & (full["G"] == oracle.KNOWN_NEW))[margin])
    assert np.max(np.abs(band["T"][acc] - full["T"][acc])) == 0.0
    # cells beyond the band are BAND (finite tentative value) or FAR (+inf)
    rest = ~acc & (band["G"] != oracle.KNOWN_FIX)
    assert np.all(np.isin(band["G"][rest], [oracle.BAND_NEW, oracle.FAR]))
    assert np.all(band["T"][rest] > W)
    assert np.all(np.isinf(band["T"][band["G"] == oracle.FAR]))


# --------------------------------------------------------------------------
# convergence (Appendix, Eq. (12))
# --------------------------------------------------------------------------

def _l2(T, exact, G, oracle):
    m = G == oracle.KNOWN_NEW
    return math.sqrt(np.mean((T[m] - exact[m]) ** 2))


def test_first_order_point_source(oracle):
    errs = []
    ns = [16, 32, 64, 128]
    for n in ns:
        p = wl.point_source(n)
        r = oracle.solve_sources(p.shape, p.sources, p.h)
        x = (np.arange(n) + 0.5) * p.h
        c = (n // 2 + 0.5) * p.h
        ex = np.sqrt((x[None, None, :] - c) ** 2 + (x[None, :, None] - c) ** 2 + (x[:, None, None] - c) ** 2)
        errs.append(_l2(r["T"], ex, r["G"], oracle))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:]))
    assert slopes[-1] > 0.7, (errs, slopes)


def test_first_order_sphere(oracle):
    errs = []
    for n in [16, 32, 64, 128]:
        p = wl.single_sphere(n, radius=0.3)
        r = oracle.solve_reinit(p.phi0, p.h)
        errs.append(_l2(r["T"], p.phi0, r["G"], oracle))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:]))
    assert slopes[-1] > 0.85, (errs, slopes)


# --------------------------------------------------------------------------
# derivatives
# --------------------------------------------------------------------------

def _loss_and_grad(oracle, shape, src, rec, h, s):
    r = oracle.solve_sources(shape, src, h, speed=1.0 / s, record=True)
    T = r["T"]
    L = sum(T[k, j, i] for i, j, k in rec)
    g = np.zeros(shape)
    for i, j, k in rec:
        g[k, j, i] += 1.0
    return L, g, r


def test_adjoint_finite_differences(oracle):
    shape = (14, 13, 15)
    rng = np.random.default_rng(21)
    h = 1.0 / 15
    modes = wl.draw_fourier_modes(rng)
    F = wl.fourier_speed(shape, modes, h=h)
    src = wl.random_cells(rng, shape, 2)
    rec = wl.random_cells(rng, shape, 6, exclude=src)
    s = 1.0 / F
    L, g, r = _loss_and_grad(oracle, shape, src, rec, h, s)
    dLds, _ = oracle.adjoint(r, h, g, speed=F)
    for trial in range(4):
        v = rng.standard_normal(shape)
        eps = 1e-6 * np.linalg.norm(s) / np.linalg.norm(v)
        Lp, _, _ = _loss_and_grad(oracle, shape, src, rec, h, s + eps * v)
        Lm, _, _ = _loss_and_grad(oracle, shape, src, rec, h, s - eps * v)
        fd = (Lp - Lm) / (2 * eps)
        ad = float(np.sum(dLds * v))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_adjoint_tangent_dot_product(oracle):
    shape = (12, 12, 12)
    rng = np.random.default_rng(22)
    h = 1.0 / 12
    F = wl.fourier_speed(shape, wl.draw_fourier_modes(rng), h=h)
    r = oracle.solve_sources(shape, wl.random_cells(rng, shape, 3), h, speed=F, record=True)
    g = rng.standard_normal(shape)
    v = rng.standard_normal(shape)
    dLds, _ = oracle.adjoint(r, h, g, speed=F)
    dT = oracle.tangent(r, h, v, speed=F)
    lhs = float(np.sum(g * dT))
    rhs = float(np.sum(dLds * v))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))
    # FIX cells get no gradient; a source's slowness cannot move T
    assert np.all(dLds[r["G"] == oracle.KNOWN_FIX] == 0.0)


# ---------------------------------------------------------------------------
# obstacles (F = 0, test case 6 of Sec. 5.1)
# ---------------------------------------------------------------------------

def test_full_wall_blocks_and_leaves_source_side_unchanged(oracle):
    """A plane of F = 0 cells across the grid with the source on one side:
    the source side is exactly the unobstructed solution (wall cells are never
    known, and they lie downwind of every cell on that side), the wall and
    everything behind it stay FAR with psi = +inf."""
    shape = (14, 13, 20)
    h = 1.0 / 20
    src = [(4, 6, 7)]
    F = np.ones(shape)
    F[:, :, 11] = 0.0
    free = oracle.solve_sources(shape, src, h)
    wall = oracle.solve_sources(shape, src, h, speed=F)
    assert np.array_equal(wall["T"][:, :, :11], free["T"][:, :, :11])
    assert np.all(np.isinf(wall["T"][:, :, 11:]))
    assert np.all(wall["G"][:, :, 11:] == oracle.FAR)


def test_wall_with_gap_detours(oracle):
    """A wall with a square gap: every value is at least the unobstructed one
    (an obstacle only removes paths), cells behind the wall are reached
    through the gap, the wall stays FAR, and fast sweeping agrees."""
    shape = (16, 16, 24)
    h = 1.0 / 24
    src = [(3, 8, 8)]
    F = np.ones(shape)
    F[:, :, 10] = 0.0
    F[6:10, 6:10, 10] = 1.0      # the gap
    free = oracle.solve_sources(shape, src, h)
    r = oracle.solve_sources(shape, src, h, speed=F)
    T, G = r["T"], r["G"]
    wall = F == 0.0
    assert np.all(np.isinf(T[wall])) and np.all(G[wall] == oracle.FAR)
    open_ = ~wall
    assert np.all(np.isfinite(T[open_]))
    assert np.all(T[open_] >= free["T"][open_] - 1e-15)
    # the corner cell just behind the wall is reached around the wall's edge
    # of the gap: its straight path crosses the wall far from the gap
    assert T[0, 0, 11] > free["T"][0, 0, 11] + h
    fixed = (G == oracle.KNOWN_FIX).astype(np.uint8)
    A, rounds = oracle.fast_sweep(np.where(fixed == 1, np.abs(T), 0.0), fixed, h, speed=F)
    assert rounds < 10000
    fin = np.isfinite(T)
    assert np.array_equal(np.isfinite(A), fin)
    assert np.max(np.abs(A[fin] - T[fin])) <= 1e-13 * np.max(T[fin])


# --------------------------------------------------------------------------
# cells of size dx * dy * dz (Sec. 2.1; h_i = 1/dx, 1/dy, 1/dz in Alg. 11)
# --------------------------------------------------------------------------

H3 = (0.05, 0.08, 0.035)


def weighted_root(vals, hs, s):
    """The unique t with sum_i max(t - v_i, 0)^2 / h_i^2 = s^2 (Eq. (2) with
    per-axis cell sizes), from np.roots of the k-term quadratic for the
    sorted values, adding terms while the root exceeds the next value."""
    pairs = sorted(zip(vals, hs))
    t = None
    for k in range(1, len(pairs) + 1):
        if t is not None and t <= pairs[k - 1][0]:
            break
        w = [1.0 / (hh * hh) for _, hh in pairs[:k]]
        v = [vv for vv, _ in pairs[:k]]
        a = sum(w)
        b = -2.0 * sum(wi * vi for wi, vi in zip(w, v))
        c = sum(wi * vi * vi for wi, vi in zip(w, v)) - s * s
        t = max(np.roots([a, b, c]).real)
    return t


def eq2_residual_h3(T, h3, F):
    """eq2_residual with the cell size of each axis."""
    A = np.abs(T)
    s = np.zeros_like(A)
    for ax in range(3):
        hax = h3[2 - ax]          # numpy axis 0 is z
        pad = [(0, 0)] * 3
        pad[ax] = (1, 1)
        P = np.pad(A, pad, constant_values=np.inf)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -2)
        hi[ax] = slice(2, None)
        with np.errstate(invalid="ignore"):
            term = np.maximum(np.maximum((A - P[tuple(lo)]) / hax, -(P[tuple(hi)] - A) / hax), 0.0)
        term = np.nan_to_num(term, nan=0.0, posinf=0.0)
        s += term * term
    return np.sqrt(s) * F - 1.0


def test_anisotropic_local_solve(oracle):
    inf = np.inf
    dx, dy, dz = H3
    # 1-D roots use the cell size of their own axis
    for a, hh in enumerate(H3):
        nb = [inf] * 6
        kn = [0] * 6
        nb[2 * a + 1] = 0.4
        kn[2 * a + 1] = 1
        assert abs(oracle.local_solve(nb, kn, inf, H3, 2.0) - (0.4 + hh / 2.0)) < 1e-15
    # 2-D and 3-D roots with unequal weights
    v = oracle.local_solve([1.0, inf, 1.02, inf, inf, inf], [1, 0, 1, 0, 0, 0], inf, H3, 1.0)
    assert abs(v - weighted_root([1.0, 1.02], [dx, dy], 1.0)) < 1e-14
    v = oracle.local_solve([1.0, inf, 1.02, inf, 0.99, inf], [1, 0, 1, 0, 1, 0], inf, H3, 1.3)
    assert abs(v - weighted_root([1.0, 1.02, 0.99], [dx, dy, dz], 1.0 / 1.3)) < 1e-13
    # a set that is causal with equal cells but not with these: the 1-D root
    # along the small z cells (0.5 + 0.035) is below the y value 0.54
    v = oracle.local_solve([inf, inf, 0.54, inf, 0.5, inf], [0, 0, 1, 0, 1, 0], inf, H3, 1.0)
    assert abs(v - weighted_root([0.54, 0.5], [dy, dz], 1.0)) < 1e-14
    assert abs(v - (0.5 + dz)) < 1e-15


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_anisotropic_axis_plane_exact(oracle, axis):
    shape = (9, 11, 13)
    normal = [0.0, 0.0, 0.0]
    normal[axis] = 1.0
    off = 0.43 * shape[2 - axis] * H3[axis]
    phi = np.broadcast_to(wl.plane_phi0(shape, tuple(normal), off, h=H3), shape).copy()
    r = oracle.solve_reinit(phi, H3)
    assert np.max(np.abs(r["T"] - phi)) < 1e-14


def test_anisotropic_point_source_closed_forms(oracle):
    shape = (5, 5, 5)
    dx, dy, dz = H3
    r = oracle.solve_sources(shape, [(2, 2, 2)], H3)
    T = r["T"]
    for k in range(3):
        assert abs(T[2, 2, 2 + k] - k * dx) < 1e-15
        assert abs(T[2, 2 + k, 2] - k * dy) < 1e-15
        assert abs(T[2 + k, 2, 2] - k * dz) < 1e-15
    # (i+1, j+1): x neighbour (i, j+1) holds dy, y neighbour (i+1, j) holds dx
    assert abs(T[2, 3, 3] - weighted_root([dy, dx], [dx, dy], 1.0)) < 1e-15
    assert abs(T[3, 3, 3] - weighted_root([T[3, 3, 2], T[3, 2, 3], T[2, 3, 3]],
                                          [dx, dy, dz], 1.0)) < 1e-15


def test_anisotropic_oblique_plane_front_exact(oracle):
    """Plane x + y = c: a front cell whose x and y segments both cross the
    plane gets the exact distance, since the crossing distances along the
    axes are |phi| / n_a and (sum_a n_a^2 / phi^2)^(-1/2) = |phi| (Algorithm 8
    with linear interpolation), whatever the cell sizes."""
    shape = (6, 20, 24)
    phi = np.broadcast_to(wl.plane_phi0(shape, (1.0, 1.0, 0.0), 0.62 * math.sqrt(2.0), h=H3),
                          shape).copy()
    T, G = oracle.init_reinit(phi, H3)
    sign = phi >= 0
    both = G == oracle.KNOWN_FIX
    for ax in (1, 2):            # numpy axes of y and x
        cross = np.zeros(shape, bool)
        for d in (-1, 1):
            rolled = np.roll(sign, d, ax)
            edge = [slice(None)] * 3
            edge[ax] = 0 if d == 1 else -1
            valid = np.ones(shape, bool)
            valid[tuple(edge)] = False   # np.roll wraps around
            cross |= valid & (rolled != sign)
        both &= cross
    assert both.sum() > 20
    assert np.max(np.abs(T[both] - phi[both])) < 1e-14


@pytest.mark.parametrize("seed,shape", [(7, (9, 13, 7)), (8, (14, 10, 16))])
def test_anisotropic_residual_and_fast_sweep(oracle, seed, shape):
    _, F, src = _rand_problem(seed, shape)
    r = oracle.solve_sources(shape, src, H3, speed=F, record=True)
    T, G = r["T"], r["G"]
    mask = G == oracle.KNOWN_NEW
    assert np.max(np.abs(eq2_residual_h3(T, H3, F)[mask])) < 1e-10
    fixed = (G == oracle.KNOWN_FIX).astype(np.uint8)
    A, rounds = oracle.fast_sweep(np.abs(T) * fixed, fixed, H3, speed=F)
    assert rounds < 10000
    assert np.max(np.abs(A - np.abs(T))) <= 1e-13 * np.max(np.abs(T))


def test_anisotropic_transposition(oracle):
    """Swapping the x and y axes together with their cell sizes transposes
    the solution."""
    shape = (7, 9, 11)
    _, F, src = _rand_problem(9, shape)
    dx, dy, dz = H3
    a = oracle.solve_sources(shape, src, (dx, dy, dz), speed=F)["T"]
    src_t = [(j, i, k) for i, j, k in src]
    b = oracle.solve_sources((7, 11, 9), src_t, (dy, dx, dz),
                             speed=np.ascontiguousarray(F.transpose(0, 2, 1)))["T"]
    assert np.max(np.abs(b.transpose(0, 2, 1) - a)) < 1e-15


def test_anisotropic_adjoint_finite_differences(oracle):
    shape = (10, 12, 9)
    rng = np.random.default_rng(31)
    modes = wl.draw_fourier_modes(rng)
    F = wl.fourier_speed(shape, modes, h=H3)
    src = wl.random_cells(rng, shape, 2)
    rec = wl.random_cells(rng, shape, 6, exclude=src)
    s = 1.0 / F
    L, g, r = _loss_and_grad(oracle, shape, src, rec, H3, s)
    dLds, _ = oracle.adjoint(r, H3, g, speed=F)
    for trial in range(3):
        v = rng.standard_normal(shape)
        eps = 1e-6 * np.linalg.norm(s) / np.linalg.norm(v)
        Lp, _, _ = _loss_and_grad(oracle, shape, src, rec, H3, s + eps * v)
        Lm, _, _ = _loss_and_grad(oracle, shape, src, rec, H3, s - eps * v)
        fd = (Lp - Lm) / (2 * eps)
        ad = float(np.sum(dLds * v))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
