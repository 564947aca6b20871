"""Pins for the oracle's second-order march (the higher-order fast marching
that Sec. 6 of the paper names as future work; the scheme is the textbook
second-order FMM: on an upwind axis whose next cell beyond the neighbour is
known and not above it, the one-sided difference (3 t - 4 psi1 + psi2)/(2h)
replaces (t - psi1)/h).

Each check comes from the mathematics, not from the oracle's own formula:

* closed forms of the local solve, derived by hand from the one-sided
  difference equation, and mixed first/second-order roots from np.roots
* a second neighbour that is unknown, non-monotone or on the other side
  leaves the first-order local solve unchanged, bit for bit
* one-sided second-order differences are exact for quadratics: a slab with
  slowness 1 + x (T = x + x^2/2, the BDF2 recurrence) and the bowl
  T = |x|^2 / 2 with slowness |x| (isotropic and with cells of unequal
  sides) are reproduced to rounding, where the first-order march errs by O(h)
* away from a point source with exact values inside a ball, the error falls
  by about 4 per halving of h (first order: about 2)
"""
import math

import numpy as np
import pytest


def _ho(oracle, nb, kn, nb2, kn2, Tc=np.inf, h=1.0, F=1.0):
    return oracle.local_solve(np.array(nb, float), np.array(kn, np.uint8), Tc, h, F,
                              nb2=np.array(nb2, float), nb2_known=np.array(kn2, np.uint8))


INF = np.inf


def test_second_order_local_solve_closed_forms(oracle):
    # one axis: (3 t - 4 a + b) / (2 h) = 1/F
    for a, b, h, F in [(1.0, 0.0, 1.0, 1.0), (2.5, 1.75, 0.5, 2.0), (0.3, 0.3, 0.1, 0.7)]:
        t = _ho(oracle, [a, INF, INF, INF, INF, INF], [1, 0, 0, 0, 0, 0],
                [b, 0, 0, 0, 0, 0], [1, 0, 0, 0, 0, 0], h=h, F=F)
        assert t == pytest.approx((4 * a - b + 2 * h / F) / 3, rel=1e-15, abs=1e-15)
        # the same from the plus side
        t = _ho(oracle, [INF, a, INF, INF, INF, INF], [0, 1, 0, 0, 0, 0],
                [0, b, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0], h=h, F=F)
        assert t == pytest.approx((4 * a - b + 2 * h / F) / 3, rel=1e-15, abs=1e-15)
    # three equal axes: 3 ((3 t - 4 a + b) / (2 h))^2 = F^-2
    a, b, h, F = 1.0, 0.8, 0.25, 1.3
    nb = [a, INF, INF, a, a, INF]
    kn = [1, 0, 0, 1, 1, 0]
    nb2 = [b, 0, 0, b, b, 0]
    t = _ho(oracle, nb, kn, nb2, kn, h=h, F=F)
    assert t == pytest.approx((4 * a - b + 2 * h / (math.sqrt(3.0) * F)) / 3, rel=1e-14)


def test_second_order_mixed_axes_against_np_roots(oracle):
    # x second order (a, b), y first order (c): the larger root of
    # ((3t - 4a + b)/(2 hx))^2 + ((t - c)/hy)^2 = F^-2
    rng = np.random.default_rng(11)
    for _ in range(50):
        hx, hy = rng.uniform(0.5, 2.0, size=2)
        F = rng.uniform(0.5, 2.0)
        a = rng.uniform(1.0, 1.2)
        b = rng.uniform(0.0, a)   # |b| <= a: the x axis is second order
        c = a + rng.uniform(-0.3, 0.3) * hy / F
        ex = (3.0 / (2 * hx)) ** 2
        ey = 1.0 / hy ** 2
        e0 = (4 * a - b) / 3
        coef = [ex + ey, -2 * (ex * e0 + ey * c), ex * e0 * e0 + ey * c * c - 1 / F ** 2]
        r = np.roots(coef)
        r = r[np.isreal(r)].real
        cands = [x for x in r if x > e0 and x > c]
        # one-axis roots for the causal fallback
        cands.append(e0 + (2 * hx / 3) / F)
        cands.append(c + hy / F)
        expect = min(cands)
        t = _ho(oracle, [a, INF, c, INF, INF, INF], [1, 0, 1, 0, 0, 0],
                [b, 0, 0, 0, 0, 0], [1, 0, 0, 0, 0, 0], h=(hx, hy, 1.0), F=F)
        assert t == pytest.approx(expect, rel=1e-12)


def test_second_order_falls_back_to_first_order(oracle):
    rng = np.random.default_rng(3)
    for _ in range(40):
        nb = rng.uniform(0.0, 1.0, size=6)
        kn = rng.integers(0, 2, size=6).astype(np.uint8)
        h = tuple(rng.uniform(0.5, 1.5, size=3))
        F = rng.uniform(0.5, 2.0)
        first = oracle.local_solve(nb, kn, np.inf, h, F)
        # second neighbours unknown, whatever their values
        t = oracle.local_solve(nb, kn, np.inf, h, F, nb2=nb - 0.5,
                               nb2_known=np.zeros(6, np.uint8))
        assert t == first
        # second neighbours known but above the first ones (not monotone)
        t = oracle.local_solve(nb, kn, np.inf, h, F, nb2=nb + 0.25,
                               nb2_known=np.ones(6, np.uint8))
        assert t == first
    # a known, monotone second neighbour on the side that is not upwind
    nb = [0.5, 0.75, INF, INF, INF, INF]
    kn = [1, 1, 0, 0, 0, 0]
    t = _ho(oracle, nb, kn, [0, 0.0, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0])
    assert t == oracle.local_solve(np.array(nb), np.array(kn, np.uint8), np.inf, 1.0, 1.0)
    assert t == 1.5


def _fix(T_exact, mask, oracle):
    T = np.where(mask, T_exact, np.inf)
    G = np.where(mask, oracle.KNOWN_FIX, oracle.FAR).astype(np.uint8)
    return T, G


def test_second_order_slab_is_exact(oracle):
    """Slowness 1 + x along x only: T = x + x^2/2.  The second-order march is
    the BDF2 recurrence, exact for quadratics; the first-order one errs by
    O(h)."""
    n, h = 48, 1.0 / 48
    x = np.arange(n) * h
    T_ex = np.broadcast_to(x + 0.5 * x * x, (3, 4, n)).copy()
    F = np.broadcast_to(1.0 / (1.0 + x), (3, 4, n)).copy()
    mask = np.zeros(T_ex.shape, bool)
    mask[..., :2] = True
    T, G = _fix(T_ex, mask, oracle)
    r2 = oracle.march(T, G, h, speed=F, accuracy=2)
    r1 = oracle.march(T, G, h, speed=F)
    assert np.abs(r2["T"] - T_ex).max() <= 1e-13
    assert np.abs(r1["T"] - T_ex).max() > 1e-3
    assert np.all(r2["G"] == np.where(mask, oracle.KNOWN_FIX, oracle.KNOWN_NEW))


@pytest.mark.parametrize("h3", [(1 / 20, 1 / 20, 1 / 20), (1 / 20, 1.5 / 20, 0.75 / 20)])
def test_second_order_bowl_is_exact(oracle, h3):
    """T = |x|^2 / 2 with slowness |x| on x, y, z > 0: every upwind axis has a
    known monotone second neighbour once the two layers at the low faces are
    fixed, and one-sided second-order differences are exact for quadratics,
    with each axis's own cell size."""
    n = 20
    coords = [(np.arange(n) + 1.0) * h for h in h3]
    Z, Y, X = np.meshgrid(coords[2], coords[1], coords[0], indexing="ij")
    T_ex = 0.5 * (X * X + Y * Y + Z * Z)
    F = 1.0 / np.sqrt(X * X + Y * Y + Z * Z)
    mask = np.indices((n, n, n)).min(axis=0) < 2
    T, G = _fix(T_ex, mask, oracle)
    r2 = oracle.march(T, G, h3, speed=F, accuracy=2)
    r1 = oracle.march(T, G, h3, speed=F)
    err2 = np.abs(r2["T"] - T_ex).max() / T_ex.max()
    err1 = np.abs(r1["T"] - T_ex).max() / T_ex.max()
    assert err2 <= 1e-13
    assert err1 > 1e-2


def _point_errors(oracle, n, accuracy, R0=0.25):
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    R = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    mask = R < R0
    T, G = _fix(R, mask, oracle)
    e = np.abs(oracle.march(T, G, h, accuracy=accuracy)["T"] - R)[~mask]
    return e.max(), e.mean()


def test_second_order_convergence(oracle):
    """Distance from a point with exact values inside a ball of radius 1/4:
    halving h divides the error by about 4 (second order) instead of about 2
    (first order)."""
    m24, a24 = _point_errors(oracle, 24, 2)
    m48, a48 = _point_errors(oracle, 48, 2)
    assert m24 / m48 > 3.2 and a24 / a48 > 3.2
    f24, _ = _point_errors(oracle, 24, 1)
    f48, _ = _point_errors(oracle, 48, 1)
    assert 1.6 < f24 / f48 < 2.4
    assert m48 < f48 / 10


def test_second_order_arguments(oracle):
    T, G = oracle.init_sources((4, 4, 4), [(1, 1, 1)])
    with pytest.raises(ValueError):
        oracle.march(T, G, 1.0, accuracy=3)
    with pytest.raises(ValueError):
        oracle.march(T, G, 1.0, accuracy=2, record=True)
    # accuracy 1 through the second entry point is the first-order march
    a = oracle.march(T, G, 1.0)
    lib = oracle._load()
    T1 = T.copy()
    G1 = G.copy()
    h3 = np.ones(3)
    rc = lib.oracle_march_ho(4, 4, 4, h3.ctypes.data, None, 1.0, np.inf,
                             T1.ctypes.data, G1.ctypes.data, None, None, 1)
    assert rc == 0 and np.array_equal(T1, a["T"]) and np.array_equal(G1, a["G"])
    rc = lib.oracle_march_ho(4, 4, 4, h3.ctypes.data, None, 1.0, np.inf,
                             T1.ctypes.data, G1.ctypes.data, None, None, 0)
    assert rc == -1


def _bucketed_march(oracle, T0, G0, h, delta, accuracy):
    """A bucketed, label-correcting march (all BAND cells within delta of the
    band minimum accepted together, every non-FIX neighbour of an accepted
    cell re-solved, a cell whose value drops becomes BAND again), written
    here with the oracle's local solve: the order of updates a data-parallel
    march uses instead of the heap."""
    T = T0.copy()
    fix = G0 == oracle.KNOWN_FIX
    known = fix.copy()
    shape = T.shape
    steps = [(0, 0, 1), (0, 1, 0), (1, 0, 0)]   # x, y, z in (k, j, i)

    def inside(q):
        return all(0 <= q[a] < shape[a] for a in range(3))

    def solve(p):
        nb, kn = np.full(6, np.inf), np.zeros(6, np.uint8)
        nb2, kn2 = np.zeros(6), np.zeros(6, np.uint8)
        for ax, d in enumerate(steps):
            for si, s in enumerate((-1, 1)):
                q = tuple(p[a] + s * d[a] for a in range(3))
                q2 = tuple(p[a] + 2 * s * d[a] for a in range(3))
                if inside(q):
                    nb[2 * ax + si], kn[2 * ax + si] = T[q], known[q]
                if inside(q2):
                    nb2[2 * ax + si], kn2[2 * ax + si] = T[q2], known[q2]
        if accuracy == 1:
            return oracle.local_solve(nb, kn, T[p], h, 1.0)
        return oracle.local_solve(nb, kn, T[p], h, 1.0, nb2=nb2, nb2_known=kn2)

    def relax(p):
        for d in steps:
            for s in (-1, 1):
                q = tuple(p[a] + s * d[a] for a in range(3))
                if inside(q) and not fix[q]:
                    t = solve(q)
                    if t < T[q]:
                        T[q] = t
                        known[q] = False

    for p in zip(*np.nonzero(fix)):
        relax(p)
    while True:
        band = ~known & np.isfinite(T)
        if not band.any():
            return T
        acc = band & (T <= T[band].min() + delta)
        known |= acc
        for p in zip(*np.nonzero(acc)):
            relax(p)


def test_second_order_result_depends_on_the_update_order(oracle):
    """Sec. 5.2's agreement of parallel and sequential marches rests on the
    first-order scheme having one discrete solution whatever the update
    order: a bucketed label-correcting march reproduces the heap march bit
    for bit.  The second-order update is not monotone in its operands, so the
    same bucketed march reaches another solution, as accurate but different
    cell by cell (the reason the second-order variant has no GPU kernel held
    to the oracle)."""
    n = 10
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    R = np.sqrt((X - 0.3) ** 2 + (Y - 0.4) ** 2 + (Z - 0.5) ** 2)
    T0, G0 = _fix(R, R < 0.2, oracle)
    seq1 = oracle.march(T0, G0, h)["T"]
    seq2 = oracle.march(T0, G0, h, accuracy=2)["T"]
    for delta in (0.0, 2 * h):
        assert np.array_equal(_bucketed_march(oracle, T0, G0, h, delta, 1), seq1)
        lc2 = _bucketed_march(oracle, T0, G0, h, delta, 2)
        assert np.abs(lc2 - seq2).max() > 1e-4
        err_seq, err_lc = np.abs(seq2 - R).max(), np.abs(lc2 - R).max()
        assert err_lc < 1.5 * err_seq


def _jacobi_bucket_march(oracle, T0, G0, h3, F, bucket):
    """Second-order bucket steps in the order of updates of the GPU's
    cell-parallel schedule, written with the oracle's local solve: each step
    accepts the BAND cells within bucket * (hmin / (sqrt 3 max F of the 8^3
    brick)) of the band minimum, solves every non-FIX cell above a neighbour
    accepted in the step from the state before the step, then applies the
    improvements (an improved cell is BAND again)."""
    T = T0.copy()
    fix = G0 == oracle.KNOWN_FIX
    known = fix.copy()
    shape = T.shape
    bd = np.empty(shape)
    for bz in range(0, shape[0], 8):
        for by in range(0, shape[1], 8):
            for bx in range(0, shape[2], 8):
                sl = (slice(bz, bz + 8), slice(by, by + 8), slice(bx, bx + 8))
                bd[sl] = min(h3) / (math.sqrt(3.0) * F[sl].max())
    steps = [(0, 0, 1), (0, 1, 0), (1, 0, 0)]

    def inside(q):
        return all(0 <= q[a] < shape[a] for a in range(3))

    def solve(p):
        nb, kn = np.full(6, np.inf), np.zeros(6, np.uint8)
        nb2, kn2 = np.zeros(6), np.zeros(6, np.uint8)
        for ax, d in enumerate(steps):
            for si, s in enumerate((-1, 1)):
                q = tuple(p[a] + s * d[a] for a in range(3))
                q2 = tuple(p[a] + 2 * s * d[a] for a in range(3))
                if inside(q):
                    nb[2 * ax + si], kn[2 * ax + si] = T[q], known[q]
                if inside(q2):
                    nb2[2 * ax + si], kn2[2 * ax + si] = T[q2], known[q2]
        return oracle.local_solve(nb, kn, T[p], h3, F[p], nb2=nb2, nb2_known=kn2)

    def step(acc):
        new = {}
        for p in zip(*np.nonzero(~fix)):
            hit = False
            for d in steps:
                for s in (-1, 1):
                    q = tuple(p[a] + s * d[a] for a in range(3))
                    hit = hit or (inside(q) and acc[q] and T[q] < T[p])
            if hit:
                t = solve(p)
                if t < T[p]:
                    new[p] = t
        for p, t in new.items():
            T[p] = t
            known[p] = False

    step(fix.copy())
    while True:
        band = ~known & np.isfinite(T)
        if not band.any():
            return T
        acc = band & (T <= T[band].min() + bucket * bd)
        known |= acc
        step(acc)


def test_second_order_bucket_steps_need_narrow_buckets(oracle):
    """With the GPU's update order (Jacobi bucket steps), a cell accepted
    with a value the same step lowers can serve as a too-large second
    neighbour and pull another cell's root below the exact value for good;
    buckets below the smallest single-axis increment (2/3) keep the
    quadratic bowl exact, wide ones (4, the first-order default) do not."""
    n = 16
    h3 = (1 / 16, 1.5 / 16, 0.75 / 16)
    coords = [(np.arange(n) + 1.0) * h for h in h3]
    Z, Y, X = np.meshgrid(coords[2], coords[1], coords[0], indexing="ij")
    T_ex = 0.5 * (X * X + Y * Y + Z * Z)
    F = 1.0 / np.sqrt(X * X + Y * Y + Z * Z)
    T0, G0 = _fix(T_ex, np.indices((n, n, n)).min(axis=0) < 2, oracle)
    narrow = _jacobi_bucket_march(oracle, T0, G0, h3, F, 0.6)
    wide = _jacobi_bucket_march(oracle, T0, G0, h3, F, 4.0)
    assert np.abs(narrow - T_ex).max() / T_ex.max() <= 1e-13
    assert np.abs(wide - T_ex).max() / T_ex.max() > 1e-9
