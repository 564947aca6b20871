"""The cell-parallel march (schedule 4), the second-order march it carries
(the higher-order fast marching named as future work in Sec. 6), and the
solve from given interface values, against the oracle.

* first order: the cell-parallel march reaches the oracle's discrete solution
  cell by cell (reinitialisation, point sources with heterogeneous speed on
  cells of unequal sides, a finite band, given interface values), as the
  brick schedules do
* second order on quadratic solutions (a slab and a bowl, also with cells
  of unequal sides): both the GPU and the oracle reproduce them to
  rounding, so they agree cell by cell
* second order elsewhere (the result depends on the order of acceptances):
  the GPU's error against the exact distance falls by about 4 per halving
  of h and stays within a small factor of the oracle's
"""
import numpy as np
import pytest
import torch

from paper_1502_07303_gb300 import workloads as wl
from parity_util import compare

pytestmark = pytest.mark.gpu

DT = {"f32": torch.float32, "f64": torch.float64}
H3 = (1.0 / 40, 1.5 / 40, 0.7 / 40)


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")
    from paper_1502_07303_gb300 import fmm as _fmm
    return _fmm


def _q(a, dt):
    return np.asarray(a, np.float32).astype(np.float64) if dt == "f32" else np.asarray(a, np.float64)


def _host(t):
    return t.cpu().numpy().astype(np.float64) if t.dtype != torch.uint8 else t.cpu().numpy()


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=DT[dt], device="cuda")


def _fixed(oracle, T_exact, mask):
    T0 = np.where(mask, T_exact, np.inf)
    G0 = np.where(mask, oracle.KNOWN_FIX, oracle.FAR).astype(np.uint8)
    return T0, G0


# ---------------------------------------------------------------------------
# first order on the cell-parallel schedule: the oracle's discrete solution
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_cell_schedule_reinit_matches_oracle(fmm, oracle, dt):
    shape = (37, 30, 45)
    rng = np.random.default_rng(8)
    phi = np.asarray(wl.spheres_phi0(shape, wl.draw_spheres(rng, 6)), np.float64)
    h = wl.spacing(shape)
    ref = oracle.solve_reinit(_q(phi, dt), h)
    with fmm.Solver(shape, h, dtype=DT[dt], schedule=4) as s:
        T, G = s.reinit(_dev(phi, dt))
        st = s.stats()
    assert st["error_flags"] == 0 and st["restarts"] > 0 and st["brick_marches"] == 0
    compare(_host(T), _host(G), ref, dt)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_cell_schedule_sources_unequal_cells_matches_oracle(fmm, oracle, dt):
    shape = (29, 33, 37)
    rng = np.random.default_rng(4)
    F = np.asarray(wl.fourier_speed(shape, wl.draw_fourier_modes(rng), h=H3), np.float64)
    src = wl.random_cells(rng, shape, 3)
    ref = oracle.solve_sources(shape, src, H3, speed=_q(F, dt))
    with fmm.Solver(shape, H3, dtype=DT[dt], speed=_dev(F, dt), sources=src, schedule=4) as s:
        T, G = s.solve()
        assert s.stats()["error_flags"] == 0
    compare(_host(T), _host(G), ref, dt)


def test_cell_schedule_finite_band_matches_oracle(fmm, oracle):
    shape = (40, 40, 40)
    h = 1.0 / 40
    phi = np.asarray(wl.sphere_phi0(shape, radius=0.25), np.float64)
    width = 6 * h
    ref = oracle.solve_reinit(phi, h, width=width)
    with fmm.Solver(shape, h, dtype=torch.float64, schedule=4, width=width) as s:
        T, G = s.reinit(_dev(phi, "f64"))
    compare(_host(T), _host(G), ref, "f64", width=width)


@pytest.mark.parametrize("schedule", [0, 1, 4])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_given_interface_values_match_oracle(fmm, oracle, schedule, dt):
    """fmm_solve_fixed: a two-sided set of FIX cells with given values (the
    interface cells of a level set, values perturbed so that they are not
    the ones Algorithm 8 would compute), FAR cells of both sides."""
    shape = (26, 31, 35)
    h = wl.spacing(shape)
    phi = np.asarray(wl.sphere_phi0(shape, radius=0.3), np.float64)
    T_init, G_init = oracle.init_reinit(phi, h)
    rng = np.random.default_rng(12)
    fix = G_init == oracle.KNOWN_FIX
    T0 = np.where(fix, T_init * rng.uniform(0.9, 1.1, shape), np.where(phi < 0, -np.inf, np.inf))
    T0 = _q(T0, dt)
    G0 = np.where(fix, oracle.KNOWN_FIX, oracle.FAR).astype(np.uint8)
    ref = oracle.march(T0, G0, h)
    with fmm.Solver(shape, h, dtype=DT[dt], schedule=schedule) as s:
        T, G = s.solve_fixed(_dev(T0, dt))
        assert s.stats()["error_flags"] == 0
    compare(_host(T), _host(G), ref, dt)


def test_given_interface_values_rejects_bad_input(fmm):
    shape = (16, 16, 16)
    with fmm.Solver(shape, 1.0 / 16, dtype=torch.float64, schedule=4) as s:
        T0 = np.full(shape, np.inf)
        T0[8, 8, 8] = 0.0
        T0[3, 3, 3] = np.nan
        with pytest.raises(fmm.FmmError) as e:
            s.solve_fixed(_dev(T0, "f64"))
        assert e.value.code == fmm.FMM_ERR_INVALID
        # a sign change between two FAR cells
        T0 = np.full(shape, np.inf)
        T0[8, 8, 8] = 0.0
        T0[:, :, :4] = -np.inf
        with pytest.raises(fmm.FmmError) as e:
            s.solve_fixed(_dev(T0, "f64"))
        assert e.value.code == fmm.FMM_ERR_INVALID
        # the handle still solves afterwards
        T0 = np.full(shape, np.inf)
        T0[8, 8, 8] = 0.0
        T, G = s.solve_fixed(_dev(T0, "f64"))
        assert float(T[8, 8, 9]) == pytest.approx(1.0 / 16, rel=1e-15)


# ---------------------------------------------------------------------------
# second order
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_second_order_slab_exact(fmm, oracle, dt):
    """Slowness 1 + x along x: T = x + x^2/2, fixed on the first two layers;
    the one-sided second-order difference is exact for it."""
    n, h = 45, 1.0 / 45
    shape = (5, 6, n)
    x = np.arange(n) * h
    T_ex = np.broadcast_to(x + 0.5 * x * x, shape).copy()
    F = _q(np.broadcast_to(1.0 / (1.0 + x), shape), dt)
    mask = np.zeros(shape, bool)
    mask[..., :2] = True
    T0, G0 = _fixed(oracle, _q(T_ex, dt), mask)
    ref = oracle.march(T0, G0, h, speed=F, accuracy=2)
    with fmm.Solver(shape, h, dtype=DT[dt], speed=_dev(F, dt), accuracy=2) as s:
        T, G = s.solve_fixed(_dev(T0, dt))
        assert s.stats()["error_flags"] == 0
    compare(_host(T), _host(G), ref, dt)
    if dt == "f64":
        assert np.abs(_host(T) - T_ex).max() <= 1e-13


@pytest.mark.parametrize("h3", [(1 / 24, 1 / 24, 1 / 24), (1 / 24, 1.5 / 24, 0.75 / 24)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_second_order_bowl_exact(fmm, oracle, dt, h3):
    """T = |x|^2 / 2 with slowness |x| on x, y, z > 0, fixed on the two
    layers at the low faces: one-sided second-order differences are exact
    for it, both marches reproduce it to rounding, so GPU and oracle agree
    cell by cell."""
    shape = (27, 21, 24)   # (nz, ny, nx), ragged bricks
    xs = [(np.arange(shape[2 - a]) + 1.0) * h3[a] for a in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    T_ex = 0.5 * (X * X + Y * Y + Z * Z)
    F = _q(1.0 / np.sqrt(X * X + Y * Y + Z * Z), dt)
    mask = np.indices(shape).min(axis=0) < 2
    T0, G0 = _fixed(oracle, _q(T_ex, dt), mask)
    ref = oracle.march(T0, G0, h3, speed=F, accuracy=2)
    with fmm.Solver(shape, h3, dtype=DT[dt], speed=_dev(F, dt), accuracy=2) as s:
        T, G = s.solve_fixed(_dev(T0, dt))
        assert s.stats()["error_flags"] == 0
    compare(_host(T), _host(G), ref, dt)
    if dt == "f64":
        assert np.abs(_host(T) - T_ex).max() / T_ex.max() <= 1e-13


def _ball_problem(n, R0=0.25):
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    R = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    return h, R, R < R0


def test_second_order_convergence(fmm, oracle):
    """Distance from a point with exact values inside a ball of radius 1/4:
    the GPU's second-order error falls by more than 3.2 per halving of h and
    stays within 1.5x the oracle's (the two marches accept in different
    orders, so their second-order solutions differ within the error)."""
    errs = []
    for n in (24, 48):
        h, R, mask = _ball_problem(n)
        T0, G0 = _fixed(oracle, R, mask)
        ref = oracle.march(T0, G0, h, accuracy=2)["T"]
        with fmm.Solver(R.shape, h, dtype=torch.float64, accuracy=2) as s:
            T, G = s.solve_fixed(_dev(T0, "f64"))
        T = _host(T)
        out = ~mask
        e_gpu = np.abs(T - R)[out]
        e_ref = np.abs(ref - R)[out]
        assert e_gpu.max() <= 1.5 * e_ref.max()
        assert np.abs(T - ref)[out].max() <= e_ref.max()
        errs.append((e_gpu.max(), e_gpu.mean()))
    assert errs[0][0] / errs[1][0] > 3.2 and errs[0][1] / errs[1][1] > 3.2


def test_second_order_reinit_sphere(fmm, oracle):
    """Reinitialisation of a sphere (Algorithm 8's interface cells): the
    second-order march's mean error against the exact distance is well below
    the first-order one's and within 1.5x of the oracle's second-order
    error."""
    n = 64
    shape = (n, n, n)
    h = 1.0 / n
    phi = np.asarray(wl.sphere_phi0(shape, radius=0.3), np.float64)
    T_i, G_i = oracle.init_reinit(phi, h)
    ref2 = oracle.march(T_i, G_i, h, accuracy=2)["T"]
    res = {}
    for acc in (1, 2):
        with fmm.Solver(shape, h, dtype=torch.float64, accuracy=acc, schedule=4) as s:
            T, G = s.reinit(_dev(phi, "f64"))
        res[acc] = np.abs(_host(T) - phi)
    assert res[2].mean() < res[1].mean() / 2.5
    assert res[2].mean() <= 1.5 * np.abs(ref2 - phi).mean()
    assert res[2].max() <= 1.5 * np.abs(ref2 - phi).max()


def test_second_order_is_reproducible(fmm):
    """The cell-parallel march applies each step's new values after all
    solves of the step (the minima are order-free atomics), so two runs give
    the same bits."""
    shape = (48, 40, 44)
    rng = np.random.default_rng(3)
    phi = np.asarray(wl.spheres_phi0(shape, wl.draw_spheres(rng, 5)), np.float64)
    h = wl.spacing(shape)
    outs = []
    for _ in range(2):
        with fmm.Solver(shape, h, dtype=torch.float64, accuracy=2) as s:
            T, G = s.reinit(_dev(phi, "f64"))
        outs.append((_host(T), _host(G)))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
