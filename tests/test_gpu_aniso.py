"""Cells of size dx * dy * dz (Sec. 2.1; the per-axis h_i of Algorithm 11):
the CUDA path against the oracle on the same seeded inputs."""

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


def _sources_problem(seed=4, shape=(29, 33, 37)):
    rng = np.random.default_rng(seed)
    modes = wl.draw_fourier_modes(rng)
    F = wl.fourier_speed(shape, modes, h=H3)
    src = wl.random_cells(rng, shape, 3)
    return shape, F, src


def _spheres_phi(shape, seed=5, count=4):
    """Signed distance to a union of spheres (the C2 law) at the centres of
    cells of size H3."""
    rng = np.random.default_rng(seed)
    x, y, z = wl._axes(shape, H3)
    ext = np.array([shape[2] * H3[0], shape[1] * H3[1], shape[0] * H3[2]])
    phi = np.full(shape, np.inf)
    for _ in range(count):
        c = rng.uniform(0.15, 0.85, 3) * ext
        r = rng.uniform(0.05, 0.15) * ext.min()
        d = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) - r
        phi = np.minimum(phi, d)
    return phi


@pytest.mark.parametrize("tape", [False, True])
@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_sources_heterogeneous(fmm, oracle, schedule, dt, tape):
    shape, F, src = _sources_problem()
    ref = oracle.solve_sources(shape, src, H3, speed=_q(F, dt))
    Fd = torch.as_tensor(F, dtype=DT[dt], device="cuda")
    with fmm.Solver(shape, H3, dtype=DT[dt], speed=Fd, sources=src, schedule=schedule,
                    record_tape=tape) as s:
        T, G = s.solve()
        assert s.stats()["error_flags"] == 0
    compare(_host(T), _host(G), ref, dt)


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_reinit_spheres(fmm, oracle, schedule, dt):
    shape = (31, 27, 36)
    phi = _spheres_phi(shape)
    ref = oracle.solve_reinit(_q(phi, dt), H3)
    with fmm.Solver(shape, H3, dtype=DT[dt], schedule=schedule) as s:
        T, G = s.reinit(torch.as_tensor(phi, dtype=DT[dt], device="cuda"))
    compare(_host(T), _host(G), ref, dt)


def test_point_source_axes_exact(fmm):
    """Along the grid lines through a point source psi is k * dx, k * dy,
    k * dz to rounding (the 1-D root of each axis)."""
    shape = (21, 23, 25)
    with fmm.Solver(shape, H3, dtype=torch.float64, sources=[(12, 11, 10)]) as s:
        T, _ = s.solve()
    T = _host(T)
    k = np.arange(-10, 11)
    assert np.max(np.abs(T[10, 11, 12 + k[2:]] - np.abs(k[2:]) * H3[0])) < 1e-14
    assert np.max(np.abs(T[10, 11 + k[1:], 12] - np.abs(k[1:]) * H3[1])) < 1e-14
    assert np.max(np.abs(T[10 + k, 11, 12] - np.abs(k) * H3[2])) < 1e-14


def test_adjoint_fp64(fmm, oracle):
    shape, F, src = _sources_problem(seed=8, shape=(22, 25, 20))
    rng = np.random.default_rng(3)
    rec = wl.random_cells(rng, shape, 8, exclude=src)
    g = np.zeros(shape)
    for i, j, k in rec:
        g[k, j, i] += 1.0
    Fd = torch.as_tensor(F, dtype=torch.float64, device="cuda")
    with fmm.Solver(shape, H3, dtype=torch.float64, speed=Fd, sources=src, record_tape=True) as s:
        s.solve()
        d = _host(s.adjoint(torch.as_tensor(g, device="cuda")))
    r = oracle.solve_sources(shape, src, H3, speed=F, record=True)
    d_ref, _ = oracle.adjoint(r, H3, g, speed=F)
    assert np.max(np.abs(d - d_ref)) <= 1e-11 * np.max(np.abs(d_ref))


def test_noalloc_entry_point(fmm, oracle):
    shape = (24, 20, 32)
    phi = _spheres_phi(shape, seed=9, count=2)
    T = torch.empty(shape, dtype=torch.float64, device="cuda")
    G = torch.empty(shape, dtype=torch.uint8, device="cuda")
    fmm.reinit_noalloc(torch.as_tensor(phi, device="cuda"), H3, T, G)
    compare(_host(T), _host(G), oracle.solve_reinit(phi, H3), "f64")


def test_spacing_arguments_checked(fmm):
    with pytest.raises(fmm.FmmError) as e:
        fmm.Solver((8, 8, 8), (0.1, -0.1, 0.1))
    assert e.value.code == fmm.FMM_ERR_INVALID
    # a checkpoint records the cell sizes
    phi = torch.as_tensor(_spheres_phi((16, 16, 16), seed=2, count=1), dtype=torch.float32,
                          device="cuda")
    with fmm.Solver((16, 16, 16), H3) as s:
        s.reinit(phi)
        image = s.checkpoint()
    with fmm.Solver((16, 16, 16), (H3[0], H3[1], H3[1])) as s2:
        with pytest.raises(fmm.FmmError) as e:
            s2.restore(image)
        assert e.value.code == fmm.FMM_ERR_INVALID


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_extreme_aspect_ratios(fmm, oracle, dt):
    """dy = 8 dx and dz = dx / 5 (weights 1/64 and 25 in Algorithm 11)."""
    h3 = (1.0 / 40, 8.0 / 40, 0.2 / 40)
    tdt = DT[dt]
    shape = (30, 12, 33)
    rng = np.random.default_rng(17)
    F = wl.fourier_speed(shape, wl.draw_fourier_modes(rng), h=h3)
    src = wl.random_cells(rng, shape, 2)
    ref = oracle.solve_sources(shape, src, h3, speed=_q(F, dt))
    with fmm.Solver(shape, h3, dtype=tdt, speed=torch.as_tensor(F, dtype=tdt, device="cuda"),
                    sources=src) as s:
        T, G = s.solve()
    compare(_host(T), _host(G), ref, dt)
    x, y, z = wl._axes(shape, h3)
    c = np.array([0.5 * shape[2] * h3[0], 0.5 * shape[1] * h3[1], 0.5 * shape[0] * h3[2]])
    phi = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) - 0.35
    ref = oracle.solve_reinit(_q(phi, dt), h3)
    with fmm.Solver(shape, h3, dtype=tdt) as s:
        T, G = s.reinit(torch.as_tensor(phi, dtype=tdt, device="cuda"))
    compare(_host(T), _host(G), ref, dt)
