"""Deterministic mode (fmm_config.deterministic): the phased schedule of
Algorithm 16 with every march pass reading its neighbours' boundary values
as they stood at the end of the previous pass, the paper's synchronous
exchange once per pass (Sec. 4.3, Algorithms 13-16).  The result must be the
same bit for bit for any number of CTAs and across a stop and resume, and
within the parity tolerance of the oracle."""
import numpy as np
import pytest
import torch

from paper_1502_07303_gb300 import workloads as wl
from parity_util import compare

pytestmark = pytest.mark.gpu

DT = {"f32": torch.float32, "f64": torch.float64}


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")
    from paper_1502_07303_gb300 import fmm as _fmm
    return _fmm


def _q(a, dt):
    """The oracle's copy of an input the GPU sees in precision dt."""
    a = np.asarray(a, np.float64)
    return a.astype(np.float32).astype(np.float64) if dt == "f32" else a


def _same_bits(a, b):
    ta, tb = a.cpu(), b.cpu()
    return ta.dtype == tb.dtype and ta.shape == tb.shape and \
        ta.contiguous().view(torch.uint8).equal(tb.contiguous().view(torch.uint8))


def _f64(t):
    return t.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_reinit_is_the_same_for_every_cta_count(fmm, oracle, dt):
    p = wl.random_spheres(shape=(45, 38, 51), count=6, seed=31)   # ragged bricks
    phi = torch.as_tensor(p.phi0, dtype=DT[dt], device="cuda")
    runs = []
    for ctas in (0, 152, 37, 0):
        with fmm.Solver(p.shape, p.h, dtype=DT[dt], deterministic=True, ctas=ctas, stride=1.0) as s:
            runs.append(s.reinit(phi))
            assert s.stats()["error_flags"] == 0
    for T, G in runs[1:]:
        assert _same_bits(T, runs[0][0]) and _same_bits(G, runs[0][1])
    compare(_f64(runs[0][0]), runs[0][1].cpu().numpy(), oracle.solve_reinit(_q(p.phi0, dt), p.h), dt)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_heterogeneous_sources_are_the_same_for_every_cta_count(fmm, oracle, dt):
    p = wl.fourier_sources(n=41, n_sources=4, n_receivers=8, seed=32)
    sp = torch.as_tensor(p.speed, dtype=DT[dt], device="cuda")
    runs = []
    for ctas in (0, 304, 19):
        with fmm.Solver(p.shape, p.h, dtype=DT[dt], speed=sp, sources=p.sources, deterministic=True,
                        ctas=ctas, stride=2.0, exchange_passes=2) as s:
            runs.append(s.solve())
    for T, G in runs[1:]:
        assert _same_bits(T, runs[0][0]) and _same_bits(G, runs[0][1])
    ref = oracle.solve_sources(p.shape, p.sources, p.h, speed=_q(p.speed, dt))
    compare(_f64(runs[0][0]), runs[0][1].cpu().numpy(), ref, dt)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_resumed_solve_is_the_uninterrupted_one(fmm, dt):
    """Stopped by its restart limit and resumed (the faces are rebuilt from
    the stopped state), the solve gives the bits of one uninterrupted run."""
    p = wl.random_spheres(n=33, count=5, seed=33)
    phi = torch.as_tensor(p.phi0, dtype=DT[dt], device="cuda")
    with fmm.Solver(p.shape, p.h, dtype=DT[dt], deterministic=True, stride=1.0) as s:
        T0, G0 = s.reinit(phi)
    with fmm.Solver(p.shape, p.h, dtype=DT[dt], deterministic=True, stride=1.0, max_restarts=4) as s:
        with pytest.raises(fmm.FmmError) as e:
            s.reinit(phi)
        assert e.value.code == fmm.FMM_ERR_TIMEOUT
        T1, G1 = s.resume()
    assert _same_bits(T1, T0) and _same_bits(G1, G0)


def test_adjoint_of_a_deterministic_solve_repeats(fmm):
    """The adjoint sums in a fixed order, so with a reproducible forward
    solve the whole forward + adjoint pair repeats bit for bit."""
    p = wl.fourier_sources(n=29, n_sources=3, n_receivers=6, seed=34)
    sp = torch.as_tensor(p.speed, dtype=torch.float64, device="cuda")
    dLdT = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    for i, j, k in p.receivers:
        dLdT[k, j, i] = 1.0
    grads = []
    for ctas in (0, 76):
        with fmm.Solver(p.shape, p.h, dtype=torch.float64, speed=sp, sources=p.sources,
                        deterministic=True, record_tape=True, ctas=ctas) as s:
            s.solve()
            grads.append(s.adjoint(dLdT))
    assert _same_bits(grads[0], grads[1])
