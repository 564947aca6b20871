"""Resuming a solve stopped by its restart limit, and checkpoints of solve
states: both must reach the oracle's fixed point, as one uninterrupted solve
does (Algorithm 16 is correct from any restart boundary)."""
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


def _host(t):
    return t.cpu().numpy().astype(np.float64) if t.dtype != torch.uint8 else t.cpu().numpy()


def _spheres(dt):
    p = wl.random_spheres(n=29, count=5, seed=4)
    phi_q = np.asarray(p.phi0, np.float32).astype(np.float64) if dt == "f32" else p.phi0
    return p, phi_q


def _stopped(fmm, s, call):
    with pytest.raises(fmm.FmmError) as e:
        call()
    assert e.value.code == fmm.FMM_ERR_TIMEOUT
    return s.stats()["restarts"]


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_resume_after_restart_limit(fmm, oracle, dt, schedule):
    p, phi_q = _spheres(dt)
    ref = oracle.solve_reinit(phi_q, p.h)
    phi = torch.as_tensor(p.phi0, dtype=DT[dt], device="cuda")
    with fmm.Solver(p.shape, p.h, dtype=DT[dt], schedule=schedule, stride=1.0,
                    max_restarts=3) as s:
        r0 = _stopped(fmm, s, lambda: s.reinit(phi))
        T, G = s.resume()
        st = s.stats()
    assert st["error_flags"] == 0 and st["restarts"] > r0
    compare(_host(T), _host(G), ref, dt)


@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_resume_in_steps(fmm, oracle, schedule):
    """Point sources with heterogeneous speed, resumed two restarts at a time."""
    p = wl.fourier_sources(n=33, n_sources=4, n_receivers=8, seed=5)
    ref = oracle.solve_sources(p.shape, p.sources, p.h, speed=p.speed)
    F = torch.as_tensor(p.speed, dtype=torch.float64, device="cuda")
    with fmm.Solver(p.shape, p.h, dtype=torch.float64, speed=F, sources=p.sources,
                    schedule=schedule, stride=0.5, max_restarts=2) as s:
        last = _stopped(fmm, s, s.solve)
        steps = 0
        while True:
            try:
                T, G = s.resume(more_restarts=2)
                break
            except fmm.FmmError as e:
                assert e.code == fmm.FMM_ERR_TIMEOUT
                now = s.stats()["restarts"]
                assert now > last
                last = now
                steps += 1
                assert steps < 1000
    assert steps >= 2
    compare(_host(T), _host(G), ref, "f64")


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_checkpoint_of_a_stopped_solve_resumes_in_another_handle(fmm, oracle, dt, schedule):
    p, phi_q = _spheres(dt)
    ref = oracle.solve_reinit(phi_q, p.h)
    phi = torch.as_tensor(p.phi0, dtype=DT[dt], device="cuda")
    kw = dict(dtype=DT[dt], schedule=schedule, stride=1.0)
    with fmm.Solver(p.shape, p.h, max_restarts=4, **kw) as s:
        _stopped(fmm, s, lambda: s.reinit(phi))
        image = s.checkpoint()
    with fmm.Solver(p.shape, p.h, **kw) as s2:
        s2.restore(image)
        T, G = s2.resume()
        assert s2.stats()["error_flags"] == 0
    compare(_host(T), _host(G), ref, dt)


def test_checkpoint_of_a_finished_solve_keeps_the_tape(fmm):
    """A finished solve with a tape, restored into a new handle, gives the
    same adjoint (bit for bit: same forward state, fixed summation order)."""
    p = wl.fourier_sources(n=30, n_sources=3, n_receivers=8, seed=6)
    F = torch.as_tensor(p.speed, dtype=torch.float64, device="cuda")
    g = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    for i, j, k in p.receivers:
        g[k, j, i] += 1.0
    kw = dict(dtype=torch.float64, speed=F, sources=p.sources, record_tape=True)
    with fmm.Solver(p.shape, p.h, **kw) as s:
        s.solve()
        d1 = s.adjoint(g)
        image = s.checkpoint()          # after the adjoint: the forward state is kept
        d1b = s.adjoint(g)
        with pytest.raises(fmm.FmmError) as e:
            s.resume()                   # finished: nothing to resume
        assert e.value.code == fmm.FMM_ERR_STATE
    assert torch.equal(d1, d1b)         # the adjoint is deterministic
    with fmm.Solver(p.shape, p.h, **kw) as s2:
        s2.restore(image)
        d2 = s2.adjoint(g)
    assert torch.equal(d1, d2)


def test_adjoint_refused_after_a_stopped_solve(fmm, oracle):
    p = wl.fourier_sources(n=30, n_sources=3, n_receivers=8, seed=6)
    F = torch.as_tensor(p.speed, dtype=torch.float64, device="cuda")
    g = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    for i, j, k in p.receivers:
        g[k, j, i] += 1.0
    gh = g.cpu().numpy()
    with fmm.Solver(p.shape, p.h, dtype=torch.float64, speed=F, sources=p.sources,
                    record_tape=True, stride=0.5, max_restarts=2) as s:
        _stopped(fmm, s, s.solve)
        with pytest.raises(fmm.FmmError) as e:
            s.adjoint(g)                 # the tape is incomplete
        assert e.value.code == fmm.FMM_ERR_STATE
        s.resume()
        d = s.adjoint(g).cpu().numpy()
    r = oracle.solve_sources(p.shape, p.sources, p.h, speed=p.speed, record=True)
    d_ref, _ = oracle.adjoint(r, p.h, gh, speed=p.speed)
    assert np.max(np.abs(d - d_ref)) <= 1e-11 * np.max(np.abs(d_ref))


def test_checkpoint_load_checks_the_handle(fmm):
    p, _ = _spheres("f32")
    phi = torch.as_tensor(p.phi0, dtype=torch.float32, device="cuda")
    with fmm.Solver(p.shape, p.h, dtype=torch.float32) as s:
        with pytest.raises(fmm.FmmError) as e:
            s.checkpoint()               # nothing solved yet
        assert e.value.code == fmm.FMM_ERR_STATE
        s.reinit(phi)
        image = s.checkpoint()
    nz, ny, nx = p.shape
    with fmm.Solver((nz, ny, nx + 1), p.h, dtype=torch.float32) as s2:
        with pytest.raises(fmm.FmmError) as e:
            s2.restore(image)            # another grid (a different image size)
        assert e.value.code == fmm.FMM_ERR_INVALID
    with fmm.Solver(p.shape, p.h, dtype=torch.float64) as s3:
        with pytest.raises(fmm.FmmError) as e:
            s3.restore(image)            # another dtype
        assert e.value.code == fmm.FMM_ERR_INVALID
    with fmm.Solver(p.shape, p.h, dtype=torch.float32) as s4:
        bad = image.copy()
        bad[0] ^= 0xFF                   # not an image of this library
        with pytest.raises(fmm.FmmError) as e:
            s4.restore(bad)
        assert e.value.code == fmm.FMM_ERR_INVALID
        with pytest.raises(fmm.FmmError) as e:
            s4.restore(image[:40])       # truncated
        assert e.value.code == fmm.FMM_ERR_INVALID
        s4.restore(image)
        with pytest.raises(fmm.FmmError) as e:
            s4.resume()                  # the image is of a finished solve
        assert e.value.code == fmm.FMM_ERR_STATE
