"""GPU adjoint (dL/d slowness) against the oracle's CPU adjoint and against
central finite differences of the GPU forward solve."""
import math

import numpy as np
import pytest
import torch

from paper_1502_07303_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")
    from paper_1502_07303_gb300 import fmm as _fmm
    return _fmm


def _problem(n, seed, n_src=3, n_rec=8):
    p = wl.fourier_sources(n=n, n_sources=n_src, n_receivers=n_rec, seed=seed)
    g = np.zeros(p.shape)
    for i, j, k in p.receivers:
        g[k, j, i] += 1.0
    return p, g


def _gpu_adjoint(fmm, p, g, dtype=torch.float64, speed=None):
    F = torch.as_tensor(p.speed if speed is None else speed, dtype=dtype, device="cuda")
    with fmm.Solver(p.shape, p.h, dtype=dtype, speed=F, sources=p.sources, record_tape=True) as s:
        T, G = s.solve()
        d = s.adjoint(torch.as_tensor(g, dtype=dtype, device="cuda"))
        st = s.stats()
    return T.cpu().numpy(), G.cpu().numpy(), d.cpu().numpy(), st


@pytest.mark.parametrize("n,seed", [(24, 3), (33, 5)])
def test_adjoint_matches_oracle_fp64(fmm, oracle, n, seed):
    p, g = _problem(n, seed)
    _, _, d_gpu, st = _gpu_adjoint(fmm, p, g)
    r = oracle.solve_sources(p.shape, p.sources, p.h, speed=p.speed, record=True)
    d_ref, _ = oracle.adjoint(r, p.h, g, speed=p.speed)
    scale = np.max(np.abs(d_ref))
    assert scale > 0
    assert np.max(np.abs(d_gpu - d_ref)) <= 1e-11 * scale
    assert st["adjoint_iterations"] >= 1


def test_adjoint_dense_cotangent_fp64(fmm, oracle):
    p, _ = _problem(20, 7)
    rng = np.random.default_rng(9)
    g = rng.standard_normal(p.shape)
    _, _, d_gpu, _ = _gpu_adjoint(fmm, p, g)
    r = oracle.solve_sources(p.shape, p.sources, p.h, speed=p.speed, record=True)
    d_ref, _ = oracle.adjoint(r, p.h, g, speed=p.speed)
    assert np.max(np.abs(d_gpu - d_ref)) <= 1e-11 * np.max(np.abs(d_ref))
    # FIX cells (the sources) get no gradient
    for i, j, k in p.sources:
        assert d_gpu[k, j, i] == 0.0


def test_adjoint_finite_differences_gpu_forward(fmm):
    """dL/ds from fmm_adjoint against central differences of L(s) computed with
    the GPU forward solve (fp64, 32^3 copy of the heterogeneous-speed case)."""
    p, g = _problem(32, 3, n_src=8, n_rec=16)
    s0 = 1.0 / p.speed
    _, _, dLds, _ = _gpu_adjoint(fmm, p, g)
    rng = np.random.default_rng(4)

    def L(s):
        F = torch.as_tensor(1.0 / s, dtype=torch.float64, device="cuda")
        with fmm.Solver(p.shape, p.h, dtype=torch.float64, speed=F, sources=p.sources) as sv:
            T, _ = sv.solve(want_tags=False)
        T = T.cpu().numpy()
        return float(sum(T[k, j, i] for i, j, k in p.receivers))

    for _ in range(4):
        v = rng.standard_normal(p.shape)
        eps = 1e-6 * np.linalg.norm(s0) / np.linalg.norm(v)
        fd = (L(s0 + eps * v) - L(s0 - eps * v)) / (2 * eps)
        ad = float(np.sum(dLds * v))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_adjoint_two_sided_reinit_fp64(fmm, oracle):
    """Adjoint of a reinitialisation (both signs) with respect to the slowness
    of every cell; the front cells are FIX and get zero."""
    pr = wl.random_spheres(shape=(28, 30, 26), count=4, seed=12)
    rng = np.random.default_rng(2)
    g = rng.standard_normal(pr.shape)
    phi = torch.as_tensor(pr.phi0, dtype=torch.float64, device="cuda")
    with fmm.Solver(pr.shape, pr.h, dtype=torch.float64, record_tape=True) as s:
        s.reinit(phi)
        d_gpu = s.adjoint(torch.as_tensor(g, device="cuda")).cpu().numpy()
    r = oracle.solve_reinit(pr.phi0, pr.h, record=True)
    d_ref, _ = oracle.adjoint(r, pr.h, g)
    assert np.max(np.abs(d_gpu - d_ref)) <= 1e-11 * np.max(np.abs(d_ref))


def test_adjoint_fp32_close_to_oracle(fmm, oracle):
    p, g = _problem(24, 3)
    F32 = np.asarray(p.speed, np.float32)
    _, _, d_gpu, _ = _gpu_adjoint(fmm, p, g, dtype=torch.float32, speed=F32)
    r = oracle.solve_sources(p.shape, p.sources, p.h, speed=F32.astype(np.float64), record=True)
    d_ref, _ = oracle.adjoint(r, p.h, g, speed=F32.astype(np.float64))
    err = np.linalg.norm(d_gpu - d_ref) / np.linalg.norm(d_ref)
    assert err < 1e-3, err


def test_adjoint_requires_tape(fmm):
    p = wl.point_source(16)
    with fmm.Solver(p.shape, p.h, dtype=torch.float64, sources=p.sources) as s:
        s.solve()
        with pytest.raises(fmm.FmmError) as e:
            s.adjoint(torch.zeros(p.shape, dtype=torch.float64, device="cuda"))
        assert e.value.code == fmm.FMM_ERR_STATE


def test_eikonal_autograd_function(fmm, oracle):
    p, g = _problem(20, 11)
    s0 = torch.as_tensor(1.0 / p.speed, dtype=torch.float64, device="cuda").requires_grad_(True)
    solver = fmm.Solver(p.shape, p.h, dtype=torch.float64, sources=p.sources, record_tape=True)
    T = fmm.EikonalFn.apply(s0, solver)
    loss = (T * torch.as_tensor(g, device="cuda")).sum()
    loss.backward()
    r = oracle.solve_sources(p.shape, p.sources, p.h, speed=p.speed, record=True)
    d_ref, _ = oracle.adjoint(r, p.h, g, speed=p.speed)
    d = s0.grad.cpu().numpy()
    assert np.max(np.abs(d - d_ref)) <= 1e-11 * np.max(np.abs(d_ref))
    solver.close()
