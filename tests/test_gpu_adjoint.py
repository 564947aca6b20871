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
    assert np.max(np.abs(d_gpu - d_ref)) <= 1e-12 * scale
    assert st["adjoint_iterations"] >= 1


def test_adjoint_dense_cotangent_fp64(fmm, oracle):
    p, _ = _problem(20, 7)
    rng = np.random.default_rng(9)
    g = rng.standard_normal(p.shape)
    _, _, d_gpu, _ = _gpu_adjoint(fmm, p, g)
    r = oracle.solve_sources(p.shape, p.sources, p.h, speed=p.speed, record=True)
    d_ref, _ = oracle.adjoint(r, p.h, g, speed=p.speed)
    assert np.max(np.abs(d_gpu - d_ref)) <= 1e-12 * np.max(np.abs(d_ref))
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
    assert np.max(np.abs(d_gpu - d_ref)) <= 1e-12 * np.max(np.abs(d_ref))


@pytest.mark.parametrize("n,seed", [(24, 3), (33, 5)])
def test_adjoint_fp32_cell_by_cell(fmm, oracle, n, seed):
    """fp32 adjoint against the oracle's fp64 adjoint on the same (float)
    speed field, cell by cell: |dL/ds_gpu - dL/ds_oracle| <= 1e-4 max|dL/ds|
    at every cell.  The bound comes from the forward rounding: fp32 psi
    carries a relative error of ~2^-24 psi, so each difference psi_p - psi_i
    ~ h/F of the reverse sweep carries ~2^-24 psi F / h relative error
    (~1e-6 at n = 33), and the sweep sums such terms along upwind paths of
    up to ~n cells (measured worst: 1.2e-6 at n = 24, 1.1e-5 at n = 33)."""
    p, g = _problem(n, seed)
    F32 = np.asarray(p.speed, np.float32)
    _, _, d_gpu, _ = _gpu_adjoint(fmm, p, g, dtype=torch.float32, speed=F32)
    r = oracle.solve_sources(p.shape, p.sources, p.h, speed=F32.astype(np.float64), record=True)
    d_ref, _ = oracle.adjoint(r, p.h, g, speed=F32.astype(np.float64))
    scale = np.max(np.abs(d_ref))
    worst = float(np.max(np.abs(d_gpu.astype(np.float64) - d_ref)))
    assert worst <= 1e-4 * scale, (worst / scale)
    # cells the oracle gives no gradient (FIX, unreached) get none
    assert np.all(d_gpu[d_ref == 0] == 0)


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
    assert np.max(np.abs(d - d_ref)) <= 1e-12 * np.max(np.abs(d_ref))
    solver.close()


def test_adjoint_finite_differences_512_fp64(fmm):
    """The bench's adjoint workload in full (512^3, Fourier speed, 8 sources,
    64 receivers, fp64, library defaults): dL/ds from fmm_adjoint against
    central differences of L(s) along two smooth random directions, each
    from two GPU forward solves (a property that holds at any size)."""
    p = wl.fourier_sources(n=512, n_sources=8, n_receivers=64, seed=3, device="cuda")
    F = p.speed.to(torch.float64).contiguous()
    rec = torch.as_tensor(np.asarray(p.receivers), device="cuda")
    g = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    g[rec[:, 2], rec[:, 1], rec[:, 0]] = 1.0
    with fmm.Solver(p.shape, p.h, dtype=torch.float64, speed=F, sources=p.sources,
                    record_tape=True) as s:
        s.solve(want_tags=False)
        dLds = s.adjoint(g)
    s0 = 1.0 / F

    def L(slow):
        with fmm.Solver(p.shape, p.h, dtype=torch.float64, speed=(1.0 / slow).contiguous(),
                        sources=p.sources) as sv:
            T, _ = sv.solve(want_tags=False)
        return float(T[rec[:, 2], rec[:, 1], rec[:, 0]].sum())

    n = p.shape[0]
    x = (torch.arange(n, device="cuda", dtype=torch.float64) + 0.5) / n
    for kx, ky, kz in ((1, 2, 3), (3, 1, 2)):
        v = (torch.sin(2 * np.pi * kx * x)[None, None, :] * torch.cos(2 * np.pi * ky * x)[None, :, None]
             * torch.sin(2 * np.pi * kz * x + 0.3)[:, None, None])
        eps = 1e-6 * float(torch.linalg.vector_norm(s0)) / float(torch.linalg.vector_norm(v))
        fd = (L(s0 + eps * v) - L(s0 - eps * v)) / (2 * eps)
        ad = float((dLds * v).sum())
        assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_every_accepted_cell_is_ordered_256(fmm, dt):
    """The reverse sweep reaches every accepted cell only if the recorded
    upwind sets point strictly downhill (no cell lists a neighbour at or
    above its own value); a causality test on rounded shifted values once
    let a 256^3 heterogeneous solve record such a pair in about a third of
    the runs, and the adjoint then stopped with cells it could not order.
    Repeated forward + adjoint runs of that workload must all complete."""
    p = wl.fourier_sources(n=256, n_sources=8, n_receivers=64, seed=3, device="cuda")
    F = p.speed.to(dt).contiguous()
    g = torch.zeros(p.shape, dtype=dt, device="cuda")
    for i, j, k in p.receivers:
        g[k, j, i] += 1.0
    with fmm.Solver(p.shape, p.h, dtype=dt, speed=F, sources=p.sources, record_tape=True,
                    tuned=False) as s:
        for _ in range(6):
            s.solve()
            d = s.adjoint(g)
            assert torch.isfinite(d).all()
