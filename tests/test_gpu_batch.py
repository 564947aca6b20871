"""Batched reinitialisation (fmm_create_batch / fmm_reinit_batch): every grid
of a batch of uneven sizes against the oracle, with the tolerances of the
single-grid parity tests."""
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


def _batch(n_grids, lo, hi, seed):
    return wl.batch(n_grids=n_grids, lo=lo, hi=hi, seed=seed)


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_batch_matches_oracle(fmm, oracle, dt):
    probs = _batch(9, 5, 41, seed=14)
    phis = [torch.as_tensor(p.phi0, dtype=DT[dt], device="cuda").contiguous() for p in probs]
    with fmm.Batch([p.shape for p in probs], [p.h for p in probs], dtype=DT[dt]) as b:
        Ts, Gs = b.reinit(phis)
        st = b.stats()
    assert st["error_flags"] == 0
    for p, T, G in zip(probs, Ts, Gs):
        phi_q = np.asarray(p.phi0, np.float32).astype(np.float64) if dt == "f32" else p.phi0
        ref = oracle.solve_reinit(phi_q, p.h)
        compare(T.cpu().numpy(), G.cpu().numpy(), ref, dt)


def test_batch_grids_do_not_interact(fmm, oracle):
    """Two copies of the same problem next to a different one give the same
    result as one copy alone (no data crosses between grids)."""
    a = wl.random_spheres(shape=(24, 17, 33), count=3, seed=3)
    c = wl.random_spheres(shape=(16, 40, 9), count=2, seed=4)
    probs = [a, c, a]
    phis = [torch.as_tensor(p.phi0, dtype=torch.float64, device="cuda") for p in probs]
    with fmm.Batch([p.shape for p in probs], [p.h for p in probs], dtype=torch.float64) as b:
        Ts, Gs = b.reinit(phis)
    for k in (0, 2):
        ref = oracle.solve_reinit(a.phi0, a.h)
        compare(Ts[k].cpu().numpy(), Gs[k].cpu().numpy(), ref, "f64")
    assert torch.equal(Gs[0], Gs[2])


def test_batch_repeat_and_single_grid(fmm, oracle):
    p = wl.random_spheres(shape=(20, 20, 20), count=2, seed=8)
    phi = torch.as_tensor(p.phi0, dtype=torch.float32, device="cuda")
    with fmm.Batch([p.shape], [p.h], dtype=torch.float32) as b:
        T1, G1 = b.reinit([phi])
        T2, G2 = b.reinit([phi])
    assert torch.equal(G1[0], G2[0])
    ref = oracle.solve_reinit(np.asarray(p.phi0, np.float32).astype(np.float64), p.h)
    compare(T2[0].cpu().numpy(), G2[0].cpu().numpy(), ref, "f32")


def test_batch_handle_rejects_single_grid_calls(fmm):
    with fmm.Batch([(8, 8, 8)], [0.1], dtype=torch.float32) as b:
        s = fmm.Solver.__new__(fmm.Solver)
        s.lib, s.handle, s.shape, s.dtype = b.lib, b.handle, (8, 8, 8), torch.float32
        with pytest.raises(fmm.FmmError) as e:
            s.solve()
        assert e.value.code == fmm.FMM_ERR_STATE
        s.handle = None


def test_bench_batch_256_grids_sampled(fmm, oracle):
    """The bench's batched workload in full (256 grids, axes in [32, 192],
    fp32, one batch handle, library defaults): six of the smaller grids
    element by element against the oracle; every grid whose phi0 changes sign
    fully accepted, every other grid (its spheres lie outside a thin grid)
    entirely FAR."""
    probs = wl.batch(n_grids=256, lo=32, hi=192, seed=4, device="cuda")
    phis = [p.phi0.to(torch.float32).contiguous() for p in probs]
    with fmm.Batch([p.shape for p in probs], [p.h for p in probs], dtype=torch.float32) as b:
        Ts, Gs = b.reinit(phis)
        st = b.stats()
    assert st["error_flags"] == 0
    for p, phi, G in zip(probs, phis, Gs):
        front = bool((phi > 0).any()) and bool((phi <= 0).any())
        if front:
            assert int((G == 0).sum()) == 0 and int((G == 1).sum()) == 0, p.name
        else:
            assert int((G != 0).sum()) == 0, p.name
    order = sorted(range(len(probs)), key=lambda i: probs[i].n_points)
    for i in order[:6]:
        p = probs[i]
        phi_q = p.phi0.to(torch.float32).to(torch.float64).cpu().numpy()
        ref = oracle.solve_reinit(phi_q, p.h)
        compare(Ts[i].cpu().numpy(), Gs[i].cpu().numpy(), ref, "f32")
