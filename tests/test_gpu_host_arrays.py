"""Host arrays through the C ABI: the entry points copy page-locked or
pageable host inputs to the device and host outputs back before they return;
results must match the oracle as device arrays do."""
import numpy as np
import pytest
import torch

from paper_1502_07303_gb300 import workloads as wl
from parity_util import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")
    from paper_1502_07303_gb300 import fmm as _fmm
    return _fmm


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_reinit_with_host_arrays(fmm, oracle, dt, pinned):
    tdt = torch.float64 if dt == "f64" else torch.float32
    p = wl.random_spheres(n=37, count=4, seed=12)
    phi = torch.as_tensor(p.phi0, dtype=tdt)
    T = torch.empty(p.shape, dtype=tdt)
    G = torch.empty(p.shape, dtype=torch.uint8)
    if pinned:
        phi, T, G = phi.pin_memory(), T.pin_memory(), G.pin_memory()
    with fmm.Solver(p.shape, p.h, dtype=tdt) as s:
        s.reinit(phi, T, G)
        # a device phi0 with host outputs, and the other way round
        Td = torch.empty(p.shape, dtype=tdt, device="cuda")
        T2 = torch.empty(p.shape, dtype=tdt)
        s.reinit(phi.cuda(), T2, None, want_tags=False)
        s.reinit(phi, Td, None, want_tags=False)
    phi_q = np.asarray(p.phi0, np.float32).astype(np.float64) if dt == "f32" else p.phi0
    ref = oracle.solve_reinit(phi_q, p.h)
    compare(T.numpy().astype(np.float64), G.numpy(), ref, dt)
    for X in (T2.numpy(), Td.cpu().numpy()):
        fin = np.isfinite(ref["T"])
        assert np.max(np.abs(X.astype(np.float64)[fin] - ref["T"][fin])) <= \
            (1e-12 if dt == "f64" else 2e-5) * np.max(np.abs(ref["T"][fin]))


def test_speed_solve_and_adjoint_with_host_arrays(fmm, oracle):
    pr = wl.fourier_sources(n=29, n_sources=3, n_receivers=8, seed=13)
    F = torch.as_tensor(pr.speed, dtype=torch.float64)          # host speed
    g = torch.zeros(pr.shape, dtype=torch.float64)
    for i, j, k in pr.receivers:
        g[k, j, i] += 1.0
    with fmm.Solver(pr.shape, pr.h, dtype=torch.float64, speed=F, sources=pr.sources,
                    record_tape=True) as s:
        T = torch.empty(pr.shape, dtype=torch.float64).pin_memory()
        G = torch.empty(pr.shape, dtype=torch.uint8)
        s.solve(T, G)
        d = s.adjoint(g)                                       # host in, host out
        assert d.device.type == "cpu"
        d_dev = s.adjoint(g.cuda())
    r = oracle.solve_sources(pr.shape, pr.sources, pr.h, speed=pr.speed, record=True)
    compare(T.numpy(), G.numpy(), r, "f64")
    d_ref, _ = oracle.adjoint(r, pr.h, g.numpy(), speed=pr.speed)
    assert np.max(np.abs(d.numpy() - d_ref)) <= 1e-11 * np.max(np.abs(d_ref))
    assert torch.equal(d, d_dev.cpu())                         # same arithmetic
