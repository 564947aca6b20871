"""Domain decomposition across ranks with the CUDA library doing every
rank's local march (fmm_dd_* entry points, paper_1502_07303_gb300/decomp.py):
the ranks are stepped one after another in one process on one GPU (each
rank's kernels finish before the next rank's start; no kernel waits on
another rank), and the assembled solution is compared element by element
with the oracle's sequential solution of the whole grid (Sec. 5.2: the
decomposed method reproduces the sequential one)."""
import math

import numpy as np
import pytest
import torch

from paper_1502_07303_gb300 import decomp
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
    return np.asarray(a, np.float32).astype(np.float64) if dt == "f32" else np.asarray(a, np.float64)


@pytest.mark.parametrize("n_ranks,stride,ghost", [(2, 2.0, 1), (3, 1.0, 1), (4, math.inf, 1),
                                                  (3, 2.0, 2)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_decomposed_reinit_matches_oracle(fmm, oracle, dt, n_ranks, stride, ghost):
    p = wl.random_spheres(shape=(45, 37, 30), count=5, seed=61)
    phi = torch.as_tensor(p.phi0, dtype=DT[dt], device="cuda")
    subs = [decomp.Subdomain(p.shape[0], n_ranks, r, ghost) for r in range(n_ranks)]
    ms = [decomp.GpuMarcher(s, p.shape, p.h, DT[dt], phi0=phi) for s in subs]
    try:
        results, restarts = decomp.solve_serial(ms, subs, stride * p.h)
        T, G = decomp.assemble(subs, results, p.shape)
    finally:
        for m in ms:
            m.close()
    compare(T.cpu().numpy(), G.cpu().numpy(), oracle.solve_reinit(_q(p.phi0, dt), p.h), dt)
    assert restarts >= 1


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_decomposed_sources_with_speed_match_oracle(fmm, oracle, dt):
    rng = np.random.default_rng(62)
    shape = (50, 30, 26)
    h = wl.spacing(shape)
    F = wl.fourier_speed(shape, wl.draw_fourier_modes(rng), h=h)
    src = wl.random_cells(rng, shape, 4)
    Fd = torch.as_tensor(F, dtype=DT[dt], device="cuda")
    subs = [decomp.Subdomain(shape[0], 3, r) for r in range(3)]
    ms = [decomp.GpuMarcher(s, shape, h, DT[dt], speed=Fd, sources=src) for s in subs]
    try:
        results, _ = decomp.solve_serial(ms, subs, 2.0 * h)
        T, G = decomp.assemble(subs, results, shape)
    finally:
        for m in ms:
            m.close()
    compare(T.cpu().numpy(), G.cpu().numpy(), oracle.solve_sources(shape, src, h, speed=_q(F, dt)), dt)


def test_dd_entry_points_check_their_arguments(fmm):
    import ctypes
    with fmm.Solver((16, 8, 8), 0.1, dtype=torch.float64, sources=[[1, 1, 1]]) as s:
        buf = torch.empty((2, 8, 8), dtype=torch.float64, device="cuda")
        rc = s.lib.fmm_dd_get_layers(s.handle, 0, 2, ctypes.c_void_p(buf.data_ptr()))
        assert rc == fmm.FMM_ERR_STATE                  # before fmm_dd_start
        assert s.lib.fmm_dd_start(s.handle, None, 0, 0) == fmm.FMM_OK
        assert s.lib.fmm_dd_get_layers(s.handle, 15, 2, ctypes.c_void_p(buf.data_ptr())) == \
            fmm.FMM_ERR_INVALID                          # past the last layer
        host = torch.empty((2, 8, 8), dtype=torch.float64)
        assert s.lib.fmm_dd_integrate(s.handle, 0, 2, ctypes.c_void_p(host.data_ptr()), None) == \
            fmm.FMM_ERR_INVALID                          # not device memory
