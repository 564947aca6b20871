"""fmm_reinit_signed_distance_noalloc against fmm_reinit_signed_distance.

The no-allocation entry point exists for callers that cannot allocate
device memory when they solve (inside a CUDA graph capture, under a memory
pool that forbids further allocations).  It keeps its workspace in a fixed
device array that every call shares, so this test makes two calls in a row
on different problems (different dtypes and sizes) and checks each result
against the ordinary handle-based entry point with the tolerances of the
other parity tests: identical tags, max |dT| <= 1e-12 max|T| in fp64 and
2e-5 max|T| in fp32.  It also checks that a grid above the stated limit is
rejected with a clear error.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_1502_07303_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")
    from paper_1502_07303_gb300 import fmm as _fmm
    return _fmm


def _check_against_handle(fmm, p, dtype):
    phi = torch.as_tensor(p.phi0, dtype=dtype, device="cuda").contiguous()
    T_na = torch.full(p.shape, float("nan"), dtype=dtype, device="cuda")
    G_na = torch.full(p.shape, 255, dtype=torch.uint8, device="cuda")
    fmm.reinit_noalloc(phi, p.h, T_na, G_na)
    with fmm.Solver(p.shape, p.h, dtype=dtype) as s:
        T_ref, G_ref = s.reinit(phi)
    torch.cuda.synchronize()
    assert torch.equal(G_na, G_ref), "tags differ from fmm_reinit_signed_distance"
    T_na, T_ref = T_na.cpu().numpy(), T_ref.cpu().numpy()
    fin = np.isfinite(T_ref)
    assert np.array_equal(fin, np.isfinite(T_na))
    scale = float(np.max(np.abs(T_ref[fin])))
    err = float(np.max(np.abs(T_na[fin] - T_ref[fin])))
    assert err <= TOL[dtype] * scale, f"max |dT| {err:.3e} > {TOL[dtype]:.0e} * {scale:.3g}"


def test_two_calls_in_a_row_match_the_handle_entry_point(fmm):
    first = wl.random_spheres(shape=(48, 48, 48), count=5, seed=31)
    second = wl.random_spheres(shape=(29, 41, 23), count=3, seed=32)
    _check_against_handle(fmm, first, torch.float64)
    _check_against_handle(fmm, second, torch.float32)


def test_grid_above_the_limit_is_rejected(fmm):
    shape = (72, 64, 64)     # 9 x 8 x 8 = 576 bricks > 512
    phi = torch.zeros(shape, dtype=torch.float32, device="cuda")
    T = torch.empty(shape, dtype=torch.float32, device="cuda")
    with pytest.raises(fmm.FmmError) as e:
        fmm.reinit_noalloc(phi, 1.0 / 72, T)
    assert e.value.code == fmm.FMM_ERR_INVALID
    assert "too large" in str(e.value)
