"""fmm_reinit_signed_distance_noalloc against fmm_reinit_signed_distance and
the oracle.

The no-allocation entry point exists for callers that cannot allocate device
memory when they solve: processes whose device memory is owned by a pool or
arena that forbids further driver allocations, and loops that must not pay
for (or fail on) an allocation mid-run.  It keeps its workspace in a fixed
device array that every call shares, so this test makes two calls in a row
on different problems (different dtypes and sizes) and checks each result
against the ordinary handle-based entry point and against the CPU oracle with
the tolerances of the other parity tests: identical tags, max |dT| <= 1e-12
max|T| in fp64 and 2e-5 max|T| in fp32.  It checks that a warm call leaves the
device's free memory unchanged, that tags_out may be NULL, that a grid above
the stated limit and a configuration fmm_create refuses are rejected with
FMM_ERR_INVALID.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_1502_07303_gb300 import workloads as wl
from parity_util import compare

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}
NAME = {torch.float64: "f64", torch.float32: "f32"}


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")
    from paper_1502_07303_gb300 import fmm as _fmm
    return _fmm


def _check(fmm, oracle, p, dtype):
    phi = torch.as_tensor(p.phi0, dtype=dtype, device="cuda").contiguous()
    T_na = torch.full(p.shape, float("nan"), dtype=dtype, device="cuda")
    G_na = torch.full(p.shape, 255, dtype=torch.uint8, device="cuda")
    fmm.reinit_noalloc(phi, p.h, T_na, G_na)
    with fmm.Solver(p.shape, p.h, dtype=dtype) as s:
        T_ref, G_ref = s.reinit(phi)
    torch.cuda.synchronize()
    # against the handle entry point
    assert torch.equal(G_na, G_ref), "tags differ from fmm_reinit_signed_distance"
    Tn, Tr = T_na.cpu().numpy(), T_ref.cpu().numpy()
    fin = np.isfinite(Tr)
    assert np.array_equal(fin, np.isfinite(Tn))
    scale = float(np.max(np.abs(Tr[fin])))
    err = float(np.max(np.abs(Tn[fin] - Tr[fin])))
    assert err <= TOL[dtype] * scale, f"max |dT| {err:.3e} > {TOL[dtype]:.0e} * {scale:.3g}"
    # against the oracle, on the level set the GPU saw
    phi_q = phi.double().cpu().numpy()
    ref = oracle.solve_reinit(phi_q, p.h)
    compare(Tn, G_na.cpu().numpy(), ref, NAME[dtype])


def test_two_calls_in_a_row_match_the_handle_entry_point_and_the_oracle(fmm, oracle):
    first = wl.random_spheres(shape=(48, 48, 48), count=5, seed=31)
    second = wl.random_spheres(shape=(29, 41, 23), count=3, seed=32)
    _check(fmm, oracle, first, torch.float64)
    _check(fmm, oracle, second, torch.float32)


def test_warm_call_allocates_nothing_and_takes_no_tags(fmm, oracle):
    p = wl.random_spheres(shape=(40, 40, 40), count=4, seed=33)
    phi = torch.as_tensor(p.phi0, dtype=torch.float32, device="cuda").contiguous()
    T1 = torch.empty(p.shape, dtype=torch.float32, device="cuda")
    T2 = torch.full(p.shape, float("nan"), dtype=torch.float32, device="cuda")
    fmm.reinit_noalloc(phi, p.h, T1)            # warm: the address lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    fmm.reinit_noalloc(phi, p.h, T2, None)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    assert torch.equal(T1.isinf(), T2.isinf())
    ref = oracle.solve_reinit(phi.double().cpu().numpy(), p.h)
    T2h = T2.cpu().numpy().astype(np.float64)
    fin = np.isfinite(ref["T"])
    scale = float(np.max(np.abs(ref["T"][fin])))
    assert float(np.max(np.abs(T2h[fin] - ref["T"][fin]))) <= 2e-5 * scale


def test_grid_above_the_limit_is_rejected(fmm):
    shape = (72, 64, 64)     # 9 x 8 x 8 = 576 bricks > 512
    phi = torch.zeros(shape, dtype=torch.float32, device="cuda")
    T = torch.empty(shape, dtype=torch.float32, device="cuda")
    with pytest.raises(fmm.FmmError) as e:
        fmm.reinit_noalloc(phi, 1.0 / 72, T)
    assert e.value.code == fmm.FMM_ERR_INVALID
    assert "too large" in str(e.value)


@pytest.mark.parametrize("field,value", [("schedule", 7), ("schedule", -1),
                                         ("exchange_passes", -2), ("exchange_passes", 65)])
def test_configuration_fmm_create_refuses_is_rejected(fmm, field, value):
    import ctypes
    lib = fmm.load()
    shape = (16, 16, 16)
    phi = torch.ones(shape, dtype=torch.float32, device="cuda")
    T = torch.empty(shape, dtype=torch.float32, device="cuda")
    cfg = fmm.FmmConfig()
    cfg.nx = cfg.ny = cfg.nz = 16
    cfg.h = 1.0 / 16
    cfg.dtype = fmm.FMM_F32
    setattr(cfg, field, value)
    rc = lib.fmm_reinit_signed_distance_noalloc(ctypes.byref(cfg), ctypes.c_void_p(phi.data_ptr()),
                                                ctypes.c_void_p(T.data_ptr()), None)
    assert rc == fmm.FMM_ERR_INVALID
    assert field in lib.fmm_last_error(None).decode()
