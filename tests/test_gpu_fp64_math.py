"""The double-precision square root and division of the fp64 march and the
adjoint (float seeds refined by Newton steps in double, csrc/fmm_fp64.cuh),
against CUDA's correctly rounded sqrt and '/' (torch's CUDA kernels) over a
seeded log-uniform sweep of operands across [1e-30, 1e30], the range edges
and the operands outside it (which take the correctly rounded operation).

Error bounds (relative to the correctly rounded result):

* sqrt: the seed y = sqrt(v) and the half reciprocal rh = 1/(2 sqrt(v)) come
  from a float v truncated to 24 bits (2^-23) and rsqrtf (about 2^-22), so
  y carries eps <= 3.4e-7 and rh eta <= 3e-7; one Newton step
  y + rh (v - y^2) leaves eps^2/2 + eta eps <= 1.6e-13.  Bound: 2e-13.
* division: the float reciprocal (2^-22) after two Newton steps is exact to
  double rounding, and the quotient gets one correction: a few ulp.
  Bound: 1e-15.

Outside [1e-30, 1e30] (for the division: a divisor outside it, or an
infinite, NaN or huge dividend) both take CUDA's correctly rounded operation
(exact).
In Algorithm 11 the square root enters u = (S + sqrt(disc)) / k with
sqrt(disc) ~ h, so 2e-13 relative is ~2e-13 h absolute per solve, far below
the fp64 parity tolerance of 1e-12 max|psi|."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SQRT_BOUND = 2e-13
DIV_BOUND = 1e-15


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")
    from paper_1502_07303_gb300 import fmm
    return fmm.load()


def _run(lib, a, b):
    A = torch.as_tensor(a, dtype=torch.float64, device="cuda").contiguous()
    B = torch.as_tensor(b, dtype=torch.float64, device="cuda").contiguous()
    S = torch.empty_like(A)
    Q = torch.empty_like(A)
    st = torch.cuda.current_stream()
    rc = lib.fmm_selftest_fp64(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                               ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(Q.data_ptr()),
                               A.numel(), ctypes.c_void_p(st.cuda_stream))
    assert rc == 0
    ref_s = torch.sqrt(A)
    ref_q = A / B
    torch.cuda.synchronize()
    return S, Q, ref_s, ref_q


def _rel(x, r):
    x, r = x.cpu().numpy(), r.cpu().numpy()
    d = np.abs(x - r)
    return np.where(r != 0, d / np.abs(r), d)


def test_sqrt_and_division_within_the_stated_bounds(lib):
    rng = np.random.default_rng(7)
    n = 1 << 22
    a = 10.0 ** rng.uniform(-30, 30, n)
    b = 10.0 ** rng.uniform(-30, 30, n) * rng.choice([-1.0, 1.0], n)
    # the range edges and their neighbours, and numbers near 1 and powers of 2
    edges = np.array([1e-30, 1e30, np.nextafter(1e-30, 1), np.nextafter(1e30, 0), 1.0,
                      np.nextafter(1.0, 2), np.nextafter(1.0, 0), 2.0, 0.5, 4.0, 3.0, 0.1])
    a = np.concatenate([a, edges, edges[::-1]])
    b = np.concatenate([b, edges[::-1], edges])
    S, Q, rs, rq = _run(lib, a, b)
    es, eq = _rel(S, rs), _rel(Q, rq)
    print(f"worst relative error: sqrt {es.max():.3e}, division {eq.max():.3e}")
    assert es.max() <= SQRT_BOUND, f"sqrt relative error {es.max():.3e}"
    assert eq.max() <= DIV_BOUND, f"division relative error {eq.max():.3e}"


def test_operands_outside_the_range_are_exact(lib):
    a = np.array([0.0, 1e-300, 5e-324, 1e-31, 1e31, 1e300, np.inf, 2.5e-310, np.nan, 1e290])
    b = np.array([1e-40, 1e40, 3.0, 1e-300, 1e300, 7.0, 2.0, 1e35, 3.0, 0.5])
    S, Q, rs, rq = _run(lib, a, b)
    torch.testing.assert_close(S, rs, rtol=0, atol=0, equal_nan=True)
    torch.testing.assert_close(Q, rq, rtol=0, atol=0, equal_nan=True)
