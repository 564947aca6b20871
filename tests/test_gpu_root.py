"""The double-grid root of Algorithm 11 (the fp64 march's double-float
solve, csrc/fmm_df.cuh, through fmm_selftest_root) against exact arithmetic
(Python's decimal module at 60 digits).

With shifted values delta_i = v_i - m of the upwind set (delta_0 = 0) the
root of sum_i (u - delta_i)^2 = q is u = (S + sqrt(k q - P)) / k, S the sum
of the delta_i, P the sum over pairs of (delta_i - delta_j)^2; the set is
causal when its largest delta is below u, and Algorithm 11 drops the largest
value while it is not.  Checked:

* the causal set: the routine's choice is the exact one, except where the
  exact u lies within 1e-13 u of the largest delta (there both sets give the
  same root to well below the parity tolerance, and rounding may decide);
* causality of the choice itself: with two or three values the root is above
  every value the chosen set uses (the upwind sets recorded for the adjoint
  must point strictly downhill);
* the root: within 1e-15 t + 4e-14 u of the exact root of the exact set (u
  in double-float carries about 1e-14 relative, t = m + u one rounding).

The cases sit on both sides of the set transition (the third value placed
within 1e-9 of the two-value root), plus general random cases and a case
found in a 256^3 solve where an unnormalized double-float comparison kept a
non-causal third value."""
import ctypes
from decimal import Decimal, getcontext

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
getcontext().prec = 60


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")
    from paper_1502_07303_gb300 import fmm
    return fmm.load()


def _exact(m, v1, v2, nd, q):
    """(k, t, margin): the causal set size, its root and u - max delta of it."""
    D = Decimal
    m, v1, v2, q = D(m), D(v1), D(v2), D(q)
    d = [D(0), v1 - m, v2 - m][:nd]
    for k in range(nd, 0, -1):
        dd = d[:k]
        S = sum(dd)
        P = sum((dd[i] - dd[j]) ** 2 for i in range(k) for j in range(i + 1, k))
        disc = k * q - P
        if disc < 0:
            continue
        u = (S + disc.sqrt()) / k
        if dd[-1] < u:
            return k, m + u, u - dd[-1], u
    return 0, None, None, None


def _run(lib, m, v1, v2, nd, q):
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    tm, t1, t2, tq = (dev(a, torch.float64) for a in (m, v1, v2, q))
    tn = dev(nd, torch.int32)
    t_out = torch.empty_like(tm)
    k_out = torch.empty_like(tn)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.fmm_selftest_root(p(tm), p(t1), p(t2), p(tn), p(tq), p(t_out), p(k_out), len(m), None)
    assert rc == 0
    torch.cuda.synchronize()
    return t_out.cpu().numpy(), k_out.cpu().numpy()


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    h = rng.choice([1 / 64, 1 / 256, 1 / 1024], n)
    F = np.exp(rng.uniform(-0.7, 0.7, n))
    q = (h / F) ** 2
    m = rng.uniform(0.0, 1.5, n)
    d1 = rng.uniform(0.0, 1.2, n) * h / F
    v1 = m + d1
    # the two-value root and a third value placed within 1e-9 of it
    u2 = (d1 + np.sqrt(np.maximum(2 * q - d1 ** 2, 0.0))) / 2
    near = m + u2 * (1 + rng.uniform(-1e-9, 1e-9, n))
    far = m + rng.uniform(0.0, 1.5, n) * h / F
    pick = rng.random(n) < 0.6
    v2 = np.where(pick, near, far)
    lo, hi = np.minimum(v1, v2), np.maximum(v1, v2)
    nd = rng.choice([1, 2, 3], n, p=[0.1, 0.2, 0.7]).astype(np.int32)
    return m, lo, hi, nd, q


def test_root_and_causal_set_match_exact_arithmetic(lib):
    m, v1, v2, nd, q = _cases(20000, seed=41)
    # the case from the 256^3 solve (exact: two values causal, the third not)
    m = np.append(m, 0.15071860094080336)
    v1 = np.append(v1, 0.1521001659784484)
    v2 = np.append(v2, 0.15323725757617793)
    nd = np.append(nd, np.int32(3)).astype(np.int32)
    q = np.append(q, 7.636608400714676e-06)
    t, k = _run(lib, m, v1, v2, nd, q)
    assert k[-1] == 2
    wrong_set, uncausal, bad_root = [], [], []
    for i in range(len(m)):
        ke, te, margin, u = _exact(m[i], v1[i], v2[i], int(nd[i]), q[i])
        if k[i] != ke and not (margin is not None and abs(margin) <= Decimal("1e-13") * u):
            wrong_set.append(i)
        used = [m[i], v1[i], v2[i]][:max(int(k[i]), 1)]
        if k[i] > 1 and not t[i] > max(used):
            uncausal.append(i)
        # the double-float u carries ~1e-14 relative, t = m + u one rounding
        if ke > 0 and abs(Decimal(float(t[i])) - te) > Decimal("1e-15") * te + Decimal("4e-14") * u:
            bad_root.append(i)
    assert not wrong_set, [(i, int(k[i])) for i in wrong_set[:5]]
    assert not uncausal, uncausal[:5]
    assert not bad_root, bad_root[:5]
