"""Parity at the full workload sizes, in the launch configuration bench.py
times (library defaults).

* 256^3, 32 random spheres (the benchmark workload): element by element
  against the oracle, fp32 and fp64.
* 512^3 heterogeneous speed, 8 sources: sampled cells re-solved one by one
  with the oracle's Algorithm 11 from the GPU's final neighbour values, and
  the Eq. (2) residual over the whole grid.
* 1024^3 signed distance to one sphere: sampled Algorithm 11 re-solves, the
  sign of every cell, and the first-order distance error bound (the oracle's
  own error grows from 0.8 h at 32^3 to 1.5 h at 192^3).
"""
import math

import numpy as np
import pytest
import torch

from paper_1502_07303_gb300 import workloads as wl
from parity_util import TOL, compare

pytestmark = pytest.mark.gpu

DT = {"f32": torch.float32, "f64": torch.float64}


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")
    from paper_1502_07303_gb300 import fmm as _fmm
    return _fmm


def residual_eq2(T, h, F):
    """max over accepted cells of |(|grad psi|_Godunov) F - 1| (Eq. (2)),
    evaluated with torch on the device from the final |psi|."""
    A = T.abs().to(torch.float64)
    s = torch.zeros_like(A)
    inf = torch.tensor(float("inf"), dtype=torch.float64, device=A.device)
    for ax in range(3):
        pad = [0, 0, 0, 0, 0, 0]
        pad[2 * (2 - ax)] = 1
        pad[2 * (2 - ax) + 1] = 1
        P = torch.nn.functional.pad(A, pad, value=float("inf"))
        lo = P.narrow(ax, 0, A.shape[ax])
        hi = P.narrow(ax, 2, A.shape[ax])
        m = torch.minimum(lo, hi)
        term = torch.clamp(A - m, min=0.0)
        term = torch.where(torch.isinf(m), torch.zeros_like(term), term) / h
        s += term * term
    F = F if torch.is_tensor(F) else torch.tensor(F, dtype=torch.float64, device=A.device)
    return torch.sqrt(s) * F.to(torch.float64) - 1.0


def sampled_local_solves(oracle, T, G, h, F, n=3000, seed=0):
    """Largest |T_cell - Algorithm 11(final neighbours)| over n sampled
    accepted non-FIX cells (the oracle re-solves each cell)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = T.shape
    # rejection sampling of accepted cells (a full index list of a 1024^3
    # grid would not fit comfortably)
    cand = np.stack([rng.integers(0, nz, 8 * n), rng.integers(0, ny, 8 * n),
                     rng.integers(0, nx, 8 * n)], axis=1)
    cg = torch.as_tensor(cand, device=T.device)
    ok = (G[cg[:, 0], cg[:, 1], cg[:, 2]] == 2).cpu().numpy()
    pick = cand[ok][:n]
    assert len(pick) > n // 2
    offs = [(0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
    cells = torch.as_tensor(pick, device=T.device)
    nb_vals, nb_known = [], []
    for dz, dy, dx in offs:
        q = cells + torch.tensor([dz, dy, dx], device=T.device)
        inside = ((q >= 0) & (q < torch.tensor([nz, ny, nx], device=T.device))).all(1)
        qc = torch.where(inside[:, None], q, torch.zeros_like(q))
        v = T[qc[:, 0], qc[:, 1], qc[:, 2]].abs().to(torch.float64)
        k = (G[qc[:, 0], qc[:, 1], qc[:, 2]] >= 2) & inside
        nb_vals.append(v.cpu().numpy())
        nb_known.append(k.cpu().numpy())
    Tc = T[cells[:, 0], cells[:, 1], cells[:, 2]].abs().to(torch.float64).cpu().numpy()
    Fc = F if np.isscalar(F) else F[cells[:, 0], cells[:, 1], cells[:, 2]].to(torch.float64).cpu().numpy()
    worst = 0.0
    for r in range(len(pick)):
        nb = np.array([nb_vals[q][r] for q in range(6)])
        kn = np.array([nb_known[q][r] for q in range(6)], dtype=np.uint8)
        fr = Fc if np.isscalar(Fc) else float(Fc[r])
        v = oracle.local_solve(nb, kn, Tc[r], h, fr)
        worst = max(worst, abs(v - Tc[r]))
    return worst


# the library defaults, and the configurations the bench's autotuner picks
# for this workload (persistent without restarts; continuous at 2 h or 4 h
# without a lead limit)
BENCH_PARAMS = [{}, {"schedule": 2, "stride": math.inf},
                {"schedule": 3, "stride": 2.0, "max_lead": 1 << 20},
                {"schedule": 3, "stride": 4.0, "max_lead": 1 << 20}]


@pytest.fixture(scope="module")
def c2():
    p = wl.random_spheres(n=256, count=32, seed=2)
    return p, {}


@pytest.mark.parametrize("params", BENCH_PARAMS,
                         ids=["defaults", "persistent-inf", "continuous-2h", "continuous-4h"])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_bench_workload_256_full_compare(fmm, oracle, c2, dt, params):
    p, refs = c2
    phi = torch.as_tensor(p.phi0, dtype=DT[dt], device="cuda")
    with fmm.Solver(p.shape, p.h, dtype=DT[dt], **params) as s:
        T, G = s.reinit(phi)
    if dt not in refs:
        phi_q = np.asarray(p.phi0, np.float32).astype(np.float64) if dt == "f32" else p.phi0
        refs[dt] = oracle.solve_reinit(phi_q, p.h)
    compare(T.cpu().numpy(), G.cpu().numpy(), refs[dt], dt)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_heterogeneous_512_sampled(fmm, oracle, dt):
    p = wl.fourier_sources(n=512, n_sources=8, n_receivers=64, seed=3, device="cuda")
    F = p.speed.to(DT[dt]).contiguous()
    with fmm.Solver(p.shape, p.h, dtype=DT[dt], speed=F, sources=p.sources) as s:
        T, G = s.solve()
    assert int((G == 0).sum()) == 0 and int((G == 1).sum()) == 0   # full march
    maxT = float(T.abs().max())
    worst = sampled_local_solves(oracle, T, G, p.h, F)
    assert worst <= TOL[dt] * maxT, (worst, maxT)
    res = residual_eq2(T, p.h, F)[G == 2]
    # Eq. (2) holds to rounding: |grad psi| F - 1 is ~eps * (psi F / h)
    bound = 1e-9 if dt == "f64" else 2e-2
    assert float(res.abs().max()) <= bound


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_sphere_1024(fmm, oracle, dt):
    n = 1024
    p = wl.single_sphere(n, device="cuda")
    phi = p.phi0.to(DT[dt]).contiguous()
    with fmm.Solver(p.shape, p.h, dtype=DT[dt]) as s:
        T, G = s.reinit(phi)
        st = s.stats()
    assert st["error_flags"] == 0
    assert int((G == 0).sum()) == 0 and int((G == 1).sum()) == 0
    # sign of psi is the sign of phi0
    assert bool(((T >= 0) == (phi >= 0)).all())
    maxT = float(T.abs().max())
    worst = sampled_local_solves(oracle, T, G, p.h, 1.0)
    assert worst <= TOL[dt] * maxT, (worst, maxT)
    # first-order accurate distance: within a few cells of the exact value
    err = (T.to(torch.float64) - p.phi0).abs().max().item()
    assert err <= 3.0 * p.h, (err, p.h)
    del T, G, phi
    torch.cuda.empty_cache()
