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


def test_bench_batch_256_grids_full_compare(fmm, oracle):
    """The bench's batched workload in full (256 grids, axes in [32, 192],
    fp32, one batch handle, library defaults): every grid element by element
    against the oracle (on the level set the GPU saw), the oracle solves
    running on a host thread pool."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    probs = wl.batch(n_grids=256, lo=32, hi=192, seed=4, device="cuda")
    phis = [p.phi0.to(torch.float32).contiguous() for p in probs]
    phis_q = [ph.to(torch.float64).cpu().numpy() for ph in phis]
    with ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as pool:
        # largest grids first, so the pool finishes evenly
        order = sorted(range(len(probs)), key=lambda i: -probs[i].n_points)
        futs = {i: pool.submit(oracle.solve_reinit, phis_q[i], probs[i].h) for i in order}
        with fmm.Batch([p.shape for p in probs], [p.h for p in probs], dtype=torch.float32) as b:
            Ts, Gs = b.reinit(phis)
            st = b.stats()
        assert st["error_flags"] == 0
        for i in range(len(probs)):
            compare(Ts[i].cpu().numpy(), Gs[i].cpu().numpy(), futs[i].result(), "f32")


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_solve_batch_mixed_problems(fmm, oracle, dt):
    """fmm_solve_batch with a level set or point sources per grid and each
    grid's own speed (field, constant or 1; obstacle cells with F = 0), every
    grid element by element against the oracle, twice in a row on one
    handle (the second call with the kinds of problem swapped around)."""
    rng = np.random.default_rng(41)
    shapes = [(19, 23, 17), (32, 24, 40), (9, 33, 21), (28, 28, 28), (16, 40, 12)]
    probs = []
    for g, sh in enumerate(shapes):
        h = wl.spacing(sh)
        sph = wl.draw_spheres(rng, 2)
        modes = wl.draw_fourier_modes(rng)
        F = wl.fourier_speed(sh, modes, h=h)
        if g == 4:
            F = F.copy()
            F[:, 20, :] = 0.0                   # a wall of obstacle cells
            F[:, 20, 3:5] = 1.0                 # with a gap
        src = wl.random_cells(rng, sh, 1 + g % 3)
        probs.append(dict(shape=sh, h=h, phi=wl.spheres_phi0(sh, sph, h=h), F=F, src=src))
    kinds = [("phi", "field"), ("src", "field"), ("phi", 1.0), ("src", 2.5), ("src", "field")]

    def q(a):
        return np.asarray(a, np.float32).astype(np.float64) if dt == "f32" else np.asarray(a, np.float64)

    with fmm.Batch(shapes, [p["h"] for p in probs], dtype=DT[dt]) as b:
        for call in range(2):
            ks = kinds if call == 0 else [(("src" if k == "phi" else "phi"), s) for k, s in kinds]
            phis, srcs, speeds = [], [], []
            for p, (kind, sp) in zip(probs, ks):
                phis.append(torch.as_tensor(p["phi"], dtype=DT[dt], device="cuda") if kind == "phi" else None)
                srcs.append(p["src"] if kind == "src" else None)
                speeds.append(torch.as_tensor(p["F"], dtype=DT[dt], device="cuda") if sp == "field" else sp)
            Ts, Gs = b.solve(phis, srcs, speeds)
            for p, (kind, sp), T, G in zip(probs, ks, Ts, Gs):
                Fo = q(p["F"]) if sp == "field" else float(sp)
                if kind == "phi":
                    ref = oracle.solve_reinit(q(p["phi"]), p["h"], speed=Fo)
                else:
                    ref = oracle.solve_sources(p["shape"], p["src"], p["h"], speed=Fo)
                compare(T.cpu().numpy(), G.cpu().numpy(), ref, dt)


def test_solve_batch_rejects_bad_problems(fmm):
    with fmm.Batch([(8, 8, 8), (8, 8, 8)], [0.1, 0.1], dtype=torch.float32) as b:
        with pytest.raises(ValueError):
            b.solve([None, None], [None, [[1, 1, 1]]])
        with pytest.raises(fmm.FmmError) as e:
            b.solve([None, None], [[[8, 0, 0]], [[1, 1, 1]]])
        assert e.value.code == fmm.FMM_ERR_INVALID
        bad = torch.full((8, 8, 8), -1.0, device="cuda")
        with pytest.raises(fmm.FmmError) as e:
            b.solve([None, None], [[[0, 0, 0]], [[1, 1, 1]]], [bad, None])
        assert e.value.code == fmm.FMM_ERR_INVALID
