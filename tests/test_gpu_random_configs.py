"""Seeded random configurations against the oracle: grid shape, cubic or
unequal cells, precision, schedule, stride, bucket width, tape, point sources
with or without a heterogeneous speed or a reinitialisation, and a restart
limit followed by resumes.  Each combination must reach the oracle's fixed
point (the readings, tolerances and tag classes of parity_util)."""
import math

import numpy as np
import pytest
import torch

from paper_1502_07303_gb300 import workloads as wl
from parity_util import compare

pytestmark = pytest.mark.gpu

N_CASES = 60


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")
    from paper_1502_07303_gb300 import fmm as _fmm
    return _fmm


def _draw(seed):
    rng = np.random.default_rng(seed)
    shape = tuple(int(v) for v in rng.integers(5, 48, 3))
    base = 1.0 / max(shape)
    h = (tuple(base * rng.uniform(0.6, 1.6) for _ in range(3)) if rng.random() < 0.5 else base)
    c = dict(shape=shape, h=h, dt="f64" if rng.random() < 0.5 else "f32",
             schedule=int(rng.integers(1, 4)),
             stride=float(rng.choice([0.0, 0.5, 1.0, 2.0, 8.0, math.inf])),
             bucket=float(rng.choice([0.0, 1.0, 2.0, 4.0, math.inf])),
             tape=bool(rng.random() < 0.3), kind="src" if rng.random() < 0.5 else "reinit")
    c["limit"] = int(rng.integers(1, 6)) if rng.random() < 0.3 and c["stride"] != math.inf else 0
    return rng, c


@pytest.mark.parametrize("seed", range(N_CASES))
def test_random_configuration(fmm, oracle, seed):
    rng, c = _draw(1000 + seed)
    shape, h, dt = c["shape"], c["h"], c["dt"]
    tdt = torch.float64 if dt == "f64" else torch.float32
    q = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if dt == "f32" else (lambda a: a)
    kw = dict(dtype=tdt, schedule=c["schedule"], stride=c["stride"], bucket=c["bucket"],
              record_tape=c["tape"], max_restarts=c["limit"])
    if c["kind"] == "src":
        F = wl.fourier_speed(shape, wl.draw_fourier_modes(rng), h=h) if rng.random() < 0.7 else None
        src = wl.random_cells(rng, shape, int(rng.integers(1, 5)))
        ref = oracle.solve_sources(shape, src, h, speed=None if F is None else q(F))
        sp = None if F is None else torch.as_tensor(F, dtype=tdt, device="cuda")
        s = fmm.Solver(shape, h, speed=sp, sources=src, **kw)
        call = s.solve
    else:
        x, y, z = wl._axes(shape, h)
        ext = np.array([x.max(), y.max(), z.max()])
        phi = np.full(shape, np.inf)
        for _ in range(int(rng.integers(1, 5))):
            ctr = rng.uniform(0.1, 0.9, 3) * ext
            r = rng.uniform(0.05, 0.3) * ext.min()
            phi = np.minimum(phi, np.sqrt((x - ctr[0]) ** 2 + (y - ctr[1]) ** 2
                                          + (z - ctr[2]) ** 2) - r)
        ref = oracle.solve_reinit(q(phi), h)
        ph = torch.as_tensor(phi, dtype=tdt, device="cuda")
        s = fmm.Solver(shape, h, **kw)
        call = lambda: s.reinit(ph)
    with s:
        try:
            T, G = call()
        except fmm.FmmError as e:
            assert e.code == fmm.FMM_ERR_TIMEOUT and c["limit"] > 0, str(e)
            for _ in range(2000):
                try:
                    T, G = s.resume(more_restarts=int(rng.integers(0, 4)))
                    break
                except fmm.FmmError as e2:
                    assert e2.code == fmm.FMM_ERR_TIMEOUT, str(e2)
            else:
                pytest.fail("the resumed solve did not finish")
        assert s.stats()["error_flags"] == 0
    compare(T.cpu().numpy().astype(np.float64), G.cpu().numpy(), ref, dt)
