"""Oracle solves of the full-size workloads, run on host threads in the
background (the C oracle releases the GIL): started once, as soon as the test
session knows it will need them, so that they overlap the GPU tests that run
first.  Not collected as tests."""
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_lock = threading.Lock()
_jobs = None
_pool = None
_inputs = None


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def start():
    """Submit the solves (idempotent); returns (inputs, jobs).

    inputs["c3"]: the 512^3 heterogeneous-speed problem (speed on the GPU);
    jobs[("c3", dt)]: oracle solve on the speed field the GPU sees in dt;
    jobs[("c5", dt)]: oracle solve of the 1024^3 sphere's octant
    i, j, k < 512 (h = 1/1024) on the level set the GPU sees in dt."""
    global _jobs, _pool, _inputs
    with _lock:
        if _jobs is not None:
            return _inputs, _jobs
        import torch

        import oracle
        from paper_1502_07303_gb300 import workloads as wl
        oracle.build()
        p3 = wl.fourier_sources(n=512, n_sources=8, n_receivers=64, seed=3, device="cuda")
        oct_phi = wl.sphere_phi0((512, 512, 512), radius=0.3, h=1.0 / 1024)
        _pool = ThreadPoolExecutor(max_workers=4)
        _jobs = {}
        for dt, tdt in (("f64", torch.float64), ("f32", torch.float32)):
            F = p3.speed.to(tdt).to(torch.float64).cpu().numpy()
            _jobs[("c3", dt)] = _pool.submit(oracle.solve_sources, p3.shape, p3.sources, p3.h, F)
            phi = oct_phi if dt == "f64" else _f32(oct_phi)
            _jobs[("c5", dt)] = _pool.submit(oracle.solve_reinit, phi, 1.0 / 1024)
        _inputs = {"c3": p3}
        return _inputs, _jobs


def shutdown():
    global _pool
    if _pool is not None:
        _pool.shutdown(wait=True)
        _pool = None
