"""Domain decomposition across ranks (Sec. 4.1, Algorithms 13-16), on the CPU:
the partition, the restart loop of paper_1502_07303_gb300/decomp.py with each
rank's local march done by the plain-Python marcher of tests/dd_reference.py,
stepped in one process and as two gloo ranks on 127.0.0.1.  The assembled
solution must be the oracle's sequential solution of the whole grid (the
paper's claim that the decomposed method reproduces the sequential one,
Sec. 5.2), within 1e-12 max|psi| and with identical accepted sets."""
import json
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch

from paper_1502_07303_gb300 import decomp
from paper_1502_07303_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def test_slabs_cover_the_grid_and_overlap_by_two_layers():
    for nz, n in ((10, 1), (10, 3), (17, 4), (9, 9)):
        s = decomp.slabs(nz, n)
        assert s[0][0] == 0 and s[-1][1] == nz
        assert all(a[1] == b[0] and a[1] > a[0] for a, b in zip(s, s[1:]))
        subs = [decomp.Subdomain(nz, n, r) for r in range(n)]
        for a, b in zip(subs, subs[1:]):
            # the upper ghost of a is b's first layer, b's lower ghost is a's last
            assert a.lz1 - 1 == b.z0 and b.lz0 == a.z1 - 1
            (pa, za), = [x for x in a.neighbours() if x[0] == b.rank]
            (pb, zb), = [x for x in b.neighbours() if x[0] == a.rank]
            assert a.lz0 + za == b.lz0 + zb == a.z1 - 1
    with pytest.raises(ValueError):
        decomp.slabs(3, 4)
    # wider overlaps: 2 * ghost shared layers at the same global positions
    for ghost in (2, 3):
        subs = [decomp.Subdomain(20, 3, r, ghost) for r in range(3)]
        for a, b in zip(subs, subs[1:]):
            (pa, za), = [x for x in a.neighbours() if x[0] == b.rank]
            (pb, zb), = [x for x in b.neighbours() if x[0] == a.rank]
            assert a.lz0 + za == b.lz0 + zb == a.z1 - ghost
            assert a.n_overlap == 2 * ghost
    with pytest.raises(ValueError):
        decomp.Subdomain(6, 3, 0, ghost=3)


def test_bounds_and_exit_test_follow_algorithm_16():
    assert decomp.next_bound([0.5, math.inf], 0.25, 1.0) == [0.75, 1.0]
    assert decomp.finished([math.inf, math.inf], 0, math.inf)
    assert not decomp.finished([math.inf, math.inf], 3, math.inf)
    assert not decomp.finished([0.2, math.inf], 0, math.inf)


def _problems():
    sph = wl.random_spheres(shape=(21, 13, 11), count=2, seed=51)
    rng = np.random.default_rng(52)
    shape = (18, 12, 10)
    h = wl.spacing(shape)
    F = wl.fourier_speed(shape, wl.draw_fourier_modes(rng), h=h)
    src = wl.random_cells(rng, shape, 3)
    return [("reinit", sph.shape, sph.h, dict(phi0=sph.phi0)),
            ("sources", shape, h, dict(sources=src, speed=F))]


def _reference(oracle, shape, h, kw):
    if "phi0" in kw:
        return oracle.solve_reinit(kw["phi0"], h)
    return oracle.solve_sources(shape, kw["sources"], h, speed=kw["speed"])


def _check(T, G, ref):
    from parity_util import compare
    compare(np.asarray(T), np.asarray(G).astype(np.uint8), ref, "f64")


@pytest.mark.parametrize("n_ranks,stride,ghost", [(2, 2.0, 1), (3, 1.0, 1), (4, math.inf, 1),
                                                  (3, 2.0, 2), (2, 1.0, 3)])
def test_serial_ranks_reproduce_the_sequential_solution(oracle, n_ranks, stride, ghost):
    from dd_reference import RefMarcher
    for name, shape, h, kw in _problems():
        subs = [decomp.Subdomain(shape[0], n_ranks, r, ghost) for r in range(n_ranks)]
        ms = [RefMarcher(s, shape, h, **kw) for s in subs]
        results, restarts = decomp.solve_serial(ms, subs, stride * h)
        T, G = decomp.assemble(subs, results, shape)
        # dd_reference's tags (FAR, BAND, KNOWN, FIX) are the public tag values
        _check(T.numpy(), G.numpy(), _reference(oracle, shape, h, kw))
        assert restarts >= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, stride_h):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    for p in (ROOT, HERE):
        if p not in sys.path:
            sys.path.insert(0, p)
    import torch.distributed as dist

    from dd_reference import RefMarcher
    dist.init_process_group("gloo", rank=rank, world_size=world)
    comm = decomp.TorchComm(dist, "cpu")
    out = {}
    for name, shape, h, kw in _problems():
        sub = decomp.Subdomain(shape[0], world, rank)
        (T, G), restarts = decomp.solve_spmd(RefMarcher(sub, shape, h, **kw), sub, comm, stride_h * h)
        np.save(os.path.join(out_dir, f"{name}_T{rank}.npy"), sub.interior(T).numpy())
        np.save(os.path.join(out_dir, f"{name}_G{rank}.npy"), sub.interior(G).numpy())
        out[name] = restarts
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(out, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_sequential_solution(oracle, tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path), 2.0), nprocs=2, join=True)
    info = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for name, shape, h, kw in _problems():
        assert info[0][name] == info[1][name]          # the ranks agree on termination
        T = np.concatenate([np.load(tmp_path / f"{name}_T{r}.npy") for r in range(2)])
        G = np.concatenate([np.load(tmp_path / f"{name}_G{r}.npy") for r in range(2)])
        assert T.shape == tuple(shape)
        _check(T, G, _reference(oracle, shape, h, kw))
