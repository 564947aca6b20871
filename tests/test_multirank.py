"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

The bench runs one independent replica per rank (no collective on the data
path); the only collectives are the barrier and the max / sum over ranks that
turn per-rank times and points into the whole-job value."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local, pg = bench.dist_setup()
    bench.barrier(pg)
    ms = bench.max_over_ranks(pg, 10.0 + rank)          # slowest rank's time
    pts = bench.sum_over_ranks(pg, 1000.0 * (rank + 1))  # points of all ranks
    value = pts / (ms / 1e3) / 1e9
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ws": ws, "rank": r, "ms": ms, "pts": pts, "value": value}, f)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_times_and_points(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, g in enumerate(got):
        assert g["ws"] == 2 and g["rank"] == r
        assert g["ms"] == 11.0          # max over ranks
        assert g["pts"] == 3000.0       # sum over ranks
        assert abs(g["value"] - 3000.0 / 0.011 / 1e9) < 1e-15


def test_reference_arm_prints_once_under_two_ranks():
    """torchrun with 2 ranks: rank 0 runs the oracle and prints one JSON line,
    rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
