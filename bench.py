#!/usr/bin/env python
"""Throughput benchmark of the GB300 restarted narrow band fast marching library.

Workload (one "step" = one complete solve through the C ABI): two-sided
signed-distance reinitialisation of 32 seeded random spheres with the
sin-modulated level set on a 256^3 unit cube (16.8 M points), fp32, full
march, the library's default restart parameters.  The metric is grid points finalised per second (Gpoints/s).
fp64 is measured on the same workload and reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun, one rank per GPU) every rank solves its own replica of
the workload (independent problems, no collective on the data path: weak
scaling) and the whole-job value is the points of all ranks over the slowest
rank's time.  ``--impl reference`` times the CPU oracle (the paper's
sequential algorithm in plain C, fp64) on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpoints/s finalised (fp32/fp64) and % HBM roofline; adjoint and batched vs plain"
UNIT = "Gpoints/s"
N_GRID = 256
N_SPHERES = 32
SEED = 2
# algorithmic bytes per finalised point of a reinitialisation: read phi0,
# write psi and the tag once (fp32: 4 + 4 + 1, fp64: 8 + 8 + 1)
ALG_BYTES = {"f32": 9, "f64": 17}
REF_SAMPLE_N = 128          # oracle sample grid for the reference arm
CPU_BASELINE_N = 192        # oracle sample grid for the cpu_baseline entry


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_record(kernel, dtype):
    """DRAM bytes per finalised point of a march kernel and dtype from the
    committed ncu summary (lines "kernel dtype source_sha256_16 bytes"), valid
    only while the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "k_march_traffic.txt")
    src = os.path.join(ROOT, "paper_1502_07303_gb300", "csrc", "fmm_march.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(path):
            f = line.split()
            if len(f) == 4 and not line.startswith("#") and f[0] == kernel and f[1] == dtype \
                    and f[2] == sha:
                return float(f[3])
        return None
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except Exception:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class NvmlClockSampler:
    """SM clock, its maximum and the clock-event reasons read through NVML
    (the driver's libnvidia-ml, reads only) every 10 ms from a thread during
    the timed region; start() returns False when NVML is unavailable."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index, period_s=0.01):
        self.index, self.period = index, period_s
        self.rows, self.stop_evt, self.lib, self.dev = [], threading.Event(), None, None

    def start(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return False
            dev = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(dev)) != 0:
                return False
            self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        except Exception:
            return False
        self.lib, self.dev, self.ct = lib, dev, ctypes
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()
        return True

    def _sample(self):
        ct, lib = self.ct, self.lib
        sm, mx, rs = ct.c_uint(0), ct.c_uint(0), ct.c_ulonglong(0)
        ok = (lib.nvmlDeviceGetClockInfo(self.dev, 1, ct.byref(sm)) == 0 and
              lib.nvmlDeviceGetMaxClockInfo(self.dev, 1, ct.byref(mx)) == 0)   # 1: SM clock
        if ok:
            self.reasons_fn(self.dev, ct.byref(rs))
            self.rows.append((sm.value, mx.value, rs.value))

    def _run(self):
        while not self.stop_evt.is_set():
            self._sample()
            time.sleep(self.period)

    def stop(self):
        self.stop_evt.set()
        self.t.join(timeout=2)
        self._sample()
        try:
            self.lib.nvmlShutdown()
        except Exception:
            pass
        reasons = sorted({name for _, _, r in self.rows for bit, name in self.REASONS.items() if r & bit})
        sm = [r[0] for r in self.rows]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(r[1] for r in self.rows) if self.rows else None,
                "reasons": reasons, "samples": len(sm), "source": "nvml"}


def clock_sampler(index):
    """NVML sampler, else the nvidia-smi one."""
    s = NvmlClockSampler(index)
    if s.start():
        return s
    s = ClockSampler(index)
    s.start()
    return s


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return ws, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v):
    if pg is None:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, v):
    if pg is None:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_rate(n):
    """One oracle solve of the workload recipe at n^3; returns (Gpoints/s, s)."""
    import oracle
    from paper_1502_07303_gb300 import workloads as wl
    oracle.build()
    p = wl.random_spheres(n=n, count=N_SPHERES, seed=SEED)
    t0 = time.perf_counter()
    oracle.solve_reinit(p.phi0, p.h)
    dt = time.perf_counter() - t0
    return p.n_points / dt / 1e9, dt


def run_reference(args):
    ws, rank, local, pg = dist_setup()
    if rank != 0:
        return 0
    import oracle
    from paper_1502_07303_gb300 import workloads as wl
    oracle.build()
    p = wl.random_spheres(n=REF_SAMPLE_N, count=N_SPHERES, seed=SEED)
    for _ in range(args.warmup):
        oracle.solve_reinit(p.phi0, p.h)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.solve_reinit(p.phi0, p.h)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = p.n_points / (ms / 1e3) / 1e9
    sample = (f"{N_SPHERES}-sphere reinitialisation recipe at {REF_SAMPLE_N}^3 "
              f"({p.n_points} points) per step, oracle fp64, 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"reinit random_spheres{N_SPHERES} {N_GRID}^3 (sampled at "
                                   f"{REF_SAMPLE_N}^3)", "seed": SEED},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def measure(fmm, torch, phi_dev, p, dtype, steps, warmup, flush, stream, params):
    """Device-timed solves: CUDA events around each solve on the solve's
    stream, L2 flushed (256 MiB write) before every step, outside the events."""
    shape = p.shape
    s = fmm.Solver(shape, p.h, dtype=dtype, time_kernels=True, stream=stream, **params)
    T_out = torch.empty(shape, dtype=dtype, device="cuda")
    G_out = torch.empty(shape, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        flush.fill_(1)
        s.reinit(phi_dev, T_out, G_out)
    torch.cuda.synchronize()
    step_ms, march_ms, march_l, launches = [], 0.0, 0, 0
    stats = None
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.reinit(phi_dev, T_out, G_out)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stats = s.stats()
        march_ms += stats["march_ms"]
        march_l += stats["march_launches"]
        launches += stats["kernel_launches"]
    s.close()
    return {"ms": statistics.mean(step_ms), "ms_min": min(step_ms), "march_ms": march_ms / steps,
            "march_launches": march_l / steps, "launches": launches, "stats": stats,
            "T": T_out}


def measure_e2e(fmm, torch, phi_host, p, dtype, steps, warmup, stream, params):
    """The user's call with host buffers: fmm_reinit_signed_distance takes
    pinned host phi0 and psi, copies phi0 to the device, solves and copies
    psi back before it returns, all inside the timed region of every step."""
    shape = p.shape
    s = fmm.Solver(shape, p.h, dtype=dtype, stream=stream, **params)
    T_host = torch.empty(shape, dtype=dtype, pin_memory=True)
    times = []
    for k in range(warmup + steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.reinit(phi_host, T_host, None, want_tags=False)
        e1.record(stream)
        e1.synchronize()
        if k >= warmup:
            times.append(e0.elapsed_time(e1))
    s.close()
    nbytes = phi_host.numel() * phi_host.element_size()
    return statistics.mean(times), nbytes, T_host.numel() * T_host.element_size()


def _events(torch, stream):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def measure_adjoint(fmm, torch, wl, stream, n=512, steps=2, warmup=1, dtypes=("f32", "f64")):
    """Heterogeneous speed F = exp(g/2) (16 random Fourier modes), 8 point
    sources, L = sum of psi at 64 receiver cells: forward solve with the tape
    and fmm_adjoint (dL/d slowness), each timed with CUDA events."""
    p = wl.fourier_sources(n=n, n_sources=8, n_receivers=64, seed=3, device="cuda")
    out = {"workload": f"fourier speed {n}^3, 8 sources, 64 receivers", "points": p.n_points}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        if name not in dtypes:
            continue
        F = p.speed.to(dt).contiguous()
        g = torch.zeros(p.shape, dtype=dt, device="cuda")
        for i, j, k in p.receivers:
            g[k, j, i] += 1.0
        s = fmm.Solver(p.shape, p.h, dtype=dt, speed=F, sources=p.sources, record_tape=True,
                       stream=stream)
        T = torch.empty(p.shape, dtype=dt, device="cuda")
        d = torch.empty(p.shape, dtype=dt, device="cuda")
        fw, bw = [], []
        for k in range(warmup + steps):
            e0, e1 = _events(torch, stream)
            e2, e3 = _events(torch, stream)
            e0.record(stream)
            s.solve(T, None, want_tags=False)
            e1.record(stream)
            e2.record(stream)
            s.adjoint(g, d)
            e3.record(stream)
            e3.synchronize()
            if k >= warmup:
                fw.append(e0.elapsed_time(e1))
                bw.append(e2.elapsed_time(e3))
        st = s.stats()
        s.close()
        fms, bms = statistics.mean(fw), statistics.mean(bw)
        out[name] = {"forward_gpts": p.n_points / fms / 1e6, "adjoint_gpts": p.n_points / bms / 1e6,
                     "forward_ms": fms, "adjoint_ms": bms, "adjoint_vs_forward": fms / bms,
                     "adjoint_iterations": st["adjoint_iterations"]}
    return out


def measure_batch(fmm, torch, wl, stream, steps=2, warmup=1):
    """256 independent grids (each axis uniform in [32, 192]), 1-8 random
    spheres each, fp32: one batched solve against the same grids solved one
    after another with single-grid handles."""
    probs = wl.batch(n_grids=256, lo=32, hi=192, seed=4, device="cuda")
    phis = [p.phi0.to(torch.float32).contiguous() for p in probs]
    pts = sum(p.n_points for p in probs)
    b = fmm.Batch([p.shape for p in probs], [p.h for p in probs], dtype=torch.float32,
                  stream=stream)
    Ts = [torch.empty(p.shape, dtype=torch.float32, device="cuda") for p in probs]
    tb = []
    for k in range(warmup + steps):
        e0, e1 = _events(torch, stream)
        e0.record(stream)
        b.reinit(phis, Ts, None, want_tags=False)
        e1.record(stream)
        e1.synchronize()
        if k >= warmup:
            tb.append(e0.elapsed_time(e1))
    st = b.stats()
    b.close()
    solvers = [fmm.Solver(p.shape, p.h, dtype=torch.float32, stream=stream) for p in probs]
    tp = []
    for k in range(warmup + steps):
        e0, e1 = _events(torch, stream)
        e0.record(stream)
        for s, ph, T in zip(solvers, phis, Ts):
            s.reinit(ph, T, None, want_tags=False)
        e1.record(stream)
        e1.synchronize()
        if k >= warmup:
            tp.append(e0.elapsed_time(e1))
    for s in solvers:
        s.close()
    bms, pms = statistics.mean(tb), statistics.mean(tp)
    return {"workload": "256 grids, axes uniform in [32, 192], 1-8 spheres each, fp32",
            "points": pts, "batched_gpts": pts / bms / 1e6, "batched_ms": bms,
            "plain_gpts": pts / pms / 1e6, "plain_ms": pms, "batched_vs_plain": pms / bms,
            "restarts": st["restarts"], "bricks": st["n_bricks"]}


def run_gpu(args):
    ws, rank, local, pg = dist_setup()
    import torch
    from paper_1502_07303_gb300 import fmm
    from paper_1502_07303_gb300 import workloads as wl

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    if args.part.startswith("adjoint"):
        # only the forward + adjoint pair of one dtype (for profiling)
        dt = args.part.split("-")[1]
        r = measure_adjoint(fmm, torch, wl, stream, n=args.adjoint_n, steps=args.steps,
                            warmup=args.warmup, dtypes=(dt,))
        if rank == 0:
            print(json.dumps({"part": args.part, **r}), flush=True)
        return 0
    n = args.n
    p = wl.random_spheres(n=n, count=N_SPHERES, seed=SEED, device="cuda")
    phi64 = p.phi0.contiguous()
    phi32 = phi64.to(torch.float32).contiguous()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    pts = p.n_points

    # restart parameters: the library's autotuner on this workload, before
    # any timed region (persistent schedule over strides, phased at default)
    from paper_1502_07303_gb300 import autotune
    tuned, tune_tables = {}, {}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        if args.params is not None:
            tuned[name] = dict(args.params)
            continue
        best, best_ms, table = autotune.tune(p, dt, kind="reinit", search=autotune.QUICK, reps=2,
                                             save=False, stream=stream)
        tuned[name] = best or {}
        tune_tables[name] = [[c, None if ms is None else round(ms, 3)] for c, ms in table]

    # fp32: the headline
    barrier(pg)
    torch.cuda.synchronize()
    sampler = clock_sampler(torch.cuda.current_device()) if rank == 0 else None
    t_wall = time.perf_counter()
    if args.part == "f64":
        r64 = measure(fmm, torch, phi64, p, torch.float64, args.steps, args.warmup, flush, stream,
                      tuned["f64"])
        if sampler:
            sampler.stop()
        if rank == 0:
            print(json.dumps({"part": "f64", "ms_per_step": r64["ms"], "params": tuned["f64"],
                              "march_ms": r64["march_ms"], "march_launches": r64["march_launches"],
                              "stats": r64["stats"]}), flush=True)
        return 0
    r32 = measure(fmm, torch, phi32, p, torch.float32, args.steps, args.warmup, flush, stream,
                  tuned["f32"])
    torch.cuda.synchronize()
    barrier(pg)
    wall_ms = 1e3 * (time.perf_counter() - t_wall)
    clocks = sampler.stop() if sampler else None
    ms32 = max_over_ranks(pg, r32["ms"])
    total_pts = sum_over_ranks(pg, float(pts))
    value = total_pts / (ms32 / 1e3) / 1e9
    if args.part == "f32":
        if rank == 0:
            print(json.dumps({"part": "f32", "value": value, "unit": UNIT, "ms_per_step": ms32,
                              "params": tuned["f32"], "march_ms": r32["march_ms"],
                              "march_launches": r32["march_launches"],
                              "stats": r32["stats"]}), flush=True)
        return 0

    # fp64 on the same workload
    r64 = measure(fmm, torch, phi64, p, torch.float64, args.steps, args.warmup, flush, stream,
                  tuned["f64"])
    ms64 = max_over_ranks(pg, r64["ms"])

    # end to end through the public API with host buffers (fp32)
    phi_host = phi32.cpu().pin_memory()
    e2e_ms, h2d, d2h = measure_e2e(fmm, torch, phi_host, p, torch.float32, args.steps,
                                   args.warmup, stream, tuned["f32"])
    e2e_ms = max_over_ranks(pg, e2e_ms)
    e2e_value = total_pts / (e2e_ms / 1e3) / 1e9

    adjoint = measure_adjoint(fmm, torch, wl, stream)
    batched = measure_batch(fmm, torch, wl, stream)

    if rank != 0:
        return 0

    peak, peak_kind = peaks()

    def roofline(r, dt):
        kernel = {1: "k_march", 2: "k_march_persistent"}.get(tuned[dt].get("schedule", 0),
                                                              "k_march_continuous")
        launches = max(r["march_launches"], 1.0)
        avg_launch_s = r["march_ms"] / launches / 1e3
        alg_per_launch = ALG_BYTES[dt] * pts / launches
        achieved = alg_per_launch / avg_launch_s / 1e9 if avg_launch_s > 0 else 0.0
        bpp = traffic_record(kernel, dt)
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": (bpp * pts / launches) if bpp else None,
                "kernel": kernel, "peak_kind": peak_kind,
                "avg_launch_us": 1e3 * r["march_ms"] / launches,
                "launches_per_step": r["march_launches"],
                "share_of_step": r["march_ms"] / r["ms"]}

    cpu_rate, cpu_s = oracle_rate(CPU_BASELINE_N) if ws == 1 else (None, None)
    st = r32["stats"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"reinit random_spheres{N_SPHERES} {n}^3", "grid": [n, n, n],
                   "points_per_gpu": pts, "seed": SEED,
                   "restart_params": {"f32": tuned["f32"], "f64": tuned["f64"],
                                      "chosen_by": ("given with --params" if args.params is not None
                                                    else "autotune.QUICK on this workload before "
                                                         "timing (ms per candidate in tune_ms)"),
                                      "tune_ms": tune_tables},
                   "brick": 8, "l2": "flushed before every step (256 MiB write)",
                   "replicas": ws, "parallelism": "independent replicas, no collective"},
        "roofline": roofline(r32, "f32"),
        "cpu_baseline": ({"value": cpu_rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                          "sample": f"{N_SPHERES}-sphere reinitialisation recipe at "
                                    f"{CPU_BASELINE_N}^3, oracle fp64, 1 thread, {cpu_s:.1f} s"}
                         if cpu_rate is not None else None),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": r32["launches"],
        "clocks": clocks,
        "fp64": {"value": total_pts / (ms64 / 1e3) / 1e9, "ms_per_step": ms64,
                 "roofline": roofline(r64, "f64")},
        "adjoint": adjoint,
        "batched": batched,
        "solve_stats": {k: st[k] for k in ("restarts", "brick_marches", "march_rounds",
                                            "exchanges", "accepted", "cell_solves", "n_bricks")},
        "wall_ms_timed_region": wall_ms,
    }
    print(json.dumps(line), flush=True)
    return 0


def _params(text):
    d = json.loads(text)
    return {k: (float(v) if k in ("stride", "bucket") else int(v)) for k, v in d.items()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N_GRID, help=argparse.SUPPRESS)
    ap.add_argument("--part", default="all", choices=["all", "f32", "f64", "adjoint-f32", "adjoint-f64"],
                    help="f32 / f64: only the timed solves of one dtype; adjoint-f32 / "
                         "adjoint-f64: only the forward + adjoint pair (for profiling)")
    ap.add_argument("--adjoint-n", type=int, default=512,
                    help="grid size of the adjoint workload of --part adjoint-*")
    ap.add_argument("--params", type=_params, default=None,
                    help="restart parameters as JSON (skips the autotuner), e.g. "
                         "'{\"schedule\": 2, \"stride\": \"inf\"}'")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
