#!/usr/bin/env python
"""Throughput benchmark of the GB300 restarted narrow band fast marching library.

Headline workload (one "step" = one complete solve through the C ABI):
signed-distance reinitialisation of one sphere of radius 0.3 centred in a
1024^3 unit cube (1.07 G points), full march, fp64 (the paper's precision),
with the restart parameters the library's autotuner picks for it.  The metric
is grid points finalised per second (Gpoints/s).  Beside it: the same solve in
fp32, the 256^3 32-sphere reinitialisation, the 64^3 point source, the 512^3
heterogeneous-speed forward solve and its adjoint, and the 256-grid batch.

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
N_GRID = 1024               # headline: single sphere, 1024^3
RADIUS = 0.3
N_C2, N_SPHERES, SEED = 256, 32, 2
# algorithmic bytes per finalised point: a reinitialisation reads phi0 and
# writes psi and the tag once (fp32: 4 + 4 + 1, fp64: 8 + 8 + 1); a point-
# source solve with constant speed writes psi and the tag; a heterogeneous
# solve also reads F
ALG_BYTES = {"reinit": {"f32": 9, "f64": 17}, "sources": {"f32": 5, "f64": 9},
             "sources_speed": {"f32": 9, "f64": 17}}
REF_SAMPLE_N = 192          # oracle sample grid of the reference arm
CPU_BASELINE_N = 256        # oracle sample grid of the cpu_baseline entry
CPU_BATCH_GRIDS = 48        # grids of the batched workload the oracle solves on all cores


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _profile_record(fname, kernel, dtype, workload):
    """A per-point figure of a march kernel from a committed ncu summary
    (lines "kernel dtype workload source_sha256_16 value"), valid only while
    the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", fname)
    src = os.path.join(ROOT, "paper_1502_07303_gb300", "csrc", "fmm_march.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(path):
            f = line.split()
            if len(f) == 5 and not line.startswith("#") and f[0] == kernel and f[1] == dtype \
                    and f[2] == workload and f[3] == sha:
                return float(f[4])
        return None
    except Exception:
        return None


def traffic_record(kernel, dtype, workload):
    """DRAM bytes (read + write) per finalised point."""
    return _profile_record("k_march_traffic.txt", kernel, dtype, workload)


def issue_record(kernel, dtype, workload):
    """Warp instructions issued per finalised point."""
    return _profile_record("k_march_issue.txt", kernel, dtype, workload)


def dpipe_record(kernel, dtype, workload):
    """Double-pipe thread instructions (DFMA + DADD + DMUL) per finalised point."""
    return _profile_record("k_march_dpipe.txt", kernel, dtype, workload)


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
    """One oracle solve of the headline recipe (single sphere) at n^3;
    returns (Gpoints/s, s)."""
    import oracle
    from paper_1502_07303_gb300 import workloads as wl
    oracle.build()
    p = wl.single_sphere(n=n, radius=RADIUS)
    t0 = time.perf_counter()
    oracle.solve_reinit(p.phi0, p.h)
    dt = time.perf_counter() - t0
    return p.n_points / dt / 1e9, dt


def oracle_batch_rate(sample):
    """The oracle on a sample of the batched workload's grids (the fp32 level
    sets the batch solves, as (phi0, h) host pairs), one grid per thread on a
    pool over all host cores; returns (Gpoints/s, s, cores, points)."""
    import concurrent.futures

    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with concurrent.futures.ThreadPoolExecutor(max_workers=cores) as pool:
        list(pool.map(lambda a: oracle.solve_reinit(a[0], a[1]), sample))
    dt = time.perf_counter() - t0
    pts = sum(a[0].size for a in sample)
    return pts / dt / 1e9, dt, cores, pts


def run_reference(args):
    ws, rank, local, pg = dist_setup()
    if rank != 0:
        return 0
    import oracle
    from paper_1502_07303_gb300 import workloads as wl
    oracle.build()
    p = wl.single_sphere(n=REF_SAMPLE_N, radius=RADIUS)
    for _ in range(args.warmup):
        oracle.solve_reinit(p.phi0, p.h)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.solve_reinit(p.phi0, p.h)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = p.n_points / (ms / 1e3) / 1e9
    sample = (f"single-sphere reinitialisation recipe (r = {RADIUS}) at {REF_SAMPLE_N}^3 "
              f"({p.n_points} points) per step, oracle fp64, 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"reinit single sphere r={RADIUS} {N_GRID}^3 (sampled at "
                                   f"{REF_SAMPLE_N}^3)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def measure(fmm, torch, p, dtype, steps, warmup, flush, stream, params, phi=None, speed=None):
    """Device-timed solves of problem p (reinitialisation of phi, or a
    point-source solve): CUDA events around each solve on the solve's
    stream, L2 flushed (256 MiB write) before every step, outside the events."""
    s = fmm.Solver(p.shape, p.h, dtype=dtype, time_kernels=True, stream=stream, speed=speed,
                   sources=None if phi is not None else p.sources, tuned=False, **params)
    T_out = torch.empty(p.shape, dtype=dtype, device="cuda")
    G_out = torch.empty(p.shape, dtype=torch.uint8, device="cuda")

    def solve():
        if phi is not None:
            s.reinit(phi, T_out, G_out)
        else:
            s.solve(T_out, G_out)
    for _ in range(warmup):
        flush.fill_(1)
        solve()
    torch.cuda.synchronize()
    step_ms, march_ms, march_l, launches = [], 0.0, 0, 0
    stats = None
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = _events(torch)
        e0.record(stream)
        solve()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stats = s.stats()
        march_ms += stats["march_ms"]
        march_l += stats["march_launches"]
        launches += stats["kernel_launches"]
    s.close()
    del T_out, G_out
    return {"ms": statistics.mean(step_ms), "ms_min": min(step_ms), "march_ms": march_ms / steps,
            "march_launches": march_l / steps, "launches": launches, "stats": stats}


def measure_e2e(fmm, torch, phi_host, p, dtype, steps, warmup, stream, params):
    """The user's call with host buffers: fmm_reinit_signed_distance takes
    pinned host phi0 and psi, copies phi0 to the device, solves and copies
    psi back before it returns, all inside the timed region of every step."""
    s = fmm.Solver(p.shape, p.h, dtype=dtype, stream=stream, tuned=False, **params)
    T_host = torch.empty(p.shape, dtype=dtype, pin_memory=True)
    times = []
    for k in range(warmup + steps):
        e0, e1 = _events(torch)
        e0.record(stream)
        s.reinit(phi_host, T_host, None, want_tags=False)
        e1.record(stream)
        e1.synchronize()
        if k >= warmup:
            times.append(e0.elapsed_time(e1))
    s.close()
    nbytes = phi_host.numel() * phi_host.element_size()
    measure_e2e.step_ms = [round(t, 1) for t in times]
    return statistics.mean(times), nbytes, T_host.numel() * T_host.element_size()


# bytes one bucket step of the cell-parallel march streams per cell (brick
# layout, fp64): accept reads psi + tag (9), relax reads psi + tag (9; the
# neighbours' values come from L1/L2), apply reads psi + tag + the new-value
# buffer (17)
CELL_STEP_BYTES = {"f64": 35, "f32": 19}


def measure_second_order(fmm, torch, wl, stream, flush, n=256, steps=3, warmup=2):
    """The cell-parallel march (schedule 4) in first and second order on the
    single-sphere reinitialisation (fp64), with the error of each against
    the exact signed distance (phi0 is exact for one sphere), and the brick
    march (first order, library defaults) on the same workload for scale.
    Roofline: the bytes the march's grid-wide passes stream per bucket step
    (CELL_STEP_BYTES per brick-layout cell) over the device time of the
    march, against the measured copy peak."""
    p = wl.single_sphere(n=n, radius=RADIUS, device="cuda")
    phi = p.phi0.contiguous()
    exact = phi.abs()
    out = {"workload": f"reinit single sphere r={RADIUS} centred, {n}^3, fp64", "points": p.n_points}
    cells = ((n + 7) // 8) ** 3 * 512
    peak, peak_kind = peaks()
    for name, prm in (("brick_first_order", {}), ("cell_first_order", {"schedule": 4}),
                      ("cell_second_order", {"schedule": 4, "accuracy": 2})):
        r = measure(fmm, torch, p, torch.float64, steps, warmup, flush, stream, prm, phi=phi)
        with fmm.Solver(p.shape, p.h, dtype=torch.float64, stream=stream, tuned=False, **prm) as s:
            T, _ = s.reinit(phi)
        err = (T.abs() - exact).abs()
        rec = {"ms": r["ms"], "gpts": p.n_points / r["ms"] / 1e6, "params": prm,
               "err_max": float(err.max()), "err_mean": float(err.mean()),
               "accepted_per_point": r["stats"]["accepted"] / p.n_points}
        if prm.get("schedule") == 4:
            # bucket steps that accepted cells, plus the one that ended the
            # march (steps enqueued after it return at once)
            nsteps = r["stats"]["restarts"] + 1
            achieved = CELL_STEP_BYTES["f64"] * cells * nsteps / (r["march_ms"] / 1e3) / 1e9
            rec["bucket_steps"] = nsteps
            rec["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                               "frac": achieved / peak, "peak_kind": peak_kind,
                               "bytes_per_cell_per_step": CELL_STEP_BYTES["f64"],
                               "kernels": "k_cell_accept + k_cell_relax + k_cell_apply",
                               "march_ms": r["march_ms"], "share_of_step": r["march_ms"] / r["ms"]}
        out[name] = rec
        del T, err
    out["second_vs_first_order_err_mean"] = out["cell_first_order"]["err_mean"] / out["cell_second_order"]["err_mean"]
    del p, phi, exact
    torch.cuda.empty_cache()
    return out


def measure_adjoint(fmm, torch, wl, stream, n=512, steps=2, warmup=1, dtypes=("f32", "f64"),
                    params=None):
    """Heterogeneous speed F = exp(g/2) (16 random Fourier modes), 8 point
    sources, L = sum of psi at 64 receiver cells: forward solve with the tape
    and fmm_adjoint (dL/d slowness), each timed with CUDA events; the plain
    forward solve without a tape beside them."""
    p = wl.fourier_sources(n=n, n_sources=8, n_receivers=64, seed=3, device="cuda")
    out = {"workload": f"fourier speed {n}^3, 8 sources, 64 receivers", "points": p.n_points}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        if name not in dtypes:
            continue
        prm = (params or {}).get(name, {})
        F = p.speed.to(dt).contiguous()
        g = torch.zeros(p.shape, dtype=dt, device="cuda")
        for i, j, k in p.receivers:
            g[k, j, i] += 1.0
        s = fmm.Solver(p.shape, p.h, dtype=dt, speed=F, sources=p.sources, record_tape=True,
                       stream=stream, tuned=False, **prm)
        plain = fmm.Solver(p.shape, p.h, dtype=dt, speed=F, sources=p.sources, stream=stream,
                           tuned=False, **prm)
        T = torch.empty(p.shape, dtype=dt, device="cuda")
        d = torch.empty(p.shape, dtype=dt, device="cuda")
        fw, bw, pl = [], [], []
        for k in range(warmup + steps):
            e0, e1 = _events(torch)
            e0.record(stream)
            plain.solve(T, None, want_tags=False)
            e1.record(stream)
            e2, e3 = _events(torch)
            e4, e5 = _events(torch)
            e2.record(stream)
            s.solve(T, None, want_tags=False)
            e3.record(stream)
            e4.record(stream)
            s.adjoint(g, d)
            e5.record(stream)
            e5.synchronize()
            if k >= warmup:
                pl.append(e0.elapsed_time(e1))
                fw.append(e2.elapsed_time(e3))
                bw.append(e4.elapsed_time(e5))
        st = s.stats()
        s.close()
        plain.close()
        pms, fms, bms = statistics.mean(pl), statistics.mean(fw), statistics.mean(bw)
        out[name] = {"forward_gpts": p.n_points / pms / 1e6, "forward_ms": pms,
                     "forward_tape_ms": fms, "adjoint_gpts": p.n_points / bms / 1e6,
                     "adjoint_ms": bms, "adjoint_vs_forward": pms / bms,
                     "adjoint_iterations": st["adjoint_iterations"], "params": prm}
    return out


def measure_batch(fmm, torch, wl, autotune, stream, steps=2, warmup=1, tune=True):
    """256 independent grids (each axis uniform in [32, 192]), 1-8 random
    spheres each, fp32: one batched solve (restart parameters from the batch
    autotuner) against the same grids solved one after another with
    single-grid handles."""
    probs = wl.batch(n_grids=256, lo=32, hi=192, seed=4, device="cuda")
    phis = [p.phi0.to(torch.float32).contiguous() for p in probs]
    pts = sum(p.n_points for p in probs)
    # host copies of the first grids for the all-cores oracle baseline
    measure_batch.sample = [(ph.double().cpu().numpy(), p.h) for ph, p in
                            zip(phis[:CPU_BATCH_GRIDS], probs[:CPU_BATCH_GRIDS])]
    best, table = {}, []
    if tune:
        best, _, table = autotune.tune_batch(probs, torch.float32, search=autotune.QUICK, reps=2,
                                             save=False, stream=stream)
        best = best or {}
    b = fmm.Batch([p.shape for p in probs], [p.h for p in probs], dtype=torch.float32,
                  stream=stream, tuned=False, **best)
    Ts = [torch.empty(p.shape, dtype=torch.float32, device="cuda") for p in probs]
    tb = []
    for k in range(warmup + steps):
        e0, e1 = _events(torch)
        e0.record(stream)
        b.reinit(phis, Ts, None, want_tags=False)
        e1.record(stream)
        e1.synchronize()
        if k >= warmup:
            tb.append(e0.elapsed_time(e1))
    st = b.stats()
    b.close()
    solvers = [fmm.Solver(p.shape, p.h, dtype=torch.float32, stream=stream, tuned=False, **best)
               for p in probs]
    tp = []
    for k in range(warmup + steps):
        e0, e1 = _events(torch)
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
            "restarts": st["restarts"], "bricks": st["n_bricks"],
            "params": dict(best, brick=8, chosen_by="autotune.tune_batch(QUICK) before timing"),
            "tune_ms": [[c, None if ms is None else round(ms, 3)] for c, ms in table]}


def tune_params(autotune, torch, p, dt, stream, kind, search=None):
    best, _, table = autotune.tune(p, dt, kind=kind, search=search or autotune.QUICK, reps=2,
                                   save=False, stream=stream)
    return best or {}, [[c, None if ms is None else round(ms, 3)] for c, ms in table]


def roofline_hbm(r, pts, alg, kernel, dt, workload, peak, peak_kind):
    """HBM roofline of the dominant kernel: algorithmic bytes of one launch
    over its average CUDA-event duration, against the measured copy peak."""
    launches = max(r["march_launches"], 1.0)
    avg_s = r["march_ms"] / launches / 1e3
    achieved = alg * pts / launches / avg_s / 1e9 if avg_s > 0 else 0.0
    bpp = traffic_record(kernel, dt, workload)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": (bpp * pts / launches) if bpp else None,
            "kernel": kernel, "peak_kind": peak_kind, "alg_bytes_per_point": alg,
            "avg_launch_us": 1e3 * r["march_ms"] / launches,
            "launches_per_step": r["march_launches"], "share_of_step": r["march_ms"] / r["ms"]}


def roofline_alu(r, pts, kernel, dt, workload, fp64_peak, sms, sm_mhz):
    """Instruction-issue roofline of the dominant kernel: warp instructions
    issued per launch (ncu's count per point x points) over the launch time,
    against the issue rate of the SMs (4 schedulers x 1 warp instruction per
    clock x SMs x the clock sampled during the run).  For fp64 the double
    pipe is given beside it: double-pipe thread instructions (DFMA + DADD +
    DMUL) per second against the measured double FMA rate
    (fmm_probe_fma_rate / 2: each of them occupies the pipe like an FMA)."""
    launches = max(r["march_launches"], 1.0)
    avg_s = r["march_ms"] / launches / 1e3
    per_pt = issue_record(kernel, dt, workload)
    peak = 4 * sms * sm_mhz * 1e6 / 1e12
    ach = per_pt * pts / launches / avg_s / 1e12 if (per_pt and avg_s > 0) else None
    out = {"bound": "alu", "pipe": "issue", "achieved": ach, "peak": peak, "unit": "Tinst/s",
           "frac": (ach / peak) if ach else None, "kernel": kernel,
           "peak_kind": f"derived: 4 warp instructions per clock per SM x {sms} SMs x {sm_mhz:.0f} MHz",
           "ops_per_point": per_pt}
    if dt == "f64":
        dp = dpipe_record(kernel, dt, workload)
        dpeak = fp64_peak / 2 / 1e12 if fp64_peak else None
        dach = dp * pts / launches / avg_s / 1e12 if (dp and avg_s > 0) else None
        out["fp64_pipe"] = {"achieved": dach, "peak": dpeak, "unit": "T double-pipe instructions/s",
                            "frac": (dach / dpeak) if (dach and dpeak) else None,
                            "peak_kind": "measured (fmm_probe_fma_rate, double FMA chains, FMAs/s)",
                            "ops_per_point": dp}
    return out


def kernel_name(params):
    return {1: "k_march", 2: "k_march_persistent"}.get(params.get("schedule", 0), "k_march_continuous")


def run_gpu(args):
    ws, rank, local, pg = dist_setup()
    import torch
    from paper_1502_07303_gb300 import autotune, fmm
    from paper_1502_07303_gb300 import workloads as wl

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    if args.part.startswith("adjoint"):
        # only the forward + adjoint pair of one dtype (for profiling)
        dt = args.part.split("-")[1]
        prm = {dt: dict(args.params)} if args.params is not None else None
        r = measure_adjoint(fmm, torch, wl, stream, n=args.adjoint_n, steps=args.steps,
                            warmup=args.warmup, dtypes=(dt,), params=prm)
        if rank == 0:
            print(json.dumps({"part": args.part, **r}), flush=True)
        return 0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    DTS = {"f32": torch.float32, "f64": torch.float64}

    if args.part == "so":
        # only the second-order / cell-parallel measurement (for profiling)
        r = measure_second_order(fmm, torch, wl, stream, flush, n=args.n or 256, steps=args.steps,
                                 warmup=args.warmup)
        if rank == 0:
            print(json.dumps({"part": args.part, **r}), flush=True)
        return 0

    if args.part in ("c2-f32", "c2-f64", "c5-f32", "c5-f64"):
        # one timed solve series of one workload and dtype (for profiling)
        w, name = args.part.split("-")
        n = args.n or (N_C2 if w == "c2" else N_GRID)
        p = (wl.random_spheres(n=n, count=N_SPHERES, seed=SEED, device="cuda") if w == "c2"
             else wl.single_sphere(n=n, radius=RADIUS, device="cuda"))
        phi = p.phi0.to(DTS[name]).contiguous()
        prm = dict(args.params) if args.params is not None else {}
        r = measure(fmm, torch, p, DTS[name], args.steps, args.warmup, flush, stream, prm, phi=phi)
        if rank == 0:
            print(json.dumps({"part": args.part, "n": n, "ms_per_step": r["ms"], "params": prm,
                              "march_ms": r["march_ms"], "march_launches": r["march_launches"],
                              "stats": r["stats"]}), flush=True)
        return 0

    n = args.n or N_GRID
    p = wl.single_sphere(n=n, radius=RADIUS, device="cuda")
    pts = p.n_points
    tuned, tune_tables = {}, {}
    phis = {"f64": p.phi0.contiguous(), "f32": p.phi0.to(torch.float32).contiguous()}
    for name in ("f64", "f32"):
        if args.params is not None:
            tuned[name] = dict(args.params)
            continue
        tuned[name], tune_tables[name] = tune_params(autotune, torch, p, DTS[name], stream, "reinit")
    # hand the tuner's device buffers back to the driver before the timed
    # runs (kept in torch's cache they slowed the later host copies of the
    # end-to-end call by half)
    torch.cuda.empty_cache()

    # the headline: fp64, then fp32 on the same workload
    barrier(pg)
    torch.cuda.synchronize()
    sampler = clock_sampler(torch.cuda.current_device()) if rank == 0 else None
    t_wall = time.perf_counter()
    r64 = measure(fmm, torch, p, torch.float64, args.steps, args.warmup, flush, stream,
                  tuned["f64"], phi=phis["f64"])
    torch.cuda.synchronize()
    barrier(pg)
    wall_ms = 1e3 * (time.perf_counter() - t_wall)
    clocks = sampler.stop() if sampler else None
    ms64 = max_over_ranks(pg, r64["ms"])
    total_pts = sum_over_ranks(pg, float(pts))
    value = total_pts / (ms64 / 1e3) / 1e9
    r32 = measure(fmm, torch, p, torch.float32, args.steps, args.warmup, flush, stream,
                  tuned["f32"], phi=phis["f32"])
    ms32 = max_over_ranks(pg, r32["ms"])

    # end to end through the public API with host buffers (fp64)
    phi_host = phis["f64"].cpu().pin_memory()
    del phis
    e2e_ms, h2d, d2h = measure_e2e(fmm, torch, phi_host, p, torch.float64, args.steps,
                                   args.warmup, stream, tuned["f64"])
    del phi_host
    e2e_ms = max_over_ranks(pg, e2e_ms)
    e2e_value = total_pts / (e2e_ms / 1e3) / 1e9
    del p
    torch.cuda.empty_cache()

    others = {}
    if not args.quick:
        # the 256^3 32-sphere reinitialisation and the 64^3 point source
        c2 = wl.random_spheres(n=N_C2, count=N_SPHERES, seed=SEED, device="cuda")
        others["c2"] = {"workload": f"reinit random_spheres{N_SPHERES} {N_C2}^3",
                        "points": c2.n_points}
        for name in ("f32", "f64"):
            phi = c2.phi0.to(DTS[name]).contiguous()
            prm, tab = tune_params(autotune, torch, c2, DTS[name], stream, "reinit")
            r = measure(fmm, torch, c2, DTS[name], args.steps, args.warmup, flush, stream, prm,
                        phi=phi)
            others["c2"][name] = {"gpts": c2.n_points / r["ms"] / 1e6, "ms": r["ms"], "params": prm,
                                  "accepted_per_point": r["stats"]["accepted"] / c2.n_points,
                                  "solves_per_point": r["stats"]["cell_solves"] / c2.n_points,
                                  "marches_per_brick": r["stats"]["brick_marches"] / r["stats"]["n_bricks"]}
            # the bit-reproducible mode (phased schedule, pass-synchronous
            # halos), library defaults otherwise: what reproducibility costs
            rd = measure(fmm, torch, c2, DTS[name], args.steps, args.warmup, flush, stream,
                         {"deterministic": True}, phi=phi)
            others["c2"][name]["deterministic"] = {
                "gpts": c2.n_points / rd["ms"] / 1e6, "ms": rd["ms"], "time_vs_default": rd["ms"] / r["ms"],
                "restarts": rd["stats"]["restarts"], "marches_per_brick":
                    rd["stats"]["brick_marches"] / rd["stats"]["n_bricks"]}
        del c2, phi
        c1 = wl.point_source(64)
        prm, _ = tune_params(autotune, torch, c1, torch.float64, stream, "sources")
        r = measure(fmm, torch, c1, torch.float64, args.steps, args.warmup, flush, stream, prm)
        others["c1"] = {"workload": "point source at cell (32, 32, 32) of 64^3, F = 1, fp64",
                        "points": c1.n_points, "gpts": c1.n_points / r["ms"] / 1e6, "ms": r["ms"],
                        "params": prm}
        adj_params = {}
        c3 = wl.fourier_sources(n=512, n_sources=8, n_receivers=64, seed=3, device="cuda")
        for name in ("f32", "f64"):
            c3t = wl.Problem(c3.name, c3.shape, c3.h, sources=c3.sources,
                             speed=c3.speed.to(DTS[name]).contiguous())
            adj_params[name], _ = tune_params(autotune, torch, c3t, DTS[name], stream, "sources_speed")
            del c3t
        del c3
        torch.cuda.empty_cache()
        others["adjoint"] = measure_adjoint(fmm, torch, wl, stream, params=adj_params)
        others["batched"] = measure_batch(fmm, torch, wl, autotune, stream)
        others["second_order"] = measure_second_order(fmm, torch, wl, stream, flush,
                                                      steps=min(args.steps, 3), warmup=1)

    if rank != 0:
        return 0
    peak, peak_kind = peaks()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    try:
        sm_mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except Exception:
        sm_mhz = 2070.0
    fp64_peak = fmm.probe_fma_rate(torch.float64, iters=1 << 15)
    fp32_fma_peak = fmm.probe_fma_rate(torch.float32, iters=1 << 20)
    wname = f"sphere{n}"
    k64, k32 = kernel_name(tuned["f64"]), kernel_name(tuned["f32"])
    cpu_rate, cpu_s = oracle_rate(CPU_BASELINE_N) if ws == 1 else (None, None)
    if ws == 1 and "batched" in others:
        # the batched workload's oracle on all host cores (a bounded sample)
        r, t, cores, bpts = oracle_batch_rate(measure_batch.sample)
        others["batched"]["cpu_baseline"] = {
            "value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the first {CPU_BATCH_GRIDS} of the 256 grids ({bpts} points), one grid per "
                      f"thread on a pool of {cores} host threads, oracle fp64, {t:.1f} s"}
    st = r64["stats"]
    st32 = r32["stats"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"reinit single sphere r={RADIUS} centred, {n}^3 unit cube, full march",
                   "grid": [n, n, n], "points_per_gpu": pts,
                   "restart_params": {"f64": tuned["f64"], "f32": tuned["f32"],
                                      "chosen_by": ("given with --params" if args.params is not None
                                                    else "autotune.QUICK on this workload before "
                                                         "timing (ms per candidate in tune_ms)"),
                                      "tune_ms": tune_tables},
                   "brick": 8, "l2": "inputs (phi0 8.6 GB fp64) larger than L2; also flushed "
                                     "before every step (256 MiB write)",
                   "replicas": ws, "parallelism": "independent replicas, no collective"},
        "roofline": roofline_hbm(r64, pts, ALG_BYTES["reinit"]["f64"], k64, "f64", wname, peak,
                                 peak_kind),
        "roofline_alu": roofline_alu(r64, pts, k64, "f64", wname, fp64_peak, sms, sm_mhz),
        "cpu_baseline": ({"value": cpu_rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                          "sample": f"single-sphere reinitialisation recipe at {CPU_BASELINE_N}^3 "
                                    f"({CPU_BASELINE_N ** 3} points), oracle fp64, 1 thread, "
                                    f"{cpu_s:.1f} s"}
                         if cpu_rate is not None else None),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "call": "fmm_reinit_signed_distance with pinned host phi0 and psi (fp64)",
                "step_ms": getattr(measure_e2e, "step_ms", None)},
        "gpu_launches": r64["launches"],
        "clocks": clocks,
        "fp32": {"value": total_pts / (ms32 / 1e3) / 1e9, "ms_per_step": ms32,
                 "roofline": roofline_hbm(r32, pts, ALG_BYTES["reinit"]["f32"], k32, "f32", wname,
                                          peak, peak_kind),
                 "roofline_alu": roofline_alu(r32, pts, k32, "f32", wname, fp64_peak, sms, sm_mhz),
                 "solve_stats": {k: st32[k] for k in ("restarts", "brick_marches", "march_rounds",
                                                      "accepted", "cell_solves", "n_bricks")}},
        "peaks_measured_here": {"fp64_fma_tflops": fp64_peak / 1e12,
                                "fp32_fma_tflops": fp32_fma_peak / 1e12},
        "solve_stats": {k: st[k] for k in ("restarts", "brick_marches", "march_rounds",
                                           "exchanges", "accepted", "cell_solves", "n_bricks")},
        "per_point": {"accepted": st["accepted"] / pts, "cell_solves": st["cell_solves"] / pts,
                      "marches_per_brick": st["brick_marches"] / st["n_bricks"]},
        "wall_ms_timed_region": wall_ms,
        **others,
    }
    print(json.dumps(line), flush=True)
    return 0


def _params(text):
    d = json.loads(text)
    return {k: (float(v) if k in ("stride", "bucket", "ahead") else int(v)) for k, v in d.items()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--quick", action="store_true",
                    help="only the headline workload (fp64 and fp32), no other configs")
    ap.add_argument("--part", default="all",
                    choices=["all", "c2-f32", "c2-f64", "c5-f32", "c5-f64", "adjoint-f32", "adjoint-f64",
                             "so"],
                    help="c2-* / c5-*: only the timed solves of one workload and dtype; "
                         "adjoint-*: only the forward + adjoint pair; so: only the cell-parallel "
                         "march in first and second order (for profiling)")
    ap.add_argument("--adjoint-n", type=int, default=512,
                    help="grid size of the adjoint workload of --part adjoint-*")
    ap.add_argument("--params", type=_params, default=None,
                    help="restart parameters as JSON (skips the autotuner), e.g. "
                         "'{\"schedule\": 3, \"stride\": 1, \"ahead\": \"inf\"}'")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
