"""Autotuner for the restart parameters of the GB300 solver.

The paper's only free parameter is the restart stride (Sec. 4.4, Sec. 5.1):
it studies 0.5-3.5 h and infinity, suggests 2 h for its CPU cluster and
advises experimenting on new platforms (Sec. 5.5).  On the GPU the stride,
the restart schedule (continuous, persistent queue or phased passes), the
look-ahead of a brick march beyond the bound, the bucket width of the local
march, the number of exchange passes per restart (phased schedule) and the
number of CTAs of the march kernel all trade restarts against
re-acceptance, so they are tuned together.  The brick is 8x8x8 (one warp per
brick, a 16-bit cell mask per lane); the CTA count sets how many bricks march
at once.

``tune`` times every candidate on a representative problem with CUDA events
and stores the fastest in a JSON cache keyed by (problem kind, dtype, size
class = round(log2(points))); ``params_for`` reads it back (an empty dict, so
the library defaults, when the class has no entry).  ``fmm.Solver`` and
``fmm.Batch`` consult the cache for every parameter the caller leaves unset.
Timing uses the CUDA library only.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import statistics

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                             "autotune.json")

PARAMS = ("schedule", "stride", "bucket", "exchange_passes", "ctas", "max_lead", "ahead")

SEARCH = {
    "schedule": [1, 2, 3],
    "stride": [0.5, 1.0, 2.0, 4.0, 8.0, math.inf],
    "bucket": [2.0, 3.0, 4.0, 6.0],
    "exchange_passes": [1, 2],
    "ctas": [0, 152 * 2, 152 * 4],
    "max_lead": [0],
    "ahead": [math.inf, 8.0],
}

# A short list for a quick tune: the continuous schedule with a whole-brick
# look-ahead over strides and bucket widths (around the fp64 optimum of 1 h
# and the fp32 one of 2 h), at the full and at a reduced CTA count, and the
# persistent schedule without restarts.
QUICK = ([{"schedule": 3, "stride": s, "bucket": 4.0, "ahead": math.inf}
          for s in (0.5, 1.0, 1.5, 2.0, 3.0, 4.0)]
         + [{"schedule": 3, "stride": 1.0, "bucket": b, "ahead": math.inf} for b in (5.0, 6.0)]
         + [{"schedule": 3, "stride": 2.0, "bucket": b, "ahead": math.inf} for b in (3.0, 6.0)]
         + [{"schedule": 3, "stride": 1.0, "bucket": 4.0, "ahead": math.inf, "ctas": 152 * 4}]
         + [{"schedule": 2, "stride": math.inf, "bucket": 4.0}])


def cache_path(path=None):
    return path or os.environ.get("FMM_GB300_TUNE_CACHE", DEFAULT_CACHE)


def size_class(n_points):
    return int(round(math.log2(max(int(n_points), 1))))


def key(kind, dtype_name, n_points):
    return f"{kind}/{dtype_name}/{size_class(n_points)}"


def _dtype_name(dtype):
    s = str(dtype)
    return "f64" if "64" in s else "f32"


def load_cache(path=None):
    p = cache_path(path)
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=None):
    p = cache_path(path)
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def params_for(kind, dtype, n_points, path=None):
    """Tuned parameters for a problem, or {} (library defaults) when the
    cache has no entry for its class."""
    entry = load_cache(path).get(key(kind, _dtype_name(dtype), n_points))
    if not entry:
        return {}
    return {k: entry[k] for k in PARAMS if k in entry}


def merge(given, kind, dtype, n_points, path=None):
    """The caller's parameters, completed from the cache: every tuned
    parameter the caller left at its default (0) takes the cached value."""
    out = dict(given)
    for k, v in params_for(kind, dtype, n_points, path).items():
        if not out.get(k):
            out[k] = v
    return out


def candidates(search=None):
    """search: a dict of value lists (the product is taken, missing keys from
    SEARCH) or an explicit list of parameter dicts."""
    if isinstance(search, (list, tuple)):
        yield from (dict(c) for c in search)
        return
    sp = dict(SEARCH)
    if search:
        sp.update(search)
    for vals in itertools.product(*(sp[n] for n in PARAMS)):
        yield dict(zip(PARAMS, vals))


def select_best(timings):
    """timings: list of (params, ms).  Fastest wins; ties keep the first."""
    best = None
    for params, ms in timings:
        if ms is None or not math.isfinite(ms):
            continue
        if best is None or ms < best[1]:
            best = (params, ms)
    return best


def _time_call(torch, fn, reps):
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return min(ts)


def tune(problem, dtype, kind=None, search=None, reps=2, path=None, save=True, log=None,
         stream=None):
    """Time every candidate on ``problem`` (a workloads.Problem with phi0 or
    sources) and store the fastest.  Returns (best_params, best_ms, table)."""
    import torch

    from . import fmm

    kind = kind or ("reinit" if problem.phi0 is not None else
                    ("sources_speed" if problem.speed is not None else "sources"))
    phi = None
    if problem.phi0 is not None:
        phi = torch.as_tensor(problem.phi0, dtype=dtype, device="cuda").contiguous()
    speed = None
    if problem.speed is not None:
        speed = torch.as_tensor(problem.speed, dtype=dtype, device="cuda").contiguous()
    table = []
    T = torch.empty(problem.shape, dtype=dtype, device="cuda")
    for params in candidates(search):
        try:
            with fmm.Solver(problem.shape, problem.h, dtype=dtype, speed=speed,
                            sources=problem.sources, stream=stream, tuned=False, **params) as s:
                if phi is not None:
                    def run():
                        s.reinit(phi, T, None, want_tags=False)
                else:
                    def run():
                        s.solve(T, None, want_tags=False)
                run()
                ms = _time_call(torch, run, reps)
        except fmm.FmmError:
            ms = None
        table.append((params, ms))
        if log:
            log(params, ms)
    best = select_best(table)
    if best is None:
        return None, None, table
    if save:
        cache = load_cache(path)
        entry = dict(best[0])
        entry["ms"] = best[1]
        entry["points"] = problem.n_points
        cache[key(kind, _dtype_name(dtype), problem.n_points)] = entry
        save_cache(cache, path)
    return best[0], best[1], table


def tune_batch(problems, dtype, search=None, reps=2, path=None, save=True, stream=None):
    """Time every candidate on a batch (a list of workloads.Problem with
    phi0, reinitialised together through fmm.Batch) and store the fastest
    under the kind "batch".  Returns (best_params, best_ms, table)."""
    import torch

    from . import fmm

    phis = [torch.as_tensor(p.phi0, dtype=dtype, device="cuda").contiguous() for p in problems]
    Ts = [torch.empty(p.shape, dtype=dtype, device="cuda") for p in problems]
    pts = sum(p.n_points for p in problems)
    table = []
    for params in candidates(search):
        try:
            with fmm.Batch([p.shape for p in problems], [p.h for p in problems], dtype=dtype,
                           stream=stream, tuned=False, **params) as b:
                def run():
                    b.reinit(phis, Ts, None, want_tags=False)
                run()
                ms = _time_call(torch, run, reps)
        except fmm.FmmError:
            ms = None
        table.append((params, ms))
    best = select_best(table)
    if best is None:
        return None, None, table
    if save:
        cache = load_cache(path)
        entry = dict(best[0])
        entry["ms"] = best[1]
        entry["points"] = pts
        cache[key("batch", _dtype_name(dtype), pts)] = entry
        save_cache(cache, path)
    return best[0], best[1], table


def summarize(table):
    ok = [ms for _, ms in table if ms is not None]
    return {"candidates": len(table), "median_ms": statistics.median(ok) if ok else None,
            "best_ms": min(ok) if ok else None}
