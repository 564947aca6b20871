"""Thin ctypes binding of libfmm_gb300.so (C ABI in include/fmm.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
PyTorch supplies device memory and the current stream.  Importing this module
loads the library and fails loudly if it is missing or was not built.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import torch

from . import autotune as _autotune
from . import build as _build

FMM_OK, FMM_ERR_INVALID, FMM_ERR_OOM, FMM_ERR_CUDA, FMM_ERR_TIMEOUT, FMM_ERR_STATE = range(6)
FMM_F32, FMM_F64 = 0, 1
TAG_FAR, TAG_BAND, TAG_KNOWN, TAG_FIX = 0, 1, 2, 3

EXPORTED = ("fmm_create", "fmm_set_speed", "fmm_solve", "fmm_reinit_signed_distance",
            "fmm_adjoint", "fmm_get_stats", "fmm_last_error", "fmm_destroy",
            "fmm_reinit_signed_distance_noalloc", "fmm_create_batch", "fmm_reinit_batch",
            "fmm_get_trace", "fmm_resume", "fmm_checkpoint_size", "fmm_checkpoint_save",
            "fmm_checkpoint_load", "fmm_selftest_fp64", "fmm_selftest_root", "fmm_probe_fma_rate",
            "fmm_solve_batch",
            "fmm_dd_start", "fmm_dd_minima", "fmm_dd_march", "fmm_dd_get_layers",
            "fmm_dd_integrate", "fmm_dd_finish", "fmm_solve_fixed")


class FmmConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("h", ctypes.c_double), ("dtype", ctypes.c_int32),
                ("record_tape", ctypes.c_int32), ("width", ctypes.c_double),
                ("stride", ctypes.c_double), ("bucket", ctypes.c_double),
                ("ctas", ctypes.c_int32), ("timeout_s", ctypes.c_int32),
                ("max_restarts", ctypes.c_int64), ("stream", ctypes.c_void_p),
                ("time_kernels", ctypes.c_int32), ("exchange_passes", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("max_lead", ctypes.c_int32),
                ("wait_limit_ms", ctypes.c_int32), ("hold_queue", ctypes.c_int32),
                ("hy", ctypes.c_double), ("hz", ctypes.c_double), ("ahead", ctypes.c_double),
                ("deterministic", ctypes.c_int32), ("accuracy", ctypes.c_int32)]


class FmmStats(ctypes.Structure):
    _fields_ = [("restarts", ctypes.c_int64), ("brick_marches", ctypes.c_int64),
                ("march_rounds", ctypes.c_int64), ("exchanges", ctypes.c_int64),
                ("accepted", ctypes.c_int64), ("n_bricks", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("march_launches", ctypes.c_int64),
                ("march_ms", ctypes.c_double), ("adjoint_iterations", ctypes.c_int64),
                ("error_flags", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("cell_solves", ctypes.c_int64)]

    def as_dict(self):
        return {k: (float(getattr(self, k)) if k == "march_ms" else int(getattr(self, k)))
                for k, _ in self._fields_ if not k.startswith("reserved")}


class FmmTraceEntry(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("phase", ctypes.c_int32),
                ("bricks", ctypes.c_int32), ("ms", ctypes.c_float)]


class FmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fmm error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(path: str | None = None):
    """Load (building first if needed) and bind the shared library."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.build()
    if not os.path.exists(p):
        raise FmmError(FMM_ERR_STATE, f"CUDA library not found at {p}")
    lib = ctypes.CDLL(p)
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    lib.fmm_create.argtypes = [ctypes.POINTER(FmmConfig), vp, dbl, vp, i64, ctypes.POINTER(vp)]
    lib.fmm_set_speed.argtypes = [vp, vp, dbl]
    lib.fmm_solve.argtypes = [vp, vp, vp]
    lib.fmm_solve_fixed.argtypes = [vp, vp, vp, vp]
    lib.fmm_reinit_signed_distance.argtypes = [vp, vp, vp, vp]
    lib.fmm_adjoint.argtypes = [vp, vp, vp]
    lib.fmm_get_stats.argtypes = [vp, ctypes.POINTER(FmmStats)]
    lib.fmm_last_error.argtypes = [vp]
    lib.fmm_last_error.restype = ctypes.c_char_p
    lib.fmm_destroy.argtypes = [vp]
    lib.fmm_destroy.restype = None
    lib.fmm_reinit_signed_distance_noalloc.argtypes = [ctypes.POINTER(FmmConfig), vp, vp, vp]
    lib.fmm_create_batch.argtypes = [ctypes.c_int, vp, vp, ctypes.POINTER(FmmConfig),
                                     ctypes.POINTER(vp)]
    lib.fmm_reinit_batch.argtypes = [vp, vp, vp, vp]
    lib.fmm_solve_batch.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.fmm_dd_start.argtypes = [vp, vp, i64, i64]
    lib.fmm_dd_minima.argtypes = [vp, ctypes.POINTER(dbl)]
    lib.fmm_dd_march.argtypes = [vp, ctypes.POINTER(dbl)]
    lib.fmm_dd_get_layers.argtypes = [vp, i64, i64, vp]
    lib.fmm_dd_integrate.argtypes = [vp, i64, i64, vp, ctypes.POINTER(i64)]
    lib.fmm_dd_finish.argtypes = [vp, vp, vp]
    lib.fmm_get_trace.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
    lib.fmm_resume.argtypes = [vp, i64, vp, vp]
    lib.fmm_checkpoint_size.argtypes = [vp, ctypes.POINTER(i64)]
    lib.fmm_checkpoint_save.argtypes = [vp, vp, i64]
    lib.fmm_checkpoint_load.argtypes = [vp, vp, i64]
    lib.fmm_selftest_fp64.argtypes = [vp, vp, vp, vp, i64, vp]
    lib.fmm_selftest_root.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, vp]
    lib.fmm_probe_fma_rate.argtypes = [ctypes.c_int32, i64, ctypes.POINTER(dbl)]
    for n in ("fmm_create", "fmm_set_speed", "fmm_solve", "fmm_reinit_signed_distance",
              "fmm_adjoint", "fmm_get_stats", "fmm_reinit_signed_distance_noalloc",
              "fmm_create_batch", "fmm_reinit_batch", "fmm_get_trace", "fmm_resume",
              "fmm_checkpoint_size", "fmm_checkpoint_save", "fmm_checkpoint_load",
              "fmm_selftest_fp64", "fmm_selftest_root", "fmm_probe_fma_rate", "fmm_solve_batch",
              "fmm_dd_start",
              "fmm_dd_minima", "fmm_dd_march", "fmm_dd_get_layers", "fmm_dd_integrate",
              "fmm_dd_finish", "fmm_solve_fixed"):
        getattr(lib, n).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _dtype_code(dtype):
    if dtype in (torch.float32, "f32", "float32", np.float32):
        return FMM_F32, torch.float32
    if dtype in (torch.float64, "f64", "float64", np.float64):
        return FMM_F64, torch.float64
    raise ValueError(f"unsupported dtype {dtype}")


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(int(s.cuda_stream))


def _dev_ptr(t: torch.Tensor, dtype=None, shape=None, name="array", host_ok=False):
    """Pointer of a contiguous tensor: on the GPU, or also in host memory
    (pinned or not) for the entry points that copy host arrays themselves."""
    if not t.is_cuda and not (host_ok and t.device.type == "cpu"):
        raise ValueError(f"{name} must be a CUDA tensor" + (" or a CPU tensor" if host_ok else ""))
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _spacing(h):
    """(dx, dy, dz) from one cell size or a 3-sequence."""
    if isinstance(h, (int, float)):
        return float(h), float(h), float(h)
    hx, hy, hz = (float(v) for v in h)
    return hx, hy, hz


class Solver:
    """One handle of the CUDA library: a grid (nz, ny, nx), cell size h (one
    value, or (dx, dy, dz) for cells of unequal sides), dtype, a speed field
    (tensor on the device or a constant) and optional point sources
    (i, j, k).  accuracy=2 selects the second-order march (on the
    cell-parallel schedule 4)."""

    def __init__(self, shape, h, dtype=torch.float32, speed=None, sources=None,
                 width=math.inf, stride=0.0, bucket=0.0, record_tape=False, ctas=0,
                 max_restarts=0, timeout_s=0, time_kernels=False, exchange_passes=0,
                 schedule=0, max_lead=0, wait_limit_ms=0, hold_queue=0, ahead=0.0, stream=None,
                 tuned=True, deterministic=False, accuracy=1):
        self.lib = load()
        nz, ny, nx = (int(v) for v in shape)
        self.shape = (nz, ny, nx)
        self.code, self.dtype = _dtype_code(dtype)
        self.stream = stream
        if deterministic or accuracy == 2 or schedule == 4:
            # the phased schedule with pass-synchronous halos, or the
            # cell-parallel march: the tuned schedules do not apply
            tuned = False
        if tuned:
            # parameters left at 0 take the autotuner's cached values (if any)
            kind = "reinit" if sources is None else (
                "sources" if speed is None or isinstance(speed, (int, float)) else "sources_speed")
            t = _autotune.merge({"stride": stride, "bucket": bucket, "ctas": ctas,
                                 "exchange_passes": exchange_passes, "schedule": schedule,
                                 "max_lead": max_lead, "ahead": ahead},
                                kind, self.dtype, nx * ny * nz)
            stride, bucket, ctas = t["stride"], t["bucket"], t["ctas"]
            exchange_passes, schedule = t["exchange_passes"], t["schedule"]
            max_lead, ahead = t["max_lead"], t["ahead"]
        cfg = FmmConfig()
        cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
        hx, hy, hz = _spacing(h)
        cfg.h, cfg.hy, cfg.hz = hx, hy, hz
        cfg.dtype = self.code
        cfg.record_tape = 1 if record_tape else 0
        cfg.width = 0.0 if math.isinf(width) else float(width)
        cfg.stride = float(stride)
        cfg.bucket = float(bucket)
        cfg.ctas = int(ctas)
        cfg.max_restarts = int(max_restarts)
        cfg.timeout_s = int(timeout_s)
        cfg.time_kernels = 1 if time_kernels else 0
        cfg.exchange_passes = int(exchange_passes)
        cfg.schedule = int(schedule)
        cfg.max_lead = int(min(max_lead, 1 << 30))
        cfg.wait_limit_ms = int(wait_limit_ms)
        cfg.hold_queue = int(hold_queue)
        cfg.ahead = float(ahead)
        cfg.deterministic = 1 if deterministic else 0
        cfg.accuracy = int(accuracy)
        cfg.stream = _stream_handle(stream)
        self.cfg = cfg
        sp_ptr, sp_const = self._speed_args(speed)
        src = None
        n_src = 0
        if sources is not None:
            src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64).reshape(-1, 3))
            n_src = len(src)
        handle = ctypes.c_void_p()
        rc = self.lib.fmm_create(ctypes.byref(cfg), sp_ptr, sp_const,
                                 None if src is None else src.ctypes.data, n_src,
                                 ctypes.byref(handle))
        if rc != FMM_OK:
            raise FmmError(rc, self.lib.fmm_last_error(None).decode())
        self.handle = handle
        self.h = hx if (hy, hz) == (hx, hx) else (hx, hy, hz)

    def _speed_args(self, speed):
        if speed is None:
            return None, 1.0
        if isinstance(speed, (int, float)):
            return None, float(speed)
        self._speed_ref = speed
        return _dev_ptr(speed, self.dtype, self.shape, "speed", host_ok=True), 0.0

    def _check(self, rc):
        if rc != FMM_OK:
            raise FmmError(rc, self.lib.fmm_last_error(self.handle).decode())

    def set_speed(self, speed):
        p, c = self._speed_args(speed)
        self._check(self.lib.fmm_set_speed(self.handle, p, c))

    def _outputs(self, T_out, tags_out, want_tags, device="cuda"):
        if T_out is None:
            T_out = torch.empty(self.shape, dtype=self.dtype, device=device)
        if tags_out is None and want_tags:
            tags_out = torch.empty(self.shape, dtype=torch.uint8, device=T_out.device)
        tp = _dev_ptr(T_out, self.dtype, self.shape, "T_out", host_ok=True)
        gp = None if tags_out is None else _dev_ptr(tags_out, torch.uint8, self.shape, "tags_out",
                                                   host_ok=True)
        return T_out, tags_out, tp, gp

    def solve(self, T_out=None, tags_out=None, want_tags=True):
        T_out, tags_out, tp, gp = self._outputs(T_out, tags_out, want_tags)
        self._check(self.lib.fmm_solve(self.handle, tp, gp))
        return T_out, tags_out

    def solve_fixed(self, T0, T_out=None, tags_out=None, want_tags=True):
        """Solve from given interface values: finite entries of T0 are FIX
        cells (side of their sign), +-inf FAR cells of that side."""
        pp = _dev_ptr(T0, self.dtype, self.shape, "T0", host_ok=True)
        T_out, tags_out, tp, gp = self._outputs(T_out, tags_out, want_tags, T0.device)
        self._check(self.lib.fmm_solve_fixed(self.handle, pp, tp, gp))
        return T_out, tags_out

    def reinit(self, phi0, T_out=None, tags_out=None, want_tags=True):
        pp = _dev_ptr(phi0, self.dtype, self.shape, "phi0", host_ok=True)
        T_out, tags_out, tp, gp = self._outputs(T_out, tags_out, want_tags, phi0.device)
        self._check(self.lib.fmm_reinit_signed_distance(self.handle, pp, tp, gp))
        return T_out, tags_out

    def resume(self, T_out=None, tags_out=None, want_tags=True, more_restarts=0):
        """Continue a solve stopped by max_restarts or timeout_s (or loaded
        with restore); more_restarts=0 means no further limit."""
        T_out, tags_out, tp, gp = self._outputs(T_out, tags_out, want_tags)
        self._check(self.lib.fmm_resume(self.handle, int(more_restarts), tp, gp))
        return T_out, tags_out

    def checkpoint(self):
        """Host image (numpy uint8) of the last solve's state."""
        n = ctypes.c_int64(0)
        self._check(self.lib.fmm_checkpoint_size(self.handle, ctypes.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        self._check(self.lib.fmm_checkpoint_save(self.handle, buf.ctypes.data, n.value))
        return buf

    def restore(self, image):
        """Load an image written by checkpoint() of a handle with the same grid,
        dtype, h, record_tape and speed."""
        buf = np.ascontiguousarray(np.asarray(image, dtype=np.uint8))
        self._check(self.lib.fmm_checkpoint_load(self.handle, buf.ctypes.data, buf.size))

    def adjoint(self, dL_dT, out=None):
        gp = _dev_ptr(dL_dT, self.dtype, self.shape, "dL_dT", host_ok=True)
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=dL_dT.device)
        op = _dev_ptr(out, self.dtype, self.shape, "dL_dslowness", host_ok=True)
        self._check(self.lib.fmm_adjoint(self.handle, gp, op))
        return out

    def stats(self):
        st = FmmStats()
        self._check(self.lib.fmm_get_stats(self.handle, ctypes.byref(st)))
        return st.as_dict()

    def trace(self):
        """Per march launch of the last solve: (restart, phase, bricks, ms);
        needs time_kernels=True."""
        n = ctypes.c_int64(0)
        self._check(self.lib.fmm_get_trace(self.handle, None, 0, ctypes.byref(n)))
        buf = (FmmTraceEntry * max(n.value, 1))()
        self._check(self.lib.fmm_get_trace(self.handle, buf, n.value, ctypes.byref(n)))
        return [(e.restart, e.phase, e.bricks, e.ms) for e in buf[: n.value]]

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fmm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def solve_sources(shape, h, sources, speed=None, dtype=torch.float32, **kw):
    """Point-source solve; returns (T, tags, stats)."""
    with Solver(shape, h, dtype=dtype, speed=speed, sources=sources, **kw) as s:
        T, G = s.solve()
        return T, G, s.stats()


def reinit(phi0, h, dtype=None, **kw):
    """Two-sided signed-distance reinitialisation of phi0 (a CUDA tensor);
    returns (T, tags, stats)."""
    dtype = phi0.dtype if dtype is None else dtype
    with Solver(tuple(phi0.shape), h, dtype=dtype, **kw) as s:
        T, G = s.reinit(phi0.to(dtype).contiguous())
        return T, G, s.stats()


class Batch:
    """Many independent grids (shapes (nz, ny, nx) with spacings hs)
    reinitialised together by fmm_create_batch / fmm_reinit_batch."""

    def __init__(self, shapes, hs, dtype=torch.float32, width=math.inf, stride=0.0, bucket=0.0,
                 exchange_passes=0, ctas=0, max_restarts=0, timeout_s=0, time_kernels=False,
                 schedule=0, max_lead=0, wait_limit_ms=0, hold_queue=0, ahead=0.0, stream=None,
                 tuned=True):
        self.lib = load()
        self.code, self.dtype = _dtype_code(dtype)
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        if tuned:
            # parameters left at 0 take the autotuner's cached values for a
            # batch of this many points (if any)
            pts = sum(a * b * c for a, b, c in self.shapes)
            t = _autotune.merge({"stride": stride, "bucket": bucket, "ctas": ctas,
                                 "exchange_passes": exchange_passes, "schedule": schedule,
                                 "max_lead": max_lead, "ahead": ahead},
                                "batch", self.dtype, pts)
            stride, bucket, ctas = t["stride"], t["bucket"], t["ctas"]
            exchange_passes, schedule = t["exchange_passes"], t["schedule"]
            max_lead, ahead = t["max_lead"], t["ahead"]
        n = len(self.shapes)
        dims = np.ascontiguousarray([[sh[2], sh[1], sh[0]] for sh in self.shapes], dtype=np.int64)
        hh = np.ascontiguousarray(hs, dtype=np.float64)
        if hh.shape != (n,):
            raise ValueError("one spacing per grid")
        cfg = FmmConfig()
        cfg.dtype = self.code
        cfg.width = 0.0 if math.isinf(width) else float(width)
        cfg.stride = float(stride)
        cfg.bucket = float(bucket)
        cfg.exchange_passes = int(exchange_passes)
        cfg.ctas = int(ctas)
        cfg.max_restarts = int(max_restarts)
        cfg.timeout_s = int(timeout_s)
        cfg.time_kernels = 1 if time_kernels else 0
        cfg.schedule = int(schedule)
        cfg.max_lead = int(min(max_lead, 1 << 30))
        cfg.wait_limit_ms = int(wait_limit_ms)
        cfg.hold_queue = int(hold_queue)
        cfg.ahead = float(ahead)
        cfg.stream = _stream_handle(stream)
        handle = ctypes.c_void_p()
        rc = self.lib.fmm_create_batch(n, dims.ctypes.data, hh.ctypes.data, ctypes.byref(cfg),
                                       ctypes.byref(handle))
        if rc != FMM_OK:
            raise FmmError(rc, self.lib.fmm_last_error(None).decode())
        self.handle = handle

    def reinit(self, phis, T_outs=None, tags_outs=None, want_tags=True):
        n = len(self.shapes)
        if len(phis) != n:
            raise ValueError("one level set per grid")
        if T_outs is None:
            T_outs = [torch.empty(sh, dtype=self.dtype, device="cuda") for sh in self.shapes]
        if tags_outs is None and want_tags:
            tags_outs = [torch.empty(sh, dtype=torch.uint8, device="cuda") for sh in self.shapes]
        P = (ctypes.c_void_p * n)(*[_dev_ptr(p, self.dtype, sh, "phi0").value
                                    for p, sh in zip(phis, self.shapes)])
        To = (ctypes.c_void_p * n)(*[_dev_ptr(t, self.dtype, sh, "T_out").value
                                     for t, sh in zip(T_outs, self.shapes)])
        Go = None
        if tags_outs is not None:
            Go = (ctypes.c_void_p * n)(*[_dev_ptr(t, torch.uint8, sh, "tags_out").value
                                         for t, sh in zip(tags_outs, self.shapes)])
        rc = self.lib.fmm_reinit_batch(self.handle, P, To, Go)
        if rc != FMM_OK:
            raise FmmError(rc, self.lib.fmm_last_error(self.handle).decode())
        return T_outs, tags_outs

    def solve(self, phis=None, sources=None, speeds=None, T_outs=None, tags_outs=None,
              want_tags=True):
        """Solve every grid (fmm_solve_batch): grid g is a reinitialisation of
        phis[g] (a CUDA tensor) or, where phis is None or phis[g] is None, a
        point-source problem with the cells sources[g] ((k, 3) of (i, j, k));
        speeds[g] is a CUDA tensor of F, a number, or None (F = 1)."""
        n = len(self.shapes)
        phis = [None] * n if phis is None else list(phis)
        sources = [None] * n if sources is None else list(sources)
        speeds = [None] * n if speeds is None else list(speeds)
        if not (len(phis) == len(sources) == len(speeds) == n):
            raise ValueError("one entry per grid")
        if T_outs is None:
            T_outs = [torch.empty(sh, dtype=self.dtype, device="cuda") for sh in self.shapes]
        if tags_outs is None and want_tags:
            tags_outs = [torch.empty(sh, dtype=torch.uint8, device="cuda") for sh in self.shapes]
        P = (ctypes.c_void_p * n)(*[None if ph is None else _dev_ptr(ph, self.dtype, sh, "phi0").value
                                    for ph, sh in zip(phis, self.shapes)])
        keep = []
        S = (ctypes.c_void_p * n)()
        N = (ctypes.c_int64 * n)()
        for g, (ph, src) in enumerate(zip(phis, sources)):
            if ph is None:
                if src is None:
                    raise ValueError(f"grid {g} needs a level set or sources")
                a = np.ascontiguousarray(np.asarray(src, dtype=np.int64).reshape(-1, 3))
                keep.append(a)
                S[g] = a.ctypes.data
                N[g] = len(a)
        V = (ctypes.c_void_p * n)()
        C = (ctypes.c_double * n)()
        for g, (sp, sh) in enumerate(zip(speeds, self.shapes)):
            if sp is None or isinstance(sp, (int, float)):
                C[g] = 1.0 if sp is None else float(sp)
            else:
                keep.append(sp)
                V[g] = _dev_ptr(sp, self.dtype, sh, "speed").value
                C[g] = 0.0
        To = (ctypes.c_void_p * n)(*[_dev_ptr(t, self.dtype, sh, "T_out").value
                                     for t, sh in zip(T_outs, self.shapes)])
        Go = None
        if tags_outs is not None:
            Go = (ctypes.c_void_p * n)(*[_dev_ptr(t, torch.uint8, sh, "tags_out").value
                                         for t, sh in zip(tags_outs, self.shapes)])
        rc = self.lib.fmm_solve_batch(self.handle, P, S, N, V, C, To, Go)
        if rc != FMM_OK:
            raise FmmError(rc, self.lib.fmm_last_error(self.handle).decode())
        return T_outs, tags_outs

    def stats(self):
        st = FmmStats()
        rc = self.lib.fmm_get_stats(self.handle, ctypes.byref(st))
        if rc != FMM_OK:
            raise FmmError(rc, "fmm_get_stats failed")
        return st.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fmm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def reinit_noalloc(phi0, h, T_out, tags_out=None, width=math.inf, stride=0.0, bucket=0.0,
                   stream=None):
    """Reinitialisation (F = 1) through fmm_reinit_signed_distance_noalloc,
    for callers that cannot allocate device memory: the library allocates
    nothing, and the caller supplies phi0, T_out and (optionally) tags_out as
    CUDA tensors.  Grids of at most 512 8x8x8 bricks (e.g. 64^3)."""
    lib = load()
    code, dt = _dtype_code(phi0.dtype)
    nz, ny, nx = phi0.shape
    cfg = FmmConfig()
    cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
    cfg.h, cfg.hy, cfg.hz = _spacing(h)
    cfg.dtype = code
    cfg.width = 0.0 if math.isinf(width) else float(width)
    cfg.stride = float(stride)
    cfg.bucket = float(bucket)
    cfg.stream = _stream_handle(stream)
    pp = _dev_ptr(phi0, dt, (nz, ny, nx), "phi0")
    tp = _dev_ptr(T_out, dt, (nz, ny, nx), "T_out")
    gp = None if tags_out is None else _dev_ptr(tags_out, torch.uint8, (nz, ny, nx), "tags_out")
    rc = lib.fmm_reinit_signed_distance_noalloc(ctypes.byref(cfg), pp, tp, gp)
    if rc != FMM_OK:
        raise FmmError(rc, lib.fmm_last_error(None).decode())
    return T_out, tags_out


def probe_fma_rate(dtype, iters=1 << 16):
    """Measured fused multiply-add throughput of the current device in
    float or double (flop/s, 2 per FMA): the arithmetic ceiling of the march
    kernels next to HBM bandwidth."""
    lib = load()
    code, _ = _dtype_code(dtype)
    out = ctypes.c_double(0.0)
    rc = lib.fmm_probe_fma_rate(code, int(iters), ctypes.byref(out))
    if rc != FMM_OK:
        raise FmmError(rc, "fmm_probe_fma_rate failed")
    return out.value


class EikonalFn(torch.autograd.Function):
    """T = EikonalFn.apply(slowness, solver): point-source travel times for a
    slowness field (1/F); backward returns dL/d(slowness) from the CUDA
    adjoint.  ``solver`` must be a Solver created with record_tape=True."""

    @staticmethod
    def forward(ctx, slowness, solver):
        speed = (1.0 / slowness).contiguous()
        solver.set_speed(speed)
        T, _ = solver.solve(want_tags=False)
        ctx.solver = solver
        return T

    @staticmethod
    def backward(ctx, gT):
        g = ctx.solver.adjoint(gT.contiguous())
        return g, None
