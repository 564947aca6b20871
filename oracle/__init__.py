"""ORACLE -- plain sequential fp64 narrow band fast marching (test infrastructure).

This package is the CPU oracle the CUDA library is checked against.  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library itself never does, and the two share
no code.  The arithmetic lives in ``fmm_oracle.c`` (plain C, fp64); this module
only builds it with gcc and marshals numpy arrays through ctypes.

Every function follows the paper (Yang & Stern, "A highly scalable massively
parallel fast marching method for the Eikonal equation"):

* ``init_sources`` / ``init_reinit``  -- Algorithm 8 (interface initialisation)
* ``march``                           -- Algorithm 9 + Algorithm 12 with
  bound = width (the sequential reference of Sec. 5.2), using Algorithm 10 and
  Algorithm 11
* ``local_solve``                     -- Algorithm 11 on one cell
* ``march(..., accuracy=2)``           -- the same march with second-order
  one-sided differences (the higher-order variant of Sec. 6)
* ``fast_sweep``                      -- an independent Gauss-Seidel solve of
  Eq. (2) (fast sweeping, cited in Sec. 1), used only to pin ``march``
* ``adjoint`` / ``tangent``           -- derivatives of the discrete Eq. (2)
  about the final upwind sets (not in the paper; derived from Eq. (2)-(3))

Arrays are numpy arrays of shape (nz, ny, nx) in C order (x fastest).  The
spacing ``h`` is one cell size for every axis or a 3-sequence (dx, dy, dz):
the cells of Sec. 2.1 are uniform in each direction, and Algorithm 11 takes
one h_i per axis.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_HDR = os.path.join(_HERE, "fmm_oracle.h")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

FAR, BAND_NEW, BAND_OLD, KNOWN_FIX, KNOWN_NEW, KNOWN_OLD = range(6)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fmm_oracle.c into oracle/_build/liboracle.so with gcc.

    -ffp-contract=off keeps every multiply and add separately rounded so the
    oracle gives the same bits on x86-64 and aarch64.
    """
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or force or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB_PATH) for p in (_SRC, _HDR))
    if stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = _bind(ctypes.CDLL(build()))
        return _lib


class use_library:
    """Context manager that routes this module's calls through another build
    of fmm_oracle.c (the mutation tests compile copies with planted mistakes
    and check that the pins reject them)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        _lib = _bind(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def compile_source(src_text, out_path):
    """Compile C source text (a copy of fmm_oracle.c) to a shared library
    with the oracle's flags."""
    d = os.path.dirname(out_path)
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                    "-fPIC", "-shared", "-I", _HERE, "-o", out_path, c_path, "-lm"],
                   check=True, cwd=d)
    return out_path


def source_text():
    with open(_SRC) as f:
        return f.read()


def _bind(lib):
    i64, dbl = ctypes.c_int64, ctypes.c_double
    vp = ctypes.c_void_p
    lib.oracle_init_sources.argtypes = [i64, i64, i64, vp, i64, vp, vp]
    lib.oracle_init_reinit.argtypes = [i64, i64, i64, vp, vp, vp, vp]
    lib.oracle_march.argtypes = [i64, i64, i64, vp, vp, dbl, dbl, vp, vp,
                                 vp, vp, vp]
    lib.oracle_local_solve.argtypes = [vp, vp, dbl, vp, dbl]
    lib.oracle_local_solve.restype = dbl
    lib.oracle_march_ho.argtypes = [i64, i64, i64, vp, vp, dbl, dbl, vp, vp,
                                    vp, vp, ctypes.c_int]
    lib.oracle_local_solve_ho.argtypes = [vp, vp, vp, vp, dbl, vp, dbl]
    lib.oracle_local_solve_ho.restype = dbl
    lib.oracle_fast_sweep.argtypes = [i64, i64, i64, vp, vp, dbl, vp, vp,
                                      i64, vp]
    lib.oracle_adjoint.argtypes = [i64, i64, i64, vp, vp, dbl, vp, vp, vp,
                                   vp, i64, vp, vp, vp]
    lib.oracle_tangent.argtypes = [i64, i64, i64, vp, vp, dbl, vp, vp, vp,
                                   vp, i64, vp, vp]
    for name in ("oracle_init_sources", "oracle_init_reinit", "oracle_march",
                 "oracle_march_ho", "oracle_fast_sweep", "oracle_adjoint",
                 "oracle_tangent"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"{what} failed with code {rc}")


def _spacing(h):
    """(dx, dy, dz) as a C array: h is one cell size for all axes or a
    3-sequence (dx, dy, dz)."""
    h3 = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (3,)))
    return h3


def _speed_args(speed, shape):
    if speed is None or np.isscalar(speed):
        return None, float(1.0 if speed is None else speed)
    sp = np.ascontiguousarray(speed, dtype=np.float64)
    if sp.shape != tuple(shape):
        raise ValueError("speed must have the grid's shape")
    return sp, 0.0


def init_sources(shape, sources):
    """Algorithm 8 for point sources.  shape = (nz, ny, nx); sources is a
    sequence of (i, j, k) cell indices.  Returns (T, G)."""
    nz, ny, nx = shape
    T = np.empty(shape, np.float64)
    G = np.empty(shape, np.uint8)
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64).reshape(-1, 3))
    _check(_load().oracle_init_sources(nx, ny, nz, _ptr(src), len(src),
                                       _ptr(T), _ptr(G)), "init_sources")
    return T, G


def init_reinit(phi0, h):
    """Algorithm 8 for a level set phi0 (front cells by linear interpolation
    of the crossing on each axis).  Returns (T, G)."""
    phi = np.ascontiguousarray(phi0, dtype=np.float64)
    nz, ny, nx = phi.shape
    T = np.empty(phi.shape, np.float64)
    G = np.empty(phi.shape, np.uint8)
    h3 = _spacing(h)
    _check(_load().oracle_init_reinit(nx, ny, nz, _ptr(h3), _ptr(phi), _ptr(T),
                                      _ptr(G)), "init_reinit")
    return T, G


def march(T, G, h, speed=None, width=np.inf, record=False, accuracy=1):
    """Algorithm 9 + Algorithm 12 (bound = width) in place on copies of T, G.

    Returns a dict with T, G and, when record=True, ``order`` (acceptance
    sequence) and ``tape`` (upwind set of each cell's final root).
    ``accuracy=2`` uses second-order one-sided differences where the cell
    beyond the upwind neighbour is known and monotone (no tape: the adjoint
    linearises the first-order scheme)."""
    if accuracy not in (1, 2):
        raise ValueError("accuracy must be 1 or 2")
    if accuracy == 2 and record:
        raise ValueError("the tape records first-order upwind sets only")
    T = np.array(T, dtype=np.float64, order="C", copy=True)
    G = np.array(G, dtype=np.uint8, order="C", copy=True)
    nz, ny, nx = T.shape
    sp, sc = _speed_args(speed, T.shape)
    n = T.size
    order = np.empty(n, np.int64) if record else None
    tape = np.empty(T.shape, np.uint8) if record else None
    n_order = ctypes.c_int64(0)
    h3 = _spacing(h)
    if accuracy == 1:
        rc = _load().oracle_march(nx, ny, nz, _ptr(h3), _ptr(sp), sc, float(width),
                                  _ptr(T), _ptr(G), _ptr(order),
                                  ctypes.addressof(n_order), _ptr(tape))
    else:
        rc = _load().oracle_march_ho(nx, ny, nz, _ptr(h3), _ptr(sp), sc,
                                     float(width), _ptr(T), _ptr(G), _ptr(order),
                                     ctypes.addressof(n_order), 2)
    _check(rc, "march")
    out = {"T": T, "G": G, "n_accepted": int(n_order.value)}
    if record:
        out["order"] = order[: n_order.value].copy()
        out["tape"] = tape
    return out


def solve_sources(shape, sources, h, speed=None, width=np.inf, record=False):
    T, G = init_sources(shape, sources)
    return march(T, G, h, speed=speed, width=width, record=record)


def solve_reinit(phi0, h, speed=None, width=np.inf, record=False):
    T, G = init_reinit(phi0, h)
    return march(T, G, h, speed=speed, width=width, record=record)


def local_solve(nb, nb_known, Tc, h, F, nb2=None, nb2_known=None):
    """Algorithm 11 on one cell from its six neighbours (-x,+x,-y,+y,-z,+z).

    With ``nb2`` (the cells two steps away in the same six directions) and
    ``nb2_known``, the second-order variant of ``march(..., accuracy=2)``."""
    nb = np.ascontiguousarray(nb, dtype=np.float64)
    kn = np.ascontiguousarray(nb_known, dtype=np.uint8)
    assert nb.shape == (6,) and kn.shape == (6,)
    h3 = _spacing(h)
    if nb2 is None:
        return float(_load().oracle_local_solve(_ptr(nb), _ptr(kn), float(Tc),
                                                _ptr(h3), float(F)))
    nb2 = np.ascontiguousarray(nb2, dtype=np.float64)
    kn2 = np.ascontiguousarray(nb2_known, dtype=np.uint8)
    assert nb2.shape == (6,) and kn2.shape == (6,)
    return float(_load().oracle_local_solve_ho(_ptr(nb), _ptr(kn), _ptr(nb2),
                                               _ptr(kn2), float(Tc), _ptr(h3),
                                               float(F)))


def fast_sweep(A0, fixed, h, speed=None, max_rounds=10000):
    """Gauss-Seidel fast sweeping on |psi|.  A0 holds the fixed values where
    ``fixed`` is set (others are ignored).  Returns (A, rounds)."""
    A = np.array(A0, dtype=np.float64, order="C", copy=True)
    fx = np.ascontiguousarray(fixed, dtype=np.uint8)
    A[fx == 0] = np.inf
    nz, ny, nx = A.shape
    sp, sc = _speed_args(speed, A.shape)
    rounds = ctypes.c_int64(0)
    h3 = _spacing(h)
    _check(_load().oracle_fast_sweep(nx, ny, nz, _ptr(h3), _ptr(sp), sc, _ptr(A),
                                     _ptr(fx), int(max_rounds),
                                     ctypes.addressof(rounds)), "fast_sweep")
    return A, int(rounds.value)


def adjoint(res, h, dLdT, speed=None):
    """dL/d(slowness) for L with gradient dLdT w.r.t. T, from a recorded
    ``march`` result.  Returns (dLds, lambda)."""
    T, G, tape, order = res["T"], res["G"], res["tape"], res["order"]
    nz, ny, nx = T.shape
    sp, sc = _speed_args(speed, T.shape)
    g = np.ascontiguousarray(dLdT, dtype=np.float64)
    dLds = np.empty(T.shape, np.float64)
    lam = np.empty(T.shape, np.float64)
    h3 = _spacing(h)
    _check(_load().oracle_adjoint(nx, ny, nz, _ptr(h3), _ptr(sp), sc, _ptr(T),
                                  _ptr(G), _ptr(tape), _ptr(order), len(order),
                                  _ptr(g), _ptr(dLds), _ptr(lam)), "adjoint")
    return dLds, lam


def tangent(res, h, v, speed=None):
    """dT = J v for a slowness perturbation v, from a recorded ``march``."""
    T, G, tape, order = res["T"], res["G"], res["tape"], res["order"]
    nz, ny, nx = T.shape
    sp, sc = _speed_args(speed, T.shape)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    dT = np.empty(T.shape, np.float64)
    h3 = _spacing(h)
    _check(_load().oracle_tangent(nx, ny, nz, _ptr(h3), _ptr(sp), sc, _ptr(T),
                                  _ptr(G), _ptr(tape), _ptr(order), len(order),
                                  _ptr(vv), _ptr(dT)), "tangent")
    return dT
