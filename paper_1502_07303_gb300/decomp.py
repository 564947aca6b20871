"""Domain decomposition of one grid across ranks (Sec. 4.1, Algorithms 13-16).

The grid is cut into slabs of z layers, one per rank.  A rank's subdomain is
its slab plus one ghost layer towards each neighbouring rank, so neighbouring
subdomains overlap by two layers (the rank's last layer and the neighbour's
first, Xi_p and Xi_q of Sec. 4.1); wider overlaps (``ghost`` > 1, a variant
the paper's conclusions name) exchange 2 * ghost layers.  Each rank marches its subdomain with the
CUDA library (``GpuMarcher``: the fmm_dd_* entry points); this module runs
the loop of Algorithm 16 around it:

    start (Algorithms 8, 9)
    loop:
        minval = AllReduce_MIN(local BAND minima per side)
        count  = AllReduce_MAX(cells replaced by the last exchange)
        exit if both minima >= width and count = 0
        bound  = min(minval + stride, width)
        march to bound (Algorithm 12)
        exchange the overlap layers with the neighbours (Algorithms 13, 14)
        integrate the received layers (Algorithm 15)
        march to bound again

The reductions carry three scalars per restart; the exchange sends two
layers of nx * ny values to each neighbour, into the receiver's own memory.
Whether the collectives run over torch.distributed (``TorchComm``: NCCL
between GPUs, gloo on CPU) or the ranks are stepped one after another in one
process (``solve_serial``: every rank's kernels run to completion before the
next rank's start, so no kernel ever waits on another rank) only changes how
data moves; the steps are the same functions.  Values are exchanged whole and
the receiver keeps the improvements (Algorithm 15's test), so the count of
Algorithm 13 is counted where the data arrive.
"""
from __future__ import annotations

import math

import numpy as np


def slabs(nz, n_ranks):
    """Interior z ranges [z0, z1) of the ranks, as even as possible."""
    if n_ranks < 1 or n_ranks > nz:
        raise ValueError("need 1 <= ranks <= nz")
    edges = [round(r * nz / n_ranks) for r in range(n_ranks + 1)]
    return [(edges[r], edges[r + 1]) for r in range(n_ranks)]


class Subdomain:
    """Rank r's slab [z0, z1) of an nz-layer grid and its subdomain
    [lz0, lz1) with `ghost` ghost layers towards each neighbour (Sec. 4.1
    uses one; wider overlaps are the variant its conclusions suggest): the
    overlap with a neighbour is 2 * ghost layers, given in local z indices."""

    def __init__(self, nz, n_ranks, rank, ghost=1):
        self.nz, self.n_ranks, self.rank, self.ghost = nz, n_ranks, rank, ghost
        self.z0, self.z1 = slabs(nz, n_ranks)[rank]
        if ghost < 1 or any(b - a < ghost for a, b in slabs(nz, n_ranks)):
            raise ValueError("every slab needs at least `ghost` layers")
        self.lz0 = self.z0 - ghost if self.z0 > 0 else 0
        self.lz1 = self.z1 + ghost if self.z1 < nz else nz
        self.nlz = self.lz1 - self.lz0
        self.n_overlap = 2 * ghost

    def neighbours(self):
        """(peer rank, first local layer of the 2 * ghost shared with it)."""
        out = []
        if self.rank > 0:
            out.append((self.rank - 1, 0))                              # ghosts, then layers from z0
        if self.rank < self.n_ranks - 1:
            out.append((self.rank + 1, self.nlz - self.n_overlap))      # layers to z1, then ghosts
        return out

    def local(self, a):
        """The subdomain's part of a global (nz, ny, nx) array."""
        return a[self.lz0:self.lz1]

    def extended(self, a):
        """The subdomain's part of a global array with one more layer beyond
        each ghost layer (where the grid has one), and the numbers of those
        extra layers below and above: the level set an interface
        initialisation of the ghost layers needs to see."""
        e0, e1 = max(self.lz0 - 1, 0), min(self.lz1 + 1, self.nz)
        return a[e0:e1], self.lz0 - e0, e1 - self.lz1

    def interior(self, a_local):
        """The slab's own layers of a subdomain array."""
        return a_local[self.z0 - self.lz0:self.z1 - self.lz0]

    def local_sources(self, sources):
        """Point sources (i, j, k) inside the subdomain, in local indices."""
        src = np.asarray(sources, dtype=np.int64).reshape(-1, 3)
        inside = (src[:, 2] >= self.lz0) & (src[:, 2] < self.lz1)
        out = src[inside].copy()
        out[:, 2] -= self.lz0
        return out


class GpuMarcher:
    """A rank's subdomain on its GPU: a handle of the CUDA library driven
    through the fmm_dd_* entry points."""

    def __init__(self, sub, shape, h, dtype, speed=None, sources=None, phi0=None, stream=None,
                 **params):
        import torch

        from . import fmm
        self.fmm, self.torch, self.sub = fmm, torch, sub
        nz, ny, nx = shape
        self.lshape = (sub.nlz, ny, nx)
        sp = None
        if speed is not None and not isinstance(speed, (int, float)):
            # a copy: a slice of the caller's field need not start on a
            # 16-byte boundary
            sp = sub.local(speed).clone(memory_format=torch.contiguous_format)
        elif speed is not None:
            sp = float(speed)
        src = None if sources is None else sub.local_sources(sources)
        self.solver = fmm.Solver(self.lshape, h, dtype=dtype, speed=sp, sources=src,
                                 stream=stream, tuned=False, **params)
        self.phi0, self.extra = None, (0, 0)
        if phi0 is not None:
            ext, lo, hi = sub.extended(phi0)
            self.phi0 = ext.to(self.solver.dtype).clone(memory_format=torch.contiguous_format)
            self.extra = (lo, hi)
        self.lib, self.handle = self.solver.lib, self.solver.handle
        self.dtype = self.solver.dtype
        self.layer_elems = ny * nx

    def _check(self, rc):
        if rc != self.fmm.FMM_OK:
            raise self.fmm.FmmError(rc, self.lib.fmm_last_error(self.handle).decode())

    def start(self):
        import ctypes
        p = None if self.phi0 is None else ctypes.c_void_p(self.phi0.data_ptr())
        self._check(self.lib.fmm_dd_start(self.handle, p, self.extra[0], self.extra[1]))

    def minima(self):
        import ctypes
        out = (ctypes.c_double * 2)()
        self._check(self.lib.fmm_dd_minima(self.handle, out))
        return [out[0], out[1]]

    def march(self, bound):
        import ctypes
        b = (ctypes.c_double * 2)(float(bound[0]), float(bound[1]))
        self._check(self.lib.fmm_dd_march(self.handle, b))

    def get_layers(self, z, n):
        import ctypes
        out = self.torch.empty((n,) + self.lshape[1:], dtype=self.dtype, device="cuda")
        self._check(self.lib.fmm_dd_get_layers(self.handle, z, n, ctypes.c_void_p(out.data_ptr())))
        return out

    def integrate(self, z, layers):
        import ctypes
        layers = layers.to(device="cuda", dtype=self.dtype).contiguous()
        n = ctypes.c_int64(0)
        self._check(self.lib.fmm_dd_integrate(self.handle, z, layers.shape[0],
                                              ctypes.c_void_p(layers.data_ptr()), ctypes.byref(n)))
        return int(n.value)

    def finish(self):
        import ctypes
        T = self.torch.empty(self.lshape, dtype=self.dtype, device="cuda")
        G = self.torch.empty(self.lshape, dtype=self.torch.uint8, device="cuda")
        self._check(self.lib.fmm_dd_finish(self.handle, ctypes.c_void_p(T.data_ptr()),
                                           ctypes.c_void_p(G.data_ptr())))
        return T, G

    def close(self):
        self.solver.close()


# ---------------------------------------------------------------------------
# the steps of Algorithm 16 for one rank
# ---------------------------------------------------------------------------

def next_bound(minval, stride, width):
    """Algorithm 16's bound per side: min(minval + stride, width)."""
    return [min(m + stride, width) for m in minval]


def finished(minval, count, width):
    """Algorithm 16's exit test."""
    return minval[0] >= width and minval[1] >= width and count == 0


def outgoing(marcher, sub):
    """Algorithm 13's outgoing buffers: the overlap layers per neighbour."""
    return {peer: marcher.get_layers(z, sub.n_overlap) for peer, z in sub.neighbours()}


def integrate(marcher, sub, incoming):
    """Algorithm 15 for every neighbour's layers; returns the replaced cells."""
    return sum(marcher.integrate(z, incoming[peer]) for peer, z in sub.neighbours())


class TorchComm:
    """The reductions and the neighbour exchange over torch.distributed."""

    def __init__(self, dist, device):
        self.dist, self.device = dist, device

    def reduce(self, minval, count):
        import torch
        d = self.dist
        t = torch.tensor([minval[0], minval[1]], dtype=torch.float64, device=self.device)
        d.all_reduce(t, op=d.ReduceOp.MIN)
        c = torch.tensor([float(count)], dtype=torch.float64, device=self.device)
        d.all_reduce(c, op=d.ReduceOp.MAX)
        return [float(t[0]), float(t[1])], int(c[0])

    def exchange(self, sends):
        """Send each peer its buffer and receive one of the same shape back."""
        d = self.dist
        recvs = {peer: buf.new_empty(buf.shape).to(self.device) for peer, buf in sends.items()}
        ops = []
        for peer, buf in sends.items():
            ops.append(d.P2POp(d.isend, buf.to(self.device).contiguous(), peer))
            ops.append(d.P2POp(d.irecv, recvs[peer], peer))
        if ops:
            for r in d.batch_isend_irecv(ops):
                r.wait()
        return recvs


def solve_spmd(marcher, sub, comm, stride, width=math.inf, max_restarts=100000):
    """This rank's part of Algorithm 16; every rank calls it.  Returns the
    subdomain's (T, G) and the number of restarts."""
    marcher.start()
    count = 0
    for restart in range(max_restarts):
        minval, total = comm.reduce(marcher.minima(), count)
        if finished(minval, total, width):
            return marcher.finish(), restart
        bound = next_bound(minval, stride, width)
        marcher.march(bound)
        count = integrate(marcher, sub, comm.exchange(outgoing(marcher, sub)))
        marcher.march(bound)
    raise RuntimeError("the restart limit was reached")


def solve_serial(marchers, subs, stride, width=math.inf, max_restarts=100000):
    """Algorithm 16 for all ranks stepped in one process (each rank's work
    completes before the next rank's starts); returns every rank's (T, G)
    and the number of restarts."""
    for m in marchers:
        m.start()
    counts = [0] * len(marchers)
    for restart in range(max_restarts):
        mins = [m.minima() for m in marchers]
        minval = [min(v[0] for v in mins), min(v[1] for v in mins)]
        if finished(minval, max(counts), width):
            return [m.finish() for m in marchers], restart
        bound = next_bound(minval, stride, width)
        for m in marchers:
            m.march(bound)
        sends = [outgoing(m, s) for m, s in zip(marchers, subs)]
        counts = [integrate(m, s, {peer: sends[peer][s.rank] for peer, _ in s.neighbours()})
                  for m, s in zip(marchers, subs)]
        for m in marchers:
            m.march(bound)
    raise RuntimeError("the restart limit was reached")


def assemble(subs, results, shape):
    """The global arrays from every rank's subdomain result (each slab's own
    layers)."""
    import torch
    T0, G0 = results[0]
    T = torch.empty(shape, dtype=T0.dtype, device=T0.device)
    G = torch.empty(shape, dtype=G0.dtype, device=G0.device)
    for s, (Tl, Gl) in zip(subs, results):
        T[s.z0:s.z1] = s.interior(Tl)
        G[s.z0:s.z1] = s.interior(Gl)
    return T, G
