"""A rank's local march on the CPU for the multi-rank tests of the domain
decomposition driver (paper_1502_07303_gb300/decomp.py): the same interface
as decomp.GpuMarcher (start, minima, march, get_layers, integrate, finish),
written in plain Python with a binary heap per side, following the paper's
algorithms step by step on a small subdomain:

* start: Algorithm 8 (the oracle's init_reinit / init_sources) and
  Algorithm 9 (every FIX cell updates its neighbours);
* march: Algorithm 12 to the given bound (pop the smallest |psi| of a side
  while it is at most the bound, accept it, Algorithm 10 on its neighbours,
  with Algorithm 11 from the oracle's local_solve);
* integrate: Algorithm 15 (a smaller incoming |psi| replaces the local one;
  the cell goes back into the heap, accepted at the next march if it is
  within the bound).

Test infrastructure only (pure-Python loops: small grids).  Not collected as
tests."""
import heapq
import math

import numpy as np
import torch

import oracle

FAR, BAND, KNOWN, FIX = 0, 1, 2, 3
_OFFS = [(0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]   # -x +x -y +y -z +z


class RefMarcher:
    def __init__(self, sub, shape, h, speed=None, sources=None, phi0=None):
        self.sub, self.h = sub, h
        nz, ny, nx = shape
        self.lshape = (sub.nlz, ny, nx)
        if speed is None or np.isscalar(speed):
            self.F = np.full(self.lshape, 1.0 if speed is None else float(speed))
        else:
            self.F = np.array(sub.local(np.asarray(speed, np.float64)))
        self.phi0 = None
        if phi0 is not None:
            ext, self.lo, self.hi = sub.extended(np.asarray(phi0, np.float64))
            self.phi0 = np.array(ext)
        self.sources = None if sources is None else sub.local_sources(sources)

    # Algorithm 10 for the cell p (side s)
    def _update_neighbours(self, p, s):
        T, G = self.T, self.G
        nz, ny, nx = self.lshape
        k, j, i = p
        Ti = abs(T[p])
        for dz, dy, dx in _OFFS:
            q = (k + dz, j + dy, i + dx)
            if not (0 <= q[0] < nz and 0 <= q[1] < ny and 0 <= q[2] < nx):
                continue
            if G[q] == FIX or not abs(T[q]) > Ti:
                continue
            t = self._solve(q)
            if t < abs(T[q]):
                T[q] = -t if s < 0 else t
                G[q] = BAND
                heapq.heappush(self.heap[s], (t, q))

    # Algorithm 11 on cell q from its known neighbours
    def _solve(self, q):
        T, G = self.T, self.G
        nz, ny, nx = self.lshape
        nb = np.full(6, np.inf)
        kn = np.zeros(6, np.uint8)
        for a, (dz, dy, dx) in enumerate(_OFFS):
            r = (q[0] + dz, q[1] + dy, q[2] + dx)
            if 0 <= r[0] < nz and 0 <= r[1] < ny and 0 <= r[2] < nx:
                nb[a] = abs(T[r])
                kn[a] = G[r] in (KNOWN, FIX)
        return oracle.local_solve(nb, kn, abs(T[q]), self.h, float(self.F[q]))

    def start(self):
        if self.phi0 is not None:
            # Algorithm 8 on the subdomain plus the layers beyond its ghost
            # layers, which are then dropped
            T, G0 = oracle.init_reinit(self.phi0, self.h)
            n = T.shape[0]
            T, G0 = T[self.lo:n - self.hi].copy(), G0[self.lo:n - self.hi].copy()
        else:
            T, G0 = oracle.init_sources(self.lshape, self.sources)
        self.T = T
        self.G = np.where(G0 == oracle.KNOWN_FIX, FIX, FAR).astype(np.uint8)
        self.heap = {-1: [], 1: []}
        for p in zip(*np.nonzero(self.G == FIX)):
            self._update_neighbours(p, -1 if T[p] < 0 else 1)

    def _top(self, s):
        h = self.heap[s]
        while h and (self.G[h[0][1]] != BAND or abs(self.T[h[0][1]]) != h[0][0]):
            heapq.heappop(h)              # stale entries
        return h[0] if h else None

    def minima(self):
        out = []
        for s in (-1, 1):
            top = self._top(s)
            out.append(math.inf if top is None else top[0])
        return out

    def march(self, bound):
        for s, b in ((-1, bound[0]), (1, bound[1])):
            while True:
                top = self._top(s)
                if top is None or top[0] > b:
                    break
                heapq.heappop(self.heap[s])
                p = top[1]
                self.G[p] = KNOWN
                self._update_neighbours(p, s)

    def get_layers(self, z, n):
        T = self.T[z:z + n].copy()
        T[self.G[z:z + n] == FAR] = np.inf
        return torch.as_tensor(T)

    def integrate(self, z, layers):
        L = layers.numpy() if torch.is_tensor(layers) else np.asarray(layers)
        n = 0
        for idx in zip(*np.nonzero(np.isfinite(L))):
            p = (z + idx[0], idx[1], idx[2])
            v = float(L[idx])
            if self.G[p] == FIX or not abs(v) < abs(self.T[p]):
                continue
            self.T[p] = v
            self.G[p] = BAND
            heapq.heappush(self.heap[-1 if v < 0 else 1], (abs(v), p))
            n += 1
        return n

    def finish(self):
        T = self.T.copy()
        T[self.G == FAR] = np.inf
        return torch.as_tensor(T), torch.as_tensor(self.G.copy())
