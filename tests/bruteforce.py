"""Brute-force references for pinning the oracle on tiny inputs.

Shares no code with ``oracle/`` or the CUDA library.  Every routine here uses
a different method from the oracle's:

* supercover membership by the exact minimum Chebyshev distance between the
  voxel centre and the segment (rational arithmetic, evaluated at every
  breakpoint of the piecewise-linear distance), instead of slab intersection;
* admissible offsets by a numpy mesh, instead of nested loops;
* joint sets by explicit enumeration of every chain root -> ... -> end,
  instead of set propagation;
* the reach pose as the lexicographically smallest chain (by linear index of
  p_1, then p_2, ...) among all valid chains, instead of a greedy traceback.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from itertools import product
from typing import Dict, List, Sequence, Tuple

import numpy as np

V = Tuple[int, int, int]


def cheb_dist_segment(a: V, b: V, c: V) -> Fraction:
    """min over t in [0,1] of max_i |a_i + t (b_i - a_i) - c_i| (exact)."""
    d = [b[i] - a[i] for i in range(3)]
    u = [a[i] - c[i] for i in range(3)]
    cands = {Fraction(0), Fraction(1)}
    for i in range(3):
        if d[i] != 0:
            cands.add(Fraction(-u[i], d[i]))
        for j in range(i + 1, 3):
            for s in (1, -1):
                # u_i + t d_i = s (u_j + t d_j)
                den = d[i] - s * d[j]
                if den != 0:
                    cands.add(Fraction(s * u[j] - u[i], den))
    best = None
    for t in cands:
        if t < 0 or t > 1:
            continue
        m = max(abs(u[i] + t * d[i]) for i in range(3))
        if best is None or m < best:
            best = m
    return best


@lru_cache(maxsize=None)
def supercover_from_origin(d: V) -> Tuple[V, ...]:
    """Voxels whose closed unit cube meets the closed segment 0 -> d."""
    lo = [min(0, d[i]) for i in range(3)]
    hi = [max(0, d[i]) for i in range(3)]
    out = []
    for z in range(lo[2] - 1, hi[2] + 2):
        for y in range(lo[1] - 1, hi[1] + 2):
            for x in range(lo[0] - 1, hi[0] + 2):
                if cheb_dist_segment((0, 0, 0), d, (x, y, z)) <= Fraction(1, 2):
                    out.append((x, y, z))
    return tuple(out)


def supercover(a: V, b: V) -> List[V]:
    d = (b[0] - a[0], b[1] - a[1], b[2] - a[2])
    return [(a[0] + v[0], a[1] + v[1], a[2] + v[2]) for v in supercover_from_origin(d)]


def shell_offsets(lo2: int, hi2: int) -> np.ndarray:
    """All integer offsets with lo2 <= |d|^2 <= hi2 (unordered)."""
    R = int(np.floor(np.sqrt(hi2))) + 1
    r = np.arange(-R, R + 1)
    X, Y, Z = np.meshgrid(r, r, r, indexing="ij")
    n2 = X * X + Y * Y + Z * Z
    m = (n2 >= lo2) & (n2 <= hi2)
    return np.stack([X[m], Y[m], Z[m]], axis=1)


def occupancy(shape, boxes) -> np.ndarray:
    """Boolean [nz][ny][nx] with every inclusive box filled (clipped)."""
    nx, ny, nz = shape
    occ = np.zeros((nz, ny, nx), dtype=bool)
    for b in np.asarray(boxes).reshape(-1, 6):
        x0, y0, z0, x1, y1, z1 = (int(v) for v in b)
        occ[max(z0, 0):z1 + 1, max(y0, 0):y1 + 1, max(x0, 0):x1 + 1] = True
    return occ


class Chains:
    """Every valid chain on a tiny grid, by explicit enumeration."""

    def __init__(self, occ: np.ndarray, bounds: Sequence[Tuple[int, int]]):
        self.occ = np.asarray(occ, dtype=bool)
        self.nz, self.ny, self.nx = self.occ.shape
        self.bounds = list(bounds)
        self.S = len(bounds)
        self.offs = [[tuple(int(v) for v in o) for o in shell_offsets(lo, hi)]
                     for lo, hi in bounds]
        self._edge: Dict[Tuple[V, V], bool] = {}

    def inside(self, p: V) -> bool:
        return 0 <= p[0] < self.nx and 0 <= p[1] < self.ny and 0 <= p[2] < self.nz

    def free(self, p: V) -> bool:
        return not self.occ[p[2], p[1], p[0]]

    def edge(self, p: V, q: V) -> bool:
        key = (p, q)
        r = self._edge.get(key)
        if r is None:
            r = self.inside(p) and self.inside(q) and all(
                self.inside(v) and self.free(v) for v in supercover(p, q))
            self._edge[key] = r
        return r

    def index(self, p: V) -> int:
        return (p[2] * self.ny + p[1]) * self.nx + p[0]

    def enumerate(self, root: V, first: int = 1, last: int = None):
        """Yield every valid chain (p_{first-1}=root, ..., p_last)."""
        last = self.S if last is None else last

        def rec(chain, k):
            if k > last:
                yield tuple(chain)
                return
            p = chain[-1]
            for d in self.offs[k - 1]:
                q = (p[0] + d[0], p[1] + d[1], p[2] + d[2])
                if self.inside(q) and self.edge(p, q):
                    chain.append(q)
                    yield from rec(chain, k + 1)
                    chain.pop()

        if not (self.inside(root) and self.free(root)):
            return
        yield from rec([root], first)

    def joint_sets(self, root: V, targets, last_offsets=None) -> Tuple[List[set], List[set], List[tuple]]:
        """(F sets, V sets, all valid chains ending in ``targets``).

        F_k collects p_k of every valid partial chain of k segments (dead
        ends included); V_k collects p_k of every full chain ending in a free
        target voxel.  ``last_offsets`` (optional) limits the last segment of
        the full chains to those offsets (F is unaffected).
        """
        targets = set(tuple(int(v) for v in t) for t in targets)
        allowed_last = None if last_offsets is None else set(tuple(int(v) for v in d) for d in last_offsets)
        F = [set() for _ in range(self.S + 1)]
        Vs = [set() for _ in range(self.S + 1)]
        good = []
        if not (self.inside(root) and self.free(root)):
            return F, Vs, good
        F[0].add(root)

        def rec(chain, k):
            if k > self.S:
                last = tuple(chain[-1][i] - chain[-2][i] for i in range(3))
                if chain[-1] in targets and (allowed_last is None or last in allowed_last):
                    good.append(tuple(chain))
                    for j, p in enumerate(chain):
                        Vs[j].add(p)
                return
            p = chain[-1]
            for d in self.offs[k - 1]:
                q = (p[0] + d[0], p[1] + d[1], p[2] + d[2])
                if self.inside(q) and self.edge(p, q):
                    F[k].add(q)
                    chain.append(q)
                    rec(chain, k + 1)
                    chain.pop()

        rec([root], 1)
        return F, Vs, good

    def lexmin(self, chains) -> tuple:
        return min(chains, key=lambda ch: tuple(self.index(p) for p in ch[1:]))


def to_set(mask: np.ndarray) -> set:
    """Voxel set (x, y, z) of a [nz][ny][nx] mask."""
    zs, ys, xs = np.nonzero(mask)
    return set(zip(xs.tolist(), ys.tolist(), zs.tolist()))
