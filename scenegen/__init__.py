"""Seeded synthetic inputs for the gap map-seeking IK workloads.

This module is shared input plumbing: the CPU oracle tests, the CUDA parity
tests and the benchmark all draw their scenes from it.  It holds none of the
method's arithmetic (no shells, supercovers, reachable sets or poses): it only
draws boxes, roots, targets, moving-box trajectories and request arrival times
from a documented pseudo-random stream.

The paper publishes no scene data (its figures only show arms among blocks,
"Fig 1", "Fig 7", "Fig 8"), so every workload is synthetic.  The five
workload shapes follow the five configurations of the benchmark:

* ``C1``: 32^3 grid, arm {8,7,6,5}, root (16,16,0), 20 boxes with per-axis
  sides U{2..6}, one target per seed.
* ``C2``/``C3``: 128^3 grid, arm {20,18,16,14,12,10,8,6}, root at the floor
  centre (64,64,0), 200 boxes with sides U{4..24}, 64 targets.  ``C3`` adds a
  32-waypoint path per target.
* ``C4``: 1024 independent problems, grid edge U{64,96,128,192}, 5-9 segments
  with lengths U{4..24}, 50-400 boxes, 8-32 waypoints.
* ``C5``: 256^3 grid, the C2 arm, 300 static boxes plus 16 moving boxes
  (sides U{6..16}, 0.5-2 voxels per tick), Poisson request arrivals.

Random numbers
--------------
Every stream is a splitmix64 generator (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014; the constants are the
published ones).  A stream's state starts at ``(seed << 8) | tag`` where the
tag names the stream (scene 1, targets 2, arrivals 3, velocities 4, problems
5).  Integers in ``[0, n)`` use Lemire's multiply-shift method with rejection
("Fast random integer generation in an interval", ACM TOMACS 2019), which is
exactly uniform.  The draw order of every generator below is part of its
definition.

Occupancy convention at every interface: a box is the inclusive voxel range
``[lo, hi]`` per axis (clipped to the grid); voxels inside any box are
occupied.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

MASK64 = (1 << 64) - 1

TAG_SCENE = 1
TAG_TARGETS = 2
TAG_ARRIVALS = 3
TAG_VELOCITIES = 4
TAG_PROBLEMS = 5


class SplitMix64:
    """splitmix64 stream with Lemire range reduction."""

    __slots__ = ("state",)

    def __init__(self, seed: int, tag: int):
        self.state = ((int(seed) << 8) | int(tag)) & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Uniform integer in [0, n), n >= 1 (Lemire, with rejection)."""
        if n <= 0:
            raise ValueError("range must be positive")
        m = self.next_u64() * n
        low = m & MASK64
        if low < n:
            threshold = ((1 << 64) - n) % n
            while low < threshold:
                m = self.next_u64() * n
                low = m & MASK64
        return m >> 64

    def between(self, lo: int, hi: int) -> int:
        """Uniform integer in the inclusive range [lo, hi]."""
        return lo + self.below(hi - lo + 1)

    def uniform01(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


@dataclass
class Scene:
    """A static scene: grid extent, root voxel and obstacle boxes.

    ``boxes`` is int32 ``[n][6]`` = (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z),
    inclusive, already clipped to the grid.
    """

    nx: int
    ny: int
    nz: int
    root: Tuple[int, int, int]
    lengths: Tuple[int, ...]
    boxes: np.ndarray
    seed: int = 0
    name: str = ""

    @property
    def shape(self) -> Tuple[int, int, int]:
        return (self.nx, self.ny, self.nz)

    def point_occupied(self, p) -> bool:
        """True when voxel ``p`` lies inside one of the boxes."""
        x, y, z = p
        b = self.boxes
        if len(b) == 0:
            return False
        inside = ((b[:, 0] <= x) & (x <= b[:, 3]) & (b[:, 1] <= y) & (y <= b[:, 4])
                  & (b[:, 2] <= z) & (z <= b[:, 5]))
        return bool(inside.any())


def _draw_box(rng: SplitMix64, n: Tuple[int, int, int], side_lo: int, side_hi: int):
    """One box: per axis a side U{side_lo..side_hi}, then a corner U{0..N-1}.

    Draw order per box: side x, side y, side z, corner x, corner y, corner z.
    """
    sides = [rng.between(side_lo, side_hi) for _ in range(3)]
    corner = [rng.below(n[a]) for a in range(3)]
    lo = corner
    hi = [min(corner[a] + sides[a] - 1, n[a] - 1) for a in range(3)]
    return lo + hi


def _covers(box, p) -> bool:
    return all(box[a] <= p[a] <= box[a + 3] for a in range(3))


def make_scene(nx: int, ny: int, nz: int, root, lengths, n_boxes: int,
               side_lo: int, side_hi: int, seed: int, name: str = "") -> Scene:
    """Draw ``n_boxes`` boxes; a box that covers the root is drawn again."""
    rng = SplitMix64(seed, TAG_SCENE)
    n = (nx, ny, nz)
    boxes: List[List[int]] = []
    while len(boxes) < n_boxes:
        b = _draw_box(rng, n, side_lo, side_hi)
        if _covers(b, root):
            continue
        boxes.append(b)
    arr = np.asarray(boxes, dtype=np.int32).reshape(-1, 6)
    return Scene(nx, ny, nz, tuple(int(v) for v in root), tuple(int(v) for v in lengths),
                 arr, seed, name)


def draw_targets(scene: Scene, count: int, seed: int) -> np.ndarray:
    """``count`` target voxels, each uniform over the free voxels within reach.

    A voxel qualifies when it is not occupied, differs from the root, and its
    squared distance to the root is at most (sum of segment lengths)^2.  Each
    target is drawn by rejection: a uniform voxel of the grid (x, then y,
    then z) is kept when it qualifies.  Rejection sampling is exactly uniform
    over the qualifying set.  Returns int32 ``[count][3]``.
    """
    rng = SplitMix64(seed, TAG_TARGETS)
    reach = sum(scene.lengths)
    r = scene.root
    out = []
    while len(out) < count:
        p = (rng.below(scene.nx), rng.below(scene.ny), rng.below(scene.nz))
        d2 = sum((p[a] - r[a]) ** 2 for a in range(3))
        if d2 > reach * reach or p == tuple(r):
            continue
        if scene.point_occupied(p):
            continue
        out.append(p)
    return np.asarray(out, dtype=np.int32).reshape(-1, 3)


# --------------------------------------------------------------------------
# The five workload shapes
# --------------------------------------------------------------------------

C1_LENGTHS = (8, 7, 6, 5)
C2_LENGTHS = (20, 18, 16, 14, 12, 10, 8, 6)


def c1_scene(seed: int) -> Scene:
    """32^3, arm {8,7,6,5}, root (16,16,0), 20 boxes with sides U{2..6}."""
    return make_scene(32, 32, 32, (16, 16, 0), C1_LENGTHS, 20, 2, 6, seed, "C1")


def c2_scene(seed: int = 1) -> Scene:
    """128^3, arm {20,18,...,6}, root (64,64,0), 200 boxes with sides U{4..24}."""
    return make_scene(128, 128, 128, (64, 64, 0), C2_LENGTHS, 200, 4, 24, seed, "C2")


def scaled_scene(n: int, lengths, n_boxes: int, side_lo: int, side_hi: int,
                 seed: int, name: str = "") -> Scene:
    """A cube grid of edge ``n`` with the root at the floor centre (n/2, n/2, 0)."""
    return make_scene(n, n, n, (n // 2, n // 2, 0), lengths, n_boxes, side_lo, side_hi,
                      seed, name)


@dataclass
class Problem:
    """One independent problem of the uneven batch (C4)."""

    scene: Scene
    target: Tuple[int, int, int]
    n_way: int


def c4_problems(count: int = 1024, seed: int = 2) -> List[Problem]:
    """Uneven batch: grid edge U{64,96,128,192}, 5-9 segments, lengths U{4..24},
    50-400 boxes with sides U{4..24}, 8-32 waypoints, one target each.

    Per problem, the problem stream draws: grid choice, segment count, each
    length, box count, waypoint count, then a scene seed and a target seed
    (both 32-bit).
    """
    rng = SplitMix64(seed, TAG_PROBLEMS)
    edges = (64, 96, 128, 192)
    out = []
    for i in range(count):
        n = edges[rng.below(4)]
        s = rng.between(5, 9)
        lengths = tuple(rng.between(4, 24) for _ in range(s))
        nb = rng.between(50, 400)
        w = rng.between(8, 32)
        scene_seed = rng.next_u64() & 0xFFFFFFFF
        target_seed = rng.next_u64() & 0xFFFFFFFF
        sc = scaled_scene(n, lengths, nb, 4, 24, scene_seed, f"C4[{i}]")
        t = draw_targets(sc, 1, target_seed)[0]
        out.append(Problem(sc, tuple(int(v) for v in t), w))
    return out


@dataclass
class MovingBoxes:
    """Boxes moving at constant velocity, reflecting at the grid walls.

    Positions and velocities are Q8 fixed point (1 voxel = 256).  ``pos`` is
    int64 ``[m][3]`` (the low corner), ``vel`` int64 ``[m][3]``, ``side``
    int64 ``[m][3]``.  The voxelised box at a tick is
    ``[floor(pos/256), floor(pos/256) + side - 1]`` per axis.
    """

    n: Tuple[int, int, int]
    pos: np.ndarray
    vel: np.ndarray
    side: np.ndarray
    tick: int = 0

    def boxes(self) -> np.ndarray:
        lo = self.pos // 256
        hi = lo + self.side - 1
        return np.concatenate([lo, hi], axis=1).astype(np.int32)

    def step(self) -> None:
        """Advance one tick; a coordinate that leaves [0, (N - side)*256] reflects."""
        self.pos = self.pos + self.vel
        top = (np.asarray(self.n, dtype=np.int64)[None, :] - self.side) * 256
        below = self.pos < 0
        self.pos = np.where(below, -self.pos, self.pos)
        self.vel = np.where(below, -self.vel, self.vel)
        above = self.pos > top
        self.pos = np.where(above, 2 * top - self.pos, self.pos)
        self.vel = np.where(above, -self.vel, self.vel)
        self.tick += 1


def make_moving_boxes(n: Tuple[int, int, int], count: int, seed: int,
                      side_lo: int = 6, side_hi: int = 16) -> MovingBoxes:
    """``count`` moving boxes: sides U{side_lo..side_hi}, corner uniform over the
    valid Q8 range, velocity a Q8 triple with 128^2 <= |v|^2 <= 512^2
    (0.5 to 2 voxels per tick) drawn component-wise U{-512..512} by rejection.
    Draw order per box: 3 sides, 3 corners, then velocity attempts.
    """
    rng = SplitMix64(seed, TAG_VELOCITIES)
    pos, vel, side = [], [], []
    for _ in range(count):
        s = [rng.between(side_lo, side_hi) for _ in range(3)]
        p = [rng.below((n[a] - s[a]) * 256 + 1) for a in range(3)]
        while True:
            v = [rng.between(-512, 512) for _ in range(3)]
            v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2]
            if 128 * 128 <= v2 <= 512 * 512:
                break
        pos.append(p)
        vel.append(v)
        side.append(s)
    return MovingBoxes(tuple(n), np.asarray(pos, np.int64), np.asarray(vel, np.int64),
                       np.asarray(side, np.int64))


def c5_scene(seed: int = 3) -> Tuple[Scene, MovingBoxes]:
    """256^3, the C2 arm, 300 static boxes (sides U{4..24}) + 16 moving boxes."""
    sc = make_scene(256, 256, 256, (128, 128, 0), C2_LENGTHS, 300, 4, 24, seed, "C5")
    mv = make_moving_boxes((256, 256, 256), 16, seed)
    return sc, mv


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: exponential gaps
    ``-ln(1 - u) / rate`` with ``u`` from the arrivals stream."""
    rng = SplitMix64(seed, TAG_ARRIVALS)
    t = 0.0
    out = []
    while True:
        t += -math.log(1.0 - rng.uniform01()) / rate_hz
        if t >= duration_s:
            break
        out.append(t)
    return np.asarray(out, dtype=np.float64)


def request_kinds(count: int, seed: int) -> np.ndarray:
    """0 = reach+path, 1 = replan of a live path; each with probability 1/2."""
    rng = SplitMix64(seed, TAG_ARRIVALS + 16)
    return np.asarray([rng.below(2) for _ in range(count)], dtype=np.int32)


__all__ = [
    "SplitMix64", "Scene", "make_scene", "draw_targets", "c1_scene", "c2_scene",
    "scaled_scene", "Problem", "c4_problems", "MovingBoxes", "make_moving_boxes",
    "c5_scene", "poisson_arrivals", "request_kinds", "C1_LENGTHS", "C2_LENGTHS",
]
