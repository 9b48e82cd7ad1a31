"""ORACLE -- test infrastructure, not product code.

Python access to the plain CPU oracle in ``ik_oracle.cpp`` (a byte-per-voxel
restatement of the gap map-seeking IK search and its path planner, written
from the paper's sections "The gap in gMS", "Testing for collisions", "The
procedure for IK solution", "Path Planning", "Smooth sequence computation",
"Filtering for smoothness" and "Dynamic Obstacles").

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA library: it
neither imports the product package nor is imported by it.

Parity status per function (details in the C++ header comment):

* ``shell``, ``supercover``, ``forward``, ``backward``, ``reach_many``,
  ``pose_valid``, ``guide``: pinned (brute force on tiny grids, closed forms,
  the worked supercover examples).
* ``waypoint_sets``, ``plan_path``, ``replan``: rules stated only in words by
  the paper; pinned by brute force over restricted balls on tiny grids and by
  invariants.  ``replan`` is pinned on every branch (kept path, forward chain
  from the current pose, the reach pose re-solved by the nearest-joint rule
  as a lexicographic minimum over all enumerated chains, unreachable
  target), and copies of it with a planted mistake fail that pin.  The paper
  prints no worked example for them.
* ``count_pairs``: pinned against a numpy shift-and-pack count.

Arrays: occupancy is uint8 ``[nz][ny][nx]`` (1 = occupied); poses are int32
``[S+1][3]`` in (x, y, z) order; sets are uint8 ``[..][nz][ny][nx]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ik_oracle.cpp")
_LIB = os.path.join(_HERE, "libik_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (plain -O2, no GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", _LIB]
        subprocess.check_call(cmd)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB)
            _lib.orc_count_pairs.restype = ctypes.c_long
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def shell_bounds(L: int, tol: float = 0.5) -> Tuple[int, int]:
    lo = ctypes.c_int()
    hi = ctypes.c_int()
    # the C ABI carries tol as a float; round it the same way
    _load().orc_shell_bounds(int(L), ctypes.c_double(float(np.float32(tol))), ctypes.byref(lo),
                             ctypes.byref(hi))
    return lo.value, hi.value


def arm_bounds(lengths: Sequence[int], tol: float = 0.5) -> Tuple[np.ndarray, np.ndarray]:
    b = [shell_bounds(L, tol) for L in lengths]
    return _i32([x[0] for x in b]), _i32([x[1] for x in b])


def shell(lo2: int, hi2: int) -> np.ndarray:
    lib = _load()
    n = lib.orc_shell(int(lo2), int(hi2), None, 0)
    out = np.zeros((max(n, 1), 3), np.int32)
    lib.orc_shell(int(lo2), int(hi2), _p(out), n)
    return out[:n]


def supercover(a, b) -> np.ndarray:
    lib = _load()
    a = _i32(a)
    b = _i32(b)
    cap = int(np.prod(np.abs(b - a) + 1))
    out = np.zeros((cap, 3), np.int32)
    n = lib.orc_supercover(_p(a), _p(b), _p(out), cap)
    return out[:n]


def rasterize(shape, boxes) -> np.ndarray:
    nx, ny, nz = shape
    boxes = _i32(boxes).reshape(-1, 6)
    occ = np.zeros((nz, ny, nx), np.uint8)
    _load().orc_rasterize(nx, ny, nz, _p(boxes), len(boxes), _p(occ))
    return occ


def _dims(occ: np.ndarray):
    nz, ny, nx = occ.shape
    return nx, ny, nz


def _limits(limits, S):
    """Per-segment direction limits: None, or a list of S entries, each None
    or (ax, ay, az, num, den) -> int32 [S][5] (zero rows = no limit)."""
    if limits is None:
        return None
    out = np.zeros((S, 5), np.int32)
    for k, c in enumerate(limits):
        if c is not None:
            out[k] = c
    return out


def forward(occ, lengths, root, tol: float = 0.5, limits=None) -> np.ndarray:
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    S = len(lengths)
    F = np.zeros((S + 1, nz, ny, nx), np.uint8)
    lim = _limits(limits, S)
    _load().orc_forward(nx, ny, nz, _p(occ), S, _p(lo2), _p(hi2), _p(_i32(root)), _p(F),
                        _p(lim) if lim is not None else None)
    return F


def backward(occ, lengths, T, tol: float = 0.5) -> np.ndarray:
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    S = len(lengths)
    B = np.zeros((S + 1, nz, ny, nx), np.uint8)
    _load().orc_backward(nx, ny, nz, _p(occ), S, _p(lo2), _p(hi2), _p(_u8(T)), _p(B))
    return B


def reach_many(occ, lengths, root, targets, want_sets: bool = False, threads: int = 1,
               tol: float = 0.5, limits=None):
    """Returns (poses [n][S+1][3], found [n], vsets [n][S+1][nz][ny][nx] or None)."""
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    S = len(lengths)
    targets = _i32(targets).reshape(-1, 3)
    n = len(targets)
    poses = np.zeros((n, S + 1, 3), np.int32)
    found = np.zeros(n, np.int32)
    vs = np.zeros((n, S + 1, nz, ny, nx), np.uint8) if want_sets else None
    lim = _limits(limits, S)
    _load().orc_reach_many(nx, ny, nz, _p(occ), S, _p(lo2), _p(hi2), _p(_i32(root)), n,
                           _p(targets), _p(poses), _p(found), _p(vs) if want_sets else None,
                           int(threads), _p(lim) if lim is not None else None)
    return poses, found, vs


def plan_between(occ, lengths, start_pose, guide_lengths, target, W: int, delta: int = 3,
                 eps2: int = 2, eps2_max: int = 8, max_relax: int = -1, tol: float = 0.5):
    """Path between arbitrary poses (section "Path between Arbitrary Poses";
    see orc_plan_between).  Returns (poses [W][S+1][3], relax [W][2], status,
    guide pose [Sv+1][3])."""
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    vlo2, vhi2 = arm_bounds(guide_lengths, tol)
    S, Sv = len(lengths), len(guide_lengths)
    poses = np.zeros((W, S + 1, 3), np.int32)
    relax = np.zeros((W, 2), np.int32)
    vpose = np.zeros((Sv + 1, 3), np.int32)
    st = ctypes.c_int32()
    _load().orc_plan_between(nx, ny, nz, _p(occ), S, _p(lo2), _p(hi2), _p(_i32(start_pose)), Sv,
                             _p(_i32(guide_lengths)), _p(vlo2), _p(vhi2), _p(_i32(target)), int(W),
                             int(delta), int(eps2), int(eps2_max), int(max_relax), _p(poses),
                             _p(relax), ctypes.byref(st), _p(vpose))
    return poses, relax, st.value, vpose


def dilate(occ, r2: int) -> np.ndarray:
    """Occupancy dilated by the ball |d|^2 <= r2 (section "Testing for
    collisions"), uint8 [nz][ny][nx]."""
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    out = np.zeros_like(occ)
    _load().orc_dilate(nx, ny, nz, _p(occ), int(r2), _p(out))
    return out


def reach_set(occ, lengths, root, T, cone=None, tol: float = 0.5):
    """Reach for a target set T ([nz][ny][nx], non-zero = target) with an
    optional approach cone (ax, ay, az, num, den) on the last segment
    (section "The gap in gMS"; see orc_reach_set).  Returns (pose [S+1][3],
    found, vsets [S+1][nz][ny][nx])."""
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    S = len(lengths)
    T = _u8(np.asarray(T) != 0)
    pose = np.zeros((S + 1, 3), np.int32)
    found = np.zeros(1, np.int32)
    vs = np.zeros((S + 1, nz, ny, nx), np.uint8)
    c = None if cone is None else _i32(cone)
    _load().orc_reach_set(nx, ny, nz, _p(occ), S, _p(lo2), _p(hi2), _p(_i32(root)), _p(T),
                          _p(c) if c is not None else None, _p(pose), _p(vs), _p(found))
    return pose, int(found[0]), vs


def pose_valid(occ, lengths, pose, tol: float = 0.5, limits=None) -> bool:
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    lim = _limits(limits, len(lengths))
    return bool(_load().orc_pose_valid(nx, ny, nz, _p(occ), len(lengths), _p(lo2), _p(hi2),
                                       _p(_i32(pose)), _p(lim) if lim is not None else None))


def guide(lengths, pose, W: int) -> np.ndarray:
    g = np.zeros((W, 3), np.int32)
    _load().orc_guide(len(lengths), _p(_i32(lengths)), _p(_i32(pose)), int(W), _p(g))
    return g


def waypoint_sets(occ, lengths, reach_pose, W: int, eps2: int = 2, eps2_max: int = 8,
                  want_sets: bool = True, threads: int = 1, tol: float = 0.5):
    """Returns (eps2_used [W], vsets [W][S+1][nz][ny][nx] or None)."""
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    S = len(lengths)
    used = np.zeros(W, np.int32)
    vs = np.zeros((W, S + 1, nz, ny, nx), np.uint8) if want_sets else None
    _load().orc_waypoint_sets(nx, ny, nz, _p(occ), S, _p(_i32(lengths)), _p(lo2), _p(hi2),
                              _p(_i32(reach_pose)), int(W), int(eps2), int(eps2_max),
                              _p(used), _p(vs) if want_sets else None, int(threads))
    return used, vs


def waypoint_sets_range(occ, lengths, reach_pose, W: int, j_lo: int, j_hi: int, eps2: int = 2,
                        eps2_max: int = 8, tol: float = 0.5):
    """Survivor sets of waypoints j_lo..j_hi-1 only: (eps2_used, vsets)."""
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    S = len(lengths)
    n = j_hi - j_lo
    used = np.zeros(n, np.int32)
    vs = np.zeros((n, S + 1, nz, ny, nx), np.uint8)
    _load().orc_waypoint_sets_range(nx, ny, nz, _p(occ), S, _p(_i32(lengths)), _p(lo2), _p(hi2),
                                    _p(_i32(reach_pose)), int(W), int(j_lo), int(j_hi), int(eps2),
                                    int(eps2_max), _p(used), _p(vs))
    return used, vs


def smooth_step(occ, lengths, vsets, ref_pose, delta: int = 3, max_relax: int = -1,
                tol: float = 0.5):
    """One smooth step from given survivor sets: (pose [S+1][3] or None, m)."""
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    S = len(lengths)
    pose = np.zeros((S + 1, 3), np.int32)
    m = ctypes.c_int32()
    _load().orc_smooth_step(nx, ny, nz, _p(occ), S, _p(lo2), _p(hi2), _p(_u8(vsets)),
                            _p(_i32(ref_pose)), int(delta), int(max_relax), _p(pose), ctypes.byref(m))
    return (pose if m.value >= 0 else None), m.value


def plan_path(occ, lengths, reach_pose, W: int, delta: int = 3, eps2: int = 2,
              eps2_max: int = 8, max_relax: int = -1, tol: float = 0.5, limits=None):
    """Returns (poses [W][S+1][3], relax [W][2], status)."""
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    S = len(lengths)
    poses = np.zeros((W, S + 1, 3), np.int32)
    relax = np.zeros((W, 2), np.int32)
    st = ctypes.c_int32()
    lim = _limits(limits, S)
    _load().orc_plan_path(nx, ny, nz, _p(occ), S, _p(_i32(lengths)), _p(lo2), _p(hi2),
                          _p(_i32(reach_pose)), int(W), int(delta), int(eps2), int(eps2_max),
                          int(max_relax), _p(poses), _p(relax), ctypes.byref(st),
                          _p(lim) if lim is not None else None)
    return poses, relax, st.value


def plan_short(occ, lengths, reach_pose, W: int, delta: int = 3, eps2: int = 2, eps2_max: int = 8,
               max_relax: int = -1, kmax: int = 2, tol: float = 0.5):
    """Short reaches: the guide is the pose of the shortest virtual arm
    (L_1 .. L_{k-1}, l for k <= kmax) that reaches the target, else the reach
    pose.  Returns (poses [W][S+1][3], relax [W][2], status, (k, l), shortcut
    pose [k+1][3] or None); poses None when the reach pose is not valid."""
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    S = len(lengths)
    poses = np.zeros((W, S + 1, 3), np.int32)
    relax = np.zeros((W, 2), np.int32)
    st = ctypes.c_int32()
    sc = np.zeros(2, np.int32)
    vpose = np.zeros((S + 1, 3), np.int32)
    rc = _load().orc_plan_short(nx, ny, nz, _p(occ), S, _p(_i32(lengths)), _p(lo2), _p(hi2),
                                ctypes.c_double(tol), _p(_i32(reach_pose)), int(W), int(delta), int(eps2),
                                int(eps2_max), int(max_relax), int(kmax), _p(poses), _p(relax),
                                ctypes.byref(st), _p(sc), _p(vpose))
    if rc < 0:
        return None, None, st.value, (0, 0), None
    k, l = int(sc[0]), int(sc[1])
    return poses, relax, st.value, (k, l), (vpose[:k + 1].copy() if k else None)


def plan_path_follow(occ, lengths, reach_pose, n: int, fold: bool, rad, eps2: int = 2,
                     eps2_max: int = 8, max_relax: int = -1, tol: float = 0.5):
    """The paper's follower and filter: the follower is joint S - fold, n
    guide points per segment of the reach polyline up to it, joint k moving
    at most rad[k-1] voxels per waypoint (-1: not filtered), the last
    segment folded along the path when fold.  Returns (poses [W][S+1][3],
    relax [W][2], status) with W = (S - fold) n + 1, or (None, None,
    status) when the reach pose is not valid."""
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    S = len(lengths)
    F = S - (1 if fold else 0)
    W = F * int(n) + 1
    rad = _i32(list(rad))
    assert rad.shape == (F,)
    poses = np.zeros((W, S + 1, 3), np.int32)
    relax = np.zeros((W, 2), np.int32)
    st = ctypes.c_int32()
    w = _load().orc_plan_path_follow(nx, ny, nz, _p(occ), S, _p(_i32(lengths)), _p(lo2), _p(hi2),
                                     _p(_i32(reach_pose)), int(n), int(bool(fold)), _p(rad),
                                     int(eps2), int(eps2_max), int(max_relax), _p(poses), _p(relax),
                                     ctypes.byref(st))
    if w < 0:
        return None, None, st.value
    return poses, relax, st.value


def replan(occ, lengths, poses_in, current: int, delta: int = 3, eps2: int = 2,
           eps2_max: int = 8, max_relax: int = -1, tol: float = 0.5):
    """Returns (poses [W][S+1][3], relax [W][2], status)."""
    occ = _u8(occ)
    nx, ny, nz = _dims(occ)
    lo2, hi2 = arm_bounds(lengths, tol)
    S = len(lengths)
    poses_in = _i32(poses_in)
    W = poses_in.shape[0]
    poses = np.zeros((W, S + 1, 3), np.int32)
    relax = np.zeros((W, 2), np.int32)
    st = ctypes.c_int32()
    _load().orc_replan(nx, ny, nz, _p(occ), S, _p(_i32(lengths)), _p(lo2), _p(hi2),
                       _p(poses_in), int(W), int(current), int(delta), int(eps2), int(eps2_max),
                       int(max_relax), _p(poses), _p(relax), ctypes.byref(st))
    return poses, relax, st.value


def count_pairs(lo2: int, hi2: int, X) -> Tuple[int, int]:
    """(active (offset, word) pairs, sum of supercover sizes over them) for D(X)."""
    X = _u8(X)
    nx, ny, nz = _dims(X)
    terms = ctypes.c_long()
    pairs = _load().orc_count_pairs(nx, ny, nz, int(lo2), int(hi2), _p(X), ctypes.byref(terms))
    return int(pairs), int(terms.value)


PATH_OK, PATH_RELAXED, PATH_BROKEN, PATH_UNREACHABLE, PATH_KEPT = range(5)
