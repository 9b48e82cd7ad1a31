"""Python binding of the C ABI in ``include/ik.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
part of the method itself: it converts arguments to pointers, calls the
library, checks the return code and shapes the outputs.  Host arrays are
numpy; device arrays are ``torch`` CUDA tensors (PyTorch supplies device
memory and streams, nothing else).

The library must have been built (``python -m paper_1906_10678_b300.build``);
importing this module without it raises ``ImportError``: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libik_b300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1906_10678_b300.build`")

_lib = ctypes.CDLL(LIB_PATH)

IK_OK, IK_ERR_ARG, IK_ERR_OOM, IK_ERR_CUDA, IK_ERR_TIMEOUT, IK_ERR_STATE, IK_ERR_UNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6)
IK_PATH_OK, IK_PATH_RELAXED, IK_PATH_BROKEN, IK_PATH_UNREACHABLE, IK_PATH_KEPT = range(5)
IK_OPT_EDGE_MASKS = 1
IK_OPT_TILE_DEPTH = 2
IK_OPT_DILATE_R2 = 3
IK_OPT_WORK_LIST = 4
IK_OPT_QUERY_PAIRS = 5
IK_OPT_TMA_MASKS = 6
IK_OPT_ROW_LANES = 7
IK_MAX_SEG = 16
IK_MAX_LEN = 100

_vp = ctypes.c_void_p
_i = ctypes.c_int


class IkArm(ctypes.Structure):
    _fields_ = [("n_seg", ctypes.c_int32), ("len", ctypes.POINTER(ctypes.c_int32)),
                ("tol", ctypes.c_float)]


class IkPathParams(ctypes.Structure):
    _fields_ = [("n_way", ctypes.c_int32), ("delta", ctypes.c_int32), ("eps2", ctypes.c_int32),
                ("eps2_max", ctypes.c_int32), ("max_relax", ctypes.c_int32)]


class IkFollowParams(ctypes.Structure):
    _fields_ = [("n_per_seg", ctypes.c_int32), ("fold", ctypes.c_int32),
                ("radius", ctypes.c_int32 * IK_MAX_SEG), ("eps2", ctypes.c_int32),
                ("eps2_max", ctypes.c_int32), ("max_relax", ctypes.c_int32),
                ("paper_radii", ctypes.c_int32)]


class IkProblem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("boxes", ctypes.POINTER(ctypes.c_int32)), ("n_boxes", ctypes.c_int32),
                ("n_seg", ctypes.c_int32), ("len", ctypes.POINTER(ctypes.c_int32)),
                ("tol", ctypes.c_float), ("root", ctypes.c_int32 * 3),
                ("target", ctypes.c_int32 * 3), ("n_way", ctypes.c_int32)]


class IkCone(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_int32 * 3), ("cos2_num", ctypes.c_int32),
                ("cos2_den", ctypes.c_int32)]


class IkBatchParams(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_int32), ("eps2", ctypes.c_int32), ("eps2_max", ctypes.c_int32),
                ("max_relax", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("ik_version", _i, [])
_sig("ik_strerror", ctypes.c_char_p, [_i])
_sig("ik_last_error_message", ctypes.c_char_p, [])
_sig("ik_create_grid", _i, [_i, _i, _i, _vp, ctypes.POINTER(_vp)])
_sig("ik_destroy_grid", _i, [_vp])
_sig("ik_grid_words", ctypes.c_size_t, [_vp])
_sig("ik_set_option", _i, [_vp, _i, _i])
_sig("ik_set_obstacles", _i, [_vp, _vp, ctypes.c_size_t, _i])
_sig("ik_set_boxes", _i, [_vp, _vp, _i, _i])
_sig("ik_get_obstacles", _i, [_vp, _vp, ctypes.c_size_t, _i])
_sig("ik_forward_sets", _i, [_vp, ctypes.POINTER(IkArm), _vp, _vp, _i])
_sig("ik_solve_reach", _i, [_vp, ctypes.POINTER(IkArm), _vp, _vp, _vp, _vp, ctypes.POINTER(_i)])
_sig("ik_solve_reach_many", _i, [_vp, ctypes.POINTER(IkArm), _vp, _vp, _i, _vp, _vp, _vp, _i])
_sig("ik_solve_reach_many_cone", _i, [_vp, ctypes.POINTER(IkArm), ctypes.POINTER(IkCone), _vp, _vp, _i,
                                      _vp, _vp, _vp, _i])
_sig("ik_solve_reach_set", _i, [_vp, ctypes.POINTER(IkArm), ctypes.POINTER(IkCone), _vp, _vp, _vp, _vp,
                                ctypes.POINTER(_i)])
_sig("ik_set_segment_limits", _i, [_vp, ctypes.POINTER(IkArm), _vp])
_sig("ik_guide", _i, [_vp, ctypes.POINTER(IkArm), _vp, _i, _vp])
_sig("ik_waypoint_sets", _i, [_vp, ctypes.POINTER(IkArm), _vp, _i, _i, _i, _vp, _vp])
_sig("ik_plan_path", _i, [_vp, ctypes.POINTER(IkArm), _vp, ctypes.POINTER(IkPathParams), _vp, _vp,
                          ctypes.POINTER(_i)])
_sig("ik_plan_path_short", _i, [_vp, ctypes.POINTER(IkArm), _vp, ctypes.POINTER(IkPathParams), _i, _vp,
                                _vp, ctypes.POINTER(_i), _vp, _vp])
_sig("ik_plan_path_follow", _i, [_vp, ctypes.POINTER(IkArm), _vp, ctypes.POINTER(IkFollowParams), _vp,
                                 _vp, ctypes.POINTER(_i)])
_sig("ik_reach_path_many", _i, [_vp, ctypes.POINTER(IkArm), _vp, _vp, _i,
                                ctypes.POINTER(IkPathParams), _vp, _vp, _vp, _vp, _vp, _i])
_sig("ik_plan_between", _i, [_vp, ctypes.POINTER(IkArm), _vp, ctypes.POINTER(IkArm), _vp,
                             ctypes.POINTER(IkPathParams), _vp, _vp, _vp, ctypes.POINTER(_i)])
_sig("ik_validate_poses", _i, [_vp, ctypes.POINTER(IkArm), _vp, _i, _vp])
_sig("ik_replan", _i, [_vp, ctypes.POINTER(IkArm), _vp, _i, _i, ctypes.POINTER(IkPathParams), _vp,
                       _vp, ctypes.POINTER(_i)])
_sig("ik_replan_many", _i, [_vp, ctypes.POINTER(IkArm), _vp, _vp, _vp, _i,
                            ctypes.POINTER(IkPathParams), _vp, _vp, _vp, _i])
_sig("ik_batch_output_sizes", _i, [_vp, _i, _vp, _vp, _vp])
_sig("ik_solve_batch", _i, [_vp, _i, ctypes.POINTER(IkBatchParams), _vp, _vp, _vp, _vp, _vp, _vp])
_sig("ik_batch_engine_create", _i, [ctypes.POINTER(_vp)])
_sig("ik_batch_engine_destroy", _i, [_vp])
_sig("ik_batch_engine_set_budget", _i, [_vp, ctypes.c_size_t])
_sig("ik_batch_engine_set_timeout", _i, [_vp, ctypes.c_int64])
_sig("ik_batch_engine_set_pairs", _i, [_vp, _i])
_sig("ik_solve_batch_async", _i, [_vp, _vp, _i, ctypes.POINTER(IkBatchParams), _vp, _vp, _vp, _vp, _vp, _vp,
                                  _vp])
_sig("ik_batch_capture_uneven", _i, [_vp, _vp, _i, ctypes.POINTER(IkBatchParams), _vp, _vp, _vp, _vp, _vp, _vp,
                                     ctypes.POINTER(_vp)])
_sig("ik_batch_graph_launch", _i, [_vp, _vp])
_sig("ik_batch_graph_destroy", _i, [_vp])
_sig("ik_batch_capture", _i, [_vp, ctypes.POINTER(IkArm), _vp, _vp, _i, _vp, _i,
                              ctypes.POINTER(IkPathParams), _vp, _vp, _vp, _vp, _vp,
                              ctypes.POINTER(_vp)])
_sig("ik_batch_launch", _i, [_vp])
_sig("ik_batch_destroy", _i, [_vp])
_sig("ik_forward_sets_noalloc", _i, [_vp, _i, _i, _i, ctypes.POINTER(IkArm), _vp, _vp, _vp])
_sig("ik_profile_enable", _i, [_vp, _i, _i])
_sig("ik_profile_read", _i, [_vp, _vp, _vp, _vp, _i])
_sig("ik_profile_name", ctypes.c_char_p, [_i])
_sig("ik_shell_offsets", _i, [_i, ctypes.c_float, _vp, _vp, _i])
_sig("ik_supercover_offsets", _i, [_vp, _vp, _i])
_sig("ik_row_table", _i, [_i, ctypes.c_float, _vp, _vp, _vp, _i, _vp, _i])
_sig("ik_row_mask_table", _i, [_i, ctypes.c_float, _vp, _i, _vp, _i])
_sig("ik_probe_peak", _i, [_i, _i, _i, _vp, _vp, _vp, _vp])

EXPORTED = [
    "ik_version", "ik_strerror", "ik_last_error_message", "ik_create_grid", "ik_destroy_grid",
    "ik_grid_words", "ik_set_option", "ik_set_obstacles", "ik_set_boxes", "ik_get_obstacles", "ik_forward_sets",
    "ik_solve_reach", "ik_solve_reach_many", "ik_solve_reach_many_cone", "ik_solve_reach_set", "ik_set_segment_limits", "ik_guide", "ik_waypoint_sets", "ik_plan_path", "ik_plan_path_follow", "ik_plan_path_short",
    "ik_reach_path_many", "ik_plan_between", "ik_validate_poses", "ik_replan", "ik_replan_many",
    "ik_batch_output_sizes", "ik_solve_batch", "ik_batch_engine_create", "ik_batch_engine_destroy",
    "ik_batch_engine_set_budget", "ik_batch_engine_set_timeout", "ik_batch_engine_set_pairs",
    "ik_solve_batch_async", "ik_batch_capture_uneven", "ik_batch_graph_launch", "ik_batch_graph_destroy",
    "ik_batch_capture",
    "ik_batch_launch", "ik_batch_destroy", "ik_forward_sets_noalloc",
    "ik_profile_enable",
    "ik_profile_read", "ik_profile_name", "ik_shell_offsets", "ik_supercover_offsets", "ik_row_table", "ik_row_mask_table",
    "ik_probe_peak",
]


class IkError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.ik_strerror(code).decode()
        extra = _lib.ik_last_error_message().decode()
        super().__init__(f"{where}: {msg} ({code}){': ' + extra if extra else ''}")
        self.code = code


def _check(rc: int, where: str) -> None:
    if rc != IK_OK:
        raise IkError(rc, where)


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_vp)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _dev_ptr(t) -> int:
    """Device pointer of a contiguous CUDA tensor."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


class Arm:
    """Keeps the length array alive while the C struct points at it."""

    def __init__(self, lengths: Sequence[int], tol: float = 0.5):
        self.lengths = _i32(lengths)
        self.c = IkArm(len(self.lengths), self.lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                       float(tol))

    @property
    def S(self) -> int:
        return len(self.lengths)


def _arm(a) -> Arm:
    return a if isinstance(a, Arm) else Arm(a)


def path_params(n_way: int, delta: int = 3, eps2: int = 2, eps2_max: int = 8,
                max_relax: int = -1) -> IkPathParams:
    return IkPathParams(int(n_way), int(delta), int(eps2), int(eps2_max), int(max_relax))


# ------------------------------------------------------------------ layout

def pack_bits(mask: np.ndarray) -> np.ndarray:
    """bool/uint8 [nz][ny][nx] -> uint32 words (x-packed, bit b = x % 32)."""
    m = np.ascontiguousarray(np.asarray(mask).astype(bool))
    nz, ny, nx = m.shape
    b = np.packbits(m.reshape(nz, ny, nx // 32, 32), axis=-1, bitorder="little")
    return np.ascontiguousarray(b).view(np.uint32).reshape(-1)


def unpack_bits(words: np.ndarray, shape) -> np.ndarray:
    """uint32 words -> bool [nz][ny][nx] for grid ``shape`` = (nx, ny, nz)."""
    nx, ny, nz = shape
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32)).reshape(-1, nz, ny, nx // 32)
    b = np.unpackbits(w.view(np.uint8).reshape(w.shape[0], nz, ny, nx // 32, 4), axis=-1,
                      bitorder="little")
    return b.reshape(w.shape[0], nz, ny, nx).astype(bool)


# --------------------------------------------------------------- functions

def ik_version() -> int:
    return _lib.ik_version()


def ik_create_grid(nx: int, ny: int, nz: int, stream: int = 0) -> int:
    h = _vp()
    _check(_lib.ik_create_grid(nx, ny, nz, _vp(stream) if stream else None, ctypes.byref(h)),
           "ik_create_grid")
    return h.value


def ik_destroy_grid(g: int) -> None:
    _check(_lib.ik_destroy_grid(g), "ik_destroy_grid")


def ik_grid_words(g: int) -> int:
    return int(_lib.ik_grid_words(g))


def ik_set_option(g: int, option: int, value: int) -> None:
    _check(_lib.ik_set_option(g, option, int(value)), "ik_set_option")


def ik_set_boxes(g: int, boxes) -> None:
    if hasattr(boxes, "is_cuda"):
        _check(_lib.ik_set_boxes(g, _dev_ptr(boxes), boxes.shape[0], 1), "ik_set_boxes")
        return
    b = _i32(boxes).reshape(-1, 6)
    _check(_lib.ik_set_boxes(g, _np_ptr(b), len(b), 0), "ik_set_boxes")


def ik_set_obstacles(g: int, words) -> None:
    if hasattr(words, "is_cuda"):
        _check(_lib.ik_set_obstacles(g, _dev_ptr(words), words.numel(), 1), "ik_set_obstacles")
        return
    w = np.ascontiguousarray(words, dtype=np.uint32)
    _check(_lib.ik_set_obstacles(g, _np_ptr(w), w.size, 0), "ik_set_obstacles")


def ik_get_obstacles(g: int) -> np.ndarray:
    out = np.zeros(ik_grid_words(g), np.uint32)
    _check(_lib.ik_get_obstacles(g, _np_ptr(out), out.size, 0), "ik_get_obstacles")
    return out


def ik_forward_sets(g: int, arm, root) -> np.ndarray:
    arm = _arm(arm)
    out = np.zeros((arm.S + 1, ik_grid_words(g)), np.uint32)
    _check(_lib.ik_forward_sets(g, ctypes.byref(arm.c), _np_ptr(_i32(root)), _np_ptr(out), 0),
           "ik_forward_sets")
    return out


def ik_solve_reach(g: int, arm, root, target, want_sets: bool = False):
    """Returns (pose [S+1][3], found, vsets [S+1][words] or None)."""
    arm = _arm(arm)
    pose = np.zeros((arm.S + 1, 3), np.int32)
    vs = np.zeros((arm.S + 1, ik_grid_words(g)), np.uint32) if want_sets else None
    f = _i()
    _check(_lib.ik_solve_reach(g, ctypes.byref(arm.c), _np_ptr(_i32(root)), _np_ptr(_i32(target)),
                               _np_ptr(pose), _np_ptr(vs), ctypes.byref(f)), "ik_solve_reach")
    return pose, bool(f.value), vs


def ik_solve_reach_many(g: int, arm, root, targets, want_sets: bool = False):
    """Host form.  Returns (poses [n][S+1][3], found [n], vsets or None)."""
    arm = _arm(arm)
    t = _i32(targets).reshape(-1, 3)
    n = len(t)
    poses = np.zeros((n, arm.S + 1, 3), np.int32)
    found = np.zeros(n, np.int32)
    vs = np.zeros((n, arm.S + 1, ik_grid_words(g)), np.uint32) if want_sets else None
    _check(_lib.ik_solve_reach_many(g, ctypes.byref(arm.c), _np_ptr(_i32(root)), _np_ptr(t), n,
                                    _np_ptr(poses), _np_ptr(found), _np_ptr(vs), 0),
           "ik_solve_reach_many")
    return poses, found, vs


def ik_solve_reach_many_device(g: int, arm, root, targets, poses, found) -> None:
    """Device form: ``targets`` int32 [n][3], ``poses`` int32 [n][S+1][3] and
    ``found`` int32 [n] are CUDA tensors."""
    arm = _arm(arm)
    n = targets.shape[0]
    _check(_lib.ik_solve_reach_many(g, ctypes.byref(arm.c), _np_ptr(_i32(root)), _dev_ptr(targets),
                                    n, _dev_ptr(poses), _dev_ptr(found), None, 1),
           "ik_solve_reach_many")


def cone(axis, cos2_num: int, cos2_den: int) -> IkCone:
    """Approach cone of the last segment: angle to ``axis`` at most theta with
    cos^2 theta = cos2_num / cos2_den."""
    c = IkCone()
    c.axis[:] = [int(v) for v in axis]
    c.cos2_num, c.cos2_den = int(cos2_num), int(cos2_den)
    return c


def _cone_ref(c):
    return None if c is None else ctypes.byref(c)


def ik_solve_reach_many_cone(g: int, arm, cone_, root, targets, want_sets: bool = False):
    """Host form of ik_solve_reach_many_cone (``cone_`` an IkCone or None).
    Returns (poses [n][S+1][3], found [n], vsets or None)."""
    arm = _arm(arm)
    t = _i32(targets).reshape(-1, 3)
    n = len(t)
    poses = np.zeros((n, arm.S + 1, 3), np.int32)
    found = np.zeros(n, np.int32)
    vs = np.zeros((n, arm.S + 1, ik_grid_words(g)), np.uint32) if want_sets else None
    _check(_lib.ik_solve_reach_many_cone(g, ctypes.byref(arm.c), _cone_ref(cone_), _np_ptr(_i32(root)),
                                         _np_ptr(t), n, _np_ptr(poses), _np_ptr(found), _np_ptr(vs), 0),
           "ik_solve_reach_many_cone")
    return poses, found, vs


def ik_solve_reach_many_cone_device(g: int, arm, cone_, root, targets, poses, found) -> None:
    """Device form: ``targets``, ``poses`` and ``found`` are int32 CUDA tensors."""
    arm = _arm(arm)
    _check(_lib.ik_solve_reach_many_cone(g, ctypes.byref(arm.c), _cone_ref(cone_), _np_ptr(_i32(root)),
                                         _dev_ptr(targets), targets.shape[0], _dev_ptr(poses),
                                         _dev_ptr(found), None, 1), "ik_solve_reach_many_cone")


def ik_solve_reach_set(g: int, arm, cone_, root, target_words, want_sets: bool = False):
    """Reach for a target set (packed words, as ``pack_bits`` gives) with an
    optional approach cone.  Returns (pose [S+1][3], found, vsets or None)."""
    arm = _arm(arm)
    tw = np.ascontiguousarray(target_words, dtype=np.uint32).reshape(-1)
    if tw.size != ik_grid_words(g):
        raise ValueError("target_words must hold ik_grid_words(g) words")
    pose = np.zeros((arm.S + 1, 3), np.int32)
    vs = np.zeros((arm.S + 1, ik_grid_words(g)), np.uint32) if want_sets else None
    found = ctypes.c_int(0)
    _check(_lib.ik_solve_reach_set(g, ctypes.byref(arm.c), _cone_ref(cone_), _np_ptr(_i32(root)),
                                   _np_ptr(tw), _np_ptr(pose), _np_ptr(vs), ctypes.byref(found)),
           "ik_solve_reach_set")
    return pose, found.value, vs


def ik_set_segment_limits(g: int, arm, limits) -> None:
    """Per-segment direction limits for this arm on this grid: ``limits`` is
    None (clear) or a list of n_seg entries, each None (free) or an IkCone /
    (axis, cos2_num, cos2_den)."""
    arm = _arm(arm)
    if limits is None:
        _check(_lib.ik_set_segment_limits(g, ctypes.byref(arm.c), None), "ik_set_segment_limits")
        return
    arr = (IkCone * arm.S)()
    for k, c in enumerate(limits):
        if c is None:
            continue
        if not isinstance(c, IkCone):
            c = cone(*c)
        arr[k] = c
    _check(_lib.ik_set_segment_limits(g, ctypes.byref(arm.c), arr), "ik_set_segment_limits")


def ik_guide(g: int, arm, reach_pose, n_way: int) -> np.ndarray:
    arm = _arm(arm)
    out = np.zeros((n_way, 3), np.int32)
    _check(_lib.ik_guide(g, ctypes.byref(arm.c), _np_ptr(_i32(reach_pose)), n_way, _np_ptr(out)),
           "ik_guide")
    return out


def ik_waypoint_sets(g: int, arm, reach_pose, n_way: int, eps2: int = 2, eps2_max: int = 8,
                     want_sets: bool = True):
    """Returns (eps2_used [W], vsets [W][S+1][words] or None)."""
    arm = _arm(arm)
    used = np.zeros(n_way, np.int32)
    vs = np.zeros((n_way, arm.S + 1, ik_grid_words(g)), np.uint32) if want_sets else None
    _check(_lib.ik_waypoint_sets(g, ctypes.byref(arm.c), _np_ptr(_i32(reach_pose)), n_way, eps2,
                                 eps2_max, _np_ptr(used), _np_ptr(vs)), "ik_waypoint_sets")
    return used, vs


def ik_plan_path(g: int, arm, reach_pose, n_way: int, delta: int = 3, eps2: int = 2,
                 eps2_max: int = 8, max_relax: int = -1):
    """Returns (poses [W][S+1][3], relax [W][2], status)."""
    arm = _arm(arm)
    pp = path_params(n_way, delta, eps2, eps2_max, max_relax)
    poses = np.zeros((n_way, arm.S + 1, 3), np.int32)
    relax = np.zeros((n_way, 2), np.int32)
    st = _i()
    _check(_lib.ik_plan_path(g, ctypes.byref(arm.c), _np_ptr(_i32(reach_pose)), ctypes.byref(pp),
                             _np_ptr(poses), _np_ptr(relax), ctypes.byref(st)), "ik_plan_path")
    return poses, relax, st.value


def ik_plan_path_short(g: int, arm, reach_pose, n_way: int, delta: int = 3, eps2: int = 2,
                       eps2_max: int = 8, max_relax: int = -1, k_max: int = 2):
    """Short reaches.  Returns (poses [W][S+1][3], relax [W][2], status,
    (k, l), shortcut pose [k+1][3] or None)."""
    arm = _arm(arm)
    pp = path_params(n_way, delta, eps2, eps2_max, max_relax)
    poses = np.zeros((n_way, arm.S + 1, 3), np.int32)
    relax = np.zeros((n_way, 2), np.int32)
    sc = np.zeros(2, np.int32)
    gp = np.zeros((int(k_max) + 1, 3), np.int32)
    st = _i()
    _check(_lib.ik_plan_path_short(g, ctypes.byref(arm.c), _np_ptr(_i32(reach_pose)), ctypes.byref(pp),
                                   int(k_max), _np_ptr(poses), _np_ptr(relax), ctypes.byref(st),
                                   _np_ptr(sc), _np_ptr(gp)), "ik_plan_path_short")
    k, l = int(sc[0]), int(sc[1])
    return poses, relax, st.value, (k, l), (gp[:k + 1].copy() if k else None)


def ik_plan_path_follow(g: int, arm, reach_pose, n_per_seg: int, fold: bool, radius=None, eps2: int = 2,
                        eps2_max: int = 8, max_relax: int = -1):
    """The paper's follower path: follower joint S - fold, n_per_seg guide
    points per segment, joint k filtered to radius[k-1] voxels (-1: not
    filtered; radius None: the library applies the paper's filter on joints
    1 and 2), the last segment folded along the path when fold.  Returns
    (poses [W][S+1][3], relax [W][2], status), W = (S - fold) n_per_seg + 1."""
    arm = _arm(arm)
    F = arm.S - (1 if fold else 0)
    fp = IkFollowParams()
    fp.n_per_seg = int(n_per_seg)
    fp.fold = 1 if fold else 0
    if radius is None:
        fp.paper_radii = 1
        for k in range(IK_MAX_SEG):
            fp.radius[k] = -1
    else:
        radius = [int(r) for r in radius]
        if len(radius) != F:
            raise ValueError(f"radius needs {F} entries (joints 1..{F})")
        fp.paper_radii = 0
        for k in range(IK_MAX_SEG):
            fp.radius[k] = radius[k] if k < F else -1
    fp.eps2, fp.eps2_max, fp.max_relax = int(eps2), int(eps2_max), int(max_relax)
    W = F * int(n_per_seg) + 1
    poses = np.zeros((W, arm.S + 1, 3), np.int32)
    relax = np.zeros((W, 2), np.int32)
    st = _i()
    _check(_lib.ik_plan_path_follow(g, ctypes.byref(arm.c), _np_ptr(_i32(reach_pose)), ctypes.byref(fp),
                                    _np_ptr(poses), _np_ptr(relax), ctypes.byref(st)),
           "ik_plan_path_follow")
    return poses, relax, st.value


def ik_reach_path_many(g: int, arm, root, targets, n_way: int, delta: int = 3, eps2: int = 2,
                       eps2_max: int = 8, max_relax: int = -1):
    """Host form.  Returns (reach [n][S+1][3], found [n], poses [n][W][S+1][3],
    relax [n][W][2], status [n])."""
    arm = _arm(arm)
    pp = path_params(n_way, delta, eps2, eps2_max, max_relax)
    t = _i32(targets).reshape(-1, 3)
    n, S = len(t), arm.S
    reach = np.zeros((n, S + 1, 3), np.int32)
    found = np.zeros(n, np.int32)
    poses = np.zeros((n, n_way, S + 1, 3), np.int32)
    relax = np.zeros((n, n_way, 2), np.int32)
    status = np.zeros(n, np.int32)
    _check(_lib.ik_reach_path_many(g, ctypes.byref(arm.c), _np_ptr(_i32(root)), _np_ptr(t), n,
                                   ctypes.byref(pp), _np_ptr(reach), _np_ptr(found), _np_ptr(poses),
                                   _np_ptr(relax), _np_ptr(status), 0), "ik_reach_path_many")
    return reach, found, poses, relax, status


def ik_reach_path_many_device(g: int, arm, root, targets, n_way: int, reach, found, poses, relax,
                              status, delta: int = 3, eps2: int = 2, eps2_max: int = 8,
                              max_relax: int = -1) -> None:
    """Device form: every array argument is a contiguous int32 CUDA tensor."""
    arm = _arm(arm)
    pp = path_params(n_way, delta, eps2, eps2_max, max_relax)
    _check(_lib.ik_reach_path_many(g, ctypes.byref(arm.c), _np_ptr(_i32(root)), _dev_ptr(targets),
                                   targets.shape[0], ctypes.byref(pp), _dev_ptr(reach),
                                   _dev_ptr(found), _dev_ptr(poses), _dev_ptr(relax),
                                   _dev_ptr(status), 1), "ik_reach_path_many")


class Batch:
    """A captured reach + path batch (``ik_batch_capture``); all arrays are
    contiguous int32 CUDA tensors that stay alive with the batch."""

    def __init__(self, g: int, arm, root, boxes, targets, n_way: int, reach, found, poses, relax,
                 status, delta: int = 3, eps2: int = 2, eps2_max: int = 8, max_relax: int = -1):
        self.arm = _arm(arm)
        self.pp = path_params(n_way, delta, eps2, eps2_max, max_relax)
        self.keep = (boxes, targets, reach, found, poses, relax, status)
        h = _vp()
        _check(_lib.ik_batch_capture(g, ctypes.byref(self.arm.c), _np_ptr(_i32(root)),
                                     _dev_ptr(boxes), boxes.shape[0], _dev_ptr(targets),
                                     targets.shape[0], ctypes.byref(self.pp), _dev_ptr(reach),
                                     _dev_ptr(found), _dev_ptr(poses), _dev_ptr(relax),
                                     _dev_ptr(status), ctypes.byref(h)), "ik_batch_capture")
        self.h = h.value

    def launch(self) -> None:
        _check(_lib.ik_batch_launch(self.h), "ik_batch_launch")

    def close(self) -> None:
        if self.h:
            _check(_lib.ik_batch_destroy(self.h), "ik_batch_destroy")
            self.h = 0


def _problem_array(problems):
    """ik_problem structs of a list of dicts (shape, boxes, lengths, root,
    target, n_way; tol 0.5), with the arrays they point at kept alive."""
    n = len(problems)
    keep = []
    arr = (IkProblem * max(n, 1))()
    for i, p in enumerate(problems):
        b = _i32(p["boxes"]).reshape(-1, 6)
        L = _i32(p["lengths"])
        keep += [b, L]
        arr[i].nx, arr[i].ny, arr[i].nz = (int(v) for v in p["shape"])
        arr[i].boxes = b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        arr[i].n_boxes = len(b)
        arr[i].n_seg = len(L)
        arr[i].len = L.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        arr[i].tol = 0.5
        arr[i].root[:] = [int(v) for v in p["root"]]
        arr[i].target[:] = [int(v) for v in p["target"]]
        arr[i].n_way = int(p["n_way"])
    return arr, keep


def ik_batch_output_sizes(problems):
    """(reach ints, poses ints, relax ints) of the packed outputs."""
    arr, keep = _problem_array(problems)
    sizes = [ctypes.c_size_t() for _ in range(3)]
    _check(_lib.ik_batch_output_sizes(ctypes.cast(arr, _vp), len(problems), *(ctypes.byref(x) for x in sizes)),
           "ik_batch_output_sizes")
    return tuple(x.value for x in sizes)


def unpack_batch(problems, found, reach, poses, relax, status):
    """Per-problem dicts of the packed outputs (numpy arrays)."""
    out, r0, p0, x0 = [], 0, 0, 0
    for i, p in enumerate(problems):
        S, W = len(p["lengths"]), int(p["n_way"])
        out.append({"found": int(found[i]), "status": int(status[i]),
                    "reach": reach[r0:r0 + 3 * (S + 1)].reshape(S + 1, 3),
                    "poses": poses[p0:p0 + 3 * (S + 1) * W].reshape(W, S + 1, 3),
                    "relax": relax[x0:x0 + 2 * W].reshape(W, 2)})
        r0 += 3 * (S + 1)
        p0 += 3 * (S + 1) * W
        x0 += 2 * W
    return out


def ik_solve_batch(problems, delta: int = 3, eps2: int = 2, eps2_max: int = 8, max_relax: int = -1,
                   blocks_per_sm: int = 0):
    """problems: list of dicts with shape (nx, ny, nz), boxes [n][6], lengths,
    root, target, n_way (tol 0.5).  Returns (list of per-problem dicts with
    found, reach, poses, relax, status; device ms of the batch)."""
    n = len(problems)
    arr, keep = _problem_array(problems)
    r_n, p_n, x_n = ik_batch_output_sizes(problems)
    found = np.zeros(n, np.int32)
    status = np.zeros(n, np.int32)
    reach = np.zeros(max(r_n, 1), np.int32)
    poses = np.zeros(max(p_n, 1), np.int32)
    relax = np.zeros(max(x_n, 1), np.int32)
    ms = ctypes.c_double()
    bp = IkBatchParams(delta, eps2, eps2_max, max_relax, blocks_per_sm)
    _check(_lib.ik_solve_batch(ctypes.cast(arr, _vp), n, ctypes.byref(bp), _np_ptr(found),
                               _np_ptr(reach), _np_ptr(poses), _np_ptr(relax), _np_ptr(status),
                               ctypes.byref(ms)), "ik_solve_batch")
    return unpack_batch(problems, found, reach, poses, relax, status), ms.value


class BatchEngine:
    """Owning wrapper of an ``ik_batch_engine`` (current device)."""

    def __init__(self):
        h = _vp()
        _check(_lib.ik_batch_engine_create(ctypes.byref(h)), "ik_batch_engine_create")
        self.h = h.value

    def set_budget(self, pool_bytes: int) -> None:
        _check(_lib.ik_batch_engine_set_budget(self.h, int(pool_bytes)), "ik_batch_engine_set_budget")

    def set_timeout(self, ns: int) -> None:
        _check(_lib.ik_batch_engine_set_timeout(self.h, int(ns)), "ik_batch_engine_set_timeout")

    def set_pairs(self, on: int) -> None:
        _check(_lib.ik_batch_engine_set_pairs(self.h, int(on)), "ik_batch_engine_set_pairs")

    def solve_async(self, problems, found, reach, poses, relax, status, job_rc, stream: int = 0,
                    delta: int = 3, eps2: int = 2, eps2_max: int = 8, max_relax: int = -1,
                    blocks_per_sm: int = 0) -> None:
        """Enqueue the batch on ``stream``; outputs are int32 CUDA tensors of
        the packed sizes (ik_batch_output_sizes) and job_rc [n]."""
        arr, keep = _problem_array(problems)
        bp = IkBatchParams(delta, eps2, eps2_max, max_relax, blocks_per_sm)
        _check(_lib.ik_solve_batch_async(self.h, ctypes.cast(arr, _vp), len(problems), ctypes.byref(bp),
                                         _dev_ptr(found), _dev_ptr(reach), _dev_ptr(poses), _dev_ptr(relax),
                                         _dev_ptr(status), _dev_ptr(job_rc), _vp(stream) if stream else None),
               "ik_solve_batch_async")

    def capture(self, problems, found, reach, poses, relax, status, job_rc, delta: int = 3, eps2: int = 2,
                eps2_max: int = 8, max_relax: int = -1, blocks_per_sm: int = 0) -> "BatchGraph":
        """The batch as a CUDA graph of one persistent launch writing into the
        given CUDA tensors (ik_batch_capture_uneven); replay with .launch()."""
        arr, keep = _problem_array(problems)
        bp = IkBatchParams(delta, eps2, eps2_max, max_relax, blocks_per_sm)
        h = _vp()
        _check(_lib.ik_batch_capture_uneven(self.h, ctypes.cast(arr, _vp), len(problems), ctypes.byref(bp),
                                            _dev_ptr(found), _dev_ptr(reach), _dev_ptr(poses), _dev_ptr(relax),
                                            _dev_ptr(status), _dev_ptr(job_rc), ctypes.byref(h)),
               "ik_batch_capture_uneven")
        return BatchGraph(h.value, (found, reach, poses, relax, status, job_rc))

    def close(self) -> None:
        if self.h:
            _lib.ik_batch_engine_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchGraph:
    """Owning wrapper of an ``ik_batch_graph`` (it keeps its output tensors
    alive)."""

    def __init__(self, h: int, outputs):
        self.h = h
        self._outputs = outputs

    def launch(self, stream: int = 0) -> None:
        _check(_lib.ik_batch_graph_launch(self.h, _vp(stream) if stream else None), "ik_batch_graph_launch")

    def close(self) -> None:
        if self.h:
            _lib.ik_batch_graph_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ik_plan_between(g: int, arm, start_pose, guide_arm, target, n_way: int, delta: int = 3,
                    eps2: int = 2, eps2_max: int = 8, max_relax: int = -1):
    """Path between arbitrary poses.  Returns (poses [W][S+1][3], relax [W][2],
    status, guide pose [Sv+1][3])."""
    arm = _arm(arm)
    garm = _arm(guide_arm)
    pp = path_params(n_way, delta, eps2, eps2_max, max_relax)
    poses = np.zeros((n_way, arm.S + 1, 3), np.int32)
    relax = np.zeros((n_way, 2), np.int32)
    gpose = np.zeros((garm.S + 1, 3), np.int32)
    st = ctypes.c_int(0)
    _check(_lib.ik_plan_between(g, ctypes.byref(arm.c), _np_ptr(_i32(start_pose)), ctypes.byref(garm.c),
                                _np_ptr(_i32(target)), ctypes.byref(pp), _np_ptr(poses), _np_ptr(relax),
                                _np_ptr(gpose), ctypes.byref(st)), "ik_plan_between")
    return poses, relax, st.value, gpose


def ik_validate_poses(g: int, arm, poses) -> np.ndarray:
    arm = _arm(arm)
    p = _i32(poses).reshape(-1, arm.S + 1, 3)
    out = np.zeros(len(p), np.int32)
    _check(_lib.ik_validate_poses(g, ctypes.byref(arm.c), _np_ptr(p), len(p), _np_ptr(out)),
           "ik_validate_poses")
    return out


def ik_replan(g: int, arm, poses, current: int, delta: int = 3, eps2: int = 2, eps2_max: int = 8,
              max_relax: int = -1):
    """Returns (poses [W][S+1][3], relax [W][2], status)."""
    arm = _arm(arm)
    p = _i32(poses)
    W = p.shape[0]
    pp = path_params(W, delta, eps2, eps2_max, max_relax)
    out = np.zeros_like(p)
    relax = np.zeros((W, 2), np.int32)
    st = _i()
    _check(_lib.ik_replan(g, ctypes.byref(arm.c), _np_ptr(p), W, current, ctypes.byref(pp),
                          _np_ptr(out), _np_ptr(relax), ctypes.byref(st)), "ik_replan")
    return out, relax, st.value


def ik_forward_sets_noalloc(occ_words, shape, arm, root, fsets_out, stream: int = 0) -> None:
    """Device form only: ``occ_words`` uint32/int32 CUDA tensor of the
    occupancy words, ``fsets_out`` CUDA tensor of (S+1) * words uint32/int32;
    no allocation happens inside the call."""
    arm = _arm(arm)
    nx, ny, nz = shape
    _check(_lib.ik_forward_sets_noalloc(_dev_ptr(occ_words), nx, ny, nz, ctypes.byref(arm.c),
                                        _np_ptr(_i32(root)), _dev_ptr(fsets_out),
                                        _vp(stream) if stream else None),
           "ik_forward_sets_noalloc")


PROBE_LOP3, PROBE_SHF, PROBE_LDS = 0, 1, 2


def ik_probe_peak(kind: int, blocks_per_sm: int = 8, iters: int = 20000, stream: int = 0) -> dict:
    """One throughput probe on the current device: {"ops_per_s", "ms", "sm_mhz"}."""
    r = np.zeros(3, np.float64)
    p = r.ctypes.data
    _check(_lib.ik_probe_peak(int(kind), int(blocks_per_sm), int(iters), _vp(stream) if stream else None,
                              _vp(p), _vp(p + 8), _vp(p + 16)), "ik_probe_peak")
    return {"ops_per_s": float(r[0]), "ms": float(r[1]), "sm_mhz": float(r[2])}


def ik_profile_enable(g: int, timing: bool = True, counting: bool = False) -> None:
    _check(_lib.ik_profile_enable(g, int(timing), int(counting)), "ik_profile_enable")


def ik_profile_read(g: int) -> dict:
    """{kernel class: {"ms", "launches", "visited", "nonzero", "mask_words", "out_words"}}."""
    cap = 32
    ms = np.zeros(cap, np.float64)
    n = np.zeros(cap, np.int64)
    c = np.zeros((cap, 8), np.uint64)
    k = _lib.ik_profile_read(g, _np_ptr(ms), _np_ptr(n), _np_ptr(c), cap)
    if k < 0:
        raise IkError(k, "ik_profile_read")
    out = {}
    for i in range(k):
        out[_lib.ik_profile_name(i).decode()] = {
            "ms": float(ms[i]), "launches": int(n[i]), "visited": int(c[i, 0]),
            "nonzero": int(c[i, 1]), "mask_words": int(c[i, 2]), "out_words": int(c[i, 3]),
            "warp_iters": int(c[i, 4]), "blocks": int(c[i, 5]), "walk_warps": int(c[i, 6]),
            "walk_lanes": int(c[i, 7])}
    return out


def ik_profile_name(i: int) -> str:
    return _lib.ik_profile_name(i).decode()


def ik_replan_many(g: int, arm, root, poses, current, delta: int = 3, eps2: int = 2,
                   eps2_max: int = 8, max_relax: int = -1):
    """Host form.  poses [n][W][S+1][3], current [n] (-1 = empty slot).
    Returns (poses, relax [n][W][2], status [n])."""
    arm = _arm(arm)
    p = _i32(poses)
    n, W = p.shape[0], p.shape[1]
    pp = path_params(W, delta, eps2, eps2_max, max_relax)
    out = np.zeros_like(p)
    relax = np.zeros((n, W, 2), np.int32)
    status = np.zeros(n, np.int32)
    _check(_lib.ik_replan_many(g, ctypes.byref(arm.c), _np_ptr(_i32(root)), _np_ptr(p),
                               _np_ptr(_i32(current)), n, ctypes.byref(pp), _np_ptr(out),
                               _np_ptr(relax), _np_ptr(status), 0), "ik_replan_many")
    return out, relax, status


def ik_replan_many_device(g: int, arm, root, poses, current, poses_out, relax_out, status_out,
                          delta: int = 3, eps2: int = 2, eps2_max: int = 8,
                          max_relax: int = -1) -> None:
    """Device form: every array is a contiguous int32 CUDA tensor."""
    arm = _arm(arm)
    pp = path_params(poses.shape[1], delta, eps2, eps2_max, max_relax)
    _check(_lib.ik_replan_many(g, ctypes.byref(arm.c), _np_ptr(_i32(root)), _dev_ptr(poses),
                               _dev_ptr(current), poses.shape[0], ctypes.byref(pp),
                               _dev_ptr(poses_out), _dev_ptr(relax_out), _dev_ptr(status_out), 1),
           "ik_replan_many")


def ik_shell_offsets(length: int, tol: float = 0.5) -> Tuple[Tuple[int, int], np.ndarray]:
    b = np.zeros(2, np.int32)
    n = _lib.ik_shell_offsets(length, tol, _np_ptr(b), None, 0)
    if n < 0:
        raise IkError(n, "ik_shell_offsets")
    out = np.zeros((max(n, 1), 3), np.int32)
    _lib.ik_shell_offsets(length, tol, _np_ptr(b), _np_ptr(out), n)
    return (int(b[0]), int(b[1])), out[:n]


def ik_row_table(length: int, tol: float = 0.5):
    """The row-lane propagation's table of one shell: (R, offsets [n][3] in
    device order, tabr [n], rowsr [(2R+1) * 2 * (2R+2)])."""
    R = np.zeros(1, np.int32)
    n = _lib.ik_row_table(length, tol, _np_ptr(R), None, None, 0, None, 0)
    if n < 0:
        raise IkError(n, "ik_row_table")
    r = int(R[0])
    offs = np.zeros((max(n, 1), 3), np.int32)
    tabr = np.zeros(max(n, 1), np.int32)
    rowsr = np.zeros((2 * r + 1) * 2 * (2 * r + 2), np.int32)
    _lib.ik_row_table(length, tol, _np_ptr(R), _np_ptr(offs), _np_ptr(tabr), n, _np_ptr(rowsr), len(rowsr))
    return r, offs[:n], tabr[:n], rowsr


def ik_row_mask_table(length: int, tol: float = 0.5):
    """The row-lane edge masks' supercover table of one shell:
    (sc_start [n + 1], sctabr [m]), offsets in ik_row_table's device order."""
    m = _lib.ik_row_mask_table(length, tol, None, 0, None, 0)
    if m < 0:
        raise IkError(m, "ik_row_mask_table")
    n = len(ik_row_table(length, tol)[1])
    start = np.zeros(n + 1, np.int32)
    tab = np.zeros(max(m, 1), np.int32)
    _lib.ik_row_mask_table(length, tol, _np_ptr(start), n + 1, _np_ptr(tab), m)
    return start, tab[:m]


def ik_supercover_offsets(d) -> np.ndarray:
    d = _i32(d)
    cap = int(np.prod(np.abs(d) + 1)) + 8
    out = np.zeros((cap, 3), np.int32)
    n = _lib.ik_supercover_offsets(_np_ptr(d), _np_ptr(out), cap)
    if n < 0:
        raise IkError(n, "ik_supercover_offsets")
    return out[:n]


class Grid:
    """Owning wrapper of an ``ik_grid`` handle."""

    def __init__(self, nx: int, ny: int, nz: int, stream: int = 0):
        self.shape = (nx, ny, nz)
        self.h = ik_create_grid(nx, ny, nz, stream)

    def close(self) -> None:
        if self.h:
            ik_destroy_grid(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
