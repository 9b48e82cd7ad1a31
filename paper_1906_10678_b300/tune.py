"""Autotuner for the propagation tiling.

For a grid shape and an arm it times one full reach + path batch with each
candidate tile depth (8 or 16 output slices per block; see
IK_OPT_TILE_DEPTH) and keeps the faster one.  Choices are cached in a JSON
file (by default ``build/ik_tuning.json`` next to the package) keyed by the
grid extents, the segment lengths and the batch shape, so a later process
reuses them without measuring.  The results of every candidate are
identical; only the time differs.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Sequence

from . import ik

CANDIDATES = (8, 16)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "build",
                             "ik_tuning.json")


def _key(shape, lengths, n_targets: int, n_way: int) -> str:
    return "x".join(str(v) for v in shape) + "|" + ",".join(str(v) for v in lengths) + \
        f"|{n_targets}|{n_way}"


def load(path: str = DEFAULT_CACHE) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tile_depth(grid_h: int, stream, shape, lengths: Sequence[int], root, boxes_d, targets_d, n_way: int,
               outs, delta: int = 3, path: str = DEFAULT_CACHE, repeats: int = 2) -> dict:
    """Best tile depth for this workload (measured once, then cached).

    ``outs`` = (reach, found, poses, relax, status) CUDA tensors sized for
    ``targets_d``; ``stream`` the torch stream of the grid.  Leaves the
    grid set to the chosen depth and returns {"depth", "ms": {...}}.
    """
    import torch
    cache = load(path)
    key = _key(shape, lengths, int(targets_d.shape[0]), n_way)
    if key in cache:
        ik.ik_set_option(grid_h, ik.IK_OPT_TILE_DEPTH, cache[key]["depth"])
        return dict(cache[key], cached=True)
    arm = ik.Arm(lengths)
    times = {}
    for depth in CANDIDATES:
        ik.ik_set_option(grid_h, ik.IK_OPT_TILE_DEPTH, depth)
        def step():
            ik.ik_set_boxes(grid_h, boxes_d)
            ik.ik_reach_path_many_device(grid_h, arm, root, targets_d, n_way, *outs, delta=delta)
        step()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(repeats):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        times[str(depth)] = e0.elapsed_time(e1) / repeats
    best = min(CANDIDATES, key=lambda d: times[str(d)])
    ik.ik_set_option(grid_h, ik.IK_OPT_TILE_DEPTH, best)
    cache[key] = {"depth": best, "ms": times}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return dict(cache[key], cached=False)
