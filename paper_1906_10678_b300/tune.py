"""Autotuner for the propagation and edge-mask tiling.

For a grid shape and an arm it times one full reach + path batch with each
candidate configuration and keeps the fastest: the tile depth (8 or 16
output slices per block, IK_OPT_TILE_DEPTH), with depth 8 one or two
queries per block on the dense levels (IK_OPT_QUERY_PAIRS) and the row-lane
kernel on or off (IK_OPT_ROW_LANES), and the edge-mask
brick staged by per-thread loads or by a TMA tensor copy (IK_OPT_TMA_MASKS,
on grids whose rows allow it).  Choices are cached in a JSON file (by
default ``build/ik_tuning.json`` next to the package) keyed by the grid
extents, the segment lengths and the batch shape, so a later process reuses
them without measuring.  The results of every candidate are identical; only
the time differs.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Sequence

from . import ik

# (tile depth, query pairs: 0 one, 1 two with padded rows, 2 two with unpadded
# rows, row lanes); depth 16 has its own kernel, which takes one query; with
# row lanes on, pairs 1 and 2 are the same kernel
CANDIDATES = ((8, 1, 1), (8, 0, 1), (8, 1, 0), (8, 2, 0), (8, 0, 0), (16, 0, 0))
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "build",
                             "ik_tuning.json")


def _key(shape, lengths, n_targets: int, n_way: int) -> str:
    return "x".join(str(v) for v in shape) + "|" + ",".join(str(v) for v in lengths) + \
        f"|{n_targets}|{n_way}|v3"


def load(path: str = DEFAULT_CACHE) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _apply(grid_h: int, cfg: dict) -> None:
    ik.ik_set_option(grid_h, ik.IK_OPT_TILE_DEPTH, int(cfg["depth"]))
    ik.ik_set_option(grid_h, ik.IK_OPT_QUERY_PAIRS, int(cfg["pairs"]))
    ik.ik_set_option(grid_h, ik.IK_OPT_TMA_MASKS, int(cfg["tma"]))
    ik.ik_set_option(grid_h, ik.IK_OPT_ROW_LANES, int(cfg.get("rows", 0)))


def tiling(grid_h: int, stream, shape, lengths: Sequence[int], root, boxes_d, targets_d, n_way: int,
           outs, delta: int = 3, path: str = DEFAULT_CACHE, repeats: int = 2) -> dict:
    """Best tiling for this workload (measured once, then cached).

    ``outs`` = (reach, found, poses, relax, status) CUDA tensors sized for
    ``targets_d``; ``stream`` the torch stream of the grid.  Leaves the
    grid set to the chosen configuration and returns {"depth", "pairs",
    "tma", "ms": {candidate: ms}}.
    """
    import torch
    cache = load(path)
    key = _key(shape, lengths, int(targets_d.shape[0]), n_way)
    if key in cache:
        _apply(grid_h, cache[key])
        return dict(cache[key], cached=True)
    arm = ik.Arm(lengths)
    tma_ok = (int(shape[0]) // 32 * 4) % 16 == 0
    cands = [dict(depth=d, pairs=p, rows=r, tma=t) for d, p, r in CANDIDATES
             for t in ((0, 1) if tma_ok else (0,))]
    times = {}
    for cfg in cands:
        _apply(grid_h, cfg)
        name = f"depth{cfg['depth']}_pairs{cfg['pairs']}_rows{cfg['rows']}_tma{cfg['tma']}"

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
        times[name] = e0.elapsed_time(e1) / repeats
    best = min(cands, key=lambda c: times[f"depth{c['depth']}_pairs{c['pairs']}_rows{c['rows']}_tma{c['tma']}"])
    _apply(grid_h, best)
    cache[key] = dict(best, ms=times)
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return dict(cache[key], cached=False)
