"""Continuous-batching IK server with moving obstacles (section "Dynamic
Obstacles": replan the remainder of a path mid-traversal).

One device-resident grid serves two request kinds:

* ``path``: reach pose + smooth path to a target;
* ``replan``: the remainder of a live path, from the waypoint the arm has
  reached, under the current obstacles.

Time advances in ticks.  At each tick the moving boxes advance one step and
the occupancy snapshot of the tick is built on the GPU; the requests that
have arrived are admitted into the free slots of the tick's batch (a fixed
number of reach+path slots and of replan slots, sized by a device-memory
budget); one captured CUDA graph rebuilds the snapshot (occupancy, edge
masks, forward sets) and solves every admitted path slot, and the admitted
replans run right after it on the same stream, batched.  For the rest of
the tick the server keeps admitting: whenever requests have arrived and
the GPU is free, they are solved as one more batch against the SAME
snapshot (the grid keeps the tick's edge masks and forward sets, so such a
batch only propagates, traces and chains), until the tick ends.  A
request's result depends only on its input and on the snapshot of the tick
that admitted it (stamped on the request), so it is the same whether it is
served alone or in a mix, at a tick's start or within it.

A path request becomes a live path when it completes; the arm is taken to
advance one waypoint per tick along it.  A replan request names a live path
and replans it from the waypoint the arm has reached.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import ik


@dataclass
class Request:
    rid: int
    kind: str                      # "path" or "replan"
    arrival: float                 # seconds on the server clock
    target: Optional[Tuple[int, int, int]] = None   # path requests
    path_id: Optional[int] = None  # replan requests: the live path to replan
    tick: int = -1                 # tick that admitted it (its snapshot)
    done: float = -1.0             # completion time on the server clock
    current: int = -1              # replan: the waypoint the arm had reached
    status: int = -1
    poses: Optional[np.ndarray] = None
    relax: Optional[np.ndarray] = None
    input_poses: Optional[np.ndarray] = None  # replan: the live path it was given


@dataclass
class LivePath:
    poses: np.ndarray
    start_tick: int


class Server:
    """Tick-synchronous continuous batching on one grid and one CUDA stream.

    ``static_boxes`` int32 [n][6]; ``moving`` a ``scenegen.MovingBoxes``
    (advanced in place, one step per tick); ``slots_path`` / ``slots_replan``
    default to what ``mem_budget`` bytes of survivor sets allow.
    ``edge_masks`` False serves from a grid that keeps no per-offset edge
    masks (segment tests walk supercovers against the tick's occupancy):
    on large grids the masks of every tick would cost more than the tick.
    """

    def __init__(self, shape, root, lengths, static_boxes, moving, n_way: int = 32,
                 delta: int = 3, tick_s: float = 3.0 / 36.0, slots_path: Optional[int] = None,
                 slots_replan: Optional[int] = None, mem_budget: float = 24e9, device: int = 0,
                 edge_masks: bool = True):
        import torch
        self.torch = torch
        torch.cuda.set_device(device)
        self.shape = tuple(shape)
        self.root = tuple(int(v) for v in root)
        self.lengths = tuple(int(v) for v in lengths)
        self.S = len(self.lengths)
        self.W = n_way
        self.delta = delta
        self.tick_s = tick_s
        self.static = np.asarray(static_boxes, np.int32).reshape(-1, 6)
        self.moving = moving
        nx, ny, nz = self.shape
        words = nx // 32 * ny * nz
        # survivor sets of one slot's waypoints dominate a slot's memory
        per_slot = self.W * (self.S + 1) * words * 4
        cap = max(1, int(mem_budget // (2 * per_slot)))
        self.slots_path = slots_path or min(64, cap)
        self.slots_replan = slots_replan or min(64, cap)
        self.stream = torch.cuda.Stream(device=device)
        self.grid = ik.Grid(nx, ny, nz, stream=self.stream.cuda_stream)
        if not edge_masks:
            ik.ik_set_option(self.grid.h, ik.IK_OPT_EDGE_MASKS, 0)
        self.arm = ik.Arm(self.lengths)
        dev = torch.device("cuda", device)
        i32 = dict(dtype=torch.int32, device=dev)
        S, W, P, R = self.S, self.W, self.slots_path, self.slots_replan
        self.boxes_d = torch.from_numpy(self._boxes()).to(dev)
        self.targets_d = torch.full((P, 3), -1, **i32)
        self.reach_d = torch.zeros((P, S + 1, 3), **i32)
        self.found_d = torch.zeros(P, **i32)
        self.poses_d = torch.zeros((P, W, S + 1, 3), **i32)
        self.relax_d = torch.zeros((P, W, 2), **i32)
        self.status_d = torch.zeros(P, **i32)
        self.batch = ik.Batch(self.grid.h, self.arm, self.root, self.boxes_d, self.targets_d, W,
                              self.reach_d, self.found_d, self.poses_d, self.relax_d, self.status_d,
                              delta=delta)
        self.rp_in_d = torch.zeros((R, W, S + 1, 3), **i32)
        self.rp_cur_d = torch.full((R,), -1, **i32)
        self.rp_out_d = torch.zeros((R, W, S + 1, 3), **i32)
        self.rp_relax_d = torch.zeros((R, W, 2), **i32)
        self.rp_status_d = torch.zeros(R, **i32)
        self.tick = 0
        self.live: Dict[int, LivePath] = {}
        self.dead = set()
        self.pending: List[Request] = []
        self.finished: List[Request] = []
        self.tick_ms: List[float] = []    # GPU work of each tick's start (snapshot + admitted)
        self.within_ms: List[float] = []  # GPU work of each batch admitted within a tick

    def _boxes(self) -> np.ndarray:
        return np.concatenate([self.static, self.moving.boxes()]).astype(np.int32)

    # ------------------------------------------------------------------ ticks

    def _admit(self, now: float):
        """The requests that have arrived by `now` and fit the slots."""
        admitted_p = [r for r in self.pending if r.kind == "path" and r.arrival <= now]
        admitted_p = admitted_p[: self.slots_path]
        admitted_r = [r for r in self.pending if r.kind == "replan" and r.arrival <= now
                      and r.path_id in self.live]
        admitted_r = admitted_r[: self.slots_replan]
        # replans of paths that ended without a reach pose have nothing to do
        dropped = [r for r in self.pending if r.kind == "replan" and r.path_id in self.dead
                   and r.arrival <= now]
        for r in dropped:
            r.status, r.done, r.tick = ik.IK_PATH_UNREACHABLE, now, self.tick
        taken = {id(r) for r in admitted_p + admitted_r + dropped}
        self.pending = [r for r in self.pending if id(r) not in taken]
        return admitted_p, admitted_r

    def run_tick(self, now: float) -> List[Request]:
        """Advance the obstacles, admit what has arrived, solve; returns the
        requests finished at the tick's start."""
        self.moving.step()
        self.tick += 1
        admitted_p, admitted_r = self._admit(now)
        return self._solve(now, admitted_p, admitted_r, snapshot=True)

    def run_within_tick(self, now: float) -> List[Request]:
        """Solve what has arrived by `now` against the current tick's
        snapshot (no rebuild); returns the finished requests (none when
        nothing has arrived)."""
        admitted_p, admitted_r = self._admit(now)
        if not admitted_p and not admitted_r:
            return []
        return self._solve(now, admitted_p, admitted_r, snapshot=False)

    def _solve(self, now: float, admitted_p, admitted_r, snapshot: bool) -> List[Request]:
        torch = self.torch
        t0 = time.perf_counter()
        with torch.cuda.stream(self.stream):
            self.boxes_d.copy_(torch.from_numpy(self._boxes()), non_blocking=False)
            tg = np.full((self.slots_path, 3), -1, np.int32)
            for i, r in enumerate(admitted_p):
                tg[i] = r.target
                r.tick = self.tick
            self.targets_d.copy_(torch.from_numpy(tg))
            pin = np.zeros((self.slots_replan, self.W, self.S + 1, 3), np.int32)
            cur = np.full(self.slots_replan, -1, np.int32)
            for i, r in enumerate(admitted_r):
                lp = self.live[r.path_id]
                r.current = min(self.W - 1, self.tick - lp.start_tick)
                r.tick = self.tick
                pin[i] = lp.poses
                cur[i] = r.current
                r.input_poses = lp.poses.copy()
            self.rp_in_d.copy_(torch.from_numpy(pin))
            self.rp_cur_d.copy_(torch.from_numpy(cur))
        if snapshot:
            # snapshot + path slots (one graph), then the replan slots
            self.batch.launch()
        elif admitted_p:
            # the tick's snapshot stays: only the admitted paths are solved
            n = len(admitted_p)
            ik.ik_reach_path_many_device(self.grid.h, self.arm, self.root, self.targets_d[:n], self.W,
                                         self.reach_d[:n], self.found_d[:n], self.poses_d[:n],
                                         self.relax_d[:n], self.status_d[:n], delta=self.delta)
        if admitted_r:
            ik.ik_replan_many_device(self.grid.h, self.arm, self.root, self.rp_in_d, self.rp_cur_d,
                                     self.rp_out_d, self.rp_relax_d, self.rp_status_d,
                                     delta=self.delta)
        self.stream.synchronize()
        (self.tick_ms if snapshot else self.within_ms).append((time.perf_counter() - t0) * 1000.0)
        done_t = now + (time.perf_counter() - t0)
        out = []
        if admitted_p:
            poses = self.poses_d.cpu().numpy()
            relax = self.relax_d.cpu().numpy()
            status = self.status_d.cpu().numpy()
            for i, r in enumerate(admitted_p):
                r.poses, r.relax, r.status = poses[i], relax[i], int(status[i])
                r.done = done_t
                if r.status != ik.IK_PATH_UNREACHABLE:
                    self.live[r.rid] = LivePath(poses[i].copy(), self.tick)
                else:
                    self.dead.add(r.rid)
                out.append(r)
        if admitted_r:
            poses = self.rp_out_d.cpu().numpy()
            relax = self.rp_relax_d.cpu().numpy()
            status = self.rp_status_d.cpu().numpy()
            for i, r in enumerate(admitted_r):
                r.poses, r.relax, r.status = poses[i], relax[i], int(status[i])
                r.done = done_t
                if r.status in (ik.IK_PATH_OK, ik.IK_PATH_RELAXED, ik.IK_PATH_BROKEN):
                    self.live[r.path_id].poses = poses[i].copy()
                out.append(r)
        self.finished.extend(out)
        return out

    def serve(self, requests: List[Request], duration: float, realtime: bool = True,
              within: bool = True) -> None:
        """Run ticks for ``duration`` seconds of server clock, admitting
        requests within each tick as they arrive (``within``; else only at
        tick starts).  With ``realtime`` the clock is the wall clock (a tick
        waits for its start time, and within it the server waits for the
        next arrival or the GPU); otherwise the clock is simulated: ticks
        follow each other back to back and, within a tick, each arrival is
        admitted at its own arrival time (deterministic admission)."""
        self.pending.extend(sorted(requests, key=lambda r: r.arrival))
        start = time.perf_counter()
        k = 0
        while True:
            t_tick = k * self.tick_s
            if t_tick > duration:
                break
            t_end = t_tick + self.tick_s
            if realtime:
                wait = start + t_tick - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                now = max(t_tick, time.perf_counter() - start)
            else:
                now = t_tick
            self.run_tick(now)
            while within:
                if realtime:
                    now = time.perf_counter() - start
                if now >= t_end:
                    break
                if self.run_within_tick(now):
                    continue
                # nothing admissible now: wait for the next arrival (or the tick's end)
                nxt = min((r.arrival for r in self.pending if r.arrival > now), default=None)
                if realtime:
                    time.sleep(max(0.0, min(t_end if nxt is None else nxt, t_end) - now))
                elif nxt is None or nxt >= t_end:
                    break
                else:
                    now = nxt
            k += 1

    def close(self) -> None:
        self.batch.close()
        self.grid.close()


def make_requests(scene, rate_hz: float, duration: float, seed: int) -> List[Request]:
    """Poisson arrivals, half reach+path (a target drawn uniformly over free
    voxels within reach) and half replans of an earlier path request
    (uniform over the path requests issued before it)."""
    import scenegen as G
    times = G.poisson_arrivals(rate_hz, duration, seed)
    kinds = G.request_kinds(len(times), seed)
    targets = G.draw_targets(scene, int((kinds == 0).sum()) + 1, seed)
    rng = G.SplitMix64(seed, 6)
    out, paths, ti = [], [], 0
    for i, (t, k) in enumerate(zip(times, kinds)):
        if k == 0 or not paths:
            out.append(Request(i, "path", float(t), target=tuple(int(v) for v in targets[ti])))
            ti += 1
            paths.append(i)
        else:
            out.append(Request(i, "replan", float(t), path_id=paths[rng.below(len(paths))]))
    return out


def latency_stats(reqs: List[Request]) -> dict:
    lat = np.asarray([(r.done - r.arrival) * 1000.0 for r in reqs if r.done >= 0])
    if len(lat) == 0:
        return {"n": 0}
    return {"n": int(len(lat)), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3)}
