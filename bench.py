"""Benchmark: reach + path solves/s on the 128^3, 8-segment workload.

One step = one pass of the whole hot path over one batch: rasterise the
scene's 200 boxes, rebuild the edge masks and forward sets for that
occupancy, solve the reach pose of 64 targets, then the 32-waypoint smooth
path of each (guide points, survivor sets of all 64 x 32 waypoints in one
batched backward pass per segment, one smooth-chain block per path).  The
batched form is the product path (``ik_reach_path_many``); the plain form
(one ``ik_solve_reach`` + ``ik_plan_path`` call per target) is reported
beside it, and so are midcourse replan latencies.

Run: ``python bench.py [--gpus N] [--steps K] [--warmup W]``; under torchrun
each rank solves its own batch (weak scaling, replicas only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reach+path solves/s & replan p50/p99 ms (128^3, 8 seg), batched vs plain, 1 B300"
UNIT = "solves/s"
N_TARGETS = 64
N_WAY = 32
DELTA = 3


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ------------------------------------------- replicas (one process per GPU)

def rank_targets(sc, n: int, rank: int):
    """Each rank solves its own seeded batch of n targets: queries are
    independent given the replicated grid, so no data moves between ranks."""
    import scenegen as G
    return G.draw_targets(sc, n, 1 + 1000 * rank)


def max_over_ranks(ms: float, dist, device) -> float:
    """The job's time: the slowest rank's (a no-op for one rank)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_targets: int, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank's targets over the slowest rank's step."""
    return n_targets * world / (ms_per_step / 1000.0)


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# Algorithmic work per non-zero (offset, output word) pair of a propagation
# (the method's word-op count with the supercover terms paid by the
# edge-mask kernel): one AND with the edge-mask word and one OR into the
# output word;
# and two words read: the shifted source word (staged in shared memory) and
# the edge-mask word.
OPS_PER_PAIR = 2
WORDS_PER_PAIR = 2


def probe_peaks(ik, stream) -> dict:
    """The library's own throughput probes (ik_probe_peak), best of three:
    3-input logic ops (the integer roofline) and conflict-free 32-bit
    shared-memory word loads (the bitset-traffic roofline), with the SM clock
    each probe saw."""
    out = {}
    for kind, name, bps in ((ik.PROBE_LOP3, "lop3", 8), (ik.PROBE_SHF, "shf", 8), (ik.PROBE_LDS, "lds", 4)):
        ik.ik_probe_peak(kind, bps, 2000, stream)
        best = max((ik.ik_probe_peak(kind, bps, 20000, stream) for _ in range(3)),
                   key=lambda r: r["ops_per_s"])
        out[name] = {"per_s": best["ops_per_s"], "sm_mhz": best["sm_mhz"]}
    return out


# DRAM bytes (read + write) per launch of the waypoint pass on this workload
# from one ncu capture of bench.py (profiles/dram_waypoint_pass_128.md), with
# the SHA-256 of the kernel and tiling sources it was taken on: reported only
# while those sources are unchanged.
TRAFFIC_CAPTURE = {"bytes_per_launch": 650030880,
                   "kernels_sha256": "c88286751ef1fb5fcc92493274501e8e05088db7dc341ac16ba5f23d77ec9dab"}


def kernel_sources_sha256() -> str:
    h = hashlib.sha256()
    for name in ("ik_kernels.cu", "ik_tables.cpp"):
        with open(os.path.join(ROOT, "paper_1906_10678_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_traffic():
    sha = kernel_sources_sha256()
    return TRAFFIC_CAPTURE["bytes_per_launch"] if sha == TRAFFIC_CAPTURE["kernels_sha256"] else None


def _kernel_roof(name, ms, launches, ops, words, peaks, clk_mhz):
    """Fractions of one kernel class against the probed peaks, scaled to the
    SM clock sampled during the timed region."""
    def at_clk(p):
        return p["per_s"] * (clk_mhz / p["sm_mhz"]) if clk_mhz and p["sm_mhz"] else p["per_s"]
    int_peak = at_clk(peaks["lop3"]) / 1e12
    lds_peak = at_clk(peaks["lds"]) / 1e12
    launches = max(1, launches)
    t = ms / launches / 1000.0
    ach_ops = ops / launches / t / 1e12 if t > 0 else 0.0
    ach_words = words / launches / t / 1e12 if t > 0 else 0.0
    return {"kernel": name, "ms_per_launch": round(ms / launches, 4), "launches": launches,
            "alg_ops_per_launch": round(ops / launches), "alg_words_per_launch": round(words / launches),
            "int": {"achieved": round(ach_ops, 4), "peak": round(int_peak, 3), "unit": "Tops/s",
                    "frac": round(ach_ops / int_peak, 5)},
            "bitset_traffic": {"achieved": round(ach_words, 4), "peak": round(lds_peak, 3),
                               "unit": "Twords/s", "frac": round(ach_words / lds_peak, 5)}}


def roofline(prof, work, peaks, clk):
    """Rooflines per kernel class (every class above 1 % of the step), and
    the line's roofline object for the dominant one (the batched backward
    propagation of the waypoint pass).

    The work is boolean and on-chip: its rooflines are the integer issue
    rate (3-input logic ops) and the shared-memory word-load rate, both
    measured by the library's probes, not HBM (the pass moves well under
    2 % of HBM bandwidth).  Algorithmic work per launch: for a propagation,
    2 word-ops and 2 word loads per non-zero (offset, output word) pair that
    the kernel's counters record on an identical step; for the edge masks,
    one OR and one word load per supercover voxel term (|SC(e)| per (offset,
    word) pair); for the smooth chain, as for a propagation, its restricted
    propagations' non-zero pairs.  The binding roofline is the one with the
    larger fraction.
    """
    clk_mhz = clk.get("sm_mhz")
    total = sum(v["ms"] for k, v in prof.items() if not k.startswith("way_k"))
    per = {}
    for cls in ("propagate_backward_waypoints", "propagate_forward", "propagate_backward_reach",
                "edge_masks", "smooth_chain"):
        p = prof.get(cls)
        if not p or not p["launches"] or p["ms"] < 0.01 * total:
            continue
        if cls == "propagate_backward_waypoints":
            w = {f: sum(v[f] for k, v in work.items() if k.startswith("way_k"))
                 for f in ("visited", "nonzero", "mask_words")}
        else:
            w = work[cls]
        if cls == "edge_masks":
            ops, words = w["nonzero"], w["nonzero"]  # supercover terms (one OR, one word each)
        else:
            ops, words = OPS_PER_PAIR * w["nonzero"], WORDS_PER_PAIR * w["nonzero"]
        r = _kernel_roof(cls, p["ms"], p["launches"], ops, words, peaks, clk_mhz)
        r["share_of_step"] = round(p["ms"] / total, 4)
        if cls.startswith("propagate"):
            r["pairs_visited"], r["pairs_nonzero"] = w["visited"], w["nonzero"]
            r["mask_words_read"] = w["mask_words"]
        elif cls == "edge_masks":
            r["pairs"], r["supercover_terms"] = w["visited"], w["nonzero"]
        else:
            r["pairs_visited"], r["pairs_nonzero"] = w["visited"], w["nonzero"]
        per[cls] = r
    top = per["propagate_backward_waypoints"]
    binding = "bitset_traffic" if top["bitset_traffic"]["frac"] >= top["int"]["frac"] else "int"
    return {"kernel": "k_propagate_rows + k_propagate_tile_list (propagate_backward_waypoints)", "bound": "alu",
            "achieved": top["int"]["achieved"], "peak": top["int"]["peak"], "unit": "Tops/s",
            "frac": top["int"]["frac"], "traffic": kernel_traffic(),
            "bitset_traffic": top["bitset_traffic"], "binding": binding,
            "alg_ops_per_launch": top["alg_ops_per_launch"], "ms_per_launch": top["ms_per_launch"],
            "pairs_visited": top["pairs_visited"], "pairs_nonzero": top["pairs_nonzero"],
            "peak_source": "ik_probe_peak (lop3.b32 / ld.shared.b32 throughput probes, best of 3, "
                           "run in this process), scaled to the SM clock sampled in the timed region",
            "peaks_measured": {k: {"per_s": round(v["per_s"] / 1e12, 3), "unit": "T/s",
                                   "sm_mhz": round(v["sm_mhz"], 1)} for k, v in peaks.items()},
            "sm_mhz_under_load": clk_mhz, "per_kernel": per}


def oracle_sample(threads: int):
    """CPU oracle, as it stands, on a bounded sample of the workload.

    The oracle's unit of work for this workload is one backward pass: the
    unmasked backward sets from a target (its reach IK) or from a waypoint
    target (each waypoint IK); a reach + 32-waypoint path needs 32 of them
    plus the forward sets once per 64-target batch.  The sample runs
    ``threads`` such passes from ``threads`` seeded target voxels, one per
    host thread, and scales: solves/s = passes/s / 32.
    """
    from concurrent.futures import ThreadPoolExecutor

    import oracle as O
    import scenegen as G

    sc = workload()
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, threads, 77)
    O.shell_bounds(1)  # load the library before timing

    def one(t):
        T = np.zeros(occ.shape, np.uint8)
        T[t[2], t[1], t[0]] = 1
        O.backward(occ, sc.lengths, T)

    a = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(one, targets))
    wall = time.perf_counter() - a
    passes_per_s = threads / wall
    return passes_per_s / 32.0, wall


def physical_cores() -> int:
    try:
        import psutil
        return psutil.cpu_count(logical=False) or os.cpu_count() or 1
    except ImportError:
        return os.cpu_count() or 1


LOWER_BOUND_NOTE = ("a lower bound on the oracle's cost (an upper bound on its solves/s): per "
                    "reach+path only its 32 backward passes are counted, not the forward sets "
                    "(shared by a batch) nor the smooth steps")


def cpu_baseline():
    """The oracle on all host threads, and single-threaded (the canonical
    figure): each thread runs one backward pass of the 128^3 scene."""
    cores = os.cpu_count() or 1
    value, wall = oracle_sample(cores)
    one, wall1 = oracle_sample(1)
    return {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} unmasked backward passes (one per host thread) from seeded "
                      f"target voxels of the 128^3 scene, {wall:.1f} s wall; solves/s = passes/s "
                      f"/ 32 (1 reach + 31 waypoint passes per reach+path)",
            "single_thread": {"value": round(one, 6), "unit": UNIT, "cores": 1,
                              "sample": f"1 backward pass, {wall1:.1f} s"},
            "note": LOWER_BOUND_NOTE}


def bench_config(world: int) -> dict:
    """The workload of the bench line (both arms)."""
    return {"workload": "C3: 128^3 grid, 200 boxes (seed 1), arm {20,18,16,14,12,10,8,6}, "
                        "64 targets, reach + 32-waypoint path, delta 3",
            "global_batch": N_TARGETS * world, "n_way": N_WAY,
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (edge masks ~1.7 GB rebuilt every step)"}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    # one oracle backward pass at 128^3 takes tens of seconds of CPU: a step
    # runs one pass per physical core in parallel (the hyperthreads add
    # little to the oracle's throughput and double each step's wall time)
    per_step = physical_cores()
    # warm-up steps: load and touch the oracle library (no oracle state to warm)
    import oracle as O
    for _ in range(args.warmup):
        O.shell_bounds(1)
    vals, walls = [], []
    for _ in range(args.steps):
        v, wall = oracle_sample(per_step)
        vals.append(v)
        walls.append(wall)
    value = float(np.mean(vals))
    ms = float(np.mean(walls)) * 1000.0
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": bench_config(world),
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": per_step, "kind": "oracle",
                         "sample": f"per step {per_step} unmasked backward passes of the 128^3 scene "
                                   f"(one per physical core; {cores} logical CPUs on the host); "
                                   f"solves/s = passes/s / 32",
                         "note": LOWER_BOUND_NOTE},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def workload(grid: int = 128):
    import scenegen as G
    if grid == 128:
        return G.c2_scene(1)
    # smaller grid of the same construction, for profiler captures only
    return G.scaled_scene(grid, G.C2_LENGTHS, max(1, 200 * grid ** 3 // 128 ** 3), 4, 24, 1,
                          f"C2@{grid}")


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1906_10678_b300 import ik
    import scenegen as G

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    global N_TARGETS
    N_TARGETS = args.targets
    sc = workload(args.grid)
    # each rank solves its own batch of targets (replicas, no collective)
    targets_np = rank_targets(sc, N_TARGETS, rank)
    S = len(sc.lengths)
    stream = torch.cuda.Stream(device=dev)
    g = ik.Grid(*sc.shape, stream=stream.cuda_stream)
    arm = ik.Arm(sc.lengths)
    boxes_d = torch.from_numpy(sc.boxes.copy()).to(dev)
    targets_d = torch.from_numpy(targets_np.copy()).to(dev)
    reach = torch.zeros((N_TARGETS, S + 1, 3), dtype=torch.int32, device=dev)
    found = torch.zeros(N_TARGETS, dtype=torch.int32, device=dev)
    poses = torch.zeros((N_TARGETS, N_WAY, S + 1, 3), dtype=torch.int32, device=dev)
    relax = torch.zeros((N_TARGETS, N_WAY, 2), dtype=torch.int32, device=dev)
    status = torch.zeros(N_TARGETS, dtype=torch.int32, device=dev)

    def step():
        ik.ik_set_boxes(g.h, boxes_d)
        ik.ik_reach_path_many_device(g.h, arm, sc.root, targets_d, N_WAY, reach, found, poses,
                                     relax, status, delta=DELTA)

    # tile depth chosen by the autotuner (measured on this very step, cached),
    # or fixed by --tile-depth
    if args.tile_depth == "auto":
        from paper_1906_10678_b300 import tune
        tuning = tune.tiling(g.h, stream, sc.shape, sc.lengths, sc.root, boxes_d, targets_d, N_WAY,
                             (reach, found, poses, relax, status), delta=DELTA)
    else:
        ik.ik_set_option(g.h, ik.IK_OPT_TILE_DEPTH, int(args.tile_depth))
        tuning = {"depth": int(args.tile_depth), "fixed": True}

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    clk = clocks.stop()
    if world > 1:
        ms = max_over_ranks(ms, dist, dev)
        dist.barrier()
    ms_per_step = ms / args.steps
    value = job_value(N_TARGETS, world, ms_per_step)
    found_np = found.cpu().numpy()
    status_np = status.cpu().numpy()
    relax_np = relax.cpu().numpy()

    if args.no_extras:
        g.close()
        print(json.dumps({"ms_per_step": ms / args.steps, "grid": args.grid,
                          "targets": N_TARGETS}))
        return
    # end to end through the public API with host buffers
    reach_h = np.zeros((N_TARGETS, S + 1, 3), np.int32)
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        a = time.perf_counter()
        ik.ik_set_boxes(g.h, sc.boxes)
        out = ik.ik_reach_path_many(g.h, arm, sc.root, targets_np, N_WAY, delta=DELTA)
        e2e_ms.append((time.perf_counter() - a) * 1000.0)
    e2e_val = N_TARGETS / (np.median(e2e_ms) / 1000.0)
    h2d = sc.boxes.nbytes + targets_np.nbytes
    d2h = sum(x.nbytes for x in out)

    # the same batch on a grid that keeps no edge masks (segment tests walk
    # supercovers on the fly): identical results, different cost profile
    nomask_ms = None
    if not args.no_extras:
        with ik.Grid(*sc.shape, stream=stream.cuda_stream) as g2:
            ik.ik_set_option(g2.h, ik.IK_OPT_EDGE_MASKS, 0)
            def step2():
                ik.ik_set_boxes(g2.h, boxes_d)
                ik.ik_reach_path_many_device(g2.h, arm, sc.root, targets_d, N_WAY, reach, found,
                                             poses, relax, status, delta=DELTA)
            step2()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                step2()
            e1.record(stream)
            torch.cuda.synchronize()
            nomask_ms = e0.elapsed_time(e1) / 2

    # per-kernel times: one more step with the library's event profiler on
    # (events recorded on the grid's stream around each launch), then one
    # with its work counters on (slower; counts only)
    ik.ik_profile_enable(g.h, timing=True, counting=False)
    step()
    prof = ik.ik_profile_read(g.h)
    ik.ik_profile_enable(g.h, timing=False, counting=True)
    step()
    work = ik.ik_profile_read(g.h)
    ik.ik_profile_enable(g.h, timing=False, counting=False)
    peaks = probe_peaks(ik, stream.cuda_stream)

    # plain single-query form on a sample of targets
    plain_ms = []
    for i in range(min(8, N_TARGETS)):
        a = time.perf_counter()
        p, f, _ = ik.ik_solve_reach(g.h, arm, sc.root, targets_np[i])
        if f:
            ik.ik_plan_path(g.h, arm, p, N_WAY, delta=DELTA)
        plain_ms.append((time.perf_counter() - a) * 1000.0)

    # midcourse replans: 16 moving boxes (sides 6-16, 0.5-2 voxels per tick)
    # added to the static scene; each tick updates the occupancy once, then
    # every path with a reach pose is replanned from waypoint c = 8.  The
    # first request after an update also pays the edge-mask and forward-set
    # rebuild of the new occupancy.
    mv = G.make_moving_boxes(sc.shape, 16, 3)
    paths = out[2]
    rep_ms, rep_status = [], []
    for tick in range(args.replan_ticks):
        for _ in range(4):
            mv.step()
        ik.ik_set_boxes(g.h, np.concatenate([sc.boxes, mv.boxes()]))
        for i in range(N_TARGETS):
            if not out[1][i]:
                continue
            a = time.perf_counter()
            _, _, st = ik.ik_replan(g.h, arm, paths[i], 8, delta=DELTA)
            rep_ms.append((time.perf_counter() - a) * 1000.0)
            rep_status.append(st)
    # the same replans batched: one ik_replan_many call per tick for all live
    # paths (device buffers, decisions on the GPU), device-timed
    live = [i for i in range(N_TARGETS) if out[1][i]]
    mv2 = G.make_moving_boxes(sc.shape, 16, 3)
    rin = torch.from_numpy(np.ascontiguousarray(paths[live])).to(dev)
    rcur = torch.full((len(live),), 8, dtype=torch.int32, device=dev)
    rout = torch.zeros_like(rin)
    rrel = torch.zeros((len(live), N_WAY, 2), dtype=torch.int32, device=dev)
    rst = torch.zeros(len(live), dtype=torch.int32, device=dev)
    many_ms = []
    for tick in range(args.replan_ticks):
        for _ in range(4):
            mv2.step()
        ik.ik_set_boxes(g.h, np.concatenate([sc.boxes, mv2.boxes()]))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ik.ik_replan_many_device(g.h, arm, sc.root, rin, rcur, rout, rrel, rst, delta=DELTA)
        e1.record(stream)
        torch.cuda.synchronize()
        many_ms.append(e0.elapsed_time(e1))
    ik.ik_set_boxes(g.h, sc.boxes)
    rep_ms = np.asarray(rep_ms)
    rep_status = np.asarray(rep_status)
    cut = rep_status != ik.IK_PATH_KEPT

    # approach cone on the last segment: the same 64 targets approached from
    # above within 45 degrees (reach poses only; the occupancy, edge masks
    # and forward sets are rebuilt every step), beside the unrestricted reach
    cone_ = ik.cone((0, 0, -1), 1, 2)
    cposes = torch.zeros((N_TARGETS, S + 1, 3), dtype=torch.int32, device=dev)
    cfound = torch.zeros(N_TARGETS, dtype=torch.int32, device=dev)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def cone_step():
        ik.ik_set_boxes(g.h, boxes_d)
        ik.ik_solve_reach_many_cone_device(g.h, arm, cone_, sc.root, targets_d, cposes, cfound)

    def reach_step():
        ik.ik_set_boxes(g.h, boxes_d)
        ik.ik_solve_reach_many_device(g.h, arm, sc.root, targets_d, cposes, cfound)

    ms_reach = timed(reach_step)
    found_reach = int(cfound.sum().item())
    ms_cone = timed(cone_step)
    cone_res = {"value": round(N_TARGETS / (ms_cone / 1000.0), 2), "unit": "reach solves/s",
                "ms_per_batch": round(ms_cone, 3), "found": int(cfound.sum().item()),
                "no_cone": {"value": round(N_TARGETS / (ms_reach / 1000.0), 2),
                            "ms_per_batch": round(ms_reach, 3), "found": found_reach},
                "cone": "axis (0,0,-1), cos^2 = 1/2 (45 degrees)",
                "note": "64 targets of the 128^3 scene, reach pose only, occupancy rebuilt per batch"}

    # served form: continuous batching with moving obstacles, Poisson
    # arrivals at 200 req/s (half reach+path, half replans of live paths).
    # Default scene: 256^3, 300 static + 16 moving boxes; --serve-scene c3
    # serves the 128^3 scene.  Edge masks are rebuilt every tick over the
    # boxes the arm can reach (about 4 GB at 256^3); --serve-no-masks serves
    # from a grid that walks supercovers instead.
    served = None
    if args.serve_seconds > 0:
        from paper_1906_10678_b300 import serve as SV
        g.close()
        if args.serve_scene == "c5":
            ssc, smv = G.c5_scene(3)
        else:
            ssc, smv = sc, G.make_moving_boxes(sc.shape, 16, 3)
        masks = not args.serve_no_masks
        srv = SV.Server(ssc.shape, ssc.root, ssc.lengths, ssc.boxes, smv, n_way=N_WAY, delta=DELTA,
                        tick_s=3.0 / 36.0, slots_path=32, slots_replan=32, edge_masks=masks)
        reqs = SV.make_requests(ssc, 200.0, args.serve_seconds + args.serve_warmup, 3)
        srv.serve(reqs, args.serve_seconds + args.serve_warmup, realtime=True)
        keep = [r for r in srv.finished if r.arrival >= args.serve_warmup and r.poses is not None]
        tick = np.asarray(srv.tick_ms)
        served = {
            "scene": ("C5: 256^3, 300 static + 16 moving boxes (sides 6-16, 0.5-2 voxels/tick)"
                      if args.serve_scene == "c5" else "C3 scene (128^3) + 16 moving boxes"),
            "edge_masks": masks,
            "seconds": args.serve_seconds, "warmup_s": args.serve_warmup, "rate_hz": 200.0,
            "tick_ms": 1000.0 * srv.tick_s, "ticks": int(len(tick)),
            "tick_gpu_ms_p50": round(float(np.percentile(tick, 50)), 3),
            "tick_gpu_ms_p99": round(float(np.percentile(tick, 99)), 3),
            "within_tick_batches": int(len(srv.within_ms)),
            "within_gpu_ms_p50": round(float(np.percentile(srv.within_ms, 50)), 3) if srv.within_ms else None,
            "within_gpu_ms_p99": round(float(np.percentile(srv.within_ms, 99)), 3) if srv.within_ms else None,
            "path": SV.latency_stats([r for r in keep if r.kind == "path"]),
            "replan": SV.latency_stats([r for r in keep if r.kind == "replan"]),
            "path_solves_per_s": round(len([r for r in keep if r.kind == "path"]) / args.serve_seconds, 2),
            "pending_at_end": len(srv.pending),
            "note": "latency = completion - arrival on the wall clock; requests are admitted at tick "
                    "starts (snapshot rebuild + batch) and within ticks as they arrive (batches "
                    "against the tick's snapshot)"}
        srv.close()
        g = None

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": bench_config(world),
            "e2e": {"value": round(e2e_val, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "plain": {"value": round(1000.0 / float(np.mean(plain_ms)), 3), "unit": UNIT,
                      "ms_per_solve": round(float(np.mean(plain_ms)), 3), "sample": len(plain_ms)},
            "replan": None if len(rep_ms) == 0 else {
                       "p50_ms": round(float(np.percentile(rep_ms, 50)), 3),
                       "p99_ms": round(float(np.percentile(rep_ms, 99)), 3),
                       "cut_p50_ms": round(float(np.percentile(rep_ms[cut], 50)), 3) if cut.any() else None,
                       "cut_p99_ms": round(float(np.percentile(rep_ms[cut], 99)), 3) if cut.any() else None,
                       "requests": int(len(rep_ms)), "cut": int(cut.sum()),
                       "status_counts": {str(k): int((rep_status == k).sum()) for k in range(5)},
                       "note": "host wall time per ik_replan call (C ABI, host buffers)",
                       "batched": {"requests_per_call": len(live), "calls": len(many_ms),
                                   "ms_per_call_p50": round(float(np.percentile(many_ms, 50)), 3),
                                   "ms_per_call_max": round(float(np.max(many_ms)), 3),
                                   "note": "ik_replan_many over every live path after each occupancy "
                                           "update (the first request after an update also pays the "
                                           "edge-mask and forward-set rebuild), device-timed"}},
            "tuning": tuning,
            "cone_reach": cone_res,
            "served": served,
            "no_edge_masks": {"ms_per_step": round(nomask_ms, 3) if nomask_ms else None,
                              "value": round(N_TARGETS / (nomask_ms / 1000.0), 3) if nomask_ms else None,
                              "note": "same batch, supercovers walked on the fly (IK_OPT_EDGE_MASKS 0)"},
            "found": int(found_np.sum()),
            "path_status_counts": {str(k): int((status_np == k).sum()) for k in range(5)},
            "max_relax": int(relax_np[..., 0].max()),
            "clocks": clk,
            # the library's kernel launches in the timed region: the per-class
            # launch counts of the profiled step (identical to a timed step)
            "gpu_launches": int(args.steps * sum(v["launches"] for k, v in prof.items()
                                                 if not k.startswith("way_k"))),
            "kernels": {k: {"ms": round(v["ms"], 3), "launches": v["launches"]}
                        for k, v in prof.items() if v["launches"] and not k.startswith("way_k")},
            "waypoint_levels": {k: {"ms": round(prof[k]["ms"], 3), "warp_iters": work[k]["warp_iters"],
                                    "visited": work[k]["visited"], "nonzero": work[k]["nonzero"],
                                    "blocks": work[k]["blocks"], "live_words": work[k]["out_words"],
                                    "walk_warps": work[k]["walk_warps"], "walk_lanes": work[k]["walk_lanes"]}
                                for k in prof if k.startswith("way_k") and prof[k]["launches"]},
        }
        line["roofline"] = roofline(prof, work, peaks, clk)
        if world == 1 and args.c4_problems > 0:
            line["extra"] = {"c4": c4_measure(args.c4_problems)}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    if g is not None:
        g.close()
    if world > 1:
        dist.destroy_process_group()


def c4_measure(n_problems: int, reps: int = 2) -> dict:
    """The uneven batch (1024 independent reach + path problems, grids 64^3
    to 192^3, 5-9 segments of lengths 4-24, 50-400 boxes, 8-32 waypoints):
    ONE persistent launch per batch, captured as a CUDA graph
    (ik_batch_capture_uneven) and replayed on a stream, device-timed with
    CUDA events after one warm-up replay; the host-output form
    ik_solve_batch is timed end to end."""
    import torch
    import scenegen as G
    from paper_1906_10678_b300 import ik
    dev = torch.device("cuda", torch.cuda.current_device())
    a = time.perf_counter()
    probs = G.c4_problems(n_problems, 2)
    gen_s = time.perf_counter() - a
    dicts = [{"shape": p.scene.shape, "boxes": p.scene.boxes, "lengths": p.scene.lengths,
              "root": p.scene.root, "target": p.target, "n_way": p.n_way} for p in probs]
    n = len(dicts)
    r_n, p_n, x_n = ik.ik_batch_output_sizes(dicts)
    i32 = dict(dtype=torch.int32, device=dev)
    found, status, rc = (torch.zeros(n, **i32) for _ in range(3))
    reach, poses, relax = torch.zeros(r_n, **i32), torch.zeros(p_n, **i32), torch.zeros(x_n, **i32)
    stream = torch.cuda.Stream(device=dev)
    eng = ik.BatchEngine()
    # the batch captured once as a CUDA graph of one persistent launch, then
    # replayed (inputs resident on the device)
    graph = eng.capture(dicts, found, reach, poses, relax, status, rc)
    graph.launch(stream.cuda_stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        graph.launch(stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    rc_np = rc.cpu().numpy()
    st = status.cpu().numpy()
    graph.close()
    eng.close()
    a = time.perf_counter()
    out, _ = ik.ik_solve_batch(dicts)
    e2e_s = time.perf_counter() - a
    return {"value": round(n / (ms / 1000.0), 2), "unit": "solves/s", "ms_per_batch": round(ms, 1),
            "launches_per_batch": 1, "cuda_graph": True, "problems": n, "found": int(found.sum().item()),
            "jobs_ok": int((rc_np == ik.IK_OK).sum()),
            "status_counts": {str(k): int((st == k).sum()) for k in range(5)},
            "e2e": {"value": round(n / e2e_s, 2), "unit": "solves/s",
                    "note": "ik_solve_batch with host buffers (upload, launch, download)"},
            "generate_s": round(gen_s, 1),
            "config": "C4: 1024 uneven problems, grids {64,96,128,192}^3, 5-9 segments, lengths 4-24, "
                      "50-400 boxes, 8-32 waypoints (seed 2); supercovers walked on the fly"}


def run_uneven(args):
    """The uneven batch as its own line."""
    import torch
    torch.cuda.set_device(0)
    r = c4_measure(args.problems, reps=max(1, args.steps))
    print(json.dumps({"metric": "uneven batch reach+path solves/s (1 B300)", "n_gpus": 1, **r}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the batched step only (for profiler captures)")
    ap.add_argument("--grid", type=int, default=128,
                    help="grid edge; 128 is the benchmark workload, smaller only for captures")
    ap.add_argument("--targets", type=int, default=64)
    ap.add_argument("--replan-ticks", type=int, default=3)
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="served run after the warm-up (0 skips the served section)")
    ap.add_argument("--workload", default="c3", choices=["c3", "c4"])
    ap.add_argument("--problems", type=int, default=1024)
    ap.add_argument("--c4-problems", type=int, default=1024,
                    help="uneven-batch problems measured beside the main line (0: skip)")
    ap.add_argument("--serve-warmup", type=float, default=5.0)
    ap.add_argument("--serve-scene", default="c5", choices=["c5", "c3"],
                    help="served workload: c5 = 256^3 with moving boxes, c3 = the 128^3 scene")
    ap.add_argument("--serve-no-masks", action="store_true",
                    help="serve from a grid without edge masks")
    ap.add_argument("--tile-depth", default="auto", choices=["auto", "8", "16"],
                    help="propagation tile depth; auto = the autotuner's choice")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "c4":
        run_uneven(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
