"""Write the oracle's full-size expected outputs for the GPU parity tests.

Calls only ``oracle/`` (and ``scenegen`` for the seeded inputs); nothing here
comes from the CUDA library.  Run on the CPU machine:

    python tests/golden/make_full_size.py [--workers 7] [--cache DIR]

and it writes, beside itself:

* ``full_c3.npz`` -- the 128^3 scene (seed 1), 64 targets (seed 1): every
  reach pose and found flag; the whole 32-waypoint path (poses, relaxation
  records, status; delta 3, eps2 2..8) of the first 16 reachable targets;
  and, for the first 4 reachable targets at waypoints 0, 8, 16, 24 and 30,
  the SHA-256 and popcount of every survivor set V_k^(j) packed as x-fastest
  little-endian bits (the library's word layout), with the eps2 used.
* ``full_c4.npz`` -- the first 32 problems of the uneven 1024-problem batch
  (seed 2; 64^3 to 192^3, 5-9 segments, 8-32 waypoints): found flag, reach
  pose, path, relaxation records, status.
* ``full_c5.npz`` -- the 256^3 serving scene (seed 3) after 5 ticks of the 16
  moving boxes, 8 targets (seed 31): reach poses and found flags, and the
  whole 32-waypoint paths of the first 2 reachable targets.

One 128^3 backward pass of the oracle takes about 40 s of one core (256^3:
about 5 min), so the whole run is a few hours on 7 cores.  Per-task results
are cached in DIR (default: a ``.cache`` folder beside this file, which git
ignores) so an interrupted run resumes.
"""
from __future__ import annotations

import argparse
import hashlib
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W_C3 = 32
C3_PATHS = 16
C3_SET_PATHS = 4
C3_SET_WAYS = (0, 8, 16, 24, 30)
C4_COUNT = 32
C5_TARGETS = 8
C5_PATHS = 2
C5_TICKS = 5
W_C5 = 32


def set_digest(v: np.ndarray):
    """(sha256 hex, popcount) of a uint8 [nz][ny][nx] set packed x-fastest,
    bit b of byte i = voxel 8 i + b (little-endian uint32 words)."""
    b = np.packbits(np.asarray(v, dtype=bool).reshape(-1), bitorder="little")
    return hashlib.sha256(b.tobytes()).hexdigest(), int(np.count_nonzero(v))


def c3_scene():
    import scenegen as G
    sc = G.c2_scene(1)
    return sc, G.draw_targets(sc, 64, 1)


def c5_scene():
    import scenegen as G
    sc, mv = G.c5_scene(3)
    for _ in range(C5_TICKS):
        mv.step()
    boxes = np.concatenate([sc.boxes, mv.boxes()]).astype(np.int32)
    return sc, boxes, G.draw_targets(sc, C5_TARGETS, 31)


# ------------------------------------------------------------------ tasks

def task_c3_path(reach):
    import oracle as O
    sc, _ = c3_scene()
    occ = O.rasterize(sc.shape, sc.boxes)
    poses, relax, st = O.plan_path(occ, sc.lengths, reach, W_C3)
    return {"poses": poses, "relax": relax, "status": np.int32(st)}


def task_c3_sets(reach, j):
    import oracle as O
    sc, _ = c3_scene()
    occ = O.rasterize(sc.shape, sc.boxes)
    used, vo = O.waypoint_sets_range(occ, sc.lengths, reach, W_C3, j, j + 1)
    hashes, pops = [], []
    for k in range(len(sc.lengths) + 1):
        h, c = set_digest(vo[0][k])
        hashes.append(h)
        pops.append(c)
    return {"hash": np.asarray(hashes, "S64"), "pop": np.asarray(pops, np.int64),
            "used": np.int32(used[0])}


def task_c4(i):
    import oracle as O
    import scenegen as G
    p = G.c4_problems(1024, 2)[i]
    sc = p.scene
    occ = O.rasterize(sc.shape, sc.boxes)
    po, fo, _ = O.reach_many(occ, sc.lengths, sc.root, np.asarray([p.target], np.int32))
    S, W = len(sc.lengths), p.n_way
    out = {"found": np.int32(fo[0]), "reach": po[0].astype(np.int32),
           "poses": np.zeros((W, S + 1, 3), np.int32), "relax": np.zeros((W, 2), np.int32),
           "status": np.int32(3)}
    if fo[0]:
        poses, relax, st = O.plan_path(occ, sc.lengths, po[0], W)
        out.update(poses=poses, relax=relax, status=np.int32(st))
    return out


def task_c5_path(reach):
    import oracle as O
    sc, boxes, _ = c5_scene()
    occ = O.rasterize(sc.shape, boxes)
    poses, relax, st = O.plan_path(occ, sc.lengths, reach, W_C5)
    return {"poses": poses, "relax": relax, "status": np.int32(st)}


TASKS = {"c3_path": task_c3_path, "c3_sets": task_c3_sets, "c4": task_c4, "c5_path": task_c5_path}


def _run(args):
    name, key, fargs, cache = args
    path = os.path.join(cache, key + ".npz")
    if os.path.exists(path):
        return key, dict(np.load(path))
    t = time.time()
    res = TASKS[name](*fargs)
    np.savez(path + ".tmp.npz", **res)
    os.replace(path + ".tmp.npz", path)
    print(f"  {key}: {time.time() - t:.0f} s", flush=True)
    return key, res


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=7)
    ap.add_argument("--cache", default=os.path.join(HERE, ".cache"))
    a = ap.parse_args()
    os.makedirs(a.cache, exist_ok=True)
    import oracle as O
    import scenegen as G

    t0 = time.time()
    # phase 1: reach poses (all targets of one scene share one call)
    sc3, t3 = c3_scene()
    p3 = os.path.join(a.cache, "c3_reach.npz")
    if not os.path.exists(p3):
        occ3 = O.rasterize(sc3.shape, sc3.boxes)
        po, fo, _ = O.reach_many(occ3, sc3.lengths, sc3.root, t3, threads=a.workers + 1)
        np.savez(p3, reach=po, found=fo)
    r3 = dict(np.load(p3))
    print(f"c3 reach: {int(r3['found'].sum())}/64 found ({time.time() - t0:.0f} s)", flush=True)
    sc5, boxes5, t5 = c5_scene()
    p5 = os.path.join(a.cache, "c5_reach.npz")
    if not os.path.exists(p5):
        occ5 = O.rasterize(sc5.shape, boxes5)
        po, fo, _ = O.reach_many(occ5, sc5.lengths, sc5.root, t5, threads=a.workers + 1)
        np.savez(p5, reach=po, found=fo)
    r5 = dict(np.load(p5))
    print(f"c5 reach: {int(r5['found'].sum())}/{C5_TARGETS} found ({time.time() - t0:.0f} s)",
          flush=True)

    # phase 2: paths and survivor sets, the longest first
    f3 = np.nonzero(r3["found"])[0]
    f5 = np.nonzero(r5["found"])[0]
    c3_paths = [int(i) for i in f3[:C3_PATHS]]
    c3_sets = [int(i) for i in f3[:C3_SET_PATHS]]
    c5_paths = [int(i) for i in f5[:C5_PATHS]]
    probs = G.c4_problems(1024, 2)[:C4_COUNT]
    jobs = [("c5_path", f"c5_path_{i}", (r5["reach"][i],), a.cache) for i in c5_paths]
    cost = lambda p: p.scene.shape[0] ** 3 * (p.n_way + 1) * sum(L ** 3 for L in p.scene.lengths)
    for i in sorted(range(C4_COUNT), key=lambda i: -cost(probs[i])):
        jobs.append(("c4", f"c4_{i}", (i,), a.cache))
    jobs += [("c3_path", f"c3_path_{i}", (r3["reach"][i],), a.cache) for i in c3_paths]
    jobs += [("c3_sets", f"c3_sets_{i}_{j}", (r3["reach"][i], j), a.cache)
             for i in c3_sets for j in C3_SET_WAYS]
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.workers) as pool:
        res = dict(pool.imap_unordered(_run, jobs))

    S3 = len(sc3.lengths)
    np.savez_compressed(
        os.path.join(HERE, "full_c3.npz"),
        targets=t3, reach=r3["reach"], found=r3["found"], path_targets=np.asarray(c3_paths, np.int32),
        poses=np.stack([res[f"c3_path_{i}"]["poses"] for i in c3_paths]),
        relax=np.stack([res[f"c3_path_{i}"]["relax"] for i in c3_paths]),
        status=np.asarray([res[f"c3_path_{i}"]["status"] for i in c3_paths], np.int32),
        set_targets=np.asarray(c3_sets, np.int32), set_ways=np.asarray(C3_SET_WAYS, np.int32),
        set_hash=np.asarray([[res[f"c3_sets_{i}_{j}"]["hash"] for j in C3_SET_WAYS] for i in c3_sets],
                            "S64").reshape(len(c3_sets), len(C3_SET_WAYS), S3 + 1),
        set_pop=np.asarray([[res[f"c3_sets_{i}_{j}"]["pop"] for j in C3_SET_WAYS] for i in c3_sets]),
        set_used=np.asarray([[res[f"c3_sets_{i}_{j}"]["used"] for j in C3_SET_WAYS] for i in c3_sets]))
    c4 = [res[f"c4_{i}"] for i in range(C4_COUNT)]
    Smax = max(len(p.scene.lengths) for p in probs)
    Wmax = max(p.n_way for p in probs)
    poses4 = np.full((C4_COUNT, Wmax, Smax + 1, 3), -1, np.int32)
    relax4 = np.full((C4_COUNT, Wmax, 2), -9, np.int32)
    reach4 = np.full((C4_COUNT, Smax + 1, 3), -1, np.int32)
    for i, (p, r) in enumerate(zip(probs, c4)):
        S, W = len(p.scene.lengths), p.n_way
        poses4[i, :W, :S + 1] = r["poses"]
        relax4[i, :W] = r["relax"]
        reach4[i, :S + 1] = r["reach"]
    np.savez_compressed(os.path.join(HERE, "full_c4.npz"),
                        found=np.asarray([r["found"] for r in c4], np.int32), reach=reach4,
                        poses=poses4, relax=relax4,
                        status=np.asarray([r["status"] for r in c4], np.int32))
    np.savez_compressed(
        os.path.join(HERE, "full_c5.npz"), targets=t5, reach=r5["reach"], found=r5["found"],
        path_targets=np.asarray(c5_paths, np.int32),
        poses=np.stack([res[f"c5_path_{i}"]["poses"] for i in c5_paths]),
        relax=np.stack([res[f"c5_path_{i}"]["relax"] for i in c5_paths]),
        status=np.asarray([res[f"c5_path_{i}"]["status"] for i in c5_paths], np.int32))
    print(f"done in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
