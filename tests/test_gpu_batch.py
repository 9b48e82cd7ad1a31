"""Captured batches (CUDA graph replay) against the ordinary calls."""
import numpy as np
import pytest

import scenegen as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ik():
    from paper_1906_10678_b300 import build
    build.build()
    from paper_1906_10678_b300 import ik as mod
    return mod


def test_graph_replay_matches_ordinary_calls(ik):
    import torch
    torch.cuda.set_device(0)
    sc = G.c1_scene(4)
    n, W, S = 6, 8, len(sc.lengths)
    stream = torch.cuda.Stream()
    g = ik.Grid(*sc.shape, stream=stream.cuda_stream)
    boxes = torch.from_numpy(sc.boxes.copy()).cuda()
    t_np = G.draw_targets(sc, n, 4)
    t_np[2] = (-1, -1, -1)  # an empty slot
    targets = torch.from_numpy(t_np.copy()).cuda()
    outs = [torch.zeros(sz, dtype=torch.int32, device="cuda")
            for sz in ((n, S + 1, 3), (n,), (n, W, S + 1, 3), (n, W, 2), (n,))]
    b = ik.Batch(g.h, sc.lengths, sc.root, boxes, targets, W, *outs)
    for rnd in range(3):
        if rnd == 1:  # new targets in place
            t2 = G.draw_targets(sc, n, 40)
            targets.copy_(torch.from_numpy(t2))
            t_np = t2
        if rnd == 2:  # new obstacles in place (same box count)
            moved = sc.boxes.copy()
            moved[:5, [0, 3]] += 2
            boxes.copy_(torch.from_numpy(moved))
        b.launch()
        stream.synchronize()
        got = [o.cpu().numpy() for o in outs]
        # ordinary calls on a second grid with the same occupancy
        with ik.Grid(*sc.shape) as g2:
            ik.ik_set_boxes(g2.h, boxes.cpu().numpy())
            valid = np.all((t_np >= 0) & (t_np < 32), axis=1)
            want = ik.ik_reach_path_many(g2.h, sc.lengths, sc.root, t_np[valid], W)
        for a, w_ in zip(got, want):
            assert (a[valid] == w_).all(), rnd
        assert (got[1][~valid] == 0).all() and (got[4][~valid] == ik.IK_PATH_UNREACHABLE).all()
    b.close()
    g.close()


def test_replan_many_matches_single_replans_and_oracle(ik):
    import oracle as O
    sc = G.c1_scene(1)
    occ = O.rasterize(sc.shape, sc.boxes)
    W, S = 8, len(sc.lengths)
    targets = G.draw_targets(sc, 8, 21)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        reach, found, paths, _, _ = ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, W)
        live = np.nonzero(found)[0]
        assert len(live) >= 3
        # an obstacle on a later joint of the first two live paths, and one on
        # the reach target of the third (its target becomes unreachable)
        extra = []
        for i in live[:2]:
            v = paths[i][W - 3][2]
            extra.append([v[0], v[1], v[2], v[0] + 1, v[1] + 1, v[2]])
        t = paths[live[2]][W - 1][S]
        extra.append([t[0], t[1], t[2], t[0], t[1], t[2]])
        boxes = np.concatenate([sc.boxes, np.asarray(extra, np.int32)])
        ik.ik_set_boxes(g.h, boxes)
        occ2 = O.rasterize(sc.shape, boxes)
        current = np.full(len(targets), 2, np.int32)
        current[~found.astype(bool)] = -1          # empty slots
        current[live[-1]] = W - 1                  # nothing left to replan
        pin = paths.copy()
        pin[current < 0] = 0
        pm, rm, sm = ik.ik_replan_many(g.h, sc.lengths, sc.root, pin, current)
        for r in range(len(targets)):
            if current[r] < 0:
                assert sm[r] == -1
                continue
            p1, r1, s1 = ik.ik_replan(g.h, sc.lengths, pin[r], int(current[r]))
            assert sm[r] == s1 and (rm[r] == r1).all() and (pm[r] == p1).all(), r
            po, ro, so = O.replan(occ2, sc.lengths, pin[r], int(current[r]))
            assert s1 == so and (r1 == ro).all() and (p1 == po).all(), r
        assert set(sm[live].tolist()) >= {ik.IK_PATH_KEPT}


def _as_dict(p):
    return {"shape": p.scene.shape, "boxes": p.scene.boxes, "lengths": p.scene.lengths,
            "root": p.scene.root, "target": p.target, "n_way": p.n_way}


def test_uneven_batch_matches_single_problem_calls(ik):
    import oracle as O
    probs = G.c4_problems(12, 2)
    out, ms = ik.ik_solve_batch([_as_dict(p) for p in probs], lanes=4)
    assert ms > 0
    for p, r in zip(probs, out):
        sc = p.scene
        with ik.Grid(*sc.shape) as g:
            ik.ik_set_boxes(g.h, sc.boxes)
            reach, found, poses, relax, status = ik.ik_reach_path_many(
                g.h, sc.lengths, sc.root, np.asarray([p.target], np.int32), p.n_way)
        assert r["found"] == found[0] and r["status"] == status[0], sc.name
        if found[0]:
            assert (r["reach"] == reach[0]).all()
            assert (r["poses"] == poses[0]).all() and (r["relax"] == relax[0]).all(), sc.name
    # one small problem against the oracle's reach
    small = [(p, r) for p, r in zip(probs, out) if p.scene.shape[0] == 64]
    if small:
        p, r = small[0]
        occ = O.rasterize(p.scene.shape, p.scene.boxes)
        po, fo, _ = O.reach_many(occ, p.scene.lengths, p.scene.root, [p.target], threads=8)
        assert fo[0] == r["found"] and (not fo[0] or (po[0] == r["reach"]).all())


def test_uneven_batch_long_segments_narrow_pitch(ik):
    """Segments of length 24 on 128^3 and 192^3 grids: their two halos take
    the narrow shared-memory pitch in the batch engine (no edge masks); the
    results equal the single-problem calls on grids with stored edge masks."""
    probs = []
    for n, lengths, seed in ((128, (24, 22, 12, 8, 6), 11), (192, (24, 16, 10, 6, 5), 12)):
        sc = G.scaled_scene(n, lengths, 150, 4, 24, seed, f"long{n}")
        t = G.draw_targets(sc, 1, seed)[0]
        probs.append(G.Problem(sc, tuple(int(v) for v in t), 12))
    out, _ = ik.ik_solve_batch([_as_dict(p) for p in probs], lanes=2)
    for p, r in zip(probs, out):
        sc = p.scene
        with ik.Grid(*sc.shape) as g:
            ik.ik_set_boxes(g.h, sc.boxes)
            reach, found, poses, relax, status = ik.ik_reach_path_many(
                g.h, sc.lengths, sc.root, np.asarray([p.target], np.int32), p.n_way)
        assert r["found"] == found[0] and r["status"] == status[0], sc.name
        if found[0]:
            assert (r["reach"] == reach[0]).all()
            assert (r["poses"] == poses[0]).all() and (r["relax"] == relax[0]).all(), sc.name
