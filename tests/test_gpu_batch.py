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
    out, ms = ik.ik_solve_batch([_as_dict(p) for p in probs])
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
    out, _ = ik.ik_solve_batch([_as_dict(p) for p in probs])
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


def _scene64():
    sc = G.scaled_scene(64, (8, 7, 6, 5), 60, 2, 8, 21, "mb64")
    import oracle as O
    occ = O.rasterize(sc.shape, sc.boxes)
    # a second root away from the first (floor centre): the nearest free voxel to (14, 48, 30)
    free = np.argwhere(occ == 0)  # (z, y, x)
    d2 = ((free - np.array([30, 48, 14])) ** 2).sum(1)
    z, y, x = free[np.argmin(d2)]
    return sc, occ, (int(x), int(y), int(z))


def _targets_near(occ, lengths, root, n, seed):
    """n free voxels within reach of root (rejection sampling, seeded)."""
    rng = np.random.default_rng(seed)
    reach = sum(lengths)
    out = []
    while len(out) < n:
        p = np.asarray(root) + rng.integers(-reach, reach + 1, 3)
        if (p < 0).any() or (p >= 64).any() or occ[p[2], p[1], p[0]]:
            continue
        if ((p - np.asarray(root)) ** 2).sum() <= reach * reach:
            out.append(p)
    return np.asarray(out, np.int32)


def test_edge_mask_boxes_for_two_roots(ik):
    """Edge masks are stored over the box each root's chains can reach; a grid
    used from two roots (boxes grown to their union) gives the results of
    fresh grids, and the reach poses of the oracle."""
    import oracle as O
    sc, occ, root2 = _scene64()
    t1 = _targets_near(occ, sc.lengths, sc.root, 5, 1)
    t2 = _targets_near(occ, sc.lengths, root2, 5, 2)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        a1 = ik.ik_reach_path_many(g.h, sc.lengths, sc.root, t1, 8)
        a2 = ik.ik_reach_path_many(g.h, sc.lengths, root2, t2, 8)
        a1b = ik.ik_reach_path_many(g.h, sc.lengths, sc.root, t1, 8)
    for root, t, got in ((sc.root, t1, a1), (root2, t2, a2), (sc.root, t1, a1b)):
        with ik.Grid(*sc.shape) as g2:
            ik.ik_set_boxes(g2.h, sc.boxes)
            want = ik.ik_reach_path_many(g2.h, sc.lengths, root, t, 8)
        for a, w_ in zip(got, want):
            assert (a == w_).all()
    po, fo, _ = O.reach_many(occ, sc.lengths, root2, t2, threads=4)
    assert (a2[1] == fo).all() and (a2[0][fo == 1] == po[fo == 1]).all()


def test_batch_replay_after_the_grid_replaced_its_buffers(ik):
    """A captured batch keeps working after ordinary calls on its grid grew
    the scratch buffers and the edge-mask boxes (the old buffers stay with the
    batch); the grid's own later calls stay correct too."""
    import torch
    torch.cuda.set_device(0)
    sc, occ, root2 = _scene64()
    n, W, S = 4, 8, len(sc.lengths)
    t1 = _targets_near(occ, sc.lengths, sc.root, n, 3)
    stream = torch.cuda.Stream()
    g = ik.Grid(*sc.shape, stream=stream.cuda_stream)
    boxes = torch.from_numpy(sc.boxes.copy()).cuda()
    targets = torch.from_numpy(t1.copy()).cuda()
    outs = [torch.zeros(sz, dtype=torch.int32, device="cuda")
            for sz in ((n, S + 1, 3), (n,), (n, W, S + 1, 3), (n, W, 2), (n,))]
    b = ik.Batch(g.h, sc.lengths, sc.root, boxes, targets, W, *outs)
    b.launch()
    stream.synchronize()
    first = [o.cpu().numpy().copy() for o in outs]
    # ordinary calls that need larger buffers and a larger mask box
    t_many = _targets_near(occ, sc.lengths, root2, 3 * n, 4)
    big = ik.ik_reach_path_many(g.h, sc.lengths, root2, t_many, 2 * W)
    for o in outs:
        o.zero_()
    b.launch()
    stream.synchronize()
    again = [o.cpu().numpy() for o in outs]
    for a, w_ in zip(again, first):
        assert (a == w_).all()
    after = ik.ik_reach_path_many(g.h, sc.lengths, sc.root, t1, W)
    b.close()
    g.close()
    with ik.Grid(*sc.shape) as g2:
        ik.ik_set_boxes(g2.h, sc.boxes)
        want1 = ik.ik_reach_path_many(g2.h, sc.lengths, sc.root, t1, W)
        want2 = ik.ik_reach_path_many(g2.h, sc.lengths, root2, t_many, 2 * W)
    for a, w_ in zip(first, want1):
        assert (a == w_).all()
    for a, w_ in zip(after, want1):
        assert (a == w_).all()
    for a, w_ in zip(big, want2):
        assert (a == w_).all()


def _packed_outputs(ik, torch, dicts):
    r_n, p_n, x_n = ik.ik_batch_output_sizes(dicts)
    i32 = dict(dtype=torch.int32, device="cuda")
    n = len(dicts)
    return [torch.full((n,), -7, **i32), torch.full((r_n,), -7, **i32), torch.full((p_n,), -7, **i32),
            torch.full((x_n,), -7, **i32), torch.full((n,), -7, **i32), torch.full((n,), -7, **i32)]


def test_uneven_batch_async_on_a_stream_equals_sync(ik):
    """ik_solve_batch_async (device outputs, a caller stream, a status per
    job) gives exactly what the synchronous form gives, twice in a row on one
    engine (the second call reuses the engine's memory)."""
    import torch
    probs = [_as_dict(p) for p in G.c4_problems(10, 5)]
    want, _ = ik.ik_solve_batch(probs)
    stream = torch.cuda.Stream()
    with ik.BatchEngine() as eng:
        for _ in range(2):
            found, reach, poses, relax, status, rc = _packed_outputs(ik, torch, probs)
            eng.solve_async(probs, found, reach, poses, relax, status, rc, stream=stream.cuda_stream)
            stream.synchronize()
            assert (rc.cpu().numpy() == ik.IK_OK).all()
            got = ik.unpack_batch(probs, found.cpu().numpy(), reach.cpu().numpy(), poses.cpu().numpy(),
                                  relax.cpu().numpy(), status.cpu().numpy())
            for a, b in zip(got, want):
                assert a["found"] == b["found"] and a["status"] == b["status"]
                assert (a["reach"] == b["reach"]).all() and (a["poses"] == b["poses"]).all()
                assert (a["relax"] == b["relax"]).all()


def test_uneven_batch_waves_equal_one_launch(ik):
    """A pool budget that fits one problem at a time (one launch per problem)
    gives the same results as the whole batch in one launch."""
    import torch
    probs = [_as_dict(p) for p in G.c4_problems(6, 6)]
    want, _ = ik.ik_solve_batch(probs)
    with ik.BatchEngine() as eng:
        eng.set_budget(1)
        found, reach, poses, relax, status, rc = _packed_outputs(ik, torch, probs)
        eng.solve_async(probs, found, reach, poses, relax, status, rc)
        torch.cuda.synchronize()
        assert (rc.cpu().numpy() == ik.IK_OK).all()
        got = ik.unpack_batch(probs, found.cpu().numpy(), reach.cpu().numpy(), poses.cpu().numpy(),
                              relax.cpu().numpy(), status.cpu().numpy())
    for a, b in zip(got, want):
        assert a["status"] == b["status"] and (a["poses"] == b["poses"]).all()


def test_uneven_batch_query_pairs_equal_single_queries(ik):
    """Waypoint items carrying two queries (sharing each supercover walk)
    give exactly the results of one query per item, on problems of every
    grid size and on one whose waypoint count is odd."""
    import torch
    probs = [_as_dict(p) for p in G.c4_problems(12, 7)]
    assert any(p["n_way"] % 2 for p in probs) and len({p["shape"][0] for p in probs}) >= 3
    outs = []
    for pairs in (0, 1):
        with ik.BatchEngine() as eng:
            eng.set_pairs(pairs)
            found, reach, poses, relax, status, rc = _packed_outputs(ik, torch, probs)
            eng.solve_async(probs, found, reach, poses, relax, status, rc)
            torch.cuda.synchronize()
            assert (rc.cpu().numpy() == ik.IK_OK).all()
            outs.append([t.cpu().numpy() for t in (found, reach, poses, relax, status)])
    for a, b in zip(*outs):
        assert (a == b).all()
    with ik.BatchEngine() as eng:
        for bad in (-1, 2):
            with pytest.raises(Exception):
                eng.set_pairs(bad)


def test_uneven_batch_captured_graph_replays_equal_sync(ik):
    """The batch captured as a CUDA graph (one persistent launch) gives the
    synchronous results on every replay, also after the caller's problem
    arrays changed (they are copied at capture)."""
    import torch
    probs = [_as_dict(p) for p in G.c4_problems(10, 8)]
    want, _ = ik.ik_solve_batch(probs)
    stream = torch.cuda.Stream()
    with ik.BatchEngine() as eng:
        outs = _packed_outputs(ik, torch, probs)
        with eng.capture(probs, *outs) as graph:
            for p in probs:  # the caller's data may change after capture
                p["boxes"] = np.zeros((0, 6), np.int32)
            for _ in range(2):
                for t in outs:
                    t.fill_(-7)
                torch.cuda.synchronize()
                graph.launch(stream.cuda_stream)
                stream.synchronize()
                found, reach, poses, relax, status, rc = outs
                assert (rc.cpu().numpy() == ik.IK_OK).all()
                got = ik.unpack_batch([_as_dict(p) for p in G.c4_problems(10, 8)], found.cpu().numpy(),
                                      reach.cpu().numpy(), poses.cpu().numpy(), relax.cpu().numpy(),
                                      status.cpu().numpy())
                for a, b in zip(got, want):
                    assert a["found"] == b["found"] and a["status"] == b["status"]
                    assert (a["reach"] == b["reach"]).all() and (a["poses"] == b["poses"]).all()
                    assert (a["relax"] == b["relax"]).all()
        with pytest.raises(Exception):
            eng.capture([], *outs)


def test_uneven_batch_timeout_is_reported_and_the_context_stays_usable(ik):
    """With a wait limit too short for any work (1 microsecond) the
    persistent launch gives up on its own: unfinished problems report
    IK_ERR_TIMEOUT in their job status (no fault, no hang), and the next call
    with the default limit on the same engine is exact."""
    import torch
    probs = [_as_dict(p) for p in G.c4_problems(4, 7)]
    want, _ = ik.ik_solve_batch(probs)
    with ik.BatchEngine() as eng:
        eng.set_timeout(1000)
        found, reach, poses, relax, status, rc = _packed_outputs(ik, torch, probs)
        eng.solve_async(probs, found, reach, poses, relax, status, rc)
        torch.cuda.synchronize()
        codes = set(rc.cpu().numpy().tolist())
        assert ik.IK_ERR_TIMEOUT in codes and codes <= {ik.IK_OK, ik.IK_ERR_TIMEOUT}
        eng.set_timeout(20 * 10 ** 9)
        found, reach, poses, relax, status, rc = _packed_outputs(ik, torch, probs)
        eng.solve_async(probs, found, reach, poses, relax, status, rc)
        torch.cuda.synchronize()
        assert (rc.cpu().numpy() == ik.IK_OK).all()
        got = ik.unpack_batch(probs, found.cpu().numpy(), reach.cpu().numpy(), poses.cpu().numpy(),
                              relax.cpu().numpy(), status.cpu().numpy())
    for a, b in zip(got, want):
        assert a["status"] == b["status"] and (a["poses"] == b["poses"]).all()


def test_engines_share_the_kernels_shared_memory_setting(ik):
    """Two engines on one device: one launches with the largest bricks (reach
    24 on a 192^3 grid), the other with small ones, then the first again.
    The kernel's shared-memory setting is shared by the engines and must not
    be lowered under the first one's feet."""
    import torch
    sc = G.scaled_scene(192, (24, 16, 10, 6, 5), 150, 4, 24, 12, "big")
    t = G.draw_targets(sc, 1, 12)[0]
    big = [{"shape": sc.shape, "boxes": sc.boxes, "lengths": sc.lengths, "root": sc.root,
            "target": tuple(int(v) for v in t), "n_way": 8}]
    small = [_as_dict(p) for p in G.c4_problems(3, 9) if p.scene.shape[0] == 64][:1] or \
        [_as_dict(G.c4_problems(1, 9)[0])]
    want, _ = ik.ik_solve_batch(big)
    with ik.BatchEngine() as e1, ik.BatchEngine() as e2:
        for eng, probs in ((e1, big), (e2, small), (e1, big)):
            found, reach, poses, relax, status, rc = _packed_outputs(ik, torch, probs)
            eng.solve_async(probs, found, reach, poses, relax, status, rc)
            torch.cuda.synchronize()
            assert (rc.cpu().numpy() == ik.IK_OK).all()
        got = ik.unpack_batch(big, found.cpu().numpy(), reach.cpu().numpy(), poses.cpu().numpy(),
                              relax.cpu().numpy(), status.cpu().numpy())
    assert got[0]["status"] == want[0]["status"] and (got[0]["poses"] == want[0]["poses"]).all()
