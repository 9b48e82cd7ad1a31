"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Sizes: the 32^3 workload (every seed of a range, several tiles and a ragged
last tile of work), non-cubic grids with ragged rows, and the 128^3 workload
(sampled: the forward sets, two targets' survivor sets, one smooth step, and
invariants for all 64 targets).  Everything is integer/boolean, so the bar
is exact equality.
"""
import numpy as np
import pytest

import oracle as O
import scenegen as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ik():
    from paper_1906_10678_b300 import build
    build.build()
    from paper_1906_10678_b300 import ik as mod
    return mod


def _grid(ik, scene):
    g = ik.Grid(*scene.shape)
    ik.ik_set_boxes(g.h, scene.boxes)
    return g


def _sets(ik, words, shape, S):
    return ik.unpack_bits(words.reshape(-1), shape).reshape(-1, S + 1, shape[2], shape[1], shape[0])


# ------------------------------------------------------------------ a1

@pytest.mark.parametrize("shape,n_boxes,seed", [((32, 32, 32), 20, 0), ((64, 40, 24), 60, 1),
                                                ((96, 17, 9), 30, 2), ((128, 128, 128), 200, 1)])
def test_rasterize(ik, shape, n_boxes, seed):
    sc = G.make_scene(*shape, (shape[0] // 2, shape[1] // 2, 0), (4,), n_boxes, 1, 24, seed)
    boxes = np.concatenate([sc.boxes, [[-5, -5, -5, 3, 2, 1], [shape[0] - 3, 0, 0, shape[0] + 9, 5, 5],
                                       [10, 10, 10, 9, 10, 10]]]).astype(np.int32)
    with ik.Grid(*shape) as g:
        ik.ik_set_boxes(g.h, boxes)
        got = ik.ik_get_obstacles(g.h)
        want = ik.pack_bits(O.rasterize(shape, boxes))
        assert (got == want).all()
        ik.ik_set_boxes(g.h, np.zeros((0, 6), np.int32))
        assert not ik.ik_get_obstacles(g.h).any()
        ik.ik_set_obstacles(g.h, want)
        assert (ik.ik_get_obstacles(g.h) == want).all()


# ------------------------------------------- forward, survivor sets, reach

@pytest.mark.parametrize("seed", range(8))
def test_forward_sets_c1(ik, seed):
    sc = G.c1_scene(seed)
    occ = O.rasterize(sc.shape, sc.boxes)
    with _grid(ik, sc) as g:
        F = ik.ik_forward_sets(g.h, sc.lengths, sc.root)
    Fo = O.forward(occ, sc.lengths, sc.root)
    assert (ik.unpack_bits(F, sc.shape) == Fo.astype(bool)).all()


@pytest.mark.parametrize("seed", range(12))
def test_reach_c1(ik, seed):
    sc = G.c1_scene(seed)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 6, seed)
    # add an occupied target and one beyond reach when available
    occd = np.argwhere(occ)
    extra = [occd[0][::-1]] if len(occd) else []
    targets = np.concatenate([targets, np.asarray(extra, np.int32).reshape(-1, 3),
                              [[0, 0, 31], [31, 31, 31]]]).astype(np.int32)
    po, fo, vo = O.reach_many(occ, sc.lengths, sc.root, targets, want_sets=True, threads=4)
    with _grid(ik, sc) as g:
        pg, fg, vg = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets, want_sets=True)
        for i in range(2):
            p1, f1, _ = ik.ik_solve_reach(g.h, sc.lengths, sc.root, targets[i])
            assert f1 == bool(fg[i]) and (p1 == pg[i]).all()
    S = len(sc.lengths)
    assert (fg == fo).all()
    assert (pg[fo == 1] == po[fo == 1]).all()
    assert (_sets(ik, vg, sc.shape, S) == vo.astype(bool)).all()


@pytest.mark.parametrize("shape,lengths,seed", [((64, 40, 24), (9, 7, 5), 3),
                                                ((96, 20, 12), (6, 6, 6, 6), 4),
                                                ((32, 9, 31), (3, 8), 5)])
def test_reach_ragged_grids(ik, shape, lengths, seed):
    root = (shape[0] // 2, shape[1] // 2, 0)
    sc = G.make_scene(*shape, root, lengths, 25, 2, 6, seed)
    occ = O.rasterize(shape, sc.boxes)
    targets = G.draw_targets(sc, 5, seed)
    po, fo, vo = O.reach_many(occ, lengths, root, targets, want_sets=True, threads=4)
    with _grid(ik, sc) as g:
        pg, fg, vg = ik.ik_solve_reach_many(g.h, lengths, root, targets, want_sets=True)
        F = ik.ik_forward_sets(g.h, lengths, root)
    assert (ik.unpack_bits(F, shape) == O.forward(occ, lengths, root).astype(bool)).all()
    assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
    assert (_sets(ik, vg, shape, len(lengths)) == vo.astype(bool)).all()


def test_edge_cases(ik):
    sc = G.c1_scene(0)
    with _grid(ik, sc) as g:
        # occupied root: nothing reachable
        boxes = np.concatenate([sc.boxes, [[16, 16, 0, 16, 16, 0]]]).astype(np.int32)
        ik.ik_set_boxes(g.h, boxes)
        F = ik.ik_forward_sets(g.h, sc.lengths, sc.root)
        assert not F.any()
        _, f, _ = ik.ik_solve_reach(g.h, sc.lengths, sc.root, (20, 20, 10))
        assert not f
        ik.ik_set_boxes(g.h, sc.boxes)
        # empty batch, targets outside the grid, bad arms
        p, f, _ = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, np.zeros((0, 3), np.int32))
        assert len(p) == 0
        with pytest.raises(ik.IkError):
            ik.ik_solve_reach(g.h, sc.lengths, sc.root, (32, 0, 0))
        with pytest.raises(ik.IkError):
            ik.ik_solve_reach(g.h, [], sc.root, (3, 3, 3))
        with pytest.raises(ik.IkError):
            ik.ik_solve_reach(g.h, [0, 3], sc.root, (3, 3, 3))
        # a one-segment arm: found iff offset in shell and segment free
        occ = O.rasterize(sc.shape, sc.boxes)
        t = [(16 + 6, 16, 0), (16, 16 + 3, 4), (16, 16, 6), (17, 18, 5)]
        pg, fg, _ = ik.ik_solve_reach_many(g.h, [6], sc.root, t)
        po, fo, _ = O.reach_many(occ, [6], sc.root, t)
        assert (fg == fo).all() and (pg == po).all()
        # grids of the smallest and largest supported extents
        with pytest.raises(ik.IkError):
            ik.Grid(16, 8, 8)
        with ik.Grid(32, 1, 1) as g1:
            pg, fg, _ = ik.ik_solve_reach_many(g1.h, [3], (0, 0, 0), [(3, 0, 0), (2, 0, 0)])
            assert fg.tolist() == [1, 0]


# ------------------------------------------- guide, waypoint sets, chain

def _reachable(sc, occ, n, seed):
    targets = G.draw_targets(sc, n, seed)
    po, fo, _ = O.reach_many(occ, sc.lengths, sc.root, targets, threads=4)
    return targets[fo == 1], po[fo == 1]


@pytest.mark.parametrize("seed", range(4))
def test_guide_and_waypoint_sets_c1(ik, seed):
    sc = G.c1_scene(seed)
    occ = O.rasterize(sc.shape, sc.boxes)
    _, reach = _reachable(sc, occ, 3, seed)
    with _grid(ik, sc) as g:
        for W in (2, 5, 8):
            r = reach[0]
            assert (ik.ik_guide(g.h, sc.lengths, r, W) == O.guide(sc.lengths, r, W)).all()
            ug, vg = ik.ik_waypoint_sets(g.h, sc.lengths, r, W, eps2=2, eps2_max=8)
            uo, vo = O.waypoint_sets(occ, sc.lengths, r, W, eps2=2, eps2_max=8, threads=4)
            assert (ug == uo).all()
            assert (_sets(ik, vg, sc.shape, len(sc.lengths)) == vo.astype(bool)).all()


@pytest.mark.parametrize("seed", range(6))
def test_plan_path_c1(ik, seed):
    sc = G.c1_scene(seed)
    occ = O.rasterize(sc.shape, sc.boxes)
    _, reach = _reachable(sc, occ, 3, 10 + seed)
    with _grid(ik, sc) as g:
        for i in range(min(2, len(reach))):
            for W, delta in ((8, 3), (12, 2)):
                pg, rg, sg = ik.ik_plan_path(g.h, sc.lengths, reach[i], W, delta=delta)
                po, ro, so = O.plan_path(occ, sc.lengths, reach[i], W, delta=delta)
                assert sg == so
                assert (rg == ro).all()
                assert (pg == po).all()


def test_plan_path_relax_cap_and_invalid_reach(ik):
    sc = G.c1_scene(2)
    occ = O.rasterize(sc.shape, sc.boxes)
    _, reach = _reachable(sc, occ, 3, 7)
    with _grid(ik, sc) as g:
        pg, rg, sg = ik.ik_plan_path(g.h, sc.lengths, reach[0], 10, delta=1, max_relax=1)
        po, ro, so = O.plan_path(occ, sc.lengths, reach[0], 10, delta=1, max_relax=1)
        assert sg == so and (rg == ro).all() and (pg == po).all()
        bad = reach[0].copy()
        bad[1] = bad[0]  # a zero-length first segment is never admissible
        assert not O.pose_valid(occ, sc.lengths, bad)
        _, _, st = ik.ik_plan_path(g.h, sc.lengths, bad, 8)
        assert st == ik.IK_PATH_UNREACHABLE


def test_reach_path_many_matches_single_calls(ik):
    sc = G.c1_scene(3)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 6, 3)
    W = 8
    with _grid(ik, sc) as g:
        reach, found, poses, relax, status = ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, W)
        for i in range(len(targets)):
            p1, f1, _ = ik.ik_solve_reach(g.h, sc.lengths, sc.root, targets[i])
            assert f1 == bool(found[i])
            if not f1:
                assert status[i] == ik.IK_PATH_UNREACHABLE
                continue
            assert (p1 == reach[i]).all()
            ps, rs, ss = ik.ik_plan_path(g.h, sc.lengths, p1, W)
            assert ss == status[i] and (rs == relax[i]).all() and (ps == poses[i]).all()
    po, ro, so = O.plan_path(occ, sc.lengths, reach[found == 1][0], W)
    i0 = int(np.argmax(found))
    assert so == status[i0] and (ro == relax[i0]).all() and (po == poses[i0]).all()


# ------------------------------------------------------------------- a9

def test_validate_poses(ik):
    sc = G.c1_scene(4)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets, reach = _reachable(sc, occ, 6, 4)
    rng = np.random.default_rng(0)
    poses = [reach[i] for i in range(len(reach))]
    for i in range(len(reach)):
        p = reach[i].copy()
        p[rng.integers(1, len(sc.lengths) + 1)] += rng.integers(-2, 3, 3)
        poses.append(p)
    poses.append(np.full_like(reach[0], 40))
    poses = np.asarray(poses, np.int32)
    with _grid(ik, sc) as g:
        v = ik.ik_validate_poses(g.h, sc.lengths, poses)
    want = [O.pose_valid(occ, sc.lengths, p) for p in poses]
    assert v.astype(bool).tolist() == want


@pytest.mark.parametrize("seed", range(4))
def test_replan_c1(ik, seed):
    sc = G.c1_scene(seed)
    occ = O.rasterize(sc.shape, sc.boxes)
    _, reach = _reachable(sc, occ, 4, 20 + seed)
    W = 8
    with _grid(ik, sc) as g:
        path, _, _ = ik.ik_plan_path(g.h, sc.lengths, reach[0], W)
        kept, _, st = ik.ik_replan(g.h, sc.lengths, path, 2)
        assert st == ik.IK_PATH_KEPT and (kept == path).all()
        for j_cut, joint in ((W - 3, 2), (W - 1, 1), (W - 2, len(sc.lengths) - 1)):
            v = path[j_cut][joint]
            box = np.array([[v[0], v[1], v[2], v[0] + 1, v[1] + 1, v[2]]], np.int32)
            boxes = np.concatenate([sc.boxes, box])
            occ2 = O.rasterize(sc.shape, boxes)
            ik.ik_set_boxes(g.h, boxes)
            for c in (1, 3):
                pg, rg, sg = ik.ik_replan(g.h, sc.lengths, path, c)
                po, ro, so = O.replan(occ2, sc.lengths, path, c)
                assert sg == so, (j_cut, c)
                assert (rg == ro).all() and (pg == po).all(), (j_cut, c)
            ik.ik_set_boxes(g.h, sc.boxes)


# ------------------------------------------------------ 128^3 (sampled)

@pytest.fixture(scope="module")
def c2(ik):
    sc = G.c2_scene(1)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 64, 1)
    return sc, occ, targets


def test_c2_forward_sets_exact(ik, c2):
    sc, occ, _ = c2
    with _grid(ik, sc) as g:
        F = ik.ik_forward_sets(g.h, sc.lengths, sc.root)
    Fo = O.forward(occ, sc.lengths, sc.root)
    assert (ik.unpack_bits(F, sc.shape) == Fo.astype(bool)).all()


def test_c2_reach_all_targets_invariants_and_two_exact(ik, c2):
    sc, occ, targets = c2
    S = len(sc.lengths)
    with _grid(ik, sc) as g:
        pg, fg, vg = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets[:2], want_sets=True)
        pall, fall, _ = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets)
    po, fo, vo = O.reach_many(occ, sc.lengths, sc.root, targets[:2], want_sets=True, threads=2)
    assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
    assert (_sets(ik, vg, sc.shape, S) == vo.astype(bool)).all()
    assert (pall[:2] == pg).all() and (fall[:2] == fg).all()
    assert fall.sum() > 32
    for i in range(len(targets)):
        if fall[i]:
            assert tuple(pall[i][0]) == sc.root and tuple(pall[i][-1]) == tuple(targets[i])
            assert O.pose_valid(occ, sc.lengths, pall[i])


def test_c3_path_sampled_exact_and_invariants(ik, c2):
    sc, occ, targets = c2
    S, W = len(sc.lengths), 32
    with _grid(ik, sc) as g:
        reach, found, poses, relax, status = ik.ik_reach_path_many(g.h, sc.lengths, sc.root,
                                                                    targets[:8], W)
    i = int(np.argmax(found))
    assert found[i]
    # exact: survivor sets and smooth step of the last two waypoints of one path
    used, vo = O.waypoint_sets_range(occ, sc.lengths, reach[i], W, W - 3, W - 1)
    for jj, j in enumerate(range(W - 3, W - 1)):
        assert relax[i][j][1] == used[jj]
    pose, m = O.smooth_step(occ, sc.lengths, vo[1], poses[i][W - 1])
    assert m == relax[i][W - 2][0]
    assert (pose == poses[i][W - 2]).all()
    pose, m = O.smooth_step(occ, sc.lengths, vo[0], poses[i][W - 2])
    assert m == relax[i][W - 3][0] and (pose == poses[i][W - 3]).all()
    # invariants on every path
    for p in range(len(found)):
        if not found[p]:
            assert status[p] == 3
            continue
        gpts = O.guide(sc.lengths, reach[p], W)
        assert (poses[p][W - 1] == reach[p]).all()
        for j in range(W):
            assert O.pose_valid(occ, sc.lengths, poses[p][j])
            if j < W - 1 and relax[p][j][0] >= 0:
                e = poses[p][j][-1] - gpts[j]
                assert int(e @ e) <= relax[p][j][1]
                d = 3 + relax[p][j][0]
                step = poses[p][j] - poses[p][j + 1]
                assert (np.sum(step * step, axis=1) <= d * d).all()
