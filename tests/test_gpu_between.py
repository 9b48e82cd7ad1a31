"""Paths between arbitrary poses (section "Path between Arbitrary Poses": a
virtual arm rooted at the start's end effector guides the end effector)
against the oracle, through the C ABI."""
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


@pytest.mark.parametrize("masks", [1, 0])
@pytest.mark.parametrize("seed", range(3))
def test_plan_between_matches_oracle_c1(ik, seed, masks):
    sc = G.c1_scene(60 + seed)
    occ = O.rasterize(sc.shape, sc.boxes)
    starts_t = G.draw_targets(sc, 6, 70 + seed)
    goals = G.draw_targets(sc, 4, 80 + seed)
    guide = (6, 5, 4)
    W = 7
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
        ik.ik_set_boxes(g.h, sc.boxes)
        pr, fr, _ = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, starts_t)
        starts = [pr[i] for i in np.nonzero(fr)[0][:2]]
        assert starts
        for start in starts:
            for t in goals:
                got = ik.ik_plan_between(g.h, sc.lengths, start, guide, t, W)
                want = O.plan_between(occ, sc.lengths, start, guide, t, W)
                assert got[2] == want[2], (start.tolist(), t)
                assert (got[0] == want[0]).all() and (got[1] == want[1]).all()
                if want[2] != O.PATH_UNREACHABLE:
                    assert (got[3] == want[3]).all()


def test_plan_between_invalid_start_and_errors(ik):
    sc = G.c1_scene(2)
    t = G.draw_targets(sc, 1, 3)[0]
    bad = np.array([[16, 16, 0], [16, 16, 1], [16, 16, 8], [16, 16, 14], [16, 16, 19]], np.int32)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        poses, relax, st, _ = ik.ik_plan_between(g.h, sc.lengths, bad, (6, 5), t, 5)
        assert st == ik.IK_PATH_UNREACHABLE and (relax[1:, 0] == -1).all()
        assert all((p == bad).all() for p in poses)
        with pytest.raises(ik.IkError) as e:
            ik.ik_plan_between(g.h, sc.lengths, bad, (6, 5), (99, 0, 0), 5)
        assert e.value.code == ik.IK_ERR_ARG


def test_plan_between_128_invariants(ik):
    """The 128^3 scene: from the reach pose of one target to another target;
    every pose valid, joints move at most delta + m between waypoints, the
    first pose is the start and a complete path ends at the target."""
    sc = G.c2_scene(1)
    occ = O.rasterize(sc.shape, sc.boxes)
    t = G.draw_targets(sc, 12, 21)
    W, delta = 16, 3
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        pr, fr, _ = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, t)
        idx = np.nonzero(fr)[0]
        start = pr[idx[0]]
        done = 0
        for i in idx[1:6]:
            poses, relax, st, gp = ik.ik_plan_between(g.h, sc.lengths, start, (16, 14, 12), t[i], W)
            assert (poses[0] == start).all()
            if st == ik.IK_PATH_UNREACHABLE:
                continue
            done += 1
            assert (gp[0] == start[-1]).all() and (gp[-1] == t[i]).all()
            for j in range(W):
                assert O.pose_valid(occ, sc.lengths, poses[j])
            for j in range(1, W):
                m = relax[j][0]
                if m >= 0:
                    d2 = ((poses[j] - poses[j - 1]) ** 2).sum(1)
                    assert (d2 <= (delta + m) ** 2).all()
            if st in (ik.IK_PATH_OK, ik.IK_PATH_RELAXED):
                assert (poses[-1][-1] == t[i]).all()
        assert done > 0
