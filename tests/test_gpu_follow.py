"""The path in the paper's form (follower joint S-1 with the last segment
folded, n guide points per segment, a filter radius per joint) equals the
oracle's, bit for bit."""
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


def _grid(ik, sc, masks):
    g = ik.Grid(*sc.shape)
    ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
    ik.ik_set_boxes(g.h, sc.boxes)
    return g


def _paper_radii(lengths, n, fold):
    """The paper's filter (section "Filtering for smoothness"), stated here
    for the oracle's input: joint 1 about half a waypoint spacing and joint 2
    about one, plus a voxel of slack; spacing = longest follower segment / n,
    rounded up."""
    F = len(lengths) - (1 if fold else 0)
    s = -(-max(lengths[:F]) // n)
    rad = [-1] * F
    rad[0] = -(-s // 2) + 1
    if F >= 2:
        rad[1] = s + 1
    return rad


@pytest.mark.parametrize("masks", [1, 0])
@pytest.mark.parametrize("seed", range(3))
def test_follow_matches_oracle_c1(ik, seed, masks):
    sc = G.c1_scene(seed)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 4, 60 + seed)
    poses, found, _ = O.reach_many(occ, sc.lengths, sc.root, targets, threads=4)
    cases = [(4, True, None),                                   # the paper's filter (joints 1, 2)
             (3, True, [1, 2, 3]),                               # every follower joint filtered
             (2, False, [2, 3, -1, -1])]                         # the end effector as follower
    n_done = 0
    with _grid(ik, sc, masks) as g:
        for i in np.nonzero(found)[0][:2]:
            for n, fold, rad in cases:
                pg, rg, sg = ik.ik_plan_path_follow(g.h, sc.lengths, poses[i], n, fold, rad)
                po, ro, so = O.plan_path_follow(occ, sc.lengths, poses[i], n, fold,
                                                _paper_radii(sc.lengths, n, fold) if rad is None else rad)
                assert sg == so
                assert (rg == ro).all()
                assert (pg == po).all()
                n_done += 1
    assert n_done > 0


def test_follow_tight_filter_relaxes_and_matches(ik):
    """Radius 0 on the filtered joints forces the relaxation ladder."""
    sc = G.c1_scene(1)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 3, 7)
    poses, found, _ = O.reach_many(occ, sc.lengths, sc.root, targets, threads=4)
    i = int(np.nonzero(found)[0][0])
    with _grid(ik, sc, 1) as g:
        pg, rg, sg = ik.ik_plan_path_follow(g.h, sc.lengths, poses[i], 3, True, [0, 0, -1], max_relax=6)
    po, ro, so = O.plan_path_follow(occ, sc.lengths, poses[i], 3, True, [0, 0, -1], max_relax=6)
    assert sg == so and (rg == ro).all() and (pg == po).all()
    assert (ro[:, 0] != 0).any()


def test_follow_invalid_reach_and_arguments(ik):
    sc = G.c1_scene(0)
    S = len(sc.lengths)
    with _grid(ik, sc, 1) as g:
        bad = np.zeros((S + 1, 3), np.int32)
        p, r, st = ik.ik_plan_path_follow(g.h, sc.lengths, bad, 2, True, [2, 3, -1])
        assert st == ik.IK_PATH_UNREACHABLE
        occ = O.rasterize(sc.shape, sc.boxes)
        t = G.draw_targets(sc, 4, 3)
        poses, found, _ = O.reach_many(occ, sc.lengths, sc.root, t, threads=4)
        reach = poses[int(np.nonzero(found)[0][0])]
        for n, rad in ((0, [2, 3, -1]), (65, [2, 3, -1]), (2, [2, -2, -1])):
            with pytest.raises(ik.IkError) as e:
                ik.ik_plan_path_follow(g.h, sc.lengths, reach, n, True, rad)
            assert e.value.code == ik.IK_ERR_ARG
        # an arm with direction limits is refused
        ik.ik_set_segment_limits(g.h, sc.lengths, [ik.cone((0, 0, 1), 0, 1)] + [None] * (S - 1))
        with pytest.raises(ik.IkError) as e:
            ik.ik_plan_path_follow(g.h, sc.lengths, reach, 2, True, [2, 3, -1])
        assert e.value.code == ik.IK_ERR_UNSUPPORTED
