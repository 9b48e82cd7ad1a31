"""Approach cones on the last segment and target clouds (section "The gap in
gMS": the backward search starts from the directions the last segment may
arrive along; section "Dynamic Obstacles": a cloud of targets) against
the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
import scenegen as G

pytestmark = pytest.mark.gpu

CONES = [((0, 0, 1), 1, 2), ((1, 0, 0), 0, 1), ((1, 1, 1), 1, 4), ((0, -1, 2), 3, 4),
         ((0, 0, -1), 1, 1), ((-3, 2, 5), 9, 10)]


@pytest.fixture(scope="module")
def ik():
    from paper_1906_10678_b300 import build
    build.build()
    from paper_1906_10678_b300 import ik as mod
    return mod


def _flat(c):
    return (*c[0], c[1], c[2])


@pytest.mark.parametrize("masks", [1, 0])
@pytest.mark.parametrize("seed", range(3))
def test_cone_reach_matches_oracle_c1(ik, seed, masks):
    sc = G.c1_scene(seed)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 6, 90 + seed)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
        ik.ik_set_boxes(g.h, sc.boxes)
        for c in CONES:
            poses, found, vs = ik.ik_solve_reach_many_cone(g.h, sc.lengths, ik.cone(*c), sc.root, targets,
                                                          want_sets=True)
            for i, t in enumerate(targets):
                T = np.zeros(occ.shape, np.uint8)
                T[t[2], t[1], t[0]] = 1
                po, fo, vo = O.reach_set(occ, sc.lengths, sc.root, T, _flat(c))
                assert found[i] == fo, (c, i)
                if fo:
                    assert (poses[i] == po).all(), (c, i)
                got = ik.unpack_bits(vs[i].reshape(-1), sc.shape).reshape(vo.shape)
                assert (got == vo.astype(bool)).all(), (c, i)


def test_no_cone_equals_plain_reach(ik):
    sc = G.c1_scene(5)
    targets = G.draw_targets(sc, 8, 3)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        a = ik.ik_solve_reach_many_cone(g.h, sc.lengths, None, sc.root, targets, want_sets=True)
        b = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets, want_sets=True)
    for x, y in zip(a, b):
        assert (x == y).all()


@pytest.mark.parametrize("seed", range(3))
def test_target_cloud_matches_oracle_c1(ik, seed):
    sc = G.c1_scene(10 + seed)
    occ = O.rasterize(sc.shape, sc.boxes)
    rng = np.random.default_rng(seed)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        for c in [None] + CONES[:3]:
            T = np.zeros(occ.shape, np.uint8)
            pts = G.draw_targets(sc, 5, 200 + seed)
            for t in pts:
                T[t[2], t[1], t[0]] = 1
            for t in rng.integers(0, 32, (4, 3)):  # some voxels anywhere (free or not)
                T[t[2], t[1], t[0]] = 1
            pose, found, vs = ik.ik_solve_reach_set(g.h, sc.lengths, None if c is None else ik.cone(*c),
                                                    sc.root, ik.pack_bits(T), want_sets=True)
            po, fo, vo = O.reach_set(occ, sc.lengths, sc.root, T, None if c is None else _flat(c))
            assert found == fo, c
            if fo:
                assert (pose == po).all(), c
            got = ik.unpack_bits(vs.reshape(-1), sc.shape).reshape(vo.shape)
            assert (got == vo.astype(bool)).all(), c


def test_cone_argument_errors(ik):
    sc = G.c1_scene(0)
    t = G.draw_targets(sc, 1, 1)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        for bad in [((0, 0, 0), 1, 2), ((0, 0, 1), 3, 2), ((0, 0, 1), 1, 0), ((0, 0, 1), -1, 2),
                    ((2000, 0, 1), 1, 2)]:
            with pytest.raises(ik.IkError) as e:
                ik.ik_solve_reach_many_cone(g.h, sc.lengths, ik.cone(*bad), sc.root, t)
            assert e.value.code == ik.IK_ERR_ARG
        # a cone that keeps no offset of the last segment's shell (length 5,
        # 21 <= |d|^2 <= 30: no offset lies exactly along (1, 2, 3), whose
        # multiples have |d|^2 = 14 t^2)
        with pytest.raises(ik.IkError) as e:
            ik.ik_solve_reach_many_cone(g.h, sc.lengths, ik.cone((1, 2, 3), 1, 1), sc.root, t)
        assert e.value.code == ik.IK_ERR_ARG
        with pytest.raises(ValueError):
            ik.ik_solve_reach_set(g.h, sc.lengths, None, sc.root, np.zeros(3, np.uint32))


def test_cone_reach_128_invariants_and_one_exact(ik):
    """The 128^3 scene, 16 targets approached from above (45 degrees): every
    found pose is valid with its last segment in the cone; one target exact
    against the oracle."""
    sc = G.c2_scene(1)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 16, 5)
    c = ((0, 0, -1), 1, 2)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        poses, found, vs = ik.ik_solve_reach_many_cone(g.h, sc.lengths, ik.cone(*c), sc.root, targets,
                                                      want_sets=True)
    assert found.sum() > 0
    S = len(sc.lengths)
    for i in np.nonzero(found)[0]:
        p = poses[i]
        assert O.pose_valid(occ, sc.lengths, p)
        s = p[S] - p[S - 1]
        assert s[2] < 0 and 2 * s[2] * s[2] >= (s * s).sum()
        assert (p[S] == targets[i]).all()
    i = int(np.nonzero(found)[0][0])
    T = np.zeros(occ.shape, np.uint8)
    T[targets[i][2], targets[i][1], targets[i][0]] = 1
    po, fo, vo = O.reach_set(occ, sc.lengths, sc.root, T, _flat(c))
    assert fo == 1 and (poses[i] == po).all()
    got = ik.unpack_bits(vs[i].reshape(-1), sc.shape).reshape(vo.shape)
    assert (got == vo.astype(bool)).all()
