"""Every form of the two-query propagation (IK_OPT_QUERY_PAIRS 0, 1 and 2,
with row lanes off so that they run) gives the oracle's sets, with and
without edge masks and with approach cones, and the same batched results
at 128^3, where form 2 (rows staged without pad words, the bits read across
a row's end masked off per offset) reads across row ends on every grid
edge."""
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


def _grid(ik, sc, pairs, masks=1):
    g = ik.Grid(*sc.shape)
    ik.ik_set_option(g.h, ik.IK_OPT_ROW_LANES, 0)
    ik.ik_set_option(g.h, ik.IK_OPT_WORK_LIST, 0)
    ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
    ik.ik_set_option(g.h, ik.IK_OPT_QUERY_PAIRS, pairs)
    ik.ik_set_boxes(g.h, sc.boxes)
    return g


@pytest.mark.parametrize("pairs", [0, 1, 2])
@pytest.mark.parametrize("masks", [1, 0])
def test_pair_forms_match_oracle_c1(ik, pairs, masks):
    sc = G.c1_scene(4)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 7, 41)  # an odd count: the last block carries one query
    po, fo, vo = O.reach_many(occ, sc.lengths, sc.root, targets, want_sets=True, threads=4)
    with _grid(ik, sc, pairs, masks) as g:
        pg, fg, vg = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets, want_sets=True)
    S = len(sc.lengths)
    assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
    got = ik.unpack_bits(vg.reshape(-1), sc.shape).reshape((-1, S + 1) + tuple(sc.shape[::-1]))
    assert (got == vo.astype(bool)).all()


@pytest.mark.parametrize("pairs", [1, 2])
def test_pair_forms_cone_reach_match_oracle_c1(ik, pairs):
    sc = G.c1_scene(5)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 5, 52)
    cone = ((0, 0, -1), 1, 2)
    with _grid(ik, sc, pairs) as g:
        poses, found, vs = ik.ik_solve_reach_many_cone(g.h, sc.lengths, ik.cone(*cone), sc.root, targets,
                                                      want_sets=True)
    for i, t in enumerate(targets):
        T = np.zeros(occ.shape, np.uint8)
        T[t[2], t[1], t[0]] = 1
        po, fo, vo = O.reach_set(occ, sc.lengths, sc.root, T, (*cone[0], cone[1], cone[2]))
        assert found[i] == fo, i
        if fo:
            assert (poses[i] == po).all(), i
        got = ik.unpack_bits(vs[i].reshape(-1), sc.shape).reshape(vo.shape)
        assert (got == vo.astype(bool)).all(), i


def test_pair_forms_agree_on_the_128_batch_and_cones(ik):
    sc = G.c2_scene(1)
    targets = G.draw_targets(sc, 16, 5)
    cone = ((0, 0, -1), 1, 2)
    outs = []
    for pairs in (1, 2):
        with _grid(ik, sc, pairs) as g:
            r = list(ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets[:8], 32))
            r += list(ik.ik_solve_reach_many_cone(g.h, sc.lengths, ik.cone(*cone), sc.root, targets,
                                                  want_sets=True))
            outs.append(r)
    for a, b in zip(*outs):
        assert (np.asarray(a) == np.asarray(b)).all()
