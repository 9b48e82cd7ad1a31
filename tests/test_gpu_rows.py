"""The row-lane propagation (IK_OPT_ROW_LANES: a lane owns a whole row of 1,
2 or 4 words) gives the oracle's sets, and the same results as the other
forms, on full and ragged tiles (ny not a multiple of 32, nz not a multiple
of 8), with one query per block and with two, with edge masks over whole
rows and over part of them."""
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


def _sets(ik, vg, shape, S):
    return ik.unpack_bits(vg.reshape(-1), shape).reshape((-1, S + 1) + tuple(shape[::-1]))


@pytest.mark.parametrize("rows", [1, 0])
@pytest.mark.parametrize("shape,lengths,n_t,seed", [((32, 32, 32), (8, 7, 6, 5), 24, 11),
                                                     ((64, 40, 21), (9, 7, 5), 6, 12),
                                                     ((128, 36, 10), (6, 5, 4), 5, 13),
                                                     ((32, 9, 31), (3, 8), 3, 14)])
def test_row_lanes_reach_sets_match_oracle(ik, rows, shape, lengths, n_t, seed):
    root = (shape[0] // 2, shape[1] // 2, 0)
    sc = G.make_scene(*shape, root, lengths, 25, 2, 6, seed)
    occ = O.rasterize(shape, sc.boxes)
    targets = G.draw_targets(sc, n_t, seed)
    po, fo, vo = O.reach_many(occ, lengths, root, targets, want_sets=True, threads=4)
    with ik.Grid(*shape) as g:
        ik.ik_set_option(g.h, ik.IK_OPT_ROW_LANES, rows)
        ik.ik_set_option(g.h, ik.IK_OPT_WORK_LIST, 0)  # every level one block per tile
        ik.ik_set_boxes(g.h, sc.boxes)
        pg, fg, vg = ik.ik_solve_reach_many(g.h, lengths, root, targets, want_sets=True)
        F = ik.ik_forward_sets(g.h, lengths, root)
        # one query at a time too (one query per block)
        p1, f1, _ = ik.ik_solve_reach(g.h, lengths, root, targets[0])
    assert (ik.unpack_bits(F, shape) == O.forward(occ, lengths, root).astype(bool)).all()
    assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
    assert (_sets(ik, vg, shape, len(lengths)) == vo.astype(bool)).all()
    assert f1 == fo[0] and (not f1 or (p1 == po[0]).all())


@pytest.mark.parametrize("pairs", [1, 0])
def test_row_lanes_waypoint_sets_and_paths_match_oracle_c1(ik, pairs):
    sc = G.c1_scene(6)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 4, 6)
    po, fo, _ = O.reach_many(occ, sc.lengths, sc.root, targets)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_option(g.h, ik.IK_OPT_QUERY_PAIRS, pairs)
        ik.ik_set_boxes(g.h, sc.boxes)
        for i in np.nonzero(fo)[0][:2]:
            used, vs = ik.ik_waypoint_sets(g.h, sc.lengths, po[i], 5)
            uo, vo = O.waypoint_sets(occ, sc.lengths, po[i], 5)
            assert (np.asarray(used) == np.asarray(uo)).all()
            got = ik.unpack_bits(np.asarray(vs).reshape(-1), sc.shape).reshape(np.asarray(vo).shape)
            assert (got == np.asarray(vo).astype(bool)).all()
            poses, relax, st = ik.ik_plan_path(g.h, sc.lengths, po[i], 5)
            oposes, orelax, ost = O.plan_path(occ, sc.lengths, po[i], 5)
            assert st == ost and (poses == oposes).all() and (relax == orelax).all()


@pytest.mark.parametrize("work_list", [0, 1])
def test_row_lanes_equal_other_forms_on_the_128_batch(ik, work_list):
    sc = G.c2_scene(1)
    targets = G.draw_targets(sc, 8, 9)
    outs = []
    for rows in (1, 0):
        with ik.Grid(*sc.shape) as g:
            ik.ik_set_option(g.h, ik.IK_OPT_ROW_LANES, rows)
            ik.ik_set_option(g.h, ik.IK_OPT_WORK_LIST, work_list)
            ik.ik_set_boxes(g.h, sc.boxes)
            outs.append(ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, 32))
    for x, y in zip(*outs):
        assert (np.asarray(x) == np.asarray(y)).all()


def test_row_lanes_option_range(ik):
    with ik.Grid(32, 32, 32) as g:
        for ok in (0, 1):
            ik.ik_set_option(g.h, ik.IK_OPT_ROW_LANES, ok)
        for bad in (-1, 2):
            with pytest.raises(Exception):
                ik.ik_set_option(g.h, ik.IK_OPT_ROW_LANES, bad)
