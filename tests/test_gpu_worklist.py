"""The batched backward pass gives the same sets whichever way it visits the
tiles of a level: one block per (tile, query), or a work list of the tiles
the level's bounding boxes reach (IK_OPT_WORK_LIST 0, 1 and 2)."""
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


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("masks", [1, 0])
def test_work_list_reach_sets_match_oracle_c1(ik, mode, masks):
    sc = G.c1_scene(2)
    occ = O.rasterize(sc.shape, sc.boxes)
    # 24 queries: the batched pass takes the work list from 16 queries up
    targets = G.draw_targets(sc, 24, 71)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
        ik.ik_set_option(g.h, ik.IK_OPT_WORK_LIST, mode)
        ik.ik_set_boxes(g.h, sc.boxes)
        pg, fg, vg = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets, want_sets=True)
    po, fo, vo = O.reach_many(occ, sc.lengths, sc.root, targets, want_sets=True, threads=4)
    assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
    assert (ik.unpack_bits(vg.reshape(-1), sc.shape).reshape(vo.shape) == vo.astype(bool)).all()


@pytest.mark.parametrize("masks", [1, 0])
def test_work_list_modes_agree_on_the_128_batch(ik, masks):
    sc = G.c2_scene(1)
    targets = G.draw_targets(sc, 8, 5)
    outs = []
    for mode in (0, 1, 2):
        with ik.Grid(*sc.shape) as g:
            ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
            ik.ik_set_option(g.h, ik.IK_OPT_WORK_LIST, mode)
            ik.ik_set_boxes(g.h, sc.boxes)
            outs.append(ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, 32))
    for other in outs[1:]:
        for x, y in zip(outs[0], other):
            assert (np.asarray(x) == np.asarray(y)).all()


def test_work_list_option_range(ik):
    with ik.Grid(32, 32, 32) as g:
        for bad in (-1, 3):
            with pytest.raises(Exception):
                ik.ik_set_option(g.h, ik.IK_OPT_WORK_LIST, bad)
