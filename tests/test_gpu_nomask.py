"""Grids without stored edge masks (segment tests walk the supercover on the
fly) give the same results, bit for bit."""
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


@pytest.mark.parametrize("seed", range(3))
def test_nomask_reach_path_replan_c1(ik, seed):
    sc = G.c1_scene(seed)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 5, 50 + seed)
    W = 8
    with _grid(ik, sc, 0) as g:
        F = ik.ik_forward_sets(g.h, sc.lengths, sc.root)
        assert (ik.unpack_bits(F, sc.shape) == O.forward(occ, sc.lengths, sc.root).astype(bool)).all()
        pg, fg, vg = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets, want_sets=True)
        po, fo, vo = O.reach_many(occ, sc.lengths, sc.root, targets, want_sets=True, threads=4)
        assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
        S = len(sc.lengths)
        assert (ik.unpack_bits(vg.reshape(-1), sc.shape).reshape(vo.shape) == vo.astype(bool)).all()
        i = int(np.argmax(fo))
        path, relax, st = ik.ik_plan_path(g.h, sc.lengths, po[i], W)
        p2, r2, s2 = O.plan_path(occ, sc.lengths, po[i], W)
        assert st == s2 and (relax == r2).all() and (path == p2).all()
        v = path[W - 3][2]
        boxes = np.concatenate([sc.boxes, [[v[0], v[1], v[2], v[0], v[1], v[2]]]]).astype(np.int32)
        ik.ik_set_boxes(g.h, boxes)
        pr, rr, sr = ik.ik_replan(g.h, sc.lengths, path, 2)
        po2, ro2, so2 = O.replan(O.rasterize(sc.shape, boxes), sc.lengths, path, 2)
        assert sr == so2 and (rr == ro2).all() and (pr == po2).all()


def test_nomask_equals_masks_on_the_128_batch(ik):
    sc = G.c2_scene(1)
    targets = G.draw_targets(sc, 8, 1)
    outs = []
    for masks in (1, 0):
        with _grid(ik, sc, masks) as g:
            outs.append(ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, 32))
    for a, b in zip(*outs):
        assert (a == b).all()


@pytest.mark.parametrize("masks", [1, 0])
def test_tile_depth_16_matches_oracle_c1(ik, masks):
    sc = G.c1_scene(6)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 4, 66)
    g = ik.Grid(*sc.shape)
    ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
    ik.ik_set_option(g.h, ik.IK_OPT_TILE_DEPTH, 16)
    ik.ik_set_boxes(g.h, sc.boxes)
    F = ik.ik_forward_sets(g.h, sc.lengths, sc.root)
    assert (ik.unpack_bits(F, sc.shape) == O.forward(occ, sc.lengths, sc.root).astype(bool)).all()
    pg, fg, vg = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets, want_sets=True)
    po, fo, vo = O.reach_many(occ, sc.lengths, sc.root, targets, want_sets=True, threads=4)
    assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
    assert (ik.unpack_bits(vg.reshape(-1), sc.shape).reshape(vo.shape) == vo.astype(bool)).all()
    i = int(np.argmax(fo))
    path, relax, st = ik.ik_plan_path(g.h, sc.lengths, po[i], 8)
    p2, r2, s2 = O.plan_path(occ, sc.lengths, po[i], 8)
    assert st == s2 and (relax == r2).all() and (path == p2).all()
    g.close()


def test_tile_depths_agree_on_the_128_batch(ik):
    sc = G.c2_scene(1)
    targets = G.draw_targets(sc, 8, 3)
    outs = []
    for depth in (8, 16):
        with ik.Grid(*sc.shape) as g:
            ik.ik_set_option(g.h, ik.IK_OPT_TILE_DEPTH, depth)
            ik.ik_set_boxes(g.h, sc.boxes)
            outs.append(ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, 32))
            outs.append(ik.ik_forward_sets(g.h, sc.lengths, sc.root))
    for a, b in zip(outs[:2], outs[2:]):
        for x, y in zip(a if isinstance(a, tuple) else (a,), b if isinstance(b, tuple) else (b,)):
            assert (x == y).all()
