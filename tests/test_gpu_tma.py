"""Edge masks with the occupancy brick staged by a TMA tensor copy (grids
whose rows are a multiple of 16 bytes): exact against the oracle on a
non-cubic grid, and identical to the per-thread staging on the 128^3
workload."""
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


def test_tma_masks_exact_on_a_ragged_128_wide_grid(ik):
    shape = (128, 40, 36)
    lengths = (8, 7, 6, 5)
    root = (70, 20, 3)
    rng = np.random.default_rng(17)
    boxes = []
    while len(boxes) < 60:
        c = rng.integers(0, shape)
        sd = rng.integers(2, 7, 3)
        b = [int(c[0]), int(c[1]), int(c[2]), int(c[0] + sd[0] - 1), int(c[1] + sd[1] - 1), int(c[2] + sd[2] - 1)]
        if all(b[a] <= root[a] <= b[a + 3] for a in range(3)):
            continue
        boxes.append(b)
    boxes = np.asarray(boxes, np.int32)
    occ = O.rasterize(shape, boxes)
    free = np.argwhere(occ == 0)[:, ::-1]
    targets = free[rng.integers(len(free), size=6)].astype(np.int32)
    Fo = O.forward(occ, lengths, root)
    po, fo, _ = O.reach_many(occ, lengths, root, targets, threads=6)
    for tma in (1, 0):
        with ik.Grid(*shape) as g:
            ik.ik_set_option(g.h, ik.IK_OPT_TMA_MASKS, tma)
            ik.ik_set_boxes(g.h, boxes)
            F = ik.ik_forward_sets(g.h, lengths, root)
            pg, fg, _ = ik.ik_solve_reach_many(g.h, lengths, root, targets)
        assert (ik.unpack_bits(F, shape) == Fo.astype(bool)).all(), tma
        assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all(), tma


def test_tma_masks_equal_plain_staging_128(ik):
    sc = G.c2_scene(1)
    targets = G.draw_targets(sc, 8, 1)
    outs = []
    for tma in (1, 0):
        with ik.Grid(*sc.shape) as g:
            ik.ik_set_option(g.h, ik.IK_OPT_TMA_MASKS, tma)
            ik.ik_set_boxes(g.h, sc.boxes)
            outs.append(ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, 16))
    for a, b in zip(*outs):
        assert (a == b).all()
