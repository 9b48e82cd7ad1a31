"""Size edge cases against the oracle, through the C ABI: segments whose
shell reach exceeds the tiled kernels' limit (the global-load propagation
runs), the largest segment count and the longest segment the ABI accepts,
and the arguments just beyond them."""
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
def test_long_segment_global_kernel(ik, masks):
    """Segment 1 of length 36 (reach 36 > 31): forward sets, survivor sets,
    reach poses and one path exact against the oracle."""
    shape = (96, 64, 48)
    sc = G.make_scene(*shape, (48, 32, 0), (36, 5, 4), 30, 2, 8, 7, "long")
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = np.concatenate([G.draw_targets(sc, 5, 8), np.asarray([sc.root], np.int32)])
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
        ik.ik_set_boxes(g.h, sc.boxes)
        F = ik.ik_forward_sets(g.h, sc.lengths, sc.root)
        pg, fg, vg = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets, want_sets=True)
        i = int(np.argmax(fg))
        path = ik.ik_plan_path(g.h, sc.lengths, pg[i], 6) if fg[i] else None
    assert (ik.unpack_bits(F, sc.shape) == O.forward(occ, sc.lengths, sc.root).astype(bool)).all()
    po, fo, vo = O.reach_many(occ, sc.lengths, sc.root, targets, want_sets=True, threads=4)
    assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
    assert (ik.unpack_bits(vg.reshape(-1), sc.shape).reshape(vo.shape) == vo.astype(bool)).all()
    assert fo.sum() > 0
    p2, r2, s2 = O.plan_path(occ, sc.lengths, po[i], 6)
    assert path[2] == s2 and (path[0] == p2).all() and (path[1] == r2).all()


def test_sixteen_segments(ik):
    """The largest segment count (16) on the 32^3 scene."""
    lengths = (3, 2, 3, 2, 2, 3, 2, 2, 3, 2, 2, 3, 2, 2, 3, 2)
    sc = G.make_scene(32, 32, 32, (16, 16, 0), lengths, 20, 2, 6, 9, "sixteen")
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 6, 10)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        pg, fg, vg = ik.ik_solve_reach_many(g.h, lengths, sc.root, targets, want_sets=True)
        out = ik.ik_reach_path_many(g.h, lengths, sc.root, targets[:2], 5)
        with pytest.raises(ik.IkError) as e:
            ik.ik_solve_reach_many(g.h, lengths + (2,), sc.root, targets)
        assert e.value.code == ik.IK_ERR_ARG
    po, fo, vo = O.reach_many(occ, lengths, sc.root, targets, want_sets=True, threads=4)
    assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
    assert (ik.unpack_bits(vg.reshape(-1), sc.shape).reshape(vo.shape) == vo.astype(bool)).all()
    for k in np.nonzero(fo[:2])[0]:
        p2, r2, s2 = O.plan_path(occ, lengths, po[k], 5)
        assert out[4][k] == s2 and (out[2][k] == p2).all()


def test_longest_segment(ik):
    """One segment of length 100 (the ABI's limit) on a free 128^3 grid: the
    forward set is every shell offset from the root that stays in the grid
    (the closed form of free space, from a numpy mesh of the shell), and a
    reach to any of them is the pose (root, target); length 101 is
    refused."""
    from bruteforce import shell_offsets
    shape = (128, 128, 128)
    root = np.array([64, 64, 10])
    lo2, hi2 = O.shell_bounds(100)
    D = shell_offsets(lo2, hi2)
    Q = D + root
    Q = Q[((Q >= 0) & (Q < 128)).all(1)]
    want = np.zeros((128, 128, 128), bool)
    want[Q[:, 2], Q[:, 1], Q[:, 0]] = True
    rng = np.random.default_rng(0)
    targets = Q[rng.integers(0, len(Q), 4)].astype(np.int32)
    with ik.Grid(*shape) as g:
        ik.ik_set_boxes(g.h, np.zeros((0, 6), np.int32))
        F = ik.ik_forward_sets(g.h, (100,), root)
        pg, fg, _ = ik.ik_solve_reach_many(g.h, (100,), root, targets)
        with pytest.raises(ik.IkError) as e:
            ik.ik_forward_sets(g.h, (101,), root)
        assert e.value.code == ik.IK_ERR_ARG
    Fb = ik.unpack_bits(F, shape)
    assert (Fb[1] == want).all() and Fb[0].sum() == 1 and Fb[0][10, 64, 64]
    assert fg.all() and (pg[:, 1] == targets).all() and (pg[:, 0] == root).all()


@pytest.mark.parametrize("masks", [1, 0])
def test_widest_rows(ik, masks):
    """Rows of 32 words (nx = 1024, the largest): the tiled kernels cannot
    stage a row plus its halo in one warp's pitch and stand aside; reach and
    survivor sets exact against the oracle on a thin 1024 x 6 x 5 grid."""
    sc = G.make_scene(1024, 6, 5, (512, 3, 0), (3, 2), 30, 1, 3, 13, "wide")
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 6, 14)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
        ik.ik_set_boxes(g.h, sc.boxes)
        F = ik.ik_forward_sets(g.h, sc.lengths, sc.root)
        pg, fg, vg = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets, want_sets=True)
    assert (ik.unpack_bits(F, sc.shape) == O.forward(occ, sc.lengths, sc.root).astype(bool)).all()
    po, fo, vo = O.reach_many(occ, sc.lengths, sc.root, targets, want_sets=True, threads=4)
    assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
    assert (ik.unpack_bits(vg.reshape(-1), sc.shape).reshape(vo.shape) == vo.astype(bool)).all()
