"""Obstacle dilation (section "Testing for collisions": obstacle volumes
dilated for the arm's thickness and a clearance margin) against the oracle,
through the C ABI."""
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


@pytest.mark.parametrize("r2", [1, 2, 3, 5])
def test_dilated_occupancy_and_reach_match_oracle(ik, r2):
    sc = G.c1_scene(20 + r2)
    raw = O.rasterize(sc.shape, sc.boxes)
    dil = O.dilate(raw, r2)
    targets = G.draw_targets(sc, 6, 7)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_option(g.h, ik.IK_OPT_DILATE_R2, r2)
        ik.ik_set_boxes(g.h, sc.boxes)
        occ = ik.unpack_bits(ik.ik_get_obstacles(g.h), sc.shape)
        assert (occ == dil.astype(bool)).all()
        pg, fg, vg = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets, want_sets=True)
        path = ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, 6)
    po, fo, vo = O.reach_many(dil, sc.lengths, sc.root, targets, want_sets=True, threads=4)
    assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
    assert (ik.unpack_bits(vg.reshape(-1), sc.shape).reshape(vo.shape) == vo.astype(bool)).all()
    for i in np.nonzero(fo)[0]:
        p2, r2_, s2 = O.plan_path(dil, sc.lengths, po[i], 6)
        assert path[4][i] == s2 and (path[2][i] == p2).all() and (path[3][i] == r2_).all()


def test_dilation_of_set_obstacles_and_option_changes(ik):
    sc = G.c1_scene(3)
    raw = O.rasterize(sc.shape, sc.boxes)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_obstacles(g.h, ik.pack_bits(raw))
        ik.ik_set_option(g.h, ik.IK_OPT_DILATE_R2, 2)  # re-dilates the current occupancy
        got = ik.unpack_bits(ik.ik_get_obstacles(g.h), sc.shape)
        assert (got == O.dilate(raw, 2).astype(bool)).all()
        ik.ik_set_option(g.h, ik.IK_OPT_DILATE_R2, 0)
        got = ik.unpack_bits(ik.ik_get_obstacles(g.h), sc.shape)
        assert (got == raw.astype(bool)).all()
        for bad in (-1, 101):
            with pytest.raises(ik.IkError) as e:
                ik.ik_set_option(g.h, ik.IK_OPT_DILATE_R2, bad)
            assert e.value.code == ik.IK_ERR_ARG


def test_captured_batch_dilates_each_replay(ik):
    import torch
    torch.cuda.set_device(0)
    sc = G.c1_scene(8)
    n, W, S = 4, 6, len(sc.lengths)
    stream = torch.cuda.Stream()
    g = ik.Grid(*sc.shape, stream=stream.cuda_stream)
    ik.ik_set_option(g.h, ik.IK_OPT_DILATE_R2, 1)
    boxes = torch.from_numpy(sc.boxes.copy()).cuda()
    t_np = G.draw_targets(sc, n, 9)
    targets = torch.from_numpy(t_np.copy()).cuda()
    outs = [torch.zeros(sz, dtype=torch.int32, device="cuda")
            for sz in ((n, S + 1, 3), (n,), (n, W, S + 1, 3), (n, W, 2), (n,))]
    b = ik.Batch(g.h, sc.lengths, sc.root, boxes, targets, W, *outs)
    moved = sc.boxes.copy()
    moved[:4, [1, 4]] += 1
    boxes.copy_(torch.from_numpy(moved))
    b.launch()
    stream.synchronize()
    got = [o.cpu().numpy() for o in outs]
    b.close()
    g.close()
    dil = O.dilate(O.rasterize(sc.shape, moved), 1)
    po, fo, _ = O.reach_many(dil, sc.lengths, sc.root, t_np, threads=4)
    assert (got[1] == fo).all() and (got[0][fo == 1] == po[fo == 1]).all()
    for i in np.nonzero(fo)[0]:
        p2, r2_, s2 = O.plan_path(dil, sc.lengths, po[i], W)
        assert got[4][i] == s2 and (got[2][i] == p2).all()
