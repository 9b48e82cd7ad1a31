"""Per-segment direction limits (section "The procedure for IK solution",
Step 1 (a); the first segment restricted to the upper hemisphere, section "The
gap in gMS") against the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
import scenegen as G

pytestmark = pytest.mark.gpu

LIMITS = [
    [(0, 0, 1, 0, 1), None, None, None],
    [(0, 0, 1, 1, 4), (1, 0, 0, 0, 1), None, (0, 0, -1, 0, 1)],
    [None, (0, 1, 1, 1, 3), (-1, 0, 1, 1, 5), None],
]


@pytest.fixture(scope="module")
def ik():
    from paper_1906_10678_b300 import build
    build.build()
    from paper_1906_10678_b300 import ik as mod
    return mod


def _ik_limits(lim):
    return [None if c is None else (c[:3], c[3], c[4]) for c in lim]


@pytest.mark.parametrize("masks", [1, 0])
@pytest.mark.parametrize("li", range(len(LIMITS)))
def test_limited_forward_and_reach_match_oracle(ik, li, masks):
    sc = G.c1_scene(30 + li)
    occ = O.rasterize(sc.shape, sc.boxes)
    lim = LIMITS[li]
    targets = G.draw_targets(sc, 6, 40 + li)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
        ik.ik_set_boxes(g.h, sc.boxes)
        ik.ik_set_segment_limits(g.h, sc.lengths, _ik_limits(lim))
        F = ik.ik_forward_sets(g.h, sc.lengths, sc.root)
        pg, fg, vg = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets, want_sets=True)
    Fo = O.forward(occ, sc.lengths, sc.root, limits=lim)
    assert (ik.unpack_bits(F, sc.shape) == Fo.astype(bool)).all()
    po, fo, vo = O.reach_many(occ, sc.lengths, sc.root, targets, want_sets=True, threads=4, limits=lim)
    assert (fg == fo).all() and (pg[fo == 1] == po[fo == 1]).all()
    assert (ik.unpack_bits(vg.reshape(-1), sc.shape).reshape(vo.shape) == vo.astype(bool)).all()


@pytest.mark.parametrize("li", range(len(LIMITS)))
def test_limited_paths_and_validation_match_oracle(ik, li):
    sc = G.c1_scene(40 + li)
    occ = O.rasterize(sc.shape, sc.boxes)
    lim = LIMITS[li]
    targets = G.draw_targets(sc, 8, 50 + li)
    W = 6
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        plain = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets)
        ik.ik_set_segment_limits(g.h, sc.lengths, _ik_limits(lim))
        out = ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, W)
        # unlimited reach poses, validated under the limits
        valid = ik.ik_validate_poses(g.h, sc.lengths, plain[0][plain[1] == 1])
        ik.ik_set_segment_limits(g.h, sc.lengths, None)
        again = ik.ik_solve_reach_many(g.h, sc.lengths, sc.root, targets)
    for a, b in zip(again[:2], plain[:2]):
        assert (a == b).all()  # clearing the limits restores the plain results
    want_valid = [O.pose_valid(occ, sc.lengths, p, limits=lim) for p in plain[0][plain[1] == 1]]
    assert list(valid.astype(bool)) == want_valid
    po, fo, _ = O.reach_many(occ, sc.lengths, sc.root, targets, threads=4, limits=lim)
    assert (out[1] == fo).all()
    for i in np.nonzero(fo)[0]:
        p2, r2, s2 = O.plan_path(occ, sc.lengths, po[i], W, limits=lim)
        assert out[4][i] == s2 and (out[2][i] == p2).all() and (out[3][i] == r2).all()


def test_limited_batch_replay_and_cone_conflict(ik):
    import torch
    torch.cuda.set_device(0)
    sc = G.c1_scene(7)
    lim = LIMITS[1]
    n, W, S = 4, 6, len(sc.lengths)
    stream = torch.cuda.Stream()
    g = ik.Grid(*sc.shape, stream=stream.cuda_stream)
    ik.ik_set_segment_limits(g.h, sc.lengths, _ik_limits(lim))
    boxes = torch.from_numpy(sc.boxes.copy()).cuda()
    t_np = G.draw_targets(sc, n, 12)
    targets = torch.from_numpy(t_np.copy()).cuda()
    outs = [torch.zeros(sz, dtype=torch.int32, device="cuda")
            for sz in ((n, S + 1, 3), (n,), (n, W, S + 1, 3), (n, W, 2), (n,))]
    b = ik.Batch(g.h, sc.lengths, sc.root, boxes, targets, W, *outs)
    moved = sc.boxes.copy()
    moved[:5, [0, 3]] += 1
    boxes.copy_(torch.from_numpy(moved))
    b.launch()
    stream.synchronize()
    got = [o.cpu().numpy() for o in outs]
    with pytest.raises(ik.IkError) as e:  # the last segment is limited: no approach cone on top
        ik.ik_solve_reach_many_cone(g.h, sc.lengths, ik.cone((0, 0, -1), 1, 2), sc.root, t_np)
    assert e.value.code == ik.IK_ERR_ARG
    b.close()
    g.close()
    occ = O.rasterize(sc.shape, moved)
    po, fo, _ = O.reach_many(occ, sc.lengths, sc.root, t_np, threads=4, limits=lim)
    assert (got[1] == fo).all() and (got[0][fo == 1] == po[fo == 1]).all()
    for i in np.nonzero(fo)[0]:
        p2, r2, s2 = O.plan_path(occ, sc.lengths, po[i], W, limits=lim)
        assert got[4][i] == s2 and (got[2][i] == p2).all()
