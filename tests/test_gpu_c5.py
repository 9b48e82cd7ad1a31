"""The 256^3 serving scene (300 static boxes and a snapshot of the 16
moving boxes) at full size, in the launch configuration the served graph
uses: the grids with and without edge masks (two independent routes through
the propagation) agree exactly on reach poses and 32-waypoint paths; sampled
poses are valid per the oracle and every step keeps to delta + m; one
waypoint's survivor sets and smooth step are exact against the oracle."""
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


def test_c5_masked_equals_maskfree_sampled_exact_and_valid(ik):
    sc, mv = G.c5_scene(3)
    for _ in range(5):
        mv.step()
    boxes = np.concatenate([sc.boxes, mv.boxes()]).astype(np.int32)
    occ = O.rasterize(sc.shape, boxes)
    targets = G.draw_targets(sc, 8, 31)
    S, W, delta = len(sc.lengths), 32, 3
    outs = []
    for masks in (1, 0):
        with ik.Grid(*sc.shape) as g:
            ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
            ik.ik_set_boxes(g.h, boxes)
            outs.append(ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, W, delta=delta))
    for a, b in zip(*outs):
        assert (a == b).all()
    reach, found, poses, relax, status = outs[0]
    assert found.sum() >= 4
    for i in np.nonzero(found)[0]:
        assert (reach[i][0] == sc.root).all() and (reach[i][S] == targets[i]).all()
        assert O.pose_valid(occ, sc.lengths, reach[i])
        assert (poses[i][W - 1] == reach[i]).all()
        for j in range(0, W, 5):
            assert O.pose_valid(occ, sc.lengths, poses[i][j])
        for j in range(W - 1):
            m = relax[i][j][0]
            if m >= 0:
                step = poses[i][j] - poses[i][j + 1]
                assert (np.sum(step * step, axis=1) <= (delta + m) ** 2).all()
    # exact: waypoint W-2 of one path, from the oracle's survivor sets
    i = int(np.nonzero(found)[0][0])
    used, vo = O.waypoint_sets_range(occ, sc.lengths, reach[i], W, W - 2, W - 1)
    assert relax[i][W - 2][1] == used[0]
    pose, m = O.smooth_step(occ, sc.lengths, vo[0], poses[i][W - 1])
    assert m == relax[i][W - 2][0] and (pose == poses[i][W - 2]).all()
