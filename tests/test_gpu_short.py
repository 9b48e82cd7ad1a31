"""Short reaches: the shortcut (virtual arm, its pose) and the path along it
equal the oracle's, bit for bit."""
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


def _near_targets(sc, occ, n, seed, r2=100):
    """Free voxels within sqrt(r2) of the root, seeded."""
    free = np.argwhere(occ == 0)[:, ::-1]
    d2 = ((free - np.array(sc.root)) ** 2).sum(axis=1)
    near = free[(d2 <= r2) & (d2 > 0)]
    rng = np.random.default_rng(seed)
    return near[rng.choice(len(near), min(n, len(near)), replace=False)].astype(np.int32)


@pytest.mark.parametrize("masks", [1, 0])
@pytest.mark.parametrize("seed", range(3))
def test_short_matches_oracle_c1(ik, seed, masks):
    sc = G.c1_scene(seed)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = _near_targets(sc, occ, 6, 80 + seed)
    poses, found, _ = O.reach_many(occ, sc.lengths, sc.root, targets, threads=4)
    W = 8
    n_short = 0
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_option(g.h, ik.IK_OPT_EDGE_MASKS, masks)
        ik.ik_set_boxes(g.h, sc.boxes)
        for i in np.nonzero(found)[0][:3]:
            pg, rg, sg, klg, vg = ik.ik_plan_path_short(g.h, sc.lengths, poses[i], W)
            po, ro, so, klo, vo = O.plan_short(occ, sc.lengths, poses[i], W)
            assert klg == klo
            assert (vg is None) == (vo is None)
            if vo is not None:
                assert (vg == vo).all()
                n_short += 1
            assert sg == so and (rg == ro).all() and (pg == po).all()
    assert n_short > 0


def test_short_falls_back_and_refuses(ik):
    sc = G.c1_scene(0)
    occ = O.rasterize(sc.shape, sc.boxes)
    S = len(sc.lengths)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        # a far target: no shortened arm of at most two segments reaches it
        t = G.draw_targets(sc, 6, 9)
        poses, found, _ = O.reach_many(occ, sc.lengths, sc.root, t, threads=4)
        for i in np.nonzero(found)[0][:2]:
            po, ro, so, klo, _ = O.plan_short(occ, sc.lengths, poses[i], 6)
            pg, rg, sg, klg, vg = ik.ik_plan_path_short(g.h, sc.lengths, poses[i], 6)
            assert klg == klo and sg == so and (rg == ro).all() and (pg == po).all()
            if klo == (0, 0):
                pp, rp, sp = ik.ik_plan_path(g.h, sc.lengths, poses[i], 6)
                assert (pp == pg).all() and (rp == rg).all() and sp == sg
        bad = np.zeros((S + 1, 3), np.int32)
        _, _, st, kl, _ = ik.ik_plan_path_short(g.h, sc.lengths, bad, 6)
        assert st == ik.IK_PATH_UNREACHABLE and kl == (0, 0)
        reach = poses[int(np.nonzero(found)[0][0])]
        for kmax in (0, S + 1):
            with pytest.raises(ik.IkError) as e:
                ik.ik_plan_path_short(g.h, sc.lengths, reach, 6, k_max=kmax)
            assert e.value.code == ik.IK_ERR_ARG
