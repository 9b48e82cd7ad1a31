"""The continuous-batching server: every result is the same alone and in the
mix (same input, same tick snapshot), and it follows the direct calls."""
import copy

import numpy as np
import pytest

import scenegen as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    from paper_1906_10678_b300 import build
    build.build()
    from paper_1906_10678_b300 import serve as mod
    return mod


def _server(serve, sc):
    mv = G.make_moving_boxes(sc.shape, 4, 3, side_lo=2, side_hi=5)
    return serve.Server(sc.shape, sc.root, sc.lengths, sc.boxes, mv, n_way=8, tick_s=1 / 12,
                        slots_path=6, slots_replan=6)


def _fresh(r):
    q = copy.copy(r)
    q.tick, q.done, q.status, q.poses, q.relax = -1, -1.0, -1, None, None
    q.arrival = 0.0
    return q


@pytest.mark.parametrize("within", [False, True])
def test_results_same_alone_and_in_the_mix(serve, within):
    """Served at tick starts only (within=False: every tick's arrivals in one
    batch with the snapshot rebuild) or also within ticks (within=True: each
    arrival solved on arrival against the tick's snapshot, without a
    rebuild), every result equals the same request served alone at its
    tick's start, and a direct call on the tick's snapshot."""
    from paper_1906_10678_b300 import ik
    sc = G.c1_scene(0)
    reqs = serve.make_requests(sc, 120.0, 1.0, 5)
    a = _server(serve, sc)
    a.serve(reqs, 1.0, realtime=False, within=within)
    done = [r for r in a.finished if r.poses is not None]
    paths = [r for r in done if r.kind == "path"]
    replans = [r for r in done if r.kind == "replan"]
    assert len(paths) >= 6 and len(replans) >= 3
    assert max(len([r for r in done if r.tick == t]) for t in range(1, a.tick + 1)) >= 3
    if within:
        assert len(a.within_ms) > 0  # some requests were admitted within a tick
    a.close()
    for r in paths[:3] + replans[:3]:
        b = _server(serve, sc)
        for _ in range(r.tick - 1):
            b.run_tick(0.0)
        q = _fresh(r)
        if r.kind == "replan":
            b.live[r.path_id] = serve.LivePath(r.input_poses.copy(), r.tick - r.current)
        b.pending.append(q)
        b.run_tick(0.0)
        assert q.tick == r.tick and q.status == r.status, r.kind
        assert (q.poses == r.poses).all() and (q.relax == r.relax).all(), r.kind
        if r.kind == "path":
            # and it equals a direct call on the tick's snapshot
            with ik.Grid(*sc.shape) as g:
                ik.ik_set_boxes(g.h, b._boxes())
                _, found, poses, relax, status = ik.ik_reach_path_many(
                    g.h, sc.lengths, sc.root, np.asarray([r.target], np.int32), 8)
            assert status[0] == r.status and (poses[0] == r.poses).all()
        b.close()
