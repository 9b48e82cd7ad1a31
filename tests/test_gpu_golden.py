"""Full-size parity against the oracle's stored outputs (tests/golden/full_*.npz,
written by tests/golden/make_full_size.py, which calls only the oracle).

Each workload runs in the launch configuration the benchmark times:

* 128^3 (64 targets, 32-waypoint paths): the whole 64 x 32 batch through
  ik_reach_path_many (the library's defaults: row lanes with two queries
  per lane, row-lane edge masks, the work list on the sparsest levels);
  every reach pose and found flag, and the poses, relaxation records and
  status of 16 whole paths, element by element; and, for 4 paths at 5
  waypoints, every survivor set V_k^(j) compared by its SHA-256 over the
  packed bits (and its popcount) -- the oracle's byte sets packed the way
  the library packs words.
* the uneven batch: the first 32 problems of the 1024-problem batch, solved
  inside the full batch by the persistent launch (waypoint items in query
  pairs), element by element.
* 256^3 (the serving scene after 5 ticks of the moving boxes): 8 reach poses
  and 2 whole paths, through a direct call and through the captured graph
  the server replays.
"""
import hashlib
import os

import numpy as np
import pytest

import scenegen as G

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ik():
    from paper_1906_10678_b300 import build
    build.build()
    from paper_1906_10678_b300 import ik as mod
    return mod


def _load(name):
    return dict(np.load(os.path.join(GOLDEN, name)))


def test_c3_batch_reach_and_paths_exact(ik):
    gold = _load("full_c3.npz")
    sc = G.c2_scene(1)
    targets = G.draw_targets(sc, 64, 1)
    assert (targets == gold["targets"]).all()
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        reach, found, poses, relax, status = ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, 32)
    assert (found == gold["found"]).all()
    f = gold["found"] == 1
    assert (reach[f] == gold["reach"][f]).all()
    for n, i in enumerate(gold["path_targets"]):
        assert status[i] == gold["status"][n], i
        assert (relax[i] == gold["relax"][n]).all(), i
        assert (poses[i] == gold["poses"][n]).all(), i


def test_c3_waypoint_survivor_sets_exact(ik):
    gold = _load("full_c3.npz")
    sc = G.c2_scene(1)
    S = len(sc.lengths)
    with ik.Grid(*sc.shape) as g:
        ik.ik_set_boxes(g.h, sc.boxes)
        for a, i in enumerate(gold["set_targets"]):
            used, vs = ik.ik_waypoint_sets(g.h, sc.lengths, gold["reach"][i], 32)
            for b, j in enumerate(gold["set_ways"]):
                assert used[j] == gold["set_used"][a][b], (i, j)
                for k in range(S + 1):
                    words = np.ascontiguousarray(vs[j][k]).astype("<u4")
                    assert int(np.unpackbits(words.view(np.uint8)).sum()) == int(gold["set_pop"][a][b][k]), \
                        (i, j, k)
                    h = hashlib.sha256(words.tobytes()).hexdigest().encode()
                    assert h == gold["set_hash"][a][b][k], (i, j, k)


def _as_dict(p):
    return {"shape": p.scene.shape, "boxes": p.scene.boxes, "lengths": p.scene.lengths,
            "root": p.scene.root, "target": p.target, "n_way": p.n_way}


def test_c4_uneven_batch_exact(ik):
    gold = _load("full_c4.npz")
    probs = G.c4_problems(1024, 2)
    out, _ = ik.ik_solve_batch([_as_dict(p) for p in probs])
    n = len(gold["found"])
    for i in range(n):
        S, W = len(probs[i].scene.lengths), probs[i].n_way
        r = out[i]
        assert r["found"] == gold["found"][i], i
        assert r["status"] == gold["status"][i], i
        if gold["found"][i]:
            assert (r["reach"] == gold["reach"][i][:S + 1]).all(), i
            assert (r["poses"] == gold["poses"][i][:W, :S + 1]).all(), i
            assert (r["relax"] == gold["relax"][i][:W]).all(), i


def test_c5_snapshot_reach_and_paths_exact_direct_and_captured(ik):
    import torch
    gold = _load("full_c5.npz")
    sc, mv = G.c5_scene(3)
    for _ in range(5):
        mv.step()
    boxes = np.concatenate([sc.boxes, mv.boxes()]).astype(np.int32)
    targets = G.draw_targets(sc, 8, 31)
    assert (targets == gold["targets"]).all()
    S, W = len(sc.lengths), 32
    f = gold["found"] == 1
    stream = torch.cuda.Stream()  # a captured graph needs a stream of its own
    with ik.Grid(*sc.shape, stream=stream.cuda_stream) as g:
        ik.ik_set_boxes(g.h, boxes)
        reach, found, poses, relax, status = ik.ik_reach_path_many(g.h, sc.lengths, sc.root, targets, W)
        assert (found == gold["found"]).all() and (reach[f] == gold["reach"][f]).all()
        for n, i in enumerate(gold["path_targets"]):
            assert status[i] == gold["status"][n] and (relax[i] == gold["relax"][n]).all()
            assert (poses[i] == gold["poses"][n]).all()
        # the server's captured graph on the same snapshot
        dev = torch.device("cuda", torch.cuda.current_device())
        i32 = dict(dtype=torch.int32, device=dev)
        boxes_d = torch.from_numpy(boxes).to(dev)
        targets_d = torch.from_numpy(targets.copy()).to(dev)
        outs = [torch.zeros((8, S + 1, 3), **i32), torch.zeros(8, **i32), torch.zeros((8, W, S + 1, 3), **i32),
                torch.zeros((8, W, 2), **i32), torch.zeros(8, **i32)]
        b = ik.Batch(g.h, sc.lengths, sc.root, boxes_d, targets_d, W, *outs)
        b.launch()
        stream.synchronize()
        creach, cfound, cposes, crelax, cstatus = (t.cpu().numpy() for t in outs)
        b.close()
    assert (cfound == gold["found"]).all() and (creach[f] == gold["reach"][f]).all()
    for n, i in enumerate(gold["path_targets"]):
        assert cstatus[i] == gold["status"][n] and (crelax[i] == gold["relax"][n]).all()
        assert (cposes[i] == gold["poses"][n]).all()
