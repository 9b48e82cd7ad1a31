"""Host logic of the continuous-batching server (no GPU): the seeded request
stream and the latency summary."""
import numpy as np

import oracle as O
import scenegen as G


def _serve():
    from paper_1906_10678_b300 import build
    build.build()
    from paper_1906_10678_b300 import serve
    return serve


def test_request_stream_is_seeded_and_well_formed():
    serve = _serve()
    sc = G.c1_scene(0)
    occ = O.rasterize(sc.shape, sc.boxes)
    a = serve.make_requests(sc, 200.0, 2.0, 5)
    b = serve.make_requests(sc, 200.0, 2.0, 5)
    assert [(r.kind, r.arrival, r.target, r.path_id) for r in a] == \
           [(r.kind, r.arrival, r.target, r.path_id) for r in b]
    assert len(a) > 100
    arrivals = [r.arrival for r in a]
    assert arrivals == sorted(arrivals) and 0.0 <= arrivals[0] and arrivals[-1] < 2.0
    paths = set()
    for r in a:
        if r.kind == "path":
            x, y, z = r.target
            assert 0 <= x < sc.shape[0] and 0 <= y < sc.shape[1] and 0 <= z < sc.shape[2]
            assert occ[z, y, x] == 0
            paths.add(r.rid)
        else:
            assert r.kind == "replan" and r.path_id in paths  # an earlier path request
    n_path = sum(r.kind == "path" for r in a)
    assert 0.3 < n_path / len(a) < 0.7


def test_latency_summary():
    serve = _serve()
    reqs = [serve.Request(i, "path", arrival=0.0, done=(i + 1) / 1000.0) for i in range(100)]
    reqs.append(serve.Request(100, "path", arrival=0.0))  # not done: left out
    st = serve.latency_stats(reqs)
    assert st["n"] == 100
    assert st["p50_ms"] == float(np.percentile(np.arange(1, 101), 50))
    assert st["p99_ms"] == round(float(np.percentile(np.arange(1, 101), 99)), 3)
    assert serve.latency_stats([]) == {"n": 0}


def test_tuner_cache_keys_and_missing_file(tmp_path):
    from paper_1906_10678_b300 import build
    build.build()
    from paper_1906_10678_b300 import tune
    assert tune.load(str(tmp_path / "absent.json")) == {}
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert tune.load(str(bad)) == {}
    k1 = tune._key((128, 128, 128), [20, 18], 64, 32)
    assert k1 == "128x128x128|20,18|64|32|v3"
    assert k1 != tune._key((128, 128, 128), [20, 18], 64, 16)
    good = tmp_path / "good.json"
    good.write_text('{"%s": {"depth": 8, "pairs": 1, "rows": 1, "tma": 0, "ms": {"depth8_pairs1_rows1_tma0": 1.0}}}'
                    % k1)
    got = tune.load(str(good))[k1]
    assert got["depth"] == 8 and got["pairs"] == 1 and got["rows"] == 1 and got["tma"] == 0
