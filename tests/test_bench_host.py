"""Host arithmetic of the benchmark (no GPU): the roofline fractions are
reproducible from the kernel counters and the probed peaks, and the oracle
sample's unit is stated."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _entry(ms, launches, visited=0, nonzero=0, mask_words=0):
    return {"ms": ms, "launches": launches, "visited": visited, "nonzero": nonzero, "mask_words": mask_words}


def test_roofline_fractions_from_counters():
    b = _bench()
    peaks = {"lop3": {"per_s": 19.2e12, "sm_mhz": 2032.0}, "shf": {"per_s": 19.0e12, "sm_mhz": 2032.0},
             "lds": {"per_s": 9.6e12, "sm_mhz": 2032.0}}
    prof = {"propagate_backward_waypoints": _entry(54.0, 8), "propagate_forward": _entry(1.3, 8),
            "propagate_backward_reach": _entry(2.5, 8), "edge_masks": _entry(5.8, 8),
            "smooth_chain": _entry(13.3, 1), "rasterize": _entry(0.03, 1)}
    work = {"way_k1": _entry(0, 0, 10e9, 4e9, 1e9), "way_k2": _entry(0, 0, 30e9, 6e9, 2e9),
            "propagate_forward": _entry(0, 0, 100e6, 50e6, 5e6), "propagate_backward_reach": _entry(0, 0, 60e6, 20e6, 3e6),
            "edge_masks": _entry(0, 0, 4e8, 9.7e9), "smooth_chain": _entry(0, 0, 150e6, 70e6)}
    for k in ("way_k3", "way_k4", "way_k5", "way_k6", "way_k7", "way_k8"):
        work[k] = _entry(0, 0, 0, 0, 0)
    r = b.roofline(prof, work, peaks, {"sm_mhz": 2032.0})
    # waypoint pass: 2 word-ops and 2 word loads per non-zero pair, per launch
    ops = 2 * (4e9 + 6e9) / 8
    t = 54.0 / 8 / 1000.0
    assert abs(r["achieved"] - ops / t / 1e12) < 1e-4
    assert abs(r["frac"] - (ops / t) / 19.2e12) < 1e-5
    assert abs(r["bitset_traffic"]["frac"] - (ops / t) / 9.6e12) < 1e-5
    assert r["binding"] == "bitset_traffic" and r["peak"] == round(19.2, 3)
    pk = r["per_kernel"]
    # edge masks: one op and one word per supercover term
    assert pk["edge_masks"]["alg_ops_per_launch"] == round(9.7e9 / 8)
    # every class above 1 % of the step is reported, the rest is not
    assert set(pk) == {"propagate_backward_waypoints", "propagate_forward", "propagate_backward_reach",
                       "edge_masks", "smooth_chain"}
    # a slower sampled clock scales the peaks down
    r2 = b.roofline(prof, work, peaks, {"sm_mhz": 1016.0})
    assert abs(r2["frac"] - 2 * r["frac"]) < 1e-4


def test_job_value_and_oracle_note():
    b = _bench()
    assert b.job_value(64, 2, 100.0) == 64 * 2 / 0.1
    assert "lower bound" in b.LOWER_BOUND_NOTE
