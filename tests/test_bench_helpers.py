"""Host-side helpers of the benchmark (no GPU): the timing-rule summary, the peak
lookup and the CPU baselines (single-graph and the sampled one of the directed mode)."""
from __future__ import annotations

import numpy as np

import bench
import graphgen


def test_step_spread_follows_the_timing_rule():
    s = bench.step_spread([3.9, 3.88, 3.87, 3.91])
    assert s["median_ms"] == (3.88 + 3.9) / 2
    assert 0 < s["ci95_ms"] < 0.05 * s["median_ms"] and s["within_5pct"]
    wide = bench.step_spread([1.0, 3.0, 1.0, 3.0])
    assert wide["within_5pct"] is False
    one = bench.step_spread([2.0])
    assert one == {"median_ms": 2.0, "ci95_ms": None, "within_5pct": None}


def test_measured_peak_is_positive():
    peak, kind = bench.measured_peak()
    assert peak > 0 and kind in ("measured", "fallback")


def test_directed_cpu_baseline_samples_the_oracle():
    n = 1 << 10
    s, d = graphgen.rmat(10, 8 * n, seed=3)
    cpu = bench.directed_cpu_baseline(n, s, d, sample_vertices=200, seed=1)
    assert cpu["kind"] == "oracle" and cpu["unit"] == "edges/s" and cpu["value"] > 0
    assert "200 random vertices" in cpu["sample"]


def test_cpu_baseline_times_the_oracle_on_all_cores_and_on_one():
    import oracle
    w = graphgen.workload("er4096")
    s, d = w.edges()
    cpu = bench.cpu_baseline(w, s, d)
    assert cpu["T"] == oracle.triangles(w.n, s, d)["T"]
    assert cpu["kind"] == "oracle" and cpu["value"] > 0 and cpu["cores"] >= 1
    one = cpu["one_thread"]
    assert one["cores"] == 1 and one["value"] > 0
    assert f"of {8 * bench.ONE_CORE_PIECES} equal-work source ranges" in one["sample"]


def test_serve_verification_compares_with_the_oracle():
    """The serve check recomputes each sampled request on the host and compares T,
    edges and both digests; a wrong value in any of them counts as a mismatch."""
    reqs = graphgen.serve_requests(seconds=0.01, rate=2000.0, n_range=(1000, 60000))
    assert len(reqs) >= 4
    results = {}
    for r in reqs:
        q, T, m, th, lh = bench.serve_oracle_one((r.id, r.workload, 1))
        results[q] = {"status": 0, "T": T, "m_simple": m, "t_hash": th, "lcc_hash": lh}
    checked, bad, desc = bench.serve_verify(reqs, results, 1.0, 1)
    small = sum(r.workload.n <= bench.SERVE_SMALL_N for r in reqs)
    assert checked == small + min(1, len(reqs) - small) and bad == 0
    assert f"({small})" in desc
    q0 = next(r.id for r in reqs if r.workload.n <= bench.SERVE_SMALL_N)
    results[q0] = dict(results[q0], lcc_hash=results[q0]["lcc_hash"] ^ 1)
    assert bench.serve_verify(reqs, results, 1.0, 0)[1] == 1


class _FakeGraph:
    """The library's caching rule: a count runs only when the graph has not counted
    under its current settings, and plans again only when a hub setting changed."""

    def __init__(self):
        self.t = {"strategy": {"small": "auto"}, "hub_min_degree": 32, "hub_max": 131072,
                  "hub_big_in": 128, "hub_core": 8192}
        self.planned = self.counted = False
        self.plans = self.counts = 0

    def tuning(self):
        return dict(self.t)

    def set_tuning(self, t):
        hub = ("hub_min_degree", "hub_max", "hub_big_in", "hub_core")
        if any(t[k] != self.t[k] for k in hub):
            self.planned = False
        self.t = dict(t)
        self.counted = False

    def count(self):
        if not self.counted:
            if not self.planned:
                self.plans += 1
                self.planned = True
            self.counts += 1
            self.counted = True
        return 7

    def timing(self):
        return {"plans": self.plans, "counts": self.counts}


def test_recount_plans_and_counts_every_time():
    g = _FakeGraph()
    for k in range(1, 4):
        assert bench.recount(g, 7) == {"plans": k, "counts": k}
    assert g.t["hub_core"] == 8192  # the settings are left as they were
    g.t["hub_core"] = 1
    assert bench.recount(g, 7) == {"plans": 4, "counts": 4} and g.t["hub_core"] == 1


def test_bench_defaults_are_one_gpu_and_minutes():
    import sys
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse_args()
    finally:
        sys.argv = argv
    assert a.gpus == 1 and a.impl == "ours" and a.mode == "single" and a.workload == "rmat23"
    assert a.warmup >= 3 and 1 <= a.steps <= 200


def test_roofline_record_reports_the_dram_fraction():
    peak, _ = bench.measured_peak()
    r = bench.roofline_record("k", alg_bytes=10 * 10 ** 9, kernel_ms=1.0, traffic=2 * 10 ** 9)
    assert abs(r["achieved"] - 10000.0) < 1e-6 and abs(r["frac"] - 10000.0 / peak) < 1e-9
    assert abs(r["dram_achieved"] - 2000.0) < 1e-6 and abs(r["dram_frac"] - 2000.0 / peak) < 1e-9
    none = bench.roofline_record("k", alg_bytes=1, kernel_ms=1.0, traffic=None)
    assert none["dram_frac"] is None and none["traffic"] is None


def test_reference_sample_ranges_cover_the_sources_once():
    import oracle
    n = 1 << 11
    s, d = graphgen.rmat(11, 8 * n, seed=4)
    off, adj, _ = oracle.build_csr(n, s, d)
    op, ap = oracle.orient(n, off, adj)
    ranges = oracle.work_ranges(op, 64 * bench.REF_SAMPLES)
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    assert all(a < b for a, b in ranges) and all(ranges[i][1] == ranges[i + 1][0] for i in range(len(ranges) - 1))
    # the eight samples together give the full count
    total = sum(oracle.tc_oriented_ranges(n, op, ap, ranges[k::bench.REF_SAMPLES], threads=2)
                for k in range(bench.REF_SAMPLES))
    np.testing.assert_array_equal(total, oracle.tc_oriented(n, op, ap))


def test_golden_check_reads_the_oracle_digests():
    import json
    import os

    import numpy as np
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "large_workloads.json")))
    assert bench.golden_check("er4096", 0, np.zeros(1, np.uint64), np.zeros(1)) is None
    rec = gold["rmat20"]
    bad = bench.golden_check("rmat20", rec["T"], np.zeros(rec["n"], np.uint64), np.zeros(rec["n"]))
    assert bad == {"T": True, "t": False, "lcc": False}
