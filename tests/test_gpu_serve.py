"""Serving loop: device-generated requests counted while others are in flight give
the same results as each request alone, and as the oracle; admission respects the
memory budget."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

GAMMA = np.uint64(0x9e3779b97f4a7c15)


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xbf58476d1ce4e5b9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94d049bb133111eb)
    return z ^ (z >> np.uint64(31))


def checksums(t, lcc):
    """Order-independent checksums of t[] and LCC[] as the server reports them."""
    with np.errstate(over="ignore"):
        key = np.arange(len(t), dtype=np.uint64) * GAMMA
        a = _mix(key ^ t.astype(np.uint64)).sum(dtype=np.uint64)
        b = _mix(key ^ lcc.view(np.uint64)).sum(dtype=np.uint64)
    return int(a), int(b)


@pytest.mark.parametrize("kind,n,m,seed,stream", [("rmat", 1000, 9000, 5, 1), ("rmat", 70001, 500000, 5, 7),
                                                  ("er_replace", 3333, 40000, 5, 2), ("rmat", 2, 17, 1, 0),
                                                  ("er_replace", 1, 5, 3, 3)])
def test_device_generator_matches_host(tc, kind, n, m, seed, stream):
    import math
    import torch
    s = torch.empty(m, dtype=torch.int32, device="cuda")
    d = torch.empty(m, dtype=torch.int32, device="cuda")
    tc.tc_generate_edges(kind, n, m, seed, stream, s, d)
    torch.cuda.synchronize()
    if kind == "rmat":
        scale = max(1, int(math.ceil(math.log2(n))))
        hs, hd = graphgen.rmat(scale, m, seed, stream, n=n)
    else:
        hs, hd = graphgen.er_replace(n, m, seed, stream)
    np.testing.assert_array_equal(s.cpu().numpy(), hs)
    np.testing.assert_array_equal(d.cpu().numpy(), hd)


def _requests(count=48):
    return graphgen.serve_requests(seconds=1e9, rate=2000.0, seed=5, n_range=(1000, 40000), limit=count)


def _serve(tc, reqs, slots, alone):
    srv = tc.Server(8 << 30, slots)
    res = {}
    try:
        for i, r in enumerate(reqs):
            srv.submit(r.id, r.workload)
            if alone:
                assert srv.wait(i + 1, 120.0)
        assert srv.wait(len(reqs), 300.0)
        for x in srv.poll(len(reqs) + 8):
            res[x["id"]] = x
        stats = srv.stats()
    finally:
        srv.stop()
    return res, stats


def test_each_result_is_the_same_alone_and_in_the_mix(tc):
    reqs = _requests()
    mix, stats = _serve(tc, reqs, slots=6, alone=False)
    alone, _ = _serve(tc, reqs, slots=1, alone=True)
    assert len(mix) == len(alone) == len(reqs)
    assert stats["max_queue"] > 1  # requests waited while others were in flight
    overlap = 0
    spans = sorted((x["start_s"], x["end_s"]) for x in mix.values())
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        overlap += b0 < a1
    assert overlap > 0  # work of different requests overlapped in time
    for r in reqs:
        a, b = mix[r.id], alone[r.id]
        assert a["status"] == b["status"] == 0
        for k in ("T", "m_simple", "t_hash", "lcc_hash"):
            assert a[k] == b[k], (r.id, k)
        ref = oracle.triangles(r.workload.n, *r.workload.edges())
        assert a["T"] == ref["T"]
        assert a["m_simple"] == ref["m_simple"]
        assert (a["t_hash"], a["lcc_hash"]) == checksums(ref["t"], ref["lcc"])


def test_admission_respects_the_budget(tc):
    reqs = _requests(24)
    est = [48 * r.workload.m + 160 * r.workload.n + (16 << 20) for r in reqs]  # the library's admission estimate
    budget = 2 * max(est)
    srv = tc.Server(budget, 8)
    try:
        for r in reqs:
            srv.submit(r.id, r.workload)
        assert srv.wait(len(reqs), 300.0)
        st = srv.stats()
        assert st["peak_bytes"] <= budget
        assert st["completed"] == len(reqs)
    finally:
        srv.stop()
    # a request larger than the whole budget still runs, alone
    srv = tc.Server(1 << 20, 2)
    try:
        srv.submit(0, reqs[0].workload)
        assert srv.wait(1, 120.0)
        (x,) = srv.poll()
        assert x["status"] == 0 and x["bytes"] > (1 << 20)
    finally:
        srv.stop()


def test_bad_requests_are_rejected(tc):
    srv = tc.Server(1 << 30, 1)
    try:
        w = graphgen.Workload("bad", "rmat", 0, 10, 5, 1, scale=1)
        with pytest.raises(tc.TCError):
            srv.submit(1, w)
    finally:
        srv.stop()


def test_plain_request_run_matches_the_server(tc):
    """tc_request_run (one request alone on the caller's stream, the path the serving
    loop is measured against) reports the same T, edges and checksums as the server
    and the oracle."""
    import torch
    reqs = _requests(12)
    served, _ = _serve(tc, reqs, slots=4, alone=False)
    side = torch.cuda.Stream()
    for r in reqs:
        x = tc.tc_request_run(r.id, r.workload, side)
        assert x["status"] == 0 and x["id"] == r.id
        for k in ("T", "m_simple", "t_hash", "lcc_hash"):
            assert x[k] == served[r.id][k], (r.id, k)
        ref = oracle.triangles(r.workload.n, *r.workload.edges())
        assert x["T"] == ref["T"] and x["m_simple"] == ref["m_simple"]
        assert (x["t_hash"], x["lcc_hash"]) == checksums(ref["t"], ref["lcc"])
    with pytest.raises(tc.TCError):
        tc.tc_request_run(0, graphgen.Workload("bad", "rmat", 0, 10, 5, 1, scale=1))
