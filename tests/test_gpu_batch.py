"""Batches of independent graphs (counted as one disjoint union) against the oracle
graph by graph, and against the single-graph entry point."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle
from tests import families as F

pytestmark = pytest.mark.gpu


def _pack(graphs):
    n = np.array([g[0] for g in graphs], dtype=np.int32)
    off = np.zeros(len(graphs) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(g[1]) for g in graphs])
    src = np.concatenate([g[1] for g in graphs] + [np.array([], np.int32)]).astype(np.int32)
    dst = np.concatenate([g[2] for g in graphs] + [np.array([], np.int32)]).astype(np.int32)
    return n, off, src, dst


def _batch_graphs(G, seed=4):
    out = []
    for w in graphgen.batch_workloads(G, seed=seed):
        s, d = w.edges()
        out.append((w.n, s, d))
    return out


def _check(tc, graphs, device):
    import torch
    n, off, src, dst = _pack(graphs)
    if device:
        s_in, d_in = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
    else:
        s_in, d_in = src, dst
    g = tc.Graph.batch(n, off, s_in, d_in)
    try:
        T = g.batch_count()
        t, lc = g.lcc()
    finally:
        g.close()
    vb = np.zeros(len(graphs) + 1, dtype=np.int64)
    vb[1:] = np.cumsum(n)
    for i, (ni, s, d) in enumerate(graphs):
        ref = oracle.triangles(ni, s, d)
        assert T[i] == ref["T"], i
        np.testing.assert_array_equal(t[vb[i]:vb[i + 1]], ref["t"])
        np.testing.assert_array_equal(lc[vb[i]:vb[i + 1]].view(np.uint64), ref["lcc"].view(np.uint64))


@pytest.mark.parametrize("device", [False, True])
def test_batch_workload_prefix_matches_oracle(tc, device):
    _check(tc, _batch_graphs(150), device)


def test_batch_with_degenerate_members(tc):
    graphs = [F.complete(5), (0, np.array([], np.int32), np.array([], np.int32)), F.wheel(9),
              (7, np.array([], np.int32), np.array([], np.int32)), F.friendship(4), F.star(20)]
    graphs = [(g[0], g[1][0], g[1][1]) if isinstance(g[1], tuple) else g for g in graphs]
    _check(tc, graphs, device=False)
    # repeated pairs and self-loops inside members
    from tests.test_oracle import _tiny
    _check(tc, [_tiny(s) for s in range(10)], device=True)


def test_batch_equals_single_graph_calls(tc):
    graphs = _batch_graphs(40, seed=9)
    n, off, src, dst = _pack(graphs)
    g = tc.Graph.batch(n, off, src, dst)
    T = g.batch_count()
    g.close()
    for i, (ni, s, d) in enumerate(graphs):
        h = tc.Graph.from_edges(ni, s, d)
        assert h.count() == T[i]
        h.close()


def test_batch_rejects_bad_local_ids(tc):
    graphs = [F.complete(4), F.complete(5)]
    graphs = [(g[0], g[1][0], g[1][1]) for g in graphs]
    n, off, src, dst = _pack(graphs)
    dst = dst.copy()
    dst[-1] = 5  # graph 1 has ids 0..4
    g = tc.Graph.batch(n, off, src, dst)
    with pytest.raises(tc.TCError) as e:
        g.batch_count()
    assert e.value.status == tc.TC_EINVAL
    g.close()
    with pytest.raises(tc.TCError):
        tc.Graph.batch(np.array([3], np.int32), np.array([1, 2], np.int64), src[:2], dst[:2])


def test_empty_batch(tc):
    g = tc.Graph.batch(np.zeros(0, np.int32), np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert len(g.batch_count()) == 0
    g.close()


def test_autotune_keeps_results_and_caches(tc):
    import time
    n = 1 << 14
    s, d = graphgen.rmat(14, 16 * n, seed=2)
    ref = oracle.triangles(n, s, d)
    g = tc.Graph.from_edges(n, s, d)
    tun = g.autotune(force=True)
    assert g.tuning() == tun
    assert g.count() == ref["T"]
    t, lc = g.lcc()
    np.testing.assert_array_equal(t, ref["t"])
    g.close()
    g = tc.Graph.from_edges(n, s, d)
    t0 = time.perf_counter()
    assert g.autotune() == tun          # same signature: taken from the cache
    assert time.perf_counter() - t0 < 0.5
    g.close()
    bad = dict(tun)
    bad["strategy"] = dict(tun["strategy"], small="bitmap")
    g = tc.Graph.from_edges(n, s, d)
    with pytest.raises(tc.TCError):
        g.set_tuning(bad)
    g.close()


@pytest.mark.parametrize("graph", [False, True])
def test_batch_run_matches_oracle_and_replays(tc, graph):
    import torch
    graphs = _batch_graphs(60, seed=11)
    n, off, src, dst = _pack(graphs)
    nt = int(n.sum())
    s_d, d_d = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
    T = torch.empty(len(n), dtype=torch.int64, device="cuda")
    t = torch.empty(nt, dtype=torch.int64, device="cuda")
    lc = torch.empty(nt, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    tuning = {"strategy": {"small": "auto", "cta": "probe", "hub": "bitmap"},
              "factor": {"small": 1.0, "cta": 1.0, "hub": 1.0}, "hub_min_degree": 16, "hub_max": 131072,
              "hub_big_in": 64}
    vb = np.zeros(len(n) + 1, dtype=np.int64)
    vb[1:] = np.cumsum(n)
    refs = [oracle.triangles(ni, si, di) for ni, si, di in graphs]
    for rep in range(3):
        T.fill_(-1)
        t.fill_(-1)
        tc.tc_batch_run(n, off, s_d, d_d, T, t, lc, tuning=tuning if rep else None, stream=stream, graph=graph)
        torch.cuda.synchronize()
        Th = T.cpu().numpy().view(np.uint64)
        th = t.cpu().numpy().view(np.uint64)
        lh = lc.cpu().numpy()
        for i, ref in enumerate(refs):
            assert Th[i] == ref["T"]
            np.testing.assert_array_equal(th[vb[i]:vb[i + 1]], ref["t"])
            np.testing.assert_array_equal(lh[vb[i]:vb[i + 1]].view(np.uint64), ref["lcc"].view(np.uint64))
    if graph:
        with pytest.raises(tc.TCError):
            tc.tc_batch_run(n, off, s_d, d_d, T, graph=True, stream=None)
        tc.tc_release_cached_graphs()


def test_batch_run_reports_bad_ids(tc):
    import torch
    n = np.array([3, 3], np.int32)
    off = np.array([0, 2, 4], np.int64)
    s = torch.tensor([0, 1, 0, 1], dtype=torch.int32, device="cuda")
    d = torch.tensor([1, 2, 1, 9], dtype=torch.int32, device="cuda")
    T = torch.empty(2, dtype=torch.int64, device="cuda")
    with pytest.raises(tc.TCError) as e:
        tc.tc_batch_run(n, off, s, d, T, stream=torch.cuda.Stream(), graph=True)
    assert e.value.status == tc.TC_EINVAL
    tc.tc_release_cached_graphs()


@pytest.mark.slow
def test_whole_batch_matches_the_oracle_digests(tc):
    """All 20,000 graphs of the batched workload (seed 4) in one batch call, through
    the CUDA-graph path the benchmark times: per-graph T and every t[v] and LCC[v]
    against tests/golden/batch_workload.json, which make_golden.py --batch wrote from
    the oracle's count of every graph."""
    import hashlib
    import json
    import os
    from concurrent.futures import ThreadPoolExecutor

    import torch
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "batch_workload.json")))
    ws = graphgen.batch_workloads(gold["graphs"], seed=gold["seed"])
    with ThreadPoolExecutor(max_workers=len(os.sched_getaffinity(0))) as ex:
        edges = list(ex.map(lambda w: w.edges(), ws))
    n = np.array([w.n for w in ws], dtype=np.int32)
    off = np.zeros(len(ws) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(e[0]) for e in edges])
    src = torch.from_numpy(np.concatenate([e[0] for e in edges]).astype(np.int32)).cuda()
    dst = torch.from_numpy(np.concatenate([e[1] for e in edges]).astype(np.int32)).cuda()
    del edges
    nt = int(n.sum())
    assert nt == gold["vertices"]
    T = torch.empty(len(ws), dtype=torch.int64, device="cuda")
    t = torch.empty(nt, dtype=torch.int64, device="cuda")
    lc = torch.empty(nt, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    tc.tc_batch_run(n, off, src, dst, T, t, lc, stream=side, graph=True)
    side.synchronize()

    def digest(a):
        return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()

    Th = T.cpu().numpy().view(np.uint64)
    assert int(Th.sum(dtype=np.uint64)) == gold["T_total"]
    assert digest(Th) == gold["T_sha256"]
    assert digest(t.cpu().numpy().view(np.uint64)) == gold["t_sha256"]
    assert digest(lc.cpu().numpy()) == gold["lcc_sha256"]
    tc.tc_release_cached_graphs()
