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
