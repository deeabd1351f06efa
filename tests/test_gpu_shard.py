"""The shard form of the count (tc_count_shard, tc_lcc_from_counts, the dist module)
against the oracle.

Each triangle is counted once, from its lowest vertex, so the shards' per-vertex
counts must sum to t(v), and their triangle counts to T, for any number of shards.
The LCC computed from the sum must equal the oracle's bit for bit. The same holds
when the shards run in separate processes that sum their counts over a gloo group:
two processes share the one GPU, and their kernels never wait on each other, since
only the host collective joins them."""
from __future__ import annotations

import socket

import numpy as np
import pytest

import graphgen
import oracle
from tests import families as F

pytestmark = pytest.mark.gpu


def _graphs():
    yield "rmat14", 1 << 14, *graphgen.rmat(14, 16 << 14, seed=2)
    yield "er4096", 4096, *graphgen.workload("er4096").edges()
    n, (s, d) = F.complete(64)  # every vertex is a hub and in the dense core
    yield "K64", n, s, d
    n, (s, d) = F.wheel(9)
    yield "wheel9", n, s, d


GRAPHS = list(_graphs())


@pytest.mark.parametrize("name,n,s,d", GRAPHS, ids=[g[0] for g in GRAPHS])
@pytest.mark.parametrize("nshards", [1, 2, 3, 7, 64])
def test_shards_sum_to_the_whole(tc, name, n, s, d, nshards):
    ref = oracle.triangles(n, s, d)
    g = tc.Graph.from_edges(n, s, d)
    try:
        tsum = np.zeros(n, dtype=np.uint64)
        Tsum = 0
        for k in range(nshards):
            T, t = g.count_shard(k, nshards)
            assert int(t.sum()) == 3 * T  # a shard's triangles add 3 to the sum of t
            tsum += t
            Tsum += T
        assert Tsum == ref["T"]
        np.testing.assert_array_equal(tsum, ref["t"])
        lcc = g.lcc_from_counts(tsum)
        np.testing.assert_array_equal(lcc.view(np.uint64), ref["lcc"].view(np.uint64))
        # the graph still counts the whole graph afterwards
        assert g.count() == ref["T"]
        t_all, _ = g.lcc()
        np.testing.assert_array_equal(t_all, ref["t"])
    finally:
        g.close()


def _expected_shard(n, s, d, shard, nshards):
    """One shard's t(v) by the rule tc.h states, recomputed on the host.

    The library ranks vertices by (degree, id), the degree being the count of
    non-loop input pairs at a vertex. The simple graph is relabelled by rank and
    oriented by label, so the oriented CSR is the library's. The cost
    d+ (d+ + 1) / 2 + 1 per rank (saturated at 2^32 - 1) cuts the ranks at
    floor(C k / N). The oracle's oriented count over the shard's source range gives
    t by rank, which is mapped back to vertex ids."""
    nl = s != d
    dm = np.bincount(s[nl], minlength=n) + np.bincount(d[nl], minlength=n)
    order = np.lexsort((np.arange(n), dm))  # rank -> vertex id
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    off, adj, _ = oracle.build_csr(n, s, d)
    rows = np.repeat(np.arange(n), np.diff(off))
    ru, rv = rank[rows], rank[adj]
    keep = ru < rv
    ru, rv = ru[keep], rv[keep]
    o = np.lexsort((rv, ru))
    ap = rv[o].astype(np.int32)
    op = np.zeros(n + 1, dtype=np.int64)
    op[1:] = np.cumsum(np.bincount(ru, minlength=n))
    dp = np.diff(op)
    cost = np.minimum(dp * (dp + 1) // 2 + 1, (1 << 32) - 1)
    prefix = np.concatenate([[0], np.cumsum(cost)])
    total = int(prefix[-1])

    def first_at_least(target):
        return int(np.searchsorted(prefix[:n], target, side="left"))

    lo = 0 if shard == 0 else first_at_least(total * shard // nshards)
    hi = n if shard + 1 == nshards else first_at_least(total * (shard + 1) // nshards)
    t_rank = oracle.tc_oriented_ranges(n, op, ap, [(lo, hi)] if hi > lo else [])
    return t_rank[rank]


@pytest.mark.parametrize("nshards", [2, 5])
def test_shards_follow_the_cost_rule(tc, nshards):
    """Each shard's share of t equals the oracle's oriented count restricted to the
    sources that the stated cut rule assigns to it."""
    n = 1 << 13
    s, d = graphgen.rmat(13, 16 * n, seed=4)
    g = tc.Graph.from_edges(n, s, d)
    try:
        for k in range(nshards):
            want = _expected_shard(n, s, d, k, nshards)
            T, t = g.count_shard(k, nshards)
            np.testing.assert_array_equal(t, want)
            assert 3 * T == int(want.sum())
    finally:
        g.close()


def test_shards_on_device_buffers(tc):
    import torch
    n = 1 << 12
    s, d = graphgen.rmat(12, 16 * n, seed=5)
    ref = oracle.triangles(n, s, d)
    g = tc.Graph.from_edges(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    try:
        tsum = torch.zeros(n, dtype=torch.int64, device="cuda")
        part = torch.empty(n, dtype=torch.int64, device="cuda")
        for k in range(3):
            g.count_shard(k, 3, part)
            tsum += part
        lcc = torch.empty(n, dtype=torch.float64, device="cuda")
        g.lcc_from_counts(tsum, lcc)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(tsum.cpu().numpy().view(np.uint64), ref["t"])
        np.testing.assert_array_equal(lcc.cpu().numpy().view(np.uint64), ref["lcc"].view(np.uint64))
    finally:
        g.close()


def test_shard_arguments_are_checked(tc):
    n, (s, d) = F.complete(5)
    g = tc.Graph.from_edges(n, s, d)
    try:
        for shard, nshards in [(0, 0), (-1, 2), (2, 2)]:
            with pytest.raises(tc.TCError):
                g.count_shard(shard, nshards)
        with pytest.raises(ValueError):
            g.count_shard(0, 2, np.empty(4, dtype=np.uint64))
        with pytest.raises(TypeError):
            g.lcc_from_counts(np.zeros(5, dtype=np.float64))
        assert g.count() == 10
    finally:
        g.close()


def test_empty_graph_shards(tc):
    g = tc.Graph.from_edges(0, np.empty(0, np.int32), np.empty(0, np.int32))
    try:
        assert g.count_shard(0, 3)[0] == 0
    finally:
        g.close()


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import paper_2202_13976_gb300 as tc
    from paper_2202_13976_gb300 import dist as tcd
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0)
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
    n = 1 << 13
    s, d = graphgen.rmat(13, 16 * n, seed=7)
    g = tc.Graph.from_edges(n, s, d)
    try:
        T, t, lcc = tcd.sharded_lcc(g, store=store, rank=rank, world=world, step="rmat13")
    finally:
        g.close()
    q.put((rank, T, t, lcc))
    dist.destroy_process_group()


def test_two_processes_sum_their_shards(tc):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = 1 << 13
    s, d = graphgen.rmat(13, 16 * n, seed=7)
    ref = oracle.triangles(n, s, d)
    for rank, T, t, lcc in out:
        assert T == ref["T"]
        np.testing.assert_array_equal(t, ref["t"])
        np.testing.assert_array_equal(lcc.view(np.uint64), ref["lcc"].view(np.uint64))
