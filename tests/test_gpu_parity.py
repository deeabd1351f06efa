"""Parity of the CUDA path (through the C ABI) with the CPU oracle: T, t[] bit-exact,
LCC bit-exact (0 ulp), input accounting exact."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle
from tests import families as F
from tests.gpu_util import assert_matches_oracle, gpu_run

pytestmark = pytest.mark.gpu

SMALL_STRATEGIES = [("hash", 1.0), ("auto", 1.0), ("auto", 8.0), ("auto", 0.125), ("merge", 1.0), ("search", 1.0)]
CTA_STRATEGIES = [("auto", 1.0), ("auto", 4.0), ("auto", 0.25), ("merge", 1.0), ("search", 1.0),
                  ("probe", 1.0), ("bitmap", 1.0)]
HUB_STRATEGIES = [("auto", 1.0), ("bitmap", 1.0), ("probe", 1.0)]
# (min_degree, max_hubs): default, none, every vertex of degree >= 1, a handful
HUB_SETTINGS = [(32, 131072), (32, 0), (1, 131072), (64, 50)]


@pytest.fixture(scope="module")
def er4096():
    w = graphgen.workload("er4096")
    s, d = w.edges()
    return w.n, s, d, oracle.triangles(w.n, s, d)


@pytest.fixture(scope="module")
def rmat14():
    n = 1 << 14
    s, d = graphgen.rmat(14, 16 * n, seed=2)
    return n, s, d, oracle.triangles(n, s, d)


def test_er4096_host_io(tc, er4096):
    n, s, d, ref = er4096
    assert_matches_oracle(tc, n, s, d, ref=ref)


def test_er4096_device_io(tc, er4096):
    n, s, d, ref = er4096
    assert_matches_oracle(tc, n, s, d, ref=ref, device_io=True)


@pytest.mark.parametrize("make", [
    lambda: F.complete(3), lambda: F.complete(34), lambda: F.complete(90), lambda: F.wheel(5),
    lambda: F.wheel(40), lambda: F.friendship(7), lambda: F.complete_tripartite(3, 5, 40),
    lambda: F.star(100), lambda: F.grid(20, 30), lambda: F.complete_bipartite(40, 50),
    lambda: F.cycle(3), lambda: F.cycle(10)])
def test_closed_forms(tc, make):
    n, (s, d) = make()
    assert_matches_oracle(tc, n, s, d)


@pytest.mark.parametrize("seed", range(24))
def test_tiny_random_with_loops_and_repeats(tc, seed):
    from tests.test_oracle import _tiny
    n, s, d = _tiny(seed)
    assert_matches_oracle(tc, n, s, d)


@pytest.mark.parametrize("hubs", HUB_SETTINGS)
@pytest.mark.parametrize("small", SMALL_STRATEGIES)
@pytest.mark.parametrize("cta", CTA_STRATEGIES)
def test_every_strategy_agrees(tc, rmat14, small, cta, hubs):
    n, s, d, ref = rmat14
    strategies = {tc.TC_BUCKET_SMALL: small, tc.TC_BUCKET_CTA: cta}
    assert_matches_oracle(tc, n, s, d, ref=ref, strategies=strategies, hubs=hubs)


@pytest.mark.parametrize("hub", HUB_STRATEGIES)
@pytest.mark.parametrize("hubs", HUB_SETTINGS)
def test_hub_strategies_agree(tc, rmat14, hub, hubs):
    n, s, d, ref = rmat14
    assert_matches_oracle(tc, n, s, d, ref=ref, strategies={tc.TC_BUCKET_HUB: hub}, hubs=hubs)


# dense core sizes: off, one vertex, a partial word, several words, the default
CORE_SETTINGS = [0, 1, 33, 200, 8192]


@pytest.mark.parametrize("core", CORE_SETTINGS)
@pytest.mark.parametrize("hubs", HUB_SETTINGS)
def test_dense_core_sizes_agree(tc, rmat14, core, hubs):
    n, s, d, ref = rmat14
    assert_matches_oracle(tc, n, s, d, ref=ref, hubs=hubs, tuning={"hub_core": core})


@pytest.mark.parametrize("core", CORE_SETTINGS)
@pytest.mark.parametrize("make", [lambda: F.complete(90), lambda: F.wheel(40),
                                  lambda: F.complete_tripartite(3, 5, 40), lambda: F.friendship(7)])
def test_dense_core_closed_forms(tc, make, core):
    n, (s, d) = make()
    assert_matches_oracle(tc, n, s, d, hubs=(1, 131072), tuning={"hub_core": core})


def test_strategy_rejects_unsupported_pairs(tc, er4096):
    n, s, d, _ = er4096
    g = tc.Graph.from_edges(n, s, d)
    for bucket, strat in [("small", "bitmap"), ("small", "probe"), ("hub", "merge"), ("hub", "search"),
                          ("cta", "hash"), ("hub", "hash")]:
        with pytest.raises(tc.TCError):
            g.set_strategy(bucket, strat)
    with pytest.raises(tc.TCError):
        g.set_hubs(-1, 10)
    g.close()


def test_plan_accounts_for_every_edge(tc, rmat14):
    n, s, d, ref = rmat14
    for hubs in HUB_SETTINGS:
        g = tc.Graph.from_edges(n, s, d)
        g.set_hubs(*hubs)
        p = g.plan_stats()
        assert sum(b["edges"] for b in p.values()) == ref["m_simple"]
        if hubs[1] == 0:
            assert p["hub"]["edges"] == 0
        assert g.count() == ref["T"]
        tim = g.timing()
        assert tim["total_ms"] > 0
        g.close()


def test_csr_input_host_and_device(tc, rmat14):
    n, s, d, ref = rmat14
    off, adj, _ = oracle.build_csr(n, s, d)
    for dev in (False, True):
        T, t, lc, _ = gpu_run(tc, n, None, None, device_io=dev, csr=(off, adj))
        assert T == ref["T"]
        np.testing.assert_array_equal(t, ref["t"])
        np.testing.assert_array_equal(lc, ref["lcc"])
    # asymmetric, unsorted, with repeats and loops
    rng = np.random.default_rng(5)
    rows = rng.integers(0, 300, 4000).astype(np.int32)
    cols = rng.integers(0, 300, 4000).astype(np.int32)
    order = np.argsort(rows, kind="stable")
    rows, cols = rows[order], cols[order]
    off2 = np.zeros(301, dtype=np.int64)
    off2[1:] = np.cumsum(np.bincount(rows, minlength=300))
    ref2 = oracle.triangles(300, rows, cols)
    for dev in (False, True):
        T, t, lc, info = gpu_run(tc, 300, None, None, device_io=dev, csr=(off2, cols))
        assert T == ref2["T"]
        np.testing.assert_array_equal(t, ref2["t"])
        np.testing.assert_array_equal(lc, ref2["lcc"])
        assert info["m_simple"] == ref2["m_simple"]


def test_empty_and_degenerate(tc):
    e = np.array([], dtype=np.int32)
    for n in (0, 1, 7):
        T, t, lc, info = gpu_run(tc, n, e, e)
        assert T == 0 and len(t) == n and (lc == 0).all() and info["m_simple"] == 0
    loops = np.arange(5, dtype=np.int32)
    T, t, lc, info = gpu_run(tc, 5, loops, loops)
    assert T == 0 and info["loops_dropped"] == 5 and info["m_simple"] == 0
    s = np.array([0, 1, 0, 0], np.int32)
    d = np.array([1, 0, 1, 1], np.int32)
    T, t, lc, info = gpu_run(tc, 2, s, d)
    assert T == 0 and info["m_simple"] == 1 and info["dups_dropped"] == 3


def test_bad_input_is_rejected(tc):
    with pytest.raises(tc.TCError) as e:
        tc.Graph.from_edges(4, np.array([0, 4], np.int32), np.array([1, 1], np.int32))
    assert e.value.status == tc.TC_EINVAL
    with pytest.raises(tc.TCError):
        tc.Graph.from_edges(4, np.array([0, -1], np.int32), np.array([1, 1], np.int32))
    import torch
    bad = torch.tensor([0, 3, 2], dtype=torch.int64, device="cuda")
    adj = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(tc.TCError):
        tc.Graph.from_csr(2, bad, adj)
    # the library stays usable after rejected inputs
    n, (s, d) = F.complete(6)
    assert_matches_oracle(tc, n, s, d)


def test_long_rows_use_block_and_global_sorters(tc):
    """Rows longer than the warp sorter (1024) and the shared-memory block sorter
    (16384) before deduplication: vertex 0 joins 100 hubs, each pair repeated 200
    times (row length 20000); each hub carries 25000 copies of an edge to its own
    satellite so that it outranks vertex 0; consecutive hubs are joined."""
    src, dst = [], []
    hubs = np.arange(1, 101, dtype=np.int32)
    for h in hubs:
        src += [0] * 200
        dst += [int(h)] * 200
        src += [int(h)] * 25000
        dst += [int(h) + 100] * 25000
    for a, b in zip(hubs[:-1], hubs[1:]):
        src.append(int(a))
        dst.append(int(b))
    # a K_1500 block gives rows of up to 1499 entries (block sorter, shared memory)
    kn = 1500
    iu, ju = np.triu_indices(kn, 1)
    s = np.concatenate([np.array(src, np.int32), (iu + 300).astype(np.int32)])
    d = np.concatenate([np.array(dst, np.int32), (ju + 300).astype(np.int32)])
    perm = np.random.default_rng(0).permutation(len(s))
    assert_matches_oracle(tc, 300 + kn, s[perm], d[perm])


@pytest.mark.parametrize("scale,ef,seed", [(12, 4, 1), (16, 16, 3), (17, 8, 4)])
def test_rmat_several_tiles(tc, scale, ef, seed):
    n = 1 << scale
    s, d = graphgen.rmat(scale, ef * n, seed=seed)
    assert_matches_oracle(tc, n, s, d)


@pytest.fixture(scope="module")
def rmat18():
    n = 1 << 18
    s, d = graphgen.rmat(18, 16 * n, seed=9)
    return n, s, d, oracle.triangles(n, s, d)


@pytest.mark.parametrize("hubs", [(32, 0), (32, 500), (32, 131072)])
def test_block_bucket_wide_windows(tc, rmat18, hubs):
    """Sources of the block bucket whose rank window (u, max N+(u)] is wider than
    the 131072-bit bitmap fall back to a hash set of N+(u): R-MAT scale 18 with
    few or no hubs has many such sources."""
    n, s, d, ref = rmat18
    for cta in [("bitmap", 1.0), ("auto", 1.0)]:
        assert_matches_oracle(tc, n, s, d, ref=ref, hubs=hubs, strategies={tc.TC_BUCKET_CTA: cta})


def test_er_ragged_sizes(tc):
    for n, m in [(1000, 7777), (65537, 400001), (3, 3)]:
        s, d = graphgen.er(n, m, seed=n)
        assert_matches_oracle(tc, n, s, d)


def test_non_default_stream(tc, er4096):
    import torch
    n, s, d, ref = er4096
    st = torch.cuda.Stream()
    T, t, lc, _ = gpu_run(tc, n, s, d, device_io=True, stream=st)
    assert T == ref["T"]
    np.testing.assert_array_equal(t, ref["t"])


def test_repeated_create_destroy_is_stable(tc, er4096):
    n, s, d, ref = er4096
    for _ in range(5):
        T, t, _, _ = gpu_run(tc, n, s, d)
        assert T == ref["T"]


@pytest.mark.parametrize("make", [
    lambda: F.complete(34), lambda: F.wheel(40), lambda: F.friendship(7), lambda: F.star(100),
    lambda: F.complete_tripartite(3, 5, 40), lambda: F.grid(20, 30)])
def test_vertex_formula_closed_forms(tc, make):
    """The paper's unoriented per-vertex formula on the GPU gives the oracle's t[]."""
    n, (s, d) = make()
    ref = oracle.triangles(n, s, d)
    g = tc.Graph.from_edges(n, s, d)
    try:
        T, t = g.vertex_formula()
    finally:
        g.close()
    assert T == ref["T"]
    np.testing.assert_array_equal(t, ref["t"])


@pytest.mark.parametrize("seed", range(6))
def test_vertex_formula_tiny_random(tc, seed):
    from tests.test_oracle import _tiny
    n, s, d = _tiny(seed)
    ref = oracle.triangles(n, s, d)
    g = tc.Graph.from_edges(n, s, d)
    try:
        T, t = g.vertex_formula()
    finally:
        g.close()
    assert T == ref["T"]
    np.testing.assert_array_equal(t, ref["t"])


def test_vertex_formula_rmat_and_er(tc, rmat14, er4096):
    import torch
    for n, s, d, ref in (rmat14, er4096):
        g = tc.Graph.from_edges(n, s, d)
        try:
            T, t = g.vertex_formula()
            td = torch.empty(n, dtype=torch.int64, device="cuda")
            T2, _ = g.vertex_formula(td)
            assert g.count() == T  # the oriented count on the same graph object agrees
        finally:
            g.close()
        assert T == ref["T"] and T2 == ref["T"]
        np.testing.assert_array_equal(t, ref["t"])
        np.testing.assert_array_equal(td.cpu().numpy().view(np.uint64), ref["t"])


def _assert_support_matches(tc, n, s, d, hubs=None):
    ru, rv, rs = oracle.edge_support(n, s, d)
    g = tc.Graph.from_edges(n, s, d)
    try:
        if hubs:
            g.set_hubs(*hubs[:2])
            if len(hubs) > 2:
                t = g.tuning()
                t["hub_big_in"] = hubs[2]
                g.set_tuning(t)
        T0 = g.count()
        u, v, sup = g.edge_support()
        assert g.count() == T0  # the graph's own tuning (dense core included) is back
    finally:
        g.close()
    np.testing.assert_array_equal(u, ru)
    np.testing.assert_array_equal(v, rv)
    np.testing.assert_array_equal(sup, rs)


@pytest.mark.parametrize("hubs", [(32, 0), (2, 131072, 1 << 30), (2, 131072, 1), (8, 64), (32, 131072)])
def test_edge_support_every_bucket(tc, hubs):
    """The support recorded by each count kernel: hubs off (small and block buckets
    only), every hub a warp's hash set, every hub a block's bitmap, a few hubs, the
    default; on an R-MAT whose sources reach past 256 out-entries."""
    n = 1 << 13
    s, d = graphgen.rmat(13, 24 * n, seed=17)
    _assert_support_matches(tc, n, s, d, hubs)


def test_edge_support_hub_longer_than_shared_counters(tc):
    """K_1100 with every vertex a big hub: N+(v) of up to 1098 entries exceeds the
    1024 shared-memory counters, so matches count globally."""
    n, (s, d) = F.complete(1100)
    _assert_support_matches(tc, n, s, d, (2, 131072, 1))


@pytest.mark.parametrize("make", [
    lambda: F.complete(34), lambda: F.wheel(40), lambda: F.friendship(7), lambda: F.star(100),
    lambda: F.complete_tripartite(3, 5, 40), lambda: F.grid(20, 30), lambda: F.cycle(3)])
def test_edge_support_closed_forms(tc, make):
    n, (s, d) = make()
    _assert_support_matches(tc, n, s, d)


@pytest.mark.parametrize("seed", range(6))
def test_edge_support_tiny_random(tc, seed):
    from tests.test_oracle import _tiny
    n, s, d = _tiny(seed)
    _assert_support_matches(tc, n, s, d)


def test_edge_support_rmat_and_er_device_io(tc, rmat14, er4096):
    import torch
    for n, s, d, ref in (rmat14, er4096):
        _assert_support_matches(tc, n, s, d)
        g = tc.Graph.from_edges(n, s, d)
        try:
            m = g.info()["m_simple"]
            bufs = [torch.empty(m, dtype=torch.int32, device="cuda") for _ in range(3)]
            u, v, sup = g.edge_support(*bufs)
            torch.cuda.synchronize()
        finally:
            g.close()
        assert int(sup.to(torch.int64).sum()) == 3 * ref["T"]
        assert bool((u < v).all())


@pytest.mark.parametrize("core", [0, 8192])
def test_hub_longer_than_shared_counters(tc, core):
    """K_1100 with every vertex a hub: big hubs with |N+(v)| up to 1098 exceed the
    1024 shared-memory counters and count their matches globally (core off), or the
    whole graph is one dense core (core on)."""
    n, (s, d) = F.complete(1100)
    assert_matches_oracle(tc, n, s, d, hubs=(1, 131072), tuning={"hub_core": core})


def test_edge_support_full_size_rmat20(tc):
    """R-MAT scale 20 (the paper's S20 EF16): the supports sum to 3T, and a sample of
    4000 edges matches |adj(u) ∩ adj(v)| computed by the oracle's Alg. 2 on its CSR."""
    import torch
    w = graphgen.workload("rmat20")
    s, d = w.edges()
    g = tc.Graph.from_edges(w.n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    try:
        T = g.count()
        m = g.info()["m_simple"]
        bufs = [torch.empty(m, dtype=torch.int32, device="cuda") for _ in range(3)]
        u, v, sup = g.edge_support(*bufs)
        torch.cuda.synchronize()
        assert g.count() == T
    finally:
        g.close()
    u, v, sup = u.cpu().numpy(), v.cpu().numpy(), sup.cpu().numpy().view(np.uint32)
    assert int(sup.sum(dtype=np.uint64)) == 3 * T
    assert (u < v).all()
    offsets, adj, _ = oracle.build_csr(w.n, s, d)
    rng = np.random.default_rng(7)
    for k in rng.choice(m, 4000, replace=False):
        a, b = int(u[k]), int(v[k])
        want = oracle.ssi(adj[offsets[a]:offsets[a + 1]], adj[offsets[b]:offsets[b + 1]])
        assert int(sup[k]) == want, (a, b)


def test_planner_streams_in_any_call_order(tc, rmat14):
    """The hub lists are built on a second stream: every order of plan, count,
    replan and destroy must see them complete (destroy right after a plan, plan
    statistics before the count, replans between counts, a count after a replan
    that turned the hubs off and on again)."""
    n, s, d, ref = rmat14
    g = tc.Graph.from_edges(n, s, d)
    g.plan_stats()
    g.close()  # released while nothing waited for the second stream yet
    g = tc.Graph.from_edges(n, s, d)
    try:
        stats = g.plan_stats()
        assert sum(stats[b]["edges"] for b in ("small", "cta", "hub", "trivial")) == ref["m_simple"]
        assert g.count() == ref["T"]
        for md, mx in [(32, 0), (1, 131072), (64, 50), (32, 131072)]:
            g.set_hubs(md, mx)
            assert g.count() == ref["T"]
            t, lcc = g.lcc()
            np.testing.assert_array_equal(t, ref["t"])
        for k in range(3):
            T, _ = g.count_shard(k, 3)
            assert T >= 0
        assert g.count() == ref["T"]
    finally:
        g.close()
