"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: brute-force triple
enumeration and dense matrix powers on tiny graphs, textbook closed forms,
scipy's sparse product for the algebraic form C = A A o A (Sec. VI-B), Python
set intersection for Alg. 1/2, hand-evaluated cases of Eq. 3, exact rational
LCC values, and invariants (relabelling, edge order, repeated pairs).
"""
from __future__ import annotations

from math import comb

import numpy as np
import pytest
import scipy.sparse as sp

import graphgen
import oracle
from tests import families as F


def run(n, src, dst):
    return oracle.triangles(n, src, dst)


# --------------------------------------------------------------------------
# Alg. 1, Alg. 2, Eq. 3

def _sorted_unique(rng, k, hi):
    return np.unique(rng.integers(0, hi, size=k)).astype(np.int32)


@pytest.mark.parametrize("seed", range(40))
def test_ssi_and_binary_search_match_set_intersection(seed):
    rng = np.random.default_rng(seed)
    A = _sorted_unique(rng, int(rng.integers(0, 60)), 200)
    B = _sorted_unique(rng, int(rng.integers(0, 300)), 200)
    want = len(set(A.tolist()) & set(B.tolist()))
    assert oracle.ssi(A, B) == want
    assert oracle.ssi(B, A) == want
    assert oracle.binary_search(A, B) == want
    assert oracle.binary_search(B, A) == want


def test_binary_search_finds_matches_at_both_ends():
    # The listing as printed never tests B[0] or B[|B|-1]; the textbook reading must.
    B = np.array([3, 5, 7, 9, 11], dtype=np.int32)
    assert oracle.binary_search(np.array([3], np.int32), B) == 1
    assert oracle.binary_search(np.array([11], np.int32), B) == 1
    assert oracle.binary_search(np.array([3, 11], np.int32), B) == 2
    assert oracle.binary_search(np.array([2, 4, 12], np.int32), B) == 0
    assert oracle.binary_search(np.array([], np.int32), B) == 0
    assert oracle.ssi(np.array([], np.int32), B) == 0


@pytest.mark.parametrize("a,b,want", [
    (8, 16, True),    # 16/8 = 2 <= log2(16) - 1 = 3
    (4, 16, False),   # 4 > 3
    (16, 16, True),   # 1 <= 3
    (4, 8, True),     # tie: 8/4 = 2 = log2(8) - 1 -> SSI
    (8, 32, True),    # tie: 4 = 4
    (7, 32, False),   # 4.57 > 4
    (1, 1, False),    # 1 > log2(1) - 1 = -1
    (2, 4, False),    # 2 > 1
    (100, 1000, False),  # 10 > log2(1000) - 1 = 8.97
    (200, 1000, True),   # 5 <= 8.97
])
def test_eq3_rule(a, b, want):
    assert oracle.prefer_ssi(a, b) is want
    assert oracle.prefer_ssi(b, a) is want  # the rule orders the lists itself


# --------------------------------------------------------------------------
# Closed forms

@pytest.mark.parametrize("n", [3, 4, 5, 9, 17, 40])
def test_complete_graph(n):
    nn, (s, d) = F.complete(n)
    r = run(nn, s, d)
    assert r["T"] == comb(n, 3)
    assert (r["t"] == comb(n - 1, 2)).all()
    assert (r["lcc"] == 1.0).all()


@pytest.mark.parametrize("make", [lambda: F.star(30), lambda: F.cycle(4), lambda: F.cycle(9),
                                  lambda: F.path(20), lambda: F.grid(7, 9),
                                  lambda: F.complete_bipartite(6, 11),
                                  lambda: F.random_tree(200, np.random.default_rng(3))])
def test_triangle_free(make):
    n, (s, d) = make()
    r = run(n, s, d)
    assert r["T"] == 0
    assert (r["t"] == 0).all()
    assert (r["lcc"] == 0.0).all()


def test_triangle_is_cycle3():
    n, (s, d) = F.cycle(3)
    r = run(n, s, d)
    assert r["T"] == 1 and (r["t"] == 1).all() and (r["lcc"] == 1.0).all()


@pytest.mark.parametrize("n", [5, 6, 7, 12, 33])
def test_wheel(n):
    nn, (s, d) = F.wheel(n)
    r = run(nn, s, d)
    assert r["T"] == n - 1
    assert r["t"][0] == n - 1 and (r["t"][1:] == 2).all()
    assert r["lcc"][0] == 2.0 / (n - 2)
    assert (r["lcc"][1:] == 2.0 / 3.0).all()


def test_wheel4_is_k4():
    n, (s, d) = F.wheel(4)
    assert run(n, s, d)["T"] == 4


@pytest.mark.parametrize("k", [1, 2, 5, 13])
def test_friendship(k):
    n, (s, d) = F.friendship(k)
    r = run(n, s, d)
    assert r["T"] == k
    assert r["t"][0] == k and (r["t"][1:] == 1).all()
    assert r["lcc"][0] == 1.0 / (2 * k - 1)
    assert (r["lcc"][1:] == 1.0).all()


@pytest.mark.parametrize("a,b,c", [(1, 1, 1), (2, 3, 4), (5, 1, 7), (6, 6, 6)])
def test_complete_tripartite(a, b, c):
    n, (s, d) = F.complete_tripartite(a, b, c)
    r = run(n, s, d)
    assert r["T"] == a * b * c
    assert (r["t"][:a] == b * c).all()
    assert (r["t"][a:a + b] == a * c).all()
    assert (r["t"][a + b:] == a * b).all()


# --------------------------------------------------------------------------
# Brute force on tiny random graphs (with loops and repeated pairs injected)

def _tiny(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 48))
    if seed % 2 == 0:
        s, d = graphgen.er(n, int(rng.integers(0, n * (n - 1) // 2 + 1)), seed=seed)
    else:
        scale = max(1, int(np.ceil(np.log2(n))))
        s, d = graphgen.rmat(scale, int(rng.integers(1, 6 * n)), seed=seed, n=n)
    # inject repeats (both orientations) and self-loops
    k = len(s)
    if k:
        pick = rng.integers(0, k, size=k // 3 + 1)
        s = np.concatenate([s, d[pick], s[pick[: len(pick) // 2]]])
        d = np.concatenate([d, s[: k][pick], d[pick[: len(pick) // 2]]])
    loops = rng.integers(0, n, size=3).astype(np.int32)
    s = np.concatenate([s, loops]).astype(np.int32)
    d = np.concatenate([d, loops]).astype(np.int32)
    perm = rng.permutation(len(s))
    return n, s[perm], d[perm]


@pytest.mark.parametrize("seed", range(60))
def test_brute_force_tiny(seed):
    n, s, d = _tiny(seed)
    r = run(n, s, d)
    T1, t1 = F.brute_triples(n, s, d)
    T2, t2 = F.brute_matrix(n, s, d)
    assert r["T"] == T1 == T2
    np.testing.assert_array_equal(r["t"], t1)
    np.testing.assert_array_equal(r["t"], t2)
    np.testing.assert_array_equal(r["lcc"], F.exact_lcc(t1, F.dense_adjacency(n, s, d).sum(1)))


# --------------------------------------------------------------------------
# Algebraic form (Sec. VI-B): C = A A o A, t = rowsum(C) / 2, with scipy.sparse

def _scipy_t(n, s, d):
    keep = s != d
    A = sp.coo_matrix((np.ones(keep.sum(), dtype=np.int64), (s[keep], d[keep])), shape=(n, n)).tocsr()
    A = ((A + A.T) > 0).astype(np.int64)
    C = (A @ A).multiply(A)
    return np.asarray(C.sum(axis=1)).ravel().astype(np.uint64) // 2, np.asarray(A.sum(axis=1)).ravel()


@pytest.mark.parametrize("name", ["er4096"])
def test_algebraic_form_er4096(name):
    w = graphgen.workload(name)
    s, d = w.edges()
    r = run(w.n, s, d)
    t, deg = _scipy_t(w.n, s, d)
    np.testing.assert_array_equal(r["t"], t)
    np.testing.assert_array_equal(r["degree"], deg)
    np.testing.assert_array_equal(r["lcc"], F.exact_lcc(t, deg))
    assert r["m_simple"] == 32768 and r["loops_dropped"] == 0 and r["dups_dropped"] == 0


@pytest.mark.parametrize("scale,ef,seed", [(10, 16, 5), (12, 8, 6)])
def test_algebraic_form_rmat(scale, ef, seed):
    n = 1 << scale
    s, d = graphgen.rmat(scale, ef * n, seed=seed)
    r = run(n, s, d)
    t, deg = _scipy_t(n, s, d)
    np.testing.assert_array_equal(r["t"], t)
    np.testing.assert_array_equal(r["lcc"], F.exact_lcc(t, deg))


# --------------------------------------------------------------------------
# The paper's per-vertex formula (Alg. 3) against the oriented count

@pytest.mark.parametrize("scale,ef,seed", [(11, 16, 1), (13, 8, 2)])
def test_per_vertex_formula_agrees(scale, ef, seed):
    n = 1 << scale
    s, d = graphgen.rmat(scale, ef * n, seed=seed)
    off, adj, _ = oracle.build_csr(n, s, d)
    op, ap = oracle.orient(n, off, adj)
    t_or = oracle.tc_oriented(n, op, ap)
    t_v = oracle.tc_vertex(n, off, adj, np.arange(n, dtype=np.int32))
    np.testing.assert_array_equal(t_or, t_v)
    # the threaded split gives the same result
    np.testing.assert_array_equal(oracle.tc_oriented(n, op, ap, threads=4), t_or)


def test_orientation_by_id_gives_same_counts():
    # Sec. II-C orients by id (j < k); the (degree, id) order must agree.
    n = 1 << 11
    s, d = graphgen.rmat(11, 8 * n, seed=9)
    off, adj, _ = oracle.build_csr(n, s, d)
    rows = np.repeat(np.arange(n), np.diff(off))
    keep = adj > rows
    op = np.zeros(n + 1, dtype=np.int64)
    op[1:] = np.cumsum(np.bincount(rows[keep], minlength=n))
    ap = adj[keep]
    np.testing.assert_array_equal(oracle.tc_oriented(n, op, ap), run(n, s, d)["t"])


# --------------------------------------------------------------------------
# Invariants and input handling

def test_relabel_edge_order_and_repeats():
    n = 1 << 10
    s, d = graphgen.rmat(10, 16 * n, seed=11)
    base = run(n, s, d)
    rng = np.random.default_rng(0)
    perm = rng.permutation(n).astype(np.int32)      # new id of old vertex
    r = run(n, perm[s], perm[d])
    np.testing.assert_array_equal(r["t"][perm], base["t"])
    np.testing.assert_array_equal(r["lcc"][perm], base["lcc"])
    order = rng.permutation(len(s))
    r = run(n, d[order], s[order])                   # reversed pairs, shuffled
    np.testing.assert_array_equal(r["t"], base["t"])
    r = run(n, np.concatenate([s, d, s]), np.concatenate([d, s, d]))
    np.testing.assert_array_equal(r["t"], base["t"])
    assert r["m_simple"] == base["m_simple"]
    assert r["dups_dropped"] == base["dups_dropped"] + 2 * (len(s) - base["loops_dropped"])


def test_sum_t_is_three_T_and_bounds():
    w = graphgen.workload("er4096")
    s, d = w.edges()
    r = run(w.n, s, d)
    assert int(r["t"].sum()) == 3 * r["T"]
    deg = r["degree"]
    assert (r["t"] <= deg * (deg - 1) // 2).all()
    assert ((r["lcc"] >= 0) & (r["lcc"] <= 1)).all()


def test_loop_and_duplicate_accounting():
    s = np.array([0, 1, 1, 2, 2, 0, 3, 3, 1], dtype=np.int32)
    d = np.array([1, 0, 2, 1, 2, 2, 3, 0, 2], dtype=np.int32)
    r = run(4, s, d)
    # edges {0,1} x2, {1,2} x3, {0,2}, {0,3}; loops (2,2), (3,3)
    assert r["loops_dropped"] == 2
    assert r["m_simple"] == 4
    assert r["dups_dropped"] == 3
    assert r["T"] == 1
    assert r["t"].tolist() == [1, 1, 1, 0]
    assert r["degree"].tolist() == [3, 2, 2, 1]
    assert r["lcc"].tolist() == [1.0 / 3.0, 1.0, 1.0, 0.0]


def test_bad_ids_rejected():
    with pytest.raises(ValueError):
        oracle.build_csr(3, np.array([0, 3], np.int32), np.array([1, 1], np.int32))
    with pytest.raises(ValueError):
        oracle.build_csr(3, np.array([-1], np.int32), np.array([1], np.int32))


def test_empty_and_isolated():
    r = run(0, np.array([], np.int32), np.array([], np.int32))
    assert r["T"] == 0 and len(r["t"]) == 0
    r = run(5, np.array([], np.int32), np.array([], np.int32))
    assert r["T"] == 0 and (r["lcc"] == 0).all()


def test_csr_input_reads_every_entry_as_a_pair():
    n, (s, d) = F.wheel(9)
    off, adj, _ = oracle.build_csr(n, s, d)
    r = oracle.triangles_csr(n, off, adj)
    assert r["T"] == 8
    # an asymmetric, unsorted CSR with repeats describes the same simple graph
    off2 = np.array([0, 2, 3, 5], dtype=np.int64)
    adj2 = np.array([2, 1, 2, 0, 1], dtype=np.int32)
    r2 = oracle.triangles_csr(3, off2, adj2)
    assert r2["T"] == 1 and r2["m_simple"] == 3 and r2["dups_dropped"] == 2


# --------------------------------------------------------------------------
# Per-edge support: |adj(u) ∩ adj(v)| for every edge, the entries of A·A ∘ A

@pytest.mark.parametrize("k", [3, 4, 7, 20])
def test_edge_support_complete_graph(k):
    n, (s, d) = F.complete(k)
    u, v, sup = oracle.edge_support(n, s, d)
    assert len(u) == comb(k, 2)
    assert (u < v).all()
    assert (sup == k - 2).all()


@pytest.mark.parametrize("make", [lambda: F.star(30), lambda: F.grid(7, 9), lambda: F.complete_bipartite(6, 9),
                                  lambda: F.cycle(12), lambda: F.random_tree(60, np.random.default_rng(3))])
def test_edge_support_triangle_free(make):
    n, (s, d) = make()
    _, _, sup = oracle.edge_support(n, s, d)
    assert (sup == 0).all()


def test_edge_support_wheel_and_friendship():
    n, (s, d) = F.wheel(9)  # hub 0, rim 1..8: each spoke lies in 2 triangles, each rim edge in 1
    u, v, sup = oracle.edge_support(n, s, d)
    assert (sup[u == 0] == 2).all() and (sup[u != 0] == 1).all()
    n, (s, d) = F.friendship(5)  # every edge lies in exactly one triangle
    _, _, sup = oracle.edge_support(n, s, d)
    assert (sup == 1).all()


@pytest.mark.parametrize("seed", range(12))
def test_edge_support_matches_dense_products(seed):
    n, s, d = _tiny(seed)
    A = F.dense_adjacency(n, s, d)
    u, v, sup = oracle.edge_support(n, s, d)
    C = (A @ A) * A  # C[i, j] = number of triangles on edge {i, j}
    assert int(A.sum()) // 2 == len(u)
    np.testing.assert_array_equal(sup.astype(np.int64), C[u, v])
    # each triangle has three edges
    assert int(sup.sum()) == 3 * oracle.triangles(n, s, d)["T"]


# --------------------------------------------------------------------------
# Directed LCC (Eq. 1): c(i) = |{e_jk : v_j, v_k in adj(v_i)}| over out-neighbours

def _tiny_directed(seed):
    """Random digraph with reciprocal pairs, repeats and self-loops."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 40))
    k = int(rng.integers(0, 3 * n * n // 4 + 1))
    s = rng.integers(0, n, size=k).astype(np.int32)
    d = rng.integers(0, n, size=k).astype(np.int32)
    if k:
        pick = rng.integers(0, k, size=k // 4 + 1)
        s = np.concatenate([s, d[pick], s[pick[: len(pick) // 2]]]).astype(np.int32)  # reversed and repeated
        d = np.concatenate([d, s[:k][pick], d[pick[: len(pick) // 2]]]).astype(np.int32)
    return n, s, d


@pytest.mark.parametrize("seed", range(40))
def test_directed_brute_force_tiny(seed):
    n, s, d = _tiny_directed(seed)
    r = oracle.directed_lcc(n, s, d)
    A = F.dense_digraph(n, s, d)
    np.testing.assert_array_equal(r["c"], F.brute_directed(n, s, d))
    # algebraic form: c = rowsum((A A) o A), the directed counterpart of Sec. VI-B
    np.testing.assert_array_equal(r["c"].astype(np.int64), ((A @ A) * A).sum(axis=1))
    np.testing.assert_array_equal(r["out_degree"], A.sum(axis=1))
    np.testing.assert_array_equal(r["lcc"], F.exact_directed_lcc(r["c"], A.sum(axis=1)))
    assert r["m_directed"] == int(A.sum())
    assert r["loops_dropped"] == int((s == d).sum())
    assert r["m_directed"] + r["loops_dropped"] + r["dups_dropped"] == len(s)


def test_directed_algebraic_form_scipy():
    n = 4096
    s, d = graphgen.er_replace(n, 40000, seed=7)
    keep = s != d
    A = sp.coo_matrix((np.ones(int(keep.sum()), dtype=np.int64), (s[keep], d[keep])), shape=(n, n)).tocsr()
    A.data[:] = 1
    A.sum_duplicates()
    A = (A > 0).astype(np.int64)
    want = np.asarray((A @ A).multiply(A).sum(axis=1)).ravel()
    r = oracle.directed_lcc(n, s, d)
    np.testing.assert_array_equal(r["c"].astype(np.int64), want)
    np.testing.assert_array_equal(r["out_degree"], np.asarray(A.sum(axis=1)).ravel())


@pytest.mark.parametrize("seed", range(8))
def test_directed_on_symmetric_input_is_eq2(seed):
    # Both directions of every edge: adj(v_i) is the undirected neighbourhood, every
    # triangle edge is counted in both directions, so Eq. 1 = Eq. 2 bit for bit.
    n, s, d = _tiny(seed)
    r = oracle.directed_lcc(n, np.concatenate([s, d]), np.concatenate([d, s]))
    u = run(n, s, d)
    np.testing.assert_array_equal(r["c"], 2 * u["t"])
    np.testing.assert_array_equal(r["lcc"], u["lcc"])
    np.testing.assert_array_equal(r["out_degree"], u["degree"])


@pytest.mark.parametrize("n", [1, 2, 3, 7, 30])
def test_directed_transitive_tournament(n):
    n, (s, d) = F.transitive_tournament(n)
    r = oracle.directed_lcc(n, s, d)
    dout = np.arange(n - 1, -1, -1)
    np.testing.assert_array_equal(r["c"], [comb(int(x), 2) for x in dout])
    np.testing.assert_array_equal(r["lcc"], np.where(dout >= 2, 0.5, 0.0))


@pytest.mark.parametrize("n", [2, 3, 5, 12])
def test_directed_complete(n):
    n, (s, d) = F.complete_digraph(n)
    r = oracle.directed_lcc(n, s, d)
    assert (r["c"] == (n - 1) * (n - 2)).all()
    np.testing.assert_array_equal(r["lcc"], np.full(n, 1.0 if n >= 3 else 0.0))


@pytest.mark.parametrize("rim", [3, 4, 9, 40])
def test_directed_wheels(rim):
    n, (s, d) = F.directed_wheel(rim, outward=True)
    r = oracle.directed_lcc(n, s, d)
    assert r["c"][0] == rim and r["lcc"][0] == 1.0 / (rim - 1)  # the rim cycle's rim edges
    assert (r["c"][1:] == 0).all() and (r["lcc"][1:] == 0.0).all()  # out-degree 1
    n, (s, d) = F.directed_wheel(rim, outward=False)
    r = oracle.directed_lcc(n, s, d)
    assert r["c"][0] == 0 and r["lcc"][0] == 0.0  # the hub has no out-edge
    assert (r["c"][1:] == 1).all() and (r["lcc"][1:] == 0.5).all()  # r -> {0, r+1}, r+1 -> 0


def test_directed_three_vertex_cases():
    cyc = oracle.directed_lcc(3, np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32))
    assert (cyc["c"] == 0).all() and (cyc["lcc"] == 0.0).all()
    ffl = oracle.directed_lcc(3, np.array([0, 0, 1], np.int32), np.array([1, 2, 2], np.int32))
    np.testing.assert_array_equal(ffl["c"], [1, 0, 0])
    np.testing.assert_array_equal(ffl["lcc"], [0.5, 0.0, 0.0])


@pytest.mark.parametrize("seed", range(6))
def test_directed_invariants(seed):
    n, s, d = _tiny_directed(seed + 50)
    r = oracle.directed_lcc(n, s, d)
    rng = np.random.default_rng(seed)
    # relabelling permutes the outputs
    perm = rng.permutation(n).astype(np.int32)
    rp = oracle.directed_lcc(n, perm[s], perm[d])
    np.testing.assert_array_equal(rp["c"][perm], r["c"])
    np.testing.assert_array_equal(rp["lcc"][perm], r["lcc"])
    # edge order and repeats do not matter
    order = rng.permutation(len(s))
    ro = oracle.directed_lcc(n, np.concatenate([s[order], s]), np.concatenate([d[order], d]))
    np.testing.assert_array_equal(ro["c"], r["c"])
    # the total counts transitive triples (i -> j, i -> k, j -> k), which reversing
    # every edge maps onto each other: sum(c) is invariant under reversal
    rr = oracle.directed_lcc(n, d, s)
    assert int(rr["c"].sum()) == int(r["c"].sum())


def test_directed_sampled_vertices_and_bad_ids():
    n, s, d = _tiny_directed(3)
    full = oracle.directed_lcc(n, s, d)
    pick = np.array([n - 1, 0, n // 2], dtype=np.int32)
    part = oracle.directed_lcc(n, s, d, vertices=pick)
    np.testing.assert_array_equal(part["c"], full["c"][pick])
    with pytest.raises(ValueError):
        oracle.directed_lcc(3, np.array([0], np.int32), np.array([3], np.int32))


# --------------------------------------------------------------------------
# Remote reads of the 1D-partitioned algorithm (Alg. 4) and their caches (Sec. IV-B)

def _brute_lru_hits(items, size_of, cap):
    """LRU by its stack property: a read hits iff the item was read before and its size
    plus the sizes of the distinct other items read since then fit in the cache."""
    hits = hb = 0
    last = {}
    for t, x in enumerate(items):
        if x in last:
            seen = set(items[last[x] + 1: t]) - {x}
            if size_of[x] + sum(size_of[y] for y in seen) <= cap:
                hits += 1
                hb += size_of[x]
        last[x] = t
    return hits, hb


def _brute_optimal_hits(items, cap):
    """Unit-size entries, ``cap`` slots: the most hits any policy can reach when every
    miss must be stored (an exhaustive search over every choice of victim)."""
    from functools import lru_cache

    @lru_cache(maxsize=None)
    def best(t, held):
        if t == len(items):
            return 0
        x = items[t]
        if x in held:
            return 1 + best(t + 1, held)
        if cap == 0:
            return best(t + 1, held)
        if len(held) < cap:
            return best(t + 1, held | {x})
        return max(best(t + 1, (held - {y}) | {x}) for y in held)

    return best(0, frozenset())


def test_cache_hand_examples():
    # LRU, unit entries, 2 slots: A B A C B -> only the second A hits (C evicts B)
    assert oracle.cache_lru([0, 1, 0, 2, 1], [1, 1, 1], 2) == (1, 1)
    assert oracle.cache_lru([0, 1, 0, 2, 1], [1, 1, 1], 3) == (2, 2)
    assert oracle.cache_lru([0, 0, 0], [5], 4) == (0, 0)  # larger than the cache: never held
    # bytes: sizes 3, 2, 2 in 5 bytes: A B C A -> C evicts A (3 + 2 + 2 > 5), A misses
    assert oracle.cache_lru([0, 1, 2, 0], [3, 2, 2], 5) == (0, 0)
    assert oracle.cache_lru([0, 1, 2, 1, 2], [3, 2, 2], 5) == (2, 4)
    assert oracle.cache_lru([2, 2, 0, 2, 2], [1, 1, 1], 1) == (2, 2)


def test_cache_score_hand_traces():
    """The degree score of Sec. IV-B2 worked by hand from its rule: on a miss the
    cached entries of lowest (degree, id) leave until the new entry fits, then it is
    stored; an entry larger than the cache is not stored and evicts nothing."""
    deg = [3, 2, 1]  # A = 0 scores highest, C = 2 lowest
    # one slot: every miss replaces the only entry, whatever the scores:
    # A; B evicts A; A evicts B; C evicts A; B evicts C -> no hit.  (A filter that
    # admits a miss only when it scores above every entry evicted so far would keep A
    # throughout and hit A's second read: 1 hit.)
    assert oracle.cache_score([0, 1, 0, 2, 1], [1, 1, 1], deg, 1) == (0, 0)
    # ... and a low-score entry hits again once it is back: C; C hits; A evicts C;
    # C evicts A; C hits
    assert oracle.cache_score([2, 2, 0, 2, 2], [1, 1, 1], deg, 1) == (2, 2)
    # two slots: A B -> {A, B}; C evicts B (lower than A) -> {A, C}; A hits; B evicts
    # C -> {A, B}; C evicts B -> {A, C}; C hits
    assert oracle.cache_score([0, 1, 2, 0, 1, 2, 2], [1, 1, 1], deg, 2) == (2, 2)
    # LRU on the same trace evicts A at C's first read: A B C A B C C -> only the last C
    assert oracle.cache_lru([0, 1, 2, 0, 1, 2, 2], [1, 1, 1], 2) == (1, 1)
    # bytes, 5-byte cache, sizes A 3, B 2, C 2: A B -> 5 bytes; C evicts B (A scores
    # higher) -> {A, C}; A hits (3 bytes); B evicts C -> {A, B}; B hits (2 bytes)
    assert oracle.cache_score([0, 1, 2, 0, 1, 1], [3, 2, 2], deg, 5) == (2, 5)
    # the victims go lowest first until the entry fits: sizes A 2, B 2, C 1, D 4 in 5
    # bytes, scores A > B > C > D; A B C fill the 5 bytes, D evicts C, B and A (2 + 4
    # is still above 5 after C and B), then A evicts D and B and C fit beside A
    deg4 = [4, 3, 2, 1]
    assert oracle.cache_score([0, 1, 2, 3, 0, 1, 2], [2, 2, 1, 4], deg4, 5) == (0, 0)
    # the same start, then D read again: it hits (4 bytes)
    assert oracle.cache_score([0, 1, 2, 3, 3], [2, 2, 1, 4], deg4, 5) == (1, 4)
    # an entry larger than the cache is not stored and leaves the cache as it was
    assert oracle.cache_score([0, 3, 0], [2, 2, 1, 9], deg4, 5) == (1, 2)
    # (LRU, by its stack reading, lets an entry larger than the cache push out the rest)
    assert oracle.cache_lru([0, 3, 0], [2, 2, 1, 9], 5) == (0, 0)
    # equal degrees: the larger id scores higher, so C evicts id 0 and keeps id 1
    assert oracle.cache_score([0, 1, 2, 0], [1, 1, 1], [5, 5, 5], 2) == (0, 0)
    assert oracle.cache_score([0, 1, 2, 1], [1, 1, 1], [5, 5, 5], 2) == (1, 1)


@pytest.mark.parametrize("seed", range(40))
def test_cache_priority_with_recency_scores_is_lru(seed):
    """With the time of the latest read as the score, evicting the lowest score is
    evicting the least recently used entry: the priority cache must give LRU's hits
    at every capacity that holds the largest entry."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 12))
    items = rng.integers(0, k, size=int(rng.integers(0, 60))).astype(np.int32)
    size_of = np.ones(k, np.uint64) if seed % 3 == 0 else rng.integers(1, 9, size=k).astype(np.uint64)
    recency = np.arange(items.size, dtype=np.int64)
    for cap in range(int(size_of.max()), 2 + int(size_of.sum())):
        assert oracle.cache_priority(items, size_of, recency, cap) == oracle.cache_lru(items, size_of, cap)


@pytest.mark.parametrize("seed", range(30))
def test_cache_priority_with_next_use_scores_is_optimal(seed):
    """Unit entries with minus the time of the next read as the score: evicting the
    lowest score evicts the entry needed furthest in the future, which is Belady's
    optimal policy among those that store every miss.  Its hits must equal the
    exhaustive optimum at every capacity."""
    rng = np.random.default_rng(seed + 100)
    k = int(rng.integers(2, 6))
    items = [int(x) for x in rng.integers(0, k, size=int(rng.integers(1, 13)))]
    nxt = []
    for t, x in enumerate(items):
        later = [u for u in range(t + 1, len(items)) if items[u] == x]
        nxt.append(-(later[0] if later else len(items) + 1))
    for cap in range(0, k + 1):
        got = oracle.cache_priority(items, np.ones(k, np.uint64), nxt, cap)
        assert got[0] == _brute_optimal_hits(tuple(items), cap), (items, cap)


@pytest.mark.parametrize("seed", range(40))
def test_cache_policies_limits(seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 12))
    items = rng.integers(0, k, size=int(rng.integers(0, 60))).astype(np.int32)
    unit = seed % 3 == 0
    size_of = np.ones(k, np.uint64) if unit else rng.integers(1, 9, size=k).astype(np.uint64)
    degree = rng.integers(0, 5, size=k).astype(np.int64)
    s = [int(x) for x in size_of]
    lst = [int(x) for x in items]
    prev_h = (0, 0)
    for cap in range(0, 2 + int(size_of.sum())):
        got = oracle.cache_lru(items, size_of, cap)
        assert got == _brute_lru_hits(lst, s, cap)
        assert got[0] >= prev_h[0]  # inclusion: a larger LRU cache never hits less
        prev_h = got
        sc = oracle.cache_score(items, size_of, degree, cap)
        # a read can only hit an entry read before that fits in the cache
        assert sc[0] <= sum(1 for t, x in enumerate(lst) if x in lst[:t] and s[x] <= cap)
    # a cache holding everything misses only the first read of each item
    big = int(size_of.sum())
    assert oracle.cache_lru(items, size_of, big)[0] == len(lst) - len(set(lst))
    assert oracle.cache_score(items, size_of, degree, big)[0] == len(lst) - len(set(lst))
    assert oracle.cache_lru(items, size_of, 0) == (0, 0)
    assert oracle.cache_score(items, size_of, degree, 0) == (0, 0)


def _cut_reads(n, s, d, parts):
    """Remote reads counted from the edges: an edge whose ends lie in different
    processes is read once from each end."""
    A = F.dense_adjacency(n, s, d)
    own = np.array([((i + 1) * parts - 1) // n for i in range(n)])
    per = np.zeros(parts, np.int64)
    for i in range(n):
        for j in range(n):
            if A[i, j] and own[i] != own[j]:
                per[own[i]] += 1
    return per, own, A


@pytest.mark.parametrize("seed,parts", [(s, p) for s in range(10) for p in (1, 2, 3, 4, 8)])
def test_remote_reads_match_the_cut(seed, parts):
    n, s, d = _tiny(seed)
    offsets, adj, _ = oracle.build_csr(n, s, d)
    items, part = oracle.remote_reads(n, offsets, adj, parts)
    per, own, A = _cut_reads(n, s, d, parts)
    np.testing.assert_array_equal(np.bincount(part, minlength=parts), per)
    assert (own[items] != part).all()
    # order: each process walks its vertices and their sorted lists in id order
    rows = np.repeat(np.arange(n), np.diff(offsets))
    remote = own[rows] != own[adj]
    np.testing.assert_array_equal(items, adj[remote])


@pytest.mark.parametrize("n,parts", [(8, 2), (12, 3), (16, 4), (9, 1)])
def test_remote_reads_complete_graph(n, parts):
    nn, (s, d) = F.complete(n)
    r = oracle.remote_cache(nn, s, d, parts, [0, 10 ** 9])
    # every vertex reads the n - n/p vertices of the other processes
    assert (r["reads"] == (n // parts) * (n - n // parts)).all()
    assert (r["distinct"] == n - n // parts).all()
    # unbounded caches miss only the first read of each remote list
    assert (r["hits"][:, :, 1] == (r["reads"] - r["distinct"])[None, :]).all()
    assert (r["hits"][:, :, 0] == 0).all()
    assert (r["read_bytes"] == 4 * (n - 1) * r["reads"]).all()


def test_remote_reads_star_top_share():
    nn, (s, d) = F.star(99)  # hub 0 and 99 leaves; two processes of 50
    r = oracle.remote_cache(nn, s, d, 2, [4 * 99, 4 * 99 - 1])
    # process 0 (hub + 49 leaves) reads the 50 leaves of process 1; they read the hub
    np.testing.assert_array_equal(r["reads"], [50, 50])
    np.testing.assert_array_equal(r["distinct"], [50, 1])
    # the top 10 by (degree, id): the hub and leaves 99..91
    np.testing.assert_array_equal(r["top_reads"], [9, 50])
    # process 1 reads the hub's 396-byte list 50 times: 49 hits iff it fits
    assert r["hits"][0, 1, 0] == 49 and r["hits"][0, 1, 1] == 0
    assert r["hits"][1, 1, 0] == 49 and r["hits"][1, 1, 1] == 0


@pytest.mark.parametrize("seed", range(4))
def test_remote_cache_brute_force(seed):
    n, s, d = _tiny(seed + 20)
    parts = 2 + seed % 3
    offsets, adj, _ = oracle.build_csr(n, s, d)
    deg = [int(x) for x in np.diff(offsets)]
    caps = [0, 4, 16, 40, 100, 400]
    r = oracle.remote_cache(n, s, d, parts, caps)
    items, part = oracle.remote_reads(n, offsets, adj, parts)
    for k in range(parts):
        it = [int(x) for x in items[part == k]]
        for c, cap in enumerate(caps):
            assert tuple(int(x) for x in (r["hits"][0, k, c], r["hit_bytes"][0, k, c])) == \
                _brute_lru_hits(it, [4 * x for x in deg], cap)
            assert tuple(int(x) for x in (r["hits"][1, k, c], r["hit_bytes"][1, k, c])) == \
                oracle.cache_score(it, [4 * x for x in deg], deg, cap)
            assert int(r["hits"][2, k, c]) == _brute_lru_hits(it, [16] * n, cap)[0]
            assert int(r["hits"][3, k, c]) == oracle.cache_score(it, [16] * n, deg, cap)[0]
