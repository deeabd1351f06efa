"""Graphs with known triangle counts, and brute-force counters, for pinning.

Everything here is independent of the oracle's arithmetic: the closed forms are
textbook results and the brute-force counters enumerate vertex triples or use a
dense matrix power.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def as_arrays(edges):
    e = np.asarray(list(edges), dtype=np.int32).reshape(-1, 2)
    return np.ascontiguousarray(e[:, 0]), np.ascontiguousarray(e[:, 1])


def complete(n):
    """K_n: T = C(n,3), t = C(n-1,2), LCC = 1."""
    return n, as_arrays(itertools.combinations(range(n), 2))


def star(leaves):
    return leaves + 1, as_arrays((0, i) for i in range(1, leaves + 1))


def cycle(n):
    return n, as_arrays((i, (i + 1) % n) for i in range(n))


def path(n):
    return n, as_arrays((i, i + 1) for i in range(n - 1))


def grid(r, c):
    e = []
    for i in range(r):
        for j in range(c):
            v = i * c + j
            if j + 1 < c:
                e.append((v, v + 1))
            if i + 1 < r:
                e.append((v, v + c))
    return r * c, as_arrays(e)


def complete_bipartite(a, b):
    return a + b, as_arrays((i, a + j) for i in range(a) for j in range(b))


def random_tree(n, rng):
    return n, as_arrays((i, int(rng.integers(0, i))) for i in range(1, n))


def wheel(n):
    """W_n: hub 0 joined to a rim cycle 1..n-1 (n-1 >= 3)."""
    k = n - 1
    e = [(0, i) for i in range(1, n)] + [(1 + i, 1 + (i + 1) % k) for i in range(k)]
    return n, as_arrays(e)


def friendship(k):
    """F_k: k triangles sharing vertex 0."""
    e = []
    for i in range(k):
        a, b = 1 + 2 * i, 2 + 2 * i
        e += [(0, a), (0, b), (a, b)]
    return 2 * k + 1, as_arrays(e)


def complete_tripartite(a, b, c):
    parts = [range(0, a), range(a, a + b), range(a + b, a + b + c)]
    e = [(x, y) for p, q in itertools.combinations(parts, 2) for x in p for y in q]
    return a + b + c, as_arrays(e)


def dense_adjacency(n, src, dst):
    A = np.zeros((n, n), dtype=np.int64)
    for u, v in zip(src.tolist(), dst.tolist()):
        if u != v:
            A[u, v] = 1
            A[v, u] = 1
    return A


def brute_triples(n, src, dst):
    """O(n^3) enumeration of vertex triples i < j < k that are pairwise adjacent."""
    A = dense_adjacency(n, src, dst)
    t = np.zeros(n, dtype=np.uint64)
    T = 0
    for i in range(n):
        for j in range(i + 1, n):
            if not A[i, j]:
                continue
            for k in range(j + 1, n):
                if A[i, k] and A[j, k]:
                    T += 1
                    t[i] += 1
                    t[j] += 1
                    t[k] += 1
    return T, t


def brute_matrix(n, src, dst):
    """t = diag(A^3) / 2 and T = trace(A^3) / 6 with a dense integer matrix power."""
    A = dense_adjacency(n, src, dst)
    d = np.diag(A @ A @ A)
    return int(d.sum()) // 6, (d // 2).astype(np.uint64)


def exact_lcc(t, deg):
    """Eq. 2 rounded once from the exact rational (0.0 for degree < 2)."""
    out = np.zeros(len(t), dtype=np.float64)
    for i, (ti, di) in enumerate(zip(t.tolist(), deg.tolist())):
        if di >= 2:
            out[i] = float(Fraction(2 * int(ti), int(di) * (int(di) - 1)))
    return out


# ---------------------------------------------------------------------------
# Directed graphs (Eq. 1): e_ij from v_i to v_j, adj(v_i) = out-neighbours.

def dense_digraph(n, src, dst):
    """0/1 matrix with A[u, v] = 1 for every pair u -> v, u != v (repeats collapse)."""
    A = np.zeros((n, n), dtype=np.int64)
    for u, v in zip(src.tolist(), dst.tolist()):
        if u != v:
            A[u, v] = 1
    return A


def brute_directed(n, src, dst):
    """c(i) = number of ordered pairs (j, k), j != k, with i -> j, i -> k and j -> k,
    by enumerating vertex triples."""
    A = dense_digraph(n, src, dst)
    c = np.zeros(n, dtype=np.uint64)
    for i in range(n):
        out = [j for j in range(n) if A[i, j]]
        for j in out:
            for k in out:
                if j != k and A[j, k]:
                    c[i] += 1
    return c


def exact_directed_lcc(c, dout):
    """Eq. 1 rounded once from the exact rational (0.0 for out-degree < 2)."""
    out = np.zeros(len(c), dtype=np.float64)
    for i, (ci, di) in enumerate(zip(c.tolist(), dout.tolist())):
        if di >= 2:
            out[i] = float(Fraction(int(ci), int(di) * (int(di) - 1)))
    return out


def transitive_tournament(n):
    """i -> j for every i < j: out(i) = {i+1, ..., n-1} and every pair j < k of it has j -> k."""
    return n, as_arrays((i, j) for i in range(n) for j in range(i + 1, n))


def complete_digraph(n):
    return n, as_arrays((i, j) for i in range(n) for j in range(n) if i != j)


def directed_wheel(rim, outward=True):
    """Hub 0 and a rim cycle 1 -> 2 -> ... -> rim -> 1; spokes hub -> rim (outward)
    or rim -> hub."""
    spokes = [(0, r) if outward else (r, 0) for r in range(1, rim + 1)]
    cyc = [(r, r % rim + 1) for r in range(1, rim + 1)]
    return rim + 1, as_arrays(spokes + cyc)
