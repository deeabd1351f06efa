"""CPU oracle for triangle counting and LCC (arxiv 2202.13976).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the library's product
path never does, and this package imports nothing from it.

The arithmetic lives in ``tc_oracle.cpp`` (plain single-threaded C++, std::sort
as the only library step); this module compiles it on first use and marshals
numpy arrays.  Every function names the passage of the paper it follows:

- ``build_csr``: Sec. II-A (simple undirected graph) and II-B (CSR).
- ``orient``: the upper-triangle offset of Sec. II-C, taken in (degree, id) order.
- ``ssi`` / ``binary_search`` / ``prefer_ssi``: Alg. 2, Alg. 1 (textbook reading),
  Eq. 3.
- ``tc_oriented``: edge-centric counting of Sec. II-C with Alg. 2.
- ``tc_vertex``: the paper's per-vertex formula (Alg. 3) with the Eq. 3 hybrid.
- ``lcc``: Eq. 2.
- ``build_digraph`` / ``directed_lcc``: directed graphs (Sec. II-A) and Eq. 1.
- ``remote_reads`` / ``cache_lru`` / ``cache_priority`` / ``cache_score`` /
  ``remote_cache``: the remote reads of the 1D-partitioned algorithm (Sec. IV-A,
  Alg. 4) and the simulated caches of Sec. IV-B (LRU; eviction of the lowest
  application-defined score, with the degree score of TC).

Parity status: every function is pinned by the ``-m "not gpu"`` tests
(brute force, closed forms, scipy's sparse product for the algebraic form
C = A A o A of Sec. VI-B, invariants).  The absolute totals of the large R-MAT
and ER workloads are printed nowhere in the paper; they are pinned only by the
agreement of the two independent formulas here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tc_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lib = None
_lock = threading.Lock()

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile tc_oracle.cpp into _oracle.so (plain -O2, single-threaded)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64 = ctypes.c_int64
            lib.or_build_csr.restype = ctypes.c_int
            lib.or_build_csr.argtypes = [i64, i64, _i32p, _i32p, _i64p, _i32p, _i64p]
            lib.or_orient.restype = None
            lib.or_orient.argtypes = [i64, _i64p, _i32p, _i64p, _i32p]
            lib.or_ssi.restype = i64
            lib.or_ssi.argtypes = [_i32p, i64, _i32p, i64]
            lib.or_binary_search.restype = i64
            lib.or_binary_search.argtypes = [_i32p, i64, _i32p, i64]
            lib.or_prefer_ssi.restype = ctypes.c_int
            lib.or_prefer_ssi.argtypes = [i64, i64]
            lib.or_tc_oriented.restype = None
            lib.or_tc_oriented.argtypes = [i64, _i64p, _i32p, _u64p, i64, i64]
            lib.or_tc_vertex.restype = None
            lib.or_tc_vertex.argtypes = [i64, _i64p, _i32p, _i32p, i64, _u64p]
            lib.or_lcc.restype = None
            lib.or_lcc.argtypes = [i64, _i64p, _u64p, _f64p]
            lib.or_edge_support.restype = i64
            lib.or_edge_support.argtypes = [i64, _i64p, _i32p, _i32p, _i32p, ctypes.POINTER(ctypes.c_uint32)]
            lib.or_build_digraph.restype = ctypes.c_int
            lib.or_build_digraph.argtypes = [i64, i64, _i32p, _i32p, _i64p, _i32p, _i64p]
            lib.or_remote_reads.restype = i64
            lib.or_remote_reads.argtypes = [i64, _i64p, _i32p, i64, _i32p, _i32p]
            lib.or_cache_lru.restype = ctypes.c_uint64
            lib.or_cache_lru.argtypes = [i64, _i32p, _u64p, ctypes.c_uint64, _u64p]
            lib.or_cache_priority.restype = ctypes.c_uint64
            lib.or_cache_priority.argtypes = [i64, _i32p, _u64p, _i64p, ctypes.c_uint64, _u64p]
            lib.or_cache_score.restype = ctypes.c_uint64
            lib.or_cache_score.argtypes = [i64, _i32p, _u64p, _i64p, ctypes.c_uint64, _u64p]
            lib.or_directed_lcc.restype = None
            lib.or_directed_lcc.argtypes = [i64, _i64p, _i32p, _i32p, i64, _u64p, _f64p]
            _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def build_csr(n: int, src, dst):
    """Sec. II-A/B: (offsets int64[n+1], adj int32[2m'], stats) of the simple graph.

    stats = {"m_simple", "loops_dropped", "dups_dropped"}.  Raises ValueError on an
    id outside [0, n)."""
    src = _c(src, np.int32)
    dst = _c(dst, np.int32)
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    m = src.size
    offsets = np.zeros(n + 1, dtype=np.int64)
    adj = np.empty(max(1, 2 * m), dtype=np.int32)
    stats = np.zeros(3, dtype=np.int64)
    rc = _load().or_build_csr(n, m, _p(src, _i32p), _p(dst, _i32p), _p(offsets, _i64p),
                              _p(adj, _i32p), _p(stats, _i64p))
    if rc != 0:
        raise ValueError("vertex id outside [0, n)")
    adj = adj[: offsets[-1]].copy()
    return offsets, adj, {"m_simple": int(stats[0]), "loops_dropped": int(stats[1]),
                          "dups_dropped": int(stats[2])}


def edges_from_csr(n: int, offsets, adj):
    """Every CSR entry (i, adj[k]) read as the undirected pair {i, adj[k]}."""
    offsets = _c(offsets, np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int32), np.diff(offsets))
    return rows, _c(adj, np.int32)[: offsets[-1]]


def degrees(offsets) -> np.ndarray:
    return np.diff(_c(offsets, np.int64))


def orient(n: int, offsets, adj):
    """Oriented CSR: u -> v iff (deg u, u) < (deg v, v); rows sorted by id."""
    offsets = _c(offsets, np.int64)
    adj = _c(adj, np.int32)
    off_plus = np.zeros(n + 1, dtype=np.int64)
    adj_plus = np.empty(max(1, adj.size // 2), dtype=np.int32)
    _load().or_orient(n, _p(offsets, _i64p), _p(adj, _i32p), _p(off_plus, _i64p), _p(adj_plus, _i32p))
    return off_plus, adj_plus[: off_plus[-1]].copy()


def ssi(A, B) -> int:
    """Alg. 2 on sorted int32 lists."""
    A = _c(A, np.int32)
    B = _c(B, np.int32)
    return int(_load().or_ssi(_p(A, _i32p), A.size, _p(B, _i32p), B.size))


def binary_search(A, B) -> int:
    """Alg. 1 (textbook reading): keys A looked up in sorted B."""
    A = _c(A, np.int32)
    B = _c(B, np.int32)
    return int(_load().or_binary_search(_p(A, _i32p), A.size, _p(B, _i32p), B.size))


def prefer_ssi(a: int, b: int) -> bool:
    """Eq. 3: SSI iff |B|/|A| <= log2|B| - 1 with |A| <= |B|."""
    return bool(_load().or_prefer_ssi(a, b))


def tc_oriented(n: int, off_plus, adj_plus, threads: int = 1) -> np.ndarray:
    """Sec. II-C edge-centric count on the oriented CSR -> t uint64[n].

    ``threads`` > 1 splits the source vertices into ranges, each run by the same
    single-threaded routine into its own array; the arrays are summed."""
    off_plus = _c(off_plus, np.int64)
    adj_plus = _c(adj_plus, np.int32)
    lib = _load()
    if threads <= 1 or n < 1024:
        t = np.zeros(n, dtype=np.uint64)
        lib.or_tc_oriented(n, _p(off_plus, _i64p), _p(adj_plus, _i32p), _p(t, _u64p), 0, n)
        return t
    # ranges of roughly equal oriented-edge work (sum over u of d+(u)^2 + d+(u))
    d = np.diff(off_plus).astype(np.float64)
    w = np.cumsum(d * d + d + 1.0)
    cuts = np.searchsorted(w, np.linspace(0, w[-1], 8 * threads + 1)[1:-1])
    bounds = [0] + [int(c) for c in cuts] + [n]
    parts = []
    jobs = list(zip(bounds[:-1], bounds[1:]))
    jl = threading.Lock()

    def worker():
        t = np.zeros(n, dtype=np.uint64)
        while True:
            with jl:
                if not jobs:
                    break
                u0, u1 = jobs.pop()
            lib.or_tc_oriented(n, _p(off_plus, _i64p), _p(adj_plus, _i32p), _p(t, _u64p), u0, u1)
        parts.append(t)

    ths = [threading.Thread(target=worker) for _ in range(threads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    return np.sum(parts, axis=0, dtype=np.uint64)


def tc_oriented_ranges(n: int, off_plus, adj_plus, ranges, threads: int = 1) -> np.ndarray:
    """The Sec. II-C oriented count restricted to the source vertices of the listed
    half-open ranges [u0, u1) -> partial t uint64[n] (every triangle whose lowest
    oriented edge starts in a listed range adds to its three corners); the ranges are
    shared among ``threads`` threads, each summing into its own array."""
    off_plus = _c(off_plus, np.int64)
    adj_plus = _c(adj_plus, np.int32)
    lib = _load()
    jobs = [(int(a), int(b)) for a, b in ranges]
    parts = []
    jl = threading.Lock()

    def worker():
        t = np.zeros(n, dtype=np.uint64)
        while True:
            with jl:
                if not jobs:
                    break
                u0, u1 = jobs.pop()
            lib.or_tc_oriented(n, _p(off_plus, _i64p), _p(adj_plus, _i32p), _p(t, _u64p), u0, u1)
        parts.append(t)

    ths = [threading.Thread(target=worker) for _ in range(max(1, threads))]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    return np.sum(parts, axis=0, dtype=np.uint64)


def work_ranges(off_plus, pieces: int):
    """``pieces`` half-open source ranges of roughly equal oriented-count work
    (d+(u)^2 + d+(u) + 1 per source u), covering [0, n)."""
    d = np.diff(_c(off_plus, np.int64)).astype(np.float64)
    n = d.size
    w = np.cumsum(d * d + d + 1.0)
    cuts = np.searchsorted(w, np.linspace(0, w[-1], pieces + 1)[1:-1]) if n else []
    bounds = [0] + [int(c) for c in cuts] + [n]
    return [(a, b) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]


def tc_vertex(n: int, offsets, adj, vertices) -> np.ndarray:
    """Alg. 3 per-vertex formula (symmetric CSR, Eq. 3 hybrid) for the listed vertices."""
    offsets = _c(offsets, np.int64)
    adj = _c(adj, np.int32)
    vertices = _c(vertices, np.int32)
    out = np.zeros(vertices.size, dtype=np.uint64)
    _load().or_tc_vertex(n, _p(offsets, _i64p), _p(adj, _i32p), _p(vertices, _i32p),
                         vertices.size, _p(out, _u64p))
    return out


def edge_support(n: int, src, dst):
    """Per-edge triangle counts of the simple graph: (u, v, support) with one entry per
    undirected edge, u < v, sorted by (u, v); support = |adj(u) ∩ adj(v)| (Alg. 2)."""
    offsets, adj, _ = build_csr(n, src, dst)
    m = int(offsets[-1]) // 2
    eu = np.empty(max(1, m), dtype=np.int32)
    ev = np.empty(max(1, m), dtype=np.int32)
    sup = np.empty(max(1, m), dtype=np.uint32)
    got = _load().or_edge_support(n, _p(offsets, _i64p), _p(adj, _i32p), _p(eu, _i32p), _p(ev, _i32p),
                                  sup.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    assert got == m
    return eu[:m], ev[:m], sup[:m]


def build_digraph(n: int, src, dst):
    """Directed simple graph (Sec. II-A: e_ij from v_i to v_j, no loops, no repeated
    pair): (offsets int64[n+1], adj int32[m'], stats) with sorted out-lists.

    stats = {"m_directed", "loops_dropped", "dups_dropped"}.  Raises ValueError on an
    id outside [0, n)."""
    src = _c(src, np.int32)
    dst = _c(dst, np.int32)
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    m = src.size
    offsets = np.zeros(n + 1, dtype=np.int64)
    adj = np.empty(max(1, m), dtype=np.int32)
    stats = np.zeros(3, dtype=np.int64)
    rc = _load().or_build_digraph(n, m, _p(src, _i32p), _p(dst, _i32p), _p(offsets, _i64p),
                                  _p(adj, _i32p), _p(stats, _i64p))
    if rc != 0:
        raise ValueError("vertex id outside [0, n)")
    adj = adj[: offsets[-1]].copy()
    return offsets, adj, {"m_directed": int(stats[0]), "loops_dropped": int(stats[1]),
                          "dups_dropped": int(stats[2])}


def directed_lcc(n: int, src, dst, vertices=None) -> dict:
    """Eq. 1 on the directed simple graph of (src[k] -> dst[k]).

    Returns {"c", "lcc", "out_degree", "m_directed", "loops_dropped", "dups_dropped"};
    c[q] = |{e_jk : v_j, v_k in adj(v_i)}| and lcc[q] = c / (deg+ (deg+ - 1)) for
    i = vertices[q] (all vertices when ``vertices`` is None)."""
    offsets, adj, stats = build_digraph(n, src, dst)
    vertices = np.arange(n, dtype=np.int32) if vertices is None else _c(vertices, np.int32)
    c = np.zeros(vertices.size, dtype=np.uint64)
    l = np.zeros(vertices.size, dtype=np.float64)
    _load().or_directed_lcc(n, _p(offsets, _i64p), _p(adj, _i32p), _p(vertices, _i32p), vertices.size,
                            _p(c, _u64p), _p(l, _f64p))
    out = {"c": c, "lcc": l, "out_degree": np.diff(offsets)[vertices]}
    out.update(stats)
    return out


def remote_reads(n: int, offsets, adj, parts: int):
    """Alg. 4 over a 1D partition into ``parts`` processes (process k owns ids
    [k n / p, (k+1) n / p)): (item int32[N], process int32[N]) of every remote read of an
    adjacency list, processes in order, each walking its vertices and their sorted
    adjacency lists in id order."""
    offsets = _c(offsets, np.int64)
    adj = _c(adj, np.int32)
    cap = max(1, adj.size)
    items = np.empty(cap, dtype=np.int32)
    part = np.empty(cap, dtype=np.int32)
    N = _load().or_remote_reads(n, _p(offsets, _i64p), _p(adj, _i32p), parts, _p(items, _i32p), _p(part, _i32p))
    return items[:N].copy(), part[:N].copy()


def cache_lru(items, size_of, capacity: int):
    """Sec. IV-B, LRU cache of ``capacity`` bytes over one process's reads; entry sizes
    size_of[item] bytes.  Returns (hits, hit bytes)."""
    items = _c(items, np.int32)
    size_of = _c(size_of, np.uint64)
    hb = ctypes.c_uint64()
    h = _load().or_cache_lru(items.size, _p(items, _i32p), _p(size_of, _u64p), int(capacity), ctypes.byref(hb))
    return int(h), int(hb.value)


def cache_priority(items, size_of, score_at, capacity: int):
    """Sec. IV-B2, a cache of ``capacity`` bytes with application-defined scores: the
    victim is the cached entry of the lowest score (the score given with its latest
    read, score_at[t]); a miss is stored after evicting the lowest entries until it
    fits, unless it is larger than the whole cache.  Returns (hits, hit bytes)."""
    items = _c(items, np.int32)
    size_of = _c(size_of, np.uint64)
    score_at = _c(score_at, np.int64)
    if score_at.shape != items.shape:
        raise ValueError("one score per read")
    hb = ctypes.c_uint64()
    h = _load().or_cache_priority(items.size, _p(items, _i32p), _p(size_of, _u64p), _p(score_at, _i64p),
                                  int(capacity), ctypes.byref(hb))
    return int(h), int(hb.value)


def cache_score(items, size_of, degree, capacity: int):
    """Sec. IV-B2, the degree score of TC: ``cache_priority`` with the score of v_j's
    entry = (degree(v_j), v_j).  Returns (hits, hit bytes)."""
    items = _c(items, np.int32)
    size_of = _c(size_of, np.uint64)
    degree = _c(degree, np.int64)
    hb = ctypes.c_uint64()
    h = _load().or_cache_score(items.size, _p(items, _i32p), _p(size_of, _u64p), _p(degree, _i64p), int(capacity),
                               ctypes.byref(hb))
    return int(h), int(hb.value)


OFFSET_ENTRY_BYTES = 16  # a (start, end) pair of 64-bit offsets


def remote_cache(n: int, src, dst, parts: int, capacities) -> dict:
    """The remote reads of Alg. 4 on the simple graph of (src, dst) and the four
    simulated caches of Sec. IV-B at every capacity (bytes).

    Returns {"reads", "top_reads", "distinct", "read_bytes": int64[parts],
    "hits", "hit_bytes": uint64[4, parts, len(capacities)]} with cache index 0 =
    adjacency lists / LRU, 1 = adjacency lists / degree score, 2 = offsets / LRU,
    3 = offsets / degree score; an adjacency entry holds 4 deg(v_j) bytes, an offsets
    entry 16.  top_reads counts the reads of the ceil(n / 10) vertices of highest
    (degree, id)."""
    offsets, adj, _ = build_csr(n, src, dst)
    deg = np.diff(offsets)
    items, part = remote_reads(n, offsets, adj, parts)
    caps = [int(c) for c in capacities]
    order = sorted(range(n), key=lambda v: (int(deg[v]), v), reverse=True)
    top = np.zeros(n, dtype=bool)
    top[order[: (n + 9) // 10]] = True
    size_adj = (4 * deg).astype(np.uint64)
    size_off = np.full(n, OFFSET_ENTRY_BYTES, dtype=np.uint64)
    hits = np.zeros((4, parts, len(caps)), dtype=np.uint64)
    hit_bytes = np.zeros((4, parts, len(caps)), dtype=np.uint64)
    reads = np.zeros(parts, dtype=np.int64)
    top_reads = np.zeros(parts, dtype=np.int64)
    distinct = np.zeros(parts, dtype=np.int64)
    read_bytes = np.zeros(parts, dtype=np.int64)
    for k in range(parts):
        it = items[part == k]
        reads[k] = it.size
        top_reads[k] = int(top[it].sum())
        distinct[k] = np.unique(it).size
        read_bytes[k] = int(size_adj[it].sum())
        for c, cap in enumerate(caps):
            hits[0, k, c], hit_bytes[0, k, c] = cache_lru(it, size_adj, cap)
            hits[1, k, c], hit_bytes[1, k, c] = cache_score(it, size_adj, deg, cap)
            hits[2, k, c], hit_bytes[2, k, c] = cache_lru(it, size_off, cap)
            hits[3, k, c], hit_bytes[3, k, c] = cache_score(it, size_off, deg, cap)
    return {"reads": reads, "top_reads": top_reads, "distinct": distinct, "read_bytes": read_bytes,
            "hits": hits, "hit_bytes": hit_bytes}


def lcc(n: int, offsets, t) -> np.ndarray:
    """Eq. 2 in fp64 (0.0 for degree < 2)."""
    offsets = _c(offsets, np.int64)
    t = _c(t, np.uint64)
    out = np.empty(n, dtype=np.float64)
    _load().or_lcc(n, _p(offsets, _i64p), _p(t, _u64p), _p(out, _f64p))
    return out


def triangles(n: int, src, dst, threads: int = 1) -> dict:
    """Whole pipeline: simple graph, orientation, oriented count, T, LCC.

    Returns {"T", "t", "lcc", "degree", "m_simple", "loops_dropped", "dups_dropped",
    "m_oriented"}.  Asserts sum(t) = 3T (each triangle adds 1 to each corner)."""
    offsets, adj, stats = build_csr(n, src, dst)
    off_plus, adj_plus = orient(n, offsets, adj)
    t = tc_oriented(n, off_plus, adj_plus, threads=threads)
    s = int(t.sum(dtype=np.uint64))
    assert s % 3 == 0, "sum of per-vertex counts is not a multiple of 3"
    out = {"T": s // 3, "t": t, "lcc": lcc(n, offsets, t), "degree": degrees(offsets),
           "m_oriented": int(off_plus[-1])}
    out.update(stats)
    return out


def triangles_csr(n: int, offsets, adj, threads: int = 1) -> dict:
    """``triangles`` for a CSR input: every entry (i, adj[k]) is the pair {i, adj[k]}."""
    src, dst = edges_from_csr(n, offsets, adj)
    return triangles(n, src, dst, threads=threads)
