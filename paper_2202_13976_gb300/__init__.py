"""Triangle counting and LCC on a GB300 GPU: Python binding of libtc (include/tc.h).

The binding only marshals arguments: every step of the computation runs in the
CUDA library.  The functions carry the C ABI's names; device buffers are passed as
PyTorch CUDA tensors (PyTorch supplies device memory and streams only), host
buffers as numpy arrays.  There is no CPU path: if libtc.so cannot be loaded every
call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB, build as _build_lib, source_digest, up_to_date

TC_OK, TC_EINVAL, TC_ENOMEM, TC_ECUDA, TC_ETIMEOUT, TC_EBUSY, TC_EINTERNAL = range(7)
TC_MEM_HOST, TC_MEM_DEVICE = 0, 1
TC_STRAT_AUTO, TC_STRAT_MERGE, TC_STRAT_SEARCH, TC_STRAT_PROBE, TC_STRAT_BITMAP, TC_STRAT_HASH = range(6)
TC_BUCKET_SMALL, TC_BUCKET_CTA, TC_BUCKET_HUB = 0, 1, 2
BUCKETS = {"small": TC_BUCKET_SMALL, "cta": TC_BUCKET_CTA, "hub": TC_BUCKET_HUB}
PHASES = ["plan_ms", "small_ms", "cta_ms", "hub_ms", "total_ms"]
STRATEGIES = {"auto": TC_STRAT_AUTO, "merge": TC_STRAT_MERGE, "search": TC_STRAT_SEARCH,
              "probe": TC_STRAT_PROBE, "bitmap": TC_STRAT_BITMAP, "hash": TC_STRAT_HASH}

# Every symbol include/tc.h declares.
EXPORTS = ["tc_graph_create_from_edges", "tc_graph_create_from_csr", "tc_count", "lcc_compute",
           "tc_graph_info", "tc_graph_size", "tc_graph_destroy", "tc_status_str",
           "tc_last_error_detail", "tc_graph_set_strategy", "tc_graph_last_timing",
           "tc_graph_plan_stats", "tc_launch_count", "tc_graph_set_hubs", "tc_count_noalloc",
           "tc_batch_create", "tc_batch_count", "tc_batch_size", "tc_graph_get_tuning",
           "tc_graph_set_tuning", "tc_graph_autotune", "tc_batch_run", "tc_release_cached_graphs",
           "tc_generate_edges", "tc_server_start", "tc_server_submit", "tc_server_poll", "tc_server_wait",
           "tc_server_get_stats", "tc_server_stop", "tc_graph_build_timing", "tc_count_vertex_formula",
           "tc_edge_support", "tc_directed_lcc", "tc_remote_cache", "tc_request_run", "tc_count_shard",
           "tc_lcc_from_counts"]
BUILD_PHASES = ["ingest_ms", "rank_ms", "count_ms", "fill_ms", "sort_ms", "degree_ms", "total_ms"]
TC_GEN_RMAT, TC_GEN_ER_REPLACE = 0, 1
GEN_KINDS = {"rmat": TC_GEN_RMAT, "er_replace": TC_GEN_ER_REPLACE}


class TcRequest(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("m", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint64)]


class TcResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("T", ctypes.c_uint64), ("m_simple", ctypes.c_int64), ("t_hash", ctypes.c_uint64),
                ("lcc_hash", ctypes.c_uint64), ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("end_s", ctypes.c_double), ("bytes", ctypes.c_uint64)]

    def to_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


TC_DIRECTED_TIMED = 1


class TcDirectedStats(ctypes.Structure):
    _fields_ = [("m_directed", ctypes.c_int64), ("m_undirected", ctypes.c_int64), ("loops_dropped", ctypes.c_int64),
                ("total", ctypes.c_uint64), ("list_entries", ctypes.c_uint64), ("build_ms", ctypes.c_float),
                ("count_ms", ctypes.c_float), ("finalize_ms", ctypes.c_float), ("pad", ctypes.c_float)]

    def to_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class TcServerStats(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("budget_bytes", ctypes.c_uint64), ("submitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("running", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("max_queue", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("in_flight_bytes", ctypes.c_uint64), ("clock_s", ctypes.c_double)]
TC_RUN_GRAPH = 1


class TcTuning(ctypes.Structure):
    """struct tc_tuning of include/tc.h."""
    _fields_ = [("strategy", ctypes.c_int32 * 3), ("factor", ctypes.c_double * 3),
                ("hub_min_degree", ctypes.c_int32), ("hub_max", ctypes.c_int32), ("hub_big_in", ctypes.c_int32),
                ("hub_core", ctypes.c_int32)]

    def to_dict(self) -> dict:
        names = {v: k for k, v in STRATEGIES.items()}
        return {"strategy": {b: names[self.strategy[i]] for b, i in BUCKETS.items()},
                "factor": {b: self.factor[i] for b, i in BUCKETS.items()},
                "hub_min_degree": self.hub_min_degree, "hub_max": self.hub_max, "hub_big_in": self.hub_big_in,
                "hub_core": self.hub_core}

    @classmethod
    def from_dict(cls, d: dict) -> "TcTuning":
        t = cls()
        for b, i in BUCKETS.items():
            s = d["strategy"][b]
            t.strategy[i] = STRATEGIES[s] if isinstance(s, str) else int(s)
            t.factor[i] = float(d["factor"][b])
        t.hub_min_degree = int(d["hub_min_degree"])
        t.hub_max = int(d["hub_max"])
        t.hub_big_in = int(d["hub_big_in"])
        t.hub_core = int(d.get("hub_core", 8192))
        return t
TC_NOALLOC_MAX_N, TC_NOALLOC_MAX_M = 16384, 262144

_lib = None


class TCError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        msg = _lib.tc_status_str(status).decode() if _lib else f"status {status}"
        super().__init__(f"{msg}{': ' + detail if detail else ''}")


def build(force: bool = False) -> str:
    """Compile libtc.so for sm_103a (nvcc) if it is missing or stale."""
    return _build_lib(force=force)


def load(path: str | None = None):
    """Load libtc.so (building it first when stale) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        if not up_to_date():
            build()
        path = LIB
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    st = ctypes.c_int
    lib.tc_graph_create_from_edges.restype = st
    lib.tc_graph_create_from_edges.argtypes = [i32, i64, P, P, ctypes.c_int, P, ctypes.POINTER(P)]
    lib.tc_graph_create_from_csr.restype = st
    lib.tc_graph_create_from_csr.argtypes = [i32, P, P, ctypes.c_int, P, ctypes.POINTER(P)]
    lib.tc_count.restype = st
    lib.tc_count.argtypes = [P, ctypes.POINTER(u64)]
    lib.lcc_compute.restype = st
    lib.lcc_compute.argtypes = [P, P, P, ctypes.c_int]
    lib.tc_count_shard.restype = st
    lib.tc_count_shard.argtypes = [P, i32, i32, P, ctypes.c_int, ctypes.POINTER(u64)]
    lib.tc_lcc_from_counts.restype = st
    lib.tc_lcc_from_counts.argtypes = [P, P, P, ctypes.c_int]
    lib.tc_count_vertex_formula.restype = st
    lib.tc_count_vertex_formula.argtypes = [P, P, ctypes.c_int, ctypes.POINTER(u64)]
    lib.tc_edge_support.restype = st
    lib.tc_edge_support.argtypes = [P, P, P, P, ctypes.c_int]
    lib.tc_remote_cache.restype = st
    lib.tc_remote_cache.argtypes = [P, i32, i32, P, P, P, P]
    lib.tc_directed_lcc.restype = st
    lib.tc_directed_lcc.argtypes = [i32, i64, P, P, ctypes.c_int, P, P, P, ctypes.POINTER(TcDirectedStats),
                                    ctypes.c_int]
    lib.tc_graph_info.restype = st
    lib.tc_graph_info.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.tc_graph_size.restype = st
    lib.tc_graph_size.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i64)]
    lib.tc_graph_destroy.restype = None
    lib.tc_graph_destroy.argtypes = [P]
    lib.tc_status_str.restype = ctypes.c_char_p
    lib.tc_status_str.argtypes = [st]
    lib.tc_last_error_detail.restype = ctypes.c_char_p
    lib.tc_last_error_detail.argtypes = []
    lib.tc_graph_set_strategy.restype = st
    lib.tc_graph_set_strategy.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    lib.tc_graph_last_timing.restype = st
    lib.tc_graph_last_timing.argtypes = [P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    lib.tc_graph_build_timing.restype = st
    lib.tc_graph_build_timing.argtypes = [P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    lib.tc_graph_set_hubs.restype = st
    lib.tc_graph_set_hubs.argtypes = [P, i32, i32]
    lib.tc_graph_plan_stats.restype = st
    lib.tc_graph_plan_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.tc_launch_count.restype = u64
    lib.tc_launch_count.argtypes = []
    lib.tc_batch_create.restype = st
    lib.tc_batch_create.argtypes = [i32, P, P, P, P, ctypes.c_int, P, ctypes.POINTER(P)]
    lib.tc_batch_count.restype = st
    lib.tc_batch_count.argtypes = [P, P, ctypes.c_int]
    lib.tc_batch_size.restype = st
    lib.tc_batch_size.argtypes = [P, ctypes.POINTER(i32)]
    TP = ctypes.POINTER(TcTuning)
    lib.tc_graph_get_tuning.restype = st
    lib.tc_graph_get_tuning.argtypes = [P, TP]
    lib.tc_graph_set_tuning.restype = st
    lib.tc_graph_set_tuning.argtypes = [P, TP]
    lib.tc_graph_autotune.restype = st
    lib.tc_graph_autotune.argtypes = [P, i32, TP]
    lib.tc_batch_run.restype = st
    lib.tc_batch_run.argtypes = [i32, P, P, P, P, P, P, P, TP, P, ctypes.c_int]
    lib.tc_release_cached_graphs.restype = None
    lib.tc_release_cached_graphs.argtypes = []
    lib.tc_generate_edges.restype = st
    lib.tc_generate_edges.argtypes = [ctypes.c_int, i32, i64, u64, u64, P, P, P]
    lib.tc_server_start.restype = st
    lib.tc_server_start.argtypes = [u64, i32, ctypes.POINTER(P)]
    lib.tc_server_submit.restype = st
    lib.tc_server_submit.argtypes = [P, ctypes.POINTER(TcRequest)]
    lib.tc_server_poll.restype = st
    lib.tc_server_poll.argtypes = [P, ctypes.POINTER(TcResult), i32, ctypes.POINTER(i32)]
    lib.tc_server_wait.restype = st
    lib.tc_server_wait.argtypes = [P, i64, ctypes.c_double]
    lib.tc_server_get_stats.restype = st
    lib.tc_server_get_stats.argtypes = [P, ctypes.POINTER(TcServerStats)]
    lib.tc_server_stop.restype = st
    lib.tc_server_stop.argtypes = [P]
    lib.tc_request_run.restype = st
    lib.tc_request_run.argtypes = [ctypes.POINTER(TcRequest), P, ctypes.POINTER(TcResult)]
    lib.tc_count_noalloc.restype = st
    lib.tc_count_noalloc.argtypes = [i32, i64, P, P, ctypes.POINTER(u64), P, P, P]
    _lib = lib
    return lib


def lib():
    return load()


def _check(status: int):
    if status != TC_OK:
        raise TCError(status, _lib.tc_last_error_detail().decode())


def _is_device(x) -> bool:
    return hasattr(x, "data_ptr") and getattr(x, "is_cuda", False)


def _ptr_kind(*arrays):
    """(pointers, mem_kind) for numpy arrays (host) or torch CUDA tensors (device)."""
    dev = [_is_device(a) for a in arrays if a is not None]
    if dev and any(dev) != all(dev):
        raise ValueError("mix of host and device buffers")
    kind = TC_MEM_DEVICE if dev and dev[0] else TC_MEM_HOST
    ptrs = []
    for a in arrays:
        if a is None:
            ptrs.append(None)
        elif kind == TC_MEM_DEVICE:
            if not a.is_contiguous():
                raise ValueError("device buffers must be contiguous")
            ptrs.append(a.data_ptr())
        else:
            if not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
                raise ValueError("host buffers must be C-contiguous numpy arrays")
            ptrs.append(a.ctypes.data)
    return ptrs, kind


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def tc_graph_create_from_edges(n: int, src, dst, stream=None) -> int:
    """Graph handle from int32 pairs (numpy arrays on the host or CUDA tensors)."""
    load()
    if len(src) != len(dst):
        raise ValueError("src and dst differ in length")
    _check_dtype(src, "int32")
    _check_dtype(dst, "int32")
    (ps, pd), kind = _ptr_kind(src, dst)
    out = ctypes.c_void_p()
    _check(_lib.tc_graph_create_from_edges(n, len(src), ps, pd, kind, _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def tc_graph_create_from_csr(n: int, offsets, adj, stream=None) -> int:
    """Graph handle from CSR arrays (int64 offsets[n+1], int32 adj)."""
    load()
    _check_dtype(offsets, "int64")
    _check_dtype(adj, "int32")
    (po, pa), kind = _ptr_kind(offsets, adj)
    out = ctypes.c_void_p()
    _check(_lib.tc_graph_create_from_csr(n, po, pa, kind, _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def _check_dtype(a, name):
    dt = str(getattr(a, "dtype", ""))
    if not dt.endswith(name):
        raise TypeError(f"expected {name} buffer, got {dt}")


def tc_count(g: int) -> int:
    T = ctypes.c_uint64()
    _check(_lib.tc_count(g, ctypes.byref(T)))
    return int(T.value)


def lcc_compute(g: int, t_out=None, lcc_out=None):
    """Fill caller-allocated t_out (uint64[n]) and lcc_out (float64[n]); either may be None."""
    if t_out is not None:
        _check_dtype(t_out, "int64")
    if lcc_out is not None:
        _check_dtype(lcc_out, "float64")
    if t_out is not None or lcc_out is not None:
        n, _ = tc_graph_size(g)
        _check_room(t_out, n, "t_out")
        _check_room(lcc_out, n, "lcc_out")
    (pt, pl), kind = _ptr_kind(t_out, lcc_out)
    _check(_lib.lcc_compute(g, pt, pl, kind))


def tc_count_shard(g: int, shard: int, nshards: int, t_out=None):
    """Triangles of one shard of the sources (cost-balanced rank ranges) and, when
    t_out (uint64[n] as int64, host numpy or CUDA tensor) is given, the shard's share
    of t(v); returns (T_shard, t_out).  The shares of all shards sum to t(v) and T."""
    if t_out is not None:
        _check_dtype(t_out, "int64")
        n, _ = tc_graph_size(g)
        _check_room(t_out, n, "t_out")
    (pt,), kind = _ptr_kind(t_out)
    T = ctypes.c_uint64()
    _check(_lib.tc_count_shard(g, shard, nshards, pt, kind, ctypes.byref(T)))
    return int(T.value), t_out


def tc_lcc_from_counts(g: int, t, lcc_out):
    """LCC (Eq. 2) into lcc_out (float64[n]) from per-vertex counts t (uint64[n] as
    int64 or uint64), both on the host or both CUDA tensors."""
    _check_dtype(t, "int64")
    _check_dtype(lcc_out, "float64")
    n, _ = tc_graph_size(g)
    _check_room(t, n, "t")
    _check_room(lcc_out, n, "lcc_out")
    (pt, pl), kind = _ptr_kind(t, lcc_out)
    _check(_lib.tc_lcc_from_counts(g, pt, pl, kind))


def tc_count_vertex_formula(g: int, t_out=None):
    """Per-vertex counts by the paper's unoriented per-vertex formula into t_out
    (uint64[n] as int64, host numpy or CUDA tensor; a numpy array is allocated when
    None); returns (T, t_out)."""
    if t_out is None:
        import numpy as np
        n, _ = tc_graph_size(g)
        t_out = np.empty(n, dtype=np.int64)
    _check_dtype(t_out, "int64")
    (pt,), kind = _ptr_kind(t_out)
    T = ctypes.c_uint64()
    _check(_lib.tc_count_vertex_formula(g, pt, kind, ctypes.byref(T)))
    return int(T.value), t_out


def tc_edge_support(g: int, u_out=None, v_out=None, support_out=None):
    """Per-edge triangle counts: (u, v, support) arrays of length m_simple (int32,
    int32, int32 holding the uint32 counts; numpy unless CUDA tensors are passed),
    u < v in the caller's ids, one entry per distinct edge."""
    if u_out is None:
        m = tc_graph_info(g)["m_simple"]
        u_out = np.empty(m, dtype=np.int32)
        v_out = np.empty(m, dtype=np.int32)
        support_out = np.empty(m, dtype=np.int32)
    for a in (u_out, v_out, support_out):
        _check_dtype(a, "int32")
    (pu, pv, ps), kind = _ptr_kind(u_out, v_out, support_out)
    _check(_lib.tc_edge_support(g, pu, pv, ps, kind))
    return u_out, v_out, support_out


CACHE_KINDS = ["adj_lru", "adj_score", "off_lru", "off_score"]


def tc_remote_cache(g: int, parts: int, capacities) -> dict:
    """Remote reads of a 1D partition into ``parts`` processes and the four caches at
    every capacity (bytes, non-decreasing): {"hits", "hit_bytes": uint64[4, parts, ncap]
    (index order CACHE_KINDS), "reads", "top_reads", "distinct", "read_bytes":
    int64[parts]}."""
    caps = np.ascontiguousarray(np.asarray(capacities, dtype=np.uint64))
    ncap = caps.size
    hits = np.zeros((4, parts, ncap), dtype=np.uint64)
    hb = np.zeros((4, parts, ncap), dtype=np.uint64)
    ps = np.zeros((parts, 4), dtype=np.int64)
    _check(_lib.tc_remote_cache(g, parts, ncap, caps.ctypes.data if ncap else None, hits.ctypes.data,
                                hb.ctypes.data, ps.ctypes.data))
    return {"hits": hits, "hit_bytes": hb, "reads": ps[:, 0].copy(), "top_reads": ps[:, 1].copy(),
            "distinct": ps[:, 2].copy(), "read_bytes": ps[:, 3].copy()}


def tc_directed_lcc(n: int, src, dst, c_out=None, lcc_out=None, stream=None, timed=False):
    """Directed LCC (Eq. 1) of the pairs src[k] -> dst[k] (int32; numpy on the host or
    CUDA tensors): fills c_out (uint64[n] as int64) and lcc_out (float64[n]), allocated
    like the inputs when None; returns (c_out, lcc_out, stats dict).  timed: phase
    times from CUDA events and the list entries the count reads."""
    load()
    if len(src) != len(dst):
        raise ValueError("src and dst differ in length")
    _check_dtype(src, "int32")
    _check_dtype(dst, "int32")
    if c_out is None or lcc_out is None:
        if _is_device(src):
            import torch
            if c_out is None:
                c_out = torch.empty(n, dtype=torch.int64, device=src.device)
            if lcc_out is None:
                lcc_out = torch.empty(n, dtype=torch.float64, device=src.device)
        else:
            if c_out is None:
                c_out = np.empty(n, dtype=np.uint64)
            if lcc_out is None:
                lcc_out = np.empty(n, dtype=np.float64)
    _check_dtype(c_out, "int64")
    _check_dtype(lcc_out, "float64")
    (ps, pd, pc, pl), kind = _ptr_kind(src, dst, c_out, lcc_out)
    st = TcDirectedStats()
    _check(_lib.tc_directed_lcc(n, len(src), ps, pd, kind, _stream_ptr(stream), pc, pl, ctypes.byref(st),
                                TC_DIRECTED_TIMED if timed else 0))
    return c_out, lcc_out, st.to_dict()


def tc_graph_info(g: int) -> dict:
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.tc_graph_info(g, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"m_simple": a.value, "loops_dropped": b.value, "dups_dropped": c.value}


def tc_graph_size(g: int) -> tuple[int, int]:
    n, m = ctypes.c_int32(), ctypes.c_int64()
    _check(_lib.tc_graph_size(g, ctypes.byref(n), ctypes.byref(m)))
    return n.value, m.value


def tc_graph_destroy(g: int) -> None:
    if g:
        _lib.tc_graph_destroy(g)


def tc_graph_set_strategy(g: int, bucket, strategy, factor: float = 1.0) -> None:
    if isinstance(bucket, str):
        bucket = BUCKETS[bucket]
    if isinstance(strategy, str):
        strategy = STRATEGIES[strategy]
    _check(_lib.tc_graph_set_strategy(g, bucket, strategy, factor))


def tc_graph_set_hubs(g: int, min_degree: int, max_hubs: int) -> None:
    _check(_lib.tc_graph_set_hubs(g, min_degree, max_hubs))


def tc_graph_last_timing(g: int) -> dict:
    ms = (ctypes.c_float * len(PHASES))()
    _check(_lib.tc_graph_last_timing(g, ms, len(PHASES)))
    return {k: ms[i] for i, k in enumerate(PHASES)}


def tc_graph_build_timing(g: int) -> dict:
    ms = (ctypes.c_float * len(BUILD_PHASES))()
    _check(_lib.tc_graph_build_timing(g, ms, len(BUILD_PHASES)))
    return {k: ms[i] for i, k in enumerate(BUILD_PHASES)}


def tc_graph_plan_stats(g: int) -> dict:
    """Per bucket: oriented edges and sum of d+(u) + d+(v) ("ids") over them."""
    nb = TC_BUCKET_HUB + 2
    e = (ctypes.c_int64 * nb)()
    i = (ctypes.c_int64 * nb)()
    _check(_lib.tc_graph_plan_stats(g, e, i))
    names = ["small", "cta", "hub", "trivial"]
    return {names[b]: {"edges": e[b], "ids": i[b]} for b in range(nb)}


def _numel(a) -> int:
    return int(a.numel()) if hasattr(a, "numel") and callable(a.numel) else int(np.asarray(a).size)


def _check_room(a, n: int, what: str):
    """Refuses an output buffer with fewer than n elements (the library writes n)."""
    if a is not None and _numel(a) < n:
        raise ValueError(f"{what} holds {_numel(a)} elements, the graph has {n} vertices")


def tc_count_noalloc(n: int, src, dst, t_out=None, lcc_out=None, stream=None) -> int:
    """T of a small graph without any allocation by the library (CUDA tensors only);
    fills t_out (int64/uint64 [n]) and lcc_out (float64 [n]) when given.  Every
    buffer is checked (device, dtype, length) before the call, since the kernel reads
    len(src) pairs from both lists and writes n entries into each output."""
    load()
    for a in (src, dst, t_out, lcc_out):
        if a is not None and not _is_device(a):
            raise ValueError("tc_count_noalloc takes device buffers")
    if _numel(src) != _numel(dst):
        raise ValueError("src and dst differ in length")
    _check_dtype(src, "int32")
    _check_dtype(dst, "int32")
    if t_out is not None:
        _check_dtype(t_out, "int64")
    if lcc_out is not None:
        _check_dtype(lcc_out, "float64")
    _check_room(t_out, n, "t_out")
    _check_room(lcc_out, n, "lcc_out")
    (ps, pd, pt, pl), _ = _ptr_kind(src, dst, t_out, lcc_out)
    T = ctypes.c_uint64()
    _check(_lib.tc_count_noalloc(n, _numel(src), ps, pd, ctypes.byref(T), pt, pl, _stream_ptr(stream)))
    return int(T.value)


def tc_batch_create(n, edge_off, src, dst, stream=None) -> int:
    """Batch handle: n (int32[G]) and edge_off (int64[G+1]) on the host, src/dst int32
    local ids (numpy on the host or CUDA tensors)."""
    load()
    n = np.ascontiguousarray(n, dtype=np.int32)
    edge_off = np.ascontiguousarray(edge_off, dtype=np.int64)
    if len(edge_off) != len(n) + 1:
        raise ValueError("edge_off needs G + 1 entries")
    _check_dtype(src, "int32")
    _check_dtype(dst, "int32")
    (ps, pd), kind = _ptr_kind(src, dst)
    out = ctypes.c_void_p()
    _check(_lib.tc_batch_create(len(n), n.ctypes.data, edge_off.ctypes.data, ps, pd, kind, _stream_ptr(stream),
                                ctypes.byref(out)))
    return out.value


def tc_batch_count(g: int, T_out=None):
    """Per-graph T into T_out (uint64/int64 [G], host or device); returns T_out."""
    G = ctypes.c_int32()
    _check(_lib.tc_batch_size(g, ctypes.byref(G)))
    if T_out is None:
        T_out = np.empty(G.value, dtype=np.uint64)
    _check_dtype(T_out, "int64")
    (pt,), kind = _ptr_kind(T_out)
    _check(_lib.tc_batch_count(g, pt, kind))
    return T_out


def tc_graph_get_tuning(g: int) -> dict:
    t = TcTuning()
    _check(_lib.tc_graph_get_tuning(g, ctypes.byref(t)))
    return t.to_dict()


def tc_graph_set_tuning(g: int, tuning: dict) -> None:
    t = TcTuning.from_dict(tuning)
    _check(_lib.tc_graph_set_tuning(g, ctypes.byref(t)))


def tc_graph_autotune(g: int, force: bool = False) -> dict:
    t = TcTuning()
    _check(_lib.tc_graph_autotune(g, 1 if force else 0, ctypes.byref(t)))
    return t.to_dict()


def tc_batch_run(n, edge_off, src, dst, T_out, t_out=None, lcc_out=None, tuning=None, stream=None,
                 graph: bool = False) -> None:
    """Whole batch in one call, device buffers (CUDA tensors); graph=True records the
    device work into a CUDA graph once and replays it on later identical calls."""
    load()
    n = np.ascontiguousarray(n, dtype=np.int32)
    edge_off = np.ascontiguousarray(edge_off, dtype=np.int64)
    for a in (src, dst, T_out, t_out, lcc_out):
        if a is not None and not _is_device(a):
            raise ValueError("tc_batch_run takes device buffers")
    (ps, pd, pT, pt, pl), _ = _ptr_kind(src, dst, T_out, t_out, lcc_out)
    tp = ctypes.byref(TcTuning.from_dict(tuning)) if tuning else None
    _check(_lib.tc_batch_run(len(n), n.ctypes.data, edge_off.ctypes.data, ps, pd, pT, pt, pl, tp,
                             _stream_ptr(stream), TC_RUN_GRAPH if graph else 0))


def tc_release_cached_graphs() -> None:
    load().tc_release_cached_graphs()


def tc_generate_edges(kind, n: int, m: int, seed: int, stream_id: int, src, dst, stream=None) -> None:
    """Device-side generation into int32 CUDA tensors src/dst of length >= m."""
    load()
    kind = GEN_KINDS[kind] if isinstance(kind, str) else kind
    (ps, pd), k = _ptr_kind(src, dst)
    if k != TC_MEM_DEVICE:
        raise ValueError("tc_generate_edges writes device buffers")
    _check(_lib.tc_generate_edges(kind, n, m, seed, stream_id, ps, pd, _stream_ptr(stream)))


class Server:
    """Serving loop (tc_server_*): requests are graph specs generated on the device."""

    def __init__(self, hbm_budget_bytes: int, slots: int = 4):
        load()
        self._h = ctypes.c_void_p()
        _check(_lib.tc_server_start(int(hbm_budget_bytes), int(slots), ctypes.byref(self._h)))

    def submit(self, rid: int, workload) -> None:
        """workload: graphgen.Workload of kind "rmat" or "er_replace"."""
        r = TcRequest(rid, GEN_KINDS[workload.kind], workload.n, workload.m, workload.seed, workload.stream)
        _check(_lib.tc_server_submit(self._h, ctypes.byref(r)))

    def poll(self, max_results: int = 4096) -> list[dict]:
        buf = (TcResult * max_results)()
        cnt = ctypes.c_int32()
        _check(_lib.tc_server_poll(self._h, buf, max_results, ctypes.byref(cnt)))
        return [buf[i].to_dict() for i in range(cnt.value)]

    def wait(self, completed: int, timeout_s: float) -> bool:
        st = _lib.tc_server_wait(self._h, int(completed), float(timeout_s))
        if st == TC_ETIMEOUT:
            return False
        _check(st)
        return True

    def stats(self) -> dict:
        s = TcServerStats()
        _check(_lib.tc_server_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def stop(self) -> None:
        if self._h:
            _check(_lib.tc_server_stop(self._h))
            self._h = ctypes.c_void_p()


def tc_request_run(rid: int, workload, stream=None) -> dict:
    """One serving request alone on ``stream`` (the plain per-graph path): the same
    result fields as a served request's; ``end_s`` = seconds the call took."""
    load()
    r = TcRequest(rid, GEN_KINDS[workload.kind], workload.n, workload.m, workload.seed, workload.stream)
    out = TcResult()
    _check(_lib.tc_request_run(ctypes.byref(r), _stream_ptr(stream), ctypes.byref(out)))
    return out.to_dict()


def tc_launch_count() -> int:
    return int(load().tc_launch_count())


class Graph:
    """Owning wrapper around a tc_graph handle."""

    def __init__(self, handle: int, n: int):
        self.handle = handle
        self.n = n

    @classmethod
    def from_edges(cls, n, src, dst, stream=None) -> "Graph":
        return cls(tc_graph_create_from_edges(n, src, dst, stream), n)

    @classmethod
    def from_csr(cls, n, offsets, adj, stream=None) -> "Graph":
        return cls(tc_graph_create_from_csr(n, offsets, adj, stream), n)

    @classmethod
    def batch(cls, n, edge_off, src, dst, stream=None) -> "Graph":
        return cls(tc_batch_create(n, edge_off, src, dst, stream), int(np.sum(n, dtype=np.int64)))

    def batch_count(self, T_out=None):
        return tc_batch_count(self.handle, T_out)

    def count(self) -> int:
        return tc_count(self.handle)

    def lcc(self, t_out=None, lcc_out=None):
        """Host numpy results when no buffers are given; else fills the buffers."""
        if t_out is None and lcc_out is None:
            t_out = np.empty(self.n, dtype=np.uint64)
            lcc_out = np.empty(self.n, dtype=np.float64)
        lcc_compute(self.handle, t_out, lcc_out)
        return t_out, lcc_out

    def count_shard(self, shard: int, nshards: int, t_out=None):
        """(T_shard, t_share) of one shard; a host uint64 array when t_out is None."""
        if t_out is None:
            t_out = np.empty(self.n, dtype=np.uint64)
        return tc_count_shard(self.handle, shard, nshards, t_out)

    def lcc_from_counts(self, t, lcc_out=None):
        """LCC from summed per-vertex counts; a host float64 array when lcc_out is None."""
        if lcc_out is None:
            lcc_out = np.empty(self.n, dtype=np.float64)
        tc_lcc_from_counts(self.handle, t, lcc_out)
        return lcc_out

    def vertex_formula(self, t_out=None):
        """(T, t) by the paper's unoriented per-vertex formula (for comparison)."""
        T, t = tc_count_vertex_formula(self.handle, t_out)
        if not hasattr(t, "cuda"):
            t = t.view("uint64")
        return T, t

    def edge_support(self, u_out=None, v_out=None, support_out=None):
        """(u, v, support) per distinct edge; numpy results come sorted by (u, v)."""
        u, v, sup = tc_edge_support(self.handle, u_out, v_out, support_out)
        if not hasattr(u, "cuda"):
            order = np.lexsort((v, u))
            u, v, sup = u[order], v[order], sup[order].view(np.uint32)
        return u, v, sup

    def remote_cache(self, parts: int, capacities) -> dict:
        """Remote reads of a 1D partition and the caches of Sec. IV-B (tc_remote_cache)."""
        return tc_remote_cache(self.handle, parts, capacities)

    def info(self) -> dict:
        return tc_graph_info(self.handle)

    def set_strategy(self, bucket, strategy, factor=1.0):
        tc_graph_set_strategy(self.handle, bucket, strategy, factor)

    def set_hubs(self, min_degree: int, max_hubs: int):
        tc_graph_set_hubs(self.handle, min_degree, max_hubs)

    def timing(self) -> dict:
        return tc_graph_last_timing(self.handle)

    def plan_stats(self) -> dict:
        return tc_graph_plan_stats(self.handle)

    def build_timing(self) -> dict:
        return tc_graph_build_timing(self.handle)

    def tuning(self) -> dict:
        return tc_graph_get_tuning(self.handle)

    def set_tuning(self, tuning: dict):
        tc_graph_set_tuning(self.handle, tuning)

    def autotune(self, force: bool = False) -> dict:
        return tc_graph_autotune(self.handle, force)

    def close(self):
        tc_graph_destroy(self.handle)
        self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                self.close()
        except Exception:
            pass
