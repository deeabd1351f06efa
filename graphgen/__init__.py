"""Seeded synthetic graph inputs (R-MAT and Erdos-Renyi G(n, m)).

This module produces edge lists only and holds none of the triangle-counting
arithmetic, so both the CPU oracle and the CUDA path may consume it.  The
generators are written in C (``graphgen.c``) for speed and compiled on first use
with the host C compiler; the compiled object is not committed.

Workloads follow the paper's synthetic graphs (Sec. V-A): R-MAT with
(a, b, c, d) = (0.57, 0.19, 0.19, 0.05).  "Scale x, edge factor y" is read as
2^x vertices and y * 2^x generated pairs before symmetrisation, deduplication
and self-loop removal; Table I's sizes (R-MAT S21 EF16: 33.6 M edges, S23 EF16:
134.2 M) fix that reading.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "_graphgen.so")
_lib = None

RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile graphgen.c into _graphgen.so next to it (atomic rename)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, i64, i32p = ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
        lib.gg_stream_key.restype = u64
        lib.gg_stream_key.argtypes = [u64, u64]
        lib.gg_draw.restype = u64
        lib.gg_draw.argtypes = [u64, u64]
        lib.gg_draw_many.restype = None
        lib.gg_draw_many.argtypes = [u64, u64, i64, ctypes.POINTER(u64)]
        lib.gg_rmat.restype = None
        lib.gg_rmat.argtypes = [u64, u64, ctypes.c_int, i64, i64, i64, ctypes.c_uint32,
                                ctypes.c_uint32, ctypes.c_uint32, i32p, i32p]
        lib.gg_er.restype = i64
        lib.gg_er.argtypes = [u64, u64, i64, i64, i32p, i32p]
        lib.gg_er_replace.restype = None
        lib.gg_er_replace.argtypes = [u64, u64, i64, i64, i64, i32p, i32p]
        _lib = lib
    return _lib


def _i32p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def stream_key(seed: int, stream: int = 0) -> int:
    return int(_load().gg_stream_key(seed, stream))


def draws(seed: int, stream: int, i0: int, count: int) -> np.ndarray:
    """Raw 64-bit draws i0 .. i0+count-1 of stream (seed, stream)."""
    out = np.empty(count, dtype=np.uint64)
    _load().gg_draw_many(stream_key(seed, stream), i0, count,
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


def rmat_thresholds(a: float, b: float, c: float) -> tuple[int, int, int]:
    """floor(cumulative probability * 2^32) for quadrants a, a+b, a+b+c."""
    return (int(math.floor(a * 2 ** 32)), int(math.floor((a + b) * 2 ** 32)),
            int(math.floor((a + b + c) * 2 ** 32)))


def rmat(scale: int, m: int, seed: int, stream: int = 0, n: int | None = None,
         abc: tuple[float, float, float] = RMAT_ABC) -> tuple[np.ndarray, np.ndarray]:
    """m generated R-MAT pairs over n <= 2^scale vertices (default n = 2^scale)."""
    if n is None:
        n = 1 << scale
    if not (1 <= n <= (1 << scale)) or scale > 31 or scale < 0:
        raise ValueError("need 1 <= n <= 2^scale, scale <= 31")
    ta, tab, tabc = rmat_thresholds(*abc)
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    if m:
        _load().gg_rmat(seed, stream, scale, n, 0, m, ta, tab, tabc, _i32p(src), _i32p(dst))
    return src, dst


def er(n: int, m: int, seed: int, stream: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """G(n, m): m distinct unordered pairs without loops (m capped at C(n,2))."""
    total = n * (n - 1) // 2 if n >= 2 else 0
    mm = min(m, total)
    src = np.empty(mm, dtype=np.int32)
    dst = np.empty(mm, dtype=np.int32)
    got = _load().gg_er(seed, stream, n, mm, _i32p(src), _i32p(dst)) if mm else 0
    if got < 0:
        raise MemoryError("graphgen: allocation failed")
    return src[:got], dst[:got]


def er_replace(n: int, m: int, seed: int, stream: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """m uniform pairs with replacement (loops and repeats kept)."""
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    if m:
        _load().gg_er_replace(seed, stream, n, 0, m, _i32p(src), _i32p(dst))
    return src, dst


# ---------------------------------------------------------------------------
# Named workloads.

@dataclass(frozen=True)
class Workload:
    name: str
    kind: str          # "rmat" or "er"
    n: int
    m: int             # generated pairs (R-MAT) or distinct edges (ER)
    seed: int
    stream: int
    scale: int = 0

    def edges(self) -> tuple[np.ndarray, np.ndarray]:
        if self.kind == "rmat":
            return rmat(self.scale, self.m, self.seed, self.stream, n=self.n)
        if self.kind == "er_replace":
            return er_replace(self.n, self.m, self.seed, self.stream)
        return er(self.n, self.m, self.seed, self.stream)


WORKLOADS = {
    # Erdos-Renyi G(4096, 32768), seed 1.
    "er4096": Workload("er4096", "er", 4096, 32768, 1, 0),
    # R-MAT scale 20, edge factor 16, seed 2.
    "rmat20": Workload("rmat20", "rmat", 1 << 20, 16 << 20, 2, 0, scale=20),
    # R-MAT scale 22, edge factor 8, seed 3: the profiling case (its oriented rows just
    # exceed the 129 MB L2, the whole graph takes about 2 GB of device memory).
    "rmat22": Workload("rmat22", "rmat", 1 << 22, 8 << 22, 3, 0, scale=22),
    # R-MAT scale 23, edge factor 8, seed 3.
    "rmat23": Workload("rmat23", "rmat", 1 << 23, 8 << 23, 3, 0, scale=23),
    # Uniform G(8,388,608, 60,000,000) of the same size, seed 3, stream 1.
    "er23": Workload("er23", "er", 1 << 23, 60_000_000, 3, 1),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def _uniform(x: np.ndarray) -> np.ndarray:
    """Top 53 bits of a draw as a double in [0, 1)."""
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass(frozen=True)
class Request:
    """One request of the serving stream: arrival time (s), graph spec."""
    id: int
    arrival: float
    workload: Workload


def serve_requests(seconds: float = 60.0, rate: float = 2000.0, seed: int = 5,
                   n_range: tuple[int, int] = (1000, 4_000_000), ef_range: tuple[float, float] = (4.0, 16.0),
                   rmat_share: float = 0.7, limit: int | None = None) -> list[Request]:
    """The serving stream: Poisson arrivals at `rate` per second for `seconds`;
    request q has n log-uniform in n_range, edge factor U(ef_range), m = round(ef n)
    generated pairs, R-MAT with probability rmat_share (scale = ceil(log2 n),
    endpoints >= n redrawn) else uniform pairs with replacement.  Stream 0 of `seed`
    drives the arrivals and specs (draws 4q .. 4q+3 for request q); request q's
    edges use stream q + 1."""
    out = []
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    t = 0.0
    q = 0
    chunk = 4096
    while True:
        d = draws(seed, 0, 4 * q, 4 * chunk)
        u = _uniform(d).reshape(-1, 4)
        for k in range(chunk):
            gap = -math.log(1.0 - float(u[k, 0])) / rate
            t += gap
            if t >= seconds or (limit is not None and q >= limit):
                return out
            n = int(math.floor(math.exp(lo + (hi - lo) * float(u[k, 1]))))
            n = max(n_range[0], min(n_range[1], n))
            ef = ef_range[0] + (ef_range[1] - ef_range[0]) * float(u[k, 2])
            m = int(round(ef * n))
            if float(u[k, 3]) < rmat_share:
                scale = max(1, int(math.ceil(math.log2(n))))
                w = Workload(f"req{q}", "rmat", n, m, seed, q + 1, scale=scale)
            else:
                w = Workload(f"req{q}", "er_replace", n, m, seed, q + 1)
            out.append(Request(q, t, w))
            q += 1


def batch_workloads(G: int = 20000, seed: int = 4) -> list[Workload]:
    """The batched workload: G graphs, n log-uniform in [32, 65536], average degree
    k ~ U(4, 32), m = round(n k / 2); even index R-MAT (scale = ceil(log2 n),
    endpoints >= n redrawn), odd index ER (m capped at C(n,2)).  Graph i's edges
    use stream i + 1 of `seed`; the per-graph parameters use stream 0."""
    d = draws(seed, 0, 0, 2 * G)
    u_n = _uniform(d[0::2])
    u_k = _uniform(d[1::2])
    out = []
    lo, hi = math.log(32.0), math.log(65536.0)
    for i in range(G):
        n = int(math.floor(math.exp(lo + (hi - lo) * float(u_n[i]))))
        n = max(32, min(65536, n))
        k = 4.0 + 28.0 * float(u_k[i])
        m = int(round(n * k / 2.0))
        if i % 2 == 0:
            scale = max(1, int(math.ceil(math.log2(n))))
            out.append(Workload(f"batch{i}", "rmat", n, m, seed, i + 1, scale=scale))
        else:
            out.append(Workload(f"batch{i}", "er", n, min(m, n * (n - 1) // 2), seed, i + 1))
    return out
