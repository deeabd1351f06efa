"""Multi-rank host logic on CPU ranks (gloo, world size 2, 127.0.0.1).

1. The benchmark's aggregation: the slowest rank's time and the whole-job value.
2. The edge-sharded count: ranks take work-balanced ranges of source vertices of
   the oriented graph, count their edges independently (the oracle's oriented
   count restricted to a range), and one sum of t[] gives the full result -- the
   only exchange the path needs when it is spread over several GPUs.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _aggregate_worker(rank, world, port, q):
    import bench
    dist = _init(rank, world, port)
    ms, value = bench.aggregate_ranks(100.0 * (rank + 1), 10, 1000, world, device="cpu")
    q.put((rank, ms, value))
    dist.destroy_process_group()


def _shard_worker(rank, world, port, q):
    import torch

    import graphgen
    import oracle
    dist = _init(rank, world, port)
    n = 1 << 13
    s, d = graphgen.rmat(13, 16 * n, seed=3)
    off, adj, _ = oracle.build_csr(n, s, d)
    op, ap = oracle.orient(n, off, adj)
    # balanced ranges by the cost of each source vertex (sum of list lengths it merges)
    dp = np.diff(op).astype(np.float64)
    w = np.cumsum(dp * dp + dp + 1.0)
    cuts = np.searchsorted(w, np.linspace(0, w[-1], world + 1)[1:-1])
    bounds = [0] + [int(c) for c in cuts] + [n]
    lo, hi = bounds[rank], bounds[rank + 1]
    rows = np.repeat(np.arange(n), np.diff(op))
    mask = (rows >= lo) & (rows < hi)  # this rank's oriented edges
    # every rank reads the whole (replicated, read-only) oriented graph and counts
    # only its source range through the oracle's range routine
    t = np.zeros(n, dtype=np.uint64)
    oracle._load().or_tc_oriented(n, oracle._p(op, oracle._i64p), oracle._p(ap, oracle._i32p),
                                  oracle._p(t, oracle._u64p), lo, hi)
    tt = torch.from_numpy(t.view(np.int64).copy())
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    full = oracle.tc_oriented(n, op, ap)
    q.put((rank, bool(np.array_equal(tt.numpy().view(np.uint64), full)), int(mask.sum())))
    dist.destroy_process_group()


def _run(target, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_bench_aggregation_takes_the_slowest_rank():
    out = _run(_aggregate_worker)
    for rank, ms, value in out:
        assert ms == 20.0                    # max(100, 200) / 10 steps
        assert value == pytest.approx(2 * 1000 / 0.020)


def test_edge_shards_sum_to_the_full_count():
    out = _run(_shard_worker)
    assert all(ok for _, ok, _ in out)
    assert all(edges > 0 for _, _, edges in out)
