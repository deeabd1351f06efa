"""Multi-rank host logic on CPU ranks (gloo, world size 2, 127.0.0.1).

1. The benchmark's aggregation: the slowest rank's time and the whole-job value.
2. The edge-sharded count: ranks take work-balanced ranges of source vertices of
   the oriented graph, count their edges independently (the oracle's oriented
   count restricted to a range), and one sum of t[] gives the full result -- the
   only exchange the path needs when it is spread over several GPUs.
3. The library's exchange step (paper_2202_13976_gb300.dist): every rank checks
   in through the store before the sum; a rank that left between steps is reported
   (RankLost, naming it) to the others within the deadline, and none of them enters
   the collective.  The failure is made on the host: the rank simply exits.
"""
from __future__ import annotations

import os
import socket
import time

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


def _exchange_worker(rank, world, port, q, absent, release):
    """All ranks join the group; `absent` (if any) then leaves before the exchange.
    The others stay until the parent has every report (`release`): rank 0 hosts the
    store, and its exit would cut the others' check-ins short."""
    import torch
    import torch.distributed as dist

    from paper_2202_13976_gb300 import dist as tcd
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0)
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
    if rank == absent:
        q.put((rank, "left", None))
        q.close()
        q.join_thread()  # the message is out before the process goes
        os._exit(0)  # gone between steps, with nothing in flight
    t = torch.arange(5, dtype=torch.int64) * (rank + 1)
    t0 = time.monotonic()
    try:
        tcd.sum_counts(t, store=store, rank=rank, world=world, step=7, timeout_s=2.0)
        q.put((rank, "sum", t.tolist()))
    except tcd.RankLost as e:
        q.put((rank, "lost", (e.missing, e.step, time.monotonic() - t0)))
    q.close()
    q.join_thread()
    release.wait(120)
    if absent is None:
        dist.destroy_process_group()
    else:
        os._exit(0)  # the group has a dead member: leave without a collective teardown


def _run_exchange(world, absent):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    release = ctx.Event()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_worker, args=(r, world, port, q, absent, release)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        out = [q.get(timeout=120) for _ in procs]
    finally:
        release.set()
    for p in procs:
        p.join(timeout=60)
    return sorted(out)


def test_exchange_sums_when_every_rank_checks_in():
    out = _run_exchange(3, None)
    want = [sum(i * (r + 1) for r in range(3)) for i in range(5)]
    assert out == [(r, "sum", want) for r in range(3)]


def test_a_rank_that_left_is_reported_not_waited_for():
    out = _run_exchange(3, 2)
    assert out[2] == (2, "left", None)
    for rank, kind, info in out[:2]:
        assert kind == "lost"
        missing, step, waited = info
        assert missing == [2] and step == 7
        assert 1.5 < waited < 30.0  # the deadline, not a hang


def test_check_in_needs_a_shared_store():
    """Single-process checks of the deadline logic on a HashStore."""
    import torch.distributed as dist

    from paper_2202_13976_gb300 import dist as tcd
    st = dist.HashStore()
    st.set("tc/check_in/a/1", b"1")
    tcd.check_in(st, 0, 2, "a", timeout_s=1.0)  # rank 1 is already there
    t0 = time.monotonic()
    with pytest.raises(tcd.RankLost) as e:
        tcd.check_in(st, 0, 3, "b", timeout_s=0.2)
    assert e.value.missing == [1, 2]
    assert time.monotonic() - t0 < 5.0
    # integer steps: a rank drops its key of two steps back once a step completes
    for step in range(4):
        tcd.check_in(st, 0, 1, step, timeout_s=1.0)
    assert not st.check(["tc/check_in/0/0"]) and not st.check(["tc/check_in/1/0"])
    assert st.check(["tc/check_in/2/0"]) and st.check(["tc/check_in/3/0"])


class _StoreThatDies:
    """A store that answers `live` checks, then fails as a TCPStore client does once
    the process hosting the store has exited."""

    def __init__(self, present, live):
        self.keys = {f"tc/check_in/s/{r}" for r in present}
        self.live = live

    def set(self, key, value):
        self.keys.add(key)

    def check(self, keys):
        if self.live == 0:
            raise RuntimeError("Connection reset by peer")
        self.live -= 1
        return all(k in self.keys for k in keys)


def test_a_store_that_stops_answering_is_reported_as_lost():
    from paper_2202_13976_gb300 import dist as tcd
    # ranks 0 and 1 are seen before the store goes; rank 2 never checked in
    t0 = time.monotonic()
    with pytest.raises(tcd.RankLost) as e:
        tcd.check_in(_StoreThatDies([0], live=3), 1, 3, "s", timeout_s=60.0)
    assert e.value.missing == [2] and e.value.store_error is not None
    assert time.monotonic() - t0 < 5.0  # at once, not at the deadline
    # a store that is gone before the first check-in confirms nobody else
    class Gone(_StoreThatDies):
        def set(self, key, value):
            raise RuntimeError("Connection refused")
    with pytest.raises(tcd.RankLost) as e:
        tcd.check_in(Gone([], live=0), 0, 3, "s", timeout_s=60.0)
    assert e.value.missing == [1, 2]
