"""One graph counted on several GPUs, one process per GPU.

Every rank holds the whole graph, which stays read-only. Each rank then:
- counts its shard of the sources with `tc_count_shard` (cost-balanced ranges of
  ranks, each triangle counted once, from its lowest vertex, Sec. III);
- adds its per-vertex counts to the other ranks' in one sum over the process group;
- computes the LCC from the summed counts (Eq. 2, `tc_lcc_from_counts`).

Failure detection happens before the sum. Every rank checks in through a
`torch.distributed` store. A rank that has not checked in by the deadline is
reported as lost (`RankLost`), so the others never block inside a collective that
cannot complete. Whether to retry, shrink the group or stop is the caller's call.
"""
from __future__ import annotations

import time

import numpy as np

__all__ = ["RankLost", "check_in", "sum_counts", "sharded_lcc"]


class RankLost(RuntimeError):
    """Ranks that did not check in for a step before the deadline.

    `store_error` is set when the store itself stopped answering (the process that
    hosts it is gone); `missing` then lists the ranks not seen before that."""

    def __init__(self, missing, step, store_error=None):
        self.missing = list(missing)
        self.step = step
        self.store_error = store_error
        why = f" (store lost: {store_error})" if store_error is not None else ""
        super().__init__(f"ranks {self.missing} did not check in for step {step!r}{why}")


def _key(step, rank: int) -> str:
    return f"tc/check_in/{step}/{rank}"


def check_in(store, rank: int, world: int, step, timeout_s: float = 30.0, poll_s: float = 0.005):
    """Marks this rank as present for `step` and waits until every rank of `world` is.

    Raises RankLost, naming the absent ranks, once `timeout_s` has passed, or as soon
    as the store stops answering.  `store` is any torch.distributed Store shared by
    the ranks (TCPStore, FileStore); `step` is any value that names the exchange
    uniquely (a step counter, a tag): a key, once set, stays set, so reusing a step
    value would find the old check-ins.  Each rank removes its key of the step before
    the previous one once this step is complete (every rank has passed that earlier
    check-in by then), when steps are integers."""
    keys = [_key(step, r) for r in range(world)]
    seen = set()
    deadline = time.monotonic() + timeout_s
    try:
        store.set(keys[rank], b"1")
    except Exception as e:  # no store: nobody can be confirmed
        raise RankLost([r for r in range(world) if r != rank], step, store_error=e) from e
    while True:
        try:
            for r, k in enumerate(keys):
                if r not in seen and store.check([k]):
                    seen.add(r)
        except Exception as e:  # the store stopped answering: its host rank is gone
            raise RankLost([r for r in range(world) if r not in seen], step, store_error=e) from e
        missing = [r for r in range(world) if r not in seen]
        if not missing:
            if isinstance(step, int) and step >= 2:
                try:
                    store.delete_key(_key(step - 2, rank))
                except Exception:  # stores without deletion keep the key
                    pass
            return
        if time.monotonic() >= deadline:
            raise RankLost(missing, step)
        time.sleep(poll_s)


def sum_counts(t, *, store, rank: int, world: int, step, timeout_s: float = 30.0, group=None):
    """Sums the int64 tensor t (per-vertex counts, plus anything appended) over the
    ranks in place, after every rank has checked in for `step`; returns t."""
    import torch.distributed as dist
    check_in(store, rank, world, step, timeout_s)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def sharded_lcc(graph, *, store, rank: int, world: int, step, timeout_s: float = 30.0, group=None,
                reduce_device: str = "cpu"):
    """(T, t, lcc) of the whole graph on every rank, from this rank's shard.

    `graph` is a `Graph` that every rank built from the same edges.  `step` names this
    exchange and must differ between calls on one store (see `check_in`), so it has
    no default.  The per-vertex
    counts and the shard's triangles travel as one int64 tensor on `reduce_device`
    ("cpu" for gloo, "cuda" for NCCL).  t is returned as uint64 and lcc as float64,
    both numpy arrays on the host."""
    import torch
    n = graph.n
    t_share = np.empty(n + 1, dtype=np.uint64)
    T_shard, _ = graph.count_shard(rank, world, t_share[:n])
    t_share[n] = T_shard
    tt = torch.from_numpy(t_share.view(np.int64)).to(reduce_device)
    sum_counts(tt, store=store, rank=rank, world=world, step=step, timeout_s=timeout_s, group=group)
    total = tt.cpu().numpy().view(np.uint64)
    t = np.ascontiguousarray(total[:n])
    lcc = graph.lcc_from_counts(t)
    return int(total[n]), t, lcc
