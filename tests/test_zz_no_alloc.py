"""The no-allocation entry point (tc_count_noalloc) against the regular one.

tc_count_noalloc serves callers that cannot allocate device memory while they run
(all free memory already handed to their own allocator, real-time code that
forbids allocation after start-up).  It keeps its intermediate arrays in one fixed
device array inside the library, so consecutive calls share that array: each case
below is run twice in a row and both results must equal those of the regular
entry point (tc_graph_create_from_edges, tc_count, lcc_compute) exactly, the
tolerance every parity test here uses.

This file is collected last on purpose: it runs after every other test, and it
also passes when run on its own in a fresh process.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
from tests import families as F

pytestmark = pytest.mark.gpu


def _cases():
    out = [("er4096",) + tuple(graphgen.workload("er4096").edges()) + (4096,)]
    n = 1 << 13
    out.append(("rmat13",) + tuple(graphgen.rmat(13, 16 * n, seed=21)) + (n,))
    # largest accepted sizes: 16384 vertices, 262144 pairs (R-MAT scale 14, edge factor 16)
    n = 1 << 14
    out.append(("rmat14_max",) + tuple(graphgen.rmat(14, 16 * n, seed=22)) + (n,))
    from tests.test_oracle import _tiny
    nn, s, d = _tiny(7)
    out.append(("tiny_loops_repeats", s, d, nn))
    nn, (s, d) = F.wheel(30)
    out.append(("wheel30", s, d, nn))
    out.append(("empty", np.array([], np.int32), np.array([], np.int32), 5))
    return out


CASES = _cases()


def _regular(tc, n, s, d):
    import torch
    g = tc.Graph.from_edges(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    try:
        T = g.count()
        t = torch.empty(n, dtype=torch.int64, device="cuda")
        lc = torch.empty(n, dtype=torch.float64, device="cuda")
        g.lcc(t, lc)
        torch.cuda.synchronize()
    finally:
        g.close()
    return T, t.cpu().numpy().view(np.uint64), lc.cpu().numpy()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_regular_entry_point_twice(tc, case):
    import torch
    _, s, d, n = case
    T0, t0, l0 = _regular(tc, n, s, d)
    src = torch.from_numpy(s).cuda()
    dst = torch.from_numpy(d).cuda()
    for _ in range(2):
        t = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        lc = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        T = tc.tc_count_noalloc(n, src, dst, t, lc)
        assert T == T0
        np.testing.assert_array_equal(t.cpu().numpy().view(np.uint64), t0)
        np.testing.assert_array_equal(lc.cpu().numpy().view(np.uint64), l0.view(np.uint64))


def test_noalloc_rejects_sizes_beyond_the_limit(tc):
    import torch
    e = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(tc.TCError) as err:
        tc.tc_count_noalloc(tc.TC_NOALLOC_MAX_N + 1, e, e)
    assert err.value.status == tc.TC_EINVAL
    big = torch.zeros(tc.TC_NOALLOC_MAX_M + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(tc.TCError):
        tc.tc_count_noalloc(100, big, big)
    bad = torch.tensor([0, 7], dtype=torch.int32, device="cuda")
    with pytest.raises(tc.TCError):
        tc.tc_count_noalloc(5, bad, torch.tensor([1, 1], dtype=torch.int32, device="cuda"))
    # still usable afterwards
    n, (s, d) = F.complete(12)
    assert tc.tc_count_noalloc(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()) == 220


def test_noalloc_second_call_takes_no_device_memory(tc):
    """After a first call (which may load the library's device code on this device),
    a further call leaves the device's free memory unchanged."""
    import torch
    nn, s, d = CASES[1][3], CASES[1][1], CASES[1][2]
    src = torch.from_numpy(s).cuda()
    dst = torch.from_numpy(d).cuda()
    t = torch.empty(nn, dtype=torch.int64, device="cuda")
    lc = torch.empty(nn, dtype=torch.float64, device="cuda")
    T0 = tc.tc_count_noalloc(nn, src, dst, t, lc)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    T1 = tc.tc_count_noalloc(nn, src, dst, t, lc)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert T1 == T0
    assert free1 == free0


def test_noalloc_on_a_side_stream(tc):
    """The same results when the call runs on a stream other than the default one."""
    import torch
    _, s, d, n = CASES[0]
    T0, t0, l0 = _regular(tc, n, s, d)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        src = torch.from_numpy(s).cuda()
        dst = torch.from_numpy(d).cuda()
        t = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        lc = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        T = tc.tc_count_noalloc(n, src, dst, t, lc, stream=side)
        side.synchronize()
        assert T == T0
        np.testing.assert_array_equal(t.cpu().numpy().view(np.uint64), t0)
        np.testing.assert_array_equal(lc.cpu().numpy().view(np.uint64), l0.view(np.uint64))
