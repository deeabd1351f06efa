"""Parity of the directed LCC (Eq. 1, tc_directed_lcc through the C ABI) with the CPU
oracle: c[] bit-exact, C[] bit-exact (0 ulp), the sum of c and the distinct directed
edge count exact."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle
from tests import families as F
from tests.test_oracle import _tiny, _tiny_directed

pytestmark = pytest.mark.gpu


def _gpu(tc, n, s, d, device_io=False):
    if device_io:
        import torch
        c, l, st = tc.tc_directed_lcc(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), timed=True)
        torch.cuda.synchronize()
        return c.cpu().numpy().view(np.uint64), l.cpu().numpy(), st["total"], st["m_directed"]
    c, l, st = tc.tc_directed_lcc(n, s, d)
    return c.view(np.uint64), l, st["total"], st["m_directed"]


def _check(tc, n, s, d, device_io=False):
    s = np.ascontiguousarray(s, dtype=np.int32)
    d = np.ascontiguousarray(d, dtype=np.int32)
    ref = oracle.directed_lcc(n, s, d)
    c, l, total, md = _gpu(tc, n, s, d, device_io)
    np.testing.assert_array_equal(c, ref["c"])
    np.testing.assert_array_equal(l.view(np.uint64), ref["lcc"].view(np.uint64))
    assert total == int(ref["c"].sum())
    assert md == ref["m_directed"]
    return ref


@pytest.mark.parametrize("seed", range(40))
def test_directed_tiny_random(tc, seed):
    n, s, d = _tiny_directed(seed)
    _check(tc, n, s, d)


@pytest.mark.parametrize("make", [
    lambda: F.transitive_tournament(1), lambda: F.transitive_tournament(2), lambda: F.transitive_tournament(45),
    lambda: F.complete_digraph(3), lambda: F.complete_digraph(60), lambda: F.directed_wheel(3),
    lambda: F.directed_wheel(200), lambda: F.directed_wheel(200, outward=False)])
def test_directed_closed_forms(tc, make):
    n, (s, d) = make()
    _check(tc, n, s, d)


def test_directed_three_vertex_cases(tc):
    _check(tc, 3, np.array([0, 1, 2]), np.array([1, 2, 0]))  # directed cycle: no pair
    _check(tc, 3, np.array([0, 0, 1]), np.array([1, 2, 2]))  # feed-forward triangle


@pytest.mark.parametrize("seed", range(6))
def test_directed_symmetric_input_is_the_undirected_lcc(tc, seed):
    n, s, d = _tiny(seed)
    both_s, both_d = np.concatenate([s, d]), np.concatenate([d, s])
    ref = _check(tc, n, both_s, both_d)
    u = oracle.triangles(n, s, d)
    np.testing.assert_array_equal(ref["c"], 2 * u["t"])
    g = tc.Graph.from_edges(n, s, d)
    try:
        t, lc = g.lcc()
    finally:
        g.close()
    c, l, _, _ = _gpu(tc, n, both_s, both_d)
    np.testing.assert_array_equal(c, 2 * t.view(np.uint64))
    np.testing.assert_array_equal(l.view(np.uint64), lc.view(np.uint64))


@pytest.mark.parametrize("scale,ef,seed", [(12, 16, 1), (14, 8, 2), (13, 24, 3)])
def test_directed_rmat(tc, scale, ef, seed):
    n = 1 << scale
    s, d = graphgen.rmat(scale, ef * n, seed=seed)
    _check(tc, n, s, d)


def test_directed_rmat_ragged_n_and_reciprocal_pairs(tc):
    n = 5003  # not a power of two: ids drawn on 2^13 and redrawn above n
    s, d = graphgen.rmat(13, 12 * n, seed=9, n=n)
    rng = np.random.default_rng(9)
    back = rng.random(len(s)) < 0.3  # 30% of the pairs also point back
    _check(tc, n, np.concatenate([s, d[back]]), np.concatenate([d, s[back]]))


def test_directed_er_device_io(tc):
    n = 4096
    s, d = graphgen.er_replace(n, 40000, seed=7)
    ref = _check(tc, n, s, d, device_io=True)
    assert ref["m_directed"] > 0


def test_directed_edge_cases(tc):
    for n, s, d in [(0, [], []), (7, [], []), (5, [1, 1, 3], [1, 1, 3]), (2, [0, 1, 0], [1, 0, 1]), (1, [0], [0])]:
        _check(tc, n, np.array(s, np.int64), np.array(d, np.int64))


def test_directed_bad_ids_leave_outputs_untouched(tc):
    n = 6
    c = np.full(n, 7, dtype=np.uint64)
    l = np.full(n, 2.5)
    for s, d in [([0, 1, 6], [1, 2, 0]), ([0, -1], [1, 2]), ([0], [1 << 20])]:
        with pytest.raises(tc.TCError) as e:
            tc.tc_directed_lcc(n, np.array(s, np.int32), np.array(d, np.int32), c, l)
        assert e.value.status == tc.TC_EINVAL
        assert (c == 7).all() and (l == 2.5).all()
    with pytest.raises(tc.TCError):
        tc.tc_directed_lcc(0, np.array([0], np.int32), np.array([0], np.int32))


def test_directed_full_size_rmat20(tc):
    """R-MAT scale 20, edge factor 16, pairs taken as directed edges: the oracle at
    sampled vertices (the highest out-degrees and a random sample), and at full size
    the properties that hold at any size: the total under reversal, and c = 2t against
    the undirected path on the symmetric input."""
    w = graphgen.workload("rmat20")
    s, d = w.edges()
    n = w.n
    c, l, total, md = _gpu(tc, n, s, d)
    dout = np.bincount(s[s != d], minlength=n)  # with repeats: ranks the candidates only
    rng = np.random.default_rng(11)
    pick = np.unique(np.concatenate([np.argsort(dout)[-4:], rng.integers(0, n, 300)])).astype(np.int32)
    ref = oracle.directed_lcc(n, s, d, vertices=pick)
    np.testing.assert_array_equal(c[pick], ref["c"])
    np.testing.assert_array_equal(l[pick].view(np.uint64), ref["lcc"].view(np.uint64))
    assert md == ref["m_directed"]
    assert total == int(c.sum())
    _, _, total_rev, md_rev = _gpu(tc, n, d, s)
    assert total_rev == total and md_rev == md
    g = tc.Graph.from_edges(n, s, d)
    try:
        t, lc = g.lcc()
    finally:
        g.close()
    c2, l2, total2, _ = _gpu(tc, n, np.concatenate([s, d]), np.concatenate([d, s]))
    np.testing.assert_array_equal(c2, 2 * t.view(np.uint64))
    np.testing.assert_array_equal(l2.view(np.uint64), lc.view(np.uint64))
    assert total2 == 2 * int(t.view(np.uint64).sum())
