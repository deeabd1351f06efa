"""Parity of the remote-read cache evaluation (tc_remote_cache through the C ABI) with
the oracle's direct simulation of every cache at every capacity: hits, hit bytes and
the per-process read counts, bit-exact."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle
from tests import families as F
from tests.test_oracle import _tiny

pytestmark = pytest.mark.gpu

CAPS = [0, 4, 16, 40, 64, 100, 256, 400, 1000, 4000, 1 << 20]


def _check(tc, n, s, d, parts, caps=CAPS):
    s = np.ascontiguousarray(s, dtype=np.int32)
    d = np.ascontiguousarray(d, dtype=np.int32)
    ref = oracle.remote_cache(n, s, d, parts, caps)
    g = tc.Graph.from_edges(n, s, d)
    try:
        got = g.remote_cache(parts, caps)
    finally:
        g.close()
    for key in ("reads", "top_reads", "distinct", "read_bytes"):
        np.testing.assert_array_equal(got[key], ref[key], err_msg=key)
    np.testing.assert_array_equal(got["hits"], ref["hits"])
    np.testing.assert_array_equal(got["hit_bytes"], ref["hit_bytes"])
    return got


@pytest.mark.parametrize("seed", range(12))
def test_cache_tiny_random(tc, seed):
    n, s, d = _tiny(seed)
    _check(tc, n, s, d, 1 + seed % 5 if n >= 5 else 1)


@pytest.mark.parametrize("make,parts", [(lambda: F.complete(40), 4), (lambda: F.star(99), 2),
                                        (lambda: F.wheel(64), 8), (lambda: F.grid(12, 17), 3)])
def test_cache_closed_form_graphs(tc, make, parts):
    n, (s, d) = make()
    _check(tc, n, s, d, parts)


@pytest.mark.parametrize("scale,ef,parts", [(10, 16, 2), (12, 8, 4), (11, 12, 8), (12, 16, 3)])
def test_cache_rmat(tc, scale, ef, parts):
    n = 1 << scale
    s, d = graphgen.rmat(scale, ef * n, seed=scale + parts)
    caps = sorted(set([0] + [int(x) for x in np.geomspace(16, 4 * ef * n, 30)]))
    _check(tc, n, s, d, parts, caps)


def test_cache_er_ragged_and_one_process(tc):
    n = 3001
    s, d = graphgen.er(n, 20000, seed=3)
    _check(tc, n, s, d, 7)
    got = _check(tc, n, s, d, 1)
    assert (got["reads"] == 0).all() and (got["hits"] == 0).all()
    _check(tc, n, s, d, n)  # one vertex per process


def test_cache_empty_and_bad_arguments(tc):
    g = tc.Graph.from_edges(5, np.array([], np.int32), np.array([], np.int32))
    try:
        got = g.remote_cache(2, [0, 10])
        assert (got["reads"] == 0).all() and (got["hits"] == 0).all()
        for parts, caps in [(0, [1]), (6, [1]), (2, [10, 5])]:
            with pytest.raises(tc.TCError) as e:
                g.remote_cache(parts, caps)
            assert e.value.status == tc.TC_EINVAL
    finally:
        g.close()


def test_cache_full_size_rmat20_two_processes(tc):
    """R-MAT scale 20, edge factor 16 on two processes, the configuration of the
    paper's cache-size study (Sec. V-C), at two cache sizes."""
    w = graphgen.workload("rmat20")
    s, d = w.edges()
    _check(tc, w.n, s, d, 2, [1 << 20, 1 << 26])
