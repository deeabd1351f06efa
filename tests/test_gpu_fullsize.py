"""Parity at the full workload sizes, in the launch configuration the benchmark
times (default strategies): T and every t[v] and LCC[v] against the oracle (its
oriented count split over the host cores), and against the digests that two
independent oracle formulas agreed on (tests/golden/large_workloads.json)."""
from __future__ import annotations

import os

import numpy as np
import pytest

import graphgen
import oracle
from tests.gpu_util import gpu_run
from tests.test_golden_large import _digest, large_golden

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["rmat20", "er23", "rmat23"])
def test_full_workload(tc, name):
    w = graphgen.workload(name)
    s, d = w.edges()
    T, t, lc, info = gpu_run(tc, w.n, s, d, device_io=True)
    ref = oracle.triangles(w.n, s, d, threads=len(os.sched_getaffinity(0)))
    assert T == ref["T"]
    assert info["m_simple"] == ref["m_simple"]
    assert info["loops_dropped"] == ref["loops_dropped"]
    np.testing.assert_array_equal(t, ref["t"])
    np.testing.assert_array_equal(lc.view(np.uint64), ref["lcc"].view(np.uint64))
    want = large_golden()[name]
    assert T == want["T"]
    assert _digest(np.ascontiguousarray(t, dtype=np.uint64)) == want["t_sha256"]
    assert _digest(np.ascontiguousarray(lc, dtype=np.float64)) == want["lcc_sha256"]
    # properties that hold at any size
    assert int(t.sum()) == 3 * T
    deg = ref["degree"]
    assert (t <= deg * (deg - 1) // 2).all()


def test_sparse_graph_with_many_vertices(tc):
    """2^27 vertex ids, 2^22 R-MAT pairs: most vertices are isolated, the rank sort
    covers 27-bit ids, the hub capacity stops at its cap far below n, and every
    n-sized pass runs over 134 M entries.  Device buffers in and out."""
    n = 1 << 27
    s, d = graphgen.rmat(27, 1 << 22, seed=11)
    T, t, lc, info = gpu_run(tc, n, s, d, device_io=True)
    ref = oracle.triangles(n, s, d, threads=len(os.sched_getaffinity(0)))
    assert T == ref["T"]
    assert info["m_simple"] == ref["m_simple"]
    np.testing.assert_array_equal(t, ref["t"])
    np.testing.assert_array_equal(lc.view(np.uint64), ref["lcc"].view(np.uint64))
