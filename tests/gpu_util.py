"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare it with the oracle."""
from __future__ import annotations

import numpy as np

import oracle


def gpu_run(tc, n, src, dst, device_io=False, strategies=None, csr=None, stream=None, hubs=None, tuning=None):
    """T, t, lcc and input accounting from the CUDA library.

    device_io: inputs and outputs as CUDA tensors (TC_MEM_DEVICE), else numpy.
    strategies: {bucket: (strategy, factor)} applied before counting.
    hubs: (min_degree, max_hubs) for the hub bucket.
    tuning: {field: value} merged into the graph's tuning before counting.
    csr: (offsets, adj) to build from CSR instead of the edge list."""
    import torch
    if csr is not None:
        off, adj = csr
        if device_io:
            g = tc.Graph.from_csr(n, torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda(), stream)
        else:
            g = tc.Graph.from_csr(n, off, adj, stream)
    elif device_io:
        g = tc.Graph.from_edges(n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), stream)
    else:
        g = tc.Graph.from_edges(n, src, dst, stream)
    try:
        for bucket, (s, f) in (strategies or {}).items():
            g.set_strategy(bucket, s, f)
        if hubs is not None:
            g.set_hubs(*hubs)
        if tuning:
            t0 = g.tuning()
            t0.update(tuning)
            g.set_tuning(t0)
        T = g.count()
        if device_io:
            t = torch.empty(n, dtype=torch.int64, device="cuda")
            lc = torch.empty(n, dtype=torch.float64, device="cuda")
            g.lcc(t, lc)
            torch.cuda.synchronize()
            t = t.cpu().numpy().view(np.uint64)
            lc = lc.cpu().numpy()
        else:
            t, lc = g.lcc()
        info = g.info()
    finally:
        g.close()
    return T, t, lc, info


def assert_matches_oracle(tc, n, src, dst, ref=None, **kw):
    ref = ref if ref is not None else oracle.triangles(n, src, dst)
    T, t, lc, info = gpu_run(tc, n, src, dst, **kw)
    assert T == ref["T"]
    np.testing.assert_array_equal(t, ref["t"])
    # 0 ulp: identical bits
    np.testing.assert_array_equal(lc.view(np.uint64), ref["lcc"].view(np.uint64))
    if "csr" not in kw:
        assert info["m_simple"] == ref["m_simple"]
        assert info["loops_dropped"] == ref["loops_dropped"]
        assert info["dups_dropped"] == ref["dups_dropped"]
    return ref
