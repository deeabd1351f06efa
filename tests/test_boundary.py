"""The C-ABI library loads and exports every symbol include/tc.h declares (no GPU
needed: only argument checks that fail before any device work are called)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(\w+)\s*\([^;{]*\)\s*;", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["tc_graph_create_from_edges", "tc_graph_create_from_csr", "tc_count",
                     "lcc_compute", "tc_graph_info", "tc_graph_destroy", "tc_status_str"]:
        assert required in names


def test_library_exports_every_declared_symbol(tc):
    lib = tc.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(declared_functions()) == sorted(tc.EXPORTS)


def test_status_strings(tc):
    lib = tc.load()
    for s in range(7):
        assert lib.tc_status_str(s).decode().startswith("TC_")
    assert lib.tc_status_str(99) == b"unknown tc_status"


def test_argument_errors_before_device_work(tc):
    lib = tc.load()
    out = ctypes.c_void_p()
    # NULL out, negative n, bad mem_kind, missing pointers: rejected on the host
    assert lib.tc_graph_create_from_edges(4, 1, None, None, 0, None, None) == tc.TC_EINVAL
    assert lib.tc_graph_create_from_edges(-1, 0, None, None, 0, None, ctypes.byref(out)) == tc.TC_EINVAL
    assert lib.tc_graph_create_from_edges(4, 1, None, None, 0, None, ctypes.byref(out)) == tc.TC_EINVAL
    assert lib.tc_graph_create_from_edges(4, 0, None, None, 7, None, ctypes.byref(out)) == tc.TC_EINVAL
    assert lib.tc_graph_create_from_edges(4, 1 << 40, None, None, 0, None, ctypes.byref(out)) == tc.TC_EINVAL
    assert lib.tc_graph_create_from_csr(4, None, None, 0, None, ctypes.byref(out)) == tc.TC_EINVAL
    assert lib.tc_count(None, None) == tc.TC_EINVAL
    assert lib.lcc_compute(None, None, None, 0) == tc.TC_EINVAL
    assert lib.tc_graph_set_strategy(None, 0, 0, 1.0) == tc.TC_EINVAL
    assert lib.tc_graph_set_hubs(None, 32, 10) == tc.TC_EINVAL
    assert lib.tc_graph_last_timing(None, None, 0) == tc.TC_EINVAL
    # directed LCC: negative sizes, missing pairs, bad mem_kind or flags
    assert lib.tc_directed_lcc(-1, 0, None, None, 0, None, None, None, None, 0) == tc.TC_EINVAL
    assert lib.tc_directed_lcc(4, -1, None, None, 0, None, None, None, None, 0) == tc.TC_EINVAL
    assert lib.tc_directed_lcc(4, 1, None, None, 0, None, None, None, None, 0) == tc.TC_EINVAL
    assert lib.tc_directed_lcc(4, 0, None, None, 7, None, None, None, None, 0) == tc.TC_EINVAL
    assert lib.tc_directed_lcc(4, 0, None, None, 0, None, None, None, None, 8) == tc.TC_EINVAL
    assert lib.tc_directed_lcc(4, 1 << 40, None, None, 0, None, None, None, None, 0) == tc.TC_EINVAL
    # remote-read caches: no graph
    assert lib.tc_remote_cache(None, 2, 0, None, None, None, None) == tc.TC_EINVAL
    lib.tc_graph_destroy(None)


def test_host_csr_offsets_validated_on_host(tc):
    import numpy as np
    lib = tc.load()
    out = ctypes.c_void_p()
    bad = np.array([0, 3, 2], dtype=np.int64)          # decreasing
    adj = np.zeros(3, dtype=np.int32)
    assert lib.tc_graph_create_from_csr(2, bad.ctypes.data, adj.ctypes.data, 0, None,
                                        ctypes.byref(out)) == tc.TC_EINVAL
    bad0 = np.array([1, 2, 3], dtype=np.int64)         # offsets[0] != 0
    assert lib.tc_graph_create_from_csr(2, bad0.ctypes.data, adj.ctypes.data, 0, None,
                                        ctypes.byref(out)) == tc.TC_EINVAL


def test_binding_rejects_wrong_dtypes(tc):
    import numpy as np
    with pytest.raises(TypeError):
        tc.tc_graph_create_from_edges(4, np.zeros(2, np.int64), np.zeros(2, np.int64))


class _FakeDeviceBuffer:
    """Stands in for a CUDA tensor in the binding's checks: they must reject it
    before any call into the library, so its pointer is never read."""

    is_cuda = True

    def __init__(self, dtype, n):
        self.dtype = dtype
        self._n = n

    def numel(self):
        return self._n

    def is_contiguous(self):
        return True

    def data_ptr(self):
        raise AssertionError("the binding passed a rejected buffer to the library")


@pytest.mark.parametrize("case", ["short_dst", "float_lcc", "short_t", "short_lcc", "int32_t_out", "host_src"])
def test_noalloc_binding_rejects_bad_buffers_before_the_call(tc, case):
    import numpy as np
    n, m = 100, 50
    src = _FakeDeviceBuffer("torch.int32", m)
    dst = _FakeDeviceBuffer("torch.int32", m)
    t = _FakeDeviceBuffer("torch.int64", n)
    lc = _FakeDeviceBuffer("torch.float64", n)
    if case == "short_dst":
        dst = _FakeDeviceBuffer("torch.int32", m - 1)
    elif case == "float_lcc":
        lc = _FakeDeviceBuffer("torch.float32", n)
    elif case == "short_t":
        t = _FakeDeviceBuffer("torch.int64", n - 1)
    elif case == "short_lcc":
        lc = _FakeDeviceBuffer("torch.float64", n - 1)
    elif case == "int32_t_out":
        t = _FakeDeviceBuffer("torch.int32", n)
    elif case == "host_src":
        src = np.zeros(m, np.int32)
    with pytest.raises((ValueError, TypeError)):
        tc.tc_count_noalloc(n, src, dst, t, lc)
