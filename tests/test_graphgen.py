"""Checks of the seeded input generators (no GPU)."""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import graphgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "workloads.json")


def test_splitmix_reference_values():
    # SplitMix64 seeded with 1234567 (Vigna's splitmix64.c): first outputs.
    # The counter form draw(key, i) = mix(key + (i+1) gamma) equals the
    # sequential generator whose state starts at key.
    g = 0x9e3779b97f4a7c15
    M = (1 << 64) - 1

    def mix(z):
        z = ((z ^ (z >> 30)) * 0xbf58476d1ce4e5b9) & M
        z = ((z ^ (z >> 27)) * 0x94d049bb133111eb) & M
        return z ^ (z >> 31)

    key = graphgen.stream_key(7, 3)
    seq = []
    state = key
    for _ in range(5):
        state = (state + g) & M
        seq.append(mix(state))
    assert graphgen.draws(7, 3, 0, 5).tolist() == seq
    # published first output of SplitMix64 with state 1234567
    assert mix((1234567 + g) & M) == 6457827717110365317


def test_rmat_pair_count_follows_table1_reading():
    # Table I: R-MAT S21 EF16 has 33.6 M edges and S23 EF16 134.2 M: y * 2^x pairs.
    assert 16 * 2 ** 21 == 33_554_432
    assert 16 * 2 ** 23 == 134_217_728
    s, d = graphgen.rmat(12, 16 << 12, seed=1)
    assert len(s) == len(d) == 16 << 12
    assert s.min() >= 0 and s.max() < 4096 and d.max() < 4096


def test_rmat_skew_and_quadrant_frequencies():
    s, d = graphgen.rmat(16, 1 << 20, seed=2)
    # top bit of the row is set for quadrants c and d: probability 0.24
    top = (s >> 15) & 1
    assert abs(top.mean() - 0.24) < 0.003
    colbit = (d >> 15) & 1
    assert abs(colbit.mean() - 0.24) < 0.003
    deg = np.bincount(s, minlength=1 << 16) + np.bincount(d, minlength=1 << 16)
    assert deg.argmax() == 0


def test_rmat_non_power_of_two_n():
    s, d = graphgen.rmat(7, 5000, seed=3, n=100)
    assert s.max() < 100 and d.max() < 100


@pytest.mark.parametrize("n,m", [(4096, 32768), (50, 1225), (50, 1000), (3000, 100), (2, 5)])
def test_er_distinct_pairs(n, m):
    s, d = graphgen.er(n, m, seed=4)
    assert len(s) == min(m, n * (n - 1) // 2)
    assert (s != d).all()
    key = np.minimum(s, d).astype(np.int64) * n + np.maximum(s, d)
    assert len(np.unique(key)) == len(key)
    assert s.min() >= 0 and max(s.max(), d.max()) < n


def test_determinism():
    a = graphgen.rmat(10, 5000, seed=8)
    b = graphgen.rmat(10, 5000, seed=8)
    c = graphgen.rmat(10, 5000, seed=8, stream=1)
    assert all((x == y).all() for x, y in zip(a, b))
    assert not (a[0] == c[0]).all()


def _digest(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def test_golden_workloads():
    """Edge lists and oracle results of the small workloads match the stored file
    (written by tests/golden/make_golden.py, which calls only graphgen and oracle)."""
    import oracle
    gold = json.load(open(GOLDEN))
    for name, want in gold.items():
        spec = want["spec"]
        if spec["kind"] == "rmat":
            s, d = graphgen.rmat(spec["scale"], spec["m"], seed=spec["seed"], stream=spec["stream"])
        else:
            s, d = graphgen.er(spec["n"], spec["m"], seed=spec["seed"], stream=spec["stream"])
        assert _digest(s, d) == want["edges_sha256"], name
        r = oracle.triangles(spec["n"], s, d)
        assert r["T"] == want["T"], name
        assert _digest(r["t"]) == want["t_sha256"], name
        assert _digest(r["lcc"]) == want["lcc_sha256"], name
        assert r["m_simple"] == want["m_simple"], name


def test_batch_specs():
    ws = graphgen.batch_workloads(200, seed=4)
    assert len(ws) == 200
    ns = np.array([w.n for w in ws])
    assert ns.min() >= 32 and ns.max() <= 65536
    assert all(w.kind == ("rmat" if i % 2 == 0 else "er") for i, w in enumerate(ws))
    for w in ws[:6]:
        s, d = w.edges()
        assert s.max() < w.n
