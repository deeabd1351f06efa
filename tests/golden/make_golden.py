"""Writes tests/golden/workloads.json: digests of the small seeded workloads and
the oracle's results on them; with --large, tests/golden/large_workloads.json: the
full-size workloads (R-MAT scale 20 and 23, the uniform graph of 8.4 M vertices)
computed by two independent formulas of the oracle, which must agree: the oriented
edge-centric count (Sec. II-C, Alg. 2) and the paper's unoriented per-vertex formula
(Alg. 3 with the Sec. II-C offset, Eq. 3 hybrid).  Calls only graphgen (inputs) and
oracle (results).

    python tests/golden/make_golden.py [--large] [--threads N]
"""
import argparse
import hashlib
import json
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

SPECS = {
    # Erdos-Renyi G(4096, 32768), seed 1
    "er4096": {"kind": "er", "n": 4096, "m": 32768, "seed": 1, "stream": 0},
    # a small R-MAT with the paper's (a, b, c, d): scale 14, edge factor 16, seed 2
    "rmat14": {"kind": "rmat", "n": 1 << 14, "scale": 14, "m": 16 << 14, "seed": 2, "stream": 0},
}


def digest(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


LARGE = ["rmat20", "er23", "rmat23"]


def vertex_formula_all(n, offsets, adj, threads):
    """Alg. 3 for every vertex, the vertices dealt round-robin to ``threads`` calls of
    the oracle's single-threaded routine (each releases the interpreter lock)."""
    t = np.zeros(n, dtype=np.uint64)
    chunks = [np.arange(i, n, 64 * threads, dtype=np.int32) for i in range(64 * threads)]

    def run(vs):
        return vs, oracle.tc_vertex(n, offsets, adj, vs)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        for vs, tv in ex.map(run, chunks):
            t[vs] = tv
    return t


def large(threads):
    out = {}
    for name in LARGE:
        w = graphgen.workload(name)
        s, d = w.edges()
        t0 = time.perf_counter()
        r = oracle.triangles(w.n, s, d, threads=threads)
        t1 = time.perf_counter()
        offsets, adj, _ = oracle.build_csr(w.n, s, d)
        tv = vertex_formula_all(w.n, offsets, adj, threads)
        t2 = time.perf_counter()
        assert np.array_equal(tv, r["t"]), f"{name}: the two formulas disagree"
        assert int(tv.sum()) == 3 * r["T"]
        out[name] = {"n": w.n, "pairs": int(len(s)), "edges_sha256": digest(s, d), "T": r["T"],
                     "m_simple": r["m_simple"], "loops_dropped": r["loops_dropped"],
                     "t_sha256": digest(r["t"]), "lcc_sha256": digest(r["lcc"]),
                     "formulas": ["oriented edge-centric count (Sec. II-C, Alg. 2)",
                                  "unoriented per-vertex formula (Alg. 3, Eq. 3 hybrid)"],
                     "seconds": {"oriented": round(t1 - t0, 1), "per_vertex": round(t2 - t1, 1)}}
        print(name, out[name]["T"], out[name]["seconds"], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "large_workloads.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--large", action="store_true")
    ap.add_argument("--threads", type=int, default=len(os.sched_getaffinity(0)))
    args = ap.parse_args()
    if args.large:
        large(args.threads)
        return
    out = {}
    for name, spec in SPECS.items():
        if spec["kind"] == "rmat":
            s, d = graphgen.rmat(spec["scale"], spec["m"], seed=spec["seed"], stream=spec["stream"])
        else:
            s, d = graphgen.er(spec["n"], spec["m"], seed=spec["seed"], stream=spec["stream"])
        r = oracle.triangles(spec["n"], s, d)
        out[name] = {"spec": spec, "edges_sha256": digest(s, d), "T": r["T"],
                     "m_simple": r["m_simple"], "t_sha256": digest(r["t"]),
                     "lcc_sha256": digest(r["lcc"])}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps({k: v["T"] for k, v in out.items()}))


if __name__ == "__main__":
    main()
