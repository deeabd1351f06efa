"""Writes tests/golden/workloads.json: digests of the small seeded workloads and
the oracle's results on them; with --large, tests/golden/large_workloads.json: the
full-size workloads (R-MAT scale 20 and 23, the uniform graph of 8.4 M vertices)
computed by two independent formulas of the oracle, which must agree: the oriented
edge-centric count (Sec. II-C, Alg. 2) and the paper's unoriented per-vertex formula
(Alg. 3 with the Sec. II-C offset, Eq. 3 hybrid).  Calls only graphgen (inputs) and
oracle (results).

With --batch, tests/golden/batch_workload.json: the oracle's results on every graph
of the 20,000-graph batch (seed 4), as digests of the per-graph T and of t[] and
LCC[] concatenated graph by graph.

    python tests/golden/make_golden.py [--large] [--batch] [--threads N]
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


def _batch_one(i):
    w = graphgen.batch_workloads(BATCH_G, seed=BATCH_SEED)[i] if _BATCH is None else _BATCH[i]
    s, d = w.edges()
    r = oracle.triangles(w.n, s, d)
    return i, r["T"], r["m_simple"], r["t"], r["lcc"]


BATCH_G, BATCH_SEED = 20000, 4
_BATCH = None


def _batch_init():
    global _BATCH
    _BATCH = graphgen.batch_workloads(BATCH_G, seed=BATCH_SEED)


def batch(threads):
    import multiprocessing as mp
    G = BATCH_G
    T = np.zeros(G, dtype=np.uint64)
    ms = np.zeros(G, dtype=np.int64)
    ts, ls = [None] * G, [None] * G
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(threads, initializer=_batch_init) as pool:
        for i, Ti, mi, ti, li in pool.imap_unordered(_batch_one, range(G), chunksize=16):
            T[i], ms[i], ts[i], ls[i] = Ti, mi, ti, li
    t_all = np.concatenate(ts).astype(np.uint64)
    l_all = np.concatenate(ls).astype(np.float64)
    out = {"graphs": G, "seed": BATCH_SEED, "vertices": int(t_all.size), "m_simple": int(ms.sum()),
           "T_total": int(T.sum(dtype=np.uint64)), "T_sha256": digest(T), "m_simple_sha256": digest(ms),
           "t_sha256": digest(t_all), "lcc_sha256": digest(l_all),
           "seconds": round(time.perf_counter() - t0, 1)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_workload.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(out, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--large", action="store_true")
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--threads", type=int, default=len(os.sched_getaffinity(0)))
    args = ap.parse_args()
    if args.large:
        large(args.threads)
        return
    if args.batch:
        batch(args.threads)
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
