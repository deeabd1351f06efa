"""Writes tests/golden/workloads.json: digests of the small seeded workloads and
the oracle's results on them.  Calls only graphgen (inputs) and oracle (results).

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

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


def main():
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
