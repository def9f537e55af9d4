"""Writes tests/golden/rmat20_unlabelled.json: reference counts for the
unlabelled R-MAT scale-20 workload (run by hand; calls only the seeded
generator and the CPU oracle).

Stored values:
  * the k-clique counts for k = 3 and 4 (each clique once), from the oracle's
    degree-ordered clique listing -- an algorithm independent of both the
    library and the oracle's backtracking matcher.  The ordered embedding
    counts of the triangle and of K4 are 3! and 4! times these (every
    permutation of a clique is an automorphic image); for the triangle this
    is tr(A^3).
  * root-range slices of the 5-cycle and the 6-vertex path: the largest
    window [lo, lo + w) of the image of query vertex 0 (w doubled from 1)
    that the backtracking oracle counts within its node budget, with the
    other query vertices of the path kept inside an id window so that a
    slice stays countable (from a single root there are far too many 6-paths:
    every vertex is two hops from a hub).  Each slice stores the count, and
    the SHA-256 of the sorted rows when the oracle can also list them.

    python tests/golden/make_rmat20_counts.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2003_01527_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "rmat20_unlabelled.json")

NODE_BUDGET = 1 << 31       # backtracking steps per slice count
LIST_CAP = 1 << 24          # rows listed for a digest
SLICES = [  # (shape, lo, window of the other query vertices or None)
    ("cycle5", 0, None),
    ("cycle5", 524_288, None),
    ("path6", 350_000, 1 << 16),
    ("path6", 700_000, 1 << 16),
]


def graph_digest(g) -> str:
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col, g.labels):
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    return h.hexdigest()


def main():
    t0 = time.time()
    g = inputs.rmat_unlabelled_graph(scale=20, seed=3)
    out = {"workload": "rmat20_unlabelled",
           "generator": "inputs.rmat_unlabelled_graph(scale=20, seed=3)",
           "graph": {"n": g.n, "nnz": g.nnz, "sha256": graph_digest(g)},
           "cliques": {}, "slices": []}
    for k in (3, 4):
        c = oracle.cliques(g, k)
        out["cliques"][str(k)] = int(c)
        print(f"{k}-cliques: {c} ({time.time() - t0:.0f}s)", flush=True)
    shapes = inputs.unlabelled_shapes()
    for shape, lo, window in SLICES:
        q = shapes[shape]
        ranges = None if window is None else {u: (0, window) for u in range(1, q.k)}
        best = None
        w = 1
        while lo + w <= g.n:
            c, _, rc = oracle.match(g, q, enumerate=False, root_range=(lo, lo + w),
                                    node_budget=NODE_BUDGET, ranges=ranges)
            if rc != oracle.OK:
                break
            best = (w, int(c))
            w *= 2
        assert best is not None, f"{shape} at {lo}: not even one root is countable"
        w, c = best
        digest = None
        if c <= LIST_CAP:
            c2, rows, rc = oracle.match(g, q, enumerate=True, root_range=(lo, lo + w),
                                        ranges=ranges)
            assert rc == oracle.OK and c2 == c
            digest = hashlib.sha256(np.ascontiguousarray(rows, dtype="<i4").tobytes()).hexdigest()
        out["slices"].append({"shape": shape, "root_lo": lo, "root_hi": lo + w,
                              "window": window, "count": c, "rows_sha256": digest})
        print(f"{shape} [{lo}, {lo + w}) window {window}: {c} ({time.time() - t0:.0f}s)",
              flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
