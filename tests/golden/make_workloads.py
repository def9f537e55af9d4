"""Writes the stored workload files under tests/golden/ (run by hand; calls only
the seeded generators and the CPU oracle).

Why slices: on a power-law R-MAT graph the hub core is close to a clique, so a
random-walk query of 5-8 vertices typically has 10^10 - 10^17 ordered
embeddings (the spanning-tree homomorphism count bounds them from above and is
reached closely for tree-like queries).  No exact method can list that many.
Each query is therefore restricted to the embeddings whose image of query
vertex 0 lies in a prefix [0, hi) of the (randomly permuted) vertex ids; hi is
the largest prefix, found by doubling then bisection, for which the oracle
finds at most CAP embeddings within its search-node budget.  The restricted
result is exactly the first `count` rows of the query's full sorted result.

Per query the file stores the query, hi, the oracle's count and the SHA-256 of
the oracle's sorted int32 rows (little endian, row major).

    python tests/golden/make_workloads.py labelled16
    python tests/golden/make_workloads.py batched18
    python tests/golden/make_workloads.py served22
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


def graph_digest(g) -> str:
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col, g.labels):
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    return h.hexdigest()


def rows_digest(rows: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(rows, dtype="<i4").tobytes()).hexdigest()


def feasible(g, q, hi, cap, budget):
    c, _, rc = oracle.match(g, q, enumerate=False, root_range=(0, hi), limit=cap,
                            node_budget=budget)
    return rc == oracle.OK, c


def find_prefix(g, q, cap, budget):
    good, bad = 0, None
    hi = 1
    while hi <= g.n:
        ok, _ = feasible(g, q, hi, cap, budget)
        if not ok:
            bad = hi
            break
        good = hi
        if hi == g.n:
            break
        hi = min(2 * hi, g.n)
    if bad is not None:
        for _ in range(6):
            if bad - good <= 1:
                break
            mid = (good + bad) // 2
            ok, _ = feasible(g, q, mid, cap, budget)
            if ok:
                good = mid
            else:
                bad = mid
    return good


def make(name, g, qs, cap, budget, meta):
    t0 = time.time()
    out = {"workload": name, "meta": meta, "cap_rows": cap, "node_budget": budget,
           "graph": {"n": g.n, "nnz": g.nnz, "sha256": graph_digest(g)}, "queries": []}
    for i, q in enumerate(qs):
        hi = find_prefix(g, q, cap, budget)
        c, rows, rc = oracle.match(g, q, enumerate=True, root_range=(0, hi))
        assert rc == oracle.OK
        out["queries"].append({
            "k": q.k, "edges": q.edges.tolist(), "labels": q.labels.tolist(),
            "walk": None if q.walk is None else q.walk.tolist(),
            "root_vertex": 0, "root_hi": hi, "count": int(c), "rows_sha256": rows_digest(rows)})
        print(f"{name} q{i}: k={q.k} m={q.m} hi={hi} count={c} ({time.time() - t0:.0f}s)",
              flush=True)
    path = os.path.join(HERE, f"{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


SERVED_WINDOW = 1 << 18


def served22():
    """The served workload: resident R-MAT scale 22 with 32 Zipf(1.0) labels
    and a pool of random-walk queries of 3-12 vertices that the request
    stream draws from.  On this graph almost every root of a query of six or
    more vertices reaches hubs with far more embeddings than the oracle can
    count, so every query vertex is restricted to the id window
    [0, SERVED_WINDOW) (ids are randomly permuted: a uniform sample of 1/16
    of the vertices), each walk is drawn inside the subgraph induced by the
    window (so it is itself an embedding there), and the root is restricted
    to a prefix [0, hi) sized by the oracle.  Queries are drawn size by size
    (k = 3..12), keeping up to 10 non-empty slices of each size from at most
    150 draws."""
    n, rp, col = inputs.rmat(22, 16, *inputs.RMAT_ABC, seed=5)
    g = inputs.make_graph(n, rp, col, inputs.zipf_labels(n, 32, 1.0, seed=105))
    W = SERVED_WINDOW
    src = np.repeat(np.arange(n), np.diff(g.row_ptr))
    keep = (src < W) & (g.col < W)
    srp, scol = inputs.csr_from_pairs(W, src[keep], g.col[keep])
    sub = inputs.make_graph(W, srp, scol, g.labels[:W])
    del src, keep
    rng = np.random.default_rng(305)
    cap, budget = 1 << 16, 1 << 25
    t0 = time.time()
    out = {"workload": "rmat22_served_slices",
           "meta": {"generator": "inputs.rmat(22, 16, *RMAT_ABC, seed=5), zipf_labels(n, 32, "
                                 "1.0, seed=105); random_walk_query in the subgraph induced by "
                                 "ids [0, 2^18), default_rng(305), k = 3..12, up to 10 "
                                 "non-empty slices per k from at most 150 draws",
                    "window": W},
           "cap_rows": cap, "node_budget": budget,
           "graph": {"n": g.n, "nnz": g.nnz, "sha256": graph_digest(g)}, "queries": []}
    for k in range(3, 13):
        kept = 0
        for _ in range(150):
            if kept >= 10:
                break
            q = inputs.random_walk_query(sub, k, rng)
            ranges = {u: (0, W) for u in range(k)}
            good, hi = 0, 1
            while hi <= W:
                c, _, rc = oracle.match(g, q, enumerate=False, root_range=(0, hi), limit=cap,
                                        node_budget=budget, ranges=ranges)
                if rc != oracle.OK:
                    break
                good = hi
                hi *= 2
            if good == 0:
                continue
            c, rows, rc = oracle.match(g, q, enumerate=True, root_range=(0, good), ranges=ranges)
            assert rc == oracle.OK
            if c == 0:
                continue
            kept += 1
            out["queries"].append({
                "k": q.k, "edges": q.edges.tolist(), "labels": q.labels.tolist(),
                "walk": q.walk.tolist(), "root_vertex": 0, "root_hi": good, "window": W,
                "count": int(c), "rows_sha256": rows_digest(rows)})
            print(f"served22 k={k} hi={good} count={c} ({time.time() - t0:.0f}s)", flush=True)
    path = os.path.join(HERE, "rmat22_served_slices.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


def main(which):
    if which == "labelled16":
        g, qs = inputs.rmat_labelled_workload(scale=16, num_labels=8, zipf_s=1.0,
                                              num_queries=20, kmin=4, kmax=8, seed=2)
        make("rmat16_labelled_slices", g, qs, cap=1 << 24, budget=1 << 29,
             meta={"generator": "inputs.rmat_labelled_workload(scale=16, num_labels=8, "
                                "zipf_s=1.0, num_queries=20, kmin=4, kmax=8, seed=2)"})
    elif which == "batched18":
        g, qs = inputs.rmat_labelled_workload(scale=18, num_labels=16, zipf_s=1.2,
                                              num_queries=256, kmin=3, kmax=10,
                                              non_tree=(2, 4), seed=4)
        make("rmat18_batched_slices", g, qs, cap=1 << 18, budget=1 << 25,
             meta={"generator": "inputs.rmat_labelled_workload(scale=18, num_labels=16, "
                                "zipf_s=1.2, num_queries=256, kmin=3, kmax=10, "
                                "non_tree=(2, 4), seed=4)"})
    elif which == "served22":
        served22()
    else:
        raise SystemExit(f"unknown workload {which}")


if __name__ == "__main__":
    main(sys.argv[1])
