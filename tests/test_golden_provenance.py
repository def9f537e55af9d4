"""The stored workload files under tests/golden/ against what wrote them
(tests/golden/make_workloads.py, make_rmat20_counts.py): the seeded
generators rebuild the same graphs (SHA-256 of the CSR and labels) and the
same queries, and the oracle, re-run on the stored slices it finishes
quickly, gives the stored counts and row digests (for the R-MAT 20 file:
its graph and its listed slice).  So no stored value can have drifted from
the oracle's.  No GPU."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2003_01527_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def graph_digest(g) -> str:
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col, g.labels):
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    return h.hexdigest()


def rows_digest(rows) -> str:
    return hashlib.sha256(np.ascontiguousarray(rows, dtype="<i4").tobytes()).hexdigest()


def check(gold, g, qs, max_count, min_checked):
    assert graph_digest(g) == gold["graph"]["sha256"]
    assert (g.n, g.nnz) == (gold["graph"]["n"], gold["graph"]["nnz"])
    assert len(qs) == len(gold["queries"])
    checked = 0
    for q, item in zip(qs, gold["queries"]):
        # the stored query is the generator's
        assert item["k"] == q.k
        assert item["edges"] == q.edges.tolist()
        assert item["labels"] == q.labels.tolist()
        if q.walk is not None:
            assert item["walk"] == q.walk.tolist()
        if item["count"] > max_count:
            continue
        count, rows, rc = oracle.match(g, q, root_range=(0, item["root_hi"]))
        assert rc == oracle.OK
        assert count == item["count"]
        assert rows_digest(rows) == item["rows_sha256"]
        checked += 1
    assert checked >= min_checked


def test_rmat16_labelled_slices(oracle_lib):
    with open(os.path.join(GOLDEN, "rmat16_labelled_slices.json")) as f:
        gold = json.load(f)
    g, qs = I.rmat_labelled_workload(scale=16, num_labels=8, zipf_s=1.0, num_queries=20,
                                     kmin=4, kmax=8, seed=2)
    # the empty slices and q10 (113,184 rows)
    check(gold, g, qs, max_count=200_000, min_checked=10)


def test_rmat18_batched_slices(oracle_lib):
    with open(os.path.join(GOLDEN, "rmat18_batched_slices.json")) as f:
        gold = json.load(f)
    g, qs = I.rmat_labelled_workload(scale=18, num_labels=16, zipf_s=1.2, num_queries=256,
                                     kmin=3, kmax=10, non_tree=(2, 4), seed=4)
    check(gold, g, qs, max_count=300_000, min_checked=256)  # every slice


def test_rmat20_unlabelled_graph_and_listed_slice(oracle_lib):
    with open(os.path.join(GOLDEN, "rmat20_unlabelled.json")) as f:
        gold = json.load(f)
    g = I.rmat_unlabelled_graph(scale=20, seed=3)
    assert graph_digest(g) == gold["graph"]["sha256"]
    assert (g.n, g.nnz) == (gold["graph"]["n"], gold["graph"]["nnz"])
    shapes = I.unlabelled_shapes()
    listed = [s for s in gold["slices"] if s["rows_sha256"] and s["window"] is None]
    assert listed
    for s in listed:
        count, rows, rc = oracle.match(g, shapes[s["shape"]],
                                       root_range=(s["root_lo"], s["root_hi"]))
        assert rc == oracle.OK
        assert count == s["count"]
        assert rows_digest(rows) == s["rows_sha256"]
