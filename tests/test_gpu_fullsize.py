"""Full-size parity for the unlabelled R-MAT scale-20 workload (triangle,
4-clique, 5-cycle, 6-vertex path; chunked under a small memory budget) and the
labelled R-MAT scale-22 graph of the served workload.

At these sizes the oracle's backtracking cannot list everything, so the
checks are: closed forms that hold at any size (edge count = nnz, ordered
3-paths = sum d(d-1)); the full triangle and 4-clique counts against the
values stored in tests/golden/rmat20_unlabelled.json, written by the oracle's
independent clique listing (ordered triangles = 3! x triangles = tr(A^3),
distinct 4-cliques); root slices of the 5-cycle and 6-path against the
oracle's stored counts and row digests; root slices the oracle lists here
(compared row for row); and consistency of a chunked full count with the
unchunked one and with the sum of slice counts.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2003_01527_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def oracle_slice(g, q, lo, width, limit=2_000_000, budget=200_000_000, ranges=None):
    """Largest root range [lo, lo+w), w <= width halved until the oracle lists
    it within the limits; returns (lo, hi, count, rows)."""
    w = width
    while w >= 1:
        c, _, rc = oracle.match(g, q, enumerate=False, root_range=(lo, lo + w), limit=limit,
                                node_budget=budget, ranges=ranges)
        if rc == oracle.OK:
            c, rows, _ = oracle.match(g, q, root_range=(lo, lo + w), ranges=ranges)
            return lo, lo + w, c, rows
        w //= 2
    return lo, lo, 0, np.zeros((0, q.k), np.int32)


GOLDEN20 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "rmat20_unlabelled.json")


def graph_digest(g) -> str:
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col, g.labels):
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    return h.hexdigest()


@pytest.fixture(scope="module")
def rmat20():
    return I.rmat_unlabelled_graph(scale=20, seed=3)


@pytest.fixture(scope="module")
def gold20(rmat20):
    with open(GOLDEN20) as f:
        gold = json.load(f)
    assert gold["graph"]["sha256"] == graph_digest(rmat20)
    return gold


def test_rmat20_closed_forms_and_chunked_counts(gsm_lib, cuda, rmat20, gold20):
    g = rmat20
    d = g.degrees()
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels, validate=True)
    assert m.count(m.query(2, [(0, 1)])) == g.nnz
    path3 = m.query(3, [(0, 1), (1, 2)])
    assert m.count(path3) == int((d * (d - 1)).sum())
    s = I.unlabelled_shapes()
    tri = s["triangle"]
    full = m.count(m.query(3, tri.edges))
    # pinned by the oracle's clique listing: 3! ordered maps per triangle
    assert full == 6 * gold20["cliques"]["3"]
    assert m.count_distinct(m.query(3, tri.edges)) == (gold20["cliques"]["3"], 6)
    assert m.count_distinct(m.query(4, s["clique4"].edges)) == (gold20["cliques"]["4"], 24)
    m.close()
    # the same counts under a 64 MB budget: frontiers are chunked
    mc = gsm_lib.Matcher(device=0, mem_budget_bytes=64 << 20)
    mc.load_graph(g.row_ptr, g.col, g.labels)
    assert mc.count(mc.query(3, tri.edges)) == full
    assert mc.last_run_stats()["chunks"] > 2
    assert mc.count(mc.query(3, [(0, 1), (1, 2)])) == int((d * (d - 1)).sum())
    # and the full count is the sum over a partition of root ranges
    cuts = [0, 300_000, 600_001, 900_000, g.n]
    parts = [mc.count(mc.query(3, tri.edges).restrict(0, a, b)) for a, b in zip(cuts, cuts[1:])]
    assert sum(parts) == full
    mc.close()


def test_rmat20_stored_slices(gsm_lib, cuda, rmat20, gold20):
    """5-cycle and 6-path root slices sized to the oracle's search budget:
    counts (and, where the oracle listed them, sorted rows) equal the stored
    oracle values."""
    g = rmat20
    shapes = I.unlabelled_shapes()
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels)
    for sl in gold20["slices"]:
        q = shapes[sl["shape"]]
        Q = m.query(q.k, q.edges).restrict(0, sl["root_lo"], sl["root_hi"])
        if sl["window"]:
            for u in range(1, q.k):
                Q.restrict(u, 0, sl["window"])
        assert m.count(Q) == sl["count"], sl
        if sl["rows_sha256"]:
            rows, count = m.enumerate(Q)
            assert count == sl["count"]
            digest = hashlib.sha256(np.ascontiguousarray(rows, dtype="<i4").tobytes())
            assert digest.hexdigest() == sl["rows_sha256"], sl
    m.close()


# The 6-path also keeps its other five vertices inside the id window
# [0, 2^14): from any single root there are far too many 6-paths (every vertex
# is two hops from a hub), and the sample must stay listable.
WINDOW = {u: (0, 1 << 14) for u in range(1, 6)}


@pytest.mark.parametrize("shape,lo,width,ranges", [("triangle", 0, 4096, None),
                                                   ("triangle", 524_288, 4096, None),
                                                   ("clique4", 1_000_000, 2048, None),
                                                   ("cycle5", 524_288, 64, None),
                                                   ("path6", 700_000, 64, WINDOW)])
def test_rmat20_slices_match_oracle(gsm_lib, cuda, rmat20, shape, lo, width, ranges):
    g = rmat20
    q = I.unlabelled_shapes()[shape]
    lo, hi, want_count, want_rows = oracle_slice(g, q, lo, width, ranges=ranges)
    assert hi > lo and want_count > 0
    m = gsm_lib.Matcher(device=0, mem_budget_bytes=256 << 20)
    m.load_graph(g.row_ptr, g.col, g.labels)
    Q = m.query(q.k, q.edges).restrict(0, lo, hi)
    for u, (a, b) in (ranges or {}).items():
        Q.restrict(u, a, b)
    rows, count = m.enumerate(Q)
    assert count == want_count
    assert np.array_equal(rows, want_rows)
    assert m.count(Q) == want_count
    m.close()


GOLDEN22 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "rmat22_served_slices.json")


@pytest.fixture(scope="module")
def rmat22():
    n, rp, col = I.rmat(22, 16, *I.RMAT_ABC, seed=5)
    return I.make_graph(n, rp, col, I.zipf_labels(n, 32, 1.0, seed=105))


def test_rmat22_served_pool(gsm_lib, cuda, rmat22):
    """The served workload's query pool on the resident R-MAT 22 graph: every
    query's sorted rows against the oracle's digest (plain form), the batched
    counts and listed rows, and the served results in both modes."""
    import time
    g = rmat22
    with open(GOLDEN22) as f:
        gold = json.load(f)
    assert gold["graph"]["sha256"] == graph_digest(g)
    pool = gold["queries"]
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels, validate=True)
    Qs = []
    for q in pool:
        Q = m.query(q["k"], q["edges"], q["labels"]).restrict(0, 0, q["root_hi"])
        for u in range(1, q["k"]):
            Q.restrict(u, 0, q["window"])
        Qs.append(Q)
    for q, Q in zip(pool, Qs):
        rows, count = m.enumerate(Q)
        assert count == q["count"]
        digest = hashlib.sha256(np.ascontiguousarray(rows, dtype="<i4").tobytes()).hexdigest()
        assert digest == q["rows_sha256"]
    want = [q["count"] for q in pool]
    assert m.run_batch(Qs) == want
    counts, rows = m.run_batch(Qs, enumerate=True)
    assert counts == want
    for q, r in zip(pool, rows):
        a = np.ascontiguousarray(r, dtype="<i4").reshape(-1)
        assert hashlib.sha256(a.tobytes()).hexdigest() == q["rows_sha256"]
    gsm_lib.gsm_server_start(m.ctx, 2, 64)
    tickets = []
    for j in range(2 * len(Qs)):
        mode = gsm_lib.GSM_MODE_ENUMERATE if j % 3 == 0 else gsm_lib.GSM_MODE_COUNT
        tickets.append((gsm_lib.gsm_submit(m.ctx, Qs[j % len(Qs)].handle, mode),
                        j % len(Qs), mode))
    done = {}
    deadline = time.time() + 120
    while len(done) < len(tickets) and time.time() < deadline:
        for t, j, mode in tickets:
            if t not in done:
                r = gsm_lib.gsm_poll(m.ctx, t)
                if r is not None:
                    done[t] = (r, j, mode)
        time.sleep(0.001)
    gsm_lib.gsm_server_stop(m.ctx)
    assert len(done) == len(tickets)
    for r, j, mode in done.values():
        assert r["status"] == 0 and r["count"] == want[j]
        if mode == gsm_lib.GSM_MODE_ENUMERATE and want[j]:
            a = np.ascontiguousarray(r["rows"], dtype="<i4").reshape(-1)
            assert hashlib.sha256(a.tobytes()).hexdigest() == pool[j]["rows_sha256"]
    m.close()
