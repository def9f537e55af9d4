"""The batched form (gsm_run_batch): every count equals the single-query
path's and the oracle's, whatever the batch mix, launch configuration or
workspace size."""
import numpy as np
import pytest

import oracle
from paper_2003_01527_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rmat12b():
    n, rp, col = I.rmat(12, 16, *I.RMAT_ABC, seed=51)
    return I.make_graph(n, rp, col, I.zipf_labels(n, 16, 1.2, seed=52))


def mixed_queries(g, num, seed):
    """Random-walk queries of 3-10 vertices (tree + 2-4 extra edges, or
    induced), restricted to a root range when the oracle needs it."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < num:
        k = int(rng.integers(3, 11))
        q = I.random_walk_query(g, k, rng, (2, 4) if rng.random() < 0.7 else None)
        hi = g.n
        for _ in range(12):
            c, _, rc = oracle.match(g, q, enumerate=False, root_range=(0, hi), limit=200_000,
                                    node_budget=20_000_000)
            if rc == oracle.OK:
                break
            hi = max(1, hi // 4)
        else:
            continue
        out.append((q, hi, c))
    return out


def test_batch_counts_match_oracle_and_single_query(gsm_lib, cuda, rmat12b):
    m = gsm_lib.Matcher(device=0)
    m.load_graph(rmat12b.row_ptr, rmat12b.col, rmat12b.labels, validate=True)
    items = mixed_queries(rmat12b, 40, seed=53)
    # extra shapes: one vertex, one edge, an absent label, an empty restriction
    extra = [(I.query_from_edges(1, [], [2]), rmat12b.n),
             (I.query_from_edges(2, [(0, 1)], [0, 1]), rmat12b.n),
             (I.query_from_edges(3, [(0, 1), (1, 2)], [0, 99, 0]), rmat12b.n),
             (I.query_from_edges(3, [(0, 1), (1, 2)], [0, 0, 0]), 0)]
    for q, hi in extra:
        c, _, _ = oracle.match(rmat12b, q, enumerate=False, root_range=(0, hi))
        items.append((q, hi, c))
    Qs = [m.query(q.k, q.edges, q.labels).restrict(0, 0, hi) for q, hi, _ in items]
    want = [c for _, _, c in items]
    got = m.run_batch(Qs)
    assert got == want
    assert [m.count(Q) for Q in Qs] == want
    st = m.batch_stats()
    assert st["graph_launches"] >= 1 and st["overflowed"] == 0
    # a second, reordered batch reuses nothing but must give the same counts
    perm = np.random.default_rng(1).permutation(len(Qs))
    assert m.run_batch([Qs[i] for i in perm]) == [want[i] for i in perm]
    # same shape again: the captured graph is reused
    built = m.batch_stats()["graphs_built"]
    assert m.run_batch(Qs) == want
    assert m.batch_stats()["graphs_built"] == built
    m.close()


def test_batch_enumerate_rows_match_oracle(gsm_lib, cuda, rmat12b):
    """The batched form in enumerate mode: every query's rows equal the
    oracle's sorted rows and gsm_enumerate's, in host and in device memory,
    for uneven query sizes (including one-vertex queries, an absent label
    and an empty restriction)."""
    g = rmat12b
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels)
    items = mixed_queries(g, 30, seed=57)
    extra = [(I.query_from_edges(1, [], [2]), g.n),
             (I.query_from_edges(2, [(0, 1)], [0, 1]), g.n),
             (I.query_from_edges(3, [(0, 1), (1, 2)], [0, 99, 0]), g.n),
             (I.query_from_edges(3, [(0, 1), (1, 2)], [0, 0, 0]), 0)]
    for q, hi in extra:
        c, _, _ = oracle.match(g, q, enumerate=False, root_range=(0, hi))
        items.append((q, hi, c))
    Qs = [m.query(q.k, q.edges, q.labels).restrict(0, 0, hi) for q, hi, _ in items]
    want = [oracle.match(g, q, root_range=(0, hi))[1] for q, hi, _ in items]
    counts, rows = m.run_batch(Qs, enumerate=True)
    assert counts == [c for _, _, c in items]
    for w, r, (q, _, _) in zip(want, rows, items):
        assert np.array_equal(r.reshape(-1, q.k), w)
    # rows on the device, and a second (reordered) batch of the same shape
    perm = np.random.default_rng(2).permutation(len(Qs))
    counts2, rows2 = m.run_batch([Qs[i] for i in perm], enumerate=True, device=True)
    assert counts2 == [counts[i] for i in perm]
    for i, r in zip(perm, rows2):
        assert np.array_equal(r.cpu().numpy().reshape(-1, items[i][0].k), want[i])
    # counts only after listing: the count graph is another shape
    assert m.run_batch(Qs) == counts
    # the rows equal the single-query path's
    for Q, w in zip(Qs[:10], want[:10]):
        alone, _ = m.enumerate(Q)
        assert np.array_equal(alone, w)
    assert m.batch_stats()["overflowed"] == 0
    m.close()


def test_batch_enumerate_arena_overflow_falls_back(gsm_lib, cuda, rmat12b):
    g = rmat12b
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels)
    gsm_lib.gsm_batch_configure(m.ctx, 0, 0, 0, 1024)  # a tiny result arena
    items = [it for it in mixed_queries(g, 12, seed=58) if it[2] > 0]
    Qs = [m.query(q.k, q.edges, q.labels).restrict(0, 0, hi) for q, hi, _ in items]
    want = [oracle.match(g, q, root_range=(0, hi))[1] for q, hi, _ in items]
    counts, rows = m.run_batch(Qs, enumerate=True)
    assert counts == [c for _, _, c in items]
    assert m.batch_stats()["overflowed"] == (1 if sum(c * q.k for q, _, c in items) > 1024 else 0)
    for w, r, (q, _, _) in zip(want, rows, items):
        assert np.array_equal(r.reshape(-1, q.k), w)
    m.close()


def test_batch_autotune_and_configurations(gsm_lib, cuda, rmat12b):
    m = gsm_lib.Matcher(device=0)
    m.load_graph(rmat12b.row_ptr, rmat12b.col, rmat12b.labels)
    items = mixed_queries(rmat12b, 16, seed=54)
    Qs = [m.query(q.k, q.edges, q.labels).restrict(0, 0, hi) for q, hi, _ in items]
    want = [c for _, _, c in items]
    assert m.run_batch(Qs, autotune=True) == want
    st = m.batch_stats()
    assert st["tuned"] == 1 and st["graphs_built"] >= 6
    assert m.run_batch(Qs) == want  # the tuned configuration is reused
    m.close()


def test_batch_overflow_falls_back(gsm_lib, cuda, rmat12b):
    m = gsm_lib.Matcher(device=0)
    m.load_graph(rmat12b.row_ptr, rmat12b.col, rmat12b.labels)
    gsm_lib.gsm_batch_configure(m.ctx, 64, 256, 4096)
    items = mixed_queries(rmat12b, 8, seed=55)
    Qs = [m.query(q.k, q.edges, q.labels).restrict(0, 0, hi) for q, hi, _ in items]
    want = [c for _, _, c in items]
    assert m.run_batch(Qs) == want
    assert m.batch_stats()["overflowed"] == 1
    m.close()


def test_batch_unlabelled_shapes(gsm_lib, cuda):
    n, rp, col = I.rmat(10, 16, *I.RMAT_ABC, seed=56)
    g = I.make_graph(n, rp, col, np.zeros(n, np.int32))
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels)
    s = I.unlabelled_shapes()
    cases = [(s["triangle"], n), (s["clique4"], 300), (s["cycle5"], 6), (s["path6"], 2)]
    Qs = [m.query(q.k, q.edges).restrict(0, 0, hi) for q, hi in cases]
    want = [oracle.count(g, q, root_range=(0, hi)) for q, hi in cases]
    assert m.run_batch(Qs) == want
    m.close()


def test_batched_workload_full_size(gsm_lib, cuda):
    """The R-MAT scale-18 batched workload at full size, as the benchmark runs
    it: one batch of all 256 query slices against the oracle's stored counts,
    and the sorted rows of the non-empty slices against its stored digests."""
    import hashlib
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "rmat18_batched_slices.json")
    with open(path) as f:
        gold = json.load(f)
    g, _ = I.rmat_labelled_workload(scale=18, num_labels=16, zipf_s=1.2, num_queries=0, seed=4)
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col, g.labels):
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    assert h.hexdigest() == gold["graph"]["sha256"]
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels)
    Qs = [m.query(q["k"], q["edges"], q["labels"]).restrict(0, 0, q["root_hi"])
          for q in gold["queries"]]
    assert m.run_batch(Qs, autotune=True) == [q["count"] for q in gold["queries"]]
    assert m.batch_stats()["overflowed"] == 0
    for q, Q in zip(gold["queries"], Qs):
        if q["count"]:
            rows, count = m.enumerate(Q)
            assert count == q["count"]
            digest = hashlib.sha256(np.ascontiguousarray(rows, dtype="<i4").tobytes()).hexdigest()
            assert digest == q["rows_sha256"]
    # the whole batch in enumerate mode: every query's rows against the digests
    counts, rows = m.run_batch(Qs, enumerate=True, device=True)
    assert counts == [q["count"] for q in gold["queries"]]
    assert m.batch_stats()["overflowed"] == 0
    for q, r in zip(gold["queries"], rows):
        got = np.ascontiguousarray(r.cpu().numpy(), dtype="<i4").reshape(-1)
        assert hashlib.sha256(got.tobytes()).hexdigest() == q["rows_sha256"]
    m.close()
