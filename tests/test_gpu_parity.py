"""GPU parity: libgsm (through its C ABI) against the CPU oracle.

Results are integers, so the bar is bit-exact: the same count and the same
sorted rows.  Small cases compare every row; the full-size power-law workload
compares the count and the SHA-256 of the sorted rows against values the
oracle wrote (tests/golden/make_workloads.py).
"""
import hashlib
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2003_01527_gb300 import inputs as I

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def M(gsm_lib, cuda, oracle_lib):
    m = gsm_lib.Matcher(device=0)
    yield m
    m.close()


def load(M, g, validate=True):
    M.load_graph(g.row_ptr, g.col, g.labels, validate=validate)


def gpu_rows(M, q, **restrict):
    Q = M.query(q.k, q.edges, q.labels)
    for u, (lo, hi) in restrict.items():
        Q.restrict(int(u[1:]), lo, hi)
    rows, count = M.enumerate(Q)
    c2 = M.count(Q)
    assert c2 == count
    return rows, count


def assert_parity(M, g, q, root_range=None):
    want_count, want_rows, rc = oracle.match(g, q, root_range=root_range)
    assert rc == oracle.OK
    kw = {} if root_range is None else {"u0": root_range}
    rows, count = gpu_rows(M, q, **kw)
    assert count == want_count
    assert rows.shape == want_rows.shape
    assert np.array_equal(rows, want_rows)
    return count


def test_tiny_er_4cycle(M):
    g, (q,) = I.tiny_er_workload()
    load(M, g)
    assert assert_parity(M, g, q) > 0


@pytest.fixture(scope="module")
def rmat12():
    n, rp, col = I.rmat(12, 16, *I.RMAT_ABC, seed=21)
    return I.make_graph(n, rp, col, I.zipf_labels(n, 8, 1.0, seed=22))


def selective_walk_queries(g, num, kmin, kmax, seed, limit=300_000, non_tree=None):
    """Random-walk queries whose full result the oracle lists quickly (the
    oracle decides which ones qualify)."""
    rng = np.random.default_rng(seed)
    out = []
    tries = 0
    while len(out) < num and tries < 40 * num:
        tries += 1
        q = I.random_walk_query(g, int(rng.integers(kmin, kmax + 1)), rng, non_tree)
        c, _, rc = oracle.match(g, q, enumerate=False, limit=limit, node_budget=50_000_000)
        if rc == oracle.OK:
            out.append(q)
    return out


def test_labelled_rmat_random_walk_queries(M, rmat12):
    load(M, rmat12)
    qs = selective_walk_queries(rmat12, 24, 3, 7, seed=23)
    assert len(qs) >= 12
    total = 0
    for q in qs:
        total += assert_parity(M, rmat12, q)
        assert M.last_run_stats()["k"] == q.k
    assert total > 0


def test_labelled_rmat_tree_plus_nontree_queries(M, rmat12):
    load(M, rmat12)
    for q in selective_walk_queries(rmat12, 12, 3, 8, seed=24, non_tree=(2, 4)):
        assert_parity(M, rmat12, q)


def test_generating_walk_is_found(M, rmat12):
    load(M, rmat12)
    rng = np.random.default_rng(25)
    for _ in range(6):
        q = I.random_walk_query(rmat12, int(rng.integers(3, 7)), rng)
        v0 = int(q.walk[0])
        rows, _ = gpu_rows(M, q, u0=(v0, v0 + 1))
        assert any(np.array_equal(r, q.walk) for r in rows)


@pytest.fixture(scope="module")
def rmat10u():
    n, rp, col = I.rmat(10, 16, *I.RMAT_ABC, seed=31)
    return I.make_graph(n, rp, col, np.zeros(n, np.int32))


def test_unlabelled_shapes(M, rmat10u):
    load(M, rmat10u)
    s = I.unlabelled_shapes()
    assert_parity(M, rmat10u, s["triangle"])
    assert_parity(M, rmat10u, s["clique4"], root_range=(0, 300))
    assert_parity(M, rmat10u, s["cycle5"], root_range=(0, 6))
    # the 6-path from two roots has 1.2e9 embeddings: its other vertices stay
    # below id 256
    q = s["path6"]
    window = {u: (0, 256) for u in range(1, 6)}
    want_count, want_rows, _ = oracle.match(rmat10u, q, root_range=(0, 2), ranges=window)
    rows, count = gpu_rows(M, q, u0=(0, 2), **{f"u{u}": r for u, r in window.items()})
    assert count == want_count > 0 and np.array_equal(rows, want_rows)


def test_unlabelled_counts_match_closed_form(M, rmat10u):
    import scipy.sparse as sp
    load(M, rmat10u)
    A = sp.csr_matrix((np.ones(rmat10u.nnz, np.int64), rmat10u.col, rmat10u.row_ptr),
                      shape=(rmat10u.n, rmat10u.n))
    tr3 = int((A @ A).multiply(A).sum())
    d = rmat10u.degrees().astype(object)
    Q = M.query(3, [(0, 1), (1, 2), (0, 2)])
    assert M.count(Q) == tr3
    Q = M.query(3, [(0, 1), (1, 2)])
    assert M.count(Q) == int(sum(x * (x - 1) for x in d))
    Q = M.query(2, [(0, 1)])
    assert M.count(Q) == rmat10u.nnz


def test_candidate_bitmaps_match_oracle(M, rmat12, gsm_lib):
    load(M, rmat12)
    rng = np.random.default_rng(26)
    for _ in range(10):
        q = I.random_walk_query(rmat12, int(rng.integers(2, 9)), rng)
        Q = M.query(q.k, q.edges, q.labels)
        bm, sizes = M.candidates(Q)
        got = gsm_lib.unpack_bitmaps(bm, rmat12.n)
        want = oracle.candidates(rmat12, q)
        assert np.array_equal(got, want)
        assert sizes.tolist() == want.sum(axis=1).tolist()


@pytest.mark.parametrize("labels", [2, 63, 64, 65, 300])
def test_candidate_bitmaps_by_label_count(M, gsm_lib, labels):
    """Up to 64 labels the filter reads the graph's neighbour label count
    table, above that it counts from the rows: both give the oracle's
    candidate sets, for queries with several same-label neighbours."""
    n, rp, col = I.rmat(11, 16, *I.RMAT_ABC, seed=27)
    g = I.make_graph(n, rp, col, I.zipf_labels(n, labels, 0.6, seed=28))
    load(M, g)
    rng = np.random.default_rng(29)
    for _ in range(6):
        q = I.random_walk_query(g, int(rng.integers(3, 9)), rng)
        lab = q.labels.copy()
        lab[1:3] = lab[0]  # repeated labels: requirements above one
        q = I.query_from_edges(q.k, q.edges, lab)
        bm, sizes = M.candidates(M.query(q.k, q.edges, q.labels))
        want = oracle.candidates(g, q)
        assert np.array_equal(gsm_lib.unpack_bitmaps(bm, g.n), want)
        assert sizes.tolist() == want.sum(axis=1).tolist()
        _, _, rc = oracle.match(g, q, enumerate=False, root_range=(0, 256), limit=200_000,
                                node_budget=20_000_000)
        if rc == oracle.OK:
            assert_parity(M, g, q, root_range=(0, 256))


def test_results_do_not_depend_on_chunking_or_block_size(gsm_lib, rmat12):
    qs = selective_walk_queries(rmat12, 4, 4, 6, seed=27)
    ref = None
    for opts in ({}, {"chunk_rows": 1}, {"chunk_rows": 7}, {"block_size": 128},
                 {"block_size": 1024}, {"block_size": 512, "chunk_rows": 33},
                 {"mem_budget_bytes": 1 << 21}, {"two_pass": True},
                 {"two_pass": True, "block_size": 1024, "chunk_rows": 33}):
        m = gsm_lib.Matcher(device=0, **opts)
        load(m, rmat12, validate=False)
        out = [m.enumerate(m.query(q.k, q.edges, q.labels)) for q in qs]
        m.close()
        if ref is None:
            ref = out
            for q, (rows, count) in zip(qs, out):
                want_count, want_rows, _ = oracle.match(rmat12, q)
                assert count == want_count and np.array_equal(rows, want_rows)
        else:
            for (a, ca), (b, cb) in zip(ref, out):
                assert ca == cb and np.array_equal(a, b), opts


@pytest.mark.parametrize("hub_bytes", [-1, 64 << 10, 0])
def test_results_do_not_depend_on_hub_bitmaps(gsm_lib, rmat12, rmat10u, hub_bytes):
    """Non-tree edges checked on hub adjacency bitmaps (all hubs, a budget for
    a few, or none: every check a binary search) give the oracle's rows."""
    m = gsm_lib.Matcher(device=0, hub_bitmap_bytes=hub_bytes)
    walks = [(q, rmat12.n, None) for q in
             selective_walk_queries(rmat12, 10, 3, 8, seed=41, non_tree=(2, 4))]
    for g, items in ((rmat12, walks),
                     (rmat10u, [(q, hi, None) for q, hi in
                                ((I.unlabelled_shapes()["clique4"], rmat10u.n),
                                 (I.unlabelled_shapes()["cycle5"], 6),
                                 (I.query_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0),
                                                         (0, 2)]), 256))])):
        m.load_graph(g.row_ptr, g.col, g.labels)
        for q, hi, _ in items:
            want_count, want_rows, _ = oracle.match(g, q, root_range=(0, hi))
            rows, count = m.enumerate(m.query(q.k, q.edges, q.labels).restrict(0, 0, hi))
            assert count == want_count and np.array_equal(rows, want_rows)
    m.close()


def test_chunking_exercised_under_small_budget(gsm_lib, rmat10u):
    m = gsm_lib.Matcher(device=0, mem_budget_bytes=1 << 20, chunk_rows=500)
    load(m, rmat10u, validate=False)
    q = I.unlabelled_shapes()["cycle5"]
    Q = m.query(q.k, q.edges, q.labels).restrict(0, 0, 40)
    rows, count = m.enumerate(Q)
    stats = m.last_run_stats()
    want_count, want_rows, _ = oracle.match(rmat10u, q, root_range=(0, 40))
    assert count == want_count and np.array_equal(rows, want_rows)
    assert stats["chunks"] > 3
    assert stats["peak_bytes"] <= 1 << 20
    m.close()


def test_budget_error_when_one_row_cannot_fit(gsm_lib, rmat10u):
    m = gsm_lib.Matcher(device=0, mem_budget_bytes=4096)
    load(m, rmat10u, validate=False)
    Q = m.query(3, [(0, 1), (1, 2)])
    with pytest.raises(gsm_lib.GsmError) as ei:
        m.count(Q)
    assert ei.value.status == gsm_lib.GSM_ERR_BUDGET
    m.close()


def test_long_path_and_cycle_queries_k16(M):
    cyc = I.graph_from_edges(20, [(i, (i + 1) % 20) for i in range(20)])
    load(M, cyc)
    path16 = I.query_from_edges(16, [(i, i + 1) for i in range(15)])
    assert M.count(M.query(16, path16.edges)) == 40
    assert_parity(M, cyc, path16)
    c16 = I.graph_from_edges(16, [(i, (i + 1) % 16) for i in range(16)])
    load(M, c16)
    q = I.query_from_edges(16, [(i, (i + 1) % 16) for i in range(16)])
    assert_parity(M, c16, q)
    assert M.count(M.query(16, q.edges)) == 32


def test_complete_graph_counts(M):
    n = 9
    kn = I.graph_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    load(M, kn)
    for name, q in I.unlabelled_shapes().items():
        assert M.count(M.query(q.k, q.edges)) == math.perm(n, q.k), name
    assert M.count(M.query(7, [(i, j) for i in range(7) for j in range(i + 1, 7)])) == \
        math.perm(9, 7)


def test_edge_cases(M, rmat12, gsm_lib):
    load(M, rmat12)
    # k = 1: every vertex with the label, ascending
    rows, count = M.enumerate(M.query(1, [], [3]))
    assert count == int((rmat12.labels == 3).sum())
    assert np.array_equal(rows[:, 0], np.nonzero(rmat12.labels == 3)[0])
    # a label absent from G
    assert M.count(M.query(2, [(0, 1)], [0, 99])) == 0
    # empty restriction
    assert M.count(M.query(2, [(0, 1)]).restrict(1, 5, 5)) == 0
    # truncated enumeration returns the first rows in order
    q = I.query_from_edges(3, [(0, 1), (1, 2)], [0, 1, 0])
    want_count, want_rows, _ = oracle.match(rmat12, q, root_range=(0, 200))
    Q = M.query(q.k, q.edges, q.labels).restrict(0, 0, 200)
    buf = np.zeros((10, 3), np.int32)
    count, st = gsm_lib.gsm_enumerate(M.ctx, Q.handle, buf, 10, 0)
    assert st == gsm_lib.GSM_ERR_TRUNCATED and count == want_count
    assert np.array_equal(buf, want_rows[:10])
    # rows of the last result can be fetched afterwards
    tail = np.zeros((5, 3), np.int32)
    gsm_lib.gsm_last_rows(M.ctx, tail, count - 5, 5, 0)
    assert np.array_equal(tail, want_rows[-5:])
    with pytest.raises(gsm_lib.GsmError):
        gsm_lib.gsm_last_rows(M.ctx, tail, count - 2, 5, 0)


def test_device_output_and_device_graph(M, cuda, rmat12):
    torch = cuda
    t = {k: torch.from_numpy(getattr(rmat12, k)).cuda() for k in ("row_ptr", "col", "labels")}
    M.load_graph(t["row_ptr"], t["col"], t["labels"], validate=True)
    q = I.query_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)], [0, 1, 0, 1])
    want_count, want_rows, _ = oracle.match(rmat12, q)
    out = torch.zeros(want_count * 4 + 8, dtype=torch.int32, device="cuda")
    _, count = M.enumerate(M.query(q.k, q.edges, q.labels), out=out)
    torch.cuda.synchronize()
    assert count == want_count
    assert np.array_equal(out[:count * 4].view(-1, 4).cpu().numpy(), want_rows)


def test_empty_and_edgeless_graphs(M):
    g0 = I.Graph(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    M.load_graph(g0.row_ptr, g0.col, g0.labels, validate=True)
    assert M.count(M.query(2, [(0, 1)])) == 0
    assert M.count(M.query(1, [])) == 0
    g1 = I.Graph(5, np.zeros(6, np.int32), np.zeros(0, np.int32), np.arange(5, dtype=np.int32))
    M.load_graph(g1.row_ptr, g1.col, g1.labels, validate=True)
    assert M.count(M.query(1, [], [2])) == 1
    assert M.count(M.query(2, [(0, 1)], [1, 2])) == 0


def test_invalid_graphs_rejected(M, gsm_lib):
    bad = {
        "self-loop": (np.array([0, 2, 3], np.int32), np.array([0, 1, 0], np.int32)),
        "asymmetric": (np.array([0, 1, 1, 1], np.int32), np.array([1], np.int32)),
        "unsorted": (np.array([0, 2, 3, 4], np.int32), np.array([2, 1, 0, 0], np.int32)),
        "duplicate": (np.array([0, 2, 4], np.int32), np.array([1, 1, 0, 0], np.int32)),
        "out of range": (np.array([0, 1, 2], np.int32), np.array([1, 7], np.int32)),
    }
    for name, (rp, col) in bad.items():
        with pytest.raises(gsm_lib.GsmError) as ei:
            M.load_graph(rp, col, None, validate=True)
        assert ei.value.status == gsm_lib.GSM_ERR_INVALID_GRAPH, name
    with pytest.raises(gsm_lib.GsmError) as ei:  # row_ptr is always checked
        M.load_graph(np.array([0, 3, 1], np.int32), np.array([1, 0, 0], np.int32), None)
    assert ei.value.status == gsm_lib.GSM_ERR_INVALID_GRAPH
    with pytest.raises(gsm_lib.GsmError) as ei:
        M.count(M.query(2, [(0, 1)]))
    assert ei.value.status == gsm_lib.GSM_ERR_NO_GRAPH


def _golden(name):
    path = os.path.join(HERE, "golden", name)
    with open(path) as f:
        return json.load(f)


def _digest(g):
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col, g.labels):
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    return h.hexdigest()


def test_power_law_workload_full_size(M):
    """The R-MAT scale-16 labelled workload at full size, in the launch
    configuration the benchmark times: every query's root slice, count and
    SHA-256 of the sorted rows against the oracle's stored values."""
    gold = _golden("rmat16_labelled_slices.json")
    g, _ = I.rmat_labelled_workload(scale=16, num_labels=8, zipf_s=1.0, num_queries=0, seed=2)
    assert _digest(g) == gold["graph"]["sha256"], "generator output differs from the stored one"
    load(M, g, validate=False)
    nonzero = 0
    for item in gold["queries"]:
        Q = M.query(item["k"], item["edges"], item["labels"]).restrict(0, 0, item["root_hi"])
        rows, count = M.enumerate(Q)
        assert count == item["count"]
        digest = hashlib.sha256(np.ascontiguousarray(rows, dtype="<i4").tobytes()).hexdigest()
        assert digest == item["rows_sha256"]
        nonzero += count > 0
    assert nonzero >= 10


def test_refined_candidates_match_oracle_and_results_do_not_change(gsm_lib, rmat12):
    rng = np.random.default_rng(28)
    qs = [I.random_walk_query(rmat12, int(rng.integers(3, 9)), rng) for _ in range(8)]
    sel = selective_walk_queries(rmat12, 4, 4, 7, seed=29)
    base = {}
    for rounds in (0, 1, 2):
        m = gsm_lib.Matcher(device=0, filter_rounds=rounds)
        load(m, rmat12, validate=False)
        for j, q in enumerate(qs):
            bm, sizes = m.candidates(m.query(q.k, q.edges, q.labels))
            got = gsm_lib.unpack_bitmaps(bm, rmat12.n)
            want = oracle.refine(rmat12, q, oracle.candidates(rmat12, q), rounds)
            assert np.array_equal(got, want), (rounds, j)
            assert sizes.tolist() == want.sum(axis=1).tolist()
        for j, q in enumerate(sel):
            rows, count = m.enumerate(m.query(q.k, q.edges, q.labels))
            if rounds == 0:
                base[j] = (count, rows)
            else:
                assert count == base[j][0] and np.array_equal(rows, base[j][1])
        m.close()


def test_sorted_prefix_ranks_across_pieces(gsm_lib):
    """Slice q9 of the R-MAT 16 workload (matching order 0, 1, 3, 4, 2, 5):
    the last level writes the rank of the sorted prefix (query vertices 0, 1)
    into the sort keys, continued across the pieces its input comes in.
    Under budgets that split the levels into more and more pieces, and with
    small launch chunks, the rows still equal the oracle's stored digest."""
    gold = _golden("rmat16_labelled_slices.json")
    g, _ = I.rmat_labelled_workload(scale=16, num_labels=8, zipf_s=1.0, num_queries=0, seed=2)
    item = gold["queries"][9]
    for budget, chunk in ((0, 0), (96 << 20, 0), (48 << 20, 100_000)):
        m = gsm_lib.Matcher(device=0, mem_budget_bytes=budget, chunk_rows=chunk)
        m.load_graph(g.row_ptr, g.col, g.labels)
        Q = m.query(item["k"], item["edges"], item["labels"]).restrict(0, 0, item["root_hi"])
        rows, count = m.enumerate(Q)
        st = m.last_run_stats()
        assert st["order"][:2] == [0, 1] and st["order"] != list(range(item["k"]))
        assert count == item["count"]
        digest = hashlib.sha256(np.ascontiguousarray(rows, dtype="<i4").tobytes()).hexdigest()
        assert digest == item["rows_sha256"], (budget, chunk)
        m.close()
