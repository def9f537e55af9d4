"""Pins of the CPU oracle against things other than itself.

* exhaustive search over all injective maps (oracle/brute.py, pure Python) on
  hundreds of tiny seeded graphs;
* closed forms from the adjacency matrix (exact integers, scipy sparse):
  edges = nnz, ordered 3-paths = sum d(d-1), 3-stars = sum d(d-1)(d-2),
  triangles = tr(A^3), labelled triangles = tr(D_a A D_b A D_c A),
  4-cycles = tr(A^4) - 2 sum d^2 + nnz,
  5-cycles = tr(A^5) - 5 tr(A^3) - 5 sum_i (d_i - 2)(A^3)_ii,
  any k-vertex query in K_n = n!/(n-k)!, labelled K_n = prod_l n_l!/(n_l-k_l)!,
  and the labelled 4-cycle (0,1,0,2) as sum_{x != z} (A D1 A)_xz (A D2 A)_xz;
* invariants: slices of f(q_0) add up, the generating walk of a random-walk
  query is one of its embeddings, removing a query edge gives a superset;
* the candidate filter of Sec. 3.2: soundness against brute force and a
  hand-worked example;
* the independent k-clique counter (degree-ordered listing) that pins the
  full-size R-MAT 20 clique counts: C(n, k) in K_n, tr(A^3)/6, k! x cliques =
  the matcher's count of K_k (which brute force pins in turn).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import brute
from paper_2003_01527_gb300 import inputs as I


def adj(g):
    return sp.csr_matrix((np.ones(g.nnz, dtype=np.int64), g.col, g.row_ptr), shape=(g.n, g.n))


def tiny_cases(num, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(num):
        n = int(rng.integers(3, 9))
        p = float(rng.uniform(0.2, 0.9))
        pairs = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
        L = int(rng.integers(1, 4))
        g = I.graph_from_edges(n, pairs if pairs else [(0, 1)], rng.integers(0, L, n))
        k = int(rng.integers(1, 5 if n >= 5 else n + 1))
        # random connected query: a random tree plus random extra edges
        qe = {(int(rng.integers(0, v)), v) for v in range(1, k)}
        for a in range(k):
            for b in range(a + 1, k):
                if rng.random() < 0.3:
                    qe.add((a, b))
        q = I.query_from_edges(k, sorted(qe), rng.integers(0, L, k))
        out.append((g, q))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_dfs_equals_brute_force(oracle_lib, seed):
    for g, q in tiny_cases(50, seed):
        want = brute.embeddings(g, q)
        count, rows, rc = oracle.match(g, q)
        assert rc == oracle.OK
        assert count == len(want)
        assert [tuple(r) for r in rows.tolist()] == want


def test_brute_force_special_graphs(oracle_lib):
    # complete graph K5, 5-cycle, star, disjoint union of two triangles
    k5 = I.graph_from_edges(5, [(i, j) for i in range(5) for j in range(i + 1, 5)])
    c5 = I.graph_from_edges(5, [(i, (i + 1) % 5) for i in range(5)])
    star = I.graph_from_edges(6, [(0, i) for i in range(1, 6)])
    two_tri = I.graph_from_edges(6, [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5)])
    shapes = I.unlabelled_shapes()
    path3 = I.query_from_edges(3, [(0, 1), (1, 2)])
    for g in (k5, c5, star, two_tri):
        for q in list(shapes.values())[:3] + [path3]:
            if q.k > g.n:
                continue
            assert oracle.count(g, q) == len(brute.embeddings(g, q))
    assert oracle.count(star, path3) == 5 * 4 + 5 * 0  # centre in the middle only
    assert oracle.count(two_tri, shapes["triangle"]) == 12
    assert oracle.count(c5, shapes["cycle5"]) == 10


def test_complete_graph_closed_forms(oracle_lib):
    for n in (5, 6, 7):
        kn = I.graph_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
        for name, q in I.unlabelled_shapes().items():
            if q.k <= n:
                assert oracle.count(kn, q) == math.perm(n, q.k), name
    # labelled K_7 with 3 vertices of label 0, 4 of label 1
    lab = [0, 0, 0, 1, 1, 1, 1]
    k7 = I.graph_from_edges(7, [(i, j) for i in range(7) for j in range(i + 1, 7)], lab)
    q = I.query_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)], [0, 1, 0, 1])
    assert oracle.count(k7, q) == math.perm(3, 2) * math.perm(4, 2)
    q = I.query_from_edges(4, [(0, 1), (1, 2), (2, 3)], [0, 0, 0, 0])
    assert oracle.count(k7, q) == 0


@pytest.fixture(scope="module")
def small_rmat():
    n, rp, col = I.rmat(9, 8, *I.RMAT_ABC, seed=11)
    return I.make_graph(n, rp, col, I.zipf_labels(n, 3, 1.0, seed=12))


def test_unlabelled_closed_forms(oracle_lib, small_rmat):
    g = I.make_graph(small_rmat.n, small_rmat.row_ptr, small_rmat.col,
                     np.zeros(small_rmat.n, dtype=np.int32))
    A = adj(g)
    d = np.asarray(A.sum(axis=1)).ravel().astype(object)
    A2 = A @ A
    A3 = A2 @ A
    tr3 = int(A3.diagonal().sum())
    tr4 = int((A2.multiply(A2.T)).sum())
    tr5 = int((A3.multiply(A2.T)).sum())
    nnz = g.nnz
    edge = I.query_from_edges(2, [(0, 1)])
    path3 = I.query_from_edges(3, [(0, 1), (1, 2)])
    star3 = I.query_from_edges(4, [(0, 1), (0, 2), (0, 3)])
    s = I.unlabelled_shapes()
    assert oracle.count(g, edge) == nnz
    assert oracle.count(g, path3) == int(sum(x * (x - 1) for x in d))
    assert oracle.count(g, star3) == int(sum(x * (x - 1) * (x - 2) for x in d))
    assert oracle.count(g, s["triangle"]) == tr3
    assert oracle.count(g, I.query_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)])) == \
        tr4 - 2 * int(sum(x * x for x in d)) + nnz
    a3d = A3.diagonal().astype(object)
    assert oracle.count(g, s["cycle5"]) == \
        tr5 - 5 * tr3 - 5 * int(sum((d[i] - 2) * a3d[i] for i in range(g.n)))


def test_clique_counter_closed_forms(oracle_lib):
    for n in (3, 4, 6, 9, 12):
        g = I.graph_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
        for k in range(3, min(n, 8) + 1):
            assert oracle.cliques(g, k) == math.comb(n, k)
    # K_{3,3} and a 6-cycle have no triangle; two disjoint K4 have 8 triangles, 2 K4
    k33 = I.graph_from_edges(6, [(i, j) for i in range(3) for j in range(3, 6)])
    c6 = I.graph_from_edges(6, [(i, (i + 1) % 6) for i in range(6)])
    two_k4 = I.graph_from_edges(8, [(a + i, a + j) for a in (0, 4) for i in range(4)
                                    for j in range(i + 1, 4)])
    assert oracle.cliques(k33, 3) == 0 and oracle.cliques(c6, 3) == 0
    assert oracle.cliques(two_k4, 3) == 8 and oracle.cliques(two_k4, 4) == 2
    assert oracle.cliques(two_k4, 5) == 0


def test_clique_counter_against_trace_and_matcher(oracle_lib, small_rmat):
    g = I.make_graph(small_rmat.n, small_rmat.row_ptr, small_rmat.col,
                     np.zeros(small_rmat.n, dtype=np.int32))
    A = adj(g)
    assert 6 * oracle.cliques(g, 3) == int((A @ A @ A).diagonal().sum())
    rng = np.random.default_rng(21)
    for t in range(12):
        n = int(rng.integers(6, 40))
        m = int(rng.integers(n, n * (n - 1) // 2 + 1))
        _, rp, col = I.erdos_renyi(n, m, seed=100 + t)
        h = I.make_graph(n, rp, col, np.zeros(n, dtype=np.int32))
        for k in (3, 4, 5):
            kk = I.query_from_edges(k, [(i, j) for i in range(k) for j in range(i + 1, k)])
            assert oracle.count(h, kk) == math.factorial(k) * oracle.cliques(h, k)
    for k in (3, 4):
        kk = I.query_from_edges(k, [(i, j) for i in range(k) for j in range(i + 1, k)])
        assert oracle.count(g, kk) == math.factorial(k) * oracle.cliques(g, k)


def test_labelled_triangle_closed_form(oracle_lib, small_rmat):
    g = small_rmat
    A = adj(g)
    D = [sp.diags((g.labels == l).astype(np.int64), dtype=np.int64) for l in range(3)]
    for (a, b, c) in [(0, 0, 0), (0, 1, 2), (1, 1, 0), (2, 0, 1)]:
        want = int((D[a] @ A @ D[b] @ A @ D[c] @ A).diagonal().sum())
        q = I.query_from_edges(3, [(0, 1), (1, 2), (0, 2)], [a, b, c])
        assert oracle.count(g, q) == want


def test_tiny_er_4cycle_closed_form(oracle_lib):
    g, (q,) = I.tiny_er_workload()
    A = adj(g)
    D1 = sp.diags((g.labels == 1).astype(np.int64), dtype=np.int64)
    D2 = sp.diags((g.labels == 2).astype(np.int64), dtype=np.int64)
    M1 = (A @ D1 @ A).tocsr()
    M2 = (A @ D2 @ A).tocsr()
    P = M1.multiply(M2).tocoo()
    zero = g.labels == 0
    want = sum(int(v) for x, z, v in zip(P.row, P.col, P.data) if x != z and zero[x] and zero[z])
    count, rows, _ = oracle.match(g, q)
    assert count == want
    assert count == rows.shape[0]


def test_root_slices_add_up(oracle_lib, small_rmat):
    q = I.query_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)], [0, 0, 1, 0])
    total, rows, _ = oracle.match(small_rmat, q)
    cuts = [0, 37, 100, 101, 300, small_rmat.n]
    parts = [oracle.match(small_rmat, q, root_range=(a, b))[1] for a, b in zip(cuts, cuts[1:])]
    joined = np.concatenate(parts)
    assert joined.shape[0] == total
    assert np.array_equal(joined, rows)  # a slice of f(q_0) is a block of the sorted result
    assert all(((p[:, 0] >= a) & (p[:, 0] < b)).all() for p, a, b in zip(parts, cuts, cuts[1:]))


def test_vertex_ranges_filter_brute_force(oracle_lib):
    """Ranges on any query vertices keep exactly the brute-force embeddings
    that fall inside them."""
    rng = np.random.default_rng(77)
    for g, q in tiny_cases(60, 300):
        ranges = {}
        for u in range(q.k):
            if rng.random() < 0.5:
                a = int(rng.integers(0, g.n))
                ranges[u] = (a, int(rng.integers(a, g.n + 1)))
        want = [f for f in brute.embeddings(g, q)
                if all(lo <= f[u] < hi for u, (lo, hi) in ranges.items())]
        count, rows, rc = oracle.match(g, q, ranges=ranges)
        assert rc == oracle.OK and count == len(want)
        assert [tuple(r) for r in rows.tolist()] == want


def test_generating_walk_is_an_embedding(oracle_lib, small_rmat):
    rng = np.random.default_rng(5)
    for _ in range(10):
        q = I.random_walk_query(small_rmat, int(rng.integers(3, 6)), rng)
        lo = int(q.walk[0])
        _, rows, _ = oracle.match(small_rmat, q, root_range=(lo, lo + 1))
        assert any(np.array_equal(r, q.walk) for r in rows)


def test_removing_an_edge_gives_a_superset(oracle_lib, small_rmat):
    q = I.query_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)], [0, 0, 0, 0])
    qq = I.query_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)], [0, 0, 0, 0])
    _, a, _ = oracle.match(small_rmat, q)
    _, b, _ = oracle.match(small_rmat, qq)
    sa = {tuple(r) for r in a.tolist()}
    sb = {tuple(r) for r in b.tolist()}
    assert sa <= sb and len(sb) > len(sa)


def test_limit_and_budget_give_up(oracle_lib, small_rmat):
    q = I.query_from_edges(3, [(0, 1), (1, 2)])
    full = oracle.count(small_rmat, q)
    c, _, rc = oracle.match(small_rmat, q, enumerate=False, limit=full)
    assert rc == oracle.OK and c == full
    _, _, rc = oracle.match(small_rmat, q, enumerate=False, limit=full - 1)
    assert rc == oracle.LIMIT
    _, _, rc = oracle.match(small_rmat, q, enumerate=False, node_budget=10)
    assert rc == oracle.BUDGET


def test_truncated_enumeration(oracle_lib, small_rmat):
    q = I.query_from_edges(3, [(0, 1), (1, 2), (0, 2)])
    count, rows, _ = oracle.match(small_rmat, q)
    c2, first, rc = oracle.match(small_rmat, q, cap_rows=5)
    assert rc == oracle.TRUNCATED and c2 == count
    assert np.array_equal(first, rows[:5])


def test_thread_count_does_not_change_result(oracle_lib, small_rmat):
    q = I.query_from_edges(4, [(0, 1), (1, 2), (2, 3)], [0, 1, 0, 0])
    _, a, _ = oracle.match(small_rmat, q, nthreads=1)
    _, b, _ = oracle.match(small_rmat, q, nthreads=4)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- filter


@pytest.mark.parametrize("seed", range(3))
def test_candidates_are_sound(oracle_lib, seed):
    """Every vertex used by an embedding passes the filter of its query vertex."""
    for g, q in tiny_cases(40, 100 + seed):
        c = oracle.candidates(g, q)
        for f in brute.embeddings(g, q):
            for u, v in enumerate(f):
                assert c[u, v] == 1


def test_candidates_hand_example(oracle_lib):
    # v0 (label 0) has neighbours v1, v2 (label 1) and v3 (label 2); v4 (label 0)
    # has neighbours v1 (1), v3 (2).
    g = I.graph_from_edges(5, [(0, 1), (0, 2), (0, 3), (4, 1), (4, 3)], [0, 1, 1, 2, 0])
    # query: centre u0 (label 0) with two label-1 neighbours
    q = I.query_from_edges(3, [(0, 1), (0, 2)], [0, 1, 1])
    c = oracle.candidates(g, q)
    assert c[0].tolist() == [1, 0, 0, 0, 0]  # v4 has only one label-1 neighbour
    assert c[1].tolist() == [0, 1, 1, 0, 0]  # label 1, degree >= 1, a label-0 neighbour
    # degree test: a label-1 leaf query neighbour of two label-0 vertices
    q2 = I.query_from_edges(3, [(0, 1), (1, 2)], [0, 1, 0])
    c2 = oracle.candidates(g, q2)
    assert c2[1].tolist() == [0, 1, 0, 0, 0]  # v2 has degree 1 < 2
    assert c2[0].tolist() == [1, 0, 0, 0, 1]


@pytest.mark.parametrize("seed", range(2))
def test_refinement_is_sound_and_monotone(oracle_lib, seed):
    """Refined candidate sets only shrink, and keep every vertex that some
    embedding uses (brute force)."""
    for g, q in tiny_cases(40, 400 + seed):
        c0 = oracle.candidates(g, q)
        c1 = oracle.refine(g, q, c0, 1)
        c3 = oracle.refine(g, q, c0, 3)
        assert (c1 <= c0).all() and (c3 <= c1).all()
        for f in brute.embeddings(g, q):
            for u, v in enumerate(f):
                assert c3[u, v] == 1


def test_refinement_hand_example(oracle_lib):
    # query: a label-0 vertex joined to a label-1 vertex that has a label-2
    # neighbour.  Data: v0(0)-v1(1), v1-v2(2), and v3(0)-v4(1) where v4 has
    # a second neighbour v5 of label 0 but no label-2 neighbour.
    g = I.graph_from_edges(6, [(0, 1), (1, 2), (3, 4), (4, 5)], [0, 1, 2, 0, 1, 0])
    q = I.query_from_edges(3, [(0, 1), (1, 2)], [0, 1, 2])
    c0 = oracle.candidates(g, q)
    assert c0[1].tolist() == [0, 1, 0, 0, 0, 0]  # v4 lacks a label-2 neighbour
    assert c0[0].tolist() == [1, 0, 0, 1, 0, 1]  # the first pass keeps v3, v5
    c1 = oracle.refine(g, q, c0, 1)
    assert c1[0].tolist() == [1, 0, 0, 0, 0, 0]  # v3, v5 have no candidate neighbour for u1
    assert c1[1].tolist() == [0, 1, 0, 0, 0, 0]


def test_validity_checks(oracle_lib):
    ok = I.graph_from_edges(3, [(0, 1), (1, 2)])
    assert oracle.validate_graph(ok) == oracle.OK
    bad_loop = I.Graph(2, np.array([0, 2, 3], np.int32), np.array([0, 1, 0], np.int32),
                       np.zeros(2, np.int32))
    assert oracle.validate_graph(bad_loop) == oracle.INVALID_GRAPH
    asym = I.Graph(3, np.array([0, 1, 1, 1], np.int32), np.array([1], np.int32),
                   np.zeros(3, np.int32))
    assert oracle.validate_graph(asym) == oracle.INVALID_GRAPH
    unsorted = I.Graph(3, np.array([0, 2, 3, 4], np.int32), np.array([2, 1, 0, 0], np.int32),
                       np.zeros(3, np.int32))
    assert oracle.validate_graph(unsorted) == oracle.INVALID_GRAPH
    disconnected = I.Query(4, np.array([[0, 1], [2, 3]], np.int32), np.zeros(4, np.int32))
    assert oracle.validate_query(disconnected) == oracle.INVALID_QUERY
    dup = I.Query(3, np.array([[0, 1], [1, 0], [1, 2]], np.int32), np.zeros(3, np.int32))
    assert oracle.validate_query(dup) == oracle.INVALID_QUERY
