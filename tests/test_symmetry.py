"""Symmetry breaking for distinct-subgraph counts (Sec. 3.1 node-ID ordering
constraints), host only: |Aut(Q)| against brute force over all vertex
permutations, and the constraints against the oracle's full embedding lists:
every orbit {f o sigma : sigma in Aut(Q)} of embeddings must keep exactly one
member."""
import itertools

import numpy as np

from paper_2003_01527_gb300 import inputs as I


def brute_automorphisms(k, edges, labels):
    es = {(a, b) for a, b in edges} | {(b, a) for a, b in edges}
    out = []
    for p in itertools.permutations(range(k)):
        if all(labels[p[u]] == labels[u] for u in range(k)) and \
                all((p[a], p[b]) in es for a, b in es):
            out.append(p)
    return out


def random_query(rng, k, num_labels):
    edges = {(int(rng.integers(0, v)), v) for v in range(1, k)}  # spanning tree
    for a, b in itertools.combinations(range(k), 2):
        if rng.random() < 0.35:
            edges.add((a, b))
    labels = rng.integers(0, num_labels, k).astype(np.int32)
    return sorted(edges), labels


def satisfies(row, pairs):
    return all(row[u] < row[v] for u, v in pairs)


def test_automorphism_counts_match_brute_force(gsm_lib):
    rng = np.random.default_rng(81)
    for _ in range(300):
        k = int(rng.integers(1, 8))
        edges, labels = random_query(rng, k, int(rng.integers(1, 4)))
        aut, pairs = gsm_lib.gsm_query_symmetry(k, edges, labels)
        assert aut == len(brute_automorphisms(k, edges, labels.tolist()))
        assert len(pairs) <= k * (k - 1) // 2
        # a query without symmetry needs no constraint
        assert (aut == 1) == (len(pairs) == 0)


def test_known_groups(gsm_lib):
    kq = lambda k: [(a, b) for a, b in itertools.combinations(range(k), 2)]
    assert gsm_lib.gsm_query_symmetry(4, kq(4))[0] == 24
    assert gsm_lib.gsm_query_symmetry(6, kq(6))[0] == 720
    cycle = lambda k: [(i, (i + 1) % k) for i in range(k)]
    assert gsm_lib.gsm_query_symmetry(5, cycle(5))[0] == 10
    assert gsm_lib.gsm_query_symmetry(8, cycle(8))[0] == 16
    path = [(i, i + 1) for i in range(15)]
    assert gsm_lib.gsm_query_symmetry(16, path)[0] == 2
    star = [(0, v) for v in range(1, 6)]
    assert gsm_lib.gsm_query_symmetry(6, star)[0] == 120
    # labels split the star's leaves into orbits of sizes 3 and 2
    assert gsm_lib.gsm_query_symmetry(6, star, [0, 1, 1, 1, 2, 2])[0] == 12
    # K_16 has 16! automorphisms; found without listing them
    assert gsm_lib.gsm_query_symmetry(16, kq(16))[0] == 20922789888000


def test_one_embedding_per_orbit(gsm_lib, oracle_lib):
    rng = np.random.default_rng(82)
    checked = 0
    while checked < 40:
        k = int(rng.integers(2, 6))
        num_labels = int(rng.integers(1, 3))
        edges, labels = random_query(rng, k, num_labels)
        n = int(rng.integers(8, 16))
        m_edges = set()
        while len(m_edges) < int(n * 2.5):
            a, b = sorted(int(x) for x in rng.choice(n, 2, replace=False))
            m_edges.add((a, b))
        g = I.graph_from_edges(n, sorted(m_edges), rng.integers(0, num_labels, n))
        q = I.query_from_edges(k, edges, labels)
        count, rows, rc = oracle_lib.match(g, q)
        assert rc == oracle_lib.OK
        if count == 0:
            continue
        aut, pairs = gsm_lib.gsm_query_symmetry(k, edges, labels)
        perms = brute_automorphisms(k, edges, labels.tolist())
        assert aut == len(perms) and count % aut == 0
        kept = [tuple(r) for r in rows.tolist() if satisfies(r, pairs)]
        assert len(kept) == count // aut
        for r in rows.tolist():
            images = {tuple(r[p[u]] for u in range(k)) for p in perms}
            assert sum(satisfies(x, pairs) for x in images) == 1
        checked += 1


def test_invalid_queries_are_rejected(gsm_lib):
    import ctypes
    with np.testing.assert_raises(gsm_lib.GsmError):
        gsm_lib.gsm_query_symmetry(3, [(0, 1)])            # disconnected
    with np.testing.assert_raises(gsm_lib.GsmError):
        gsm_lib.gsm_query_symmetry(0, [])                  # k outside 1..16
    with np.testing.assert_raises(gsm_lib.GsmError):
        gsm_lib.gsm_query_symmetry(3, [(0, 1), (1, 1)])    # self-loop
    # too little room for the constraints: the count is still reported
    e = np.array([0, 1, 1, 2, 2, 0], dtype=np.int32)       # triangle: 3 constraints
    aut, n = ctypes.c_uint64(), ctypes.c_int32()
    pairs = np.zeros(2, dtype=np.int32)
    st = gsm_lib._lib.gsm_query_symmetry(3, 3, e.ctypes.data, None, ctypes.byref(aut),
                                         pairs.ctypes.data, 1, ctypes.byref(n))
    assert st == gsm_lib.GSM_ERR_INVALID_ARG and n.value == 3 and aut.value == 6
