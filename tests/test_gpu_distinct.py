"""Distinct-subgraph counts (gsm_count_distinct): ordered embeddings come in
groups of |Aut(Q)|, so distinct x |Aut(Q)| must equal the oracle's ordered
count, and |Aut(Q)| must equal an exhaustive count of the label- and
edge-preserving permutations of Q."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2003_01527_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def brute_aut(q):
    edges = {(int(a), int(b)) for a, b in q.edges} | {(int(b), int(a)) for a, b in q.edges}
    lab = [int(x) for x in q.labels]
    n = 0
    for p in itertools.permutations(range(q.k)):
        if all(lab[p[u]] == lab[u] for u in range(q.k)) and \
                all((p[a], p[b]) in edges for a, b in edges):
            n += 1
    return n


def test_distinct_counts_unlabelled(gsm_lib, cuda):
    n, rp, col = I.rmat(10, 16, *I.RMAT_ABC, seed=71)
    g = I.make_graph(n, rp, col, np.zeros(n, np.int32))
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels)
    shapes = dict(I.unlabelled_shapes())
    shapes["star3"] = I.query_from_edges(4, [(0, 1), (0, 2), (0, 3)])
    shapes["diamond"] = I.query_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)])
    shapes["path3"] = I.query_from_edges(3, [(0, 1), (1, 2)])
    for name, q in shapes.items():
        if name in ("path6", "cycle5"):
            continue  # too many ordered embeddings for the oracle on this graph
        distinct, aut = m.count_distinct(m.query(q.k, q.edges))
        assert aut == brute_aut(q), name
        assert distinct * aut == oracle.count(g, q), name
    m.close()


def test_distinct_counts_labelled(gsm_lib, cuda):
    n, rp, col = I.rmat(12, 16, *I.RMAT_ABC, seed=72)
    g = I.make_graph(n, rp, col, I.zipf_labels(n, 3, 1.0, seed=73))
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels)
    rng = np.random.default_rng(74)
    done = 0
    while done < 10:
        q = I.random_walk_query(g, int(rng.integers(3, 7)), rng)
        c, _, rc = oracle.match(g, q, enumerate=False, limit=2_000_000, node_budget=50_000_000)
        if rc != oracle.OK:
            continue
        distinct, aut = m.count_distinct(m.query(q.k, q.edges, q.labels))
        assert aut == brute_aut(q)
        assert distinct * aut == c
        done += 1
    m.close()


def test_distinct_counts_in_complete_graphs(gsm_lib, cuda):
    m = gsm_lib.Matcher(device=0)
    kn = I.graph_from_edges(9, [(i, j) for i in range(9) for j in range(i + 1, 9)])
    m.load_graph(kn.row_ptr, kn.col, kn.labels)
    k4 = I.unlabelled_shapes()["clique4"]
    assert m.count_distinct(m.query(4, k4.edges)) == (math.comb(9, 4), 24)
    c5 = I.unlabelled_shapes()["cycle5"]
    # 5-cycles in K9: choose 5 vertices, (5-1)!/2 cycles on them
    assert m.count_distinct(m.query(5, c5.edges)) == (math.comb(9, 5) * 12, 10)
    with pytest.raises(gsm_lib.GsmError):
        m.count_distinct(m.query(4, k4.edges).restrict(0, 0, 3))
    m.close()
