"""The seeded generators produce valid inputs with the stated shapes."""
import numpy as np

import oracle
from paper_2003_01527_gb300 import inputs as I


def test_rmat_is_valid_and_seeded(oracle_lib):
    n, rp, col = I.rmat(10, 16, *I.RMAT_ABC, seed=7)
    g = I.make_graph(n, rp, col, np.zeros(n, np.int32))
    assert oracle.validate_graph(g) == oracle.OK
    n2, rp2, col2 = I.rmat(10, 16, *I.RMAT_ABC, seed=7)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    deg = g.degrees()
    assert deg.max() > 8 * deg.mean()  # power-law: hubs far above the mean


def test_er_shape(oracle_lib):
    g, (q,) = I.tiny_er_workload()
    assert g.n == 2000 and g.nnz == 16000
    assert oracle.validate_graph(g) == oracle.OK
    assert set(np.unique(g.labels).tolist()) == {0, 1, 2, 3}
    assert q.labels.tolist() == [0, 1, 0, 2] and q.m == 4


def test_zipf_labels_follow_the_law():
    lab = I.zipf_labels(200000, 8, 1.0, seed=3)
    freq = np.bincount(lab, minlength=8) / lab.size
    p = 1.0 / np.arange(1, 9)
    p /= p.sum()
    assert np.allclose(freq, p, atol=0.01)


def test_random_walk_queries(oracle_lib):
    n, rp, col = I.rmat(10, 16, *I.RMAT_ABC, seed=9)
    g = I.make_graph(n, rp, col, I.zipf_labels(n, 4, 1.0, seed=10))
    rng = np.random.default_rng(1)
    for k in range(3, 9):
        q = I.random_walk_query(g, k, rng)
        assert q.k == k and oracle.validate_query(q) == oracle.OK
        assert len(set(q.walk.tolist())) == k
        assert np.array_equal(q.labels, g.labels[q.walk])
        for a, b in q.edges:  # induced edges exist in G
            assert I.has_edge(g, int(q.walk[a]), int(q.walk[b]))
    q = I.random_walk_query(g, 8, rng, non_tree=(2, 4))
    assert q.m >= 7 and q.m <= 7 + 4
