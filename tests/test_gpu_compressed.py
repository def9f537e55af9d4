"""Compressed partial results (GSM_OPT_COMPRESSED_FRONTIERS: frontier rows
kept as (parent row, new vertex)) against the CPU oracle and against the
uncompressed path: same counts, same sorted rows, under chunking too."""
import numpy as np
import pytest

import oracle
from paper_2003_01527_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rmat12():
    n, rp, col = I.rmat(12, 16, *I.RMAT_ABC, seed=21)
    return I.make_graph(n, rp, col, I.zipf_labels(n, 8, 1.0, seed=22))


def walk_queries(g, num, kmin, kmax, seed, limit=200_000):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < num:
        q = I.random_walk_query(g, int(rng.integers(kmin, kmax + 1)), rng)
        c, rows, rc = oracle.match(g, q, limit=limit, node_budget=20_000_000)
        if rc == oracle.OK:
            out.append((q, c, rows))
    return out


@pytest.mark.parametrize("opts", [{}, {"mem_budget_bytes": 1 << 21, "chunk_rows": 200},
                                  {"block_size": 1024}])
def test_compressed_rows_match_oracle(gsm_lib, cuda, rmat12, opts):
    g = rmat12
    items = walk_queries(g, 12, 3, 8, seed=61)
    m = gsm_lib.Matcher(device=0, compressed=True, time_kernels=True, **opts)
    m.load_graph(g.row_ptr, g.col, g.labels)
    for q, c, rows in items:
        Q = m.query(q.k, q.edges, q.labels)
        got, count = m.enumerate(Q)
        assert count == c and np.array_equal(got, rows)
        assert m.count(Q) == c
    launches = {st["name"]: st["launches"] for st in m.kernel_stats()}
    assert launches["extend_fused"] > 0 and launches["extend_write"] == 0
    m.close()


def test_compressed_deep_query_and_symmetry(gsm_lib, cuda):
    # a 16-vertex path in a 20-cycle: width-15 rows decoded through 14 parents
    cyc = I.graph_from_edges(20, [(i, (i + 1) % 20) for i in range(20)])
    path16 = I.query_from_edges(16, [(i, i + 1) for i in range(15)])
    want_count, want_rows, rc = oracle.match(cyc, path16)
    assert rc == oracle.OK and want_count == 40
    m = gsm_lib.Matcher(device=0, compressed=True)
    m.load_graph(cyc.row_ptr, cyc.col, cyc.labels)
    rows, count = m.enumerate(m.query(16, path16.edges))
    assert count == want_count and np.array_equal(rows, want_rows)
    # distinct counts (ordering constraints) agree with the plain path
    n, rp, col = I.rmat(10, 16, *I.RMAT_ABC, seed=31)
    g = I.make_graph(n, rp, col, np.zeros(n, np.int32))
    plain = gsm_lib.Matcher(device=0)
    plain.load_graph(g.row_ptr, g.col, g.labels)
    m.load_graph(g.row_ptr, g.col, g.labels)
    for name in ("triangle", "clique4", "cycle5"):
        q = I.unlabelled_shapes()[name]
        assert m.count_distinct(m.query(q.k, q.edges)) == \
            plain.count_distinct(plain.query(q.k, q.edges))
    q = I.unlabelled_shapes()["cycle5"]
    a = m.enumerate(m.query(q.k, q.edges).restrict(0, 0, 8))
    b = plain.enumerate(plain.query(q.k, q.edges).restrict(0, 0, 8))
    assert a[1] == b[1] and np.array_equal(a[0], b[0])
    plain.close()
    m.close()
