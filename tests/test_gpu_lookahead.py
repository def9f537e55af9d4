"""The k-look-ahead of the verification levels (Sec. 3.2, 1- and
2-look-ahead): results equal the oracle's with it off, at 1 and at 2, in every
frontier layout, and it only ever removes partial embeddings (every
intermediate frontier is at most as large as without it), removing some on
the power-law workloads."""
import numpy as np
import pytest

import oracle
from paper_2003_01527_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def slices(g, num, seed, kmin=4, kmax=8):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < num:
        q = I.random_walk_query(g, int(rng.integers(kmin, kmax + 1)), rng)
        hi = g.n
        for _ in range(14):
            c, _, rc = oracle.match(g, q, enumerate=False, root_range=(0, hi), limit=300_000,
                                    node_budget=20_000_000)
            if rc == oracle.OK:
                out.append((q, hi, c))
                break
            hi = max(1, hi // 4)
    return out


@pytest.fixture(scope="module")
def labelled():
    n, rp, col = I.rmat(12, 16, *I.RMAT_ABC, seed=71)
    return I.make_graph(n, rp, col, I.zipf_labels(n, 8, 1.0, seed=72))


@pytest.fixture(scope="module")
def unlabelled():
    n, rp, col = I.rmat(11, 8, *I.RMAT_ABC, seed=73)
    return I.make_graph(n, rp, col, np.zeros(n, np.int32))


@pytest.mark.parametrize("opts", [{}, {"two_pass": True}, {"compressed": True}])
def test_lookahead_results_equal_oracle(gsm_lib, cuda, labelled, opts):
    g = labelled
    items = slices(g, 14, seed=74)
    want = [oracle.match(g, q, root_range=(0, hi))[1] for q, hi, _ in items]
    frontiers = {}
    for la in (0, 1, 2):
        m = gsm_lib.Matcher(device=0, lookahead=la, **opts)
        m.load_graph(g.row_ptr, g.col, g.labels)
        fr = []
        for (q, hi, c), w in zip(items, want):
            Q = m.query(q.k, q.edges, q.labels).restrict(0, 0, hi)
            rows, count = m.enumerate(Q)
            assert count == c and np.array_equal(rows, w)
            assert m.count(Q) == c
            fr.append(m.last_run_stats()["frontier"])
        frontiers[la] = fr
        m.close()
    # pruning only removes rows: level by level no larger than without it,
    # and the 2-look-ahead no larger than the 1-look-ahead
    for a, b, c in zip(frontiers[0], frontiers[1], frontiers[2]):
        assert all(y <= x for x, y in zip(a, b))
        assert all(z <= y for y, z in zip(b, c))
    if not opts:
        assert sum(map(sum, frontiers[1])) < sum(map(sum, frontiers[0]))


def test_lookahead_unlabelled_shapes(gsm_lib, cuda, unlabelled):
    g = unlabelled
    s = I.unlabelled_shapes()
    window = {u: (0, 512) for u in range(1, 6)}
    cases = [(s["cycle5"], 16, None), (s["path6"], 4, window), (s["clique4"], g.n, None),
             (I.query_from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 4), (1, 3)]), 4, None)]
    want = [oracle.match(g, q, root_range=(0, hi), ranges=rg)[:2] for q, hi, rg in cases]
    for la in (1, 2):
        m = gsm_lib.Matcher(device=0, lookahead=la)
        m.load_graph(g.row_ptr, g.col, g.labels)
        for (q, hi, rg), (want_count, want_rows) in zip(cases, want):
            Q = m.query(q.k, q.edges).restrict(0, 0, hi)
            for u, (a, b) in (rg or {}).items():
                Q.restrict(u, a, b)
            rows, count = m.enumerate(Q)
            assert count == want_count and np.array_equal(rows, want_rows)
        m.close()


def test_lookahead_distinct_counts(gsm_lib, cuda, unlabelled):
    g = unlabelled
    s = I.unlabelled_shapes()
    m0 = gsm_lib.Matcher(device=0)
    m2 = gsm_lib.Matcher(device=0, lookahead=2)
    for m in (m0, m2):
        m.load_graph(g.row_ptr, g.col, g.labels)
    for shape in ("triangle", "clique4"):
        q = s[shape]
        assert m0.count_distinct(m0.query(q.k, q.edges)) == m2.count_distinct(m2.query(q.k, q.edges))
    m0.close()
    m2.close()


def test_invalid_lookahead(gsm_lib, cuda):
    opt = gsm_lib.gsm_default_options()
    opt.lookahead = 3
    with pytest.raises(gsm_lib.GsmError) as e:
        gsm_lib.gsm_create(0, opt)
    assert e.value.status == gsm_lib.GSM_ERR_INVALID_ARG
