"""Full-size parity for the unlabelled R-MAT scale-20 workload (triangle,
4-clique, 5-cycle, 6-vertex path; chunked under a small memory budget) and the
labelled R-MAT scale-22 graph of the served workload.

At these sizes the oracle cannot list everything, so the checks are:
closed forms that hold at any size (edge count = nnz, ordered 3-paths =
sum d(d-1)), root slices the oracle lists one by one (compared row for row),
consistency of a chunked full count with the unchunked one and with the sum
of slice counts, and ordered triangle counts divisible by 6.
"""
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


@pytest.fixture(scope="module")
def rmat20():
    return I.rmat_unlabelled_graph(scale=20, seed=3)


def test_rmat20_closed_forms_and_chunked_counts(gsm_lib, cuda, rmat20):
    g = rmat20
    d = g.degrees()
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels, validate=True)
    assert m.count(m.query(2, [(0, 1)])) == g.nnz
    path3 = m.query(3, [(0, 1), (1, 2)])
    assert m.count(path3) == int((d * (d - 1)).sum())
    tri = I.unlabelled_shapes()["triangle"]
    full = m.count(m.query(3, tri.edges))
    assert full % 6 == 0 and full > 0
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


@pytest.fixture(scope="module")
def rmat22():
    n, rp, col = I.rmat(22, 16, *I.RMAT_ABC, seed=5)
    return I.make_graph(n, rp, col, I.zipf_labels(n, 32, 1.0, seed=105))


def test_rmat22_labelled_slices_and_serving(gsm_lib, cuda, rmat22):
    import time
    g = rmat22
    rng = np.random.default_rng(205)
    items = []
    while len(items) < 6:
        q = I.random_walk_query(g, int(rng.integers(3, 13)), rng)
        lo = int(rng.integers(0, g.n - 4096))
        lo, hi, c, rows = oracle_slice(g, q, lo, 4096, limit=500_000, budget=50_000_000)
        if hi > lo:
            items.append((q, lo, hi, c, rows))
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels, validate=True)
    Qs = []
    for q, lo, hi, c, rows in items:
        Q = m.query(q.k, q.edges, q.labels).restrict(0, lo, hi)
        got, count = m.enumerate(Q)
        assert count == c and np.array_equal(got, rows)
        Qs.append(Q)
    assert m.run_batch(Qs) == [c for _, _, _, c, _ in items]
    gsm_lib.gsm_server_start(m.ctx, 2, 16)
    tickets = [(gsm_lib.gsm_submit(m.ctx, Qs[j % len(Qs)].handle), j % len(Qs))
               for j in range(4 * len(Qs))]
    done = {}
    deadline = time.time() + 120
    while len(done) < len(tickets) and time.time() < deadline:
        for t, j in tickets:
            if t not in done:
                r = gsm_lib.gsm_poll(m.ctx, t)
                if r is not None:
                    done[t] = (r, j)
        time.sleep(0.001)
    gsm_lib.gsm_server_stop(m.ctx)
    assert len(done) == len(tickets)
    for r, j in done.values():
        assert r["status"] == 0 and r["count"] == items[j][3]
    m.close()
