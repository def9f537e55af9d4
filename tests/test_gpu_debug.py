"""The GSM_DEBUG build (libgsm_debug.so: device bounds checks at the hot
kernels' indexed accesses, which report a failed check as GSM_ERR_INTERNAL
instead of faulting) gives the oracle's results with no check failing:
listings and counts of random-walk query slices on a labelled R-MAT graph
(sorted and already-canonical matching orders), the labelled tiny ER query,
unlabelled triangles and 4-cycles, and a listing batch.  The build is made
on first use and run in a child process (one library per process)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from paper_2003_01527_gb300 import gsm, inputs as I

assert gsm.DEBUG and gsm.LIB_PATH.endswith("libgsm_debug.so"), gsm.LIB_PATH
checked = 0
n, rp, col = I.rmat(12, 16, *I.RMAT_ABC, seed=81)
g = I.make_graph(n, rp, col, I.zipf_labels(n, 8, 1.0, seed=82))
rng = np.random.default_rng(83)
m = gsm.Matcher(device=0)
m.load_graph(g.row_ptr, g.col, g.labels)
qs = []
while len(qs) < 10:
    q = I.random_walk_query(g, int(rng.integers(4, 8)), rng)
    hi = g.n
    for _ in range(14):
        c, _, rc = oracle.match(g, q, enumerate=False, root_range=(0, hi), limit=200_000,
                                node_budget=10_000_000)
        if rc == oracle.OK:
            qs.append((q, hi))
            break
        hi = max(1, hi // 4)
noncanonical = 0
for q, hi in qs:
    want_count, want_rows, _ = oracle.match(g, q, root_range=(0, hi))
    Q = m.query(q.k, q.edges, q.labels).restrict(0, 0, hi)
    rows, count = m.enumerate(Q)
    assert count == want_count and np.array_equal(rows, want_rows)
    assert m.count(Q) == want_count
    noncanonical += tuple(m.last_run_stats()["order"]) != tuple(range(q.k))
    checked += 2
Qs = [m.query(q.k, q.edges, q.labels).restrict(0, 0, hi) for q, hi in qs]
counts, rows = m.run_batch(Qs, enumerate=True)
for (q, hi), c, r in zip(qs, counts, rows):
    want_count, want_rows, _ = oracle.match(g, q, root_range=(0, hi))
    assert c == want_count and np.array_equal(r, want_rows)
    checked += 1
m.close()
gt, (qt,) = I.tiny_er_workload()
m = gsm.Matcher(device=0)
m.load_graph(gt.row_ptr, gt.col, gt.labels)
want_count, want_rows, _ = oracle.match(gt, qt)
rows, count = m.enumerate(m.query(qt.k, qt.edges, qt.labels))
assert count == want_count and np.array_equal(rows, want_rows)
m.close()
checked += 1
n, rp, col = I.rmat(11, 8, *I.RMAT_ABC, seed=84)
gu = I.make_graph(n, rp, col, np.zeros(n, np.int32))
m = gsm.Matcher(device=0)
m.load_graph(gu.row_ptr, gu.col, gu.labels)
s = I.unlabelled_shapes()
for q in (s["triangle"], I.query_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)])):
    assert m.count(m.query(q.k, q.edges)) == oracle.count(gu, q)
    checked += 1
m.close()
print("OK", checked, "non-canonical orders:", noncanonical)
"""


def test_debug_build_gives_the_oracles_results():
    from paper_2003_01527_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, GSM_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert r.stdout.strip().startswith("OK"), r.stdout
