"""The per-kernel measurements (GSM_OPT_TIME_KERNELS, GSM_OPT_COUNT_PROBES):
counting them changes no result, and the probe-byte term of the byte model
(4 * ceil(log2 deg) per non-tree edge check made) behaves as its definition
says -- zero for a tree query, positive for a cycle, and bounded by one check
per candidate and non-tree edge at the largest degree."""
import math

import numpy as np
import pytest

import oracle
from paper_2003_01527_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def graph():
    n, rp, col = I.rmat(11, 8, *I.RMAT_ABC, seed=91)
    return I.make_graph(n, rp, col, np.zeros(n, np.int32))


def fused(stats):
    return next(s for s in stats if s["name"] == "extend_fused")


def test_probe_bytes_follow_their_definition(gsm_lib, cuda, graph):
    g = graph
    s = I.unlabelled_shapes()
    m = gsm_lib.Matcher(device=0, time_kernels=True, count_probes=True)
    m0 = gsm_lib.Matcher(device=0)
    for x in (m, m0):
        x.load_graph(g.row_ptr, g.col, g.labels)
    max_deg = int(np.diff(g.row_ptr).max())
    cases = [("path3", I.query_from_edges(3, [(0, 1), (1, 2)]), 0),
             ("star4", I.query_from_edges(4, [(0, 1), (0, 2), (0, 3)]), 0),
             ("triangle", s["triangle"], 1), ("cycle4", I.query_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)]), 1)]
    for name, q, nontree in cases:
        want = oracle.count(g, q)
        m.kernel_stats(reset=True)
        assert m.count(m.query(q.k, q.edges)) == want
        # the last level of a count is not a single-pass level: list instead
        rows, c = m.enumerate(m.query(q.k, q.edges))
        assert c == want and m0.count(m0.query(q.k, q.edges)) == want
        st = fused(m.kernel_stats(reset=True))
        checked = sum(m.last_run_stats()["candidates"])
        if nontree == 0:
            assert st["probe_bytes"] == 0, name
        else:
            assert st["probe_bytes"] > 0, name
            assert st["probe_bytes"] <= 2 * checked * nontree * 4 * math.ceil(math.log2(max_deg)), name
        assert st["probe_bytes"] <= st["algo_bytes"]
    m.close()
    m0.close()
