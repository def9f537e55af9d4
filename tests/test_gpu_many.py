"""gsm_enumerate_many (listing many queries with the copies overlapping the
next query's compute) against the CPU oracle, with host and device outputs,
chunked frontiers, empty results and truncation."""
import numpy as np
import pytest
import torch

import oracle
from paper_2003_01527_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rmat12():
    n, rp, col = I.rmat(12, 16, *I.RMAT_ABC, seed=21)
    return I.make_graph(n, rp, col, I.zipf_labels(n, 8, 1.0, seed=22))


def workload(g, num, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < num:
        q = I.random_walk_query(g, int(rng.integers(3, 8)), rng)
        c, rows, rc = oracle.match(g, q, limit=200_000, node_budget=20_000_000)
        if rc == oracle.OK:
            out.append((q, c, rows))
    return out


@pytest.mark.parametrize("opts", [{}, {"copy_slots": 1}, {"two_pass": True},
                                  {"copy_slots": 2, "mem_budget_bytes": 1 << 21, "chunk_rows": 300},
                                  {"host_workers": 1}, {"host_workers": 4, "copy_slots": 1},
                                  {"host_workers": 3, "filter_rounds": 1}])
def test_many_host_and_device_match_oracle(gsm_lib, cuda, rmat12, opts):
    g = rmat12
    items = workload(g, 12, seed=41)
    # a query whose label is absent from the graph: no embedding
    items.insert(0, (I.query_from_edges(3, [(0, 1), (1, 2)], [0, 99, 0]), 0,
                     np.zeros((0, 3), np.int32)))
    m = gsm_lib.Matcher(device=0, time_kernels=True, **opts)
    m.load_graph(g.row_ptr, g.col, g.labels, validate=True)
    Qs = [m.query(q.k, q.edges, q.labels) for q, _, _ in items]
    host = [torch.zeros(max(c, 1) * q.k, dtype=torch.int32).pin_memory() for q, c, _ in items]
    dev = [torch.zeros(max(c, 1) * q.k, dtype=torch.int32, device="cuda") for q, c, _ in items]
    for outs in (host, dev, host):
        counts = m.enumerate_many(Qs, outs)
        assert counts == [c for _, c, _ in items]
        for (q, c, rows), o in zip(items, outs):
            got = o.cpu().numpy()[:c * q.k].reshape(c, q.k)
            assert np.array_equal(got, rows)
    # which form of the verification levels ran
    launches = {st["name"]: st["launches"] for st in m.kernel_stats()}
    if opts.get("two_pass"):
        assert launches["extend_fused"] == 0 and launches["extend_write"] > 0
    else:
        assert launches["extend_fused"] > 0
    # the last query's rows stay readable through gsm_last_rows
    q, c, rows = items[-1]
    buf = np.zeros((max(c, 1), q.k), np.int32)
    gsm_lib.gsm_last_rows(m.ctx, buf, 0, c, 0)
    assert np.array_equal(buf[:c], rows)
    m.close()


def test_many_truncation_keeps_counts_and_prefixes(gsm_lib, cuda, rmat12):
    g = rmat12
    items = [it for it in workload(g, 6, seed=43) if it[1] >= 4][:3]
    assert items
    m = gsm_lib.Matcher(device=0, host_workers=2)
    m.load_graph(g.row_ptr, g.col, g.labels)
    Qs = [m.query(q.k, q.edges, q.labels) for q, _, _ in items]
    caps = [c // 2 for _, c, _ in items]
    outs = [np.zeros(max(cap, 1) * q.k, np.int32) for (q, _, _), cap in zip(items, caps)]
    counts, st = gsm_lib.gsm_enumerate_many(m.ctx, [Q.handle for Q in Qs], outs, caps, 0)
    assert st == gsm_lib.GSM_ERR_TRUNCATED
    assert counts.tolist() == [c for _, c, _ in items]
    for (q, c, rows), o, cap in zip(items, outs, caps):
        assert np.array_equal(o[:cap * q.k].reshape(cap, q.k), rows[:cap])
    m.close()


def test_many_workers_follow_graph_reloads(gsm_lib, cuda, rmat12):
    """The listing workers share the resident graph: after the graph is
    replaced they list against the new one."""
    g = rmat12
    items = workload(g, 6, seed=45)
    tg, (tq,) = I.tiny_er_workload()
    want_count, want_rows, _ = oracle.match(tg, tq)
    m = gsm_lib.Matcher(device=0, host_workers=2)
    for _ in range(2):
        m.load_graph(g.row_ptr, g.col, g.labels)
        Qs = [m.query(q.k, q.edges, q.labels) for q, _, _ in items]
        outs = [np.zeros(max(c, 1) * q.k, np.int32) for q, c, _ in items]
        assert m.enumerate_many(Qs, outs) == [c for _, c, _ in items]
        for (q, c, rows), o in zip(items, outs):
            assert np.array_equal(o[:c * q.k].reshape(c, q.k), rows)
        m.load_graph(tg.row_ptr, tg.col, tg.labels)
        Q = m.query(tq.k, tq.edges, tq.labels)
        outs = [np.zeros(max(want_count, 1) * tq.k, np.int32) for _ in range(3)]
        assert m.enumerate_many([Q, Q, Q], outs) == [want_count] * 3
        for o in outs:
            assert np.array_equal(o[:want_count * tq.k].reshape(-1, tq.k), want_rows)
    m.close()


def test_label_values_far_apart_give_same_rows(gsm_lib, cuda, rmat12):
    """Label values are only names: spreading them over the int32 range (the
    sort-based densification) lists the same rows as the original values (the
    table-based one)."""
    g = rmat12
    items = workload(g, 4, seed=47)
    big = (g.labels.astype(np.int64) * 100_000_007 - 2**30).astype(np.int32)
    assert len(np.unique(big)) == len(np.unique(g.labels))
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, big, validate=True)
    for q, c, rows in items:
        qbig = (q.labels.astype(np.int64) * 100_000_007 - 2**30).astype(np.int32)
        got, count = m.enumerate(m.query(q.k, q.edges, qbig))
        assert count == c and np.array_equal(got, rows)
    m.close()
