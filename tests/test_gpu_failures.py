"""Failure paths of the library, made on the host or through bounded device
waits -- no GPU fault and no hang:

* the device allocator fails (the alloc hook returns NULL, at every point of
  a run in turn): the call returns GSM_ERR_OOM, and the same context then
  gives the oracle's result;
* a single-pass level's look-back wait runs out: one tile withholds its
  survivor count (GSM_OPT_INJECT_LOOKBACK_STALL), the tiles after it give up
  after lookback_spin_limit polls, the call returns GSM_ERR_TIMEOUT, the
  caller's buffer is left untouched, and the same context then counts
  exactly;
* a look-back wait of the final row sort runs out (GSM_OPT_INJECT_SORT_STALL:
  one tile of every sort pass withholds its digit counts): GSM_ERR_TIMEOUT,
  nothing written past the rows, and the context then lists exactly;
* a look-back wait of a level's work scan runs out (GSM_OPT_INJECT_SCAN_STALL:
  one tile of every pivot-and-scan launch withholds its work total):
  GSM_ERR_TIMEOUT, the caller's buffer untouched, and the context still
  counts exactly.
"""
import hashlib

import numpy as np
import pytest

import oracle
from paper_2003_01527_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def small_case():
    g, (q,) = I.tiny_er_workload()
    return g, q


def test_alloc_failure_at_every_allocation_of_a_run(gsm_lib, cuda):
    g, q = small_case()
    want_count, want_rows, _ = oracle.match(g, q)
    # allocations a fresh context makes for one listing, after the graph load
    state = {"calls": 0, "fail_at": None}

    def hook(nbytes):
        state["calls"] += 1
        return state["fail_at"] is None or state["calls"] != state["fail_at"]

    m = gsm_lib.Matcher(device=0, alloc_hook=hook)
    m.load_graph(g.row_ptr, g.col, g.labels)
    before = state["calls"]
    rows, count = m.enumerate(m.query(q.k, q.edges, q.labels))
    assert count == want_count and np.array_equal(rows, want_rows)
    per_run = state["calls"] - before
    m.close()
    assert per_run >= 3
    for nth in range(1, per_run + 1):
        state["calls"], state["fail_at"] = 0, None
        m = gsm_lib.Matcher(device=0, alloc_hook=hook)
        m.load_graph(g.row_ptr, g.col, g.labels)
        Q = m.query(q.k, q.edges, q.labels)
        state["fail_at"] = state["calls"] + nth
        with pytest.raises(gsm_lib.GsmError) as e:
            m.enumerate(Q)
        assert e.value.status == gsm_lib.GSM_ERR_OOM
        state["fail_at"] = None
        # the context is still usable and exact
        rows, count = m.enumerate(Q)
        assert count == want_count and np.array_equal(rows, want_rows)
        assert m.count(Q) == want_count
        m.close()


def test_every_allocation_failing_then_recovering(gsm_lib, cuda):
    g, q = small_case()
    want = oracle.count(g, q)
    state = {"fail": False}
    m = gsm_lib.Matcher(device=0, alloc_hook=lambda nbytes: not state["fail"])
    m.load_graph(g.row_ptr, g.col, g.labels)
    Q = m.query(q.k, q.edges, q.labels)
    state["fail"] = True
    for call in (lambda: m.count(Q), lambda: m.enumerate(Q), lambda: m.candidates(Q)):
        with pytest.raises(gsm_lib.GsmError) as e:
            call()
        assert e.value.status == gsm_lib.GSM_ERR_OOM
    state["fail"] = False
    assert m.count(Q) == want
    m.close()


def test_lookback_wait_runs_out(gsm_lib, cuda):
    import bench
    g, queries = bench.load_workload()
    sl = queries[0]  # its levels have hundreds of tiles
    torch = cuda
    m = gsm_lib.Matcher(device=0, lookback_spin_limit=64, inject_lookback_stall=True)
    m.load_graph(g.row_ptr, g.col, g.labels)
    Q = m.query(sl["k"], sl["edges"], sl["labels"]).restrict(0, 0, sl["root_hi"])
    out = torch.full((sl["count"] * sl["k"] + 1024,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(gsm_lib.GsmError) as e:
        m.enumerate(Q, out=out)
    assert e.value.status == gsm_lib.GSM_ERR_TIMEOUT
    assert bool((out == -7).all())  # nothing was copied out
    # the same context still runs kernels and counts exactly: the edge query
    # labelled (0, 0) has one level, counted without a look-back; its count is
    # the number of directed edges between label-0 vertices
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    want = int(((g.labels[src] == 0) & (g.labels[g.col] == 0)).sum())
    assert m.count(m.query(2, [(0, 1)], [0, 0])) == want
    m.close()
    # and without the injection the slice is exact (under a bound the
    # levels' own waits never reach)
    m = gsm_lib.Matcher(device=0, lookback_spin_limit=4096)
    m.load_graph(g.row_ptr, g.col, g.labels)
    Q = m.query(sl["k"], sl["edges"], sl["labels"]).restrict(0, 0, sl["root_hi"])
    assert m.count(Q) == sl["count"]
    m.close()


def test_sort_wait_runs_out(gsm_lib, cuda):
    import bench
    g, queries = bench.load_workload()
    sl = queries[13]  # its matching order is not canonical: the rows are sorted
    torch = cuda
    # a bound the levels' own waits never reach, short enough for the test
    m = gsm_lib.Matcher(device=0, lookback_spin_limit=4096, inject_sort_stall=True)
    m.load_graph(g.row_ptr, g.col, g.labels)
    Q = m.query(sl["k"], sl["edges"], sl["labels"]).restrict(0, 0, sl["root_hi"])
    n = sl["count"] * sl["k"]
    out = torch.full((n + 1024,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(gsm_lib.GsmError) as e:
        m.enumerate(Q, out=out)
    assert e.value.status == gsm_lib.GSM_ERR_TIMEOUT
    assert "sort" in str(e.value)
    assert bool((out[n:] == -7).all())  # no write past the rows
    # counting needs no sort: exact on the same context
    assert m.count(Q) == sl["count"]
    m.close()
    m = gsm_lib.Matcher(device=0, lookback_spin_limit=4096)
    m.load_graph(g.row_ptr, g.col, g.labels)
    Q = m.query(sl["k"], sl["edges"], sl["labels"]).restrict(0, 0, sl["root_hi"])
    _, c = m.enumerate(Q, out=out)
    rows = out[:n].cpu().numpy().astype("<i4")
    assert c == sl["count"]
    assert hashlib.sha256(rows.tobytes()).hexdigest() == sl["rows_sha256"]
    m.close()


def test_work_scan_wait_runs_out(gsm_lib, cuda):
    import bench
    g, queries = bench.load_workload()
    sl = queries[0]
    torch = cuda
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels)
    Q = m.query(sl["k"], sl["edges"], sl["labels"]).restrict(0, 0, sl["root_hi"])
    assert m.count(Q) == sl["count"]
    # a level after the first has more rows than one scan tile (1,024)
    assert max(m.last_run_stats()["frontier"][1:]) > 2048
    m.close()
    # a bound the levels' own waits never reach, short enough for the test
    m = gsm_lib.Matcher(device=0, lookback_spin_limit=4096, inject_scan_stall=True)
    m.load_graph(g.row_ptr, g.col, g.labels)
    Q = m.query(sl["k"], sl["edges"], sl["labels"]).restrict(0, 0, sl["root_hi"])
    out = torch.full((sl["count"] * sl["k"] + 1024,), -7, dtype=torch.int32, device="cuda")
    for call in (lambda: m.enumerate(Q, out=out), lambda: m.count(Q)):
        with pytest.raises(gsm_lib.GsmError) as e:
            call()
        assert e.value.status == gsm_lib.GSM_ERR_TIMEOUT
        assert "work-scan" in str(e.value)
    assert bool((out == -7).all())  # nothing was copied out
    # the same context still runs kernels and counts exactly: a one-vertex
    # query has no level and so no work scan
    assert m.count(m.query(1, [], [0])) == int((g.labels == 0).sum())
    m.close()


def test_invalid_spin_limit(gsm_lib, cuda):
    opt = gsm_lib.gsm_default_options()
    opt.lookback_spin_limit = -1
    with pytest.raises(gsm_lib.GsmError) as e:
        gsm_lib.gsm_create(0, opt)
    assert e.value.status == gsm_lib.GSM_ERR_INVALID_ARG
