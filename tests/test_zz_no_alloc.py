"""gsm_candidates_static: the allocation-free candidate filter.

Callers that cannot allocate device memory (their device memory is already
claimed by another allocator, or a latency-critical loop cannot take the
synchronisation of cudaMalloc/cudaFree) use this entry point with a graph
they keep on the device.  Its bitmaps and sizes must equal those of
gsm_candidates, call after call: the fixed device array it works in keeps the
previous call's contents, so the second call checks that nothing stale leaks.
They are also checked against the oracle's candidate predicate, with and
without a restriction range on a query vertex.

This file is collected last on purpose, and also passes alone in a fresh
process.
"""
import numpy as np
import pytest

import oracle
from paper_2003_01527_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_static_candidates_match_gsm_candidates_twice(gsm_lib, cuda):
    torch = cuda
    gl = gsm_lib
    n, rp, col = I.rmat(13, 16, *I.RMAT_ABC, seed=41)
    g = I.make_graph(n, rp, col, I.zipf_labels(n, 6, 1.0, seed=42))
    d = {k: torch.from_numpy(getattr(g, k)).cuda() for k in ("row_ptr", "col", "labels")}
    m = gl.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels)
    rng = np.random.default_rng(43)
    queries = [I.random_walk_query(g, int(rng.integers(3, 9)), rng) for _ in range(2)]
    # two calls in a row (different queries, so stale counters or bitmap words
    # from the first call would show), then the first query again
    for q in queries + queries[:1]:
        Q = m.query(q.k, q.edges, q.labels)
        want_bm, want_sizes = m.candidates(Q)
        nw = (g.n + 31) // 32
        got_bm = np.full((q.k, nw), 0xFFFFFFFF, dtype=np.uint32)
        got_sizes = np.zeros(q.k, dtype=np.uint64)
        torch.cuda.synchronize()
        gl.gsm_candidates_static(g.n, g.nnz, d["row_ptr"], d["col"], d["labels"], Q.handle,
                                 got_bm, got_sizes)
        assert np.array_equal(got_bm, want_bm)
        assert np.array_equal(got_sizes, want_sizes)
        assert int(got_sizes.sum()) > 0
    # device outputs, on a caller stream
    q = queries[1]
    Q = m.query(q.k, q.edges, q.labels)
    want_bm, want_sizes = m.candidates(Q)
    s = torch.cuda.Stream()
    out_bm = torch.zeros(q.k * ((g.n + 31) // 32), dtype=torch.int32, device="cuda")
    out_sizes = torch.zeros(q.k, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    gl.gsm_candidates_static(g.n, g.nnz, d["row_ptr"], d["col"], d["labels"], Q.handle,
                             out_bm, out_sizes, gl.GSM_OUT_DEVICE, s)
    assert np.array_equal(out_bm.cpu().numpy().view(np.uint32).reshape(q.k, -1), want_bm)
    assert np.array_equal(out_sizes.cpu().numpy().view(np.uint64), want_sizes)
    m.close()


def test_static_candidates_match_oracle_with_restrictions(gsm_lib, cuda, oracle_lib):
    """The allocation-free filter against the oracle's candidate predicate
    (bit for bit), unrestricted and with query vertices restricted to id
    ranges, two calls in a row each."""
    torch = cuda
    gl = gsm_lib
    n, rp, col = I.rmat(12, 16, *I.RMAT_ABC, seed=44)
    g = I.make_graph(n, rp, col, I.zipf_labels(n, 4, 1.0, seed=45))
    d = {k: torch.from_numpy(getattr(g, k)).cuda() for k in ("row_ptr", "col", "labels")}
    m = gl.Matcher(device=0)
    rng = np.random.default_rng(46)
    nw = (g.n + 31) // 32
    for rep in range(2):
        q = I.random_walk_query(g, int(rng.integers(3, 8)), rng)
        want = oracle.candidates(g, q).astype(bool)
        for ranges in ({}, {0: (100, 1500), q.k - 1: (0, 2048)}):
            Q = m.query(q.k, q.edges, q.labels)
            w = want.copy()
            for u, (lo, hi) in ranges.items():
                Q.restrict(u, lo, hi)
                w[u, :lo] = False
                w[u, hi:] = False
            got_bm = np.zeros((q.k, nw), dtype=np.uint32)
            got_sizes = np.zeros(q.k, dtype=np.uint64)
            torch.cuda.synchronize()
            gl.gsm_candidates_static(g.n, g.nnz, d["row_ptr"], d["col"], d["labels"], Q.handle,
                                     got_bm, got_sizes)
            assert np.array_equal(gl.unpack_bitmaps(got_bm, g.n).astype(bool), w)
            assert got_sizes.tolist() == w.sum(axis=1).tolist()
    m.close()


def test_static_candidates_reject_oversize(gsm_lib, cuda):
    gl = gsm_lib
    torch = cuda
    words = gl.GSM_STATIC_SCRATCH_BITMAP_BYTES // 4
    n = 32 * (words // 16) + 32  # one bitmap word per query vertex too many at k = 16
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    lab = torch.zeros(n, dtype=torch.int32, device="cuda")
    q = gl.gsm_query_create(None, 16, 15, np.array([[i, i + 1] for i in range(15)],
                                                      np.int32).reshape(-1), None)
    with pytest.raises(gl.GsmError) as ei:
        gl.gsm_candidates_static(n, 0, rp, None, lab, q, None, None)
    assert ei.value.status == gl.GSM_ERR_TOO_LARGE
    gl.gsm_query_destroy(q)
