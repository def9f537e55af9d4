"""The served form: queries submitted while others run are batched with
them, and every result equals the one the query gets alone (gsm_count) and
the oracle's."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2003_01527_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served_setup(gsm_lib, cuda):
    n, rp, col = I.rmat(12, 16, *I.RMAT_ABC, seed=61)
    g = I.make_graph(n, rp, col, I.zipf_labels(n, 16, 1.0, seed=62))
    rng = np.random.default_rng(63)
    items = []
    while len(items) < 60:
        q = I.random_walk_query(g, int(rng.integers(3, 13)), rng)
        hi = g.n
        for _ in range(12):
            c, _, rc = oracle.match(g, q, enumerate=False, root_range=(0, hi), limit=100_000,
                                    node_budget=20_000_000)
            if rc == oracle.OK:
                items.append((q, hi, c))
                break
            hi = max(1, hi // 4)
    return g, items


def test_served_results_equal_alone(gsm_lib, served_setup):
    g, items = served_setup
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels)
    Qs = [m.query(q.k, q.edges, q.labels).restrict(0, 0, hi) for q, hi, _ in items]
    alone = [m.count(Q) for Q in Qs]
    assert alone == [c for _, _, c in items]
    gsm_lib.gsm_server_start(m.ctx, 2, 32)
    tickets = {}
    rng = np.random.default_rng(64)

    def producer():
        # Poisson arrivals at ~2,000 queries/s, each query submitted 3 times
        for rep in range(3):
            for j in rng.permutation(len(Qs)):
                time.sleep(float(rng.exponential(1 / 2000)))
                tickets[gsm_lib.gsm_submit(m.ctx, Qs[j].handle)] = int(j)

    th = threading.Thread(target=producer)
    th.start()
    results = {}
    deadline = time.time() + 120
    while (th.is_alive() or len(results) < len(tickets)) and time.time() < deadline:
        for t in list(tickets):
            if t in results:
                continue
            r = gsm_lib.gsm_poll(m.ctx, t)
            if r is not None:
                results[t] = r
        time.sleep(0.001)
    th.join()
    gsm_lib.gsm_server_stop(m.ctx)
    assert len(results) == len(tickets) == 3 * len(Qs)
    for t, r in results.items():
        assert r["status"] == 0
        assert r["count"] == alone[tickets[t]]
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_done_ns"]
    st = m.batch_stats()
    assert st["batches"] >= 2
    m.close()


def test_server_rejects_misuse(gsm_lib, served_setup):
    g, items = served_setup
    m = gsm_lib.Matcher(device=0)
    with pytest.raises(gsm_lib.GsmError):
        gsm_lib.gsm_server_start(m.ctx, 2, 8)  # no graph yet
    m.load_graph(g.row_ptr, g.col, g.labels)
    gsm_lib.gsm_server_start(m.ctx, 1, 8)
    with pytest.raises(gsm_lib.GsmError):
        gsm_lib.gsm_server_start(m.ctx, 1, 8)  # already running
    with pytest.raises(gsm_lib.GsmError):
        gsm_lib.gsm_poll(m.ctx, 12345)  # unknown ticket
    q, hi, c = items[0]
    Q = m.query(q.k, q.edges, q.labels).restrict(0, 0, hi)
    t = gsm_lib.gsm_submit(m.ctx, Q.handle)
    r = None
    for _ in range(20000):
        r = gsm_lib.gsm_poll(m.ctx, t)
        if r is not None:
            break
        time.sleep(0.0005)
    assert r is not None and r["count"] == c
    gsm_lib.gsm_server_stop(m.ctx)
    m.close()


def test_served_enumerate_mode_rows(gsm_lib, served_setup):
    """Requests in enumerate mode, mixed with count-mode requests under Poisson
    arrivals: every listed result equals the oracle's sorted rows and the rows
    the query gets alone (gsm_enumerate); count-mode results carry no rows."""
    g, items = served_setup
    items = [it for it in items if it[2] <= 200_000][:30]
    m = gsm_lib.Matcher(device=0)
    m.load_graph(g.row_ptr, g.col, g.labels)
    Qs = [m.query(q.k, q.edges, q.labels).restrict(0, 0, hi) for q, hi, _ in items]
    want = []
    for (q, hi, c), Q in zip(items, Qs):
        cnt, rows, _ = oracle.match(g, q, root_range=(0, hi))
        alone, count = m.enumerate(Q)
        assert count == cnt == c and np.array_equal(alone, rows)
        want.append(rows)
    gsm_lib.gsm_server_start(m.ctx, 2, 16)
    rng = np.random.default_rng(65)
    tickets = {}
    for rep in range(2):
        for j in rng.permutation(len(Qs)):
            time.sleep(float(rng.exponential(1 / 2000)))
            mode = gsm_lib.GSM_MODE_ENUMERATE if (rep + j) % 2 == 0 else gsm_lib.GSM_MODE_COUNT
            tickets[gsm_lib.gsm_submit(m.ctx, Qs[j].handle, mode)] = (int(j), mode)
    results = {}
    deadline = time.time() + 120
    while len(results) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t not in results:
                r = gsm_lib.gsm_poll(m.ctx, t)
                if r is not None:
                    results[t] = r
        time.sleep(0.001)
    gsm_lib.gsm_server_stop(m.ctx)
    assert len(results) == len(tickets)
    listed = 0
    for t, r in results.items():
        j, mode = tickets[t]
        assert r["status"] == 0 and r["count"] == items[j][2]
        if mode == gsm_lib.GSM_MODE_ENUMERATE:
            rows = r.get("rows", np.zeros((0, items[j][0].k), np.int32))
            assert np.array_equal(rows.reshape(-1, items[j][0].k), want[j])
            listed += 1
        else:
            assert "rows" not in r
    assert listed >= len(Qs) // 2
    m.close()
