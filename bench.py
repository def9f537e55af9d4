"""Benchmark: embeddings/s and queries/s of the GPU subgraph matcher.

Workload (the power-law labelled configuration): an R-MAT scale-16 graph
(65,536 vertices, edge factor 16, a=.57 b=.19 c=.19, symmetrised, deduplicated,
self-loops removed) with 8 Zipf(1.0) vertex labels, and 20 random-walk
queries of 4-8 vertices (induced edges, inherited labels).  Each query is
restricted to a prefix [0, hi) of the image of query vertex 0 because the full
results of these queries reach 10^10-10^17 rows; hi and the expected count and
row digest of every slice were written by the CPU oracle
(tests/golden/make_workloads.py).

A step = all 20 query slices through the whole path (filter, order, every
verification level, sorting into canonical order), listed by one
gsm_enumerate_many call into device buffers.  The graph is resident; L2 is
flushed before each timed step (the graph is smaller than L2).  The headline
pass records no per-kernel events; a second pass of the same steps on a
context that does gives the per-kernel split and the roofline of the
dominant kernel.  The end-to-end figure (`e2e`) uploads the graph from pinned
host memory and lists every slice into pinned host buffers through the same
call.

Further legs on the same line:
  `compressed_frontiers`: the slices with frontier rows kept as (parent row,
      new vertex), time and peak frontier memory against the default layout.
  `lookahead`: the slices with the k-look-ahead off, at 1 and at 2:
      candidates checked, partial embeddings kept, time per step.
  `batched_vs_plain`: R-MAT scale 18 (16 Zipf(1.2) labels, 256 random-walk
      queries of 3-10 vertices with 2-4 non-tree edges, oracle-sized root
      slices) counted one query per call versus as one batch (one CUDA graph),
      the same in enumerate mode (sorted rows in device memory), then served
      under Poisson arrivals at 50-10,000 queries/s.
  `unlabelled_counts`: unlabelled R-MAT scale 20: the 3-path count (checked
      against sum d(d-1)), ordered and distinct triangle and 4-clique counts
      (checked against k! x the oracle's clique count), and the 5-cycle and
      6-path on stored root slices (checked against the oracle's counts).
  `served_rmat22`: the served form on resident R-MAT scale 22 with 32
      Zipf(1.0) labels, 2,000 Poisson arrivals per rate at 50-2,000 queries/s
      (and 5,000 and 10,000 beyond the configured range) from a pool of
      random-walk queries of 3-12 vertices, against the plain form run
      serially on the same arrival stream.
Every count and row digest is checked against the oracle's stored values.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One JSON line on rank 0.  `--impl reference` times the CPU oracle on a fixed
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden", "rmat16_labelled_slices.json")
GOLDEN_BATCH = os.path.join(ROOT, "tests", "golden", "rmat18_batched_slices.json")
GOLDEN_RMAT20 = os.path.join(ROOT, "tests", "golden", "rmat20_unlabelled.json")
GOLDEN_SERVED = os.path.join(ROOT, "tests", "golden", "rmat22_served_slices.json")
SERVED22_RATES = (50, 100, 200, 500, 1000, 2000, 5000, 10000)
SERVE_RATES = (50, 100, 200, 500, 1000, 2000, 5000, 10000)
METRIC = "embeddings/sec & queries/sec at 1 GB300 (batched vs plain, bit-exact); p50/p99"
UNIT = "embeddings/s"
WORKLOAD = ("R-MAT scale 16 (65,536 vertices, edge factor 16), 8 Zipf(1.0) labels, "
            "20 random-walk queries of 4-8 vertices, each on an oracle-sized root slice")


def load_workload():
    from paper_2003_01527_gb300 import inputs as I
    with open(GOLDEN) as f:
        gold = json.load(f)
    g, _ = I.rmat_labelled_workload(scale=16, num_labels=8, zipf_s=1.0, num_queries=0, seed=2)
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col, g.labels):
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    if h.hexdigest() != gold["graph"]["sha256"]:
        raise SystemExit("generated graph differs from the stored workload")
    return g, gold["queries"]


def load_batch_workload():
    from paper_2003_01527_gb300 import inputs as I
    with open(GOLDEN_BATCH) as f:
        gold = json.load(f)
    g, _ = I.rmat_labelled_workload(scale=18, num_labels=16, zipf_s=1.2, num_queries=0, seed=4)
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col, g.labels):
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    if h.hexdigest() != gold["graph"]["sha256"]:
        raise SystemExit("generated batch graph differs from the stored workload")
    return g, gold["queries"]


def pct(xs, p):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(p / 100 * (len(xs) - 1))))] if xs else None


def batched_and_served(gsm, torch, device, serve_seconds):
    """The batched form (one CUDA graph for all 256 queries) against 256
    single-query launches, then the served form under Poisson arrivals, on the
    R-MAT 18 workload; every count checked against the oracle's."""
    g, queries = load_batch_workload()
    M = gsm.Matcher(device=device)
    M.load_graph(g.row_ptr, g.col, g.labels, validate=True)
    Qs = [M.query(q["k"], q["edges"], q["labels"]).restrict(0, 0, q["root_hi"]) for q in queries]
    want = [q["count"] for q in queries]
    emb = sum(want)
    # plain: one query per call
    for _ in range(2):
        got = [M.count(Q) for Q in Qs]
    if got != want:
        raise SystemExit("plain counts differ from the oracle's")
    reps = 3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        for Q in Qs:
            M.count(Q)
    plain_s = (time.perf_counter() - t0) / reps
    lat = []
    for Q in Qs:
        t1 = time.perf_counter()
        M.count(Q)
        lat.append((time.perf_counter() - t1) * 1e3)
    # batched: autotune on the first call, then time
    got = M.run_batch(Qs, autotune=True)
    if got != want:
        raise SystemExit("batched counts differ from the oracle's")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        got = M.run_batch(Qs)
    batch_s = (time.perf_counter() - t0) / reps
    if got != want:
        raise SystemExit("batched counts differ from the oracle's")
    bst = M.batch_stats()
    out = {"workload": "R-MAT scale 18 (262,144 vertices, edge factor 16), 16 Zipf(1.2) labels, "
                       f"{len(Qs)} random-walk queries of 3-10 vertices (tree + 2-4 non-tree "
                       "edges), each on an oracle-sized root slice",
           "embeddings_per_pass": emb,
           "plain": {"queries_per_sec": round(len(Qs) / plain_s, 1),
                     "embeddings_per_sec": round(emb / plain_s, 1),
                     "ms_per_pass": round(plain_s * 1e3, 3),
                     "latency_ms_p50": round(pct(lat, 50), 4),
                     "latency_ms_p99": round(pct(lat, 99), 4)},
           "batched": {"queries_per_sec": round(len(Qs) / batch_s, 1),
                       "embeddings_per_sec": round(emb / batch_s, 1),
                       "ms_per_pass": round(batch_s * 1e3, 3),
                       "graph_kernels": bst["kernels_per_graph"],
                       "block_size": bst["block_size"], "grid": bst["grid"],
                       "tuned": bst["tuned"]},
           "bit_exact": True}
    # enumerate mode: every query's sorted rows in device memory, the batch
    # (one graph, rows canonicalised per query) against one gsm_enumerate per
    # query; rows checked against the oracle's digests
    outs = [torch.empty(max(c, 1) * q["k"], dtype=torch.int32, device="cuda")
            for c, q in zip(want, queries)]

    def digests_ok(rows_list):
        for q, r in zip(queries, rows_list):
            a = np.ascontiguousarray(r, dtype="<i4").reshape(-1)
            if hashlib.sha256(a.tobytes()).hexdigest() != q["rows_sha256"]:
                return False
        return True

    for Q, o in zip(Qs, outs):
        M.enumerate(Q, out=o)
    if not digests_ok([o[:c * q["k"]].cpu().numpy() for o, c, q in zip(outs, want, queries)]):
        raise SystemExit("plain enumerate rows differ from the oracle's")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        for Q, o in zip(Qs, outs):
            M.enumerate(Q, out=o)
    torch.cuda.synchronize()
    plain_e = (time.perf_counter() - t0) / reps
    got, rows = M.run_batch(Qs, enumerate=True, device=True)
    if got != want or not digests_ok([r.cpu().numpy() for r in rows]):
        raise SystemExit("batched enumerate rows differ from the oracle's")
    del rows
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        got, rows = M.run_batch(Qs, enumerate=True, device=True)
        del rows
    torch.cuda.synchronize()
    batch_e = (time.perf_counter() - t0) / reps
    out["enumerate"] = {
        "mode": "sorted rows in device memory",
        "plain": {"queries_per_sec": round(len(Qs) / plain_e, 1),
                  "embeddings_per_sec": round(emb / plain_e, 1),
                  "ms_per_pass": round(plain_e * 1e3, 3)},
        "batched": {"queries_per_sec": round(len(Qs) / batch_e, 1),
                    "embeddings_per_sec": round(emb / batch_e, 1),
                    "ms_per_pass": round(batch_e * 1e3, 3)},
        "bit_exact": True}
    # served: Poisson arrivals over the same query stream
    served = []
    rng = np.random.default_rng(7)
    gsm.gsm_server_start(M.ctx, 2, 256)  # captures every batch shape once
    for rate in SERVE_RATES:
        n_req = max(20, int(rate * serve_seconds))
        gaps = rng.exponential(1.0 / rate, n_req)
        order = rng.integers(0, len(Qs), n_req)
        tickets = []
        t_start = time.perf_counter()
        next_t = t_start
        results = {}
        for j in range(n_req):
            next_t += gaps[j]
            wait = next_t - time.perf_counter()
            if wait > 0:
                time.sleep(wait)  # sleeping, not spinning: the server thread stays free
            tickets.append((gsm.gsm_submit(M.ctx, Qs[order[j]].handle), int(order[j])))
        while len(results) < len(tickets):
            for t, qi in tickets:
                if t not in results:
                    r = gsm.gsm_poll(M.ctx, t)
                    if r is not None:
                        results[t] = (r, qi)
            time.sleep(0.0002)
        wall = time.perf_counter() - t_start
        lat = [(r["t_done_ns"] - r["t_submit_ns"]) / 1e6 for r, _ in results.values()]
        ok = all(r["count"] == want[qi] and r["status"] == 0 for r, qi in results.values())
        if not ok:
            raise SystemExit(f"served counts differ from the oracle's at {rate} q/s")
        served.append({"rate_qps": rate, "requests": n_req,
                       "throughput_qps": round(n_req / wall, 1),
                       "embeddings_per_sec": round(sum(want[qi] for _, qi in tickets) / wall, 1),
                       "latency_ms_p50": round(pct(lat, 50), 3),
                       "latency_ms_p99": round(pct(lat, 99), 3)})
    gsm.gsm_server_stop(M.ctx)
    out["served"] = served
    M.close()
    return out


def load_served_workload():
    from paper_2003_01527_gb300 import inputs as I
    with open(GOLDEN_SERVED) as f:
        gold = json.load(f)
    n, rp, col = I.rmat(22, 16, *I.RMAT_ABC, seed=5)
    g = I.make_graph(n, rp, col, I.zipf_labels(n, 32, 1.0, seed=105))
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col, g.labels):
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    if h.hexdigest() != gold["graph"]["sha256"]:
        raise SystemExit("generated R-MAT 22 graph differs from the stored workload")
    return g, gold["queries"]


def served_rmat22(gsm, torch, device, requests_per_rate, rates=SERVED22_RATES):
    """The served form on the resident R-MAT scale-22 graph (4,194,304
    vertices, 32 Zipf(1.0) labels): Poisson arrivals at each rate (the
    configured 50-2,000 queries/s, then 5,000 and 10,000 to find where each
    form saturates), requests drawn from a pool of random-walk queries of
    3-12 vertices on oracle-sized slices, against the plain form (one
    gsm_count per request, run serially on a second context) fed the same
    arrival stream.  Every count is checked against the oracle's."""
    g, queries = load_served_workload()
    S = gsm.Matcher(device=device)  # serves
    P = gsm.Matcher(device=device)  # plain, serial
    S.load_graph(g.row_ptr, g.col, g.labels, validate=True)
    P.load_graph(g.row_ptr, g.col, g.labels)
    def make_q(m, q):
        Q = m.query(q["k"], q["edges"], q["labels"]).restrict(0, 0, q["root_hi"])
        for u in range(1, q["k"]):
            Q.restrict(u, 0, q["window"])
        return Q

    SQ = [make_q(S, q) for q in queries]
    PQ = [make_q(P, q) for q in queries]
    want = [q["count"] for q in queries]
    if [P.count(Q) for Q in PQ] != want:
        raise SystemExit("R-MAT 22 plain counts differ from the oracle's")
    del g
    rng = np.random.default_rng(9)
    gsm.gsm_server_start(S.ctx, 2, 256)
    rows = []
    for rate in rates:
        n_req = requests_per_rate
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
        pick = rng.integers(0, len(queries), n_req)
        emb = int(sum(want[j] for j in pick))
        # served: submit at the arrival times, results polled afterwards
        # (latency = the library's submit -> done timestamps)
        tickets = []
        t0 = time.perf_counter()
        for a, j in zip(arrivals, pick):
            wait = t0 + a - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            tickets.append((gsm.gsm_submit(S.ctx, SQ[j].handle), int(j)))
        results = {}
        while len(results) < len(tickets):
            for t, j in tickets:
                if t not in results:
                    r = gsm.gsm_poll(S.ctx, t)
                    if r is not None:
                        results[t] = (r, j)
            time.sleep(0.0002)
        last_done = max(r["t_done_ns"] for r, _ in results.values())
        first_sub = min(r["t_submit_ns"] for r, _ in results.values())
        wall_s = (last_done - first_sub) / 1e9
        if not all(r["status"] == 0 and r["count"] == want[j] for r, j in results.values()):
            raise SystemExit(f"served R-MAT 22 counts differ from the oracle's at {rate} q/s")
        lat = [(r["t_done_ns"] - r["t_submit_ns"]) / 1e6 for r, _ in results.values()]
        # plain, serially, on the same arrival stream
        plat = []
        t0 = time.perf_counter()
        done = t0
        for a, j in zip(arrivals, pick):
            arr = t0 + a
            wait = arr - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            if P.count(PQ[j]) != want[j]:
                raise SystemExit(f"plain R-MAT 22 count differs at {rate} q/s")
            done = time.perf_counter()
            plat.append((done - arr) * 1e3)
        pwall = done - (t0 + arrivals[0])
        rows.append({"rate_qps": rate, "requests": n_req, "embeddings": emb,
                     "served": {"throughput_qps": round(n_req / wall_s, 1),
                                "embeddings_per_sec": round(emb / wall_s, 1),
                                "latency_ms_p50": round(pct(lat, 50), 3),
                                "latency_ms_p99": round(pct(lat, 99), 3)},
                     "plain_serial": {"throughput_qps": round(n_req / pwall, 1),
                                      "embeddings_per_sec": round(emb / pwall, 1),
                                      "latency_ms_p50": round(pct(plat, 50), 3),
                                      "latency_ms_p99": round(pct(plat, 99), 3)}})
    gsm.gsm_server_stop(S.ctx)
    st = S.batch_stats()
    S.close()
    P.close()
    ks = sorted({q["k"] for q in queries})
    return {"workload": "R-MAT scale 22 (4,194,304 vertices, edge factor 16), 32 Zipf(1.0) "
                        f"labels, resident; a pool of {len(queries)} random-walk queries of "
                        f"{ks[0]}-{ks[-1]} vertices (induced edges), every query vertex "
                        f"restricted to ids below {queries[0]['window']} and the root to an "
                        "oracle-sized prefix",
            "lanes": 2, "max_batch": 256, "batches": st["batches"],
            "bit_exact": True, "rates": rows}


def compressed_frontiers(gsm, torch, device, g, queries, steps):
    """The same query slices with compressed partial results (frontier rows
    as (parent row, new vertex)): time per step, peak budgeted frontier memory
    against the uncompressed path, rows checked against the oracle digests."""
    out = {}
    for name, compressed in (("columns", False), ("compressed", True)):
        M = gsm.Matcher(device=device, compressed=compressed)
        M.load_graph(g.row_ptr, g.col, g.labels)
        Qs = [M.query(q["k"], q["edges"], q["labels"]).restrict(0, 0, q["root_hi"])
              for q in queries]
        outs = [torch.empty(max(q["count"], 1) * q["k"], dtype=torch.int32, device="cuda")
                for q in queries]
        peak = 0
        for Q, o in zip(Qs, outs):  # one query per call: the peak of each
            M.enumerate(Q, out=o)
            peak = max(peak, M.last_run_stats()["peak_bytes"])
        for q, o in zip(queries, outs):
            rows = o[:q["count"] * q["k"]].cpu().numpy().astype("<i4")
            if hashlib.sha256(rows.tobytes()).hexdigest() != q["rows_sha256"]:
                raise SystemExit(f"{name} frontiers: result mismatch on a query slice")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(M.stream)
        for _ in range(steps):
            counts = M.enumerate_many(Qs, outs)
        ev1.record(M.stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        out[name] = {"ms_per_step": round(ms, 3),
                     "embeddings_per_sec": round(sum(counts) / (ms / 1e3), 1),
                     "peak_budgeted_bytes": int(peak)}
        M.close()
    out["bit_exact"] = True
    return out


def lookahead_leg(gsm, torch, device, g, queries, steps):
    """The same query slices with the k-look-ahead of Sec. 3.2 off, at 1 and
    at 2: candidates checked and partial embeddings kept over all levels,
    and time per step; rows checked against the oracle digests."""
    out = {}
    for la in (0, 1, 2):
        M = gsm.Matcher(device=device, lookahead=la)
        M.load_graph(g.row_ptr, g.col, g.labels)
        Qs = [M.query(q["k"], q["edges"], q["labels"]).restrict(0, 0, q["root_hi"])
              for q in queries]
        outs = [torch.empty(max(q["count"], 1) * q["k"], dtype=torch.int32, device="cuda")
                for q in queries]
        cand, kept = 0, 0
        for Q, o, q in zip(Qs, outs, queries):
            M.enumerate(Q, out=o)
            st = M.last_run_stats()
            cand += sum(st["candidates"])
            kept += sum(st["frontier"][1:q["k"]])
            rows = o[:q["count"] * q["k"]].cpu().numpy().astype("<i4")
            if hashlib.sha256(rows.tobytes()).hexdigest() != q["rows_sha256"]:
                raise SystemExit(f"look-ahead {la}: result mismatch on a query slice")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(M.stream)
        for _ in range(steps):
            counts = M.enumerate_many(Qs, outs)
        ev1.record(M.stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        out[f"lookahead_{la}"] = {"ms_per_step": round(ms, 3),
                                  "embeddings_per_sec": round(sum(counts) / (ms / 1e3), 1),
                                  "candidates_checked": int(cand),
                                  "partial_embeddings_kept": int(kept)}
        M.close()
    out["bit_exact"] = True
    return out


def unlabelled_counts(gsm, torch, device, ordered_k4=True):
    """Unlabelled R-MAT scale 20 (1,048,576 vertices, edge factor 16): the
    ordered 3-path count pinned by sum d(d-1); ordered and distinct
    (symmetry-broken) triangle counts and distinct and ordered 4-clique
    counts, pinned by the oracle's clique listing stored in
    tests/golden/rmat20_unlabelled.json (ordered = k! x cliques); and the
    5-cycle and 6-path on the stored root slices, each count equal to the
    oracle's."""
    from paper_2003_01527_gb300 import inputs as I
    g = I.rmat_unlabelled_graph(scale=20, seed=3)
    with open(GOLDEN_RMAT20) as f:
        gold = json.load(f)
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col, g.labels):
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    if h.hexdigest() != gold["graph"]["sha256"]:
        raise SystemExit("generated R-MAT 20 graph differs from the stored workload")
    tri_n, k4_n = gold["cliques"]["3"], gold["cliques"]["4"]
    d = g.degrees()
    M = gsm.Matcher(device=device)
    M.load_graph(g.row_ptr, g.col, g.labels)
    s = I.unlabelled_shapes()
    out = {"workload": "R-MAT scale 20 (1,048,576 vertices, edge factor 16), unlabelled",
           "nnz": g.nnz, "pins": "3-path: sum d(d-1); triangle, 4-clique: k! x the oracle's "
                                 "clique count; 5-cycle, 6-path slices: the oracle's counts"}

    def timed(fn):
        fn()  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, (time.perf_counter() - t0) * 1e3

    p3 = M.query(3, [(0, 1), (1, 2)])
    c, ms = timed(lambda: M.count(p3))
    if c != int((d * (d - 1)).sum()):
        raise SystemExit("3-path count differs from sum d(d-1)")
    out["path3"] = {"ordered": c, "ms": round(ms, 3), "embeddings_per_sec": round(c / ms * 1e3, 1)}
    q = M.query(3, s["triangle"].edges)
    c, ms = timed(lambda: M.count(q))
    (dc, aut), dms = timed(lambda: M.count_distinct(q))
    if c != 6 * tri_n or dc != tri_n or aut != 6:
        raise SystemExit("triangle counts differ from the oracle's clique count")
    out["triangle"] = {"ordered": c, "ordered_ms": round(ms, 3),
                       "ordered_embeddings_per_sec": round(c / ms * 1e3, 1),
                       "distinct": dc, "automorphisms": aut, "distinct_ms": round(dms, 3)}
    q = M.query(4, s["clique4"].edges)
    (dc, aut), dms = timed(lambda: M.count_distinct(q))
    if dc != k4_n or aut != 24:
        raise SystemExit("distinct 4-clique count differs from the oracle's clique count")
    out["clique4"] = {"distinct": dc, "automorphisms": aut, "distinct_ms": round(dms, 3)}
    if ordered_k4:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c = M.count(q)
        ms = (time.perf_counter() - t0) * 1e3
        if c != 24 * k4_n:
            raise SystemExit("ordered 4-clique count differs from 4! x the oracle's")
        out["clique4"].update({"ordered": c, "ordered_ms": round(ms, 1),
                               "ordered_embeddings_per_sec": round(c / ms * 1e3, 1)})
    slices = []
    for sl in gold["slices"]:
        qs = s[sl["shape"]]
        Q = M.query(qs.k, qs.edges).restrict(0, sl["root_lo"], sl["root_hi"])
        if sl["window"]:
            for u in range(1, qs.k):
                Q.restrict(u, 0, sl["window"])
        c, ms = timed(lambda: M.count(Q))
        if c != sl["count"]:
            raise SystemExit(f"{sl['shape']} slice count differs from the oracle's")
        slices.append({"shape": sl["shape"], "roots": [sl["root_lo"], sl["root_hi"]],
                       "other_vertices_below": sl["window"], "ordered": c,
                       "ms": round(ms, 3), "embeddings_per_sec": round(c / ms * 1e3, 1)})
    out["slices"] = slices
    M.close()
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.mark = 0

    def start(self, settle_s: float = 5.0):
        """Starts nvidia-smi and returns once its first sample is in (at most
        settle_s), so that its start-up does not overlap the timed steps."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while not self.lines and self.proc.poll() is None and time.time() - t0 < settle_s:
            time.sleep(0.005)
        self.mark = len(self.lines)  # samples from here on belong to the timed region

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self, wait_s: float = 0.5):
        """Ends sampling; the record is the samples taken since start()
        returned (waiting up to wait_s for one when the timed region was
        shorter than the sampling interval)."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t0 = time.time()
        while len(self.lines) <= self.mark and self.proc.poll() is None and \
                time.time() - t0 < wait_s:
            time.sleep(0.005)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.mark:]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def combine_ranks(ms_per_step, embeddings_per_step, queries, world, dist=None, device="cpu"):
    """Whole-job figures of `world` replicas (every rank runs the same
    workload on its own GPU; no data-path collective): the step time is the
    maximum over ranks, throughput counts every rank's work."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms_per_step], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_per_step = float(t.item())
    value = embeddings_per_step * world / (ms_per_step / 1e3)
    qps = queries * world / (ms_per_step / 1e3)
    return ms_per_step, value, qps


def rank_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------- GPU arm


def run_gpu(args):
    import torch
    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2003_01527_gb300 import build
    build.build()
    from paper_2003_01527_gb300 import gsm

    g, queries = load_workload()
    if args.queries:
        keep = [int(x) for x in args.queries.split(",")]
        queries = [queries[i] for i in keep]
    # two contexts on the same graph: M (no per-kernel events, six host
    # workers) is timed for the headline; MK records CUDA events around every
    # kernel and lists the queries one after the other (so no other query's
    # kernels fall between a kernel's events), timed in a second pass for the
    # per-kernel split and the roofline
    M = gsm.Matcher(device=local, time_kernels=False, filter_rounds=args.filter_rounds,
                    block_size=args.block_size)
    MK = gsm.Matcher(device=local, time_kernels=True, filter_rounds=args.filter_rounds,
                     block_size=args.block_size, host_workers=1)
    M.load_graph(g.row_ptr, g.col, g.labels, validate=True)
    MK.load_graph(g.row_ptr, g.col, g.labels)
    Qs = [M.query(q["k"], q["edges"], q["labels"]).restrict(0, 0, q["root_hi"]) for q in queries]
    QKs = [MK.query(q["k"], q["edges"], q["labels"]).restrict(0, 0, q["root_hi"])
           for q in queries]
    outs = [torch.empty(max(q["count"], 1) * q["k"], dtype=torch.int32, device="cuda")
            for q in queries]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    def step(m, qs):
        # one gsm_enumerate_many call: every query slice listed into its
        # device buffer, each copy overlapping the following queries
        counts = m.enumerate_many(qs, outs)
        return sum(counts), m.last_run_stats()["kernel_launches"]

    # warm-up, and bit-exact check against the stored oracle digests
    for _ in range(max(args.warmup, 3)):
        step(M, Qs)
        step(MK, QKs)
    for m, qs in ((M, Qs), (MK, QKs)):
        for q, Q, out in zip(queries, qs, outs):
            _, c = m.enumerate(Q, out=out)
            rows = out[:c * q["k"]].cpu().numpy().astype("<i4")
            if c != q["count"] or hashlib.sha256(rows.tobytes()).hexdigest() != q["rows_sha256"]:
                raise SystemExit(f"result mismatch on a query slice (count {c} vs {q['count']})")

    def timed_steps(m, qs, clocks=False):
        """K steps, L2 flushed before each, CUDA events on the library's stream."""
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.start()
        ms, emb, nl = 0.0, 0, 0
        for _ in range(args.steps):
            flush.fill_(1)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(m.stream)
            e, l = step(m, qs)
            ev1.record(m.stream)
            torch.cuda.synchronize()
            ms += ev0.elapsed_time(ev1)
            emb += e
            nl += l
        ck = sampler.stop() if sampler else None
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        return ms, emb, nl, ck

    ms_total, embeddings, launches, clocks = timed_steps(M, Qs, clocks=True)
    MK.kernel_stats(reset=True)
    ms_k, _, _, _ = timed_steps(MK, QKs)
    kstats = MK.kernel_stats(reset=True)
    MK.close()
    # the probe term of the byte model (binary-search bytes of the non-tree
    # edge checks) is counted on a third context, one untimed step, so that
    # counting costs the timed pass nothing; it is the same every step
    MP = gsm.Matcher(device=local, count_probes=True, host_workers=1)
    MP.load_graph(g.row_ptr, g.col, g.labels)
    MP.kernel_stats(reset=True)
    step(MP, [MP.query(q["k"], q["edges"], q["labels"]).restrict(0, 0, q["root_hi"])
              for q in queries])
    probe_step = {s["name"]: s["probe_bytes"] for s in MP.kernel_stats(reset=True)}
    MP.close()
    for s in kstats:
        pb = probe_step.get(s["name"], 0.0) * args.steps
        s["probe_bytes"] = pb
        s["algo_bytes"] += pb

    per_step = embeddings / args.steps
    ms_per_step, value, qps = combine_ranks(ms_total / args.steps, per_step, len(queries), world,
                                            dist, device="cuda")

    # dominant kernel and its roofline
    dom = max(kstats, key=lambda s: s["total_ms"])
    peak, peak_kind = peaks()
    achieved = dom["algo_bytes"] / (dom["total_ms"] / 1e3) / 1e9 if dom["total_ms"] else 0.0
    # the same without the byte model's binary-search probe term (the non-tree
    # edge checks), for comparison with the model that left it out
    achieved_np = ((dom["algo_bytes"] - dom.get("probe_bytes", 0.0)) / (dom["total_ms"] / 1e3)
                   / 1e9 if dom["total_ms"] else 0.0)
    # DRAM bytes per launch of the dominant kernel from an ncu capture
    # (profiles/traffic.json); null when the kernel's source file changed since
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            with open(prof) as f:
                tr = json.load(f).get(dom["name"])
            if tr:
                h = hashlib.sha256()
                for name in tr["sources"]:
                    with open(os.path.join(ROOT, "paper_2003_01527_gb300", "csrc", name),
                              "rb") as f:
                        h.update(f.read())
                if tr.get("sources_sha256") == h.hexdigest():
                    traffic = tr["dram_bytes_per_launch"]
        except Exception:
            traffic = None

    # end to end through the public API with host buffers: graph upload from
    # pinned host memory, every query listed by gsm_enumerate_many into pinned
    # host memory (the copy of one query's rows overlaps the next query)
    pin = {k: torch.from_numpy(getattr(g, k)).pin_memory() for k in ("row_ptr", "col", "labels")}
    host_out = [torch.empty(max(q["count"], 1) * q["k"], dtype=torch.int32).pin_memory()
                for q in queries]
    h2d = sum(t.numel() * 4 for t in pin.values())
    d2h = sum(q["count"] * q["k"] * 4 for q in queries)
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        M.load_graph(pin["row_ptr"].numpy(), pin["col"].numpy(), pin["labels"].numpy())
        M.enumerate_many(Qs, host_out)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value = per_step * world / (statistics.median(e2e_ms) / 1e3)
    for q, out in zip(queries, host_out):
        rows = out[:q["count"] * q["k"]].numpy().astype("<i4")
        if hashlib.sha256(rows.tobytes()).hexdigest() != q["rows_sha256"]:
            raise SystemExit("end-to-end result mismatch on a query slice")

    cpu = cpu_baseline(g, queries) if (rank == 0 and world == 1 and not args.no_cpu) else None
    batched = None
    unlabelled = None
    compressed = None
    lookahead = None
    if not args.queries:
        compressed = compressed_frontiers(gsm, torch, local, g, queries, 5)
        lookahead = lookahead_leg(gsm, torch, local, g, queries, 5)
    served22 = None
    if not args.no_batch and not args.queries:
        batched = batched_and_served(gsm, torch, local, args.serve_seconds)
        unlabelled = unlabelled_counts(gsm, torch, local, ordered_k4=not args.no_ordered_k4)
    if not args.no_serve22 and not args.queries:
        served22 = served_rmat22(gsm, torch, local, args.serve22_requests)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded R-MAT + random-walk queries)",
        "config": {"workload": WORKLOAD, "queries": len(queries),
                   "embeddings_per_step": per_step, "mode": "enumerate, sorted rows on device",
                   "l2": "flushed (512 MB write) before every timed step",
                   "filter_rounds": args.filter_rounds,
                   "block_size": args.block_size or 256,
                   "parallelism": f"replicas x{world}"},
        "queries_per_sec": round(qps, 2),
        "roofline": {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "peak_source": peak_kind,
                     "probe_GB": round(dom.get("probe_bytes", 0.0) / 1e9, 4),
                     "frac_without_probe_term": round(achieved_np / peak, 4)},
        "kernels": {s["name"]: {"launches": s["launches"], "ms": round(s["total_ms"], 3),
                                "algo_GB": round(s["algo_bytes"] / 1e9, 4),
                                "probe_GB": round(s.get("probe_bytes", 0.0) / 1e9, 4)}
                    for s in kstats if s["launches"]},
        "kernel_split": {"note": "per-kernel CUDA events on every launch, from a second "
                                 "timed pass of the same steps with one host worker (the "
                                 "headline pass records no per-kernel events and lists "
                                 "with the default six workers)",
                         "ms_per_step_with_events": round(ms_k / args.steps, 4)},
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(statistics.median(e2e_ms), 3)},
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "batched_vs_plain": batched,
        "unlabelled_counts": unlabelled,
        "compressed_frontiers": compressed,
        "lookahead": lookahead,
        "served_rmat22": served22,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    M.close()
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------------- CPU oracle


# The oracle's sample of the plain workload: the first 1/16 of the root range
# of every non-empty query slice (a fixed list, the same for every step and
# for both CPU legs), and, for the single-core figure, the first five of
# those sub-slices.
ORACLE_SAMPLE_DIV = 16
ORACLE_ONE_CORE_SLICES = 5


def oracle_slices(queries, one_core=False):
    out = [(i, max(1, q["root_hi"] // ORACLE_SAMPLE_DIV)) for i, q in enumerate(queries)
           if q["count"] > 0]
    return out[:ORACLE_ONE_CORE_SLICES] if one_core else out


def oracle_sample(g, queries, one_core=False):
    """The oracle on its fixed sample (oracle_slices): (embeddings listed and
    sorted, seconds, slice names, threads used)."""
    import oracle
    from paper_2003_01527_gb300 import inputs as I
    nthreads = 1 if one_core else 0
    t_total, emb, used = 0.0, 0, []
    for i, hi in oracle_slices(queries, one_core):
        q = queries[i]
        qq = I.query_from_edges(q["k"], q["edges"], q["labels"])
        t0 = time.perf_counter()
        c, _, rc = oracle.match(g, qq, enumerate=True, root_range=(0, hi), nthreads=nthreads)
        t_total += time.perf_counter() - t0
        emb += c
        used.append(f"q{i}[0,{hi})")
    return emb, t_total, used, (1 if one_core else oracle.max_threads())


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(g, queries):
    emb, secs, used, cores = oracle_sample(g, queries)
    emb1, secs1, used1, _ = oracle_sample(g, queries, one_core=True)
    return {"value": round(emb / secs, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(used)} query slices, first 1/{ORACLE_SAMPLE_DIV} of each root range "
                      f"({', '.join(used)}): {emb} embeddings listed and sorted in {secs:.2f} s",
            "one_core": {"value": round(emb1 / secs1, 1), "cores": 1,
                         "sample": f"{', '.join(used1)}: {emb1} embeddings in {secs1:.2f} s"},
            "cpu_model": cpu_model(), "nproc": os.cpu_count()}


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    g, queries = load_workload()
    for _ in range(args.warmup):
        oracle_sample(g, queries)
    emb, secs = 0, 0.0
    samples, cores = [], 0
    for _ in range(args.steps):
        e, t, used, cores = oracle_sample(g, queries)
        emb += e
        secs += t
        samples = used
    value = emb / secs
    sample = (f"{len(samples)} query slices, first 1/{ORACLE_SAMPLE_DIV} of each root range "
              f"({', '.join(samples)}), the same every step")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(secs / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded R-MAT + random-walk queries)",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores,
                         "kind": "oracle", "sample": sample, "cpu_model": cpu_model(),
                         "nproc": os.cpu_count()},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gsm", choices=["gsm", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched and served measurements")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="seconds of Poisson arrivals per served rate (R-MAT 18 leg)")
    ap.add_argument("--no-serve22", action="store_true",
                    help="skip the served R-MAT 22 leg")
    ap.add_argument("--serve22-requests", type=int, default=2000,
                    help="requests per arrival rate of the served R-MAT 22 leg")
    ap.add_argument("--no-ordered-k4", action="store_true",
                    help="skip the ordered 4-clique count of the R-MAT 20 leg")
    ap.add_argument("--filter-rounds", type=int, default=0,
                    help="candidate refinement rounds after the first filter pass")
    ap.add_argument("--block-size", type=int, default=0,
                    help="threads per CTA of the verification kernels (0 = the library's)")
    ap.add_argument("--queries", default="",
                    help="comma-separated query indices (a smaller case for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
