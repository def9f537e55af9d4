"""The C ABI library: loads, exports every declared entry point, and its host
logic (query validation, matching order) behaves as documented.  No device
work here."""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gsm_\w+)\s*\(", src))
    return names - {"gsm_alloc_fn", "gsm_free_fn"}


def test_library_exports_every_declared_symbol(gsm_lib):
    lib = ctypes.CDLL(gsm_lib.LIB_PATH)
    declared = declared_entry_points()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(gsm_lib.EXPORTED)


def header_constants():
    """Every integer #define of include/gsm.h, evaluated (plain literals,
    parenthesised negatives, unsigned shifts)."""
    out = {}
    src = open(os.path.join(ROOT, "include", "gsm.h")).read()
    for name, expr in re.findall(r"^#define\s+(GSM_\w+)\s+([^/\n]+)", src, flags=re.M):
        expr = re.sub(r"(\d+)u\b", r"\1", expr.strip())
        if re.fullmatch(r"[\d\s()<\-+]+", expr):
            out[name] = eval(expr)  # integer literal arithmetic only (checked above)
    return out


def test_binding_constants_match_the_header(gsm_lib):
    consts = header_constants()
    assert {"GSM_OK", "GSM_ERR_TIMEOUT", "GSM_OPT_INJECT_SCAN_STALL",
            "GSM_STATIC_SCRATCH_BITMAP_BYTES"} <= set(consts)
    for name, value in consts.items():
        assert getattr(gsm_lib, name) == value, name
    # the option flags are distinct bits
    flags = [v for n, v in consts.items() if n.startswith("GSM_OPT_")]
    assert all(f > 0 and f & (f - 1) == 0 for f in flags)
    assert len(set(flags)) == len(flags)


def test_status_strings(gsm_lib):
    assert gsm_lib.gsm_status_string(0) == "GSM_OK"
    assert gsm_lib.gsm_status_string(-6) == "GSM_ERR_BUDGET"
    assert gsm_lib.gsm_status_string(-99) == "GSM_ERR_UNKNOWN"
    # every status the header defines has its own name
    for name, value in header_constants().items():
        if name == "GSM_OK" or name == "GSM_PENDING" or name.startswith("GSM_ERR_"):
            assert gsm_lib.gsm_status_string(value) == name, name


def test_query_validation_without_device(gsm_lib):
    g = gsm_lib
    e = np.array([0, 1, 1, 2], np.int32)
    q = g.gsm_query_create(None, 3, 2, e, None)
    g.gsm_query_destroy(q)
    bad = [
        (0, np.zeros(0, np.int32)),                       # k = 0
        (17, np.array([0, 1], np.int32)),                 # k > 16
        (3, np.array([0, 1], np.int32)),                  # disconnected
        (3, np.array([0, 1, 1, 0, 1, 2], np.int32)),      # duplicate edge
        (2, np.array([0, 0, 0, 1], np.int32)),            # self-loop
        (2, np.array([0, 2], np.int32)),                  # out of range
    ]
    for k, edges in bad:
        with pytest.raises(g.GsmError) as ei:
            g.gsm_query_create(None, k, edges.size // 2, edges if edges.size else None, None)
        assert ei.value.status == g.GSM_ERR_INVALID_QUERY


def test_restrict_rejects_bad_ranges(gsm_lib):
    g = gsm_lib
    q = g.gsm_query_create(None, 2, 1, np.array([0, 1], np.int32), None)
    g.gsm_query_restrict(q, 0, 5, 9)
    for u, lo, hi in [(2, 0, 1), (-1, 0, 1), (0, 5, 4), (0, -1, 3)]:
        with pytest.raises(g.GsmError):
            g.gsm_query_restrict(q, u, lo, hi)
    g.gsm_query_destroy(q)


def _check_order(k, edges, sizes, order, parent):
    adj = [set() for _ in range(k)]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    assert sorted(order.tolist()) == list(range(k))
    pos = {u: i for i, u in enumerate(order.tolist())}
    assert parent[0] == -1
    for i in range(1, k):
        u = order[i]
        earlier = [j for j in range(i) if order[j] in adj[u]]
        assert earlier, "order must follow a spanning tree"
        assert parent[i] == min(earlier)
    # first vertex: fewest candidates, then larger degree, then lower id
    key = lambda u: (sizes[u], -len(adj[u]), u)
    assert order[0] == min(range(k), key=key)
    placed = {order[0]}
    for i in range(1, k):
        cand = [u for u in range(k) if u not in placed and adj[u] & placed]
        best = min(cand, key=lambda u: (-len(adj[u] & placed), sizes[u], -len(adj[u]), u))
        assert order[i] == best
        placed.add(order[i])


def test_plan_order_rules(gsm_lib):
    rng = np.random.default_rng(0)
    for _ in range(200):
        k = int(rng.integers(1, 11))
        edges = {(int(rng.integers(0, v)), v) for v in range(1, k)}
        for a, b in itertools.combinations(range(k), 2):
            if rng.random() < 0.25:
                edges.add((a, b))
        edges = sorted(edges)
        sizes = rng.integers(1, 50, k).astype(np.uint64)
        order, parent = gsm_lib.gsm_plan_order(k, edges, sizes)
        _check_order(k, edges, sizes.tolist(), order, parent)


def test_plan_order_example(gsm_lib):
    # 4-cycle 0-1-2-3 with chord 1-3; vertex 2 has the fewest candidates
    order, parent = gsm_lib.gsm_plan_order(4, [(0, 1), (1, 2), (2, 3), (3, 0), (1, 3)],
                                           [10, 10, 3, 10])
    assert order.tolist() == [2, 1, 3, 0]
    assert parent.tolist() == [-1, 0, 0, 1]
