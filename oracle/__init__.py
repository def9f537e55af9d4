"""CPU oracle for subgraph matching -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package.  The product library never imports, links
or executes it, and the two share no code.

``oracle.cpp`` holds the plain depth-first backtracking matcher (the
definition of Result(Q, G) of Sec. 1 / Sec. 3.2 of the paper, written out)
and the candidate-filter predicate of Sec. 3.2; ``brute.py`` holds the
exhaustive search over all injective maps that pins the backtracker on tiny
graphs.  Every function here is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID_ARG, INVALID_GRAPH, INVALID_QUERY, BUDGET, TRUNCATED, LIMIT = 0, -1, -2, -3, -6, -8, -12


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
            lib.oracle_validate_graph.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p]
            lib.oracle_validate_graph.restype = ctypes.c_int
            lib.oracle_validate_query.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p]
            lib.oracle_validate_query.restype = ctypes.c_int
            lib.oracle_candidates.argtypes = [ctypes.c_int32, i32p, i32p, i32p, ctypes.c_int32,
                                              ctypes.c_int32, i32p, i32p, u8p]
            lib.oracle_candidates.restype = ctypes.c_int
            lib.oracle_match.argtypes = [ctypes.c_int32, i32p, i32p, i32p, ctypes.c_int32,
                                         ctypes.c_int32, i32p, i32p, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32,
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
            lib.oracle_match.restype = ctypes.c_int
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_refine_round.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32,
                                                ctypes.c_int32, i32p, i32p, u8p, u8p]
            lib.oracle_refine_round.restype = ctypes.c_int
            lib.oracle_cliques.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(ctypes.c_uint64)]
            lib.oracle_cliques.restype = ctypes.c_int
            _lib = lib
    return _lib


def _edges(q):
    e = np.ascontiguousarray(np.asarray(q.edges, dtype=np.int32).reshape(-1))
    return e if e.size else np.zeros(1, dtype=np.int32)


def validate_graph(g) -> int:
    return _load().oracle_validate_graph(g.n, g.nnz, g.row_ptr, g.col)


def validate_query(q) -> int:
    return _load().oracle_validate_query(q.k, q.m, _edges(q))


def candidates(g, q) -> np.ndarray:
    """uint8[k, n]: 1 where data vertex v passes the filter for query vertex u."""
    out = np.zeros((q.k, g.n), dtype=np.uint8)
    rc = _load().oracle_candidates(g.n, g.row_ptr, g.col, g.labels, q.k, q.m, _edges(q),
                                   np.ascontiguousarray(q.labels, dtype=np.int32), out)
    if rc != OK:
        raise ValueError(f"oracle_candidates failed: {rc}")
    return out


def refine(g, q, cand: np.ndarray, rounds: int) -> np.ndarray:
    """`rounds` rounds of candidate refinement applied to uint8[k, n] sets."""
    cur = np.ascontiguousarray(cand, dtype=np.uint8)
    for _ in range(rounds):
        nxt = np.zeros_like(cur)
        rc = _load().oracle_refine_round(g.n, g.row_ptr, g.col, q.k, q.m, _edges(q),
                                         np.ascontiguousarray(q.labels, dtype=np.int32), cur, nxt)
        if rc != OK:
            raise ValueError(f"oracle_refine_round failed: {rc}")
        cur = nxt
    return cur


def cliques(g, k: int, nthreads: int = 0) -> int:
    """Number of k-cliques of g (each once), by degree-ordered listing: an
    algorithm independent of ``match``; K_k has k! ordered embeddings per
    clique."""
    lo, hi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = _load().oracle_cliques(g.n, g.row_ptr, g.col, k, nthreads, ctypes.byref(lo),
                                ctypes.byref(hi))
    if rc != OK:
        raise ValueError(f"oracle_cliques failed: {rc}")
    return lo.value + (hi.value << 64)


def max_threads() -> int:
    return _load().oracle_max_threads()


def match(g, q, enumerate: bool = True, root_range=None, cap_rows: int | None = None,
          nthreads: int = 0, limit: int = 0, node_budget: int = 0, ranges=None):
    """Returns (count, rows, status).

    count  -- exact Python int (128-bit on the C side).
    rows   -- int32[min(count, cap), k] sorted lexicographically (enumerate)
              or None.
    root_range -- (lo, hi): only embeddings with f(q_0) in [lo, hi).
    limit / node_budget -- search controls: status LIMIT (more than `limit`
              embeddings) or BUDGET (more than `node_budget` search steps)
              means the search gave up and count is meaningless.
    ranges -- {u: (lo, hi)}: only embeddings with f(u) in [lo, hi) for each
              listed query vertex u.
    """
    lo, hi = (0, g.n) if root_range is None else root_range
    lib = _load()
    qlab = np.ascontiguousarray(q.labels, dtype=np.int32)
    clo, chi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rng_arr = None
    if ranges:
        rng_arr = np.zeros(2 * q.k, dtype=np.int64)
        rng_arr[1::2] = g.n
        for u, (a, b) in ranges.items():
            rng_arr[2 * u], rng_arr[2 * u + 1] = a, b

    def call(enum, out_ptr, cap):
        return lib.oracle_match(g.n, g.row_ptr, g.col, g.labels, q.k, q.m, _edges(q), qlab,
                                lo, hi, enum, out_ptr, cap, ctypes.byref(clo), ctypes.byref(chi),
                                nthreads, limit, node_budget,
                                None if rng_arr is None else rng_arr.ctypes.data)

    if not enumerate:
        rc = call(0, None, 0)
        if rc in (LIMIT, BUDGET):
            return None, None, rc
        if rc != OK:
            raise ValueError(f"oracle_match failed: {rc}")
        return clo.value + (chi.value << 64), None, rc
    if cap_rows is None:
        # a counting pass first so the output buffer can be sized exactly
        rc = call(0, None, 0)
        if rc in (LIMIT, BUDGET):
            return None, None, rc
        if rc != OK:
            raise ValueError(f"oracle_match failed: {rc}")
        cap_rows = clo.value + (chi.value << 64)
    out = np.zeros((max(cap_rows, 1), q.k), dtype=np.int32)
    rc = call(1, out.ctypes.data, cap_rows)
    if rc in (LIMIT, BUDGET):
        return None, None, rc
    if rc not in (OK, TRUNCATED):
        raise ValueError(f"oracle_match failed: {rc}")
    count = clo.value + (chi.value << 64)
    return count, out[:min(count, cap_rows)], rc


def count(g, q, root_range=None, nthreads: int = 0) -> int:
    return match(g, q, enumerate=False, root_range=root_range, nthreads=nthreads)[0]
