"""Exhaustive search over all injective maps -- TEST INFRASTRUCTURE ONLY.

Pins the backtracking oracle on tiny graphs (n <= 9, k <= 5): every one of the
n!/(n-k)! injective maps V(Q) -> V(G) is tested against the definition of an
embedding (Sec. 1 / Sec. 3.2 of the paper: label preserving and edge
preserving, non-induced), with no pruning and no ordering.  Pure Python on
purpose: it shares nothing with the C++ backtracker.
"""
from __future__ import annotations

import itertools

import numpy as np


def adjacency_sets(g):
    return [set(int(x) for x in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]) for v in range(g.n)]


def embeddings(g, q) -> list[tuple[int, ...]]:
    adj = adjacency_sets(g)
    lab = [int(x) for x in g.labels]
    qlab = [int(x) for x in q.labels]
    qedges = [(int(a), int(b)) for a, b in np.asarray(q.edges).reshape(-1, 2)]
    out = []
    for f in itertools.permutations(range(g.n), q.k):
        if any(lab[f[u]] != qlab[u] for u in range(q.k)):
            continue
        if all(f[b] in adj[f[a]] for a, b in qedges):
            out.append(tuple(f))
    out.sort()
    return out
