"""Seeded synthetic inputs for subgraph matching.

This module is shared by the CUDA path's tests, the benchmark and the CPU
oracle's tests.  It draws random graphs and random queries and nothing else:
it holds none of the matching arithmetic (no filtering, ordering, extension or
counting).

Workload shapes follow the paper's experiments (Sec. 4): power-law Kronecker
graphs (Graph500 kron, here R-MAT with a=.57 b=.19 c=.19 d=.05, edge factor
16), a small Erdos-Renyi graph, power-law (Zipf) vertex labels, and query
graphs cut out of the data graph by random walks (the label-scaling test of
Sec. 4.3, after Yan et al.).

Every graph is returned as sorted, symmetric CSR with no self-loops and no
duplicate entries:

    Graph(n, row_ptr int32[n+1], col int32[nnz], labels int32[n])

Every query is

    Query(k, edges int32[m, 2] (undirected, u < v), labels int32[k], walk)

where ``walk`` (int32[k]) is the data-graph vertex each query vertex was cut
from, so ``walk`` is itself one embedding of the query.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col: np.ndarray      # int32[nnz], each row ascending
    labels: np.ndarray   # int32[n]

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)


@dataclasses.dataclass
class Query:
    k: int
    edges: np.ndarray   # int32[m, 2], undirected, u < v, sorted
    labels: np.ndarray  # int32[k]
    walk: np.ndarray | None = None  # int32[k]: the generating embedding

    @property
    def m(self) -> int:
        return int(self.edges.shape[0])


# ---------------------------------------------------------------- graphs


def csr_from_pairs(n: int, src: np.ndarray, dst: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Symmetrise, drop self-loops and duplicates, and build sorted CSR."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    keys = np.concatenate([(src << 32) | dst, (dst << 32) | src])
    keys.sort()  # sorted distinct keys, as np.unique gives, but far faster here
    if keys.shape[0]:
        keep = np.empty(keys.shape[0], dtype=bool)
        keep[0] = True
        np.not_equal(keys[1:], keys[:-1], out=keep[1:])
        keys = keys[keep]
    rows = (keys >> 32).astype(np.int64)
    col = (keys & 0xFFFFFFFF).astype(np.int32)
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("graph too large for int32 CSR")
    return row_ptr.astype(np.int32), col


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 0) -> tuple[int, np.ndarray, np.ndarray]:
    """R-MAT / Graph500-Kronecker edge sampler.

    Draws edge_factor * 2**scale directed pairs; at every bit level the pair
    falls into quadrant a (0,0), b (0,1), c (1,0) or d = 1-a-b-c (1,1), with no
    noise.  Vertex ids are then relabelled by a seeded random permutation,
    which is what Graph500 does to hide the R-MAT locality.  Returns
    (n, row_ptr, col) after symmetrisation, self-loop removal and
    de-duplication.
    """
    rng = np.random.default_rng(seed)
    n = 1 << scale
    m = edge_factor << scale
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for bit in range(scale):
        u = rng.random(m, dtype=np.float32)
        s_bit = u >= ab
        d_bit = ((u >= a) & (u < ab)) | (u >= abc)
        src |= s_bit.astype(np.int64) << bit
        dst |= d_bit.astype(np.int64) << bit
        del u, s_bit, d_bit
    perm = rng.permutation(n).astype(np.int64)
    src = perm[src]
    dst = perm[dst]
    row_ptr, col = csr_from_pairs(n, src, dst)
    return n, row_ptr, col


def erdos_renyi(n: int, num_edges: int, seed: int = 0) -> tuple[int, np.ndarray, np.ndarray]:
    """G(n, M): a uniformly random set of M distinct undirected edges."""
    rng = np.random.default_rng(seed)
    max_edges = n * (n - 1) // 2
    if num_edges > max_edges:
        raise ValueError("too many edges")
    chosen = np.empty(0, dtype=np.int64)
    while chosen.shape[0] < num_edges:
        draw = 2 * (num_edges - chosen.shape[0]) + 16
        u = rng.integers(0, n, draw, dtype=np.int64)
        v = rng.integers(0, n, draw, dtype=np.int64)
        keep = u != v
        lo = np.minimum(u[keep], v[keep])
        hi = np.maximum(u[keep], v[keep])
        keys = np.concatenate([chosen, lo * n + hi])
        # keep first occurrences in draw order
        _, first = np.unique(keys, return_index=True)
        chosen = keys[np.sort(first)]
    chosen = chosen[:num_edges]
    row_ptr, col = csr_from_pairs(n, chosen // n, chosen % n)
    return n, row_ptr, col


def zipf_labels(n: int, num_labels: int, s: float, seed: int) -> np.ndarray:
    """Vertex labels with P(l) proportional to (l+1)^-s, l = 0..L-1."""
    rng = np.random.default_rng(seed)
    if num_labels <= 1:
        return np.zeros(n, dtype=np.int32)
    p = np.arange(1, num_labels + 1, dtype=np.float64) ** (-s)
    p /= p.sum()
    return rng.choice(num_labels, size=n, p=p).astype(np.int32)


def uniform_labels(n: int, num_labels: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, num_labels, n, dtype=np.int64).astype(np.int32)


def make_graph(n: int, row_ptr: np.ndarray, col: np.ndarray, labels: np.ndarray) -> Graph:
    return Graph(n=n, row_ptr=np.ascontiguousarray(row_ptr, dtype=np.int32),
                 col=np.ascontiguousarray(col, dtype=np.int32),
                 labels=np.ascontiguousarray(labels, dtype=np.int32))


def graph_from_edges(n: int, edges, labels=None) -> Graph:
    """Small graphs written out by hand (tests)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    row_ptr, col = csr_from_pairs(n, e[:, 0], e[:, 1])
    if labels is None:
        labels = np.zeros(n, dtype=np.int32)
    return make_graph(n, row_ptr, col, np.asarray(labels, dtype=np.int32))


def has_edge(g: Graph, u: int, v: int) -> bool:
    lo, hi = int(g.row_ptr[u]), int(g.row_ptr[u + 1])
    i = np.searchsorted(g.col[lo:hi], v)
    return bool(i < hi - lo and g.col[lo + i] == v)


# ---------------------------------------------------------------- queries


def query_from_edges(k: int, edges, labels=None) -> Query:
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    lo = np.minimum(e[:, 0], e[:, 1])
    hi = np.maximum(e[:, 0], e[:, 1])
    e = np.unique(np.stack([lo, hi], axis=1), axis=0) if e.shape[0] else e
    if labels is None:
        labels = np.zeros(k, dtype=np.int32)
    return Query(k=k, edges=np.ascontiguousarray(e, dtype=np.int32),
                 labels=np.asarray(labels, dtype=np.int32))


def _walk(g: Graph, k: int, rng: np.random.Generator, starts: np.ndarray):
    """Random walk until k distinct vertices are seen (restart after 100k steps).

    Returns (visited vertices in first-visit order, first-visit tree edges as
    pairs of walk positions)."""
    while True:
        cur = int(starts[rng.integers(0, starts.shape[0])])
        visited = [cur]
        pos = {cur: 0}
        tree = []
        steps = 0
        while len(visited) < k and steps < 100 * k:
            lo, hi = int(g.row_ptr[cur]), int(g.row_ptr[cur + 1])
            nxt = int(g.col[lo + rng.integers(0, hi - lo)])
            if nxt not in pos:
                pos[nxt] = len(visited)
                tree.append((pos[cur], pos[nxt]))
                visited.append(nxt)
            cur = nxt
            steps += 1
        if len(visited) == k:
            return np.asarray(visited, dtype=np.int64), tree


def random_walk_query(g: Graph, k: int, rng: np.random.Generator,
                      non_tree: tuple[int, int] | None = None) -> Query:
    """A connected query of k vertices cut out of g by a random walk.

    non_tree=None: all induced edges among the walked vertices (labels
    inherited).  non_tree=(lo, hi): the walk's first-visit tree edges plus
    min(U{lo..hi}, available) induced non-tree edges; the walk is redrawn up to
    100 times to reach the drawn number, else the best walk is kept.
    """
    deg = g.degrees()
    starts = np.nonzero(deg > 0)[0]
    if starts.shape[0] == 0:
        raise ValueError("graph has no edges")
    want = None if non_tree is None else int(rng.integers(non_tree[0], non_tree[1] + 1))
    best = None
    for _ in range(100 if want is not None else 1):
        verts, tree = _walk(g, k, rng, starts)
        induced = [(i, j) for i in range(k) for j in range(i + 1, k)
                   if has_edge(g, int(verts[i]), int(verts[j]))]
        if want is None:
            edges = induced
            cand = (verts, edges)
            best = cand
            break
        tree_set = {(min(a, b), max(a, b)) for a, b in tree}
        extra = [e for e in induced if e not in tree_set]
        take = min(want, len(extra))
        if take:
            pick = rng.choice(len(extra), size=take, replace=False)
            chosen = [extra[i] for i in sorted(pick)]
        else:
            chosen = []
        cand = (verts, sorted(tree_set) + chosen, take)
        if best is None or take > best[2]:
            best = cand
        if take == want:
            break
    verts, edges = best[0], best[1]
    q = query_from_edges(k, edges, g.labels[verts])
    q.walk = verts.astype(np.int32)
    return q


# ---------------------------------------------------------------- workloads

RMAT_ABC = (0.57, 0.19, 0.19)


def tiny_er_workload(seed: int = 1):
    """ER graph, 2,000 vertices, 8,000 edges (avg degree 8), 4 uniform labels;
    the query is the 4-cycle labelled (0, 1, 0, 2)."""
    n, rp, col = erdos_renyi(2000, 8000, seed=seed)
    g = make_graph(n, rp, col, uniform_labels(n, 4, seed + 100))
    q = query_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)], [0, 1, 0, 2])
    return g, [q]


def rmat_labelled_workload(scale: int = 16, num_labels: int = 8, zipf_s: float = 1.0,
                           num_queries: int = 20, kmin: int = 4, kmax: int = 8,
                           non_tree=None, seed: int = 2):
    """R-MAT graph with Zipf labels and random-walk queries (induced edges by
    default, or tree + non_tree=(lo, hi) extra edges)."""
    n, rp, col = rmat(scale, 16, *RMAT_ABC, seed=seed)
    g = make_graph(n, rp, col, zipf_labels(n, num_labels, zipf_s, seed + 100))
    rng = np.random.default_rng(seed + 200)
    qs = [random_walk_query(g, int(rng.integers(kmin, kmax + 1)), rng, non_tree)
          for _ in range(num_queries)]
    return g, qs


def rmat_unlabelled_graph(scale: int = 20, seed: int = 3) -> Graph:
    n, rp, col = rmat(scale, 16, *RMAT_ABC, seed=seed)
    return make_graph(n, rp, col, np.zeros(n, dtype=np.int32))


def unlabelled_shapes():
    """Triangle, 4-clique, 5-cycle and 6-vertex path, unlabelled."""
    tri = query_from_edges(3, [(0, 1), (1, 2), (0, 2)])
    k4 = query_from_edges(4, [(i, j) for i in range(4) for j in range(i + 1, 4)])
    c5 = query_from_edges(5, [(i, (i + 1) % 5) for i in range(5)])
    p6 = query_from_edges(6, [(i, i + 1) for i in range(5)])
    return {"triangle": tri, "clique4": k4, "cycle5": c5, "path6": p6}
