// CPU oracle for subgraph matching -- TEST INFRASTRUCTURE ONLY.
//
// This file is the slow, obviously correct reference that the CUDA path is
// checked against.  Only the test suite, the smoke check and the benchmark's
// CPU-baseline leg may load it; the product library never links or calls it,
// and the two share no code (no headers, helpers or tables).
//
// What it computes (Sec. 1 and Sec. 3.2 of the paper: "the enumeration of all
// subgraph isomorphisms" between an undirected labelled data graph G and a
// connected labelled query graph Q):
//
//   Result(Q, G) = { f : V(Q) -> V(G) | f injective,
//                    lab(f(u)) = qlab(u) for every u,
//                    {u,u'} in E(Q)  =>  {f(u),f(u')} in E(G) }
//
// i.e. non-induced embeddings as ordered injective maps, each written as the
// k-tuple (f(q_0), ..., f(q_{k-1})) in query-vertex-id order, the list sorted
// lexicographically.  The count is |Result|.
//
// Algorithm: the depth-first backtracking that Sec. 2 describes for CPU tree
// search (Ullmann-style): query vertices are taken in the BFS order of Q from
// query vertex 0 (neighbours in ascending id), which is deliberately not the
// order the GPU path picks; depth 0 tries every data vertex with the right
// label, depth i tries the neighbours of the image of the BFS parent, and a
// candidate is accepted iff its label matches, it is not yet used, and every
// query edge to an already-placed vertex is present in G.  Rows are sorted
// once at the end.
//
// Also here: the definition of the candidate filter of Sec. 3.2 (label, degree
// and neighbourhood test) written out per (query vertex, data vertex) pair,
// the graph/query validity checks of the library's contract, and an
// independent k-clique counter (degree-ordered listing) that pins the
// matcher's clique counts on graphs too large for the backtracking.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

// error codes mirror the meaning (not the header) of the library's contract
enum { OR_OK = 0, OR_INVALID_ARG = -1, OR_INVALID_GRAPH = -2, OR_INVALID_QUERY = -3,
       OR_BUDGET = -6, OR_TRUNCATED = -8, OR_LIMIT = -12 };

static bool row_has(const int32_t* rp, const int32_t* col, int32_t x, int32_t y) {
  // plain binary search of y in the ascending row of x
  int64_t lo = rp[x], hi = rp[x + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] < y) lo = mid + 1; else hi = mid;
  }
  return lo < rp[x + 1] && col[lo] == y;
}

// A data graph is valid iff its CSR is well formed, every row is strictly
// ascending (sorted, no duplicate), no vertex lists itself, and the pattern is
// symmetric (undirected).
int oracle_validate_graph(int32_t n, int64_t nnz, const int32_t* rp, const int32_t* col) {
  if (n < 0 || nnz < 0) return OR_INVALID_ARG;
  if (rp[0] != 0 || (int64_t)rp[n] != nnz) return OR_INVALID_GRAPH;
  for (int32_t v = 0; v < n; ++v) {
    if (rp[v + 1] < rp[v]) return OR_INVALID_GRAPH;
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      int32_t w = col[e];
      if (w < 0 || w >= n || w == v) return OR_INVALID_GRAPH;
      if (e > rp[v] && col[e - 1] >= w) return OR_INVALID_GRAPH;
    }
  }
  for (int32_t v = 0; v < n; ++v)
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e)
      if (!row_has(rp, col, col[e], v)) return OR_INVALID_GRAPH;
  return OR_OK;
}

// A query is valid iff 1 <= k <= 16, every edge joins two distinct query
// vertices, no undirected edge is listed twice, and Q is connected.
int oracle_validate_query(int32_t k, int32_t m, const int32_t* edges) {
  if (k < 1 || k > 16 || m < 0 || m > k * (k - 1) / 2) return OR_INVALID_QUERY;
  bool adj[16][16] = {};
  for (int32_t e = 0; e < m; ++e) {
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || a >= k || b < 0 || b >= k || a == b) return OR_INVALID_QUERY;
    if (adj[a][b]) return OR_INVALID_QUERY;
    adj[a][b] = adj[b][a] = true;
  }
  bool seen[16] = {};
  int32_t stack[16], top = 0, reached = 1;
  seen[0] = true;
  stack[top++] = 0;
  while (top) {
    int32_t u = stack[--top];
    for (int32_t w = 0; w < k; ++w)
      if (adj[u][w] && !seen[w]) { seen[w] = true; ++reached; stack[top++] = w; }
  }
  return reached == k ? OR_OK : OR_INVALID_QUERY;
}

// Candidate predicate of the filtering step (Sec. 3.2, "filter nodes based on
// Q's (NE, label, deg)"), in its per-label form: v is a candidate for u iff
//   lab(v) = qlab(u),  deg(v) >= deg_Q(u),  and for every label l
//   |{w in N(v): lab(w) = l}| >= |{u' in N_Q(u): qlab(u') = l}|.
// Writes out[u * n + v] = 1 / 0.
int oracle_candidates(int32_t n, const int32_t* rp, const int32_t* col, const int32_t* lab,
                      int32_t k, int32_t m, const int32_t* edges, const int32_t* qlab,
                      uint8_t* out) {
  if (oracle_validate_query(k, m, edges) != OR_OK) return OR_INVALID_QUERY;
  std::vector<std::map<int32_t, int64_t>> need(k);
  std::vector<int64_t> qdeg(k, 0);
  for (int32_t e = 0; e < m; ++e) {
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    qdeg[a]++; qdeg[b]++;
    need[a][qlab[b]]++;
    need[b][qlab[a]]++;
  }
  for (int32_t v = 0; v < n; ++v) {
    std::map<int32_t, int64_t> have;
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) have[lab[col[e]]]++;
    int64_t deg = rp[v + 1] - rp[v];
    for (int32_t u = 0; u < k; ++u) {
      bool ok = lab[v] == qlab[u] && deg >= qdeg[u];
      for (auto& kv : need[u]) {
        auto it = have.find(kv.first);
        int64_t c = it == have.end() ? 0 : it->second;
        if (c < kv.second) ok = false;
      }
      out[(int64_t)u * n + v] = ok ? 1 : 0;
    }
  }
  return OR_OK;
}

// One round of candidate refinement (the repeated local pruning of Sec. 3.2,
// "after each iteration of pruning, NE and degree information of the data
// graph is updated"), in per-label form: v stays a candidate of u iff it was
// one and, for every label l, v has at least as many neighbours in the union
// of the candidate sets of u's query neighbours with label l as u has such
// query neighbours.  cand_in / cand_out: uint8[k * n] (u-major); they may not
// alias.
int oracle_refine_round(int32_t n, const int32_t* rp, const int32_t* col, int32_t k, int32_t m,
                        const int32_t* edges, const int32_t* qlab, const uint8_t* cand_in,
                        uint8_t* cand_out) {
  if (oracle_validate_query(k, m, edges) != OR_OK) return OR_INVALID_QUERY;
  bool adj[16][16] = {};
  for (int32_t e = 0; e < m; ++e) {
    adj[edges[2 * e]][edges[2 * e + 1]] = true;
    adj[edges[2 * e + 1]][edges[2 * e]] = true;
  }
  for (int32_t u = 0; u < k; ++u) {
    // query neighbours of u grouped by label
    std::map<int32_t, std::vector<int32_t>> groups;
    for (int32_t w = 0; w < k; ++w)
      if (adj[u][w]) groups[qlab[w]].push_back(w);
    for (int32_t v = 0; v < n; ++v) {
      bool keep = cand_in[(int64_t)u * n + v] != 0;
      for (auto& gr : groups) {
        if (!keep) break;
        int64_t have = 0;
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
          const int32_t x = col[e];
          bool in_union = false;
          for (int32_t w : gr.second) in_union = in_union || cand_in[(int64_t)w * n + x] != 0;
          if (in_union) ++have;
        }
        if (have < (int64_t)gr.second.size()) keep = false;
      }
      cand_out[(int64_t)u * n + v] = keep ? 1 : 0;
    }
  }
  return OR_OK;
}

struct Search {
  const int32_t* rp;
  const int32_t* col;
  const int32_t* lab;
  const int32_t* qlab;
  int32_t k;
  int32_t order[16];
  int32_t parent[16];      // BFS parent (query id) of order[i], -1 for the root
  bool adj[16][16];
  bool enumerate;
  int64_t rlo[16], rhi[16];  // f(u) must lie in [rlo[u], rhi[u])
  // search controls (not part of the definition): stop once more than
  // `limit` embeddings or more than `node_budget` search steps (nodes entered
  // plus candidates examined) were taken
  uint64_t limit, node_budget;
  mutable std::atomic<uint64_t> shared_count{0}, shared_nodes{0};
  mutable std::atomic<int> stop{0};  // 1 = limit exceeded, 2 = budget exceeded
};

struct Worker {
  const Search* s;
  int32_t f[16];           // f[query id] = data vertex
  unsigned __int128 count = 0;
  uint64_t pend_count = 0, pend_nodes = 0;
  std::vector<int32_t> rows;

  void flush() {
    const Search& S = *s;
    uint64_t c = S.shared_count.fetch_add(pend_count) + pend_count;
    uint64_t nd = S.shared_nodes.fetch_add(pend_nodes) + pend_nodes;
    pend_count = pend_nodes = 0;
    if (S.limit && c > S.limit) S.stop.store(1);
    if (S.node_budget && nd > S.node_budget) S.stop.store(2);
  }

  void dfs(int32_t depth) {
    const Search& S = *s;
    if (S.stop.load(std::memory_order_relaxed)) return;
    if (++pend_nodes >= 4096) flush();
    if (depth == S.k) {
      ++count;
      if (++pend_count >= 4096) flush();
      if (S.enumerate) rows.insert(rows.end(), f, f + S.k);
      return;
    }
    int32_t u = S.order[depth];
    int32_t p = f[S.parent[u]];
    for (int64_t e = S.rp[p]; e < S.rp[p + 1]; ++e) {
      int32_t w = S.col[e];
      // every examined candidate counts towards the search budget, so a
      // node that scans a hub row is bounded too
      if (++pend_nodes >= 4096) {
        flush();
        if (S.stop.load(std::memory_order_relaxed)) return;
      }
      if (S.lab[w] != S.qlab[u]) continue;
      if (w < S.rlo[u] || w >= S.rhi[u]) continue;
      bool ok = true;
      for (int32_t j = 0; j < depth && ok; ++j) {
        int32_t uj = S.order[j];
        if (f[uj] == w) ok = false;
        else if (S.adj[u][uj] && !row_has(S.rp, S.col, f[uj], w)) ok = false;
      }
      if (!ok) continue;
      f[u] = w;
      dfs(depth + 1);
    }
  }
};

// Counts (and with enumerate != 0, lists) Result(Q, G) restricted to
// f(q_0) in [root_lo, root_hi).  The count is returned as two 64-bit halves of
// an unsigned 128-bit integer.  Rows are written sorted, at most cap_rows of
// them; OR_TRUNCATED if more exist.  nthreads <= 0 uses every core.
// ranges (may be NULL): int64[2k], f(u) restricted to [ranges[2u], ranges[2u+1])
// for every query vertex u, i.e. only embeddings inside those ranges count.
// limit > 0: give up (OR_LIMIT) once more than `limit` embeddings exist;
// node_budget > 0: give up (OR_BUDGET) after that many search steps.  Neither
// changes what is counted when the call returns OR_OK / OR_TRUNCATED.
int oracle_match(int32_t n, const int32_t* rp, const int32_t* col, const int32_t* lab,
                 int32_t k, int32_t m, const int32_t* edges, const int32_t* qlab,
                 int64_t root_lo, int64_t root_hi, int32_t enumerate,
                 int32_t* out, uint64_t cap_rows, uint64_t* count_lo, uint64_t* count_hi,
                 int32_t nthreads, uint64_t limit, uint64_t node_budget,
                 const int64_t* ranges) {
  if (oracle_validate_query(k, m, edges) != OR_OK) return OR_INVALID_QUERY;
  Search S;
  S.rp = rp; S.col = col; S.lab = lab; S.qlab = qlab; S.k = k;
  S.enumerate = enumerate != 0;
  S.limit = limit;
  S.node_budget = node_budget;
  for (int32_t u = 0; u < 16; ++u) {
    S.rlo[u] = (ranges && u < k) ? ranges[2 * u] : 0;
    S.rhi[u] = (ranges && u < k) ? ranges[2 * u + 1] : (int64_t)n;
  }
  std::memset(S.adj, 0, sizeof(S.adj));
  for (int32_t e = 0; e < m; ++e) {
    S.adj[edges[2 * e]][edges[2 * e + 1]] = true;
    S.adj[edges[2 * e + 1]][edges[2 * e]] = true;
  }
  // BFS of Q from vertex 0, neighbours ascending
  bool seen[16] = {};
  int32_t head = 0, tail = 0;
  S.order[tail++] = 0; seen[0] = true; S.parent[0] = -1;
  while (head < tail) {
    int32_t u = S.order[head++];
    for (int32_t w = 0; w < k; ++w)
      if (S.adj[u][w] && !seen[w]) { seen[w] = true; S.parent[w] = u; S.order[tail++] = w; }
  }
  int32_t root = S.order[0];
  int64_t lo = std::max<int64_t>(std::max<int64_t>(0, root_lo), S.rlo[root]);
  int64_t hi = std::min<int64_t>(std::min<int64_t>(n, root_hi), S.rhi[root]);
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  int nt = 1;
#endif
  std::vector<Worker> workers(nt);
  std::vector<std::vector<int32_t>> per_root_rows;  // rows grouped by root, ascending root
  int64_t span = hi > lo ? hi - lo : 0;
  if (S.enumerate) per_root_rows.resize(span);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
#endif
  for (int64_t v = lo; v < hi; ++v) {
#ifdef _OPENMP
    Worker& W = workers[omp_get_thread_num()];
#else
    Worker& W = workers[0];
#endif
    W.s = &S;
    if (lab[v] != qlab[root]) continue;
    W.f[root] = (int32_t)v;
    W.rows.clear();
    W.dfs(1);
    if (S.enumerate) per_root_rows[v - lo].swap(W.rows);
  }
  if (S.stop.load()) return S.stop.load() == 1 ? OR_LIMIT : OR_BUDGET;
  unsigned __int128 total = 0;
  for (auto& W : workers) total += W.count;
  *count_lo = (uint64_t)total;
  *count_hi = (uint64_t)(total >> 64);
  if (limit && total > limit) return OR_LIMIT;
  if (!S.enumerate) return OR_OK;
  std::vector<int32_t> all;
  for (auto& r : per_root_rows) all.insert(all.end(), r.begin(), r.end());
  size_t nrows = all.size() / (size_t)k;
  std::vector<size_t> idx(nrows);
  for (size_t i = 0; i < nrows; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
    return std::lexicographical_compare(all.begin() + a * k, all.begin() + a * k + k,
                                        all.begin() + b * k, all.begin() + b * k + k);
  });
  uint64_t ncopy = std::min<uint64_t>(nrows, cap_rows);
  for (uint64_t i = 0; i < ncopy; ++i)
    std::memcpy(out + i * k, all.data() + idx[i] * k, sizeof(int32_t) * k);
  return nrows > cap_rows ? OR_TRUNCATED : OR_OK;
}

// Number of k-cliques of an undirected graph (3 <= k <= 8), each clique
// counted once, by the textbook degree-ordered listing (Chiba and Nishizeki's
// arboricity method): rank the vertices by (degree, id), keep every edge
// only from its lower- to its higher-ranked end (N+(v)), and grow cliques
// along increasing rank, each step keeping the common out-neighbours of the
// vertices chosen so far.  It shares nothing with the backtracking matcher
// above (different order, no query, no injectivity test), so it pins the
// matcher's count of the k-clique query at sizes the matcher cannot reach:
// ordered embeddings of K_k = k! x this count.  The count is returned as two
// 64-bit halves of an unsigned 128-bit integer.
int oracle_cliques(int32_t n, const int32_t* rp, const int32_t* col, int32_t k,
                   int32_t nthreads, uint64_t* count_lo, uint64_t* count_hi) {
  if (n < 0 || k < 3 || k > 8) return OR_INVALID_ARG;
  auto higher = [&](int32_t a, int32_t b) {  // rank(b) > rank(a)
    const int32_t da = rp[a + 1] - rp[a], db = rp[b + 1] - rp[b];
    return db > da || (db == da && b > a);
  };
  std::vector<int64_t> op(n + 1, 0);
  for (int32_t v = 0; v < n; ++v) {
    int64_t c = 0;
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) c += higher(v, col[e]) ? 1 : 0;
    op[v + 1] = op[v] + c;
  }
  std::vector<int32_t> out(op[n] > 0 ? op[n] : 1);
  for (int32_t v = 0; v < n; ++v) {
    int64_t p = op[v];
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e)
      if (higher(v, col[e])) out[p++] = col[e];
  }
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  int nt = 1;
#endif
  std::vector<unsigned __int128> part(nt, 0);
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
  {
#ifdef _OPENMP
    const int tid = omp_get_thread_num();
#else
    const int tid = 0;
#endif
    // mark[x] == stamp[d] iff x is in the candidate list of depth d
    std::vector<uint64_t> mark(n > 0 ? n : 1, 0);
    uint64_t next_stamp = 0;
    std::vector<std::vector<int32_t>> lists(k);
    unsigned __int128 local = 0;
    // depth d holds the common out-neighbours of the d chosen vertices
    std::function<void(int32_t)> grow = [&](int32_t d) {
      const std::vector<int32_t>& cur = lists[d];
      if (d == k - 1) {
        local += cur.size();
        return;
      }
      const uint64_t stamp = ++next_stamp;
      for (int32_t x : cur) mark[x] = stamp;
      for (int32_t u : cur) {
        std::vector<int32_t>& nxt = lists[d + 1];
        nxt.clear();
        for (int64_t e = op[u]; e < op[u + 1]; ++e)
          if (mark[out[e]] == stamp) nxt.push_back(out[e]);
        if ((int32_t)nxt.size() >= k - 1 - d) {
          grow(d + 1);
          for (int32_t x : nxt) mark[x] = stamp;  // deeper levels re-marked them
        }
      }
    };
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
    for (int32_t v = 0; v < n; ++v) {
      lists[1].assign(out.begin() + op[v], out.begin() + op[v + 1]);
      if ((int32_t)lists[1].size() >= k - 1) grow(1);
    }
    part[tid] = local;
  }
  unsigned __int128 total = 0;
  for (auto p : part) total += p;
  *count_lo = (uint64_t)total;
  *count_hi = (uint64_t)(total >> 64);
  return OR_OK;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
