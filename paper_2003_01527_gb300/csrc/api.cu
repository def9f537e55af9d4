// libgsm host side: the C ABI of include/gsm.h, device-memory management, the
// matching-order planner, and the level driver that runs one verification
// level per query vertex (paper Sec. 3.2, Algorithm 1) depth-first over
// frontier chunks so intermediate results stay inside a fixed budget.
#include <algorithm>
#include <array>
#include <atomic>
#include <climits>
#include <functional>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>

#include <nvtx3/nvToolsExt.h>

#include "batch.h"
#include "gsm.h"
#include "compressed.cuh"
#include "kernels.cuh"
#include "query_access.h"

using namespace gsm;

// ------------------------------------------------------------------ context

namespace {

struct KStat {
  const char *name;
  uint64_t launches = 0;
  double total_ms = 0, algo_bytes = 0;
  uint64_t items = 0;
  double probe_bytes = 0;  // part of algo_bytes
};

enum KernelId { K_FILTER, K_LIST, K_PIVOT, K_COUNT, K_WRITE, K_SORT, K_FUSED, K_NUM };
const char *kKernelNames[K_NUM] = {"filter", "bitmap_to_list", "pivot_scan",
                                   "extend_count", "extend_write", "sort_rows", "extend_fused"};

struct Pending {
  int kid;
  cudaEvent_t a, b;
  double bytes;
  uint64_t items;
};

struct Block {
  char *ptr;
  size_t cap;
};

}  // namespace

struct gsm_query {
  int32_t k = 0, m = 0;
  std::vector<int32_t> edges;
  int32_t labels[kMaxK] = {};
  uint32_t adj[kMaxK] = {};
  int32_t lo[kMaxK], hi[kMaxK];
};

struct gsm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  gsm_options opt{};
  size_t budget = 0;
  std::string err;

  // graph
  bool has_graph = false;
  bool borrowed_graph = false;  // a worker context: the graph belongs to its parent
  std::vector<gsm_ctx *> workers;  // gsm_enumerate_many's parallel listing contexts
  int32_t n = 0;
  int64_t nnz = 0;
  int32_t max_deg = 0;
  int32_t *d_rp = nullptr, *d_col = nullptr, *d_lab = nullptr;
  int32_t *d_lcol = nullptr, *d_llab = nullptr;  // rows ordered by (label, id)
  int32_t *d_hub = nullptr;        // hub index of every vertex, -1 = none
  uint32_t *d_hub_bits = nullptr;  // adjacency bitmaps of the hubs
  int32_t *d_hub_seg = nullptr;    // label segment starts of the hubs' rows
  size_t hub_seg_bytes = 0;
  uint8_t *d_nlc = nullptr;        // neighbour label counts, nlc_stride per vertex
  int32_t nlc_stride = 0;
  int32_t hub_count = 0, hub_min_deg = 0;
  size_t hub_bits_bytes = 0;
  std::vector<int32_t> label_values;  // sorted distinct labels; dense id = index

  // query-lifetime buffers (outside the budget)
  void *bitmaps = nullptr;
  size_t bitmaps_cap = 0;
  void *bitmaps2 = nullptr;  // second buffer of the refinement rounds
  size_t bitmaps2_cap = 0;
  void *mfilter = nullptr;  // gsm_enumerate_many: descriptors, sizes and bitmaps of all queries
  size_t mfilter_cap = 0;
  unsigned long long *d_small = nullptr;  // [0..15] sizes, [16] total, [17] err
  void *acc[2] = {nullptr, nullptr};
  size_t acc_cap[2] = {0, 0};
  // gsm_enumerate_many: the result buffers (acc, sort_keys) come in several
  // slots used in turn; while the rows of one query are copied out on
  // copy_stream, the next queries compute into the other slots.  A slot's
  // `copied` event marks the end of its last copy out; the compute stream
  // waits for it before reusing the slot.  The active slot's buffers are
  // acc / sort_keys above, the others are parked.
  struct ResultSlot {
    void *acc[2] = {nullptr, nullptr};
    size_t acc_cap[2] = {0, 0};
    void *sort_keys = nullptr;
    size_t sort_keys_cap = 0;
    cudaEvent_t copied = nullptr;
    bool pending = false;
  };
  std::deque<ResultSlot> parked;
  cudaEvent_t active_copied = nullptr;
  bool active_pending = false;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t rows_ready = nullptr;
  void *sort_tmp = nullptr;  // radix-sort histograms (scale with the result)
  size_t sort_tmp_cap = 0;
  void *d_prefix = nullptr;  // PrefixState of the last level's prefix ranks
  size_t d_prefix_cap = 0;
  void *sort_keys = nullptr;  // the second buffer of the packed-key radix passes
  size_t sort_keys_cap = 0;
  const int32_t *last_rows = nullptr;  // sorted rows of the last gsm_enumerate
  uint64_t last_count = 0;
  int32_t last_k = 0;

  // budgeted memory: frontier stack (segmented) and scratch; the scratch
  // area may take up to a quarter of the budget, the stack the rest
  std::vector<Block> blocks;
  size_t top_block = 0, top_used = 0;  // stack pointer
  size_t stack_alloc = 0;              // bytes allocated for stack blocks
  size_t stack_limit = 0, scratch_limit = 0;
  size_t live_bytes = 0, peak_bytes = 0;
  void *scratch = nullptr;
  size_t scratch_cap = 0;

  // small device->host reads: a kernel writes them into mapped pinned memory
  // (the copy engines stay free for result copies in flight)
  int64_t *h_stage = nullptr;
  void *d_stage = nullptr;  // device view of h_stage
  // mapped flag words after the 4 KB of h_stage: [0] = a sort's look-back
  // wait ran out (set by the sort kernels, read and cleared by the host)
  uint32_t *h_flags = nullptr, *d_flags = nullptr;
  int32_t num_sms = 0;

  // batched form: per-label sorted degrees (order estimates without the
  // filter's results); lanes = stream + fixed-capacity workspace + graphs
  std::vector<std::vector<int32_t>> deg_by_label;
  int64_t batch_caps[4] = {0, 0, 0, 0};  // rows, elements, candidates, result elements (0 = default)
  struct BatchLane {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool ready = false;
    int64_t cap_rows = 0, cap_elems = 0, cap_items = 0;
    int32_t max_nq = 0;
    int64_t max_words_total = 0;
    std::vector<std::pair<void *, size_t>> allocs;
    gsm::BatchArgs a{};
    void *bitmaps = nullptr;
    size_t bitmaps_cap = 0;
    FilterDesc *h_fds = nullptr;
    BatchQuery *h_qs = nullptr;
    uint32_t **h_bm = nullptr;
    unsigned long long *h_counts = nullptr;
    int32_t *h_overflow = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_done = nullptr;
    uint32_t *zero_bitmap = nullptr;  // root bitmap of padding queries
    int32_t mb = 0, kb = 0;           // shape of the issued batch (padded)
    // enumerate batches: the result arena (allocated on first use), the step
    // sizes read back after a batch, each selected query's matching order and
    // whether it lists rows, and the buffers of the canonical sort
    int32_t enumerate = 0;
    int64_t cap_final = 0;
    BatchStep *h_state = nullptr;
    std::vector<std::array<int32_t, kMaxK>> orders;
    std::vector<int32_t> lists;
    // device buffers of the canonical sorts: keys (2), sort scratch, the
    // small-sort items, the staged rows of host results, the segment tables
    void *srt[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t srt_cap[6] = {0, 0, 0, 0, 0, 0};
    gsm::SmallSortItem *h_items = nullptr;  // pinned staging of the items
    size_t h_items_cap = 0;
    gsm::SortSegment *h_segs = nullptr;  // pinned staging of the segment tables
    size_t h_segs_cap = 0;
    std::map<std::tuple<int32_t, int32_t, int32_t, int32_t, int32_t, int32_t>, cudaGraphExec_t>
        graphs;
    // a batch in flight (server): which requests, how many queries
    std::vector<uint64_t> tickets;
    std::vector<int32_t> sel;
    int32_t m = 0;
    bool busy = false;
  };
  BatchLane lane0;  // gsm_run_batch, on the context's stream
  std::map<std::pair<int32_t, int32_t>, std::pair<int32_t, int32_t>> tuned;  // bucket -> (block, grid)
  struct Server;
  Server *server = nullptr;
  gsm_batch_stats bstats{};

  // stats
  KStat kstats[K_NUM];
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  gsm_run_stats run{};
};

namespace {

struct Fail {
  gsm_status code;
};

GraphDev graph_dev(const gsm_ctx *ctx) {
  return GraphDev{ctx->n,
                  ctx->nnz,
                  ctx->d_rp,
                  ctx->d_col,
                  ctx->d_lab,
                  ctx->d_lcol,
                  ctx->d_llab,
                  (int32_t)std::max<size_t>(1, ctx->label_values.size()),
                  ctx->hub_count ? ctx->d_hub : nullptr,
                  ctx->hub_count ? ctx->d_hub_bits : nullptr,
                  (ctx->n + 31) / 32,
                  ctx->hub_count ? ctx->d_hub_seg : nullptr,
                  ctx->d_nlc,
                  ctx->nlc_stride,
                  ctx->d_flags ? ctx->d_flags + 1 : nullptr};
}

void set_err(gsm_ctx *c, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  c->err = buf;
}

#define CU(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      set_err(ctx, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
              __LINE__);                                                             \
      throw Fail{GSM_ERR_CUDA};                                                      \
    }                                                                                \
  } while (0)

#define FAIL(code, ...)        \
  do {                         \
    set_err(ctx, __VA_ARGS__); \
    throw Fail{code};          \
  } while (0)

void *dev_alloc(gsm_ctx *ctx, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void *p = nullptr;
  if (ctx->opt.alloc) {
    p = ctx->opt.alloc(ctx->opt.alloc_ctx, bytes, ctx->stream);
    if (!p) FAIL(GSM_ERR_OOM, "device allocation of %zu bytes failed", bytes);
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      FAIL(GSM_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
  }
  return p;
}

void dev_free(gsm_ctx *ctx, void *p, size_t bytes) {
  if (!p) return;
  if (ctx->opt.free)
    ctx->opt.free(ctx->opt.alloc_ctx, p, bytes, ctx->stream);
  else
    cudaFree(p);
}

// Grows a buffer that is outside the budget; keeps the contents if asked.
void ensure_buf(gsm_ctx *ctx, void **p, size_t *cap, size_t bytes, bool keep, size_t keep_bytes) {
  if (*cap >= bytes && *p) return;
  size_t want = std::max(bytes, *cap + *cap / 2);
  void *q = dev_alloc(ctx, want);
  if (keep && keep_bytes) CU(cudaMemcpyAsync(q, *p, keep_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  dev_free(ctx, *p, *cap);
  *p = q;
  *cap = want;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// ---- budgeted stack ----

struct Mark {
  size_t block, used, live;
};

Mark stack_mark(gsm_ctx *c) { return {c->top_block, c->top_used, c->live_bytes}; }
void stack_release(gsm_ctx *c, Mark m) {
  c->top_block = m.block;
  c->top_used = m.used;
  c->live_bytes = m.live;
}

// First block index a push may use when the top block is full: the top
// block itself if nothing live is in it, else the one above.
size_t stack_start(const gsm_ctx *c) {
  if (c->blocks.empty()) return 0;
  return c->top_used == 0 ? c->top_block : c->top_block + 1;
}

// Can pushes totalling `bytes` (each already aligned) be made without
// exceeding the stack's share of the budget?  Either they all fit in what is
// left of the top block, or one block (cached or new) can hold all of them.
bool stack_fits(gsm_ctx *c, size_t bytes) {
  const auto &B = c->blocks;
  if (c->top_block < B.size() && B[c->top_block].cap - c->top_used >= bytes) return true;
  const size_t start = stack_start(c);
  size_t free_above = 0;
  for (size_t b = start; b < B.size(); ++b) {
    if (B[b].cap >= bytes) return true;
    free_above += B[b].cap;
  }
  return c->stack_alloc - free_above + bytes <= c->stack_limit;
}

void *stack_push(gsm_ctx *ctx, size_t bytes) {
  bytes = align_up(bytes);
  auto &B = ctx->blocks;
  char *p = nullptr;
  if (ctx->top_block < B.size() && B[ctx->top_block].cap - ctx->top_used >= bytes) {
    p = B[ctx->top_block].ptr + ctx->top_used;
    ctx->top_used += bytes;
  } else {
    const size_t start = stack_start(ctx);
    for (size_t b = start; b < B.size() && !p; ++b) {
      if (B[b].cap >= bytes) {
        std::swap(B[b], B[start]);  // blocks at or above start hold nothing live
        p = B[start].ptr;
      }
    }
    if (!p) {
      // drop the cached blocks at or above start, then allocate a new one
      while (B.size() > start) {
        dev_free(ctx, B.back().ptr, B.back().cap);
        ctx->stack_alloc -= B.back().cap;
        B.pop_back();
      }
      const size_t avail = ctx->stack_limit - std::min(ctx->stack_limit, ctx->stack_alloc);
      if (bytes > avail)
        FAIL(GSM_ERR_BUDGET,
             "frontier chunk of %zu bytes exceeds the memory budget (%zu of %zu bytes of stack "
             "in use)", bytes, ctx->stack_alloc, ctx->stack_limit);
      const size_t last = B.empty() ? 0 : B.back().cap;
      const size_t want =
          std::max(bytes, std::min(avail, std::max<size_t>(last * 2, size_t(64) << 20)));
      B.push_back(Block{(char *)dev_alloc(ctx, want), want});
      ctx->stack_alloc += want;
      p = B[start].ptr;
    }
    ctx->top_block = start;
    ctx->top_used = bytes;
  }
  ctx->live_bytes += bytes;
  ctx->peak_bytes = std::max(ctx->peak_bytes, ctx->live_bytes + ctx->scratch_cap);
  return p;
}

// Scratch: reused by every step, contents dead between steps.
void *scratch_get(gsm_ctx *ctx, size_t bytes) {
  bytes = align_up(bytes);
  if (ctx->scratch_cap >= bytes) return ctx->scratch;
  if (bytes > ctx->scratch_limit)
    FAIL(GSM_ERR_BUDGET, "scratch of %zu bytes exceeds its share of the budget (%zu)", bytes,
         ctx->scratch_limit);
  const size_t want = std::min(ctx->scratch_limit, std::max(bytes, ctx->scratch_cap * 2));
  if (ctx->scratch) {
    CU(cudaStreamSynchronize(ctx->stream));
    dev_free(ctx, ctx->scratch, ctx->scratch_cap);
  }
  ctx->scratch = nullptr;
  ctx->scratch_cap = 0;
  ctx->scratch = dev_alloc(ctx, want);
  ctx->scratch_cap = want;
  ctx->peak_bytes = std::max(ctx->peak_bytes, ctx->live_bytes + ctx->scratch_cap);
  return ctx->scratch;
}

// Carves consecutive aligned pieces out of one scratch request.
struct Carve {
  size_t off = 0;
  template <typename T>
  size_t add(int64_t elems) {
    size_t o = off;
    off = align_up(off + sizeof(T) * (size_t)std::max<int64_t>(elems, 1));
    return o;
  }
};

// Copies `bytes` (a multiple of 4, at most 4096) from device memory into
// ctx->h_stage once the stream's earlier work is done.
void fetch(gsm_ctx *ctx, const void *dptr, size_t bytes) {
  launch_fetch(dptr, ctx->d_stage, bytes, ctx->stream);
  ctx->run.kernel_launches += 1;
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(ctx->stream));
}

// GSM_OPT_INJECT_SORT_STALL: the tile of every sort pass that withholds its
// counts (-1: none).
int32_t sort_stall_tile(const gsm_ctx *ctx) {
  return (ctx->opt.flags & GSM_OPT_INJECT_SORT_STALL) ? 1 : -1;
}

// Raises GSM_ERR_TIMEOUT if a sort's look-back wait ran out since the last
// check, or GSM_ERR_INTERNAL if a bounds check of the GSM_DEBUG build failed
// (and clears the flags); call once the kernels' stream has been
// synchronised.
void check_sort_flag(gsm_ctx *ctx) {
  volatile uint32_t *f = ctx->h_flags;
  if (f && f[1]) {
    const uint32_t site = f[1];
    f[1] = 0;
    FAIL(GSM_ERR_INTERNAL, "a device bounds check failed (site %u)", site);
  }
  if (f && f[0]) {
    f[0] = 0;
    FAIL(GSM_ERR_TIMEOUT, "a sort tile waited too long for its predecessors");
  }
}

// NVTX ranges (header-only NVTX 3: a cheap no-op unless a profiler is
// attached) around a listing call, the filter, every verification-level
// launch and the sort, so that a profile can be cut to one level
// (ncu --nvtx --nvtx-include "gsm level 3/").
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

const char *level_range(int32_t i) {
  static const char *kNames[] = {"gsm level 0",  "gsm level 1",  "gsm level 2",  "gsm level 3",
                                 "gsm level 4",  "gsm level 5",  "gsm level 6",  "gsm level 7",
                                 "gsm level 8",  "gsm level 9",  "gsm level 10", "gsm level 11",
                                 "gsm level 12", "gsm level 13", "gsm level 14", "gsm level 15"};
  return (i >= 0 && i < 16) ? kNames[i] : "gsm level";
}

int64_t read_i64(gsm_ctx *ctx, const int64_t *dptr) {
  fetch(ctx, dptr, sizeof(int64_t));
  return ((volatile int64_t *)ctx->h_stage)[0];
}

// ---- kernel timing ----

cudaEvent_t get_event(gsm_ctx *ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CU(cudaEventCreate(&e));
  return e;
}

template <typename F>
void timed(gsm_ctx *ctx, int kid, double bytes, uint64_t items, int launches, F &&launch) {
  const bool on = ctx->opt.flags & GSM_OPT_TIME_KERNELS;
  Pending p{kid, nullptr, nullptr, bytes, items};
  if (on) {
    p.a = get_event(ctx);
    p.b = get_event(ctx);
    CU(cudaEventRecord(p.a, ctx->stream));
  }
  launch();
  CU(cudaGetLastError());
  ctx->run.kernel_launches += launches;
  if (on) {
    CU(cudaEventRecord(p.b, ctx->stream));
    ctx->pending.push_back(p);
  } else {
    KStat &s = ctx->kstats[kid];
    s.launches += 1;
    s.algo_bytes += bytes;
    s.items += items;
  }
}

void resolve_timings(gsm_ctx *ctx) {
  if (ctx->pending.empty()) return;
  CU(cudaStreamSynchronize(ctx->stream));
  for (auto &p : ctx->pending) {
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, p.a, p.b));
    KStat &s = ctx->kstats[p.kid];
    s.launches += 1;
    s.total_ms += ms;
    s.algo_bytes += p.bytes;
    s.items += p.items;
    ctx->event_pool.push_back(p.a);
    ctx->event_pool.push_back(p.b);
  }
  ctx->pending.clear();
}

// ------------------------------------------------------------------ planner

int popc(uint32_t x) { return __builtin_popcount(x); }

// Matching order of Sec. 3.2 (after VF3): first the vertex with the fewest
// candidates (ties: larger degree, lower id); then repeatedly the unplaced
// vertex with the most edges to placed vertices (d_M), then fewest candidates
// (the P_f estimate), then larger degree, then lower id.  Since Q is
// connected the chosen vertex always has a placed neighbour, so the order
// follows a spanning tree; each vertex's parent is its earliest-placed
// neighbour.
void plan(int32_t k, const uint32_t *adj, const uint64_t *sizes, int32_t *order,
          int32_t *parent) {
  uint32_t placed = 0;
  for (int32_t i = 0; i < k; ++i) {
    int32_t best = -1;
    for (int32_t u = 0; u < k; ++u) {
      if (placed >> u & 1u) continue;
      const int dm = popc(adj[u] & placed);
      if (i > 0 && dm == 0) continue;
      if (best < 0) {
        best = u;
        continue;
      }
      const int dmb = popc(adj[best] & placed);
      const uint64_t su = sizes ? sizes[u] : 0, sb = sizes ? sizes[best] : 0;
      const int du = popc(adj[u]), db = popc(adj[best]);
      bool better;
      if (dm != dmb) better = dm > dmb;
      else if (su != sb) better = su < sb;
      else if (du != db) better = du > db;
      else better = u < best;
      if (better) best = u;
    }
    order[i] = best;
    placed |= 1u << best;
    parent[i] = -1;
    for (int32_t j = 0; j < i; ++j)
      if (adj[best] >> order[j] & 1u) {
        parent[i] = j;
        break;
      }
  }
}

gsm_status validate_query_edges(int32_t k, int32_t m, const int32_t *edges, uint32_t *adj) {
  if (k < 1 || k > kMaxK) return GSM_ERR_INVALID_QUERY;
  if (m < 0 || m > k * (k - 1) / 2) return GSM_ERR_INVALID_QUERY;
  if (m > 0 && !edges) return GSM_ERR_INVALID_ARG;
  for (int32_t u = 0; u < k; ++u) adj[u] = 0;
  for (int32_t e = 0; e < m; ++e) {
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || a >= k || b < 0 || b >= k || a == b) return GSM_ERR_INVALID_QUERY;
    if (adj[a] >> b & 1u) return GSM_ERR_INVALID_QUERY;
    adj[a] |= 1u << b;
    adj[b] |= 1u << a;
  }
  uint32_t seen = 1u, frontier = 1u;
  while (frontier) {
    uint32_t next = 0;
    for (int32_t u = 0; u < k; ++u)
      if (frontier >> u & 1u) next |= adj[u];
    frontier = next & ~seen;
    seen |= next;
  }
  return seen == ((k == 32) ? 0xffffffffu : ((1u << k) - 1u)) ? GSM_OK : GSM_ERR_INVALID_QUERY;
}

// ------------------------------------------------------------------ symmetry

// Is there an automorphism of the labelled query (a label-preserving
// permutation that maps edges to edges and non-edges to non-edges) with
// sigma(x) = x for every x in `fixed` and sigma(a) = b?  Backtracking over
// query vertices in id order.
bool aut_exists(int32_t k, const uint32_t *adj, const int32_t *lab, uint32_t fixed, int32_t a,
                int32_t b) {
  int32_t sigma[kMaxK];
  for (int32_t u = 0; u < kMaxK; ++u) sigma[u] = -1;
  for (int32_t u = 0; u < k; ++u)
    if (fixed >> u & 1u) sigma[u] = u;
  if (sigma[a] >= 0 && sigma[a] != b) return false;
  sigma[a] = b;
  uint32_t used = 0;
  for (int32_t u = 0; u < k; ++u)
    if (sigma[u] >= 0) {
      if (used >> sigma[u] & 1u) return false;
      used |= 1u << sigma[u];
    }
  // consistency of the preassigned part
  for (int32_t u = 0; u < k; ++u)
    for (int32_t v = 0; v < k; ++v)
      if (sigma[u] >= 0 && sigma[v] >= 0 &&
          ((adj[u] >> v & 1u) != (adj[sigma[u]] >> sigma[v] & 1u)))
        return false;
  for (int32_t u = 0; u < k; ++u)
    if (sigma[u] >= 0 && (lab[u] != lab[sigma[u]] || popc(adj[u]) != popc(adj[sigma[u]])))
      return false;
  // extend to the free vertices
  int32_t freev[kMaxK], nf = 0;
  for (int32_t u = 0; u < k; ++u)
    if (sigma[u] < 0) freev[nf++] = u;
  std::function<bool(int32_t)> go = [&](int32_t t) -> bool {
    if (t == nf) return true;
    const int32_t u = freev[t];
    for (int32_t v = 0; v < k; ++v) {
      if (used >> v & 1u) continue;
      if (lab[v] != lab[u] || popc(adj[v]) != popc(adj[u])) continue;
      bool ok = true;
      for (int32_t x = 0; x < k && ok; ++x)
        if (sigma[x] >= 0 && ((adj[u] >> x & 1u) != (adj[v] >> sigma[x] & 1u))) ok = false;
      if (!ok) continue;
      sigma[u] = v;
      used |= 1u << v;
      if (go(t + 1)) return true;
      sigma[u] = -1;
      used &= ~(1u << v);
    }
    return false;
  };
  return go(0);
}

// Ordering constraints that keep exactly one embedding per orbit of Aut(Q)
// (the node-ID ordering of equivalent query vertices the paper proposes,
// Sec. 3.1, built along a stabilizer chain): repeatedly take the lowest-id
// vertex u whose orbit under the automorphisms fixing the vertices chosen so
// far is non-trivial, require f(u) < f(v) for every other v of that orbit,
// and fix u.  |Aut(Q)| is the product of the orbit sizes.
uint64_t symmetry_constraints(int32_t k, const uint32_t *adj, const int32_t *lab,
                              std::vector<std::pair<int32_t, int32_t>> *less) {
  uint32_t fixed = 0;
  uint64_t order = 1;
  for (;;) {
    int32_t pick = -1;
    std::vector<int32_t> orbit;
    for (int32_t u = 0; u < k && pick < 0; ++u) {
      if (fixed >> u & 1u) continue;
      std::vector<int32_t> o{u};
      for (int32_t v = 0; v < k; ++v)
        if (v != u && !(fixed >> v & 1u) && aut_exists(k, adj, lab, fixed, u, v)) o.push_back(v);
      if (o.size() > 1) {
        pick = u;
        orbit = o;
      }
    }
    if (pick < 0) break;
    for (int32_t v : orbit)
      if (v != pick) less->push_back({pick, v});
    order *= orbit.size();
    fixed |= 1u << pick;
  }
  return order;
}

// ------------------------------------------------------------------ driver

struct Run {
  gsm_ctx *ctx;
  const gsm_query *q;
  bool enumerate;
  int32_t k;
  int32_t order[kMaxK], parent[kMaxK];
  LevelDesc lv[kMaxK];
  GraphDev g;
  int32_t block;
  int32_t spin_limit;  // polls a look-back wait may take
  int32_t stall_tile;  // GSM_OPT_INJECT_LOOKBACK_STALL: the tile that withholds its count
  int32_t scan_stall_tile;  // GSM_OPT_INJECT_SCAN_STALL: the same for the work scan
  int64_t wcap;        // max candidates per extend launch
  int64_t chunk_rows;  // max rows per extend launch (0 = unbounded)
  uint64_t acc_rows = 0;  // final rows so far, in ctx->acc[0]
  int64_t acc_ld = 0;     // rows ctx->acc[0] holds
  // layout of the final rows in ctx->acc[0]: row-major rows (the result) when
  // the matching order leaves them in canonical order, else packed sort keys
  int32_t acc_mode = kSinkRows;
  int32_t key_bits = 0, key_nw = 0;
  size_t acc_row_bytes() const {
    return acc_mode == kSinkKeys ? (size_t)key_nw * sizeof(uint64_t) : (size_t)k * sizeof(int32_t);
  }
  unsigned __int128 count = 0;
  unsigned long long *d_total;
  // the last level's keys carry the dense rank of the prefix (query vertices
  // 0..rank_p-1, placed first in that order) when rank_p > 0: ranks of the
  // rows of the last level's input piece in `rank`, running state in prefix
  int32_t rank_p = 0, rank_pos = 0;
  PrefixState *prefix = nullptr;
  const int32_t *rank = nullptr;
};

void recurse(Run &R, int32_t i, const int32_t *F, int64_t ld, int64_t rows);
void recurse_rest(Run &R, int32_t i, const int32_t *F, int64_t ld, int64_t rows,
                  const int32_t *pstart, const uint8_t *pslot, const int64_t *woff, int64_t W);
void process_fused(Run &R, int32_t i, const int32_t *F, int64_t ld, const int32_t *pstart,
                   const uint8_t *pslot, const int64_t *woff, int64_t ra, int64_t rb, int64_t wa,
                   int64_t wb);

// Largest result staging (bytes) the single-pass last level may reserve for
// its upper bound of one row per candidate.
constexpr double kFusedResultBytes = 4.0 * (1ull << 30);

// Grows the final-row accumulator to hold `rows` rows, keeping the R.acc_rows
// rows already written (row-major rows, or key words of leading dimension
// R.acc_ld).
void ensure_acc(Run &R, uint64_t rows) {
  gsm_ctx *ctx = R.ctx;
  if ((int64_t)rows <= R.acc_ld) return;
  const int64_t ld = std::max<int64_t>((int64_t)rows, R.acc_ld + R.acc_ld / 2);
  const size_t bytes = (size_t)ld * R.acc_row_bytes();
  void *q = dev_alloc(ctx, bytes);
  if (R.acc_rows && R.acc_mode == kSinkKeys)
    CU(cudaMemcpy2DAsync(q, ld * sizeof(uint64_t), ctx->acc[0], R.acc_ld * sizeof(uint64_t),
                         R.acc_rows * sizeof(uint64_t), R.key_nw, cudaMemcpyDeviceToDevice,
                         ctx->stream));
  else if (R.acc_rows)
    CU(cudaMemcpyAsync(q, ctx->acc[0], R.acc_rows * R.acc_row_bytes(), cudaMemcpyDeviceToDevice,
                       ctx->stream));
  dev_free(ctx, ctx->acc[0], ctx->acc_cap[0]);
  ctx->acc[0] = q;
  ctx->acc_cap[0] = bytes;
  R.acc_ld = ld;
}

void process_sub(Run &R, int32_t i, const int32_t *F, int64_t ld, const int32_t *pstart,
                 const uint8_t *pslot, const int64_t *woff, int64_t ra, int64_t rb, int64_t wa,
                 int64_t wb) {
  gsm_ctx *ctx = R.ctx;
  const Range range(level_range(i));
  const LevelDesc &d = R.lv[i];
  const bool last = i == R.k - 1;
  const int64_t W = wb - wa, nrows = rb - ra;
  if (W <= 0) return;
  const int64_t tile_items = (int64_t)R.block * kItemsPerThread;
  const int64_t tiles = extend_tiles(wa, wb, R.block);
  const double read_bytes = (double)nrows * (4.0 * i + 13.0) + 4.0 * (double)W;
  ctx->run.chunks += 1;
  const bool count_only = last && !R.enumerate;
  const int32_t w_out = i + 1;
  if (!count_only && !(ctx->opt.flags & GSM_OPT_TWO_PASS)) {
    // single pass (count and write together) when the output has room for
    // every candidate surviving: W rows of the next frontier (plus its
    // per-row arrays) on the stack, or W result rows
    bool fits;
    if (last) {
      fits = (double)W * (double)R.acc_row_bytes() <= kFusedResultBytes;
    } else {
      const size_t need = align_up((size_t)W * w_out * sizeof(int32_t)) +
                          align_up(4 * (size_t)W) + align_up((size_t)W) +
                          align_up(8 * ((size_t)W + 1));
      fits = (int64_t)W * w_out < (int64_t(1) << 31) - 1 && stack_fits(ctx, need);
    }
    if (fits) {
      process_fused(R, i, F, ld, pstart, pslot, woff, ra, rb, wa, wb);
      return;
    }
  }
  Carve cv;
  const size_t o_row = cv.add<int32_t>(tiles + 1);
  const size_t o_mask = count_only ? 0 : cv.add<uint32_t>(tiles * (tile_items / 32));
  const size_t o_cnt = count_only ? 0 : cv.add<int32_t>(tiles);
  const size_t o_off = count_only ? 0 : cv.add<int64_t>(tiles + 1);
  const size_t o_tmp = count_only ? 0 : cv.add<int64_t>(scan_tmp_elems(tiles));
  char *sc = (char *)scratch_get(ctx, cv.off);
  int32_t *tile_row = (int32_t *)(sc + o_row);
  timed(ctx, K_PIVOT, 8.0 * (nrows + tiles), (uint64_t)tiles, 1, [&] {
    launch_tile_rows(woff, ra, rb, wa, wb, R.block, tile_row, nullptr, ctx->stream);
  });
  if (count_only) {
    timed(ctx, K_COUNT, read_bytes, (uint64_t)W, 1, [&] {
      launch_extend_count(R.g, d, F, ld, pstart, pslot, woff, tile_row, wa, wb, R.block, nullptr,
                          nullptr, R.d_total, ctx->stream);
    });
    return;
  }
  uint32_t *masks = (uint32_t *)(sc + o_mask);
  int32_t *tile_cnt = (int32_t *)(sc + o_cnt);
  int64_t *tile_off = (int64_t *)(sc + o_off);
  int64_t *tmp = (int64_t *)(sc + o_tmp);
  timed(ctx, K_COUNT, read_bytes + W / 8.0, (uint64_t)W, 1, [&] {
    launch_extend_count(R.g, d, F, ld, pstart, pslot, woff, tile_row, wa, wb, R.block, masks,
                        tile_cnt, nullptr, ctx->stream);
  });
  timed(ctx, K_PIVOT, 12.0 * tiles, (uint64_t)tiles, scan_kernels(tiles),
        [&] { launch_scan_i32(tile_cnt, tile_off, tiles, tmp, ctx->stream); });
  const int64_t S = read_i64(ctx, tile_off + tiles);
  if (S == 0) return;
  if (last) {
    ensure_acc(R, R.acc_rows + (uint64_t)S);
    RowSink sink{R.acc_mode, R.k, R.key_bits, R.key_nw, R.acc_ld, (int64_t)R.acc_rows,
                 ctx->acc[0]};
    sink.rank = R.rank;
    sink.rank_pos = R.rank_pos;
    timed(ctx, K_WRITE, (double)S * R.acc_row_bytes(), (uint64_t)S, 1, [&] {
      launch_extend_write(R.g, d, F, ld, pstart, woff, tile_row, wa, wb, R.block, masks,
                          tile_off, sink, ctx->stream);
    });
    R.acc_rows += (uint64_t)S;
    return;
  }
  const size_t bytes = (size_t)S * w_out * sizeof(int32_t);
  // the next level also pushes pivot start, pivot slot and work offsets
  const size_t need = align_up(bytes) + align_up(4 * (size_t)S) + align_up((size_t)S) +
                      align_up(8 * ((size_t)S + 1));
  // elements of a frontier are indexed with 32 bits inside the kernels
  const bool too_many = (int64_t)S * w_out >= (int64_t(1) << 31) - 1;
  if (too_many || !stack_fits(ctx, need)) {
    if (nrows <= 1)
      FAIL(GSM_ERR_BUDGET, "the %lld partial results of one row need %zu bytes, over the budget",
           (long long)S, bytes);
    const int64_t mid = ra + nrows / 2;
    const int64_t wmid = read_i64(ctx, woff + mid);
    process_sub(R, i, F, ld, pstart, pslot, woff, ra, mid, wa, wmid);
    process_sub(R, i, F, ld, pstart, pslot, woff, mid, rb, wmid, wb);
    return;
  }
  const Mark mk = stack_mark(ctx);
  int32_t *Fn = (int32_t *)stack_push(ctx, bytes);
  const RowSink sink{kSinkColumns, w_out, 0, 0, S, 0, Fn};
  timed(ctx, K_WRITE, 4.0 * S * w_out, (uint64_t)S, 1, [&] {
    launch_extend_write(R.g, d, F, ld, pstart, woff, tile_row, wa, wb, R.block, masks, tile_off,
                        sink, ctx->stream);
  });
  recurse(R, i + 1, Fn, S, S);
  stack_release(ctx, mk);
}

// The single-pass form of process_sub's count and write passes
// (k_extend_fused); the caller checked that the output has room for W rows.
void process_fused(Run &R, int32_t i, const int32_t *F, int64_t ld, const int32_t *pstart,
                   const uint8_t *pslot, const int64_t *woff, int64_t ra, int64_t rb, int64_t wa,
                   int64_t wb) {
  gsm_ctx *ctx = R.ctx;
  const Range range(level_range(i));
  const LevelDesc &d = R.lv[i];
  const bool last = i == R.k - 1;
  const int64_t W = wb - wa, nrows = rb - ra;
  const int64_t tiles = extend_tiles(wa, wb, R.block);
  const int32_t w_out = i + 1;
  Carve cv;
  const size_t o_row = cv.add<int32_t>(tiles + 1);
  // the level's look-back words, then (not last) those of the next level's
  // pivot choice and work scan (sized for up to W rows); k_tile_rows zeroes
  // both
  const int64_t pwords = last ? 0 : pivot_scan_words(W);
  const size_t o_lb = cv.add<unsigned long long>(tiles + kLbExtra + pwords);
  char *sc = (char *)scratch_get(ctx, cv.off);
  int32_t *tile_row = (int32_t *)(sc + o_row);
  unsigned long long *lb = (unsigned long long *)(sc + o_lb);
  timed(ctx, K_PIVOT, 8.0 * (nrows + tiles) + 8.0 * (tiles + pwords), (uint64_t)tiles, 1, [&] {
    launch_tile_rows(woff, ra, rb, wa, wb, R.block, tile_row, lb, ctx->stream, pwords);
  });
  const double read_bytes = (double)nrows * (4.0 * i + 13.0) + 4.0 * (double)W;
  const Mark mk = stack_mark(ctx);
  RowSink sink;
  int32_t *Fn = nullptr;
  if (last) {
    ensure_acc(R, R.acc_rows + (uint64_t)W);
    sink = RowSink{R.acc_mode, R.k, R.key_bits, R.key_nw, R.acc_ld, (int64_t)R.acc_rows,
                   ctx->acc[0]};
    sink.rank = R.rank;
    sink.rank_pos = R.rank_pos;
  } else {
    Fn = (int32_t *)stack_push(ctx, (size_t)W * w_out * sizeof(int32_t));
    sink = RowSink{kSinkColumns, w_out, 0, 0, W, 0, Fn};
  }
  timed(ctx, K_FUSED, read_bytes, (uint64_t)W, 1, [&] {
    launch_extend_fused(R.g, d, F, ld, pstart, pslot, woff, tile_row, wa, wb, R.block, lb, sink,
                        R.spin_limit, R.stall_tile, ctx->stream);
  });
  const int64_t *S_dev = (const int64_t *)(lb + tiles + 1);
  if (last) {
    fetch(ctx, S_dev, 3 * sizeof(unsigned long long));
    const int64_t S = ((volatile int64_t *)ctx->h_stage)[0];
    if (((volatile int64_t *)ctx->h_stage)[1])
      FAIL(GSM_ERR_TIMEOUT, "a verification tile waited too long for its predecessors");
    const double probes = (double)((volatile int64_t *)ctx->h_stage)[2];
    ctx->kstats[K_FUSED].algo_bytes += (double)S * (double)R.acc_row_bytes() + probes;
    ctx->kstats[K_FUSED].probe_bytes += probes;
    R.acc_rows += (uint64_t)S;
    return;
  }
  // the next level's pivot choice and work scan run before the host learns
  // S (they read it on the device; their arrays were reserved for W rows),
  // and their last CTA writes both levels' totals to the host stage, so one
  // read-back serves both levels
  const LevelDesc &dn = R.lv[i + 1];
  int32_t *pstart2 = (int32_t *)stack_push(ctx, sizeof(int32_t) * W);
  uint8_t *pslot2 = (uint8_t *)stack_push(ctx, W);
  int64_t *woff2 = (int64_t *)stack_push(ctx, sizeof(int64_t) * (W + 1));
  timed(ctx, K_PIVOT, 0.0, 0, 1, [&] {
    launch_pivot_scan(R.g, dn, Fn, W, W, pstart2, pslot2, woff2, lb + tiles + kLbExtra,
                      R.spin_limit, ctx->d_stage, R.scan_stall_tile, ctx->stream, S_dev);
  });
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(ctx->stream));
  const int64_t S = ((volatile int64_t *)ctx->h_stage)[0];
  if (((volatile int64_t *)ctx->h_stage)[1])
    FAIL(GSM_ERR_TIMEOUT,
         "a verification or work-scan tile waited too long for its predecessors");
  const int64_t W2 = ((volatile int64_t *)ctx->h_stage)[2];
  const double probes = (double)((volatile int64_t *)ctx->h_stage)[3];
  ctx->kstats[K_FUSED].algo_bytes += (double)S * 4.0 * w_out + probes;
  ctx->kstats[K_FUSED].probe_bytes += probes;
  ctx->kstats[K_PIVOT].algo_bytes += (double)S * (4.0 * dn.nb + 8.0 * dn.nb + 13.0);
  ctx->kstats[K_PIVOT].items += (uint64_t)S;
  if (S > 0) recurse_rest(R, i + 1, Fn, W, S, pstart2, pslot2, woff2, W2);
  stack_release(ctx, mk);
}

// Row boundaries of the launches over rows [0, rows) of a level whose work
// offsets are woff (W candidates in all): pieces of at most R.wcap
// candidates, merged with multiples of chunk_rows; bw receives the work
// offset at every boundary.
void level_chunks(Run &R, const int64_t *woff, int64_t rows, int64_t W,
                  std::vector<int64_t> &bnd, std::vector<int64_t> &bw) {
  gsm_ctx *ctx = R.ctx;
  const bool split_w = W > R.wcap;
  const bool split_r = R.chunk_rows > 0 && rows > R.chunk_rows;
  if (!split_w && !split_r) {
    bnd = {0, rows};
    bw = {0, W};
    return;
  }
  if (split_w) {
    const int64_t step = std::max<int64_t>(1, R.wcap - ctx->max_deg);
    const int64_t J = (W + step - 1) / step;
    Carve cv;
    const size_t o_b = cv.add<int64_t>(J + 1), o_w = cv.add<int64_t>(J + 1);
    char *sc = (char *)scratch_get(ctx, cv.off);
    launch_split_points(woff, rows, step, J, (int64_t *)(sc + o_b), (int64_t *)(sc + o_w),
                        ctx->stream);
    CU(cudaGetLastError());
    bnd.resize(J + 1);
    CU(cudaMemcpyAsync(bnd.data(), sc + o_b, sizeof(int64_t) * (J + 1), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    bnd[0] = 0;
  } else {
    bnd = {0, rows};
  }
  if (split_r) {
    std::vector<int64_t> extra;
    for (int64_t r = R.chunk_rows; r < rows; r += R.chunk_rows) extra.push_back(r);
    bnd.insert(bnd.end(), extra.begin(), extra.end());
  }
  std::sort(bnd.begin(), bnd.end());
  bnd.erase(std::unique(bnd.begin(), bnd.end()), bnd.end());
  // work offset at every boundary
  bw.resize(bnd.size());
  for (size_t j = 0; j < bnd.size(); ++j) {
    CU(cudaMemcpyAsync(&bw[j], woff + bnd[j], sizeof(int64_t), cudaMemcpyDeviceToHost,
                       ctx->stream));
  }
  CU(cudaStreamSynchronize(ctx->stream));
}

// Extends rows of width i (F, `rows` of them, leading dimension ld) through
// the remaining levels.
void recurse(Run &R, int32_t i, const int32_t *F, int64_t ld, int64_t rows) {
  gsm_ctx *ctx = R.ctx;
  if (rows <= 0) return;
  const LevelDesc &d = R.lv[i];
  const Mark mk = stack_mark(ctx);
  int32_t *pstart = (int32_t *)stack_push(ctx, sizeof(int32_t) * rows);
  uint8_t *pslot = (uint8_t *)stack_push(ctx, rows);
  int64_t *woff = (int64_t *)stack_push(ctx, sizeof(int64_t) * (rows + 1));
  const int64_t pwords = pivot_scan_words(rows);
  auto *plb = (unsigned long long *)scratch_get(ctx, sizeof(unsigned long long) * pwords);
  CU(cudaMemsetAsync(plb, 0, sizeof(unsigned long long) * pwords, ctx->stream));
  timed(ctx, K_PIVOT, (double)rows * (4.0 * d.nb + 8.0 * d.nb + 13.0), (uint64_t)rows, 1,
        [&] {
    launch_pivot_scan(R.g, d, F, ld, rows, pstart, pslot, woff, plb, R.spin_limit,
                      ctx->d_stage, R.scan_stall_tile, ctx->stream);
  });
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(ctx->stream));
  if (((volatile int64_t *)ctx->h_stage)[1])
    FAIL(GSM_ERR_TIMEOUT, "a work-scan tile waited too long for its predecessors");
  const int64_t W = ((volatile int64_t *)ctx->h_stage)[2];
  recurse_rest(R, i, F, ld, rows, pstart, pslot, woff, W);
  stack_release(ctx, mk);
}

// The part of recurse after the pivot and work scan (W = total candidates).
void recurse_rest(Run &R, int32_t i, const int32_t *F, int64_t ld, int64_t rows,
                  const int32_t *pstart, const uint8_t *pslot, const int64_t *woff, int64_t W) {
  R.ctx->run.frontier[i] += (uint64_t)rows;
  R.ctx->run.candidates[i] += (uint64_t)W;
  if (i == R.k - 1 && R.rank_p > 0 && rows > 0) {
    // prefix ranks of this piece of the last level's input (the caller's
    // stack mark releases them)
    gsm_ctx *ctx = R.ctx;
    int32_t *flags = (int32_t *)stack_push(ctx, sizeof(int32_t) * rows);
    int64_t *offs = (int64_t *)stack_push(ctx, sizeof(int64_t) * (rows + 1));
    int64_t *tmp = (int64_t *)stack_push(ctx, sizeof(int64_t) * scan_tmp_elems(rows));
    int32_t *rank = (int32_t *)stack_push(ctx, sizeof(int32_t) * rows);
    ctx->run.kernel_launches +=
        launch_prefix_ranks(F, ld, rows, R.rank_p, R.prefix, flags, offs, tmp, rank, ctx->stream);
    CU(cudaGetLastError());
    R.rank = rank;
  }
  std::vector<int64_t> bnd, bw;
  level_chunks(R, woff, rows, W, bnd, bw);
  for (size_t j = 0; j + 1 < bnd.size(); ++j)
    process_sub(R, i, F, ld, pstart, pslot, woff, bnd[j], bnd[j + 1], bw[j], bw[j + 1]);
  if (i == R.k - 1) R.rank = nullptr;
}

// ---- compressed frontiers (GSM_OPT_COMPRESSED_FRONTIERS): a row of width i
// is (parent row of width i-1, new vertex); levels otherwise as above, always
// in the single pass

void recurse_c(Run &R, int32_t i, const CFrontier &f, int64_t rows);

void process_c(Run &R, int32_t i, const CFrontier &f, const int32_t *pstart, const uint8_t *pslot,
               const int64_t *woff, int64_t ra, int64_t rb, int64_t wa, int64_t wb) {
  gsm_ctx *ctx = R.ctx;
  const Range range(level_range(i));
  const LevelDesc &d = R.lv[i];
  const bool last = i == R.k - 1;
  const int64_t W = wb - wa, nrows = rb - ra;
  if (W <= 0) return;
  const bool count_only = last && !R.enumerate;
  if (!count_only) {
    // room for one output row per candidate, else split the rows
    bool fits;
    if (last) {
      fits = (double)W * (double)R.acc_row_bytes() <= kFusedResultBytes;
    } else {
      const size_t need = 2 * align_up(4 * (size_t)W) + align_up(4 * (size_t)W) +
                          align_up((size_t)W) + align_up(8 * ((size_t)W + 1));
      fits = stack_fits(ctx, need);
    }
    if (!fits) {
      if (nrows <= 1)
        FAIL(GSM_ERR_BUDGET, "the %lld candidates of one row need more than the budget",
             (long long)W);
      const int64_t mid = ra + nrows / 2;
      const int64_t wmid = read_i64(ctx, woff + mid);
      process_c(R, i, f, pstart, pslot, woff, ra, mid, wa, wmid);
      process_c(R, i, f, pstart, pslot, woff, mid, rb, wmid, wb);
      return;
    }
  }
  ctx->run.chunks += 1;
  const int64_t tiles = extend_tiles(wa, wb, R.block);
  Carve cv;
  const size_t o_row = cv.add<int32_t>(tiles + 1);
  const size_t o_lb = cv.add<unsigned long long>(tiles + kLbExtra);
  char *sc = (char *)scratch_get(ctx, cv.off);
  int32_t *tile_row = (int32_t *)(sc + o_row);
  unsigned long long *lb = (unsigned long long *)(sc + o_lb);
  timed(ctx, K_PIVOT, 8.0 * (nrows + tiles) + 8.0 * tiles, (uint64_t)tiles, 1, [&] {
    launch_tile_rows(woff, ra, rb, wa, wb, R.block, tile_row, lb, ctx->stream);
  });
  // candidate reads: the pivot start and the row (decoded through i-1
  // parent indices, 8 bytes each) per row, 4 bytes per candidate
  const double read_bytes = (double)nrows * (8.0 * i + 5.0) + 4.0 * (double)W;
  const Mark mk = stack_mark(ctx);
  CSink sink{};
  int32_t *Pn = nullptr, *Vn = nullptr;
  if (count_only) {
    sink.mode = kCSinkCount;
    sink.total = R.d_total;
  } else if (last) {
    ensure_acc(R, R.acc_rows + (uint64_t)W);
    sink.mode = R.acc_mode == kSinkKeys ? kCSinkKeys : kCSinkRows;
    sink.rows = RowSink{R.acc_mode, R.k, R.key_bits, R.key_nw, R.acc_ld, (int64_t)R.acc_rows,
                        ctx->acc[0]};
  } else {
    Pn = (int32_t *)stack_push(ctx, 4 * (size_t)W);
    Vn = (int32_t *)stack_push(ctx, 4 * (size_t)W);
    sink.mode = kCSinkPairs;
    sink.pn = Pn;
    sink.vn = Vn;
  }
  timed(ctx, K_FUSED, read_bytes, (uint64_t)W, 1, [&] {
    launch_cextend(R.g, d, f, i, pstart, pslot, woff, tile_row, wa, wb, R.block, lb, sink,
                   R.spin_limit, ctx->stream);
  });
  if (count_only) return;
  fetch(ctx, lb + tiles + 1, 2 * sizeof(unsigned long long));
  const int64_t S = ((volatile int64_t *)ctx->h_stage)[0];
  if (((volatile int64_t *)ctx->h_stage)[1])
    FAIL(GSM_ERR_TIMEOUT, "a verification tile waited too long for its predecessors");
  ctx->kstats[K_FUSED].algo_bytes += (double)S * (last ? (double)R.acc_row_bytes() : 8.0);
  if (last) {
    R.acc_rows += (uint64_t)S;
    return;
  }
  if (S > 0) {
    CFrontier next = f;
    next.V[i + 1] = Vn;
    next.P[i + 1] = Pn;
    recurse_c(R, i + 1, next, S);
  }
  stack_release(ctx, mk);
}

void recurse_c(Run &R, int32_t i, const CFrontier &f, int64_t rows) {
  gsm_ctx *ctx = R.ctx;
  if (rows <= 0) return;
  const LevelDesc &d = R.lv[i];
  const Mark mk = stack_mark(ctx);
  int32_t *pstart = (int32_t *)stack_push(ctx, sizeof(int32_t) * rows);
  uint8_t *pslot = (uint8_t *)stack_push(ctx, rows);
  int64_t *woff = (int64_t *)stack_push(ctx, sizeof(int64_t) * (rows + 1));
  int64_t *tmp = (int64_t *)scratch_get(ctx, sizeof(int64_t) * scan_tmp_elems(rows));
  timed(ctx, K_PIVOT, (double)rows * (8.0 * i + 8.0 * d.nb + 13.0 + 16.0), (uint64_t)rows,
        1 + scan_kernels(rows), [&] {
    launch_cpivot(R.g, d, f, i, rows, pstart, pslot, woff, ctx->stream);
    launch_scan_i64(woff, woff, rows, tmp, ctx->stream);
  });
  const int64_t W = read_i64(ctx, woff + rows);
  ctx->run.frontier[i] += (uint64_t)rows;
  ctx->run.candidates[i] += (uint64_t)W;
  std::vector<int64_t> bnd, bw;
  level_chunks(R, woff, rows, W, bnd, bw);
  for (size_t j = 0; j + 1 < bnd.size(); ++j)
    process_c(R, i, f, pstart, pslot, woff, bnd[j], bnd[j + 1], bw[j], bw[j + 1]);
  stack_release(ctx, mk);
}

void fill_filter(gsm_ctx *ctx, const gsm_query *q, const int32_t *dense, FilterDesc &fd) {
  std::memset(&fd, 0, sizeof(fd));
  fd.k = q->k;
  fd.n_words = (ctx->n + 31) / 32;
  for (int32_t u = 0; u < q->k; ++u) {
    fd.qlab[u] = dense[u];
    fd.qdeg[u] = popc(q->adj[u]);
    fd.lo[u] = std::max<int32_t>(0, q->lo[u]);
    fd.hi[u] = std::min<int32_t>(ctx->n, q->hi[u]);
  }
  if (ctx->label_values.size() <= 1) return;  // one label: counts equal degrees
  for (int32_t u = 0; u < q->k; ++u) {
    int32_t lab_of[kMaxK], cnt_of[kMaxK], nl = 0;
    for (int32_t w = 0; w < q->k; ++w) {
      if (!(q->adj[u] >> w & 1u)) continue;
      int32_t j = 0;
      while (j < nl && lab_of[j] != dense[w]) ++j;
      if (j == nl) {
        lab_of[nl] = dense[w];
        cnt_of[nl++] = 0;
      }
      cnt_of[j]++;
    }
    for (int32_t j = 0; j < nl; ++j) {
      int32_t s = 0;
      while (s < fd.nslots && fd.slot_label[s] != lab_of[j]) ++s;
      if (s == fd.nslots) fd.slot_label[fd.nslots++] = lab_of[j];
      fd.req_slot[u][fd.nreq[u]] = s;
      fd.req_cnt[u][fd.nreq[u]++] = cnt_of[j];
    }
  }
}

// Maps query labels to the graph's dense label ids; false if one is absent.
bool dense_labels(gsm_ctx *ctx, const gsm_query *q, int32_t *dense) {
  for (int32_t u = 0; u < q->k; ++u) {
    auto it = std::lower_bound(ctx->label_values.begin(), ctx->label_values.end(), q->labels[u]);
    if (it == ctx->label_values.end() || *it != q->labels[u]) return false;
    dense[u] = (int32_t)(it - ctx->label_values.begin());
  }
  return true;
}

// Filtering step: fills the k candidate bitmaps and returns |C(u)|; then
// opt.filter_rounds refinement rounds (double-buffered, so every round reads
// the previous round's sets only).
void run_filter(gsm_ctx *ctx, const gsm_query *q, const int32_t *dense, uint64_t *sizes) {
  const Range range("gsm filter");
  FilterDesc fd;
  fill_filter(ctx, q, dense, fd);
  const size_t bytes = (size_t)q->k * fd.n_words * sizeof(uint32_t);
  ensure_buf(ctx, &ctx->bitmaps, &ctx->bitmaps_cap, bytes, false, 0);
  CU(cudaMemsetAsync(ctx->d_small, 0, sizeof(unsigned long long) * kMaxK, ctx->stream));
  GraphDev g = graph_dev(ctx);
  timed(ctx, K_FILTER, 12.0 * ctx->n + bytes, (uint64_t)ctx->n, 1, [&] {
    launch_filter(g, fd, (uint32_t *)ctx->bitmaps, ctx->d_small, ctx->stream);
  });
  const int32_t rounds = std::max<int32_t>(0, ctx->opt.filter_rounds);
  if (rounds > 0 && q->k > 1) {
    RefineDesc rd;
    std::memset(&rd, 0, sizeof(rd));
    rd.k = q->k;
    rd.n_words = fd.n_words;
    for (int32_t u = 0; u < q->k; ++u) {
      for (int32_t w = 0; w < q->k; ++w) {
        if (!(q->adj[u] >> w & 1u)) continue;
        int32_t gi = 0;
        while (gi < rd.ngroups[u] && dense[__builtin_ctz(rd.group_mask[u][gi])] != dense[w]) ++gi;
        if (gi == rd.ngroups[u]) rd.ngroups[u]++;
        rd.group_mask[u][gi] |= 1u << w;
        rd.group_need[u][gi]++;
      }
    }
    ensure_buf(ctx, &ctx->bitmaps2, &ctx->bitmaps2_cap, bytes, false, 0);
    for (int32_t r = 0; r < rounds; ++r) {
      CU(cudaMemsetAsync(ctx->d_small, 0, sizeof(unsigned long long) * kMaxK, ctx->stream));
      timed(ctx, K_FILTER, 4.0 * ctx->nnz + 2.0 * bytes, (uint64_t)ctx->n, 1, [&] {
        launch_refine(g, rd, (const uint32_t *)ctx->bitmaps, (uint32_t *)ctx->bitmaps2,
                      ctx->d_small, ctx->stream);
      });
      std::swap(ctx->bitmaps, ctx->bitmaps2);
      std::swap(ctx->bitmaps_cap, ctx->bitmaps2_cap);
    }
  }
  fetch(ctx, ctx->d_small, sizeof(uint64_t) * q->k);
  std::memcpy(sizes, ctx->h_stage, sizeof(uint64_t) * q->k);
}

// The whole matcher for one query.  out == nullptr and !enumerate: count only.
// pre (optional): the query's candidate bitmaps and sizes, already computed
// by a batched filter launch (gsm_enumerate_many).
struct Prefiltered {
  const uint32_t *bitmaps;
  const uint64_t *sizes;
};

void run_query(gsm_ctx *ctx, const gsm_query *q, bool enumerate, int32_t *out, uint64_t cap_rows,
               int32_t flags, uint64_t *count_out, bool *truncated,
               const std::vector<std::pair<int32_t, int32_t>> *less = nullptr,
               bool copy_async = false, const Prefiltered *pre = nullptr) {
  if (!ctx->has_graph) FAIL(GSM_ERR_NO_GRAPH, "no data graph loaded");
  const Range range(enumerate ? "gsm query (list)" : "gsm query (count)");
  std::memset(&ctx->run, 0, sizeof(ctx->run));
  // nothing is live between calls (an earlier call may have failed mid-way)
  ctx->top_block = 0;
  ctx->top_used = 0;
  ctx->live_bytes = 0;
  ctx->last_rows = nullptr;
  ctx->last_count = 0;
  ctx->last_k = q->k;
  ctx->peak_bytes = 0;
  Run R;
  R.ctx = ctx;
  R.q = q;
  R.enumerate = enumerate;
  R.k = q->k;
  R.g = graph_dev(ctx);
  R.block = ctx->opt.block_size > 0 ? ctx->opt.block_size : 256;
  R.spin_limit = ctx->opt.lookback_spin_limit > 0 ? ctx->opt.lookback_spin_limit : kLbSpinLimit;
  R.stall_tile = (ctx->opt.flags & GSM_OPT_INJECT_LOOKBACK_STALL) ? 1 : -1;
  R.scan_stall_tile = (ctx->opt.flags & GSM_OPT_INJECT_SCAN_STALL) ? 1 : -1;
  R.chunk_rows = ctx->opt.chunk_rows;
  // masks take W/8 bytes and tile arrays 12 bytes per tile of scratch
  R.wcap = std::max<int64_t>((int64_t)ctx->max_deg + 1,
                             std::min<int64_t>((int64_t(1) << 30) - 4096,
                                               (int64_t)(ctx->scratch_limit / 2) * 7));
  R.d_total = ctx->d_small + kMaxK;
  ctx->run.k = q->k;
  *truncated = false;
  *count_out = 0;

  int32_t dense[kMaxK];
  uint64_t sizes[kMaxK] = {};
  if (!dense_labels(ctx, q, dense)) return;  // a query label absent from G: no embedding
  if (pre)
    std::memcpy(sizes, pre->sizes, sizeof(uint64_t) * q->k);
  else
    run_filter(ctx, q, dense, sizes);
  for (int32_t u = 0; u < q->k; ++u) ctx->run.cand_size[u] = sizes[u];
  for (int32_t u = 0; u < q->k; ++u)
    if (sizes[u] == 0) return;
  plan(q->k, q->adj, sizes, R.order, R.parent);
  for (int32_t i = 0; i < q->k; ++i) ctx->run.order[i] = R.order[i];
  // The levels emit rows in lexicographic order of the matching order.  If
  // query vertices sort_cols .. k-1 are placed in increasing id order, rows
  // that agree on columns 0 .. sort_cols-1 already stand in canonical order,
  // so only those columns need sorting; sort_cols == 0 (identity order): the
  // last level writes the result rows directly.
  int32_t sort_cols = q->k - 1;
  {
    int32_t pos[kMaxK];
    for (int32_t j = 0; j < q->k; ++j) pos[R.order[j]] = j;
    while (sort_cols > 0 && pos[sort_cols - 1] < pos[sort_cols]) --sort_cols;
  }
  int key_bits = 1;
  while (key_bits < 31 && (int64_t(1) << key_bits) < ctx->n) ++key_bits;
  R.acc_mode = sort_cols == 0 ? kSinkRows : kSinkKeys;
  R.key_bits = key_bits;
  R.key_nw = packed_words(q->k, key_bits);
  // rows leave the levels sorted by the columns of query vertices 0..p-1 when
  // the matching order starts with them; the last level then writes their
  // dense rank into the keys' spare bits (any int32 fits), so that the sort
  // keys those columns by it
  if (enumerate && R.acc_mode == kSinkKeys && !(ctx->opt.flags & GSM_OPT_COMPRESSED_FRONTIERS) &&
      R.key_nw <= 2 && sort_rank_pos(q->k, key_bits, sort_cols) + 31 <= 64 * R.key_nw) {
    int32_t p = 0;
    while (p < q->k && R.order[p] == p) ++p;
    if (p >= 1 && p < sort_cols) {
      R.rank_p = p;
      R.rank_pos = sort_rank_pos(q->k, key_bits, sort_cols);
      ensure_buf(ctx, &ctx->d_prefix, &ctx->d_prefix_cap, sizeof(PrefixState), false, 0);
      R.prefix = (PrefixState *)ctx->d_prefix;
      launch_prefix_state_reset(R.prefix, ctx->stream);
      ctx->run.kernel_launches += 1;
    }
  }

  const int32_t nw = (ctx->n + 31) / 32;
  const uint32_t *bm = pre ? pre->bitmaps : (const uint32_t *)ctx->bitmaps;
  for (int32_t i = 1; i < q->k; ++i) {
    LevelDesc &d = R.lv[i];
    std::memset(&d, 0, sizeof(d));
    const int32_t u = R.order[i];
    d.i = i;
    for (int32_t j = 0; j < i; ++j) {
      const int32_t uj = R.order[j];
      if (q->adj[u] >> uj & 1u)
        d.bpos[d.nb++] = j;  // ascending position: the first is the tree parent
      else if (dense[uj] == dense[u])
        d.inj[d.ninj++] = j;
    }
    for (int32_t j = 0; j <= i; ++j) d.out_col[j] = (i == q->k - 1) ? R.order[j] : j;
    d.bitmap = bm + (size_t)u * nw;
    d.lab = dense[u];
    d.la = std::max<int32_t>(0, ctx->opt.lookahead);
    d.cand = bm;
    d.n_words = nw;
    d.count_probes = (ctx->opt.flags & GSM_OPT_COUNT_PROBES) ? 1 : 0;
    if (d.la) {
      // query neighbours of pi_i placed after it, grouped by label
      uint32_t placed = 0;
      for (int32_t j = 0; j <= i; ++j) placed |= 1u << R.order[j];
      for (int32_t w = 0; w < q->k; ++w) {
        if (!(q->adj[u] >> w & 1u) || (placed >> w & 1u)) continue;
        int32_t t = 0;
        while (t < d.nla && d.la_lab[t] != dense[w]) ++t;
        if (t == d.nla) {
          d.la_lab[t] = dense[w];
          d.nla++;
        }
        d.la_need[t]++;
        d.la_uq[t] |= 1u << w;
      }
      for (int32_t t = 0; t < d.nla; ++t)
        for (int32_t j = 0; j < i; ++j) {
          const int32_t uj = R.order[j];
          if (dense[uj] != d.la_lab[t]) continue;
          if (q->adj[u] >> uj & 1u)
            d.la_known[t]++;
          else
            d.la_pos[t] |= 1u << j;
        }
    }
    if (less) {
      // ordering constraints between pi_i and vertices placed before it
      for (const auto &c : *less) {
        for (int32_t j = 0; j < i; ++j) {
          if (c.first == u && c.second == R.order[j]) d.lt[d.nlt++] = j;   // f(u) < f(pi_j)
          if (c.second == u && c.first == R.order[j]) d.gt[d.ngt++] = j;   // f(pi_j) < f(u)
        }
      }
    }
  }

  CU(cudaMemsetAsync(R.d_total, 0, sizeof(unsigned long long), ctx->stream));
  const Mark mk = stack_mark(ctx);
  const int64_t R1 = (int64_t)sizes[R.order[0]];
  int32_t *F1 = (int32_t *)stack_push(ctx, sizeof(int32_t) * R1);
  {
    Carve cv;
    const size_t o_cnt = cv.add<int32_t>(nw), o_off = cv.add<int64_t>(nw + 1),
                 o_tmp = cv.add<int64_t>(scan_tmp_elems(nw));
    char *sc = (char *)scratch_get(ctx, cv.off);
    timed(ctx, K_LIST, nw * 4.0 + 4.0 * R1, (uint64_t)R1, 2 + scan_kernels(nw), [&] {
      launch_bitmap_to_list(bm + (size_t)R.order[0] * nw, nw, (int32_t *)(sc + o_cnt),
                            (int64_t *)(sc + o_off), (int64_t *)(sc + o_tmp), F1, ctx->stream);
    });
  }
  ctx->run.frontier[1] = (uint64_t)R1;
  R.acc_ld = (int64_t)(ctx->acc_cap[0] / R.acc_row_bytes());
  if (q->k == 1) {
    if (enumerate) {
      ensure_acc(R, (uint64_t)R1);
      CU(cudaMemcpyAsync(ctx->acc[0], F1, sizeof(int32_t) * R1, cudaMemcpyDeviceToDevice,
                         ctx->stream));
    }
    R.acc_rows = (uint64_t)R1;
  } else if (ctx->opt.flags & GSM_OPT_COMPRESSED_FRONTIERS) {
    CFrontier f{};
    f.V[1] = F1;
    recurse_c(R, 1, f, R1);
  } else {
    recurse(R, 1, F1, R1, R1);
  }
  stack_release(ctx, mk);

  uint64_t total;
  if (enumerate || q->k == 1) {
    total = R.acc_rows;
  } else {
    fetch(ctx, R.d_total, sizeof(uint64_t));
    total = (uint64_t)ctx->h_stage[0];
  }
  ctx->run.frontier[q->k] = total;
  *count_out = total;
  if (!enumerate) return;

  // canonical order: the final rows are already the result (identity-like
  // order), or their packed keys are sorted on columns 0 .. sort_cols-1 and
  // unpacked row-major into acc[1]
  int32_t *rows = (int32_t *)ctx->acc[0];
  if (R.acc_mode == kSinkKeys && total > 0) {
    const int32_t nw = R.key_nw;
    const size_t bytes = (size_t)total * q->k * sizeof(int32_t);
    const size_t key_bytes = (size_t)R.acc_ld * nw * sizeof(uint64_t);
    ensure_buf(ctx, &ctx->sort_keys, &ctx->sort_keys_cap, key_bytes, false, 0);
    ensure_buf(ctx, &ctx->acc[1], &ctx->acc_cap[1], bytes, false, 0);
    // the rows leave the levels sorted by the columns the matching order
    // places first in id order (0, 1, ..., p-1), with at most |F_p|
    // distinct prefixes
    SortPrefix pre;
    while (pre.cols < q->k && R.order[pre.cols] == pre.cols) ++pre.cols;
    pre.groups = pre.cols > 0 ? (int64_t)ctx->run.frontier[pre.cols] : 0;
    if (pre.cols == 0 || pre.groups <= 0) pre = SortPrefix();
    pre.ranked = R.rank_p > 0 && pre.cols == R.rank_p;  // the last level wrote the ranks
    // outside the budget, like the result buffers it serves
    ensure_buf(ctx, &ctx->sort_tmp, &ctx->sort_tmp_cap,
               sort_scratch_bytes((int64_t)total, q->k, R.key_bits, sort_cols, pre), false, 0);
    const Range sort_range("gsm sort");
    bool ranked = false;
    const int digits =
        sort_digit_passes((int64_t)total, q->k, R.key_bits, sort_cols, pre, &ranked);
    // key bytes read + written per digit pass; the prefix rank reads the
    // keys twice, writes the flags, scans them and rewrites the keys
    const double moved = 2.0 * (double)total * nw * sizeof(uint64_t) * digits +
                         (ranked ? (double)total * (3.0 * nw * 8.0 + 4.0 + 12.0) : 0.0);
    int launches = 0;
    timed(ctx, K_SORT, moved + (double)bytes, total, 0, [&] {
      launches = launch_sort_rows_packed(nullptr, 0, (int64_t)total, q->k, R.key_bits, sort_cols,
                                         (uint64_t *)ctx->acc[0], (uint64_t *)ctx->sort_keys,
                                         R.acc_ld, (int32_t *)ctx->acc[1], ctx->sort_tmp,
                                         R.spin_limit, ctx->d_flags, sort_stall_tile(ctx),
                                         ctx->stream, pre);
    });
    ctx->run.kernel_launches += launches;
    rows = (int32_t *)ctx->acc[1];
  }
  ctx->last_rows = rows;
  ctx->last_count = total;
  const uint64_t ncopy = std::min<uint64_t>(total, cap_rows);
  const cudaMemcpyKind kind =
      (flags & GSM_OUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (copy_async) {
    // copy out on the copy stream once the rows are complete; the compute
    // stream goes on with the next query in the other result slot
    if (ncopy) {
      CU(cudaEventRecord(ctx->rows_ready, ctx->stream));
      CU(cudaStreamWaitEvent(ctx->copy_stream, ctx->rows_ready, 0));
      CU(cudaMemcpyAsync(out, rows, (size_t)ncopy * q->k * sizeof(int32_t), kind,
                         ctx->copy_stream));
      CU(cudaEventRecord(ctx->active_copied, ctx->copy_stream));
      ctx->active_pending = true;
    }
  } else {
    if (ncopy)
      CU(cudaMemcpyAsync(out, rows, (size_t)ncopy * q->k * sizeof(int32_t), kind, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    check_sort_flag(ctx);
  }
  *truncated = total > cap_rows;
}

template <typename F>
gsm_status guarded(gsm_ctx *ctx, F &&f) {
  try {
    f();
    return GSM_OK;
  } catch (const Fail &e) {
    return e.code;
  } catch (const std::exception &e) {
    set_err(ctx, "internal error: %s", e.what());
    return GSM_ERR_OOM;
  }
}

// Adjacency bitmaps of the hubs: vertices of degree >= kHubMinDegree, the
// highest degrees first, as many as fit opt.hub_bitmap_bytes (ceil(n/32)
// words each).  A non-tree edge check against a hub is then one bit probe
// instead of a binary search of its long row.
constexpr int32_t kHubMinDegree = 32;
constexpr int64_t kHubBytesDefault = int64_t(512) << 20;

void build_hubs(gsm_ctx *ctx, const std::vector<int32_t> &h_rp) {
  const int32_t n = ctx->n;
  const int64_t budget =
      ctx->opt.hub_bitmap_bytes == 0 ? kHubBytesDefault : ctx->opt.hub_bitmap_bytes;
  const int32_t words = (n + 31) / 32;
  if (budget <= 0 || n == 0) return;
  const int64_t cap = budget / ((int64_t)words * 4);
  std::vector<int32_t> hubs;
  for (int32_t v = 0; v < n; ++v)
    if (h_rp[v + 1] - h_rp[v] >= kHubMinDegree) hubs.push_back(v);
  std::sort(hubs.begin(), hubs.end(), [&](int32_t a, int32_t b) {
    const int32_t da = h_rp[a + 1] - h_rp[a], db = h_rp[b + 1] - h_rp[b];
    return da != db ? da > db : a < b;
  });
  if ((int64_t)hubs.size() > cap) hubs.resize((size_t)cap);
  if (hubs.empty()) return;
  const int32_t H = (int32_t)hubs.size();
  std::vector<int32_t> idx(n, -1);
  for (int32_t h = 0; h < H; ++h) idx[hubs[h]] = h;
  ctx->d_hub = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * n);
  ctx->hub_bits_bytes = (size_t)H * words * sizeof(uint32_t);
  ctx->d_hub_bits = (uint32_t *)dev_alloc(ctx, ctx->hub_bits_bytes);
  int32_t *d_list = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * H);
  CU(cudaMemcpyAsync(ctx->d_hub, idx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                     ctx->stream));
  CU(cudaMemcpyAsync(d_list, hubs.data(), sizeof(int32_t) * H, cudaMemcpyHostToDevice,
                     ctx->stream));
  GraphDev g = graph_dev(ctx);
  launch_hub_bitmaps(g, d_list, H, words, ctx->d_hub_bits, ctx->stream);
  CU(cudaGetLastError());
  // label segment table of the hubs (labelled graphs, up to 4,096 labels)
  const int64_t L = (int64_t)ctx->label_values.size();
  if (L > 1 && L <= 4096) {
    ctx->hub_seg_bytes = sizeof(int32_t) * (size_t)H * (size_t)(L + 1);
    ctx->d_hub_seg = (int32_t *)dev_alloc(ctx, ctx->hub_seg_bytes);
    g.num_labels = (int32_t)L;
    launch_hub_segments(g, d_list, H, ctx->d_hub_seg, ctx->stream);
    CU(cudaGetLastError());
  }
  CU(cudaStreamSynchronize(ctx->stream));
  dev_free(ctx, d_list, sizeof(int32_t) * H);
  ctx->hub_count = H;
  ctx->hub_min_deg = h_rp[hubs.back() + 1] - h_rp[hubs.back()];
}

void clear_all_graphs(gsm_ctx *ctx);

void free_graph(gsm_ctx *ctx) {
  for (gsm_ctx *w : ctx->workers) free_graph(w);  // they borrow it (kept for the next graph)
  clear_all_graphs(ctx);
  if (ctx->borrowed_graph) {
    ctx->d_rp = ctx->d_col = ctx->d_lab = ctx->d_lcol = ctx->d_llab = ctx->d_hub = nullptr;
    ctx->d_hub_bits = nullptr;
    ctx->d_hub_seg = nullptr;
    ctx->d_nlc = nullptr;
    ctx->nlc_stride = 0;
    ctx->hub_count = 0;
    ctx->has_graph = false;
    ctx->borrowed_graph = false;
    ctx->label_values.clear();
    return;
  }
  if (ctx->d_rp) dev_free(ctx, ctx->d_rp, sizeof(int32_t) * (ctx->n + 1));
  if (ctx->d_col) dev_free(ctx, ctx->d_col, sizeof(int32_t) * std::max<int64_t>(ctx->nnz, 1));
  if (ctx->d_lab) dev_free(ctx, ctx->d_lab, sizeof(int32_t) * std::max<int32_t>(ctx->n, 1));
  if (ctx->d_lcol) dev_free(ctx, ctx->d_lcol, sizeof(int32_t) * std::max<int64_t>(ctx->nnz, 1));
  if (ctx->d_llab) dev_free(ctx, ctx->d_llab, sizeof(int32_t) * std::max<int64_t>(ctx->nnz, 1));
  if (ctx->d_hub) dev_free(ctx, ctx->d_hub, sizeof(int32_t) * std::max<int32_t>(ctx->n, 1));
  if (ctx->d_hub_bits) dev_free(ctx, ctx->d_hub_bits, ctx->hub_bits_bytes);
  if (ctx->d_hub_seg) dev_free(ctx, ctx->d_hub_seg, ctx->hub_seg_bytes);
  if (ctx->d_nlc) dev_free(ctx, ctx->d_nlc, (size_t)ctx->n * ctx->nlc_stride);
  ctx->d_nlc = nullptr;
  ctx->nlc_stride = 0;
  ctx->d_hub = nullptr;
  ctx->d_hub_bits = nullptr;
  ctx->d_hub_seg = nullptr;
  ctx->hub_seg_bytes = 0;
  ctx->hub_count = 0;
  ctx->hub_bits_bytes = 0;
  ctx->d_rp = ctx->d_col = ctx->d_lab = nullptr;
  ctx->d_lcol = ctx->d_llab = nullptr;
  ctx->has_graph = false;
  ctx->label_values.clear();
}

}  // namespace

// ------------------------------------------------------------------ batched form

namespace {

using Lane = gsm_ctx::BatchLane;

constexpr int64_t kBatchCapRows = int64_t(1) << 24;
constexpr int64_t kBatchCapElems = int64_t(1) << 27;
constexpr int64_t kBatchCapItems = int64_t(1) << 28;
constexpr int64_t kBatchCapFinal = int64_t(1) << 28;  // result arena elements (1 GiB)

template <typename T>
T *lane_alloc(gsm_ctx *ctx, Lane &L, int64_t elems) {
  const size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(elems, 1);
  void *p = dev_alloc(ctx, bytes);
  L.allocs.push_back({p, bytes});
  return (T *)p;
}

void lane_free_one(gsm_ctx *ctx, Lane &L, const void *p) {
  for (auto it = L.allocs.begin(); it != L.allocs.end(); ++it)
    if (it->first == p) {
      dev_free(ctx, it->first, it->second);
      L.allocs.erase(it);
      return;
    }
}

void lane_clear_graphs(Lane &L) {
  for (auto &kv : L.graphs) cudaGraphExecDestroy(kv.second);
  L.graphs.clear();
}

// Releases a lane's device memory, pinned buffers and graphs (not its stream).
void lane_release(gsm_ctx *ctx, Lane &L) {
  lane_clear_graphs(L);
  for (auto &pa : L.allocs) dev_free(ctx, pa.first, pa.second);
  L.allocs.clear();
  if (L.h_fds) cudaFreeHost(L.h_fds);
  if (L.h_qs) cudaFreeHost(L.h_qs);
  if (L.h_bm) cudaFreeHost(L.h_bm);
  if (L.h_counts) cudaFreeHost(L.h_counts);
  if (L.h_overflow) cudaFreeHost(L.h_overflow);
  if (L.h_state) cudaFreeHost(L.h_state);
  if (L.h_items) cudaFreeHost(L.h_items);
  L.h_items = nullptr;
  L.h_items_cap = 0;
  if (L.h_segs) cudaFreeHost(L.h_segs);
  L.h_segs = nullptr;
  L.h_segs_cap = 0;
  for (int j = 0; j < 6; ++j)
    if (L.srt[j]) dev_free(ctx, L.srt[j], L.srt_cap[j]);
  if (L.bitmaps) dev_free(ctx, L.bitmaps, L.bitmaps_cap);
  for (cudaEvent_t e : {L.ev0, L.ev1, L.ev_done})
    if (e) cudaEventDestroy(e);
  cudaStream_t st = L.stream;
  const bool own = L.own_stream;
  L = Lane();
  L.stream = st;
  L.own_stream = own;
}

// Fixed-capacity buffers (once), per-query arrays (grown with the batch).
void lane_workspace(gsm_ctx *ctx, Lane &L, int32_t nq, int64_t words_total) {
  BatchArgs &a = L.a;
  if (!L.ready) {
    L.cap_rows = ctx->batch_caps[0] ? ctx->batch_caps[0] : kBatchCapRows;
    L.cap_elems = ctx->batch_caps[1] ? ctx->batch_caps[1] : kBatchCapElems;
    L.cap_items = ctx->batch_caps[2] ? ctx->batch_caps[2] : kBatchCapItems;
    a.cap_rows = L.cap_rows;
    a.cap_elems = L.cap_elems;
    a.cap_items = L.cap_items;
    for (int j = 0; j < 2; ++j) {
      a.F[j] = lane_alloc<int32_t>(ctx, L, L.cap_elems);
      a.rseg[j] = lane_alloc<int32_t>(ctx, L, L.cap_rows);
    }
    a.pstart = lane_alloc<int32_t>(ctx, L, L.cap_rows);
    a.pslot = lane_alloc<uint8_t>(ctx, L, L.cap_rows);
    a.woff = lane_alloc<int64_t>(ctx, L, L.cap_rows + 1);
    const int64_t tiles = L.cap_items / 128 + 3;
    a.tile_row = lane_alloc<int32_t>(ctx, L, tiles);
    a.tile_cnt = lane_alloc<int32_t>(ctx, L, tiles);
    a.tile_off = lane_alloc<int64_t>(ctx, L, tiles);
    a.masks = lane_alloc<uint32_t>(ctx, L, L.cap_items / 32 + 256);  // + a tile of the largest block
    a.fmasks = lane_alloc<uint32_t>(ctx, L, L.cap_items / 32 + 256);
    a.ftile_cnt = lane_alloc<int32_t>(ctx, L, tiles);
    a.ftile_off = lane_alloc<int64_t>(ctx, L, tiles);
    a.state = lane_alloc<BatchStep>(ctx, L, kMaxK + 1);
    CU(cudaMallocHost(&L.h_state, sizeof(BatchStep) * (kMaxK + 1)));
    a.overflow = lane_alloc<int32_t>(ctx, L, 1);
    a.partials = lane_alloc<int64_t>(ctx, L, (int64_t)ctx->num_sms * 32 + 1);
    CU(cudaMallocHost(&L.h_overflow, sizeof(int32_t)));
    const int32_t nw = (ctx->n + 31) / 32;
    L.zero_bitmap = lane_alloc<uint32_t>(ctx, L, nw);
    CU(cudaMemsetAsync(L.zero_bitmap, 0, sizeof(uint32_t) * std::max(nw, 1), L.stream));
    CU(cudaEventCreate(&L.ev0));
    CU(cudaEventCreate(&L.ev1));
    CU(cudaEventCreateWithFlags(&L.ev_done, cudaEventDisableTiming));
    L.ready = true;
  }
  bool moved = false;
  if (nq > L.max_nq) {
    if (L.max_nq) {
      lane_free_one(ctx, L, a.fds);
      lane_free_one(ctx, L, a.bm_out);
      lane_free_one(ctx, L, a.qs);
      lane_free_one(ctx, L, a.counts);
      lane_free_one(ctx, L, a.sizes);
      cudaFreeHost(L.h_fds);
      cudaFreeHost(L.h_qs);
      cudaFreeHost(L.h_bm);
      cudaFreeHost(L.h_counts);
    }
    const int32_t cap = std::max(nq, 2 * L.max_nq);
    a.fds = lane_alloc<FilterDesc>(ctx, L, cap);
    a.bm_out = lane_alloc<uint32_t *>(ctx, L, cap);
    a.qs = lane_alloc<BatchQuery>(ctx, L, cap);
    a.counts = lane_alloc<unsigned long long>(ctx, L, cap);
    a.sizes = lane_alloc<unsigned long long>(ctx, L, (int64_t)cap * kMaxK);
    CU(cudaMallocHost(&L.h_fds, sizeof(FilterDesc) * cap));
    CU(cudaMallocHost(&L.h_qs, sizeof(BatchQuery) * cap));
    CU(cudaMallocHost(&L.h_bm, sizeof(uint32_t *) * cap));
    CU(cudaMallocHost(&L.h_counts, sizeof(unsigned long long) * cap));
    L.max_nq = cap;
    moved = true;
  }
  if (words_total > L.max_words_total) {
    if (L.max_words_total) {
      lane_free_one(ctx, L, a.wcnt);
      lane_free_one(ctx, L, a.woffs);
    }
    const int64_t cap = std::max<int64_t>(words_total, 2 * L.max_words_total);
    a.wcnt = lane_alloc<int32_t>(ctx, L, cap);
    a.woffs = lane_alloc<int64_t>(ctx, L, cap + 1);
    L.max_words_total = cap;
    moved = true;
  }
  if (moved) lane_clear_graphs(L);  // captured graphs hold the old pointers
}

// The result arena of enumerate batches, allocated on first use (captured
// graphs of enumerate batches hold its address, so it never moves).
void lane_final(gsm_ctx *ctx, Lane &L) {
  if (L.a.final_rows) return;
  L.cap_final = ctx->batch_caps[3] ? ctx->batch_caps[3] : kBatchCapFinal;
  L.a.cap_final = L.cap_final;
  L.a.final_rows = lane_alloc<int32_t>(ctx, L, L.cap_final);
}

// Grows lane sort buffer j to `bytes` (contents not kept).
void *lane_srt(gsm_ctx *ctx, Lane &L, int j, size_t bytes) {
  if (L.srt_cap[j] < bytes) CU(cudaStreamSynchronize(L.stream));  // the old buffer may be in use
  ensure_buf(ctx, &L.srt[j], &L.srt_cap[j], bytes, false, 0);
  return L.srt[j];
}

// Columns 0 .. sort_cols-1 of rows that the levels emitted in lexicographic
// order of the matching order still need sorting (see run_query); 0: none.
int32_t unsorted_columns(int32_t k, const int32_t *order) {
  int32_t pos[kMaxK];
  for (int32_t j = 0; j < k; ++j) pos[order[j]] = j;
  int32_t sort_cols = k - 1;
  while (sort_cols > 0 && pos[sort_cols - 1] < pos[sort_cols]) --sort_cols;
  return sort_cols;
}

// Element offset in the result arena of every selected query that listed
// rows (-1 for the others), from the step sizes read back after the batch:
// step k-1 holds the queries of k vertices, in batch order.
std::vector<int64_t> lane_row_offsets(const Lane &L, const unsigned long long *counts) {
  std::vector<int64_t> off(L.m, -1);
  int64_t next[kMaxK + 1];
  for (int32_t i = 0; i <= kMaxK; ++i) next[i] = L.h_state[i].FB;
  for (int32_t t = 0; t < L.m; ++t) {
    const int32_t k = L.h_qs[t].k;
    if (!L.lists[t] || k < 2) continue;
    off[t] = next[k - 1];
    next[k - 1] += (int64_t)counts[t] * k;
  }
  return off;
}

// Estimated |C(u)|: vertices with u's label and at least u's degree (the
// label / degree probability the paper borrows from VF3), scaled by u's
// restriction range.
uint64_t estimate_candidates(gsm_ctx *ctx, const gsm_query *q, int32_t u, int32_t dense_label) {
  const auto &d = ctx->deg_by_label[dense_label];
  const int32_t qdeg = popc(q->adj[u]);
  uint64_t c = (uint64_t)(d.end() - std::lower_bound(d.begin(), d.end(), qdeg));
  const int64_t lo = std::max<int64_t>(0, q->lo[u]), hi = std::min<int64_t>(ctx->n, q->hi[u]);
  if (hi - lo < ctx->n && ctx->n > 0) {
    const double f = hi > lo ? (double)(hi - lo) / ctx->n : 0.0;
    c = c ? std::max<uint64_t>(1, (uint64_t)(c * f)) : 0;
  }
  return c;
}

// Plans q with the histogram estimates; returns the largest estimated
// frontier (rows) over its levels: est_1 = |C(pi_0)|, and each level
// multiplies by the mean degree, the fraction of vertices in C(pi_i), and
// (mean degree / n) per non-tree edge.
double plan_estimated(gsm_ctx *ctx, const gsm_query *q, const int32_t *dense, int32_t *order) {
  uint64_t est[kMaxK];
  for (int32_t u = 0; u < q->k; ++u) est[u] = estimate_candidates(ctx, q, u, dense[u]);
  int32_t parent[kMaxK];
  plan(q->k, q->adj, est, order, parent);
  const double n = std::max<double>(1.0, ctx->n);
  const double dbar = ctx->nnz / n;
  double rows = (double)est[order[0]], peak = rows;
  uint32_t placed = 1u << order[0];
  for (int32_t i = 1; i < q->k; ++i) {
    const int32_t u = order[i];
    const int nb = popc(q->adj[u] & placed);
    rows *= dbar * ((double)est[u] / n);
    for (int j = 1; j < nb; ++j) rows *= dbar / n;
    peak = std::max(peak, rows);
    placed |= 1u << u;
  }
  return peak;
}

cudaGraphExec_t lane_graph(gsm_ctx *ctx, Lane &L, int32_t m, int32_t kmax, int32_t n_words,
                           int32_t block, int32_t grid) {
  const auto key = std::make_tuple(m, kmax, n_words, block, grid, L.enumerate);
  auto it = L.graphs.find(key);
  if (it != L.graphs.end()) return it->second;
  if (L.enumerate) lane_final(ctx, L);
  BatchArgs a = L.a;
  a.enumerate = L.enumerate;
  a.nq = m;
  a.kmax = kmax;
  a.n_words = n_words;
  a.block = block;
  a.grid = grid;
  GraphDev g = graph_dev(ctx);
  cudaGraph_t graph = nullptr;
  CU(cudaStreamBeginCapture(L.stream, cudaStreamCaptureModeThreadLocal));
  const int launches = batch_enqueue(g, a, L.stream);
  cudaError_t e = cudaStreamEndCapture(L.stream, &graph);
  if (e != cudaSuccess) {
    set_err(ctx, "capturing the batch graph failed: %s", cudaGetErrorString(e));
    throw Fail{GSM_ERR_CUDA};
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    set_err(ctx, "instantiating the batch graph failed: %s", cudaGetErrorString(e));
    throw Fail{GSM_ERR_CUDA};
  }
  L.graphs[key] = exec;
  ctx->bstats.graphs_built += 1;
  ctx->bstats.kernels_per_graph = (uint64_t)launches;
  return exec;
}

// Batch shapes are bucketed so that few graphs serve every batch: the number
// of queries is rounded up to a power of two (the extra slots hold padding
// queries that match nothing); the largest query size is kept exact, since
// every level costs its launches even when it has no rows.
int32_t bucket_queries(int32_t m) {
  int32_t b = 1;
  while (b < m) b <<= 1;
  return b;
}
int32_t bucket_size(int32_t k) { return k; }

// Host part of a batch: labels, filter descriptions, orders, level
// descriptions, uploaded (asynchronously) to the lane, padded to the bucketed
// shape (L.mb queries).  L.sel = indices of the queries that can match (a
// label absent from G means 0).  lists (may be null): lists[j] != 0 if query
// j lists its rows (queries of two or more vertices write them into the
// result arena).  Returns the bucketed largest query size.
int32_t lane_prepare(gsm_ctx *ctx, Lane &L, const gsm_query *const *qs, int32_t nq,
                     const int32_t *lists = nullptr) {
  const int32_t n_words = (ctx->n + 31) / 32;
  L.sel.clear();
  L.orders.clear();
  L.lists.clear();
  L.enumerate = 0;
  std::vector<std::array<int32_t, kMaxK>> dense_of;
  int64_t total_k = 0;
  for (int32_t j = 0; j < nq; ++j) {
    std::array<int32_t, kMaxK> dn{};
    if (!dense_labels(ctx, qs[j], dn.data())) continue;
    L.sel.push_back(j);
    dense_of.push_back(dn);
    total_k += qs[j]->k;
  }
  L.m = (int32_t)L.sel.size();
  if (L.m == 0) return 0;
  L.mb = bucket_queries(L.m);
  const size_t bm_bytes = (size_t)total_k * n_words * sizeof(uint32_t);
  if (L.bitmaps_cap < bm_bytes) {
    // graphs stay valid: bitmap addresses travel in the per-batch descriptors
    CU(cudaStreamSynchronize(L.stream));
    ensure_buf(ctx, &L.bitmaps, &L.bitmaps_cap, bm_bytes, false, 0);
  }
  lane_workspace(ctx, L, L.mb, (int64_t)L.mb * n_words);
  uint32_t *bm = (uint32_t *)L.bitmaps;
  int32_t kmax = 1;
  int64_t off = 0;
  for (int32_t t = 0; t < L.m; ++t) {
    const gsm_query *q = qs[L.sel[t]];
    const int32_t *dense = dense_of[t].data();
    fill_filter(ctx, q, dense, L.h_fds[t]);
    int32_t order[kMaxK];
    plan_estimated(ctx, q, dense, order);
    uint32_t *base = bm + off;
    off += (int64_t)q->k * n_words;
    L.h_bm[t] = base;
    BatchQuery &bq = L.h_qs[t];
    std::memset(&bq, 0, sizeof(bq));
    bq.k = q->k;
    bq.root_bitmap = base + (size_t)order[0] * n_words;
    bq.enumerate = (lists && lists[L.sel[t]] && q->k >= 2) ? 1 : 0;
    L.enumerate |= bq.enumerate;
    for (int32_t j = 0; j < q->k; ++j) bq.out_col[j] = order[j];
    std::array<int32_t, kMaxK> ord{};
    for (int32_t j = 0; j < q->k; ++j) ord[j] = order[j];
    L.orders.push_back(ord);
    L.lists.push_back(lists && lists[L.sel[t]] ? 1 : 0);
    for (int32_t i = 1; i < q->k; ++i) {
      BatchLevel &lv = bq.lv[i];
      const int32_t u = order[i];
      for (int32_t j = 0; j < i; ++j) {
        const int32_t uj = order[j];
        if (q->adj[u] >> uj & 1u)
          lv.bpos[lv.nb++] = j;
        else if (dense[uj] == dense[u])
          lv.inj[lv.ninj++] = j;
      }
      lv.last = i == q->k - 1;
      lv.lab = dense[u];
      lv.bitmap = base + (size_t)u * n_words;
    }
    kmax = std::max(kmax, q->k);
  }
  for (int32_t t = L.m; t < L.mb; ++t) {  // padding: no filter work, nothing to count
    std::memset(&L.h_fds[t], 0, sizeof(FilterDesc));
    L.h_bm[t] = L.zero_bitmap;
    std::memset(&L.h_qs[t], 0, sizeof(BatchQuery));
    L.h_qs[t].k = 1;
    L.h_qs[t].root_bitmap = L.zero_bitmap;
  }
  CU(cudaMemcpyAsync((void *)L.a.fds, L.h_fds, sizeof(FilterDesc) * L.mb, cudaMemcpyHostToDevice,
                     L.stream));
  CU(cudaMemcpyAsync((void *)L.a.bm_out, L.h_bm, sizeof(uint32_t *) * L.mb,
                     cudaMemcpyHostToDevice, L.stream));
  CU(cudaMemcpyAsync((void *)L.a.qs, L.h_qs, sizeof(BatchQuery) * L.mb, cudaMemcpyHostToDevice,
                     L.stream));
  L.kb = bucket_size(kmax);
  return L.kb;
}

// Issues the prepared batch: graph launch, then the counts and the overflow
// flag back to pinned memory, then ev_done (all asynchronous).
void lane_issue(gsm_ctx *ctx, Lane &L, int32_t kmax, int32_t block, int32_t grid) {
  const int32_t n_words = (ctx->n + 31) / 32;
  cudaGraphExec_t exec = lane_graph(ctx, L, L.mb, kmax, n_words, block, grid);
  CU(cudaEventRecord(L.ev0, L.stream));
  CU(cudaGraphLaunch(exec, L.stream));
  CU(cudaEventRecord(L.ev1, L.stream));
  CU(cudaMemcpyAsync(L.h_counts, L.a.counts, sizeof(unsigned long long) * L.m,
                     cudaMemcpyDeviceToHost, L.stream));
  CU(cudaMemcpyAsync(L.h_overflow, L.a.overflow, sizeof(int32_t), cudaMemcpyDeviceToHost,
                     L.stream));
  CU(cudaMemcpyAsync(L.h_state, L.a.state, sizeof(BatchStep) * (kMaxK + 1),
                     cudaMemcpyDeviceToHost, L.stream));
  CU(cudaEventRecord(L.ev_done, L.stream));
  ctx->bstats.graph_launches += 1;
  ctx->bstats.block_size = block;
  ctx->bstats.grid = grid;
}

// Waits for the issued batch; returns the overflow flag, *ms = graph time.
bool lane_wait(gsm_ctx *ctx, Lane &L, float *ms) {
  CU(cudaEventSynchronize(L.ev_done));
  if (ms) CU(cudaEventElapsedTime(ms, L.ev0, L.ev1));
  return *L.h_overflow != 0;
}

std::pair<int32_t, int32_t> batch_config(gsm_ctx *ctx, int32_t m, int32_t kmax, bool *tuned) {
  int32_t mb = 1;
  while (mb < m) mb <<= 1;
  auto it = ctx->tuned.find({mb, kmax});
  *tuned = it != ctx->tuned.end();
  if (*tuned) return it->second;
  return {256, ctx->num_sms * 4};
}

// Result rows of one query through the single-query path (count rows into a
// new buffer: host memory, or device memory from the context's allocator).
void single_query_rows(gsm_ctx *ctx, const gsm_query *q, bool on_device, gsm_result *r) {
  uint64_t c = 0;
  bool trunc = false;
  run_query(ctx, q, true, nullptr, 0, 0, &c, &trunc);
  r->count = c;
  r->k = q->k;
  r->on_device = on_device ? 1 : 0;
  r->rows = nullptr;
  if (c == 0) return;
  const size_t bytes = (size_t)c * q->k * sizeof(int32_t);
  if (on_device) {
    r->rows = (int32_t *)dev_alloc(ctx, bytes);
    CU(cudaMemcpyAsync(r->rows, ctx->last_rows, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    r->rows = (int32_t *)std::malloc(bytes);
    if (!r->rows) FAIL(GSM_ERR_OOM, "host allocation of %zu bytes failed", bytes);
    CU(cudaMemcpyAsync(r->rows, ctx->last_rows, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  }
  CU(cudaStreamSynchronize(ctx->stream));
}

// Result rows of a listing batch share one allocation (host, or device
// memory from the context's allocator): every result's rows pointer points
// into the block, which is released with the last of them.  Keyed by the
// rows pointer; process-wide, so host rows can be released without a
// context.
struct RowBlock {
  void *base;
  size_t bytes;
  bool on_device;
  int32_t refs;
};
std::mutex g_blocks_mu;
std::unordered_map<const void *, RowBlock *> g_block_of;

// Drops one reference to the block holding p.  Returns false if p is not in
// a block; otherwise *last = the block to free (null while others remain).
bool block_unref(const void *p, RowBlock **last) {
  std::lock_guard<std::mutex> lk(g_blocks_mu);
  auto it = g_block_of.find(p);
  if (it == g_block_of.end()) return false;
  RowBlock *b = it->second;
  g_block_of.erase(it);
  *last = --b->refs == 0 ? b : nullptr;
  return true;
}

// Host rows handed out by the library (a block member or a malloc'd array).
void release_host_rows(int32_t *p) {
  if (!p) return;
  RowBlock *b = nullptr;
  if (!block_unref(p, &b)) {
    std::free(p);
    return;
  }
  if (b) {
    std::free(b->base);
    delete b;
  }
}

void release_rows(gsm_ctx *ctx, gsm_result *r) {
  if (!r->rows) return;
  RowBlock *b = nullptr;
  if (block_unref(r->rows, &b)) {
    if (b) {
      if (b->on_device)
        dev_free(ctx, b->base, b->bytes);
      else
        std::free(b->base);
      delete b;
    }
  } else if (r->on_device) {
    dev_free(ctx, r->rows, (size_t)r->count * r->k * sizeof(int32_t));
  } else {
    std::free(r->rows);
  }
  r->rows = nullptr;
}

// Grows pinned host staging *p to hold `bytes` (contents not kept; the
// lane's stream is synchronised first, as an earlier upload may read it).
template <typename T>
T *lane_pinned(gsm_ctx *ctx, Lane &L, T **p, size_t *cap, size_t bytes) {
  if (*cap < bytes) {
    CU(cudaStreamSynchronize(L.stream));
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    const size_t want = std::max(bytes, size_t(4096));
    CU(cudaHostAlloc((void **)p, want, cudaHostAllocDefault));
    *cap = want;
  }
  return *p;
}

// Rows of the selected queries t of a finished listing batch on lane L with
// want[t] (k >= 2), canonicalised into results[L.sel[t]], all in one block
// (host, or device memory from the context's allocator).  Results of at most
// kSmallSortRows rows are sorted together by one launch (a CTA each); larger
// ones whose matching order is not canonical are sorted together per query
// size, as one segmented sort (the query's index within the group as the
// key's most significant part: the arena already holds each query's rows
// contiguously, queries in batch order), straight into their place in the
// block; the rest are copied.  Host results are staged on the device and
// copied back in one transfer; the caller synchronises the lane's stream.
void lane_batch_rows(gsm_ctx *ctx, Lane &L, const std::vector<int64_t> &off,
                     const std::vector<char> &want, bool on_device, gsm_result *results) {
  // the groups (per k, in batch order) take the front of the block, their
  // rows contiguous; every other result follows at a 16-byte aligned offset
  std::map<int32_t, std::vector<int32_t>> groups;
  std::vector<int32_t> rest;
  std::vector<int32_t> sort_cols(L.m, 0);
  for (int32_t t = 0; t < L.m; ++t) {
    const int32_t k = L.h_qs[t].k;
    if (!want[t] || k < 2) continue;
    gsm_result &r = results[L.sel[t]];
    r.count = L.h_counts[t];
    r.k = k;
    r.on_device = on_device ? 1 : 0;
    r.rows = nullptr;
    if (r.count == 0) continue;
    sort_cols[t] = unsorted_columns(k, L.orders[t].data());
    if (r.count > (uint64_t)kSmallSortRows && sort_cols[t] > 0)
      groups[k].push_back(t);
    else
      rest.push_back(t);
  }
  if (groups.empty() && rest.empty()) return;
  std::vector<size_t> pos(L.m, 0);
  size_t total = 0;
  for (const auto &kv : groups) {
    for (int32_t t : kv.second) {
      pos[t] = total;
      total += (size_t)L.h_counts[t] * kv.first;
    }
    total = (total + 3) & ~size_t(3);
  }
  for (int32_t t : rest) {
    pos[t] = total;
    total += ((size_t)L.h_counts[t] * L.h_qs[t].k + 3) & ~size_t(3);
  }
  const size_t bytes = total * sizeof(int32_t);
  void *base = on_device ? dev_alloc(ctx, bytes) : std::malloc(bytes);
  if (!base) FAIL(GSM_ERR_OOM, "host allocation of %zu bytes failed", bytes);
  {
    int32_t nres = (int32_t)rest.size();
    for (const auto &kv : groups) nres += (int32_t)kv.second.size();
    RowBlock *b = new RowBlock{base, bytes, on_device, nres};
    std::lock_guard<std::mutex> lk(g_blocks_mu);
    auto own = [&](int32_t t) {
      int32_t *p = (int32_t *)base + pos[t];
      results[L.sel[t]].rows = p;
      g_block_of[p] = b;
    };
    for (const auto &kv : groups)
      for (int32_t t : kv.second) own(t);
    for (int32_t t : rest) own(t);
  }
  int32_t *dst = on_device ? (int32_t *)base : (int32_t *)lane_srt(ctx, L, 4, bytes);
  int32_t bits = 1;
  while (bits < 31 && (int64_t(1) << bits) < ctx->n) ++bits;
  // segmented sorts, one per query size
  if (!groups.empty()) {
    size_t nsegs = 0;
    for (const auto &kv : groups) nsegs += kv.second.size();
    SortSegment *h =
        lane_pinned(ctx, L, &L.h_segs, &L.h_segs_cap, nsegs * sizeof(SortSegment));
    SortSegment *d = (SortSegment *)lane_srt(ctx, L, 5, nsegs * sizeof(SortSegment));
    size_t e = 0;
    for (const auto &kv : groups) {
      int64_t first = 0;
      for (int32_t t : kv.second) {
        h[e++] = SortSegment{L.a.final_rows + off[t], first, (int64_t)L.h_counts[t]};
        first += (int64_t)L.h_counts[t];
      }
    }
    CU(cudaMemcpyAsync(d, h, nsegs * sizeof(SortSegment), cudaMemcpyHostToDevice, L.stream));
    e = 0;
    for (const auto &kv : groups) {
      const int32_t k = kv.first, nseg = (int32_t)kv.second.size();
      int64_t N = 0;
      int32_t S = 1;
      for (int32_t t : kv.second) {
        N += (int64_t)L.h_counts[t];
        S = std::max(S, sort_cols[t]);
      }
      SortPrefix pre;
      pre.given_bits = 1;
      while ((int64_t(1) << pre.given_bits) < nseg) ++pre.given_bits;
      const int32_t nw = sort_key_words(k, bits, pre);
      uint64_t *ka = (uint64_t *)lane_srt(ctx, L, 0, (size_t)N * nw * sizeof(uint64_t));
      uint64_t *kb = (uint64_t *)lane_srt(ctx, L, 1, (size_t)N * nw * sizeof(uint64_t));
      void *scratch = lane_srt(ctx, L, 2, sort_scratch_bytes(N, k, bits, S, pre));
      launch_pack_segments(d + e, nseg, N, k, bits, pre.given_bits, nw, ka, N, L.stream);
      launch_sort_rows_packed(nullptr, 0, N, k, bits, S, ka, kb, N, dst + pos[kv.second[0]],
                              scratch, ctx->opt.lookback_spin_limit, ctx->d_flags,
                              sort_stall_tile(ctx), L.stream, pre);
      CU(cudaGetLastError());
      e += (size_t)nseg;
    }
  }
  std::vector<SmallSortItem> items;
  int32_t max_k = 2;
  for (int32_t t : rest) {
    const int32_t k = L.h_qs[t].k;
    const int64_t N = (int64_t)L.h_counts[t];
    const int32_t *src = L.a.final_rows + off[t];
    if (N <= kSmallSortRows) {
      items.push_back({src, dst + pos[t], (int32_t)N, k, sort_cols[t] > 0 ? 1 : 0});
      max_k = std::max(max_k, k);
    } else {  // canonical order already
      CU(cudaMemcpyAsync(dst + pos[t], src, (size_t)N * k * sizeof(int32_t),
                         cudaMemcpyDeviceToDevice, L.stream));
    }
  }
  if (!items.empty()) {
    const size_t ib = items.size() * sizeof(SmallSortItem);
    SmallSortItem *h = lane_pinned(ctx, L, &L.h_items, &L.h_items_cap, ib);
    std::memcpy(h, items.data(), ib);
    void *d_items = lane_srt(ctx, L, 3, ib);
    CU(cudaMemcpyAsync(d_items, h, ib, cudaMemcpyHostToDevice, L.stream));
    launch_sort_small((const SmallSortItem *)d_items, (int32_t)items.size(), max_k, L.stream);
    CU(cudaGetLastError());
  }
  if (!on_device) CU(cudaMemcpyAsync(base, dst, bytes, cudaMemcpyDeviceToHost, L.stream));
}

void run_batch(gsm_ctx *ctx, const gsm_query *const *qs, int32_t nq, uint64_t *counts,
               gsm_result *results, int32_t flags) {
  const Range range("gsm batch");
  if (!ctx->has_graph) FAIL(GSM_ERR_NO_GRAPH, "no data graph loaded");
  const auto t0 = std::chrono::steady_clock::now();
  Lane &L = ctx->lane0;
  L.stream = ctx->stream;
  const bool on_device = flags & GSM_OUT_DEVICE;
  for (int32_t j = 0; j < nq; ++j) {
    counts[j] = 0;
    if (results) {
      std::memset(&results[j], 0, sizeof(gsm_result));
      results[j].k = qs[j]->k;
      results[j].on_device = on_device ? 1 : 0;
    }
  }
  ctx->bstats.batches += 1;
  ctx->bstats.overflowed = 0;
  std::vector<int32_t> lists(nq, results ? 1 : 0);
  const int32_t kmax = lane_prepare(ctx, L, qs, nq, lists.data());
  if (L.m == 0) return;
  bool tuned = false;
  auto cfg = batch_config(ctx, L.m, kmax, &tuned);
  bool overflow = false;
  float ms = 0;
  if (!tuned && (flags & GSM_BATCH_AUTOTUNE)) {
    const int32_t cand[][2] = {{128, 8}, {256, 4}, {256, 8}, {512, 2}, {512, 4}, {1024, 2}};
    float best = 1e30f;
    for (const auto &c : cand) {
      float t = 0;
      lane_issue(ctx, L, kmax, c[0], ctx->num_sms * c[1]);
      overflow = lane_wait(ctx, L, &t);
      if (overflow) break;  // every configuration gives the same results
      if (t < best) {
        best = t;
        cfg = {c[0], ctx->num_sms * c[1]};
      }
    }
    ms = best;
    if (!overflow) {
      int32_t mb = 1;
      while (mb < L.m) mb <<= 1;
      ctx->tuned[{mb, kmax}] = cfg;
      tuned = true;
    }
  } else {
    lane_issue(ctx, L, kmax, cfg.first, cfg.second);
    overflow = lane_wait(ctx, L, &ms);
  }
  ctx->bstats.tuned = tuned ? 1 : 0;
  ctx->bstats.block_size = cfg.first;
  ctx->bstats.grid = cfg.second;
  try {
    if (overflow) {
      // the workspace was too small for this batch: run it query by query
      ctx->bstats.overflowed = 1;
      ctx->bstats.fallbacks += 1;
      for (int32_t t = 0; t < L.m; ++t) {
        const int32_t j = L.sel[t];
        if (results) {
          single_query_rows(ctx, qs[j], on_device, &results[j]);
          counts[j] = results[j].count;
        } else {
          uint64_t c = 0;
          bool trunc = false;
          run_query(ctx, qs[j], false, nullptr, 0, 0, &c, &trunc);
          counts[j] = c;
        }
      }
    } else {
      for (int32_t t = 0; t < L.m; ++t) counts[L.sel[t]] = L.h_counts[t];
      if (results) {
        const std::vector<int64_t> off = lane_row_offsets(L, L.h_counts);
        for (int32_t t = 0; t < L.m; ++t) {
          const int32_t j = L.sel[t];
          if (qs[j]->k == 1)  // one-vertex queries: their candidate list
            single_query_rows(ctx, qs[j], on_device, &results[j]);
        }
        lane_batch_rows(ctx, L, off, std::vector<char>(L.m, 1), on_device, results);
        CU(cudaStreamSynchronize(L.stream));
        check_sort_flag(ctx);
      }
    }
  } catch (...) {
    if (results)
      for (int32_t j = 0; j < nq; ++j) release_rows(ctx, &results[j]);
    throw;
  }
  if (results)
    for (int32_t j = 0; j < nq; ++j) results[j].count = counts[j];
  ctx->bstats.last_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

// ------------------------------------------------------------------ served form
//
// A request loop on a thread of its own.  Submitted queries wait in a FIFO;
// whenever a lane (stream + batch workspace) is free, the loop admits waiting
// queries into a new batch while their estimated peak frontiers fit half the
// lane's frontier capacity (at least one query per batch), launches it, and
// goes back to admitting: a request that arrives while batches are running
// joins the next free lane, so its work overlaps theirs on the device.  A
// lane's results are collected by polling its completion event.  A batch
// that overflows its workspace is recounted query by query (a bad estimate
// costs latency, not correctness).

struct gsm_ctx::Server {
  struct Req {
    uint64_t ticket = 0;
    const gsm_query *q = nullptr;
    int32_t mode = GSM_MODE_COUNT;
    double est_rows = 0;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    uint64_t count = 0;
    int32_t *rows = nullptr;  // enumerate mode: host rows, handed over by gsm_poll
    gsm_status status = GSM_PENDING;
  };
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<Req> waiting;
  std::unordered_map<uint64_t, Req> inflight, finished;
  uint64_t next_ticket = 1;
  int32_t max_batch = 256;
  std::vector<std::unique_ptr<Lane>> lanes;
  gsm_status fatal = GSM_OK;
};

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Completes the batch of a lane whose ev_done has fired: counts, and the
// sorted rows of the requests in enumerate mode.
void server_complete(gsm_ctx *ctx, gsm_ctx::Server &S, Lane &L) {
  const bool overflow = *L.h_overflow != 0;
  std::vector<const gsm_query *> qs;
  std::vector<int32_t> modes;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    for (uint64_t t : L.tickets) {
      qs.push_back(S.inflight[t].q);
      modes.push_back(S.inflight[t].mode);
    }
  }
  const size_t nr = L.tickets.size();
  std::vector<uint64_t> counts(nr, 0);
  std::vector<gsm_result> res(nr);
  for (auto &r : res) std::memset(&r, 0, sizeof(r));
  gsm_status st = guarded(ctx, [&] {
    try {
      if (overflow) {
        ctx->bstats.fallbacks += 1;
        for (size_t t = 0; t < nr; ++t) {
          if (modes[t] == GSM_MODE_ENUMERATE) {
            single_query_rows(ctx, qs[t], false, &res[t]);
            counts[t] = res[t].count;
          } else {
            bool trunc = false;
            run_query(ctx, qs[t], false, nullptr, 0, 0, &counts[t], &trunc);
          }
        }
      } else {
        for (int32_t t = 0; t < L.m; ++t) counts[L.sel[t]] = L.h_counts[t];
        if (L.enumerate || std::count(modes.begin(), modes.end(), GSM_MODE_ENUMERATE)) {
          const std::vector<int64_t> off = lane_row_offsets(L, L.h_counts);
          std::vector<char> want(L.m, 0);
          for (int32_t t = 0; t < L.m; ++t) {
            const int32_t j = L.sel[t];
            if (modes[j] != GSM_MODE_ENUMERATE) continue;
            if (qs[j]->k == 1)
              single_query_rows(ctx, qs[j], false, &res[j]);
            else
              want[t] = 1;
          }
          lane_batch_rows(ctx, L, off, want, false, res.data());
          CU(cudaStreamSynchronize(L.stream));
          check_sort_flag(ctx);
        }
      }
    } catch (...) {
      for (auto &r : res) release_rows(ctx, &r);
      throw;
    }
  });
  if (st != GSM_OK)
    for (auto &r : res) release_rows(ctx, &r);
  const int64_t t_done = now_ns();
  std::lock_guard<std::mutex> lk(S.mu);
  for (size_t t = 0; t < nr; ++t) {
    auto node = S.inflight.extract(L.tickets[t]);
    node.mapped().count = counts[t];
    node.mapped().rows = res[t].rows;
    node.mapped().status = st;
    node.mapped().t_done = t_done;
    S.finished.insert(std::move(node));
  }
  L.tickets.clear();
  L.busy = false;
}

void server_loop(gsm_ctx *ctx) {
  gsm_ctx::Server &S = *ctx->server;
  cudaSetDevice(ctx->device);
  for (;;) {
    bool progressed = false;
    // collect finished lanes
    for (auto &lp : S.lanes) {
      Lane &L = *lp;
      if (L.busy && cudaEventQuery(L.ev_done) == cudaSuccess) {
        server_complete(ctx, S, L);
        progressed = true;
      }
    }
    // admit waiting requests into free lanes
    for (auto &lp : S.lanes) {
      Lane &L = *lp;
      if (L.busy) continue;
      std::vector<const gsm_query *> qs;
      std::vector<int32_t> lists;
      {
        std::lock_guard<std::mutex> lk(S.mu);
        if (S.waiting.empty()) break;
        const double budget = 0.5 * (double)(ctx->batch_caps[0] ? ctx->batch_caps[0]
                                                                 : kBatchCapRows);
        double used = 0;
        const int64_t t_admit = now_ns();
        while (!S.waiting.empty() && (int32_t)qs.size() < S.max_batch) {
          gsm_ctx::Server::Req &r = S.waiting.front();
          if (!qs.empty() && used + r.est_rows > budget) break;
          used += r.est_rows;
          r.t_admit = t_admit;
          qs.push_back(r.q);
          lists.push_back(r.mode == GSM_MODE_ENUMERATE ? 1 : 0);
          L.tickets.push_back(r.ticket);
          S.inflight.emplace(r.ticket, r);
          S.waiting.pop_front();
        }
      }
      gsm_status st = guarded(ctx, [&] {
        const int32_t kmax = lane_prepare(ctx, L, qs.data(), (int32_t)qs.size(), lists.data());
        if (L.m > 0) {
          bool tuned;
          auto cfg = batch_config(ctx, L.m, kmax, &tuned);
          lane_issue(ctx, L, kmax, cfg.first, cfg.second);
        } else {
          *L.h_overflow = 0;
          CU(cudaEventRecord(L.ev_done, L.stream));
        }
        ctx->bstats.batches += 1;
      });
      if (st != GSM_OK) {
        std::lock_guard<std::mutex> lk(S.mu);
        for (uint64_t t : L.tickets) {
          auto node = S.inflight.extract(t);
          node.mapped().status = st;
          node.mapped().t_done = now_ns();
          S.finished.insert(std::move(node));
        }
        L.tickets.clear();
        continue;
      }
      L.busy = true;
      progressed = true;
    }
    std::unique_lock<std::mutex> lk(S.mu);
    bool any_busy = false;
    for (auto &lp : S.lanes) any_busy = any_busy || lp->busy;
    if (S.stop && S.waiting.empty() && !any_busy) break;
    if (!progressed) {
      // nothing to do right now: sleep until a submission (or, with work on
      // the device, briefly, then poll the lanes again)
      if (any_busy)
        S.cv.wait_for(lk, std::chrono::microseconds(20));
      else
        S.cv.wait(lk, [&] { return S.stop || !S.waiting.empty(); });
    }
  }
}

}  // namespace

namespace {

void clear_all_graphs(gsm_ctx *ctx) {
  lane_clear_graphs(ctx->lane0);
  if (ctx->server)
    for (auto &lp : ctx->server->lanes) lane_clear_graphs(*lp);
}

}  // namespace

namespace gsm {

int32_t query_k(const gsm_query *q) { return q->k; }

void query_describe(const gsm_query *q, int32_t *labels, uint32_t *adj, int32_t *lo,
                    int32_t *hi) {
  for (int32_t u = 0; u < q->k; ++u) {
    labels[u] = q->labels[u];
    adj[u] = q->adj[u];
    lo[u] = q->lo[u];
    hi[u] = q->hi[u];
  }
}

}  // namespace gsm

// ------------------------------------------------------------------ C ABI

extern "C" {

void gsm_default_options(gsm_options *opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
}

const char *gsm_status_string(gsm_status s) {
  switch (s) {
    case GSM_OK: return "GSM_OK";
    case GSM_PENDING: return "GSM_PENDING";
    case GSM_ERR_INVALID_ARG: return "GSM_ERR_INVALID_ARG";
    case GSM_ERR_INVALID_GRAPH: return "GSM_ERR_INVALID_GRAPH";
    case GSM_ERR_INVALID_QUERY: return "GSM_ERR_INVALID_QUERY";
    case GSM_ERR_NO_GRAPH: return "GSM_ERR_NO_GRAPH";
    case GSM_ERR_OOM: return "GSM_ERR_OOM";
    case GSM_ERR_BUDGET: return "GSM_ERR_BUDGET";
    case GSM_ERR_OVERFLOW: return "GSM_ERR_OVERFLOW";
    case GSM_ERR_TRUNCATED: return "GSM_ERR_TRUNCATED";
    case GSM_ERR_TIMEOUT: return "GSM_ERR_TIMEOUT";
    case GSM_ERR_CUDA: return "GSM_ERR_CUDA";
    case GSM_ERR_TOO_LARGE: return "GSM_ERR_TOO_LARGE";
    case GSM_ERR_INTERNAL: return "GSM_ERR_INTERNAL";
    default: return "GSM_ERR_UNKNOWN";
  }
}

gsm_status gsm_create(gsm_ctx **out, int32_t device, const gsm_options *opt) {
  if (!out) return GSM_ERR_INVALID_ARG;
  *out = nullptr;
  if (opt && opt->block_size != 0 &&
      (opt->block_size < 128 || opt->block_size > 1024 || opt->block_size % 32))
    return GSM_ERR_INVALID_ARG;
  if (opt && (opt->chunk_rows < 0 || opt->filter_rounds < 0 || opt->filter_rounds > 64 ||
              opt->copy_slots < 0 || opt->copy_slots > 64 || opt->lookback_spin_limit < 0 ||
              opt->lookahead < 0 || opt->lookahead > 2 || opt->host_workers < 0 ||
              opt->host_workers > 16))
    return GSM_ERR_INVALID_ARG;
  gsm_ctx *ctx = new gsm_ctx();
  if (opt) ctx->opt = *opt;
  ctx->device = device;
  for (int i = 0; i < K_NUM; ++i) ctx->kstats[i].name = kKernelNames[i];
  gsm_status st = guarded(ctx, [&] {
    CU(cudaSetDevice(device));
    if (ctx->opt.stream) {
      ctx->stream = (cudaStream_t)ctx->opt.stream;
    } else {
      CU(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
      ctx->own_stream = true;
    }
    size_t free_b = 0, total_b = 0;
    CU(cudaMemGetInfo(&free_b, &total_b));
    ctx->budget = ctx->opt.mem_budget_bytes ? ctx->opt.mem_budget_bytes : free_b / 10 * 9;
    ctx->scratch_limit = ctx->budget / 4;
    ctx->stack_limit = ctx->budget - ctx->scratch_limit;
    CU(cudaHostAlloc(&ctx->h_stage, 4096 + 64, cudaHostAllocMapped));
    CU(cudaHostGetDevicePointer(&ctx->d_stage, ctx->h_stage, 0));
    ctx->h_flags = (uint32_t *)((char *)ctx->h_stage + 4096);
    ctx->d_flags = (uint32_t *)((char *)ctx->d_stage + 4096);
    std::memset(ctx->h_flags, 0, 64);
    CU(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
    ctx->d_small = (unsigned long long *)dev_alloc(ctx, 256);
  });
  if (st != GSM_OK) {
    gsm_destroy(ctx);
    return st;
  }
  *out = ctx;
  return GSM_OK;
}

void gsm_destroy(gsm_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->server) gsm_server_stop(ctx);
  for (gsm_ctx *w : ctx->workers) gsm_destroy(w);
  ctx->workers.clear();
  try {
    lane_release(ctx, ctx->lane0);
    free_graph(ctx);
    for (auto &b : ctx->blocks) dev_free(ctx, b.ptr, b.cap);
    dev_free(ctx, ctx->scratch, ctx->scratch_cap);
    dev_free(ctx, ctx->bitmaps, ctx->bitmaps_cap);
    dev_free(ctx, ctx->bitmaps2, ctx->bitmaps2_cap);
    dev_free(ctx, ctx->mfilter, ctx->mfilter_cap);
    dev_free(ctx, ctx->acc[0], ctx->acc_cap[0]);
    dev_free(ctx, ctx->acc[1], ctx->acc_cap[1]);
    dev_free(ctx, ctx->sort_tmp, ctx->sort_tmp_cap);
    dev_free(ctx, ctx->sort_keys, ctx->sort_keys_cap);
    dev_free(ctx, ctx->d_prefix, ctx->d_prefix_cap);
    for (auto &p : ctx->parked) {
      dev_free(ctx, p.acc[0], p.acc_cap[0]);
      dev_free(ctx, p.acc[1], p.acc_cap[1]);
      dev_free(ctx, p.sort_keys, p.sort_keys_cap);
    }
    dev_free(ctx, ctx->d_small, 256);
  } catch (...) {
  }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  for (auto &p : ctx->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  if (ctx->rows_ready) cudaEventDestroy(ctx->rows_ready);
  if (ctx->active_copied) cudaEventDestroy(ctx->active_copied);
  for (auto &p : ctx->parked)
    if (p.copied) cudaEventDestroy(p.copied);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char *gsm_last_error(const gsm_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

gsm_status gsm_load_graph(gsm_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col, const int32_t *labels, int32_t flags) {
  if (!ctx) return GSM_ERR_INVALID_ARG;
  if (n < 0 || nnz < 0 || !row_ptr || (nnz > 0 && !col) ||
      (flags & ~(GSM_DEVICE_PTRS | GSM_VALIDATE))) {
    set_err(ctx, "invalid graph arguments");
    return GSM_ERR_INVALID_ARG;
  }
  if (n >= 0x7fffffff || nnz >= (int64_t(1) << 31)) {
    set_err(ctx, "graph too large for int32 CSR (n=%d nnz=%lld)", n, (long long)nnz);
    return GSM_ERR_TOO_LARGE;
  }
  return guarded(ctx, [&] {
    CU(cudaSetDevice(ctx->device));
    CU(cudaStreamSynchronize(ctx->stream));
    free_graph(ctx);
    const bool dev = flags & GSM_DEVICE_PTRS;
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    std::vector<int32_t> h_rp(n + 1), h_lab(n);
    if (dev) {
      CU(cudaMemcpy(h_rp.data(), row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost));
      if (labels)
        CU(cudaMemcpy(h_lab.data(), labels, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(h_rp.data(), row_ptr, sizeof(int32_t) * (n + 1));
      if (labels && n) std::memcpy(h_lab.data(), labels, sizeof(int32_t) * n);
    }
    ctx->n = n;
    ctx->nnz = nnz;
    ctx->d_rp = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * (n + 1));
    ctx->d_col = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * std::max<int64_t>(nnz, 1));
    ctx->d_lab = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * std::max<int32_t>(n, 1));
    CU(cudaMemcpyAsync(ctx->d_rp, h_rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice,
                       ctx->stream));
    if (nnz)
      CU(cudaMemcpyAsync(ctx->d_col, col, sizeof(int32_t) * nnz, kind, ctx->stream));
    // dense label ids: index into the sorted distinct label values (a table
    // over the value range when it is small, else a sort)
    std::vector<int32_t> vals, dense(n);
    {
      int64_t lo = 0, hi = -1;
      if (n) {
        const auto mm = std::minmax_element(h_lab.begin(), h_lab.end());
        lo = *mm.first;
        hi = *mm.second;
      }
      if (n && hi - lo < 4 * (int64_t)n + 4096) {
        std::vector<int32_t> id((size_t)(hi - lo + 1), -1);
        for (int32_t v = 0; v < n; ++v) id[(size_t)(h_lab[v] - lo)] = 0;
        for (size_t x = 0; x < id.size(); ++x)
          if (id[x] == 0) {
            id[x] = (int32_t)vals.size();
            vals.push_back((int32_t)(lo + (int64_t)x));
          }
        for (int32_t v = 0; v < n; ++v) dense[v] = id[(size_t)(h_lab[v] - lo)];
      } else {
        vals = h_lab;
        std::sort(vals.begin(), vals.end());
        vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
        for (int32_t v = 0; v < n; ++v)
          dense[v] = (int32_t)(std::lower_bound(vals.begin(), vals.end(), h_lab[v]) - vals.begin());
      }
      if (vals.empty()) vals.push_back(0);
    }
    ctx->label_values = vals;
    if (n)
      CU(cudaMemcpyAsync(ctx->d_lab, dense.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                         ctx->stream));
    int32_t md = 0;
    bool rp_ok = h_rp[0] == 0 && (int64_t)h_rp[n] == nnz;
    for (int32_t v = 0; v < n; ++v) {
      const int32_t dv = h_rp[v + 1] - h_rp[v];
      if (dv < 0) rp_ok = false;
      md = std::max(md, dv);
    }
    ctx->max_deg = md;
    // degrees of every label in ascending order: a counting sort by degree,
    // then a stable split by label
    ctx->deg_by_label.assign(vals.size(), {});
    if (n && rp_ok) {
      std::vector<int32_t> start((size_t)md + 2, 0), by_deg(n);
      for (int32_t v = 0; v < n; ++v) start[(size_t)(h_rp[v + 1] - h_rp[v]) + 1]++;
      for (size_t d = 1; d < start.size(); ++d) start[d] += start[d - 1];
      for (int32_t v = 0; v < n; ++v) by_deg[start[(size_t)(h_rp[v + 1] - h_rp[v])]++] = v;
      std::vector<int32_t> per_label(vals.size(), 0);
      for (int32_t v = 0; v < n; ++v) per_label[dense[v]]++;
      for (size_t l = 0; l < vals.size(); ++l) ctx->deg_by_label[l].reserve(per_label[l]);
      for (int32_t v : by_deg) ctx->deg_by_label[dense[v]].push_back(h_rp[v + 1] - h_rp[v]);
    }
    CU(cudaStreamSynchronize(ctx->stream));
    if (flags & GSM_VALIDATE) {
      if (!rp_ok) {
        free_graph(ctx);
        FAIL(GSM_ERR_INVALID_GRAPH, "row_ptr is not a valid CSR offset array");
      }
      GraphDev g{n, nnz, ctx->d_rp, ctx->d_col, ctx->d_lab, nullptr, nullptr, 1};
      g.dbg = ctx->d_flags ? ctx->d_flags + 1 : nullptr;
      int32_t *err = (int32_t *)(ctx->d_small + kMaxK + 1);
      CU(cudaMemsetAsync(err, 0, sizeof(int32_t), ctx->stream));
      launch_validate(g, err, ctx->stream);
      launch_validate_rows(g, err, ctx->stream);
      CU(cudaGetLastError());
      int32_t h_err = 0;
      fetch(ctx, err, sizeof(int32_t));
      std::memcpy(&h_err, ctx->h_stage, sizeof(int32_t));
      if (h_err) {
        free_graph(ctx);
        FAIL(GSM_ERR_INVALID_GRAPH,
             "invalid data graph (%s%s%s)", (h_err & 1) ? "unsorted/duplicate/self-loop/range " : "",
             (h_err & 2) ? "asymmetric " : "", (h_err & 4) ? "row_ptr" : "");
      }
    } else if (!rp_ok) {
      free_graph(ctx);
      FAIL(GSM_ERR_INVALID_GRAPH, "row_ptr is not a valid CSR offset array");
    }
    // label-segmented copy of the rows (ordered by (neighbour label, id))
    ctx->d_lcol = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * std::max<int64_t>(nnz, 1));
    ctx->d_llab = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * std::max<int64_t>(nnz, 1));
    if (nnz > 0) {
      if (ctx->label_values.size() <= 1) {
        CU(cudaMemcpyAsync(ctx->d_lcol, ctx->d_col, sizeof(int32_t) * nnz,
                           cudaMemcpyDeviceToDevice, ctx->stream));
        CU(cudaMemsetAsync(ctx->d_llab, 0, sizeof(int32_t) * nnz, ctx->stream));
      } else {
        const int32_t bits = label_segment_bits(n, (int32_t)ctx->label_values.size());
        const int32_t nw = packed_words(3, bits);
        Carve cv;
        const size_t o_cols = cv.add<int32_t>(3 * nnz), o_rows = cv.add<int32_t>(3 * nnz),
                     o_keys = cv.add<uint64_t>(2 * nnz * nw),
                     o_s = cv.add<char>((int64_t)sort_scratch_bytes(nnz, 3, bits, 2));
        char *tmpbuf = (char *)dev_alloc(ctx, cv.off);
        GraphDev g = graph_dev(ctx);
        launch_label_segments(g, (int32_t)ctx->label_values.size(), (int32_t *)(tmpbuf + o_cols),
                              (uint64_t *)(tmpbuf + o_keys), (int32_t *)(tmpbuf + o_rows),
                              tmpbuf + o_s, ctx->d_flags, ctx->d_lcol, ctx->d_llab, ctx->stream);
        CU(cudaGetLastError());
        CU(cudaStreamSynchronize(ctx->stream));
        dev_free(ctx, tmpbuf, cv.off);
        check_sort_flag(ctx);
      }
      CU(cudaStreamSynchronize(ctx->stream));
    }
    build_hubs(ctx, h_rp);
    // neighbour label counts for the filter (labelled graphs with few labels)
    const int32_t L = (int32_t)ctx->label_values.size();
    if (L > 1 && L <= kNlcMaxLabels && (size_t)n * L <= (size_t(1) << 30)) {
      ctx->nlc_stride = L;
      ctx->d_nlc = (uint8_t *)dev_alloc(ctx, std::max<size_t>((size_t)n * L, 1));
      launch_label_counts(graph_dev(ctx), ctx->d_nlc, L, ctx->stream);
      CU(cudaGetLastError());
      CU(cudaStreamSynchronize(ctx->stream));
    }
    ctx->has_graph = true;
  });
}

gsm_status gsm_query_create(gsm_ctx *ctx, int32_t k, int32_t m, const int32_t *edges,
                            const int32_t *labels, gsm_query **out) {
  if (!out) return GSM_ERR_INVALID_ARG;
  *out = nullptr;
  uint32_t adj[kMaxK];
  gsm_status st = validate_query_edges(k, m, edges, adj);
  if (st != GSM_OK) {
    if (ctx) set_err(ctx, "invalid query graph");
    return st;
  }
  gsm_query *q = new gsm_query();
  q->k = k;
  q->m = m;
  q->edges.assign(edges, edges + 2 * m);
  for (int32_t u = 0; u < k; ++u) {
    q->labels[u] = labels ? labels[u] : 0;
    q->adj[u] = adj[u];
    q->lo[u] = 0;
    q->hi[u] = 0x7fffffff;
  }
  *out = q;
  return GSM_OK;
}

void gsm_query_destroy(gsm_query *q) { delete q; }

gsm_status gsm_query_restrict(gsm_query *q, int32_t u, int32_t lo, int32_t hi) {
  if (!q || u < 0 || u >= q->k || lo < 0 || hi < lo) return GSM_ERR_INVALID_ARG;
  q->lo[u] = lo;
  q->hi[u] = hi;
  return GSM_OK;
}

gsm_status gsm_count(gsm_ctx *ctx, const gsm_query *q, uint64_t *count) {
  if (!ctx || !q || !count) return GSM_ERR_INVALID_ARG;
  bool trunc = false;
  gsm_status st = guarded(ctx, [&] {
    CU(cudaSetDevice(ctx->device));
    run_query(ctx, q, false, nullptr, 0, 0, count, &trunc);
    resolve_timings(ctx);
    ctx->run.peak_bytes = ctx->peak_bytes;
  });
  return st;
}

namespace {
// The candidate filter of every query of a gsm_enumerate_many call in one
// launch (no refinement rounds), with one read-back of all candidate-set
// sizes; pre[j].bitmaps stays null for a query with a label absent from G.
void prefilter_many(gsm_ctx *ctx, int32_t nq, const gsm_query *const *queries,
                    std::vector<Prefiltered> &pre, std::vector<uint64_t> &sizes) {
  const Range range("gsm filter (all queries)");
  const int32_t nw = (ctx->n + 31) / 32;
  std::vector<FilterDesc> fds;
  std::vector<int32_t> sel;
  std::vector<size_t> bm_off;
  size_t bm_words = 0;
  for (int32_t j = 0; j < nq; ++j) {
    int32_t dense[kMaxK];
    if (!dense_labels(ctx, queries[j], dense)) continue;
    FilterDesc fd;
    fill_filter(ctx, queries[j], dense, fd);
    fds.push_back(fd);
    sel.push_back(j);
    bm_off.push_back(bm_words);
    bm_words += (size_t)queries[j]->k * nw;
  }
  pre.assign(nq, Prefiltered{nullptr, nullptr});
  sizes.assign((size_t)nq * kMaxK, 0);
  const int32_t m = (int32_t)sel.size();
  if (m == 0) return;
  Carve cv;
  const size_t o_fd = cv.add<FilterDesc>(m), o_ptr = cv.add<uint32_t *>(m),
               o_sz = cv.add<unsigned long long>((int64_t)m * kMaxK),
               o_bm = cv.add<uint32_t>((int64_t)bm_words);
  ensure_buf(ctx, &ctx->mfilter, &ctx->mfilter_cap, cv.off, false, 0);
  char *base = (char *)ctx->mfilter;
  uint32_t *bm = (uint32_t *)(base + o_bm);
  std::vector<uint32_t *> ptrs(m);
  for (int32_t t = 0; t < m; ++t) ptrs[t] = bm + bm_off[t];
  CU(cudaMemcpyAsync(base + o_fd, fds.data(), sizeof(FilterDesc) * m, cudaMemcpyHostToDevice,
                     ctx->stream));
  CU(cudaMemcpyAsync(base + o_ptr, ptrs.data(), sizeof(uint32_t *) * m, cudaMemcpyHostToDevice,
                     ctx->stream));
  unsigned long long *d_sizes = (unsigned long long *)(base + o_sz);
  GraphDev g = graph_dev(ctx);
  timed(ctx, K_FILTER, 12.0 * ctx->n * m + 4.0 * (double)bm_words, (uint64_t)ctx->n * m, 1, [&] {
    launch_filter_many(g, (const FilterDesc *)(base + o_fd), (uint32_t *const *)(base + o_ptr),
                       d_sizes, m, nw, ctx->stream);
  });
  std::vector<uint64_t> h((size_t)m * kMaxK);
  CU(cudaMemcpyAsync(h.data(), d_sizes, sizeof(uint64_t) * h.size(), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  for (int32_t t = 0; t < m; ++t) {
    const int32_t j = sel[t];
    std::memcpy(&sizes[(size_t)j * kMaxK], &h[(size_t)t * kMaxK], sizeof(uint64_t) * kMaxK);
    pre[j] = Prefiltered{ptrs[t], &sizes[(size_t)j * kMaxK]};
  }
}
}  // namespace

namespace {
// Parks the active result buffers and takes the oldest parked slot (creating
// slots until there are `slots` of them); what the compute stream does next
// waits until that slot's last copy out has finished.
void next_result_slot(gsm_ctx *ctx, int32_t slots) {
  gsm_ctx::ResultSlot cur;
  for (int j = 0; j < 2; ++j) {
    cur.acc[j] = ctx->acc[j];
    cur.acc_cap[j] = ctx->acc_cap[j];
  }
  cur.sort_keys = ctx->sort_keys;
  cur.sort_keys_cap = ctx->sort_keys_cap;
  cur.copied = ctx->active_copied;
  cur.pending = ctx->active_pending;
  ctx->parked.push_back(cur);
  while ((int32_t)ctx->parked.size() < slots) ctx->parked.emplace_front();
  gsm_ctx::ResultSlot nxt = ctx->parked.front();
  ctx->parked.pop_front();
  for (int j = 0; j < 2; ++j) {
    ctx->acc[j] = nxt.acc[j];
    ctx->acc_cap[j] = nxt.acc_cap[j];
  }
  ctx->sort_keys = nxt.sort_keys;
  ctx->sort_keys_cap = nxt.sort_keys_cap;
  ctx->active_copied = nxt.copied;
  ctx->active_pending = nxt.pending;
  if (!ctx->active_copied)
    CU(cudaEventCreateWithFlags(&ctx->active_copied, cudaEventDisableTiming));
  if (ctx->active_pending) {
    CU(cudaStreamWaitEvent(ctx->stream, ctx->active_copied, 0));
    ctx->active_pending = false;
  }
}
}  // namespace

namespace {

// Points a worker at the parent's current graph (every call: the parent may
// have loaded another graph since).
void share_graph(const gsm_ctx *ctx, gsm_ctx *w) {
  w->n = ctx->n;
  w->nnz = ctx->nnz;
  w->max_deg = ctx->max_deg;
  w->d_rp = ctx->d_rp;
  w->d_col = ctx->d_col;
  w->d_lab = ctx->d_lab;
  w->d_lcol = ctx->d_lcol;
  w->d_llab = ctx->d_llab;
  w->d_hub = ctx->d_hub;
  w->d_hub_bits = ctx->d_hub_bits;
  w->d_hub_seg = ctx->d_hub_seg;
  w->d_nlc = ctx->d_nlc;
  w->nlc_stride = ctx->nlc_stride;
  w->hub_count = ctx->hub_count;
  w->label_values = ctx->label_values;
  w->has_graph = ctx->has_graph;
  w->borrowed_graph = true;
}

// A worker context of gsm_enumerate_many: its own stream, workspace, result
// slots and small-read buffer, and a share of the parent's memory budget; it
// lists on the parent's resident graph (borrowed, never freed by the worker)
// and lives as long as the parent.
gsm_ctx *make_worker(gsm_ctx *ctx, int32_t nworkers) {
  gsm_options o = ctx->opt;
  o.stream = nullptr;
  o.mem_budget_bytes = std::max<size_t>(ctx->budget / (size_t)nworkers, size_t(1) << 20);
  gsm_ctx *w = nullptr;
  const gsm_status st = gsm_create(&w, ctx->device, &o);
  if (st != GSM_OK) FAIL(st, "creating a listing worker failed");
  return w;
}

// The listing loop of gsm_enumerate_many on one context: takes query indices
// from `next` until none is left (or another worker failed), lists each into
// its output through the context's result slots and copy stream.
struct ManyState {
  int32_t nq;
  const gsm_query *const *queries;
  int32_t *const *outs;
  const uint64_t *cap_rows;
  uint64_t *counts;
  int32_t flags;
  const std::vector<Prefiltered> *pre = nullptr;
  int32_t nworkers = 1;
  std::atomic<int32_t> next{0};
  std::atomic<int32_t> failed{0};
  std::atomic<int32_t> first_trunc{INT32_MAX};
};

void list_many(gsm_ctx *ctx, ManyState &M, uint64_t *launches, uint64_t *peak, bool *had_last,
               gsm_run_stats *last_run) {
  gsm_ctx *c = ctx;
  if (!c->copy_stream) {
    CU(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&c->rows_ready, cudaEventDisableTiming));
  }
  const int32_t slots = c->opt.copy_slots > 0 ? c->opt.copy_slots : (M.nworkers > 1 ? 2 : 8);
  for (;;) {
    if (M.failed.load()) break;
    const int32_t j = M.next.fetch_add(1);
    if (j >= M.nq) break;
    next_result_slot(c, slots);
    bool trunc = false;
    const Prefiltered *p = (M.pre && (*M.pre)[j].bitmaps) ? &(*M.pre)[j] : nullptr;
    run_query(c, M.queries[j], true, M.outs[j], M.cap_rows[j], M.flags, &M.counts[j], &trunc,
              nullptr, true, p);
    *launches += c->run.kernel_launches;
    *peak = std::max<uint64_t>(*peak, c->peak_bytes);
    if (trunc) {
      int32_t cur = M.first_trunc.load();
      while (j < cur && !M.first_trunc.compare_exchange_weak(cur, j)) {
      }
    }
    if (j == M.nq - 1) {
      *had_last = true;
      *last_run = c->run;
    }
  }
  CU(cudaStreamSynchronize(c->copy_stream));
  CU(cudaStreamSynchronize(c->stream));
  resolve_timings(c);
  check_sort_flag(c);
}

}  // namespace

gsm_status gsm_enumerate_many(gsm_ctx *ctx, int32_t nq, const gsm_query *const *queries,
                              int32_t *const *outs, const uint64_t *cap_rows, uint64_t *counts,
                              int32_t flags) {
  if (!ctx || nq < 0 || (flags & ~GSM_OUT_DEVICE)) return GSM_ERR_INVALID_ARG;
  if (nq > 0 && (!queries || !outs || !cap_rows || !counts)) return GSM_ERR_INVALID_ARG;
  for (int32_t j = 0; j < nq; ++j)
    if (!queries[j] || (cap_rows[j] > 0 && !outs[j])) return GSM_ERR_INVALID_ARG;
  ManyState M;
  M.nq = nq;
  M.queries = queries;
  M.outs = outs;
  M.cap_rows = cap_rows;
  M.counts = counts;
  M.flags = flags;
  const int32_t nworkers =
      std::min<int32_t>(ctx->opt.host_workers > 0 ? ctx->opt.host_workers : 6, std::max(nq, 1));
  M.nworkers = nworkers;
  gsm_status st = guarded(ctx, [&] {
    CU(cudaSetDevice(ctx->device));
    if (!ctx->has_graph) FAIL(GSM_ERR_NO_GRAPH, "no data graph loaded");
    uint64_t launches = 0, peak = 0;
    // without refinement rounds the filter of every query runs as one launch
    std::vector<Prefiltered> pre;
    std::vector<uint64_t> pre_sizes;
    if (ctx->opt.filter_rounds == 0 && nq > 1) {
      prefilter_many(ctx, nq, queries, pre, pre_sizes);
      M.pre = &pre;
      launches += 1;
    }
    gsm_run_stats last{};
    if (nworkers <= 1) {
      bool had_last = false;
      list_many(ctx, M, &launches, &peak, &had_last, &last);
    } else {
      // several host threads, each on a worker context of its own, so one
      // query's kernels fill another's waits on the host
      while ((int32_t)ctx->workers.size() < nworkers)
        ctx->workers.push_back(make_worker(ctx, nworkers));
      for (int32_t w = 0; w < nworkers; ++w) share_graph(ctx, ctx->workers[w]);
      std::vector<gsm_status> wst(nworkers, GSM_OK);
      std::vector<uint64_t> wl(nworkers, 0), wp(nworkers, 0);
      std::vector<char> wlast(nworkers, 0);
      std::vector<gsm_run_stats> wrun(nworkers);
      std::vector<std::thread> th;
      for (int32_t w = 0; w < nworkers; ++w)
        th.emplace_back([&, w] {
          gsm_ctx *c = ctx->workers[w];
          wst[w] = guarded(c, [&] {
            CU(cudaSetDevice(c->device));
            bool had = false;
            list_many(c, M, &wl[w], &wp[w], &had, &wrun[w]);
            wlast[w] = had ? 1 : 0;
          });
          if (wst[w] != GSM_OK) M.failed.store(1);
        });
      for (auto &t : th) t.join();
      for (int32_t w = 0; w < nworkers; ++w) {
        gsm_ctx *c = ctx->workers[w];
        if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
        c->active_pending = false;
        for (auto &p : c->parked) p.pending = false;
      }
      for (int32_t w = 0; w < nworkers; ++w)
        if (wst[w] != GSM_OK) {
          ctx->err = ctx->workers[w]->err;
          throw Fail{wst[w]};
        }
      for (int32_t w = 0; w < nworkers; ++w) {
        gsm_ctx *c = ctx->workers[w];
        launches += wl[w];
        peak = std::max(peak, wp[w]);
        for (int k = 0; k < K_NUM; ++k) {  // per-kernel figures of the whole call
          ctx->kstats[k].launches += c->kstats[k].launches;
          ctx->kstats[k].total_ms += c->kstats[k].total_ms;
          ctx->kstats[k].algo_bytes += c->kstats[k].algo_bytes;
          ctx->kstats[k].items += c->kstats[k].items;
          ctx->kstats[k].probe_bytes += c->kstats[k].probe_bytes;
          const char *nm = c->kstats[k].name;
          c->kstats[k] = KStat();
          c->kstats[k].name = nm;
        }
        if (wlast[w]) {
          last = wrun[w];
          ctx->last_rows = c->last_rows;  // the rows of the call's last query
          ctx->last_count = c->last_count;
          ctx->last_k = c->last_k;
        }
      }
    }
    resolve_timings(ctx);
    if (nworkers > 1) ctx->run = last;
    ctx->run.kernel_launches = launches;
    ctx->run.peak_bytes = peak;
  });
  // no copy into the caller's buffers outlives the call, whatever happened
  if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
  ctx->active_pending = false;
  for (auto &p : ctx->parked) p.pending = false;
  const int32_t first_trunc = M.first_trunc.load();
  if (st == GSM_OK && first_trunc < nq) {
    set_err(ctx, "query %d: %llu embeddings, capacity %llu rows", first_trunc,
            (unsigned long long)counts[first_trunc], (unsigned long long)cap_rows[first_trunc]);
    return GSM_ERR_TRUNCATED;
  }
  return st;
}

gsm_status gsm_enumerate(gsm_ctx *ctx, const gsm_query *q, int32_t *out, uint64_t cap_rows,
                         uint64_t *count, int32_t flags) {
  if (!ctx || !q || !count || (cap_rows > 0 && !out) || (flags & ~GSM_OUT_DEVICE))
    return GSM_ERR_INVALID_ARG;
  bool trunc = false;
  gsm_status st = guarded(ctx, [&] {
    CU(cudaSetDevice(ctx->device));
    run_query(ctx, q, true, out, cap_rows, flags, count, &trunc);
    resolve_timings(ctx);
    ctx->run.peak_bytes = ctx->peak_bytes;
  });
  if (st == GSM_OK && trunc) {
    set_err(ctx, "%llu embeddings, capacity %llu rows", (unsigned long long)*count,
            (unsigned long long)cap_rows);
    return GSM_ERR_TRUNCATED;
  }
  return st;
}

gsm_status gsm_last_rows(gsm_ctx *ctx, int32_t *out, uint64_t first, uint64_t nrows,
                         int32_t flags) {
  if (!ctx || (nrows > 0 && !out) || (flags & ~GSM_OUT_DEVICE)) return GSM_ERR_INVALID_ARG;
  if (first > ctx->last_count || nrows > ctx->last_count - first) {
    set_err(ctx, "rows [%llu, %llu) outside the last result of %llu rows",
            (unsigned long long)first, (unsigned long long)(first + nrows),
            (unsigned long long)ctx->last_count);
    return GSM_ERR_INVALID_ARG;
  }
  if (nrows == 0) return GSM_OK;
  return guarded(ctx, [&] {
    CU(cudaSetDevice(ctx->device));
    CU(cudaMemcpyAsync(out, ctx->last_rows + first * ctx->last_k,
                       (size_t)nrows * ctx->last_k * sizeof(int32_t),
                       (flags & GSM_OUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  });
}

gsm_status gsm_candidates(gsm_ctx *ctx, const gsm_query *q, uint32_t *bitmaps, uint64_t *sizes) {
  if (!ctx || !q) return GSM_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    if (!ctx->has_graph) FAIL(GSM_ERR_NO_GRAPH, "no data graph loaded");
    CU(cudaSetDevice(ctx->device));
    int32_t dense[kMaxK];
    uint64_t sz[kMaxK] = {};
    const size_t nw = (ctx->n + 31) / 32;
    if (!dense_labels(ctx, q, dense)) {
      if (bitmaps) std::memset(bitmaps, 0, sizeof(uint32_t) * nw * q->k);
      if (sizes) std::memset(sizes, 0, sizeof(uint64_t) * q->k);
      return;
    }
    run_filter(ctx, q, dense, sz);
    if (sizes) std::memcpy(sizes, sz, sizeof(uint64_t) * q->k);
    if (bitmaps) {
      CU(cudaMemcpyAsync(bitmaps, ctx->bitmaps, sizeof(uint32_t) * nw * q->k,
                         cudaMemcpyDeviceToHost, ctx->stream));
      CU(cudaStreamSynchronize(ctx->stream));
    }
    resolve_timings(ctx);
  });
}

gsm_status gsm_count_distinct(gsm_ctx *ctx, const gsm_query *q, uint64_t *count,
                              uint64_t *automorphisms) {
  if (!ctx || !q || !count) return GSM_ERR_INVALID_ARG;
  for (int32_t u = 0; u < q->k; ++u)
    if (q->lo[u] != 0 || q->hi[u] != 0x7fffffff) {
      set_err(ctx, "distinct counting needs an unrestricted query");
      return GSM_ERR_INVALID_ARG;
    }
  return guarded(ctx, [&] {
    CU(cudaSetDevice(ctx->device));
    std::vector<std::pair<int32_t, int32_t>> less;
    const uint64_t aut = symmetry_constraints(q->k, q->adj, q->labels, &less);
    bool trunc = false;
    run_query(ctx, q, false, nullptr, 0, 0, count, &trunc, &less);
    if (automorphisms) *automorphisms = aut;
    resolve_timings(ctx);
    ctx->run.peak_bytes = ctx->peak_bytes;
  });
}

gsm_status gsm_run_batch(gsm_ctx *ctx, const gsm_query *const *qs, int32_t nq, uint64_t *counts,
                         gsm_result *results, int32_t flags) {
  if (!ctx || nq < 0 || nq > 65535 || (nq > 0 && (!qs || !counts)) ||
      (flags & ~(GSM_BATCH_AUTOTUNE | GSM_OUT_DEVICE)))
    return GSM_ERR_INVALID_ARG;
  for (int32_t j = 0; j < nq; ++j)
    if (!qs[j]) return GSM_ERR_INVALID_ARG;
  if (ctx->server) {
    set_err(ctx, "the server is running");
    return GSM_ERR_INVALID_ARG;
  }
  return guarded(ctx, [&] {
    CU(cudaSetDevice(ctx->device));
    run_batch(ctx, qs, nq, counts, results, flags);
    resolve_timings(ctx);
  });
}

void gsm_result_free(gsm_ctx *ctx, gsm_result *r) {
  if (!r || !r->rows) return;
  if (r->on_device) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
  }
  try {
    release_rows(ctx, r);
  } catch (...) {
  }
}

gsm_status gsm_batch_configure(gsm_ctx *ctx, uint64_t cap_rows, uint64_t cap_elems,
                               uint64_t cap_items, uint64_t cap_result_elems) {
  if (!ctx || cap_rows >= (uint64_t(1) << 31) || cap_elems >= (uint64_t(1) << 31) ||
      cap_items >= (uint64_t(1) << 30) || cap_result_elems >= (uint64_t(1) << 40))
    return GSM_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    CU(cudaSetDevice(ctx->device));
    CU(cudaStreamSynchronize(ctx->stream));
    if (ctx->server) FAIL(GSM_ERR_INVALID_ARG, "the server is running");
    lane_release(ctx, ctx->lane0);
    ctx->batch_caps[0] = (int64_t)cap_rows;
    ctx->batch_caps[1] = (int64_t)cap_elems;
    ctx->batch_caps[2] = (int64_t)cap_items;
    ctx->batch_caps[3] = (int64_t)cap_result_elems;
  });
}

gsm_status gsm_server_start(gsm_ctx *ctx, int32_t lanes, int32_t max_batch) {
  if (!ctx || lanes < 1 || lanes > 8 || max_batch < 1 || max_batch > 65535 || ctx->server)
    return GSM_ERR_INVALID_ARG;
  if (!ctx->has_graph) return GSM_ERR_NO_GRAPH;
  auto *S = new gsm_ctx::Server();
  S->max_batch = max_batch;
  gsm_status st = guarded(ctx, [&] {
    CU(cudaSetDevice(ctx->device));
    for (int32_t j = 0; j < lanes; ++j) {
      auto L = std::make_unique<Lane>();
      CU(cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking));
      L->own_stream = true;
      S->lanes.push_back(std::move(L));
    }
  });
  if (st != GSM_OK) {
    for (auto &L : S->lanes)
      if (L->stream) cudaStreamDestroy(L->stream);
    delete S;
    return st;
  }
  // Size every lane for the largest batch and capture the graphs of every
  // shape bucket now, so serving neither allocates nor captures.
  st = guarded(ctx, [&] {
    const int32_t n_words = (ctx->n + 31) / 32;
    const int32_t mb_max = bucket_queries(max_batch);
    for (auto &Lp : S->lanes) {
      Lane &L = *Lp;
      lane_workspace(ctx, L, mb_max, (int64_t)mb_max * n_words);
      const size_t bm_bytes = std::min<size_t>((size_t)mb_max * kMaxK * n_words * 4,
                                               size_t(1) << 30);
      ensure_buf(ctx, &L.bitmaps, &L.bitmaps_cap, bm_bytes, false, 0);
      for (int32_t e = 0; e <= 1; ++e) {  // count and enumerate batches
        L.enumerate = e;
        for (int32_t mb = 1; mb <= mb_max; mb <<= 1)
          for (int32_t kb = 1; kb <= kMaxK; ++kb) {
            bool tuned;
            auto cfg = batch_config(ctx, mb, kb, &tuned);
            lane_graph(ctx, L, mb, kb, n_words, cfg.first, cfg.second);
          }
      }
      L.enumerate = 0;
      CU(cudaStreamSynchronize(L.stream));
    }
  });
  if (st != GSM_OK) {
    for (auto &L : S->lanes) {
      try {
        lane_release(ctx, *L);
      } catch (...) {
      }
      if (L->stream) cudaStreamDestroy(L->stream);
    }
    delete S;
    return st;
  }
  ctx->server = S;
  S->th = std::thread(server_loop, ctx);
  return GSM_OK;
}

gsm_status gsm_submit(gsm_ctx *ctx, const gsm_query *q, int32_t mode, uint64_t *ticket) {
  if (!ctx || !q || !ticket || !ctx->server ||
      (mode != GSM_MODE_COUNT && mode != GSM_MODE_ENUMERATE))
    return GSM_ERR_INVALID_ARG;
  gsm_ctx::Server &S = *ctx->server;
  gsm_ctx::Server::Req r;
  r.q = q;
  r.mode = mode;
  r.t_submit = now_ns();
  int32_t dense[kMaxK], order[kMaxK];
  r.est_rows = dense_labels(ctx, q, dense) ? plan_estimated(ctx, q, dense, order) : 0.0;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    r.ticket = S.next_ticket++;
    *ticket = r.ticket;
    S.waiting.push_back(r);
  }
  S.cv.notify_one();
  return GSM_OK;
}

gsm_status gsm_poll(gsm_ctx *ctx, uint64_t ticket, gsm_result *out) {
  if (!ctx || !out || !ctx->server) return GSM_ERR_INVALID_ARG;
  gsm_ctx::Server &S = *ctx->server;
  std::lock_guard<std::mutex> lk(S.mu);
  auto it = S.finished.find(ticket);
  if (it == S.finished.end()) {
    if (S.inflight.count(ticket)) return GSM_PENDING;
    for (const auto &r : S.waiting)
      if (r.ticket == ticket) return GSM_PENDING;
    return GSM_ERR_INVALID_ARG;
  }
  out->count = it->second.count;
  out->status = it->second.status;
  out->t_submit_ns = it->second.t_submit;
  out->t_admit_ns = it->second.t_admit;
  out->t_done_ns = it->second.t_done;
  out->k = it->second.q->k;
  out->on_device = 0;
  out->rows = it->second.rows;  // the caller owns them now
  S.finished.erase(it);
  return GSM_OK;
}

gsm_status gsm_server_stop(gsm_ctx *ctx) {
  if (!ctx || !ctx->server) return GSM_ERR_INVALID_ARG;
  gsm_ctx::Server *S = ctx->server;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->th.joinable()) S->th.join();
  cudaSetDevice(ctx->device);
  for (auto &L : S->lanes) {
    try {
      lane_release(ctx, *L);
    } catch (...) {
    }
    if (L->own_stream && L->stream) cudaStreamDestroy(L->stream);
  }
  for (auto &kv : S->finished) release_host_rows(kv.second.rows);  // never polled
  ctx->server = nullptr;
  delete S;
  return GSM_OK;
}

gsm_status gsm_batch_get_stats(gsm_ctx *ctx, gsm_batch_stats *out) {
  if (!ctx || !out) return GSM_ERR_INVALID_ARG;
  *out = ctx->bstats;
  return GSM_OK;
}

gsm_status gsm_plan_order(int32_t k, int32_t m, const int32_t *edges, const uint64_t *cand_sizes,
                          int32_t *order, int32_t *parent) {
  if (!order || !parent) return GSM_ERR_INVALID_ARG;
  uint32_t adj[kMaxK];
  gsm_status st = validate_query_edges(k, m, edges, adj);
  if (st != GSM_OK) return st;
  plan(k, adj, cand_sizes, order, parent);
  return GSM_OK;
}

gsm_status gsm_query_symmetry(int32_t k, int32_t m, const int32_t *edges, const int32_t *labels,
                              uint64_t *automorphisms, int32_t *pairs, int32_t cap,
                              int32_t *npairs) {
  if (!automorphisms || !npairs || cap < 0 || (cap > 0 && !pairs)) return GSM_ERR_INVALID_ARG;
  uint32_t adj[kMaxK];
  gsm_status st = validate_query_edges(k, m, edges, adj);
  if (st != GSM_OK) return st;
  int32_t lab[kMaxK] = {};
  if (labels)
    for (int32_t u = 0; u < k; ++u) lab[u] = labels[u];
  std::vector<std::pair<int32_t, int32_t>> less;
  *automorphisms = symmetry_constraints(k, adj, lab, &less);
  *npairs = (int32_t)less.size();
  if ((int32_t)less.size() > cap) return GSM_ERR_INVALID_ARG;
  for (size_t t = 0; t < less.size(); ++t) {
    pairs[2 * t] = less[t].first;
    pairs[2 * t + 1] = less[t].second;
  }
  return GSM_OK;
}

gsm_status gsm_kernel_stats(gsm_ctx *ctx, gsm_kernel_stat *out, int32_t max, int32_t *n,
                            int32_t reset) {
  if (!ctx || (max > 0 && !out)) return GSM_ERR_INVALID_ARG;
  for (int32_t i = 0; i < K_NUM && i < max; ++i) {
    std::memset(&out[i], 0, sizeof(out[i]));
    std::snprintf(out[i].name, sizeof(out[i].name), "%s", ctx->kstats[i].name);
    out[i].launches = ctx->kstats[i].launches;
    out[i].total_ms = ctx->kstats[i].total_ms;
    out[i].algo_bytes = ctx->kstats[i].algo_bytes;
    out[i].items = ctx->kstats[i].items;
    out[i].probe_bytes = ctx->kstats[i].probe_bytes;
  }
  if (n) *n = K_NUM;
  if (reset)
    for (int32_t i = 0; i < K_NUM; ++i) {
      const char *nm = ctx->kstats[i].name;
      ctx->kstats[i] = KStat();
      ctx->kstats[i].name = nm;
    }
  return GSM_OK;
}

gsm_status gsm_last_run_stats(gsm_ctx *ctx, gsm_run_stats *out) {
  if (!ctx || !out) return GSM_ERR_INVALID_ARG;
  *out = ctx->run;
  return GSM_OK;
}

}  // extern "C"
