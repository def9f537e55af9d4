/*
 * gsm.h -- C ABI of libgsm, a GB300 (sm_103a) subgraph matcher.
 *
 * Problem (paper Sec. 1 and Sec. 3.2, "Our proposed algorithm: GSM"): given an
 * undirected, vertex-labelled data graph G stored as CSR and a small connected
 * labelled query graph Q, count or list every subgraph isomorphism of Q into G.
 * An embedding is an injective map f : V(Q) -> V(G) with lab(f(u)) = qlab(u)
 * for every query vertex u and {f(u), f(u')} in E(G) for every query edge
 * {u, u'} (non-induced).  Embeddings are ordered maps: automorphic images are
 * distinct results.  A result row is (f(q_0), ..., f(q_{k-1})) in query-vertex
 * id order; rows are returned sorted lexicographically.
 *
 * Method (Sec. 3.2, Algorithm 1): per-query-vertex candidate filtering from
 * label, degree and neighbourhood signatures; a host-side matching order along
 * a query spanning tree; then one breadth-first verification level per query
 * vertex, each checking label, injectivity and every non-tree query edge of a
 * candidate in one step, with compaction of the survivors (Sec. 3.3), and
 * intermediate results held under a fixed device-memory budget.
 *
 * Conventions
 *  - Every call returns a gsm_status: GSM_OK (0), GSM_PENDING (1), or a
 *    negative error.  No C++ exception crosses this boundary.  After an error
 *    gsm_last_error(ctx) describes it.
 *  - A gsm_ctx is used by one host thread at a time.
 *  - Pointers are host pointers unless a flag says they are device pointers
 *    (device pointers must belong to the context's device).
 *  - Sizes are element counts unless named *_bytes.
 */
#ifndef GSM_H_
#define GSM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gsm_status;

#define GSM_OK 0
#define GSM_PENDING 1
#define GSM_ERR_INVALID_ARG (-1)   /* a null pointer, a size out of range, a bad flag */
#define GSM_ERR_INVALID_GRAPH (-2) /* CSR not sorted/symmetric, self-loop, duplicate */
#define GSM_ERR_INVALID_QUERY (-3) /* k outside 1..16, bad edge, duplicate, disconnected */
#define GSM_ERR_NO_GRAPH (-4)      /* matching before gsm_load_graph */
#define GSM_ERR_OOM (-5)           /* the device allocator failed */
#define GSM_ERR_BUDGET (-6)        /* one unit of work does not fit the memory budget */
#define GSM_ERR_OVERFLOW (-7)      /* the count exceeds 2^64 - 1 */
#define GSM_ERR_TRUNCATED (-8)     /* more rows than the caller's capacity */
#define GSM_ERR_TIMEOUT (-9)       /* a bounded device wait gave up */
#define GSM_ERR_CUDA (-10)         /* a CUDA runtime call failed */
#define GSM_ERR_TOO_LARGE (-11)    /* nnz >= 2^31 or n >= 2^31 - 1 */
#define GSM_ERR_INTERNAL (-12)     /* a device bounds check failed (GSM_DEBUG build only) */

typedef struct gsm_ctx gsm_ctx;
typedef struct gsm_query gsm_query;

/* Device memory hooks.  alloc returns a device pointer aligned to 256 bytes
 * (or NULL on failure); free releases it.  `stream` is the context's stream. */
typedef void *(*gsm_alloc_fn)(void *alloc_ctx, size_t bytes, void *stream);
typedef void (*gsm_free_fn)(void *alloc_ctx, void *ptr, size_t bytes, void *stream);

#define GSM_OPT_TIME_KERNELS 1 /* record per-kernel CUDA-event times (gsm_kernel_stats) */
/* Verify and write every level in two passes (count with survivor masks, then
 * write).  Without it a level takes one pass (decoupled look-back over its
 * tiles) whenever its output has room for one row per candidate, and two
 * passes otherwise; results are identical either way. */
#define GSM_OPT_TWO_PASS 2
/* Compressed partial results (the lossless form of Sec. 3.2's hashed partial
 * results): a frontier row of width i is stored as (parent row, new vertex),
 * 8 bytes whatever i, instead of i vertex ids, and decoded through the parent
 * rows of the earlier levels (kept alive by the depth-first chunking).  Less
 * memory and write traffic per level for deep queries, i-1 dependent loads
 * per row read; results are identical.  Levels always take the single pass
 * (rows are split until one row per candidate fits). */
#define GSM_OPT_COMPRESSED_FRONTIERS 4
/* Fault injection for tests of the bounded waits: in every single-pass level
 * of the default frontier layout, the second tile never publishes its
 * survivor count, so the waits of the tiles after it run out
 * (lookback_spin_limit) and the call returns GSM_ERR_TIMEOUT.  Nothing hangs
 * and every row stays inside its buffer; the context stays usable. */
#define GSM_OPT_INJECT_LOOKBACK_STALL 8
/* The same for the final sort of listing calls: in every single-sweep pass
 * of the canonical row sort the second tile never publishes its digit
 * counts; the call returns GSM_ERR_TIMEOUT and the context stays usable. */
#define GSM_OPT_INJECT_SORT_STALL 16
/* Count the algorithmic bytes of the non-tree edge checks of single-pass
 * levels, 4 * ceil(log2 deg) per check made (the binary-search probes of the
 * byte model), into gsm_kernel_stat.probe_bytes (and algo_bytes).  Costs two
 * row-pointer loads per check; results are unchanged. */
#define GSM_OPT_COUNT_PROBES 32
/* The same for the work scan of the advance setup (the pivot choice and the
 * scan of every row's candidate count, one kernel per level): its second
 * tile never publishes its work total, so the waits of the tiles after it
 * run out; the call returns GSM_ERR_TIMEOUT, no offset is used, and the
 * context stays usable.  Only levels of more than 1,024 rows have a second
 * tile. */
#define GSM_OPT_INJECT_SCAN_STALL 64

typedef struct gsm_options {
  /* Cap on device memory for intermediate frontiers and scratch, in bytes.
   * 0 = 90% of the device memory free at gsm_create.  The graph, candidate
   * bitmaps and final result buffers are not counted.  A single-pass level
   * reserves its output for one row per candidate when that fits the cap;
   * otherwise it sizes the output exactly (two passes) or splits its rows. */
  size_t mem_budget_bytes;
  /* cudaStream_t every kernel and copy is issued on; NULL = a stream the
   * library creates and owns. */
  void *stream;
  gsm_alloc_fn alloc; /* NULL = cudaMalloc */
  gsm_free_fn free;   /* NULL = cudaFree */
  void *alloc_ctx;
  int32_t block_size;     /* threads per CTA of the extend kernels; 0 = 256; 128..1024, x32 */
  int64_t chunk_rows;     /* max frontier rows per extend launch; 0 = from the budget */
  /* Candidate-refinement rounds after the first filter pass (Sec. 3.2, 0..64):
   * a round keeps v in C(u) iff, for every label l, v has at least as many
   * neighbours in the union of the candidate sets of u's label-l query
   * neighbours as u has such neighbours.  Results do not depend on it;
   * gsm_candidates returns the refined sets.  The batched form ignores it. */
  int32_t filter_rounds;
  int32_t flags;          /* GSM_OPT_* */
  /* Result staging slots gsm_enumerate_many uses in turn, per worker (0 = 8
   * with one host worker, 2 with several; at most 64): each holds the staging
   * buffers of one query's rows until they are copied out, so up to this
   * many of a worker's queries can be ahead of its copies. */
  int32_t copy_slots;
  /* Bound of every wait of a single-pass level on the counts of earlier
   * tiles (polls of about 32 ns; 0 = 2^20).  A wait that runs out ends the
   * call with GSM_ERR_TIMEOUT; the rows written stay inside the buffers. */
  int32_t lookback_spin_limit;
  /* k-look-ahead of the verification levels (Sec. 3.2, "1- and 2-look-ahead";
   * 0 = off, 1, 2): a candidate w for pi_i is dropped when the query
   * neighbours of pi_i placed later cannot all be mapped to distinct
   * neighbours of w outside the partial embedding (1: by label counts; 2:
   * also by their candidate sets, over the first 64 same-label neighbours).
   * Both tests are necessary conditions, so results do not depend on it; it
   * trades extra work per surviving candidate for smaller frontiers.  The
   * batched form ignores it. */
  int32_t lookahead;
  /* Device memory for adjacency bitmaps of the data graph's hubs (vertices of
   * degree >= 32, highest degree first, ceil(n/32) x 4 bytes each), used to
   * check non-tree edges against a hub with one bit probe instead of a binary
   * search of its row.  0 = 512 MiB; negative = no bitmaps.  Built by
   * gsm_load_graph, outside the memory budget; results do not depend on it. */
  int64_t hub_bitmap_bytes;
  /* Host threads gsm_enumerate_many lists its queries with (0 = 6, at most
   * 16): each thread has a worker context of its own (stream, workspace with
   * an equal share of the memory budget, result slots) on the shared
   * resident graph, so one query's kernels run while another waits for a
   * read-back.  1 = one query after the other on the context itself.  (On
   * the 20-slice R-MAT 16 listing, 1 / 2 / 4 / 6 / 8 workers: 6.70 / 5.93 /
   * 5.47 / 5.39 / 5.42 ms with 2-4 slots.) */
  int32_t host_workers;
} gsm_options;

/* Fills *opt with the defaults described above. */
void gsm_default_options(gsm_options *opt);

/* Creates a context on CUDA device `device`.  opt may be NULL (defaults).
 * Errors: GSM_ERR_INVALID_ARG, GSM_ERR_CUDA. */
gsm_status gsm_create(gsm_ctx **out, int32_t device, const gsm_options *opt);

/* Releases every resource of the context (queries must be destroyed first). */
void gsm_destroy(gsm_ctx *ctx);

/* Message of the last error on this context ("" if none).  Owned by ctx. */
const char *gsm_last_error(const gsm_ctx *ctx);

/* Static name of a status code. */
const char *gsm_status_string(gsm_status s);

#define GSM_DEVICE_PTRS 1 /* row_ptr/col/labels are device pointers */
#define GSM_VALIDATE 2    /* check sortedness, symmetry, self-loops, duplicates */

/* Loads the data graph G (paper Sec. 3.3: CSR, no preprocessing).
 *   n        vertices, 0 <= n < 2^31 - 1
 *   nnz      directed CSR entries (= 2|E|), < 2^31
 *   row_ptr  int32[n+1], row_ptr[0] = 0, row_ptr[n] = nnz, non-decreasing
 *   col      int32[nnz], row v = col[row_ptr[v] .. row_ptr[v+1]), strictly
 *            ascending, no v in its own row, and w in row v <=> v in row w
 *   labels   int32[n] vertex labels (any int32 values), or NULL for all-zero
 * The library copies the arrays (caller may free them on return) and keeps the
 * copy resident; a second call replaces the graph.  row_ptr is always checked
 * (GSM_ERR_INVALID_GRAPH); the rules on col are checked on the device with
 * GSM_VALIDATE and are otherwise the caller's guarantee.  Errors:
 * GSM_ERR_INVALID_ARG, GSM_ERR_TOO_LARGE, GSM_ERR_INVALID_GRAPH, GSM_ERR_OOM,
 * GSM_ERR_CUDA. */
gsm_status gsm_load_graph(gsm_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col, const int32_t *labels, int32_t flags);

/* Creates a query graph Q (host memory only).
 *   k       query vertices, 1..16
 *   m       undirected edges
 *   edges   int32[2m]: edge e joins edges[2e] and edges[2e+1]; no self-loop,
 *           no edge listed twice (in either direction); Q must be connected
 *   labels  int32[k] query labels, or NULL for all-zero labels
 * Errors: GSM_ERR_INVALID_ARG, GSM_ERR_INVALID_QUERY. */
gsm_status gsm_query_create(gsm_ctx *ctx, int32_t k, int32_t m, const int32_t *edges,
                            const int32_t *labels, gsm_query **out);

void gsm_query_destroy(gsm_query *q);

/* Restricts the results of q to embeddings with lo <= f(u) < hi (a root-range
 * slice; with u = 0 the slice is a contiguous block of the sorted result).
 * Calling it again for the same u replaces the range.
 * Errors: GSM_ERR_INVALID_ARG (u out of range, lo > hi, negative bound). */
gsm_status gsm_query_restrict(gsm_query *q, int32_t u, int32_t lo, int32_t hi);

/* Counts the embeddings of q in the loaded graph.
 * Errors: GSM_ERR_NO_GRAPH, GSM_ERR_BUDGET, GSM_ERR_OOM, GSM_ERR_OVERFLOW,
 * GSM_ERR_CUDA. */
gsm_status gsm_count(gsm_ctx *ctx, const gsm_query *q, uint64_t *count);

/* Counts distinct subgraphs: embeddings up to the automorphisms of the
 * labelled query (the paper's own count |M|/|Q| in Algorithm 1, obtained as
 * Sec. 3.1 proposes, by node-ID ordering constraints between equivalent query
 * vertices, so each subgraph is produced once).  *count = gsm_count(q) /
 * |Aut(Q)|; *automorphisms (may be NULL) receives |Aut(Q)|.  The query must
 * not be restricted.  Errors: as gsm_count, plus GSM_ERR_INVALID_ARG. */
gsm_status gsm_count_distinct(gsm_ctx *ctx, const gsm_query *q, uint64_t *count,
                              uint64_t *automorphisms);

#define GSM_OUT_DEVICE 1 /* `out` is a device pointer */

/* Lists the embeddings of q: out is int32[cap_rows * k], row-major, rows in
 * ascending lexicographic order, column j = f(q_j).  *count receives the total
 * number of embeddings.  If it exceeds cap_rows the first cap_rows rows are
 * written and GSM_ERR_TRUNCATED is returned.  out may be NULL iff cap_rows = 0.
 * Final rows are staged in library-owned device buffers outside the budget:
 * count x k x 4 bytes of rows plus, unless the matching order already gives
 * canonical order, two packed sort keys of ceil(k * log2(n) / 64) x 8 bytes
 * per row and about 1.5 bytes per row of histograms.  A single-pass last
 * level reserves room for one row per candidate it checks (at most 4 GiB;
 * beyond that it takes two passes), so the staging can exceed the count.
 * Errors: as gsm_count, plus GSM_ERR_TRUNCATED. */
gsm_status gsm_enumerate(gsm_ctx *ctx, const gsm_query *q, int32_t *out, uint64_t cap_rows,
                         uint64_t *count, int32_t flags);

/* gsm_enumerate for nq queries: queries[j] lists into outs[j] (capacity
 * cap_rows[j] rows), counts[j] receives its total.  Same row layout and order
 * as gsm_enumerate; all outs[] are host pointers, or all device pointers with
 * GSM_OUT_DEVICE.  The paper has no counterpart: it is the serving form of
 * the listing.  The candidate filter of all queries runs as one launch (when
 * filter_rounds is 0), then gsm_options.host_workers host threads take the
 * queries in turn, each on a worker context of its own (stream, workspace,
 * result slots; created on first use, kept with the context, sharing its
 * graph), so one query's kernels overlap another's waits.  Each worker copies
 * a query's rows out on a copy stream while its next queries compute, so the
 * result staging buffers of gsm_enumerate exist once per slot and worker
 * (gsm_options.copy_slots).  The call returns after every copy has finished
 * (also on error); host buffers should be pinned for the copies to overlap.
 * gsm_last_rows then refers to the last query; gsm_last_run_stats counts the
 * kernel launches of the whole call and the peak budgeted bytes over its
 * queries (per worker), and its other fields describe the last query;
 * gsm_kernel_stats adds up every worker's kernels.  Errors: as gsm_enumerate
 * (GSM_ERR_TRUNCATED if any query overflowed its capacity: every count is
 * still set, every output holds its first cap_rows[j] rows); on another error
 * the counts of queries not yet run are unspecified. */
gsm_status gsm_enumerate_many(gsm_ctx *ctx, int32_t nq, const gsm_query *const *queries,
                              int32_t *const *outs, const uint64_t *cap_rows, uint64_t *counts,
                              int32_t flags);

/* Copies rows [first, first + nrows) of the last gsm_enumerate result on this
 * context (kept in library buffers until the next gsm_count / gsm_enumerate /
 * gsm_candidates / gsm_run_batch call) into out (host, or device with
 * GSM_OUT_DEVICE).
 * Errors: GSM_ERR_INVALID_ARG (range outside the last result), GSM_ERR_CUDA. */
gsm_status gsm_last_rows(gsm_ctx *ctx, int32_t *out, uint64_t first, uint64_t nrows,
                         int32_t flags);

/* Candidate sets of the filtering step (paper Sec. 3.2, Algorithm 1
 * Filter_candidate_set): bit v of bitmap u (word v/32, bit v%32) is set iff
 * lab(v) = qlab(u), deg(v) >= deg_Q(u), for every label l the number of
 * neighbours of v with label l is at least the number of query neighbours of u
 * with label l, and v lies in u's restriction range (if any).
 *   bitmaps  host uint32[k * ceil(n/32)] (may be NULL)
 *   sizes    host uint64[k]: |C(u)| (may be NULL) */
gsm_status gsm_candidates(gsm_ctx *ctx, const gsm_query *q, uint32_t *bitmaps, uint64_t *sizes);

/* ---- Batched form: many queries against the resident graph at once ----
 *
 * The paper runs one query at a time; this form runs a whole batch of
 * queries (uneven sizes, 1..16 vertices) as one CUDA graph: a batched
 * candidate filter, then every verification level of every query over one
 * concatenated frontier (Algorithm 1's levels, all queries in lock step),
 * with no host synchronisation until the counts come back.  The matching
 * order of each query uses label/degree histograms of G as its P_f estimate
 * (the VF3 estimate the paper cites in Sec. 3.2) instead of the candidate
 * counts, so the order is known before the filter runs.  Results equal
 * gsm_count's (and gsm_enumerate's rows) for every query.  The batch works in
 * a fixed-capacity workspace (about 1.4 GB, allocated on first use, outside
 * the memory budget: 2^24 frontier rows, 2^27 frontier elements, 2^28
 * candidates per level, and for listing batches a result arena of 2^28 ints);
 * a batch that would exceed it is rerun query by query on the single-query
 * path.
 */
typedef struct gsm_batch_stats {
  int32_t block_size;        /* threads per CTA used by the last batch */
  int32_t grid;              /* persistent CTAs used by the last batch */
  int32_t tuned;             /* 1 if the autotuner chose them */
  int32_t overflowed;        /* 1 if the last batch fell back to gsm_count */
  uint64_t batches;          /* batches run */
  uint64_t graph_launches;   /* CUDA graph launches */
  uint64_t graphs_built;     /* graphs captured and instantiated */
  uint64_t fallbacks;        /* batches rerun on the single-query path */
  uint64_t kernels_per_graph;
  double last_ms;            /* host wall time of the last gsm_run_batch */
} gsm_batch_stats;

#define GSM_BATCH_AUTOTUNE 1 /* time candidate (block size, grid) pairs for new batch shapes */

/* The result of one query of the batched or served form.  In count mode
 * rows is NULL.  In enumerate mode rows holds the count x k result rows
 * (row-major int32, query-id column order, sorted lexicographically, as
 * gsm_enumerate returns them), NULL when count is 0; the buffer belongs to
 * the library until gsm_result_free.  on_device = 1: rows is device memory
 * of the context's device (from the context's allocator), else host memory. */
typedef struct gsm_result {
  uint64_t count;
  gsm_status status;     /* GSM_OK or the error that ended the query */
  int64_t t_submit_ns;   /* served form: steady-clock timestamps (same clock for all) */
  int64_t t_admit_ns;
  int64_t t_done_ns;
  int32_t k;             /* row width (enumerate mode) */
  int32_t on_device;
  int32_t *rows;
} gsm_result;

/* Releases r->rows (through the context's allocator when on_device) and sets
 * it to NULL; ctx is the context that produced the result.  NULL rows are
 * fine. */
void gsm_result_free(gsm_ctx *ctx, gsm_result *r);

/* Runs qs[0..nq) as one batch.  counts[j] receives what gsm_count would
 * return for qs[j].  results = NULL: count only.  Otherwise every query also
 * lists its rows: results[j] receives the count and the sorted rows of qs[j]
 * (host memory, or device memory with GSM_OUT_DEVICE), which the caller
 * releases with gsm_result_free.  Shapes (number of queries, largest query,
 * count or list) seen before reuse their captured graph.  With
 * GSM_BATCH_AUTOTUNE, the first batch of a shape is run once per candidate
 * configuration (every run gives the same results) and the fastest is kept
 * for that shape.  nq <= 65535.
 * Errors: GSM_ERR_INVALID_ARG, GSM_ERR_NO_GRAPH, GSM_ERR_OOM, GSM_ERR_CUDA, and
 * the errors of gsm_count / gsm_enumerate on the fallback path (on an error
 * no rows are left allocated). */
gsm_status gsm_run_batch(gsm_ctx *ctx, const gsm_query *const *qs, int32_t nq, uint64_t *counts,
                         gsm_result *results, int32_t flags);

gsm_status gsm_batch_get_stats(gsm_ctx *ctx, gsm_batch_stats *out);

/* Sets the batch workspace capacities (0 keeps the default): frontier rows
 * (< 2^31), frontier elements (rows x width, < 2^31), candidates per level
 * (< 2^30) and result-arena ints of listing batches (< 2^40).  Frees the
 * current workspace; the next batch allocates the new one.
 * Errors: GSM_ERR_INVALID_ARG. */
gsm_status gsm_batch_configure(gsm_ctx *ctx, uint64_t cap_rows, uint64_t cap_elems,
                               uint64_t cap_items, uint64_t cap_result_elems);

/* ---- Served form: a request loop with continuous batching ----
 *
 * gsm_server_start starts a thread that owns the context until
 * gsm_server_stop: meanwhile only gsm_submit, gsm_poll, gsm_result_free and
 * gsm_server_stop may be called on the context (from any threads).  Submitted
 * queries wait in arrival order; whenever one of `lanes` batch lanes (a stream
 * with its own batch workspace) is free, the waiting queries are admitted
 * into a new batch while the sum of their estimated peak frontier sizes (from
 * label/degree histograms, Sec. 3.2's P_f) stays within half a lane's
 * frontier capacity -- at least one query per batch, at most max_batch.
 * Queries that arrive while batches run are admitted as soon as a lane frees,
 * so their work overlaps the running batches on the device.  A batch that
 * overflows its workspace is rerun query by query.  Every result equals
 * gsm_count's (gsm_enumerate's rows) for that query.
 */

/* lanes 1..8, max_batch 1..65535.  Captures the batch graphs of every shape
 * (count and enumerate mode) before it returns, so serving does not capture.
 * Errors: GSM_ERR_INVALID_ARG (also if a server already runs),
 * GSM_ERR_NO_GRAPH, GSM_ERR_CUDA. */
gsm_status gsm_server_start(gsm_ctx *ctx, int32_t lanes, int32_t max_batch);

#define GSM_MODE_COUNT 0      /* the result carries the count only */
#define GSM_MODE_ENUMERATE 1  /* ... and the sorted rows, in host memory */

/* Queues q in `mode`; *ticket identifies it.  q must stay alive until its
 * result has been polled.  Thread-safe.  Errors: GSM_ERR_INVALID_ARG (no
 * server, bad mode). */
gsm_status gsm_submit(gsm_ctx *ctx, const gsm_query *q, int32_t mode, uint64_t *ticket);

/* GSM_PENDING while the query waits or runs; once done, fills *out, forgets
 * the ticket and returns GSM_OK (out->status holds the query's own status;
 * in enumerate mode out->rows passes to the caller, who releases it with
 * gsm_result_free).  Thread-safe.  Errors: GSM_ERR_INVALID_ARG (unknown
 * ticket, no server). */
gsm_status gsm_poll(gsm_ctx *ctx, uint64_t ticket, gsm_result *out);

/* Finishes every submitted query, stops the thread and frees the lanes
 * (results not yet polled are dropped, their rows released). */
gsm_status gsm_server_stop(gsm_ctx *ctx);

/* Size of the fixed device array behind gsm_candidates_static: bitmap words of
 * one call, k * ceil(n/32) * 4 bytes, must fit in it (e.g. n <= 4,194,304 at
 * k = 16).  A further 256 bytes hold the counters. */
#define GSM_STATIC_SCRATCH_BITMAP_BYTES (8u << 20)

/* gsm_candidates without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory -- a process whose device memory is already claimed by
 * another allocator (a serving process whose caching allocator reserved the
 * free HBM up front, where cudaMalloc would fail or fragment that pool), or
 * code in a latency-critical loop that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree may perform.
 *
 * It computes the same bitmaps and sizes as gsm_candidates, from a graph the
 * caller keeps in device memory, and needs no context:
 *   n, nnz, row_ptr, col, labels   the data graph on the current device, in
 *            the layout of gsm_load_graph (labels required, raw values; the
 *            caller guarantees the CSR rules -- nothing is validated)
 *   q        the query (its restrictions apply)
 *   bitmaps  uint32[k * ceil(n/32)] and sizes uint64[k] (either may be NULL),
 *            host memory, or device memory with flags = GSM_OUT_DEVICE
 *   stream   cudaStream_t to run on (NULL = the legacy default stream); the
 *            call returns after the stream has finished the work
 * Working memory is one fixed file-scope device array
 * (GSM_STATIC_SCRATCH_BITMAP_BYTES + 256 bytes) that every GPU which loads the
 * library holds until the process exits.  The library allocates nothing: no
 * cudaMalloc, no cudaFree, no allocator hook.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents
 * (the counters are cleared at the start of every call), so calls whose work
 * overlaps on the GPU -- from two streams or two host threads -- race and give
 * wrong results.
 * Errors: GSM_ERR_INVALID_ARG, GSM_ERR_TOO_LARGE (k * ceil(n/32) * 4 bytes over
 * the array, or the graph over the int32 CSR limits), GSM_ERR_CUDA. */
gsm_status gsm_candidates_static(int32_t n, int64_t nnz, const int32_t *row_ptr,
                                 const int32_t *col, const int32_t *labels, const gsm_query *q,
                                 uint32_t *bitmaps, uint64_t *sizes, int32_t flags, void *stream);

/* The symmetry breaking behind gsm_count_distinct (host only, no device
 * work): Sec. 3.1's node-ID ordering constraints between equivalent query
 * vertices, built along a stabilizer chain of Aut(Q) (the automorphisms of
 * the query that keep labels and edges).  *automorphisms = |Aut(Q)|;
 * constraint t is f(pairs[2t]) < f(pairs[2t+1]) for an embedding f, and of
 * the |Aut(Q)| embeddings f o sigma (sigma in Aut(Q)) exactly one meets every
 * constraint.  labels may be NULL (all 0).  cap = room in pairs (in pairs of
 * int32); *npairs = the number of constraints (at most k(k-1)/2), also when
 * cap is too small.  Errors: GSM_ERR_INVALID_QUERY, GSM_ERR_INVALID_ARG (null
 * outputs, or cap < *npairs). */
gsm_status gsm_query_symmetry(int32_t k, int32_t m, const int32_t *edges, const int32_t *labels,
                              uint64_t *automorphisms, int32_t *pairs, int32_t cap,
                              int32_t *npairs);

/* The matching order of Sec. 3.2 (host only, no device work): order[i] is the
 * i-th query vertex placed, parent[i] the position (< i) of its spanning-tree
 * parent (-1 for i = 0).  The first vertex minimises the candidate count
 * (ties: larger query degree, then lower id); every later one maximises the
 * number of edges to placed vertices, then minimises the candidate count, then
 * maximises the query degree, then takes the lower id.  The parent is the
 * earliest-placed neighbour.  cand_sizes = uint64[k] (NULL = all equal).
 * Errors: GSM_ERR_INVALID_QUERY. */
gsm_status gsm_plan_order(int32_t k, int32_t m, const int32_t *edges, const uint64_t *cand_sizes,
                          int32_t *order, int32_t *parent);

/* Per-kernel measurements, collected while GSM_OPT_TIME_KERNELS is set. */
typedef struct gsm_kernel_stat {
  char name[32];
  uint64_t launches;
  double total_ms;       /* sum of CUDA-event durations on the context's stream */
  double algo_bytes;     /* algorithmic bytes moved by those launches */
  uint64_t items;        /* work items (candidates checked, rows written, ...) */
  double probe_bytes;    /* part of algo_bytes: the non-tree edge checks' binary-search
                            probes, 4 * ceil(log2 deg) per check made (single-pass levels,
                            with GSM_OPT_COUNT_PROBES) */
} gsm_kernel_stat;

/* Copies up to max entries into out, returns the number of kernels tracked
 * through *n.  reset != 0 clears the counters afterwards. */
gsm_status gsm_kernel_stats(gsm_ctx *ctx, gsm_kernel_stat *out, int32_t max, int32_t *n,
                            int32_t reset);

/* Work counters of the last gsm_count / gsm_enumerate call. */
typedef struct gsm_run_stats {
  int32_t k;
  int32_t order[16];
  uint64_t cand_size[16];    /* |C(u)| per query vertex id */
  uint64_t frontier[16];     /* rows at level i (i = 1..k; [0] unused) */
  uint64_t candidates[16];   /* candidates checked while extending level i -> i+1 */
  uint64_t chunks;           /* extend sub-chunks launched */
  uint64_t peak_bytes;       /* high-water mark of budgeted device memory */
  uint64_t kernel_launches;  /* kernels launched by the call */
} gsm_run_stats;

gsm_status gsm_last_run_stats(gsm_ctx *ctx, gsm_run_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* GSM_H_ */
