// Internal interface between the host driver (api.cu) and the device kernels
// (kernels.cu, sort.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gsm {

constexpr int kMaxK = 16;

// Items (candidate edges) one CTA of the extend kernels covers: blockDim.x
// threads x kItemsPerThread, item j of thread t is tile_base + j*blockDim + t,
// so a warp touches 32 consecutive candidates of (usually) one CSR row.
constexpr int kItemsPerThread = 4;

// Filter description of one query (Sec. 3.2 filtering: label, degree and the
// per-label neighbour counts that refine the paper's neighbourhood encoding).
struct FilterDesc {
  int32_t k;
  int32_t n_words;                 // ceil(n/32): stride between bitmaps
  int32_t qlab[kMaxK];             // dense label id of query vertex u
  int32_t qdeg[kMaxK];             // deg_Q(u)
  int32_t lo[kMaxK], hi[kMaxK];    // restriction of f(u) to [lo, hi)
  int32_t nreq[kMaxK];             // number of (slot, count) requirements of u
  int32_t req_slot[kMaxK][kMaxK];  // label slot of requirement r of u
  int32_t req_cnt[kMaxK][kMaxK];   // neighbours needed with that label
  int32_t nslots;                  // distinct labels used by requirements
  int32_t slot_label[kMaxK];       // dense label id of each slot
};

// One verification level: extends rows of width i (positions 0..i-1 hold the
// images of pi_0..pi_{i-1}) by a vertex for pi_i.
struct LevelDesc {
  int32_t i;                  // input row width
  int32_t nb;                 // mapped query neighbours of pi_i (tree parent + non-tree)
  int32_t bpos[kMaxK];        // their row positions
  int32_t ninj;               // positions that need an explicit injectivity test
  int32_t inj[kMaxK];
  int32_t out_col[kMaxK + 1]; // output column of position j (0..i); identity except last level
  const uint32_t *bitmap;     // C(pi_i)
  int32_t nlt, lt[kMaxK];     // symmetry breaking: the new vertex must be < row[lt[t]]
  int32_t ngt, gt[kMaxK];     //                     and > row[gt[t]]
  int32_t lab;                // dense label of pi_i: only that segment of a row is traversed
  // k-look-ahead (Sec. 3.2; la = 0 off, 1 or 2): the query neighbours of
  // pi_i placed after it, grouped by label.  Group t: label la_lab[t],
  // la_need[t] such neighbours, la_known[t] mapped neighbours of pi_i with
  // that label (adjacent to a candidate by the level's own checks), la_pos[t]
  // = positions of the other placed vertices with that label (bit j), la_uq[t]
  // = the group's query vertices (bit u; their candidate bitmaps are
  // cand + u * n_words).
  int32_t la, nla;
  int32_t la_lab[kMaxK], la_need[kMaxK], la_known[kMaxK];
  uint32_t la_pos[kMaxK], la_uq[kMaxK];
  const uint32_t *cand;
  int32_t n_words;
  // 1 (GSM_OPT_COUNT_PROBES): the single-pass level adds the algorithmic
  // bytes of its non-tree edge checks, 4 * ceil(log2 deg) per check made
  // (the binary-search probes of the byte model), to lookback word tiles + 3
  int32_t count_probes;
};

struct GraphDev {
  int32_t n;
  int64_t nnz;
  const int32_t *rp;
  const int32_t *col;   // rows ascending by id
  const int32_t *lab;   // dense label ids
  const int32_t *lcol;  // the same rows ordered by (label, id): label segments
  const int32_t *llab;  // dense label of lcol[e]
  int32_t num_labels;   // 1: every row is one segment and lcol equals col
  // adjacency bitmaps of the high-degree vertices ("hubs"): hub[v] = index h
  // of v's bitmap or -1, bit w of hub_bits[h * hub_words ..] set iff w is a
  // neighbour of v.  hub = null: no bitmaps, every test searches the row.
  const int32_t *hub;
  const uint32_t *hub_bits;
  int32_t hub_words;
  // label segments of the hubs' rows (null: none): the neighbours of hub h
  // with label l are lcol[hub_seg[h * (num_labels + 1) + l] .. the next entry)
  const int32_t *hub_seg;
  // neighbour label counts (null: none): nlc[v * nlc_stride + l] = the number
  // of neighbours of v with label l, saturated at 255 (a query needs at most
  // 15, so the saturated count decides every requirement exactly)
  const uint8_t *nlc;
  int32_t nlc_stride;
  // GSM_DEBUG builds: the mapped word a failed bounds check writes its site
  // to (null: not reported)
  uint32_t *dbg;
};

// Bounds checks of the GSM_DEBUG build at the hot kernels' indexed accesses:
// GSM_IN_BOUNDS(dbg, cond, site) is true when cond holds; otherwise it
// records `site` in *dbg and is false, and the caller skips the access (no
// trap; the host reports GSM_ERR_INTERNAL).  In other builds it is true and
// costs nothing.
#ifdef GSM_DEBUG
__device__ __forceinline__ bool gsm_in_bounds(uint32_t *dbg, bool ok, uint32_t site) {
  if (!ok && dbg) *(volatile uint32_t *)dbg = site;
  return ok;
}
#define GSM_IN_BOUNDS(dbg, cond, site) gsm_in_bounds((dbg), (cond), (site))
#else
#define GSM_IN_BOUNDS(dbg, cond, site) true
#endif
// check sites
constexpr uint32_t kDbgPivotVertex = 1, kDbgCandidate = 2, kDbgRow = 3, kDbgNeighbour = 4,
                   kDbgOutputRow = 5, kDbgSortPosition = 6;

// ---- launchers (all asynchronous on `s`) ----

// err[0] |= 1 on a malformed row (unsorted/duplicate/self-loop/out of range),
// |= 2 on an asymmetric entry, |= 4 on a bad row_ptr.
void launch_validate(const GraphDev &g, int32_t *err, cudaStream_t s);
// Row checks; only valid to run once launch_validate reported a sane row_ptr.
void launch_validate_rows(const GraphDev &g, int32_t *err, cudaStream_t s);

// Label-segmented rows: out_col/out_lab = every row of g ordered by (label
// of the neighbour, neighbour id).  Uses the packed row sort on the edges as
// 3-column rows (row, label, id); edge_cols and rows_out need 3*nnz int32,
// keys 2 * nnz * packed_words(3, bits) uint64, sort_scratch
// sort_scratch_bytes(nnz, 3, bits, 2) bytes (bits = label_segment_bits);
// err as for launch_sort_rows_packed.  Returns kernels launched.
int launch_label_segments(const GraphDev &g, int32_t num_labels, int32_t *edge_cols,
                          uint64_t *keys, int32_t *rows_out, void *sort_scratch, uint32_t *err,
                          int32_t *out_col, int32_t *out_lab, cudaStream_t s);
int32_t label_segment_bits(int32_t n, int32_t num_labels);

// Adjacency bitmaps of the H hubs (vertex ids hubs[0..H)): bitmap h (words
// bits[h * words ..], zeroed here) gets bit w for every neighbour w.
void launch_hub_bitmaps(const GraphDev &g, const int32_t *hubs, int32_t H, int32_t words,
                        uint32_t *bits, cudaStream_t s);
// seg[h * (g.num_labels + 1) + l] = start of label l's segment in the
// (label, id)-ordered row of hub hubs[h] (l = num_labels: the row's end).
void launch_hub_segments(const GraphDev &g, const int32_t *hubs, int32_t H, int32_t *seg,
                         cudaStream_t s);

// The neighbour label count table of every vertex (labels < g.num_labels <=
// stride), from the label-segmented rows.
constexpr int32_t kNlcMaxLabels = 64;
void launch_label_counts(const GraphDev &g, uint8_t *nlc, int32_t stride, cudaStream_t s);

// Writes k bitmaps of n_words words and adds |C(u)| into sizes[u].
void launch_filter(const GraphDev &g, const FilterDesc &d, uint32_t *bitmaps,
                   unsigned long long *sizes, cudaStream_t s);

// One refinement round (Sec. 3.2 repeated pruning): v stays in C(u) iff it
// was there and, for every label group of u's query neighbours, v has at least
// as many neighbours in the union of the group's candidate sets as the group
// has members.  Reads bm_in, writes bm_out (k bitmaps each), adds the new
// |C(u)| into sizes[u].
struct RefineDesc {
  int32_t k;
  int32_t n_words;
  int32_t ngroups[kMaxK];
  uint32_t group_mask[kMaxK][kMaxK];  // query neighbours of u in group g
  int32_t group_need[kMaxK][kMaxK];   // their number
};
void launch_refine(const GraphDev &g, const RefineDesc &d, const uint32_t *bm_in,
                   uint32_t *bm_out, unsigned long long *sizes, cudaStream_t s);

// Exclusive scan: out[0..n] with out[n] = total.  tmp needs scan_tmp_elems(n)
// int64 elements.  The int64 form may run in place (in == out).
int64_t scan_tmp_elems(int64_t n);
// Kernels one scan of n elements launches (n <= 0: a memset, no kernel).
int scan_kernels(int64_t n);
void launch_scan_i32(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s);
void launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s);

// Bitmap -> ascending vertex list.  cnt: int32[n_words], off: int64[n_words+1]
// (scratch), tmp: scan_tmp_elems(n_words).
void launch_bitmap_to_list(const uint32_t *bitmap, int32_t n_words, int32_t *cnt, int64_t *off,
                           int64_t *tmp, int32_t *out, cudaStream_t s);

// Frontiers are column-major: position c of row r is F[c*ld + r].

// Advance setup of a level (Sec. 3.3): per row, pick the mapped neighbour of
// pi_i whose pi_i-label segment is shortest (the pivot) and record that
// segment's CSR start and the neighbour's slot in d.bpos (pstart, pslot: R
// entries); woff (R + 1 entries) receives the exclusive scan of the segment
// lengths, woff[R] = the level's candidate total.  One launch: the scan uses
// a decoupled look-back over tiles of rows.  F has leading dimension ld >= R.
// lookback: pivot_scan_words(R) words, zeroed before the launch (a memset,
// or launch_tile_rows' extra words); a look-back wait longer than spin_limit
// polls sets the error word.  stage (optional, device view of mapped host
// memory, 4 words) receives, once the kernel is done: [0] the row count,
// [1] non-zero if a wait ran out (this scan's or, with R_dev, the producing
// level's), [2] woff[R], [3] R_dev[2] (0 without R_dev).  stall_tile (-1 =
// none) is fault injection for tests: that tile never publishes its
// look-back word, so the waits of the tiles after it run out.
// With R_dev the row count is read on the device (R_dev[0]; R is its upper
// bound), R_dev[1] is the error word of the level that wrote F (when it is
// set, some rows were never written and no row is read) and R_dev[2] its
// probe bytes: the words a single-pass level leaves after its total.
int64_t pivot_scan_words(int64_t R);
void launch_pivot_scan(const GraphDev &g, const LevelDesc &d, const int32_t *F, int64_t ld,
                       int64_t R, int32_t *pstart, uint8_t *pslot, int64_t *woff,
                       unsigned long long *lookback, int32_t spin_limit, void *stage,
                       int32_t stall_tile, cudaStream_t s, const int64_t *R_dev = nullptr);

// Number of extend tiles for candidates [wa, wb).
int64_t extend_tiles(int64_t wa, int64_t wb, int32_t block);

// tile_row[0..tiles]: first row of every tile of candidates [wa, wb) of rows
// [ra, rb) (woff = exclusive work offsets of the level).
// Limits of one extend launch: wb - wa < 2^30, rows < 2^31, ld * (i+1) < 2^31.
// Also zeroes lookback[0 .. tiles + kLbExtra + extra_words) when lookback is
// non-null (the extra words: a following launch_pivot_scan's look-back).
void launch_tile_rows(const int64_t *woff, int64_t ra, int64_t rb, int64_t wa, int64_t wb,
                      int32_t block, int32_t *tile_row, unsigned long long *lookback,
                      cudaStream_t s, int64_t extra_words = 0);

// Verification pass over candidates [wa, wb): writes one survivor bit per
// candidate into masks (if non-null), one survivor count per tile into
// tile_cnt (if non-null), and adds the total into *total (if non-null).
void launch_extend_count(const GraphDev &g, const LevelDesc &d, const int32_t *F, int64_t ld,
                         const int32_t *pstart, const uint8_t *pslot, const int64_t *woff,
                         const int32_t *tile_row, int64_t wa, int64_t wb, int32_t block,
                         uint32_t *masks, int32_t *tile_cnt, unsigned long long *total,
                         cudaStream_t s);

// Where the write pass puts a row.  kSinkColumns: column-major int32 (the
// frontier layout), column c of row r at out[c*ld + r].  kSinkRows: row-major
// int32, out[r*k + c] (the result layout).  kSinkKeys: the packed sort key of
// the row (see launch_sort_rows_packed), word w of row r at out[w*ld + r].
enum SinkMode : int32_t { kSinkColumns = 0, kSinkRows = 1, kSinkKeys = 2 };
constexpr int kMaxKeyWords = 8;  // 16 columns x 31 bits < 512
struct RowSink {
  int32_t mode;
  int32_t k;     // row width (kSinkRows, kSinkKeys)
  int32_t bits;  // key bits per column (kSinkKeys)
  int32_t nw;    // key words (kSinkKeys)
  int64_t ld;    // elements per column / per key word
  int64_t row0;  // row of the first survivor
  void *out;
  // kSinkKeys with 1-2 words: rank[r] (the dense rank of parent row r's
  // sorted prefix) is or-ed into every key written from row r, at bit
  // rank_pos (above the k columns); null: none
  const int32_t *rank = nullptr;
  int32_t rank_pos = 0;
};

// Dense ranks of the prefix (positions 0..p-1) of the rows of a frontier
// piece whose rows stand sorted by it, continuing the ranks of the pieces
// before it (pieces in order): state holds the last rank given (-1 at the
// start of a query) and the prefix it was given to.
struct PrefixState {
  long long last;
  int32_t prefix[kMaxK];
};
// Resets *st for a new query.
void launch_prefix_state_reset(PrefixState *st, cudaStream_t s);
// rank[r] for rows [0, rows) of F (leading dimension ld); flags and offs
// (rows + 1 int64) and tmp (scan_tmp_elems(rows) int64) are scratch.
// Returns the kernels launched.
int launch_prefix_ranks(const int32_t *F, int64_t ld, int64_t rows, int32_t p, PrefixState *st,
                        int32_t *flags, int64_t *offs, int64_t *tmp, int32_t *rank,
                        cudaStream_t s);

// Write pass: survivor q of tile t becomes row sink.row0 + tile_off[t] + rank;
// input position c goes to column d.out_col[c], the new vertex to column
// d.out_col[d.i].
void launch_extend_write(const GraphDev &g, const LevelDesc &d, const int32_t *F, int64_t ld,
                         const int32_t *pstart, const int64_t *woff, const int32_t *tile_row,
                         int64_t wa, int64_t wb, int32_t block, const uint32_t *masks,
                         const int64_t *tile_off, const RowSink &sink, cudaStream_t s);

// Single-pass form of the count and write passes (not for the count-only
// last level): survivors of candidates [wa, wb) go to rows sink.row0 + 0, 1,
// ... in candidate order, exactly where the two passes put them.  lookback
// needs extend_tiles(wa, wb, block) + kLbExtra words, zeroed (launch_tile_rows
// does it); afterwards word tiles + 1 holds the survivor count, word
// tiles + 2 is non-zero if a tile gave up waiting for its predecessors (after
// spin_limit polls) and word tiles + 3 holds the probe bytes (count_probes).
// The sink needs room for wb - wa rows.  The grid is persistent (at most the
// CTAs that fit on the device at once).  stall_tile (-1 = none) is fault
// injection for tests: that tile never publishes its look-back word, so later
// tiles' waits run out.
constexpr int kLbExtra = 4;
constexpr unsigned long long kLbAggregate = 1ull << 62, kLbInclusive = 2ull << 62;
constexpr unsigned long long kLbValue = (1ull << 62) - 1;
constexpr int32_t kLbSpinLimit = 1 << 20;  // default bound of a look-back wait (polls)
void launch_extend_fused(const GraphDev &g, const LevelDesc &d, const int32_t *F, int64_t ld,
                         const int32_t *pstart, const uint8_t *pslot, const int64_t *woff,
                         const int32_t *tile_row, int64_t wa, int64_t wb, int32_t block,
                         unsigned long long *lookback, const RowSink &sink, int32_t spin_limit,
                         int32_t stall_tile, cudaStream_t s);

// Row boundaries for work-bounded sub-chunks: bounds[j] = the row r with
// woff[r] <= j*step < woff[r+1] (clamped to [0, R]); bounds[J] = R.
void launch_split_points(const int64_t *woff, int64_t R, int64_t step, int64_t J,
                         int64_t *bounds, int64_t *bound_w, cudaStream_t s);

// Copies `bytes` (a multiple of 4, at most 4096) from src to dst with one
// small kernel; dst is typically the device view of mapped pinned host memory,
// so small reads back to the host do not queue behind copy-engine transfers.
void launch_fetch(const void *src, void *dst, size_t bytes, cudaStream_t s);

// Sorting many small results at once (one CTA each): rows src (count x k,
// row-major) into canonical lexicographic order at dst (count x k); sort = 0
// copies.  count <= kSmallSortRows when sort != 0.
constexpr int32_t kSmallSortRows = 1024;
struct SmallSortItem {
  const int32_t *src;
  int32_t *dst;
  int32_t count, k, sort;
};
// Dynamic shared memory k_sort_small needs for rows of at most max_k ints.
size_t small_sort_smem(int32_t max_k);
// items: device array of nitems entries; max_k = the widest row among them.
void launch_sort_small(const SmallSortItem *items, int32_t nitems, int32_t max_k,
                       cudaStream_t s);

// Lexicographic sort of N rows of k int32 (values < 2^bits) by column 0,
// then 1, ...  Each row is a k*bits-bit integer, sum_j c_j << ((k-1-j)*bits),
// held as packed_words(k, bits) little-endian 64-bit words (word w of row r at
// keys[w*ld + r], ld >= N).  If `a` is non-null the keys are first packed into
// keys_a from the column-major rows a (leading dimension lda); otherwise
// keys_a already holds them.  LSD radix passes over byte digits move the keys
// between keys_a and keys_b, and the last pass writes the rows row-major into
// `out` (N x k, must not overlap keys_a / keys_b; it may alias `a`).  Only
// columns 0 .. sort_cols-1 are sorted on (1 <= sort_cols <= k): the caller
// guarantees that rows with equal values there already stand in order of
// the remaining columns, which the stable passes keep.  Keys of one or two
// words (N < 2^30) take single-sweep passes (one histogram launch, then one
// launch per digit whose tiles find their offsets by a decoupled look-back);
// wider keys take per-tile histograms and a scan per digit.  scratch:
// sort_scratch_bytes(N, k, bits, sort_cols) bytes of device memory, 256-byte
// aligned, contents not kept.  err: null, or two words: a look-back wait
// longer than spin_limit polls (<= 0: the library default) sets err[0] to 1
// and leaves the rows out of order, every write still inside `out`; a failed
// bounds check of the GSM_DEBUG build writes its site to err[1].
// stall_tile >= 0 (fault injection for tests): that tile of every
// single-sweep pass never publishes its counts.  Returns the number of
// kernels launched.
// Optional knowledge of the input order: the rows already stand sorted by
// their first `cols` columns (1 <= cols < sort_cols), with at most `groups`
// distinct prefixes.  The sort then orders those columns by the prefix's
// dense rank (ceil(log2 groups) bits or-ed in at sort_rank_pos, when the
// key words have room and it saves digit passes: one flag pass, a scan and
// one rank pass instead of the prefix's own digits); the result is the same.
//
// given_bits > 0 instead: the keys already carry a dense rank of their group
// (rows of one group contiguous, groups in order) in given_bits bits above
// the k columns, and the key is ceil((k*bits + given_bits)/64) words wide;
// the sort orders the groups by it (segmented sort of many row sets at once).
struct SortPrefix {
  int32_t cols = 0;
  int64_t groups = 0;
  int32_t given_bits = 0;
  // with cols: the keys already carry the prefix's dense rank at
  // sort_rank_pos (written by the last level, RowSink::rank): the sort
  // computes none
  bool ranked = false;
};
// One segment of a segmented sort: the rows [src, src + count*k) (row-major)
// become compact rows first .. first + count - 1, group `index`.
struct SortSegment {
  const int32_t *src;
  int64_t first, count;
};
// Packs the segments' rows (segs: device array of nseg entries, ascending
// `first`, N rows in all) into keys of nw words (word w of row r at
// keys[w*ld + r]) with the segment's index in bits [k*bits, k*bits + seg_bits).
void launch_pack_segments(const SortSegment *segs, int32_t nseg, int64_t N, int32_t k,
                          int32_t bits, int32_t seg_bits, int32_t nw, uint64_t *keys, int64_t ld,
                          cudaStream_t s);
int32_t packed_words(int32_t k, int32_t bits);
size_t sort_scratch_bytes(int64_t N, int32_t k, int32_t bits, int32_t sort_cols,
                          SortPrefix pre = SortPrefix());
// Bit where a prefix rank goes in the keys of a sort on sort_cols columns:
// above the k columns and above every bit the plain digit passes read, so
// that keys carrying a rank sort right whether or not the sort uses it.
int32_t sort_rank_pos(int32_t k, int32_t bits, int32_t sort_cols);
// Key words of a sort (wider with given_bits).
int32_t sort_key_words(int32_t k, int32_t bits, SortPrefix pre = SortPrefix());
// Digit passes the sort makes (and whether it ranks the prefix).
int32_t sort_digit_passes(int64_t N, int32_t k, int32_t bits, int32_t sort_cols,
                          SortPrefix pre = SortPrefix(), bool *prefix_rank = nullptr);
int launch_sort_rows_packed(const int32_t *a, int64_t lda, int64_t N, int32_t k, int32_t bits,
                            int32_t sort_cols, uint64_t *keys_a, uint64_t *keys_b, int64_t ld,
                            int32_t *out, void *scratch, int32_t spin_limit, uint32_t *err,
                            int32_t stall_tile, cudaStream_t s, SortPrefix pre = SortPrefix());

}  // namespace gsm
