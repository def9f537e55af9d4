// Device helpers of the verification kernels (extend count, write, single
// pass): tile row staging, the candidate check and the row writer.
#pragma once

#include "kernels.cuh"
#include "segments.cuh"

namespace gsm {

__device__ __forceinline__ bool bitmap_has(const uint32_t *__restrict__ bm, int32_t v) {
  return (__ldg(bm + (v >> 5)) >> (v & 31)) & 1u;
}

// Inside one launch every index is 32-bit: candidates are numbered locally
// from wa (a launch covers fewer than 2^30), rows and frontier elements stay
// below 2^31 (the host code chunks frontiers to that), only output addresses of
// the final rows are 64-bit.
//
// A tile's rows [r0, r0+span): their work offsets, relative to wa, are staged
// in shared memory when they fit (span <= tile items: always, unless rows
// without work pile up); items then find their row by binary search there,
// otherwise in the global offsets.
struct TileRows {
  int32_t r0;
  int32_t span;
  bool staged;
};

__device__ __forceinline__ TileRows stage_rows(const int64_t *__restrict__ woff,
                                               const int32_t *__restrict__ tile_row, int64_t wa,
                                               int32_t tile_items, int32_t *s_woff,
                                               int32_t tile) {
  TileRows t;
  t.r0 = tile_row[tile];
  t.span = tile_row[tile + 1] + 1 - t.r0;
  t.staged = t.span <= tile_items;
  if (t.staged)
    for (int32_t j = threadIdx.x; j <= t.span; j += blockDim.x)
      s_woff[j] = (int32_t)(woff[t.r0 + j] - wa);
  __syncthreads();
  return t;
}

// Row of local item x and the local offset where that row's candidates start.
__device__ __forceinline__ int32_t item_row(const TileRows &t, const int32_t *s_woff,
                                            const int64_t *__restrict__ woff, int64_t wa,
                                            int32_t x, int32_t *row_start) {
  int32_t lo = 0, hi = t.span;  // largest j in [0, span) with offset(r0+j) <= x
  if (t.staged) {
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (s_woff[mid] <= x) lo = mid; else hi = mid;
    }
    *row_start = s_woff[lo];
  } else {
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (woff[t.r0 + mid] - wa <= x) lo = mid; else hi = mid;
    }
    *row_start = (int32_t)(woff[t.r0 + lo] - wa);
  }
  return t.r0 + lo;
}

// Position c of row r of a column-major frontier (leading dimension ld).
struct ColumnRow {
  const int32_t *__restrict__ F;
  int32_t ld, r;
  __device__ __forceinline__ int32_t operator()(int c) const { return F[c * ld + r]; }
};

// Index of the parent row a written row comes from (for the sink's prefix
// ranks); -1 where the row type has none.
__device__ __forceinline__ int32_t parent_index(const ColumnRow &r) { return r.r; }
template <typename Row>
__device__ __forceinline__ int32_t parent_index(const Row &) {
  return -1;
}

// The checks of Sec. 3.2 verification that need no adjacency search, for
// candidate w of a partial embedding (row(c) = the image of pi_c): label +
// signature (bitmap of C(pi_i)), injectivity against same-label, non-adjacent
// positions, and the ordering constraints of distinct counting.  Desc is a
// level description with the fields of LevelDesc used here (the single-query
// LevelDesc or the batched form's BatchLevel).
template <typename Desc, typename Row>
__device__ __forceinline__ bool check_local(const Desc &d, const Row &row, int32_t w) {
  if (!bitmap_has(d.bitmap, w)) return false;
  for (int t = 0; t < d.ninj; ++t)
    if (row(d.inj[t]) == w) return false;
  for (int t = 0; t < d.nlt; ++t)
    if (!(w < row(d.lt[t]))) return false;
  for (int t = 0; t < d.ngt; ++t)
    if (!(w > row(d.gt[t]))) return false;
  return true;
}

// The whole one-step check: check_local plus the presence of every query
// edge to a mapped neighbour other than the pivot (binary search in that
// neighbour's label segment).
template <typename Desc, typename Row>
__device__ __forceinline__ bool check_candidate(const GraphDev &g, const Desc &d,
                                                const Row &row, int32_t w, int slot) {
  if (!check_local(d, row, w)) return false;
  for (int b = 0; b < d.nb; ++b) {
    if (b == slot) continue;
    if (!row_contains_l(g, row(d.bpos[b]), d.lab, w)) return false;
  }
  return true;
}

// check_candidate that also adds to *probe_bytes 4 * ceil(log2 deg(x)) for
// every non-tree edge check it makes against a mapped vertex x (the bytes a
// binary search of x's row reads; the check itself may be one bitmap probe).
template <typename Desc, typename Row>
__device__ __forceinline__ bool check_candidate_probes(const GraphDev &g, const Desc &d,
                                                       const Row &row, int32_t w, int slot,
                                                       uint32_t *probe_bytes) {
  if (!check_local(d, row, w)) return false;
  for (int b = 0; b < d.nb; ++b) {
    if (b == slot) continue;
    const int32_t x = row(d.bpos[b]);
    const int32_t deg = __ldg(g.rp + x + 1) - __ldg(g.rp + x);
    *probe_bytes += deg > 1 ? 4u * (32u - __clz((uint32_t)(deg - 1))) : 0u;
    if (!row_contains_l(g, x, d.lab, w)) return false;
  }
  return true;
}

// Entries of w's (label, id)-ordered row scanned at most per group by the
// 2-look-ahead before it gives up (and keeps the candidate).
constexpr int32_t kLaScan = 64;

// The k-look-ahead of Sec. 3.2 for a candidate w of pi_i that passed the
// level's checks: does the partial embedding extended by w still leave room
// for the query neighbours of pi_i placed later?  For every label group t of
// those neighbours:
//   1-look-ahead: w keeps at least la_need[t] neighbours with the label that
//   are not in the row (its label segment, minus the mapped neighbours of
//   pi_i, which are adjacent to w, minus the other same-label row vertices
//   adjacent to w), since an embedding maps the group to distinct unused
//   neighbours of w;
//   2-look-ahead: at least la_need[t] of those unused neighbours are
//   candidates of some query vertex of the group (checked over the first
//   kLaScan entries of the segment; a longer segment is not pruned).
// Both conditions hold for every embedding that extends the row, so pruning
// on them never changes the result.
template <typename Row>
__device__ __forceinline__ bool lookahead_ok(const GraphDev &g, const LevelDesc &d,
                                             const Row &row, int32_t w) {
  for (int t = 0; t < d.nla; ++t) {
    const int2 seg = label_segment(g, w, d.la_lab[t]);
    int32_t avail = seg.y - seg.x - d.la_known[t];
    for (uint32_t m = d.la_pos[t]; m; m &= m - 1) {
      const int32_t x = row(__ffs(m) - 1);
      // x carries the label, so it is in w's row iff it is in the segment
      int32_t lo = seg.x, len = seg.y - seg.x;
      while (len > 0) {
        const int32_t half = len >> 1;
        if (__ldg(g.lcol + lo + half) < x) {
          lo += half + 1;
          len -= half + 1;
        } else {
          len = half;
        }
      }
      if (lo < seg.y && __ldg(g.lcol + lo) == x) --avail;
    }
    if (avail < d.la_need[t]) return false;
    if (d.la >= 2) {
      const int32_t end = min(seg.y, seg.x + kLaScan);
      int32_t found = 0;
      for (int32_t e = seg.x; e < end && found < d.la_need[t]; ++e) {
        const int32_t x = __ldg(g.lcol + e);
        bool cand = false;
        for (uint32_t u = d.la_uq[t]; u && !cand; u &= u - 1)
          cand = bitmap_has(d.cand + (size_t)(__ffs(u) - 1) * d.n_words, x);
        if (!cand) continue;
        bool used = false;  // a row vertex (only same-label positions can be)
        for (int c = 0; c < d.i && !used; ++c) used = row(c) == x;
        if (!used) ++found;
      }
      if (found < d.la_need[t] && end == seg.y) return false;
    }
  }
  return true;
}

// Writes the partial embedding `src` (src(c) = image of pi_c, c < d.i)
// extended by w as output row `row` of the sink (see RowSink): position c goes
// to column d.out_col[c], w to d.out_col[d.i].
template <int kMode, typename Row>
__device__ __forceinline__ void put_row(const RowSink &sink, const LevelDesc &d, const Row &src,
                                        int32_t w, int64_t row) {
  const int32_t i = d.i;
  if (kMode == kSinkColumns) {
    int32_t *o = (int32_t *)sink.out + row;
    for (int c = 0; c < i; ++c) o[d.out_col[c] * sink.ld] = src(c);
    o[d.out_col[i] * sink.ld] = w;
  } else if (kMode == kSinkRows) {
    int32_t *o = (int32_t *)sink.out + row * sink.k;
    for (int c = 0; c < i; ++c) o[d.out_col[c]] = src(c);
    o[d.out_col[i]] = w;
  } else if (sink.nw <= 2) {
    // packed key of one or two words: column j occupies bits
    // [(k-1-j)*b, (k-j)*b); each column is read once and or-ed into the
    // word(s) it overlaps
    uint64_t *o = (uint64_t *)sink.out + row;
    uint64_t w0 = 0, w1 = 0;
    for (int c = 0; c <= i; ++c) {
      const uint64_t v = (uint32_t)(c < i ? src(c) : w);
      const int32_t p = (sink.k - 1 - d.out_col[c]) * sink.bits;
      if (p >= 64) {
        w1 |= v << (p - 64);
      } else {
        w0 |= v << p;
        if (p + sink.bits > 64) w1 |= v >> (64 - p);
      }
    }
    if (sink.rank) {
      const int32_t pr = parent_index(src);
      if (pr >= 0) {
        const uint64_t v = (uint32_t)__ldg(sink.rank + pr);
        const int32_t p = sink.rank_pos;
        if (p >= 64) {
          w1 |= v << (p - 64);
        } else {
          w0 |= v << p;
          if (p > 32) w1 |= v >> (64 - p);
        }
      }
    }
    o[0] = w0;
    if (sink.nw == 2) o[sink.ld] = w1;
  } else {
    // packed key: column j occupies bits [(k-1-j)*b, (k-j)*b); word t
    // collects the columns that overlap bits [64t, 64t+64)
    uint64_t *o = (uint64_t *)sink.out + row;
    for (int t = 0; t < sink.nw; ++t) {
      uint64_t kw = 0;
      for (int c = 0; c <= i; ++c) {
        const uint64_t v = (uint32_t)(c < i ? src(c) : w);
        const int32_t lo = (sink.k - 1 - d.out_col[c]) * sink.bits - 64 * t;
        if (lo >= 0 && lo < 64)
          kw |= v << lo;
        else if (lo < 0 && lo + sink.bits > 0)
          kw |= v >> (-lo);
      }
      o[t * sink.ld] = kw;
    }
  }
}

__device__ __forceinline__ unsigned long long load_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}


// Exclusive rank of this thread's c items among the block's (threads in
// order) and the block total; s_warp holds 33 ints; contains two barriers.
__device__ __forceinline__ int32_t block_rank(int32_t c, int32_t *s_warp, int32_t *total) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kAll, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nwarps = blockDim.x >> 5;
    const int32_t v = lane < nwarps ? s_warp[lane] : 0;
    int32_t wi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(kAll, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < nwarps) s_warp[lane] = wi - v;
    if (lane == 31) s_warp[32] = wi;
  }
  __syncthreads();
  *total = s_warp[32];
  return incl - c + s_warp[warp];
}

// Decoupled look-back, in two halves so that a CTA can verify its next tile
// between them.  lookback_publish: tile `tile` has T survivors; tile 0
// publishes its inclusive prefix, every other tile its own count, and the
// level total (word tiles + 1) gains T.  Any thread may call it.
__device__ __forceinline__ void lookback_publish(unsigned long long *lookback, int32_t tile,
                                                 int32_t tiles, unsigned long long T) {
  atomicExch(lookback + tile, (tile == 0 ? kLbInclusive : kLbAggregate) | T);
  if (T) atomicAdd(lookback + tiles + 1, T);
}

// lookback_resolve, run by one whole warp after lookback_publish: reads the
// published words of the 32 preceding tiles at a time (lane l: tile
// window_end - l) until one holds an inclusive prefix, publishes the tile's
// own inclusive prefix, and returns the number of survivors of all earlier
// tiles in every lane.  A wait longer than spin_limit polls sets word
// tiles + 2 and returns the (smaller) sum found so far, so every row the
// caller writes stays inside the level's reserved output.  publish = false
// keeps the tile's word unwritten (fault injection: later tiles wait on it).
__device__ __forceinline__ unsigned long long lookback_resolve(unsigned long long *lookback,
                                                               int32_t tile, int32_t tiles,
                                                               unsigned long long T, int lane,
                                                               int32_t spin_limit,
                                                               bool publish = true) {
  constexpr unsigned kAll = 0xffffffffu;
  if (tile == 0) return 0;
  unsigned long long prefix = 0;
  int32_t window_end = tile - 1;
  int32_t polls = 0;
  bool gave_up = false;
  while (true) {
    const int32_t j = window_end - lane;
    unsigned long long st = j >= 0 ? load_relaxed(lookback + j) : kLbInclusive;
    unsigned long long flag = st & ~kLbValue;
    // wait until every tile of the window has published
    while (__any_sync(kAll, flag == 0)) {
      if (++polls > spin_limit) {
        gave_up = true;
        break;
      }
      __nanosleep(32);
      if (flag == 0) {
        st = load_relaxed(lookback + j);
        flag = st & ~kLbValue;
      }
    }
    if (gave_up) break;
    const uint32_t has_prefix = __ballot_sync(kAll, flag == kLbInclusive);
    // tiles up to the nearest inclusive prefix (the lowest such lane)
    const int32_t stop = has_prefix ? __ffs(has_prefix) - 1 : 31;
    unsigned long long v = lane <= stop ? (st & kLbValue) : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kAll, v, o);
    prefix += v;
    if (has_prefix) break;
    window_end -= 32;
  }
  if (lane == 0) {
    if (gave_up) atomicExch(lookback + tiles + 2, 1ull);
    if (publish) atomicExch(lookback + tile, kLbInclusive | (prefix + T));
  }
  return prefix;
}

// Both halves at once (the tile waits for its prefix right after counting).
__device__ __forceinline__ unsigned long long lookback_prefix(unsigned long long *lookback,
                                                              int32_t tile, int32_t tiles,
                                                              unsigned long long T, int lane,
                                                              int32_t spin_limit) {
  if (lane == 0) lookback_publish(lookback, tile, tiles, T);
  __syncwarp();
  return lookback_resolve(lookback, tile, tiles, T, lane, spin_limit);
}

}  // namespace gsm
