// Device kernels of the matcher: graph validation, candidate filtering,
// candidate-list compaction, scans, and the two passes of one verification
// level (count/verify with survivor bitmask, then write).
//
// Paper mapping (Sec. 3.2, Algorithm 1; Sec. 3.3):
//   k_filter            Filter_candidate_set (label / degree / neighbourhood)
//   k_bitmap_*          the first frontier: compaction of C(pi_0)
//   k_pivot_scan        Advance setup: which mapped neighbour's row to traverse,
//                       and the scan of the rows' work
//   k_extend_count      Advance + Compute: check label, injectivity and every
//                       non-tree edge of each traversed candidate in one step
//   k_scan_*            the compaction scan
//   k_extend_write      Write_to_Partial: survivors to consecutive rows
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdio>
#include <type_traits>

#include "filter_body.cuh"
#include "segments.cuh"
#include "kernels.cuh"
#include "verify.cuh"

namespace gsm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanThreads = 256;
constexpr int kScanIpt = 8;
constexpr int kScanTile = kScanThreads * kScanIpt;

// Binary search of key in the ascending slice col[beg, end).
__device__ __forceinline__ bool row_contains(const int32_t *__restrict__ col, int32_t beg,
                                             int32_t end, int32_t key) {
  int32_t lo = beg, len = end - beg;
  while (len > 0) {
    int32_t half = len >> 1;
    if (__ldg(col + lo + half) < key) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo < end && __ldg(col + lo) == key;
}

// First index in [lo, hi) with a[idx] > key, or hi.
__device__ __forceinline__ int64_t upper_bound_i64(const int64_t *__restrict__ a, int64_t lo,
                                                   int64_t hi, int64_t key) {
  int64_t len = hi - lo;
  while (len > 0) {
    int64_t half = len >> 1;
    if (a[lo + half] <= key) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo;
}

// ------------------------------------------------------------ validation

__global__ void k_validate_rp(int32_t n, int64_t nnz, const int32_t *__restrict__ rp,
                              int32_t *err) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
    int32_t x = rp[v];
    bool bad = x < 0 || x > nnz;
    if (v == 0 && x != 0) bad = true;
    if (v == n && (int64_t)x != nnz) bad = true;
    if (v < n && rp[v + 1] < x) bad = true;
    if (bad) atomicOr(err, 4);
  }
}

// One warp per vertex; lanes stride over the row.
__global__ void k_validate_rows(int32_t n, const int32_t *__restrict__ rp,
                                const int32_t *__restrict__ col, int32_t *err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int32_t b = rp[v], e = rp[v + 1];
    int32_t flags = 0;
    for (int32_t idx = b + lane; idx < e; idx += 32) {
      const int32_t w = col[idx];
      if (w < 0 || w >= n || w == (int32_t)v || (idx > b && col[idx - 1] >= w)) {
        flags |= 1;
        continue;
      }
      if (!row_contains(col, rp[w], rp[w + 1], (int32_t)v)) flags |= 2;
    }
    if (flags) atomicOr(err, flags);
  }
}

// ------------------------------------------------------------ filter

__global__ void __launch_bounds__(256) k_filter(GraphDev g, FilterDesc d,
                                                uint32_t *__restrict__ bitmaps,
                                                unsigned long long *__restrict__ sizes) {
  filter_warps(g, d, bitmaps, sizes, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
               ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// ------------------------------------------------------------ refinement

// One warp per (query vertex u, word of 32 data vertices).  Each candidate v
// of the word is scanned by the whole warp 256 neighbours at a time; a lane
// counts, per label group, neighbours in the union of the group's candidate
// sets, and the scan stops once every group has enough.
__global__ void __launch_bounds__(256) k_refine(GraphDev g, RefineDesc d,
                                                const uint32_t *__restrict__ bm_in,
                                                uint32_t *__restrict__ bm_out,
                                                unsigned long long *__restrict__ sizes) {
  const int lane = threadIdx.x & 31;
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = (int64_t)d.k * d.n_words;
  for (int64_t item = warp_id; item < total; item += n_warps) {
    const int32_t u = (int32_t)(item / d.n_words);
    const int64_t grp = item % d.n_words;
    uint32_t word = bm_in[(int64_t)u * d.n_words + grp];
    uint32_t out = word;
    const int ng = d.ngroups[u];
    if (ng > 0) {
      uint32_t todo = word;
      while (todo) {
        const int bit = __ffs(todo) - 1;
        todo &= todo - 1;
        const int32_t v = (int32_t)(grp * 32 + bit);
        const int32_t b = g.rp[v], e = g.rp[v + 1];
        int32_t cnt[kMaxK];
#pragma unroll
        for (int x = 0; x < kMaxK; ++x) cnt[x] = 0;
        bool pass = false;
        for (int32_t base = b; base < e && !pass; base += 256) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int32_t idx = base + j * 32 + lane;
            if (idx < e) {
              const int32_t w = __ldg(g.col + idx);
              uint32_t in = 0;  // query vertices whose candidate set holds w
              for (int uu = 0; uu < d.k; ++uu)
                in |= ((__ldg(bm_in + (int64_t)uu * d.n_words + (w >> 5)) >> (w & 31)) & 1u) << uu;
#pragma unroll
              for (int x = 0; x < kMaxK; ++x)
                if (x < ng && (in & d.group_mask[u][x])) ++cnt[x];
            }
          }
          bool all = true;
#pragma unroll
          for (int x = 0; x < kMaxK; ++x)
            if (x < ng) all = all && __reduce_add_sync(kFull, cnt[x]) >= d.group_need[u][x];
          pass = all;  // warp-uniform
        }
        if (!pass) out &= ~(1u << bit);
      }
    }
    if (lane == 0) {
      bm_out[(int64_t)u * d.n_words + grp] = out;
      if (out) atomicAdd(sizes + u, (unsigned long long)__popc(out));
    }
  }
}

// ------------------------------------------------------------ scans

__device__ __forceinline__ int64_t warp_incl_scan(int64_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive block scan of one value per thread (blockDim.x <= 1024); returns
// the exclusive prefix and writes the block total to *total.
__device__ int64_t block_excl_scan(int64_t x, int64_t *s_warp, int64_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  int64_t incl = warp_incl_scan(x, lane);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int64_t t = lane < nw ? s_warp[lane] : 0;
    int64_t ti = warp_incl_scan(t, lane);
    if (lane < nw) s_warp[lane] = ti - t;
    if (lane == 31) s_warp[32] = ti;
  }
  __syncthreads();
  int64_t r = incl - x + s_warp[warp];
  *total = s_warp[32];
  __syncthreads();
  return r;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const T *in, int64_t n,
                                                              int64_t *partial) {
  __shared__ int64_t s_warp[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t sum = 0;
#pragma unroll
  for (int j = 0; j < kScanIpt; ++j) {
    int64_t idx = base + j * kScanThreads + threadIdx.x;
    if (idx < n) sum += in[idx];
  }
  int64_t total;
  block_excl_scan(sum, s_warp, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_partials(int64_t *partial, int64_t nb) {
  __shared__ int64_t s_warp[33];
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    int64_t idx = base + threadIdx.x;
    int64_t x = idx < nb ? partial[idx] : 0;
    int64_t total;
    int64_t ex = block_excl_scan(x, s_warp, &total);
    if (idx < nb) partial[idx] = ex + carry;
    carry += total;
  }
  if (threadIdx.x == 0) partial[nb] = carry;
}

// In-place safe: a CTA reads its whole tile before writing it, and out[n]
// lies past the input.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const T *in, int64_t n,
                                                            const int64_t *__restrict__ partial,
                                                            int64_t nb, int64_t *out) {
  __shared__ int64_t s_val[kScanTile];
  __shared__ int64_t s_warp[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int j = 0; j < kScanIpt; ++j) {
    int64_t idx = base + j * kScanThreads + threadIdx.x;
    s_val[j * kScanThreads + threadIdx.x] = idx < n ? (int64_t)in[idx] : 0;
  }
  __syncthreads();
  int64_t loc[kScanIpt];
  int64_t sum = 0;
#pragma unroll
  for (int j = 0; j < kScanIpt; ++j) {
    loc[j] = sum;
    sum += s_val[threadIdx.x * kScanIpt + j];
  }
  int64_t total;
  int64_t ex = block_excl_scan(sum, s_warp, &total);
  const int64_t off = partial[blockIdx.x] + ex;
#pragma unroll
  for (int j = 0; j < kScanIpt; ++j) s_val[threadIdx.x * kScanIpt + j] = off + loc[j];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kScanIpt; ++j) {
    int64_t idx = base + j * kScanThreads + threadIdx.x;
    if (idx < n) out[idx] = s_val[j * kScanThreads + threadIdx.x];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = partial[nb];
}

// Whole scan in one CTA for short inputs (one launch instead of three): tiles
// of kOneThreads x kScanIpt elements in order, with a running carry.
// In-place safe for the same reason as k_scan_down.
constexpr int kOneThreads = 512;
constexpr int64_t kOneCtaMax = 4 * kOneThreads * kScanIpt;  // longest input taken
template <typename T>
__global__ void __launch_bounds__(kOneThreads) k_scan_one_cta(const T *in, int64_t n,
                                                              int64_t *out) {
  constexpr int kTile = kOneThreads * kScanIpt;
  __shared__ int64_t s_val[kTile];
  __shared__ int64_t s_warp[33];
  int64_t carry = 0;
  for (int64_t base = 0; base < n; base += kTile) {
#pragma unroll
    for (int j = 0; j < kScanIpt; ++j) {
      const int64_t idx = base + j * kOneThreads + threadIdx.x;
      s_val[j * kOneThreads + threadIdx.x] = idx < n ? (int64_t)in[idx] : 0;
    }
    __syncthreads();
    int64_t loc[kScanIpt];
    int64_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanIpt; ++j) {
      loc[j] = sum;
      sum += s_val[threadIdx.x * kScanIpt + j];
    }
    int64_t total;
    const int64_t off = carry + block_excl_scan(sum, s_warp, &total);
#pragma unroll
    for (int j = 0; j < kScanIpt; ++j) s_val[threadIdx.x * kScanIpt + j] = off + loc[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanIpt; ++j) {
      const int64_t idx = base + j * kOneThreads + threadIdx.x;
      if (idx < n) out[idx] = s_val[j * kOneThreads + threadIdx.x];
    }
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

// ------------------------------------------------------------ bitmap -> list

__global__ void k_bitmap_popc(const uint32_t *__restrict__ bm, int32_t n_words,
                              int32_t *__restrict__ cnt) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_words; w += stride)
    cnt[w] = __popc(bm[w]);
}

__global__ void k_bitmap_emit(const uint32_t *__restrict__ bm, int32_t n_words,
                              const int64_t *__restrict__ off, int32_t *__restrict__ out) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_words; w += stride) {
    uint32_t word = bm[w];
    int64_t pos = off[w];
    while (word) {
      int b = __ffs(word) - 1;
      word &= word - 1;
      out[pos++] = (int32_t)(w * 32 + b);
    }
  }
}

// ------------------------------------------------------------ extend
//
// Frontiers are column-major (SoA): position c of row r of a frontier with
// leading dimension ld is F[c*ld + r], so a warp reading one position of 32
// consecutive rows, or writing one position of 32 consecutive survivors,
// touches 128 contiguous bytes.

// Advance setup of a level in one pass: every row's pivot and the
// exclusive scan of the rows' work into woff (woff[R] = the total).
// Tiles of kPsRows consecutive rows are taken by ticket; a tile's offset
// comes from the decoupled look-back of the single-pass level
// (lookback_prefix), so the scan needs no second launch.  lookback:
// ptiles + kLbExtra zeroed words (tile words, then the ticket, the total,
// the error word and the count of finished CTAs).  The CTA that finishes
// last writes woff[R] and, with stage (mapped host memory), stage[0] = the
// row count, stage[1] = the error words (the producing level's and this
// scan's, OR-ed), stage[2] = the total and stage[3] = the producing level's
// probe bytes.  R_dev: as for launch_pivot_scan.
constexpr int kPsThreads = 256, kPsIpt = 4;
constexpr int64_t kPsRows = (int64_t)kPsThreads * kPsIpt;
__global__ void __launch_bounds__(kPsThreads, 4) k_pivot_scan(
    GraphDev g, LevelDesc d, const int32_t *__restrict__ F, int64_t ld, int64_t R,
    int32_t ptiles, int32_t *__restrict__ pstart, uint8_t *__restrict__ pslot,
    int64_t *__restrict__ woff, const int64_t *R_dev, unsigned long long *lookback,
    int32_t spin_limit, long long *stage, int32_t stall_tile) {
  __shared__ int64_t s_val[kPsRows];
  __shared__ int64_t s_warp[33];
  __shared__ int32_t s_tile;
  __shared__ unsigned long long s_prefix;
  // the actual row count (R is then the launch's bound); a set error word
  // beside it means the level that wrote the rows gave up a wait, so some
  // rows were never written: read none of them
  long long rows_in = R, lvl_err = 0, lvl_probes = 0;
  if (R_dev) {
    rows_in = R_dev[0];
    lvl_err = R_dev[1];
    lvl_probes = R_dev[2];
    R = lvl_err ? 0 : min(R, (int64_t)rows_in);
  }
  const int32_t ntiles = (int32_t)((R + kPsRows - 1) / kPsRows);  // <= ptiles
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int32_t)atomicAdd(lookback + ptiles, 1ull);
    __syncthreads();
    const int32_t tile = s_tile;
    if (tile >= ntiles) break;  // uniform across the block
    const int64_t base = (int64_t)tile * kPsRows;
    // rows base + j*kPsThreads + t: each load and store of a warp covers 32
    // consecutive rows.  Per row, the pivot is the mapped neighbour of pi_i
    // whose pi_i-label segment is shortest (only pi_i's label can match);
    // its length is the row's work.  Neighbour slot b is taken for all of a
    // thread's rows at once, so their loads are in flight together.
    int32_t best[kPsIpt], bstart[kPsIpt], bslot[kPsIpt];
#pragma unroll
    for (int j = 0; j < kPsIpt; ++j) {
      best[j] = base + j * kPsThreads + threadIdx.x < R ? 0x7fffffff : 0;
      bstart[j] = 0;
      bslot[j] = 0;
    }
    for (int b = 0; b < d.nb; ++b) {
      int32_t x[kPsIpt];
#pragma unroll
      for (int j = 0; j < kPsIpt; ++j)  // rows past R, or with no work left, read nothing
        x[j] = best[j] ? F[(int64_t)d.bpos[b] * ld + base + j * kPsThreads + threadIdx.x] : 0;
#pragma unroll
      for (int j = 0; j < kPsIpt; ++j) {
        if (!best[j]) continue;
        if (!GSM_IN_BOUNDS(g.dbg, x[j] >= 0 && x[j] < g.n, kDbgPivotVertex)) {
          best[j] = 0;  // the row gets no candidates
          bstart[j] = 0;
          bslot[j] = b;
          continue;
        }
        const int2 seg = label_segment(g, x[j], d.lab);
        if (seg.y - seg.x < best[j]) {
          best[j] = seg.y - seg.x;
          bstart[j] = seg.x;
          bslot[j] = b;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kPsIpt; ++j) {
      const int64_t r = base + j * kPsThreads + threadIdx.x;
      if (r < R) {
        pstart[r] = bstart[j];
        pslot[r] = (uint8_t)bslot[j];
      }
      s_val[j * kPsThreads + threadIdx.x] = r < R ? best[j] : 0;
    }
    __syncthreads();
    // thread t scans rows base + t*kPsIpt .. + kPsIpt - 1
    int64_t loc[kPsIpt];
    int64_t sum = 0;
#pragma unroll
    for (int j = 0; j < kPsIpt; ++j) {
      loc[j] = sum;
      sum += s_val[threadIdx.x * kPsIpt + j];
    }
    int64_t total;
    const int64_t ex = block_excl_scan(sum, s_warp, &total);
    if (warp == 0) {
      // stall_tile (fault injection) adds its work to the total but never
      // publishes its tile word, so the waits of the tiles after it run out
      if (lane == 0) {
        if (tile != stall_tile)
          lookback_publish(lookback, tile, ptiles, (unsigned long long)total);
        else if (total)
          atomicAdd(lookback + ptiles + 1, (unsigned long long)total);
      }
      __syncwarp();
      const unsigned long long p = lookback_resolve(lookback, tile, ptiles,
                                                    (unsigned long long)total, lane, spin_limit,
                                                    tile != stall_tile);
      if (lane == 0) s_prefix = p;
    }
    __syncthreads();
    const int64_t off = (int64_t)s_prefix + ex;
#pragma unroll
    for (int j = 0; j < kPsIpt; ++j) s_val[threadIdx.x * kPsIpt + j] = off + loc[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPsIpt; ++j) {
      const int64_t r = base + j * kPsThreads + threadIdx.x;
      if (r < R) woff[r] = s_val[j * kPsThreads + threadIdx.x];
    }
    __syncthreads();  // s_val and s_tile are reused by the next tile
  }
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's offsets and look-back words before its count
    const unsigned long long done = atomicAdd(lookback + ptiles + 3, 1ull);
    if (done == gridDim.x - 1) {  // every other CTA has finished
      __threadfence();
      const long long W = (long long)atomicAdd(lookback + ptiles + 1, 0ull);
      const long long err = (long long)atomicAdd(lookback + ptiles + 2, 0ull);
      woff[R] = W;
      if (stage) {
        stage[0] = rows_in;
        stage[1] = lvl_err | err;
        stage[2] = W;
        stage[3] = lvl_probes;
      }
    }
  }
}

// tile_row[t] = the row whose candidates include local item t*tile_items
// (rows partition the items, so exactly one row writes each entry);
// tile_row[tiles] = rb - 1.  Rows < 2^31.  Also zeroes lookback[0, lb_words).
__global__ void k_tile_rows(const int64_t *__restrict__ woff, int64_t ra, int64_t rb, int64_t wa,
                            int64_t tile_items, int64_t tiles, int32_t *__restrict__ tile_row,
                            unsigned long long *__restrict__ lookback, int64_t lb_words) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < lb_words; t += stride)
    lookback[t] = 0;
  for (int64_t r = ra + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rb; r += stride) {
    const int64_t s = woff[r] - wa, e = woff[r + 1] - wa;
    if (e <= s) continue;
    for (int64_t t = (s + tile_items - 1) / tile_items; t * tile_items < e; ++t)
      tile_row[t] = (int32_t)r;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tile_row[tiles] = (int32_t)(rb - 1);
}

// Verification pass.  Thread t of a tile takes the kItemsPerThread consecutive
// candidates 4t .. 4t+3: one row search serves all of them (rows change inside
// the group only at a row boundary), and the warp's 128 candidates are
// consecutive, so its candidate loads cover contiguous bytes.  The survivor
// bits stay in candidate order: each lane's 4-bit group is shifted into place
// and OR-ed across the 8 lanes that share a 32-bit mask word.
template <bool kMasks>
__global__ void __launch_bounds__(1024) k_extend_count(
    GraphDev g, LevelDesc d, const int32_t *__restrict__ F, int32_t ld,
    const int32_t *__restrict__ pstart, const uint8_t *__restrict__ pslot,
    const int64_t *__restrict__ woff, const int32_t *__restrict__ tile_row, int64_t wa,
    int32_t W, uint32_t *__restrict__ masks, int32_t *__restrict__ tile_cnt,
    unsigned long long *__restrict__ total) {
  static_assert(kItemsPerThread == 4, "one 4-bit group per lane");
  extern __shared__ int32_t s_woff[];
  __shared__ int32_t s_count;
  const int32_t B = blockDim.x;
  const int32_t tile_items = B * kItemsPerThread;
  const int32_t x0 = blockIdx.x * tile_items;
  const int32_t x1 = min(x0 + tile_items, W);
  if (threadIdx.x == 0) s_count = 0;
  const TileRows t = stage_rows(woff, tile_row, wa, tile_items, s_woff, blockIdx.x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t xb = x0 + warp * 128 + lane * kItemsPerThread;
  uint32_t bits = 0;
  if (xb < x1) {
    int32_t rs;
    int32_t r = item_row(t, s_woff, woff, wa, xb, &rs);
    int32_t rr = r - t.r0;
    int32_t re = t.staged ? s_woff[rr + 1] : (int32_t)(woff[r + 1] - wa);
    int32_t pst = pstart[r], slot = pslot[r];
#pragma unroll
    for (int j = 0; j < kItemsPerThread; ++j) {
      const int32_t x = xb + j;
      if (x >= x1) break;
      while (x >= re) {  // next row (rows without work are skipped)
        ++rr;
        ++r;
        rs = re;
        re = t.staged ? s_woff[rr + 1] : (int32_t)(woff[r + 1] - wa);
        pst = pstart[r];
        slot = pslot[r];
      }
      const int32_t w = __ldg(g.lcol + pst + (x - rs));
      if (check_candidate(g, d, ColumnRow{F, ld, r}, w, slot) &&
          (!d.la || lookahead_ok(g, d, ColumnRow{F, ld, r}, w)))
        bits |= 1u << j;
    }
  }
  uint32_t word = bits << (4 * (lane & 7));
  word |= __shfl_xor_sync(kFull, word, 1);
  word |= __shfl_xor_sync(kFull, word, 2);
  word |= __shfl_xor_sync(kFull, word, 4);
  int32_t cnt = 0;
  if ((lane & 7) == 0) {
    if (kMasks) masks[(x0 + warp * 128) / 32 + (lane >> 3)] = word;
    cnt = __popc(word);
  }
  cnt = __reduce_add_sync(kFull, cnt);
  if (lane == 0 && cnt) atomicAdd(&s_count, cnt);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (tile_cnt) tile_cnt[blockIdx.x] = s_count;
    if (total && s_count) atomicAdd(total, (unsigned long long)s_count);
  }
}

// Position (0..31) of the n-th (0-based) set bit of m; m has more than n.
__device__ __forceinline__ int nth_set_bit(uint32_t m, int n) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w; w >>= 1) {
    const uint32_t lo = m & ((1u << w) - 1u);
    const int c = __popc(lo);
    if (n >= c) {
      n -= c;
      m >>= w;
      pos += w;
    } else {
      m = lo;
    }
  }
  return pos;
}

// Write pass: survivor q of tile t becomes output row sink.row0 + tile_off[t]
// + q; thread q of the CTA handles it (survivors are dense over the threads,
// whatever the survival rate), so each store of a warp covers 32 consecutive
// rows.  Position c of the input row goes to column out_col[c], the new
// vertex to column out_col[i], of a column-major frontier, a row-major result
// row, or the row's packed sort key (the last level writes the final layout
// directly, so no separate transpose or packing pass reads the rows again).
template <int kMode>
__global__ void __launch_bounds__(1024) k_extend_write(
    GraphDev g, LevelDesc d, const int32_t *__restrict__ F, int32_t ld,
    const int32_t *__restrict__ pstart, const int64_t *__restrict__ woff,
    const int32_t *__restrict__ tile_row, int64_t wa, int32_t W,
    const uint32_t *__restrict__ masks, const int64_t *__restrict__ tile_off, RowSink sink) {
  extern __shared__ int32_t s_woff[];
  __shared__ uint32_t s_mask[kItemsPerThread * 1024 / 32];
  __shared__ int32_t s_wpre[kItemsPerThread * 1024 / 32];
  const int64_t base = tile_off[blockIdx.x];
  const int32_t cnt = (int32_t)(tile_off[blockIdx.x + 1] - base);
  if (cnt == 0) return;  // uniform across the block
  const int32_t B = blockDim.x;
  const int32_t tile_items = B * kItemsPerThread;
  const int32_t tile_words = tile_items / 32;
  const int32_t x0 = blockIdx.x * tile_items;
  for (int32_t w = threadIdx.x; w < tile_words; w += B)
    s_mask[w] = masks[blockIdx.x * tile_words + w];
  const TileRows t = stage_rows(woff, tile_row, wa, tile_items, s_woff, blockIdx.x);
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    int32_t carry = 0;
    for (int32_t c = 0; c < tile_words; c += 32) {
      const int32_t idx = c + lane;
      const int32_t v = idx < tile_words ? __popc(s_mask[idx]) : 0;
      int32_t incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      if (idx < tile_words) s_wpre[idx] = carry + incl - v;
      carry += __shfl_sync(kFull, incl, 31);
    }
  }
  __syncthreads();
  for (int32_t q = threadIdx.x; q < cnt; q += B) {
    // word holding survivor q: the last word whose prefix count is <= q
    int32_t lo = 0, hi = tile_words;
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (s_wpre[mid] <= q) lo = mid; else hi = mid;
    }
    const int32_t x = x0 + lo * 32 + nth_set_bit(s_mask[lo], q - s_wpre[lo]);
    int32_t rs;
    const int32_t r = item_row(t, s_woff, woff, wa, x, &rs);
    const int32_t w = __ldg(g.lcol + pstart[r] + (x - rs));
    put_row<kMode>(sink, d, ColumnRow{F, ld, r}, w, sink.row0 + base + q);
  }
}

// Count and write in one pass (single-pass compaction), persistent: every CTA
// takes tiles (1,024 candidates at 256 threads) from a ticket counter until
// none is left.  For each tile it verifies the candidates, ranks the
// survivors with a block scan, keeps them (row, vertex) in one of two
// shared-memory buffers and publishes its survivor count (decoupled
// look-back).  The tile's own look-back and writes wait until the CTA has
// verified its next tile: by then the earlier tiles have published, so the
// look-back rarely waits and the SM is not idle at the barrier.  Survivors
// are written directly at their final rows, in candidate order, as the
// two-pass form would write them.
//
// Thread t of a tile takes the 4 consecutive candidates 4t .. 4t+3 (one row
// search for all four, in the tile's staged work offsets).  Non-tree edges
// to hubs are checked on the hubs' adjacency bitmaps (one probe), the others
// by binary search of the row (row_contains_l).  Result rows of an even width
// are stored by their own thread with 16- or 8-byte stores; the others are
// assembled in shared memory and stored contiguously.
//
// lookback: tiles words, then the ticket, the survivor total and an error
// word, all zero at launch.  A look-back that polls more than spin_limit
// times sets the error word and goes on with the prefix found so far (rows
// stay in bounds; the host reports the error).  stall_tile >= 0 is fault
// injection for tests: that tile never publishes its word, so the waits of
// the tiles after it run out.
constexpr size_t kFusedSmemAttr = 200 * 1024;  // dynamic shared memory a CTA may use
constexpr size_t kFusedStageMax = 96 * 1024;   // ... with the tile's result rows staged

// kMaxThreads = 256: up to 256 threads per CTA, registers capped so that six
// CTAs fit on an SM; 1024: any block size.
template <int kMode, int kMaxThreads, bool kProbes>
__global__ void __launch_bounds__(kMaxThreads, kMaxThreads == 256 ? 6 : 1) k_extend_fused(
    GraphDev g, LevelDesc d, const int32_t *__restrict__ F, int32_t ld,
    const int32_t *__restrict__ pstart, const uint8_t *__restrict__ pslot,
    const int64_t *__restrict__ woff, const int32_t *__restrict__ tile_row, int64_t wa,
    int32_t W, int32_t tiles, unsigned long long *__restrict__ lookback, RowSink sink,
    bool stage_out, int32_t spin_limit, int32_t stall_tile) {
  static_assert(kItemsPerThread == 4, "four candidates per thread");
  constexpr unsigned kAll = 0xffffffffu;
  extern __shared__ int32_t smem[];
  __shared__ int32_t s_tile;
  __shared__ int32_t s_warp[33];
  __shared__ long long s_prefix;
  const int32_t B = blockDim.x;
  const int32_t tile_items = B * kItemsPerThread;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // shared memory: staged work offsets | survivor pairs x 2 | assembled
  // result rows (stage_out only)
  int32_t *s_woff = smem;
  int32_t *s_pairs = s_woff + tile_items + 4;
  int32_t *s_out = s_pairs + 4 * tile_items;
  int32_t pend = -1, pend_T = 0, pend_buf = 0, buf = 0;

  // lookback + write of a verified tile whose survivors are in buffer pb
  auto finish = [&](int32_t tile, int32_t T, int32_t pb) {
    if (warp == 0) {
      const unsigned long long prefix =
          lookback_resolve(lookback, tile, tiles, (unsigned long long)T, lane, spin_limit,
                           tile != stall_tile);
      if (lane == 0) s_prefix = (long long)prefix;
    }
    __syncthreads();
    const int32_t *pairs = s_pairs + pb * 2 * tile_items;
    const int64_t base = sink.row0 + s_prefix;
    // (GSM_DEBUG) the level reserved W rows from sink.row0
    if (!GSM_IN_BOUNDS(g.dbg, s_prefix >= 0 && s_prefix + T <= W, kDbgOutputRow)) return;
    if (kMode == kSinkRows && (sink.k & 1) == 0) {
      // result rows in the matching order (the identity here: rows are only
      // written directly when it is canonical); an even row width is stored
      // with 16- or 8-byte stores, so each warp store covers 32 whole rows
      const int32_t k = sink.k, i = d.i;
      for (int32_t q = threadIdx.x; q < T; q += B) {
        const int32_t r = pairs[2 * q], w = pairs[2 * q + 1];
        int32_t *dst = (int32_t *)sink.out + (base + q) * k;
        auto col = [&](int c) { return c < i ? F[c * ld + r] : w; };
        if ((k & 3) == 0) {
          for (int c = 0; c < k; c += 4)
            *reinterpret_cast<int4 *>(dst + c) = make_int4(col(c), col(c + 1), col(c + 2),
                                                           col(c + 3));
        } else {
          for (int c = 0; c < k; c += 2)
            *reinterpret_cast<int2 *>(dst + c) = make_int2(col(c), col(c + 1));
        }
      }
    } else if (kMode == kSinkRows && stage_out) {
      // the tile's result rows are one contiguous block of T*k ints:
      // assemble them in shared memory, then store them contiguously
      const int32_t k = sink.k;
      for (int32_t q = threadIdx.x; q < T; q += B) {
        const int32_t r = pairs[2 * q];
        for (int cc = 0; cc < d.i; ++cc) s_out[q * k + d.out_col[cc]] = F[cc * ld + r];
        s_out[q * k + d.out_col[d.i]] = pairs[2 * q + 1];
      }
      __syncthreads();
      int32_t *dst = (int32_t *)sink.out + base * k;
      for (int32_t e = threadIdx.x; e < T * k; e += B) dst[e] = s_out[e];
    } else {
      // survivor q is written by thread q (q, q + B, ...): each store of a
      // warp covers 32 consecutive output rows
      for (int32_t q = threadIdx.x; q < T; q += B)
        put_row<kMode>(sink, d, ColumnRow{F, ld, pairs[2 * q]}, pairs[2 * q + 1], base + q);
    }
  };

  for (;;) {
    if (threadIdx.x == 0) s_tile = (int32_t)atomicAdd(lookback + tiles, 1ull);
    __syncthreads();
    const int32_t tile = s_tile;
    if (tile >= tiles) break;  // uniform across the block
    const int32_t x0 = tile * tile_items;
    const int32_t x1 = min(x0 + tile_items, W);
    const TileRows t = stage_rows(woff, tile_row, wa, tile_items, s_woff, tile);
    const int32_t xb = x0 + warp * 128 + lane * kItemsPerThread;
    uint32_t bits = 0, probes = 0;
    int32_t rj[kItemsPerThread], wj[kItemsPerThread];
    if (xb < x1) {
      int32_t rs;
      int32_t r = item_row(t, s_woff, woff, wa, xb, &rs);
      int32_t rr = r - t.r0;
      int32_t re = t.staged ? s_woff[rr + 1] : (int32_t)(woff[r + 1] - wa);
      int32_t pst = pstart[r], slot = pslot[r];
#pragma unroll
      for (int j = 0; j < kItemsPerThread; ++j) {
        rj[j] = r;
        wj[j] = 0;
        const int32_t x = xb + j;
        if (x >= x1) continue;
        while (x >= re) {  // next row (rows without work are skipped)
          ++rr;
          ++r;
          rs = re;
          re = t.staged ? s_woff[rr + 1] : (int32_t)(woff[r + 1] - wa);
          pst = pstart[r];
          slot = pslot[r];
        }
        if (!GSM_IN_BOUNDS(g.dbg, pst + (x - rs) >= 0 && pst + (x - rs) < g.nnz, kDbgCandidate) ||
            !GSM_IN_BOUNDS(g.dbg, r >= 0 && r < ld, kDbgRow))
          continue;
        const int32_t w = __ldg(g.lcol + pst + (x - rs));
        rj[j] = r;
        wj[j] = w;
        bool ok;
        if constexpr (kProbes)
          ok = check_candidate_probes(g, d, ColumnRow{F, ld, r}, w, slot, &probes);
        else
          ok = check_candidate(g, d, ColumnRow{F, ld, r}, w, slot);
        if (ok && (!d.la || lookahead_ok(g, d, ColumnRow{F, ld, r}, w))) bits |= 1u << j;
      }
    }
    if constexpr (kProbes) {
#pragma unroll
      for (int o = 16; o; o >>= 1) probes += __shfl_xor_sync(kAll, probes, o);
      if (lane == 0 && probes) atomicAdd(lookback + tiles + 3, (unsigned long long)probes);
    }
    // rank of this thread's survivors in the tile (thread order is
    // candidate order); the survivors go to the free pair buffer
    const int32_t c = __popc(bits);
    int32_t T;
    const int32_t rank = block_rank(c, s_warp, &T);
    {
      int32_t *s_pair = s_pairs + buf * 2 * tile_items;
      int32_t q = rank;
#pragma unroll
      for (int j = 0; j < kItemsPerThread; ++j)
        if ((bits >> j) & 1u) {
          s_pair[2 * q] = rj[j];
          s_pair[2 * q + 1] = wj[j];
          ++q;
        }
    }
    if (threadIdx.x == 0) {
      if (tile != stall_tile)
        lookback_publish(lookback, tile, tiles, (unsigned long long)T);
      else if (T)
        atomicAdd(lookback + tiles + 1, (unsigned long long)T);  // the total stays right
    }
    __syncthreads();
    if (pend >= 0) finish(pend, pend_T, pend_buf);
    pend = tile;
    pend_T = T;
    pend_buf = buf;
    buf ^= 1;
  }
  if (pend >= 0) finish(pend, pend_T, pend_buf);
}

__global__ void k_split_points(const int64_t *__restrict__ woff, int64_t R, int64_t step,
                               int64_t J, int64_t *bounds, int64_t *bound_w) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j > J) return;
  int64_t r;
  if (j == J) {
    r = R;
  } else {
    r = upper_bound_i64(woff, 0, R + 1, j * step) - 1;
    if (r < 0) r = 0;
    if (r > R) r = R;
  }
  bounds[j] = r;
  bound_w[j] = woff[r];
}

__global__ void k_fetch(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, int32_t n) {
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// flags[r] = 1 where row r's prefix (positions 0..p-1) differs from row
// r-1's, or, for r = 0, from the prefix the last earlier piece ended with.
__global__ void k_prefix_change(const int32_t *__restrict__ F, int64_t ld, int64_t rows,
                                int32_t p, const PrefixState *__restrict__ st,
                                int32_t *__restrict__ flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
    bool diff = false;
    for (int32_t c = 0; c < p; ++c) {
      const int32_t prev = r > 0 ? F[(int64_t)c * ld + r - 1] : st->prefix[c];
      diff = diff || F[(int64_t)c * ld + r] != prev;
    }
    flags[r] = diff ? 1 : 0;
  }
}

// rank[r] = the last rank of the earlier pieces + the changes up to r
// (offs: exclusive scan of the flags, offs[rows] = their total).
__global__ void k_prefix_rank(const int64_t *__restrict__ offs, int64_t rows,
                              const PrefixState *__restrict__ st, int32_t *__restrict__ rank) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const long long last = st->last;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride)
    rank[r] = (int32_t)(last + offs[r + 1]);
}

// After the piece: the state takes its last rank and last row's prefix.
__global__ void k_prefix_advance(const int32_t *__restrict__ F, int64_t ld, int64_t rows,
                                 int32_t p, const int64_t *__restrict__ offs,
                                 PrefixState *__restrict__ st) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && rows > 0) {
    st->last += offs[rows];
    for (int32_t c = 0; c < p; ++c) st->prefix[c] = F[(int64_t)c * ld + rows - 1];
  }
}

__global__ void k_prefix_reset(PrefixState *st) {
  if (threadIdx.x == 0) {
    st->last = -1;
    for (int32_t c = 0; c < kMaxK; ++c) st->prefix[c] = -1;  // no vertex id: a change
  }
}

// One warp per hub: every neighbour's bit of the hub's bitmap.
__global__ void k_hub_bits(GraphDev g, const int32_t *__restrict__ hubs, int32_t H,
                           int32_t words, uint32_t *__restrict__ bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t h = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < H; h += warps) {
    const int32_t v = hubs[h];
    uint32_t *b = bits + h * words;
    for (int32_t e = g.rp[v] + lane; e < g.rp[v + 1]; e += 32) {
      const int32_t w = g.col[e];
      atomicOr(b + (w >> 5), 1u << (w & 31));
    }
  }
}

// One warp per vertex: the lanes count the vertex's neighbours per label in
// shared memory (the labels of its label-segmented row), then write the
// saturated counts.
__global__ void __launch_bounds__(256) k_label_counts(GraphDev g, uint8_t *__restrict__ nlc,
                                                      int32_t stride) {
  __shared__ int32_t s_cnt[8][kNlcMaxLabels];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < g.n; v += warps) {
    for (int l = lane; l < stride; l += 32) s_cnt[warp][l] = 0;
    __syncwarp();
    const int32_t b = g.rp[v], e = g.rp[v + 1];
    for (int32_t x = b + lane; x < e; x += 32) atomicAdd(&s_cnt[warp][g.llab[x]], 1);
    __syncwarp();
    for (int l = lane; l < stride; l += 32) nlc[v * stride + l] = (uint8_t)min(s_cnt[warp][l], 255);
    __syncwarp();
  }
}

// One warp per hub: lane l finds where labels l, l + 32, ... start in the
// hub's (label, id)-ordered row (lower bound of the label).
__global__ void k_hub_segments(GraphDev g, const int32_t *__restrict__ hubs, int32_t H,
                               int32_t *__restrict__ seg) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t L = g.num_labels;
  for (int64_t h = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < H; h += warps) {
    const int32_t v = hubs[h];
    const int32_t b = g.rp[v], e = g.rp[v + 1];
    for (int32_t l = lane; l <= L; l += 32) {
      int32_t lo = b, len = e - b;
      while (len > 0) {
        const int32_t half = len >> 1;
        if (g.llab[lo + half] < l) {
          lo += half + 1;
          len -= half + 1;
        } else {
          len = half;
        }
      }
      seg[h * (L + 1) + l] = lo;
    }
  }
}

inline int grid_for(int64_t n, int threads, int cap = 152 * 32) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// Edge e of row v becomes the 3-column row (v, label of col[e], col[e]),
// column-major with leading dimension nnz.
// One warp per vertex (rows of power-law graphs are very uneven).
__global__ void k_edge_rows(GraphDev g, int32_t *__restrict__ cols) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < g.n; v += warps) {
    const int32_t e1 = g.rp[v + 1];
    for (int32_t e = g.rp[v] + lane; e < e1; e += 32) {
      const int32_t w = g.col[e];
      cols[e] = (int32_t)v;
      cols[g.nnz + e] = g.lab[w];
      cols[2 * g.nnz + e] = w;
    }
  }
}

// Row-major (v, label, id) triples -> the label and id columns.
__global__ void k_split_segments(const int32_t *__restrict__ rows, int64_t nnz,
                                 int32_t *__restrict__ out_col, int32_t *__restrict__ out_lab) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    out_lab[e] = rows[3 * e + 1];
    out_col[e] = rows[3 * e + 2];
  }
}

}  // namespace

int32_t label_segment_bits(int32_t n, int32_t num_labels) {
  int32_t bits = 1;
  const int64_t m = std::max<int64_t>(n, num_labels);
  while (bits < 31 && (int64_t(1) << bits) < m) ++bits;
  return bits;
}

int launch_label_segments(const GraphDev &g, int32_t num_labels, int32_t *edge_cols,
                          uint64_t *keys, int32_t *rows_out, void *sort_scratch, uint32_t *err,
                          int32_t *out_col, int32_t *out_lab, cudaStream_t s) {
  if (g.nnz == 0) return 0;
  k_edge_rows<<<grid_for((int64_t)g.n * 32, 256, 152 * 8), 256, 0, s>>>(g, edge_cols);
  const int32_t bits = label_segment_bits(g.n, num_labels);
  const int32_t nw = packed_words(3, bits);
  // CSR rows are already ordered by (row, id): sorting on (row, label) is enough
  int launches = 1 + launch_sort_rows_packed(edge_cols, g.nnz, g.nnz, 3, bits, 2, keys,
                                             keys + (size_t)g.nnz * nw, g.nnz, rows_out,
                                             sort_scratch, 0, err, -1, s);
  k_split_segments<<<grid_for(g.nnz, 256), 256, 0, s>>>(rows_out, g.nnz, out_col, out_lab);
  return launches + 1;
}

void launch_fetch(const void *src, void *dst, size_t bytes, cudaStream_t s) {
  const int32_t n = (int32_t)(std::min<size_t>(bytes, 4096) / 4);
  if (n > 0) k_fetch<<<1, 128, 0, s>>>((const uint32_t *)src, (uint32_t *)dst, n);
}

void launch_validate(const GraphDev &g, int32_t *err, cudaStream_t s) {
  k_validate_rp<<<grid_for((int64_t)g.n + 1, 256), 256, 0, s>>>(g.n, g.nnz, g.rp, err);
  // rows are only read if row_ptr is sane; the host checks err in between
}

void launch_validate_rows(const GraphDev &g, int32_t *err, cudaStream_t s) {
  k_validate_rows<<<grid_for((int64_t)g.n * 32, 256, 152 * 8), 256, 0, s>>>(g.n, g.rp, g.col, err);
}

void launch_hub_bitmaps(const GraphDev &g, const int32_t *hubs, int32_t H, int32_t words,
                        uint32_t *bits, cudaStream_t s) {
  if (H <= 0) return;
  cudaMemsetAsync(bits, 0, sizeof(uint32_t) * (size_t)H * words, s);
  k_hub_bits<<<grid_for((int64_t)H * 32, 256, 152 * 8), 256, 0, s>>>(g, hubs, H, words, bits);
}

void launch_prefix_state_reset(PrefixState *st, cudaStream_t s) {
  k_prefix_reset<<<1, 32, 0, s>>>(st);
}

int launch_prefix_ranks(const int32_t *F, int64_t ld, int64_t rows, int32_t p, PrefixState *st,
                        int32_t *flags, int64_t *offs, int64_t *tmp, int32_t *rank,
                        cudaStream_t s) {
  if (rows <= 0) return 0;
  const unsigned g = grid_for(rows, 256, 152 * 8);
  k_prefix_change<<<g, 256, 0, s>>>(F, ld, rows, p, st, flags);
  launch_scan_i32(flags, offs, rows, tmp, s);
  k_prefix_rank<<<g, 256, 0, s>>>(offs, rows, st, rank);
  k_prefix_advance<<<1, 32, 0, s>>>(F, ld, rows, p, offs, st);
  return 3 + scan_kernels(rows);
}

void launch_label_counts(const GraphDev &g, uint8_t *nlc, int32_t stride, cudaStream_t s) {
  if (g.n <= 0) return;
  k_label_counts<<<grid_for((int64_t)g.n * 32, 256, 152 * 16), 256, 0, s>>>(g, nlc, stride);
}

void launch_hub_segments(const GraphDev &g, const int32_t *hubs, int32_t H, int32_t *seg,
                         cudaStream_t s) {
  if (H <= 0) return;
  k_hub_segments<<<grid_for((int64_t)H * 32, 256, 152 * 8), 256, 0, s>>>(g, hubs, H, seg);
}

void launch_filter(const GraphDev &g, const FilterDesc &d, uint32_t *bitmaps,
                   unsigned long long *sizes, cudaStream_t s) {
  const int threads = 256;
  int64_t warps_needed = d.n_words;
  int blocks = grid_for(warps_needed * 32, threads, 152 * 16);
  k_filter<<<blocks, threads, 0, s>>>(g, d, bitmaps, sizes);
}

void launch_refine(const GraphDev &g, const RefineDesc &d, const uint32_t *bm_in,
                   uint32_t *bm_out, unsigned long long *sizes, cudaStream_t s) {
  const int64_t warps = (int64_t)d.k * d.n_words;
  k_refine<<<grid_for(warps * 32, 256, 152 * 16), 256, 0, s>>>(g, d, bm_in, bm_out, sizes);
}

int64_t scan_tmp_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

template <typename T>
void scan_impl(const T *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) {
    cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    return;
  }
  if (n <= kOneCtaMax) {
    k_scan_one_cta<T><<<1, kOneThreads, 0, s>>>(in, n, out);
    return;
  }
  k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
  k_scan_partials<<<1, 1024, 0, s>>>(tmp, nb);
  k_scan_down<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp, nb, out);
}

int scan_kernels(int64_t n) {
  if (n <= 0) return 0;
  return n <= kOneCtaMax ? 1 : 3;
}

void launch_scan_i32(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
  scan_impl<int32_t>(in, out, n, tmp, s);
}

void launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
  scan_impl<int64_t>(in, out, n, tmp, s);
}

void launch_bitmap_to_list(const uint32_t *bitmap, int32_t n_words, int32_t *cnt, int64_t *off,
                           int64_t *tmp, int32_t *out, cudaStream_t s) {
  k_bitmap_popc<<<grid_for(n_words, 256), 256, 0, s>>>(bitmap, n_words, cnt);
  launch_scan_i32(cnt, off, n_words, tmp, s);
  k_bitmap_emit<<<grid_for(n_words, 256), 256, 0, s>>>(bitmap, n_words, off, out);
}

int64_t pivot_scan_words(int64_t R) {
  return std::max<int64_t>(1, (R + kPsRows - 1) / kPsRows) + kLbExtra;
}

void launch_pivot_scan(const GraphDev &g, const LevelDesc &d, const int32_t *F, int64_t ld,
                       int64_t R, int32_t *pstart, uint8_t *pslot, int64_t *woff,
                       unsigned long long *lookback, int32_t spin_limit, void *stage,
                       int32_t stall_tile, cudaStream_t s, const int64_t *R_dev) {
  const int64_t ptiles = pivot_scan_words(R) - kLbExtra;
  const int grid = (int)std::min<int64_t>(ptiles, 152 * 4);  // the CTAs resident at once
  k_pivot_scan<<<grid, kPsThreads, 0, s>>>(g, d, F, ld, R, (int32_t)ptiles, pstart, pslot, woff,
                                           R_dev, lookback, spin_limit, (long long *)stage,
                                           stall_tile);
}

int64_t extend_tiles(int64_t wa, int64_t wb, int32_t block) {
  const int64_t tile_items = (int64_t)block * kItemsPerThread;
  return (wb - wa + tile_items - 1) / tile_items;
}

void launch_tile_rows(const int64_t *woff, int64_t ra, int64_t rb, int64_t wa, int64_t wb,
                      int32_t block, int32_t *tile_row, unsigned long long *lookback,
                      cudaStream_t s, int64_t extra_words) {
  const int64_t tiles = extend_tiles(wa, wb, block);
  if (tiles <= 0 && extra_words <= 0) return;
  const int64_t lb_words = lookback ? tiles + kLbExtra + extra_words : 0;
  const int64_t n = std::max<int64_t>(rb - ra, lb_words);
  k_tile_rows<<<grid_for(n, 256, 152 * 64), 256, 0, s>>>(
      woff, ra, rb, wa, (int64_t)block * kItemsPerThread, tiles, tile_row, lookback, lb_words);
}

void launch_extend_count(const GraphDev &g, const LevelDesc &d, const int32_t *F, int64_t ld,
                         const int32_t *pstart, const uint8_t *pslot, const int64_t *woff,
                         const int32_t *tile_row, int64_t wa, int64_t wb, int32_t block,
                         uint32_t *masks, int32_t *tile_cnt, unsigned long long *total,
                         cudaStream_t s) {
  const int64_t tiles = extend_tiles(wa, wb, block);
  if (tiles <= 0) return;
  const size_t smem = (size_t)((int64_t)block * kItemsPerThread + 1) * sizeof(int32_t);
  if (masks)
    k_extend_count<true><<<(unsigned)tiles, block, smem, s>>>(
        g, d, F, (int32_t)ld, pstart, pslot, woff, tile_row, wa, (int32_t)(wb - wa), masks,
        tile_cnt, total);
  else
    k_extend_count<false><<<(unsigned)tiles, block, smem, s>>>(
        g, d, F, (int32_t)ld, pstart, pslot, woff, tile_row, wa, (int32_t)(wb - wa), masks,
        tile_cnt, total);
}

void launch_extend_write(const GraphDev &g, const LevelDesc &d, const int32_t *F, int64_t ld,
                         const int32_t *pstart, const int64_t *woff, const int32_t *tile_row,
                         int64_t wa, int64_t wb, int32_t block, const uint32_t *masks,
                         const int64_t *tile_off, const RowSink &sink, cudaStream_t s) {
  const int64_t tiles = extend_tiles(wa, wb, block);
  if (tiles <= 0) return;
  const size_t smem = (size_t)((int64_t)block * kItemsPerThread + 1) * sizeof(int32_t);
  const int32_t W = (int32_t)(wb - wa);
  if (sink.mode == kSinkRows)
    k_extend_write<kSinkRows><<<(unsigned)tiles, block, smem, s>>>(
        g, d, F, (int32_t)ld, pstart, woff, tile_row, wa, W, masks, tile_off, sink);
  else if (sink.mode == kSinkKeys)
    k_extend_write<kSinkKeys><<<(unsigned)tiles, block, smem, s>>>(
        g, d, F, (int32_t)ld, pstart, woff, tile_row, wa, W, masks, tile_off, sink);
  else
    k_extend_write<kSinkColumns><<<(unsigned)tiles, block, smem, s>>>(
        g, d, F, (int32_t)ld, pstart, woff, tile_row, wa, W, masks, tile_off, sink);
}

namespace {
// One persistent launch of k_extend_fused<kMode, ..., kProbes>: as many CTAs as fit on the
// device at once (at most one per tile).  The dynamic shared-memory limit is
// raised once per device for this instance.
template <int kMode, int kMaxThreads, bool kProbes>
void launch_fused_mode(const GraphDev &g, const LevelDesc &d, const int32_t *F, int64_t ld,
                       const int32_t *pstart, const uint8_t *pslot, const int64_t *woff,
                       const int32_t *tile_row, int64_t wa, int32_t W, int32_t tiles,
                       int32_t block, size_t smem, unsigned long long *lookback,
                       const RowSink &sink, bool stage, int32_t spin_limit, int32_t stall_tile,
                       cudaStream_t s) {
  static std::atomic<unsigned long long> attr_set{0};  // bit per device
  // occupancy of the last (block, smem) this host thread launched with
  static thread_local int per_sm_cache[64][2] = {};
  static thread_local size_t smem_cache[64] = {};
  static thread_local int blocks_cache[64] = {};
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int di = dev & 63;
  if (!((attr_set.load() >> di) & 1ull)) {
    cudaFuncSetAttribute(k_extend_fused<kMode, kMaxThreads, kProbes>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemAttr);
    attr_set.fetch_or(1ull << di);
  }
  int per_sm = 0;
  if (blocks_cache[di] == block && smem_cache[di] == smem && per_sm_cache[di][0]) {
    per_sm = per_sm_cache[di][1];
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_extend_fused<kMode, kMaxThreads, kProbes>,
                                                  block, smem);
    blocks_cache[di] = block;
    smem_cache[di] = smem;
    per_sm_cache[di][0] = 1;
    per_sm_cache[di][1] = per_sm;
  }
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)std::max(per_sm, 1) * sms);
  k_extend_fused<kMode, kMaxThreads, kProbes><<<(unsigned)grid, block, smem, s>>>(
      g, d, F, (int32_t)ld, pstart, pslot, woff, tile_row, wa, W, tiles, lookback, sink, stage,
      spin_limit, stall_tile);
}
}  // namespace

void launch_extend_fused(const GraphDev &g, const LevelDesc &d, const int32_t *F, int64_t ld,
                         const int32_t *pstart, const uint8_t *pslot, const int64_t *woff,
                         const int32_t *tile_row, int64_t wa, int64_t wb, int32_t block,
                         unsigned long long *lookback, const RowSink &sink, int32_t spin_limit,
                         int32_t stall_tile, cudaStream_t s) {
  const int64_t tiles = extend_tiles(wa, wb, block);
  if (tiles <= 0) return;
  const int32_t W = (int32_t)(wb - wa), T = (int32_t)tiles;
  // staged work offsets, two survivor-pair buffers, the warps' windows, and
  // (kSinkRows) the assembled result rows of one tile when they fit
  const int64_t items = (int64_t)block * kItemsPerThread;
  const size_t base_ints = (size_t)(items + 4 + 4 * items);
  size_t smem = base_ints * sizeof(int32_t);
  // odd result widths are assembled in shared memory (even ones are stored
  // directly)
  const size_t smem_rows = (base_ints + (size_t)items * sink.k) * sizeof(int32_t);
  const bool stage = sink.mode == kSinkRows && (sink.k & 1) && smem_rows <= kFusedStageMax;
  if (stage) smem = smem_rows;
  auto go = [&](auto small, auto probes) {
    constexpr int kMax = decltype(small)::value ? 256 : 1024;
    constexpr bool kP = decltype(probes)::value;
    if (sink.mode == kSinkRows)
      launch_fused_mode<kSinkRows, kMax, kP>(g, d, F, ld, pstart, pslot, woff, tile_row, wa, W,
                                             T, block, smem, lookback, sink, stage, spin_limit,
                                             stall_tile, s);
    else if (sink.mode == kSinkKeys)
      launch_fused_mode<kSinkKeys, kMax, kP>(g, d, F, ld, pstart, pslot, woff, tile_row, wa, W,
                                             T, block, smem, lookback, sink, false, spin_limit,
                                             stall_tile, s);
    else
      launch_fused_mode<kSinkColumns, kMax, kP>(g, d, F, ld, pstart, pslot, woff, tile_row, wa,
                                                W, T, block, smem, lookback, sink, false,
                                                spin_limit, stall_tile, s);
  };
  // the probe-byte accounting is a separate instance, so the default one
  // carries no trace of it
  if (block <= 256 && !d.count_probes)
    go(std::true_type{}, std::false_type{});
  else if (block <= 256)
    go(std::true_type{}, std::true_type{});
  else if (!d.count_probes)
    go(std::false_type{}, std::false_type{});
  else
    go(std::false_type{}, std::true_type{});
}

void launch_split_points(const int64_t *woff, int64_t R, int64_t step, int64_t J,
                         int64_t *bounds, int64_t *bound_w, cudaStream_t s) {
  k_split_points<<<(unsigned)((J + 1 + 255) / 256), 256, 0, s>>>(woff, R, step, J, bounds,
                                                                  bound_w);
}

}  // namespace gsm
