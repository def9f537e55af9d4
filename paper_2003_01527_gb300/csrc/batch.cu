// Batched form: many query graphs against one resident data graph, all
// levels of all queries issued as one fixed sequence of persistent kernels
// (captured once as a CUDA graph by the host driver).
//
// The queries advance together, one verification level per step (Sec. 3.2,
// Algorithm 1), over one concatenated frontier whose rows carry the index of
// their query ("segment").  No kernel needs a size from the host: every
// launch has a fixed grid and reads the sizes of its step (rows, candidates,
// tiles, survivors) from device memory, so the whole sequence runs without a
// host synchronisation.  Buffers have fixed capacities; a step that would
// exceed them sets an overflow flag, produces nothing further, and the host
// reruns the batch on the single-query path.
#include <algorithm>
#include <cstddef>

#include "batch.h"
#include "filter_body.cuh"
#include "segments.cuh"
#include "verify.cuh"

namespace gsm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPScanThreads = 256;
constexpr int kPScanTile = 2048;  // 8 elements per thread

__device__ __forceinline__ int64_t warp_incl(int64_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive scan of one value per thread of the block; *total = block sum.
__device__ int64_t block_scan(int64_t x, int64_t *s_warp, int64_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t incl = warp_incl(x, lane);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int64_t t = lane < nw ? s_warp[lane] : 0;
    const int64_t ti = warp_incl(t, lane);
    if (lane < nw) s_warp[lane] = ti - t;
    if (lane == 31) s_warp[32] = ti;
  }
  __syncthreads();
  const int64_t r = incl - x + s_warp[warp];
  *total = s_warp[32];
  __syncthreads();
  return r;
}

// ---- scans whose length lives in device memory (fixed grid of G blocks;
// block b owns a contiguous range of ceil(n/G) elements)

template <typename T>
__global__ void __launch_bounds__(kPScanThreads) k_pscan_reduce(const T *in, const int64_t *n_ptr,
                                                                int64_t *partials) {
  __shared__ int64_t s_warp[33];
  const int64_t n = *n_ptr;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(n, lo + chunk);
  int64_t sum = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) sum += (int64_t)in[i];
  int64_t total;
  block_scan(sum, s_warp, &total);
  if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_pscan_top(int64_t *partials, int32_t nb) {
  __shared__ int64_t s_warp[33];
  int64_t carry = 0;
  for (int32_t base = 0; base < nb; base += blockDim.x) {
    const int32_t idx = base + threadIdx.x;
    const int64_t x = idx < nb ? partials[idx] : 0;
    int64_t total;
    const int64_t ex = block_scan(x, s_warp, &total);
    if (idx < nb) partials[idx] = ex + carry;
    carry += total;
  }
  if (threadIdx.x == 0) partials[nb] = carry;
}

// In place safe (in == out for int64): each tile is read whole before it is
// written, and later tiles are untouched until their turn.
template <typename T>
__global__ void __launch_bounds__(kPScanThreads) k_pscan_down(const T *in, const int64_t *n_ptr,
                                                              const int64_t *partials,
                                                              int64_t *out) {
  __shared__ int64_t s_val[kPScanTile];
  __shared__ int64_t s_warp[33];
  const int64_t n = *n_ptr;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(n, lo + chunk);
  int64_t carry = partials[blockIdx.x];
  for (int64_t base = lo; base < hi; base += kPScanTile) {
    for (int j = threadIdx.x; j < kPScanTile; j += blockDim.x) {
      const int64_t idx = base + j;
      s_val[j] = idx < hi ? (int64_t)in[idx] : 0;
    }
    __syncthreads();
    int64_t loc[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      loc[j] = sum;
      sum += s_val[threadIdx.x * 8 + j];
    }
    int64_t total;
    const int64_t ex = block_scan(sum, s_warp, &total);
#pragma unroll
    for (int j = 0; j < 8; ++j) s_val[threadIdx.x * 8 + j] = carry + ex + loc[j];
    __syncthreads();
    for (int j = threadIdx.x; j < kPScanTile; j += blockDim.x) {
      const int64_t idx = base + j;
      if (idx < hi) out[idx] = s_val[j];
    }
    carry += total;
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = partials[gridDim.x];
}

// ---- set-up, filter and level 1

// Zeroes the step sizes and stores the number of root-bitmap words (the
// length of the level-1 scan) where the scan can read it.
__global__ void k_b_init(BatchStep *state, int64_t words) {
  for (int j = threadIdx.x; j <= kMaxK; j += blockDim.x) state[j] = BatchStep{0, 0, 0, 0, 0, 0};
  __syncthreads();
  if (threadIdx.x == 0) state[0].W = words;
}

__global__ void __launch_bounds__(256) k_b_filter(GraphDev g, const FilterDesc *__restrict__ fds,
                                                  uint32_t *const *__restrict__ bm_out,
                                                  unsigned long long *__restrict__ sizes) {
  __shared__ FilterDesc s_d;
  const int32_t q = blockIdx.y;
  for (int j = threadIdx.x; j < (int)(sizeof(FilterDesc) / 4); j += blockDim.x)
    reinterpret_cast<int32_t *>(&s_d)[j] = reinterpret_cast<const int32_t *>(fds + q)[j];
  __syncthreads();
  if (s_d.k == 0) return;  // padding slot of a bucketed batch
  filter_warps(g, s_d, bm_out[q], sizes + (int64_t)q * kMaxK,
               ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
               ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// Word counts of every query's root bitmap; one-vertex queries are counted
// here and contribute no rows.
__global__ void k_b_list_popc(const BatchQuery *__restrict__ qs, int32_t nq, int32_t n_words,
                              int32_t *__restrict__ wcnt, unsigned long long *__restrict__ counts) {
  const int64_t total = (int64_t)nq * n_words;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int32_t q = (int32_t)(i / n_words), w = (int32_t)(i % n_words);
    const int32_t c = __popc(__ldg(qs[q].root_bitmap + w));
    if (qs[q].k == 1) {
      if (c) atomicAdd(counts + q, (unsigned long long)c);
      wcnt[i] = 0;
    } else {
      wcnt[i] = c;
    }
  }
}

// Level-1 size check: rows = total set bits; over capacity -> overflow.
__global__ void k_b_list_check(const int64_t *__restrict__ woffs, int64_t words,
                               BatchStep *state, int64_t cap_rows, int32_t *overflow) {
  const int64_t R = woffs[words];
  if (R > cap_rows) {
    *overflow = 1;
    state[1].R = 0;
  } else {
    state[1].R = R;
  }
}

__global__ void k_b_list_emit(const BatchQuery *__restrict__ qs, int32_t nq, int32_t n_words,
                              const int64_t *__restrict__ woffs, const BatchStep *state,
                              int32_t *__restrict__ F, int32_t *__restrict__ rseg) {
  const int64_t total = (int64_t)nq * n_words;
  if (state[1].R != woffs[total]) return;  // overflowed: nothing to write
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int32_t q = (int32_t)(i / n_words), w = (int32_t)(i % n_words);
    if (qs[q].k == 1) continue;
    uint32_t word = __ldg(qs[q].root_bitmap + w);
    int64_t pos = woffs[i];
    while (word) {
      const int b = __ffs(word) - 1;
      word &= word - 1;
      F[pos] = w * 32 + b;
      rseg[pos] = q;
      ++pos;
    }
  }
}

// ---- one step: level i -> i+1 (frontier rows of width i, column-major,
// leading dimension R = state[i].R)

__global__ void k_b_pivot(GraphDev g, const BatchQuery *__restrict__ qs, int32_t i,
                          const BatchStep *state, const int32_t *__restrict__ F,
                          const int32_t *__restrict__ rseg, int32_t *__restrict__ pstart,
                          uint8_t *__restrict__ pslot, int64_t *__restrict__ work) {
  const int32_t R = (int32_t)state[i].R;
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    const BatchLevel &L = qs[rseg[r]].lv[i];
    int32_t best = 0x7fffffff, best_start = 0, best_slot = 0;
    for (int b = 0; b < L.nb; ++b) {
      const int32_t x = F[L.bpos[b] * R + r];
      const int2 seg = label_segment(g, x, L.lab);  // only pi_i's label can match
      if (seg.y - seg.x < best) {
        best = seg.y - seg.x;
        best_start = seg.x;
        best_slot = b;
      }
    }
    pstart[r] = best_start;
    pslot[r] = (uint8_t)best_slot;
    work[r] = best;
  }
}

// Candidates W = woff[R]; over capacity -> overflow and no tiles.
__global__ void k_b_check_work(int32_t i, BatchStep *state, const int64_t *__restrict__ woff,
                               int64_t cap_items, int32_t tile_items, int32_t *overflow) {
  const int64_t R = state[i].R;
  const int64_t W = R > 0 ? woff[R] : 0;
  if (W > cap_items) {
    *overflow = 1;
    state[i].W = 0;
    state[i].tiles = 0;
  } else {
    state[i].W = W;
    state[i].tiles = (W + tile_items - 1) / tile_items;
  }
}

__global__ void k_b_tile_rows(int32_t i, const BatchStep *state, const int64_t *__restrict__ woff,
                              int32_t tile_items, int32_t *__restrict__ tile_row) {
  const int32_t R = (int32_t)state[i].R;
  const int64_t tiles = state[i].tiles;
  if (tiles == 0) return;
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    const int64_t s = woff[r], e = woff[r + 1];
    for (int64_t t = (s + tile_items - 1) / tile_items; t * tile_items < e; ++t)
      tile_row[t] = r;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tile_row[tiles] = R - 1;
}

// Rows of one tile, with their work offsets staged in shared memory.
struct BTile {
  int32_t r0, span;
  bool staged;
};

__device__ __forceinline__ BTile b_stage(const int64_t *__restrict__ woff,
                                         const int32_t *__restrict__ tile_row, int64_t t,
                                         int32_t tile_items, int32_t *s_woff) {
  BTile b;
  b.r0 = tile_row[t];
  b.span = tile_row[t + 1] + 1 - b.r0;
  b.staged = b.span <= tile_items;
  if (b.staged)
    for (int32_t j = threadIdx.x; j <= b.span; j += blockDim.x) s_woff[j] = (int32_t)woff[b.r0 + j];
  __syncthreads();
  return b;
}

__device__ __forceinline__ int32_t b_row(const BTile &b, const int32_t *s_woff,
                                         const int64_t *__restrict__ woff, int32_t x,
                                         int32_t *row_start) {
  int32_t lo = 0, hi = b.span;
  if (b.staged) {
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (s_woff[mid] <= x) lo = mid; else hi = mid;
    }
    *row_start = s_woff[lo];
  } else {
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (woff[b.r0 + mid] <= x) lo = mid; else hi = mid;
    }
    *row_start = (int32_t)woff[b.r0 + lo];
  }
  return b.r0 + lo;
}

// Verification pass of one step.  A survivor of a query at its last level
// is counted into counts[q] (and, for a query that lists its rows, marked in
// fmasks and counted towards its tile in ftile_cnt); other survivors get
// their mask bit and count towards their tile.  The check is the
// single-query path's (check_candidate).  Thread t of a tile takes the 4
// consecutive candidates 4t .. 4t+3 (one row search for all four); the mask
// bits stay in candidate order (4-bit groups OR-ed across the 8 lanes of a
// mask word).
__global__ void __launch_bounds__(1024) k_b_count(
    GraphDev g, const BatchQuery *__restrict__ qs, int32_t i, const BatchStep *state,
    const int32_t *__restrict__ F, const int32_t *__restrict__ rseg,
    const int32_t *__restrict__ pstart, const uint8_t *__restrict__ pslot,
    const int64_t *__restrict__ woff, const int32_t *__restrict__ tile_row,
    uint32_t *__restrict__ masks, int32_t *__restrict__ tile_cnt,
    unsigned long long *__restrict__ counts, uint32_t *__restrict__ fmasks,
    int32_t *__restrict__ ftile_cnt) {
  static_assert(kItemsPerThread == 4, "one 4-bit group per lane");
  extern __shared__ int32_t s_woff[];
  __shared__ int32_t s_count, s_fcount;
  const int32_t R = (int32_t)state[i].R;
  const int32_t W = (int32_t)state[i].W;
  const int64_t tiles = state[i].tiles;
  const int32_t B = blockDim.x;
  const int32_t tile_items = B * kItemsPerThread;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    if (threadIdx.x == 0) s_count = s_fcount = 0;
    const BTile b = b_stage(woff, tile_row, t, tile_items, s_woff);
    const int32_t x0 = (int32_t)t * tile_items, x1 = min(x0 + tile_items, W);
    const int32_t xb = x0 + warp * 128 + lane * kItemsPerThread;
    uint32_t bits = 0, fbits = 0;
    int32_t qj[kItemsPerThread] = {-1, -1, -1, -1};  // query of a last-level survivor
    if (xb < x1) {
      int32_t rs;
      int32_t r = b_row(b, s_woff, woff, xb, &rs);
      int32_t rr = r - b.r0;
      int32_t re = b.staged ? s_woff[rr + 1] : (int32_t)woff[r + 1];
      int32_t q = rseg[r], pst = pstart[r], slot = pslot[r];
#pragma unroll
      for (int j = 0; j < kItemsPerThread; ++j) {
        const int32_t x = xb + j;
        if (x >= x1) break;
        while (x >= re) {
          ++rr;
          ++r;
          rs = re;
          re = b.staged ? s_woff[rr + 1] : (int32_t)woff[r + 1];
          q = rseg[r];
          pst = pstart[r];
          slot = pslot[r];
        }
        const BatchLevel &L = qs[q].lv[i];
        const int32_t w = __ldg(g.lcol + pst + (x - rs));
        if (check_candidate(g, L, ColumnRow{F, R, r}, w, slot)) {
          if (L.last) {
            qj[j] = q;
            if (fmasks && qs[q].enumerate) fbits |= 1u << j;
          } else {
            bits |= 1u << j;
          }
        }
      }
    }
    // last-level survivors: one atomic per query per warp and item slot
    // (a warp's rows mostly belong to one query: ballots settle that case,
    // match_any only a warp that straddles queries)
#pragma unroll
    for (int j = 0; j < kItemsPerThread; ++j) {
      const uint32_t has = __ballot_sync(kFull, qj[j] >= 0);
      if (!has) continue;
      const int first = __ffs(has) - 1;
      const int32_t qa = __shfl_sync(kFull, qj[j], first);
      if (__ballot_sync(kFull, qj[j] == qa) == has) {
        if (lane == first) atomicAdd(counts + qa, (unsigned long long)__popc(has));
      } else {
        const uint32_t peers = __match_any_sync(kFull, qj[j]);
        if (qj[j] >= 0 && lane == __ffs(peers) - 1)
          atomicAdd(counts + qj[j], (unsigned long long)__popc(peers));
      }
    }
    uint32_t word = bits << (4 * (lane & 7));
    word |= __shfl_xor_sync(kFull, word, 1);
    word |= __shfl_xor_sync(kFull, word, 2);
    word |= __shfl_xor_sync(kFull, word, 4);
    int32_t cnt = 0;
    if ((lane & 7) == 0) {
      masks[(x0 + warp * 128) / 32 + (lane >> 3)] = word;
      cnt = __popc(word);
    }
    cnt = __reduce_add_sync(kFull, cnt);
    if (lane == 0 && cnt) atomicAdd(&s_count, cnt);
    if (fmasks) {
      uint32_t fw = fbits << (4 * (lane & 7));
      fw |= __shfl_xor_sync(kFull, fw, 1);
      fw |= __shfl_xor_sync(kFull, fw, 2);
      fw |= __shfl_xor_sync(kFull, fw, 4);
      int32_t fc = 0;
      if ((lane & 7) == 0) {
        fmasks[(x0 + warp * 128) / 32 + (lane >> 3)] = fw;
        fc = __popc(fw);
      }
      fc = __reduce_add_sync(kFull, fc);
      if (lane == 0 && fc) atomicAdd(&s_fcount, fc);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      tile_cnt[t] = s_count;
      if (ftile_cnt) ftile_cnt[t] = s_fcount;
    }
    __syncthreads();
  }
}

// Survivors S = tile_off[tiles]; the next level gets them unless they exceed
// the frontier capacity.
__global__ void k_b_advance(int32_t i, BatchStep *state, const int64_t *__restrict__ tile_off,
                            int64_t cap_rows, int64_t cap_elems, int32_t *overflow) {
  const int64_t tiles = state[i].tiles;
  const int64_t S = tiles > 0 ? tile_off[tiles] : 0;
  state[i].S = S;
  if (S > cap_rows || S * (i + 1) > cap_elems) {
    *overflow = 1;
    state[i + 1].R = 0;
  } else {
    state[i + 1].R = S;
  }
}

__device__ __forceinline__ int b_nth_bit(uint32_t m, int n) {
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

__global__ void __launch_bounds__(1024) k_b_write(
    GraphDev g, int32_t i, const BatchStep *state, const int32_t *__restrict__ F,
    const int32_t *__restrict__ rseg, const int32_t *__restrict__ pstart,
    const int64_t *__restrict__ woff, const int32_t *__restrict__ tile_row,
    const uint32_t *__restrict__ masks, const int64_t *__restrict__ tile_off,
    int32_t *__restrict__ Fn, int32_t *__restrict__ rseg_n) {
  extern __shared__ int32_t s_woff[];
  __shared__ uint32_t s_mask[kItemsPerThread * 1024 / 32];
  __shared__ int32_t s_wpre[kItemsPerThread * 1024 / 32];
  const int32_t R = (int32_t)state[i].R;
  const int64_t tiles = state[i].tiles;
  const int64_t S = state[i + 1].R;
  if (S == 0 || S != state[i].S) return;  // nothing survives, or overflow
  const int32_t B = blockDim.x;
  const int32_t tile_items = B * kItemsPerThread;
  const int32_t tile_words = tile_items / 32;
  const int lane = threadIdx.x & 31;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t base = tile_off[t];
    const int32_t cnt = (int32_t)(tile_off[t + 1] - base);
    if (cnt == 0) continue;  // uniform across the block
    for (int32_t w = threadIdx.x; w < tile_words; w += B) s_mask[w] = masks[t * tile_words + w];
    const BTile b = b_stage(woff, tile_row, t, tile_items, s_woff);
    if (threadIdx.x < 32) {
      int32_t carry = 0;
      for (int32_t c = 0; c < tile_words; c += 32) {
        const int32_t idx = c + lane;
        const int32_t v = idx < tile_words ? __popc(s_mask[idx]) : 0;
        int32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        if (idx < tile_words) s_wpre[idx] = carry + incl - v;
        carry += __shfl_sync(kFull, incl, 31);
      }
    }
    __syncthreads();
    const int32_t x0 = (int32_t)t * tile_items;
    for (int32_t q = threadIdx.x; q < cnt; q += B) {
      int32_t lo = 0, hi = tile_words;
      while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (s_wpre[mid] <= q) lo = mid; else hi = mid;
      }
      const int32_t x = x0 + lo * 32 + b_nth_bit(s_mask[lo], q - s_wpre[lo]);
      int32_t rs;
      const int32_t r = b_row(b, s_woff, woff, x, &rs);
      const int32_t w = __ldg(g.lcol + pstart[r] + (x - rs));
      const int64_t pos = base + q;
      for (int c = 0; c < i; ++c) Fn[c * S + pos] = F[c * R + r];
      Fn[i * S + pos] = w;
      rseg_n[pos] = rseg[r];
    }
    __syncthreads();
  }
}

// Result rows of step i: FS = ftile_off[tiles]; they take arena elements
// [FB, FB + FS*(i+1)) and the next step's rows start after them.  Over the
// arena's capacity: overflow, and no row is written.
__global__ void k_b_fadvance(int32_t i, BatchStep *state, const int64_t *__restrict__ ftile_off,
                             int64_t cap_final, int32_t *overflow) {
  const int64_t tiles = state[i].tiles;
  const int64_t FS = tiles > 0 ? ftile_off[tiles] : 0;
  const int64_t FB = state[i].FB;
  if (FB + FS * (i + 1) > cap_final) {
    *overflow = 1;
    state[i].FS = 0;
    state[i + 1].FB = FB;
  } else {
    state[i].FS = FS;
    state[i + 1].FB = FB + FS * (i + 1);
  }
}

// Writes the result rows of step i: result survivor q of tile t becomes row
// ftile_off[t] + q of the step, row-major from arena element FB, position c
// of the frontier row going to column out_col[c] of its query (the new
// vertex to column out_col[i]).
__global__ void __launch_bounds__(1024) k_b_fwrite(
    GraphDev g, const BatchQuery *__restrict__ qs, int32_t i, const BatchStep *state,
    const int32_t *__restrict__ F, const int32_t *__restrict__ rseg,
    const int32_t *__restrict__ pstart, const int64_t *__restrict__ woff,
    const int32_t *__restrict__ tile_row, const uint32_t *__restrict__ fmasks,
    const int64_t *__restrict__ ftile_off, int32_t *__restrict__ final_rows) {
  extern __shared__ int32_t s_woff[];
  __shared__ uint32_t s_mask[kItemsPerThread * 1024 / 32];
  __shared__ int32_t s_wpre[kItemsPerThread * 1024 / 32];
  const int32_t R = (int32_t)state[i].R;
  const int64_t tiles = state[i].tiles;
  const int64_t FS = state[i].FS, FB = state[i].FB;
  if (FS == 0) return;  // nothing to write, or over capacity
  const int32_t B = blockDim.x;
  const int32_t tile_items = B * kItemsPerThread;
  const int32_t tile_words = tile_items / 32;
  const int lane = threadIdx.x & 31;
  const int32_t width = i + 1;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t base = ftile_off[t];
    const int32_t cnt = (int32_t)(ftile_off[t + 1] - base);
    if (cnt == 0) continue;  // uniform across the block
    for (int32_t w = threadIdx.x; w < tile_words; w += B) s_mask[w] = fmasks[t * tile_words + w];
    const BTile b = b_stage(woff, tile_row, t, tile_items, s_woff);
    if (threadIdx.x < 32) {
      int32_t carry = 0;
      for (int32_t c = 0; c < tile_words; c += 32) {
        const int32_t idx = c + lane;
        const int32_t v = idx < tile_words ? __popc(s_mask[idx]) : 0;
        int32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        if (idx < tile_words) s_wpre[idx] = carry + incl - v;
        carry += __shfl_sync(kFull, incl, 31);
      }
    }
    __syncthreads();
    const int32_t x0 = (int32_t)t * tile_items;
    for (int32_t q = threadIdx.x; q < cnt; q += B) {
      int32_t lo = 0, hi = tile_words;
      while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (s_wpre[mid] <= q) lo = mid; else hi = mid;
      }
      const int32_t x = x0 + lo * 32 + b_nth_bit(s_mask[lo], q - s_wpre[lo]);
      int32_t rs;
      const int32_t r = b_row(b, s_woff, woff, x, &rs);
      const int32_t w = __ldg(g.lcol + pstart[r] + (x - rs));
      const int32_t *oc = qs[rseg[r]].out_col;
      int32_t *dst = final_rows + FB + (base + q) * width;
      for (int c = 0; c < i; ++c) dst[oc[c]] = F[c * R + r];
      dst[oc[i]] = w;
    }
    __syncthreads();
  }
}

// Address of a field of state[i] (device memory; no host access).
const int64_t *step_field(const BatchStep *state, int32_t i, size_t off) {
  return reinterpret_cast<const int64_t *>(reinterpret_cast<const char *>(state) +
                                           (size_t)i * sizeof(BatchStep) + off);
}

template <typename T>
void pscan(const T *in, const int64_t *n_ptr, int64_t *out, int64_t *partials, int32_t G,
           cudaStream_t s) {
  k_pscan_reduce<T><<<G, kPScanThreads, 0, s>>>(in, n_ptr, partials);
  k_pscan_top<<<1, 1024, 0, s>>>(partials, G);
  k_pscan_down<T><<<G, kPScanThreads, 0, s>>>(in, n_ptr, partials, out);
}

}  // namespace

void launch_filter_many(const GraphDev &g, const FilterDesc *fds, uint32_t *const *bm_out,
                        unsigned long long *sizes, int32_t nq, int32_t n_words,
                        cudaStream_t s) {
  if (nq <= 0) return;
  cudaMemsetAsync(sizes, 0, sizeof(unsigned long long) * nq * kMaxK, s);
  const int gx = (int)std::min<int64_t>((n_words + 7) / 8, 128);
  k_b_filter<<<dim3(std::max(gx, 1), nq), 256, 0, s>>>(g, fds, bm_out, sizes);
}

int batch_enqueue(const GraphDev &g, const BatchArgs &a, cudaStream_t s) {
  const int32_t B = a.block, G = a.grid;
  const int32_t tile_items = B * kItemsPerThread;
  const size_t smem = (size_t)(tile_items + 1) * sizeof(int32_t);
  int launches = 0;
  cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * a.nq, s);
  cudaMemsetAsync(a.sizes, 0, sizeof(unsigned long long) * a.nq * kMaxK, s);
  cudaMemsetAsync(a.overflow, 0, sizeof(int32_t), s);
  k_b_init<<<1, 32, 0, s>>>(a.state, (int64_t)a.nq * a.n_words);
  // filter: one CTA row per query
  const int gx = (int)std::min<int64_t>((a.n_words + 7) / 8, 128);
  k_b_filter<<<dim3(std::max(gx, 1), a.nq), 256, 0, s>>>(g, a.fds, a.bm_out, a.sizes);
  ++launches;
  // level 1: every query's candidate list for its first matched vertex
  k_b_list_popc<<<G, 256, 0, s>>>(a.qs, a.nq, a.n_words, a.wcnt, a.counts);
  pscan<int32_t>(a.wcnt, step_field(a.state, 0, offsetof(BatchStep, W)), a.woffs, a.partials,
                 G, s);
  k_b_list_check<<<1, 1, 0, s>>>(a.woffs, (int64_t)a.nq * a.n_words, a.state,
                                 std::min(a.cap_rows, a.cap_elems), a.overflow);
  k_b_list_emit<<<G, 256, 0, s>>>(a.qs, a.nq, a.n_words, a.woffs, a.state, a.F[0], a.rseg[0]);
  launches += 7;
  for (int32_t i = 1; i < a.kmax; ++i) {
    const int cur = (i - 1) & 1, nxt = i & 1;
    k_b_pivot<<<G, 256, 0, s>>>(g, a.qs, i, a.state, a.F[cur], a.rseg[cur], a.pstart, a.pslot,
                                a.woff);
    pscan<int64_t>(a.woff, step_field(a.state, i, offsetof(BatchStep, R)), a.woff, a.partials,
                   G, s);
    k_b_check_work<<<1, 1, 0, s>>>(i, a.state, a.woff, a.cap_items, tile_items, a.overflow);
    k_b_tile_rows<<<G, 256, 0, s>>>(i, a.state, a.woff, tile_items, a.tile_row);
    k_b_count<<<G, B, smem, s>>>(g, a.qs, i, a.state, a.F[cur], a.rseg[cur], a.pstart, a.pslot,
                                 a.woff, a.tile_row, a.masks, a.tile_cnt, a.counts,
                                 a.enumerate ? a.fmasks : nullptr,
                                 a.enumerate ? a.ftile_cnt : nullptr);
    pscan<int32_t>(a.tile_cnt, step_field(a.state, i, offsetof(BatchStep, tiles)), a.tile_off,
                   a.partials, G, s);
    k_b_advance<<<1, 1, 0, s>>>(i, a.state, a.tile_off, a.cap_rows, a.cap_elems, a.overflow);
    k_b_write<<<G, B, smem, s>>>(g, i, a.state, a.F[cur], a.rseg[cur], a.pstart, a.woff,
                                 a.tile_row, a.masks, a.tile_off, a.F[nxt], a.rseg[nxt]);
    launches += 12;
    if (a.enumerate) {
      pscan<int32_t>(a.ftile_cnt, step_field(a.state, i, offsetof(BatchStep, tiles)),
                     a.ftile_off, a.partials, G, s);
      k_b_fadvance<<<1, 1, 0, s>>>(i, a.state, a.ftile_off, a.cap_final, a.overflow);
      k_b_fwrite<<<G, B, smem, s>>>(g, a.qs, i, a.state, a.F[cur], a.rseg[cur], a.pstart, a.woff,
                                    a.tile_row, a.fmasks, a.ftile_off, a.final_rows);
      launches += 5;
    }
  }
  return launches;
}

}  // namespace gsm
