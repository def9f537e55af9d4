// Compressed frontiers (see compressed.cuh): the pivot and single-pass level
// kernels for rows kept as (parent row, new vertex).  A row of width i is
// decoded by i-1 dependent loads through the parent indices; the candidate
// check, ranking, look-back and result writes are those of the
// column-frontier kernels (verify.cuh).
#include <climits>

#include "compressed.cuh"
#include "segments.cuh"
#include "verify.cuh"

namespace gsm {
namespace {

// Positions 0..i-1 of row r of the width-i frontier of f.
__device__ __forceinline__ void decode_row(const CFrontier &f, int32_t i, int32_t r,
                                           int32_t *vals) {
  for (int32_t j = i; j >= 1; --j) {
    vals[j - 1] = __ldg(f.V[j] + r);
    if (j > 1) r = __ldg(f.P[j] + r);
  }
}

struct ArrayRow {
  const int32_t *v;
  __device__ __forceinline__ int32_t operator()(int c) const { return v[c]; }
};

__global__ void k_cpivot(GraphDev g, LevelDesc d, CFrontier f, int32_t i, int64_t R,
                         int32_t *__restrict__ pstart, uint8_t *__restrict__ pslot,
                         int64_t *__restrict__ work) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int32_t vals[kMaxK];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += stride) {
    decode_row(f, i, (int32_t)r, vals);
    int32_t best = INT_MAX, best_start = 0, best_slot = 0;
    for (int b = 0; b < d.nb; ++b) {
      const int2 seg = label_segment(g, vals[d.bpos[b]], d.lab);
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

// Tiles, candidate order and survivor order as k_extend_fused; the row of a
// candidate is decoded once per thread and row change.
template <int kMode>
__global__ void __launch_bounds__(1024) k_cextend(
    GraphDev g, LevelDesc d, CFrontier f, int32_t i, const int32_t *__restrict__ pstart,
    const uint8_t *__restrict__ pslot, const int64_t *__restrict__ woff,
    const int32_t *__restrict__ tile_row, int64_t wa, int32_t W, int32_t tiles,
    unsigned long long *__restrict__ lookback, CSink sink, int32_t spin_limit) {
  static_assert(kItemsPerThread == 4, "four candidates per thread");
  extern __shared__ int32_t s_woff[];
  __shared__ int32_t s_tile;
  __shared__ int32_t s_warp[33];
  __shared__ long long s_prefix;
  if (threadIdx.x == 0) s_tile = (int32_t)atomicAdd(lookback + tiles, 1ull);
  __syncthreads();
  const int32_t tile = s_tile;
  const int32_t B = blockDim.x;
  const int32_t tile_items = B * kItemsPerThread;
  const int32_t x0 = tile * tile_items;
  const int32_t x1 = min(x0 + tile_items, W);
  const TileRows t = stage_rows(woff, tile_row, wa, tile_items, s_woff, tile);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t xb = x0 + warp * 128 + lane * kItemsPerThread;
  uint32_t bits = 0;
  int32_t rj[kItemsPerThread], wj[kItemsPerThread];
  int32_t vals[kMaxK];
  if (xb < x1) {
    int32_t rs;
    int32_t r = item_row(t, s_woff, woff, wa, xb, &rs);
    int32_t rr = r - t.r0;
    int32_t re = t.staged ? s_woff[rr + 1] : (int32_t)(woff[r + 1] - wa);
    int32_t pst = pstart[r], slot = pslot[r];
    decode_row(f, i, r, vals);
#pragma unroll
    for (int j = 0; j < kItemsPerThread; ++j) {
      rj[j] = r;
      wj[j] = 0;
      const int32_t x = xb + j;
      if (x >= x1) continue;
      if (x >= re) {
        while (x >= re) {  // next row (rows without work are skipped)
          ++rr;
          ++r;
          rs = re;
          re = t.staged ? s_woff[rr + 1] : (int32_t)(woff[r + 1] - wa);
        }
        pst = pstart[r];
        slot = pslot[r];
        decode_row(f, i, r, vals);
      }
      const int32_t w = __ldg(g.lcol + pst + (x - rs));
      rj[j] = r;
      wj[j] = w;
      if (check_candidate(g, d, ArrayRow{vals}, w, slot) &&
          (!d.la || lookahead_ok(g, d, ArrayRow{vals}, w)))
        bits |= 1u << j;
    }
  }
  const int32_t c = __popc(bits);
  int32_t T;
  const int32_t rank = block_rank(c, s_warp, &T);
  if (kMode == kCSinkCount) {
    if (threadIdx.x == 0 && T) atomicAdd(sink.total, (unsigned long long)T);
    return;
  }
  {
    int32_t *s_pair = s_woff;
    int32_t q = rank;
#pragma unroll
    for (int j = 0; j < kItemsPerThread; ++j)
      if ((bits >> j) & 1u) {
        s_pair[2 * q] = rj[j];
        s_pair[2 * q + 1] = wj[j];
        ++q;
      }
  }
  if (warp == 0) {
    const unsigned long long prefix = lookback_prefix(lookback, tile, tiles, T, lane, spin_limit);
    if (lane == 0) s_prefix = (long long)prefix;
  }
  __syncthreads();
  for (int32_t q = threadIdx.x; q < T; q += B) {
    const int32_t r = s_woff[2 * q], w = s_woff[2 * q + 1];
    if (kMode == kCSinkPairs) {
      const int64_t row = sink.row0 + s_prefix + q;
      sink.pn[row] = r;
      sink.vn[row] = w;
    } else {
      decode_row(f, i, r, vals);
      constexpr int kRowMode = kMode == kCSinkRows ? kSinkRows : kSinkKeys;
      put_row<kRowMode>(sink.rows, d, ArrayRow{vals}, w, sink.rows.row0 + s_prefix + q);
    }
  }
}

inline int grid_rows(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (int)b;
}

}  // namespace

void launch_cpivot(const GraphDev &g, const LevelDesc &d, const CFrontier &f, int32_t i,
                   int64_t R, int32_t *pstart, uint8_t *pslot, int64_t *work, cudaStream_t s) {
  if (R <= 0) return;
  k_cpivot<<<grid_rows(R), 256, 0, s>>>(g, d, f, i, R, pstart, pslot, work);
}

void launch_cextend(const GraphDev &g, const LevelDesc &d, const CFrontier &f, int32_t i,
                    const int32_t *pstart, const uint8_t *pslot, const int64_t *woff,
                    const int32_t *tile_row, int64_t wa, int64_t wb, int32_t block,
                    unsigned long long *lookback, const CSink &sink, int32_t spin_limit,
                    cudaStream_t s) {
  const int64_t tiles = extend_tiles(wa, wb, block);
  if (tiles <= 0) return;
  // the staged work offsets, later the survivor pairs (2 ints per item)
  const size_t smem = (size_t)((int64_t)block * kItemsPerThread * 2 + 1) * sizeof(int32_t);
  const int32_t W = (int32_t)(wb - wa), T = (int32_t)tiles;
  switch (sink.mode) {
    case kCSinkPairs:
      k_cextend<kCSinkPairs><<<(unsigned)tiles, block, smem, s>>>(
          g, d, f, i, pstart, pslot, woff, tile_row, wa, W, T, lookback, sink, spin_limit);
      break;
    case kCSinkRows:
      k_cextend<kCSinkRows><<<(unsigned)tiles, block, smem, s>>>(
          g, d, f, i, pstart, pslot, woff, tile_row, wa, W, T, lookback, sink, spin_limit);
      break;
    case kCSinkKeys:
      k_cextend<kCSinkKeys><<<(unsigned)tiles, block, smem, s>>>(
          g, d, f, i, pstart, pslot, woff, tile_row, wa, W, T, lookback, sink, spin_limit);
      break;
    default:
      k_cextend<kCSinkCount><<<(unsigned)tiles, block, smem, s>>>(
          g, d, f, i, pstart, pslot, woff, tile_row, wa, W, T, lookback, sink, spin_limit);
      break;
  }
}

}  // namespace gsm
