// Output canonicalisation: lexicographic sort of the final embedding rows.
//
// The verification levels emit rows in matching order; the library returns
// them in query-vertex-id order, sorted lexicographically, so the result is
// independent of the order the planner picked.  This is a least-significant-
// digit radix sort over 8-bit digits that moves whole rows (k int32 each):
// columns are processed from the last to the first, low digit to high digit,
// and every pass is stable, so after the last pass the rows are ordered by
// column 0, then column 1, and so on.
#include "kernels.cuh"

namespace gsm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSortThreads = 256;
constexpr int kSortChunks = 8;  // rows per CTA = 256 * 8
constexpr int kSortTile = kSortThreads * kSortChunks;
constexpr int kBins = 256;

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const int32_t *__restrict__ rows,
                                                            int64_t N, int32_t k, int32_t col,
                                                            int32_t shift,
                                                            int32_t *__restrict__ hist,
                                                            int64_t nblocks) {
  __shared__ int32_t s_hist[kBins];
  s_hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
  for (int c = 0; c < kSortChunks; ++c) {
    const int64_t idx = base + c * kSortThreads + threadIdx.x;
    if (idx < N) {
      const uint32_t dgt = ((uint32_t)rows[idx * k + col] >> shift) & 0xffu;
      atomicAdd(&s_hist[dgt], 1);
    }
  }
  __syncthreads();
  // digit-major layout, so one exclusive scan gives every (digit, block) its
  // global output offset
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_hist[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(
    const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t N, int32_t k, int32_t col,
    int32_t shift, const int64_t *__restrict__ hist_off, int64_t nblocks) {
  __shared__ int64_t s_base[kBins];
  __shared__ int32_t s_wcnt[kSortThreads / 32][kBins + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s_base[threadIdx.x] = hist_off[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  const uint32_t lt = (1u << lane) - 1u;
  for (int c = 0; c < kSortChunks; ++c) {
    for (int w = 0; w < kSortThreads / 32; ++w) s_wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t idx = base + c * kSortThreads + threadIdx.x;
    const bool valid = idx < N;
    const uint32_t dgt = valid ? ((uint32_t)in[idx * k + col] >> shift) & 0xffu : kBins;
    const uint32_t peers = __match_any_sync(kFull, dgt);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) s_wcnt[warp][dgt] = __popc(peers);
    __syncthreads();
    if (valid) {
      int64_t pos = s_base[dgt] + rank;
      for (int w = 0; w < warp; ++w) pos += s_wcnt[w][dgt];
      const int32_t *src = in + idx * k;
      int32_t *dst = out + pos * k;
      for (int j = 0; j < k; ++j) dst[j] = src[j];
    }
    __syncthreads();
    int32_t add = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) add += s_wcnt[w][threadIdx.x];
    s_base[threadIdx.x] += add;
    __syncthreads();
  }
}

}  // namespace

int64_t sort_hist_elems(int64_t N) {
  const int64_t nb = (N + kSortTile - 1) / kSortTile;
  return nb * kBins;
}

int launch_sort_rows(int32_t *a, int32_t *b, int64_t N, int32_t k, int32_t bits, int32_t *hist,
                     int64_t *hist_off, int64_t *tmp, cudaStream_t s, int *launches) {
  if (N <= 1) return 0;
  const int64_t nb = (N + kSortTile - 1) / kSortTile;
  int32_t *src = a, *dst = b;
  int which = 0;
  for (int32_t col = k - 1; col >= 0; --col) {
    for (int32_t shift = 0; shift < bits; shift += 8) {
      k_sort_hist<<<(unsigned)nb, kSortThreads, 0, s>>>(src, N, k, col, shift, hist, nb);
      launch_scan_i32(hist, hist_off, nb * kBins, tmp, s);
      k_sort_scatter<<<(unsigned)nb, kSortThreads, 0, s>>>(src, dst, N, k, col, shift, hist_off,
                                                           nb);
      if (launches) *launches += 5;
      int32_t *t = src;
      src = dst;
      dst = t;
      which ^= 1;
    }
  }
  return which;
}

}  // namespace gsm
