// Output canonicalisation: lexicographic sort of the final embedding rows.
//
// The verification levels emit rows in matching order; the library returns
// them in query-vertex-id order, sorted lexicographically, so the result is
// independent of the order the planner picked.  This is a least-significant-
// digit radix sort over 8-bit digits that moves whole rows (k int32 each):
// columns are processed from the last to the first, low digit to high digit,
// and every pass is stable, so after the last pass the rows are ordered by
// column 0, then column 1, and so on.  Rows arrive column-major (the layout
// of the frontiers); intermediate passes keep that layout, the last pass
// writes row-major, the layout of the result.
#include <utility>

#include "kernels.cuh"

namespace gsm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSortThreads = 256;
constexpr int kSortChunks = 8;  // rows per CTA = 256 * 8
constexpr int kSortTile = kSortThreads * kSortChunks;
constexpr int kBins = 256;

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const int32_t *__restrict__ col_in,
                                                            int64_t N,
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
      const uint32_t dgt = ((uint32_t)col_in[idx] >> shift) & 0xffu;
      atomicAdd(&s_hist[dgt], 1);
    }
  }
  __syncthreads();
  // digit-major layout, so one exclusive scan gives every (digit, block) its
  // global output offset
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_hist[threadIdx.x];
}

// One stable pass: row idx moves to hist_off[digit][block] + (rank among the
// block's earlier rows with that digit).  Input column-major (ld_in); output
// column-major (ld_out) or, for the last pass, row-major.
template <bool kRowOut>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(
    const int32_t *__restrict__ in, int64_t ld_in, int32_t *__restrict__ out, int64_t ld_out,
    int64_t N, int32_t k, int32_t col, int32_t shift, const int64_t *__restrict__ hist_off,
    int64_t nblocks) {
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
    const uint32_t dgt =
        valid ? ((uint32_t)in[(int64_t)col * ld_in + idx] >> shift) & 0xffu : kBins;
    const uint32_t peers = __match_any_sync(kFull, dgt);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) s_wcnt[warp][dgt] = __popc(peers);
    __syncthreads();
    if (valid) {
      int64_t pos = s_base[dgt] + rank;
      for (int w = 0; w < warp; ++w) pos += s_wcnt[w][dgt];
      for (int j = 0; j < k; ++j) {
        const int32_t v = in[(int64_t)j * ld_in + idx];
        if (kRowOut)
          out[pos * k + j] = v;
        else
          out[(int64_t)j * ld_out + pos] = v;
      }
    }
    __syncthreads();
    int32_t add = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) add += s_wcnt[w][threadIdx.x];
    s_base[threadIdx.x] += add;
    __syncthreads();
  }
}

// Column-major -> row-major through a shared-memory tile of 256 rows: each
// column is read with contiguous loads, and the tile's k*256 output ints,
// which are contiguous in the result, are written with contiguous stores.
__global__ void __launch_bounds__(256) k_transpose_rows(const int32_t *__restrict__ in,
                                                        int64_t ld, int32_t *__restrict__ out,
                                                        int64_t N, int32_t k) {
  __shared__ int32_t s_tile[256 * (kMaxK + 1)];
  const int64_t r0 = (int64_t)blockIdx.x * 256;
  const int32_t rows = (int32_t)min((int64_t)256, N - r0);
  const int32_t w = k + 1;  // padded row pitch: conflict-free column writes
  for (int32_t c = 0; c < k; ++c)
    if ((int32_t)threadIdx.x < rows)
      s_tile[threadIdx.x * w + c] = in[(int64_t)c * ld + r0 + threadIdx.x];
  __syncthreads();
  int32_t *dst = out + r0 * k;
  for (int32_t e = threadIdx.x; e < rows * k; e += blockDim.x) {
    const int32_t rr = e / k, c = e - rr * k;
    dst[e] = s_tile[rr * w + c];
  }
}

// ---- packed keys: row (c_0, ..., c_{k-1}) becomes the K = k*b-bit integer
// sum_j c_j << ((k-1-j)*b), held as nw little-endian 64-bit words (word 0 =
// least significant); ordering these integers is ordering the rows.  Words
// are column-major (word w of row r at keys[w*N + r]).

constexpr int kMaxWords = 8;  // 16 columns x 31 bits < 512

__global__ void __launch_bounds__(256) k_pack_keys(const int32_t *__restrict__ in, int64_t ld,
                                                   int64_t N, int32_t k, int32_t b, int32_t nw,
                                                   uint64_t *__restrict__ keys) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  uint64_t w[kMaxWords];
#pragma unroll
  for (int i = 0; i < kMaxWords; ++i) w[i] = 0;
  for (int32_t j = 0; j < k; ++j) {
    const uint64_t v = (uint32_t)in[(int64_t)j * ld + r];
    const int32_t pos = (k - 1 - j) * b;  // bit offset of column j
    const int32_t wi = pos >> 6, sh = pos & 63;
#pragma unroll
    for (int i = 0; i < kMaxWords; ++i) {
      if (i == wi) w[i] |= v << sh;
      if (i == wi + 1 && sh + b > 64) w[i] |= v >> (64 - sh);
    }
  }
#pragma unroll
  for (int i = 0; i < kMaxWords; ++i)
    if (i < nw) keys[(int64_t)i * N + r] = w[i];
}

__global__ void __launch_bounds__(kSortThreads) k_hist_keys(const uint64_t *__restrict__ word,
                                                            int64_t N, int32_t shift,
                                                            int32_t *__restrict__ hist,
                                                            int64_t nblocks) {
  __shared__ int32_t s_hist[kBins];
  s_hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
  for (int c = 0; c < kSortChunks; ++c) {
    const int64_t idx = base + c * kSortThreads + threadIdx.x;
    if (idx < N) atomicAdd(&s_hist[(word[idx] >> shift) & 0xffu], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_hist[threadIdx.x];
}

// One stable pass over packed keys; the last pass unpacks each key into a
// row-major int32 row of `out` instead of moving the key.
template <bool kUnpack>
__global__ void __launch_bounds__(kSortThreads) k_scatter_keys(
    const uint64_t *__restrict__ in, uint64_t *__restrict__ out_keys,
    int32_t *__restrict__ out_rows, int64_t N, int32_t nw, int32_t k, int32_t b, int32_t dword,
    int32_t shift, const int64_t *__restrict__ hist_off, int64_t nblocks) {
  __shared__ int64_t s_base[kBins];
  __shared__ int32_t s_wcnt[kSortThreads / 32][kBins + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s_base[threadIdx.x] = hist_off[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  const uint32_t lt = (1u << lane) - 1u;
  const uint64_t mask_b = (b >= 64) ? ~0ull : ((1ull << b) - 1ull);
  for (int c = 0; c < kSortChunks; ++c) {
    for (int w = 0; w < kSortThreads / 32; ++w) s_wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t idx = base + c * kSortThreads + threadIdx.x;
    const bool valid = idx < N;
    const uint32_t dgt =
        valid ? (uint32_t)((in[(int64_t)dword * N + idx] >> shift) & 0xffu) : kBins;
    const uint32_t peers = __match_any_sync(kFull, dgt);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) s_wcnt[warp][dgt] = __popc(peers);
    __syncthreads();
    if (valid) {
      int64_t pos = s_base[dgt] + rank;
      for (int w = 0; w < warp; ++w) pos += s_wcnt[w][dgt];
      if (kUnpack) {
        uint64_t wv[kMaxWords];
#pragma unroll
        for (int i = 0; i < kMaxWords; ++i) wv[i] = i < nw ? in[(int64_t)i * N + idx] : 0;
        int32_t *dst = out_rows + pos * k;
        for (int32_t j = 0; j < k; ++j) {
          const int32_t bp = (k - 1 - j) * b;
          const int32_t wi = bp >> 6, sh = bp & 63;
          uint64_t v = 0;
#pragma unroll
          for (int i = 0; i < kMaxWords; ++i) {
            if (i == wi) v |= wv[i] >> sh;
            if (i == wi + 1 && sh + b > 64) v |= wv[i] << (64 - sh);
          }
          dst[j] = (int32_t)(v & mask_b);
        }
      } else {
        for (int32_t i = 0; i < nw; ++i) out_keys[(int64_t)i * N + pos] = in[(int64_t)i * N + idx];
      }
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

int launch_sort_rows(int32_t *a, int64_t lda, int32_t *b, int64_t ldb, int64_t N, int32_t k,
                     int32_t bits, bool presorted, int32_t *hist, int64_t *hist_off, int64_t *tmp,
                     cudaStream_t s, int *launches) {
  if (N <= 0) return 0;
  if (presorted || N == 1) {
    k_transpose_rows<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(a, lda, b, N, k);
    if (launches) *launches += 1;
    return 1;
  }
  const int64_t nb = (N + kSortTile - 1) / kSortTile;
  const int passes_per_col = (bits + 7) / 8;
  const int total = k * passes_per_col;
  int32_t *src = a, *dst = b;
  int64_t ld_src = lda, ld_dst = ldb;
  int which = 0;
  int pass = 0;
  for (int32_t col = k - 1; col >= 0; --col) {
    for (int32_t shift = 0; shift < bits; shift += 8) {
      ++pass;
      k_sort_hist<<<(unsigned)nb, kSortThreads, 0, s>>>(src + (int64_t)col * ld_src, N, shift,
                                                        hist, nb);
      launch_scan_i32(hist, hist_off, nb * kBins, tmp, s);
      if (pass == total)
        k_sort_scatter<true><<<(unsigned)nb, kSortThreads, 0, s>>>(
            src, ld_src, dst, ld_dst, N, k, col, shift, hist_off, nb);
      else
        k_sort_scatter<false><<<(unsigned)nb, kSortThreads, 0, s>>>(
            src, ld_src, dst, ld_dst, N, k, col, shift, hist_off, nb);
      if (launches) *launches += 5;
      std::swap(src, dst);
      std::swap(ld_src, ld_dst);
      which ^= 1;
    }
  }
  return which;
}

}  // namespace gsm

namespace gsm {

int32_t packed_words(int32_t k, int32_t bits) { return (k * bits + 63) / 64; }

int launch_sort_rows_packed(const int32_t *a, int64_t lda, int64_t N, int32_t k, int32_t bits,
                            uint64_t *keys_a, uint64_t *keys_b, int32_t *out, int32_t *hist,
                            int64_t *hist_off, int64_t *tmp, cudaStream_t s) {
  if (N <= 0) return 0;
  int launches = 0;
  const int32_t nw = packed_words(k, bits);
  k_pack_keys<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(a, lda, N, k, bits, nw, keys_a);
  ++launches;
  const int64_t nb = (N + kSortTile - 1) / kSortTile;
  const int32_t digits = (k * bits + 7) / 8;
  uint64_t *src = keys_a, *dst = keys_b;
  for (int32_t dg = 0; dg < digits; ++dg) {
    const int32_t dword = (dg * 8) >> 6, shift = (dg * 8) & 63;
    k_hist_keys<<<(unsigned)nb, kSortThreads, 0, s>>>(src + (int64_t)dword * N, N, shift, hist, nb);
    launch_scan_i32(hist, hist_off, nb * kBins, tmp, s);
    if (dg == digits - 1)
      k_scatter_keys<true><<<(unsigned)nb, kSortThreads, 0, s>>>(
          src, dst, out, N, nw, k, bits, dword, shift, hist_off, nb);
    else
      k_scatter_keys<false><<<(unsigned)nb, kSortThreads, 0, s>>>(
          src, dst, out, N, nw, k, bits, dword, shift, hist_off, nb);
    launches += 5;
    std::swap(src, dst);
  }
  return launches;
}

}  // namespace gsm
