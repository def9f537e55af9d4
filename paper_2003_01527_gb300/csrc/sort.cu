// Output canonicalisation: lexicographic sort of the final embedding rows.
//
// The verification levels emit rows in matching order; the library returns
// them in query-vertex-id order, sorted lexicographically, so the result is
// independent of the order the planner picked.  Row (c_0, ..., c_{k-1})
// becomes the k*b-bit integer sum_j c_j << ((k-1-j)*b), held as nw
// little-endian 64-bit words (word 0 = least significant); ordering these
// integers is ordering the rows.  A least-significant-digit radix sort over
// 8-bit digits of that integer, with stable passes, orders them; the last pass
// unpacks every key into a row-major int32 row, the layout of the result.
// Words are column-major (word w of row r at keys[w*ld + r]).
#include <algorithm>
#include <utility>

#include "kernels.cuh"

namespace gsm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSortThreads = 256;
constexpr int kSortChunks = 8;  // rows per CTA = 256 * 8
constexpr int kSortTile = kSortThreads * kSortChunks;
constexpr int kBins = 256;

constexpr int kMaxWords = kMaxKeyWords;

__global__ void __launch_bounds__(256) k_pack_keys(const int32_t *__restrict__ in, int64_t ld,
                                                   int64_t N, int32_t k, int32_t b, int32_t nw,
                                                   uint64_t *__restrict__ keys, int64_t kld) {
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
    if (i < nw) keys[(int64_t)i * kld + r] = w[i];
}

// Byte digit of the packed key at bit position p (a digit may straddle two
// words; bits above the key's width are zero).
__device__ __forceinline__ uint32_t key_digit(const uint64_t *__restrict__ in, int64_t ld,
                                              int64_t idx, int32_t nw, int32_t p) {
  const int32_t wi = p >> 6, sh = p & 63;
  uint64_t v = in[(int64_t)wi * ld + idx] >> sh;
  if (sh > 56 && wi + 1 < nw) v |= in[(int64_t)(wi + 1) * ld + idx] << (64 - sh);
  return (uint32_t)(v & 0xffu);
}

__global__ void __launch_bounds__(kSortThreads) k_hist_keys(const uint64_t *__restrict__ in,
                                                            int64_t ld, int64_t N, int32_t nw,
                                                            int32_t p,
                                                            int32_t *__restrict__ hist,
                                                            int64_t nblocks) {
  __shared__ int32_t s_hist[kBins];
  s_hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
  for (int c = 0; c < kSortChunks; ++c) {
    const int64_t idx = base + c * kSortThreads + threadIdx.x;
    if (idx < N) atomicAdd(&s_hist[key_digit(in, ld, idx, nw, p)], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_hist[threadIdx.x];
}

// One stable pass over packed keys; the last pass unpacks each key into a
// row-major int32 row of `out` instead of moving the key.
template <bool kUnpack>
__global__ void __launch_bounds__(kSortThreads) k_scatter_keys(
    const uint64_t *__restrict__ in, uint64_t *__restrict__ out_keys,
    int32_t *__restrict__ out_rows, int64_t ld, int64_t N, int32_t nw, int32_t k, int32_t b,
    int32_t p, const int64_t *__restrict__ hist_off, int64_t nblocks) {
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
    const uint32_t dgt = valid ? key_digit(in, ld, idx, nw, p) : kBins;
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
        for (int i = 0; i < kMaxWords; ++i) wv[i] = i < nw ? in[(int64_t)i * ld + idx] : 0;
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
        for (int32_t i = 0; i < nw; ++i) out_keys[(int64_t)i * ld + pos] = in[(int64_t)i * ld + idx];
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

}  // namespace gsm

namespace gsm {

int32_t packed_words(int32_t k, int32_t bits) { return (k * bits + 63) / 64; }

int launch_sort_rows_packed(const int32_t *a, int64_t lda, int64_t N, int32_t k, int32_t bits,
                            int32_t sort_cols, uint64_t *keys_a, uint64_t *keys_b, int64_t ld,
                            int32_t *out, int32_t *hist, int64_t *hist_off, int64_t *tmp,
                            cudaStream_t s) {
  if (N <= 0) return 0;
  int launches = 0;
  const int32_t nw = packed_words(k, bits);
  if (a) {
    k_pack_keys<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(a, lda, N, k, bits, nw, keys_a, ld);
    ++launches;
  }
  const int64_t nb = (N + kSortTile - 1) / kSortTile;
  // only the bits of columns 0 .. sort_cols-1 are digits; the rest of the key
  // is carried along (its order is already right among equal prefixes)
  sort_cols = std::min(std::max(sort_cols, 1), k);
  const int32_t lo_bit = (k - sort_cols) * bits;
  const int32_t digits = (sort_cols * bits + 7) / 8;
  uint64_t *src = keys_a, *dst = keys_b;
  for (int32_t dg = 0; dg < digits; ++dg) {
    const int32_t p = lo_bit + 8 * dg;
    k_hist_keys<<<(unsigned)nb, kSortThreads, 0, s>>>(src, ld, N, nw, p, hist, nb);
    launch_scan_i32(hist, hist_off, nb * kBins, tmp, s);
    if (dg == digits - 1)
      k_scatter_keys<true><<<(unsigned)nb, kSortThreads, 0, s>>>(src, dst, out, ld, N, nw, k,
                                                                 bits, p, hist_off, nb);
    else
      k_scatter_keys<false><<<(unsigned)nb, kSortThreads, 0, s>>>(src, dst, out, ld, N, nw, k,
                                                                  bits, p, hist_off, nb);
    launches += 5;
    std::swap(src, dst);
  }
  return launches;
}

}  // namespace gsm
