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
#include <atomic>
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

// Column j of row r is in[j * cs + r * rs] (column-major: cs = ld, rs = 1;
// row-major: cs = 1, rs = k).
__global__ void __launch_bounds__(256) k_pack_keys(const int32_t *__restrict__ in, int64_t cs,
                                                   int64_t rs, int64_t N, int32_t k, int32_t b,
                                                   int32_t nw, uint64_t *__restrict__ keys,
                                                   int64_t kld) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  // word t collects the columns that overlap bits [64t, 64t+64)
  for (int32_t t = 0; t < nw; ++t) {
    uint64_t w = 0;
    for (int32_t j = 0; j < k; ++j) {
      const uint64_t v = (uint32_t)in[(int64_t)j * cs + r * rs];
      const int32_t lo = (k - 1 - j) * b - 64 * t;
      if (lo >= 0 && lo < 64)
        w |= v << lo;
      else if (lo < 0 && lo + b > 0)
        w |= v >> (-lo);
    }
    keys[(int64_t)t * kld + r] = w;
  }
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

// The same pass for keys of NW <= 2 words, a tile at a time: every thread
// first loads all its keys (item c*256 + t of the tile for chunk c), so the
// loads of a tile are in flight together; each warp then counts its digits
// per chunk with match_any into s_cnt[(chunk, warp)][digit], one exclusive
// scan per digit over the 64 (chunk, warp) entries turns the counts into tile
// offsets, and every key goes straight to hist_off + offset + rank.
template <int NW>
__device__ __forceinline__ uint32_t tile_digit(const uint64_t (&kk)[NW], int32_t wi, int32_t sh) {
  uint64_t lo = kk[0], hi = 0;
  if (NW > 1) {
    if (wi == 0) {
      hi = kk[NW - 1];
    } else {
      lo = kk[NW - 1];
    }
  }
  uint64_t v = lo >> sh;
  if (sh > 56) v |= hi << (64 - sh);
  return (uint32_t)(v & 0xffu);
}

template <int NW, bool kUnpack>
__global__ void __launch_bounds__(kSortThreads) k_scatter_tile(
    const uint64_t *__restrict__ in, uint64_t *__restrict__ out_keys,
    int32_t *__restrict__ out_rows, int64_t ld, int64_t N, int32_t k, int32_t b, int32_t p,
    const int64_t *__restrict__ hist_off, int64_t nblocks) {
  constexpr int kWarps = kSortThreads / 32;
  constexpr int kSlots = kSortChunks * kWarps;
  __shared__ __align__(16) uint16_t s_cnt[kSlots][kBins];
  __shared__ int64_t s_base[kBins];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  uint64_t key[kSortChunks][NW];
#pragma unroll
  for (int c = 0; c < kSortChunks; ++c) {
    const int64_t idx = base + c * kSortThreads + threadIdx.x;
#pragma unroll
    for (int w = 0; w < NW; ++w) key[c][w] = idx < N ? in[(int64_t)w * ld + idx] : 0;
  }
  s_base[threadIdx.x] = hist_off[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  {
    uint4 *z = reinterpret_cast<uint4 *>(&s_cnt[0][0]);
    constexpr int kVec = kSlots * kBins * 2 / 16;
    for (int e = threadIdx.x; e < kVec; e += kSortThreads) z[e] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  const int32_t wi = p >> 6, sh = p & 63;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t dg[kSortChunks];
  int32_t rk[kSortChunks];
#pragma unroll
  for (int c = 0; c < kSortChunks; ++c) {
    const bool valid = base + c * kSortThreads + threadIdx.x < N;
    dg[c] = valid ? tile_digit<NW>(key[c], wi, sh) : kBins;
    const uint32_t peers = __match_any_sync(kFull, dg[c]);
    rk[c] = __popc(peers & lt);
    if (valid && rk[c] == 0) s_cnt[c * kWarps + warp][dg[c]] = (uint16_t)__popc(peers);
  }
  __syncthreads();
  {
    int32_t run = 0;
    for (int e = 0; e < kSlots; ++e) {
      const int32_t v = s_cnt[e][threadIdx.x];
      s_cnt[e][threadIdx.x] = (uint16_t)run;
      run += v;
    }
  }
  __syncthreads();
  const uint64_t mask_b = (1ull << b) - 1ull;
#pragma unroll
  for (int c = 0; c < kSortChunks; ++c) {
    if (dg[c] == kBins) continue;
    const int64_t pos = s_base[dg[c]] + s_cnt[c * kWarps + warp][dg[c]] + rk[c];
    if (kUnpack) {
      int32_t *dst = out_rows + pos * k;
      for (int32_t j = 0; j < k; ++j) {
        const int32_t bp = (k - 1 - j) * b;
        const int32_t bw = bp >> 6, bs = bp & 63;
        uint64_t v = (NW > 1 && bw == 1) ? key[c][NW - 1] : key[c][0];
        v >>= bs;
        if (NW > 1 && bw == 0 && bs + b > 64) v |= key[c][NW - 1] << (64 - bs);
        dst[j] = (int32_t)(v & mask_b);
      }
    } else {
#pragma unroll
      for (int w = 0; w < NW; ++w) out_keys[(int64_t)w * ld + pos] = key[c][w];
    }
  }
}

// One CTA per item: `count` (<= kSmallSortRows) row-major rows of k int32 are
// loaded into shared memory and their indices bitonic-sorted by a
// lexicographic comparison of the rows (rows are distinct embeddings, so the
// order is total); then the rows are written in that order.  sort = 0: a
// plain copy (any count).
__device__ __forceinline__ bool row_less(const int32_t *s_rows, int32_t k, int32_t a, int32_t b) {
  if (a < 0) return false;  // padding sorts last
  if (b < 0) return true;
  const int32_t *x = s_rows + a * k, *y = s_rows + b * k;
  for (int32_t c = 0; c < k; ++c)
    if (x[c] != y[c]) return x[c] < y[c];
  return false;
}

__global__ void __launch_bounds__(256) k_sort_small(const SmallSortItem *__restrict__ items) {
  extern __shared__ int32_t s_mem[];
  const SmallSortItem it = items[blockIdx.x];
  const int32_t k = it.k, N = it.count;
  if (!it.sort || N <= 1) {
    const int64_t e_end = (int64_t)N * k;
    for (int64_t e = threadIdx.x; e < e_end; e += blockDim.x) it.dst[e] = it.src[e];
    return;
  }
  int32_t P = 1;
  while (P < N) P <<= 1;
  int32_t *s_idx = s_mem;       // P indices
  int32_t *s_rows = s_mem + P;  // N rows
  for (int32_t e = threadIdx.x; e < N * k; e += blockDim.x) s_rows[e] = it.src[e];
  for (int32_t e = threadIdx.x; e < P; e += blockDim.x) s_idx[e] = e < N ? e : -1;
  __syncthreads();
  for (int32_t size = 2; size <= P; size <<= 1) {
    for (int32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (int32_t t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
        const int32_t i = 2 * t - (t & (stride - 1));  // lower element of the pair
        const int32_t j = i + stride;
        const bool up = (i & size) == 0;
        const int32_t a = s_idx[i], b = s_idx[j];
        if (row_less(s_rows, k, b, a) == up) {
          s_idx[i] = b;
          s_idx[j] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int32_t e = threadIdx.x; e < N * k; e += blockDim.x) {
    const int32_t q = e / k, c = e - q * k;
    it.dst[e] = s_rows[s_idx[q] * k + c];
  }
}

}  // namespace

int64_t sort_hist_elems(int64_t N) {
  const int64_t nb = (N + kSortTile - 1) / kSortTile;
  return nb * kBins;
}

size_t small_sort_smem(int32_t max_k) {
  return sizeof(int32_t) * (size_t)kSmallSortRows * (1 + max_k);
}

void launch_sort_small(const SmallSortItem *items, int32_t nitems, int32_t max_k,
                       cudaStream_t s) {
  if (nitems <= 0) return;
  const size_t smem = small_sort_smem(max_k);
  static std::atomic<unsigned long long> attr_set{0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!((attr_set.load() >> (dev & 63)) & 1ull)) {
    cudaFuncSetAttribute(k_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)small_sort_smem(kMaxK));
    attr_set.fetch_or(1ull << (dev & 63));
  }
  k_sort_small<<<(unsigned)nitems, 256, smem, s>>>(items);
}

}  // namespace gsm

namespace gsm {

int32_t packed_words(int32_t k, int32_t bits) { return (k * bits + 63) / 64; }

void launch_pack_rows(const int32_t *rows, int64_t N, int32_t k, int32_t bits, uint64_t *keys,
                      int64_t ld, cudaStream_t s) {
  if (N <= 0) return;
  k_pack_keys<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(rows, 1, k, N, k, bits,
                                                          packed_words(k, bits), keys, ld);
}

int launch_sort_rows_packed(const int32_t *a, int64_t lda, int64_t N, int32_t k, int32_t bits,
                            int32_t sort_cols, uint64_t *keys_a, uint64_t *keys_b, int64_t ld,
                            int32_t *out, int32_t *hist, int64_t *hist_off, int64_t *tmp,
                            cudaStream_t s) {
  if (N <= 0) return 0;
  int launches = 0;
  const int32_t nw = packed_words(k, bits);
  if (a) {
    k_pack_keys<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(a, lda, 1, N, k, bits, nw, keys_a,
                                                            ld);
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
    const bool last = dg == digits - 1;
    if (nw == 1 && last)
      k_scatter_tile<1, true><<<(unsigned)nb, kSortThreads, 0, s>>>(src, dst, out, ld, N, k,
                                                                    bits, p, hist_off, nb);
    else if (nw == 1)
      k_scatter_tile<1, false><<<(unsigned)nb, kSortThreads, 0, s>>>(src, dst, out, ld, N, k,
                                                                     bits, p, hist_off, nb);
    else if (nw == 2 && last)
      k_scatter_tile<2, true><<<(unsigned)nb, kSortThreads, 0, s>>>(src, dst, out, ld, N, k,
                                                                    bits, p, hist_off, nb);
    else if (nw == 2)
      k_scatter_tile<2, false><<<(unsigned)nb, kSortThreads, 0, s>>>(src, dst, out, ld, N, k,
                                                                     bits, p, hist_off, nb);
    else if (last)
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
