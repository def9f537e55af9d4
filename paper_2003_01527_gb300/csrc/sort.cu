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

// Lanes of the warp whose value v (kBits bits) equals this lane's: the
// intersection, over the bits, of the lanes that agree on the bit.  kBits
// ballots; cheaper here than __match_any_sync for byte digits.
template <int kBits>
__device__ __forceinline__ uint32_t equal_lanes(uint32_t v) {
  uint32_t peers = kFull;
#pragma unroll
  for (int i = 0; i < kBits; ++i) {
    const bool bit = (v >> i) & 1u;
    const uint32_t on = __ballot_sync(kFull, bit);
    peers &= bit ? on : ~on;
  }
  return peers;
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
    const uint32_t peers = equal_lanes<9>(dgt);
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

// Byte digit at bit (64 wi + sh) of a key of NW <= 2 words held in registers.
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

// ---- single-sweep passes (keys of at most two words, N < 2^30) ----
//
// One histogram launch counts the digits of every pass in one read of the
// keys; then each pass is one launch.  A CTA takes the next tile by ticket,
// counts its digits, publishes the per-digit counts, and finds the count of
// each digit in all earlier tiles by a decoupled look-back over the
// published words of the tiles before it (per digit a 32-bit word: flag in
// the top two bits, count or inclusive prefix below).  The tile's keys are
// then staged in shared memory in their sorted order, so that consecutive
// threads write consecutive positions of a digit's run.  Tiles only wait on
// tiles with smaller tickets, which are already running, so the waits end;
// each is still bounded (spin_limit polls, then *err = 1 and the sum found so
// far, which keeps every write inside the output).
constexpr uint32_t kSwAggregate = 1u << 30;
constexpr uint32_t kSwInclusive = 2u << 30;
constexpr uint32_t kSwFlags = 3u << 30;
constexpr uint32_t kSwValue = kSwAggregate - 1u;
constexpr int kMaxDigits = 16;  // two words of key
constexpr int kLookWin = 8;     // look-back words read at once

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Exclusive scan of one value per thread over the kWarps warps of the CTA.
template <int kWarps>
__device__ __forceinline__ uint32_t cta_excl_scan(uint32_t v, uint32_t *s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < kWarps ? s_warp[lane] : 0;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < kWarps) s_warp[lane] = wi - w;
  }
  __syncthreads();
  const uint32_t r = x - v + s_warp[warp];
  __syncthreads();
  return r;
}

// Column j of the packed key kk (k columns of b bits, column 0 highest).
template <int NW>
__device__ __forceinline__ int32_t key_column(const uint64_t (&kk)[NW], int32_t k, int32_t b,
                                              int32_t j) {
  const int32_t bp = (k - 1 - j) * b;
  const int32_t wi = bp >> 6, sh = bp & 63;
  uint64_t v = (NW > 1 && wi == 1) ? kk[NW - 1] : kk[0];
  v >>= sh;
  if (NW > 1 && wi == 0 && sh + b > 64) v |= kk[NW - 1] << (64 - sh);
  return (int32_t)(v & ((1ull << b) - 1ull));
}

// Histograms of `digits` byte digits (at bits pos.p[0..digits)) of all N keys, added
// into ghist[d * 256 + digit]; the last CTA to finish then writes their
// exclusive scans, gexcl[d * 256 + digit] = the number of keys whose digit d
// is smaller (done: a zeroed counter).  Grid-stride over tiles of kSortTile
// keys; shared-memory atomics into two copies of the counts (even and odd
// warps) to halve the contention of skewed digits.
struct DigitPos {
  int32_t p[kMaxDigits];  // bit position of each digit pass, lowest first
};

template <int NW>
__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const uint64_t *__restrict__ in,
                                                             int64_t ld, int64_t N, DigitPos pos,
                                                             int32_t digits, uint32_t *ghist,
                                                             uint32_t *__restrict__ gexcl,
                                                             uint32_t *done) {
  __shared__ uint32_t s_h[2][kMaxDigits * kBins];
  __shared__ uint32_t s_warp[kSortThreads / 32];
  __shared__ bool s_last;
  uint32_t *h = s_h[(threadIdx.x >> 5) & 1];
  for (int e = threadIdx.x; e < 2 * kMaxDigits * kBins; e += kSortThreads) (&s_h[0][0])[e] = 0;
  __syncthreads();
  const int64_t tiles = (N + kSortTile - 1) / kSortTile;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t base = tile * kSortTile;
    uint64_t key[kSortChunks][NW];
#pragma unroll
    for (int c = 0; c < kSortChunks; ++c) {
      const int64_t idx = base + c * kSortThreads + threadIdx.x;
#pragma unroll
      for (int w = 0; w < NW; ++w) key[c][w] = idx < N ? __ldg(in + (int64_t)w * ld + idx) : 0;
    }
#pragma unroll
    for (int c = 0; c < kSortChunks; ++c) {
      if (base + c * kSortThreads + threadIdx.x >= N) continue;
#pragma unroll
      for (int32_t d = 0; d < kMaxDigits; ++d) {  // unrolled: pos is indexed statically
        if (d >= digits) break;
        const int32_t p = pos.p[d];
        atomicAdd(&h[d * kBins + tile_digit<NW>(key[c], p >> 6, p & 63)], 1u);
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < digits * kBins; e += kSortThreads) {
    const uint32_t v = s_h[0][e] + s_h[1][e];
    if (v) atomicAdd(&ghist[e], v);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int32_t d = 0; d < digits; ++d) {
    const uint32_t v = ld_relaxed_u32(ghist + d * kBins + threadIdx.x);
    gexcl[d * kBins + threadIdx.x] = cta_excl_scan<kSortThreads / 32>(v, s_warp);
  }
}

// One stable pass on the byte digit at bit p.  gexcl: the 256 exclusive
// digit offsets over all keys; status: tiles * 256 look-back words, zero
// before the pass; ticket: zero before the pass.  Warp w of a tile holds keys
// w*256 + c*32 + lane (c = 0..7), so (warp, chunk, lane) is key order: the
// warps first count their digits (early counts), thread t then turns the
// counts of digit t into tile-local starts per warp and publishes the tile's
// count; the warps rank their chunks in order (ballots; one leader per digit
// advances the warp's running start) and stage the keys in shared memory in
// sorted order; only then does thread t look back for the earlier tiles'
// counts of digit t (they have had the ranking's time to publish), and
// consecutive threads write consecutive positions of a digit's run.  The
// last pass (kUnpack) writes each key as a row-major int32 row of out_rows
// instead of moving the key.
// Threads of a single-sweep CTA: 512 for one-word keys (tiles of 4,096 keys:
// half the tiles to look back over), 256 for two-word keys (registers).
template <int NW>
__host__ __device__ constexpr int sweep_threads() {
  return NW == 1 ? 512 : 256;
}

template <int NW, bool kUnpack>
__global__ void __launch_bounds__(sweep_threads<NW>(), NW == 1 ? 2 : 3) k_onesweep(
    const uint64_t *__restrict__ in, uint64_t *__restrict__ out_keys,
    int32_t *__restrict__ out_rows, int64_t ld, int64_t N, int32_t k, int32_t b, int32_t p,
    const uint32_t *__restrict__ gexcl, uint32_t *status, uint32_t *ticket, int32_t spin_limit,
    uint32_t *err, int64_t stall_tile) {
  constexpr int kT = sweep_threads<NW>();
  constexpr int kTile = kT * kSortChunks;
  constexpr int kWarps = kT / 32;
  extern __shared__ __align__(16) uint64_t s_keys[];  // NW * kTile: word w of key i at w*kTile + i
  __shared__ uint32_t s_wc[kWarps][kBins];
  __shared__ int64_t s_off[kBins];
  __shared__ uint32_t s_warp[kWarps];
  __shared__ int64_t s_tile;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool owner = t < kBins;  // thread t < 256 owns digit t
  for (int e = t; e < kWarps * kBins; e += kT) (&s_wc[0][0])[e] = 0;
  if (t == 0) s_tile = (int64_t)atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t base = tile * kTile;
  const int64_t wbase = base + warp * (kTile / kWarps);
  uint64_t key[kSortChunks][NW];
#pragma unroll
  for (int c = 0; c < kSortChunks; ++c) {
    const int64_t idx = wbase + c * 32 + lane;
#pragma unroll
    for (int w = 0; w < NW; ++w) key[c][w] = idx < N ? __ldg(in + (int64_t)w * ld + idx) : 0;
  }
  const int32_t wi = p >> 6, sh = p & 63;
  uint32_t dg[kSortChunks];
#pragma unroll
  for (int c = 0; c < kSortChunks; ++c) {
    dg[c] = wbase + c * 32 + lane < N ? tile_digit<NW>(key[c], wi, sh) : kBins;
    if (dg[c] < kBins) atomicAdd(&s_wc[warp][dg[c]], 1u);
  }
  __syncthreads();
  uint32_t cnt = 0;
  if (owner) {
#pragma unroll
    for (int w = 0; w < kWarps; ++w) cnt += s_wc[w][t];
  }
  uint32_t *mine = status + tile * kBins + t;
  const bool publish = owner && tile != stall_tile;  // fault injection: never publish
  if (publish) st_relaxed_u32(mine, (tile == 0 ? kSwInclusive : kSwAggregate) | cnt);
  const uint32_t lx = cta_excl_scan<kWarps>(cnt, s_warp);  // before digit t in this tile
  if (owner) {
    uint32_t run = lx;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t v = s_wc[w][t];
      s_wc[w][t] = run;
      run += v;
    }
  }
  __syncthreads();
  // rank the warp's chunks in order and stage the keys (a lane without a
  // key, only in the last tile, has digit kBins: a ninth bit)
  const uint32_t lt = (1u << lane) - 1u;
  const bool full = base + kTile <= N;
#pragma unroll
  for (int c = 0; c < kSortChunks; ++c) {
    const uint32_t peers = full ? equal_lanes<8>(dg[c]) : equal_lanes<9>(dg[c]);
    const int leader = __ffs(peers) - 1;
    uint32_t start = 0;
    if (lane == leader && dg[c] < kBins) {
      start = s_wc[warp][dg[c]];
      s_wc[warp][dg[c]] = start + __popc(peers);
    }
    start = __shfl_sync(kFull, start, leader);
    if (dg[c] < kBins) {
      const uint32_t li = start + __popc(peers & lt);
#pragma unroll
      for (int w = 0; w < NW; ++w) s_keys[w * kTile + li] = key[c][w];
    }
    __syncwarp();
  }
  // look back kLookWin tiles at a time (independent loads), summing counts
  // up to the nearest inclusive prefix; a tile not yet published stops the
  // window there and is polled again (a poll that makes no progress counts
  // against spin_limit)
  uint32_t excl = 0;
  if (owner && tile > 0) {
    int64_t j = tile - 1;
    int32_t polls = 0;
    uint32_t nap = 32;  // ns, doubled per fruitless poll up to 1 us
    bool done = false;
    while (!done) {
      uint32_t st[kLookWin];
#pragma unroll
      for (int w = 0; w < kLookWin; ++w)
        st[w] = j - w >= 0 ? ld_relaxed_u32(status + (j - w) * kBins + t) : kSwInclusive;
      int used = 0;
#pragma unroll
      for (int w = 0; w < kLookWin; ++w) {
        if (done || used != w) continue;  // stopped earlier in the window
        const uint32_t f = st[w] & kSwFlags;
        if (f == 0) continue;
        excl += st[w] & kSwValue;
        used = w + 1;
        if (f == kSwInclusive) done = true;
      }
      if (done) break;
      j -= used;
      if (used == 0) {
        if (++polls > spin_limit) {
          if (err) *(volatile uint32_t *)err = 1u;
          break;
        }
        __nanosleep(nap);
        nap = nap < 1024 ? 2 * nap : nap;
      }
    }
    if (publish) st_relaxed_u32(mine, kSwInclusive | (excl + cnt));
  }
  if (owner) s_off[t] = (int64_t)__ldg(gexcl + t) + excl - lx;
  __syncthreads();
  const int32_t n_tile = (int32_t)(N - base < kTile ? N - base : kTile);
  for (int32_t i = t; i < n_tile; i += kT) {
    uint64_t kk[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) kk[w] = s_keys[w * kTile + i];
    const int64_t pos = s_off[tile_digit<NW>(kk, wi, sh)] + i;
    if (!GSM_IN_BOUNDS(err ? err + 1 : nullptr, pos >= 0 && pos < N, kDbgSortPosition)) continue;
    if (kUnpack) {
      int32_t *dst = out_rows + pos * k;
      if ((k & 1) == 0) {
        for (int32_t j = 0; j < k; j += 2)
          *reinterpret_cast<int2 *>(dst + j) =
              make_int2(key_column<NW>(kk, k, b, j), key_column<NW>(kk, k, b, j + 1));
      } else {
        for (int32_t j = 0; j < k; ++j) dst[j] = key_column<NW>(kk, k, b, j);
      }
    } else {
#pragma unroll
      for (int w = 0; w < NW; ++w) out_keys[(int64_t)w * ld + pos] = kk[w];
    }
  }
}

// flags[i] = 1 where key i's prefix (the key bits selected by m0 in word 0
// and m1 in word 1) differs from key i-1's; flags[0] = 0.
template <int NW>
__global__ void __launch_bounds__(256) k_prefix_flags(const uint64_t *__restrict__ keys,
                                                      int64_t ld, int64_t N, uint64_t m0,
                                                      uint64_t m1, int32_t *__restrict__ flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    if (i == 0) {
      flags[0] = 0;
      continue;
    }
    uint64_t d = (__ldg(keys + i) ^ __ldg(keys + i - 1)) & m0;
    if (NW > 1) d |= (__ldg(keys + ld + i) ^ __ldg(keys + ld + i - 1)) & m1;
    flags[i] = d != 0;
  }
}

// Key i gains the dense rank of its prefix, incl[i] = offs[i + 1] (the
// prefix changes up to i), at bit rank_pos (rank_bits bits, above the k
// columns).
template <int NW>
__global__ void __launch_bounds__(256) k_put_rank(uint64_t *__restrict__ keys, int64_t ld,
                                                  int64_t N, const int64_t *__restrict__ offs,
                                                  int32_t rank_pos, int32_t rank_bits) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int32_t w = rank_pos >> 6, sh = rank_pos & 63;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    const uint64_t rank = (uint64_t)__ldg(offs + i + 1);
    keys[(int64_t)w * ld + i] |= rank << sh;
    if (NW > 1 && w == 0 && sh > 0 && sh + rank_bits > 64) keys[ld + i] |= rank >> (64 - sh);
  }
}

// Packed keys of the segments' rows (see launch_pack_segments): compact row
// i belongs to the last segment whose `first` is <= i (binary search).
__global__ void __launch_bounds__(256) k_pack_segments(const SortSegment *__restrict__ segs,
                                                       int32_t nseg, int64_t N, int32_t k,
                                                       int32_t b, int32_t seg_bits, int32_t nw,
                                                       uint64_t *__restrict__ keys, int64_t ld) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    int32_t lo = 0, hi = nseg;  // largest j with segs[j].first <= i
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (segs[mid].first <= i) lo = mid; else hi = mid;
    }
    const int32_t *row = segs[lo].src + (i - segs[lo].first) * k;
    for (int32_t t = 0; t < nw; ++t) {
      uint64_t w = 0;
      for (int32_t j = 0; j < k; ++j) {
        const uint64_t v = (uint32_t)__ldg(row + j);
        const int32_t p = (k - 1 - j) * b - 64 * t;
        if (p >= 0 && p < 64)
          w |= v << p;
        else if (p < 0 && p + b > 0)
          w |= v >> (-p);
      }
      const int32_t q = k * b - 64 * t;  // the segment index
      const uint64_t sv = (uint64_t)lo;
      if (q >= 0 && q < 64)
        w |= sv << q;
      else if (q < 0 && q + seg_bits > 0)
        w |= sv >> (-q);
      keys[(int64_t)t * ld + i] = w;
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

int32_t sort_rank_pos(int32_t k, int32_t bits, int32_t sort_cols) {
  sort_cols = std::min(std::max(sort_cols, 1), k);
  const int32_t lo = (k - sort_cols) * bits;
  return std::max(k * bits, lo + 8 * ((sort_cols * bits + 7) / 8));
}

int32_t sort_key_words(int32_t k, int32_t bits, SortPrefix pre) {
  return (k * bits + std::max(pre.given_bits, 0) + 63) / 64;
}


namespace {

// Where the pieces of a sort's scratch go: the single-sweep passes (keys of
// at most two words, N < 2^30) need the digit histograms, one ticket and
// tiles * 256 look-back words per pass; the general passes a histogram per
// tile and its scan.
struct SortLayout {
  bool sweep;
  int32_t nw, digits, lo_bit;
  DigitPos pos;                // bit position of each digit pass
  int32_t prefix_cols, rank_bits, rank_pos;  // rank_bits = 0: no prefix rank
  bool given;                                // a group rank came with the keys
  bool ranked;                               // the prefix rank came with the keys
  int64_t tiles;
  size_t o_ghist, o_gexcl, o_ticket, o_status, o_hist, o_hoff, o_tmp, o_flags, o_offs, o_rtmp,
      bytes;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

SortLayout sort_layout(int64_t N, int32_t k, int32_t bits, int32_t sort_cols, SortPrefix pre) {
  SortLayout L{};
  L.nw = sort_key_words(k, bits, pre);
  sort_cols = std::min(std::max(sort_cols, 1), k);
  L.lo_bit = (k - sort_cols) * bits;
  L.digits = (sort_cols * bits + 7) / 8;
  if (pre.given_bits > 0) {
    // a group rank is already in the keys, right above the k columns: the
    // sort field is the contiguous bits of the sorted columns and the rank
    L.digits = (sort_cols * bits + pre.given_bits + 7) / 8;
    pre = SortPrefix();  // no rank to compute
    L.given = true;
  }
  // prefix rank: the sorted leading columns keyed by their dense rank above
  // the k columns, when the key words have room and it saves passes
  if (pre.cols >= 1 && pre.cols < sort_cols && pre.groups >= 1 && L.nw <= 2) {
    int32_t rb = 1;
    while (rb < 62 && (int64_t(1) << rb) < pre.groups) ++rb;
    const int32_t low = ((sort_cols - pre.cols) * bits + 7) / 8, high = (rb + 7) / 8;
    const int32_t rp = sort_rank_pos(k, bits, sort_cols);
    if (rp + rb <= 64 * L.nw && low + high < L.digits) {
      L.prefix_cols = pre.cols;
      L.rank_bits = rb;
      L.ranked = pre.ranked;
      L.rank_pos = rp;
      for (int32_t d = 0; d < low; ++d) L.pos.p[d] = L.lo_bit + 8 * d;
      for (int32_t d = 0; d < high; ++d) L.pos.p[low + d] = L.rank_pos + 8 * d;
      L.digits = low + high;
    }
  }
  if (!L.rank_bits)
    for (int32_t d = 0; d < std::min(L.digits, kMaxDigits); ++d) L.pos.p[d] = L.lo_bit + 8 * d;
  L.sweep = L.nw <= 2 && N < (int64_t(1) << 30) && L.digits <= kMaxDigits;
  const int64_t tile = L.sweep ? (int64_t)(L.nw == 1 ? sweep_threads<1>() : sweep_threads<2>()) *
                                     kSortChunks
                               : kSortTile;
  L.tiles = (N + tile - 1) / tile;  // tiles of the passes
  size_t off = 0;
  if (L.sweep) {
    L.o_ghist = off;
    off = align256(off + sizeof(uint32_t) * (size_t)L.digits * kBins);
    L.o_gexcl = off;
    off = align256(off + sizeof(uint32_t) * (size_t)L.digits * kBins);
    L.o_ticket = off;  // one per pass, then the histogram's done counter
    off = align256(off + sizeof(uint32_t) * (size_t)(L.digits + 1));
    L.o_status = off;
    off = align256(off + sizeof(uint32_t) * (size_t)L.digits * (size_t)L.tiles * kBins);
  } else {
    const int64_t H = L.tiles * kBins;
    L.o_hist = off;
    off = align256(off + sizeof(int32_t) * (size_t)H);
    L.o_hoff = off;
    off = align256(off + sizeof(int64_t) * (size_t)(H + 1));
    L.o_tmp = off;
    off = align256(off + sizeof(int64_t) * (size_t)scan_tmp_elems(H));
  }
  if (L.rank_bits && !L.ranked) {
    L.o_flags = off;
    off = align256(off + sizeof(int32_t) * (size_t)N);
    L.o_offs = off;
    off = align256(off + sizeof(int64_t) * (size_t)(N + 1));
    L.o_rtmp = off;
    off = align256(off + sizeof(int64_t) * (size_t)scan_tmp_elems(N));
  }
  L.bytes = std::max<size_t>(off, 256);
  return L;
}

int sm_count() {
  static std::atomic<int> cached[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int v = cached[dev & 63].load();
  if (!v) {
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 1;
    cached[dev & 63].store(v);
  }
  return v;
}

template <int NW>
void sweep_pass(bool last, const uint64_t *src, uint64_t *dst, int32_t *out, int64_t ld,
                int64_t N, int32_t k, int32_t bits, int32_t p, const uint32_t *gexcl,
                uint32_t *status, uint32_t *ticket, int32_t spin_limit, uint32_t *err,
                int64_t stall_tile, int64_t tiles, cudaStream_t s) {
  // the staged tile lives in dynamic shared memory (two-word keys take the
  // CTA past the 48 KB of static shared memory)
  constexpr int kT = sweep_threads<NW>();
  constexpr size_t kDyn = sizeof(uint64_t) * NW * kT * kSortChunks;
  static std::atomic<unsigned long long> attr_set{0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!((attr_set.load() >> (dev & 63)) & 1ull)) {
    cudaFuncSetAttribute(k_onesweep<NW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kDyn);
    cudaFuncSetAttribute(k_onesweep<NW, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kDyn);
    attr_set.fetch_or(1ull << (dev & 63));
  }
  if (last)
    k_onesweep<NW, true><<<(unsigned)tiles, kT, kDyn, s>>>(
        src, dst, out, ld, N, k, bits, p, gexcl, status, ticket, spin_limit, err, stall_tile);
  else
    k_onesweep<NW, false><<<(unsigned)tiles, kT, kDyn, s>>>(
        src, dst, out, ld, N, k, bits, p, gexcl, status, ticket, spin_limit, err, stall_tile);
}

}  // namespace

size_t sort_scratch_bytes(int64_t N, int32_t k, int32_t bits, int32_t sort_cols,
                          SortPrefix pre) {
  return sort_layout(std::max<int64_t>(N, 1), k, bits, sort_cols, pre).bytes;
}

int32_t sort_digit_passes(int64_t N, int32_t k, int32_t bits, int32_t sort_cols,
                          SortPrefix pre, bool *prefix_rank) {
  const SortLayout L = sort_layout(std::max<int64_t>(N, 1), k, bits, sort_cols, pre);
  if (prefix_rank) *prefix_rank = L.rank_bits > 0 && !L.ranked;  // ranks computed here
  return L.digits;
}

int launch_sort_rows_packed(const int32_t *a, int64_t lda, int64_t N, int32_t k, int32_t bits,
                            int32_t sort_cols, uint64_t *keys_a, uint64_t *keys_b, int64_t ld,
                            int32_t *out, void *scratch, int32_t spin_limit, uint32_t *err,
                            int32_t stall_tile, cudaStream_t s, SortPrefix pre) {
  if (N <= 0) return 0;
  int launches = 0;
  const SortLayout L = sort_layout(N, k, bits, sort_cols, pre);
  const int32_t nw = L.nw;
  if (a) {
    k_pack_keys<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(a, lda, 1, N, k, bits, nw, keys_a,
                                                            ld);
    ++launches;
  }
  char *sc = (char *)scratch;
  if (L.rank_bits && !L.ranked) {
    // the prefix's dense rank: change flags, their scan, the rank or-ed in
    // above the k columns (the prefix bits themselves stay, for the unpack)
    const int32_t plo = (k - L.prefix_cols) * bits, phi = k * bits;
    auto word_mask = [&](int32_t w) {
      const int32_t lo = std::max(plo - 64 * w, 0), hi = std::min(phi - 64 * w, 64);
      if (hi <= lo) return 0ull;
      const unsigned long long top = hi >= 64 ? ~0ull : ((1ull << hi) - 1ull);
      return top & ~((1ull << lo) - 1ull);
    };
    int32_t *flags = (int32_t *)(sc + L.o_flags);
    int64_t *offs = (int64_t *)(sc + L.o_offs);
    const unsigned g = (unsigned)std::min<int64_t>((N + 255) / 256, (int64_t)sm_count() * 8);
    if (nw == 1) {
      k_prefix_flags<1><<<g, 256, 0, s>>>(keys_a, ld, N, word_mask(0), 0ull, flags);
      launch_scan_i32(flags, offs, N, (int64_t *)(sc + L.o_rtmp), s);
      k_put_rank<1><<<g, 256, 0, s>>>(keys_a, ld, N, offs, L.rank_pos, L.rank_bits);
    } else {
      k_prefix_flags<2><<<g, 256, 0, s>>>(keys_a, ld, N, word_mask(0), word_mask(1), flags);
      launch_scan_i32(flags, offs, N, (int64_t *)(sc + L.o_rtmp), s);
      k_put_rank<2><<<g, 256, 0, s>>>(keys_a, ld, N, offs, L.rank_pos, L.rank_bits);
    }
    launches += 2 + scan_kernels(N);
  }
  uint64_t *src = keys_a, *dst = keys_b;
  if (L.sweep) {
    if (spin_limit <= 0) spin_limit = kLbSpinLimit;
    cudaMemsetAsync(sc, 0, L.o_status + sizeof(uint32_t) * (size_t)L.digits * (size_t)L.tiles * kBins,
                    s);
    uint32_t *ghist = (uint32_t *)(sc + L.o_ghist);
    uint32_t *gexcl = (uint32_t *)(sc + L.o_gexcl);
    uint32_t *ticket = (uint32_t *)(sc + L.o_ticket);
    uint32_t *status = (uint32_t *)(sc + L.o_status);
    const unsigned grid = (unsigned)std::min<int64_t>(L.tiles, (int64_t)sm_count() * 4);
    if (nw == 1)
      k_digit_hist<1><<<grid, kSortThreads, 0, s>>>(keys_a, ld, N, L.pos, L.digits, ghist,
                                                    gexcl, ticket + L.digits);
    else
      k_digit_hist<2><<<grid, kSortThreads, 0, s>>>(keys_a, ld, N, L.pos, L.digits, ghist,
                                                    gexcl, ticket + L.digits);
    ++launches;
    for (int32_t dg = 0; dg < L.digits; ++dg) {
      const int32_t p = L.pos.p[dg];
      const bool last = dg == L.digits - 1;
      uint32_t *st = status + (size_t)dg * (size_t)L.tiles * kBins;
      if (nw == 1)
        sweep_pass<1>(last, src, dst, out, ld, N, k, bits, p, gexcl + dg * kBins, st, ticket + dg,
                      spin_limit, err, stall_tile, L.tiles, s);
      else
        sweep_pass<2>(last, src, dst, out, ld, N, k, bits, p, gexcl + dg * kBins, st, ticket + dg,
                      spin_limit, err, stall_tile, L.tiles, s);
      ++launches;
      std::swap(src, dst);
    }
    return launches;
  }
  // general passes: a histogram per tile, its scan, then the scatter
  int32_t *hist = (int32_t *)(sc + L.o_hist);
  int64_t *hist_off = (int64_t *)(sc + L.o_hoff);
  int64_t *tmp = (int64_t *)(sc + L.o_tmp);
  const int64_t nb = L.tiles;
  for (int32_t dg = 0; dg < L.digits; ++dg) {
    const int32_t p = dg < kMaxDigits ? L.pos.p[dg] : L.lo_bit + 8 * dg;
    k_hist_keys<<<(unsigned)nb, kSortThreads, 0, s>>>(src, ld, N, nw, p, hist, nb);
    launch_scan_i32(hist, hist_off, nb * kBins, tmp, s);
    const bool last = dg == L.digits - 1;
    if (last)
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

void launch_pack_segments(const SortSegment *segs, int32_t nseg, int64_t N, int32_t k,
                          int32_t bits, int32_t seg_bits, int32_t nw, uint64_t *keys, int64_t ld,
                          cudaStream_t s) {
  if (N <= 0 || nseg <= 0) return;
  const unsigned g = (unsigned)std::min<int64_t>((N + 255) / 256, (int64_t)sm_count() * 8);
  k_pack_segments<<<g, 256, 0, s>>>(segs, nseg, N, k, bits, seg_bits, nw, keys, ld);
}

}  // namespace gsm
