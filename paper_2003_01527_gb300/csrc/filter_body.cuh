// Candidate filter body shared by the single-query and batched kernels
// (Sec. 3.2 filtering: label, degree and per-label neighbour counts).
#pragma once

#include "kernels.cuh"

namespace gsm {

// Requirement test of query vertex set `vneed` against per-slot neighbour
// counts cnt[] (slot s counts neighbours labelled d.slot_label[s]).
template <typename Desc>
__device__ __forceinline__ uint32_t nlc_pass(const Desc &d, uint32_t vneed,
                                             const int32_t (&cnt)[kMaxK]) {
  uint32_t pass = 0;
  for (int u = 0; u < d.k; ++u) {
    if (!((vneed >> u) & 1u)) continue;
    bool ok = true;
    for (int r = 0; r < d.nreq[u]; ++r) {
      const int slot = d.req_slot[u][r];
      int32_t c = 0;
#pragma unroll
      for (int s = 0; s < kMaxK; ++s) c = (s == slot) ? cnt[s] : c;
      ok = ok && c >= d.req_cnt[u][r];
    }
    if (ok) pass |= 1u << u;
  }
  return pass;
}

// The same test against v's row of the graph's label-count table: each
// requirement reads its one count byte (the row is L1-resident), with no
// register array to index.
template <typename Desc>
__device__ __forceinline__ uint32_t nlc_pass_row(const Desc &d, uint32_t vneed,
                                                 const uint8_t *__restrict__ row) {
  uint32_t pass = 0;
  for (uint32_t m = vneed; m; m &= m - 1) {
    const int u = __ffs(m) - 1;
    bool ok = true;
    for (int r = 0; r < d.nreq[u] && ok; ++r)
      ok = (int32_t)__ldg(row + d.slot_label[d.req_slot[u][r]]) >= d.req_cnt[u][r];
    if (ok) pass |= 1u << u;
  }
  return pass;
}

// One warp handles 32 consecutive data vertices per iteration (warps
// warp_id, warp_id + n_warps, ...).  Each lane first applies the label /
// degree / range test for its own vertex.  With the graph's neighbour label
// count table the requirements are read from it; otherwise they are counted
// from the rows, as follows.  A vertex that also needs per-label
// neighbour counts is first counted by its own lane over its first
// kLaneScan neighbours (most rows of a power-law graph end there); only a
// vertex whose requirements are still unmet and whose row goes on is then
// scanned by the whole warp (coalesced reads of the CSR row, labels gathered
// through L2).  The k bitmap words of the group are formed by ballots.  Lane u
// adds |C(u)| into sizes[u].
constexpr int kLaneScan = 32;
template <typename Desc>
__device__ __forceinline__ void filter_warps(const GraphDev &g, const Desc &d,
                                             uint32_t *__restrict__ bitmaps,
                                             unsigned long long *__restrict__ sizes,
                                             int64_t warp_id, int64_t n_warps) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned long long my_size = 0;  // lane u accumulates |C(u)|
  for (int64_t grp = warp_id; grp < d.n_words; grp += n_warps) {
    const int64_t v64 = grp * 32 + lane;
    const bool valid = v64 < g.n;
    const int32_t v = (int32_t)v64;
    int32_t lv = -1, deg = -1;
    if (valid) {
      lv = g.lab[v];
      deg = g.rp[v + 1] - g.rp[v];
    }
    uint32_t pre = 0, need = 0;
    if (valid)
      for (int u = 0; u < d.k; ++u) {
        if (lv == d.qlab[u] && deg >= d.qdeg[u] && v >= d.lo[u] && v < d.hi[u]) {
          pre |= 1u << u;
          if (d.nreq[u] > 0) need |= 1u << u;
        }
      }
    uint32_t result = pre & ~need;
    bool rest = false;
    if (need && g.nlc) {  // the counts are in the graph's table
      result |= nlc_pass_row(d, need, g.nlc + (int64_t)v * g.nlc_stride);
      need = 0;
    } else if (need) {
      const int32_t b = g.rp[v], e = g.rp[v + 1];
      const int32_t e1 = min(e, b + kLaneScan);
      int32_t cnt[kMaxK];
#pragma unroll
      for (int s = 0; s < kMaxK; ++s) cnt[s] = 0;
#pragma unroll 4
      for (int32_t idx = b; idx < e1; ++idx) {
        const int32_t lw = __ldg(g.lab + __ldg(g.col + idx));
#pragma unroll
        for (int s = 0; s < kMaxK; ++s)
          if (s < d.nslots && lw == d.slot_label[s]) ++cnt[s];
      }
      const uint32_t pass = nlc_pass(d, need, cnt);
      result |= pass;
      rest = pass != need && e > e1;
      need = rest ? need : 0;
    }
    uint32_t todo = __ballot_sync(kFull, rest);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int32_t vv = (int32_t)(grp * 32 + src);
      const uint32_t vneed = __shfl_sync(kFull, need, src);
      const int32_t b = g.rp[vv], e = g.rp[vv + 1];
      int32_t cnt[kMaxK], tot[kMaxK];
#pragma unroll
      for (int s = 0; s < kMaxK; ++s) cnt[s] = tot[s] = 0;
      uint32_t pass = 0;
      // Scan the row 256 neighbours at a time and stop as soon as every
      // requirement holds (counts only grow), so hubs end after one chunk.
      for (int32_t base = b; base < e; base += 256) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int32_t idx = base + j * 32 + lane;
          if (idx < e) {
            const int32_t lw = __ldg(g.lab + __ldg(g.col + idx));
#pragma unroll
            for (int s = 0; s < kMaxK; ++s)
              if (s < d.nslots && lw == d.slot_label[s]) ++cnt[s];
          }
        }
#pragma unroll
        for (int s = 0; s < kMaxK; ++s)
          if (s < d.nslots) tot[s] = __reduce_add_sync(kFull, cnt[s]);
        pass = nlc_pass(d, vneed, tot);
        if (pass == vneed) break;  // warp-uniform: tot is the same in every lane
      }
      if (lane == src) result |= pass;
    }
    for (int u = 0; u < d.k; ++u) {  // d.k is warp-uniform
      const uint32_t word = __ballot_sync(kFull, (result >> u) & 1u);
      if (lane == u) {
        bitmaps[(int64_t)u * d.n_words + grp] = word;
        my_size += __popc(word);
      }
    }
  }
  if (lane < d.k && my_size) atomicAdd(sizes + lane, my_size);
}

}  // namespace gsm
