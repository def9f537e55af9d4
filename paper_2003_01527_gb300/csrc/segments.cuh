// Label-segmented adjacency: besides the id-sorted rows, the library keeps
// every row ordered by (neighbour label, neighbour id), so the neighbours of a
// vertex with one label form one contiguous, id-sorted segment.
#pragma once

#include "kernels.cuh"

namespace gsm {

// [first, second) = the neighbours of x with label l (rows of lcol are
// ordered by (label, id), so they are one contiguous, id-sorted segment).
__device__ __forceinline__ int2 label_segment(const GraphDev &g, int32_t x, int32_t l) {
  if (g.num_labels > 1 && g.hub_seg) {  // a hub: its segment table
    const int32_t h = __ldg(g.hub + x);
    if (h >= 0) {
      const int32_t *t = g.hub_seg + (size_t)h * (g.num_labels + 1) + l;
      return make_int2(__ldg(t), __ldg(t + 1));
    }
  }
  const int32_t b = __ldg(g.rp + x), e = __ldg(g.rp + x + 1);
  if (g.num_labels == 1) return make_int2(b, e);
  int32_t lo = b, len = e - b;  // first entry with label >= l
  while (len > 0) {
    const int32_t half = len >> 1;
    if (__ldg(g.llab + lo + half) < l) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  int32_t hi = lo;
  len = e - lo;  // first entry with label > l
  while (len > 0) {
    const int32_t half = len >> 1;
    if (__ldg(g.llab + hi + half) <= l) {
      hi += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return make_int2(lo, hi);
}

// Is w (label l) a neighbour of x?  One bit of x's adjacency bitmap when x
// is a hub, else one binary search on the (label, id) order of x's row.
__device__ __forceinline__ bool row_contains_l(const GraphDev &g, int32_t x, int32_t l,
                                               int32_t w) {
  if (!GSM_IN_BOUNDS(g.dbg, x >= 0 && x < g.n, kDbgNeighbour)) return false;
  if (g.hub) {
    const int32_t h = __ldg(g.hub + x);
    if (h >= 0)
      return (__ldg(g.hub_bits + (size_t)h * g.hub_words + (w >> 5)) >> (w & 31)) & 1u;
  }
  const int32_t e = __ldg(g.rp + x + 1);
  int32_t lo = __ldg(g.rp + x), len = e - lo;
  if (g.num_labels == 1) {  // one label: a plain search of the id-sorted row
    while (len > 0) {
      const int32_t half = len >> 1;
      if (__ldg(g.lcol + lo + half) < w) {
        lo += half + 1;
        len -= half + 1;
      } else {
        len = half;
      }
    }
    return lo < e && __ldg(g.lcol + lo) == w;
  }
  while (len > 0) {
    const int32_t half = len >> 1;
    const int32_t ml = __ldg(g.llab + lo + half);
    if (ml < l || (ml == l && __ldg(g.lcol + lo + half) < w)) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo < e && __ldg(g.llab + lo) == l && __ldg(g.lcol + lo) == w;
}

}  // namespace gsm
