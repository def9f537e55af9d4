// Internal interface of the batched form (batch.cu) for the host driver.
#pragma once

#include <cstddef>
#include <cstdint>

#include "kernels.cuh"

namespace gsm {

// Verification level i of one query (extending rows of width i by pi_i).
struct BatchLevel {
  int32_t nb;               // mapped query neighbours of pi_i
  int32_t bpos[kMaxK];      // their row positions
  int32_t ninj;             // same-label, non-adjacent positions
  int32_t inj[kMaxK];
  int32_t last;             // 1 if pi_i is the query's last vertex
  int32_t lab;              // dense label of pi_i (the row segment traversed)
  const uint32_t *bitmap;   // C(pi_i)
  int32_t nlt, lt[kMaxK];   // ordering constraints (none in the batched form)
  int32_t ngt, gt[kMaxK];
};

struct BatchQuery {
  int32_t k;
  int32_t enumerate;            // 1: the last level writes result rows
  int32_t out_col[kMaxK];       // result column of row position j (= pi_j)
  const uint32_t *root_bitmap;  // C(pi_0)
  BatchLevel lv[kMaxK];         // lv[1 .. k-1]
};

// Device-side sizes of one level (rows at level i, candidates checked while
// extending it, tiles, survivors that continue; FB = first element of the
// step's result rows in the result arena, FS = result rows the step writes).
struct BatchStep {
  int64_t R, W, tiles, S, FB, FS;
};

struct BatchArgs {
  int32_t nq, kmax, n_words;
  int32_t block, grid;
  int64_t cap_rows, cap_elems, cap_items;
  const FilterDesc *fds;          // [nq]
  uint32_t *const *bm_out;        // [nq] bitmap output of each query
  const BatchQuery *qs;           // [nq]
  unsigned long long *counts;     // [nq] results
  unsigned long long *sizes;      // [nq * kMaxK] |C(u)|
  int32_t *overflow;
  BatchStep *state;               // [kMaxK + 1]
  int32_t *wcnt;                  // [nq * n_words]
  int64_t *woffs;                 // [nq * n_words + 1]
  int64_t *partials;              // [grid + 1]
  int32_t *F[2], *rseg[2];        // frontiers: cap_elems / cap_rows each
  int32_t *pstart;                // [cap_rows]
  uint8_t *pslot;                 // [cap_rows]
  int64_t *woff;                  // [cap_rows + 1]
  int32_t *tile_row;              // [cap_items / 128 + 2]
  uint32_t *masks;                // [cap_items / 32 + 32]
  int32_t *tile_cnt;              // [cap_items / 128 + 2]
  int64_t *tile_off;              // [cap_items / 128 + 3]
  // enumerate batches (enumerate = 1): result rows of the queries that list
  // them.  The rows of step i (queries with k = i + 1) are row-major, k ints
  // each, in query-id column order, from element state[i].FB on; within a
  // step the queries follow batch order, each query's rows in lexicographic
  // order of its matching order.
  int32_t enumerate;
  int64_t cap_final;              // arena elements
  int32_t *final_rows;            // [cap_final]
  uint32_t *fmasks;               // [cap_items / 32 + 256]
  int32_t *ftile_cnt;             // [cap_items / 128 + 2]
  int64_t *ftile_off;             // [cap_items / 128 + 3]
};

// The candidate filter of nq queries in one launch: query j's FilterDesc is
// fds[j], its k bitmaps go to bm_out[j], |C(u)| to sizes[j * kMaxK + u]
// (zeroed here).  fds and bm_out are device arrays.
void launch_filter_many(const GraphDev &g, const FilterDesc *fds, uint32_t *const *bm_out,
                        unsigned long long *sizes, int32_t nq, int32_t n_words,
                        cudaStream_t s);

// Issues the whole batch on stream s (no host synchronisation, fixed launch
// shapes, so the sequence can be captured as a CUDA graph).  Returns the
// number of kernels launched.
int batch_enqueue(const GraphDev &g, const BatchArgs &a, cudaStream_t s);

}  // namespace gsm
