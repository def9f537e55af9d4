// Compressed partial results (Sec. 3.2 stores partial results as hashed
// tuples; this is the lossless form of that idea): a frontier row of width i
// is kept as (parent row in the width-(i-1) frontier, vertex placed at
// position i-1) -- 8 bytes per row whatever the width -- and decoded by
// following parent indices back to the width-1 frontier.  Internal interface
// between api.cu and compressed.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace gsm {

// The chain of frontiers that row indices of width i refer to: V[j][r] is the
// vertex at position j-1 of row r of the width-j frontier, P[j][r] (j >= 2)
// the row of the width-(j-1) frontier it extends.  V[1] is the level-1 list.
struct CFrontier {
  const int32_t *V[kMaxK + 1];
  const int32_t *P[kMaxK + 1];
};

// Pivot choice of launch_pivot_scan for the R rows of width i of f.
void launch_cpivot(const GraphDev &g, const LevelDesc &d, const CFrontier &f, int32_t i,
                   int64_t R, int32_t *pstart, uint8_t *pslot, int64_t *work, cudaStream_t s);

// Output of a compressed level.  kCSinkPairs: survivor q of the level becomes
// row0 + q of the next frontier (pn = its parent row, vn = its new vertex);
// kCSinkRows / kCSinkKeys: the decoded result row or its packed sort key, as
// RowSink's kSinkRows / kSinkKeys; kCSinkCount: survivors are only counted.
enum CSinkMode : int32_t { kCSinkPairs = 0, kCSinkRows = 1, kCSinkKeys = 2, kCSinkCount = 3 };
struct CSink {
  int32_t mode;
  RowSink rows;  // kCSinkRows / kCSinkKeys
  int32_t *pn, *vn;
  int64_t row0;                // kCSinkPairs
  unsigned long long *total;   // kCSinkCount: survivors are added here
};

// One single-pass level over candidates [wa, wb) of the width-i rows of f
// (the same tiles, check, ranking and look-back as launch_extend_fused):
// lookback needs extend_tiles(wa, wb, block) + kLbExtra zeroed words (word
// tiles + 1 receives the survivor count, tiles + 2 an error flag set after a
// wait of more than spin_limit polls; the count mode only uses the ticket
// word).  The output needs room for wb - wa rows.
void launch_cextend(const GraphDev &g, const LevelDesc &d, const CFrontier &f, int32_t i,
                    const int32_t *pstart, const uint8_t *pslot, const int64_t *woff,
                    const int32_t *tile_row, int64_t wa, int64_t wb, int32_t block,
                    unsigned long long *lookback, const CSink &sink, int32_t spin_limit,
                    cudaStream_t s);

}  // namespace gsm
