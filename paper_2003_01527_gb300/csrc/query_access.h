// Read access to the opaque gsm_query (defined in api.cu) for other
// translation units of the library.  Not part of the public ABI.
#pragma once

#include <cstdint>

#include "gsm.h"

namespace gsm {

int32_t query_k(const gsm_query *q);
// Copies the labels, adjacency bitmasks and restriction ranges of q.
void query_describe(const gsm_query *q, int32_t *labels, uint32_t *adj, int32_t *lo,
                    int32_t *hi);

}  // namespace gsm
