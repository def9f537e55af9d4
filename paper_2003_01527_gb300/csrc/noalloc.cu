// gsm_candidates_static: the candidate filter for callers that cannot allocate
// device memory.
//
// Who needs it: a process whose device memory is already claimed by another
// allocator (for example a serving process whose caching allocator reserved
// the free HBM up front, so cudaMalloc fails or fragments that pool), and code
// in a latency-critical loop that cannot afford the device-wide
// synchronisation cudaMalloc/cudaFree may perform.  Such callers pass their
// own device-resident graph and receive the same candidate bitmaps as
// gsm_candidates, with no allocation by the library.
//
// The filter's working memory -- the bitmap staging area and the per-query-
// vertex counters it accumulates -- is one fixed array in this file, so every
// GPU that loads the library holds it until the process exits.
#include <cstring>
#include <mutex>

#include "gsm.h"
#include "kernels.cuh"
#include "query_access.h"

using namespace gsm;

namespace {

// Layout: 256 bytes of counters (16 x uint64), then the bitmaps.
constexpr size_t kCounterBytes = 256;
constexpr size_t kBitmapBytes = GSM_STATIC_SCRATCH_BITMAP_BYTES;
static_assert(kBitmapBytes % 256 == 0, "bitmap area must keep 256-byte alignment");
static __device__ __align__(256) unsigned char g_static_scratch[kCounterBytes + kBitmapBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};  // device address, per device

// Once per device, with that device current: the host-side name of the array
// is not a device address, so ask the runtime for the real one.
cudaError_t scratch_address(int device, unsigned char **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" gsm_status gsm_candidates_static(int32_t n, int64_t nnz, const int32_t *row_ptr,
                                            const int32_t *col, const int32_t *labels,
                                            const gsm_query *q, uint32_t *bitmaps,
                                            uint64_t *sizes, int32_t flags, void *stream) {
  if (!q || !row_ptr || !labels || (nnz > 0 && !col) || n < 0 || nnz < 0 ||
      (flags & ~GSM_OUT_DEVICE))
    return GSM_ERR_INVALID_ARG;
  if (n >= 0x7fffffff || nnz >= (int64_t(1) << 31)) return GSM_ERR_TOO_LARGE;
  const int32_t k = query_k(q);
  const int64_t n_words = ((int64_t)n + 31) / 32;
  if ((size_t)k * (size_t)n_words * sizeof(uint32_t) > kBitmapBytes) return GSM_ERR_TOO_LARGE;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
    return GSM_ERR_CUDA;
  unsigned char *base = nullptr;
  if (scratch_address(device, &base) != cudaSuccess) return GSM_ERR_CUDA;
  unsigned long long *d_sizes = reinterpret_cast<unsigned long long *>(base);
  uint32_t *d_bitmaps = reinterpret_cast<uint32_t *>(base + kCounterBytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // The filter description is built from the raw labels: a query vertex
  // matches a data vertex with the same label value, and each neighbour
  // requirement counts neighbours with a given label value.
  FilterDesc fd;
  std::memset(&fd, 0, sizeof(fd));
  int32_t qlab[kMaxK];
  uint32_t adj[kMaxK];
  int32_t lo[kMaxK], hi[kMaxK];
  query_describe(q, qlab, adj, lo, hi);
  fd.k = k;
  fd.n_words = (int32_t)n_words;
  for (int32_t u = 0; u < k; ++u) {
    fd.qlab[u] = qlab[u];
    fd.qdeg[u] = __builtin_popcount(adj[u]);
    fd.lo[u] = lo[u] < 0 ? 0 : lo[u];
    fd.hi[u] = hi[u] > n ? n : hi[u];
    int32_t lab_of[kMaxK], cnt_of[kMaxK], nl = 0;
    for (int32_t w = 0; w < k; ++w) {
      if (!(adj[u] >> w & 1u)) continue;
      int32_t j = 0;
      while (j < nl && lab_of[j] != qlab[w]) ++j;
      if (j == nl) {
        lab_of[nl] = qlab[w];
        cnt_of[nl++] = 0;
      }
      cnt_of[j]++;
    }
    for (int32_t j = 0; j < nl; ++j) {
      int32_t sl = 0;
      while (sl < fd.nslots && fd.slot_label[sl] != lab_of[j]) ++sl;
      if (sl == fd.nslots) fd.slot_label[fd.nslots++] = lab_of[j];
      fd.req_slot[u][fd.nreq[u]] = sl;
      fd.req_cnt[u][fd.nreq[u]++] = cnt_of[j];
    }
  }

  // The counters accumulate, and the array keeps the previous call's
  // contents: clear them first.  (The bitmap words are all overwritten.)
  if (cudaMemsetAsync(d_sizes, 0, kCounterBytes, s) != cudaSuccess) return GSM_ERR_CUDA;
  GraphDev g{n, nnz, row_ptr, col, labels, nullptr, nullptr, 0};  // the filter reads id-sorted rows
  g.dbg = nullptr;
  launch_filter(g, fd, d_bitmaps, d_sizes, s);
  if (cudaGetLastError() != cudaSuccess) return GSM_ERR_CUDA;
  const cudaMemcpyKind kind =
      (flags & GSM_OUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (bitmaps && n_words &&
      cudaMemcpyAsync(bitmaps, d_bitmaps, (size_t)k * n_words * sizeof(uint32_t), kind, s) !=
          cudaSuccess)
    return GSM_ERR_CUDA;
  if (sizes && cudaMemcpyAsync(sizes, d_sizes, (size_t)k * sizeof(uint64_t), kind, s) !=
                   cudaSuccess)
    return GSM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GSM_ERR_CUDA;
  return GSM_OK;
}
