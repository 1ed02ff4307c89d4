// linkpred_topk_noalloc: the top-k link-prediction kernels with their
// scratch (the per-slice candidate lists) in a fixed, file-scope device
// array instead of memory obtained from cudaMalloc.
//
// Who needs this: code that must not allocate device memory while it runs
// -- a serving loop whose latency budget has no room for an allocation
// (cudaMalloc may synchronise the whole device), or a process whose device
// memory is already reserved by another framework's caching allocator, so
// that a fresh cudaMalloc would fail although the caller's own buffers are
// in place.  Such callers pass every input and output; this entry point
// touches no allocator (no cudaMalloc/cudaFree, no library routine that
// allocates).  It checks the query ids on the host (one small copy into a
// fixed host array) and synchronises the caller's stream before and after
// its kernels.
#include <atomic>
#include <cstring>
#include <mutex>

#include "index.h"
#include "kernels_dense.h"

namespace {

// Scratch: up to kNoAllocEntries candidate (id, score) pairs.  Each GPU that
// loads the library holds this array (3 MiB) until the process exits.
constexpr int64_t kNoAllocEntries = int64_t(1) << 18;
static __device__ __align__(256) int32_t g_topk_ids[kNoAllocEntries];
static __device__ __align__(256) double g_topk_scores[kNoAllocEntries];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t* g_ids_ptr[kMaxDevices] = {};
double* g_sc_ptr[kMaxDevices] = {};

// Device addresses of the scratch arrays for the current device, looked up
// once per device (cudaGetSymbolAddress; the host-side symbols are only
// stand-ins and must never be passed to a kernel).
void scratch_for_current_device(int32_t** ids, double** sc) {
  int dev = 0;
  KATZ_CUDA(cudaGetDevice(&dev));
  KATZ_REQUIRE(dev >= 0 && dev < kMaxDevices, KATZ_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> l(g_mu);
  if (!g_ids_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    KATZ_CUDA(cudaGetSymbolAddress(&p, g_topk_ids));
    KATZ_CUDA(cudaGetSymbolAddress(&q, g_topk_scores));
    g_ids_ptr[dev] = static_cast<int32_t*>(p);
    g_sc_ptr[dev] = static_cast<double*>(q);
  }
  *ids = g_ids_ptr[dev];
  *sc = g_sc_ptr[dev];
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int linkpred_topk_noalloc(const katz_index* idx, const int32_t* q, int32_t b,
                                     const void* K, int32_t k_dtype, int64_t ldk, int32_t k,
                                     int32_t* ids_out, double* scores_out, void* stream) {
  try {
    KATZ_REQUIRE(idx && q && K && ids_out && scores_out, KATZ_EINVAL, "null argument");
    KATZ_REQUIRE(b > 0 && b <= 1024, KATZ_EINVAL, "b must be in [1, 1024]");
    KATZ_REQUIRE(k > 0 && k <= 64, KATZ_EINVAL, "k must be in [1, 64]");
    KATZ_REQUIRE(k_dtype == KATZ_F32 || k_dtype == KATZ_F64, KATZ_EINVAL, "k_dtype");
    KATZ_REQUIRE(ldk >= b, KATZ_EINVAL, "ldk < b");
    KATZ_REQUIRE(on_device(q) && on_device(K) && on_device(ids_out) && on_device(scores_out),
                 KATZ_EINVAL, "linkpred_topk_noalloc needs device pointers for all buffers");
    // at least one slice (8 lists of k entries per query column) must fit
    const int64_t per_slice = int64_t(8) * b * k;
    KATZ_REQUIRE(per_slice <= kNoAllocEntries, KATZ_EINVAL,
                 "b * k = " + std::to_string(int64_t(b) * k) + " exceeds the no-alloc scratch (" +
                     std::to_string(kNoAllocEntries / 8) + ")");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // validate the query ids through a fixed host array (no allocation)
    int32_t hq[1024];
    KATZ_CUDA(cudaMemcpyAsync(hq, q, 4 * size_t(b), cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    for (int j = 0; j < b; ++j)
      KATZ_REQUIRE(hq[j] >= 0 && hq[j] < idx->n, KATZ_EINVAL, "query id out of range");
    int32_t* wid = nullptr;
    double* wsc = nullptr;
    scratch_for_current_device(&wid, &wsc);
    const int64_t want = std::max<int64_t>(1, std::min<int64_t>(16, idx->n / 65536 + 1));
    const int slices = (int)std::min<int64_t>(want, kNoAllocEntries / per_slice);
    if (k_dtype == KATZ_F32)
      katz::topk_columns_ws<float>(idx->W.view(), static_cast<const float*>(K), ldk, idx->n, q, b,
                                   k, ids_out, scores_out, wid, wsc, slices, s);
    else
      katz::topk_columns_ws<double>(idx->W.view(), static_cast<const double*>(K), ldk, idx->n, q,
                                    b, k, ids_out, scores_out, wid, wsc, slices, s);
    KATZ_CUDA(cudaStreamSynchronize(s));
    return KATZ_OK;
  } catch (const katz::Error& e) {
    katz::set_last_error(e.what());
    return e.code;
  }
}
