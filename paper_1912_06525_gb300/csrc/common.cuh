// Shared definitions of the Katz CUDA library (host + device).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstdio>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/katz.h"

namespace katz {

// ------------------------------------------------------------ error handling
// Internal failures throw katz::Error; the C layer turns it into a status
// code plus katz_last_error().
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define KATZ_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      if (e_ == cudaErrorMemoryAllocation)                                           \
        throw ::katz::Error(KATZ_ENOMEM, std::string("cuda: ") + cudaGetErrorString(e_) + \
                                             " at " + __FILE__ + ":" + std::to_string(__LINE__)); \
      throw ::katz::Error(KATZ_ECUDA, std::string("cuda: ") + cudaGetErrorString(e_) + \
                                          " at " + __FILE__ + ":" + std::to_string(__LINE__)); \
    }                                                                                \
  } while (0)

// Every kernel launch site calls this right after the launch; it also
// counts launches (katz_launch_count).
#define KATZ_CHECK_LAUNCH()                  \
  do {                                       \
    KATZ_CUDA(cudaGetLastError());           \
    ::katz::count_launch();                  \
  } while (0)

#define KATZ_REQUIRE(cond, code, msg)                     \
  do {                                                    \
    if (!(cond)) throw ::katz::Error((code), (msg));      \
  } while (0)

// Sets the message katz_last_error() returns on this thread.
void set_last_error(const std::string& msg);

// ------------------------------------------------------------ measurement
void count_launch();
int64_t launch_count();
// CUDA-event timing of tagged launches (enabled by katz_profile_enable).
bool profiling();
void prof_begin(cudaStream_t s);
void prof_end(const char* tag, double alg_bytes, cudaStream_t s);
// true when the host-side fault injection (katz_fault_inject_alloc) makes
// this device allocation fail
bool alloc_fault();

// Named NVTX range over a scope: the phases of a query show up in ncu /
// nsys timelines (`--nvtx`); without a tool attached it costs a call.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------ device memory
// Owning device buffer (cudaMalloc / cudaFree).
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    if (count) {
      if (alloc_fault()) throw Error(KATZ_ENOMEM, "injected device allocation failure");
      KATZ_CUDA(cudaMalloc(&p, count * sizeof(T)));
    }
    n = count;
  }
  // grow-only reallocation (contents not kept)
  void ensure(size_t count) { if (count > n) alloc(count); }
  void release() { if (p) cudaFree(p); p = nullptr; n = 0; }
  size_t bytes() const { return n * sizeof(T); }
};

// Named, grow-only device scratch owned by an index.
class Workspace {
 public:
  template <class T>
  T* get(const std::string& name, size_t count) {
    auto& b = bufs_[name];
    b.ensure(count * sizeof(T));
    return reinterpret_cast<T*>(b.p);
  }
  void clear() { bufs_.clear(); }
  void release(const std::string& name) { bufs_.erase(name); }
  size_t bytes() const {
    size_t t = 0;
    for (auto& kv : bufs_) t += kv.second.bytes();
    return t;
  }

 private:
  std::map<std::string, DBuf<uint8_t>> bufs_;
};

// ------------------------------------------------------------ sparse views
// CSR view on device: rows [0, nrows) with global column ids.  `val` may be
// null (unit weights); `vdt` is the stored value type.
struct Csr {
  int64_t nrows = 0;
  int64_t ncols = 0;
  int64_t nnz = 0;
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const void* val = nullptr;
  int vdt = KATZ_UNIT;
};

// Owning CSR on device.
struct DevCsr {
  int64_t nrows = 0, ncols = 0, nnz = 0;
  int vdt = KATZ_UNIT;
  DBuf<int64_t> rowptr;
  DBuf<int32_t> col;
  DBuf<uint8_t> val;  // raw bytes of the stored type
  Csr view() const {
    Csr c;
    c.nrows = nrows; c.ncols = ncols; c.nnz = nnz;
    c.rowptr = rowptr.p; c.col = col.p;
    c.val = (vdt == KATZ_UNIT) ? nullptr : val.p;
    c.vdt = vdt;
    return c;
  }
  size_t bytes() const { return rowptr.bytes() + col.bytes() + val.bytes(); }
};

// Host CSR (int64 rowptr, int32 col, double values or empty for unit).
struct HostCsr {
  int64_t nrows = 0, ncols = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;  // empty = unit weights
  int64_t nnz() const { return rowptr.empty() ? 0 : rowptr.back(); }
};

// Upload a host CSR with values stored as `vdt` (rounded to nearest even).
void upload_csr(const HostCsr& h, int vdt, DevCsr& d, cudaStream_t s);

inline size_t vdt_size(int vdt) {
  switch (vdt) {
    case KATZ_F64: return 8;
    case KATZ_F32: return 4;
    case KATZ_BF16: return 2;
    default: return 0;
  }
}

// ------------------------------------------------------------ device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class T> struct VecOf;
template <> struct VecOf<float> { using type = float4; static constexpr int width = 4; };
template <> struct VecOf<double> { using type = double2; static constexpr int width = 2; };

inline int num_sms() {
  static int sms = -1;
  if (sms < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
  }
  return sms;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace katz
