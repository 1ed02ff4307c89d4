// Device and host helpers shared by the tcgen05 GEMMs: mbarriers with
// bounded waits, 2-D TMA tile loads, the shared-memory matrix descriptor of a
// K-major 128-byte-swizzled tile, and tensor-map encoding.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace katz {
namespace tcu {

constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with parity `phase`; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major, 128-byte swizzled tile:
// start address >> 4 (bits 0-13), leading byte offset 16 B (unused for this
// layout, bits 16-29), stride byte offset 1024 B between 8-row groups
// (bits 32-45), descriptor version 1 (bits 46-47), swizzle mode 2 =
// 128-byte (bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFF);
  d |= uint64_t(1) << 16;
  d |= uint64_t(1024 >> 4) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(2) << 61;
  return d;
}


typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    KATZ_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                               cudaEnableDefault, &q));
    KATZ_REQUIRE(p != nullptr && q == cudaDriverEntryPointSuccess, KATZ_ECUDA,
                 "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D BF16 tensor map: rows x K (K contiguous, row stride ld elements),
// box = box_rows x 64, 128-byte swizzle, zero fill out of bounds.
// 2-D tensor map of a row-major rows x K matrix (K contiguous, row stride ld
// elements of esize bytes), box = box_rows x (128 / esize) elements, 128-byte
// swizzle, zero fill out of bounds.
inline CUtensorMap make_map(const void* ptr, CUtensorMapDataType dtype, int esize, int64_t rows,
                            int64_t K, int64_t ld, int box_rows) {
  KATZ_REQUIRE(reinterpret_cast<uintptr_t>(ptr) % 16 == 0 && (ld * esize) % 16 == 0, KATZ_EINVAL,
               "tc_gemm: operands need 16-byte aligned base and row stride");
  CUtensorMap m;
  const cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(ld * esize)};
  const cuuint32_t box[2] = {cuuint32_t(128 / esize), cuuint32_t(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(&m, dtype, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  KATZ_REQUIRE(r == CUDA_SUCCESS, KATZ_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(r));
  return m;
}


}  // namespace tcu
}  // namespace katz
