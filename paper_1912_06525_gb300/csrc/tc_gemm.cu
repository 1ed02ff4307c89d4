// Rank-r correction GEMMs of the Schur preconditioner (Eq. 14) on the
// 5th-generation tensor cores: tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulator in tensor memory), operands staged by TMA into 128-byte
// swizzled shared memory, a 4-stage mbarrier pipeline, one elected thread
// issuing the MMAs and the tensor-memory accumulator read back with
// tcgen05.ld for the epilogue.
//
// Computes D = A * B^T for A (M x K) and B (N x K), both BF16 row-major with
// K contiguous ("K-major"), and either
//   mode 0:  C (FP32, M x N, row-major ldc) = alpha * D + beta * C
//   mode 1:  Ct (BF16, N x M, row-major ldct) = alpha * D   (transposed)
// Every wait on an mbarrier is bounded; on timeout the CTA records an error
// in *err and skips the rest of its work.
#include <cuda.h>

#include <atomic>

#include "kernels.h"
#include "tc_gemm.h"
#include "tc_util.cuh"

namespace katz {

namespace {

using namespace tcu;

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
constexpr int TILE_A = BM * BK * 2, TILE_B = BN * BK * 2;  // bytes per stage
// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) |
         (uint32_t(M >> 4) << 24);
}

__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   int M, int N, int K, float alpha, float beta, float* C, int64_t ldc,
                   __nv_bfloat16* Ct, int64_t ldct, int mode, int* err, int stall) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned tiles (required by the 128-byte swizzle atoms)
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* tA = base;
  unsigned char* tB = base + STAGES * TILE_A;
  uint64_t* full = reinterpret_cast<uint64_t*>(tB + STAGES * TILE_B);
  uint64_t* empty = full + STAGES;
  uint64_t* accb = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accb + 1);
  __shared__ int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nkb = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    failed = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(accb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer (stall: a test switch under which no copy is issued, so
    // the MMA issuer's bounded wait on the first stage runs out with nothing
    // in flight)
    for (int kb = 0; kb < nkb && !stall; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(empty + s, ((kb / STAGES) - 1) & 1)) {
        atomicExch(&failed, 1);
        break;
      }
      if (failed) break;
      mbar_expect_tx(full + s, TILE_A + TILE_B);
      tma_load_2d(tA + s * TILE_A, &mapA, kb * BK, m0, full + s);
      tma_load_2d(tB + s * TILE_B, &mapB, kb * BK, n0, full + s);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = instr_desc(BM, BN);
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(full + s, (kb / STAGES) & 1)) {
        atomicExch(&failed, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(tA + s * TILE_A), b0 = smem_u32(tB + s * TILE_B);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t ad = smem_desc(a0 + kk * 32), bd = smem_desc(b0 + kk * 32);
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(empty + s))
          : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(accb))
        : "memory");
  }
  __syncwarp();

  // epilogue: warp w owns accumulator lanes (rows) 32w .. 32w+31
  const bool ok = mbar_wait(accb, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) atomicExch(&failed, 1);
  __syncthreads();
  if (!failed) {
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col >= N) break;
          const float a = alpha * __uint_as_float(v[j]);
          if (mode == 0) {
            float* cp = C + int64_t(row) * ldc + col;
            *cp = beta == 0.f ? a : a + beta * (*cp);
          } else {
            Ct[int64_t(col) * ldct + row] = __float2bfloat16(a);
          }
        }
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

// Column-major conversion: Xt[j][i] = bf16(X[i][j]) for the K-major B operand.
__global__ void to_bf16_transposed_kernel(const float* X, int64_t ldx, int64_t rows, int cols,
                                          __nv_bfloat16* Xt, int64_t ldxt) {
  __shared__ float tile[32][33];
  const int64_t r0 = int64_t(blockIdx.x) * 32;
  const int c0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k;
    const int c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < rows && c < cols) ? X[r * ldx + c] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k;
    const int64_t r = r0 + threadIdx.x;
    if (c < cols && r < rows) Xt[int64_t(c) * ldxt + r] = __float2bfloat16(tile[threadIdx.x][k]);
  }
}

std::atomic<int> g_stall_copies{0};

}  // namespace

void set_test_stall_copies(bool on) { g_stall_copies.store(on ? 1 : 0); }

size_t tc_gemm_smem_bytes() { return size_t(STAGES) * (TILE_A + TILE_B) + 1024 + 256; }

void tc_gemm(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int M,
             int N, int K, float alpha, float beta, float* C, int64_t ldc, __nv_bfloat16* Ct,
             int64_t ldct, int mode, int* err, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  const CUtensorMap ma = tcu::make_map(A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, M, K, lda, BM);
  const CUtensorMap mb = tcu::make_map(B, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, N, K, ldb, BN);
  const size_t smem = tc_gemm_smem_bytes();
  static bool attr = false;
  if (!attr) {
    KATZ_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    attr = true;
  }
  dim3 grid((unsigned)ceil_div(N, BN), (unsigned)ceil_div(M, BM));
  prof_begin(s);
  tc_gemm_kernel<<<grid, 128, smem, s>>>(ma, mb, M, N, K, alpha, beta, C, ldc, Ct, ldct, mode,
                                         err, g_stall_copies.load());
  KATZ_CHECK_LAUNCH();
  if (profiling())
    prof_end("tc_gemm", 2.0 * (double(M) * K + double(N) * K) +
                            (mode == 0 ? 4.0 * M * N * (beta != 0.f ? 2 : 1) : 2.0 * M * N),
             s);
}

void to_bf16_transposed(const float* X, int64_t ldx, int64_t rows, int cols, __nv_bfloat16* Xt,
                        int64_t ldxt, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  dim3 grid((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(cols, 32));
  to_bf16_transposed_kernel<<<grid, dim3(32, 8), 0, s>>>(X, ldx, rows, cols, Xt, ldxt);
  KATZ_CHECK_LAUNCH();
}

}  // namespace katz
