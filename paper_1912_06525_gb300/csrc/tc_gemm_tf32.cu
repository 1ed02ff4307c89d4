// FP32-accurate dense products on the 5th-generation tensor cores: three
// TF32 tcgen05.mma products per k-block (kind::tf32, FP32 accumulator in
// tensor memory) with each FP32 operand split into a TF32 high part and the
// remainder, A B ~ Ah Bh + Ah Bl + Al Bh (the dropped Al Bl is below 2^-22
// of |A||B|).  Operands are staged by TMA (128-byte swizzle, K-major) into a
// 3-stage mbarrier pipeline; one thread issues the MMAs; the epilogue reads
// the accumulator with tcgen05.ld.  Every mbarrier wait is bounded; on
// timeout the CTA raises *err and skips its output.
#include "tc_gemm.h"
#include "tc_util.cuh"

namespace katz {

namespace {

using namespace tcu;

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3;
constexpr int TILE = BM * BK * 4;  // bytes of one 128 x 32 FP32 tile (BM == BN)

// Round an FP32 value to TF32 (10 stored mantissa bits), to nearest, ties
// to even; infinities and NaNs pass through.
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u += 0x00000fffu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xffffe000u);
}

// Instruction descriptor, kind::tf32: FP32 accumulator (bits 4-5 = 1), A and
// B TF32 (bits 7-9 = 2, 10-12 = 2), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__global__ void __launch_bounds__(128, 1)
    tc_gemm_tf32x3_kernel(const __grid_constant__ CUtensorMap mAh,
                          const __grid_constant__ CUtensorMap mAl,
                          const __grid_constant__ CUtensorMap mBh,
                          const __grid_constant__ CUtensorMap mBl, int M, int N, int K,
                          float alpha, float beta, const float* Cin, int64_t ldcin, float* C,
                          int64_t ldc, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // stage s: Ah, Al, Bh, Bl tiles
  auto tile = [&](int s, int which) { return base + (s * 4 + which) * TILE; };
  uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * 4 * TILE);
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
    // TMA producer
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(empty + s, ((kb / STAGES) - 1) & 1)) {
        atomicExch(&failed, 1);
        break;
      }
      if (failed) break;
      mbar_expect_tx(full + s, 4 * TILE);
      tma_load_2d(tile(s, 0), &mAh, kb * BK, m0, full + s);
      tma_load_2d(tile(s, 1), &mAl, kb * BK, m0, full + s);
      tma_load_2d(tile(s, 2), &mBh, kb * BK, n0, full + s);
      tma_load_2d(tile(s, 3), &mBl, kb * BK, n0, full + s);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 MMAs of K = 8 per 32-element (128-byte) k-block and operand pair
    constexpr uint32_t idesc = instr_desc_tf32(BM, BN);
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(full + s, (kb / STAGES) & 1)) {
        atomicExch(&failed, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(tile(s, 0)), al = smem_u32(tile(s, 1)),
                     bh = smem_u32(tile(s, 2)), bl = smem_u32(tile(s, 3));
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk) {
        const uint32_t o = kk * 32;
        mma_tf32(tmem, smem_desc(ah + o), smem_desc(bh + o), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(ah + o), smem_desc(bl + o), idesc, 1u);
        mma_tf32(tmem, smem_desc(al + o), smem_desc(bh + o), idesc, 1u);
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
          C[int64_t(row) * ldc + col] =
              beta == 0.f ? a : a + beta * Cin[int64_t(row) * ldcin + col];
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

// hi/lo = TF32 split of V (FP64 or FP32, rows x cols, ldv) into FP32 arrays (ldo).
template <class T>
__global__ void split_kernel(const T* V, int64_t ldv, int64_t rows, int cols, float* hi,
                             float* lo, int64_t ldo) {
  const int64_t total = rows * cols;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / cols;
    const int c = int(e - i * cols);
    const double v = V[i * ldv + c];
    const float h = tf32_round(float(v));
    hi[i * ldo + c] = h;
    lo[i * ldo + c] = float(v - double(h));
  }
}

// hi/lo (cols x rows, ldo) = TF32 split of X^T for X (rows x cols, FP32, ldx).
__global__ void split_t_kernel(const float* X, int64_t ldx, int64_t rows, int cols, float* hi,
                               float* lo, int64_t ldo) {
  __shared__ float t[32][33];
  const int64_t r0 = int64_t(blockIdx.x) * 32;
  const int c0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k;
    const int c = c0 + threadIdx.x;
    t[k][threadIdx.x] = (r < rows && c < cols) ? X[r * ldx + c] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k;
    const int64_t r = r0 + threadIdx.x;
    if (c < cols && r < rows) {
      const float x = t[threadIdx.x][k];
      const float h = tf32_round(x);
      hi[int64_t(c) * ldo + r] = h;
      lo[int64_t(c) * ldo + r] = x - h;
    }
  }
}

}  // namespace

size_t tc_gemm_tf32x3_smem_bytes() { return size_t(STAGES) * 4 * TILE + 1024 + 256; }

void tc_gemm_tf32x3(const float* Ah, const float* Al, int64_t lda, const float* Bh,
                    const float* Bl, int64_t ldb, int M, int N, int K, float alpha, float beta,
                    const float* Cin, int64_t ldcin, float* C, int64_t ldc, int* err,
                    cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  KATZ_REQUIRE(K > 0 && (beta == 0.f || Cin), KATZ_EINVAL, "tc_gemm_tf32x3: bad arguments");
  const CUtensorMap mah = make_map(Ah, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, M, K, lda, BM);
  const CUtensorMap mal = make_map(Al, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, M, K, lda, BM);
  const CUtensorMap mbh = make_map(Bh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, N, K, ldb, BN);
  const CUtensorMap mbl = make_map(Bl, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, N, K, ldb, BN);
  const size_t smem = tc_gemm_tf32x3_smem_bytes();
  static bool attr = false;
  if (!attr) {
    KATZ_CUDA(cudaFuncSetAttribute(tc_gemm_tf32x3_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const dim3 grid((unsigned)ceil_div(N, BN), (unsigned)ceil_div(M, BM));
  prof_begin(s);
  tc_gemm_tf32x3_kernel<<<grid, 128, smem, s>>>(mah, mal, mbh, mbl, M, N, K, alpha, beta, Cin,
                                                ldcin, C, ldc, err);
  KATZ_CHECK_LAUNCH();
  if (profiling())
    prof_end("tc_gemm_tf32x3", 3.0 * 2.0 * double(M) * N * K, s);
}

template <class T>
void split_tf32(const T* V, int64_t ldv, int64_t rows, int cols, float* hi, float* lo,
                int64_t ldo, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  const int64_t total = rows * cols;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256),
                                                                      int64_t(num_sms()) * 16));
  split_kernel<T><<<g, 256, 0, s>>>(V, ldv, rows, cols, hi, lo, ldo);
  KATZ_CHECK_LAUNCH();
}
template void split_tf32<double>(const double*, int64_t, int64_t, int, float*, float*, int64_t,
                                 cudaStream_t);
template void split_tf32<float>(const float*, int64_t, int64_t, int, float*, float*, int64_t,
                                cudaStream_t);

void split_tf32_transposed(const float* X, int64_t ldx, int64_t rows, int cols, float* hi,
                           float* lo, int64_t ldo, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  const dim3 grid((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(cols, 32));
  split_t_kernel<<<grid, dim3(32, 8), 0, s>>>(X, ldx, rows, cols, hi, lo, ldo);
  KATZ_CHECK_LAUNCH();
}

}  // namespace katz
