// tcgen05 (5th-generation tensor core) GEMM for the rank-r correction of
// the Schur preconditioner.
#pragma once

#include "common.cuh"

namespace katz {

// D = A * B^T with A (M x K) and B (N x K) BF16 row-major (K contiguous,
// row strides lda/ldb elements, multiples of 8, 16-byte aligned bases).
// mode 0: C (FP32, M x N, ldc) = alpha*D + beta*C.
// mode 1: Ct (BF16, N x M, ldct) = alpha*D (transposed store).
// err (device int) is set if a pipeline wait timed out.
void tc_gemm(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int M,
             int N, int K, float alpha, float beta, float* C, int64_t ldc, __nv_bfloat16* Ct,
             int64_t ldct, int mode, int* err, cudaStream_t s);

size_t tc_gemm_smem_bytes();

// Test switch (process-wide): while on, tc_gemm's producer issues no TMA
// copy, so the kernel's bounded wait runs out and *err is set.
void set_test_stall_copies(bool on);

// C (FP32, M x N, ldc) = alpha * A B^T + beta * Cin (ldcin; Cin may be C)
// with FP32-level accuracy from three TF32 tensor-core products: A = Ah + Al
// (M x K) and B = Bh + Bl (N x K), K contiguous, row strides multiples of 4
// elements, 16-byte aligned bases (see split_tf32).  err (device int) is set
// if a pipeline wait timed out.
void tc_gemm_tf32x3(const float* Ah, const float* Al, int64_t lda, const float* Bh,
                    const float* Bl, int64_t ldb, int M, int N, int K, float alpha, float beta,
                    const float* Cin, int64_t ldcin, float* C, int64_t ldc, int* err,
                    cudaStream_t s);

// hi = TF32 rounding of V, lo = V - hi (FP32), rows x cols (ldv -> ldo).
template <class T>
void split_tf32(const T* V, int64_t ldv, int64_t rows, int cols, float* hi, float* lo,
                int64_t ldo, cudaStream_t s);
// The same for X^T: hi/lo are cols x rows (ldo) for X rows x cols (ldx).
void split_tf32_transposed(const float* X, int64_t ldx, int64_t rows, int cols, float* hi,
                           float* lo, int64_t ldo, cudaStream_t s);

// Xt (cols x rows, BF16, ldxt) = X^T for X (rows x cols, FP32, ldx).
void to_bf16_transposed(const float* X, int64_t ldx, int64_t rows, int cols, __nv_bfloat16* Xt,
                        int64_t ldxt, cudaStream_t s);

}  // namespace katz
