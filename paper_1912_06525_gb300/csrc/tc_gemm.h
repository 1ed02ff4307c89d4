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

// Xt (cols x rows, BF16, ldxt) = X^T for X (rows x cols, FP32, ldx).
void to_bf16_transposed(const float* X, int64_t ldx, int64_t rows, int cols, __nv_bfloat16* Xt,
                        int64_t ldxt, cudaStream_t s);

}  // namespace katz
