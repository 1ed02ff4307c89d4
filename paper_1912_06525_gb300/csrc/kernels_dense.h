// Dense helpers used by the index build and the Schur-complement solve.
#pragma once

#include "common.cuh"

namespace katz {

// C = alpha op(A) op(B) + beta C (row-major); lower_only skips tiles
// strictly above the diagonal.
template <class VT>
void gemm2(bool transA, bool transB, int64_t M, int64_t N, int64_t K, double alpha, const VT* A,
           int64_t lda, const VT* B, int64_t ldb, double beta, VT* C, int64_t ldc, bool lower_only,
           cudaStream_t s);

// Y = a X for a rows x cols sub-matrix.
template <class VT>
void copy2d(const VT* X, int64_t ldx, VT* Y, int64_t ldy, int64_t rows, int64_t cols, double a,
            cudaStream_t s);

// Inverses of the M11 diagonal blocks of one size class S (FP64, S x S
// zero-padded, [count][S][S]); Wperm is W in index order.
void block_inverses(const Csr& Wperm, const int64_t* start, const int32_t* size, int64_t count,
                    int S, double beta, double* inv, int* flag, cudaStream_t s);

// In-place inverse of an SPD n x n matrix by blocked Gauss-Jordan.
// ws: 2*n*64 + 64*64 doubles.  flag set on a non-positive pivot.
void spd_inverse_inplace(double* A, int64_t n, int64_t lda, double* ws, int* flag,
                         cudaStream_t s);

// Top-k per column with explicit scratch (slices*8*b*k ids and scores):
// for column j the k nodes i != q[j] of highest K[i][j] (score descending,
// id ascending), leaving out q[j]'s neighbours when mask_nbrs.
template <class VT>
void topk_columns_ws(const Csr& W, const VT* K, int64_t ldk, int64_t n, const int32_t* q, int b,
                     int k, int32_t* ids, double* scores, int32_t* ws_id, double* ws_sc,
                     int slices, cudaStream_t s, bool mask_nbrs = true);

}  // namespace katz
