// Float-float (double-FP32) residual and solution updates for the
// mixed-precision refinement.
#pragma once

#include "kernels.h"

namespace katz {

// R = B - M K with K = Kh + Kl (FP32 pair), M = I - beta A, B = beta W e_q
// scattered to rows pos(i) (pos null = identity).  A's stored weights must
// be exact in FP32.  maxdeg = max degree of the query nodes.
void ff_residual(const Csr& A, const Csr& W, const int32_t* q, const int32_t* pos, int b,
                 double beta, const float* Kh, const float* Kl, int64_t ld, float* R,
                 int64_t maxdeg, cudaStream_t s);

// (Kh, Kl) += D elementwise (TwoSum), total = rows * ld.
void ff_add(float* Kh, float* Kl, const float* D, int64_t total, cudaStream_t s);

// out[i, c] = Kh[map(i), c] + Kl[map(i), c] in FP32 or FP64.
void ff_out(const float* Kh, const float* Kl, int64_t ld, const int32_t* map, int64_t n, int b,
            void* out, int out_dt, int64_t ldk, cudaStream_t s);

// Zero the columns c with conv[c] != 0 (and the padding columns c >= b).
void mask_columns(float* R, int64_t ld, int64_t len, int b, const int* conv, cudaStream_t s);

// Unit-weight graphs: K in 64-bit fixed point, K[i][c] = Kfx[i][c] 2^-sh[c].
// R = B - M K with exact integer sparse sums (see fx_residual.cu).
void fx_residual(const Csr& A, const Csr& W, const int32_t* q, const int32_t* pos, int b,
                 double beta, const long long* K, const int* sh, int64_t ld, float* R,
                 int64_t maxdeg, cudaStream_t s);
// K (+)= round(D 2^sh) (init: K = ...), rows x ld.
void fx_add(long long* K, const float* D, int64_t rows, int64_t ld, const int* sh, int b,
            bool init, cudaStream_t s);
void fx_out(const long long* K, int64_t ld, const int* sh, const int32_t* map, int64_t n, int b,
            void* out, int out_dt, int64_t ldk, cudaStream_t s);

}  // namespace katz
