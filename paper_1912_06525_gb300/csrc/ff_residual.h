// Float-float (double-FP32) refinement residual and solution output for the
// mixed-precision query path.
#pragma once

#include "kernels.h"

namespace katz {

// Rows longer than kHeavyRowNnz split into kHeavySeg-entry segments (one
// CTA each) whose float-float partial sums meet in `scratch` (2 * nseg * ld
// floats) before the row epilogue; the row kernel then skips them.
struct HeavyRows {
  const int32_t* rows = nullptr;     // n heavy row ids
  const int32_t* seg_ptr = nullptr;  // n + 1 segment offsets
  const int32_t* seg_row = nullptr;  // nseg: heavy-row index of each segment
  int64_t n = 0, nseg = 0;
  float* scratch = nullptr;
};

// One refinement pass with the gathered FP32 operand X (M = I - beta A,
// A's stored weights exact in FP32):
//   init   : (Rh, Rl) = -X + beta A X            (float-float sums)
//   update : Rh = Rh (+ Rl if non-null) - X + beta A X   (Rl not written)
// and rr[c] += sum_i Rh[i][c]^2 for c < b when rr is non-null (the caller
// zeroes rr).  Blocks are ld-padded FP32, 16-byte aligned; cfg: the tuned
// CTAs per SM or null; hv (optional): the heavy rows of A, split.
void ffr_update(const Csr& A, double beta, const float* X, float* Rh, float* Rl, bool init,
                int64_t ld, int b, double* rr, const SpmmCfg* cfg, cudaStream_t s,
                const HeavyRows* hv = nullptr);

// (Kh, Kl) += D elementwise (TwoSum), total = rows * ld; kl_zero: Kl is
// taken as zero (not read) and written.
void ff_add(float* Kh, float* Kl, const float* D, int64_t total, cudaStream_t s,
            bool kl_zero = false);

// (Rh, Rl)[pos(i), j] += beta W[q_j, i] for the stored entries of the query
// rows (the sparse right-hand side); rr (optional) is adjusted by the change
// of Rh^2, which cancels badly when Rh ~ -b: prefer fresh column norms.
// maxdeg bounds the query rows' lengths.
void ffr_add_rhs(const Csr& W, const int32_t* q, const int32_t* pos, int b, double beta, float* Rh,
                 float* Rl, int64_t ld, double* rr, int64_t maxdeg, cudaStream_t s);

// out[i, c] = Kh (+ Kl if non-null) (+ D if non-null) at row map(i), column
// c, rounded once to FP32 or FP64.
void ff_out(const float* Kh, const float* Kl, const float* D, int64_t ld, const int32_t* map,
            int64_t n, int b, void* out, int out_dt, int64_t ldk, cudaStream_t s);

}  // namespace katz
