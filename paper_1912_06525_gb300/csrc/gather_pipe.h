// Pipelined row-gather kernels for the wide sparse products of the query
// path (the large-block Chebyshev step and the first refinement residual).
//
// One CTA per SM takes row blocks (<= 31 rows, ~512 stored entries) in
// increasing order from a global counter.  A producer warp streams, with
// cp.async.bulk (TMA bulk copies, completion counted on mbarriers), the row
// of the gathered operand X named by every stored entry of its rows into a
// shared-memory ring, and the rows' own operands into a second ring;
// consumer warps (one 128-column slice each) accumulate from shared memory
// and run the fused epilogue.  The bytes in flight live in shared memory,
// not in registers, so one CTA keeps ~200 KB of gathers outstanding per SM.
// Every wait is bounded (2 s); on timeout the kernel raises *err, drains
// the copies it issued and returns.
#pragma once

#include "kernels.h"

namespace katz {

// Row blocks of a CSR for the pipelined kernels: [bstart[k], bstart[k+1]),
// at most 31 rows and about 512 stored entries (+4 per row) each;
// bentry[k] = rowptr[bstart[k]]; ctr: the per-launch block counters.
struct PipeSplit {
  DBuf<int64_t> bstart, bentry;
  DBuf<int> ctr;
  int64_t nblocks = 0;
};
void pipe_split_build(const std::vector<int64_t>& rowptr, int64_t nrows, PipeSplit& ps,
                      cudaStream_t s);

// Whether the pipelined kernels take a block of padded width ld over this
// split (narrow blocks stay on the register kernels).
bool pipe_eligible(const PipeSplit& ps, int64_t ld);

// x_{k+1} = x_k + ak (x_k - x_{k-1}) + ck (B - x_k + beta A x_k) with
// x_k = sx * Xk and x_{k-1} = sp * Xprev, for the ld-padded FP32 blocks; Xprev null means
// x_{k-1} = 0; Xout may alias Xprev (not Xk).  unit: every stored weight is
// 1 (weights are not read).
void pipe_cheb_step(const Csr& A, const PipeSplit& ps, bool unit, double beta, double ak,
                    double ck, const float* Xk, const float* Xprev, const float* B, float* Xout,
                    int64_t ld, int* err, cudaStream_t s, double sx = 1.0, double sp = 1.0);

// First refinement-residual pass in float-float arithmetic with the
// gathered FP32 operand X (M = I - beta A): (Rh, Rl) = -X + beta A X, and
// rr[c] += sum_i Rh[i][c]^2 for the columns c < b when rr is non-null (the
// caller zeroes rr).
void pipe_residual(const Csr& A, const PipeSplit& ps, bool unit, double beta, const float* X,
                   float* Rh, float* Rl, int64_t ld, int b, double* rr, int* err, cudaStream_t s);

}  // namespace katz
