// Launchers of the Katz CUDA kernels.  Dense n x b blocks are node-major
// (entry (i, j) at X[i*ld + j]); ld is a multiple of 4 floats / 2 doubles so
// rows can be moved with 16-byte vector loads.
#pragma once

#include "common.cuh"

namespace katz {

// Rows with more stored entries than this are handled by the split-row
// kernel (several warps per row, one column slice each) so that a few hub
// rows do not serialise the sweep.
constexpr int64_t kHeavyRowNnz = 384;
// stored entries per segment of a heavy row in the split residual kernels
constexpr int64_t kHeavySeg = 512;

// Launch shape of the CSR SpMM (chosen by the autotuner or the default).
struct SpmmCfg {
  int warps_per_cta = 8;   // row groups of 32 threads per CTA
  int col_tile = 0;        // columns per CTA tile (0 = whole row up to 1024 floats / 512 doubles)
  int ctas_per_sm = 8;     // grid = SMs * ctas_per_sm (grid-stride over rows)
  bool pipe = false;       // the pipelined (TMA bulk-copy) kernel measured faster here
  bool pipe_first = false; // ... for the first refinement-residual pass
  int fused_cps = 0;       // CTAs per SM of the fused Chebyshev / residual kernel (0: ctas_per_sm)
  int gather_depth = 0;    // fused Chebyshev step: gathered rows loaded together (0, 4 or 8)
  bool row_pipeline = false;  // fused Chebyshev step: the row-pipelined kernel
  int row_chunk = 0;  // fused Chebyshev step: CTA c takes rows [c, c+1) * row_chunk (0: the
                      // warps stride over all rows)
};

// Y[i,:] = gamma * Z[i,:] + alpha * sum_k A[i,k] X[k,:]   for i < A.nrows.
// If `dots` is non-null: dots[c] += sum_i Y[i,c] * V[i,c] (FP64 accumulate).
// heavy/n_heavy: rows of A handled by the split-row kernel (nnz > kHeavyRowNnz).
template <class VT>
void spmm(const Csr& A, const int32_t* heavy, int64_t n_heavy, double alpha,
          const VT* X, int64_t ldx, double gamma, const VT* Z, int64_t ldz, VT* Y,
          int64_t ldy, int b, const VT* V, int64_t ldv, double* dots, cudaStream_t s,
          const SpmmCfg* cfg = nullptr);

// Fused Chebyshev step for (I - beta A) x = b (FP32), with x_k = sx * Xk and
// x_{k-1} = sp * Xprev:
//   x_{k+1} = x_k + ak (x_k - x_{k-1}) + ck (b - x_k + beta A x_k)
// Xk != Xout; Xprev null means x_{k-1} = 0; Xprev may equal Xout.
void cheb_step(const Csr& A, double beta, double ak, double ck, const float* Xk,
               const float* Xprev, const float* B, float* Xout, int64_t ld, int b, cudaStream_t s,
               const SpmmCfg* cfg = nullptr, double sx = 1.0, double sp = 1.0);

// The same step with iterates in FP32 rows or in the split form (two BF16
// planes hi = bf16(x), lo = bf16(x - hi) in an FP32-sized rows x ld buffer,
// lo starting at element rows * ld).  in_mode: 0 FP32 Xk; 1 split Xk whose
// product gathers hi alone; 2 split Xk gathered as hi + lo.  prev_mode: 0
// none (Xprev null), 1 FP32, 2 split.  out_split: write x_{k+1} split.
// tm_mask bits 1, 2, 4: Xk, Xprev, Xout are tile-major (FP32 only, b > 128,
// ld % 8 == 0): column tile t (256 columns) of row i at (t * rows + i) * 256,
// the buffer holding ceil(b / 256) * 256 columns per row.
void cheb_step_ex(const Csr& A, double beta, double ak, double ck, const void* Xk, int in_mode,
                  const void* Xprev, int prev_mode, const float* B, void* Xout, int out_split,
                  int64_t ld, int b, cudaStream_t s, const SpmmCfg* cfg = nullptr,
                  double sx = 1.0, double sp = 1.0, int tm_mask = 0);

// dots[c] += sum_{i<len} A[i,c] * B[i,c]
template <class VT>
void coldot(const VT* A, int64_t lda, const VT* B, int64_t ldb, int64_t len, int b,
            double* dots, cudaStream_t s);

// Column state of a multi-RHS (P)CG: per column c
//   rz[c]   = r^T z of the current iterate (FP64), pq[c] = p^T A p,
//   rz_new  = accumulation target of the next r^T z, rr = ||r||^2,
//   thr2[c] = squared stopping threshold on ||r||_2, active[c] in {0,1},
//   iters[c] = iterations taken, flags: bit0 breakdown (p^T A p <= 0).
struct ColState {
  double* rz = nullptr;
  double* pq = nullptr;
  double* rz_new = nullptr;
  double* rr = nullptr;
  double* thr2 = nullptr;
  int* active = nullptr;
  int* iters = nullptr;
  int* flags = nullptr;
  int* n_active = nullptr;  // single counter
};

// X += a P, R -= a Q with a[c] = rz[c]/pq[c] on active columns; when
// `acc_rr` accumulates rr[c] += ||R[:,c]||^2 (plain CG: z = r).
template <class VT>
void cg_update_xr(VT* X, const VT* P, VT* R, const VT* Q, int64_t ld, int64_t len, int b,
                  const ColState& st, bool acc_rr, cudaStream_t s);

// P = Z + (rz_new/rz) P on active columns (Z may equal R for plain CG).
template <class VT>
void cg_update_p(VT* P, const VT* Z, int64_t ld, int64_t len, int b, const ColState& st,
                 cudaStream_t s);

// One-block kernels on the column state.
// After pq is reduced: flag breakdown (pq <= 0 on an active column).
void colstate_check_pq(const ColState& st, int b, cudaStream_t s);
// After rz_new / rr are reduced: iters++, rz <- rz_new, active <- rr > thr2,
// n_active <- count; rz_new, pq, rr zeroed for the next iteration.
// `keep_rz` leaves rz unchanged (the p-update still needs the old value) and
// instead finishes with colstate_rotate.
void colstate_advance(const ColState& st, int b, cudaStream_t s);
void colstate_rotate(const ColState& st, int b, cudaStream_t s);

// Y = a*X (+ Y if accumulate); X, Y len x b with their own ld.
template <class VT>
void scale_copy(const VT* X, int64_t ldx, VT* Y, int64_t ldy, int64_t len, int b, double a,
                bool accumulate, cudaStream_t s);

// Y(double) += X(float) ; or convert between precisions.
void add_f32_to_f64(const float* X, int64_t ldx, double* Y, int64_t ldy, int64_t len, int b,
                    cudaStream_t s);
void convert_f64_to_f32(const double* X, int64_t ldx, float* Y, int64_t ldy, int64_t len, int b,
                        cudaStream_t s);
void convert_f32_to_f64(const float* X, int64_t ldx, double* Y, int64_t ldy, int64_t len, int b,
                        cudaStream_t s);

// Gather/scatter rows between node order and index order:
//   Y[i,:] = X[map[i],:]   (gather, i < len)
template <class VT>
void gather_rows(const VT* X, int64_t ldx, const int32_t* map, VT* Y, int64_t ldy, int64_t len,
                 int b, cudaStream_t s);

// RHS of Eq. 3: B[:, j] = beta * W e_{q_j} placed at rows pos[W-neighbour]
// (pos = iperm for index order, or null for node order).  B must be zeroed.
template <class VT>
void build_rhs(const Csr& W, const int32_t* q, int b, double beta, const int32_t* pos, VT* B,
               int64_t ldb, cudaStream_t s);

// Per-column squared norms (FP64) and max-abs of B (for the stopping rule).
template <class VT>
void col_norms(const VT* B, int64_t ld, int64_t len, int b, double* norm2, double* maxabs,
               cudaStream_t s);

// thr2[c] = (tol * base[c])^2 where base = sqrt(norm2) or maxabs*(1-c).
void make_thresholds(const double* norm2, const double* maxabs, int b, double tol, int kind,
                     double one_minus_c, double* thr2, cudaStream_t s);

// Dense M11 block solve: Y_blk = Minv_blk X_blk for every block of one size
// class.  inv: [count][S][S] row-major (zero padded); start[count] first
// row of each block; size[count] its true size (<= S).
template <class VT>
void block_solve(const VT* inv, const int64_t* start, const int32_t* size, int64_t count, int S,
                 const VT* X, int64_t ldx, VT* Y, int64_t ldy, int b, cudaStream_t s);

// C (MxN) = alpha * op(A) B + beta * C, row-major; op(A) = A (MxK, lda) or
// A^T with A stored KxM (transA).  B KxN (ldb), C ldc.  SIMT FP32/FP64.
template <class VT>
void gemm(bool transA, int64_t M, int64_t N, int64_t K, double alpha, const VT* A, int64_t lda,
          const VT* B, int64_t ldb, double beta, VT* C, int64_t ldc, cudaStream_t s);

}  // namespace katz
