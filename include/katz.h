/*
 * katz.h - C ABI of the GB300 Katz-query library (libkatz.so).
 *
 * The library answers Katz proximity queries on an undirected graph
 * (Coskun, Baggag, Koyuturk, "Fast Computation of Katz Index for Efficient
 * Processing of Link Prediction Queries"):
 *
 *     K = sum_{l>=1} beta^l W^l = (I - beta W)^{-1} - I        (Eqs. 1-2)
 *     k_q = column q of K solves  M k_q = beta W e_q,  M = I - beta W  (Eq. 3)
 *
 * with the paper's LRC-Katz method (block partition of M, Lemma 1, Eqs.
 * 4-7, low-rank corrected Schur preconditioner Eq. 14, Algorithms 1-2) and,
 * as the comparison method, plain conjugate gradients on M.  The paper's
 * damping factor alpha is written beta here and its adjacency G is W.
 *
 * Conventions for every entry point
 *   - Return value: KATZ_OK (0) or one of the KATZ_E* codes below.  No call
 *     aborts the process; katz_last_error() gives a one-line reason for the
 *     last failure on the calling thread.
 *   - Graph arrays passed to katz_index_build are host pointers; the index
 *     copies them and owns all device memory it allocates.
 *   - Vector/matrix arguments marked "host or device" may be either; the
 *     library inspects the pointer.  Host buffers are staged through device
 *     memory owned by the index (pinned host memory copies fastest).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All work is issued on it; every call returns only after its
 *     results are complete and visible to the host and to later work on
 *     that stream.
 *   - Dense n x b blocks (one column per query) are NODE-MAJOR: entry
 *     (node i, query j) is at X[i*ld + j], ld >= b.
 *   - An index is not thread safe: calls on one index must not overlap.
 */
#ifndef KATZ_H
#define KATZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define KATZ_OK 0
#define KATZ_EINVAL 1  /* bad argument: malformed/asymmetric CSR, query id out of range, b <= 0 */
#define KATZ_ENOTSPD 2 /* beta * lambda_max >= 1 detected: M is not positive definite (Section 3.1) */
#define KATZ_ENOCONV 3 /* an iteration or refinement cap was hit; outputs and stats are still filled */
#define KATZ_ENOMEM 4  /* a device or host allocation failed */
#define KATZ_ECUDA 5   /* a CUDA runtime error */

/* ---- element types ---- */
#define KATZ_UNIT 0 /* values: pattern only, every stored weight is exactly 1 */
#define KATZ_F64 1
#define KATZ_F32 2
#define KATZ_BF16 3

/* ---- query precision modes ---- */
#define KATZ_PREC_F32 0   /* FP32 solve only (no refinement) */
#define KATZ_PREC_MIXED 1 /* FP32 inner solves + FP64 residual iterative refinement */
#define KATZ_PREC_F64 2   /* every vector and reduction in FP64 (reference speed path) */

/* ---- stopping criteria ---- */
/* Kernel of the wide fused sparse products (KATZ_PREC_MIXED and F32 paths):
 * AUTO uses what katz_autotune measured faster for the operator and width
 * (the register kernel if untuned); REGISTER: warp-per-row register
 * gathers; PIPELINED: TMA bulk-copy gathers into a shared-memory ring
 * (used where applicable: padded width >= 64, weights unit/FP32/BF16). */
#define KATZ_GATHER_AUTO 0
#define KATZ_GATHER_REGISTER 1
#define KATZ_GATHER_PIPELINED 2
#define KATZ_GATHER_ROWPIPE 3 /* the row-pipelined register kernel for the Chebyshev steps
                                 (FP32 iterates, b > 128; each warp fetches the next row's
                                 indices and this row's own operands during this row's
                                 gathers), the register kernel elsewhere */
#define KATZ_GATHER_CHUNKED 4 /* the register kernels of the Chebyshev steps and of the
                                 refinement residual with each CTA taking a contiguous run of
                                 rows (the tuned run lengths, else 64 rows) */

/* Gathers of the Chebyshev steps on the large M11 blocks (KATZ_PREC_MIXED
 * and F32 paths).  F32: FP32 iterates and FP32 gathers.  The other modes
 * keep the iterates as two BF16 planes hi = bf16(x), lo = bf16(x - hi)
 * (FP32 storage size, x to 2^-18 relative), so that a step's product can
 * gather the hi plane alone: half the bytes per gathered row, at ~2^-9
 * relative error per gathered term.  BF16: hi-plane gathers on every step
 * after the first; MIXED: the same, except that the last step of a solve
 * asked for a tolerance below 1e-4 gathers hi + lo.  AUTO: FP32 iterates,
 * the intermediate ones stored tile-major (each 256-column tile's rows
 * contiguous) for batches wider than 128 columns. */
#define KATZ_CHEB_AUTO 0
#define KATZ_CHEB_F32 1
#define KATZ_CHEB_BF16 2
#define KATZ_CHEB_MIXED 3

#define KATZ_TOL_RESIDUAL 0  /* stop column j when ||b_j - M k_j||_2 <= tol * ||b_j||_2 */
#define KATZ_TOL_ERROR_INF 1 /* stop when ||b_j - M k_j||_2 <= tol * (1 - beta*lambda) * ||b_j||_inf,
                                lambda a rigorous upper bound on lambda_max (katz_lambda_bounds),
                                which guarantees ||k_j - k_j*||_inf <= tol * ||k_j*||_inf for
                                non-negative weights (||M^{-1}||_2 <= 1/(1 - beta*lambda),
                                k* >= b >= 0) */

typedef struct katz_index katz_index; /* opaque; owns all device memory of one graph */

/* Symmetric CSR adjacency W of an undirected graph, HOST pointers.
 * rowptr[n+1] (int64, rowptr[0] = 0, non-decreasing), col[nnz] (int32 in
 * [0, n), no self-loops, W symmetric with equal weights both ways), val[nnz]
 * weights (> 0) or NULL for unit weights. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
} katz_csr;

typedef struct {
  int32_t value_dtype;   /* storage of W values on the device: KATZ_UNIT/F64/F32/BF16
                            (values are rounded to nearest-even; UNIT requires all ones) */
  int32_t build_lrc;     /* 0: graph only (CG queries); 1: also the LRC-Katz index (Algorithm 1) */
  int32_t rank;          /* r: number of eigenpairs of R kept (Eq. 14); 0 allowed */
  int32_t n_hubs;        /* highest-degree nodes forced into the separator */
  int32_t block_max;     /* largest M11 diagonal block stored as a dense inverse */
  int32_t split;         /* 1: split components larger than block_max by BFS level sets;
                            0: keep them whole (their M11 block is solved iteratively) */
  int32_t lanczos_steps; /* Lanczos steps on R; 0 = max(2r, r+20) */
  int32_t n2_max;        /* largest separator whose Schur complement S is stored dense
                            (0 = 16384).  Larger separators (up to 49,152 nodes) apply S
                            implicitly in each PCG iteration, S P = M22 P - M12^T M11^{-1}
                            (M12 P) with one M11 solve (Lemma 1); M22^{-1} stays dense */
  uint64_t seed;         /* SplitMix64 seed of the Lanczos start vector */
  int32_t coupling_gemm; /* store beta*M11^{-1} W12 (n1 x n2, TF32 hi/lo parts) so that LRC
                            queries form K1 = Y1 + beta M11^{-1} W12 K2 (Eq. 6) on the tensor
                            cores instead of a second M11 solve when that is cheaper:
                            0 = when it fits in a third of device memory, 1 = always,
                            -1 = never */
  int32_t rhs_coupling;  /* store Z = beta M11^{-1} W12 (n1 x n2, FP32; the build solves for
                            it anyway to form S) so that the first Schur right-hand side of a
                            query, F = B2 - M12^T M11^{-1} B1 = B2 + Z^T B1 (Eq. 7, M11
                            symmetric), is gathered from the deg(q) rows of Z that the sparse
                            B1 = beta W e_q touches instead of costing an M11 solve of the
                            whole n1 x b block: 0 = where M11 has blocks solved iteratively,
                            S is dense and Z fits in a quarter of device memory, 1 = always
                            (single graph, dense S), -1 = never */
} katz_build_opts;

typedef struct {
  double tol;          /* see tol_kind */
  int32_t tol_kind;    /* KATZ_TOL_RESIDUAL or KATZ_TOL_ERROR_INF */
  int32_t precision;   /* KATZ_PREC_* */
  int32_t max_iter;    /* cap on iterations of each inner CG / PCG solve (0 = 2000) */
  int32_t max_refine;  /* cap on FP64 refinement steps (0 = 12) */
  int32_t rhs_width;   /* columns solved together: the b queries are solved in chunks of
                          rhs_width columns, one after another, each written to its own
                          column range of K_out (0 = all b at once).  At most 1,024
                          columns are solved together, so b > 1,024 needs
                          1 <= rhs_width <= 1,024; negative -> KATZ_EINVAL.  With
                          chunks, katz_stats holds the maxima of iters, refine_steps
                          and max_rel_res over the chunks, the sums of ms[0..5], the
                          column-weighted mean of ms[6] and the maximum of ms[7] */
  int32_t warm_start;  /* 1: start from the learned warm start (needs a trained network; mixed
                          precision): LRC starts its Schur PCG from K2 = W_r c_hat; CG on M
                          starts from the whole vector [M11^{-1} B1 + beta M11^{-1} W12 W_r
                          c_hat; W_r c_hat], each column scaled to its energy-optimal multiple
                          gamma = b^T x / x^T M x (zero if that is not positive) */
  int32_t gather_kernel; /* KATZ_GATHER_*: kernel of the wide sparse products (Chebyshev
                            steps of the large M11 blocks, refinement residual) */
  int32_t cheb_gather;   /* KATZ_CHEB_*: precision of the Chebyshev steps' gathers */
} katz_query_opts;

typedef struct {
  int32_t iters;        /* inner iterations summed over refinement steps (max over columns) */
  int32_t refine_steps; /* FP64 residual evaluations performed */
  double max_rel_res;   /* max_j ||b_j - M k_j||_2 / ||b_j||_2 of the returned K (FP64) */
  double ms[8];         /* [0] total ms, [1] RHS ms, [2] first inner solve ms, [3] residual ms,
                           [4] CUDA-graph replays (multi-graph), [5] warm-start fallbacks
                           (columns started from zero), [6] mean scale of the CG warm
                           start's guesses, [7] 1 when the first Schur right-hand side
                           came from the stored Z (rhs_coupling) instead of an M11 solve */
} katz_stats;

typedef struct {
  int64_t n, nnz, n1, n2;
  int32_t n_blocks, n_large_blocks, rank, value_dtype;
  double beta;
  double lambda_max_R; /* largest Ritz value sigma_1 of R (0 if rank 0) */
  int64_t device_bytes;
  double lambda_max_W; /* largest Lanczos Ritz value of W (a lower bound on lambda_max) */
  double lambda_upper; /* rigorous upper bound on lambda_max of W (Collatz-Wielandt); the SPD
                          check and the KATZ_TOL_ERROR_INF rule use it */
  int32_t schur_implicit; /* 1: the separator exceeds n2_max and S is applied implicitly */
  int32_t rhs_coupling;   /* 1: Z = beta M11^{-1} W12 is stored (see katz_build_opts) */
} katz_index_info;

/* ---------------------------------------------------------------- graph */

/* Largest eigenvalue lambda_max of the symmetric W (= ||W||_2 for W >= 0),
 * the bound of Section 3.1 (beta < 1/||W||_2), by FP64 Lanczos on the GPU
 * (`steps` iterations, 0 = 64).  W is host CSR as above.  *out receives
 * the largest Ritz value, an estimate from below.  Errors: KATZ_EINVAL on
 * a malformed CSR. */
int katz_lambda_max(const katz_csr* W, int32_t steps, double* out, void* stream);

/* Both sides of lambda_max of W (host CSR, weights > 0) after `steps`
 * Lanczos steps (0 = 64): *ritz (may be NULL) the largest Ritz value, which
 * never exceeds lambda_max, and *upper (may be NULL) a rigorous upper
 * bound, max_i (W x)_i / x_i for the positive vector x = |y| + f max|y| of
 * the top Ritz vector y (the Collatz-Wielandt bound for W >= 0; the
 * smallest over a few floors f, each valid).  The index build refuses beta
 * unless beta * upper < 1 (M certified positive definite, Section 3.1),
 * and the KATZ_TOL_ERROR_INF stopping rule uses 1 - beta * upper as the
 * lower bound on the smallest eigenvalue of M.  Errors: KATZ_EINVAL. */
int katz_lambda_bounds(const katz_csr* W, int32_t steps, double* ritz, double* upper,
                       void* stream);

/* Build the query index for damping `beta` (Algorithm 1, "Preprocess").
 * Always: validates W (CSR shape, symmetry), uploads it.  With
 * opts->build_lrc: partitions and reorders M (Section 3.2, Steps 2-3;
 * project reading: hubs + BFS level-set separators), inverts the M11
 * diagonal blocks (Step 4: Cholesky, then the inverse), forms M12, M22,
 * the dense Schur complement S = M22 - M12^T M11^{-1} M12 (Lemma 1),
 * M22^{-1} (blocked Gauss-Jordan), and the top `rank` eigenpairs of
 * R = L^{-1} M12^T M11^{-1} M12 L^{-T} (Eqs. 8-11, M22 = L L^T).  R is
 * similar to M22^{-1} T (T = M12^T M11^{-1} M12), so Lanczos runs on that
 * operator in the M22 inner product; its Ritz vectors are W_r = L^{-T} U_r
 * directly and L is never formed.  Stored: W_r D^{1/2}, D = diag(sigma/(1-sigma)).
 * lambda_max is measured at build; beta*lambda_max >= 1 -> KATZ_ENOTSPD.
 * On success *out owns the index (free with katz_index_free). */
int katz_index_build(const katz_csr* W, double beta, const katz_build_opts* opts,
                     void* stream, katz_index** out);

void katz_index_free(katz_index* idx);

/* Persist a built index (the stored artefact of Algorithm 1, Section 3.2)
 * to a file and read it back, so that queries can be served without
 * repeating the partition, the block inverses, the Schur complement and the
 * Lanczos low-rank correction.  The file holds every stored field: graph
 * and reordered blocks, M11 block inverses, M12, S, M22^{-1}, W_r D^{1/2},
 * sigma, beta, lambda_max, the autotuned launch shapes and the warm-start
 * network with its optimiser state.  Format: versioned little-endian
 * records with per-field tags and a checksum.
 * katz_index_save: waits for all device work, then writes `path` (host
 *   string; an existing file is replaced; a partial file is removed on
 *   failure).  KATZ_EINVAL if the file cannot be written.
 * katz_index_load: allocates a new index on the current device and fills
 *   it from `path`; *out owns it (free with katz_index_free).  Queries on
 *   the loaded index run exactly as on the saved one.  KATZ_EINVAL for a
 *   missing, truncated, corrupt (checksum), foreign (magic) or other-version
 *   file; *out is NULL on failure. */
int katz_index_save(const katz_index* idx, const char* path);
int katz_index_load(const char* path, katz_index** out);

int katz_index_get_info(const katz_index* idx, katz_index_info* info);

/* Copy the partition (host outputs): perm[n] (perm[new] = old node),
 * block_ptr[n_blocks+1].  Either pointer may be NULL. */
int katz_index_get_partition(const katz_index* idx, int64_t* perm, int64_t* block_ptr);

/* The partition alone (Section 3.2, Steps 2-3; project reading: the
 * n_hubs highest-degree nodes plus, when `split`, BFS median-level
 * separators of components larger than block_max).  Host-only: runs no GPU
 * code.  perm[n] (perm[new] = old node), block_ptr[n+1] (host, caller
 * owned; entries after the last block are untouched), *n_blocks and *n1
 * receive the block count and the number of non-separator nodes. */
int katz_partition(const katz_csr* W, int32_t n_hubs, int32_t block_max, int32_t split,
                   int64_t* perm, int64_t* block_ptr, int64_t* n_blocks, int64_t* n1);

/* Copy the kept Ritz values sigma_1 >= ... >= sigma_r of R (host, rank). */
int katz_index_get_sigma(const katz_index* idx, double* sigma);

/* ---------------------------------------------------------------- queries */

/* Katz vectors of b query nodes by LRC-Katz (Algorithm 2 with Lemma 1):
 * RHS b_j = beta W e_{q_j} (Eq. 3); F = B2 - M12^T M11^{-1} B1 (Eq. 7); PCG
 * on S K2 = F preconditioned by S~^{-1} = M22^{-1} + W_r D W_r^T (Eq. 14);
 * K1 = M11^{-1}(B1 - M12 K2) (Eq. 6); merge and un-permute.  With
 * KATZ_PREC_MIXED the LRC solve runs in FP32 and FP64-class residuals of the
 * full system (float-float, ~2^-48 relative to their terms; FP64 for
 * FP64-valued graphs) drive iterative refinement until opts->tol is met.
 * q[b]: int32 node ids (host or device); b <= 1,024 unless opts->rhs_width
 * splits the batch into chunks of at most 1,024.  K_out: n x b node-major, ld = ldk,
 * element type out_dtype (KATZ_F32 or KATZ_F64), host or device.
 * stats may be NULL; iters_out[b] / rel_res_out[b] (host, may be NULL)
 * receive per-column iteration counts and the relative residuals
 * ||b_j - M k_j||_2 / ||b_j||_2 of the returned K (NaN with KATZ_PREC_F32,
 * which evaluates no residual).  Needs an index built with build_lrc = 1. */
int katz_query_batch(const katz_index* idx, const int32_t* q, int32_t b,
                     const katz_query_opts* opts, void* K_out, int32_t out_dtype,
                     int64_t ldk, katz_stats* stats, int32_t* iters_out,
                     double* rel_res_out, void* stream);

/* Same contract, solved by plain multi-RHS conjugate gradients on M (the
 * comparison method of Sections 1 and 4) from a zero initial guess, or,
 * with opts->warm_start = 1 on an index with a trained warm-start network,
 * from the network's whole-vector guess described at katz_query_opts.
 * An index built without the LRC part serves this call alone. */
int cg_query_batch(const katz_index* idx, const int32_t* q, int32_t b,
                   const katz_query_opts* opts, void* K_out, int32_t out_dtype,
                   int64_t ldk, katz_stats* stats, int32_t* iters_out,
                   double* rel_res_out, void* stream);

/* Katz link prediction (Section 3.3): for each query column j of K (n x b
 * node-major, ld = ldk, k_dtype KATZ_F32 or KATZ_F64, device or host),
 * rank every node except q_j and its neighbours by K[:, j] descending, ties
 * by node id ascending, and write the first `k` ids (int32) and scores
 * (double) to ids_out[b*k] / scores_out[b*k] (host or device, row j =
 * query j).  Missing candidates get id -1, score 0.  k <= 64. */
int linkpred_topk(const katz_index* idx, const int32_t* q, int32_t b,
                  const void* K, int32_t k_dtype, int64_t ldk, int32_t k,
                  int32_t* ids_out, double* scores_out, void* stream);

/* Sparse-Katz link prediction (Algorithm 3, Section 3.3, Fig. 2) for b
 * queries q (host or device, 1 <= b <= 1024):
 *   1. k_q by LRC-Katz (plain CG if the index has no LRC part), with the
 *      accuracy that *opts asks for (as katz_query_batch);
 *   2. the Top-s list: the s highest k_q[j] over j outside {q} and q's
 *      neighbours (the linkpred_topk list);
 *   3. the T landmarks: the T highest k_q[j] over j != q (neighbours
 *      included), and their Katz vectors k_t, the columns of K_T (one solve
 *      per DISTINCT landmark of the batch, batched up to 1,024 columns);
 *   4. rho_c = Pearson correlation of row q and row c of K_T (the
 *      T-vectors (k_t[q])_t and (k_t[c])_t), in FP64; 0 when either row is
 *      constant (always when T = 1);
 *   5. the Top-s list re-ordered by rho descending, ties in Katz order.
 * Scores are compared in FP32 (the stored Katz vectors) for the selections
 * of steps 2-3, score descending and node id ascending.
 * Outputs (host or device, row j = query j): ids_out[b*s] re-ranked
 * candidates (-1 at the tail when fewer than s exist), rho_out[b*s] their
 * correlations (0 for -1), landmarks_out[b*T] (may be NULL) the landmarks
 * in Katz order.  1 <= s, T <= 64 and T < n, else KATZ_EINVAL.  stats (may
 * be NULL): iterations, refinement steps and residual as the maximum over
 * all the solves of the call, ms[0] its wall time, ms[6] the number of
 * distinct landmarks solved.  KATZ_ENOCONV if any
 * solve hit its cap (outputs still filled). */
int sparse_katz_topk(const katz_index* idx, const int32_t* q, int32_t b, int32_t s, int32_t T,
                     const katz_query_opts* opts, int32_t* ids_out, double* rho_out,
                     int32_t* landmarks_out, katz_stats* stats, void* stream);

/* linkpred_topk without any device allocation.  The paper has no
 * counterpart: this serves callers that must not allocate device memory
 * while they run -- a serving loop whose latency budget has no room for an
 * allocation (cudaMalloc may synchronise the device), or a process whose
 * device memory is already reserved by another framework's caching
 * allocator, so that a fresh cudaMalloc would fail although the caller's
 * own buffers are in place.  Same arguments and results as linkpred_topk,
 * except that q, K, ids_out and scores_out must all be DEVICE pointers.
 * The candidate lists live in a fixed scratch array inside the library
 * (3 MiB per GPU that loads the library, held until the process exits)
 * that holds up to 2^18 entries: b * k must not exceed 32,768, else
 * KATZ_EINVAL.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  The first call on each device looks up the scratch array's
 * device address (cudaGetSymbolAddress, with that device current), so make
 * that first call before any stream capture.  The call copies the query
 * ids to the host to check them and synchronises `stream` before its
 * kernels and again when they are done.  All calls share the one scratch
 * array (it keeps the last call's contents): calls that overlap on the
 * GPU -- on different streams or threads -- race and must be serialised by
 * the caller. */
int linkpred_topk_noalloc(const katz_index* idx, const int32_t* q, int32_t b, const void* K,
                          int32_t k_dtype, int64_t ldk, int32_t k, int32_t* ids_out,
                          double* scores_out, void* stream);

/* Y = M X = X - beta W X for n x b node-major blocks in node order
 * (X, Y device pointers, ld = b, dtype KATZ_F32 or KATZ_F64).  The sparse
 * product of Eq. 3, exposed for step-level testing. */
int katz_apply_M(const katz_index* idx, const void* X, void* Y, int32_t b,
                 int32_t dtype, void* stream);

/* Autotuner: times the candidate launch shapes of the multi-RHS CSR
 * product (columns per warp-row tile in {128..1024} x CTAs per SM in
 * {2..64}) on the index's operators for right-hand-side width b, keeps the
 * fastest per operator for later queries with that b, and caches the
 * choice per (rows, nnz, b, value type) in the process; for the fused
 * kernels (the large-block Chebyshev step, the refinement-residual pass)
 * it times their own grids (CTAs per SM in {8..128}); on the large-block
 * operator it also chooses between the register and the pipelined (TMA
 * bulk-copy) Chebyshev step, and on the full operators between the two
 * kernels of the first and of the later refinement-residual passes.
 * out (11 ints): out[0] = chosen column tile (0 = default), out[1] = CTAs
 * per SM, out[2] = 1 if the pipelined Chebyshev step was chosen, out[3] /
 * out[4] = 1 if the pipelined kernel was chosen for the first / later
 * residual passes of LRC queries, out[5] / out[6] = CTAs per SM of the
 * Chebyshev step / of the residual pass (0 if not tuned), out[7] = rows
 * the Chebyshev step gathers together per lane (0: the compiler's
 * schedule, 4 or 8), out[8] = 1 if the row-pipelined Chebyshev kernel (the
 * next row's indices and this row's own operands fetched during this
 * row's gathers) was chosen, out[9] = rows per CTA of the Chebyshev step
 * when each CTA takes a contiguous run of rows (0: its warps stride over
 * all rows), out[10] = rows per CTA of the refinement-residual passes in
 * the same sense; ms[0] = best
 * time, ms[1] = time of the default shape (per product, FP32 vectors). */
int katz_autotune(katz_index* idx, int32_t b, int32_t* out, double* ms, void* stream);

/* D = A * B^T on the tcgen05 tensor cores (BF16 operands, FP32
 * accumulation in tensor memory): the kernel used for the rank-r
 * correction products W^ (W^T R) of the preconditioner (Eq. 14), exposed
 * for step-level testing.  A (M x K) and B (N x K) are device BF16
 * row-major with K contiguous, row strides lda/ldb multiples of 8 elements,
 * 16-byte aligned.  C (device FP32, M x N, ldc) = alpha*D + beta*C.
 * Errors: KATZ_EINVAL on bad shapes/alignment, KATZ_ECUDA if the pipeline
 * reported a timeout. */
int katz_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, int32_t M, int32_t N,
                   int32_t K, float alpha, float beta, float* C, int64_t ldc, void* stream);

/* Test hook (no GPU fault is involved): while `on` is non-zero, the
 * rank-r tensor-core GEMM (katz_gemm_bf16 and the preconditioner products)
 * issues no TMA copy, so the wait of its MMA-issuing thread on the first
 * pipeline stage runs out after its bounded spin (about two seconds) with
 * nothing in flight; the kernel releases its tensor memory and reports the
 * timeout, and the call returns KATZ_ECUDA.  Switch it off again (on = 0)
 * for normal work; the library and the CUDA context stay usable.
 * Process-wide.  Always returns KATZ_OK. */
int katz_test_stall_copies(int32_t on);

/* FP32-accurate tensor-core product C = alpha * A B^T + beta * C from three
 * TF32 tcgen05 products of the TF32 high/low parts of A and B (the kernel of
 * the coupling product K1 = Y1 + beta M11^{-1} W12 K2), exposed for
 * step-level testing.  A (M x K), B (N x K), C (M x N): device FP32
 * row-major, row strides lda/ldb multiples of 4 elements, 16-byte aligned.
 * Errors: KATZ_EINVAL on bad shapes/alignment, KATZ_ENOMEM, KATZ_ECUDA if
 * the pipeline reported a timeout. */
int katz_gemm_tf32x3(const float* A, int64_t lda, const float* B, int64_t ldb, int32_t M,
                     int32_t N, int32_t K, float alpha, float beta, float* C, int64_t ldc,
                     void* stream);

/* ------------------------------------------------- learned warm start */

typedef struct {
  int32_t hidden;       /* hidden width (256) */
  int32_t epochs;       /* passes over the training queries */
  int32_t batch;        /* minibatch rows */
  float lr;             /* AdamW learning rate */
  float weight_decay;   /* AdamW decoupled weight decay */
  uint64_t seed;        /* SplitMix64 seed of the initial weights and the row order */
} katz_train_opts;

typedef struct {
  double initial_loss, final_loss; /* MSE of the first minibatch / whole training set */
  int32_t steps;                   /* AdamW steps taken */
  double ms;                       /* wall time (target solves + training) */
} katz_train_stats;

/* Train the warm-start network on Katz vectors the method itself computes.
 * For each training query q (host ids, n_train of them) the LRC solve gives
 * k_q; the target is c* = W_r^T M22 k2 (the M22-orthogonal coordinates of
 * the separator part in the Lanczos basis W_r, W_r^T M22 W_r = I).  Input
 * features (32): degree / mean degree, log(1 + degree) (standardised) and
 * 30 spectral coordinates (row of W_r for separator nodes, of
 * beta M11^{-1} W12 W_r otherwise; unit RMS per column).  Network: 32 ->
 * hidden (exact GELU) -> r, BF16 weights, FP32 accumulation and FP32
 * master weights, MSE loss, AdamW.  Afterwards katz_query_batch with
 * opts->warm_start = 1 starts the Schur PCG from K2 = W_r MLP(x_q) (a
 * column whose warm residual is not below ||F|| starts from zero instead),
 * and cg_query_batch with opts->warm_start = 1 starts CG on M from the
 * guess's extension to the whole vector (see katz_query_opts). */
int katz_warmstart_train(katz_index* idx, const int32_t* q_train, int32_t n_train,
                         const katz_train_opts* opts, katz_train_stats* stats, void* stream);

/* One forward/backward of the warm-start network on device data, for
 * gradient checks.  X (m x din), T (m x dout) FP32; params FP32 in the
 * layout W1 (dh x din), b1 (dh), W2 (dout x dh), b2 (dout) -- the weights
 * are rounded to BF16 as in training; grads (same layout) receive the
 * gradients of the mean squared error 0.5/m * ||Y - T||^2, *loss its value. */
int katz_mlp_loss_grad(int32_t m, int32_t din, int32_t dh, int32_t dout, const float* X,
                       const float* T, const float* params, float* grads, double* loss,
                       void* stream);

/* ------------------------------------------------- many graphs at once */

typedef struct katz_multi katz_multi; /* opaque; g independent graphs */

/* Index g independent graphs of uneven size for batched queries.  Ws[g]:
 * host CSRs as for katz_index_build; betas[g]: each graph's damping.  The
 * graphs are stored as one block-diagonal CSR; lambda_max of every graph is
 * measured and beta_g * lambda_g >= 1 gives KATZ_ENOTSPD.  value_dtype:
 * KATZ_UNIT, KATZ_F32 or KATZ_BF16 (weights exact in FP32). */
int katz_multi_build(int32_t g, const katz_csr* Ws, const double* betas, int32_t value_dtype,
                     void* stream, katz_multi** out);

void katz_multi_free(katz_multi* m);

/* The same g graphs with a per-graph LRC index (Algorithm 1 on every graph
 * at once).  The graphs form one block-diagonal graph whose weights carry
 * each graph's damping (W~ = beta_g W_g on graph g's block, beta = 1), so
 * M = I - W~ and its Schur complement are block diagonal:
 *   - rank target r_g per graph, log-scaled from opts->rank / 4 (smallest
 *     graph) to opts->rank (largest; 0 = 32; at most 64);
 *   - separator: each graph's own highest-degree nodes (ties: smaller id),
 *     max(1, round(opts->n_hubs * n_g / sum n), 2 r_g) of them, at most 256
 *     and n_g - 1 (opts->n_hubs = 0: min(8192, sum n / 1000), at least g);
 *     every other component is an M11 block (dense inverse, or Chebyshev if
 *     larger than block_max);
 *   - S_g for all graphs from one column-packed M11 solve (separator node l
 *     of every graph shares column l); S_g, M22_g^{-1} and W^_g are stored
 *     block by block (one dense block per graph, no union-wide array);
 *   - rank r_g = min(target, separator): Lanczos on every graph's block at
 *     once with per-graph scalars.
 * opts->value_dtype: KATZ_UNIT, KATZ_F32 or KATZ_BF16 (as katz_multi_build;
 * the index stores the scaled weights in FP32).  opts->split,
 * lanczos_steps, seed as for katz_index_build; n2_max is raised to the
 * separator size.  Both katz_multi_query (CG) and katz_multi_query_lrc run
 * on the result.  KATZ_ENOTSPD if some beta_g * lambda_g >= 1. */
int katz_index_build_many(int32_t g, const katz_csr* Ws, const double* betas,
                          const katz_build_opts* opts, void* stream, katz_multi** out);

/* Per-graph shape of an index from katz_index_build_many (host outputs, any
 * may be NULL): n2_out[g] separator size, ranks_out[g] rank r_g,
 * sigma_out[sum r_g] the Ritz values of R_g (Eq. 11), graph-major,
 * descending within a graph.  KATZ_EINVAL without the LRC part. */
int katz_multi_get_info(const katz_multi* m, int64_t* n2_out, int32_t* ranks_out,
                        double* sigma_out);

/* qpg queries of every graph (Eq. 3 per graph), solved together: one
 * multi-RHS CG on the block-diagonal system with per-(graph, query) CG
 * scalars and stopping, the iteration sequence captured once in a CUDA graph
 * and replayed, float-float residual refinement to opts->tol.
 * q[g*qpg]: graph-local node ids (host or device), graph-major.
 * K_out: (sum of n_g) x qpg node-major (ld = ldk), rows in graph order;
 * column j of graph g's rows is the Katz vector of graph g's j-th query.
 * iters_out / rel_res_out (host, g*qpg, may be NULL).  qpg <= 64. */
int katz_multi_query(const katz_multi* m, const int32_t* q, int32_t qpg,
                     const katz_query_opts* opts, void* K_out, int32_t out_dtype, int64_t ldk,
                     katz_stats* stats, int32_t* iters_out, double* rel_res_out, void* stream);

/* katz_multi_query with the per-graph LRC solve (Algorithm 2 per graph, all
 * graphs in every launch) as the inner solver of the same float-float
 * residual refinement and per-(graph, query) stopping.  The inner PCG on
 * the block-diagonal S keeps one set of CG coefficients per (graph, query)
 * pair, each stopping on its own rows' residual; its iterations are
 * captured once into a CUDA graph and replayed (stats->ms[4] counts the
 * replays of both inner solvers).  Same arguments and
 * outputs; iters_out counts each pair's inner PCG iterations.  KATZ_EINVAL
 * if m was not built by katz_index_build_many. */
int katz_multi_query_lrc(const katz_multi* m, const int32_t* q, int32_t qpg,
                         const katz_query_opts* opts, void* K_out, int32_t out_dtype, int64_t ldk,
                         katz_stats* stats, int32_t* iters_out, double* rel_res_out,
                         void* stream);

/* ---------------------------------------------------------- measurement */

/* Number of kernels this library has launched in this process (all calls). */
int64_t katz_launch_count(void);

/* Test hook (host-side fault injection; no GPU fault is involved): after
 * `after` more device allocations by the library, the next one fails as if
 * the device were out of memory -- no cudaMalloc is made for it -- and the
 * call in progress returns KATZ_ENOMEM after releasing what it allocated.
 * The hook then switches itself off; after < 0 switches it off at once.
 * Process-wide.  Always returns KATZ_OK. */
int katz_fault_inject_alloc(int64_t after);

/* Start (on != 0) or stop timing tagged kernel launches with CUDA events on
 * their launching stream; every call resets the totals.  Tags:
 * "spmm_f32" / "spmm_f64" (CSR products, Eq. 3 and the couplings),
 * "cheb_step" / "cheb_step_bf16g" (fused Chebyshev steps on the large M11
 * blocks), "ff_residual" (refinement-residual passes), "ff_out" (the
 * float-float solution to the output), "block_solve_f32" /
 * "block_solve_f64" (M11 blocks), "gemm_f32" / "gemm_f64" (dense Schur /
 * preconditioner products), "tc_gemm" / "tc_gemm_tf32x3" (tcgen05
 * products; the latter counts FLOPs instead of bytes), "topk" (link
 * prediction). */
int katz_profile_enable(int32_t on);

/* Totals for one tag since the last katz_profile_enable: launches, summed
 * device time in ms, and summed algorithmic bytes (CSR arrays + dense
 * operands read once + outputs written once). */
int katz_profile_read(const char* tag, int64_t* launches, double* total_ms, double* alg_bytes);

const char* katz_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KATZ_H */
