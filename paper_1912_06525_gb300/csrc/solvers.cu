// Query solvers: plain multi-RHS CG on M (the comparison method), the
// LRC-Katz solve (Lemma 1 with PCG on the Schur complement, Algorithm 2),
// and the mixed-precision driver that wraps either one in FP64 iterative
// refinement.
#include <cfloat>
#include <chrono>
#include <cmath>

#include "index.h"
#include "ff_residual.h"
#include "kernels_dense.h"
#include "tc_gemm.h"

namespace katz {

// ----------------------------------------------------------- small kernels
__global__ void colstate_init_kernel(ColState st, int b, int use_rr) {
  __shared__ int cnt;
  if (threadIdx.x == 0) { cnt = 0; *st.flags = 0; }
  __syncthreads();
  int local = 0;
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    const double r2 = use_rr ? st.rr[c] : st.rz[c];
    const int a = r2 > st.thr2[c];
    st.active[c] = a;
    st.iters[c] = 0;
    st.pq[c] = 0.0;
    st.rz_new[c] = 0.0;
    if (st.rr) st.rr[c] = 0.0;
    local += a;
  }
  atomicAdd(&cnt, local);
  __syncthreads();
  if (threadIdx.x == 0) *st.n_active = cnt;
}

// RHS norms straight from the sparse structure: b_j = beta W e_{q_j}.
template <int WT>
__global__ void rhs_norms_kernel(Csr W, const int32_t* q, double beta, double* norm2,
                                 double* maxabs) {
  const int j = blockIdx.x;
  const int64_t k0 = W.rowptr[q[j]], k1 = W.rowptr[q[j] + 1];
  double s = 0, m = 0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    double w = 1.0;
    if (WT == KATZ_F64) w = static_cast<const double*>(W.val)[k];
    else if (WT == KATZ_F32) w = static_cast<const float*>(W.val)[k];
    else if (WT == KATZ_BF16) w = __bfloat162float(static_cast<const __nv_bfloat16*>(W.val)[k]);
    const double v = beta * w;
    s += v * v;
    m = fmax(m, fabs(v));
  }
  s = warp_sum(s);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(norm2 + j, s);
    atomicMax(reinterpret_cast<unsigned long long*>(maxabs) + j,
              (unsigned long long)__double_as_longlong(m));
  }
}

// Residual correction: R[pos(i), j] += beta W[q_j, i] (adds the sparse RHS).
template <int WT>
__global__ void rhs_add_kernel(Csr W, const int32_t* q, double beta, const int32_t* pos,
                               double* R, int64_t ld) {
  const int j = blockIdx.x;
  const int64_t k0 = W.rowptr[q[j]], k1 = W.rowptr[q[j] + 1];
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    double w = 1.0;
    if (WT == KATZ_F64) w = static_cast<const double*>(W.val)[k];
    else if (WT == KATZ_F32) w = static_cast<const float*>(W.val)[k];
    else if (WT == KATZ_BF16) w = __bfloat162float(static_cast<const __nv_bfloat16*>(W.val)[k]);
    const int64_t i = W.col[k];
    const int64_t r = pos ? pos[i] : i;
    R[r * ld + j] += beta * w;
  }
}

// First Schur right-hand side of a query from the stored Z = beta M11^{-1} W12
// (Eq. 7; M11 symmetric, so M12^T M11^{-1} = -Z^T):
//   F[:, c] = B2[:, c] + Z^T B1[:, c],  B1[:, c] = beta W[q_c, :] restricted to
// the rows pos(u) < n1.  Column c reads the deg(q_c) rows of Z that B1 touches:
// the (row, weight) pairs are staged in shared memory 256 at a time (pairs of
// separator nodes become (0, 0)), then every thread adds its KP entries of
// the staged rows, four rows in flight, in FP64.  grid (b, ceil(n2 / (256 KP))).
template <int WT>
__global__ void __launch_bounds__(256) schur_rhs_from_z_kernel(
    Csr W, const int32_t* __restrict__ q, double beta, const int32_t* __restrict__ pos,
    int64_t n1, const float* __restrict__ Z, int64_t ldz, int64_t n2,
    const float* __restrict__ R2, int64_t ld, float* __restrict__ F) {
  constexpr int KP = 8;
  __shared__ int64_t srow[256];
  __shared__ double sw[256];
  const int c = blockIdx.x;
  const int64_t k0 = int64_t(blockIdx.y) * 256 * KP + threadIdx.x;
  double acc[KP];
#pragma unroll
  for (int i = 0; i < KP; ++i) acc[i] = 0.0;
  const int64_t e0 = W.rowptr[q[c]], e1 = W.rowptr[q[c] + 1];
  for (int64_t base = e0; base < e1; base += 256) {
    const int cnt = int(e1 - base < 256 ? e1 - base : 256);
    __syncthreads();
    if (threadIdx.x < cnt) {
      const int64_t e = base + threadIdx.x;
      const int64_t r = pos[W.col[e]];
      const bool in1 = r < n1;
      srow[threadIdx.x] = in1 ? r : 0;
      double w = 1.0;
      if (WT == KATZ_F64) w = static_cast<const double*>(W.val)[e];
      else if (WT == KATZ_F32) w = static_cast<const float*>(W.val)[e];
      else if (WT == KATZ_BF16) w = __bfloat162float(static_cast<const __nv_bfloat16*>(W.val)[e]);
      sw[threadIdx.x] = in1 ? beta * w : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) {
      const float* zr = Z + srow[j] * ldz;
      const double w = sw[j];
#pragma unroll
      for (int i = 0; i < KP; ++i) {
        const int64_t k = k0 + int64_t(i) * 256;
        if (k < n2) acc[i] = fma(w, double(__ldg(zr + k)), acc[i]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < KP; ++i) {
    const int64_t k = k0 + int64_t(i) * 256;
    if (k < n2) F[k * ld + c] = float(double(R2[k * ld + c]) + acc[i]);
  }
}

// T[pos(u), c] += beta W[q_c, u] for the rows pos(u) < rows: the M11 part of
// the query right-hand sides added to a dense block (no duplicate entries in
// a CSR row, so one block per column writes distinct rows).
template <int WT>
__global__ void rhs_add_rows_kernel(Csr W, const int32_t* q, double beta, const int32_t* pos,
                                    int64_t rows, float* T, int64_t ld) {
  const int c = blockIdx.x;
  const int64_t k0 = W.rowptr[q[c]], k1 = W.rowptr[q[c] + 1];
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    double w = 1.0;
    if (WT == KATZ_F64) w = static_cast<const double*>(W.val)[k];
    else if (WT == KATZ_F32) w = static_cast<const float*>(W.val)[k];
    else if (WT == KATZ_BF16) w = __bfloat162float(static_cast<const __nv_bfloat16*>(W.val)[k]);
    const int64_t r = pos[W.col[k]];
    if (r < rows) T[r * ld + c] += float(beta * w);
  }
}

// Whether the first LRC pass of a query takes its Schur right-hand side
// from the stored Z (and then reads only the separator rows of its
// right-hand side block).
static bool first_rhs_from_z(const katz_index& idx) {
  return idx.has_z && idx.n1 > 0 && idx.n2 > 0 && !idx.seg_blocked;
}

static void schur_rhs_from_z(const katz_index& idx, const int32_t* q, int b, const float* R2,
                             int64_t ld, float* F, cudaStream_t s) {
  const dim3 grid((unsigned)b, (unsigned)ceil_div(idx.n2, 256 * 8));
  const Csr W = idx.W.view();
  switch (W.vdt) {
    case KATZ_UNIT:
      schur_rhs_from_z_kernel<KATZ_UNIT><<<grid, 256, 0, s>>>(W, q, idx.beta, idx.iperm.p, idx.n1,
                                                              idx.Zc.p, idx.ldZ, idx.n2, R2, ld, F);
      break;
    case KATZ_F64:
      schur_rhs_from_z_kernel<KATZ_F64><<<grid, 256, 0, s>>>(W, q, idx.beta, idx.iperm.p, idx.n1,
                                                             idx.Zc.p, idx.ldZ, idx.n2, R2, ld, F);
      break;
    case KATZ_F32:
      schur_rhs_from_z_kernel<KATZ_F32><<<grid, 256, 0, s>>>(W, q, idx.beta, idx.iperm.p, idx.n1,
                                                             idx.Zc.p, idx.ldZ, idx.n2, R2, ld, F);
      break;
    default:
      schur_rhs_from_z_kernel<KATZ_BF16><<<grid, 256, 0, s>>>(W, q, idx.beta, idx.iperm.p, idx.n1,
                                                              idx.Zc.p, idx.ldZ, idx.n2, R2, ld, F);
      break;
  }
  KATZ_CHECK_LAUNCH();
}

// Per column: converged = rr <= thr2; inner threshold
//   thr2_in = max(tau^2 rr, (0.3)^2 thr2)
// and, for converged columns, a threshold every residual meets (their
// inner CG does no iteration and returns a zero correction).
__global__ void inner_thresholds_kernel(const double* rr, const double* thr2, double tau, int b,
                                        int* conv, double* thr2_in, int* n_open) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int local = 0;
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    const int cv = rr[c] <= thr2[c];
    conv[c] = cv;
    thr2_in[c] = cv ? DBL_MAX : fmax(tau * tau * rr[c], 0.09 * thr2[c]);
    local += !cv;
  }
  atomicAdd(&cnt, local);
  __syncthreads();
  if (threadIdx.x == 0) *n_open = cnt;
}

template <class D>
__global__ void masked_from_f64_kernel(const double* X, D* Y, int64_t ld, int64_t len, int b,
                                       const int* conv) {
  const int64_t total = len * ld;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t c = e % ld;
    Y[e] = (c < b && !conv[c]) ? D(X[e]) : D(0);
  }
}

template <class S>
__global__ void gather_out_kernel(const double* K64, const S* K32, int64_t ld, const int32_t* map,
                                  int64_t n, int b, void* out, int out_dt, int64_t ldk) {
  const int64_t total = n * b;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / b, c = e - i * b;
    const int64_t r = map ? map[i] : i;
    const double v = K64 ? K64[r * ld + c] : double(K32[r * ld + c]);
    if (out_dt == KATZ_F64)
      static_cast<double*>(out)[i * ldk + c] = v;
    else
      static_cast<float*>(out)[i * ldk + c] = float(v);
  }
}

static unsigned flat_blocks(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), int64_t(num_sms()) * 16));
}

// Column arrays that receive vectorised reductions are padded to a multiple
// of 4 entries (a reduction over a 4-wide vector writes all 4 lanes).
static int bpad(int b) { return (b + 3) / 4 * 4; }
// Leading dimension of the query's n x b blocks: a multiple of 8 elements
// for wide batches (32-byte row accesses in the fused gather kernels),
// else of 4.
static int64_t query_ld(int b) { return b > 128 ? (b + 7) / 8 * 8 : (b + 3) / 4 * 4; }

// ------------------------------------------------------------ col state
static ColState make_state(Workspace& ws, const std::string& tag, int b, bool with_rr) {
  ColState st;
  st.rz = ws.get<double>(tag + ".rz", bpad(b));
  st.pq = ws.get<double>(tag + ".pq", bpad(b));
  st.rz_new = ws.get<double>(tag + ".rzn", bpad(b));
  st.rr = with_rr ? ws.get<double>(tag + ".rr", bpad(b)) : nullptr;
  st.thr2 = ws.get<double>(tag + ".thr2", b);
  st.active = ws.get<int>(tag + ".act", b);
  st.iters = ws.get<int>(tag + ".it", b);
  st.flags = ws.get<int>(tag + ".flags", 1);
  st.n_active = ws.get<int>(tag + ".nact", 1);
  return st;
}

static int read_int(const int* dev, cudaStream_t s) {
  int h = 0;
  KATZ_CUDA(cudaMemcpyAsync(&h, dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  return h;
}

// Adds the state's per-column iteration counts to iters (host; grown to b
// columns if shorter).
static void harvest_iters(const ColState& st, int b, std::vector<int32_t>* iters, cudaStream_t s) {
  if (!iters) return;
  if (iters->size() < size_t(b)) iters->resize(b, 0);
  std::vector<int32_t> h(b);
  KATZ_CUDA(cudaMemcpyAsync(h.data(), st.iters, sizeof(int) * b, cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  for (int c = 0; c < b; ++c) (*iters)[c] += h[c];
}

// ----------------------------------------------------------- plain CG
// Solves (I - beta A) X = B for len x b blocks (ld), zero start, stopping
// column c when ||r_c||^2 <= thr2[c].  Returns KATZ_OK / ENOTSPD / ENOCONV.
template <class VT>
int cg_solve(const GraphPart& A, double beta, const VT* B, int64_t ld, int64_t len, int b, VT* X,
             const double* thr2, int max_iter, Workspace& ws, const std::string& tag,
             std::vector<int32_t>* iters, cudaStream_t s) {
  VT* R = ws.get<VT>(tag + ".R", size_t(len) * ld);
  VT* P = ws.get<VT>(tag + ".P", size_t(len) * ld);
  VT* Q = ws.get<VT>(tag + ".Q", size_t(len) * ld);
  ColState st = make_state(ws, tag, b, false);
  KATZ_CUDA(cudaMemcpyAsync(st.thr2, thr2, sizeof(double) * b, cudaMemcpyDeviceToDevice, s));
  KATZ_CUDA(cudaMemsetAsync(X, 0, sizeof(VT) * len * ld, s));
  KATZ_CUDA(cudaMemcpyAsync(R, B, sizeof(VT) * len * ld, cudaMemcpyDeviceToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(P, B, sizeof(VT) * len * ld, cudaMemcpyDeviceToDevice, s));
  KATZ_CUDA(cudaMemsetAsync(st.rz, 0, sizeof(double) * b, s));
  coldot<VT>(R, ld, R, ld, len, b, st.rz, s);
  colstate_init_kernel<<<1, 1024, 0, s>>>(st, b, 0);
  KATZ_CHECK_LAUNCH();
  int active = read_int(st.n_active, s);
  int it = 0;
  for (; it < max_iter && active > 0; ++it) {
    spmm<VT>(A.view(), A.heavy.p, A.n_heavy, -beta, P, ld, 1.0, P, ld, Q, ld, b, P, ld, st.pq, s,
             A.cfg(b));
    colstate_check_pq(st, b, s);
    cg_update_xr<VT>(X, P, R, Q, ld, len, b, st, true, s);
    colstate_advance(st, b, s);
    cg_update_p<VT>(P, R, ld, len, b, st, s);
    colstate_rotate(st, b, s);
    active = read_int(st.n_active, s);
  }
  harvest_iters(st, b, iters, s);
  const int flags = read_int(st.flags, s);
  if (flags & 1) return KATZ_ENOTSPD;
  return active > 0 ? KATZ_ENOCONV : KATZ_OK;
}

// thr2[c] = (tol * ||X_c||_2)^2 for a dense block.
template <class VT>
static void rel_thresholds(const VT* X, int64_t ld, int64_t len, int b, double tol, double* thr2,
                           Workspace& ws, const std::string& tag, cudaStream_t s) {
  double* n2 = ws.get<double>(tag + ".n2", bpad(b));
  double* mx = ws.get<double>(tag + ".mx", bpad(b));
  col_norms<VT>(X, ld, len, b, n2, mx, s);
  make_thresholds(n2, mx, b, tol, KATZ_TOL_RESIDUAL, 1.0, thr2, s);
}

// ----------------------------------------------------------- M11^{-1}
template <class VT>
static const VT* inv_of(const BlockClass& c);
template <>
const float* inv_of<float>(const BlockClass& c) { return c.inv32.p; }
template <>
const double* inv_of<double>(const BlockClass& c) { return c.inv64.p; }

// Pipelined or register kernel for a fused product, by the query's choice
// (AUTO: what the autotuner measured faster, register if untuned); first:
// the first refinement-residual pass.
static bool use_pipe(const katz_index& idx, const SpmmCfg* cfg, bool first = false) {
  if (idx.gather_pref == KATZ_GATHER_PIPELINED) return true;
  if (idx.gather_pref == KATZ_GATHER_REGISTER || idx.gather_pref == KATZ_GATHER_ROWPIPE ||
      idx.gather_pref == KATZ_GATHER_CHUNKED)
    return false;
  return cfg && (first ? cfg->pipe_first : cfg->pipe);
}

// Y1 = M11^{-1} X1: dense block inverses for the small blocks (Step 4) and,
// for blocks kept whole, CG on that diagonal block to relative tolerance tolL.
// Chebyshev iteration (Saad, Iterative Methods, Alg. 12.1) on the large
// M11 blocks, in three-term form, for the spectrum of M11 in
// [theta - d, theta + d] = [1 - beta*lam11, 1 - beta*lam11_min]:
//   x_1 = b / theta,
//   x_{k+1} = x_k + rho_k rho_{k-1} (x_k - x_{k-1}) + (2 rho_k / d) r_k,
//   rho_0 = d / theta, rho_k = 1 / (2 theta / d - rho_{k-1}).
// The iteration count follows from the bound 2 c^K <= tol with
// c = (sqrt(kappa)-1)/(sqrt(kappa)+1), kappa = (theta + d) / (theta - d).
// No inner products, no host synchronisation, one fused kernel per step
// (x_1 enters the first one as b scaled by 1/theta).
// Iterates x_2 .. x_{K-1} are kept in the split BF16 form (two scratch
// buffers, x_{k+1} overwriting x_{k-1} row by row) unless the query asks
// for FP32 gathers; their products gather the hi plane alone except, under
// KATZ_CHEB_MIXED, the last step of a solve asked for a tolerance below
// kHiGatherTol: a step's gather error (~2^-9 relative per term, ~1e-4 of
// beta W x after the sum) is damped by each later step by about the
// convergence factor c (~0.05 on the benchmark graph), so the hi-plane
// gathers leave the solve within its tolerance when a hi + lo step closes
// it.  x_K is written to Y in FP32.
constexpr double kHiGatherTol = 1e-4;

static void m11_chebyshev(katz_index& idx, const float* X, float* Y, int b, int64_t ld,
                          double tol, cudaStream_t s) {
  const int64_t len = idx.n1 - idx.n1s;
  const double lo = 1.0 - idx.beta * idx.lam11, hi = 1.0 - idx.beta * idx.lam11_min;
  const double theta = 0.5 * (lo + hi), d = 0.5 * (hi - lo);
  const int K = cheb_steps(idx, tol);
  if (K == 1) {
    scale_copy<float>(X, ld, Y, ld, len, int(ld), 1.0 / theta, false, s);
    return;
  }
  const double sigma = theta / d;
  double rho_prev = d / theta;  // rho_0 = 1/sigma
  const SpmmCfg* cfg = idx.W11L.cfg(b);
  SpmmCfg forced;  // the query asked for the row-pipelined kernel
  if (idx.gather_pref == KATZ_GATHER_ROWPIPE) {
    forced = cfg ? *cfg : SpmmCfg{};
    forced.row_pipeline = true;
    cfg = &forced;
  } else if (idx.gather_pref == KATZ_GATHER_REGISTER && cfg &&
             (cfg->row_pipeline || cfg->row_chunk > 0)) {
    forced = *cfg;
    forced.row_pipeline = false;
    forced.row_chunk = 0;
    cfg = &forced;
  } else if (idx.gather_pref == KATZ_GATHER_CHUNKED) {
    forced = cfg ? *cfg : SpmmCfg{};
    forced.row_pipeline = false;
    if (forced.row_chunk == 0) forced.row_chunk = 64;
    cfg = &forced;
  }
  const bool pipe = use_pipe(idx, cfg) && pipe_eligible(idx.W11L.ps, ld) &&
                    (idx.unit_weights || idx.W11L.csr.vdt != KATZ_F64);
  const bool tile_major = idx.cheb_pref == KATZ_CHEB_AUTO && !pipe && b > 128 && ld % 8 == 0;
  if (tile_major) {
    // FP32 iterates x_2 .. x_{K-1} in tile-major scratch (T for even k, U for
    // odd k): a column tile's rows are contiguous, so the gathers of one
    // tile sweep stay within rows x 1 KB instead of spreading over rows x ld
    const int64_t wcols = (b + 255) / 256 * 256;
    float* T = idx.ws.get<float>("ch.T", size_t(len) * wcols);
    float* U = K > 3 ? idx.ws.get<float>("ch.U", size_t(len) * wcols) : nullptr;
    auto slot = [&](int j) -> float* { return (j % 2 == 0) ? T : U; };
    for (int k = 1; k < K; ++k) {
      const double rho = 1.0 / (2.0 * sigma - rho_prev);
      const double ak = rho * rho_prev, ck = 2.0 * rho / d;
      const bool last = k == K - 1;
      const float* xk = k == 1 ? X : slot(k);
      const float* xprev = k == 1 ? nullptr : (k == 2 ? X : slot(k - 1));
      float* out = last ? Y : slot(k + 1);
      const int mask = (k >= 2 ? 1 : 0) | (k >= 3 ? 2 : 0) | (last ? 0 : 4);
      const double sx = k == 1 ? 1.0 / theta : 1.0, sp = k == 2 ? 1.0 / theta : 1.0;
      cheb_step_ex(idx.W11L.view(), idx.beta, ak, ck, xk, 0, xprev, xprev ? 1 : 0, X, out, 0, ld,
                   b, s, cfg, sx, sp, mask);
      rho_prev = rho;
    }
    return;
  }
  if (idx.cheb_pref == KATZ_CHEB_F32 || idx.cheb_pref == KATZ_CHEB_AUTO || pipe) {
    // FP32 iterates: x_k for k >= 2 alternates between Y and T so that x_K
    // lands in Y (x_{k+1} overwrites x_{k-1} row by row)
    float* T = idx.ws.get<float>("ch.T", size_t(len) * ld);
    auto slot = [&](int k) { return ((K - k) % 2 == 0) ? Y : T; };
    int* perr = idx.ws.get<int>("pipe.err", 1);
    for (int k = 1; k < K; ++k) {
      const double rho = 1.0 / (2.0 * sigma - rho_prev);
      const double ak = rho * rho_prev, ck = 2.0 * rho / d;
      // x_1 = X / theta is never stored: it enters as Xk (k = 1) or Xprev (k = 2)
      const float* xk = k == 1 ? X : slot(k);
      const float* xprev = k == 1 ? nullptr : (k == 2 ? X : slot(k - 1));
      const double sx = k == 1 ? 1.0 / theta : 1.0, sp = k == 2 ? 1.0 / theta : 1.0;
      if (pipe)
        pipe_cheb_step(idx.W11L.view(), idx.W11L.ps, idx.unit_weights, idx.beta, ak, ck, xk,
                       xprev, X, slot(k + 1), ld, perr, s, sx, sp);
      else
        cheb_step(idx.W11L.view(), idx.beta, ak, ck, xk, xprev, X, slot(k + 1), ld, b, s, cfg, sx,
                  sp);
      rho_prev = rho;
    }
    return;
  }
  // split iterates x_2 .. x_{K-1} in T and U (x_j in T for even j)
  float* T = idx.ws.get<float>("ch.T", size_t(len) * ld);
  float* U = K > 3 ? idx.ws.get<float>("ch.U", size_t(len) * ld) : nullptr;
  auto slot = [&](int j) -> void* { return (j % 2 == 0) ? static_cast<void*>(T) : U; };
  const bool last_exact = idx.cheb_pref == KATZ_CHEB_MIXED && tol < kHiGatherTol;
  for (int k = 1; k < K; ++k) {
    const double rho = 1.0 / (2.0 * sigma - rho_prev);
    const double ak = rho * rho_prev, ck = 2.0 * rho / d;
    const bool last = k == K - 1;
    const void* xk = k == 1 ? static_cast<const void*>(X) : slot(k);
    const int in_mode = k == 1 ? 0 : (last && last_exact ? 2 : 1);
    const void* xprev = k == 1 ? nullptr : (k == 2 ? static_cast<const void*>(X) : slot(k - 1));
    const int prev_mode = k == 1 ? 0 : (k == 2 ? 1 : 2);
    void* out = last ? static_cast<void*>(Y) : slot(k + 1);
    const double sx = k == 1 ? 1.0 / theta : 1.0, sp = k == 2 ? 1.0 / theta : 1.0;
    cheb_step_ex(idx.W11L.view(), idx.beta, ak, ck, xk, in_mode, xprev, prev_mode, X, out,
                 last ? 0 : 1, ld, b, s, cfg, sx, sp);
    rho_prev = rho;
  }
}

template <class VT>
int m11_solve(katz_index& idx, const VT* X, VT* Y, int b, int64_t ld, double tolL, int max_iter,
              std::vector<int32_t>* iters, cudaStream_t s) {
  for (auto& c : idx.classes)
    block_solve<VT>(inv_of<VT>(c), c.start.p, c.size.p, c.count, c.S, X, ld, Y, ld, b, s);
  int st = KATZ_OK;
  if constexpr (sizeof(VT) == 4) {
    if (idx.n1 > idx.n1s && idx.lam11 > 0) {
      m11_chebyshev(idx, reinterpret_cast<const float*>(X) + idx.n1s * ld,
                    reinterpret_cast<float*>(Y) + idx.n1s * ld, b, ld, tolL, s);
      return st;
    }
  }
  if (idx.n1 > idx.n1s) {
    const int64_t len = idx.n1 - idx.n1s;
    double* thr2 = idx.ws.get<double>("L.thr", b);
    rel_thresholds<VT>(X + idx.n1s * ld, ld, len, b, tolL, thr2, idx.ws, "L", s);
    st = cg_solve<VT>(idx.W11L, idx.beta, X + idx.n1s * ld, ld, len, b, Y + idx.n1s * ld, thr2,
                      max_iter, idx.ws, "L", iters, s);
  }
  return st;
}

// ------------------------------------------------- PCG on S K2 = F
template <class VT> struct Dense;
template <> struct Dense<float> {
  static const float* S(const katz_index& i) { return i.S32.p; }
  static const float* Minv(const katz_index& i) { return i.M22inv32.p; }
  static const float* Wr(const katz_index& i) { return i.Wr32.p; }
};
template <> struct Dense<double> {
  static const double* S(const katz_index& i) { return i.S64.p; }
  static const double* Minv(const katz_index& i) { return i.M22inv64.p; }
  static const double* Wr(const katz_index& i) { return i.Wr64.p; }
};

// Y = alpha A X + beta Y for the dense n2 x n2 matrices A = S or M22^{-1}
// and an n2 x ld block X: on the tensor cores (three TF32 products, FP32
// accuracy; all ld columns so zero padding stays zero) where the index keeps
// A's TF32 parts, else the FP32/FP64 SIMT GEMM.
// Y = alpha S X + beta Y (beta 0 or 1) for a separator too large to store S:
//   S X = M22 X - M12^T M11^{-1} M12 X = X - b W22 X - b W21 M11^{-1} (b W12 X)
// (Lemma 1, Eqs. 4-7; b the damping).  The M11 solve runs to 1e-7 relative
// (FP32) or 1e-14 (FP64), below what the PCG asks of S P.
template <class VT>
static void implicit_S(katz_index& idx, const VT* X, int64_t ld, int b, double alpha, double beta,
                       VT* Y, cudaStream_t s) {
  KATZ_REQUIRE(beta == 0.0 || beta == 1.0, KATZ_EINVAL, "implicit S: beta must be 0 or 1");
  const int64_t n1 = idx.n1, n2 = idx.n2;
  VT* Tm = idx.ws.get<VT>("Si.T", size_t(n2) * ld);
  spmm<VT>(idx.W22.view(), idx.W22.heavy.p, idx.W22.n_heavy, -idx.beta, X, ld, 1.0, X, ld, Tm, ld,
           b, nullptr, 0, nullptr, s, idx.W22.cfg(b));
  if (n1 > 0) {
    VT* U = idx.ws.get<VT>("Si.U", size_t(n1) * ld);
    VT* V = idx.ws.get<VT>("Si.V", size_t(n1) * ld);
    spmm<VT>(idx.W12.view(), idx.W12.heavy.p, idx.W12.n_heavy, idx.beta, X, ld, 0.0, nullptr, ld,
             U, ld, b, nullptr, 0, nullptr, s, idx.W12.cfg(b));
    const int st = m11_solve<VT>(idx, U, V, b, ld, sizeof(VT) == 4 ? 1e-7 : 1e-14, 5000,
                                 nullptr, s);
    KATZ_REQUIRE(st != KATZ_ENOTSPD, KATZ_ENOTSPD, "M11 is not positive definite");
    spmm<VT>(idx.W21.view(), idx.W21.heavy.p, idx.W21.n_heavy, -idx.beta, V, ld, 1.0, Tm, ld, Tm,
             ld, b, nullptr, 0, nullptr, s, idx.W21.cfg(b));
  }
  scale_copy<VT>(Tm, ld, Y, ld, n2, int(ld), alpha, beta != 0.0, s);
}

template <class VT>
static void dense_n2(katz_index& idx, bool minv, const VT* X, int64_t ld, int b, double alpha,
                     double beta, VT* Y, cudaStream_t s) {
  const int64_t n2 = idx.n2;
  if (!minv && idx.s_implicit) {
    implicit_S<VT>(idx, X, ld, b, alpha, beta, Y, s);
    return;
  }
  if constexpr (sizeof(VT) == 4) {
    if (idx.dense_tc) {
      float* Xh = idx.ws.get<float>("S.Xh", size_t(ld) * idx.ld2);
      float* Xl = idx.ws.get<float>("S.Xl", size_t(ld) * idx.ld2);
      split_tf32_transposed(reinterpret_cast<const float*>(X), ld, n2, int(ld), Xh, Xl, idx.ld2, s);
      tc_gemm_tf32x3(minv ? idx.Mh.p : idx.Sh.p, minv ? idx.Ml.p : idx.Sl.p, idx.ld2, Xh, Xl,
                     idx.ld2, int(n2), int(ld), int(n2), float(alpha), float(beta),
                     reinterpret_cast<const float*>(Y), ld, reinterpret_cast<float*>(Y), ld,
                     idx.ws.get<int>("S.err", 1), s);
      return;
    }
  }
  gemm<VT>(false, n2, b, n2, alpha, minv ? Dense<VT>::Minv(idx) : Dense<VT>::S(idx), idx.ld2, X,
           ld, beta, Y, ld, s);
}

// Z = S~^{-1} R = M22^{-1} R + W^ (W^T R), with W^ = W_r D^{1/2} (Eq. 14).
// FP32 path: the two rank-r products run on the tcgen05 tensor cores with
// BF16 operands (a preconditioner only needs to be a fixed SPD
// approximation; W^ and R^T are rounded once each, so the correction stays
// symmetric positive semi-definite up to the FP32 accumulation).
template <class VT>
static void precond(katz_index& idx, const VT* R, VT* Z, VT* Tm, int b, int64_t ld,
                    cudaStream_t s) {
  const int64_t n2 = idx.n2;
  dense_n2<VT>(idx, true, R, ld, b, 1.0, 0.0, Z, s);
  if constexpr (sizeof(VT) == 4) {
    if (idx.rank > 0) {
      __nv_bfloat16* Rt = idx.ws.get<__nv_bfloat16>("S.Rt", size_t(b) * idx.ldn2);
      __nv_bfloat16* Tt = idx.ws.get<__nv_bfloat16>("S.Tt", size_t(b) * idx.ldr);
      int* err = idx.ws.get<int>("S.err", 1);
      to_bf16_transposed(reinterpret_cast<const float*>(R), ld, n2, b, Rt, idx.ldn2, s);
      // Tt (b x r) = (W^T R)^T
      tc_gemm(idx.WbT.p, idx.ldn2, Rt, idx.ldn2, idx.rank, b, (int)n2, 1.f, 0.f, nullptr, 0, Tt,
              idx.ldr, 1, err, s);
      // Z += W^ T
      tc_gemm(idx.Wb.p, idx.ldr, Tt, idx.ldr, (int)n2, b, idx.rank, 1.f, 1.f,
              reinterpret_cast<float*>(Z), ld, nullptr, 0, 0, err, s);
    }
    (void)Tm;
    return;
  }
  if (idx.rank > 0) {
    gemm<VT>(true, idx.rank, b, n2, 1.0, Dense<VT>::Wr(idx), idx.rank, R, ld, 0.0, Tm, ld, s);
    gemm<VT>(false, n2, b, idx.rank, 1.0, Dense<VT>::Wr(idx), idx.rank, Tm, ld, 1.0, Z, ld, s);
  }
}

// Preconditioned CG (Hestenes-Stiefel form) on S K2 = F with S~^{-1} as the
// preconditioner; zero start; column c stops when ||F_c - S K2_c||^2 <= thr2[c].
// Columns whose warm residual is not below ||F||: restart from zero.
template <class VT>
__global__ void warm_fallback_kernel(VT* K2, VT* R, const VT* F, int64_t ld, int64_t len, int b,
                                     double* rr, const double* ff) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < len * b;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / b;
    const int c = int(e - i * b);
    if (rr[c] >= ff[c]) {
      K2[i * ld + c] = VT(0);
      R[i * ld + c] = F[i * ld + c];
    }
  }
}
__global__ void warm_fallback_rr_kernel(double* rr, const double* ff, int b, int* n_fallback) {
  for (int c = threadIdx.x; c < b; c += blockDim.x)
    if (rr[c] >= ff[c]) {
      rr[c] = ff[c];
      atomicAdd(n_fallback, 1);
    }
}

template <class VT>
int pcg_schur(katz_index& idx, const VT* F, VT* K2, int b, int64_t ld, const double* thr2,
              int max_iter, std::vector<int32_t>* iters, cudaStream_t s, const VT* X0 = nullptr) {
  const int64_t n2 = idx.n2;
  Workspace& ws = idx.ws;
  VT* R = ws.get<VT>("S.R", size_t(n2) * ld);
  VT* Z = ws.get<VT>("S.Z", size_t(n2) * ld);
  VT* P = ws.get<VT>("S.P", size_t(n2) * ld);
  VT* Q = ws.get<VT>("S.Q", size_t(n2) * ld);
  VT* Tm = ws.get<VT>("S.T", size_t(std::max(1, idx.rank)) * ld);
  ColState st = make_state(ws, "S", b, true);
  KATZ_CUDA(cudaMemsetAsync(ws.get<int>("S.err", 1), 0, sizeof(int), s));
  KATZ_CUDA(cudaMemcpyAsync(st.thr2, thr2, sizeof(double) * b, cudaMemcpyDeviceToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(R, F, sizeof(VT) * n2 * ld, cudaMemcpyDeviceToDevice, s));
  KATZ_CUDA(cudaMemsetAsync(st.rr, 0, sizeof(double) * b, s));
  if (X0) {
    // warm start: R = F - S K2(0), per-column fallback to zero
    KATZ_CUDA(cudaMemcpyAsync(K2, X0, sizeof(VT) * n2 * ld, cudaMemcpyDeviceToDevice, s));
    dense_n2<VT>(idx, false, K2, ld, b, -1.0, 1.0, R, s);
    double* ff = ws.get<double>("S.ff", bpad(b));
    int* nfb = ws.get<int>("S.nfb", 1);
    KATZ_CUDA(cudaMemsetAsync(ff, 0, sizeof(double) * b, s));
    KATZ_CUDA(cudaMemsetAsync(nfb, 0, sizeof(int), s));
    coldot<VT>(F, ld, F, ld, n2, b, ff, s);
    coldot<VT>(R, ld, R, ld, n2, b, st.rr, s);
    warm_fallback_kernel<VT><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n2 * b, 256), 4096)), 256, 0, s>>>(
        K2, R, F, ld, n2, b, st.rr, ff);
    KATZ_CHECK_LAUNCH();
    warm_fallback_rr_kernel<<<1, 1024, 0, s>>>(st.rr, ff, b, nfb);
    KATZ_CHECK_LAUNCH();
  } else {
    KATZ_CUDA(cudaMemsetAsync(K2, 0, sizeof(VT) * n2 * ld, s));
    coldot<VT>(R, ld, R, ld, n2, b, st.rr, s);
  }
  precond<VT>(idx, R, Z, Tm, b, ld, s);
  KATZ_CUDA(cudaMemcpyAsync(P, Z, sizeof(VT) * n2 * ld, cudaMemcpyDeviceToDevice, s));
  KATZ_CUDA(cudaMemsetAsync(st.rz, 0, sizeof(double) * b, s));
  coldot<VT>(R, ld, Z, ld, n2, b, st.rz, s);
  colstate_init_kernel<<<1, 1024, 0, s>>>(st, b, 1);
  KATZ_CHECK_LAUNCH();
  int active = read_int(st.n_active, s);
  for (int it = 0; it < max_iter && active > 0; ++it) {
    dense_n2<VT>(idx, false, P, ld, b, 1.0, 0.0, Q, s);
    coldot<VT>(P, ld, Q, ld, n2, b, st.pq, s);
    colstate_check_pq(st, b, s);
    cg_update_xr<VT>(K2, P, R, Q, ld, n2, b, st, false, s);
    coldot<VT>(R, ld, R, ld, n2, b, st.rr, s);
    precond<VT>(idx, R, Z, Tm, b, ld, s);
    coldot<VT>(R, ld, Z, ld, n2, b, st.rz_new, s);
    colstate_advance(st, b, s);
    cg_update_p<VT>(P, Z, ld, n2, b, st, s);
    colstate_rotate(st, b, s);
    active = read_int(st.n_active, s);
  }
  harvest_iters(st, b, iters, s);
  const int flags = read_int(st.flags, s);
  KATZ_REQUIRE(read_int(ws.get<int>("S.err", 1), s) == 0, KATZ_ECUDA,
               "tcgen05 GEMM pipeline timed out");
  if (flags & 1) return KATZ_ENOTSPD;
  return active > 0 ? KATZ_ENOCONV : KATZ_OK;
}

// Chebyshev steps the large M11 blocks need for relative tolerance tol.
int cheb_steps(const katz_index& idx, double tol) {
  const double lo = 1.0 - idx.beta * idx.lam11, hi = 1.0 - idx.beta * idx.lam11_min;
  const double kappa = hi / lo;
  const double cf = (std::sqrt(kappa) - 1.0) / (std::sqrt(kappa) + 1.0);
  return cf <= 0 ? 1 : std::max(1, int(std::ceil(std::log(tol / 2.0) / std::log(cf))));
}

// Whether the back-substitution K1 = M11^{-1}(R1 + beta W12 K2) is cheaper as
// K1 = Y1 + (beta M11^{-1} W12) K2 on the tensor cores: the second M11 solve
// gathers ~4 ld bytes per stored entry of the large blocks per Chebyshev step
// (~10 TB/s from L2); the product costs 6 n1 n2 ld flops at the ~0.25
// PFLOP/s measured for the three-TF32 GEMM with 128 x 128 tiles (bound by
// streaming both split operands through L2).
bool coupling_gemm_pays(const katz_index& idx, int64_t ld, double tol) {
  if (idx.n1 <= idx.n1s || idx.lam11 <= 0) return false;
  const double t_solve = cheb_steps(idx, tol) * double(idx.W11L.csr.nnz) * 4.0 * ld / 1.0e13;
  const double t_gemm = 6.0 * double(idx.n1) * double(idx.n2) * ld / 0.25e15;
  return t_gemm < t_solve;
}

// --------------------------------------------------------- LRC solve
// D = M^{-1} Rin for n x b blocks in index order (Lemma 1):
//   Y1 = M11^{-1} R1;  F = R2 - M12^T Y1 = R2 + beta W21 Y1   (Eq. 7)
//   S K2 = F by PCG with S~^{-1}                              (Eq. 14)
//   K1 = M11^{-1}(R1 - M12 K2) = M11^{-1}(R1 + beta W12 K2)   (Eq. 6)
template <class VT>
int lrc_solve(katz_index& idx, const VT* Rin, VT* D, int b, int64_t ld, double tol_s,
              double tol_l, int max_iter, std::vector<int32_t>* iters, cudaStream_t s,
              const VT* K2_0 = nullptr, const int32_t* q_rhs = nullptr, double tol_y1 = 0.0) {
  const int64_t n1 = idx.n1, n2 = idx.n2;
  const VT* R1 = Rin;
  const VT* R2 = Rin + n1 * ld;
  VT* D1 = D;
  VT* D2 = D + n1 * ld;
  VT* Y1 = idx.ws.get<VT>("lrc.Y1", size_t(std::max<int64_t>(n1, 1)) * ld);
  int status = KATZ_OK;
  auto merge = [&](int st) { if (st != KATZ_OK && status == KATZ_OK) status = st; };
  // Rin = beta W e_q (q_rhs given) and Z stored: F from the rows of Z, no Y1
  const bool from_z = sizeof(VT) == 4 && q_rhs && first_rhs_from_z(idx);
  // a one-step Y1 on an M11 that is one large block is R1 / theta: folded
  // into the coupling product below instead of being written out (not
  // where the tensor-core back-substitution reads Y1)
  const double tol_y = tol_y1 > 0 ? tol_y1 : tol_l;
  const bool y1_scaled = sizeof(VT) == 4 && !from_z && n1 > 0 && n2 > 0 && idx.n1s == 0 &&
                         idx.lam11 > 0 && !idx.has_h && cheb_steps(idx, tol_y) == 1;
  const double theta = 1.0 - 0.5 * idx.beta * (idx.lam11 + idx.lam11_min);
  if (n1 > 0 && !from_z && !y1_scaled) {
    NvtxRange r("katz.m11_solve");
    merge(m11_solve<VT>(idx, R1, Y1, b, ld, tol_y, max_iter, nullptr, s));
  }
  if (n2 > 0) {
    NvtxRange r("katz.schur_pcg");
    VT* F = idx.ws.get<VT>("lrc.F", size_t(n2) * ld);
    if (from_z) {
      if constexpr (sizeof(VT) == 4) schur_rhs_from_z(idx, q_rhs, b, R2, ld, F, s);
    } else if (y1_scaled)
      spmm<VT>(idx.W21.view(), idx.W21.heavy.p, idx.W21.n_heavy, idx.beta / theta, R1, ld, 1.0, R2,
               ld, F, ld, b, nullptr, 0, nullptr, s, idx.W21.cfg(b));
    else if (n1 > 0)
      spmm<VT>(idx.W21.view(), idx.W21.heavy.p, idx.W21.n_heavy, idx.beta, Y1, ld, 1.0, R2, ld, F,
               ld, b, nullptr, 0, nullptr, s, idx.W21.cfg(b));
    else
      KATZ_CUDA(cudaMemcpyAsync(F, R2, sizeof(VT) * n2 * ld, cudaMemcpyDeviceToDevice, s));
    if (idx.seg_blocked) {
      // many graphs: block-diagonal S with per-(graph, column) PCG scalars
      if constexpr (sizeof(VT) == 4) {
        merge(seg_pcg(idx, F, D2, b, ld, tol_s, max_iter, idx.seg_iters, s));
        if (iters) {
          iters->resize(b, 0);
          for (int g = 0; g < idx.sb.G; ++g)
            for (int c = 0; c < b; ++c)
              (*iters)[c] = std::max((*iters)[c], idx.seg_iters[size_t(g) * b + c]);
        }
      } else {
        throw Error(KATZ_EINVAL, "a many-graph index answers FP32 (mixed-precision) queries");
      }
    } else {
      double* thr2 = idx.ws.get<double>("lrc.thrF", b);
      rel_thresholds<VT>(F, ld, n2, b, tol_s, thr2, idx.ws, "lrcF", s);
      merge(pcg_schur<VT>(idx, F, D2, b, ld, thr2, max_iter, iters, s, K2_0));
    }
  }
  if (n1 > 0) {
    NvtxRange r("katz.backsolve");
    if constexpr (sizeof(VT) == 4) {
      if (n2 > 0 && !from_z && idx.has_h && coupling_gemm_pays(idx, ld, tol_l)) {
        // K1 = Y1 + (beta M11^{-1} W12) K2 on the tensor cores (all ld columns,
        // so the zero padding columns stay zero)
        float* Bh = idx.ws.get<float>("lrc.K2h", size_t(ld) * idx.ldH);
        float* Bl = idx.ws.get<float>("lrc.K2l", size_t(ld) * idx.ldH);
        split_tf32_transposed(reinterpret_cast<const float*>(D2), ld, n2, int(ld), Bh, Bl,
                              idx.ldH, s);
        tc_gemm_tf32x3(idx.Hh.p, idx.Hl.p, idx.ldH, Bh, Bl, idx.ldH, int(n1), int(ld), int(n2),
                       1.f, 1.f, reinterpret_cast<const float*>(Y1), ld,
                       reinterpret_cast<float*>(D1), ld, idx.ws.get<int>("pipe.err", 1), s);
        return status;
      }
    }
    const VT* T1 = R1;
    if (from_z) {
      // R1 is not read on this path: T1 = beta W12 K2 plus the sparse B1
      if constexpr (sizeof(VT) == 4) {
        spmm<VT>(idx.W12.view(), idx.W12.heavy.p, idx.W12.n_heavy, idx.beta, D2, ld, 0.0, nullptr,
                 ld, Y1, ld, b, nullptr, 0, nullptr, s, idx.W12.cfg(b));
        const Csr W = idx.W.view();
        switch (W.vdt) {
          case KATZ_UNIT: rhs_add_rows_kernel<KATZ_UNIT><<<b, 128, 0, s>>>(W, q_rhs, idx.beta, idx.iperm.p, n1, Y1, ld); break;
          case KATZ_F64: rhs_add_rows_kernel<KATZ_F64><<<b, 128, 0, s>>>(W, q_rhs, idx.beta, idx.iperm.p, n1, Y1, ld); break;
          case KATZ_F32: rhs_add_rows_kernel<KATZ_F32><<<b, 128, 0, s>>>(W, q_rhs, idx.beta, idx.iperm.p, n1, Y1, ld); break;
          default: rhs_add_rows_kernel<KATZ_BF16><<<b, 128, 0, s>>>(W, q_rhs, idx.beta, idx.iperm.p, n1, Y1, ld); break;
        }
        KATZ_CHECK_LAUNCH();
        T1 = Y1;
      }
    } else if (n2 > 0) {
      spmm<VT>(idx.W12.view(), idx.W12.heavy.p, idx.W12.n_heavy, idx.beta, D2, ld, 1.0, R1, ld, Y1,
               ld, b, nullptr, 0, nullptr, s, idx.W12.cfg(b));
      T1 = Y1;
    }
    merge(m11_solve<VT>(idx, T1, D1, b, ld, tol_l, max_iter, nullptr, s));
  }
  return status;
}

// ------------------------------------------------------- apply M (test)
template <class VT>
void apply_M(const katz_index& idx, const VT* X, VT* Y, int b, int64_t ld, cudaStream_t s) {
  spmm<VT>(idx.W.view(), idx.W.heavy.p, idx.W.n_heavy, -idx.beta, X, ld, 1.0, X, ld, Y, ld, b,
           nullptr, 0, nullptr, s);
}
template void apply_M<float>(const katz_index&, const float*, float*, int, int64_t, cudaStream_t);
template void apply_M<double>(const katz_index&, const double*, double*, int, int64_t,
                              cudaStream_t);

// ------------------------------------------------- query driver
template <class VT>
static int inner_solve(katz_index& idx, bool use_lrc, const VT* Rin, VT* D, int b, int64_t ld,
                       const double* thr2_in, double tol_rel, int max_iter,
                       std::vector<int32_t>* iters, cudaStream_t s, const VT* K2_0 = nullptr,
                       const int32_t* q_rhs = nullptr, double tol_y1 = 0.0) {
  if (use_lrc)
    return lrc_solve<VT>(idx, Rin, D, b, ld, tol_rel, tol_rel, max_iter, iters, s, K2_0, q_rhs,
                         tol_y1);
  // shares the scratch of the large-block M11 solve (never live at once)
  return cg_solve<VT>(idx.W, idx.beta, Rin, ld, idx.n, b, D, thr2_in, max_iter, idx.ws, "L",
                      iters, s);
}

static void rhs_norms(const Csr& W, const int32_t* q, int b, double beta, double* norm2,
                      double* maxabs, cudaStream_t s) {
  KATZ_CUDA(cudaMemsetAsync(norm2, 0, sizeof(double) * b, s));
  KATZ_CUDA(cudaMemsetAsync(maxabs, 0, sizeof(double) * b, s));
  switch (W.vdt) {
    case KATZ_UNIT: rhs_norms_kernel<KATZ_UNIT><<<b, 128, 0, s>>>(W, q, beta, norm2, maxabs); break;
    case KATZ_F64: rhs_norms_kernel<KATZ_F64><<<b, 128, 0, s>>>(W, q, beta, norm2, maxabs); break;
    case KATZ_F32: rhs_norms_kernel<KATZ_F32><<<b, 128, 0, s>>>(W, q, beta, norm2, maxabs); break;
    default: rhs_norms_kernel<KATZ_BF16><<<b, 128, 0, s>>>(W, q, beta, norm2, maxabs); break;
  }
  KATZ_CHECK_LAUNCH();
}

static void rhs_add(const Csr& W, const int32_t* q, int b, double beta, const int32_t* pos,
                    double* R, int64_t ld, cudaStream_t s) {
  switch (W.vdt) {
    case KATZ_UNIT: rhs_add_kernel<KATZ_UNIT><<<b, 128, 0, s>>>(W, q, beta, pos, R, ld); break;
    case KATZ_F64: rhs_add_kernel<KATZ_F64><<<b, 128, 0, s>>>(W, q, beta, pos, R, ld); break;
    case KATZ_F32: rhs_add_kernel<KATZ_F32><<<b, 128, 0, s>>>(W, q, beta, pos, R, ld); break;
    default: rhs_add_kernel<KATZ_BF16><<<b, 128, 0, s>>>(W, q, beta, pos, R, ld); break;
  }
  KATZ_CHECK_LAUNCH();
}

// R64 = B - M K64 (FP64) and rr[c] = ||R64_c||^2.
static void residual64(katz_index& idx, bool use_lrc, const int32_t* q, int b, int64_t ld,
                       const double* K64, double* R64, double* rr, cudaStream_t s) {
  const GraphPart& G = use_lrc ? idx.Wp : idx.W;
  const int32_t* pos = use_lrc ? idx.iperm.p : nullptr;
  spmm<double>(G.view(), G.heavy.p, G.n_heavy, idx.beta, K64, ld, -1.0, K64, ld, R64, ld, b,
               nullptr, 0, nullptr, s);
  rhs_add(idx.W.view(), q, b, idx.beta, pos, R64, ld, s);
  KATZ_CUDA(cudaMemsetAsync(rr, 0, sizeof(double) * b, s));
  coldot<double>(R64, ld, R64, ld, idx.n, b, rr, s);
}

// Tolerance the solve must meet so that the returned K meets o.tol: an
// infinity-norm error bound loses up to 2^-24 (1 + tol) more to the final
// rounding to FP32 output.
static double solve_tol(const katz_query_opts& o, const QueryOut& out) {
  if (o.tol_kind != KATZ_TOL_ERROR_INF || out.dtype != KATZ_F32) return o.tol;
  return std::max(0.5 * o.tol, o.tol - std::ldexp(1.0 + o.tol, -24));
}

// CG warm start, energy-optimal scaling of the guess x (node order): with
// M x = b - R from the first residual pass, the M-norm error of gamma x,
// ||k - gamma x||_M^2 = ||k||_M^2 - 2 gamma b^T x + gamma^2 x^T M x, is
// smallest at gamma = b^T x / x^T M x = b^T x / (b^T x - x^T R) (k = M^{-1} b),
// never larger than the zero start's ||k||_M (gamma = 0 when b^T x <= 0).
// bx[c] = b_c^T x_c = beta sum_{j in N(q_c)} w_j x[j][c], gathered here.
template <int WT>
__global__ void rhs_dot_kernel(Csr W, const int32_t* q, double beta, const float* X, int64_t ld,
                               double* bx) {
  const int c = blockIdx.x;
  const int64_t k0 = W.rowptr[q[c]], k1 = W.rowptr[q[c] + 1];
  double acc = 0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    double w = 1.0;
    if (WT == KATZ_F64) w = static_cast<const double*>(W.val)[k];
    else if (WT == KATZ_F32) w = static_cast<const float*>(W.val)[k];
    else if (WT == KATZ_BF16) w = __bfloat162float(static_cast<const __nv_bfloat16*>(W.val)[k]);
    acc += beta * w * double(X[int64_t(W.col[k]) * ld + c]);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) atomicAdd(bx + c, acc);
}
__global__ void warm_gamma_kernel(const double* bx, const double* xr, int b, double* gamma,
                                  int* n_zero) {
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    const double den = bx[c] - xr[c];
    const double g = (bx[c] > 0.0 && den > 0.0) ? bx[c] / den : 0.0;
    gamma[c] = g;
    if (g == 0.0) atomicAdd(n_zero, 1);
  }
}
__global__ void scale_cols_kernel(float* X, int64_t ld, int64_t n, int b, const double* gamma) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n * ld;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(e % ld);
    if (c < b) X[e] = float(double(X[e]) * gamma[c]);
  }
}

// Mixed-precision query for graphs whose weights are exact in FP32: FP32
// solves, the solution kept as a float-float pair (Kh, Kl) and the residual
// as (Rh, Rl), both updated by one pass per refinement step that gathers the
// step's FP32 correction (R <- R - M D, K <- K + D), accurate to ~2^-48
// relative to the terms.  Every column stops when its residual meets the
// error-bound threshold.
static int query_mixed_ff(katz_index& idx, bool use_lrc, const int32_t* q, const int32_t* q_host,
                          int b, const katz_query_opts& o, const QueryOut& out, katz_stats* stats,
                          std::vector<int32_t>& iters, std::vector<double>& relres,
                          cudaStream_t s) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  const int64_t n = idx.n;
  const int64_t ld = query_ld(b);
  const int max_iter = o.max_iter > 0 ? o.max_iter : 2000;
  const int max_refine = o.max_refine > 0 ? o.max_refine : 12;
  const int32_t* pos = use_lrc ? idx.iperm.p : nullptr;
  const GraphPart& G = use_lrc ? idx.Wp : idx.W;
  const SpmmCfg* gcfg = G.cfg(b);
  SpmmCfg gforced;  // the query asked for one row schedule of the residual passes
  if (idx.gather_pref == KATZ_GATHER_CHUNKED) {
    gforced = gcfg ? *gcfg : SpmmCfg{};
    if (gforced.row_chunk == 0) gforced.row_chunk = 64;
    gcfg = &gforced;
  } else if (idx.gather_pref == KATZ_GATHER_REGISTER && gcfg && gcfg->row_chunk > 0) {
    gforced = *gcfg;
    gforced.row_chunk = 0;
    gcfg = &gforced;
  }
  const bool pipe_ok = pipe_eligible(G.ps, ld) && (idx.unit_weights || G.csr.vdt != KATZ_F64);
  Workspace& ws = idx.ws;
  iters.assign(b, 0);
  relres.assign(b, 0.0);
  int64_t maxdeg = 0;
  for (int j = 0; j < b; ++j) maxdeg = std::max<int64_t>(maxdeg, idx.deg_h[q_host[j]]);

  double* bn2 = ws.get<double>("q.bn2", b);
  double* bmx = ws.get<double>("q.bmx", b);
  double* thr2 = ws.get<double>("q.thr2", b);
  double* thr2_in = ws.get<double>("q.thr2in", b);
  double* rr = ws.get<double>("q.rr", bpad(b));
  int* conv = ws.get<int>("q.conv", b);
  int* nopen = ws.get<int>("q.nopen", 1);
  int* perr = ws.get<int>("pipe.err", 1);
  rhs_norms(idx.W.view(), q, b, idx.beta, bn2, bmx, s);
  const double omc = std::max(1e-300, 1.0 - idx.beta * idx.lambda_up);
  make_thresholds(bn2, bmx, b, solve_tol(o, out), o.tol_kind, omc, thr2, s);
  const double tau = 2e-6;
  double tol_rel = (o.tol_kind == KATZ_TOL_RESIDUAL) ? o.tol : o.tol * omc;
  tol_rel = std::max(tol_rel * 0.3, tau);

  float* Rh = ws.get<float>("q.Rin", size_t(n) * ld);  // FP32 residual = RHS of the solves
  float* Rl = ws.get<float>("q.Rl", size_t(n) * ld);
  float* D = ws.get<float>("q.D", size_t(n) * ld);
  float* Kh = ws.get<float>("q.Kh", size_t(n) * ld);
  float* Kl = ws.get<float>("q.Kl", size_t(n) * ld);
  // the first LRC pass that forms its Schur right-hand side from Z reads
  // only the separator rows of the right-hand side (the first residual pass
  // then writes every row)
  if (use_lrc && first_rhs_from_z(idx))
    KATZ_CUDA(cudaMemsetAsync(Rh + idx.n1 * ld, 0, sizeof(float) * idx.n2 * ld, s));
  else
    KATZ_CUDA(cudaMemsetAsync(Rh, 0, sizeof(float) * n * ld, s));
  {
    NvtxRange nr("katz.rhs");
    build_rhs<float>(idx.W.view(), q, b, idx.beta, pos, Rh, ld, s);
  }
  inner_thresholds_kernel<<<1, 1024, 0, s>>>(bn2, thr2, tau, b, conv, thr2_in, nopen);
  KATZ_CHECK_LAUNCH();
  const float* K20 = nullptr;
  const bool cg_warm = o.warm_start && !use_lrc;
  if (o.warm_start) {
    KATZ_REQUIRE(idx.lrc && idx.mlp.ready, KATZ_EINVAL,
                 "warm_start needs an index with the LRC part and a trained warm-start network");
    if (use_lrc) {
      float* g = ws.get<float>("q.K20", size_t(std::max<int64_t>(idx.n2, 1)) * ld);
      warm_start_guess(idx, q, b, g, ld, s);
      K20 = g;
    }
  }
  const auto t1 = clk::now();
  int status = KATZ_OK;
  if (cg_warm) {
    // CG from the network's guess: the first residual pass below evaluates
    // b - M K0 for it, and columns whose guess is not better than zero
    // (||b - M K0|| >= ||b||) restart from zero
    KATZ_CUDA(cudaMemsetAsync(Kh, 0, sizeof(float) * n * ld, s));
    warm_cg_guess(idx, q, b, Kh, ld, s);
  } else {
    // (the first right-hand side is beta W e_q itself: the Schur system's
    // comes from the stored Z where there is one)
    status = inner_solve<float>(idx, use_lrc, Rh, Kh, b, ld, thr2_in, tol_rel, max_iter, &iters,
                                s, K20, q);
  }
  bool kl_zero = true;  // Kl (the low part of K) is zero and not yet written
  KATZ_CUDA(cudaStreamSynchronize(s));
  const auto t2 = clk::now();
  double ms_res = 0;
  int refine = 0;
  bool pending = false;  // D holds a correction not yet added to K
  bool loose_y1_used = false;  // the last correction took Y1 from one Chebyshev step
  bool warm_checked = false;
  int64_t warm_fallbacks = 0;  // columns whose guess was scaled to zero
  double warm_gamma_mean = 0;
  HeavyRows hv;  // the residual operator's heavy rows, split
  if (status == KATZ_OK || status == KATZ_ENOCONV) {
    for (;;) {
      const auto r0 = clk::now();
      KATZ_CUDA(cudaMemsetAsync(rr, 0, sizeof(double) * bpad(b), s));
      // R = b - M K0 (K0 = Kh, Kl = 0) on the first pass, then R -= M D for
      // each correction D, which joins K (K += D) only when another correction
      // is about to overwrite D, else in the output.  The first pass adds the
      // sparse b after the sweep, so its norms are taken afterwards (summing
      // squares before and correcting by b_i^2 - r_i^2 would cancel
      // catastrophically); later passes fuse them.
      NvtxRange nr(refine == 0 ? "katz.residual_first" : "katz.residual_update");
      if (refine == 0) {
        if (pipe_ok && use_pipe(idx, gcfg, true))
          pipe_residual(G.view(), G.ps, idx.unit_weights, idx.beta, Kh, Rh, Rl, ld, b, nullptr,
                        perr, s);
        else
          ffr_update(G.view(), idx.beta, Kh, Rh, Rl, true, ld, b, nullptr, gcfg, s,
                     heavy_rows(G, ld, ws, hv));
        ffr_add_rhs(idx.W.view(), q, pos, b, idx.beta, Rh, Rl, ld, nullptr, maxdeg, s);
        coldot<float>(Rh, ld, Rh, ld, n, b, rr, s);
        if (cg_warm && !warm_checked) {
          // scale each column of the guess to its energy-optimal multiple
          // (zero where the guess points away from k), then the first pass
          // again for the scaled guess
          warm_checked = true;
          double* bx = ws.get<double>("q.wbx", bpad(b));
          double* xr = ws.get<double>("q.wxr", bpad(b));
          double* gam = ws.get<double>("q.wg", bpad(b));
          int* nz = ws.get<int>("q.nfb", 1);
          KATZ_CUDA(cudaMemsetAsync(bx, 0, sizeof(double) * b, s));
          KATZ_CUDA(cudaMemsetAsync(xr, 0, sizeof(double) * b, s));
          KATZ_CUDA(cudaMemsetAsync(nz, 0, sizeof(int), s));
          switch (idx.W.csr.vdt) {
            case KATZ_UNIT: rhs_dot_kernel<KATZ_UNIT><<<b, 128, 0, s>>>(idx.W.view(), q, idx.beta, Kh, ld, bx); break;
            case KATZ_F64: rhs_dot_kernel<KATZ_F64><<<b, 128, 0, s>>>(idx.W.view(), q, idx.beta, Kh, ld, bx); break;
            case KATZ_F32: rhs_dot_kernel<KATZ_F32><<<b, 128, 0, s>>>(idx.W.view(), q, idx.beta, Kh, ld, bx); break;
            default: rhs_dot_kernel<KATZ_BF16><<<b, 128, 0, s>>>(idx.W.view(), q, idx.beta, Kh, ld, bx); break;
          }
          KATZ_CHECK_LAUNCH();
          coldot<float>(Kh, ld, Rh, ld, n, b, xr, s);
          warm_gamma_kernel<<<1, 1024, 0, s>>>(bx, xr, b, gam, nz);
          KATZ_CHECK_LAUNCH();
          scale_cols_kernel<<<(unsigned)std::max<int64_t>(
                                  1, std::min<int64_t>(ceil_div(n * ld, 256), 4096)),
                              256, 0, s>>>(Kh, ld, n, b, gam);
          KATZ_CHECK_LAUNCH();
          warm_fallbacks = read_int(nz, s);
          {
            std::vector<double> hg(b);
            KATZ_CUDA(cudaMemcpyAsync(hg.data(), gam, 8 * size_t(b), cudaMemcpyDeviceToHost, s));
            KATZ_CUDA(cudaStreamSynchronize(s));
            warm_gamma_mean = 0;
            for (double g : hg) warm_gamma_mean += g / b;
          }
          continue;  // first pass again for the scaled guess
        }
      } else {
        // Rl carries the first pass's low part into the first update only
        ffr_update(G.view(), idx.beta, D, Rh, refine == 1 ? Rl : nullptr, false, ld, b, rr, gcfg,
                   s, heavy_rows(G, ld, ws, hv));
      }
      inner_thresholds_kernel<<<1, 1024, 0, s>>>(rr, thr2, tau, b, conv, thr2_in, nopen);
      KATZ_CHECK_LAUNCH();
      ++refine;
      const int open = read_int(nopen, s);
      // a correction with the one-step Y1 that left columns open: later
      // corrections (of this and later queries) solve for Y1 in full
      if (open > 0 && loose_y1_used) idx.loose_y1 = false;
      loose_y1_used = false;
      KATZ_REQUIRE(read_int(perr, s) == 0, KATZ_ECUDA,
                   "pipelined gather kernel: a wait on its shared-memory ring timed out");
      ms_res += std::chrono::duration<double, std::milli>(clk::now() - r0).count();
      if (open == 0) { status = KATZ_OK; break; }
      if (refine > max_refine) { status = KATZ_ENOCONV; break; }
      // the correction solve only has to bring every open column below its
      // threshold: relative tolerance = tightest 0.3 * thr_c / ||r_c||
      double tol_step = 1.0;
      {
        std::vector<double> hr(b), ht(b);
        KATZ_CUDA(cudaMemcpyAsync(hr.data(), rr, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
        KATZ_CUDA(cudaMemcpyAsync(ht.data(), thr2, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
        KATZ_CUDA(cudaStreamSynchronize(s));
        for (int c = 0; c < b; ++c)
          if (hr[c] > ht[c] && hr[c] > 0) tol_step = std::min(tol_step, 0.3 * std::sqrt(ht[c] / hr[c]));
        tol_step = std::max(tol_step, tau);
      }
      if (pending) {  // D is about to be overwritten
        ff_add(Kh, Kl, D, n * ld, s, kl_zero);
        kl_zero = false;
      }
      // Y1 of a correction feeds only its Schur right-hand side; where the
      // index has not seen that fail, it is the first Chebyshev iterate
      loose_y1_used = use_lrc && idx.loose_y1 && idx.n1 > idx.n1s && idx.lam11 > 0 && idx.n2 > 0;
      const int st = inner_solve<float>(idx, use_lrc, Rh, D, b, ld, thr2_in, tol_step, max_iter,
                                        &iters, s, nullptr, nullptr, loose_y1_used ? 1.0 : 0.0);
      if (st == KATZ_ENOTSPD) { pending = false; status = st; break; }
      pending = true;
    }
    std::vector<double> hr(b), hb(b);
    KATZ_CUDA(cudaMemcpyAsync(hr.data(), rr, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaMemcpyAsync(hb.data(), bn2, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < b; ++c) relres[c] = hb[c] > 0 ? std::sqrt(hr[c] / hb[c]) : std::sqrt(hr[c]);
    ff_out(Kh, kl_zero ? nullptr : Kl, pending ? D : nullptr, ld, pos, n, b, out.K, out.dtype,
           out.ldk, s);
    KATZ_CUDA(cudaStreamSynchronize(s));
  }
  const auto t3 = clk::now();
  if (stats) {
    int mx = 0;
    double mr = 0;
    for (int c = 0; c < b; ++c) {
      mx = std::max(mx, iters[c]);
      mr = std::max(mr, relres[c]);
    }
    stats->iters = mx;
    stats->refine_steps = refine;
    stats->max_rel_res = mr;
    stats->ms[0] = std::chrono::duration<double, std::milli>(t3 - t0).count();
    stats->ms[1] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    stats->ms[2] = std::chrono::duration<double, std::milli>(t2 - t1).count();
    stats->ms[3] = ms_res;
    // the first Schur right-hand side came from the stored Z (no M11 solve)
    stats->ms[7] = (use_lrc && !cg_warm && idx.has_z && idx.n1 > 0 && idx.n2 > 0) ? 1.0 : 0.0;
    if (o.warm_start && use_lrc) {
      int h = 0;
      KATZ_CUDA(cudaMemcpy(&h, ws.get<int>("S.nfb", 1), sizeof(int), cudaMemcpyDeviceToHost));
      stats->ms[5] = h;  // columns whose warm start fell back to zero
    } else if (o.warm_start) {
      stats->ms[5] = double(warm_fallbacks);
      stats->ms[6] = warm_gamma_mean;  // mean energy-optimal scale of the guesses
    }
  }
  return status;
}

template <class VT>
static int query_impl(katz_index& idx, bool use_lrc, const int32_t* q, int b,
                      const katz_query_opts& o, const QueryOut& out, katz_stats* stats,
                      std::vector<int32_t>& iters, std::vector<double>& relres, cudaStream_t s) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  const int64_t n = idx.n;
  const int64_t ld = query_ld(b);
  const int max_iter = o.max_iter > 0 ? o.max_iter : 2000;
  const int max_refine = o.max_refine > 0 ? o.max_refine : 12;
  const bool mixed = o.precision == KATZ_PREC_MIXED;
  const int32_t* pos = use_lrc ? idx.iperm.p : nullptr;
  Workspace& ws = idx.ws;
  iters.assign(b, 0);
  relres.assign(b, 0.0);

  double* bn2 = ws.get<double>("q.bn2", b);
  double* bmx = ws.get<double>("q.bmx", b);
  double* thr2 = ws.get<double>("q.thr2", b);
  double* thr2_in = ws.get<double>("q.thr2in", b);
  double* rr = ws.get<double>("q.rr", bpad(b));
  int* conv = ws.get<int>("q.conv", b);
  int* nopen = ws.get<int>("q.nopen", 1);
  rhs_norms(idx.W.view(), q, b, idx.beta, bn2, bmx, s);
  const double omc = std::max(1e-300, 1.0 - idx.beta * idx.lambda_up);
  make_thresholds(bn2, bmx, b, solve_tol(o, out), o.tol_kind, omc, thr2, s);
  // inner solves aim below the outer target but not below what the inner
  // precision can deliver
  const double tau = (sizeof(VT) == 4) ? 2e-6 : 1e-13;
  double tol_rel = (o.tol_kind == KATZ_TOL_RESIDUAL) ? o.tol : o.tol * omc;
  tol_rel = std::max(tol_rel * 0.3, tau);

  // step 0: solve with the exact RHS in the inner precision
  VT* Rin = ws.get<VT>("q.Rin", size_t(n) * ld);
  VT* Dv = ws.get<VT>("q.D", size_t(n) * ld);
  KATZ_CUDA(cudaMemsetAsync(Rin, 0, sizeof(VT) * n * ld, s));
  build_rhs<VT>(idx.W.view(), q, b, idx.beta, pos, Rin, ld, s);
  inner_thresholds_kernel<<<1, 1024, 0, s>>>(bn2, thr2, tau, b, conv, thr2_in, nopen);
  KATZ_CHECK_LAUNCH();
  const auto t1 = clk::now();
  int status = inner_solve<VT>(idx, use_lrc, Rin, Dv, b, ld, thr2_in, tol_rel, max_iter, &iters, s);
  KATZ_CUDA(cudaStreamSynchronize(s));
  const auto t2 = clk::now();
  double ms_res = 0;
  int refine = 0;
  double* K64 = nullptr;
  if (status == KATZ_OK || status == KATZ_ENOCONV) {
    if (mixed || sizeof(VT) == 8) {
      K64 = ws.get<double>("q.K64", size_t(n) * ld);
      double* R64 = ws.get<double>("q.R64", size_t(n) * ld);
      if constexpr (sizeof(VT) == 4)
        convert_f32_to_f64(reinterpret_cast<const float*>(Dv), ld, K64, ld, n, (int)ld, s);
      else
        KATZ_CUDA(cudaMemcpyAsync(K64, Dv, sizeof(double) * n * ld, cudaMemcpyDeviceToDevice, s));
      for (;;) {
        const auto r0 = clk::now();
        residual64(idx, use_lrc, q, b, ld, K64, R64, rr, s);
        inner_thresholds_kernel<<<1, 1024, 0, s>>>(rr, thr2, tau, b, conv, thr2_in, nopen);
        KATZ_CHECK_LAUNCH();
        ++refine;
        const int open = read_int(nopen, s);
        ms_res += std::chrono::duration<double, std::milli>(clk::now() - r0).count();
        if (open == 0) { status = KATZ_OK; break; }
        if (refine > max_refine) { status = KATZ_ENOCONV; break; }
        masked_from_f64_kernel<VT><<<flat_blocks(n * ld), 256, 0, s>>>(R64, Rin, ld, n, b, conv);
        KATZ_CHECK_LAUNCH();
        const int st = inner_solve<VT>(idx, use_lrc, Rin, Dv, b, ld, thr2_in, tol_rel, max_iter,
                                       &iters, s);
        if (st == KATZ_ENOTSPD) { status = st; break; }
        if constexpr (sizeof(VT) == 4)
          add_f32_to_f64(reinterpret_cast<const float*>(Dv), ld, K64, ld, n, (int)ld, s);
        else
          scale_copy<double>(reinterpret_cast<const double*>(Dv), ld, K64, ld, n, (int)ld, 1.0,
                             true, s);
      }
      std::vector<double> hr(b), hb(b);
      KATZ_CUDA(cudaMemcpyAsync(hr.data(), rr, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
      KATZ_CUDA(cudaMemcpyAsync(hb.data(), bn2, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
      KATZ_CUDA(cudaStreamSynchronize(s));
      for (int c = 0; c < b; ++c) relres[c] = hb[c] > 0 ? std::sqrt(hr[c] / hb[c]) : std::sqrt(hr[c]);
    } else {
      for (int c = 0; c < b; ++c) relres[c] = std::nan("");
    }
    // output (node order)
    if (K64)
      gather_out_kernel<float><<<flat_blocks(n * b), 256, 0, s>>>(K64, nullptr, ld, pos, n, b, out.K,
                                                                  out.dtype, out.ldk);
    else
      gather_out_kernel<VT><<<flat_blocks(n * b), 256, 0, s>>>(nullptr, Dv, ld, pos, n, b, out.K,
                                                               out.dtype, out.ldk);
    KATZ_CHECK_LAUNCH();
    KATZ_CUDA(cudaStreamSynchronize(s));
  }
  const auto t3 = clk::now();
  if (stats) {
    int mx = 0;
    double mr = 0;
    for (int c = 0; c < b; ++c) {
      mx = std::max(mx, iters[c]);
      if (!std::isnan(relres[c])) mr = std::max(mr, relres[c]);
    }
    stats->iters = mx;
    stats->refine_steps = refine;
    stats->max_rel_res = mr;
    stats->ms[0] = std::chrono::duration<double, std::milli>(t3 - t0).count();
    stats->ms[1] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    stats->ms[2] = std::chrono::duration<double, std::milli>(t2 - t1).count();
    stats->ms[3] = ms_res;
  }
  return status;
}

int run_queries(katz_index& idx, bool use_lrc, const int32_t* q_dev, const int32_t* q_host, int b,
                const katz_query_opts& o, const QueryOut& out, katz_stats* st,
                std::vector<int32_t>& iters, std::vector<double>& relres, cudaStream_t s) {
  KATZ_REQUIRE(!use_lrc || idx.lrc, KATZ_EINVAL, "index was built without the LRC part");
  KATZ_REQUIRE(b > 0 && b <= 1024, KATZ_EINVAL, "b must be in [1, 1024]");
  // FP64-valued graphs keep the FP64 residual (their weights need not be
  // exact in FP32); the others use the float-float residual
  KATZ_REQUIRE(o.gather_kernel >= KATZ_GATHER_AUTO && o.gather_kernel <= KATZ_GATHER_CHUNKED,
               KATZ_EINVAL, "gather_kernel must be a KATZ_GATHER_* value");
  idx.gather_pref = o.gather_kernel;
  KATZ_REQUIRE(o.cheb_gather >= KATZ_CHEB_AUTO && o.cheb_gather <= KATZ_CHEB_MIXED, KATZ_EINVAL,
               "cheb_gather must be a KATZ_CHEB_* value");
  idx.cheb_pref = o.cheb_gather;
  int* perr = idx.ws.get<int>("pipe.err", 1);
  KATZ_CUDA(cudaMemsetAsync(perr, 0, sizeof(int), s));
  int status;
  if (o.precision == KATZ_PREC_MIXED && idx.vdt != KATZ_F64)
    status = query_mixed_ff(idx, use_lrc, q_dev, q_host, b, o, out, st, iters, relres, s);
  else if (o.precision == KATZ_PREC_F64)
    status = query_impl<double>(idx, use_lrc, q_dev, b, o, out, st, iters, relres, s);
  else
    status = query_impl<float>(idx, use_lrc, q_dev, b, o, out, st, iters, relres, s);
  KATZ_REQUIRE(read_int(perr, s) == 0, KATZ_ECUDA,
               "pipelined gather kernel: a wait on its shared-memory ring timed out");
  return status;
}

int lrc_solve_f32(katz_index& idx, const float* R, float* D, int b, int64_t ld, double tol_rel,
                  int max_iter, std::vector<int32_t>* iters, cudaStream_t s) {
  return lrc_solve<float>(idx, R, D, b, ld, tol_rel, tol_rel, max_iter, iters, s);
}

int run_queries_internal(katz_index& idx, const int32_t* q_dev, const int32_t* q_host, int b,
                         const katz_query_opts& o, void* Kout, int out_dt, int64_t ldk,
                         cudaStream_t s) {
  QueryOut out;
  out.K = Kout;
  out.dtype = out_dt;
  out.ldk = ldk;
  std::vector<int32_t> it;
  std::vector<double> rr;
  return run_queries(idx, true, q_dev, q_host, b, o, out, nullptr, it, rr, s);
}

template int cg_solve<float>(const GraphPart&, double, const float*, int64_t, int64_t, int, float*,
                             const double*, int, Workspace&, const std::string&,
                             std::vector<int32_t>*, cudaStream_t);
template int cg_solve<double>(const GraphPart&, double, const double*, int64_t, int64_t, int,
                              double*, const double*, int, Workspace&, const std::string&,
                              std::vector<int32_t>*, cudaStream_t);
template int m11_solve<double>(katz_index&, const double*, double*, int, int64_t, double, int,
                               std::vector<int32_t>*, cudaStream_t);
template int m11_solve<float>(katz_index&, const float*, float*, int, int64_t, double, int,
                              std::vector<int32_t>*, cudaStream_t);

}  // namespace katz
