// Block-diagonal Schur complement of an index over many disjoint graphs
// (Lemma 1 on a block-diagonal M: with each graph's own separator, S,
// M22^{-1} and the rank-r correction W^ W^T of Eq. 14 are block diagonal,
// one block per graph).  The blocks are stored packed, graph by graph, and
// every product runs one CTA per graph; the Schur PCG keeps one set of CG
// coefficients per (graph, column) so that each pair stops on its own.
#include <algorithm>
#include <cmath>

#include "index.h"

namespace katz {

namespace {

unsigned flat_blocks(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 65535));
}

__global__ void scatter_T_kernel(const double* E, int64_t ldc, int64_t n2, const int32_t* sg,
                                 const int64_t* gsep, const int64_t* moff, int l0, int cw,
                                 double* Tb) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n2 * cw;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = e / cw;
    const int l = int(e - p * cw);
    const int g = sg[p];
    const int64_t n = gsep[g + 1] - gsep[g], li = p - gsep[g], lj = l0 + l;
    if (lj < n) Tb[moff[g] + li * n + lj] = E[p * ldc + l];
  }
}

// M22 blocks: I - beta W22 restricted to each graph's separator (W22 holds
// local separator column indices; its rows of graph g only reach graph g).
template <int WT>
__global__ void m22_blocks_kernel(Csr W22, double beta, const int32_t* sg, const int64_t* gsep,
                                  const int64_t* moff, double* M) {
  for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < W22.nrows;
       p += int64_t(gridDim.x) * blockDim.x) {
    const int g = sg[p];
    const int64_t n = gsep[g + 1] - gsep[g], li = p - gsep[g];
    double* row = M + moff[g] + li * n;
    row[li] += 1.0;
    for (int64_t k = W22.rowptr[p]; k < W22.rowptr[p + 1]; ++k) {
      double w = 1.0;
      if (WT == KATZ_F64) w = static_cast<const double*>(W22.val)[k];
      else if (WT == KATZ_F32) w = static_cast<const float*>(W22.val)[k];
      else if (WT == KATZ_BF16) w = __bfloat162float(static_cast<const __nv_bfloat16*>(W22.val)[k]);
      row[W22.col[k] - gsep[g]] -= beta * w;
    }
  }
}

__global__ void sub_kernel(const double* A, const double* B, double* C, int64_t total) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x)
    C[e] = A[e] - B[e];
}

__global__ void to_f32_kernel(const double* A, float* B, int64_t total) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x)
    B[e] = float(A[e]);
}

// In-place inverse of each SPD block by Gauss-Jordan elimination without
// pivoting (one CTA per graph): at step k every entry off row and column k
// loses A[i][k] A[k][j] / p (p = A[k][k] > 0), then column k becomes
// -A[i][k] / p, row k A[k][j] / p and the pivot 1 / p.  A pivot <= 0 means
// the block is not positive definite (flag).
__global__ void block_gj_inverse_kernel(double* M, const int64_t* gsep, const int64_t* moff,
                                        int* flag) {
  const int g = blockIdx.x;
  const int64_t n = gsep[g + 1] - gsep[g];
  double* A = M + moff[g];
  __shared__ double piv;
  for (int64_t k = 0; k < n; ++k) {
    if (threadIdx.x == 0) piv = A[k * n + k];
    __syncthreads();
    const double p = piv;
    if (!(p > 0.0)) {
      if (threadIdx.x == 0) atomicExch(flag, 1);
      return;
    }
    for (int64_t e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int64_t i = e / n, j = e - i * n;
      if (i != k && j != k) A[e] -= A[i * n + k] * A[k * n + j] / p;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      if (i == k) continue;
      A[i * n + k] = -A[i * n + k] / p;
      A[k * n + i] = A[k * n + i] / p;
    }
    __syncthreads();
    if (threadIdx.x == 0) A[k * n + k] = 1.0 / p;
    __syncthreads();
  }
}

__global__ void block_mv64_kernel(const double* A, const int64_t* gsep, const int64_t* moff,
                                  const double* x, int64_t incx, double* y, int64_t incy) {
  const int g = blockIdx.x;
  const int64_t g0 = gsep[g], n = gsep[g + 1] - g0;
  const double* Ag = A + moff[g];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j) acc += Ag[i * n + j] * x[(g0 + j) * incx];
    y[(g0 + i) * incy] = acc;
  }
}

}  // namespace

void seg_scatter_T(const SegBlocks& sb, const double* E, int64_t ldc, int64_t n2, int l0, int cw,
                   double* Tb, cudaStream_t s) {
  if (n2 <= 0 || cw <= 0) return;
  scatter_T_kernel<<<flat_blocks(n2 * cw), 256, 0, s>>>(E, ldc, n2, sb.sg.p, sb.gsep.p, sb.moff.p,
                                                        l0, cw, Tb);
  KATZ_CHECK_LAUNCH();
}

bool seg_build_blocks(SegBlocks& sb, const Csr& W22, double beta, const double* Tb,
                      double* M22b, cudaStream_t s) {
  const int64_t nm = sb.nmat;
  KATZ_CUDA(cudaMemsetAsync(M22b, 0, 8 * size_t(std::max<int64_t>(nm, 1)), s));
  if (W22.nrows > 0) {
    const unsigned nb = flat_blocks(W22.nrows);
    switch (W22.vdt) {
      case KATZ_UNIT: m22_blocks_kernel<KATZ_UNIT><<<nb, 256, 0, s>>>(W22, beta, sb.sg.p, sb.gsep.p, sb.moff.p, M22b); break;
      case KATZ_F64: m22_blocks_kernel<KATZ_F64><<<nb, 256, 0, s>>>(W22, beta, sb.sg.p, sb.gsep.p, sb.moff.p, M22b); break;
      case KATZ_F32: m22_blocks_kernel<KATZ_F32><<<nb, 256, 0, s>>>(W22, beta, sb.sg.p, sb.gsep.p, sb.moff.p, M22b); break;
      default: m22_blocks_kernel<KATZ_BF16><<<nb, 256, 0, s>>>(W22, beta, sb.sg.p, sb.gsep.p, sb.moff.p, M22b); break;
    }
    KATZ_CHECK_LAUNCH();
  }
  sb.S64.alloc(std::max<int64_t>(nm, 1));
  sb.Minv64.alloc(std::max<int64_t>(nm, 1));
  sub_kernel<<<flat_blocks(nm), 256, 0, s>>>(M22b, Tb, sb.S64.p, nm);
  KATZ_CHECK_LAUNCH();
  KATZ_CUDA(cudaMemcpyAsync(sb.Minv64.p, M22b, 8 * size_t(nm), cudaMemcpyDeviceToDevice, s));
  DBuf<int> flag(1);
  KATZ_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  block_gj_inverse_kernel<<<sb.G, 256, 0, s>>>(sb.Minv64.p, sb.gsep.p, sb.moff.p, flag.p);
  KATZ_CHECK_LAUNCH();
  sb.S32.alloc(std::max<int64_t>(nm, 1));
  sb.Minv32.alloc(std::max<int64_t>(nm, 1));
  to_f32_kernel<<<flat_blocks(nm), 256, 0, s>>>(sb.S64.p, sb.S32.p, nm);
  to_f32_kernel<<<flat_blocks(nm), 256, 0, s>>>(sb.Minv64.p, sb.Minv32.p, nm);
  KATZ_CHECK_LAUNCH();
  int h = 0;
  KATZ_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  return h == 0;
}

void seg_block_mv64(const SegBlocks& sb, const double* A, const double* x, int64_t incx, double* y,
                    int64_t incy, cudaStream_t s) {
  if (sb.G <= 0) return;
  block_mv64_kernel<<<sb.G, 128, 0, s>>>(A, sb.gsep.p, sb.moff.p, x, incx, y, incy);
  KATZ_CHECK_LAUNCH();
}

}  // namespace katz

// ------------------------------------------------ Schur PCG, per graph
namespace katz {

namespace {

constexpr int kMaxB = 64;  // columns of a many-graph batch (queries per graph)

// out[g * b + c] = sum over graph g's rows of A[p][c] B[p][c] (FP64), one CTA
// per graph: thread t sums column t % 64 over rows t / 64, 4 apart.
__global__ void segcoldot_kernel(const float* A, const float* B, int64_t ld, int b,
                                 const int64_t* gsep, double* out) {
  __shared__ double part[256];
  const int g = blockIdx.x;
  const int c = threadIdx.x % kMaxB, r0 = threadIdx.x / kMaxB;
  double acc = 0.0;
  if (c < b)
    for (int64_t p = gsep[g] + r0; p < gsep[g + 1]; p += 4)
      acc += double(A[p * ld + c]) * double(B[p * ld + c]);
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < kMaxB && c < b)
    out[int64_t(g) * b + c] = part[c] + part[c + 64] + part[c + 128] + part[c + 192];
}

// Y_g = alpha A_g X_g + beta Y_g for the FP32 blocks A_g (n_g x n_g).
__global__ void block_mm32_kernel(const float* A, const int64_t* gsep, const int64_t* moff,
                                  const float* X, int64_t ld, int b, float alpha, float beta,
                                  float* Y) {
  const int g = blockIdx.x;
  const int64_t g0 = gsep[g], n = gsep[g + 1] - g0;
  const float* Ag = A + moff[g];
  for (int64_t e = threadIdx.x; e < n * b; e += blockDim.x) {
    const int64_t i = e / b;
    const int c = int(e - i * b);
    float acc = 0.f;
    for (int64_t j = 0; j < n; ++j) acc = fmaf(Ag[i * n + j], X[(g0 + j) * ld + c], acc);
    float* y = Y + (g0 + i) * ld + c;
    *y = beta == 0.f ? alpha * acc : alpha * acc + beta * (*y);
  }
}

// Z_g += W_g (W_g^T R_g) with W_g = W^ block (n_g x r_g), one CTA per graph.
__global__ void block_lowrank_kernel(const float* Wb, const int64_t* woff, const int32_t* rk,
                                     const int64_t* gsep, const float* R, int64_t ld, int b,
                                     float* Z) {
  __shared__ float T[kSegBlockMax / 4 * kMaxB];  // r_g x b, r_g <= 64
  const int g = blockIdx.x;
  const int r = rk[g];
  if (r == 0) return;
  const int64_t g0 = gsep[g], n = gsep[g + 1] - g0;
  const float* W = Wb + woff[g];
  for (int e = threadIdx.x; e < r * b; e += blockDim.x) {
    const int k = e / b, c = e - (e / b) * b;
    float acc = 0.f;
    for (int64_t i = 0; i < n; ++i) acc = fmaf(W[i * r + k], R[(g0 + i) * ld + c], acc);
    T[k * b + c] = acc;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < n * b; e += blockDim.x) {
    const int64_t i = e / b;
    const int c = int(e - i * b);
    float acc = 0.f;
    for (int k = 0; k < r; ++k) acc = fmaf(W[i * r + k], T[k * b + c], acc);
    Z[(g0 + i) * ld + c] += acc;
  }
}

// Per-pair state: alpha = rz / pq (breakdown pq <= 0 stops the pair and sets
// flag bit 0), then the update X += alpha P, R -= alpha Q on active pairs.
__global__ void seg_alpha_kernel(const double* rz, const double* pq, int pairs, int* active,
                                 double* alpha, int* flags) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < pairs; k += gridDim.x * blockDim.x) {
    alpha[k] = 0.0;
    if (!active[k]) continue;
    if (!(pq[k] > 0.0)) {
      active[k] = 0;
      atomicOr(flags, 1);
      continue;
    }
    alpha[k] = rz[k] / pq[k];
  }
}
__global__ void seg_xr_kernel(float* X, const float* P, float* R, const float* Q, int64_t ld,
                              int64_t n2, int b, const int32_t* sg, const double* alpha) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n2 * b;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = e / b;
    const int c = int(e - p * b);
    const double a = alpha[int64_t(sg[p]) * b + c];
    if (a == 0.0) continue;
    const int64_t o = p * ld + c;
    X[o] = float(double(X[o]) + a * double(P[o]));
    R[o] = float(double(R[o]) - a * double(Q[o]));
  }
}
// convergence (rr <= thr2 stops the pair) and beta = rz_new / rz; counts
// the pairs still open and their iterations
__global__ void seg_beta_kernel(const double* rr, const double* thr2, double* rz,
                                const double* rz_new, int pairs, int* active, double* beta,
                                int* iters, int* n_active) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < pairs; k += gridDim.x * blockDim.x) {
    beta[k] = 0.0;
    if (!active[k]) continue;
    ++iters[k];
    if (rr[k] <= thr2[k]) {
      active[k] = 0;
      continue;
    }
    beta[k] = rz[k] > 0.0 ? rz_new[k] / rz[k] : 0.0;
    rz[k] = rz_new[k];
    atomicAdd(n_active, 1);
  }
}
__global__ void seg_p_kernel(float* P, const float* Z, int64_t ld, int64_t n2, int b,
                             const int32_t* sg, const int* active, const double* beta) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n2 * b;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = e / b;
    const int c = int(e - p * b);
    const int64_t k = int64_t(sg[p]) * b + c;
    if (!active[k]) continue;
    const int64_t o = p * ld + c;
    P[o] = float(double(Z[o]) + beta[k] * double(P[o]));
  }
}
__global__ void seg_init_kernel(const double* ff, const double* rr, double tol2, int pairs,
                                double* thr2, int* active, int* iters, int* n_active) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < pairs; k += gridDim.x * blockDim.x) {
    thr2[k] = tol2 * ff[k];
    iters[k] = 0;
    active[k] = rr[k] > thr2[k] ? 1 : 0;
    if (active[k]) atomicAdd(n_active, 1);
  }
}

}  // namespace

// Z = S~^{-1} R = M22^{-1} R + W^ (W^T R) block by block (Eq. 14).
static void seg_precond(const SegBlocks& sb, const float* R, float* Z, int64_t ld, int b,
                        cudaStream_t s) {
  block_mm32_kernel<<<sb.G, 256, 0, s>>>(sb.Minv32.p, sb.gsep.p, sb.moff.p, R, ld, b, 1.f, 0.f, Z);
  KATZ_CHECK_LAUNCH();
  if (sb.nw > 0) {
    block_lowrank_kernel<<<sb.G, 256, 0, s>>>(sb.W32.p, sb.woff.p, sb.rk.p, sb.gsep.p, R, ld, b, Z);
    KATZ_CHECK_LAUNCH();
  }
}

int seg_pcg(katz_index& idx, const float* F, float* K2, int b, int64_t ld, double tol,
            int max_iter, std::vector<int32_t>& iters_gc, cudaStream_t s) {
  const SegBlocks& sb = idx.sb;
  KATZ_REQUIRE(b >= 1 && b <= kMaxB, KATZ_EINVAL, "many-graph Schur PCG: b must be in [1, 64]");
  const int64_t n2 = idx.n2;
  const int pairs = sb.G * b;
  Workspace& ws = idx.ws;
  float* R = ws.get<float>("sp.R", size_t(n2) * ld);
  float* Z = ws.get<float>("sp.Z", size_t(n2) * ld);
  float* P = ws.get<float>("sp.P", size_t(n2) * ld);
  float* Q = ws.get<float>("sp.Q", size_t(n2) * ld);
  double* ff = ws.get<double>("sp.ff", pairs);
  double* rr = ws.get<double>("sp.rr", pairs);
  double* rz = ws.get<double>("sp.rz", pairs);
  double* rzn = ws.get<double>("sp.rzn", pairs);
  double* pq = ws.get<double>("sp.pq", pairs);
  double* thr2 = ws.get<double>("sp.thr", pairs);
  double* al = ws.get<double>("sp.al", pairs);
  double* be = ws.get<double>("sp.be", pairs);
  int* active = ws.get<int>("sp.act", pairs);
  int* it = ws.get<int>("sp.it", pairs);
  int* flags = ws.get<int>("sp.flags", 2);  // [0] breakdown, [1] open pairs
  const unsigned pb = (unsigned)std::max(1, std::min(64, (pairs + 255) / 256));
  const unsigned vb = flat_blocks(n2 * b);
  KATZ_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), s));
  KATZ_CUDA(cudaMemsetAsync(K2, 0, sizeof(float) * n2 * ld, s));
  KATZ_CUDA(cudaMemcpyAsync(R, F, sizeof(float) * n2 * ld, cudaMemcpyDeviceToDevice, s));
  segcoldot_kernel<<<sb.G, 256, 0, s>>>(F, F, ld, b, sb.gsep.p, ff);
  KATZ_CHECK_LAUNCH();
  KATZ_CUDA(cudaMemcpyAsync(rr, ff, 8 * size_t(pairs), cudaMemcpyDeviceToDevice, s));
  seg_init_kernel<<<pb, 256, 0, s>>>(ff, rr, tol * tol, pairs, thr2, active, it, flags + 1);
  KATZ_CHECK_LAUNCH();
  seg_precond(sb, R, Z, ld, b, s);
  KATZ_CUDA(cudaMemcpyAsync(P, Z, sizeof(float) * n2 * ld, cudaMemcpyDeviceToDevice, s));
  segcoldot_kernel<<<sb.G, 256, 0, s>>>(R, Z, ld, b, sb.gsep.p, rz);
  KATZ_CHECK_LAUNCH();
  auto open_pairs = [&]() {
    int h = 0;
    KATZ_CUDA(cudaMemcpyAsync(&h, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    return h;
  };
  int open = open_pairs();
  // one PCG iteration of every pair; converged pairs are masked, so extra
  // iterations change nothing
  auto iteration = [&](cudaStream_t st) {
    block_mm32_kernel<<<sb.G, 256, 0, st>>>(sb.S32.p, sb.gsep.p, sb.moff.p, P, ld, b, 1.f, 0.f, Q);
    KATZ_CHECK_LAUNCH();
    segcoldot_kernel<<<sb.G, 256, 0, st>>>(P, Q, ld, b, sb.gsep.p, pq);
    KATZ_CHECK_LAUNCH();
    seg_alpha_kernel<<<pb, 256, 0, st>>>(rz, pq, pairs, active, al, flags);
    KATZ_CHECK_LAUNCH();
    seg_xr_kernel<<<vb, 256, 0, st>>>(K2, P, R, Q, ld, n2, b, sb.sg.p, al);
    KATZ_CHECK_LAUNCH();
    segcoldot_kernel<<<sb.G, 256, 0, st>>>(R, R, ld, b, sb.gsep.p, rr);
    KATZ_CHECK_LAUNCH();
    seg_precond(sb, R, Z, ld, b, st);
    segcoldot_kernel<<<sb.G, 256, 0, st>>>(R, Z, ld, b, sb.gsep.p, rzn);
    KATZ_CHECK_LAUNCH();
    KATZ_CUDA(cudaMemsetAsync(flags + 1, 0, sizeof(int), st));
    seg_beta_kernel<<<pb, 256, 0, st>>>(rr, thr2, rz, rzn, pairs, active, be, it, flags + 1);
    KATZ_CHECK_LAUNCH();
    seg_p_kernel<<<vb, 256, 0, st>>>(P, Z, ld, n2, b, sb.sg.p, active, be);
    KATZ_CHECK_LAUNCH();
  };
  // kItersPerReplay iterations captured once into a CUDA graph (on a stream
  // of its own, ordered after the caller's by events) and replayed until no
  // pair is open; the host reads the open count once per replay
  if (open > 0) {
    constexpr int kItersPerReplay = 4;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      if (ev) cudaEventDestroy(ev);
      if (cs) cudaStreamDestroy(cs);
    };
    try {
      KATZ_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      KATZ_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      KATZ_CUDA(cudaEventRecord(ev, s));
      KATZ_CUDA(cudaStreamWaitEvent(cs, ev, 0));
      KATZ_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      try {
        for (int t = 0; t < kItersPerReplay; ++t) iteration(cs);
      } catch (...) {
        cudaStreamEndCapture(cs, &graph);
        throw;
      }
      KATZ_CUDA(cudaStreamEndCapture(cs, &graph));
      KATZ_CUDA(cudaGraphInstantiate(&exec, graph, 0));
      for (int done = 0; done < max_iter && open > 0; done += kItersPerReplay) {
        KATZ_CUDA(cudaGraphLaunch(exec, cs));
        ++idx.seg_replays;
        int h = 0;
        KATZ_CUDA(cudaMemcpyAsync(&h, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, cs));
        KATZ_CUDA(cudaStreamSynchronize(cs));
        open = h;
      }
      KATZ_CUDA(cudaEventRecord(ev, cs));
      KATZ_CUDA(cudaStreamWaitEvent(s, ev, 0));
    } catch (...) {
      cleanup();
      throw;
    }
    cleanup();
  }
  iters_gc.resize(pairs);
  int fl = 0;
  KATZ_CUDA(cudaMemcpyAsync(iters_gc.data(), it, 4 * size_t(pairs), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaMemcpyAsync(&fl, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  if (fl & 1) return KATZ_ENOTSPD;
  return open > 0 ? KATZ_ENOCONV : KATZ_OK;
}

}  // namespace katz
