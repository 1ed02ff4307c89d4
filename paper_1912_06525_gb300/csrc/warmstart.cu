// Learned warm start for the Schur-complement solve.
//
// Node features (32): degree / mean degree, log(1 + degree), and 30
// coordinates of a spectral embedding taken from the index's Lanczos basis
// W_r (the Ritz vectors of R, W_r^T M22 W_r = I): a separator node uses its
// row of W_r, a non-separator node its row of the harmonic extension
// beta M11^{-1} W12 W_r; every column is scaled to unit RMS.
// Target for query q: c* = W_r^T M22 k2(q), the M22-orthogonal coordinates
// of the separator part of the Katz vector computed by the method itself.
// Warm start: K2(0) = W_r c_hat with c_hat = MLP(x_q), used as the initial
// guess of the PCG on S (a column falls back to zero when its warm residual
// is not smaller than ||F||).
#include <algorithm>
#include <chrono>
#include <cmath>

#include "index.h"
#include "kernels_dense.h"

namespace katz {

int run_queries_internal(katz_index& idx, const int32_t* q_dev, const int32_t* q_host, int b,
                         const katz_query_opts& o, void* Kout, int out_dt, int64_t ldk,
                         cudaStream_t s);
template <class VT>
int m11_solve(katz_index& idx, const VT* X, VT* Y, int b, int64_t ld, double tolL, int max_iter,
              std::vector<int32_t>* iters, cudaStream_t s);

namespace {

constexpr int kFeat = 32, kEmb = 30;

// feat[i] for node i (node order)
__global__ void features_kernel(const int64_t* rowptr, const int32_t* iperm, int64_t n, int64_t n1,
                                const float* H, const float* Wr, int64_t ldr, int r,
                                float mean_deg, float* feat) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n * kFeat;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / kFeat;
    const int f = int(e - i * kFeat);
    float v = 0.f;
    if (f == 0) {
      v = float(rowptr[i + 1] - rowptr[i]) / mean_deg;
    } else if (f == 1) {
      v = log1pf(float(rowptr[i + 1] - rowptr[i]));
    } else {
      const int c = f - 2;
      if (c < r) {
        const int64_t p = iperm[i];
        v = p < n1 ? H[p * ldr + c] : Wr[(p - n1) * ldr + c];
      }
    }
    feat[e] = v;
  }
}

// feat[:, f] /= rms (columns 2.. only; degree columns standardised below)
__global__ void col_scale_kernel(float* feat, int64_t n, const double* s2, const double* s1) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n * kFeat;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int f = int(e % kFeat);
    const double mean = s1[f] / double(n);
    const double var = fmax(s2[f] / double(n) - (f < 2 ? mean * mean : 0.0), 1e-30);
    feat[e] = float((double(feat[e]) - (f < 2 ? mean : 0.0)) / sqrt(var));
  }
}

__global__ void col_moments_kernel(const float* feat, int64_t n, double* s2, double* s1) {
  const int f = threadIdx.x % kFeat;
  const int lanes = blockDim.x / kFeat;
  double a = 0, b = 0;
  for (int64_t i = int64_t(blockIdx.x) * lanes + threadIdx.x / kFeat; i < n;
       i += int64_t(gridDim.x) * lanes) {
    const double v = feat[i * kFeat + f];
    a += v * v;
    b += v;
  }
  atomicAdd(s2 + f, a);
  atomicAdd(s1 + f, b);
}

__global__ void gather_feat_kernel(const float* feat, const int32_t* q, int b, float* X) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < b * kFeat; e += gridDim.x * blockDim.x)
    X[e] = feat[int64_t(q[e / kFeat]) * kFeat + e % kFeat];
}

// separator part of K (node order, n x b) in index order: k2[s][j] = K[perm[n1+s]][j]
__global__ void gather_sep_kernel(const float* K, int64_t ldk, const int32_t* perm, int64_t n1,
                                  int64_t n2, int b, float* k2, int64_t ld) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n2 * b;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t sidx = e / b;
    const int j = int(e - sidx * b);
    k2[sidx * ld + j] = K[int64_t(perm[n1 + sidx]) * ldk + j];
  }
}

unsigned blocks(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), int64_t(num_sms()) * 16));
}

}  // namespace

// Node features (computed once per index).
void warm_features(katz_index& idx, cudaStream_t s) {
  if (idx.feat.p) return;
  KATZ_REQUIRE(idx.lrc && idx.rank > 0, KATZ_EINVAL, "warm start needs an LRC index with rank > 0");
  const int64_t n = idx.n, n1 = idx.n1, n2 = idx.n2;
  const int r = idx.rank;
  const int64_t ldr = idx.ldr4;
  // H = beta M11^{-1} W12 W_r  (n1 x r)
  float* U = idx.ws.get<float>("wf.U", size_t(std::max<int64_t>(n1, 1)) * ldr);
  float* H = idx.ws.get<float>("wf.H", size_t(std::max<int64_t>(n1, 1)) * ldr);
  if (n1 > 0) {
    spmm<float>(idx.W12.view(), idx.W12.heavy.p, idx.W12.n_heavy, idx.beta, idx.Wr32u.p, ldr, 0.0,
                nullptr, ldr, U, ldr, r, nullptr, 0, nullptr, s);
    m11_solve<float>(idx, U, H, r, ldr, 1e-5, 500, nullptr, s);
  }
  idx.feat.alloc(size_t(n) * kFeat);
  const float mean_deg = float(double(idx.nnz) / double(std::max<int64_t>(n, 1)));
  features_kernel<<<blocks(n * kFeat), 256, 0, s>>>(idx.W.csr.rowptr.p, idx.iperm.p, n, n1, H,
                                                     idx.Wr32u.p, ldr, r, mean_deg, idx.feat.p);
  KATZ_CHECK_LAUNCH();
  double* mom = idx.ws.get<double>("wf.mom", 2 * kFeat);
  KATZ_CUDA(cudaMemsetAsync(mom, 0, 16 * kFeat, s));
  col_moments_kernel<<<256, 256, 0, s>>>(idx.feat.p, n, mom, mom + kFeat);
  KATZ_CHECK_LAUNCH();
  col_scale_kernel<<<blocks(n * kFeat), 256, 0, s>>>(idx.feat.p, n, mom, mom + kFeat);
  KATZ_CHECK_LAUNCH();
  // keep H (the harmonic extension of the basis) for the CG warm start
  if (n1 > 0) {
    idx.Hr.alloc(size_t(n1) * ldr);
    KATZ_CUDA(cudaMemcpyAsync(idx.Hr.p, H, 4 * size_t(n1) * ldr, cudaMemcpyDeviceToDevice, s));
  }
  idx.ws.release("wf.U");
  idx.ws.release("wf.H");
  KATZ_CUDA(cudaStreamSynchronize(s));
  (void)n2;
}

// H = beta M11^{-1} W12 W_r (n1 x ldr4), recomputed when an index was loaded
// from a file (the features are stored, H is not).
static void ensure_harmonic_basis(katz_index& idx, cudaStream_t s) {
  const int64_t n1 = idx.n1, ldr = idx.ldr4;
  if (idx.Hr.p || n1 == 0) return;
  float* U = idx.ws.get<float>("wf.U", size_t(n1) * ldr);
  idx.Hr.alloc(size_t(n1) * ldr);
  spmm<float>(idx.W12.view(), idx.W12.heavy.p, idx.W12.n_heavy, idx.beta, idx.Wr32u.p, ldr, 0.0,
              nullptr, ldr, U, ldr, idx.rank, nullptr, 0, nullptr, s);
  m11_solve<float>(idx, U, idx.Hr.p, idx.rank, ldr, 1e-5, 500, nullptr, s);
  idx.ws.release("wf.U");
}

// Targets c* (b x r, row j = query j) from K (node order, n x b, ldk).
static void targets_from_K(katz_index& idx, const float* K, int64_t ldk, int b, float* T,
                           cudaStream_t s) {
  const int64_t n2 = idx.n2, ld = (b + 3) / 4 * 4;
  const int r = idx.rank;
  float* k2 = idx.ws.get<float>("wt.k2", size_t(n2) * ld);
  float* mk = idx.ws.get<float>("wt.mk", size_t(n2) * ld);
  KATZ_CUDA(cudaMemsetAsync(k2, 0, 4 * n2 * ld, s));
  gather_sep_kernel<<<blocks(n2 * b), 256, 0, s>>>(K, ldk, idx.perm.p, idx.n1, n2, b, k2, ld);
  KATZ_CHECK_LAUNCH();
  // M22 k2 = k2 - beta W22 k2
  spmm<float>(idx.W22.view(), idx.W22.heavy.p, idx.W22.n_heavy, -idx.beta, k2, ld, 1.0, k2, ld, mk,
              ld, b, nullptr, 0, nullptr, s);
  // T (b x r) = (W_r^T M22 k2)^T = mk^T W_r
  gemm2<float>(true, false, b, r, n2, 1.0, mk, ld, idx.Wr32u.p, idx.ldr4, 0.0, T, r, false, s);
}

// C (b x r) = MLP(features of q): the predicted coordinates c_hat.
static const float* warm_coeffs(katz_index& idx, const int32_t* q, int b, cudaStream_t s) {
  const int r = idx.rank;
  float* X = idx.ws.get<float>("ws.X", size_t(b) * kFeat);
  float* Hp = idx.ws.get<float>("ws.Hp", size_t(b) * idx.mlp.dh);
  float* Hh = idx.ws.get<float>("ws.H", size_t(b) * idx.mlp.dh);
  float* C = idx.ws.get<float>("ws.C", size_t(b) * r);
  gather_feat_kernel<<<blocks(int64_t(b) * kFeat), 256, 0, s>>>(idx.feat.p, q, b, X);
  KATZ_CHECK_LAUNCH();
  idx.mlp.forward(X, b, Hp, Hh, C, s);
  return C;
}

// K2(0) (n2 x b, ld) = W_r C^T with C = MLP(features of q) (b x r)
void warm_start_guess(katz_index& idx, const int32_t* q, int b, float* K20, int64_t ld,
                      cudaStream_t s) {
  const float* C = warm_coeffs(idx, q, b, s);
  KATZ_CUDA(cudaMemsetAsync(K20, 0, 4 * idx.n2 * ld, s));
  gemm2<float>(false, true, idx.n2, b, idx.rank, 1.0, idx.Wr32u.p, idx.ldr4, C, idx.rank, 0.0, K20,
               ld, false, s);
}

namespace {
// Xn[i] = Xi[iperm[i]] (rows of b columns, both ld): index order -> node order
__global__ void unpermute_rows_kernel(const float* Xi, const int32_t* iperm, int64_t n, int b,
                                      int64_t ld, float* Xn) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n * b;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / b;
    const int j = int(e - i * b);
    Xn[i * ld + j] = Xi[int64_t(iperm[i]) * ld + j];
  }
}
}  // namespace

// Initial guess of CG on M (node order, n x b, ld; padding columns zero):
// the whole Katz vector the LRC decomposition predicts from c_hat,
//   K2(0) = W_r c_hat,  K1(0) = M11^{-1} B1 + beta M11^{-1} W12 W_r c_hat
// (Eq. 6 with K2 replaced by the network's separator part; the first term
// is one M11 solve of the right-hand side to 1e-4, the second the stored
// harmonic extension H of the basis times c_hat).  Its error is the
// harmonic extension of the separator error K2 - W_r c_hat alone.
void warm_cg_guess(katz_index& idx, const int32_t* q, int b, float* X, int64_t ld,
                   cudaStream_t s) {
  KATZ_REQUIRE(idx.lrc && idx.rank > 0 && idx.mlp.ready && idx.feat.p, KATZ_EINVAL,
               "warm start needs an LRC index with a trained warm-start network");
  ensure_harmonic_basis(idx, s);
  const int64_t n = idx.n, n1 = idx.n1, n2 = idx.n2;
  const int r = idx.rank;
  float* Bi = idx.ws.get<float>("wg.B", size_t(n) * ld);
  float* Xi = idx.ws.get<float>("wg.X", size_t(n) * ld);
  KATZ_CUDA(cudaMemsetAsync(Bi, 0, 4 * size_t(n) * ld, s));
  KATZ_CUDA(cudaMemsetAsync(Xi, 0, 4 * size_t(n) * ld, s));
  const float* C = warm_coeffs(idx, q, b, s);
  // separator rows: W_r c_hat
  gemm2<float>(false, true, n2, b, r, 1.0, idx.Wr32u.p, idx.ldr4, C, r, 0.0, Xi + n1 * ld, ld,
               false, s);
  if (n1 > 0) {
    build_rhs<float>(idx.W.view(), q, b, idx.beta, idx.iperm.p, Bi, ld, s);
    m11_solve<float>(idx, Bi, Xi, b, ld, 1e-4, 500, nullptr, s);
    gemm2<float>(false, true, n1, b, r, 1.0, idx.Hr.p, idx.ldr4, C, r, 1.0, Xi, ld, false, s);
  }
  unpermute_rows_kernel<<<blocks(n * b), 256, 0, s>>>(Xi, idx.iperm.p, n, b, ld, X);
  KATZ_CHECK_LAUNCH();
}

double warmstart_train(katz_index& idx, const int32_t* q_host, int n_train, int hidden, int epochs,
                       int batch, float lr, float wd, uint64_t seed, double* init_loss, int* steps,
                       cudaStream_t s) {
  KATZ_REQUIRE(n_train > 0 && hidden > 0 && epochs > 0 && batch > 0, KATZ_EINVAL,
               "bad training options");
  warm_features(idx, s);
  const int r = idx.rank;
  // 1. targets: the method's own Katz vectors, in batches of up to 1024
  DBuf<float> Xall(size_t(n_train) * kFeat), Tall(size_t(n_train) * r);
  DBuf<int32_t> qd(n_train);
  KATZ_CUDA(cudaMemcpyAsync(qd.p, q_host, 4 * size_t(n_train), cudaMemcpyHostToDevice, s));
  gather_feat_kernel<<<blocks(int64_t(n_train) * kFeat), 256, 0, s>>>(idx.feat.p, qd.p, n_train,
                                                                      Xall.p);
  KATZ_CHECK_LAUNCH();
  katz_query_opts o{};
  o.tol = 1e-6;
  o.tol_kind = KATZ_TOL_ERROR_INF;
  o.precision = KATZ_PREC_MIXED;
  const int chunk = 1024;
  float* Kb = idx.ws.get<float>("wt.K", size_t(idx.n) * chunk);
  for (int j0 = 0; j0 < n_train; j0 += chunk) {
    const int bb = std::min(chunk, n_train - j0);
    const int st = run_queries_internal(idx, qd.p + j0, q_host + j0, bb, o, Kb, KATZ_F32, bb, s);
    KATZ_REQUIRE(st == KATZ_OK || st == KATZ_ENOCONV, st, "target solve failed");
    targets_from_K(idx, Kb, bb, bb, Tall.p + int64_t(j0) * r, s);
  }
  idx.ws.release("wt.K");
  // 2. training (minibatch AdamW, rows in a fixed seeded order per epoch)
  idx.mlp.init(kFeat, hidden, r, seed, s);
  std::vector<int32_t> order(n_train);
  for (int i = 0; i < n_train; ++i) order[i] = i;
  uint64_t st = seed ^ 0x5DEECE66Dull;
  auto rnd = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  float* Xb = idx.ws.get<float>("wt.Xb", size_t(batch) * kFeat);
  float* Tb = idx.ws.get<float>("wt.Tb", size_t(batch) * r);
  DBuf<int32_t> ordd(n_train);
  double loss = 0;
  *init_loss = -1;
  *steps = 0;
  std::vector<float> hx(size_t(n_train) * kFeat), ht(size_t(n_train) * r);
  KATZ_CUDA(cudaMemcpyAsync(hx.data(), Xall.p, 4 * hx.size(), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaMemcpyAsync(ht.data(), Tall.p, 4 * ht.size(), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  std::vector<float> bx(size_t(batch) * kFeat), bt(size_t(batch) * r);
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = n_train - 1; i > 0; --i) std::swap(order[i], order[rnd() % uint64_t(i + 1)]);
    for (int b0 = 0; b0 < n_train; b0 += batch) {
      const int m = std::min(batch, n_train - b0);
      for (int t = 0; t < m; ++t) {
        std::copy_n(hx.data() + size_t(order[b0 + t]) * kFeat, kFeat, bx.data() + size_t(t) * kFeat);
        std::copy_n(ht.data() + size_t(order[b0 + t]) * r, r, bt.data() + size_t(t) * r);
      }
      KATZ_CUDA(cudaMemcpyAsync(Xb, bx.data(), 4 * size_t(m) * kFeat, cudaMemcpyHostToDevice, s));
      KATZ_CUDA(cudaMemcpyAsync(Tb, bt.data(), 4 * size_t(m) * r, cudaMemcpyHostToDevice, s));
      loss = idx.mlp.loss_grad(Xb, Tb, m, idx.ws, s);
      if (*init_loss < 0) *init_loss = loss;
      idx.mlp.adamw(lr, wd, s);
      ++*steps;
    }
  }
  // final loss over the whole training set
  loss = idx.mlp.loss_grad(Xall.p, Tall.p, n_train, idx.ws, s);
  (void)ordd;
  return loss;
}

}  // namespace katz
