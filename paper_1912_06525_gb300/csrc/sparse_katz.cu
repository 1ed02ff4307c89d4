// Sparse-Katz re-ranking of link-prediction lists (Algorithm 3, Section
// 3.3, Fig. 2), batched over b queries:
//   1. K = [k_q] for the b queries (LRC-Katz, or CG on an index without the
//      LRC part);
//   2. per column, the Top-s link candidates (q and its neighbours left
//      out) and the T landmark nodes (the T highest scores, only q left
//      out), by the two-pass top-k kernels;
//   3. the Katz vectors k_t of the DISTINCT landmarks of the batch (queries
//      often share landmarks, e.g. hubs; k_t does not depend on which query
//      chose t), solved in batches of up to 1,024 columns; after each batch
//      one kernel keeps only the entries the correlation needs, row q and
//      the s candidate rows of K_T, for every (query, landmark) pair whose
//      landmark is in the batch;
//   4. one CTA per query: rho_c = Pearson correlation of rows q and c of
//      K_T in FP64, and the candidates re-ordered by rho descending (ties
//      in Katz order).
#include <algorithm>
#include <chrono>

#include "index.h"
#include "kernels_dense.h"

namespace katz {
namespace {

constexpr int kSkMax = 64;      // s and T
constexpr int kSkChunk = 1024;  // landmark columns per solve

// Pair g = j * T + t (landmark t of query j) uses column umap[g] - c0 of
// this batch of distinct-landmark solves when c0 <= umap[g] < c0 + w.  Row 0
// of the block grid copies K_T[q_j][col] to X[j][t]; row 1 + i copies
// K_T[cand_j,i][col] to Y[j][i][t] (0 for a missing candidate).
__global__ void sk_gather_kernel(const float* __restrict__ KT, int64_t ldk, int64_t c0, int w,
                                 const int32_t* __restrict__ umap, int64_t pairs,
                                 const int32_t* __restrict__ q, const int32_t* __restrict__ cand,
                                 int s, int T, double* __restrict__ X, double* __restrict__ Y) {
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= pairs) return;
  const int64_t c = int64_t(umap[g]) - c0;
  if (c < 0 || c >= w) return;
  const int i = blockIdx.y;
  const int64_t j = g / T, t = g % T;
  const int64_t row = i == 0 ? int64_t(q[j]) : int64_t(cand[j * s + i - 1]);
  const double v = row >= 0 ? double(KT[row * ldk + c]) : 0.0;
  if (i == 0)
    X[j * T + t] = v;
  else
    Y[(j * s + i - 1) * T + t] = v;
}

// One CTA (kSkMax threads) per query: thread i correlates candidate i.
// Candidates come in Katz order with missing ones (-1) at the tail; the
// valid ones are ranked by (rho descending, Katz position ascending), the
// missing ones keep their places.
__global__ void __launch_bounds__(kSkMax) sk_rank_kernel(const double* __restrict__ X,
                                                         const double* __restrict__ Y,
                                                         const int32_t* __restrict__ cand, int s,
                                                         int T, int32_t* __restrict__ ids,
                                                         double* __restrict__ rho_out) {
  __shared__ double rho[kSkMax];
  __shared__ int ok[kSkMax];
  const int j = blockIdx.x, i = threadIdx.x;
  const double* x = X + int64_t(j) * T;
  double mx = 0.0;
  for (int t = 0; t < T; ++t) mx += x[t];
  mx /= T;
  const int id = i < s ? cand[int64_t(j) * s + i] : -1;
  double r = 0.0;
  if (id >= 0) {
    const double* y = Y + (int64_t(j) * s + i) * T;
    double my = 0.0;
    for (int t = 0; t < T; ++t) my += y[t];
    my /= T;
    double sxy = 0.0, sxx = 0.0, syy = 0.0;
    for (int t = 0; t < T; ++t) {
      const double dx = x[t] - mx, dy = y[t] - my;
      sxy += dx * dy;
      sxx += dx * dx;
      syy += dy * dy;
    }
    r = (sxx > 0.0 && syy > 0.0) ? sxy / sqrt(sxx * syy) : 0.0;
  }
  rho[i] = r;
  ok[i] = id >= 0;
  __syncthreads();
  if (i >= s) return;
  int pos = i;
  if (id >= 0) {
    pos = 0;
    for (int u = 0; u < s; ++u)
      if (ok[u] && (rho[u] > r || (rho[u] == r && u < i))) ++pos;
  }
  ids[int64_t(j) * s + pos] = id;
  rho_out[int64_t(j) * s + pos] = r;
}

void merge_stats(katz_stats* acc, const katz_stats& st) {
  acc->iters = std::max(acc->iters, st.iters);
  acc->refine_steps = std::max(acc->refine_steps, st.refine_steps);
  acc->max_rel_res = std::max(acc->max_rel_res, st.max_rel_res);
}

}  // namespace

int sparse_katz(katz_index& idx, const int32_t* q_dev, const int32_t* q_host, int b, int s_top,
                int T, const katz_query_opts& o, int32_t* ids, double* rho, int32_t* land_out,
                katz_stats* st, cudaStream_t s) {
  KATZ_REQUIRE(s_top >= 1 && s_top <= kSkMax, KATZ_EINVAL, "s must be in [1, 64]");
  KATZ_REQUIRE(T >= 1 && T <= kSkMax, KATZ_EINVAL, "T must be in [1, 64]");
  KATZ_REQUIRE(T <= idx.n - 1, KATZ_EINVAL, "T must be below the number of nodes");
  KATZ_REQUIRE(b >= 1 && b <= 1024, KATZ_EINVAL, "b must be in [1, 1024]");
  const auto t0 = std::chrono::steady_clock::now();
  const bool lrc = idx.lrc;
  const int64_t n = idx.n;
  katz_stats acc{};
  katz_stats one{};
  std::vector<int32_t> it;
  std::vector<double> rr;
  // 1. the query columns
  QueryOut out;
  out.K = idx.ws.get<float>("sk.K", size_t(n) * b);
  out.dtype = KATZ_F32;
  out.ldk = b;
  int status = run_queries(idx, lrc, q_dev, q_host, b, o, out, &one, it, rr, s);
  if (status != KATZ_OK && status != KATZ_ENOCONV) return status;
  merge_stats(&acc, one);
  // 2. candidates and landmarks
  const int kmax = std::max(s_top, T);
  const int slices = (int)std::max<int64_t>(1, std::min<int64_t>(16, n / 65536 + 1));
  int32_t* wid = idx.ws.get<int32_t>("sk.tid", size_t(slices) * 8 * b * kmax);
  double* wsc = idx.ws.get<double>("sk.tsc", size_t(slices) * 8 * b * kmax);
  int32_t* cand = idx.ws.get<int32_t>("sk.cand", size_t(b) * s_top);
  double* csc = idx.ws.get<double>("sk.csc", size_t(b) * kmax);
  int32_t* land = idx.ws.get<int32_t>("sk.land", size_t(b) * T);
  const float* K0 = static_cast<const float*>(out.K);
  topk_columns_ws<float>(idx.W.view(), K0, b, n, q_dev, b, s_top, cand, csc, wid, wsc, slices, s,
                         true);
  topk_columns_ws<float>(idx.W.view(), K0, b, n, q_dev, b, T, land, csc, wid, wsc, slices, s,
                         false);
  std::vector<int32_t> land_h(size_t(b) * T);
  KATZ_CUDA(cudaMemcpyAsync(land_h.data(), land, 4 * land_h.size(), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  for (int32_t v : land_h)
    KATZ_REQUIRE(v >= 0 && v < n, KATZ_ECUDA, "landmark selection returned an invalid node");
  // 3. the distinct landmarks (ascending ids) and each pair's index among them
  const int64_t pairs = int64_t(b) * T;
  std::vector<int32_t> uniq(land_h.begin(), land_h.end());
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  std::vector<int32_t> umap_h(pairs);
  for (int64_t g = 0; g < pairs; ++g)
    umap_h[g] = int32_t(std::lower_bound(uniq.begin(), uniq.end(), land_h[g]) - uniq.begin());
  const int64_t nu = (int64_t)uniq.size();
  int32_t* uq = idx.ws.get<int32_t>("sk.uq", size_t(nu));
  int32_t* umap = idx.ws.get<int32_t>("sk.umap", size_t(pairs));
  KATZ_CUDA(cudaMemcpyAsync(uq, uniq.data(), 4 * size_t(nu), cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(umap, umap_h.data(), 4 * size_t(pairs), cudaMemcpyHostToDevice, s));
  if (st) st->ms[6] = double(nu);
  // landmark solves, keeping rows q and the candidates of K_T
  double* X = idx.ws.get<double>("sk.X", size_t(b) * T);
  double* Y = idx.ws.get<double>("sk.Y", size_t(b) * s_top * T);
  const int wmax = (int)std::min<int64_t>(kSkChunk, nu);
  float* KT = idx.ws.get<float>("sk.KT", size_t(n) * wmax);
  for (int64_t c0 = 0; c0 < nu; c0 += wmax) {
    const int w = (int)std::min<int64_t>(wmax, nu - c0);
    QueryOut ot;
    ot.K = KT;
    ot.dtype = KATZ_F32;
    ot.ldk = w;
    one = katz_stats{};
    const int st2 = run_queries(idx, lrc, uq + c0, uniq.data() + c0, w, o, ot, &one, it, rr, s);
    if (st2 != KATZ_OK && st2 != KATZ_ENOCONV) return st2;
    if (st2 == KATZ_ENOCONV) status = KATZ_ENOCONV;
    merge_stats(&acc, one);
    dim3 grid((unsigned)ceil_div(pairs, 128), (unsigned)(s_top + 1));
    sk_gather_kernel<<<grid, 128, 0, s>>>(KT, w, c0, w, umap, pairs, q_dev, cand, s_top, T, X, Y);
    KATZ_CHECK_LAUNCH();
  }
  // 4. correlation and re-ranking
  sk_rank_kernel<<<(unsigned)b, kSkMax, 0, s>>>(X, Y, cand, s_top, T, ids, rho);
  KATZ_CHECK_LAUNCH();
  if (land_out)
    KATZ_CUDA(cudaMemcpyAsync(land_out, land, 4 * size_t(b) * T, cudaMemcpyDeviceToDevice, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  if (st) {
    const double nu_d = st->ms[6];
    *st = acc;
    st->ms[0] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                    .count();
    st->ms[6] = nu_d;
  }
  return status;
}

}  // namespace katz
