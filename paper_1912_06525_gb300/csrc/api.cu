// extern "C" boundary of libkatz.so (declared in include/katz.h).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "index.h"
#include "kernels_dense.h"
#include "tc_gemm.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

template <class F>
int guarded(F&& f) {
  try {
    g_last_error.clear();
    return f();
  } catch (const katz::Error& e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(KATZ_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(KATZ_ECUDA, e.what());
  }
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Validate a host CSR and copy it into katz::HostCsr.
katz::HostCsr read_csr(const katz_csr* W) {
  KATZ_REQUIRE(W && W->rowptr && (W->col || W->nnz == 0), KATZ_EINVAL, "null CSR");
  KATZ_REQUIRE(W->n >= 0 && W->n < (int64_t(1) << 31), KATZ_EINVAL, "n out of range");
  KATZ_REQUIRE(W->rowptr[0] == 0 && W->rowptr[W->n] == W->nnz, KATZ_EINVAL,
               "rowptr must start at 0 and end at nnz");
  katz::HostCsr h;
  h.nrows = h.ncols = W->n;
  h.rowptr.assign(W->rowptr, W->rowptr + W->n + 1);
  h.col.assign(W->col, W->col + W->nnz);
  if (W->val) h.val.assign(W->val, W->val + W->nnz);
  for (int64_t i = 0; i < W->n; ++i) {
    KATZ_REQUIRE(h.rowptr[i + 1] >= h.rowptr[i], KATZ_EINVAL, "rowptr not monotone");
    for (int64_t k = h.rowptr[i]; k < h.rowptr[i + 1]; ++k) {
      const int64_t c = h.col[k];
      KATZ_REQUIRE(c >= 0 && c < W->n, KATZ_EINVAL, "column index out of range");
      KATZ_REQUIRE(c != i, KATZ_EINVAL, "self-loop at node " + std::to_string(i));
      if (W->val) KATZ_REQUIRE(h.val[k] > 0 && std::isfinite(h.val[k]), KATZ_EINVAL,
                               "weights must be positive and finite");
    }
  }
  // symmetry: the transpose pattern (with values) must equal the original
  std::vector<int64_t> cnt(W->n + 1, 0);
  for (int64_t k = 0; k < W->nnz; ++k) cnt[h.col[k] + 1]++;
  for (int64_t i = 0; i < W->n; ++i) cnt[i + 1] += cnt[i];
  KATZ_REQUIRE(cnt == h.rowptr, KATZ_EINVAL, "W is not symmetric (row/column counts differ)");
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
  std::vector<int32_t> tcol(W->nnz);
  std::vector<double> tval(W->val ? W->nnz : 0);
  for (int64_t i = 0; i < W->n; ++i)
    for (int64_t k = h.rowptr[i]; k < h.rowptr[i + 1]; ++k) {
      const int64_t d = pos[h.col[k]]++;
      tcol[d] = (int32_t)i;
      if (W->val) tval[d] = h.val[k];
    }
  // compare row by row as multisets (sort both)
  std::vector<std::pair<int32_t, double>> a, b;
  for (int64_t i = 0; i < W->n; ++i) {
    a.clear();
    b.clear();
    for (int64_t k = h.rowptr[i]; k < h.rowptr[i + 1]; ++k) {
      a.emplace_back(h.col[k], W->val ? h.val[k] : 1.0);
      b.emplace_back(tcol[k], W->val ? tval[k] : 1.0);
    }
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    KATZ_REQUIRE(a == b, KATZ_EINVAL, "W is not symmetric at row " + std::to_string(i));
    for (size_t t = 1; t < a.size(); ++t)
      KATZ_REQUIRE(a[t].first != a[t - 1].first, KATZ_EINVAL,
                   "duplicate entry in row " + std::to_string(i));
  }
  return h;
}

// Device copy of the query ids (validated against n); the host copy is
// returned in *host when given.
const int32_t* stage_queries(katz_index* idx, const int32_t* q, int32_t b, cudaStream_t s,
                             std::vector<int32_t>* host = nullptr) {
  KATZ_REQUIRE(q != nullptr && b > 0, KATZ_EINVAL, "empty query list");
  std::vector<int32_t> h(b);
  if (is_device_ptr(q)) {
    KATZ_CUDA(cudaMemcpyAsync(h.data(), q, 4 * size_t(b), cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
  } else {
    std::memcpy(h.data(), q, 4 * size_t(b));
  }
  for (int j = 0; j < b; ++j)
    KATZ_REQUIRE(h[j] >= 0 && h[j] < idx->n, KATZ_EINVAL,
                 "query id " + std::to_string(h[j]) + " out of range");
  int32_t* d = idx->ws.get<int32_t>("api.q", b);
  KATZ_CUDA(cudaMemcpyAsync(d, h.data(), 4 * size_t(b), cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  if (host) *host = h;
  return d;
}

int do_query(const katz_index* cidx, bool lrc, const int32_t* q, int32_t b,
             const katz_query_opts* opts, void* K_out, int32_t out_dtype, int64_t ldk,
             katz_stats* stats, int32_t* iters_out, double* rel_res_out, void* stream) {
  return guarded([&]() {
    KATZ_REQUIRE(cidx && opts && K_out, KATZ_EINVAL, "null argument");
    KATZ_REQUIRE(out_dtype == KATZ_F32 || out_dtype == KATZ_F64, KATZ_EINVAL, "out_dtype");
    KATZ_REQUIRE(ldk >= b, KATZ_EINVAL, "ldk < b");
    KATZ_REQUIRE(opts->tol > 0, KATZ_EINVAL, "tol must be positive");
    katz_index* idx = const_cast<katz_index*>(cidx);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> qh;
    const int32_t* qd = stage_queries(idx, q, b, s, &qh);
    katz::QueryOut out;
    out.dtype = out_dtype;
    out.ldk = ldk;
    const bool dev = is_device_ptr(K_out);
    const size_t es = out_dtype == KATZ_F64 ? 8 : 4;
    if (dev) {
      out.K = K_out;
    } else {
      out.K = idx->ws.get<uint8_t>("api.K", es * size_t(idx->n) * ldk);
    }
    KATZ_REQUIRE(opts->rhs_width >= 0, KATZ_EINVAL, "rhs_width must be >= 0");
    const int32_t w = opts->rhs_width > 0 ? std::min(opts->rhs_width, b) : b;
    KATZ_REQUIRE(w <= 1024, KATZ_EINVAL,
                 "at most 1024 columns are solved together: b > 1024 needs rhs_width in [1, 1024]");
    std::vector<int32_t> it;
    std::vector<double> rr;
    int st = KATZ_OK;
    if (w == b) {
      st = katz::run_queries(*idx, lrc, qd, qh.data(), b, *opts, out, stats, it, rr, s);
    } else {
      // Column chunks of w queries, one solve each, in order; the chunk's
      // output is the column range [j0, j0 + bj) of K (node-major, so the
      // base moves by j0 elements and the leading dimension stays ldk).
      katz_stats acc{};
      double gamma_sum = 0;
      for (int32_t j0 = 0; j0 < b; j0 += w) {
        const int32_t bj = std::min(w, b - j0);
        katz::QueryOut oj = out;
        oj.K = static_cast<uint8_t*>(out.K) + es * size_t(j0);
        katz_stats sj{};
        std::vector<int32_t> itj;
        std::vector<double> rrj;
        const int stj = katz::run_queries(*idx, lrc, qd + j0, qh.data() + j0, bj, *opts, oj,
                                          stats ? &sj : nullptr, itj, rrj, s);
        if (stj != KATZ_OK && stj != KATZ_ENOCONV) {
          st = stj;
          break;
        }
        if (stj == KATZ_ENOCONV) st = KATZ_ENOCONV;
        it.insert(it.end(), itj.begin(), itj.end());
        rr.insert(rr.end(), rrj.begin(), rrj.end());
        if (stats) {
          acc.iters = std::max(acc.iters, sj.iters);
          acc.refine_steps = std::max(acc.refine_steps, sj.refine_steps);
          acc.max_rel_res = std::max(acc.max_rel_res, sj.max_rel_res);
          for (int k : {0, 1, 2, 3, 4, 5}) acc.ms[k] += sj.ms[k];
          gamma_sum += sj.ms[6] * bj;
          acc.ms[7] = std::max(acc.ms[7], sj.ms[7]);
        }
      }
      if (stats) {
        acc.ms[6] = gamma_sum / b;
        *stats = acc;
      }
    }
    if (!dev && (st == KATZ_OK || st == KATZ_ENOCONV)) {
      // the b columns of each row only: the caller's entries between b and
      // ldk stay as they were, as with a device K_out
      KATZ_CUDA(cudaMemcpy2DAsync(K_out, es * size_t(ldk), out.K, es * size_t(ldk),
                                  es * size_t(b), size_t(idx->n), cudaMemcpyDeviceToHost, s));
      KATZ_CUDA(cudaStreamSynchronize(s));
    }
    if (iters_out) std::memcpy(iters_out, it.data(), 4 * it.size());
    if (rel_res_out) std::memcpy(rel_res_out, rr.data(), 8 * rr.size());
    if (st == KATZ_ENOCONV) g_last_error = "iteration or refinement cap reached";
    if (st == KATZ_ENOTSPD) g_last_error = "CG breakdown: p^T A p <= 0 (M not positive definite)";
    return st;
  });
}

}  // namespace

void katz::set_last_error(const std::string& msg) { g_last_error = msg; }

extern "C" {

const char* katz_last_error(void) { return g_last_error.c_str(); }

int katz_lambda_bounds(const katz_csr* W, int32_t steps, double* ritz, double* upper,
                       void* stream) {
  return guarded([&]() {
    KATZ_REQUIRE(ritz || upper, KATZ_EINVAL, "null outputs");
    katz::HostCsr h = read_csr(W);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    katz::GraphPart g;
    katz::upload_csr(h, h.val.empty() ? KATZ_UNIT : KATZ_F64, g.csr, s);
    std::vector<int32_t> heavy;
    for (int64_t i = 0; i < h.nrows; ++i)
      if (h.rowptr[i + 1] - h.rowptr[i] > katz::kHeavyRowNnz) heavy.push_back((int32_t)i);
    g.n_heavy = (int64_t)heavy.size();
    g.heavy.alloc(std::max<size_t>(1, heavy.size()));
    if (!heavy.empty())
      KATZ_CUDA(cudaMemcpy(g.heavy.p, heavy.data(), 4 * heavy.size(), cudaMemcpyHostToDevice));
    katz::Workspace ws;
    double up = 0;
    const double r = katz::lambda_max_gpu(g, h.nrows, steps > 0 ? steps : 64, ws, s, 0, nullptr,
                                          upper ? &up : nullptr);
    if (ritz) *ritz = r;
    if (upper) *upper = up;
    return KATZ_OK;
  });
}

int katz_lambda_max(const katz_csr* W, int32_t steps, double* out, void* stream) {
  if (!out) return guarded([&]() -> int { throw katz::Error(KATZ_EINVAL, "null output"); });
  return katz_lambda_bounds(W, steps, out, nullptr, stream);
}

int katz_index_build(const katz_csr* W, double beta, const katz_build_opts* opts, void* stream,
                     katz_index** out) {
  return guarded([&]() {
    KATZ_REQUIRE(out && opts, KATZ_EINVAL, "null argument");
    *out = nullptr;
    KATZ_REQUIRE(beta > 0 && std::isfinite(beta), KATZ_EINVAL, "beta must be positive");
    KATZ_REQUIRE(opts->value_dtype >= KATZ_UNIT && opts->value_dtype <= KATZ_BF16, KATZ_EINVAL,
                 "value_dtype");
    katz::HostCsr h = read_csr(W);
    if (opts->value_dtype == KATZ_UNIT)
      for (double v : h.val)
        KATZ_REQUIRE(v == 1.0, KATZ_EINVAL, "value_dtype UNIT needs all weights equal to 1");
    auto* idx = new katz_index();
    try {
      katz::build_index(*idx, h, beta, *opts, static_cast<cudaStream_t>(stream));
    } catch (...) {
      delete idx;
      throw;
    }
    *out = idx;
    return KATZ_OK;
  });
}

void katz_index_free(katz_index* idx) { delete idx; }

int katz_index_save(const katz_index* idx, const char* path) {
  return guarded([&]() {
    KATZ_REQUIRE(idx && path, KATZ_EINVAL, "null argument");
    KATZ_CUDA(cudaDeviceSynchronize());
    katz::save_index(*idx, path);
    return KATZ_OK;
  });
}

int katz_index_load(const char* path, katz_index** out) {
  return guarded([&]() {
    KATZ_REQUIRE(out && path, KATZ_EINVAL, "null argument");
    *out = nullptr;
    std::unique_ptr<katz_index> idx = katz::load_index(path);
    KATZ_CUDA(cudaDeviceSynchronize());
    *out = idx.release();
    return KATZ_OK;
  });
}

int katz_index_get_info(const katz_index* idx, katz_index_info* info) {
  return guarded([&]() {
    KATZ_REQUIRE(idx && info, KATZ_EINVAL, "null argument");
    std::memset(info, 0, sizeof(*info));
    info->n = idx->n;
    info->nnz = idx->nnz;
    info->n1 = idx->n1;
    info->n2 = idx->n2;
    info->n_blocks = idx->lrc ? (int32_t)(idx->part.block_ptr.size() - 1) : 0;
    info->n_large_blocks = idx->n_large;
    info->rank = idx->rank;
    info->value_dtype = idx->vdt;
    info->beta = idx->beta;
    info->lambda_max_R = idx->sigma.empty() ? 0.0 : idx->sigma[0];
    info->lambda_max_W = idx->lambda;
    info->lambda_upper = idx->lambda_up;
    info->schur_implicit = idx->s_implicit ? 1 : 0;
    info->rhs_coupling = idx->has_z ? 1 : 0;
    int64_t bytes = idx->W.csr.bytes() + idx->Wp.csr.bytes() + idx->W12.csr.bytes() +
                    idx->W21.csr.bytes() + idx->W11L.csr.bytes() + idx->W22.csr.bytes() +
                    idx->S32.bytes() + idx->S64.bytes() + idx->M22inv32.bytes() +
                    idx->M22inv64.bytes() + idx->Wr32.bytes() + idx->Wr64.bytes() +
                    idx->Wb.bytes() + idx->WbT.bytes() + idx->Wr32u.bytes() + idx->Hh.bytes() +
                    idx->Hl.bytes() + idx->Zc.bytes() + idx->Sh.bytes() + idx->Sl.bytes() +
                    idx->Mh.bytes() + idx->Ml.bytes() + idx->Hr.bytes() + idx->feat.bytes() +
                    (int64_t)idx->ws.bytes();
    for (auto& c : idx->classes) bytes += c.inv32.bytes() + c.inv64.bytes();
    info->device_bytes = bytes;
    return KATZ_OK;
  });
}

int katz_index_get_partition(const katz_index* idx, int64_t* perm, int64_t* block_ptr) {
  return guarded([&]() {
    KATZ_REQUIRE(idx && idx->lrc, KATZ_EINVAL, "index has no partition");
    if (perm) std::memcpy(perm, idx->part.perm.data(), 8 * idx->part.perm.size());
    if (block_ptr)
      std::memcpy(block_ptr, idx->part.block_ptr.data(), 8 * idx->part.block_ptr.size());
    return KATZ_OK;
  });
}

int katz_partition(const katz_csr* W, int32_t n_hubs, int32_t block_max, int32_t split,
                   int64_t* perm, int64_t* block_ptr, int64_t* n_blocks, int64_t* n1) {
  return guarded([&]() {
    KATZ_REQUIRE(perm && block_ptr && n_blocks && n1, KATZ_EINVAL, "null output");
    KATZ_REQUIRE(block_max > 0, KATZ_EINVAL, "block_max must be positive");
    katz::HostCsr h = read_csr(W);
    katz::Partition p = katz::partition_graph(h, std::max(0, n_hubs), block_max, split != 0);
    std::memcpy(perm, p.perm.data(), 8 * p.perm.size());
    std::memcpy(block_ptr, p.block_ptr.data(), 8 * p.block_ptr.size());
    *n_blocks = (int64_t)p.block_ptr.size() - 1;
    *n1 = p.n1;
    return KATZ_OK;
  });
}

int katz_index_get_sigma(const katz_index* idx, double* sigma) {
  return guarded([&]() {
    KATZ_REQUIRE(idx && sigma, KATZ_EINVAL, "null argument");
    std::memcpy(sigma, idx->sigma.data(), 8 * idx->sigma.size());
    return KATZ_OK;
  });
}

int katz_query_batch(const katz_index* idx, const int32_t* q, int32_t b,
                     const katz_query_opts* opts, void* K_out, int32_t out_dtype, int64_t ldk,
                     katz_stats* stats, int32_t* iters_out, double* rel_res_out, void* stream) {
  return do_query(idx, true, q, b, opts, K_out, out_dtype, ldk, stats, iters_out, rel_res_out,
                  stream);
}

int cg_query_batch(const katz_index* idx, const int32_t* q, int32_t b,
                   const katz_query_opts* opts, void* K_out, int32_t out_dtype, int64_t ldk,
                   katz_stats* stats, int32_t* iters_out, double* rel_res_out, void* stream) {
  return do_query(idx, false, q, b, opts, K_out, out_dtype, ldk, stats, iters_out, rel_res_out,
                  stream);
}

int linkpred_topk(const katz_index* cidx, const int32_t* q, int32_t b, const void* K,
                  int32_t k_dtype, int64_t ldk, int32_t k, int32_t* ids_out, double* scores_out,
                  void* stream) {
  return guarded([&]() {
    KATZ_REQUIRE(cidx && K && ids_out && scores_out, KATZ_EINVAL, "null argument");
    KATZ_REQUIRE(k > 0 && k <= 64, KATZ_EINVAL, "k must be in [1, 64]");
    KATZ_REQUIRE(k_dtype == KATZ_F32 || k_dtype == KATZ_F64, KATZ_EINVAL, "k_dtype");
    KATZ_REQUIRE(ldk >= b, KATZ_EINVAL, "ldk < b");
    katz_index* idx = const_cast<katz_index*>(cidx);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int32_t* qd = stage_queries(idx, q, b, s);
    const size_t es = k_dtype == KATZ_F64 ? 8 : 4;
    const void* Kd = K;
    if (!is_device_ptr(K)) {
      void* t = idx->ws.get<uint8_t>("api.Kin", es * size_t(idx->n) * ldk);
      KATZ_CUDA(cudaMemcpyAsync(t, K, es * size_t(idx->n) * ldk, cudaMemcpyHostToDevice, s));
      Kd = t;
    }
    const int slices = (int)std::max<int64_t>(1, std::min<int64_t>(16, idx->n / 65536 + 1));
    int32_t* wid = idx->ws.get<int32_t>("tk.id", size_t(slices) * 8 * b * k);
    double* wsc = idx->ws.get<double>("tk.sc", size_t(slices) * 8 * b * k);
    const bool dev_ids = is_device_ptr(ids_out), dev_sc = is_device_ptr(scores_out);
    int32_t* ids = dev_ids ? ids_out : idx->ws.get<int32_t>("tk.oid", size_t(b) * k);
    double* sc = dev_sc ? scores_out : idx->ws.get<double>("tk.osc", size_t(b) * k);
    if (k_dtype == KATZ_F32)
      katz::topk_columns_ws<float>(idx->W.view(), static_cast<const float*>(Kd), ldk, idx->n, qd, b,
                                   k, ids, sc, wid, wsc, slices, s);
    else
      katz::topk_columns_ws<double>(idx->W.view(), static_cast<const double*>(Kd), ldk, idx->n, qd,
                                    b, k, ids, sc, wid, wsc, slices, s);
    if (!dev_ids)
      KATZ_CUDA(cudaMemcpyAsync(ids_out, ids, 4 * size_t(b) * k, cudaMemcpyDeviceToHost, s));
    if (!dev_sc)
      KATZ_CUDA(cudaMemcpyAsync(scores_out, sc, 8 * size_t(b) * k, cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    return KATZ_OK;
  });
}

int sparse_katz_topk(const katz_index* cidx, const int32_t* q, int32_t b, int32_t s_top,
                     int32_t T, const katz_query_opts* opts, int32_t* ids_out, double* rho_out,
                     int32_t* landmarks_out, katz_stats* stats, void* stream) {
  return guarded([&]() {
    KATZ_REQUIRE(cidx && opts && ids_out && rho_out, KATZ_EINVAL, "null argument");
    KATZ_REQUIRE(opts->tol > 0, KATZ_EINVAL, "tol must be positive");
    katz_index* idx = const_cast<katz_index*>(cidx);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> qh;
    const int32_t* qd = stage_queries(idx, q, b, s, &qh);
    const bool dev_ids = is_device_ptr(ids_out), dev_rho = is_device_ptr(rho_out);
    const bool dev_land = landmarks_out && is_device_ptr(landmarks_out);
    int32_t* ids = dev_ids ? ids_out : idx->ws.get<int32_t>("sk.oid", size_t(b) * s_top);
    double* rho = dev_rho ? rho_out : idx->ws.get<double>("sk.orho", size_t(b) * s_top);
    int32_t* land = !landmarks_out ? nullptr
                    : dev_land     ? landmarks_out
                                   : idx->ws.get<int32_t>("sk.oland", size_t(b) * T);
    const int st = katz::sparse_katz(*idx, qd, qh.data(), b, s_top, T, *opts, ids, rho, land,
                                     stats, s);
    if (st != KATZ_OK && st != KATZ_ENOCONV) return st;
    if (!dev_ids)
      KATZ_CUDA(cudaMemcpyAsync(ids_out, ids, 4 * size_t(b) * s_top, cudaMemcpyDeviceToHost, s));
    if (!dev_rho)
      KATZ_CUDA(cudaMemcpyAsync(rho_out, rho, 8 * size_t(b) * s_top, cudaMemcpyDeviceToHost, s));
    if (landmarks_out && !dev_land)
      KATZ_CUDA(cudaMemcpyAsync(landmarks_out, land, 4 * size_t(b) * T, cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    if (st == KATZ_ENOCONV) g_last_error = "iteration or refinement cap reached";
    return st;
  });
}

int katz_warmstart_train(katz_index* idx, const int32_t* q_train, int32_t n_train,
                         const katz_train_opts* opts, katz_train_stats* stats, void* stream) {
  return guarded([&]() {
    KATZ_REQUIRE(idx && q_train && opts && n_train > 0, KATZ_EINVAL, "bad training arguments");
    KATZ_REQUIRE(idx->lrc && idx->rank > 0, KATZ_EINVAL, "warm start needs an LRC index with rank > 0");
    std::vector<int32_t> h(n_train);
    if (is_device_ptr(q_train)) {
      KATZ_CUDA(cudaMemcpy(h.data(), q_train, 4 * size_t(n_train), cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(h.data(), q_train, 4 * size_t(n_train));
    }
    for (int32_t v : h) KATZ_REQUIRE(v >= 0 && v < idx->n, KATZ_EINVAL, "training id out of range");
    const auto t0 = std::chrono::steady_clock::now();
    double init = 0;
    int steps = 0;
    const double fin = katz::warmstart_train(
        *idx, h.data(), n_train, opts->hidden > 0 ? opts->hidden : 256,
        opts->epochs > 0 ? opts->epochs : 20, opts->batch > 0 ? opts->batch : 256,
        opts->lr > 0 ? opts->lr : 1e-3f, opts->weight_decay, opts->seed, &init, &steps,
        static_cast<cudaStream_t>(stream));
    if (stats) {
      stats->initial_loss = init;
      stats->final_loss = fin;
      stats->steps = steps;
      stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return KATZ_OK;
  });
}

int katz_mlp_loss_grad(int32_t m, int32_t din, int32_t dh, int32_t dout, const float* X,
                       const float* T, const float* params, float* grads, double* loss,
                       void* stream) {
  return guarded([&]() {
    KATZ_REQUIRE(m > 0 && din > 0 && dh > 0 && dout > 0 && X && T && params && grads && loss,
                 KATZ_EINVAL, "bad arguments");
    KATZ_REQUIRE(is_device_ptr(X) && is_device_ptr(T) && is_device_ptr(params) &&
                     is_device_ptr(grads),
                 KATZ_EINVAL, "device pointers required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    katz::Mlp net;
    net.din = din;
    net.dh = dh;
    net.dout = dout;
    std::vector<float> h(net.n_params());
    KATZ_CUDA(cudaMemcpy(h.data(), params, 4 * h.size(), cudaMemcpyDeviceToHost));
    net.set_params(h.data(), s);
    katz::Workspace ws;
    *loss = net.loss_grad(X, T, m, ws, s);
    KATZ_CUDA(cudaMemcpyAsync(grads, net.grads.p, 4 * h.size(), cudaMemcpyDeviceToDevice, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    return KATZ_OK;
  });
}

int katz_multi_build(int32_t g, const katz_csr* Ws, const double* betas, int32_t value_dtype,
                     void* stream, katz_multi** out) {
  return guarded([&]() {
    KATZ_REQUIRE(out && Ws && betas && g > 0, KATZ_EINVAL, "bad multi-graph arguments");
    *out = nullptr;
    std::vector<katz::HostCsr> hs;
    hs.reserve(g);
    for (int32_t i = 0; i < g; ++i) {
      hs.push_back(read_csr(&Ws[i]));
      if (value_dtype == KATZ_UNIT)
        for (double v : hs.back().val)
          KATZ_REQUIRE(v == 1.0, KATZ_EINVAL, "value_dtype UNIT needs all weights equal to 1");
    }
    auto* m = new katz_multi();
    try {
      katz::multi_build(*m, hs, betas, value_dtype, static_cast<cudaStream_t>(stream));
    } catch (...) {
      delete m;
      throw;
    }
    *out = m;
    return KATZ_OK;
  });
}

int katz_index_build_many(int32_t g, const katz_csr* Ws, const double* betas,
                          const katz_build_opts* opts, void* stream, katz_multi** out) {
  return guarded([&]() {
    KATZ_REQUIRE(out && Ws && betas && opts && g > 0, KATZ_EINVAL, "bad multi-graph arguments");
    *out = nullptr;
    std::vector<katz::HostCsr> hs;
    hs.reserve(g);
    for (int32_t i = 0; i < g; ++i) {
      hs.push_back(read_csr(&Ws[i]));
      if (opts->value_dtype == KATZ_UNIT)
        for (double v : hs.back().val)
          KATZ_REQUIRE(v == 1.0, KATZ_EINVAL, "value_dtype UNIT needs all weights equal to 1");
    }
    auto* m = new katz_multi();
    try {
      katz::multi_build_lrc(*m, hs, betas, *opts, static_cast<cudaStream_t>(stream));
    } catch (...) {
      delete m;
      throw;
    }
    *out = m;
    return KATZ_OK;
  });
}

int katz_multi_get_info(const katz_multi* m, int64_t* n2_out, int32_t* ranks_out,
                        double* sigma_out) {
  return guarded([&]() {
    KATZ_REQUIRE(m && m->lrc, KATZ_EINVAL, "multi-graph index has no LRC part");
    const katz_index& L = *m->lrc;
    std::vector<int64_t> n2g(m->g, 0);
    for (int64_t p = 0; p < L.n2; ++p) {
      const int64_t node = L.part.perm[L.n1 + p];
      const int32_t gi = int32_t(std::upper_bound(m->seg_ptr_h.begin(), m->seg_ptr_h.end(), node) -
                                 m->seg_ptr_h.begin()) - 1;
      n2g[gi]++;
    }
    if (n2_out) std::memcpy(n2_out, n2g.data(), 8 * n2g.size());
    if (ranks_out)
      for (int32_t gi = 0; gi < m->g; ++gi)
        ranks_out[gi] = gi < (int32_t)L.seg_rank.size() ? L.seg_rank[gi] : 0;
    if (sigma_out && !L.sigma.empty()) std::memcpy(sigma_out, L.sigma.data(), 8 * L.sigma.size());
    return KATZ_OK;
  });
}

void katz_multi_free(katz_multi* m) { delete m; }

static int multi_query_api(const katz_multi* cm, const int32_t* q, int32_t qpg,
                           const katz_query_opts* opts, void* K_out, int32_t out_dtype,
                           int64_t ldk, katz_stats* stats, int32_t* iters_out,
                           double* rel_res_out, void* stream, bool use_lrc) {
  return guarded([&]() {
    KATZ_REQUIRE(cm && q && opts && K_out && qpg > 0 && qpg <= 64, KATZ_EINVAL, "bad arguments");
    KATZ_REQUIRE(out_dtype == KATZ_F32 || out_dtype == KATZ_F64, KATZ_EINVAL, "out_dtype");
    KATZ_REQUIRE(ldk >= qpg && opts->tol > 0, KATZ_EINVAL, "ldk < qpg or tol <= 0");
    katz_multi* m = const_cast<katz_multi*>(cm);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t total = int64_t(m->g) * qpg;
    std::vector<int32_t> h(total);
    if (is_device_ptr(q)) {
      KATZ_CUDA(cudaMemcpyAsync(h.data(), q, 4 * size_t(total), cudaMemcpyDeviceToHost, s));
      KATZ_CUDA(cudaStreamSynchronize(s));
    } else {
      std::memcpy(h.data(), q, 4 * size_t(total));
    }
    for (int32_t g = 0; g < m->g; ++g)
      for (int j = 0; j < qpg; ++j) {
        const int32_t v = h[size_t(g) * qpg + j];
        KATZ_REQUIRE(v >= 0 && v < m->seg_ptr_h[g + 1] - m->seg_ptr_h[g], KATZ_EINVAL,
                     "query id out of range in graph " + std::to_string(g));
      }
    int32_t* qd = m->ws.get<int32_t>("api.q", total);
    KATZ_CUDA(cudaMemcpyAsync(qd, h.data(), 4 * size_t(total), cudaMemcpyHostToDevice, s));
    const bool dev = is_device_ptr(K_out);
    const size_t es = out_dtype == KATZ_F64 ? 8 : 4;
    void* Kd = dev ? K_out : m->ws.get<uint8_t>("api.K", es * size_t(m->n) * ldk);
    std::vector<int32_t> it;
    std::vector<double> rr;
    const int st =
        katz::multi_query(*m, qd, qpg, *opts, Kd, out_dtype, ldk, stats, it, rr, s, use_lrc);
    if (!dev && (st == KATZ_OK || st == KATZ_ENOCONV)) {
      KATZ_CUDA(cudaMemcpyAsync(K_out, Kd, es * size_t(m->n) * ldk, cudaMemcpyDeviceToHost, s));
      KATZ_CUDA(cudaStreamSynchronize(s));
    }
    if (iters_out) std::memcpy(iters_out, it.data(), 4 * it.size());
    if (rel_res_out) std::memcpy(rel_res_out, rr.data(), 8 * rr.size());
    if (st == KATZ_ENOCONV) g_last_error = "iteration or refinement cap reached";
    if (st == KATZ_ENOTSPD) g_last_error = "CG breakdown: p^T A p <= 0";
    return st;
  });
}

int katz_multi_query(const katz_multi* m, const int32_t* q, int32_t qpg,
                     const katz_query_opts* opts, void* K_out, int32_t out_dtype, int64_t ldk,
                     katz_stats* stats, int32_t* iters_out, double* rel_res_out, void* stream) {
  return multi_query_api(m, q, qpg, opts, K_out, out_dtype, ldk, stats, iters_out, rel_res_out,
                         stream, false);
}

int katz_multi_query_lrc(const katz_multi* m, const int32_t* q, int32_t qpg,
                         const katz_query_opts* opts, void* K_out, int32_t out_dtype, int64_t ldk,
                         katz_stats* stats, int32_t* iters_out, double* rel_res_out,
                         void* stream) {
  return multi_query_api(m, q, qpg, opts, K_out, out_dtype, ldk, stats, iters_out, rel_res_out,
                         stream, true);
}

int katz_autotune(katz_index* idx, int32_t b, int32_t* out, double* ms, void* stream) {
  return guarded([&]() {
    KATZ_REQUIRE(idx && out && ms && b > 0 && b <= 1024, KATZ_EINVAL, "bad autotune arguments");
    const katz::TuneResult r = katz::autotune(*idx, b, static_cast<cudaStream_t>(stream));
    out[0] = r.col_tile;
    out[1] = r.ctas_per_sm;
    out[2] = r.cheb_pipe ? 1 : 0;
    out[3] = r.res_first_pipe ? 1 : 0;
    out[4] = r.res_pipe ? 1 : 0;
    out[5] = r.cheb_cps;
    out[6] = r.res_cps;
    out[7] = r.cheb_depth;
    out[8] = r.cheb_rowpipe ? 1 : 0;
    out[9] = r.cheb_chunk;
    out[10] = r.res_chunk;
    ms[0] = r.ms_best;
    ms[1] = r.ms_default;
    return KATZ_OK;
  });
}

int katz_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, int32_t M, int32_t N,
                   int32_t K, float alpha, float beta, float* C, int64_t ldc, void* stream) {
  return guarded([&]() {
    KATZ_REQUIRE(A && B && C && M > 0 && N > 0 && K > 0, KATZ_EINVAL, "bad GEMM arguments");
    KATZ_REQUIRE(lda >= K && ldb >= K && ldc >= N && lda % 8 == 0 && ldb % 8 == 0, KATZ_EINVAL,
                 "GEMM strides: lda, ldb >= K and multiples of 8; ldc >= N");
    KATZ_REQUIRE(is_device_ptr(A) && is_device_ptr(B) && is_device_ptr(C), KATZ_EINVAL,
                 "GEMM operands must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    katz::DBuf<int> err(1);
    KATZ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    katz::tc_gemm(static_cast<const __nv_bfloat16*>(A), lda, static_cast<const __nv_bfloat16*>(B),
                  ldb, M, N, K, alpha, beta, C, ldc, nullptr, 0, 0, err.p, s);
    int h = 0;
    KATZ_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    KATZ_REQUIRE(h == 0, KATZ_ECUDA, "tcgen05 GEMM pipeline timed out");
    return KATZ_OK;
  });
}

int katz_test_stall_copies(int32_t on) {
  katz::set_test_stall_copies(on != 0);
  return KATZ_OK;
}

int katz_gemm_tf32x3(const float* A, int64_t lda, const float* B, int64_t ldb, int32_t M,
                     int32_t N, int32_t K, float alpha, float beta, float* C, int64_t ldc,
                     void* stream) {
  return guarded([&]() {
    KATZ_REQUIRE(A && B && C && M > 0 && N > 0 && K > 0, KATZ_EINVAL, "bad GEMM arguments");
    KATZ_REQUIRE(lda >= K && ldb >= K && ldc >= N && lda % 4 == 0 && ldb % 4 == 0, KATZ_EINVAL,
                 "GEMM strides: lda, ldb >= K and multiples of 4; ldc >= N");
    KATZ_REQUIRE(is_device_ptr(A) && is_device_ptr(B) && is_device_ptr(C), KATZ_EINVAL,
                 "GEMM operands must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t ldk = (int64_t(K) + 3) / 4 * 4;
    katz::DBuf<float> Ah(size_t(M) * ldk), Al(size_t(M) * ldk), Bh(size_t(N) * ldk),
        Bl(size_t(N) * ldk);
    katz::split_tf32<float>(A, lda, M, K, Ah.p, Al.p, ldk, s);
    katz::split_tf32<float>(B, ldb, N, K, Bh.p, Bl.p, ldk, s);
    katz::DBuf<int> err(1);
    KATZ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    katz::tc_gemm_tf32x3(Ah.p, Al.p, ldk, Bh.p, Bl.p, ldk, M, N, K, alpha, beta, C, ldc, C, ldc,
                         err.p, s);
    int h = 0;
    KATZ_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    KATZ_REQUIRE(h == 0, KATZ_ECUDA, "tcgen05 GEMM pipeline timed out");
    return KATZ_OK;
  });
}

int katz_apply_M(const katz_index* cidx, const void* X, void* Y, int32_t b, int32_t dtype,
                 void* stream) {
  return guarded([&]() {
    KATZ_REQUIRE(cidx && X && Y && b > 0, KATZ_EINVAL, "null argument");
    KATZ_REQUIRE(dtype == KATZ_F32 || dtype == KATZ_F64, KATZ_EINVAL, "dtype");
    KATZ_REQUIRE(is_device_ptr(X) && is_device_ptr(Y), KATZ_EINVAL, "X and Y must be device memory");
    katz_index* idx = const_cast<katz_index*>(cidx);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = idx->n, ld = (b + 3) / 4 * 4;
    // staged through padded buffers so vector loads stay 16-byte aligned
    if (dtype == KATZ_F32) {
      float* xs = idx->ws.get<float>("am.x", size_t(n) * ld);
      float* ys = idx->ws.get<float>("am.y", size_t(n) * ld);
      KATZ_CUDA(cudaMemsetAsync(xs, 0, 4 * size_t(n) * ld, s));
      katz::copy2d<float>(static_cast<const float*>(X), b, xs, ld, n, b, 1.0, s);
      katz::apply_M<float>(*idx, xs, ys, b, ld, s);
      katz::copy2d<float>(ys, ld, static_cast<float*>(Y), b, n, b, 1.0, s);
    } else {
      double* xs = idx->ws.get<double>("am.x", size_t(n) * ld);
      double* ys = idx->ws.get<double>("am.y", size_t(n) * ld);
      KATZ_CUDA(cudaMemsetAsync(xs, 0, 8 * size_t(n) * ld, s));
      katz::copy2d<double>(static_cast<const double*>(X), b, xs, ld, n, b, 1.0, s);
      katz::apply_M<double>(*idx, xs, ys, b, ld, s);
      katz::copy2d<double>(ys, ld, static_cast<double*>(Y), b, n, b, 1.0, s);
    }
    KATZ_CUDA(cudaStreamSynchronize(s));
    return KATZ_OK;
  });
}

}  // extern "C"
