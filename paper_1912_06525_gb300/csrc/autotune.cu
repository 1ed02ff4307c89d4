// SpMM launch-shape autotuner.  For a right-hand-side width b it times the
// candidate shapes (columns per warp-row tile x CTAs per SM) of the
// multi-RHS CSR product on each operator of an index with CUDA events, keeps
// the fastest per operator, and caches the choice per (rows, nnz, b, value
// type) for the process so indexes of the same graph reuse it.
#include <mutex>
#include <tuple>

#include "index.h"

namespace katz {

namespace {
std::mutex g_mu;
std::map<std::tuple<int64_t, int64_t, int, int>, SpmmCfg> g_cache;

double time_cfg(const GraphPart& g, const SpmmCfg& c, const float* X, float* Y, int b, int64_t ld,
                cudaStream_t s, int reps) {
  cudaEvent_t e0, e1;
  KATZ_CUDA(cudaEventCreate(&e0));
  KATZ_CUDA(cudaEventCreate(&e1));
  spmm<float>(g.view(), g.heavy.p, g.n_heavy, -0.5, X, ld, 1.0, X, ld, Y, ld, b, nullptr, 0,
              nullptr, s, &c);  // warm-up
  KATZ_CUDA(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r)
    spmm<float>(g.view(), g.heavy.p, g.n_heavy, -0.5, X, ld, 1.0, X, ld, Y, ld, b, nullptr, 0,
                nullptr, s, &c);
  KATZ_CUDA(cudaEventRecord(e1, s));
  KATZ_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  KATZ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

// Best shape for one operator (square operators only: X and Y share rows).
SpmmCfg tune_part(GraphPart& g, int b, Workspace& ws, cudaStream_t s, double* best_ms,
                  double* def_ms) {
  const auto key = std::make_tuple(g.csr.nrows, g.csr.nnz, b, g.csr.vdt);
  {
    std::lock_guard<std::mutex> l(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      g.tuned[b] = it->second;
      return it->second;
    }
  }
  const int64_t ld = (b + 3) / 4 * 4;
  const int64_t rows = std::max(g.csr.nrows, g.csr.ncols);
  float* X = ws.get<float>("tune.X", size_t(rows) * ld);
  float* Y = ws.get<float>("tune.Y", size_t(rows) * ld);
  KATZ_CUDA(cudaMemsetAsync(X, 0, sizeof(float) * rows * ld, s));
  const int reps = g.csr.nnz > 20000000 ? 2 : 5;
  SpmmCfg best{};
  *def_ms = time_cfg(g, best, X, Y, b, ld, s, reps);
  *best_ms = *def_ms;
  for (int tile : {128, 256, 512, 1024}) {
    if (tile > 4 * ld && tile != 128) continue;
    for (int cps : {2, 4, 8, 16}) {
      SpmmCfg c;
      c.col_tile = tile;
      c.ctas_per_sm = cps;
      const double ms = time_cfg(g, c, X, Y, b, ld, s, reps);
      if (ms < *best_ms) {
        *best_ms = ms;
        best = c;
      }
    }
  }
  g.tuned[b] = best;
  std::lock_guard<std::mutex> l(g_mu);
  g_cache[key] = best;
  return best;
}
}  // namespace

TuneResult autotune(katz_index& idx, int b, cudaStream_t s) {
  TuneResult r;
  double best = 0, def = 0;
  SpmmCfg c = tune_part(idx.W, b, idx.ws, s, &best, &def);
  r.col_tile = c.col_tile;
  r.ctas_per_sm = c.ctas_per_sm;
  r.ms_best = best;
  r.ms_default = def;
  if (idx.lrc) {
    double b2, d2;
    tune_part(idx.Wp, b, idx.ws, s, &b2, &d2);
    if (idx.W11L.csr.nrows > 0) tune_part(idx.W11L, b, idx.ws, s, &b2, &d2);
  }
  // release the tuning scratch
  idx.ws.release("tune.X");
  idx.ws.release("tune.Y");
  return r;
}

}  // namespace katz
