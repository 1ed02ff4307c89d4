// SpMM launch-shape autotuner.  For a right-hand-side width b it times the
// candidate shapes (columns per warp-row tile x CTAs per SM) of the
// multi-RHS CSR product on each operator of an index with CUDA events, keeps
// the fastest per operator, and caches the choice per (rows, nnz, b, value
// type) for the process so indexes of the same graph reuse it.  Where the
// pipelined (TMA bulk-copy) kernels apply it also times them against the
// register kernels -- the fused Chebyshev step on the large-block operator,
// the refinement residual on the full operators -- and keeps the faster.
#include <mutex>
#include <tuple>

#include "ff_residual.h"
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

enum class Fused { none, cheb, residual };

// Mean time of `reps` launches of the fused product (after one warm-up).
template <class F>
double time_launches(F&& launch, cudaStream_t s, int reps) {
  cudaEvent_t e0, e1;
  KATZ_CUDA(cudaEventCreate(&e0));
  KATZ_CUDA(cudaEventCreate(&e1));
  launch();
  KATZ_CUDA(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) launch();
  KATZ_CUDA(cudaEventRecord(e1, s));
  KATZ_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  KATZ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

// Is the pipelined kernel faster than the register one for the fused
// product?  Residual: *first for the first pass (the later passes have no
// pipelined kernel).
bool pipe_faster(const GraphPart& g, Fused kind, bool unit, const SpmmCfg& c, float* X, float* Y,
                 float* Z, int b, int64_t ld, Workspace& ws, cudaStream_t s, int reps,
                 bool* first) {
  int* err = ws.get<int>("pipe.err", 1);
  KATZ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  bool faster;
  if (kind == Fused::cheb) {
    const double t_reg =
        time_launches([&] { cheb_step(g.view(), 0.01, 0.1, 1.0, X, X, X, Y, ld, b, s, &c); }, s, reps);
    const double t_pipe = time_launches(
        [&] { pipe_cheb_step(g.view(), g.ps, unit, 0.01, 0.1, 1.0, X, X, X, Y, ld, err, s); }, s, reps);
    faster = t_pipe < t_reg;
  } else {
    HeavyRows hv;
    const HeavyRows* hvp = heavy_rows(g, ld, ws, hv);
    const double t_reg = time_launches(
        [&] { ffr_update(g.view(), 0.01, X, Y, Z, true, ld, b, nullptr, &c, s, hvp); }, s, reps);
    const double t_pipe = time_launches(
        [&] { pipe_residual(g.view(), g.ps, unit, 0.01, X, Y, Z, ld, b, nullptr, err, s); }, s,
        reps);
    *first = t_pipe < t_reg;
    faster = false;  // later passes: register kernel
  }
  int herr = 0;
  KATZ_CUDA(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
  KATZ_REQUIRE(herr == 0, KATZ_ECUDA, "pipelined gather kernel: a wait timed out");
  return faster;
}

// Best shape for one operator (square operators only: X and Y share rows);
// kind: the fused product to choose the register or pipelined kernel for.
SpmmCfg tune_part(GraphPart& g, int b, Workspace& ws, cudaStream_t s, double* best_ms,
                  double* def_ms, Fused kind = Fused::none, bool unit = false) {
  const auto key = std::make_tuple(g.csr.nrows, g.csr.nnz, b, g.csr.vdt * 4 + int(kind));
  {
    std::lock_guard<std::mutex> l(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      g.tuned[b] = it->second;
      return it->second;
    }
  }
  // the queries' leading dimension (multiple of 8 for batches above 128)
  const int64_t ld = b > 128 ? (b + 7) / 8 * 8 : (b + 3) / 4 * 4;
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
    for (int cps : {2, 4, 8, 16, 32, 64}) {
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
  if (kind != Fused::none && g.csr.nrows > 0 && (kind == Fused::cheb || g.csr.vdt != KATZ_F64)) {
    // the fused kernel's own grid: its warps take one column tile of the
    // rows at a time, and more resident-then-queued CTAs per SM than the
    // plain product keeps the active rows' gathers in L2
    float* Z = ws.get<float>("tune.Z", size_t(rows) * ld);
    KATZ_CUDA(cudaMemsetAsync(Z, 0, sizeof(float) * rows * ld, s));
    HeavyRows hv;
    const HeavyRows* hvp = heavy_rows(g, ld, ws, hv);
    double* rr = ws.get<double>("tune.rr", size_t(ld));
    // residual: the first pass (float-float sums) and a later one (R -= M D
    // with the column norms) share the launch shape; both are timed
    auto fused_ms = [&](const SpmmCfg& c) {
      if (kind == Fused::cheb)
        return time_launches(
            [&] { cheb_step(g.view(), 0.01, 0.1, 1.0, X, X, X, Y, ld, b, s, &c); }, s, reps);
      return time_launches(
                 [&] { ffr_update(g.view(), 0.01, X, Y, Z, true, ld, b, nullptr, &c, s, hvp); }, s,
                 reps) +
             time_launches(
                 [&] { ffr_update(g.view(), 0.01, X, Y, Z, false, ld, b, rr, &c, s, hvp); }, s,
                 reps);
    };
    double bestf = 0;
    for (int cps : {8, 16, 32, 64, 128}) {
      SpmmCfg c = best;
      c.fused_cps = cps;
      const double ms = fused_ms(c);
      if (best.fused_cps == 0 || ms < bestf) {
        bestf = ms;
        best.fused_cps = cps;
      }
    }
    if (kind == Fused::residual) {
      // contiguous row runs per CTA
      for (int rc : {32, 64, 128, 256}) {
        SpmmCfg c = best;
        c.row_chunk = rc;
        const double ms = fused_ms(c);
        if (ms < bestf) {
          bestf = ms;
          best.row_chunk = rc;
        }
      }
    }
    if (kind == Fused::cheb) {
      // gathered rows loaded together per lane, and the row-pipelined kernel
      for (int gd : {4, 8}) {
        SpmmCfg c = best;
        c.gather_depth = gd;
        const double ms = time_launches(
            [&] { cheb_step(g.view(), 0.01, 0.1, 1.0, X, X, X, Y, ld, b, s, &c); }, s, reps);
        if (ms < bestf) {
          bestf = ms;
          best.gather_depth = gd;
        }
      }
      // contiguous row chunks per CTA (the resident CTAs' rows neighbours)
      for (int rc : {32, 64, 128, 256}) {
        SpmmCfg c = best;
        c.row_chunk = rc;
        const double ms = time_launches(
            [&] { cheb_step(g.view(), 0.01, 0.1, 1.0, X, X, X, Y, ld, b, s, &c); }, s, reps);
        if (ms < bestf) {
          bestf = ms;
          best.row_chunk = rc;
        }
      }
      {
        SpmmCfg c = best;
        c.row_pipeline = true;
        const double ms = time_launches(
            [&] { cheb_step(g.view(), 0.01, 0.1, 1.0, X, X, X, Y, ld, b, s, &c); }, s, reps);
        if (ms < bestf) {
          bestf = ms;
          best.row_pipeline = true;
        }
      }
    }
    ws.release("tune.Z");
    ws.release("tune.rr");
  }
  if (kind != Fused::none && pipe_eligible(g.ps, ld) && (unit || g.csr.vdt != KATZ_F64)) {
    float* Z = ws.get<float>("tune.Z", size_t(rows) * ld);
    KATZ_CUDA(cudaMemsetAsync(Z, 0, sizeof(float) * rows * ld, s));
    bool first = false;
    best.pipe = pipe_faster(g, kind, unit, best, X, Y, Z, b, ld, ws, s, reps, &first);
    best.pipe_first = first;
    ws.release("tune.Z");
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
  SpmmCfg c = tune_part(idx.W, b, idx.ws, s, &best, &def, Fused::residual, idx.unit_weights);
  r.col_tile = c.col_tile;
  r.ctas_per_sm = c.ctas_per_sm;
  r.ms_best = best;
  r.ms_default = def;
  if (idx.lrc) {
    double b2, d2;
    const SpmmCfg cp = tune_part(idx.Wp, b, idx.ws, s, &b2, &d2, Fused::residual, idx.unit_weights);
    r.res_first_pipe = cp.pipe_first;
    r.res_pipe = cp.pipe;
    r.res_cps = cp.fused_cps;
    r.res_chunk = cp.row_chunk;
    if (idx.W11L.csr.nrows > 0) {
      const SpmmCfg cc = tune_part(idx.W11L, b, idx.ws, s, &b2, &d2, Fused::cheb, idx.unit_weights);
      r.cheb_pipe = cc.pipe;
      r.cheb_cps = cc.fused_cps;
      r.cheb_depth = cc.gather_depth;
      r.cheb_rowpipe = cc.row_pipeline;
      r.cheb_chunk = cc.row_chunk;
    }
    // the couplings (W12 rows stream the M11 block, W21 rows are hubs)
    if (idx.n1 > 0 && idx.n2 > 0) {
      tune_part(idx.W12, b, idx.ws, s, &b2, &d2);
      tune_part(idx.W21, b, idx.ws, s, &b2, &d2);
    }
  } else {
    r.res_cps = c.fused_cps;
    r.res_chunk = c.row_chunk;
  }
  // release the tuning scratch
  idx.ws.release("tune.X");
  idx.ws.release("tune.Y");
  return r;
}

}  // namespace katz
