// The query index (Algorithm 1 output) and the solver entry points.
#pragma once

#include <map>
#include <memory>
#include <string>

#include "ff_residual.h"
#include "gather_pipe.h"
#include "kernels.h"
#include "mlp.h"

namespace katz {

// Dense inverses of one size class of M11 diagonal blocks.
struct BlockClass {
  int S = 0;
  int64_t count = 0;
  DBuf<int64_t> start;
  DBuf<int32_t> size;
  DBuf<float> inv32;
  DBuf<double> inv64;
};

// A CSR with the list of its heavy rows, its per-CTA row split for the
// pipelined gather kernels, and the SpMM launch shapes the autotuner picked
// for it (per right-hand-side width b).
struct GraphPart {
  DevCsr csr;
  DBuf<int32_t> heavy;
  int64_t n_heavy = 0;
  // heavy rows cut into segments of kHeavySeg entries for the residual
  // kernels: segments [hseg_ptr[h], hseg_ptr[h+1]) belong to heavy[h],
  // hseg_row[g] = h
  DBuf<int32_t> hseg_ptr, hseg_row;
  int64_t n_hseg = 0;
  PipeSplit ps;
  std::map<int, SpmmCfg> tuned;
  Csr view() const { return csr.view(); }
  const SpmmCfg* cfg(int b) const {
    auto it = tuned.find(b);
    return it == tuned.end() ? nullptr : &it->second;
  }
};

// The heavy rows of g split for the residual kernels, with their scratch
// for width ld taken from ws (null when g has no heavy rows).
inline const HeavyRows* heavy_rows(const GraphPart& g, int64_t ld, Workspace& ws,
                                   HeavyRows& hv) {
  if (g.n_hseg == 0) return nullptr;
  hv.rows = g.heavy.p;
  hv.seg_ptr = g.hseg_ptr.p;
  hv.seg_row = g.hseg_row.p;
  hv.n = g.n_heavy;
  hv.nseg = g.n_hseg;
  hv.scratch = ws.get<float>("ffr.heavy", size_t(2) * g.n_hseg * ld);
  return &hv;
}

struct Partition {
  std::vector<int64_t> perm;       // perm[new] = old
  std::vector<int64_t> block_ptr;  // blocks of M11 in index order
  int64_t n1 = 0, n2 = 0;
};

}  // namespace katz

// Every field except `ws`, `gather_pref` and `cheb_pref` is stored by save_index
// (index_io.cu): a field added here is added to its list too.
// Block-diagonal Schur objects of an index over many disjoint graphs: the
// separator rows of graph g are [gsep[g], gsep[g+1]) (graph-major, n2_g of
// them); S_g, M22_g^{-1} (n2_g x n2_g, row-major) are packed at moff[g]
// (the sum of the earlier n2_h^2) and W^_g = W_g D_g^{1/2} (n2_g x r_g,
// row-major) at woff[g].  Products with them run one CTA per graph.
struct SegBlocks {
  int32_t G = 0;
  int64_t nmat = 0, nw = 0;
  std::vector<int64_t> gsep_h, moff_h, woff_h;
  std::vector<int32_t> rk_h;
  katz::DBuf<int64_t> gsep, moff, woff;
  katz::DBuf<int32_t> rk, sg;  // rank of each graph; graph of each separator row
  katz::DBuf<float> S32, Minv32, W32;
  katz::DBuf<double> S64, Minv64, W64;
};
// Largest separator of one graph in a block-diagonal (many-graph) index.
constexpr int64_t kSegBlockMax = 256;

// Largest separator of a single-graph LRC index: M22 and M22^{-1} are kept
// dense (n2 x n2 FP64 and FP32) even when S is applied implicitly.
constexpr int64_t kDenseM22Max = 49152;

struct katz_index {
  int64_t n = 0, nnz = 0;
  // lambda: largest Lanczos Ritz value of W (a lower bound on lambda_max);
  // lambda_up: rigorous upper bound, used for the SPD check and the
  // error-bound stopping rule
  double beta = 0, lambda = 0, lambda_up = 0;
  std::vector<int32_t> deg_h;  // node degrees (host), bound the RHS fix-up grid
  int64_t maxdeg = 0;
  bool unit_weights = false;  // every stored weight is exactly 1 (fixed-point residual)
  int vdt = KATZ_UNIT;
  katz::GraphPart W;  // node order

  // LRC-Katz index (Algorithm 1)
  bool lrc = false;
  int rank = 0, block_max = 0, split = 1;
  int64_t n1 = 0, n2 = 0, n1s = 0;  // rows [0,n1s) in dense blocks, [n1s,n1) in large blocks
  int n_large = 0;
  // spectral bounds of the large-block W11 for the Chebyshev solve:
  // spectrum(W11_large) in [lam11_min, lam11] (lam11 = 0: use CG), so
  // spectrum(M11_large) in [1 - beta*lam11, 1 - beta*lam11_min]
  double lam11 = 0, lam11_min = 0;
  // kernel preference of the query being run (KATZ_GATHER_*), set per query
  int gather_pref = KATZ_GATHER_AUTO;
  int cheb_pref = KATZ_CHEB_AUTO;  // per query, like gather_pref
  // LRC corrections (refinement passes after the first) take Y1 = M11^{-1}R1
  // from one Chebyshev step (it only feeds their Schur right-hand side)
  // until a correction made that way leaves a column above its threshold
  bool loose_y1 = true;
  katz::Partition part;
  katz::DBuf<int32_t> perm, iperm;
  katz::GraphPart Wp;    // W in index order (full), for FP64 residuals
  katz::GraphPart W12;   // n1 x n2 block of W (M12 = -beta W12)
  katz::GraphPart W21;   // n2 x n1 (= W12^T)
  katz::GraphPart W11L;  // intra-block edges of the large blocks, local rows/cols
  std::vector<katz::BlockClass> classes;
  int64_t ld2 = 0;  // leading dimension of the dense n2 x n2 objects
  katz::DBuf<float> S32, M22inv32, Wr32;  // Wr scaled by sqrt(sigma/(1-sigma)) per column
  katz::DBuf<double> S64, M22inv64, Wr64;
  // BF16 copies of W^ for the tcgen05 rank-r products: Wb (n2 x ldr) and
  // WbT (r x ldn2), row strides multiples of 8 elements
  katz::DBuf<__nv_bfloat16> Wb, WbT;
  int64_t ldr = 0, ldn2 = 0;
  // unscaled Lanczos basis W_r (n2 x ldr4, FP32, W_r^T M22 W_r = I), W22
  // (the separator block of W), and the learned warm start
  katz::DBuf<float> Wr32u;
  int64_t ldr4 = 0;
  katz::GraphPart W22;
  // beta * M11^{-1} W12 (n1 x n2, row stride ldH) as TF32 high/low parts for
  // the tensor-core back-substitution K1 = Y1 + beta M11^{-1} W12 K2 (Eq. 6)
  katz::DBuf<float> Hh, Hl;
  int64_t ldH = 0;
  bool has_h = false;
  // Z = beta M11^{-1} W12 (n1 x n2 FP32, row stride ldZ): the first Schur
  // right-hand side of a query, F = B2 - M12^T M11^{-1} B1 = B2 + Z^T B1
  // (Eq. 7), from the deg(q) rows of Z that B1 = beta W e_q touches
  katz::DBuf<float> Zc;
  int64_t ldZ = 0;
  bool has_z = false;
  // S and M22^{-1} (n2 x ld2) as TF32 high/low parts for the tensor-core
  // Schur products of the FP32 solve (large separators only)
  katz::DBuf<float> Sh, Sl, Mh, Ml;
  bool dense_tc = false;
  // separators above n2_max: S is never formed; PCG applies
  // S P = M22 P - beta^2 W21 M11^{-1} (W12 P) (Lemma 1, Eqs. 4-7)
  bool s_implicit = false;
  // many graphs: S, M22^{-1} and W^ kept block by block (seg_blocked), the
  // Schur PCG with per-graph scalars; seg_iters[g * b + c] its iterations
  bool seg_blocked = false;
  SegBlocks sb;
  std::vector<int32_t> seg_iters;
  int64_t seg_replays = 0;  // CUDA-graph replays of the many-graph Schur PCG
  katz::Mlp mlp;
  katz::DBuf<float> feat;  // n x 32 node features
  katz::DBuf<float> Hr;    // beta M11^{-1} W12 W_r (n1 x ldr4), for the CG warm start
  std::vector<double> sigma;
  int lanczos_steps = 0;
  // an index of disjoint graphs: each graph's rank (its sigma and basis
  // columns follow one another, graph-major); empty for one graph
  std::vector<int> seg_rank;

  katz::Workspace ws;
};

// g independent graphs stored as one block-diagonal CSR (multi-graph batch).
struct katz_multi {
  int32_t g = 0;
  // per-graph LRC index over the union with each graph's damping folded
  // into its weights (beta = 1): built by katz_index_build_many
  std::unique_ptr<katz_index> lrc;
  int64_t n = 0, nnz = 0;
  int vdt = KATZ_F32;
  std::vector<int64_t> seg_ptr_h;
  std::vector<double> beta_h, lambda_h;  // lambda_h: rigorous upper bounds on lambda_max
  std::vector<int32_t> deg_h;
  katz::GraphPart W;
  katz::DBuf<int64_t> seg_ptr;
  katz::DBuf<int32_t> seg;
  katz::DBuf<float> bseg_hi, bseg_lo;
  katz::DBuf<double> bseg64;
  katz::Workspace ws;
  cudaStream_t cap_stream = nullptr;
  ~katz_multi() {
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

namespace katz {

// Host partitioner (Section 3.2, Steps 2-3, with the BFS level-set reading);
// hub_list, when given, is the hub set instead of the n_hubs largest degrees.
Partition partition_graph(const HostCsr& W, int64_t n_hubs, int64_t block_max, bool split,
                          const std::vector<int64_t>* hub_list = nullptr);

// Index of g disjoint graphs stored as one block-diagonal graph: which graph
// each node belongs to (node ids graph-major), the separator (each graph's
// own hubs) and each graph's rank of the low-rank correction.  The Schur
// complement and its correction are then block diagonal: S is formed by
// column-packed solves (separator node l of every graph shares column l) and
// Lanczos runs on every graph at once with per-graph scalars.
struct SegSpec {
  int32_t G = 0;
  std::vector<int32_t> node_graph;
  std::vector<int64_t> hubs;
  std::vector<int> ranks;
};

// Block-diagonal Schur pieces of a many-graph index (seg_blocks.cu).
// Scatter the packed T columns of column block [l0, l0 + cw) into the
// per-graph T blocks (Tb, packed like S).
void seg_scatter_T(const SegBlocks& sb, const double* E, int64_t ldc, int64_t n2, int l0, int cw,
                   double* Tb, cudaStream_t s);
// S_g = M22_g - T_g and M22_g^{-1} (in place, Gauss-Jordan on the SPD block)
// for every graph; W22 is the union's separator block (local columns).
// Returns false if a block is not positive definite.
bool seg_build_blocks(SegBlocks& sb, const Csr& W22, double beta, const double* Tb,
                      double* M22b, cudaStream_t s);
// y_g = A_g x_g for FP64 block-diagonal A (packed at moff), strided x / y.
void seg_block_mv64(const SegBlocks& sb, const double* A, const double* x, int64_t incx, double* y,
                    int64_t incy, cudaStream_t s);
// Schur PCG with per-graph scalars on S K2 = F (n2 x b, ld): every (graph,
// column) pair has its own CG coefficients and stops when
// ||F - S K2||_2 <= tol ||F||_2 on its rows.  iters_gc (G * b) receives the
// iterations of each pair.
int seg_pcg(katz_index& idx, const float* F, float* K2, int b, int64_t ld, double tol,
            int max_iter, std::vector<int32_t>& iters_gc, cudaStream_t s);

// Largest Ritz value of W after `steps` FP64 Lanczos steps on the GPU
// (start: all-ones if seed == 0, else SplitMix64(seed)); *lmin (optional)
// gets the smallest, *lup (optional) a rigorous upper bound on lambda_max
// for W >= 0 (Collatz-Wielandt bound from the top Ritz vector).
double lambda_max_gpu(const GraphPart& W, int64_t n, int steps, Workspace& ws, cudaStream_t s,
                      uint64_t seed = 0, double* lmin = nullptr, double* lup = nullptr);

void build_index(katz_index& idx, const HostCsr& W, double beta, const katz_build_opts& o,
                 cudaStream_t s, const SegSpec* seg = nullptr);

// Versioned binary file of every stored field of an index (device buffers
// staged through host memory); load validates magic, version, field tags,
// sizes and a checksum and throws KATZ_EINVAL on any mismatch.
void save_index(const katz_index& idx, const char* path);
std::unique_ptr<katz_index> load_index(const char* path);

struct QueryOut {
  void* K = nullptr;  // device
  int dtype = KATZ_F32;
  int64_t ldk = 0;
};

// Runs a batch of queries (q on device) by LRC (use_lrc) or plain CG and
// writes K (device).  Fills per-column iterations / residuals (host).
int run_queries(katz_index& idx, bool use_lrc, const int32_t* q_dev, const int32_t* q_host, int b,
                const katz_query_opts& o, const QueryOut& out, katz_stats* st,
                std::vector<int32_t>& iters, std::vector<double>& relres, cudaStream_t s);

template <class VT>
void apply_M(const katz_index& idx, const VT* X, VT* Y, int b, int64_t ld, cudaStream_t s);

// One FP32 LRC solve D ~ M^{-1} R (Lemma 1, Eqs. 6-7, PCG on S with the
// preconditioner of Eq. 14) of ld-padded blocks in INDEX order, to relative
// tolerance tol_rel; per-column iterations in *iters.
int lrc_solve_f32(katz_index& idx, const float* R, float* D, int b, int64_t ld, double tol_rel,
                  int max_iter, std::vector<int32_t>* iters, cudaStream_t s);

void multi_build(katz_multi& m, const std::vector<HostCsr>& Ws, const double* betas, int vdt,
                 cudaStream_t s);
// multi_build plus the per-graph LRC index (hubs per graph in proportion
// to its size from a total of o.n_hubs; ranks from o.rank / 4 on the
// smallest graph to o.rank on the largest, log-scaled, capped by the
// graph's separator)
void multi_build_lrc(katz_multi& m, const std::vector<HostCsr>& Ws, const double* betas,
                     const katz_build_opts& o, cudaStream_t s);
int multi_query(katz_multi& m, const int32_t* q_dev, int qpg, const katz_query_opts& o, void* Kout,
                int out_dt, int64_t ldk, katz_stats* stats, std::vector<int32_t>& iters,
                std::vector<double>& relres, cudaStream_t s, bool use_lrc = false);

// Sparse-Katz (Algorithm 3) for b queries: ids/rho (device, b x s) get the
// re-ranked Top-s candidates and their Pearson correlations, land (device,
// b x T, may be null) the landmarks.
int sparse_katz(katz_index& idx, const int32_t* q_dev, const int32_t* q_host, int b, int s_top,
                int T, const katz_query_opts& o, int32_t* ids, double* rho, int32_t* land,
                katz_stats* st, cudaStream_t s);

double warmstart_train(katz_index& idx, const int32_t* q_host, int n_train, int hidden, int epochs,
                       int batch, float lr, float wd, uint64_t seed, double* init_loss, int* steps,
                       cudaStream_t s);
void warm_start_guess(katz_index& idx, const int32_t* q, int b, float* K20, int64_t ld,
                      cudaStream_t s);
// Initial guess of CG on M from the network (node order, n x b, ld).
void warm_cg_guess(katz_index& idx, const int32_t* q, int b, float* X, int64_t ld,
                   cudaStream_t s);

// Chebyshev steps of the large M11 blocks for relative tolerance tol, and
// whether the tensor-core back-substitution is cheaper than the second M11
// solve at width ld and that tolerance (cost model).
int cheb_steps(const katz_index& idx, double tol);
bool coupling_gemm_pays(const katz_index& idx, int64_t ld, double tol);

struct TuneResult {
  int col_tile = 0, ctas_per_sm = 0, rhs_width = 0;
  bool cheb_pipe = false;  // the pipelined Chebyshev step was faster on the large block
  bool res_first_pipe = false, res_pipe = false;  // ... residual passes (LRC operator)
  int cheb_depth = 0;
  bool cheb_rowpipe = false;  // the row-pipelined Chebyshev kernel was faster
  int cheb_chunk = 0;         // rows per CTA of the Chebyshev step (0: strided)
  int res_chunk = 0;          // rows per CTA of the residual passes (0: strided)
  int cheb_cps = 0, res_cps = 0;  // CTAs per SM of the fused kernels
  double ms_best = 0, ms_default = 0;
};
// Times candidate SpMM launch shapes on every operator of the index for
// width b (FP32 vectors) and records the fastest; returns the result for W.
TuneResult autotune(katz_index& idx, int b, cudaStream_t s);

}  // namespace katz
