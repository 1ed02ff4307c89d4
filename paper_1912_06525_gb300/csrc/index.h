// The query index (Algorithm 1 output) and the solver entry points.
#pragma once

#include <map>
#include <memory>
#include <string>

#include "kernels.h"

namespace katz {

// Named, grow-only device scratch owned by an index.
class Workspace {
 public:
  template <class T>
  T* get(const std::string& name, size_t count) {
    auto& b = bufs_[name];
    b.ensure(count * sizeof(T));
    return reinterpret_cast<T*>(b.p);
  }
  void clear() { bufs_.clear(); }
  void release(const std::string& name) { bufs_.erase(name); }
  size_t bytes() const {
    size_t t = 0;
    for (auto& kv : bufs_) t += kv.second.bytes();
    return t;
  }

 private:
  std::map<std::string, DBuf<uint8_t>> bufs_;
};

// Dense inverses of one size class of M11 diagonal blocks.
struct BlockClass {
  int S = 0;
  int64_t count = 0;
  DBuf<int64_t> start;
  DBuf<int32_t> size;
  DBuf<float> inv32;
  DBuf<double> inv64;
};

// A CSR with the list of its heavy rows and the SpMM launch shapes the
// autotuner picked for it (per right-hand-side width b).
struct GraphPart {
  DevCsr csr;
  DBuf<int32_t> heavy;
  int64_t n_heavy = 0;
  std::map<int, SpmmCfg> tuned;
  Csr view() const { return csr.view(); }
  const SpmmCfg* cfg(int b) const {
    auto it = tuned.find(b);
    return it == tuned.end() ? nullptr : &it->second;
  }
};

struct Partition {
  std::vector<int64_t> perm;       // perm[new] = old
  std::vector<int64_t> block_ptr;  // blocks of M11 in index order
  int64_t n1 = 0, n2 = 0;
};

}  // namespace katz

struct katz_index {
  int64_t n = 0, nnz = 0;
  double beta = 0, lambda = 0;
  std::vector<int32_t> deg_h;  // node degrees (host), bound the RHS fix-up grid
  int vdt = KATZ_UNIT;
  katz::GraphPart W;  // node order

  // LRC-Katz index (Algorithm 1)
  bool lrc = false;
  int rank = 0, block_max = 0, split = 1;
  int64_t n1 = 0, n2 = 0, n1s = 0;  // rows [0,n1s) in dense blocks, [n1s,n1) in large blocks
  int n_large = 0;
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
  std::vector<double> sigma;
  int lanczos_steps = 0;

  katz::Workspace ws;
};

namespace katz {

// Host partitioner (Section 3.2, Steps 2-3, with the BFS level-set reading).
Partition partition_graph(const HostCsr& W, int64_t n_hubs, int64_t block_max, bool split);

// Largest eigenvalue of W by FP64 Lanczos on the GPU.
double lambda_max_gpu(const GraphPart& W, int64_t n, int steps, Workspace& ws, cudaStream_t s);

void build_index(katz_index& idx, const HostCsr& W, double beta, const katz_build_opts& o,
                 cudaStream_t s);

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

struct TuneResult {
  int col_tile = 0, ctas_per_sm = 0, rhs_width = 0;
  double ms_best = 0, ms_default = 0;
};
// Times candidate SpMM launch shapes on every operator of the index for
// width b (FP32 vectors) and records the fastest; returns the result for W.
TuneResult autotune(katz_index& idx, int b, cudaStream_t s);

}  // namespace katz
