// Index construction (Algorithm 1, "Preprocess") and lambda_max.
//
// Host side (native C++): CSR validation, the vertex-separator partition and
// reordering (Section 3.2, Steps 2-3), and assembly of the permuted CSR
// blocks.  Device side: M11 block inverses (Step 4), the Schur complement S
// (Lemma 1), M22^{-1}, and the Lanczos process on R (Eqs. 8-11).
#include <algorithm>
#include <cmath>
#include <deque>
#include <numeric>
#include <thread>

#include "index.h"
#include "tc_gemm.h"
#include "kernels_dense.h"

namespace katz {

template <class VT>
int cg_solve(const GraphPart& A, double beta, const VT* B, int64_t ld, int64_t len, int b, VT* X,
             const double* thr2, int max_iter, Workspace& ws, const std::string& tag,
             std::vector<int32_t>* iters, cudaStream_t s);
template <class VT>
int m11_solve(katz_index& idx, const VT* X, VT* Y, int b, int64_t ld, double tolL, int max_iter,
              std::vector<int32_t>* iters, cudaStream_t s);

// ------------------------------------------------------------ uploads
void upload_csr(const HostCsr& h, int vdt, DevCsr& d, cudaStream_t s) {
  d.nrows = h.nrows;
  d.ncols = h.ncols;
  d.nnz = h.nnz();
  d.vdt = vdt;
  d.rowptr.alloc(h.nrows + 1);
  KATZ_CUDA(cudaMemcpyAsync(d.rowptr.p, h.rowptr.data(), sizeof(int64_t) * (h.nrows + 1),
                            cudaMemcpyHostToDevice, s));
  d.col.alloc(std::max<int64_t>(d.nnz, 1));
  if (d.nnz)
    KATZ_CUDA(cudaMemcpyAsync(d.col.p, h.col.data(), sizeof(int32_t) * d.nnz,
                              cudaMemcpyHostToDevice, s));
  const size_t es = vdt_size(vdt);
  if (es && d.nnz) {
    std::vector<uint8_t> raw(es * d.nnz);
    for (int64_t k = 0; k < d.nnz; ++k) {
      const double w = h.val.empty() ? 1.0 : h.val[k];
      if (vdt == KATZ_F64) reinterpret_cast<double*>(raw.data())[k] = w;
      else if (vdt == KATZ_F32) reinterpret_cast<float*>(raw.data())[k] = float(w);
      else reinterpret_cast<__nv_bfloat16*>(raw.data())[k] = __double2bfloat16(w);
    }
    d.val.alloc(raw.size());
    KATZ_CUDA(cudaMemcpyAsync(d.val.p, raw.data(), raw.size(), cudaMemcpyHostToDevice, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
  } else {
    KATZ_CUDA(cudaStreamSynchronize(s));
  }
}

static void upload_part(const HostCsr& h, int vdt, GraphPart& g, cudaStream_t s) {
  upload_csr(h, vdt, g.csr, s);
  if (h.nrows > 0) pipe_split_build(h.rowptr, h.nrows, g.ps, s);
  std::vector<int32_t> heavy;
  for (int64_t i = 0; i < h.nrows; ++i)
    if (h.rowptr[i + 1] - h.rowptr[i] > kHeavyRowNnz) heavy.push_back((int32_t)i);
  g.n_heavy = (int64_t)heavy.size();
  g.heavy.alloc(std::max<size_t>(heavy.size(), 1));
  std::vector<int32_t> seg_ptr(heavy.size() + 1, 0), seg_row;
  for (size_t hh = 0; hh < heavy.size(); ++hh) {
    const int64_t len = h.rowptr[heavy[hh] + 1] - h.rowptr[heavy[hh]];
    const int64_t nseg = ceil_div(len, kHeavySeg);
    for (int64_t k = 0; k < nseg; ++k) seg_row.push_back((int32_t)hh);
    seg_ptr[hh + 1] = (int32_t)seg_row.size();
  }
  g.n_hseg = (int64_t)seg_row.size();
  g.hseg_ptr.alloc(seg_ptr.size());
  g.hseg_row.alloc(std::max<size_t>(seg_row.size(), 1));
  KATZ_CUDA(cudaMemcpyAsync(g.hseg_ptr.p, seg_ptr.data(), sizeof(int32_t) * seg_ptr.size(),
                            cudaMemcpyHostToDevice, s));
  if (!heavy.empty()) {
    KATZ_CUDA(cudaMemcpyAsync(g.heavy.p, heavy.data(), sizeof(int32_t) * heavy.size(),
                              cudaMemcpyHostToDevice, s));
    KATZ_CUDA(cudaMemcpyAsync(g.hseg_row.p, seg_row.data(), sizeof(int32_t) * seg_row.size(),
                              cudaMemcpyHostToDevice, s));
  }
  KATZ_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------ partition
// Node-for-node the reading stated with the oracle's partition():
//  1. the n_hubs nodes of largest degree (ties: smaller id) -> separator;
//  2. components of the rest are blocks; when splitting, a block larger than
//     block_max is cut at the median BFS level (BFS from its smallest id;
//     the last node reached roots a second BFS; first level k with
//     2*cum_k >= size), recursively;
//  3. blocks by (size, smallest id), ids ascending inside; separator last.
namespace {
struct Bfs {
  const HostCsr& W;
  std::vector<int32_t> stamp;  // allowed iff stamp[v] == cur
  std::vector<int32_t> level;
  std::vector<int32_t> seen;
  int32_t cur = 0, seen_epoch = 0;
  explicit Bfs(const HostCsr& w) : W(w), stamp(w.nrows, -1), level(w.nrows, -1), seen(w.nrows, 0) {}
  // FIFO order from `start` over nodes stamped `cur`
  void run(int64_t start, std::vector<int64_t>& order) {
    ++seen_epoch;
    order.clear();
    order.push_back(start);
    seen[start] = seen_epoch;
    level[start] = 0;
    for (size_t h = 0; h < order.size(); ++h) {
      const int64_t u = order[h];
      for (int64_t k = W.rowptr[u]; k < W.rowptr[u + 1]; ++k) {
        const int64_t v = W.col[k];
        if (stamp[v] == cur && seen[v] != seen_epoch) {
          seen[v] = seen_epoch;
          level[v] = level[u] + 1;
          order.push_back(v);
        }
      }
    }
  }
};
}  // namespace

Partition partition_graph(const HostCsr& W, int64_t n_hubs, int64_t block_max, bool split,
                          const std::vector<int64_t>* hub_list) {
  const int64_t n = W.nrows;
  std::vector<char> sep(n, 0);
  if (hub_list) {
    for (int64_t v : *hub_list) {
      KATZ_REQUIRE(v >= 0 && v < n, KATZ_EINVAL, "hub id out of range");
      sep[v] = 1;
    }
  } else if (n_hubs > 0) {
    std::vector<int64_t> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    auto deg = [&](int64_t v) { return W.rowptr[v + 1] - W.rowptr[v]; };
    const int64_t h = std::min(n_hubs, n);
    std::partial_sort(ord.begin(), ord.begin() + h, ord.end(), [&](int64_t a, int64_t b) {
      return deg(a) != deg(b) ? deg(a) > deg(b) : a < b;
    });
    for (int64_t i = 0; i < h; ++i) sep[ord[i]] = 1;
  }
  Bfs bfs(W);
  std::vector<std::vector<int64_t>> blocks, pending;
  std::vector<int64_t> order;
  // components of the nodes stamped `stampv` among `nodes` (ascending)
  auto components = [&](const std::vector<int64_t>& nodes, int32_t stampv) {
    std::vector<std::vector<int64_t>> out;
    bfs.cur = stampv;
    const int32_t mark = bfs.seen_epoch + 1;  // nodes visited in this sweep
    (void)mark;
    std::vector<char> done;
    for (int64_t s : nodes) {
      if (bfs.stamp[s] != stampv) continue;
      bfs.run(s, order);
      std::vector<int64_t> comp(order.begin(), order.end());
      for (int64_t v : comp) bfs.stamp[v] = -2 - stampv;  // leave the pool
      std::sort(comp.begin(), comp.end());
      out.push_back(std::move(comp));
    }
    return out;
  };
  int32_t next_stamp = 0;
  {
    std::vector<int64_t> all;
    all.reserve(n);
    for (int64_t v = 0; v < n; ++v)
      if (!sep[v]) { all.push_back(v); bfs.stamp[v] = next_stamp; }
    pending = components(all, next_stamp);
    ++next_stamp;
  }
  while (!pending.empty()) {
    std::vector<int64_t> c = std::move(pending.back());
    pending.pop_back();
    if (!split || (int64_t)c.size() <= block_max) {
      blocks.push_back(std::move(c));
      continue;
    }
    const int32_t st = next_stamp++;
    for (int64_t v : c) bfs.stamp[v] = st;
    bfs.cur = st;
    bfs.run(c[0], order);
    const int64_t root = order.back();
    bfs.run(root, order);
    int32_t depth = 0;
    for (int64_t v : order) depth = std::max(depth, bfs.level[v]);
    std::vector<int64_t> cnt(depth + 1, 0);
    for (int64_t v : order) cnt[bfs.level[v]]++;
    int64_t cum = 0;
    int32_t kcut = 0;
    for (int32_t k = 0; k <= depth; ++k) {
      cum += cnt[k];
      if (2 * cum >= (int64_t)c.size()) { kcut = k; break; }
    }
    std::vector<int64_t> rest;
    for (int64_t v : c) {
      if (bfs.level[v] == kcut) { sep[v] = 1; bfs.stamp[v] = -1; }
      else rest.push_back(v);
    }
    const int32_t st2 = next_stamp++;
    for (int64_t v : rest) bfs.stamp[v] = st2;
    auto sub = components(rest, st2);
    for (auto& x : sub) pending.push_back(std::move(x));
  }
  std::sort(blocks.begin(), blocks.end(), [](const std::vector<int64_t>& a, const std::vector<int64_t>& b) {
    return a.size() != b.size() ? a.size() < b.size() : a[0] < b[0];
  });
  Partition p;
  p.perm.reserve(n);
  p.block_ptr.push_back(0);
  for (auto& b : blocks) {
    for (int64_t v : b) p.perm.push_back(v);
    p.block_ptr.push_back((int64_t)p.perm.size());
  }
  p.n1 = (int64_t)p.perm.size();
  for (int64_t v = 0; v < n; ++v)
    if (sep[v]) p.perm.push_back(v);
  p.n2 = n - p.n1;
  return p;
}

// -------------------------------------------- tridiagonal eigen (host)
// Eigen-decomposition of the symmetric tridiagonal Lanczos matrix by
// implicit-shift QL iterations (Golub and Van Loan, Sec. 8.3): d = diagonal,
// e = sub-diagonal; on return d holds the eigenvalues and column j of Z
// (k x k, row-major) the eigenvector of d[j].
static void tridiag_ql(std::vector<double>& d, std::vector<double> e, std::vector<double>& Z, int k) {
  e.resize(k, 0.0);
  Z.assign(size_t(k) * k, 0.0);
  for (int i = 0; i < k; ++i) Z[size_t(i) * k + i] = 1.0;
  for (int l = 0; l < k; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;
      for (; m < k - 1; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= 1e-16 * dd) break;
      }
      if (m == l) break;
      if (iter > 200) throw std::runtime_error("tridiagonal QL did not converge");
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + std::copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      bool split = false;
      for (int i = m - 1; i >= l; --i) {
        double f = s * e[i];
        const double bb = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[m] = 0.0;
          split = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * bb;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - bb;
        for (int t = 0; t < k; ++t) {
          f = Z[size_t(t) * k + i + 1];
          Z[size_t(t) * k + i + 1] = s * Z[size_t(t) * k + i] + c * f;
          Z[size_t(t) * k + i] = c * Z[size_t(t) * k + i] - s * f;
        }
      }
      if (split) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
}
static std::vector<double> splitmix64_uniform(uint64_t seed, int64_t count) {
  std::vector<double> out(count);
  for (int64_t i = 0; i < count; ++i) {
    uint64_t z = seed + uint64_t(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    out[i] = double(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
  return out;
}

static double dget(const double* p, cudaStream_t s) {
  double h = 0;
  KATZ_CUDA(cudaMemcpyAsync(&h, p, sizeof(double), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  return h;
}

// ----------------------------------------------------------- lambda_max
// x_i = |y_i| + floor on column 0 of an ld-strided vector.
__global__ void abs_floor_kernel(const double* y, double* x, int64_t ld, int64_t n, double fl) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    x[i * ld] = fabs(y[i * ld]) + fl;
}
// out = max_i (W x)_i / x_i for x > 0: non-negative doubles order like their
// bit patterns, so atomicMax on the bits gives the maximum.
__global__ void cw_ratio_kernel(const double* wx, const double* x, int64_t ld, int64_t n,
                                unsigned long long* out) {
  double m = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    m = fmax(m, wx[i * ld] / x[i * ld]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// x <- a w + c x on column 0 of ld-strided vectors.
__global__ void axpby_col_kernel(const double* w, double* x, int64_t ld, int64_t n, double a,
                                 double c) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    x[i * ld] = a * w[i * ld] + c * x[i * ld];
}

// Plain Lanczos on W from the normalised all-ones vector; the largest Ritz
// value of the tridiagonal matrix is returned.  The Ritz value is a lower
// bound on lambda_max.  With `lup`, also a rigorous UPPER bound: for
// W >= 0 and any x > 0, lambda_max = rho(W) <= max_i (W x)_i / x_i (the
// Collatz-Wielandt bound: D^{-1} W D with D = diag(x) has these row sums
// and the same spectrum).  x starts as |y| + f max|y| for the top Ritz
// vector y (rebuilt by a second pass of the recurrence with the stored
// coefficients); the floor f keeps x > 0.  Where y vanishes (components
// that do not carry lambda_max) or is below its rounding, the ratio is
// governed by the floor instead, so x is also smoothed by a few steps of
// the positive map x <- (W x + s x) / (2 s), s the Ritz value, which moves
// every component towards its own Perron vector and never raises the
// largest ratio.  Every (floor, step) gives a valid bound; the smallest is
// kept, times 1 + 1e-11 for the rounding of the ratios.
double lambda_max_gpu(const GraphPart& W, int64_t n, int steps, Workspace& ws, cudaStream_t s,
                      uint64_t seed, double* lmin, double* lup) {
  if (lmin) *lmin = 0.0;
  if (lup) *lup = 0.0;
  if (n == 0 || W.csr.nnz == 0) return 0.0;
  const int64_t ld = 2;
  double* v = ws.get<double>("lm.v", n * ld);
  double* vp = ws.get<double>("lm.vp", n * ld);
  double* w = ws.get<double>("lm.w", n * ld);
  double* dd = ws.get<double>("lm.d", 2);
  // start: the normalised all-ones vector (close to the Perron vector), or a
  // SplitMix64 vector, which also has weight on the lower end of the spectrum
  std::vector<double> start(n * ld, 0.0);
  if (seed == 0) {
    for (int64_t i = 0; i < n; ++i) start[i * ld] = 1.0 / std::sqrt(double(n));
  } else {
    const std::vector<double> u = splitmix64_uniform(seed, n);
    double nrm = 0;
    for (int64_t i = 0; i < n; ++i) nrm += (u[i] - 0.5) * (u[i] - 0.5);
    nrm = std::sqrt(nrm);
    for (int64_t i = 0; i < n; ++i) start[i * ld] = (u[i] - 0.5) / nrm;
  }
  KATZ_CUDA(cudaMemcpyAsync(v, start.data(), sizeof(double) * n * ld, cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemsetAsync(vp, 0, sizeof(double) * n * ld, s));
  std::vector<double> al, be;
  double bprev = 0;
  for (int j = 0; j < steps; ++j) {
    spmm<double>(W.view(), W.heavy.p, W.n_heavy, 1.0, v, ld, 0.0, nullptr, ld, w, ld, 1, nullptr,
                 0, nullptr, s);
    KATZ_CUDA(cudaMemsetAsync(dd, 0, sizeof(double) * 2, s));
    coldot<double>(v, ld, w, ld, n, 1, dd, s);
    const double a = dget(dd, s);
    al.push_back(a);
    scale_copy<double>(v, ld, w, ld, n, 1, -a, true, s);
    if (j > 0) scale_copy<double>(vp, ld, w, ld, n, 1, -bprev, true, s);
    KATZ_CUDA(cudaMemsetAsync(dd, 0, sizeof(double) * 2, s));
    coldot<double>(w, ld, w, ld, n, 1, dd, s);
    const double bn = std::sqrt(dget(dd, s));
    if (bn <= 1e-12 * std::max(1.0, std::fabs(a)) || j == steps - 1) break;
    be.push_back(bn);
    std::swap(vp, v);                                           // vp <- v
    scale_copy<double>(w, ld, v, ld, n, 1, 1.0 / bn, false, s);  // v <- w / bn
    bprev = bn;
  }
  const int m = (int)al.size();
  std::vector<double> ev(al), Z;
  be.resize(std::max(0, m - 1));
  tridiag_ql(ev, be, Z, m);
  if (lmin) *lmin = *std::min_element(ev.begin(), ev.end());
  const int top = int(std::max_element(ev.begin(), ev.end()) - ev.begin());
  if (lup) {
    // second pass: y = sum_j Z[j][top] v_j with the stored coefficients
    double* y = ws.get<double>("lm.y", n * ld);
    KATZ_CUDA(cudaMemcpyAsync(v, start.data(), sizeof(double) * n * ld, cudaMemcpyHostToDevice, s));
    KATZ_CUDA(cudaMemsetAsync(vp, 0, sizeof(double) * n * ld, s));
    KATZ_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * n * ld, s));
    for (int j = 0; j < m; ++j) {
      scale_copy<double>(v, ld, y, ld, n, 1, Z[size_t(j) * m + top], true, s);
      if (j == m - 1) break;
      spmm<double>(W.view(), W.heavy.p, W.n_heavy, 1.0, v, ld, 0.0, nullptr, ld, w, ld, 1,
                   nullptr, 0, nullptr, s);
      scale_copy<double>(v, ld, w, ld, n, 1, -al[j], true, s);
      if (j > 0) scale_copy<double>(vp, ld, w, ld, n, 1, -be[j - 1], true, s);
      std::swap(vp, v);
      scale_copy<double>(w, ld, v, ld, n, 1, 1.0 / be[j], false, s);
    }
    double* nrm = ws.get<double>("lm.n", 2);
    double* mx = ws.get<double>("lm.mx", 2);
    col_norms<double>(y, ld, n, 1, nrm, mx, s);
    const double ymax = dget(mx, s);
    double best = HUGE_VAL;
    const double sig = std::max(ev[top], 1e-300);
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 4096));
    for (double f : {1e-12, 1e-8, 1e-4, 1e-1}) {
      // x = |y| + f max|y| (the all-ones vector when y vanishes)
      abs_floor_kernel<<<nb, 256, 0, s>>>(y, v, ld, n, ymax > 0 ? f * ymax : 1.0);
      KATZ_CHECK_LAUNCH();
      for (int k = 0; k <= 16; ++k) {
        spmm<double>(W.view(), W.heavy.p, W.n_heavy, 1.0, v, ld, 0.0, nullptr, ld, w, ld, 1,
                     nullptr, 0, nullptr, s);
        KATZ_CUDA(cudaMemsetAsync(dd, 0, sizeof(double), s));
        cw_ratio_kernel<<<nb, 256, 0, s>>>(w, v, ld, n, reinterpret_cast<unsigned long long*>(dd));
        KATZ_CHECK_LAUNCH();
        best = std::min(best, dget(dd, s));
        axpby_col_kernel<<<nb, 256, 0, s>>>(w, v, ld, n, 0.5 / sig, 0.5);
        KATZ_CHECK_LAUNCH();
      }
      if (ymax <= 0) break;
    }
    *lup = best * (1.0 + 1e-11);
  }
  return ev[top];
}

// --------------------------------------------------------- device helpers
__global__ void identity_cols_kernel(double* E, int64_t ld, int64_t rows, int64_t j0, int cw) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cw; c += gridDim.x * blockDim.x)
    if (j0 + c < rows) E[(j0 + c) * ld + c] = 1.0;
}

__global__ void dense_from_csr_kernel(Csr A, double beta, double* D, int64_t ld) {
  for (int64_t i = blockIdx.x; i < A.nrows; i += gridDim.x) {
    if (threadIdx.x == 0) D[i * ld + i] = 1.0;
    for (int64_t k = A.rowptr[i] + threadIdx.x; k < A.rowptr[i + 1]; k += blockDim.x) {
      double w = 1.0;
      if (A.vdt == KATZ_F64) w = static_cast<const double*>(A.val)[k];
      else if (A.vdt == KATZ_F32) w = static_cast<const float*>(A.val)[k];
      else if (A.vdt == KATZ_BF16) w = __bfloat162float(static_cast<const __nv_bfloat16*>(A.val)[k]);
      D[i * ld + A.col[k]] -= beta * w;
    }
  }
}

__global__ void sub_kernel(const double* A, const double* B, double* C, int64_t total) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x)
    C[e] = A[e] - B[e];
}

// Z[:, j0 + c] = V[:, c] for c < cw (V: rows x ldv FP64, Z: rows x ldz FP32)
__global__ void cols_to_f32_kernel(const double* V, int64_t ldv, int64_t rows, int cw, float* Z,
                                   int64_t ldz, int64_t j0) {
  const int64_t total = rows * cw;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / cw, c = e % cw;
    Z[i * ldz + j0 + c] = float(V[i * ldv + c]);
  }
}

__global__ void to_f32_kernel(const double* A, float* B, int64_t total) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x)
    B[e] = float(A[e]);
}

static unsigned blocks_for(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), int64_t(num_sms()) * 16));
}

// ------------------------------------- block-diagonal (per-graph) pieces
// For an index of disjoint graphs: separator rows of graph g are
// [gsep[g], gsep[g+1]) (node ids graph-major, separator in ascending node
// order) and sg[p] is the graph of separator row p.

// E[p][l] = 1 for separator rows p whose local index (p - gsep[g]) is l0 + l,
// l < cw: column l of the packed right-hand side holds the local separator
// node l0 + l of EVERY graph at once.
__global__ void packed_identity_kernel(double* E, int64_t ldc, int64_t n2, const int32_t* sg,
                                       const int64_t* gsep, int l0, int cw) {
  for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n2;
       p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t l = p - gsep[sg[p]] - l0;
    if (l >= 0 && l < cw) E[p * ldc + l] = 1.0;
  }
}

// T[p][gsep[g] + l0 + l] = Tp[p][l] for p in graph g (the packed columns
// back to their places in the block-diagonal n2 x n2 matrix).
__global__ void packed_scatter_kernel(const double* Tp, int64_t ldc, double* T, int64_t ld2,
                                      int64_t n2, const int32_t* sg, const int64_t* gsep, int l0,
                                      int cw) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n2 * cw;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = e / cw;
    const int l = int(e - p * cw);
    const int g = sg[p];
    const int64_t q = gsep[g] + l0 + l;
    if (q < gsep[g + 1]) T[p * ld2 + q] = Tp[p * ldc + l];
  }
}

// out[g] = sum over the rows p of graph g of x[p * incx] * y[p * incy]
// (one CTA of 128 threads per graph, fixed summation order).
__global__ void segdot_kernel(const double* x, int64_t incx, const double* y, int64_t incy,
                              const int64_t* gsep, double* out) {
  __shared__ double red[4];
  const int g = blockIdx.x;
  double acc = 0.0;
  for (int64_t p = gsep[g] + threadIdx.x; p < gsep[g + 1]; p += blockDim.x)
    acc += x[p * incx] * y[p * incy];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) out[g] = red[0] + red[1] + red[2] + red[3];
}

// C[k * G + g] = sum over the rows p of graph g of Q[p][k] * u[p], k < kk.
__global__ void seg_coeff_kernel(const double* Q, int64_t ldq, const double* u,
                                 const int64_t* gsep, int kk, int G, double* C) {
  const int g = blockIdx.x;
  for (int k = threadIdx.x; k < kk; k += blockDim.x) {
    double acc = 0.0;
    for (int64_t p = gsep[g]; p < gsep[g + 1]; ++p) acc += Q[p * ldq + k] * u[p];
    C[int64_t(k) * G + g] = acc;
  }
}

// w[p] -= sum_{k < kk} Q[p][k] * C[k * G + g(p)]
__global__ void seg_reorth_kernel(const double* Q, int64_t ldq, const double* C, int kk, int G,
                                  const int32_t* sg, int64_t n2, double* w) {
  for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n2;
       p += int64_t(gridDim.x) * blockDim.x) {
    const int g = sg[p];
    double acc = 0.0;
    for (int k = 0; k < kk; ++k) acc += Q[p * ldq + k] * C[int64_t(k) * G + g];
    w[p] -= acc;
  }
}

// Q[p][col] = w[p] * scale[g(p)]
__global__ void seg_scale_kernel(const double* w, const double* scale, const int32_t* sg,
                                 int64_t n2, double* Q, int64_t ldq, int col) {
  for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n2;
       p += int64_t(gridDim.x) * blockDim.x)
    Q[p * ldq + col] = w[p] * scale[sg[p]];
}

// Stores the basis W_r (host, n2 x rk row-major, W_r^T M22 W_r = I on each
// graph's block) with idx.sigma: the unscaled FP32 copy, W^ = W_r D^{1/2}
// (D = diag(sigma / (1 - sigma))) in FP64 / FP32, and the BF16 copies of
// W^ for the tensor-core products of the preconditioner (Eq. 14).
static void store_basis(katz_index& idx, std::vector<double>& Wh, int rk, cudaStream_t s) {
  const int64_t n2 = idx.n2;
  idx.rank = rk;
  idx.ldr4 = (rk + 3) / 4 * 4;
  {
    std::vector<float> wu(size_t(n2) * idx.ldr4, 0.f);
    for (int64_t i = 0; i < n2; ++i)
      for (int c = 0; c < rk; ++c) wu[size_t(i) * idx.ldr4 + c] = float(Wh[size_t(i) * rk + c]);
    idx.Wr32u.alloc(wu.size());
    KATZ_CUDA(cudaMemcpyAsync(idx.Wr32u.p, wu.data(), 4 * wu.size(), cudaMemcpyHostToDevice, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<float> Wf(Wh.size());
  for (int c = 0; c < rk; ++c) {
    const double sg = std::min(std::max(idx.sigma[c], 0.0), 1.0 - 1e-12);
    const double f = std::sqrt(sg / (1.0 - sg));
    for (int64_t i = 0; i < n2; ++i) {
      Wh[size_t(i) * rk + c] *= f;
      Wf[size_t(i) * rk + c] = float(Wh[size_t(i) * rk + c]);
    }
  }
  idx.ldr = (rk + 7) / 8 * 8;
  idx.ldn2 = (n2 + 7) / 8 * 8;
  std::vector<__nv_bfloat16> wb(size_t(n2) * idx.ldr, __float2bfloat16(0.f)),
      wbt(size_t(rk) * idx.ldn2, __float2bfloat16(0.f));
  for (int64_t i = 0; i < n2; ++i)
    for (int c = 0; c < rk; ++c) {
      const __nv_bfloat16 v = __double2bfloat16(Wh[size_t(i) * rk + c]);
      wb[size_t(i) * idx.ldr + c] = v;
      wbt[size_t(c) * idx.ldn2 + i] = v;
    }
  idx.Wb.alloc(wb.size());
  idx.WbT.alloc(wbt.size());
  KATZ_CUDA(cudaMemcpyAsync(idx.Wb.p, wb.data(), 2 * wb.size(), cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(idx.WbT.p, wbt.data(), 2 * wbt.size(), cudaMemcpyHostToDevice, s));
  idx.Wr64.alloc(Wh.size());
  idx.Wr32.alloc(Wf.size());
  KATZ_CUDA(cudaMemcpyAsync(idx.Wr64.p, Wh.data(), 8 * Wh.size(), cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(idx.Wr32.p, Wf.data(), 4 * Wf.size(), cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
}

// Lanczos on every graph's block at once (the same iteration as the
// single-graph build below, with every scalar kept per graph): on graph g,
// A_g = M22_g^{-1} T_g in the M22_g inner product, full reorthogonalisation,
// extended until the top r_g Ritz residuals converge, stopped early when the
// Krylov space fills the graph's separator.  Returns the basis (host, n2 x
// sum r_g, graph g's columns at its offset, zero outside its rows) and sets
// idx.sigma (graph-major).
// The per-graph bases W_g (packed, n2_g x r_g each) scaled by
// D_g^{1/2} = diag(sqrt(sigma / (1 - sigma))) into W^_g (Eq. 14).
static void store_seg_basis(katz_index& idx, std::vector<double>& Wh, const std::vector<int>& rkg,
                            cudaStream_t s) {
  SegBlocks& sb = idx.sb;
  const int G = sb.G;
  sb.rk_h.assign(rkg.begin(), rkg.end());
  sb.woff_h.assign(G + 1, 0);
  for (int g = 0; g < G; ++g)
    sb.woff_h[g + 1] = sb.woff_h[g] + (sb.gsep_h[g + 1] - sb.gsep_h[g]) * rkg[g];
  sb.nw = sb.woff_h[G];
  int so = 0;  // offset of graph g's Ritz values in idx.sigma
  for (int g = 0; g < G; ++g) {
    const int r = rkg[g];
    KATZ_REQUIRE(r <= kSegBlockMax / 4, KATZ_EINVAL, "per-graph rank above 64");
    const int64_t n = sb.gsep_h[g + 1] - sb.gsep_h[g];
    for (int c = 0; c < r; ++c) {
      const double sg = std::min(std::max(idx.sigma[so + c], 0.0), 1.0 - 1e-12);
      const double f = std::sqrt(sg / (1.0 - sg));
      for (int64_t i = 0; i < n; ++i) Wh[sb.woff_h[g] + i * r + c] *= f;
    }
    so += r;
  }
  idx.rank = so;
  std::vector<float> Wf(Wh.begin(), Wh.end());
  sb.W64.alloc(Wh.size());
  sb.W32.alloc(Wf.size());
  sb.woff.alloc(sb.woff_h.size());
  sb.rk.alloc(std::max(G, 1));
  KATZ_CUDA(cudaMemcpyAsync(sb.W64.p, Wh.data(), 8 * Wh.size(), cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(sb.W32.p, Wf.data(), 4 * Wf.size(), cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(sb.woff.p, sb.woff_h.data(), 8 * sb.woff_h.size(),
                            cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(sb.rk.p, sb.rk_h.data(), 4 * sb.rk_h.size(), cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
}

static std::vector<double> seg_lanczos(katz_index& idx, const SegSpec& seg,
                                       const std::vector<int64_t>& gsep_h, const int32_t* sg,
                                       const int64_t* gsep, const double* T, const double* M22,
                                       int64_t ld2, uint64_t seed, int lanczos_steps, int* rk_out,
                                       std::vector<int>* rk_graph, cudaStream_t s) {
  const int G = seg.G;
  const int64_t n2 = idx.n2;
  std::vector<int> r(G), mg(G), capg(G), check(G);
  int capmax = 0;
  for (int g = 0; g < G; ++g) {
    const int64_t ng = gsep_h[g + 1] - gsep_h[g];
    r[g] = (int)std::min<int64_t>(std::max(0, seg.ranks[g]), ng);
    int m = lanczos_steps > 0 ? lanczos_steps : std::max(2 * r[g], r[g] + 20);
    mg[g] = (int)std::min<int64_t>(std::max(m, r[g]), ng);
    capg[g] = r[g] > 0 ? (int)std::min<int64_t>(ng, std::max(4 * mg[g], mg[g] + 200)) : 0;
    check[g] = mg[g];
    capmax = std::max(capmax, capg[g]);
  }
  rk_graph->assign(G, 0);
  *rk_out = 0;
  idx.sigma.clear();
  if (capmax == 0) return {};
  const int64_t ldq = capmax + 1;
  DBuf<double> Q(size_t(n2) * ldq), t(n2), wv(n2), u(n2), dots(G), C(size_t(ldq) * G),
      scale(G);
  KATZ_CUDA(cudaMemsetAsync(Q.p, 0, Q.bytes(), s));
  std::vector<double> v0 = splitmix64_uniform(seed, n2);
  KATZ_CUDA(cudaMemcpyAsync(wv.p, v0.data(), 8 * n2, cudaMemcpyHostToDevice, s));
  std::vector<double> hd(G), hs(G);
  auto segdot = [&](const double* x, int64_t incx, const double* y) {  // per graph x^T y
    segdot_kernel<<<G, 128, 0, s>>>(x, incx, y, 1, gsep, dots.p);
    KATZ_CHECK_LAUNCH();
    KATZ_CUDA(cudaMemcpyAsync(hd.data(), dots.p, 8 * G, cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    return hd;
  };
  const SegBlocks& sb = idx.sb;
  auto mdot = [&](const double* x) {  // per graph x^T M22 x
    seg_block_mv64(sb, M22, x, 1, u.p, 1, s);
    return segdot(x, 1, u.p);
  };
  auto put = [&](int col) {
    KATZ_CUDA(cudaMemcpyAsync(scale.p, hs.data(), 8 * G, cudaMemcpyHostToDevice, s));
    seg_scale_kernel<<<blocks_for(n2), 256, 0, s>>>(wv.p, scale.p, sg, n2, Q.p, ldq, col);
    KATZ_CHECK_LAUNCH();
  };
  std::vector<char> active(G, 0);
  {
    const std::vector<double> nr = mdot(wv.p);
    for (int g = 0; g < G; ++g) {
      active[g] = r[g] > 0 && nr[g] > 0;
      hs[g] = active[g] ? 1.0 / std::sqrt(nr[g]) : 0.0;
    }
    put(0);
  }
  std::vector<std::vector<double>> al(G), be(G);
  std::vector<double> ev, Y;
  for (int j = 0; j < capmax; ++j) {
    bool any = false;
    for (int g = 0; g < G; ++g) any |= active[g] != 0;
    if (!any) break;
    // t = T q_j ; w = M22^{-1} t ; alpha = q_j^T t (block by block)
    seg_block_mv64(sb, T, Q.p + j, ldq, t.p, 1, s);
    seg_block_mv64(sb, sb.Minv64.p, t.p, 1, wv.p, 1, s);
    const std::vector<double> a = segdot(Q.p + j, ldq, t.p);
    for (int g = 0; g < G; ++g)
      if (active[g]) al[g].push_back(a[g]);
    for (int pass = 0; pass < 2; ++pass) {
      seg_block_mv64(sb, M22, wv.p, 1, u.p, 1, s);
      seg_coeff_kernel<<<G, 128, 0, s>>>(Q.p, ldq, u.p, gsep, j + 1, G, C.p);
      KATZ_CHECK_LAUNCH();
      seg_reorth_kernel<<<blocks_for(n2), 256, 0, s>>>(Q.p, ldq, C.p, j + 1, G, sg, n2, wv.p);
      KATZ_CHECK_LAUNCH();
    }
    const std::vector<double> bsq = mdot(wv.p);
    for (int g = 0; g < G; ++g) {
      hs[g] = 0.0;
      if (!active[g]) continue;
      const int64_t ng = gsep_h[g + 1] - gsep_h[g];
      const double bj = std::sqrt(std::max(0.0, bsq[g]));
      const int kk = (int)al[g].size();
      bool stop = bj <= 1e-14 * std::max(1.0, std::fabs(al[g].back())) || kk >= ng;
      if (!stop && (kk >= check[g] || kk == capg[g])) {
        ev = al[g];
        tridiag_ql(ev, be[g], Y, kk);
        std::vector<int> o2(kk);
        std::iota(o2.begin(), o2.end(), 0);
        std::sort(o2.begin(), o2.end(), [&](int x, int y) { return ev[x] > ev[y]; });
        bool ok = true;
        for (int c = 0; c < std::min(r[g], kk); ++c)
          ok &= bj * std::fabs(Y[size_t(kk - 1) * kk + o2[c]]) <=
                1e-8 * std::max(1.0, std::fabs(ev[o2[c]]));
        if (ok || kk == capg[g]) stop = true;
        else check[g] = kk + std::max(10, kk / 2);
      }
      if (stop) {
        active[g] = 0;
      } else {
        be[g].push_back(bj);
        hs[g] = 1.0 / bj;
      }
    }
    put(j + 1);
  }
  // Ritz vectors per graph: W_g = Q_g Y_g (top r_g)
  std::vector<double> Qh(size_t(n2) * ldq);
  KATZ_CUDA(cudaMemcpyAsync(Qh.data(), Q.p, 8 * Qh.size(), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  std::vector<std::vector<double>> Ysel(G);
  std::vector<int> off(G + 1, 0);
  for (int g = 0; g < G; ++g) {
    const int k = (int)al[g].size();
    int rk = 0;
    if (r[g] > 0 && k > 0) {
      ev = al[g];
      std::vector<double> sub(be[g].begin(), be[g].begin() + std::max(0, k - 1));
      tridiag_ql(ev, sub, Y, k);
      std::vector<int> ord(k);
      std::iota(ord.begin(), ord.end(), 0);
      std::sort(ord.begin(), ord.end(), [&](int x, int y) { return ev[x] > ev[y]; });
      rk = std::min(r[g], k);
      Ysel[g].assign(size_t(k) * rk, 0.0);
      for (int c = 0; c < rk; ++c) {
        idx.sigma.push_back(ev[ord[c]]);
        for (int i = 0; i < k; ++i) Ysel[g][size_t(i) * rk + c] = Y[size_t(i) * k + ord[c]];
      }
    }
    (*rk_graph)[g] = rk;
    off[g + 1] = off[g] + rk;
  }
  const int rk_tot = off[G];
  *rk_out = rk_tot;
  // W_g (n2_g x r_g, row-major) packed graph after graph
  int64_t nw = 0;
  for (int g = 0; g < G; ++g) nw += (gsep_h[g + 1] - gsep_h[g]) * (*rk_graph)[g];
  std::vector<double> Wh(size_t(std::max<int64_t>(nw, 1)), 0.0);
  int64_t wo = 0;
  for (int g = 0; g < G; ++g) {
    const int rk = (*rk_graph)[g];
    const int k = (int)al[g].size();
    for (int64_t p = gsep_h[g]; p < gsep_h[g + 1]; ++p)
      for (int c = 0; c < rk; ++c) {
        double acc = 0.0;
        for (int i = 0; i < k; ++i) acc += Qh[size_t(p) * ldq + i] * Ysel[g][size_t(i) * rk + c];
        Wh[wo + (p - gsep_h[g]) * rk + c] = acc;
      }
    wo += (gsep_h[g + 1] - gsep_h[g]) * rk;
  }
  idx.lanczos_steps = 0;
  for (int g = 0; g < G; ++g) idx.lanczos_steps = std::max(idx.lanczos_steps, (int)al[g].size());
  return Wh;
}

// ------------------------------------------------------------- build
void build_index(katz_index& idx, const HostCsr& W, double beta, const katz_build_opts& o,
                 cudaStream_t s, const SegSpec* seg) {
  idx.n = W.nrows;
  idx.nnz = W.nnz();
  idx.beta = beta;
  idx.vdt = o.value_dtype;
  idx.deg_h.resize(W.nrows);
  idx.maxdeg = 0;
  for (int64_t i = 0; i < W.nrows; ++i) {
    idx.deg_h[i] = (int32_t)(W.rowptr[i + 1] - W.rowptr[i]);
    idx.maxdeg = std::max<int64_t>(idx.maxdeg, idx.deg_h[i]);
  }
  idx.unit_weights = true;
  for (double v : W.val)
    if (v != 1.0) { idx.unit_weights = false; break; }
  // graphs whose stored weights are all 1 keep no values on the device: every
  // product then runs its unit-weight kernel (no weight loads or products)
  const int sdt = idx.unit_weights ? int(KATZ_UNIT) : o.value_dtype;
  upload_part(W, sdt, idx.W, s);
  // Ritz value (a lower bound on lambda_max) and a rigorous upper bound: M is
  // certified SPD and the error-bound stopping rule is sound only with the
  // upper bound
  idx.lambda = lambda_max_gpu(idx.W, idx.n, 96, idx.ws, s, 0, nullptr, &idx.lambda_up);
  KATZ_REQUIRE(beta * idx.lambda < 1.0, KATZ_ENOTSPD,
               "beta * lambda_max = " + std::to_string(beta * idx.lambda) +
                   " >= 1: M = I - beta W is not positive definite");
  KATZ_REQUIRE(beta * idx.lambda_up < 1.0, KATZ_ENOTSPD,
               "beta * (upper bound on lambda_max) = " + std::to_string(beta * idx.lambda_up) +
                   " >= 1: M = I - beta W cannot be certified positive definite");
  if (!o.build_lrc) return;

  idx.lrc = true;
  idx.rank = std::max(0, o.rank);
  idx.block_max = o.block_max > 0 ? o.block_max : 64;
  idx.split = o.split;
  KATZ_REQUIRE(idx.block_max <= 128, KATZ_EINVAL, "block_max must be <= 128");
  const int64_t n2_max = o.n2_max > 0 ? o.n2_max : 16384;
  Partition& P = idx.part;
  P = partition_graph(W, std::max(0, o.n_hubs), idx.block_max, o.split != 0,
                      seg ? &seg->hubs : nullptr);
  const int64_t n = idx.n, n1 = P.n1, n2 = P.n2;
  idx.n1 = n1;
  idx.n2 = n2;
  // separators above n2_max keep S implicit (single graphs); M22 and its
  // inverse stay dense, which bounds the separator at kDenseM22Max
  idx.s_implicit = !seg && n2 > n2_max;
  KATZ_REQUIRE((seg && n2 <= n2_max) || (!seg && n2 <= kDenseM22Max), KATZ_EINVAL,
               "separator has " + std::to_string(n2) + " nodes > " +
                   std::to_string(seg ? n2_max : kDenseM22Max));
  // disjoint graphs: each graph's separator rows (contiguous, graph-major)
  std::vector<int64_t> gsep_h;
  DBuf<int32_t> sg_d;
  DBuf<int64_t> gsep_d;
  int64_t width = 0;  // largest separator of one graph
  if (seg) {
    KATZ_REQUIRE((int64_t)seg->node_graph.size() == n && seg->G > 0, KATZ_EINVAL,
                 "segment map does not match the graph");
    gsep_h.assign(seg->G + 1, 0);
    std::vector<int32_t> sgh(std::max<int64_t>(n2, 1), 0);
    int32_t prev = -1;
    for (int64_t p = 0; p < n2; ++p) {
      const int32_t g = seg->node_graph[P.perm[P.n1 + p]];
      KATZ_REQUIRE(g >= prev, KATZ_EINVAL, "graph ids must be graph-major");
      prev = g;
      sgh[p] = g;
      gsep_h[g + 1]++;
    }
    for (int g = 0; g < seg->G; ++g) {
      width = std::max(width, gsep_h[g + 1]);
      gsep_h[g + 1] += gsep_h[g];
    }
    sg_d.alloc(sgh.size());
    gsep_d.alloc(gsep_h.size());
    KATZ_CUDA(cudaMemcpyAsync(sg_d.p, sgh.data(), 4 * sgh.size(), cudaMemcpyHostToDevice, s));
    KATZ_CUDA(cudaMemcpyAsync(gsep_d.p, gsep_h.data(), 8 * gsep_h.size(), cudaMemcpyHostToDevice,
                              s));
    // block-by-block storage of S, M22^{-1} and W^ (one block per graph)
    KATZ_REQUIRE(width <= kSegBlockMax, KATZ_EINVAL,
                 "a graph's separator has " + std::to_string(width) + " nodes > " +
                     std::to_string(kSegBlockMax));
    SegBlocks& sb = idx.sb;
    idx.seg_blocked = true;
    sb.G = seg->G;
    sb.gsep_h = gsep_h;
    sb.moff_h.assign(seg->G + 1, 0);
    for (int g = 0; g < seg->G; ++g) {
      const int64_t ng = gsep_h[g + 1] - gsep_h[g];
      sb.moff_h[g + 1] = sb.moff_h[g] + ng * ng;
    }
    sb.nmat = sb.moff_h[seg->G];
    sb.gsep.alloc(gsep_h.size());
    sb.moff.alloc(sb.moff_h.size());
    sb.sg.alloc(sgh.size());
    KATZ_CUDA(cudaMemcpyAsync(sb.gsep.p, gsep_h.data(), 8 * gsep_h.size(), cudaMemcpyHostToDevice, s));
    KATZ_CUDA(cudaMemcpyAsync(sb.moff.p, sb.moff_h.data(), 8 * sb.moff_h.size(),
                              cudaMemcpyHostToDevice, s));
    KATZ_CUDA(cudaMemcpyAsync(sb.sg.p, sgh.data(), 4 * sgh.size(), cudaMemcpyHostToDevice, s));
  }
  std::vector<int32_t> iperm(n), perm32(n);
  for (int64_t i = 0; i < n; ++i) {
    perm32[i] = (int32_t)P.perm[i];
    iperm[P.perm[i]] = (int32_t)i;
  }
  idx.perm.alloc(n);
  idx.iperm.alloc(n);
  KATZ_CUDA(cudaMemcpyAsync(idx.perm.p, perm32.data(), 4 * n, cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(idx.iperm.p, iperm.data(), 4 * n, cudaMemcpyHostToDevice, s));

  // --- large-block region
  const int64_t nblocks = (int64_t)P.block_ptr.size() - 1;
  int64_t first_large = nblocks;
  for (int64_t bi = 0; bi < nblocks; ++bi)
    if (P.block_ptr[bi + 1] - P.block_ptr[bi] > idx.block_max) { first_large = bi; break; }
  idx.n1s = P.block_ptr[first_large];
  idx.n_large = (int)(nblocks - first_large);

  // --- permuted CSR pieces (host), rows in index order, columns sorted
  HostCsr Wp, W12, W21, W22, W11L;
  Wp.nrows = Wp.ncols = n;
  W12.nrows = n1; W12.ncols = n2;
  W21.nrows = n2; W21.ncols = n1;
  W22.nrows = W22.ncols = n2;
  W11L.nrows = W11L.ncols = n1 - idx.n1s;
  const bool has_val = !W.val.empty();
  Wp.rowptr.assign(n + 1, 0);
  Wp.col.resize(idx.nnz);
  if (has_val) Wp.val.resize(idx.nnz);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t o0 = P.perm[i];
    Wp.rowptr[i + 1] = Wp.rowptr[i] + (W.rowptr[o0 + 1] - W.rowptr[o0]);
  }
  {
    const int nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t)
      th.emplace_back([&, t]() {
        std::vector<std::pair<int32_t, double>> tmp;
        for (int64_t i = t; i < n; i += nth) {
          const int64_t o0 = P.perm[i];
          tmp.clear();
          for (int64_t k = W.rowptr[o0]; k < W.rowptr[o0 + 1]; ++k)
            tmp.emplace_back(iperm[W.col[k]], has_val ? W.val[k] : 1.0);
          std::sort(tmp.begin(), tmp.end(),
                    [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                      return a.first < b.first;
                    });
          int64_t d = Wp.rowptr[i];
          for (auto& e : tmp) {
            Wp.col[d] = e.first;
            if (has_val) Wp.val[d] = e.second;
            ++d;
          }
        }
      });
    for (auto& x : th) x.join();
  }
  auto sub = [&](HostCsr& out, int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
    out.rowptr.assign(r1 - r0 + 1, 0);
    for (int64_t i = r0; i < r1; ++i) {
      int64_t cnt = 0;
      for (int64_t k = Wp.rowptr[i]; k < Wp.rowptr[i + 1]; ++k)
        cnt += (Wp.col[k] >= c0 && Wp.col[k] < c1);
      out.rowptr[i - r0 + 1] = out.rowptr[i - r0] + cnt;
    }
    out.col.resize(out.rowptr.back());
    if (has_val) out.val.resize(out.rowptr.back());
    int64_t d = 0;
    for (int64_t i = r0; i < r1; ++i)
      for (int64_t k = Wp.rowptr[i]; k < Wp.rowptr[i + 1]; ++k)
        if (Wp.col[k] >= c0 && Wp.col[k] < c1) {
          out.col[d] = (int32_t)(Wp.col[k] - c0);
          if (has_val) out.val[d] = Wp.val[k];
          ++d;
        }
  };
  sub(W12, 0, n1, n1, n);
  sub(W21, n1, n, 0, n1);
  sub(W22, n1, n, n1, n);
  sub(W11L, idx.n1s, n1, idx.n1s, n1);
  upload_part(Wp, sdt, idx.Wp, s);
  upload_part(W12, sdt, idx.W12, s);
  upload_part(W21, sdt, idx.W21, s);
  upload_part(W11L, sdt, idx.W11L, s);
  if (W11L.nrows > 0 && W11L.nnz() > 0) {
    // Lanczos Ritz values lie inside the spectrum: widen both ends by 2% of
    // its width; the lower end never below -lambda_max (W11 >= 0)
    double up = 0, bot = 0;
    const double top = lambda_max_gpu(idx.W11L, W11L.nrows, 96, idx.ws, s, 0, nullptr, &up);
    lambda_max_gpu(idx.W11L, W11L.nrows, 96, idx.ws, s, 0x243F6A8885A308D3ull, &bot);
    // the upper end is the rigorous bound (so no eigenvalue of M11 lies below
    // the interval, where the iteration would diverge); the lower end widened
    // by 2% of the width (an eigenvalue slightly above it costs only speed)
    const double lam = up;
    idx.lam11 = beta * lam < 0.999 ? lam : 0.0;
    idx.lam11_min = std::max(-lam, std::min(0.0, bot - 0.02 * (top - bot)));
  } else if (W11L.nrows > 0) {
    idx.lam11 = 1e-300;  // no edges: M11 = I
  }
  upload_part(W22, sdt, idx.W22, s);
  const GraphPart& W22d = idx.W22;

  // --- M11 dense block inverses by size class (Step 4)
  DBuf<int> flag(1);
  KATZ_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  idx.classes.clear();
  int64_t bi = 0;
  while (bi < first_large) {
    const int64_t sz = P.block_ptr[bi + 1] - P.block_ptr[bi];
    int S = 1;
    while (S < sz) S *= 2;
    std::vector<int64_t> st;
    std::vector<int32_t> sizes;
    while (bi < first_large) {
      const int64_t z = P.block_ptr[bi + 1] - P.block_ptr[bi];
      if (z > S) break;
      st.push_back(P.block_ptr[bi]);
      sizes.push_back((int32_t)z);
      ++bi;
    }
    BlockClass c;
    c.S = S;
    c.count = (int64_t)st.size();
    c.start.alloc(c.count);
    c.size.alloc(c.count);
    KATZ_CUDA(cudaMemcpyAsync(c.start.p, st.data(), 8 * c.count, cudaMemcpyHostToDevice, s));
    KATZ_CUDA(cudaMemcpyAsync(c.size.p, sizes.data(), 4 * c.count, cudaMemcpyHostToDevice, s));
    c.inv64.alloc(size_t(c.count) * S * S);
    c.inv32.alloc(size_t(c.count) * S * S);
    block_inverses(idx.Wp.view(), c.start.p, c.size.p, c.count, S, beta, c.inv64.p, flag.p, s);
    to_f32_kernel<<<blocks_for(c.count * S * S), 256, 0, s>>>(c.inv64.p, c.inv32.p,
                                                              c.count * int64_t(S) * S);
    KATZ_CHECK_LAUNCH();
    idx.classes.push_back(std::move(c));
  }
  int hflag = 0;
  KATZ_CUDA(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  KATZ_REQUIRE(hflag == 0, KATZ_ENOTSPD, "an M11 diagonal block is not positive definite");

  if (n2 == 0) {
    idx.rank = 0;
    return;
  }
  // --- T = M12^T M11^{-1} M12 = beta^2 W21 M11^{-1} W12 (FP64, by columns)
  const int64_t ld2 = (n2 + 3) / 4 * 4;
  idx.ld2 = ld2;
  // (many graphs: the per-graph blocks T_g, packed; else dense n2 x n2)
  DBuf<double> T(idx.s_implicit ? size_t(1)
                 : seg         ? size_t(std::max<int64_t>(idx.sb.nmat, 1))
                               : size_t(n2) * ld2);
  KATZ_CUDA(cudaMemsetAsync(T.p, 0, T.bytes(), s));
  {
    const int cw_max = (int)std::min<int64_t>(256, (n2 + 1) / 2 * 2);
    const int64_t ldc = (cw_max + 3) / 4 * 4;
    DBuf<double> E(size_t(n2) * ldc), U(size_t(std::max<int64_t>(n1, 1)) * ldc),
        V(size_t(std::max<int64_t>(n1, 1)) * ldc);
    // V = beta M11^{-1} W12 by column chunks; kept (TF32 parts) for the
    // tensor-core back-substitution where the large M11 blocks are solved
    // iteratively and the two n1 x n2 FP32 arrays fit
    idx.ldH = (n2 + 3) / 4 * 4;
    {
      size_t free_b = 0, total_b = 0;
      KATZ_CUDA(cudaMemGetInfo(&free_b, &total_b));
      const double bytes = 2.0 * 4.0 * double(n1) * double(idx.ldH);
      // automatic: where the cost model favours the product at the FP32
      // inner tolerance (2e-6) and the parts fit
      idx.has_h = !seg && !idx.s_implicit && n1 > 0 && (o.coupling_gemm > 0 ||
                             (o.coupling_gemm == 0 && coupling_gemm_pays(idx, 1024, 2e-6) &&
                              bytes <= double(total_b) / 3.0 && bytes <= 0.8 * double(free_b)));
    }
    if (idx.has_h) {
      idx.Hh.alloc(size_t(n1) * idx.ldH);
      idx.Hl.alloc(size_t(n1) * idx.ldH);
    }
    // Z = beta M11^{-1} W12 in FP32 for the first Schur right-hand side of a
    // query (automatic: where the first M11 solve of a query is iterative)
    idx.ldZ = (n2 + 3) / 4 * 4;
    {
      size_t free_b = 0, total_b = 0;
      KATZ_CUDA(cudaMemGetInfo(&free_b, &total_b));
      const double bytes = 4.0 * double(n1) * double(idx.ldZ);
      idx.has_z = !seg && !idx.s_implicit && n1 > 0 && o.rhs_coupling >= 0 &&
                  (o.rhs_coupling > 0 || (n1 > idx.n1s && bytes <= double(total_b) / 4.0 &&
                                          bytes <= 0.6 * double(free_b)));
    }
    if (idx.has_z) {
      idx.Zc.alloc(size_t(n1) * idx.ldZ);
      KATZ_CUDA(cudaMemsetAsync(idx.Zc.p, 0, idx.Zc.bytes(), s));
    }
    // disjoint graphs: packed columns, T_g of every graph from one solve of
    // width (largest separator), scattered back to the block diagonal
    for (int64_t l0 = 0; seg && l0 < width; l0 += cw_max) {
      const int cw = (int)std::min<int64_t>(cw_max, width - l0);
      if (n1 == 0) break;
      KATZ_CUDA(cudaMemsetAsync(E.p, 0, E.bytes(), s));
      packed_identity_kernel<<<blocks_for(n2), 256, 0, s>>>(E.p, ldc, n2, sg_d.p, gsep_d.p,
                                                            (int)l0, cw);
      KATZ_CHECK_LAUNCH();
      KATZ_CUDA(cudaMemsetAsync(U.p, 0, U.bytes(), s));
      spmm<double>(idx.W12.view(), idx.W12.heavy.p, idx.W12.n_heavy, beta, E.p, ldc, 0.0, nullptr,
                   ldc, U.p, ldc, cw, nullptr, 0, nullptr, s);
      const int st = m11_solve<double>(idx, U.p, V.p, cw, ldc, 1e-14, 5000, nullptr, s);
      KATZ_REQUIRE(st != KATZ_ENOTSPD, KATZ_ENOTSPD, "M11 is not positive definite");
      spmm<double>(idx.W21.view(), idx.W21.heavy.p, idx.W21.n_heavy, beta, V.p, ldc, 0.0, nullptr,
                   ldc, E.p, ldc, cw, nullptr, 0, nullptr, s);
      seg_scatter_T(idx.sb, E.p, ldc, n2, (int)l0, cw, T.p, s);
    }
    for (int64_t j0 = 0; !seg && !idx.s_implicit && j0 < n2; j0 += cw_max) {
      const int cw = (int)std::min<int64_t>(cw_max, n2 - j0);
      if (n1 == 0) break;
      KATZ_CUDA(cudaMemsetAsync(E.p, 0, E.bytes(), s));
      identity_cols_kernel<<<1, 256, 0, s>>>(E.p, ldc, n2, j0, cw);
      KATZ_CHECK_LAUNCH();
      KATZ_CUDA(cudaMemsetAsync(U.p, 0, U.bytes(), s));
      spmm<double>(idx.W12.view(), idx.W12.heavy.p, idx.W12.n_heavy, beta, E.p, ldc, 0.0, nullptr,
                   ldc, U.p, ldc, cw, nullptr, 0, nullptr, s);
      const int st = m11_solve<double>(idx, U.p, V.p, cw, ldc, 1e-14, 5000, nullptr, s);
      KATZ_REQUIRE(st != KATZ_ENOTSPD, KATZ_ENOTSPD, "M11 is not positive definite");
      if (idx.has_h)
        split_tf32<double>(V.p, ldc, n1, cw, idx.Hh.p + j0, idx.Hl.p + j0, idx.ldH, s);
      if (idx.has_z) {
        cols_to_f32_kernel<<<(unsigned)std::min<int64_t>(ceil_div(n1 * cw, 256), 8192), 256, 0,
                             s>>>(V.p, ldc, n1, cw, idx.Zc.p, idx.ldZ, j0);
        KATZ_CHECK_LAUNCH();
      }
      spmm<double>(idx.W21.view(), idx.W21.heavy.p, idx.W21.n_heavy, beta, V.p, ldc, 0.0, nullptr,
                   ldc, T.p + j0, ld2, cw, nullptr, 0, nullptr, s);
    }
  }
  if (seg) {
    // --- per graph: M22_g, S_g = M22_g - T_g, M22_g^{-1}, then Lanczos on
    // each graph's block at once
    DBuf<double> M22b(size_t(std::max<int64_t>(idx.sb.nmat, 1)));
    KATZ_REQUIRE(seg_build_blocks(idx.sb, W22d.view(), beta, T.p, M22b.p, s), KATZ_ENOTSPD,
                 "a graph's M22 block is not positive definite");
    idx.sigma.clear();
    if (idx.rank > 0) {
      int rk = 0;
      std::vector<int> rkg;
      std::vector<double> Wh = seg_lanczos(idx, *seg, gsep_h, sg_d.p, gsep_d.p, T.p, M22b.p, 0,
                                           o.seed, o.lanczos_steps, &rk, &rkg, s);
      idx.seg_rank = rkg;
      if (rk > 0) store_seg_basis(idx, Wh, rkg, s);
      else idx.rank = 0;
    }
    return;
  }
  // --- M22 (dense), S = M22 - T, M22^{-1}
  DBuf<double> M22(size_t(n2) * ld2);
  KATZ_CUDA(cudaMemsetAsync(M22.p, 0, M22.bytes(), s));
  dense_from_csr_kernel<<<(unsigned)std::min<int64_t>(n2, 65535), 128, 0, s>>>(W22d.view(), beta,
                                                                               M22.p, ld2);
  KATZ_CHECK_LAUNCH();
  if (!idx.s_implicit) {
    idx.S64.alloc(size_t(n2) * ld2);
    sub_kernel<<<blocks_for(n2 * ld2), 256, 0, s>>>(M22.p, T.p, idx.S64.p, n2 * ld2);
    KATZ_CHECK_LAUNCH();
  }
  idx.M22inv64.alloc(size_t(n2) * ld2);
  KATZ_CUDA(cudaMemcpyAsync(idx.M22inv64.p, M22.p, M22.bytes(), cudaMemcpyDeviceToDevice, s));
  {
    DBuf<double> gws(size_t(n2) * 64 * 2 + 64 * 64);
    KATZ_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    spd_inverse_inplace(idx.M22inv64.p, n2, ld2, gws.p, flag.p, s);
    KATZ_CUDA(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    KATZ_REQUIRE(hflag == 0, KATZ_ENOTSPD, "M22 is not positive definite");
  }
  // separators large enough for the dense n2 x n2 x b products to dominate
  // keep S and M22^{-1} as TF32 parts for the tensor cores (their ~2^-22
  // rounding in S P costs the PCG about one iteration on hard problems,
  // which only pays when the products are a large share of the solve)
  idx.dense_tc = !seg && n2 >= 4096;
  if (idx.dense_tc) {
    for (auto* d : {&idx.Mh, &idx.Ml}) d->alloc(size_t(n2) * ld2);
    split_tf32<double>(idx.M22inv64.p, ld2, n2, int(n2), idx.Mh.p, idx.Ml.p, ld2, s);
    if (!idx.s_implicit) {
      for (auto* d : {&idx.Sh, &idx.Sl}) d->alloc(size_t(n2) * ld2);
      split_tf32<double>(idx.S64.p, ld2, n2, int(n2), idx.Sh.p, idx.Sl.p, ld2, s);
    }
  }
  idx.M22inv32.alloc(size_t(n2) * ld2);
  to_f32_kernel<<<blocks_for(n2 * ld2), 256, 0, s>>>(idx.M22inv64.p, idx.M22inv32.p, n2 * ld2);
  KATZ_CHECK_LAUNCH();
  if (!idx.s_implicit) {
    idx.S32.alloc(size_t(n2) * ld2);
    to_f32_kernel<<<blocks_for(n2 * ld2), 256, 0, s>>>(idx.S64.p, idx.S32.p, n2 * ld2);
    KATZ_CHECK_LAUNCH();
  }

  // --- Lanczos for the top-r eigenpairs of R = L^{-1} T L^{-T}.  R is
  // similar to A = M22^{-1} T, which is self-adjoint in <x,y> = x^T M22 y;
  // Lanczos on A in that inner product gives R's eigenvalues and, for each
  // Ritz vector u of R, w = L^{-T} u directly (w^T M22 w = 1).  L itself is
  // never formed.  Full reorthogonalisation (two Gram-Schmidt passes).
  idx.sigma.clear();
  if (idx.rank > 0) {
    const int r = (int)std::min<int64_t>(idx.rank, n2);
    int m = o.lanczos_steps > 0 ? o.lanczos_steps : std::max(2 * r, r + 20);
    m = (int)std::min<int64_t>(std::max(m, r), n2);
    // capacity for extending past m until the top-r Ritz residuals converge
    const int cap = (int)std::min<int64_t>(n2, std::max(4 * m, m + 200));
    const int64_t ldq = cap + 1;
    DBuf<double> Q(size_t(n2) * ldq), t(n2), wv(n2), u(n2), cvec(ldq), sc(2);
    std::vector<double> v0 = splitmix64_uniform(o.seed, n2);
    KATZ_CUDA(cudaMemcpyAsync(wv.p, v0.data(), 8 * n2, cudaMemcpyHostToDevice, s));
    auto mdot = [&](const double* x, const double* y) {  // x^T M22 y
      gemm<double>(false, n2, 1, n2, 1.0, M22.p, ld2, y, 1, 0.0, u.p, 1, s);
      gemm<double>(true, 1, 1, n2, 1.0, x, 1, u.p, 1, 0.0, sc.p, 1, s);
      return dget(sc.p, s);
    };
    double nrm = std::sqrt(mdot(wv.p, wv.p));
    copy2d<double>(wv.p, 1, Q.p, ldq, n2, 1, 1.0 / nrm, s);
    std::vector<double> al, be, ev, Y;
    int check = m;
    // implicit S: T q = beta^2 W21 M11^{-1} (W12 q) by one FP64 M11 solve
    DBuf<double> q2, u2, v2;
    if (idx.s_implicit) {
      q2.alloc(size_t(n2) * 2);
      u2.alloc(size_t(std::max<int64_t>(n1, 1)) * 2);
      v2.alloc(size_t(std::max<int64_t>(n1, 1)) * 2);
      KATZ_CUDA(cudaMemsetAsync(q2.p, 0, q2.bytes(), s));
    }
    for (int j = 0; j < cap; ++j) {
      // t = T q_j ; w = M22^{-1} t
      if (!idx.s_implicit) {
        gemm<double>(false, n2, 1, n2, 1.0, T.p, ld2, Q.p + j, ldq, 0.0, t.p, 1, s);
      } else if (n1 == 0) {
        KATZ_CUDA(cudaMemsetAsync(t.p, 0, t.bytes(), s));
      } else {
        copy2d<double>(Q.p + j, ldq, q2.p, 2, n2, 1, 1.0, s);
        spmm<double>(idx.W12.view(), idx.W12.heavy.p, idx.W12.n_heavy, beta, q2.p, 2, 0.0,
                     nullptr, 2, u2.p, 2, 1, nullptr, 0, nullptr, s);
        const int st = m11_solve<double>(idx, u2.p, v2.p, 1, 2, 1e-14, 5000, nullptr, s);
        KATZ_REQUIRE(st != KATZ_ENOTSPD, KATZ_ENOTSPD, "M11 is not positive definite");
        spmm<double>(idx.W21.view(), idx.W21.heavy.p, idx.W21.n_heavy, beta, v2.p, 2, 0.0,
                     nullptr, 2, q2.p, 2, 1, nullptr, 0, nullptr, s);
        copy2d<double>(q2.p, 2, t.p, 1, n2, 1, 1.0, s);
      }
      gemm<double>(false, n2, 1, n2, 1.0, idx.M22inv64.p, ld2, t.p, 1, 0.0, wv.p, 1, s);
      gemm<double>(true, 1, 1, n2, 1.0, Q.p + j, ldq, t.p, 1, 0.0, sc.p, 1, s);
      al.push_back(dget(sc.p, s));
      for (int pass = 0; pass < 2; ++pass) {
        // w -= Q c, c = Q^T M22 w   (columns 0..j)
        gemm<double>(false, n2, 1, n2, 1.0, M22.p, ld2, wv.p, 1, 0.0, u.p, 1, s);
        gemm<double>(true, j + 1, 1, n2, 1.0, Q.p, ldq, u.p, 1, 0.0, cvec.p, 1, s);
        gemm<double>(false, n2, 1, j + 1, -1.0, Q.p, ldq, cvec.p, 1, 1.0, wv.p, 1, s);
      }
      const double bj = std::sqrt(std::max(0.0, mdot(wv.p, wv.p)));
      const int kk = j + 1;
      if (bj <= 1e-14 * std::max(1.0, std::fabs(al.back()))) break;  // invariant subspace
      if (kk >= check || kk == cap) {
        // residual estimates beta_k |y_k,i| of the top-r Ritz pairs
        ev = al;
        std::vector<double> sub(be);
        tridiag_ql(ev, sub, Y, kk);
        std::vector<int> o2(kk);
        std::iota(o2.begin(), o2.end(), 0);
        std::sort(o2.begin(), o2.end(), [&](int a, int b) { return ev[a] > ev[b]; });
        bool ok = true;
        for (int c = 0; c < std::min(r, kk); ++c)
          ok &= bj * std::fabs(Y[size_t(kk - 1) * kk + o2[c]]) <=
                1e-8 * std::max(1.0, std::fabs(ev[o2[c]]));
        if (ok || kk == cap) break;
        check = kk + std::max(10, kk / 2);
      }
      be.push_back(bj);
      copy2d<double>(wv.p, 1, Q.p + j + 1, ldq, n2, 1, 1.0 / bj, s);
    }
    const int k = (int)al.size();
    ev = al;
    {
      std::vector<double> sub(be.begin(), be.begin() + std::max(0, k - 1));
      tridiag_ql(ev, sub, Y, k);
    }
    std::vector<int> ordr(k);
    std::iota(ordr.begin(), ordr.end(), 0);
    std::sort(ordr.begin(), ordr.end(), [&](int a, int b) { return ev[a] > ev[b]; });
    const int rk = std::min(r, k);
    idx.rank = rk;
    std::vector<double> Ysel(size_t(k) * rk);
    for (int c = 0; c < rk; ++c) {
      idx.sigma.push_back(ev[ordr[c]]);
      for (int i = 0; i < k; ++i) Ysel[size_t(i) * rk + c] = Y[size_t(i) * k + ordr[c]];
    }
    idx.lanczos_steps = k;
    DBuf<double> Yd(Ysel.size()), Wd(size_t(n2) * rk);
    KATZ_CUDA(cudaMemcpyAsync(Yd.p, Ysel.data(), 8 * Ysel.size(), cudaMemcpyHostToDevice, s));
    gemm<double>(false, n2, rk, k, 1.0, Q.p, ldq, Yd.p, rk, 0.0, Wd.p, rk, s);
    std::vector<double> Wh(size_t(n2) * rk);
    KATZ_CUDA(cudaMemcpyAsync(Wh.data(), Wd.p, 8 * Wh.size(), cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    store_basis(idx, Wh, rk, s);
  }
}

}  // namespace katz
