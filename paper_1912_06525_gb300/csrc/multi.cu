// Many independent graphs of uneven size answered together.
//
// The graphs are stored as one block-diagonal CSR (graph g owns rows
// seg_ptr[g] .. seg_ptr[g+1]) with each graph's own damping beta_g applied
// per row, so M = I - diag(beta_seg(i)) W is block diagonal and one
// multi-RHS solve with qpg columns answers qpg queries of EVERY graph at
// once: column j of graph g's rows is the Katz vector of that graph's j-th
// query (Eq. 3 per graph).  All CG scalars are kept per (graph, column), so
// each graph converges on its own; every kernel launch covers all graphs
// (load balance comes from the row-level parallelism, whatever the graph
// sizes).  The CG iteration sequence is captured once into a CUDA graph
// and replayed; each replay runs kItersPerGraph iterations; the host reads
// the count of unconverged (graph, column) pairs between replays.  FP64-
// class accuracy comes from float-float residual refinement, as for a
// single graph.
#include <chrono>
#include <cmath>
#include <numeric>
#include <algorithm>

#include "index.h"

namespace katz {

namespace {

constexpr int kItersPerGraph = 8;
constexpr int kRowsPerCta = 256;

struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

template <int WT>
__device__ __forceinline__ float wgt(const void* val, int64_t k) {
  if constexpr (WT == KATZ_UNIT) return 1.f;
  else if constexpr (WT == KATZ_F32) return static_cast<const float*>(val)[k];
  else return __bfloat162float(static_cast<const __nv_bfloat16*>(val)[k]);
}

// Y = X - beta_seg(i) * (W X)_i   (thread per (row, column); small b)
template <int WT>
__global__ void seg_spmm_kernel(Csr A, const int32_t* __restrict__ seg, const float* __restrict__ bseg,
                                const float* __restrict__ X, float* __restrict__ Y, int64_t ld,
                                int b) {
  const int64_t total = A.nrows * b;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / b;
    const int c = int(e - i * b);
    float acc = 0.f;
    for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k)
      acc += wgt<WT>(A.val, k) * __ldg(X + int64_t(A.col[k]) * ld + c);
    Y[i * ld + c] = X[i * ld + c] - bseg[seg[i]] * acc;
  }
}

// Contiguous row chunk per CTA; thread = (row lane, column).  Per-(segment,
// column) partial sums are flushed to FP64 atomics when the segment
// changes (rare: graphs are contiguous), so reductions stay cheap.
struct SegAcc {
  double part = 0;
  int seg = -1;
};
__device__ __forceinline__ void seg_flush(SegAcc& a, double* out, int ldst, int c) {
  if (a.seg >= 0 && a.part != 0.0) atomicAdd(out + int64_t(a.seg) * ldst + c, a.part);
  a.part = 0;
}

__global__ void seg_coldot_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                  int64_t ld, int64_t len, int b, const int32_t* __restrict__ seg,
                                  double* out, int ldst) {
  const int c = threadIdx.x % b;
  const int lanes = blockDim.x / b;
  const int rl = threadIdx.x / b;
  if (rl >= lanes) return;
  const int64_t r0 = int64_t(blockIdx.x) * kRowsPerCta;
  const int64_t r1 = min(len, r0 + kRowsPerCta);
  SegAcc a;
  for (int64_t i = r0 + rl; i < r1; i += lanes) {
    const int sg = seg[i];
    if (sg != a.seg) {
      seg_flush(a, out, ldst, c);
      a.seg = sg;
    }
    a.part += double(A[i * ld + c] * B[i * ld + c]);
  }
  seg_flush(a, out, ldst, c);
}

// X += a P, R -= a Q with a = rz/pq of (segment, column); rr += ||R||^2.
__global__ void seg_update_xr_kernel(float* __restrict__ X, const float* __restrict__ P,
                                     float* __restrict__ R, const float* __restrict__ Q, int64_t ld,
                                     int64_t len, int b, const int32_t* __restrict__ seg,
                                     ColState st, int ldst) {
  const int c = threadIdx.x % b;
  const int lanes = blockDim.x / b;
  const int rl = threadIdx.x / b;
  if (rl >= lanes) return;
  const int64_t r0 = int64_t(blockIdx.x) * kRowsPerCta;
  const int64_t r1 = min(len, r0 + kRowsPerCta);
  SegAcc a;
  float alpha = 0.f;
  bool act = false;
  for (int64_t i = r0 + rl; i < r1; i += lanes) {
    const int sg = seg[i];
    if (sg != a.seg) {
      seg_flush(a, st.rz_new, ldst, c);
      a.seg = sg;
      const int64_t k = int64_t(sg) * ldst + c;
      act = st.active[k] != 0;
      alpha = act ? float(st.rz[k] / st.pq[k]) : 0.f;
    }
    if (!act) continue;
    const int64_t e = i * ld + c;
    X[e] += alpha * P[e];
    const float r = R[e] - alpha * Q[e];
    R[e] = r;
    a.part += double(r) * double(r);
  }
  seg_flush(a, st.rz_new, ldst, c);
}

__global__ void seg_update_p_kernel(float* __restrict__ P, const float* __restrict__ R, int64_t ld,
                                    int64_t len, int b, const int32_t* __restrict__ seg, ColState st,
                                    int ldst) {
  const int64_t total = len * b;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / b;
    const int c = int(e - i * b);
    const int64_t k = int64_t(seg[i]) * ldst + c;
    if (!st.active[k]) continue;
    const float be = float(st.rz_new[k] / st.rz[k]);
    P[i * ld + c] = R[i * ld + c] + be * P[i * ld + c];
  }
}

// (segment, column) state updates; the same rules as the single-graph CG.
__global__ void seg_state_kernel(ColState st, int total, int phase, int* n_active) {
  // phase 0: init from rz; 1: check pq; 2: advance; 3: rotate
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int local = 0;
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    if (phase == 0) {
      st.active[k] = st.rz[k] > st.thr2[k];
      st.iters[k] = 0;
      st.pq[k] = 0;
      st.rz_new[k] = 0;
      local += st.active[k];
    } else if (phase == 1) {
      if (st.active[k] && !(st.pq[k] > 0.0)) {
        atomicOr(st.flags, 1);
        st.active[k] = 0;
      }
    } else if (phase == 2) {
      if (st.active[k]) {
        st.iters[k] += 1;
        st.active[k] = st.rz_new[k] > st.thr2[k];
        local += st.active[k];
      }
    } else {
      st.rz[k] = st.rz_new[k];
      st.rz_new[k] = 0;
      st.pq[k] = 0;
    }
  }
  if (phase == 0 || phase == 2) {
    atomicAdd(&cnt, local);
    __syncthreads();
    if (threadIdx.x == 0) *n_active = cnt;
  }
}

// RHS: column j of graph g holds beta_g W_g e_{q_gj} in graph g's rows.
template <int WT>
__global__ void seg_rhs_kernel(Csr A, const int64_t* seg_ptr, const float* bseg, const int32_t* q,
                               int qpg, float* B, int64_t ld, double* bn2, double* bmx,
                               const double* bseg64) {
  const int g = blockIdx.x / qpg, j = blockIdx.x % qpg;
  const int64_t row = seg_ptr[g] + q[blockIdx.x];
  double s = 0, m = 0;
  for (int64_t k = A.rowptr[row] + threadIdx.x; k < A.rowptr[row + 1]; k += blockDim.x) {
    const float w = wgt<WT>(A.val, k);
    if (B) B[int64_t(A.col[k]) * ld + j] = bseg[g] * w;
    const double v = bseg64[g] * double(w);
    s += v * v;
    m = fmax(m, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0 && bn2) {
    atomicAdd(bn2 + blockIdx.x, s);
    atomicMax(reinterpret_cast<unsigned long long*>(bmx) + blockIdx.x,
              (unsigned long long)__double_as_longlong(m));
  }
}

// R = B - M K in float-float: thread per (row, column); the RHS term of the
// row's own queries is added before rounding.
template <int WT>
__global__ void seg_ff_residual_kernel(Csr A, const int32_t* __restrict__ seg,
                                       const int64_t* __restrict__ seg_ptr,
                                       const float* __restrict__ bh_seg,
                                       const float* __restrict__ bl_seg, const int32_t* q, int qpg,
                                       const float* __restrict__ Kh, const float* __restrict__ Kl,
                                       int64_t ld, float* __restrict__ R) {
  const int64_t total = A.nrows * qpg;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / qpg;
    const int c = int(e - i * qpg);
    const int g = seg[i];
    const int64_t qrow = seg_ptr[g] + q[int64_t(g) * qpg + c];
    FF acc = {0.f, 0.f};
    float wq = 0.f;  // W[i, q] (the RHS entry is beta_g * wq)
    for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
      const int64_t j = A.col[k];
      const float w = wgt<WT>(A.val, k);
      if (j == qrow) wq = w;
      const float xh = Kh[j * ld + c], xl = Kl[j * ld + c];
      const float p = w * xh;
      const float pe = __fmaf_rn(w, xh, -p);
      const FF s = two_sum(acc.hi, p);
      acc.hi = s.hi;
      acc.lo += s.lo + pe + w * xl;
    }
    acc = fast_two_sum(acc.hi, acc.lo);
    const float beh = bh_seg[g], bel = bl_seg[g];
    // beta * (acc + wq) - k  (wq enters the same product: b_i = beta * W[i,q])
    const FF t = two_sum(acc.hi, wq);
    const float ah = t.hi, al = t.lo + acc.lo;
    const float ph = beh * ah;
    const float pe = __fmaf_rn(beh, ah, -ph) + beh * al + bel * ah;
    const FF s1 = two_sum(ph, -Kh[i * ld + c]);
    R[i * ld + c] = s1.hi + (s1.lo + pe - Kl[i * ld + c]);
  }
}

__global__ void seg_ff_add_kernel(float* Kh, float* Kl, const float* D, int64_t total) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const FF s = two_sum(Kh[e], D[e]);
    const FF t = fast_two_sum(s.hi, s.lo + Kl[e]);
    Kh[e] = t.hi;
    Kl[e] = t.lo;
  }
}

// conv / inner thresholds per (segment, column) and masking of converged
// (segment, column) entries of R.
__global__ void seg_inner_kernel(const double* rr, const double* thr2, double tau, int total,
                                 int* conv, double* thr2_in, int* n_open) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int local = 0;
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    const int cv = rr[k] <= thr2[k];
    conv[k] = cv;
    thr2_in[k] = cv ? 0.0 : fmax(tau * tau * rr[k], 0.09 * thr2[k]);
    local += !cv;
  }
  atomicAdd(&cnt, local);
  __syncthreads();
  if (threadIdx.x == 0) *n_open = cnt;
}

__global__ void seg_mask_kernel(float* R, int64_t ld, int64_t len, int b, const int32_t* seg,
                                const int* conv, int ldst) {
  const int64_t total = len * ld;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / ld;
    const int c = int(e - i * ld);
    if (c >= b || conv[int64_t(seg[i]) * ldst + c]) R[e] = 0.f;
  }
}

__global__ void seg_out_kernel(const float* Kh, const float* Kl, int64_t ld, int64_t n, int b,
                               void* out, int out_dt, int64_t ldk) {
  const int64_t total = n * b;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / b, c = e - i * b;
    if (out_dt == KATZ_F64)
      static_cast<double*>(out)[i * ldk + c] = double(Kh[i * ld + c]) + double(Kl[i * ld + c]);
    else
      static_cast<float*>(out)[i * ldk + c] = Kh[i * ld + c] + Kl[i * ld + c];
  }
}

// Y[pos[i]] = X[i] (to index order) or Y[i] = X[pos[i]] (back), ld columns.
__global__ void permute_rows_kernel(const float* __restrict__ X, float* __restrict__ Y,
                                    const int32_t* __restrict__ pos, int64_t n, int64_t ld,
                                    bool to_index) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n * ld;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / ld, c = e - i * ld;
    if (to_index)
      Y[int64_t(pos[i]) * ld + c] = X[e];
    else
      Y[e] = X[int64_t(pos[i]) * ld + c];
  }
}

unsigned flat(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), int64_t(num_sms()) * 16));
}

}  // namespace

void multi_build(katz_multi& m, const std::vector<HostCsr>& Ws, const double* betas, int vdt,
                 cudaStream_t s) {
  KATZ_REQUIRE(vdt == KATZ_UNIT || vdt == KATZ_F32 || vdt == KATZ_BF16, KATZ_EINVAL,
               "multi-graph values must be UNIT, F32 or BF16 (exact in FP32)");
  m.g = (int32_t)Ws.size();
  m.vdt = vdt;
  HostCsr U;
  m.seg_ptr_h.assign(1, 0);
  for (auto& w : Ws) m.seg_ptr_h.push_back(m.seg_ptr_h.back() + w.nrows);
  m.n = m.seg_ptr_h.back();
  U.nrows = U.ncols = m.n;
  U.rowptr.assign(1, 0);
  std::vector<int32_t> segv(m.n);
  for (int32_t gi = 0; gi < m.g; ++gi) {
    const HostCsr& w = Ws[gi];
    const int64_t off = m.seg_ptr_h[gi];
    for (int64_t i = 0; i < w.nrows; ++i) {
      for (int64_t k = w.rowptr[i]; k < w.rowptr[i + 1]; ++k) {
        U.col.push_back((int32_t)(w.col[k] + off));
        if (!w.val.empty() || vdt != KATZ_UNIT) U.val.push_back(w.val.empty() ? 1.0 : w.val[k]);
      }
      U.rowptr.push_back((int64_t)U.col.size());
      segv[off + i] = gi;
    }
  }
  m.nnz = U.nnz();
  upload_csr(U, vdt, m.W.csr, s);
  m.W.heavy.alloc(1);
  m.deg_h.resize(m.n);
  for (int64_t i = 0; i < m.n; ++i) m.deg_h[i] = (int32_t)(U.rowptr[i + 1] - U.rowptr[i]);
  // per-graph lambda_max (FP64 Lanczos) and the damping bound
  m.beta_h.assign(betas, betas + m.g);
  m.lambda_h.resize(m.g);
  for (int32_t gi = 0; gi < m.g; ++gi) {
    GraphPart one;
    upload_csr(Ws[gi], vdt, one.csr, s);
    one.heavy.alloc(1);
    // the rigorous upper bound (Collatz-Wielandt) certifies M_g SPD and makes
    // the per-graph error-bound stopping rule sound
    double up = 0;
    const double ritz = lambda_max_gpu(one, Ws[gi].nrows, 48, m.ws, s, 0, nullptr, &up);
    m.lambda_h[gi] = up;
    KATZ_REQUIRE(betas[gi] > 0 && betas[gi] * ritz < 1.0, KATZ_ENOTSPD,
                 "graph " + std::to_string(gi) + ": beta * lambda_max >= 1");
    KATZ_REQUIRE(betas[gi] * up < 1.0, KATZ_ENOTSPD,
                 "graph " + std::to_string(gi) +
                     ": beta * (upper bound on lambda_max) >= 1, M cannot be certified SPD");
  }
  m.ws.clear();
  std::vector<float> bh(m.g), bl(m.g);
  for (int32_t gi = 0; gi < m.g; ++gi) {
    bh[gi] = float(betas[gi]);
    bl[gi] = float(betas[gi] - double(bh[gi]));
  }
  m.seg_ptr.alloc(m.g + 1);
  m.seg.alloc(std::max<int64_t>(m.n, 1));
  m.bseg_hi.alloc(m.g);
  m.bseg_lo.alloc(m.g);
  m.bseg64.alloc(m.g);
  KATZ_CUDA(cudaMemcpyAsync(m.seg_ptr.p, m.seg_ptr_h.data(), 8 * (m.g + 1), cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(m.seg.p, segv.data(), 4 * m.n, cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(m.bseg_hi.p, bh.data(), 4 * m.g, cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(m.bseg_lo.p, bl.data(), 4 * m.g, cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(m.bseg64.p, betas, 8 * m.g, cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  KATZ_CUDA(cudaStreamCreateWithFlags(&m.cap_stream, cudaStreamNonBlocking));
}

void multi_build_lrc(katz_multi& m, const std::vector<HostCsr>& Ws, const double* betas,
                     const katz_build_opts& o, cudaStream_t s) {
  KATZ_REQUIRE(o.value_dtype == KATZ_UNIT || o.value_dtype == KATZ_F32 ||
                   o.value_dtype == KATZ_BF16, KATZ_EINVAL,
               "multi-graph values must be UNIT, F32 or BF16 (exact in FP32)");
  multi_build(m, Ws, betas, o.value_dtype, s);
  const int G = m.g;
  // the union with each graph's damping folded into its weights: M = I - W~,
  // W~ = beta_g W_g on graph g's block (beta = 1 for the index)
  HostCsr U;
  U.nrows = U.ncols = m.n;
  U.rowptr.assign(1, 0);
  SegSpec seg;
  seg.G = G;
  seg.node_graph.resize(m.n);
  int64_t n_min = INT64_MAX, n_max = 0;
  for (int g = 0; g < G; ++g) {
    const HostCsr& w = Ws[g];
    const int64_t off = m.seg_ptr_h[g];
    n_min = std::min(n_min, w.nrows);
    n_max = std::max(n_max, w.nrows);
    for (int64_t i = 0; i < w.nrows; ++i) {
      for (int64_t k = w.rowptr[i]; k < w.rowptr[i + 1]; ++k) {
        U.col.push_back((int32_t)(w.col[k] + off));
        U.val.push_back(betas[g] * (w.val.empty() ? 1.0 : w.val[k]));
      }
      U.rowptr.push_back((int64_t)U.col.size());
      seg.node_graph[off + i] = g;
    }
  }
  // hubs: the largest degrees of each graph (ties: smaller id): a share of
  // the separator budget in proportion to the graph's size, and at least
  // twice the graph's rank (the rank r_g is log-scaled with the graph's
  // size from r/4 to r), at most kSegBlockMax (the block storage's limit)
  const int64_t budget =
      o.n_hubs > 0 ? o.n_hubs : std::max<int64_t>(G, std::min<int64_t>(8192, m.n / 1000));
  const int r_hi = o.rank > 0 ? o.rank : 32, r_lo = std::max(1, r_hi / 4);
  KATZ_REQUIRE(r_hi <= kSegBlockMax / 4, KATZ_EINVAL, "per-graph rank must be <= 64");
  seg.ranks.resize(G);
  for (int g = 0; g < G; ++g) {
    const HostCsr& w = Ws[g];
    const int64_t ng = w.nrows;
    const double t = n_max > n_min ? std::log(double(ng) / n_min) / std::log(double(n_max) / n_min)
                                   : 1.0;
    const int64_t r_target = std::llround(r_lo + (r_hi - r_lo) * t);
    int64_t h = std::max<int64_t>(1, (int64_t)std::llround(double(budget) * ng / double(m.n)));
    h = std::max<int64_t>(h, 2 * r_target);
    h = std::min<int64_t>({h, kSegBlockMax, std::max<int64_t>(0, ng - 1)});
    std::vector<int64_t> ord(ng);
    std::iota(ord.begin(), ord.end(), 0);
    auto deg = [&](int64_t v) { return w.rowptr[v + 1] - w.rowptr[v]; };
    std::partial_sort(ord.begin(), ord.begin() + h, ord.end(), [&](int64_t a, int64_t b) {
      return deg(a) != deg(b) ? deg(a) > deg(b) : a < b;
    });
    for (int64_t i = 0; i < h; ++i) seg.hubs.push_back(m.seg_ptr_h[g] + ord[i]);
    seg.ranks[g] = (int)std::min<int64_t>(h, r_target);
  }
  katz_build_opts bo = o;
  bo.value_dtype = KATZ_F32;
  bo.build_lrc = 1;
  bo.rank = r_hi;
  bo.n_hubs = 0;
  bo.coupling_gemm = -1;
  bo.n2_max = (int32_t)std::max<int64_t>(o.n2_max > 0 ? o.n2_max : 16384,
                                         (int64_t)seg.hubs.size());
  m.lrc.reset(new katz_index());
  build_index(*m.lrc, U, 1.0, bo, s, &seg);
}

namespace {

template <int WT>
void launch_seg_spmm(katz_multi& m, const float* X, float* Y, int64_t ld, int b, cudaStream_t s) {
  seg_spmm_kernel<WT><<<flat(m.n * b), 256, 0, s>>>(m.W.view(), m.seg.p, m.bseg_hi.p, X, Y, ld, b);
  KATZ_CHECK_LAUNCH();
}

void seg_spmm(katz_multi& m, const float* X, float* Y, int64_t ld, int b, cudaStream_t s) {
  if (m.vdt == KATZ_UNIT) launch_seg_spmm<KATZ_UNIT>(m, X, Y, ld, b, s);
  else if (m.vdt == KATZ_F32) launch_seg_spmm<KATZ_F32>(m, X, Y, ld, b, s);
  else launch_seg_spmm<KATZ_BF16>(m, X, Y, ld, b, s);
}

int read1(const int* d, cudaStream_t s) {
  int h = 0;
  KATZ_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  return h;
}

// One CG iteration on all graphs (no host synchronisation inside).
void seg_cg_iteration(katz_multi& m, float* X, float* R, float* P, float* Q, int64_t ld, int b,
                      const ColState& st, int total, cudaStream_t s) {
  const unsigned chunks = (unsigned)ceil_div(m.n, kRowsPerCta);
  seg_spmm(m, P, Q, ld, b, s);
  seg_coldot_kernel<<<chunks, 256, 0, s>>>(P, Q, ld, m.n, b, m.seg.p, st.pq, b);
  KATZ_CHECK_LAUNCH();
  seg_state_kernel<<<1, 1024, 0, s>>>(st, total, 1, st.n_active);
  KATZ_CHECK_LAUNCH();
  seg_update_xr_kernel<<<chunks, 256, 0, s>>>(X, P, R, Q, ld, m.n, b, m.seg.p, st, b);
  KATZ_CHECK_LAUNCH();
  seg_state_kernel<<<1, 1024, 0, s>>>(st, total, 2, st.n_active);
  KATZ_CHECK_LAUNCH();
  seg_update_p_kernel<<<flat(m.n * b), 256, 0, s>>>(P, R, ld, m.n, b, m.seg.p, st, b);
  KATZ_CHECK_LAUNCH();
  seg_state_kernel<<<1, 1024, 0, s>>>(st, total, 3, st.n_active);
  KATZ_CHECK_LAUNCH();
}

// Segmented CG from zero on B (= R on entry is copied); X out.  Replays a
// captured CUDA graph of kItersPerGraph iterations until no pair is active
// or max_iter is reached.  Returns KATZ_OK / ENOTSPD / ENOCONV.
int seg_cg(katz_multi& m, const float* B, float* X, int64_t ld, int b, const double* thr2,
           int max_iter, int* graph_replays, cudaStream_t s) {
  const int total = m.g * b;
  float* R = m.ws.get<float>("m.R", size_t(m.n) * ld);
  float* P = m.ws.get<float>("m.P", size_t(m.n) * ld);
  float* Q = m.ws.get<float>("m.Q", size_t(m.n) * ld);
  ColState st;
  st.rz = m.ws.get<double>("m.rz", total);
  st.pq = m.ws.get<double>("m.pq", total);
  st.rz_new = m.ws.get<double>("m.rzn", total);
  st.thr2 = m.ws.get<double>("m.thr2", total);
  st.active = m.ws.get<int>("m.act", total);
  st.iters = m.ws.get<int>("m.it", total);
  st.flags = m.ws.get<int>("m.flags", 1);
  st.n_active = m.ws.get<int>("m.nact", 1);
  KATZ_CUDA(cudaMemcpyAsync(st.thr2, thr2, 8 * size_t(total), cudaMemcpyDeviceToDevice, s));
  KATZ_CUDA(cudaMemsetAsync(X, 0, sizeof(float) * m.n * ld, s));
  KATZ_CUDA(cudaMemcpyAsync(R, B, sizeof(float) * m.n * ld, cudaMemcpyDeviceToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(P, B, sizeof(float) * m.n * ld, cudaMemcpyDeviceToDevice, s));
  KATZ_CUDA(cudaMemsetAsync(st.rz, 0, 8 * size_t(total), s));
  KATZ_CUDA(cudaMemsetAsync(st.flags, 0, sizeof(int), s));
  seg_coldot_kernel<<<(unsigned)ceil_div(m.n, kRowsPerCta), 256, 0, s>>>(R, R, ld, m.n, b,
                                                                          m.seg.p, st.rz, b);
  KATZ_CHECK_LAUNCH();
  seg_state_kernel<<<1, 1024, 0, s>>>(st, total, 0, st.n_active);
  KATZ_CHECK_LAUNCH();
  int active = read1(st.n_active, s);
  if (active == 0) return KATZ_OK;
  // capture kItersPerGraph iterations on the index's own stream
  cudaEvent_t ev;
  KATZ_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  KATZ_CUDA(cudaEventRecord(ev, s));
  KATZ_CUDA(cudaStreamWaitEvent(m.cap_stream, ev, 0));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  KATZ_CUDA(cudaStreamBeginCapture(m.cap_stream, cudaStreamCaptureModeThreadLocal));
  try {
    for (int t = 0; t < kItersPerGraph; ++t)
      seg_cg_iteration(m, X, R, P, Q, ld, b, st, total, m.cap_stream);
  } catch (...) {
    cudaStreamEndCapture(m.cap_stream, &graph);
    if (graph) cudaGraphDestroy(graph);
    cudaEventDestroy(ev);
    throw;
  }
  KATZ_CUDA(cudaStreamEndCapture(m.cap_stream, &graph));
  KATZ_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  int done = 0;
  while (active > 0 && done < max_iter) {
    KATZ_CUDA(cudaGraphLaunch(exec, m.cap_stream));
    done += kItersPerGraph;
    if (graph_replays) ++*graph_replays;
    active = read1(st.n_active, m.cap_stream);
  }
  KATZ_CUDA(cudaEventRecord(ev, m.cap_stream));
  KATZ_CUDA(cudaStreamWaitEvent(s, ev, 0));
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  cudaEventDestroy(ev);
  if (read1(st.flags, s) & 1) return KATZ_ENOTSPD;
  return active > 0 ? KATZ_ENOCONV : KATZ_OK;
}

}  // namespace

int multi_query(katz_multi& m, const int32_t* q_dev, int qpg, const katz_query_opts& o, void* Kout,
                int out_dt, int64_t ldk, katz_stats* stats, std::vector<int32_t>& iters,
                std::vector<double>& relres, cudaStream_t s, bool use_lrc) {
  KATZ_REQUIRE(!use_lrc || m.lrc, KATZ_EINVAL,
               "LRC multi-graph queries need an index built by katz_index_build_many");
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  KATZ_REQUIRE(qpg > 0 && qpg <= 64, KATZ_EINVAL, "queries per graph must be in [1, 64]");
  const int b = qpg;
  const int total = m.g * b;
  const int64_t ld = (b + 3) / 4 * 4;
  const int max_iter = o.max_iter > 0 ? o.max_iter : 2000;
  const int max_refine = o.max_refine > 0 ? o.max_refine : 12;
  float* R = m.ws.get<float>("q.R", size_t(m.n) * ld);
  float* D = m.ws.get<float>("q.D", size_t(m.n) * ld);
  float* Kh = m.ws.get<float>("q.Kh", size_t(m.n) * ld);
  float* Kl = m.ws.get<float>("q.Kl", size_t(m.n) * ld);
  double* bn2 = m.ws.get<double>("q.bn2", total);
  double* bmx = m.ws.get<double>("q.bmx", total);
  double* thr2 = m.ws.get<double>("q.thr2", total);
  double* thr2_in = m.ws.get<double>("q.thr2in", total);
  double* rr = m.ws.get<double>("q.rr", total);
  int* conv = m.ws.get<int>("q.conv", total);
  int* nopen = m.ws.get<int>("q.nopen", 1);
  // per-(graph, column) one-minus-c for the error-bound stopping rule
  std::vector<double> omc(total);
  for (int g = 0; g < m.g; ++g)
    for (int c = 0; c < b; ++c) omc[size_t(g) * b + c] = std::max(1e-300, 1.0 - m.beta_h[g] * m.lambda_h[g]);
  double* omc_d = m.ws.get<double>("q.omc", total);
  KATZ_CUDA(cudaMemcpyAsync(omc_d, omc.data(), 8 * size_t(total), cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemsetAsync(R, 0, sizeof(float) * m.n * ld, s));
  KATZ_CUDA(cudaMemsetAsync(bn2, 0, 8 * size_t(total), s));
  KATZ_CUDA(cudaMemsetAsync(bmx, 0, 8 * size_t(total), s));
#define KATZ_RHS(WT)                                                                             \
  seg_rhs_kernel<WT><<<total, 128, 0, s>>>(m.W.view(), m.seg_ptr.p, m.bseg_hi.p, q_dev, b, R, ld, \
                                           bn2, bmx, m.bseg64.p)
  if (m.vdt == KATZ_UNIT) KATZ_RHS(KATZ_UNIT);
  else if (m.vdt == KATZ_F32) KATZ_RHS(KATZ_F32);
  else KATZ_RHS(KATZ_BF16);
#undef KATZ_RHS
  KATZ_CHECK_LAUNCH();
  // thresholds: (tol * base)^2 with base = ||b||_2 or (1 - c) ||b||_inf
  {
    std::vector<double> hn(total), hm(total), th(total);
    KATZ_CUDA(cudaMemcpyAsync(hn.data(), bn2, 8 * size_t(total), cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaMemcpyAsync(hm.data(), bmx, 8 * size_t(total), cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < total; ++k) {
      const double base = o.tol_kind == KATZ_TOL_ERROR_INF ? hm[k] * omc[k] : std::sqrt(hn[k]);
      th[k] = (o.tol * base) * (o.tol * base);
    }
    KATZ_CUDA(cudaMemcpyAsync(thr2, th.data(), 8 * size_t(total), cudaMemcpyHostToDevice, s));
  }
  const double tau = 2e-6;
  seg_inner_kernel<<<1, 1024, 0, s>>>(bn2, thr2, tau, total, conv, thr2_in, nopen);
  KATZ_CHECK_LAUNCH();
  int replays = 0;
  std::vector<int32_t> it_acc(total, 0);
  // the per-graph LRC solve of all graphs at once (the union index), in its
  // index order; its PCG stops each column at relative tolerance tol_rel
  std::vector<int32_t> lit;
  auto lrc_inner = [&](const float* Rn, float* Xn, double tol_rel) {
    katz_index& L = *m.lrc;
    float* Rp = m.ws.get<float>("ml.Rp", size_t(m.n) * ld);
    float* Dp = m.ws.get<float>("ml.Dp", size_t(m.n) * ld);
    permute_rows_kernel<<<flat(m.n * ld), 256, 0, s>>>(Rn, Rp, L.iperm.p, m.n, ld, true);
    KATZ_CHECK_LAUNCH();
    lit.assign(b, 0);
    const int64_t rep0 = L.seg_replays;
    const int st = lrc_solve_f32(L, Rp, Dp, b, ld, tol_rel, max_iter, &lit, s);
    replays += int(L.seg_replays - rep0);
    permute_rows_kernel<<<flat(m.n * ld), 256, 0, s>>>(Dp, Xn, L.iperm.p, m.n, ld, false);
    KATZ_CHECK_LAUNCH();
    // per-(graph, query) PCG iterations of the block-diagonal solve
    const bool per_graph = L.seg_blocked && (int64_t)L.seg_iters.size() == int64_t(m.g) * b;
    for (int g = 0; g < m.g; ++g)
      for (int c = 0; c < b && c < (int)lit.size(); ++c)
        it_acc[size_t(g) * b + c] += per_graph ? L.seg_iters[size_t(g) * b + c] : lit[c];
    return st;
  };
  double omc_min = 1.0;
  for (double v : omc) omc_min = std::min(omc_min, v);
  double tol_first = (o.tol_kind == KATZ_TOL_RESIDUAL) ? o.tol : o.tol * omc_min;
  tol_first = std::max(0.3 * tol_first, tau);
  int status = use_lrc ? lrc_inner(R, Kh, tol_first)
                       : seg_cg(m, R, Kh, ld, b, thr2_in, max_iter, &replays, s);
  auto harvest = [&]() {
    if (use_lrc) return;
    std::vector<int32_t> h(total);
    KATZ_CUDA(cudaMemcpyAsync(h.data(), m.ws.get<int>("m.it", total), 4 * size_t(total),
                              cudaMemcpyDeviceToHost, s));
    KATZ_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < total; ++k) it_acc[k] += h[k];
  };
  harvest();
  KATZ_CUDA(cudaMemsetAsync(Kl, 0, sizeof(float) * m.n * ld, s));
  int refine = 0;
  if (status == KATZ_OK || status == KATZ_ENOCONV) {
    for (;;) {
#define KATZ_RES(WT)                                                                            \
  seg_ff_residual_kernel<WT><<<flat(m.n * b), 256, 0, s>>>(m.W.view(), m.seg.p, m.seg_ptr.p,    \
                                                          m.bseg_hi.p, m.bseg_lo.p, q_dev, b, Kh, \
                                                          Kl, ld, R)
      if (m.vdt == KATZ_UNIT) KATZ_RES(KATZ_UNIT);
      else if (m.vdt == KATZ_F32) KATZ_RES(KATZ_F32);
      else KATZ_RES(KATZ_BF16);
#undef KATZ_RES
      KATZ_CHECK_LAUNCH();
      KATZ_CUDA(cudaMemsetAsync(rr, 0, 8 * size_t(total), s));
      seg_coldot_kernel<<<(unsigned)ceil_div(m.n, kRowsPerCta), 256, 0, s>>>(R, R, ld, m.n, b,
                                                                              m.seg.p, rr, b);
      KATZ_CHECK_LAUNCH();
      seg_inner_kernel<<<1, 1024, 0, s>>>(rr, thr2, tau, total, conv, thr2_in, nopen);
      KATZ_CHECK_LAUNCH();
      ++refine;
      if (read1(nopen, s) == 0) { status = KATZ_OK; break; }
      if (refine > max_refine) { status = KATZ_ENOCONV; break; }
      seg_mask_kernel<<<flat(m.n * ld), 256, 0, s>>>(R, ld, m.n, b, m.seg.p, conv, b);
      KATZ_CHECK_LAUNCH();
      double tol_step = 1.0;
      if (use_lrc) {  // tightest 0.3 * thr / ||r|| over the open pairs
        std::vector<double> hr(total), ht(total);
        KATZ_CUDA(cudaMemcpyAsync(hr.data(), rr, 8 * size_t(total), cudaMemcpyDeviceToHost, s));
        KATZ_CUDA(cudaMemcpyAsync(ht.data(), thr2, 8 * size_t(total), cudaMemcpyDeviceToHost, s));
        KATZ_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < total; ++k)
          if (hr[k] > ht[k] && hr[k] > 0) tol_step = std::min(tol_step, 0.3 * std::sqrt(ht[k] / hr[k]));
        tol_step = std::max(tol_step, tau);
      }
      const int st = use_lrc ? lrc_inner(R, D, tol_step)
                             : seg_cg(m, R, D, ld, b, thr2_in, max_iter, &replays, s);
      harvest();
      if (st == KATZ_ENOTSPD) { status = st; break; }
      seg_ff_add_kernel<<<flat(m.n * ld), 256, 0, s>>>(Kh, Kl, D, m.n * ld);
      KATZ_CHECK_LAUNCH();
    }
    seg_out_kernel<<<flat(m.n * b), 256, 0, s>>>(Kh, Kl, ld, m.n, b, Kout, out_dt, ldk);
    KATZ_CHECK_LAUNCH();
  }
  std::vector<double> hr(total), hb(total);
  KATZ_CUDA(cudaMemcpyAsync(hr.data(), rr, 8 * size_t(total), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaMemcpyAsync(hb.data(), bn2, 8 * size_t(total), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  iters = it_acc;
  relres.resize(total);
  double mr = 0;
  int mx = 0;
  for (int k = 0; k < total; ++k) {
    relres[k] = hb[k] > 0 ? std::sqrt(hr[k] / hb[k]) : std::sqrt(hr[k]);
    mr = std::max(mr, relres[k]);
    mx = std::max(mx, iters[k]);
  }
  if (stats) {
    stats->iters = mx;
    stats->refine_steps = refine;
    stats->max_rel_res = mr;
    stats->ms[0] = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    stats->ms[4] = replays;
  }
  return status;
}

}  // namespace katz
