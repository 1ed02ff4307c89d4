// Dense kernels: SIMT GEMM (FP32/FP64), batched M11 block inverses (Step 4:
// Cholesky of each diagonal block, then the inverse), the small pivot-block
// inverse of the blocked Gauss-Jordan used for M22^{-1}, and top-k of Katz
// columns for link prediction (Section 3.3).
#include "kernels.h"
#include "kernels_dense.h"

namespace katz {

// ---------------------------------------------------------------- GEMM
// 64x64 output tile per CTA, K step 16, 256 threads each owning a 4x4
// micro-tile.  op(A) is A (M x K, row-major) or A^T (A stored K x M);
// op(B) likewise.  lower_only skips tiles strictly above the diagonal.
template <class VT, bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_kernel(int64_t M, int64_t N, int64_t K, VT alpha,
                                                   const VT* __restrict__ A, int64_t lda,
                                                   const VT* __restrict__ B, int64_t ldb, VT beta,
                                                   VT* __restrict__ C, int64_t ldc,
                                                   int lower_only) {
  __shared__ VT As[16][64 + 4];
  __shared__ VT Bs[16][64 + 4];
  const int64_t m0 = int64_t(blockIdx.y) * 64, n0 = int64_t(blockIdx.x) * 64;
  if (lower_only && n0 > m0 + 63) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  VT acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = VT(0);
  for (int64_t k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int mm, kk;
      if (!TA) { mm = e >> 4; kk = e & 15; } else { kk = e >> 6; mm = e & 63; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      VT v = VT(0);
      if (gm < M && gk < K) v = TA ? A[gk * lda + gm] : A[gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int nn, kk;
      if (!TB) { kk = e >> 6; nn = e & 63; } else { nn = e >> 4; kk = e & 15; }
      const int64_t gn = n0 + nn, gk = k0 + kk;
      VT v = VT(0);
      if (gn < N && gk < K) v = TB ? B[gn * ldb + gk] : B[gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      VT a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      VT* cp = C + gm * ldc + gn;
      *cp = beta == VT(0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*cp);
    }
  }
}

// FP32, neither operand transposed: 128 x 64 output tile per CTA, K step
// 16, each of the 256 threads owning an 8 x 4 micro-tile (rows ty + 16 i,
// columns tx + 16 j), so a K step costs 12 shared loads per 32 FMAs.  Every
// output element sums its K products in the same order as gemm_kernel.
__global__ void __launch_bounds__(256) sgemm_nn_kernel(int64_t M, int64_t N, int64_t K,
                                                       float alpha, const float* __restrict__ A,
                                                       int64_t lda, const float* __restrict__ B,
                                                       int64_t ldb, float beta,
                                                       float* __restrict__ C, int64_t ldc) {
  __shared__ float As[16][128 + 4];
  __shared__ float Bs[16][64 + 4];
  const int64_t m0 = int64_t(blockIdx.y) * 128, n0 = int64_t(blockIdx.x) * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int64_t k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = threadIdx.x + 256 * r;
      const int mm = e >> 4, kk = e & 15;
      const int64_t gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? A[gm * lda + gk] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = threadIdx.x + 256 * r;
      const int kk = e >> 6, nn = e & 63;
      const int64_t gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < K) ? B[gk * ldb + gn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[8], bb[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      float* cp = C + gm * ldc + gn;
      *cp = beta == 0.f ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*cp);
    }
  }
}

template <class VT>
void gemm2(bool transA, bool transB, int64_t M, int64_t N, int64_t K, double alpha, const VT* A,
           int64_t lda, const VT* B, int64_t ldb, double beta, VT* C, int64_t ldc, bool lower_only,
           cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((unsigned)ceil_div(N, 64), (unsigned)ceil_div(M, 64));
  const int lo = lower_only ? 1 : 0;
  prof_begin(s);
#define KATZ_G(TA, TB)                                                                   \
  gemm_kernel<VT, TA, TB><<<grid, 256, 0, s>>>(M, N, K, VT(alpha), A, lda, B, ldb, VT(beta), C, \
                                               ldc, lo)
  if constexpr (sizeof(VT) == 4) {
    if (!transA && !transB && !lower_only && M >= 128) {
      const dim3 g2((unsigned)ceil_div(N, 64), (unsigned)ceil_div(M, 128));
      sgemm_nn_kernel<<<g2, 256, 0, s>>>(M, N, K, float(alpha), A, lda, B, ldb, float(beta), C,
                                         ldc);
      KATZ_CHECK_LAUNCH();
      if (profiling())
        prof_end("gemm_f32", 4.0 * (double(M) * K + double(K) * N + double(M) * N), s);
      return;
    }
  }
  if (!transA && !transB) KATZ_G(false, false);
  else if (transA && !transB) KATZ_G(true, false);
  else if (!transA && transB) KATZ_G(false, true);
  else KATZ_G(true, true);
#undef KATZ_G
  KATZ_CHECK_LAUNCH();
  if (profiling())
    prof_end(sizeof(VT) == 4 ? "gemm_f32" : "gemm_f64",
             double(sizeof(VT)) * (double(M) * K + double(K) * N + double(M) * N), s);
}
template void gemm2<float>(bool, bool, int64_t, int64_t, int64_t, double, const float*, int64_t,
                           const float*, int64_t, double, float*, int64_t, bool, cudaStream_t);
template void gemm2<double>(bool, bool, int64_t, int64_t, int64_t, double, const double*, int64_t,
                            const double*, int64_t, double, double*, int64_t, bool, cudaStream_t);

template <class VT>
void gemm(bool transA, int64_t M, int64_t N, int64_t K, double alpha, const VT* A, int64_t lda,
          const VT* B, int64_t ldb, double beta, VT* C, int64_t ldc, cudaStream_t s) {
  gemm2<VT>(transA, false, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, false, s);
}
template void gemm<float>(bool, int64_t, int64_t, int64_t, double, const float*, int64_t,
                          const float*, int64_t, double, float*, int64_t, cudaStream_t);
template void gemm<double>(bool, int64_t, int64_t, int64_t, double, const double*, int64_t,
                           const double*, int64_t, double, double*, int64_t, cudaStream_t);

// ------------------------------------------------- M11 block inverses
// One CTA per diagonal block of M11 = I - beta W11.  The block is assembled
// in shared memory from the (index-ordered) CSR rows, factorised in place
// (M_blk = L1 L1^T, right-looking Cholesky), and its inverse written as
// L1^{-T} L1^{-1}: thread j solves L1 y = e_j then L1^T x = y.  Output is the
// S x S zero-padded inverse in FP64; a non-positive pivot sets *flag.
__global__ void block_inverse_kernel(Csr W, const int64_t* start, const int32_t* size, int S,
                                     double beta, double* inv, int* flag) {
  extern __shared__ double Ls[];  // S x S
  const int64_t blk = blockIdx.x;
  const int64_t a = start[blk];
  const int n = size[blk];
  double* out = inv + blk * int64_t(S) * S;
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
    Ls[e] = 0.0;
    out[e] = 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    Ls[r * S + r] = 1.0;
    for (int64_t k = W.rowptr[a + r]; k < W.rowptr[a + r + 1]; ++k) {
      const int64_t c = int64_t(W.col[k]) - a;
      if (c >= 0 && c < n) {
        double w = 1.0;
        if (W.vdt == KATZ_F64) w = static_cast<const double*>(W.val)[k];
        else if (W.vdt == KATZ_F32) w = static_cast<const float*>(W.val)[k];
        else if (W.vdt == KATZ_BF16) w = __bfloat162float(static_cast<const __nv_bfloat16*>(W.val)[k]);
        Ls[r * S + c] -= beta * w;
      }
    }
  }
  __syncthreads();
  // right-looking Cholesky, lower triangle
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = Ls[j * S + j];
      if (!(d > 0.0)) { bad = 1; Ls[j * S + j] = 1.0; }
      else Ls[j * S + j] = sqrt(d);
    }
    __syncthreads();
    const double dj = Ls[j * S + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) Ls[i * S + j] /= dj;
    __syncthreads();
    const int m = n - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k <= i) Ls[i * S + k] -= Ls[i * S + j] * Ls[k * S + j];
    }
    __syncthreads();
  }
  if (bad && threadIdx.x == 0) atomicOr(flag, 1);
  // inverse: row j of the (symmetric) inverse = solution of M x = e_j
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double* x = out + int64_t(j) * S;  // scratch: row j
    for (int i = 0; i < n; ++i) {  // forward: L y = e_j
      double v = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) v -= Ls[i * S + k] * x[k];
      x[i] = (i < j) ? 0.0 : v / Ls[i * S + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // backward: L^T x = y
      double v = x[i];
      for (int k = i + 1; k < n; ++k) v -= Ls[k * S + i] * x[k];
      x[i] = v / Ls[i * S + i];
    }
  }
}

void block_inverses(const Csr& Wperm, const int64_t* start, const int32_t* size, int64_t count,
                    int S, double beta, double* inv, int* flag, cudaStream_t s) {
  if (count <= 0) return;
  const size_t smem = size_t(S) * S * sizeof(double);
  if (smem > 48 * 1024)
    KATZ_CUDA(cudaFuncSetAttribute(block_inverse_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int threads = S >= 64 ? 256 : 128;
  block_inverse_kernel<<<(unsigned)count, threads, smem, s>>>(Wperm, start, size, S, beta, inv,
                                                              flag);
  KATZ_CHECK_LAUNCH();
}

// ---------------------------------------- pivot-block inverse (Gauss-Jordan)
// In-place inverse of an nb x nb SPD block (nb <= 64) held at P (ld).  Plain
// Gauss-Jordan without pivoting, which is stable for SPD matrices; a
// non-positive pivot sets *flag.
__global__ void small_spd_inverse_kernel(double* P, int64_t ld, int nb, int* flag) {
  __shared__ double A[64][65];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) A[e / nb][e % nb] = P[(e / nb) * ld + e % nb];
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    const double piv = A[k][k];
    if (!(piv > 0.0)) {  // uniform across the CTA: every thread reads the same value
      if (threadIdx.x == 0) bad = 1;
      break;
    }
    const double ip = 1.0 / piv;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      const int i = e / nb, j = e % nb;
      if (i != k && j != k) A[i][j] -= A[i][k] * A[k][j] * ip;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
      if (j != k) {
        A[k][j] *= ip;
        A[j][k] = -A[j][k] * ip;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) A[k][k] = ip;
    __syncthreads();
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) atomicOr(flag, 1);
    return;
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) P[(e / nb) * ld + e % nb] = A[e / nb][e % nb];
}

void small_spd_inverse(double* P, int64_t ld, int nb, int* flag, cudaStream_t s) {
  small_spd_inverse_kernel<<<1, 64, 0, s>>>(P, ld, nb, flag);
  KATZ_CHECK_LAUNCH();
}

// strided sub-matrix copy (rows x cols), optional scale
template <class VT>
__global__ void copy2d_kernel(const VT* X, int64_t ldx, VT* Y, int64_t ldy, int64_t rows,
                              int64_t cols, VT a) {
  const int64_t total = rows * cols;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    Y[i * ldy + j] = a * X[i * ldx + j];
  }
}
template <class VT>
void copy2d(const VT* X, int64_t ldx, VT* Y, int64_t ldy, int64_t rows, int64_t cols, double a,
            cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  int64_t g = std::min<int64_t>(ceil_div(rows * cols, 256), int64_t(num_sms()) * 16);
  copy2d_kernel<VT><<<(unsigned)std::max<int64_t>(1, g), 256, 0, s>>>(X, ldx, Y, ldy, rows, cols,
                                                                    VT(a));
  KATZ_CHECK_LAUNCH();
}
template void copy2d<float>(const float*, int64_t, float*, int64_t, int64_t, int64_t, double,
                            cudaStream_t);
template void copy2d<double>(const double*, int64_t, double*, int64_t, int64_t, int64_t, double,
                             cudaStream_t);

// Dense SPD inverse in place by blocked Gauss-Jordan (pivot blocks of 64):
//   Pinv = A_kk^{-1};  Rp = Pinv A_k,: ;  A -= A_:,k Rp ;
//   A_k,: = Rp ; A_:,k = -A_:,k Pinv ; A_kk = Pinv.
// ws must hold n*64 (Rp) + n*64 (column copy) + 64*64 doubles.
void spd_inverse_inplace(double* A, int64_t n, int64_t lda, double* ws, int* flag,
                         cudaStream_t s) {
  const int64_t NB = 64;
  double* Rp = ws;
  double* Cc = ws + n * NB;
  double* Pinv = Cc + n * NB;
  for (int64_t k = 0; k < n; k += NB) {
    const int64_t nb = std::min(NB, n - k);
    copy2d<double>(A + k * lda + k, lda, Pinv, NB, nb, nb, 1.0, s);
    small_spd_inverse(Pinv, NB, (int)nb, flag, s);
    // Rp (nb x n) = Pinv * A[k:k+nb, :]
    gemm2<double>(false, false, nb, n, nb, 1.0, Pinv, NB, A + k * lda, lda, 0.0, Rp, n, false, s);
    // Cc (n x nb) = A[:, k:k+nb]
    copy2d<double>(A + k, lda, Cc, NB, n, nb, 1.0, s);
    // A -= Cc * Rp
    gemm2<double>(false, false, n, n, nb, -1.0, Cc, NB, Rp, n, 1.0, A, lda, false, s);
    // row block k := Rp
    copy2d<double>(Rp, n, A + k * lda, lda, nb, n, 1.0, s);
    // column block k := -Cc * Pinv
    gemm2<double>(false, false, n, nb, nb, -1.0, Cc, NB, Pinv, NB, 0.0, A + k, lda, false, s);
    // pivot block := Pinv
    copy2d<double>(Pinv, NB, A + k * lda + k, lda, nb, nb, 1.0, s);
  }
}

// ---------------------------------------------------------------- top-k
// Candidate order: score descending, node id ascending (a strict total
// order, so every implementation selects the same set).
template <class T>
__device__ __forceinline__ bool better(T sa, int ia, T sb, int ib) {
  return sa > sb || (sa == sb && ia < ib);
}

constexpr int kTopMax = 64;
constexpr int kTopUnroll = 16;  // rows loaded ahead per warp (2 KB in flight per warp)
constexpr int kTopFilterDeg = 512;  // neighbour lists filtered bit by bit up to this length
constexpr int kTopSmemK = 32;       // lists of up to this length kept in shared memory

// Pass 1: CTA = (row slice, 8 tiles of 32 query columns); warp w takes
// column tile blockIdx.y * 8 + w and lane c its column tile * 32 + c, so
// the CTA's warps read neighbouring 128-byte segments of the same rows (a
// 1 KB stretch of each row of K at a time) and each warp walks every row
// of the slice, kTopUnroll rows ahead.  Each (warp, column) keeps a sorted
// top-k list in local memory (scores in K's own type, so the order is
// decided in that precision) with its k-th entry held in registers; a
// candidate is tested against q's neighbours (skipped when mask_nbrs is
// false) only when it beats the k-th entry: first against a 512-bit filter
// of the neighbour ids in shared memory (bit id mod 512; all bits set for
// more than kTopFilterDeg neighbours), then, where the bit is set, by binary
// search in the sorted CSR row.  SL: the lists live in shared memory (entry
// t of the thread's list at [t][threadIdx.x], k <= kTopSmemK), else in local
// memory.  Lists go to the scratch as [column][slice][k].
template <class VT, bool SL>
__global__ void __launch_bounds__(256) topk_partial_kernel(Csr W, const VT* K, int64_t ldk,
                                                           int64_t n, const int32_t* q, int b,
                                                           int k, int64_t rows_per_slice,
                                                           bool mask_nbrs, int32_t* pid,
                                                           double* psc) {
  // filter word w of the thread's column at nbm[w][threadIdx.x] (each
  // thread writes and reads its own column only)
  __shared__ uint32_t nbm[16][256];
  extern __shared__ __align__(16) unsigned char tk_smem[];
  VT* s_sc = reinterpret_cast<VT*>(tk_smem);
  int* s_id = reinterpret_cast<int*>(tk_smem + sizeof(VT) * 256 * size_t(k));
  VT l_sc[SL ? 1 : kTopMax];
  int l_id[SL ? 1 : kTopMax];
  auto LS = [&](int t) -> VT& {
    if constexpr (SL) return s_sc[t * 256 + threadIdx.x];
    else return l_sc[t];
  };
  auto LI = [&](int t) -> int& {
    if constexpr (SL) return s_id[t * 256 + threadIdx.x];
    else return l_id[t];
  };
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = (blockIdx.y * 8 + warp) * 32 + lane;
  const bool cv = j < b;
  const int64_t r0 = int64_t(blockIdx.x) * rows_per_slice;
  const int64_t r1 = min(n, r0 + rows_per_slice);
  const int64_t qq = cv ? q[j] : -1;
  const int64_t nb0 = cv && mask_nbrs ? W.rowptr[qq] : 0;
  const int64_t nb1 = cv && mask_nbrs ? W.rowptr[qq + 1] : 0;
  {
    const uint32_t fill = nb1 - nb0 > kTopFilterDeg ? 0xffffffffu : 0u;
#pragma unroll
    for (int w = 0; w < 16; ++w) nbm[w][threadIdx.x] = fill;
    if (fill == 0u)
      for (int64_t e = nb0; e < nb1; ++e) {
        const int c = W.col[e];
        nbm[(c >> 5) & 15][threadIdx.x] |= 1u << (c & 31);
      }
  }
  int cnt = 0;
  VT thv = VT(0);  // k-th entry once the list is full
  int thi = 0;
  // every score below the gate loses: -infinity until the list is full,
  // then the k-th entry's score (equal scores are decided by the id)
  VT gate = -VT(INFINITY);
  // a candidate that passed the gate: q itself and q's neighbours are
  // skipped, the rest is inserted in order if it beats the k-th entry
  auto offer = [&](VT v, int64_t i) {
    if (i == qq) return;
    if (cnt == k && !better(v, (int)i, thv, thi)) return;
    if ((nbm[(i >> 5) & 15][threadIdx.x] >> (i & 31)) & 1u) {
      int64_t lo = nb0, hi = nb1;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (W.col[mid] < i) lo = mid + 1; else hi = mid;
      }
      if (lo < nb1 && W.col[lo] == i) return;
    }
    int p = cnt < k ? cnt++ : k - 1;
    while (p > 0 && better(v, (int)i, LS(p - 1), LI(p - 1))) {
      LS(p) = LS(p - 1);
      LI(p) = LI(p - 1);
      --p;
    }
    LS(p) = v;
    LI(p) = (int)i;
    if (cnt == k) {
      thv = LS(k - 1);
      thi = LI(k - 1);
      gate = thv;
    }
  };
  if (cv) {
    // whole batches of kTopUnroll rows: all loads issued first, then one
    // comparison per row against the gate on the common path
    int64_t i0 = r0;
    for (; i0 + kTopUnroll <= r1; i0 += kTopUnroll) {
      VT vals[kTopUnroll];
#pragma unroll
      for (int u = 0; u < kTopUnroll; ++u) vals[u] = K[(i0 + u) * ldk + j];
#pragma unroll
      for (int u = 0; u < kTopUnroll; ++u)
        if (vals[u] >= gate) offer(vals[u], i0 + u);
    }
    for (; i0 < r1; ++i0) {
      const VT v = K[i0 * ldk + j];
      if (v >= gate) offer(v, i0);
    }
    const int lists = gridDim.x;
    const int64_t out = (int64_t(j) * lists + blockIdx.x) * k;
    for (int t = 0; t < k; ++t) {
      pid[out + t] = t < cnt ? LI(t) : -1;
      psc[out + t] = t < cnt ? double(LS(t)) : 0.0;
    }
  }
}

// Pass 2: one warp per column merges its sorted lists (k-way selection):
// lane l holds the heads of lists l, l + 32, ... (lists <= 128), the best
// head of the warp is found by a shuffle reduction and advanced.  Ids are
// unique across a column's lists (the row slices are disjoint), so the
// (score, id) order picks one winner per step.
__global__ void topk_merge_warp_kernel(const int32_t* pid, const double* psc, int lists, int k,
                                       int b, int32_t* ids, double* scores) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (j >= b) return;
  const int64_t base = j * lists * k;
  int head[4] = {0, 0, 0, 0};
  for (int t = 0; t < k; ++t) {
    double bs = 0.0;
    int bid = -1, bm = -1;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int l = lane + 32 * m;
      if (l >= lists || head[m] >= k) continue;
      const int64_t o = base + int64_t(l) * k + head[m];
      const int id = pid[o];
      if (id < 0) continue;
      const double sc = psc[o];
      if (bm < 0 || better(sc, id, bs, bid)) { bs = sc; bid = id; bm = m; }
    }
    int wl = bm >= 0 ? lane : -1;  // lane holding the warp's best head so far
    for (int off = 16; off > 0; off >>= 1) {
      const double os = __shfl_xor_sync(0xffffffffu, bs, off);
      const int oid = __shfl_xor_sync(0xffffffffu, bid, off);
      const int ol = __shfl_xor_sync(0xffffffffu, wl, off);
      if (ol >= 0 && (wl < 0 || better(os, oid, bs, bid))) { bs = os; bid = oid; wl = ol; }
    }
    if (wl < 0) {
      if (lane == 0) {
        ids[j * k + t] = -1;
        scores[j * k + t] = 0.0;
      }
      continue;
    }
    if (lane == wl) {
#pragma unroll
      for (int m = 0; m < 4; ++m) head[m] += m == bm ? 1 : 0;
    }
    if (lane == 0) {
      ids[j * k + t] = bid;
      scores[j * k + t] = bs;
    }
  }
}

template <class VT>
void topk_columns_ws(const Csr& W, const VT* K, int64_t ldk, int64_t n, const int32_t* q, int b,
                     int k, int32_t* ids, double* scores, int32_t* ws_id, double* ws_sc,
                     int slices, cudaStream_t s, bool mask_nbrs) {
  KATZ_REQUIRE(slices * 8 <= 2 * kTopMax && k <= kTopMax, KATZ_EINVAL, "topk: too many lists");
  // 8 row slices per requested slice: 8 lists of k per column and slice, as
  // the scratch is sized
  const int64_t rows_per = ceil_div(n, int64_t(slices) * 8);
  dim3 grid((unsigned)(slices * 8), (unsigned)ceil_div(b, 256));
  prof_begin(s);
  if (k <= kTopSmemK) {
    const size_t smem = size_t(256) * k * (sizeof(VT) + sizeof(int));
    KATZ_CUDA(cudaFuncSetAttribute(topk_partial_kernel<VT, true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    topk_partial_kernel<VT, true><<<grid, 256, smem, s>>>(W, K, ldk, n, q, b, k, rows_per,
                                                          mask_nbrs, ws_id, ws_sc);
  } else {
    topk_partial_kernel<VT, false><<<grid, 256, 0, s>>>(W, K, ldk, n, q, b, k, rows_per,
                                                        mask_nbrs, ws_id, ws_sc);
  }
  KATZ_CHECK_LAUNCH();
  topk_merge_warp_kernel<<<(unsigned)ceil_div(int64_t(b) * 32, 256), 256, 0, s>>>(
      ws_id, ws_sc, slices * 8, k, b, ids, scores);
  KATZ_CHECK_LAUNCH();
  // algorithmic: K read once, the lists written and read once, the result
  if (profiling())
    prof_end("topk",
             double(n) * b * sizeof(VT) + 2.0 * 12.0 * double(slices) * 8 * b * k + 12.0 * b * k,
             s);
}
template void topk_columns_ws<float>(const Csr&, const float*, int64_t, int64_t, const int32_t*,
                                     int, int, int32_t*, double*, int32_t*, double*, int,
                                     cudaStream_t, bool);
template void topk_columns_ws<double>(const Csr&, const double*, int64_t, int64_t,
                                      const int32_t*, int, int, int32_t*, double*, int32_t*,
                                      double*, int, cudaStream_t, bool);

}  // namespace katz
