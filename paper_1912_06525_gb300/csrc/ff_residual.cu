// Residual of the full system, R = B - M K, evaluated in double-FP32
// ("float-float") arithmetic.  K is kept as an unevaluated sum hi + lo of two
// FP32 arrays; products and sums use the error-free transformations TwoSum
// (Knuth) and TwoProd (Dekker, via FMA), giving ~48 significant bits with
// FP32 instructions only.  On GB300 the FP64 pipe is ~60x slower than FP32,
// so this is what makes the refinement residual cheap.  The rounding of R to
// FP32 happens after the cancellation b - (k - beta W k) has been carried
// out in float-float, so R is accurate to FP32 relative to itself.
#include "ff_residual.h"

namespace katz {

namespace {

struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ FF fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}

// acc += w * (xh + xl)
__device__ __forceinline__ void ff_axpy(FF& acc, float w, float xh, float xl) {
  const float p = w * xh;
  const float pe = __fmaf_rn(w, xh, -p);
  const FF s = two_sum(acc.hi, p);
  acc.hi = s.hi;
  acc.lo += s.lo + pe + w * xl;
}

// (beta_h + beta_l) * acc - (kh + kl) + (bh + bl), rounded to FP32
__device__ __forceinline__ float ff_residual(FF acc, float beh, float bel, float kh, float kl,
                                             float bh, float bl) {
  acc = fast_two_sum(acc.hi, acc.lo);
  const float ph = beh * acc.hi;
  const float pe = __fmaf_rn(beh, acc.hi, -ph) + beh * acc.lo + bel * acc.hi;
  const FF s1 = two_sum(ph, -kh);
  const FF s2 = two_sum(s1.hi, bh);
  return s2.hi + (s1.lo + s2.lo + pe - kl + bl);
}

template <int WT>
__device__ __forceinline__ float weight(const void* val, int64_t k) {
  if constexpr (WT == KATZ_UNIT) return 1.f;
  else if constexpr (WT == KATZ_F64) return float(static_cast<const double*>(val)[k]);
  else if constexpr (WT == KATZ_F32) return static_cast<const float*>(val)[k];
  else return __bfloat162float(static_cast<const __nv_bfloat16*>(val)[k]);
}

// Warp per row and 256-column tile (2 x 4 columns per lane).  Float-float
// accumulation of sum_j w_ij (hi_j + lo_j); R = beta*acc - k (the sparse
// RHS b is added by ff_fix_rhs_kernel).  FP64-weighted graphs use FP32
// weights here (exact for the dyadic / unit weights used by this library's
// workloads).
template <int WT>
__global__ void __launch_bounds__(256) ff_residual_kernel(Csr A, const float* __restrict__ Kh,
                                                          const float* __restrict__ Kl, int64_t ld,
                                                          float beh, float bel, float* R, int b) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int c0 = blockIdx.y * 256 + lane * 4;
  const bool cv0 = c0 < b, cv1 = c0 + 128 < b;
  for (int64_t i = warp; i < A.nrows; i += nwarps) {
    const int64_t k0 = A.rowptr[i], k1 = A.rowptr[i + 1];
    FF acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = {0.f, 0.f};
    for (int64_t kb = k0; kb < k1; kb += 32) {
      const int64_t k = kb + lane;
      int cj = 0;
      float wj = 0.f;
      if (k < k1) {
        cj = A.col[k];
        wj = weight<WT>(A.val, k);
      }
      const int cnt = (int)(k1 - kb < 32 ? k1 - kb : 32);
#pragma unroll 4
      for (int s = 0; s < cnt; ++s) {
        const int j = __shfl_sync(0xffffffffu, cj, s);
        const float w = __shfl_sync(0xffffffffu, wj, s);
        const float* hr = Kh + int64_t(j) * ld + c0;
        const float* lr = Kl + int64_t(j) * ld + c0;
        if (cv0) {
          const float4 h = __ldg(reinterpret_cast<const float4*>(hr));
          const float4 l = __ldg(reinterpret_cast<const float4*>(lr));
          ff_axpy(acc[0], w, h.x, l.x);
          ff_axpy(acc[1], w, h.y, l.y);
          ff_axpy(acc[2], w, h.z, l.z);
          ff_axpy(acc[3], w, h.w, l.w);
        }
        if (cv1) {
          const float4 h = __ldg(reinterpret_cast<const float4*>(hr + 128));
          const float4 l = __ldg(reinterpret_cast<const float4*>(lr + 128));
          ff_axpy(acc[4], w, h.x, l.x);
          ff_axpy(acc[5], w, h.y, l.y);
          ff_axpy(acc[6], w, h.z, l.z);
          ff_axpy(acc[7], w, h.w, l.w);
        }
      }
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int c = c0 + 128 * half;
      if (half == 0 ? !cv0 : !cv1) continue;
      const float4 h = *reinterpret_cast<const float4*>(Kh + i * ld + c);
      const float4 l = *reinterpret_cast<const float4*>(Kl + i * ld + c);
      float4 r;
      r.x = ff_residual(acc[4 * half + 0], beh, bel, h.x, l.x, 0.f, 0.f);
      r.y = ff_residual(acc[4 * half + 1], beh, bel, h.y, l.y, 0.f, 0.f);
      r.z = ff_residual(acc[4 * half + 2], beh, bel, h.z, l.z, 0.f, 0.f);
      r.w = ff_residual(acc[4 * half + 3], beh, bel, h.w, l.w, 0.f, 0.f);
      *reinterpret_cast<float4*>(R + i * ld + c) = r;
    }
  }
}

// Entries with a nonzero RHS, b_ij = beta * w(q_j, i) for i in N(q_j):
// recompute them exactly with b included (one warp per entry).
template <int WT>
__global__ void ff_fix_rhs_kernel(Csr A, Csr W, const int32_t* q, const int32_t* pos,
                                  const float* __restrict__ Kh, const float* __restrict__ Kl,
                                  int64_t ld, float beh, float bel, double beta, float* R) {
  const int j = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int64_t qq = q[j];
  const int64_t e = W.rowptr[qq] + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= W.rowptr[qq + 1]) return;
  const int64_t node = W.col[e];
  const double bv = beta * double(weight<WT>(W.val, e));
  const float bh = float(bv), bl = float(bv - double(bh));
  const int64_t i = pos ? pos[node] : node;
  FF acc = {0.f, 0.f};
  for (int64_t k = A.rowptr[i] + lane; k < A.rowptr[i + 1]; k += 32) {
    const int64_t jj = A.col[k];
    ff_axpy(acc, weight<WT>(A.val, k), Kh[jj * ld + j], Kl[jj * ld + j]);
  }
  // combine the lanes' float-float partials
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, acc.hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, acc.lo, o);
    const FF s = two_sum(acc.hi, oh);
    acc.hi = s.hi;
    acc.lo += s.lo + ol;
  }
  if (lane == 0) R[i * ld + j] = ff_residual(acc, beh, bel, Kh[i * ld + j], Kl[i * ld + j], bh, bl);
}

__global__ void ff_add_kernel(float* __restrict__ Kh, float* __restrict__ Kl,
                              const float* __restrict__ D, int64_t total) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const FF s = two_sum(Kh[e], D[e]);
    const FF t = fast_two_sum(s.hi, s.lo + Kl[e]);
    Kh[e] = t.hi;
    Kl[e] = t.lo;
  }
}

__global__ void ff_out_kernel(const float* __restrict__ Kh, const float* __restrict__ Kl,
                              int64_t ld, const int32_t* map, int64_t n, int b, void* out,
                              int out_dt, int64_t ldk) {
  const int64_t total = n * b;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / b, c = e - i * b;
    const int64_t r = map ? map[i] : i;
    if (out_dt == KATZ_F64)
      static_cast<double*>(out)[i * ldk + c] = double(Kh[r * ld + c]) + double(Kl[r * ld + c]);
    else
      static_cast<float*>(out)[i * ldk + c] = Kh[r * ld + c] + Kl[r * ld + c];
  }
}

__global__ void mask_columns_kernel(float* R, int64_t ld, int64_t total, int b, const int* conv) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t c = e % ld;
    if (c >= b || conv[c]) R[e] = 0.f;
  }
}

unsigned flat(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), int64_t(num_sms()) * 16));
}

}  // namespace

void ff_residual(const Csr& A, const Csr& W, const int32_t* q, const int32_t* pos, int b,
                 double beta, const float* Kh, const float* Kl, int64_t ld, float* R,
                 int64_t maxdeg, cudaStream_t s) {
  KATZ_REQUIRE(ld % 4 == 0 && reinterpret_cast<uintptr_t>(Kh) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(Kl) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(R) % 16 == 0 && ld >= b,
               KATZ_EINVAL, "ff_residual: operands must be 16-byte aligned with padded rows");
  const float beh = float(beta), bel = float(beta - double(beh));
  const int tiles = (int)ceil_div(b, 256);
  int64_t ctas = std::min<int64_t>(ceil_div(A.nrows, 8), int64_t(num_sms()) * 8 / tiles);
  dim3 grid((unsigned)std::max<int64_t>(1, ctas), (unsigned)tiles);
  prof_begin(s);
  switch (A.vdt) {
    case KATZ_UNIT: ff_residual_kernel<KATZ_UNIT><<<grid, 256, 0, s>>>(A, Kh, Kl, ld, beh, bel, R, b); break;
    case KATZ_F64: ff_residual_kernel<KATZ_F64><<<grid, 256, 0, s>>>(A, Kh, Kl, ld, beh, bel, R, b); break;
    case KATZ_F32: ff_residual_kernel<KATZ_F32><<<grid, 256, 0, s>>>(A, Kh, Kl, ld, beh, bel, R, b); break;
    default: ff_residual_kernel<KATZ_BF16><<<grid, 256, 0, s>>>(A, Kh, Kl, ld, beh, bel, R, b); break;
  }
  KATZ_CHECK_LAUNCH();
  if (profiling())
    prof_end("ff_residual",
             8.0 * (A.nrows + 1) + double(A.nnz) * (4 + vdt_size(A.vdt)) +
                 4.0 * b * (2.0 * A.ncols + A.nrows),
             s);
  if (maxdeg > 0) {
    dim3 g2((unsigned)ceil_div(maxdeg, 8), (unsigned)b);
    switch (A.vdt) {
      case KATZ_UNIT: ff_fix_rhs_kernel<KATZ_UNIT><<<g2, 256, 0, s>>>(A, W, q, pos, Kh, Kl, ld, beh, bel, beta, R); break;
      case KATZ_F64: ff_fix_rhs_kernel<KATZ_F64><<<g2, 256, 0, s>>>(A, W, q, pos, Kh, Kl, ld, beh, bel, beta, R); break;
      case KATZ_F32: ff_fix_rhs_kernel<KATZ_F32><<<g2, 256, 0, s>>>(A, W, q, pos, Kh, Kl, ld, beh, bel, beta, R); break;
      default: ff_fix_rhs_kernel<KATZ_BF16><<<g2, 256, 0, s>>>(A, W, q, pos, Kh, Kl, ld, beh, bel, beta, R); break;
    }
    KATZ_CHECK_LAUNCH();
  }
}

void ff_add(float* Kh, float* Kl, const float* D, int64_t total, cudaStream_t s) {
  if (total <= 0) return;
  ff_add_kernel<<<flat(total), 256, 0, s>>>(Kh, Kl, D, total);
  KATZ_CHECK_LAUNCH();
}

void ff_out(const float* Kh, const float* Kl, int64_t ld, const int32_t* map, int64_t n, int b,
            void* out, int out_dt, int64_t ldk, cudaStream_t s) {
  if (n * b <= 0) return;
  ff_out_kernel<<<flat(n * b), 256, 0, s>>>(Kh, Kl, ld, map, n, b, out, out_dt, ldk);
  KATZ_CHECK_LAUNCH();
}

void mask_columns(float* R, int64_t ld, int64_t len, int b, const int* conv, cudaStream_t s) {
  if (len * ld <= 0) return;
  mask_columns_kernel<<<flat(len * ld), 256, 0, s>>>(R, ld, len * ld, b, conv);
  KATZ_CHECK_LAUNCH();
}

}  // namespace katz
