// Refinement residual of the full system in double-FP32 ("float-float")
// arithmetic, gathering one FP32 operand X per pass (M = I - beta A):
//   first pass : (Rh, Rl) = -M X for the first FP32 solution X = K0 (the
//                sums in float-float: TwoSum (Knuth) / TwoProd (Dekker, via
//                FMA), ~48 significant bits with FP32 instructions only, as
//                GB300's FP64 pipe is ~60x slower); the sparse b is added
//                after it in float-float;
//   later passes: Rh = Rh (+ Rl) - M X for an FP32 correction X = D, FP32
//                sums for short rows (|M D| is of the order of |R|).
// Rh, rounded to FP32 after the cancellation, is the right-hand side of the
// next FP32 correction solve.  The solution is kept as Kh + Kl (+ the last
// correction, folded in by ff_out or ff_add).
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

template <int WT>
__device__ __forceinline__ float weight(const void* val, int64_t k) {
  if constexpr (WT == KATZ_UNIT) return 1.f;
  else if constexpr (WT == KATZ_F64) return float(static_cast<const double*>(val)[k]);
  else if constexpr (WT == KATZ_F32) return static_cast<const float*>(val)[k];
  else return __bfloat162float(static_cast<const __nv_bfloat16*>(val)[k]);
}

// acc += w * x (w * x exact through FMA)
template <bool UNIT>
__device__ __forceinline__ void ff_acc(FF& acc, float w, float x) {
  if constexpr (UNIT) {
    const FF t = two_sum(acc.hi, x);
    acc.hi = t.hi;
    acc.lo += t.lo;
  } else {
    const float p = w * x;
    const float pe = __fmaf_rn(w, x, -p);
    const FF t = two_sum(acc.hi, p);
    acc.hi = t.hi;
    acc.lo += t.lo + pe;
  }
}

// (rh, rl) + beta * acc - x, renormalised (beta = beh + bel)
__device__ __forceinline__ FF ff_res(FF acc, float beh, float bel, float x, float rh, float rl) {
  const FF s = fast_two_sum(acc.hi, acc.lo);
  const float ph = beh * s.hi;
  const float pe = __fmaf_rn(beh, s.hi, -ph) + beh * s.lo + bel * s.hi;
  const FF t1 = two_sum(ph, -x);
  const FF t2 = two_sum(t1.hi, rh);
  return fast_two_sum(t2.hi, t1.lo + t2.lo + pe + rl);
}

constexpr int64_t kFp32Row = 64;  // longest row summed in FP32 by the update passes

// acc[v][w] = sum_k w_ik X[col k][tile + (v * 32 + t) * 4 + w] over the stored
// entries [k0, k1) of a row, float-float (FFACC) or FP32 (returned as hi).
template <int WT, int VPT, bool FFACC>
__device__ __forceinline__ void row_sum(const Csr& A, const float* __restrict__ X, int64_t ld,
                                        int64_t tile0, int t, const bool (&cval)[VPT], int64_t k0,
                                        int64_t k1, FF (&acc)[VPT][4]) {
  constexpr bool UNIT = WT == KATZ_UNIT;
  float sacc[VPT][4];
#pragma unroll
  for (int v = 0; v < VPT; ++v)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      acc[v][w] = {0.f, 0.f};
      sacc[v][w] = 0.f;
    }
  for (int64_t kb = k0; kb < k1; kb += 32) {
    const int64_t k = kb + t;
    int cj = 0;
    float wj = 0.f;
    if (k < k1) {
      cj = A.col[k];
      if constexpr (!UNIT) wj = weight<WT>(A.val, k);
    }
    const int cnt = (int)(k1 - kb < 32 ? k1 - kb : 32);
#pragma unroll 4
    for (int s2 = 0; s2 < cnt; ++s2) {
      const int j = __shfl_sync(0xffffffffu, cj, s2);
      float wv = 1.f;
      if constexpr (!UNIT) wv = __shfl_sync(0xffffffffu, wj, s2);
      const float* xr = X + int64_t(j) * ld + tile0 + t * 4;
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        if (cval[v]) {
          const float4 x = __ldg(reinterpret_cast<const float4*>(xr + v * 128));
          if constexpr (FFACC) {
            ff_acc<UNIT>(acc[v][0], wv, x.x);
            ff_acc<UNIT>(acc[v][1], wv, x.y);
            ff_acc<UNIT>(acc[v][2], wv, x.z);
            ff_acc<UNIT>(acc[v][3], wv, x.w);
          } else {
            sacc[v][0] = __fmaf_rn(wv, x.x, sacc[v][0]);
            sacc[v][1] = __fmaf_rn(wv, x.y, sacc[v][1]);
            sacc[v][2] = __fmaf_rn(wv, x.z, sacc[v][2]);
            sacc[v][3] = __fmaf_rn(wv, x.w, sacc[v][3]);
          }
        }
      }
    }
  }
  if constexpr (!FFACC) {
#pragma unroll
    for (int v = 0; v < VPT; ++v)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[v][w] = {sacc[v][w], 0.f};
  }
}

// Row epilogue: (Rh, Rl)[i] from the row sums acc, X[i] and (update) the
// previous residual; sq accumulates Rh^2 per lane column.
template <int VPT, bool INIT>
__device__ __forceinline__ void row_epilogue(int64_t i, const FF (&acc)[VPT][4],
                                             const float* __restrict__ X, float* Rh, float* Rl,
                                             int64_t ld, int64_t tile0, int t,
                                             const bool (&cval)[VPT], float beh, float bel,
                                             float (&sq)[VPT][4]) {
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    if (!cval[v]) continue;
    const int64_t o = i * ld + tile0 + (v * 32 + t) * 4;
    const float4 x4 = __ldg(reinterpret_cast<const float4*>(X + o));
    const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
    float rh0[4] = {0.f, 0.f, 0.f, 0.f}, rl0[4] = {0.f, 0.f, 0.f, 0.f};
    if constexpr (!INIT) {
      const float4 a1 = *reinterpret_cast<const float4*>(Rh + o);
      rh0[0] = a1.x; rh0[1] = a1.y; rh0[2] = a1.z; rh0[3] = a1.w;
      if (Rl) {
        const float4 a2 = *reinterpret_cast<const float4*>(Rl + o);
        rl0[0] = a2.x; rl0[1] = a2.y; rl0[2] = a2.z; rl0[3] = a2.w;
      }
    }
    float rh[4], rl[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const FF r = ff_res(acc[v][w], beh, bel, xs[w], rh0[w], rl0[w]);
      rh[w] = r.hi;
      rl[w] = r.lo;
      sq[v][w] = __fmaf_rn(r.hi, r.hi, sq[v][w]);
    }
    *reinterpret_cast<float4*>(Rh + o) = make_float4(rh[0], rh[1], rh[2], rh[3]);
    if constexpr (INIT)
      *reinterpret_cast<float4*>(Rl + o) = make_float4(rl[0], rl[1], rl[2], rl[3]);
  }
}

// ---------------------------------------- wide rows, packed arithmetic
// Two FP32 values in one 64-bit register, operated on by the packed
// f32x2 instructions of sm_100+ (one instruction for two columns, the same
// IEEE round-to-nearest operations as two scalar ones, never contracted).
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t pack2(float a, float b) {
  return uint64_t(__float_as_uint(a)) | (uint64_t(__float_as_uint(b)) << 32);
}
__device__ __forceinline__ float lo2(uint64_t v) { return __uint_as_float(uint32_t(v)); }
__device__ __forceinline__ float hi2(uint64_t v) { return __uint_as_float(uint32_t(v >> 32)); }
// 8 consecutive FP32 values as 4 packed pairs (one 32-byte access)
__device__ __forceinline__ void ld8_ro(const float* p, uint64_t (&o)[4]) {
  asm("ld.global.nc.v4.b64 {%0,%1,%2,%3}, [%4];"
      : "=l"(o[0]), "=l"(o[1]), "=l"(o[2]), "=l"(o[3])
      : "l"(p));
}
__device__ __forceinline__ void ld8(const float* p, uint64_t (&o)[4]) {
  asm volatile("ld.global.v4.b64 {%0,%1,%2,%3}, [%4];"
               : "=l"(o[0]), "=l"(o[1]), "=l"(o[2]), "=l"(o[3])
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void st8(float* p, const float (&v)[8]) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]),
               "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
// (hi, lo) += x elementwise for two pairs of columns: TwoSum (Knuth) of hi
// and x, its rounding error added to lo
__device__ __forceinline__ void ff_acc2(uint64_t& hi, uint64_t& lo, uint64_t x) {
  const uint64_t s = add2(hi, x);
  const uint64_t bb = sub2(s, hi);
  const uint64_t e = add2(sub2(hi, sub2(s, bb)), sub2(x, bb));
  hi = s;
  lo = add2(lo, e);
}

// Row sums over the stored entries [k0, k1) of one row for the lane's 8
// columns c0 .. c0+7: float-float (FFACC; the product w x split exactly by
// FMA for weighted graphs) or FP32, as packed pairs.
template <int WT, bool FFACC>
__device__ __forceinline__ void row_sum8(const Csr& A, const float* __restrict__ X, int64_t ld,
                                         int64_t c0, bool cval, int t, int64_t k0, int64_t k1,
                                         uint64_t (&hi)[4], uint64_t (&lo)[4]) {
  constexpr bool UNIT = WT == KATZ_UNIT;
#pragma unroll
  for (int q = 0; q < 4; ++q) hi[q] = lo[q] = 0;
  for (int64_t kb = k0; kb < k1; kb += 32) {
    const int64_t k = kb + t;
    int cj = 0;
    float wj = 0.f;
    if (k < k1) {
      cj = A.col[k];
      if constexpr (!UNIT) wj = weight<WT>(A.val, k);
    }
    const int cnt = (int)(k1 - kb < 32 ? k1 - kb : 32);
#pragma unroll 4
    for (int s2 = 0; s2 < cnt; ++s2) {
      const int j = __shfl_sync(0xffffffffu, cj, s2);
      float wv = 1.f;
      if constexpr (!UNIT) wv = __shfl_sync(0xffffffffu, wj, s2);
      if (cval) {
        uint64_t x[4];
        ld8_ro(X + int64_t(j) * ld + c0, x);
        if constexpr (UNIT) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if constexpr (FFACC) ff_acc2(hi[q], lo[q], x[q]);
            else hi[q] = add2(hi[q], x[q]);
          }
        } else {
          const uint64_t w2 = pack2(wv, wv);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if constexpr (FFACC) {
              const uint64_t pr = mul2(w2, x[q]);
              const uint64_t pe = fma2(w2, x[q], pr ^ 0x8000000080000000ull);  // w x - p, exact
              ff_acc2(hi[q], lo[q], pr);
              lo[q] = add2(lo[q], pe);
            } else {
              hi[q] = fma2(w2, x[q], hi[q]);
            }
          }
        }
      }
    }
  }
}

// Per-CTA column sums of Rh^2 (red: [8 warps][TILE] in shared memory, each
// warp's lanes add their sq), then one FP64 atomic per column and CTA.
template <int VPT>
__device__ __forceinline__ void flush_sq(double (*red)[128 * VPT], int wib, int t,
                                         float (&sq)[VPT][4]) {
#pragma unroll
  for (int v = 0; v < VPT; ++v)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      red[wib][(v * 32 + t) * 4 + w] += sq[v][w];
      sq[v][w] = 0.f;
    }
}

template <int VPT>
__device__ __forceinline__ void column_atomics(double (*red)[128 * VPT], int64_t tile0, int b,
                                               double* rr) {
  for (int c = threadIdx.x; c < 128 * VPT; c += blockDim.x) {
    double sum = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) sum += red[q][c];
    if (tile0 + c < b && sum != 0.0) atomicAdd(rr + tile0 + c, sum);
  }
}

__device__ __forceinline__ FF ff_plus(FF a, FF b) {
  const FF t = two_sum(a.hi, b.hi);
  return fast_two_sum(t.hi, t.lo + a.lo + b.lo);
}

// Warp per row, VPT float4 column groups per lane per tile of 128 * VPT
// columns (the warps stride over all rows, or with chunk > 0 CTA c takes the
// rows [c, c + 1) * chunk, its warps interleaved); rows longer than kHeavyRowNnz are left to the split
// kernels when skip_heavy.  Column sums of Rh^2: FP32 over at most 64 rows
// per lane, then FP64 in shared memory per warp, then one atomic per column
// and CTA.
template <int WT, int VPT, bool INIT>
__global__ void __launch_bounds__(256) ffr_rows_kernel(Csr A, const float* __restrict__ X,
                                                       float* Rh, float* Rl, int64_t ld, float beh,
                                                       float bel, double* rr, int b,
                                                       bool skip_heavy, int64_t chunk) {
  constexpr int TILE = 128 * VPT;
  __shared__ double red[8][TILE];
  const int t = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t tile0 = int64_t(blockIdx.y) * TILE;
  for (int c = threadIdx.x; c < 8 * TILE; c += blockDim.x) (&red[0][0])[c] = 0.0;
  bool cval[VPT];
#pragma unroll
  for (int v = 0; v < VPT; ++v) cval[v] = tile0 + (v * 32 + t) * 4 < ld;
  float sq[VPT][4];
#pragma unroll
  for (int v = 0; v < VPT; ++v)
#pragma unroll
    for (int w = 0; w < 4; ++w) sq[v][w] = 0.f;
  int nsq = 0;
  __syncthreads();
  int64_t i0 = warp, i1 = A.nrows, is = nwarps;
  if (chunk > 0) {
    i0 = int64_t(blockIdx.x) * chunk + wib;
    i1 = min(A.nrows, int64_t(blockIdx.x + 1) * chunk);
    is = blockDim.x >> 5;
  }
  for (int64_t i = i0; i < i1; i += is) {
    const int64_t k0 = A.rowptr[i], k1 = A.rowptr[i + 1];
    if (skip_heavy && k1 - k0 > kHeavyRowNnz) continue;
    FF acc[VPT][4];
    // the first pass (X = K0) cancels to the residual's size and needs the
    // float-float sum; later passes gather a correction X = D with
    // |M D| ~ |r|, where FP32 sums of short rows carry errors ~1e-7 of the
    // result (rows longer than kFp32Row keep the float-float sum)
    if (INIT || k1 - k0 > kFp32Row)
      row_sum<WT, VPT, true>(A, X, ld, tile0, t, cval, k0, k1, acc);
    else
      row_sum<WT, VPT, false>(A, X, ld, tile0, t, cval, k0, k1, acc);
    row_epilogue<VPT, INIT>(i, acc, X, Rh, Rl, ld, tile0, t, cval, beh, bel, sq);
    if (++nsq == 64) {
      flush_sq<VPT>(red, wib, t, sq);
      nsq = 0;
    }
  }
  flush_sq<VPT>(red, wib, t, sq);
  __syncthreads();
  if (rr) column_atomics<VPT>(red, tile0, b, rr);
}

// Warp per row (either row schedule of ffr_rows_kernel) on 256-column tiles, 8 consecutive columns
// per lane moved by 32-byte accesses and summed with packed f32x2
// instructions; otherwise as ffr_rows_kernel (same sums, same epilogue).
template <int WT, bool INIT>
__global__ void __launch_bounds__(256) ffr_rows8_kernel(Csr A, const float* __restrict__ X,
                                                        float* Rh, float* Rl, int64_t ld,
                                                        float beh, float bel, double* rr, int b,
                                                        bool skip_heavy, int64_t chunk) {
  constexpr int TILE = 256;
  __shared__ double red[8][TILE];
  const int t = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t tile0 = int64_t(blockIdx.y) * TILE;
  const int64_t c0 = tile0 + 8 * t;
  const bool cval = c0 < ld;
  for (int c = threadIdx.x; c < 8 * TILE; c += blockDim.x) (&red[0][0])[c] = 0.0;
  float sq[8];
#pragma unroll
  for (int w = 0; w < 8; ++w) sq[w] = 0.f;
  int nsq = 0;
  __syncthreads();
  int64_t i0 = warp, i1 = A.nrows, is = nwarps;
  if (chunk > 0) {
    i0 = int64_t(blockIdx.x) * chunk + wib;
    i1 = min(A.nrows, int64_t(blockIdx.x + 1) * chunk);
    is = blockDim.x >> 5;
  }
  for (int64_t i = i0; i < i1; i += is) {
    const int64_t k0 = A.rowptr[i], k1 = A.rowptr[i + 1];
    if (skip_heavy && k1 - k0 > kHeavyRowNnz) continue;
    uint64_t hi[4], lo[4];
    if (INIT || k1 - k0 > kFp32Row)
      row_sum8<WT, true>(A, X, ld, c0, cval, t, k0, k1, hi, lo);
    else
      row_sum8<WT, false>(A, X, ld, c0, cval, t, k0, k1, hi, lo);
    if (cval) {
      const int64_t o = i * ld + c0;
      uint64_t xq[4], a[4] = {0, 0, 0, 0}, l[4] = {0, 0, 0, 0};
      ld8_ro(X + o, xq);
      if constexpr (!INIT) {
        ld8(Rh + o, a);
        if (Rl) ld8(Rl + o, l);
      }
      float rh[8], rl[8];
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const int q = w >> 1;
        const bool up = w & 1;
        const FF acc = {up ? hi2(hi[q]) : lo2(hi[q]), up ? hi2(lo[q]) : lo2(lo[q])};
        const float xw = up ? hi2(xq[q]) : lo2(xq[q]);
        const float r0 = up ? hi2(a[q]) : lo2(a[q]);
        const float l0 = up ? hi2(l[q]) : lo2(l[q]);
        const FF r = ff_res(acc, beh, bel, xw, r0, l0);
        rh[w] = r.hi;
        rl[w] = r.lo;
        sq[w] = __fmaf_rn(r.hi, r.hi, sq[w]);
      }
      st8(Rh + o, rh);
      if constexpr (INIT) st8(Rl + o, rl);
    }
    if (++nsq == 64) {
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        red[wib][8 * t + w] += sq[w];
        sq[w] = 0.f;
      }
      nsq = 0;
    }
  }
#pragma unroll
  for (int w = 0; w < 8; ++w) red[wib][8 * t + w] += sq[w];
  __syncthreads();
  if (rr) column_atomics<2>(red, tile0, b, rr);
}

// Heavy rows, pass 1: CTA = (segment of kHeavySeg entries, column tile);
// each warp sums kHeavySeg / 8 entries in float-float, the 8 partials are
// added in warp order in shared memory and stored as (P[g], P[nseg + g]).
template <int WT, int VPT>
__global__ void __launch_bounds__(256) ffr_heavy_partial_kernel(Csr A, const float* __restrict__ X,
                                                                int64_t ld, HeavyRows hv) {
  constexpr int TILE = 128 * VPT;
  constexpr int64_t kPerWarp = kHeavySeg / 8;
  __shared__ FF red[8][TILE];
  const int t = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t g = blockIdx.x;
  const int64_t tile0 = int64_t(blockIdx.y) * TILE;
  const int h = hv.seg_row[g];
  const int64_t row = hv.rows[h];
  const int64_t r0 = A.rowptr[row], r1 = A.rowptr[row + 1];
  const int64_t s0 = r0 + (g - hv.seg_ptr[h]) * kHeavySeg;
  const int64_t k0 = min(r1, s0 + wib * kPerWarp), k1 = min(r1, s0 + (wib + 1) * kPerWarp);
  bool cval[VPT];
#pragma unroll
  for (int v = 0; v < VPT; ++v) cval[v] = tile0 + (v * 32 + t) * 4 < ld;
  FF acc[VPT][4];
  row_sum<WT, VPT, true>(A, X, ld, tile0, t, cval, k0, k1, acc);
#pragma unroll
  for (int v = 0; v < VPT; ++v)
#pragma unroll
    for (int w = 0; w < 4; ++w) red[wib][(v * 32 + t) * 4 + w] = acc[v][w];
  __syncthreads();
  for (int c = threadIdx.x; c < TILE; c += blockDim.x) {
    if (tile0 + c >= ld) continue;
    FF sum = red[0][c];
#pragma unroll
    for (int q = 1; q < 8; ++q) sum = ff_plus(sum, red[q][c]);
    const int64_t o = g * ld + tile0 + c;
    hv.scratch[o] = sum.hi;
    hv.scratch[hv.nseg * ld + o] = sum.lo;
  }
}

// Heavy rows, pass 1, on 256-column tiles of 32-byte lanes with packed
// f32x2 float-float sums (the partials' layout as ffr_heavy_partial_kernel).
template <int WT>
__global__ void __launch_bounds__(256) ffr_heavy_partial8_kernel(Csr A, const float* __restrict__ X,
                                                                 int64_t ld, HeavyRows hv) {
  constexpr int TILE = 256;
  constexpr int64_t kPerWarp = kHeavySeg / 8;
  __shared__ FF red[8][TILE];
  const int t = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t g = blockIdx.x;
  const int64_t tile0 = int64_t(blockIdx.y) * TILE;
  const int64_t c0 = tile0 + 8 * t;
  const bool cval = c0 < ld;
  const int h = hv.seg_row[g];
  const int64_t row = hv.rows[h];
  const int64_t r0 = A.rowptr[row], r1 = A.rowptr[row + 1];
  const int64_t s0 = r0 + (g - hv.seg_ptr[h]) * kHeavySeg;
  const int64_t k0 = min(r1, s0 + wib * kPerWarp), k1 = min(r1, s0 + (wib + 1) * kPerWarp);
  uint64_t hi[4], lo[4];
  row_sum8<WT, true>(A, X, ld, c0, cval, t, k0, k1, hi, lo);
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const int q = w >> 1;
    const bool up = w & 1;
    red[wib][8 * t + w] = {up ? hi2(hi[q]) : lo2(hi[q]), up ? hi2(lo[q]) : lo2(lo[q])};
  }
  __syncthreads();
  for (int c = threadIdx.x; c < TILE; c += blockDim.x) {
    if (tile0 + c >= ld) continue;
    FF sum = red[0][c];
#pragma unroll
    for (int q = 1; q < 8; ++q) sum = ff_plus(sum, red[q][c]);
    const int64_t o = g * ld + tile0 + c;
    hv.scratch[o] = sum.hi;
    hv.scratch[hv.nseg * ld + o] = sum.lo;
  }
}

// Heavy rows, pass 2: warp per heavy row; its segment partials are added
// in segment order, then the row epilogue and the Rh^2 column sums.
template <int VPT, bool INIT>
__global__ void __launch_bounds__(256) ffr_heavy_finish_kernel(const float* __restrict__ X,
                                                               float* Rh, float* Rl, int64_t ld,
                                                               float beh, float bel, double* rr,
                                                               int b, HeavyRows hv) {
  constexpr int TILE = 128 * VPT;
  __shared__ double red[8][TILE];
  const int t = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t h = int64_t(blockIdx.x) * 8 + wib;
  const int64_t tile0 = int64_t(blockIdx.y) * TILE;
  for (int c = threadIdx.x; c < 8 * TILE; c += blockDim.x) (&red[0][0])[c] = 0.0;
  bool cval[VPT];
#pragma unroll
  for (int v = 0; v < VPT; ++v) cval[v] = tile0 + (v * 32 + t) * 4 < ld;
  float sq[VPT][4];
#pragma unroll
  for (int v = 0; v < VPT; ++v)
#pragma unroll
    for (int w = 0; w < 4; ++w) sq[v][w] = 0.f;
  __syncthreads();
  if (h < hv.n) {
    FF acc[VPT][4];
#pragma unroll
    for (int v = 0; v < VPT; ++v)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[v][w] = {0.f, 0.f};
    for (int64_t g = hv.seg_ptr[h]; g < hv.seg_ptr[h + 1]; ++g) {
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        if (!cval[v]) continue;
        const int64_t o = g * ld + tile0 + (v * 32 + t) * 4;
        const float4 ph = *reinterpret_cast<const float4*>(hv.scratch + o);
        const float4 pl = *reinterpret_cast<const float4*>(hv.scratch + hv.nseg * ld + o);
        acc[v][0] = ff_plus(acc[v][0], {ph.x, pl.x});
        acc[v][1] = ff_plus(acc[v][1], {ph.y, pl.y});
        acc[v][2] = ff_plus(acc[v][2], {ph.z, pl.z});
        acc[v][3] = ff_plus(acc[v][3], {ph.w, pl.w});
      }
    }
    row_epilogue<VPT, INIT>(hv.rows[h], acc, X, Rh, Rl, ld, tile0, t, cval, beh, bel, sq);
  }
  flush_sq<VPT>(red, wib, t, sq);
  __syncthreads();
  if (rr) column_atomics<VPT>(red, tile0, b, rr);
}

// (Rh, Rl)[pos(i), j] += beta w_{q_j i}; rr[j] += new Rh^2 - old Rh^2.
template <int WT>
__global__ void ffr_add_rhs_kernel(Csr W, const int32_t* q, const int32_t* pos, double beta,
                                   float* Rh, float* Rl, int64_t ld, double* rr) {
  const int j = blockIdx.y;
  const int64_t qq = q[j];
  const int64_t e = W.rowptr[qq] + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= W.rowptr[qq + 1]) return;
  const int64_t node = W.col[e];
  const int64_t i = pos ? pos[node] : node;
  const double bv = beta * double(weight<WT>(W.val, e));
  const float bh = float(bv), bl = float(bv - double(bh));
  const int64_t o = i * ld + j;
  const float old = Rh[o];
  const FF t = two_sum(old, bh);
  const FF r = fast_two_sum(t.hi, t.lo + Rl[o] + bl);
  Rh[o] = r.hi;
  Rl[o] = r.lo;
  if (rr) atomicAdd(rr + j, double(r.hi) * r.hi - double(old) * old);
}

__global__ void ff_add_kernel(float* __restrict__ Kh, float* __restrict__ Kl,
                              const float* __restrict__ D, int64_t total, bool kl_zero) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const FF t = two_sum(Kh[e], D[e]);
    const FF u = fast_two_sum(t.hi, kl_zero ? t.lo : t.lo + Kl[e]);
    Kh[e] = u.hi;
    Kl[e] = u.lo;
  }
}

// out = Kh + Kl (+ D), rounded once to the output type
__global__ void ff_out_kernel(const float* __restrict__ Kh, const float* __restrict__ Kl,
                              const float* __restrict__ D, int64_t ld, const int32_t* map,
                              int64_t n, int b, void* out, int out_dt, int64_t ldk) {
  const int64_t total = n * b;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / b, c = e - i * b;
    const int64_t r = map ? map[i] : i;
    const int64_t o = r * ld + c;
    const float d = D ? D[o] : 0.f;
    const float kl = Kl ? Kl[o] : 0.f;
    if (out_dt == KATZ_F64) {
      static_cast<double*>(out)[i * ldk + c] = (double(Kh[o]) + double(d)) + double(kl);
    } else {
      const FF t = two_sum(Kh[o], d);
      static_cast<float*>(out)[i * ldk + c] = t.hi + (t.lo + kl);
    }
  }
}

// The same, a warp per output row (rows grid-stride) and 4 columns per lane
// moved as float4 (FP32 output, every leading dimension a multiple of 4 and
// 16-byte aligned bases): no per-element index division.
__global__ void ff_out_rows_kernel(const float* __restrict__ Kh, const float* __restrict__ Kl,
                                   const float* __restrict__ D, int64_t ld, const int32_t* map,
                                   int64_t n, int b, float* out, int64_t ldk) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n;
       i += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    const int64_t r = map ? map[i] : i;
    for (int c = lane * 4; c < b; c += 128) {
      const int64_t o = r * ld + c;
      const float4 h = __ldg(reinterpret_cast<const float4*>(Kh + o));
      const float4 l = Kl ? __ldg(reinterpret_cast<const float4*>(Kl + o)) : make_float4(0, 0, 0, 0);
      const float4 d = D ? __ldg(reinterpret_cast<const float4*>(D + o)) : make_float4(0, 0, 0, 0);
      const FF t0 = two_sum(h.x, d.x), t1 = two_sum(h.y, d.y), t2 = two_sum(h.z, d.z),
               t3 = two_sum(h.w, d.w);
      const float4 v = make_float4(t0.hi + (t0.lo + l.x), t1.hi + (t1.lo + l.y),
                                   t2.hi + (t2.lo + l.z), t3.hi + (t3.lo + l.w));
      if (c + 4 <= b) {
        *reinterpret_cast<float4*>(out + i * ldk + c) = v;
      } else {  // ragged tail inside ld: only the columns < b
        const float vv[4] = {v.x, v.y, v.z, v.w};
        for (int w = 0; c + w < b; ++w) out[i * ldk + c + w] = vv[w];
      }
    }
  }
}

unsigned flat(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), int64_t(num_sms()) * 16));
}

}  // namespace

void ffr_update(const Csr& A, double beta, const float* X, float* Rh, float* Rl, bool init,
                int64_t ld, int b, double* rr, const SpmmCfg* cfg, cudaStream_t s,
                const HeavyRows* hv) {
  KATZ_REQUIRE(ld % 4 == 0 && ld >= b && reinterpret_cast<uintptr_t>(X) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(Rh) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(Rl) % 16 == 0 && (Rl || !init),
               KATZ_EINVAL, "ffr_update: operands must be 16-byte aligned with padded rows");
  if (A.nrows <= 0) return;
  const float beh = float(beta), bel = float(beta - double(beh));
  const int vpt = ld > 128 ? 2 : 1;
  const int64_t tiles = ceil_div(ld, 128 * vpt);
  const int cps = cfg && cfg->fused_cps > 0     ? cfg->fused_cps
                  : cfg && cfg->ctas_per_sm > 0 ? cfg->ctas_per_sm
                                                : 8;
  const int64_t chunk = cfg && cfg->row_chunk > 0 ? cfg->row_chunk : 0;
  const int64_t ctas = chunk > 0 ? ceil_div(A.nrows, chunk)
                                 : std::min<int64_t>(ceil_div(A.nrows, 8),
                                                     std::max<int64_t>(1, int64_t(num_sms()) *
                                                                              cps / tiles));
  KATZ_REQUIRE(ctas < (int64_t(1) << 31), KATZ_EINVAL, "ffr_update: row chunk too small");
  const dim3 grid((unsigned)std::max<int64_t>(1, ctas), (unsigned)tiles);
  const bool split = hv && hv->nseg > 0;
  KATZ_REQUIRE(!split || (hv->scratch && reinterpret_cast<uintptr_t>(hv->scratch) % 16 == 0),
               KATZ_EINVAL, "ffr_update: heavy-row scratch must be 16-byte aligned");
  // 32-byte lane accesses where the rows and bases allow them (same tiles
  // of 256 columns)
  const bool wide = vpt == 2 && ld % 8 == 0 &&
                    ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Rh) |
                      reinterpret_cast<uintptr_t>(Rl)) % 32) == 0;
  prof_begin(s);
#define KATZ_FFR(WT, V, I) \
  ffr_rows_kernel<WT, V, I><<<grid, 256, 0, s>>>(A, X, Rh, Rl, ld, beh, bel, rr, b, split, chunk)
#define KATZ_FFR8(WT, I) \
  ffr_rows8_kernel<WT, I><<<grid, 256, 0, s>>>(A, X, Rh, Rl, ld, beh, bel, rr, b, split, chunk)
#define KATZ_FFR_W(WT)                                                     \
  if (wide) {                                                              \
    if (init) KATZ_FFR8(WT, true); else KATZ_FFR8(WT, false);              \
  } else if (vpt == 2) {                                                   \
    if (init) KATZ_FFR(WT, 2, true); else KATZ_FFR(WT, 2, false);          \
  } else {                                                                 \
    if (init) KATZ_FFR(WT, 1, true); else KATZ_FFR(WT, 1, false);          \
  }
  switch (A.vdt) {
    case KATZ_UNIT: KATZ_FFR_W(KATZ_UNIT); break;
    case KATZ_F32: KATZ_FFR_W(KATZ_F32); break;
    case KATZ_BF16: KATZ_FFR_W(KATZ_BF16); break;
    default: KATZ_FFR_W(KATZ_F64); break;
  }
#undef KATZ_FFR_W
#undef KATZ_FFR8
#undef KATZ_FFR
  KATZ_CHECK_LAUNCH();
  if (split) {
    const dim3 pg((unsigned)hv->nseg, (unsigned)tiles);
    const dim3 fg((unsigned)ceil_div(hv->n, 8), (unsigned)tiles);
#define KATZ_FFH(WT)                                                                        \
  if (wide) ffr_heavy_partial8_kernel<WT><<<pg, 256, 0, s>>>(A, X, ld, *hv);               \
  else if (vpt == 2) ffr_heavy_partial_kernel<WT, 2><<<pg, 256, 0, s>>>(A, X, ld, *hv);    \
  else ffr_heavy_partial_kernel<WT, 1><<<pg, 256, 0, s>>>(A, X, ld, *hv)
    switch (A.vdt) {
      case KATZ_UNIT: KATZ_FFH(KATZ_UNIT); break;
      case KATZ_F32: KATZ_FFH(KATZ_F32); break;
      case KATZ_BF16: KATZ_FFH(KATZ_BF16); break;
      default: KATZ_FFH(KATZ_F64); break;
    }
#undef KATZ_FFH
    KATZ_CHECK_LAUNCH();
    if (vpt == 2) {
      if (init) ffr_heavy_finish_kernel<2, true><<<fg, 256, 0, s>>>(X, Rh, Rl, ld, beh, bel, rr, b, *hv);
      else ffr_heavy_finish_kernel<2, false><<<fg, 256, 0, s>>>(X, Rh, Rl, ld, beh, bel, rr, b, *hv);
    } else {
      if (init) ffr_heavy_finish_kernel<1, true><<<fg, 256, 0, s>>>(X, Rh, Rl, ld, beh, bel, rr, b, *hv);
      else ffr_heavy_finish_kernel<1, false><<<fg, 256, 0, s>>>(X, Rh, Rl, ld, beh, bel, rr, b, *hv);
    }
    KATZ_CHECK_LAUNCH();
  }
  if (profiling())
    prof_end("ff_residual",
             8.0 * (A.nrows + 1) + double(A.nnz) * (4 + vdt_size(A.vdt)) +
                 4.0 * ld * (A.ncols + A.nrows * (init ? 3.0 : (Rl ? 4.0 : 3.0))),
             s);
}

void ffr_add_rhs(const Csr& W, const int32_t* q, const int32_t* pos, int b, double beta, float* Rh,
                 float* Rl, int64_t ld, double* rr, int64_t maxdeg, cudaStream_t s) {
  if (maxdeg <= 0 || b <= 0) return;
  const dim3 grid(unsigned(ceil_div(maxdeg, 256)), unsigned(b));
  switch (W.vdt) {
    case KATZ_UNIT: ffr_add_rhs_kernel<KATZ_UNIT><<<grid, 256, 0, s>>>(W, q, pos, beta, Rh, Rl, ld, rr); break;
    case KATZ_F64: ffr_add_rhs_kernel<KATZ_F64><<<grid, 256, 0, s>>>(W, q, pos, beta, Rh, Rl, ld, rr); break;
    case KATZ_F32: ffr_add_rhs_kernel<KATZ_F32><<<grid, 256, 0, s>>>(W, q, pos, beta, Rh, Rl, ld, rr); break;
    default: ffr_add_rhs_kernel<KATZ_BF16><<<grid, 256, 0, s>>>(W, q, pos, beta, Rh, Rl, ld, rr); break;
  }
  KATZ_CHECK_LAUNCH();
}

void ff_add(float* Kh, float* Kl, const float* D, int64_t total, cudaStream_t s, bool kl_zero) {
  if (total <= 0) return;
  ff_add_kernel<<<flat(total), 256, 0, s>>>(Kh, Kl, D, total, kl_zero);
  KATZ_CHECK_LAUNCH();
}

void ff_out(const float* Kh, const float* Kl, const float* D, int64_t ld, const int32_t* map,
            int64_t n, int b, void* out, int out_dt, int64_t ldk, cudaStream_t s) {
  if (n * b <= 0) return;
  const bool rows = out_dt == KATZ_F32 && ld % 4 == 0 && ldk % 4 == 0 &&
                    ((reinterpret_cast<uintptr_t>(Kh) | reinterpret_cast<uintptr_t>(Kl) |
                      reinterpret_cast<uintptr_t>(D) | reinterpret_cast<uintptr_t>(out)) % 16) == 0;
  prof_begin(s);
  if (rows) {
    const unsigned blocks =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 8), int64_t(num_sms()) * 16));
    ff_out_rows_kernel<<<blocks, 256, 0, s>>>(Kh, Kl, D, ld, map, n, b, static_cast<float*>(out),
                                              ldk);
  } else {
    ff_out_kernel<<<flat(n * b), 256, 0, s>>>(Kh, Kl, D, ld, map, n, b, out, out_dt, ldk);
  }
  KATZ_CHECK_LAUNCH();
  // algorithmic: Kh (Kl, D) read once, K written once
  if (profiling())
    prof_end("ff_out",
             double(n) * b * (4.0 * (1 + (Kl ? 1 : 0) + (D ? 1 : 0)) + (out_dt == KATZ_F64 ? 8.0 : 4.0)),
             s);
}

}  // namespace katz
