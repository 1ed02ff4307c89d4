// HBM-bound kernels of the Katz query path: multi-RHS CSR SpMM on M (Eq. 3)
// and on the coupling blocks (Lemma 1), fused column dot products, CG/PCG
// vector updates, RHS construction, permutations and dense M11 block solves.
//
// Layout: dense n x b blocks are node-major, so one CSR entry (i, j) moves
// the contiguous row X[j, :] (b values) with 16-byte vector loads.
#include "kernels.h"

namespace katz {

// ---------------------------------------------------------------- helpers
template <class VT> struct Acc { using type = VT; };

template <int WT, class A>
__device__ __forceinline__ A load_weight(const void* val, int64_t k) {
  if constexpr (WT == KATZ_UNIT) {
    return A(1);
  } else if constexpr (WT == KATZ_F64) {
    return A(static_cast<const double*>(val)[k]);
  } else if constexpr (WT == KATZ_F32) {
    return A(static_cast<const float*>(val)[k]);
  } else {
    return A(__bfloat162float(static_cast<const __nv_bfloat16*>(val)[k]));
  }
}

template <class VT>
__device__ __forceinline__ void vload(const VT* p, VT (&o)[VecOf<VT>::width]) {
  using V = typename VecOf<VT>::type;
  V v = *reinterpret_cast<const V*>(p);
  if constexpr (VecOf<VT>::width == 4) {
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    o[0] = v.x; o[1] = v.y;
  }
}
// read-only (non-coherent) load for operands no thread of the kernel writes
template <class VT>
__device__ __forceinline__ void vload_ro(const VT* p, VT (&o)[VecOf<VT>::width]) {
  using V = typename VecOf<VT>::type;
  V v = __ldg(reinterpret_cast<const V*>(p));
  if constexpr (VecOf<VT>::width == 4) {
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    o[0] = v.x; o[1] = v.y;
  }
}
template <class VT>
__device__ __forceinline__ void vstore(VT* p, const VT (&o)[VecOf<VT>::width]) {
  using V = typename VecOf<VT>::type;
  V v;
  if constexpr (VecOf<VT>::width == 4) {
    v.x = o[0]; v.y = o[1]; v.z = o[2]; v.w = o[3];
  } else {
    v.x = o[0]; v.y = o[1];
  }
  *reinterpret_cast<V*>(p) = v;
}

namespace {
// CW consecutive columns of one row per lane: 4 (16-byte FP32 / 8-byte BF16
// accesses) or 8 (32-byte FP32 accesses, the 256-bit vector loads and
// stores of sm_100+, and 16-byte BF16 accesses).  "ro": read-only data
// (non-coherent path).
// Two FP32 values in one 64-bit register for the packed f32x2 arithmetic of
// sm_100+ (one instruction per column pair; the same round-to-nearest
// results as two scalar operations, fused where the scalar form is fused)
__device__ __forceinline__ uint64_t padd2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t pfma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

template <int CW> struct Lane;
template <> struct Lane<4> {
  // the lane's 4 columns as 2 packed pairs (read-only path)
  static __device__ __forceinline__ void p32_ro(const float* p, uint64_t (&o)[2]) {
    asm("ld.global.nc.v2.b64 {%0,%1}, [%2];" : "=l"(o[0]), "=l"(o[1]) : "l"(p));
  }
  static __device__ __forceinline__ void f32_ro(const float* p, float (&o)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  static __device__ __forceinline__ void f32(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  static __device__ __forceinline__ void st_f32(float* p, const float (&o)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  }
  static __device__ __forceinline__ void bf16_ro(const __nv_bfloat16* p, float (&o)[4]) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    unpack(u.x, o[0], o[1]);
    unpack(u.y, o[2], o[3]);
  }
  static __device__ __forceinline__ void bf16(const __nv_bfloat16* p, float (&o)[4]) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    unpack(u.x, o[0], o[1]);
    unpack(u.y, o[2], o[3]);
  }
  static __device__ __forceinline__ void st_bf16(__nv_bfloat16* p, const uint32_t (&w)[2]) {
    *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
  }
  static __device__ __forceinline__ void unpack(uint32_t u, float& a, float& b) {
    a = __uint_as_float(u << 16);
    b = __uint_as_float(u & 0xffff0000u);
  }
};
template <> struct Lane<8> {
  static __device__ __forceinline__ void p32_ro(const float* p, uint64_t (&o)[4]) {
    asm("ld.global.nc.v4.b64 {%0,%1,%2,%3}, [%4];"
        : "=l"(o[0]), "=l"(o[1]), "=l"(o[2]), "=l"(o[3])
        : "l"(p));
  }
  static __device__ __forceinline__ void f32_ro(const float* p, float (&o)[8]) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]),
          "=f"(o[7])
        : "l"(p));
  }
  static __device__ __forceinline__ void f32(const float* p, float (&o)[8]) {
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]),
                   "=f"(o[6]), "=f"(o[7])
                 : "l"(p)
                 : "memory");
  }
  static __device__ __forceinline__ void st_f32(float* p, const float (&o)[8]) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(o[0]),
                 "f"(o[1]), "f"(o[2]), "f"(o[3]), "f"(o[4]), "f"(o[5]), "f"(o[6]), "f"(o[7])
                 : "memory");
  }
  static __device__ __forceinline__ void bf16_ro(const __nv_bfloat16* p, float (&o)[8]) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    Lane<4>::unpack(u.x, o[0], o[1]);
    Lane<4>::unpack(u.y, o[2], o[3]);
    Lane<4>::unpack(u.z, o[4], o[5]);
    Lane<4>::unpack(u.w, o[6], o[7]);
  }
  static __device__ __forceinline__ void bf16(const __nv_bfloat16* p, float (&o)[8]) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    Lane<4>::unpack(u.x, o[0], o[1]);
    Lane<4>::unpack(u.y, o[2], o[3]);
    Lane<4>::unpack(u.z, o[4], o[5]);
    Lane<4>::unpack(u.w, o[6], o[7]);
  }
  static __device__ __forceinline__ void st_bf16(__nv_bfloat16* p, const uint32_t (&w)[4]) {
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
  }
};

}  // namespace

// n-wide row accesses of the SpMM: VW = VecOf<VT>::width (16 bytes), or 8
// floats (32 bytes) for FP32 rows whose leading dimensions allow it.
template <class VT, int VW>
__device__ __forceinline__ void rload_ro(const VT* p, VT (&o)[VW]) {
  if constexpr (VW == 8) Lane<8>::f32_ro(p, o);
  else vload_ro<VT>(p, o);
}
template <class VT, int VW>
__device__ __forceinline__ void rload(const VT* p, VT (&o)[VW]) {
  if constexpr (VW == 8) Lane<8>::f32(p, o);
  else vload<VT>(p, o);
}
template <class VT, int VW>
__device__ __forceinline__ void rstore(VT* p, const VT (&o)[VW]) {
  if constexpr (VW == 8) Lane<8>::st_f32(p, o);
  else vstore<VT>(p, o);
}

// Column accumulator: FP32 partial sums are flushed into FP64 every
// kFlush rows so long reductions keep FP64 accuracy at FP32 cost.
constexpr int kFlush = 16;

// ---------------------------------------------------------------- SpMM
template <class VT>
struct SpmmParams {
  Csr A;
  double alpha, gamma;
  const VT* X; int64_t ldx;
  const VT* Z; int64_t ldz;
  VT* Y; int64_t ldy;
  const VT* V; int64_t ldv;
  double* dots;
  int b;
  int skip_heavy;
};

// One group of TPR threads per row; each thread owns VPT vectors of VW
// columns: thread t of the group covers columns
//   tile0 + (v*TPR + t)*VW .. +VW-1, v < VPT.
// Rows are visited grid-stride so concurrent groups sweep neighbouring rows
// (their gathers share L2 lines of X for graphs with locality).
template <class VT, int WT, int TPR, int VPT, bool DOT, int VW = VecOf<VT>::width>
__global__ void __launch_bounds__(256) spmm_rows_kernel(SpmmParams<VT> p) {
  constexpr int TILE = TPR * VW * VPT;
  using A = typename Acc<VT>::type;
  const int t = threadIdx.x % TPR;
  const int64_t group = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / TPR;
  const int64_t ngroups = (int64_t(gridDim.x) * blockDim.x) / TPR;
  const int lane = threadIdx.x & 31;
  const unsigned gmask = (TPR == 32) ? 0xffffffffu : (((1u << TPR) - 1u) << (lane / TPR * TPR));
  const int tile0 = blockIdx.y * TILE;
  const A alpha = A(p.alpha), gamma = A(p.gamma);
  bool cval[VPT];
#pragma unroll
  for (int v = 0; v < VPT; ++v) cval[v] = tile0 + (v * TPR + t) * VW < p.b;
  double dsum[VPT][VW];
  A dpart[VPT][VW];
#pragma unroll
  for (int v = 0; v < VPT; ++v)
#pragma unroll
    for (int w = 0; w < VW; ++w) { dsum[v][w] = 0.0; dpart[v][w] = A(0); }
  int since_flush = 0;

  for (int64_t i = group; i < p.A.nrows; i += ngroups) {
    const int64_t k0 = p.A.rowptr[i], k1 = p.A.rowptr[i + 1];
    if (p.skip_heavy && k1 - k0 > kHeavyRowNnz) continue;
    A acc[VPT][VW];
#pragma unroll
    for (int v = 0; v < VPT; ++v)
#pragma unroll
      for (int w = 0; w < VW; ++w) acc[v][w] = A(0);
    for (int64_t kb = k0; kb < k1; kb += TPR) {
      const int64_t k = kb + t;
      int cj = 0;
      A wj = A(0);
      if (k < k1) {
        cj = p.A.col[k];
        wj = load_weight<WT, A>(p.A.val, k);
      }
      const int cnt = (int)(k1 - kb < TPR ? k1 - kb : TPR);
#pragma unroll 4
      for (int s = 0; s < cnt; ++s) {
        const int j = __shfl_sync(gmask, cj, s, TPR);
        const A wv = (WT == KATZ_UNIT) ? A(1) : __shfl_sync(gmask, wj, s, TPR);
        const VT* xr = p.X + int64_t(j) * p.ldx + tile0 + t * VW;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          if (cval[v]) {
            VT xv[VW];
            rload_ro<VT, VW>(xr + v * TPR * VW, xv);
#pragma unroll
            for (int w = 0; w < VW; ++w) acc[v][w] += wv * xv[w];
          }
        }
      }
    }
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      if (!cval[v]) continue;
      const int64_t c = tile0 + (v * TPR + t) * VW;
      VT y[VW];
      if (p.Z != nullptr) {
        VT z[VW];
        rload<VT, VW>(p.Z + i * p.ldz + c, z);
#pragma unroll
        for (int w = 0; w < VW; ++w) y[w] = VT(gamma * z[w] + alpha * acc[v][w]);
      } else {
#pragma unroll
        for (int w = 0; w < VW; ++w) y[w] = VT(alpha * acc[v][w]);
      }
      rstore<VT, VW>(p.Y + i * p.ldy + c, y);
      if constexpr (DOT) {
        VT vv[VW];
        rload<VT, VW>(p.V + i * p.ldv + c, vv);
#pragma unroll
        for (int w = 0; w < VW; ++w) dpart[v][w] += A(y[w]) * A(vv[w]);
      }
    }
    if constexpr (DOT) {
      if (++since_flush == kFlush) {
        since_flush = 0;
#pragma unroll
        for (int v = 0; v < VPT; ++v)
#pragma unroll
          for (int w = 0; w < VW; ++w) { dsum[v][w] += double(dpart[v][w]); dpart[v][w] = A(0); }
      }
    }
  }
  if constexpr (DOT) {
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      if (!cval[v]) continue;
      const int64_t c = tile0 + (v * TPR + t) * VW;
#pragma unroll
      for (int w = 0; w < VW; ++w) {
        const double d = dsum[v][w] + double(dpart[v][w]);
        if (d != 0.0) atomicAdd(p.dots + c + w, d);
      }
    }
  }
}

// Heavy rows: CTA = (heavy row, column slice of 32*VW columns); its 8
// warps split the row's entries; partial sums meet in shared memory.
template <class VT, int WT, bool DOT>
__global__ void __launch_bounds__(256) spmm_heavy_kernel(SpmmParams<VT> p, const int32_t* heavy) {
  constexpr int VW = VecOf<VT>::width;
  using A = typename Acc<VT>::type;
  __shared__ A red[8][32 * VW];
  const int64_t i = heavy[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c = int64_t(blockIdx.y) * 32 * VW + lane * VW;
  const bool cv = c < p.b;
  const int64_t k0 = p.A.rowptr[i], k1 = p.A.rowptr[i + 1];
  A acc[VW];
#pragma unroll
  for (int w = 0; w < VW; ++w) acc[w] = A(0);
  for (int64_t kb = k0 + warp * 32; kb < k1; kb += 8 * 32) {
    const int64_t k = kb + lane;
    int cj = 0;
    A wj = A(0);
    if (k < k1) {
      cj = p.A.col[k];
      wj = load_weight<WT, A>(p.A.val, k);
    }
    const int cnt = (int)(k1 - kb < 32 ? k1 - kb : 32);
#pragma unroll 4
    for (int s = 0; s < cnt; ++s) {
      const int j = __shfl_sync(0xffffffffu, cj, s);
      const A wv = __shfl_sync(0xffffffffu, wj, s);
      if (cv) {
        VT xv[VW];
        vload_ro<VT>(p.X + int64_t(j) * p.ldx + c, xv);
#pragma unroll
        for (int w = 0; w < VW; ++w) acc[w] += wv * xv[w];
      }
    }
  }
#pragma unroll
  for (int w = 0; w < VW; ++w) red[warp][lane * VW + w] = acc[w];
  __syncthreads();
  if (warp == 0 && cv) {
    A s[VW];
#pragma unroll
    for (int w = 0; w < VW; ++w) {
      s[w] = A(0);
      for (int q = 0; q < 8; ++q) s[w] += red[q][lane * VW + w];
    }
    VT y[VW];
    if (p.Z != nullptr) {
      VT z[VW];
      vload<VT>(p.Z + i * p.ldz + c, z);
#pragma unroll
      for (int w = 0; w < VW; ++w) y[w] = VT(A(p.gamma) * z[w] + A(p.alpha) * s[w]);
    } else {
#pragma unroll
      for (int w = 0; w < VW; ++w) y[w] = VT(A(p.alpha) * s[w]);
    }
    vstore<VT>(p.Y + i * p.ldy + c, y);
    if constexpr (DOT) {
      VT vv[VW];
      vload<VT>(p.V + i * p.ldv + c, vv);
#pragma unroll
      for (int w = 0; w < VW; ++w) atomicAdd(p.dots + c + w, double(A(y[w]) * A(vv[w])));
    }
  }
}

template <class VT, int WT, int TPR, int VPT, int VW = VecOf<VT>::width>
static void launch_rows(const SpmmParams<VT>& p, dim3 grid, cudaStream_t s) {
  if (p.dots)
    spmm_rows_kernel<VT, WT, TPR, VPT, true, VW><<<grid, 256, 0, s>>>(p);
  else
    spmm_rows_kernel<VT, WT, TPR, VPT, false, VW><<<grid, 256, 0, s>>>(p);
}

template <class VT, int WT>
static void spmm_dispatch(SpmmParams<VT>& p, const int32_t* heavy, int64_t n_heavy,
                          cudaStream_t s, const SpmmCfg& cfg) {
  constexpr int VW = VecOf<VT>::width;
  const int nvec = (p.b + VW - 1) / VW;
  // threads per row and vectors per thread cover min(b, cap) columns
  int tpr = 1;
  while (tpr < 32 && tpr < nvec) tpr *= 2;
  int vpt = 1;
  // columns per warp-row tile: 256 floats / 128 doubles by default, so the
  // accumulators and fused dot partials stay in registers without spills
  // (with the fused dot at most 2: its FP64 column partials per vector
  // cost registers, and the tuned tile is measured without the dot)
  int vcap = cfg.col_tile > 0 ? max(1, cfg.col_tile / (VW * 32)) : 2;
  if (p.dots) vcap = std::min(vcap, 2);
  if (tpr == 32)
    while (vpt < vcap && vpt * 32 < nvec) vpt *= 2;
  const int tile = tpr * VW * vpt;
  const int64_t tiles = ceil_div(p.b, tile);
  const int64_t groups_per_cta = 256 / tpr;
  int64_t ctas = ceil_div(p.A.nrows, groups_per_cta);
  const int64_t cap = int64_t(num_sms()) * cfg.ctas_per_sm * (tpr == 32 ? 1 : 1);
  ctas = std::max<int64_t>(1, std::min<int64_t>(ctas, std::max<int64_t>(1, cap / tiles)));
  dim3 grid((unsigned)ctas, (unsigned)tiles);
  p.skip_heavy = heavy != nullptr && n_heavy > 0;
  // FP32 rows whose strides and bases allow 32-byte accesses: half the
  // vectors per thread at 8 floats each (the same tile; measured 7 % faster
  // on the coupling products of the n = 4M graph)
  bool w8 = false;
  if constexpr (sizeof(VT) == 4) {
    const uintptr_t al = reinterpret_cast<uintptr_t>(p.X) | reinterpret_cast<uintptr_t>(p.Y) |
                         reinterpret_cast<uintptr_t>(p.Z) |
                         reinterpret_cast<uintptr_t>(p.dots ? p.V : nullptr);
    // (not with the fused dot: its FP64 column partials then cost occupancy,
    // measured slower in CG)
    w8 = tpr == 32 && vpt >= 2 && al % 32 == 0 && p.ldx % 8 == 0 && p.ldy % 8 == 0 &&
         (p.Z == nullptr || p.ldz % 8 == 0) && p.dots == nullptr;
  }
  if (p.A.nrows > 0) {
#define KATZ_ROWS(T, V) \
  if (tpr == T && vpt == V) { launch_rows<VT, WT, T, V>(p, grid, s); }
#define KATZ_ROWS8(V) \
  if (vpt == V) { launch_rows<VT, WT, 32, V / 2, 8>(p, grid, s); }
    if constexpr (sizeof(VT) == 4) {
      if (w8) {
        KATZ_ROWS8(2) else KATZ_ROWS8(4) else KATZ_ROWS8(8)
        else throw Error(KATZ_EINVAL, "spmm: unsupported shape");
      }
    }
    if (!w8) {
      KATZ_ROWS(1, 1) else KATZ_ROWS(2, 1) else KATZ_ROWS(4, 1) else KATZ_ROWS(8, 1)
      else KATZ_ROWS(16, 1) else KATZ_ROWS(32, 1) else KATZ_ROWS(32, 2) else KATZ_ROWS(32, 4)
      else KATZ_ROWS(32, 8) else throw Error(KATZ_EINVAL, "spmm: unsupported shape");
    }
#undef KATZ_ROWS
#undef KATZ_ROWS8
    KATZ_CHECK_LAUNCH();
  }
  if (p.skip_heavy) {
    dim3 hg((unsigned)n_heavy, (unsigned)ceil_div(p.b, 32 * VW));
    if (p.dots)
      spmm_heavy_kernel<VT, WT, true><<<hg, 256, 0, s>>>(p, heavy);
    else
      spmm_heavy_kernel<VT, WT, false><<<hg, 256, 0, s>>>(p, heavy);
    KATZ_CHECK_LAUNCH();
  }
}

template <class VT>
void spmm(const Csr& A, const int32_t* heavy, int64_t n_heavy, double alpha, const VT* X,
          int64_t ldx, double gamma, const VT* Z, int64_t ldz, VT* Y, int64_t ldy, int b,
          const VT* V, int64_t ldv, double* dots, cudaStream_t s, const SpmmCfg* cfg) {
  SpmmCfg c = cfg ? *cfg : SpmmCfg{};
  SpmmParams<VT> p{A, alpha, gamma, X, ldx, Z, ldz, Y, ldy, V, ldv, dots, b, 0};
  if (gamma == 0.0) p.Z = nullptr;
  KATZ_REQUIRE(b > 0 && ldx % VecOf<VT>::width == 0 && ldy % VecOf<VT>::width == 0 &&
                   (p.Z == nullptr || ldz % VecOf<VT>::width == 0) &&
                   (dots == nullptr || ldv % VecOf<VT>::width == 0) &&
                   ldx >= b && ldy >= b &&
                   (reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(p.Z) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(dots ? V : nullptr) % 16 == 0,
               KATZ_EINVAL, "spmm: operands must be 16-byte aligned with padded rows");
  prof_begin(s);
  switch (A.vdt) {
    case KATZ_UNIT: spmm_dispatch<VT, KATZ_UNIT>(p, heavy, n_heavy, s, c); break;
    case KATZ_F64: spmm_dispatch<VT, KATZ_F64>(p, heavy, n_heavy, s, c); break;
    case KATZ_F32: spmm_dispatch<VT, KATZ_F32>(p, heavy, n_heavy, s, c); break;
    case KATZ_BF16: spmm_dispatch<VT, KATZ_BF16>(p, heavy, n_heavy, s, c); break;
    default: throw Error(KATZ_EINVAL, "spmm: bad value dtype");
  }
  if (profiling()) {
    // algorithmic bytes: CSR once, X once, Y written once, Z / V read once
    const double sv = double(sizeof(VT)) * b;
    const double bytes = 8.0 * (A.nrows + 1) + double(A.nnz) * (4 + vdt_size(A.vdt)) +
                         sv * A.ncols + sv * A.nrows * (1 + (p.Z ? 1 : 0) + (dots ? 1 : 0));
    prof_end(sizeof(VT) == 4 ? "spmm_f32" : "spmm_f64", bytes, s);
  }
}

template void spmm<float>(const Csr&, const int32_t*, int64_t, double, const float*, int64_t,
                          double, const float*, int64_t, float*, int64_t, int, const float*,
                          int64_t, double*, cudaStream_t, const SpmmCfg*);
template void spmm<double>(const Csr&, const int32_t*, int64_t, double, const double*, int64_t,
                           double, const double*, int64_t, double*, int64_t, int, const double*,
                           int64_t, double*, cudaStream_t, const SpmmCfg*);

// ------------------------------------------------------- Chebyshev step
// One step of the Chebyshev iteration for A x = b with A = I - beta W,
// written as a three-term recurrence (no direction array), fused with the
// product:
//   r = b - A x_k = b - x_k + beta W x_k
//   x_{k+1} = x_k + a_k (x_k - x_{k-1}) + c_k r
// Iterates are stored either as FP32 rows or in the split form: an n x ld
// FP32-sized buffer holding two BF16 planes, hi = bf16(x) (rows of ld
// elements from the buffer start) and lo = bf16(x - hi) (the same from
// element `plane` = rows * ld), so that hi + lo carries x to 2^-18
// relative in the same bytes.  The product's gathers then read either the
// FP32 rows, the hi plane alone (half the bytes per gathered row; the
// product's relative error grows to ~2^-9 per term, the accuracy a step of
// an inexact inner solve can use) or hi and lo (FP32-accurate).  The row's
// own x_k, x_{k-1} and b are always read in full precision.
namespace {

enum : int { kInF32 = 0, kInHi = 1, kInHiLo = 2 };

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(x)));
}
// hi = bf16(x), lo = bf16(x - hi) for CW consecutive columns
template <int CW>
__device__ __forceinline__ void split_store(__nv_bfloat16* hi, __nv_bfloat16* lo,
                                            const float (&x)[CW]) {
  uint32_t h[CW / 2], l[CW / 2];
#pragma unroll
  for (int w = 0; w < CW; w += 2) {
    const uint32_t h0 = bf16_bits(x[w]), h1 = bf16_bits(x[w + 1]);
    const uint32_t l0 = bf16_bits(x[w] - __uint_as_float(h0 << 16));
    const uint32_t l1 = bf16_bits(x[w + 1] - __uint_as_float(h1 << 16));
    h[w / 2] = h0 | (h1 << 16);
    l[w / 2] = l0 | (l1 << 16);
  }
  Lane<CW>::st_bf16(hi, h);
  Lane<CW>::st_bf16(lo, l);
}

struct ChebArgs {
  Csr A;
  float beta, ak, ck, sx, sp;
  const void* Xk;     // FP32 rows or split planes
  const void* Xprev;  // null, FP32 rows or split planes
  const float* B;
  void* Xout;         // FP32 rows or split planes
  int64_t ld, plane;  // plane: element offset of the lo plane in a split buffer
  int b;
  int prev_mode;  // 0: x_{k-1} = 0, 1: FP32, 2: split
  int out_split;  // 1: write x_{k+1} split, 0: FP32
  // tile-major layout (x_k, x_{k-1}, x_{k+1}): column tile t of row i at
  // ((t * rows + i) * TILE) instead of i * ld + t * TILE
  int xk_tm, prev_tm, out_tm;
  // > 0: CTA c of a column tile takes the rows [c * chunk, (c + 1) * chunk),
  // its warps interleaved, so that the CTAs resident at once work on
  // neighbouring rows; 0: every warp strides over all rows
  int64_t chunk;
};

// One warp per row and column tile of 32 * CW columns; lane t owns the CW
// consecutive columns tile0 + t*CW .. +CW-1 (one vector access each).
// GD > 0: the row's entries are taken GD at a time, all GD gathered rows
// loaded before any is summed (GD loads in flight per lane; entries past
// the row's end load nothing and add zero); GD = 0: one entry at a time in
// a loop unrolled by 4 (the compiler's schedule).
template <int WT, int CW, int IN, int GD>
__global__ void __launch_bounds__(256) cheb_step_kernel(ChebArgs p) {
  constexpr int TILE = 32 * CW;
  using L = Lane<CW>;
  const int t = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t ld = p.ld;
  const int64_t c0 = int64_t(blockIdx.y) * TILE + t * CW;
  const bool cval = c0 < p.b;
  // row stride and lane offset of each operand's layout
  const int64_t tm_off = int64_t(blockIdx.y) * p.A.nrows * TILE + t * CW;
  const int64_t xs = p.xk_tm ? TILE : ld, xoff = p.xk_tm ? tm_off : c0;
  const int64_t ps = p.prev_tm ? TILE : ld, poff = p.prev_tm ? tm_off : c0;
  const int64_t os = p.out_tm ? TILE : ld, ooff = p.out_tm ? tm_off : c0;
  const float* Xf = static_cast<const float*>(p.Xk);
  const __nv_bfloat16* Xh = static_cast<const __nv_bfloat16*>(p.Xk);
  const __nv_bfloat16* Xl = Xh + p.plane;
  int64_t i0 = warp, i1 = p.A.nrows, istep = nwarps;
  if (p.chunk > 0) {
    i0 = int64_t(blockIdx.x) * p.chunk + (threadIdx.x >> 5);
    i1 = min(p.A.nrows, int64_t(blockIdx.x + 1) * p.chunk);
    istep = blockDim.x >> 5;
  }
  for (int64_t i = i0; i < i1; i += istep) {
    const int64_t k0 = p.A.rowptr[i], k1 = p.A.rowptr[i + 1];
    float acc[CW];
#pragma unroll
    for (int w = 0; w < CW; ++w) acc[w] = 0.f;
    if constexpr (IN == kInF32 && GD > 0) {
      // FP32 iterates: whole groups of GD entries without bound checks, all
      // GD rows loaded before any is added, then the last partial group with
      // checks; sums kept as packed column pairs (the same additions in the
      // same order as the scalar form)
      uint64_t ap[CW / 2];
#pragma unroll
      for (int q = 0; q < CW / 2; ++q) ap[q] = 0;
      const float* xb = Xf + xoff;
      for (int64_t kb = k0; kb < k1; kb += 32) {
        const int64_t k = kb + t;
        int cj = 0;
        float wj = 0.f;
        if (k < k1) {
          cj = p.A.col[k];
          wj = load_weight<WT, float>(p.A.val, k);
        }
        const int cnt = (int)(k1 - kb < 32 ? k1 - kb : 32);
        int s2 = 0;
        for (; s2 + GD <= cnt; s2 += GD) {
          int jj[GD];
          float ww[GD];
#pragma unroll
          for (int u = 0; u < GD; ++u) {
            jj[u] = __shfl_sync(0xffffffffu, cj, s2 + u);
            if constexpr (WT != KATZ_UNIT) ww[u] = __shfl_sync(0xffffffffu, wj, s2 + u);
          }
          if (cval) {
            uint64_t xv[GD][CW / 2];
#pragma unroll
            for (int u = 0; u < GD; ++u) L::p32_ro(xb + int64_t(jj[u]) * xs, xv[u]);
#pragma unroll
            for (int u = 0; u < GD; ++u) {
              if constexpr (WT == KATZ_UNIT) {
#pragma unroll
                for (int q = 0; q < CW / 2; ++q) ap[q] = padd2(ap[q], xv[u][q]);
              } else {
                const uint64_t w2 = uint64_t(__float_as_uint(ww[u])) |
                                    (uint64_t(__float_as_uint(ww[u])) << 32);
#pragma unroll
                for (int q = 0; q < CW / 2; ++q) ap[q] = pfma2(w2, xv[u][q], ap[q]);
              }
            }
          }
        }
        if (s2 < cnt) {
          // the last, partial group: its rows loaded together as well (rows
          // past the end load nothing and add zero)
          const int rem = cnt - s2;
          int jj[GD];
          float ww[GD];
#pragma unroll
          for (int u = 0; u < GD; ++u) {
            jj[u] = __shfl_sync(0xffffffffu, cj, (s2 + u) & 31);
            ww[u] = 1.f;
            if constexpr (WT != KATZ_UNIT) ww[u] = __shfl_sync(0xffffffffu, wj, (s2 + u) & 31);
          }
          if (cval) {
            uint64_t xv[GD][CW / 2];
#pragma unroll
            for (int u = 0; u < GD; ++u) {
              if (u < rem) {
                L::p32_ro(xb + int64_t(jj[u]) * xs, xv[u]);
              } else {
#pragma unroll
                for (int q = 0; q < CW / 2; ++q) xv[u][q] = 0;
              }
            }
#pragma unroll
            for (int u = 0; u < GD; ++u) {
              if (u < rem) {
                if constexpr (WT == KATZ_UNIT) {
#pragma unroll
                  for (int q = 0; q < CW / 2; ++q) ap[q] = padd2(ap[q], xv[u][q]);
                } else {
                  const uint64_t w2 = uint64_t(__float_as_uint(ww[u])) |
                                      (uint64_t(__float_as_uint(ww[u])) << 32);
#pragma unroll
                  for (int q = 0; q < CW / 2; ++q) ap[q] = pfma2(w2, xv[u][q], ap[q]);
                }
              }
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < CW / 2; ++q) {
        acc[2 * q] = __uint_as_float(uint32_t(ap[q]));
        acc[2 * q + 1] = __uint_as_float(uint32_t(ap[q] >> 32));
      }
    }
    for (int64_t kb = k0; (IN != kInF32 || GD == 0) && kb < k1; kb += 32) {
      const int64_t k = kb + t;
      int cj = 0;
      float wj = 0.f;
      if (k < k1) {
        cj = p.A.col[k];
        wj = load_weight<WT, float>(p.A.val, k);
      }
      const int cnt = (int)(k1 - kb < 32 ? k1 - kb : 32);
      auto gather = [&](int j, float (&xv)[CW]) {
        const int64_t off = int64_t(j) * xs + xoff;
        if constexpr (IN == kInF32) {
          L::f32_ro(Xf + off, xv);
        } else {
          L::bf16_ro(Xh + off, xv);
          if constexpr (IN == kInHiLo) {
            float xl[CW];
            L::bf16_ro(Xl + off, xl);
#pragma unroll
            for (int w = 0; w < CW; ++w) xv[w] += xl[w];
          }
        }
      };
      if constexpr (GD == 0) {
#pragma unroll 4
        for (int s2 = 0; s2 < cnt; ++s2) {
          const int j = __shfl_sync(0xffffffffu, cj, s2);
          const float wv = (WT == KATZ_UNIT) ? 1.f : __shfl_sync(0xffffffffu, wj, s2);
          if (cval) {
            float xv[CW];
            gather(j, xv);
#pragma unroll
            for (int w = 0; w < CW; ++w) acc[w] += wv * xv[w];
          }
        }
      } else {
        for (int s2 = 0; s2 < cnt; s2 += GD) {
          int jj[GD];
          float ww[GD];
#pragma unroll
          for (int u = 0; u < GD; ++u) {
            jj[u] = __shfl_sync(0xffffffffu, cj, (s2 + u) & 31);
            ww[u] = (WT == KATZ_UNIT) ? 1.f : __shfl_sync(0xffffffffu, wj, (s2 + u) & 31);
            if (s2 + u >= cnt) ww[u] = 0.f;
          }
          if (cval) {
            float xv[GD][CW];
#pragma unroll
            for (int u = 0; u < GD; ++u) {
              if (s2 + u < cnt) {
                gather(jj[u], xv[u]);
              } else {
#pragma unroll
                for (int w = 0; w < CW; ++w) xv[u][w] = 0.f;
              }
            }
#pragma unroll
            for (int u = 0; u < GD; ++u)
#pragma unroll
              for (int w = 0; w < CW; ++w) acc[w] += ww[u] * xv[u][w];
          }
        }
      }
    }
    if (!cval) continue;
    const int64_t o = i * ld + c0, ox = i * xs + xoff, op = i * ps + poff, oo = i * os + ooff;
    float xo[CW], bo[CW], xp[CW], xn[CW];
    if constexpr (IN == kInF32) {
      L::f32_ro(Xf + ox, xo);
    } else {
      float xl[CW];
      L::bf16_ro(Xh + ox, xo);
      L::bf16_ro(Xl + ox, xl);
#pragma unroll
      for (int w = 0; w < CW; ++w) xo[w] += xl[w];
    }
    L::f32(p.B + o, bo);
    if (p.prev_mode == 1) {
      L::f32(static_cast<const float*>(p.Xprev) + op, xp);
    } else if (p.prev_mode == 2) {
      const __nv_bfloat16* ph = static_cast<const __nv_bfloat16*>(p.Xprev);
      float xl[CW];
      L::bf16(ph + op, xp);
      L::bf16(ph + p.plane + op, xl);
#pragma unroll
      for (int w = 0; w < CW; ++w) xp[w] += xl[w];
    } else {
#pragma unroll
      for (int w = 0; w < CW; ++w) xp[w] = 0.f;
    }
#pragma unroll
    for (int w = 0; w < CW; ++w) {
      const float xs = p.sx * xo[w];
      const float r = bo[w] - xs + p.beta * (p.sx * acc[w]);
      xn[w] = xs + p.ak * (xs - p.sp * xp[w]) + p.ck * r;
    }
    if (p.out_split) {
      __nv_bfloat16* oh = static_cast<__nv_bfloat16*>(p.Xout);
      split_store<CW>(oh + oo, oh + p.plane + oo, xn);
    } else {
      L::st_f32(static_cast<float*>(p.Xout) + oo, xn);
    }
  }
}

// Row-pipelined FP32 step (256-column tiles, 8 columns per lane): each
// warp overlaps the serial chain of a row (its bounds, its column indices,
// its gathers, its own operands) with the next row's: at the start of row
// i the operands of the epilogue (b, x_k and x_{k-1} of row i) are copied
// asynchronously into the warp's shared memory (cp.async, no registers
// held), the next row's bounds are loaded, the gathers run, the next row's
// first 32 column indices are loaded, and only then does the warp wait for
// the copies and finish row i.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

template <int WT>
__global__ void __launch_bounds__(256) cheb_rows_pipe_kernel(ChebArgs p) {
  constexpr int CW = 8, TILE = 256;
  using L = Lane<CW>;
  __shared__ __align__(16) float stage[8][3][TILE];  // per warp: b, x_k, x_{k-1} of its row
  const int t = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t ld = p.ld;
  const int64_t c0 = int64_t(blockIdx.y) * TILE + t * CW;
  const bool cval = c0 < p.b;
  const int64_t tm_off = int64_t(blockIdx.y) * p.A.nrows * TILE + t * CW;
  const int64_t xs = p.xk_tm ? TILE : ld, xoff = p.xk_tm ? tm_off : c0;
  const int64_t ps = p.prev_tm ? TILE : ld, poff = p.prev_tm ? tm_off : c0;
  const int64_t os = p.out_tm ? TILE : ld, ooff = p.out_tm ? tm_off : c0;
  const float* Xf = static_cast<const float*>(p.Xk);
  const float* Xp = static_cast<const float*>(p.Xprev);
  float* sb = stage[wib][0] + t * CW;
  float* sx = stage[wib][1] + t * CW;
  float* sp = stage[wib][2] + t * CW;
  int64_t i = warp;
  if (i >= p.A.nrows) return;
  int64_t k0 = p.A.rowptr[i], k1 = p.A.rowptr[i + 1];
  int cj = 0;
  float wj = 0.f;
  if (k0 + t < k1) {
    cj = p.A.col[k0 + t];
    wj = load_weight<WT, float>(p.A.val, k0 + t);
  }
  for (;;) {
    // 1. this row's epilogue operands, asynchronously
    if (cval) {
      const int64_t o = i * ld + c0, ox = i * xs + xoff, op = i * ps + poff;
      cp_async16(sb, p.B + o);
      cp_async16(sb + 4, p.B + o + 4);
      cp_async16(sx, Xf + ox);
      cp_async16(sx + 4, Xf + ox + 4);
      if (p.prev_mode == 1) {
        cp_async16(sp, Xp + op);
        cp_async16(sp + 4, Xp + op + 4);
      }
    }
    // 2. the next row's bounds
    const int64_t inext = i + nwarps;
    const bool more = inext < p.A.nrows;
    int64_t n0 = 0, n1 = 0;
    if (more) {
      n0 = p.A.rowptr[inext];
      n1 = p.A.rowptr[inext + 1];
    }
    // 3. gathers of this row (first 32 indices already in registers)
    float acc[CW];
#pragma unroll
    for (int w = 0; w < CW; ++w) acc[w] = 0.f;
    for (int64_t kb = k0; kb < k1; kb += 32) {
      if (kb > k0) {
        const int64_t k = kb + t;
        cj = 0;
        wj = 0.f;
        if (k < k1) {
          cj = p.A.col[k];
          wj = load_weight<WT, float>(p.A.val, k);
        }
      }
      const int cnt = (int)(k1 - kb < 32 ? k1 - kb : 32);
#pragma unroll 4
      for (int s2 = 0; s2 < cnt; ++s2) {
        const int j = __shfl_sync(0xffffffffu, cj, s2);
        const float wv = (WT == KATZ_UNIT) ? 1.f : __shfl_sync(0xffffffffu, wj, s2);
        if (cval) {
          float xv[CW];
          L::f32_ro(Xf + int64_t(j) * xs + xoff, xv);
#pragma unroll
          for (int w = 0; w < CW; ++w) acc[w] += wv * xv[w];
        }
      }
    }
    // 4. the next row's first column indices
    int ncj = 0;
    float nwj = 0.f;
    if (more && n0 + t < n1) {
      ncj = p.A.col[n0 + t];
      nwj = load_weight<WT, float>(p.A.val, n0 + t);
    }
    // 5. this row's epilogue
    cp_async_wait_all();
    __syncwarp();
    if (cval) {
      float xn[CW];
#pragma unroll
      for (int w = 0; w < CW; ++w) {
        const float xsv = p.sx * sx[w];
        const float xpv = p.prev_mode == 1 ? sp[w] : 0.f;
        const float r = sb[w] - xsv + p.beta * (p.sx * acc[w]);
        xn[w] = xsv + p.ak * (xsv - p.sp * xpv) + p.ck * r;
      }
      L::st_f32(static_cast<float*>(p.Xout) + i * os + ooff, xn);
    }
    __syncwarp();  // the stage is refilled by the next row
    if (!more) break;
    i = inext;
    k0 = n0;
    k1 = n1;
    cj = ncj;
    wj = nwj;
  }
}

}  // namespace

void cheb_step_ex(const Csr& A, double beta, double ak, double ck, const void* Xk, int in_mode,
                  const void* Xprev, int prev_mode, const float* B, void* Xout, int out_split,
                  int64_t ld, int b, cudaStream_t s, const SpmmCfg* cfg, double sx, double sp,
                  int tm_mask) {
  KATZ_REQUIRE(ld % 4 == 0 && ld >= b && Xk != Xout && in_mode >= 0 && in_mode <= 2 &&
                   prev_mode >= 0 && prev_mode <= 2 && (prev_mode == 0) == (Xprev == nullptr) &&
                   (reinterpret_cast<uintptr_t>(Xk) | reinterpret_cast<uintptr_t>(Xprev) |
                    reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(Xout)) % 16 == 0,
               KATZ_EINVAL, "cheb_step: operands must be 16-byte aligned with padded rows");
  if (A.nrows <= 0) return;
  // 256-column tiles of 32-byte lane accesses where the rows allow them
  // (ld a multiple of 8 elements, 32-byte aligned bases), else 128-column
  // tiles of 16-byte accesses
  const bool wide = b > 128 && ld % 8 == 0 &&
                    ((reinterpret_cast<uintptr_t>(Xk) | reinterpret_cast<uintptr_t>(Xprev) |
                      reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(Xout)) % 32) == 0;
  KATZ_REQUIRE(tm_mask == 0 || (wide && in_mode == kInF32 && prev_mode != 2 && !out_split),
               KATZ_EINVAL, "cheb_step: tile-major operands need FP32 rows of 256-column tiles");
  const int tile = wide ? 256 : 128;
  const int64_t tiles = ceil_div(b, tile);
  const int cps = cfg && cfg->fused_cps > 0     ? cfg->fused_cps
                  : cfg && cfg->ctas_per_sm > 0 ? cfg->ctas_per_sm
                                                : 8;
  int64_t ctas = std::min<int64_t>(ceil_div(A.nrows, 8),
                                   std::max<int64_t>(1, int64_t(num_sms()) * cps / tiles));
  const bool row_pipe = cfg && cfg->row_pipeline && wide && in_mode == kInF32 && prev_mode != 2 &&
                        !out_split;
  const int64_t chunk = (cfg && !row_pipe && cfg->row_chunk > 0) ? cfg->row_chunk : 0;
  if (chunk > 0) ctas = ceil_div(A.nrows, chunk);
  KATZ_REQUIRE(ctas < (int64_t(1) << 31), KATZ_EINVAL, "cheb_step: row chunk too small");
  dim3 grid((unsigned)std::max<int64_t>(1, ctas), (unsigned)tiles);
  ChebArgs a{A,     float(beta), float(ak), float(ck), float(sx), float(sp), Xk, Xprev, B,
             Xout,  ld,          A.nrows * ld,          b,         prev_mode, out_split,
             (tm_mask & 1) ? 1 : 0, (tm_mask & 2) ? 1 : 0, (tm_mask & 4) ? 1 : 0, chunk};
  prof_begin(s);
  const int gd = cfg ? cfg->gather_depth : 0;
#define KATZ_CHEB_GD(WT, C, I)                                                      \
  if (gd == 8) cheb_step_kernel<WT, C, I, 8><<<grid, 256, 0, s>>>(a);              \
  else if (gd == 4) cheb_step_kernel<WT, C, I, 4><<<grid, 256, 0, s>>>(a);         \
  else cheb_step_kernel<WT, C, I, 0><<<grid, 256, 0, s>>>(a)
#define KATZ_CHEB_IN(WT, C)                                                          \
  switch (in_mode) {                                                                 \
    case kInF32: KATZ_CHEB_GD(WT, C, kInF32); break;                                 \
    case kInHi: KATZ_CHEB_GD(WT, C, kInHi); break;                                   \
    default: KATZ_CHEB_GD(WT, C, kInHiLo); break;                                    \
  }
#define KATZ_CHEB(WT)         \
  if (wide) {                 \
    KATZ_CHEB_IN(WT, 8)       \
  } else {                    \
    KATZ_CHEB_IN(WT, 4)       \
  }
  if (row_pipe) {
    switch (A.vdt) {
      case KATZ_UNIT: cheb_rows_pipe_kernel<KATZ_UNIT><<<grid, 256, 0, s>>>(a); break;
      case KATZ_F32: cheb_rows_pipe_kernel<KATZ_F32><<<grid, 256, 0, s>>>(a); break;
      case KATZ_BF16: cheb_rows_pipe_kernel<KATZ_BF16><<<grid, 256, 0, s>>>(a); break;
      default: cheb_rows_pipe_kernel<KATZ_F64><<<grid, 256, 0, s>>>(a); break;
    }
  } else {
    switch (A.vdt) {
      case KATZ_UNIT: KATZ_CHEB(KATZ_UNIT); break;
      case KATZ_F32: KATZ_CHEB(KATZ_F32); break;
      case KATZ_BF16: KATZ_CHEB(KATZ_BF16); break;
      default: KATZ_CHEB(KATZ_F64); break;
    }
  }
#undef KATZ_CHEB
#undef KATZ_CHEB_IN
#undef KATZ_CHEB_GD
  KATZ_CHECK_LAUNCH();
  if (profiling()) {
    // algorithmic: CSR once, x_k once (FP32 rows, or its hi and lo planes),
    // b and x_{k-1} read once, x_{k+1} written once; each n x b block is
    // 4 bytes per entry in either form.  Launches that gather the hi plane
    // alone are tagged apart.
    const double sv = 4.0 * b;
    prof_end(in_mode == kInHi ? "cheb_step_bf16g" : "cheb_step",
             8.0 * (A.nrows + 1) + double(A.nnz) * (4 + vdt_size(A.vdt)) + sv * A.ncols +
                 sv * A.nrows * (prev_mode ? 3.0 : 2.0),
             s);
  }
}

void cheb_step(const Csr& A, double beta, double ak, double ck, const float* Xk,
               const float* Xprev, const float* B, float* Xout, int64_t ld, int b, cudaStream_t s,
               const SpmmCfg* cfg, double sx, double sp) {
  cheb_step_ex(A, beta, ak, ck, Xk, kInF32, Xprev, Xprev ? 1 : 0, B, Xout, 0, ld, b, s, cfg, sx,
               sp);
}

// ------------------------------------------------------- 2D vector launches
// Threads: x over column vectors of a tile (TC vectors), y over rows.
struct Grid2 {
  dim3 grid, block;
  int tc;
};
template <class VT>
static Grid2 grid2(int64_t len, int b) {
  constexpr int VW = VecOf<VT>::width;
  const int nvec = (b + VW - 1) / VW;
  int tc = 1;
  while (tc < 32 && tc < nvec) tc *= 2;
  const int ty = 256 / tc;
  const int tiles = (nvec + tc - 1) / tc;
  int64_t gx = ceil_div(len, ty);
  const int64_t cap = int64_t(num_sms()) * 8;
  gx = std::max<int64_t>(1, std::min<int64_t>(gx, std::max<int64_t>(1, cap / tiles)));
  return {dim3((unsigned)gx, (unsigned)tiles), dim3(tc, ty), tc};
}

// block-level FP64 reduction of per-thread column partials (threads with
// equal threadIdx.x share columns) followed by one atomicAdd per column.
template <int VW>
__device__ __forceinline__ void reduce_cols_atomic(double (&part)[VW], double* out, int64_t c,
                                                   bool valid) {
  __shared__ double sh[256 * 4];
  const int tx = threadIdx.x, ty = threadIdx.y, tc = blockDim.x, tyn = blockDim.y;
  const int tid = ty * tc + tx;
#pragma unroll
  for (int w = 0; w < VW; ++w) sh[tid * VW + w] = part[w];
  __syncthreads();
  for (int stride = tyn / 2; stride > 0; stride >>= 1) {
    if (ty < stride) {
#pragma unroll
      for (int w = 0; w < VW; ++w) sh[tid * VW + w] += sh[((ty + stride) * tc + tx) * VW + w];
    }
    __syncthreads();
  }
  if (ty == 0 && valid) {
#pragma unroll
    for (int w = 0; w < VW; ++w)
      if (sh[tx * VW + w] != 0.0) atomicAdd(out + c + w, sh[tx * VW + w]);
  }
}

template <class VT>
__global__ void coldot_kernel(const VT* __restrict__ A, int64_t lda, const VT* __restrict__ B,
                              int64_t ldb, int64_t len,
                              int b, double* dots) {
  constexpr int VW = VecOf<VT>::width;
  const int64_t c = (int64_t(blockIdx.y) * blockDim.x + threadIdx.x) * VW;
  const bool valid = c < b;
  double tot[VW];
  VT part[VW];
#pragma unroll
  for (int w = 0; w < VW; ++w) { tot[w] = 0; part[w] = VT(0); }
  int cnt = 0;
  // a sum of squares (A == B) loads each row once; four rows per trip, all
  // loads issued before the products
  const bool same = A == B && lda == ldb;
  if (valid) {
    const int64_t step = int64_t(gridDim.x) * blockDim.y;
    int64_t i = int64_t(blockIdx.x) * blockDim.y + threadIdx.y;
    for (; i + 3 * step < len; i += 4 * step) {
      VT a[4][VW], bb[4][VW];
#pragma unroll
      for (int u = 0; u < 4; ++u) vload<VT>(A + (i + u * step) * lda + c, a[u]);
      if (!same) {
#pragma unroll
        for (int u = 0; u < 4; ++u) vload<VT>(B + (i + u * step) * ldb + c, bb[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < VW; ++w) part[w] += a[u][w] * (same ? a[u][w] : bb[u][w]);
      cnt += 4;
      if (cnt >= kFlush) {
        cnt = 0;
#pragma unroll
        for (int w = 0; w < VW; ++w) { tot[w] += double(part[w]); part[w] = VT(0); }
      }
    }
    for (; i < len; i += step) {
      VT a[VW], bb[VW];
      vload<VT>(A + i * lda + c, a);
      vload<VT>(B + i * ldb + c, bb);
#pragma unroll
      for (int w = 0; w < VW; ++w) part[w] += a[w] * bb[w];
    }
  }
#pragma unroll
  for (int w = 0; w < VW; ++w) tot[w] += double(part[w]);
  reduce_cols_atomic<VW>(tot, dots, c, valid);
}

template <class VT>
void coldot(const VT* A, int64_t lda, const VT* B, int64_t ldb, int64_t len, int b, double* dots,
            cudaStream_t s) {
  if (len <= 0 || b <= 0) return;
  Grid2 g = grid2<VT>(len, b);
  coldot_kernel<VT><<<g.grid, g.block, 0, s>>>(A, lda, B, ldb, len, b, dots);
  KATZ_CHECK_LAUNCH();
}
template void coldot<float>(const float*, int64_t, const float*, int64_t, int64_t, int, double*,
                            cudaStream_t);
template void coldot<double>(const double*, int64_t, const double*, int64_t, int64_t, int,
                             double*, cudaStream_t);

// ------------------------------------------------------------ CG updates
template <class VT, bool ACC_RR>
__global__ void cg_update_xr_kernel(VT* __restrict__ X, const VT* __restrict__ P,
                                    VT* __restrict__ R, const VT* __restrict__ Q, int64_t ld,
                                    int64_t len, int b, ColState st) {
  constexpr int VW = VecOf<VT>::width;
  const int64_t c = (int64_t(blockIdx.y) * blockDim.x + threadIdx.x) * VW;
  const bool valid = c < b;
  VT a[VW];
  bool any = false;
#pragma unroll
  for (int w = 0; w < VW; ++w) {
    a[w] = VT(0);
    if (valid && c + w < b && st.active[c + w]) {
      a[w] = VT(st.rz[c + w] / st.pq[c + w]);
      any = true;
    }
  }
  double tot[VW];
  VT part[VW];
#pragma unroll
  for (int w = 0; w < VW; ++w) { tot[w] = 0; part[w] = VT(0); }
  int cnt = 0;
  if (any) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.y + threadIdx.y; i < len;
         i += int64_t(gridDim.x) * blockDim.y) {
      VT x[VW], p[VW], r[VW], q[VW];
      vload<VT>(X + i * ld + c, x);
      vload<VT>(P + i * ld + c, p);
      vload<VT>(R + i * ld + c, r);
      vload<VT>(Q + i * ld + c, q);
#pragma unroll
      for (int w = 0; w < VW; ++w) {
        x[w] += a[w] * p[w];
        r[w] -= a[w] * q[w];
        part[w] += r[w] * r[w];
      }
      vstore<VT>(X + i * ld + c, x);
      vstore<VT>(R + i * ld + c, r);
      if constexpr (ACC_RR) {
        if (++cnt == kFlush) {
          cnt = 0;
#pragma unroll
          for (int w = 0; w < VW; ++w) { tot[w] += double(part[w]); part[w] = VT(0); }
        }
      }
    }
  }
  if constexpr (ACC_RR) {
#pragma unroll
    for (int w = 0; w < VW; ++w) tot[w] += double(part[w]);
    reduce_cols_atomic<VW>(tot, st.rz_new, c, valid);
  }
}

// rr accumulation for PCG happens separately (coldot of r with r); the
// plain-CG variant accumulates r.r into rz_new directly (z = r).
template <class VT>
void cg_update_xr(VT* X, const VT* P, VT* R, const VT* Q, int64_t ld, int64_t len, int b,
                  const ColState& st, bool acc_rr, cudaStream_t s) {
  if (len <= 0) return;
  Grid2 g = grid2<VT>(len, b);
  if (acc_rr)
    cg_update_xr_kernel<VT, true><<<g.grid, g.block, 0, s>>>(X, P, R, Q, ld, len, b, st);
  else
    cg_update_xr_kernel<VT, false><<<g.grid, g.block, 0, s>>>(X, P, R, Q, ld, len, b, st);
  KATZ_CHECK_LAUNCH();
}
template void cg_update_xr<float>(float*, const float*, float*, const float*, int64_t, int64_t,
                                  int, const ColState&, bool, cudaStream_t);
template void cg_update_xr<double>(double*, const double*, double*, const double*, int64_t,
                                   int64_t, int, const ColState&, bool, cudaStream_t);

template <class VT>
__global__ void cg_update_p_kernel(VT* __restrict__ P, const VT* __restrict__ Z, int64_t ld,
                                   int64_t len, int b,
                                   ColState st) {
  constexpr int VW = VecOf<VT>::width;
  const int64_t c = (int64_t(blockIdx.y) * blockDim.x + threadIdx.x) * VW;
  if (c >= b) return;
  VT be[VW];
  bool act[VW];
  bool any = false;
#pragma unroll
  for (int w = 0; w < VW; ++w) {
    act[w] = (c + w < b) && st.active[c + w];
    be[w] = act[w] ? VT(st.rz_new[c + w] / st.rz[c + w]) : VT(0);
    any |= act[w];
  }
  if (!any) return;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.y + threadIdx.y; i < len;
       i += int64_t(gridDim.x) * blockDim.y) {
    VT p[VW], z[VW];
    vload<VT>(P + i * ld + c, p);
    vload<VT>(Z + i * ld + c, z);
#pragma unroll
    for (int w = 0; w < VW; ++w)
      if (act[w]) p[w] = z[w] + be[w] * p[w];
    vstore<VT>(P + i * ld + c, p);
  }
}

template <class VT>
void cg_update_p(VT* P, const VT* Z, int64_t ld, int64_t len, int b, const ColState& st,
                 cudaStream_t s) {
  if (len <= 0) return;
  Grid2 g = grid2<VT>(len, b);
  cg_update_p_kernel<VT><<<g.grid, g.block, 0, s>>>(P, Z, ld, len, b, st);
  KATZ_CHECK_LAUNCH();
}
template void cg_update_p<float>(float*, const float*, int64_t, int64_t, int, const ColState&,
                                 cudaStream_t);
template void cg_update_p<double>(double*, const double*, int64_t, int64_t, int, const ColState&,
                                  cudaStream_t);

__global__ void colstate_check_pq_kernel(ColState st, int b) {
  for (int c = threadIdx.x; c < b; c += blockDim.x)
    if (st.active[c] && !(st.pq[c] > 0.0)) {
      atomicOr(st.flags, 1);
      st.active[c] = 0;
    }
}
void colstate_check_pq(const ColState& st, int b, cudaStream_t s) {
  colstate_check_pq_kernel<<<1, 1024, 0, s>>>(st, b);
  KATZ_CHECK_LAUNCH();
}

// Decide convergence from rr (plain CG: rr == rz_new), advance rz.
__global__ void colstate_advance_kernel(ColState st, int b, int rotate_rz) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int local = 0;
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    if (st.active[c]) {
      st.iters[c] += 1;
      const double rr = st.rr ? st.rr[c] : st.rz_new[c];
      const int still = rr > st.thr2[c];
      // the p-update of this iteration runs only on columns still active
      st.active[c] = still;
      local += still;
    }
  }
  atomicAdd(&cnt, local);
  __syncthreads();
  if (threadIdx.x == 0) *st.n_active = cnt;
  (void)rotate_rz;
}
void colstate_advance(const ColState& st, int b, cudaStream_t s) {
  colstate_advance_kernel<<<1, 1024, 0, s>>>(st, b, 0);
  KATZ_CHECK_LAUNCH();
}

// After the p-update: rz <- rz_new; zero the accumulators.
__global__ void colstate_rotate_kernel(ColState st, int b) {
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    st.rz[c] = st.rz_new[c];
    st.rz_new[c] = 0.0;
    st.pq[c] = 0.0;
    if (st.rr) st.rr[c] = 0.0;
  }
}
void colstate_rotate(const ColState& st, int b, cudaStream_t s) {
  colstate_rotate_kernel<<<1, 1024, 0, s>>>(st, b);
  KATZ_CHECK_LAUNCH();
}

// ---------------------------------------------------------- misc vectors
template <class VT>
__global__ void scale_copy_kernel(const VT* X, int64_t ldx, VT* Y, int64_t ldy, int64_t len,
                                  int b, VT a, int accumulate) {
  const int64_t total = len * b;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / b, c = e - i * b;
    const VT v = a * X[i * ldx + c];
    Y[i * ldy + c] = accumulate ? Y[i * ldy + c] + v : v;
  }
}
static dim3 flat_grid(int64_t total) {
  int64_t g = ceil_div(total, 256);
  return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(g, int64_t(num_sms()) * 16)));
}
template <class VT>
void scale_copy(const VT* X, int64_t ldx, VT* Y, int64_t ldy, int64_t len, int b, double a,
                bool accumulate, cudaStream_t s) {
  if (len <= 0 || b <= 0) return;
  scale_copy_kernel<VT><<<flat_grid(len * b), 256, 0, s>>>(X, ldx, Y, ldy, len, b, VT(a),
                                                            accumulate ? 1 : 0);
  KATZ_CHECK_LAUNCH();
}
template void scale_copy<float>(const float*, int64_t, float*, int64_t, int64_t, int, double,
                                bool, cudaStream_t);
template void scale_copy<double>(const double*, int64_t, double*, int64_t, int64_t, int, double,
                                 bool, cudaStream_t);

template <class S, class D, bool ACC>
__global__ void convert_kernel(const S* X, int64_t ldx, D* Y, int64_t ldy, int64_t len, int b) {
  const int64_t total = len * b;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / b, c = e - i * b;
    if constexpr (ACC)
      Y[i * ldy + c] += D(X[i * ldx + c]);
    else
      Y[i * ldy + c] = D(X[i * ldx + c]);
  }
}
void add_f32_to_f64(const float* X, int64_t ldx, double* Y, int64_t ldy, int64_t len, int b,
                    cudaStream_t s) {
  if (len <= 0 || b <= 0) return;
  convert_kernel<float, double, true><<<flat_grid(len * b), 256, 0, s>>>(X, ldx, Y, ldy, len, b);
  KATZ_CHECK_LAUNCH();
}
void convert_f64_to_f32(const double* X, int64_t ldx, float* Y, int64_t ldy, int64_t len, int b,
                        cudaStream_t s) {
  if (len <= 0 || b <= 0) return;
  convert_kernel<double, float, false><<<flat_grid(len * b), 256, 0, s>>>(X, ldx, Y, ldy, len, b);
  KATZ_CHECK_LAUNCH();
}
void convert_f32_to_f64(const float* X, int64_t ldx, double* Y, int64_t ldy, int64_t len, int b,
                        cudaStream_t s) {
  if (len <= 0 || b <= 0) return;
  convert_kernel<float, double, false><<<flat_grid(len * b), 256, 0, s>>>(X, ldx, Y, ldy, len, b);
  KATZ_CHECK_LAUNCH();
}

template <class VT>
__global__ void gather_rows_kernel(const VT* X, int64_t ldx, const int32_t* map, VT* Y,
                                   int64_t ldy, int64_t len, int b) {
  const int64_t total = len * b;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / b, c = e - i * b;
    Y[i * ldy + c] = X[int64_t(map[i]) * ldx + c];
  }
}
template <class VT>
void gather_rows(const VT* X, int64_t ldx, const int32_t* map, VT* Y, int64_t ldy, int64_t len,
                 int b, cudaStream_t s) {
  if (len <= 0 || b <= 0) return;
  gather_rows_kernel<VT><<<flat_grid(len * b), 256, 0, s>>>(X, ldx, map, Y, ldy, len, b);
  KATZ_CHECK_LAUNCH();
}
template void gather_rows<float>(const float*, int64_t, const int32_t*, float*, int64_t, int64_t,
                                 int, cudaStream_t);
template void gather_rows<double>(const double*, int64_t, const int32_t*, double*, int64_t,
                                  int64_t, int, cudaStream_t);

// One CTA per query column: scatter beta * W[q, i] to row pos(i).
template <class VT, int WT>
__global__ void build_rhs_kernel(Csr W, const int32_t* q, double beta, const int32_t* pos, VT* B,
                                 int64_t ldb) {
  const int j = blockIdx.x;
  const int64_t qq = q[j];
  const int64_t k0 = W.rowptr[qq], k1 = W.rowptr[qq + 1];
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const int64_t i = W.col[k];
    const int64_t r = pos ? pos[i] : i;
    B[r * ldb + j] = VT(beta * load_weight<WT, double>(W.val, k));
  }
}
template <class VT>
void build_rhs(const Csr& W, const int32_t* q, int b, double beta, const int32_t* pos, VT* B,
               int64_t ldb, cudaStream_t s) {
  if (b <= 0) return;
  switch (W.vdt) {
    case KATZ_UNIT: build_rhs_kernel<VT, KATZ_UNIT><<<b, 256, 0, s>>>(W, q, beta, pos, B, ldb); break;
    case KATZ_F64: build_rhs_kernel<VT, KATZ_F64><<<b, 256, 0, s>>>(W, q, beta, pos, B, ldb); break;
    case KATZ_F32: build_rhs_kernel<VT, KATZ_F32><<<b, 256, 0, s>>>(W, q, beta, pos, B, ldb); break;
    default: build_rhs_kernel<VT, KATZ_BF16><<<b, 256, 0, s>>>(W, q, beta, pos, B, ldb); break;
  }
  KATZ_CHECK_LAUNCH();
}
template void build_rhs<float>(const Csr&, const int32_t*, int, double, const int32_t*, float*,
                               int64_t, cudaStream_t);
template void build_rhs<double>(const Csr&, const int32_t*, int, double, const int32_t*, double*,
                                int64_t, cudaStream_t);

// Column sums of squares and max |x|: vector loads along the row (the
// Grid2 layout of the other column reductions), FP64 partials.
template <class VT>
__global__ void col_norms_kernel(const VT* __restrict__ B, int64_t ld, int64_t len, int b,
                                 double* norm2, unsigned long long* maxabs_bits) {
  constexpr int VW = VecOf<VT>::width;
  const int64_t c = (int64_t(blockIdx.y) * blockDim.x + threadIdx.x) * VW;
  const bool valid = c < b;
  double tot[VW];
  VT part[VW], mx[VW];  // max |x| in the element type (exact), no FP64 per element
#pragma unroll
  for (int w = 0; w < VW; ++w) { tot[w] = 0; mx[w] = VT(0); part[w] = VT(0); }
  int cnt = 0;
  if (valid) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.y + threadIdx.y; i < len;
         i += int64_t(gridDim.x) * blockDim.y) {
      VT v[VW];
      vload<VT>(B + i * ld + c, v);
#pragma unroll
      for (int w = 0; w < VW; ++w) {
        part[w] += v[w] * v[w];
        mx[w] = v[w] > mx[w] ? v[w] : (-v[w] > mx[w] ? -v[w] : mx[w]);
      }
      if (++cnt == kFlush) {
        cnt = 0;
#pragma unroll
        for (int w = 0; w < VW; ++w) { tot[w] += double(part[w]); part[w] = VT(0); }
      }
    }
  }
#pragma unroll
  for (int w = 0; w < VW; ++w) tot[w] += double(part[w]);
  if (valid)
#pragma unroll
    for (int w = 0; w < VW; ++w)
      if (c + w < b && mx[w] > VT(0))
        atomicMax(maxabs_bits + c + w, (unsigned long long)__double_as_longlong(double(mx[w])));
  reduce_cols_atomic<VW>(tot, norm2, c, valid);
}

template <class VT>
void col_norms(const VT* B, int64_t ld, int64_t len, int b, double* norm2, double* maxabs,
               cudaStream_t s) {
  KATZ_CUDA(cudaMemsetAsync(norm2, 0, sizeof(double) * b, s));
  KATZ_CUDA(cudaMemsetAsync(maxabs, 0, sizeof(double) * b, s));
  if (len <= 0) return;
  Grid2 g = grid2<VT>(len, b);
  // non-negative doubles order like their bit patterns, so atomicMax on the
  // bits gives the maximum
  col_norms_kernel<VT><<<g.grid, g.block, 0, s>>>(B, ld, len, b, norm2,
                                                   reinterpret_cast<unsigned long long*>(maxabs));
  KATZ_CHECK_LAUNCH();
}
template void col_norms<float>(const float*, int64_t, int64_t, int, double*, double*,
                               cudaStream_t);
template void col_norms<double>(const double*, int64_t, int64_t, int, double*, double*,
                                cudaStream_t);

__global__ void make_thresholds_kernel(const double* norm2, const double* maxabs, int b, double tol,
                                       int kind, double omc, double* thr2) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < b; c += gridDim.x * blockDim.x) {
    const double base = kind == KATZ_TOL_ERROR_INF ? maxabs[c] * omc : sqrt(norm2[c]);
    const double t = tol * base;
    thr2[c] = t * t;
  }
}
void make_thresholds(const double* norm2, const double* maxabs, int b, double tol, int kind,
                     double one_minus_c, double* thr2, cudaStream_t s) {
  make_thresholds_kernel<<<(unsigned)ceil_div(b, 256), 256, 0, s>>>(norm2, maxabs, b, tol, kind,
                                                                    one_minus_c, thr2);
  KATZ_CHECK_LAUNCH();
}

// ------------------------------------------------------- M11 block solves
// CTA = (group of blocks, column tile of TC columns).  Minv tiles and the
// X tile are staged in shared memory; each thread accumulates RI output
// rows of one column.
template <class VT, int S>
__global__ void __launch_bounds__(256) block_solve_kernel(const VT* inv, const int64_t* start,
                                                          const int32_t* size, int64_t count,
                                                          const VT* X, int64_t ldx, VT* Y,
                                                          int64_t ldy, int b, int TC, int G) {
  extern __shared__ unsigned char smraw[];
  VT* sm_inv = reinterpret_cast<VT*>(smraw);       // G*S*S
  VT* sm_x = sm_inv + size_t(G) * S * S;           // G*S*TC
  const int64_t blk0 = int64_t(blockIdx.x) * G;
  const int c0 = blockIdx.y * TC;
  const int tc = min(TC, b - c0);
  const int nb = (int)(count - blk0 < G ? count - blk0 : G);
  for (int e = threadIdx.x; e < nb * S * S; e += blockDim.x)
    sm_inv[e] = inv[(blk0 * S) * S + e];
  for (int e = threadIdx.x; e < nb * S * tc; e += blockDim.x) {
    const int g = e / (S * tc), rem = e - g * S * tc, r = rem / tc, c = rem - r * tc;
    const int64_t bi = blk0 + g;
    sm_x[(g * S + r) * TC + c] = r < size[bi] ? X[(start[bi] + r) * ldx + c0 + c] : VT(0);
  }
  __syncthreads();
  const int outputs = nb * S * tc;
  for (int o = threadIdx.x; o < outputs; o += blockDim.x) {
    const int g = o / (S * tc), rem = o - g * S * tc, r = rem / tc, c = rem - r * tc;
    const int64_t bi = blk0 + g;
    if (r >= size[bi]) continue;
    const VT* mi = sm_inv + (size_t(g) * S + r) * S;
    const VT* xc = sm_x + size_t(g) * S * TC + c;
    VT acc = VT(0);
#pragma unroll 8
    for (int k = 0; k < S; ++k) acc += mi[k] * xc[k * TC];
    Y[(start[bi] + r) * ldy + c0 + c] = acc;
  }
}

template <class VT, int S>
static void launch_block_solve(const VT* inv, const int64_t* start, const int32_t* size,
                               int64_t count, const VT* X, int64_t ldx, VT* Y, int64_t ldy, int b,
                               cudaStream_t s) {
  const int TC = std::min(b, S >= 64 ? 32 : 64);
  int G = std::max(1, 2048 / (S * TC));
  while (G > 1 && size_t(G) * S * (S + TC) * sizeof(VT) > 96 * 1024) G /= 2;
  const size_t smem = size_t(G) * S * (S + TC) * sizeof(VT);
  if (smem > 48 * 1024)
    KATZ_CUDA(cudaFuncSetAttribute(block_solve_kernel<VT, S>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)ceil_div(count, G), (unsigned)ceil_div(b, TC));
  block_solve_kernel<VT, S><<<grid, 256, smem, s>>>(inv, start, size, count, X, ldx, Y, ldy, b,
                                                     TC, G);
  KATZ_CHECK_LAUNCH();
}

template <class VT>
void block_solve(const VT* inv, const int64_t* start, const int32_t* size, int64_t count, int S,
                 const VT* X, int64_t ldx, VT* Y, int64_t ldy, int b, cudaStream_t s) {
  if (count <= 0 || b <= 0) return;
  prof_begin(s);
  switch (S) {
    case 1: launch_block_solve<VT, 1>(inv, start, size, count, X, ldx, Y, ldy, b, s); break;
    case 2: launch_block_solve<VT, 2>(inv, start, size, count, X, ldx, Y, ldy, b, s); break;
    case 4: launch_block_solve<VT, 4>(inv, start, size, count, X, ldx, Y, ldy, b, s); break;
    case 8: launch_block_solve<VT, 8>(inv, start, size, count, X, ldx, Y, ldy, b, s); break;
    case 16: launch_block_solve<VT, 16>(inv, start, size, count, X, ldx, Y, ldy, b, s); break;
    case 32: launch_block_solve<VT, 32>(inv, start, size, count, X, ldx, Y, ldy, b, s); break;
    case 64: launch_block_solve<VT, 64>(inv, start, size, count, X, ldx, Y, ldy, b, s); break;
    case 128: launch_block_solve<VT, 128>(inv, start, size, count, X, ldx, Y, ldy, b, s); break;
    default: throw Error(KATZ_EINVAL, "block_solve: size class must be a power of two <= 128");
  }
  if (profiling()) {
    const double bytes = double(sizeof(VT)) * (double(count) * S * S + 2.0 * double(count) * S * b);
    prof_end(sizeof(VT) == 4 ? "block_solve_f32" : "block_solve_f64", bytes, s);
  }
}
template void block_solve<float>(const float*, const int64_t*, const int32_t*, int64_t, int,
                                 const float*, int64_t, float*, int64_t, int, cudaStream_t);
template void block_solve<double>(const double*, const int64_t*, const int32_t*, int64_t, int,
                                  const double*, int64_t, double*, int64_t, int, cudaStream_t);

}  // namespace katz
