// Pipelined row-gather kernels (see gather_pipe.h).
//
// Work unit: a row block (at most 31 consecutive rows, about 512 stored
// entries), handed out in increasing order by a global atomic counter, so
// the rows in flight on all SMs at any moment lie in a narrow window of the
// row order (the rows they gather share L2) and heavy rows balance
// themselves across SMs.
//
// Per CTA: one producer warp and tw/128 consumer warps (4 columns a lane).
//   entry ring: S slots; slot (position mod S) holds X[col[e]][tile] of the
//     e-th stored entry the CTA processes, and its weight; barriers "full"
//     (one arrive with the byte count, completed by the bulk copy) and
//     "empty" (one arrive per consumer warp);
//   head ring: HS stages, one row each: its id and entry count (written by
//     the producer, published by the "meta" barrier) and the row's own
//     operands (NH tile rows on the stage's "full" barrier); "empty" barrier.
// The producer issues rows in order (head, then entries) and only waits for
// slots and stages released by rows it issued earlier, so the pipeline
// cannot deadlock; block ids, block bounds and the first row-pointer and
// column windows of the next blocks are fetched three blocks ahead so that
// their latency hides behind the current block.
#include <algorithm>

#include "gather_pipe.h"

namespace katz {

namespace {

constexpr int kBatch = 8;         // stored entries a consumer warp takes per wait
constexpr int kMaxThreads = 544;  // producer warp + at most 16 consumer warps
constexpr int kBlockRows = 31;    // rows per block (row pointers fit one warp register)
constexpr int64_t kBlockWeight = 512;  // stored entries + 4 per row, per block
constexpr int kMaxTiles = 8;
constexpr int kMaxSlots = 256;
constexpr int kSmemBudget = 220 * 1024;
constexpr uint64_t kTimeoutNs = 2000000000ull;  // bound on every wait

enum { kCheb2 = 0, kCheb3 = 1, kResInit = 2 };
__host__ __device__ constexpr int n_heads(int mode) {
  return mode == kCheb2 ? 2 : mode == kCheb3 ? 3 : 1;
}

struct PipeArgs {
  Csr A;
  const int64_t* bstart;  // row blocks [bstart[k], bstart[k+1])
  const int64_t* bentry;  // rowptr[bstart[k]]
  int64_t nblocks;
  int* ctr;               // block counters, one per column tile (zeroed per launch)
  int64_t ld;
  int tw, nslots, hstages, ngroups, nwg, chunk;
  const float* X;
  const float* H[3];
  float* O[2];
  float beta, beh, bel, ak, ck, sx, sp;
  double* rr;
  int b;
  int* err;
};

// bytes of barriers and per-stage / per-slot metadata ahead of the rings
__host__ __device__ constexpr uint32_t pipe_meta_bytes(int S, int HS) {
  return (8u * (2 * S + 3 * HS) + 8u * HS + 8u * HS + 8u * S + 127u) & ~127u;
}

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool bar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait of one thread: false on timeout or when the CTA aborted.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, const volatile int* abort) {
  if (bar_test(bar, parity)) return true;
  const uint64_t t0 = gtime();
  while (!bar_try(bar, parity)) {
    if ((abort && *abort) || gtime() - t0 > kTimeoutNs) return false;
  }
  return true;
}
// Wait for the copy of stream position P into a slot: the slot's tag must
// name P (the producer tags a slot before arming its barrier) before the
// phase parity is trusted, since a consumer group may reach a slot while an
// earlier occupant, owned by another group, is still in flight.
__device__ __forceinline__ bool slot_wait(uint32_t bar, uint32_t parity, const volatile uint32_t* tag,
                                          uint32_t P, const volatile int* abort) {
  if (*tag == P && bar_test(bar, parity)) return true;
  const uint64_t t0 = gtime();
  for (;;) {
    if (*tag == P && bar_try(bar, parity)) return true;
    if (*abort || gtime() - t0 > kTimeoutNs) return false;
  }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

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
__device__ __forceinline__ float load_w(const void* val, int64_t k) {
  if constexpr (WT == KATZ_F32) return __ldg(static_cast<const float*>(val) + k);
  else return __bfloat162float(static_cast<const __nv_bfloat16*>(val)[k]);
}

// acc += w * x (float-float; w * x exact through FMA)
template <bool UNIT>
__device__ __forceinline__ void ff_acc(FF& acc, float w, float x) {
  if constexpr (UNIT) {
    const FF s = two_sum(acc.hi, x);
    acc.hi = s.hi;
    acc.lo += s.lo;
  } else {
    const float p = w * x;
    const float pe = __fmaf_rn(w, x, -p);
    const FF s = two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo += s.lo + pe;
  }
}

// Bounds of one row block; rs < 0 past the last block.
struct Blk {
  int64_t rs, re, es, ee;
};
__device__ __forceinline__ Blk blk_bounds(const PipeArgs& a, int64_t k) {
  Blk b;
  if (k < a.nblocks) {
    b.rs = a.bstart[k];
    b.re = a.bstart[k + 1];
    b.es = a.bentry[k];
    b.ee = a.bentry[k + 1];
  } else {
    b.rs = b.re = -1;
    b.es = b.ee = 0;
  }
  return b;
}
// Register windows of a block: lane l holds rowptr[rs + l] (l <= rows) and
// the column ids / weights of entries es + l and es + 32 + l.
struct Win {
  int64_t rp;
  int cw, cn;
  float wv, wn;
};
template <int WT>
__device__ __forceinline__ Win blk_windows(const PipeArgs& a, const Blk& b, int lane) {
  Win w;
  w.rp = (b.rs >= 0 && lane <= b.re - b.rs) ? a.A.rowptr[b.rs + lane] : 0;
  w.cw = (b.es + lane < b.ee) ? a.A.col[b.es + lane] : 0;
  w.cn = (b.es + 32 + lane < b.ee) ? a.A.col[b.es + 32 + lane] : 0;
  w.wv = w.wn = 1.f;
  if constexpr (WT != KATZ_UNIT) {
    w.wv = (b.es + lane < b.ee) ? load_w<WT>(a.A.val, b.es + lane) : 0.f;
    w.wn = (b.es + 32 + lane < b.ee) ? load_w<WT>(a.A.val, b.es + 32 + lane) : 0.f;
  }
  return w;
}

// One stored entry of a consumer lane: acc += w * x over its 4 columns,
// float-float (FFSUM, into af) or FP32 (into acc).
template <bool FFSUM, bool UNIT>
__device__ __forceinline__ void take(const unsigned char* src, float w, float (&acc)[4],
                                     FF (&af)[4]) {
  const float4 x = *reinterpret_cast<const float4*>(src);
  if constexpr (FFSUM) {
    ff_acc<UNIT>(af[0], w, x.x);
    ff_acc<UNIT>(af[1], w, x.y);
    ff_acc<UNIT>(af[2], w, x.z);
    ff_acc<UNIT>(af[3], w, x.w);
  } else {
    acc[0] = __fmaf_rn(w, x.x, acc[0]);
    acc[1] = __fmaf_rn(w, x.y, acc[1]);
    acc[2] = __fmaf_rn(w, x.z, acc[2]);
    acc[3] = __fmaf_rn(w, x.w, acc[3]);
  }
}

template <int MODE, int WT>
__global__ void __launch_bounds__(kMaxThreads, 1) pipe_kernel(const __grid_constant__ PipeArgs a) {
  constexpr int NH = n_heads(MODE);
  constexpr bool RES = MODE >= kResInit;
  constexpr bool UNIT = WT == KATZ_UNIT;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int abort_flag;
  const int S = a.nslots, HS = a.hstages, NG = a.ngroups, NWG = a.nwg;
  // barriers; per head stage: row id, entry count, ring position of the
  // first entry; per slot: weight; then the two rings
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  int64_t* hrow = reinterpret_cast<int64_t*>(bars + 2 * S + 3 * HS);
  int* hdeg = reinterpret_cast<int*>(hrow + HS);
  uint32_t* hpos = reinterpret_cast<uint32_t*>(hdeg + HS);  // stream position of the first entry
  float* wring = reinterpret_cast<float*>(hpos + HS);
  uint32_t* tag = reinterpret_cast<uint32_t*>(wring + S);  // stream position a slot holds
  const uint32_t meta_bytes = pipe_meta_bytes(S, HS);
  const uint32_t full0 = su32(smem), empty0 = full0 + 8u * S, hmeta0 = empty0 + 8u * S,
                 hfull0 = hmeta0 + 8u * HS, hempty0 = hfull0 + 8u * HS;
  const uint32_t RS = uint32_t(a.tw) * 4u;  // slot stride (bytes)
  const uint32_t ring = full0 + meta_bytes, hring = ring + uint32_t(S) * RS;
  const unsigned char* ring_p = smem + meta_bytes;
  const unsigned char* hring_p = ring_p + size_t(S) * RS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int i = 0; i < S; ++i) {
      bar_init(full0 + 8u * i, 1);
      bar_init(empty0 + 8u * i, NWG);
    }
    for (int i = 0; i < HS; ++i) {
      bar_init(hmeta0 + 8u * i, 1);
      bar_init(hfull0 + 8u * i, 1);
      bar_init(hempty0 + 8u * i, NWG);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t tile0 = int64_t(blockIdx.y) * a.tw;
  const int twc = int(a.ld - tile0 < a.tw ? a.ld - tile0 : a.tw);
  const uint32_t RB = uint32_t(twc) * 4u;  // bytes copied per tile row
  volatile int* abort = &abort_flag;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    const int CH = a.chunk;  // entries issued per step (<= 32, <= S)
    int* ctr = a.ctr + blockIdx.y;
    int kA = (lane == 0) ? atomicAdd(ctr, 1) : 0;
    Blk cB = blk_bounds(a, __shfl_sync(FULL, kA, 0));
    Win cW = blk_windows<WT>(a, cB, lane);
    kA = (lane == 0) ? atomicAdd(ctr, 1) : 0;
    Blk sB = blk_bounds(a, __shfl_sync(FULL, kA, 0));
    kA = (lane == 0) ? atomicAdd(ctr, 1) : 0;
    int64_t p = 0, hp = 0;     // entries / rows issued
    int pslot = 0, hslot = 0;  // p mod S, hp mod HS
    uint32_t pround = 0, hround = 0;
    bool ok = true;
    for (;;) {
      // rotate the look-ahead: current <- (cB, cW) <- (sB, its windows) <- bounds(kA) <- next id
      const Blk cur = cB;
      Win w = cW;
      if (cur.rs < 0) break;
      cB = sB;
      cW = blk_windows<WT>(a, cB, lane);
      sB = blk_bounds(a, __shfl_sync(FULL, kA, 0));
      kA = (lane == 0) ? atomicAdd(ctr, 1) : 0;
      int64_t wb = cur.es;  // window base: cw covers entries wb..wb+31, cn the next 32
      const int nr = int(cur.re - cur.rs);
      for (int r = 0; r < nr && ok; ++r) {
        const int64_t i = cur.rs + r;
        const int64_t e0 = __shfl_sync(FULL, w.rp, r), e1 = __shfl_sync(FULL, w.rp, r + 1);
        if (hround > 0) {
          ok = __all_sync(FULL, bar_wait(hempty0 + 8u * hslot, (hround - 1) & 1, abort));
          if (!ok) break;
        }
        if (lane == 0) {
          hrow[hslot] = i;
          hdeg[hslot] = int(e1 - e0);
          hpos[hslot] = uint32_t(p);
          bar_arrive(hmeta0 + 8u * hslot);
          bar_expect(hfull0 + 8u * hslot, NH * RB);
        }
        __syncwarp();
        if (lane < NH)
          bulk_g2s(hring + uint32_t(hslot * NH + lane) * RS, a.H[lane] + i * a.ld + tile0, RB,
                   hfull0 + 8u * hslot);
        ++hp;
        if (++hslot == HS) {
          hslot = 0;
          ++hround;
        }
        for (int64_t e = e0; e < e1;) {
          const int c = int(e1 - e < CH ? e1 - e : CH);
          const bool mine = lane < c;
          int slot = pslot + lane;
          uint32_t rd = pround;
          if (slot >= S) {  // lanes < c <= S wrap at most once
            slot -= S;
            ++rd;
          }
          ok = __all_sync(FULL, !mine || rd == 0 || bar_wait(empty0 + 8u * slot, (rd - 1) & 1, abort));
          if (!ok) break;
          const int idx = int(e - wb) + lane;  // < 64: e - wb < 32 at every step
          const int jw = __shfl_sync(FULL, w.cw, idx & 31), jn = __shfl_sync(FULL, w.cn, idx & 31);
          float wt = 1.f;
          if constexpr (!UNIT) {
            const float a0 = __shfl_sync(FULL, w.wv, idx & 31), a1 = __shfl_sync(FULL, w.wn, idx & 31);
            wt = idx < 32 ? a0 : a1;
          }
          if (mine) {
            const int j = idx < 32 ? jw : jn;
            if constexpr (!UNIT) wring[slot] = wt;
            tag[slot] = uint32_t(p + lane);
            bar_expect(full0 + 8u * slot, RB);
            bulk_g2s(ring + uint32_t(slot) * RS, a.X + int64_t(j) * a.ld + tile0, RB,
                     full0 + 8u * slot);
          }
          e += c;
          p += c;
          pslot += c;
          if (pslot >= S) {
            pslot -= S;
            ++pround;
          }
          if (e - wb >= 32) {
            wb += 32;
            w.cw = w.cn;
            w.cn = (wb + 32 + lane < cur.ee) ? a.A.col[wb + 32 + lane] : 0;
            if constexpr (!UNIT) {
              w.wv = w.wn;
              w.wn = (wb + 32 + lane < cur.ee) ? load_w<WT>(a.A.val, wb + 32 + lane) : 0.f;
            }
          }
        }
      }
      if (!ok) break;
    }
    // end markers (row id -1), one for each consumer group
    for (int g = 0; g < NG && ok; ++g) {
      if (hround > 0) ok = __all_sync(FULL, bar_wait(hempty0 + 8u * hslot, (hround - 1) & 1, abort));
      if (ok && lane == 0) {
        hrow[hslot] = -1;
        hdeg[hslot] = 0;
        bar_arrive(hmeta0 + 8u * hslot);
      }
      if (++hslot == HS) {
        hslot = 0;
        ++hround;
      }
    }
    if (!ok && lane == 0) {
      *abort = 1;
      atomicExch(a.err, 1);
    }
    // no bulk copy may still target this CTA's shared memory at exit
    for (int s = lane; s < S; s += 32)
      if (s < p) {
        const int64_t last = s + ((p - 1 - s) / S) * S;
        bar_wait(full0 + 8u * s, uint32_t(last / S) & 1, nullptr);
      }
    for (int s = lane; s < HS; s += 32)
      if (s < hp) {
        const int64_t last = s + ((hp - 1 - s) / HS) * HS;
        bar_wait(hfull0 + 8u * s, uint32_t(last / HS) & 1, nullptr);
      }
    return;
  }

  // -------------------------------------------------------------- consumers
  // group g takes the rows issued at positions g, g + NG, ...; its NWG warps
  // split the tile's columns (4 per lane)
  const int cwarp = warp - 1;
  const int grp = cwarp / NWG;
  if (grp >= NG) return;
  const int col = (cwarp - grp * NWG) * 128 + lane * 4;
  const bool cv = col < twc;
  int hs = grp;  // head stage of the group's next row, and its phase parity
  uint32_t hpar = 0;
  float sq[4] = {0.f, 0.f, 0.f, 0.f};
  double sqd[4] = {0.0, 0.0, 0.0, 0.0};
  int nsq = 0;
  bool failed = false;
  for (;;) {
    if (!__all_sync(FULL, bar_wait(hmeta0 + 8u * hs, hpar, abort))) {
      failed = true;
      break;
    }
    const int64_t i = hrow[hs];
    if (i < 0) break;
    const int deg = hdeg[hs];
    const uint32_t P0 = hpos[hs];
    int slot = int(P0 % uint32_t(S));
    uint32_t par = (P0 / uint32_t(S)) & 1u;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    FF af[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    // float-float sums for the residual pass, FP32 for the Chebyshev step
    constexpr bool ffsum = RES;
    // entries in batches of up to kBatch: one vote over their barriers, the
    // shared-memory loads issued back to back, the slots released in parallel
    for (int t = 0; t < deg;) {
      const int cnt = deg - t < kBatch ? deg - t : kBatch;
      int sl = slot + lane;
      uint32_t pl = par;
      if (sl >= S) {
        sl -= S;
        pl ^= 1u;
      }
      if (!__all_sync(FULL, lane >= cnt ||
                                slot_wait(full0 + 8u * sl, pl, tag + sl, P0 + uint32_t(t + lane), abort))) {
        failed = true;
        break;
      }
      if (cv) {
        if constexpr (ffsum) {
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            if (u < cnt) {
              const int su = slot + u < S ? slot + u : slot + u - S;
              take<true, UNIT>(ring_p + size_t(su) * RS + col * 4, UNIT ? 1.f : wring[su], acc, af);
            }
          }
        } else if (cnt == kBatch) {
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int su = slot + u < S ? slot + u : slot + u - S;
            take<false, UNIT>(ring_p + size_t(su) * RS + col * 4, UNIT ? 1.f : wring[su], acc, af);
          }
        } else {
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            if (u < cnt) {
              const int su = slot + u < S ? slot + u : slot + u - S;
              take<false, UNIT>(ring_p + size_t(su) * RS + col * 4, UNIT ? 1.f : wring[su], acc, af);
            }
          }
        }
      }
      __syncwarp();
      if (lane < cnt) bar_arrive(empty0 + 8u * sl);
      slot += cnt;
      if (slot >= S) {
        slot -= S;
        par ^= 1u;
      }
      t += cnt;
    }
    if (failed) break;
    if (!__all_sync(FULL, bar_wait(hfull0 + 8u * hs, hpar, abort))) {
      failed = true;
      break;
    }
    if (cv) {
      const unsigned char* hb = hring_p + size_t(hs) * NH * RS + col * 4;
      const int64_t o = i * a.ld + tile0 + col;
      if constexpr (!RES) {
        const float4 xk = *reinterpret_cast<const float4*>(hb);
        const float4 bv = *reinterpret_cast<const float4*>(hb + RS);
        float4 xp = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (NH == 3) xp = *reinterpret_cast<const float4*>(hb + 2 * RS);
        const float xs[4] = {xk.x, xk.y, xk.z, xk.w}, bs[4] = {bv.x, bv.y, bv.z, bv.w},
                    ps[4] = {xp.x, xp.y, xp.z, xp.w};
        float out[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float x = a.sx * xs[t];
          const float r = bs[t] - x + a.beta * (a.sx * acc[t]);
          out[t] = x + a.ak * (x - a.sp * ps[t]) + a.ck * r;
        }
        *reinterpret_cast<float4*>(a.O[0] + o) = make_float4(out[0], out[1], out[2], out[3]);
      } else {
        const float4 xv = *reinterpret_cast<const float4*>(hb);
        const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
        float rh[4], rl[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          // beta * acc as ph + pe
          const FF s = fast_two_sum(af[t].hi, af[t].lo);
          const float ph = a.beh * s.hi;
          const float pe = __fmaf_rn(a.beh, s.hi, -ph) + a.beh * s.lo + a.bel * s.hi;
          const FF t1 = two_sum(ph, -xs[t]);
          const FF r = fast_two_sum(t1.hi, t1.lo + pe);
          rh[t] = r.hi;
          rl[t] = r.lo;
          sq[t] = __fmaf_rn(r.hi, r.hi, sq[t]);
        }
        *reinterpret_cast<float4*>(a.O[0] + o) = make_float4(rh[0], rh[1], rh[2], rh[3]);
        *reinterpret_cast<float4*>(a.O[1] + o) = make_float4(rl[0], rl[1], rl[2], rl[3]);
        if (++nsq == 64) {  // FP32 partial sums over at most 64 rows
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            sqd[t] += sq[t];
            sq[t] = 0.f;
          }
          nsq = 0;
        }
      }
    }
    __syncwarp();
    if (lane == 0) bar_arrive(hempty0 + 8u * hs);
    hs += NG;
    if (hs >= HS) {
      hs -= HS;
      hpar ^= 1u;
    }
  }
  if (failed && lane == 0) {
    *abort = 1;
    atomicExch(a.err, 1);
  }
  if constexpr (RES) {
    if (cv && a.rr) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int64_t c = tile0 + col + t;
        const double v = sqd[t] + sq[t];
        if (c < a.b && v != 0.0) atomicAdd(a.rr + c, v);
      }
    }
  }
}


struct PipeShape {
  int tw, tiles, nwg, ngroups, nslots, hstages, chunk;
  size_t smem;
};

// Column tile <= 1024 floats, one consumer warp per 128 columns, enough
// consumer groups for 16 consumer warps (at most 8 groups), 2-4 head stages
// per group within 64 KB, the rest of the shared memory for the entry ring.
PipeShape pipe_shape(int64_t ld, int nh) {
  PipeShape p;
  p.tw = int(std::min<int64_t>(ld, 1024));
  p.tiles = int(ceil_div(ld, p.tw));
  p.nwg = int(ceil_div(p.tw, 128));
  p.ngroups = std::max(1, std::min(8, 16 / p.nwg));
  const int RS = p.tw * 4;
  const int k = std::max(2, std::min(4, (64 * 1024) / (nh * RS * p.ngroups)));
  p.hstages = p.ngroups * k;
  const int avail = kSmemBudget - p.hstages * nh * RS - int(pipe_meta_bytes(kMaxSlots, p.hstages));
  p.nslots = std::min(kMaxSlots, avail / RS);
  p.chunk = std::min(32, p.nslots - kBatch);  // keeps a waiting batch from blocking the producer
  p.smem = size_t(pipe_meta_bytes(p.nslots, p.hstages)) + size_t(p.nslots + p.hstages * nh) * RS;
  return p;
}

template <int MODE>
void pipe_launch(const Csr& A, const PipeSplit& ps, bool unit, PipeArgs& a, cudaStream_t s) {
  const PipeShape sh = pipe_shape(a.ld, n_heads(MODE));
  KATZ_REQUIRE(sh.nslots >= 16 && sh.tiles <= kMaxTiles && A.nnz < (int64_t(1) << 32), KATZ_EINVAL,
               "pipelined gather: row too wide");
  a.A = A;
  a.bstart = ps.bstart.p;
  a.bentry = ps.bentry.p;
  a.nblocks = ps.nblocks;
  a.ctr = ps.ctr.p;
  a.tw = sh.tw;
  a.nslots = sh.nslots;
  a.hstages = sh.hstages;
  a.ngroups = sh.ngroups;
  a.nwg = sh.nwg;
  a.chunk = sh.chunk;
  KATZ_CUDA(cudaMemsetAsync(ps.ctr.p, 0, sizeof(int) * kMaxTiles, s));
  const dim3 grid(unsigned(num_sms()), unsigned(sh.tiles)),
      block(unsigned(32 * (1 + sh.ngroups * sh.nwg)));
  auto go = [&](auto kern) {
    KATZ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sh.smem)));
    kern<<<grid, block, sh.smem, s>>>(a);
    KATZ_CHECK_LAUNCH();
  };
  switch (unit ? int(KATZ_UNIT) : A.vdt) {
    case KATZ_UNIT: go(pipe_kernel<MODE, KATZ_UNIT>); break;
    case KATZ_F32: go(pipe_kernel<MODE, KATZ_F32>); break;
    case KATZ_BF16: go(pipe_kernel<MODE, KATZ_BF16>); break;
    default: throw Error(KATZ_EINVAL, "pipelined gather: weights must be unit, FP32 or BF16");
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

void pipe_split_build(const std::vector<int64_t>& rowptr, int64_t nrows, PipeSplit& ps,
                      cudaStream_t s) {
  std::vector<int64_t> bs{0};
  int rows = 0;
  int64_t w = 0;
  for (int64_t i = 0; i < nrows; ++i) {
    ++rows;
    w += rowptr[i + 1] - rowptr[i] + 4;
    if (rows == kBlockRows || w >= kBlockWeight) {
      bs.push_back(i + 1);
      rows = 0;
      w = 0;
    }
  }
  if (bs.back() != nrows) bs.push_back(nrows);
  std::vector<int64_t> be(bs.size());
  for (size_t k = 0; k < bs.size(); ++k) be[k] = rowptr[bs[k]];
  ps.nblocks = int64_t(bs.size()) - 1;
  ps.bstart.alloc(bs.size());
  ps.bentry.alloc(be.size());
  ps.ctr.alloc(kMaxTiles);
  KATZ_CUDA(cudaMemcpyAsync(ps.bstart.p, bs.data(), sizeof(int64_t) * bs.size(),
                            cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemcpyAsync(ps.bentry.p, be.data(), sizeof(int64_t) * be.size(),
                            cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
}

bool pipe_eligible(const PipeSplit& ps, int64_t ld) { return ps.nblocks > 0 && ld >= 64; }

void pipe_cheb_step(const Csr& A, const PipeSplit& ps, bool unit, double beta, double ak,
                    double ck, const float* Xk, const float* Xprev, const float* B, float* Xout,
                    int64_t ld, int* err, cudaStream_t s, double sx, double sp) {
  KATZ_REQUIRE(ld % 4 == 0 && Xk != Xout && aligned16(Xk) && aligned16(B) && aligned16(Xout) &&
                   (!Xprev || aligned16(Xprev)),
               KATZ_EINVAL, "pipe_cheb_step: operands must be 16-byte aligned, Xout != Xk");
  if (A.nrows <= 0) return;
  PipeArgs a{};
  a.ld = ld;
  a.X = Xk;
  a.H[0] = Xk;
  a.H[1] = B;
  a.H[2] = Xprev;
  a.O[0] = Xout;
  a.beta = float(beta);
  a.ak = float(ak);
  a.ck = float(ck);
  a.sx = float(sx);
  a.sp = float(sp);
  a.err = err;
  prof_begin(s);
  if (Xprev) pipe_launch<kCheb3>(A, ps, unit, a, s);
  else pipe_launch<kCheb2>(A, ps, unit, a, s);
  if (profiling()) {
    const double sv = 4.0 * ld;
    prof_end("cheb_step",
             8.0 * (A.nrows + 1) + double(A.nnz) * (4 + (unit ? 0 : vdt_size(A.vdt))) +
                 sv * A.ncols + sv * A.nrows * (Xprev ? 3.0 : 2.0),
             s);
  }
}

void pipe_residual(const Csr& A, const PipeSplit& ps, bool unit, double beta, const float* X,
                   float* Rh, float* Rl, int64_t ld, int b, double* rr, int* err, cudaStream_t s) {
  KATZ_REQUIRE(ld % 4 == 0 && aligned16(X) && aligned16(Rh) && aligned16(Rl), KATZ_EINVAL,
               "pipe_residual: operands must be 16-byte aligned");
  if (A.nrows <= 0) return;
  PipeArgs a{};
  a.ld = ld;
  a.X = X;
  a.H[0] = X;
  a.O[0] = Rh;
  a.O[1] = Rl;
  a.beh = float(beta);
  a.bel = float(beta - double(a.beh));
  a.rr = rr;
  a.b = b;
  a.err = err;
  prof_begin(s);
  pipe_launch<kResInit>(A, ps, unit, a, s);
  if (profiling())
    prof_end("ff_residual",
             8.0 * (A.nrows + 1) + double(A.nnz) * (4 + (unit ? 0 : vdt_size(A.vdt))) +
                 4.0 * ld * (A.ncols + 3.0 * A.nrows),
             s);
}

}  // namespace katz
