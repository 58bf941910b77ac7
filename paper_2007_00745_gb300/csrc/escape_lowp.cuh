// escape_lowp.cuh -- the escape-time step in reduced precision: binary32, and
// double-float (a value is an unevaluated sum h + l of two binary32 numbers).
//
// The paper iterates in double precision (Sec. I, Eq. 1-2); these variants
// trade count accuracy for throughput on GB300, whose FP32 pipe issues about
// 128 lanes per clock per SM against about 1.7 for FP64.  Each is defined by its
// exact operation sequence, so its counts are reproducible bit for bit, and
// each keeps the binary64 order of one iteration:
//     zr2 = zr*zr; zi2 = zi*zi; stop if zr2 + zi2 > R2;
//     zi = (2*zr)*zi + ci;  zr = (zr2 - zi2) + cr.
//
// Binary32: c and R2 are the binary64 values rounded once to binary32 (round
// to nearest-even), then every operation is one binary32 operation.
//
// Double-float: a binary64 x becomes h = RN32(x), l = RN32(x - h).  Sums and
// products are the double-word algorithms of Joldes, Muller and Popescu (ACM
// TOMS 44(2), 2017): the accurate sum (two exact two-sums, two fast-two-sum
// renormalisations; relative error below 3u^2, u = 2^-24) and the product with
// three fused multiply-adds (relative error below 4u^2).  2*x doubles both
// parts; the escape test compares (h, l) pairs lexicographically.
//
// Neither variant needs the exactness machinery of the binary64 step.  The
// binary32 lanes apply the iteration budget once per block of steps (see
// resolve()): the count only grows while the orbit has not escaped, so adding
// the block's iterations saturated at iterMax gives the count the bounded loop
// would give.  The double-float lanes check the budget every iteration.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "escape_core.cuh"
#include "mb_internal.h"

namespace mb {

// ---- binary32 ------------------------------------------------------------
//
// The binary32 step is so cheap that bookkeeping would cost as much as the
// arithmetic, so a block of steps only ORs each step's escape test into one
// flag (no per-step count), and each scheduling step runs F32_ITERS iterations
// (a block of UNROLL steps is UNROLL * F32_ITERS iterations, which spreads the
// per-block overhead over four times as many iterations).  Between blocks, a
// lane whose flag is clear just adds the block's iterations to its count; a
// lane whose flag is set replays the block from its checkpoint with the same
// binary32 operations, one iteration at a time, to find the exact escape (once
// per pixel).
constexpr int F32_ITERS = 4;

struct LaneF32 {
  float zr, zi, cr, ci, r2;
  float szr, szi;   // state at the start of the block
  uint32_t cnt, lim;
  bool live;
  bool esc;         // some step of this block escaped
};

__device__ __forceinline__ void lane_clear(LaneF32& L) {
  L.zr = L.zi = L.cr = L.ci = L.szr = L.szi = 0.0f;
  L.r2 = 4.0f;
  L.cnt = L.lim = 0;
  L.live = false;
  L.esc = false;
}

__device__ __forceinline__ void lane_start(LaneF32& L, double cr, double ci, uint32_t lim, double r2) {
  L.cr = __double2float_rn(cr);
  L.ci = __double2float_rn(ci);
  L.r2 = __double2float_rn(r2);
  L.zr = 0.0f;
  L.zi = 0.0f;
  L.cnt = 0;
  L.lim = lim;
  L.live = lim != 0u;
  L.esc = false;
}

__device__ __forceinline__ void block_begin(LaneF32& L) {
  L.szr = L.zr;
  L.szi = L.zi;
  L.esc = false;
}

// One binary32 iteration.  After an escape the lane keeps computing (its z runs
// off to infinity); resolve() discards those steps.
__device__ __forceinline__ void f32_iter(float& zr, float& zi, float cr, float ci, float r2, bool& esc) {
  float zr2 = __fmul_rn(zr, zr);
  float zi2 = __fmul_rn(zi, zi);
  esc = __fadd_rn(zr2, zi2) > r2;
  float t = __fmul_rn(__fadd_rn(zr, zr), zi);
  zi = __fadd_rn(t, ci);
  zr = __fadd_rn(__fsub_rn(zr2, zi2), cr);
}

template <bool FILT, bool EMUL>
__device__ __forceinline__ void step(LaneF32& L, double, EscThr, bool = false) {
#pragma unroll
  for (int k = 0; k < F32_ITERS; ++k) {
    bool e;
    f32_iter(L.zr, L.zi, L.cr, L.ci, L.r2, e);
    L.esc = L.esc || e;
  }
}

// Settle a block: count it whole, or replay it to the escape, never past the
// budget (a lane that reaches iterMax is done, with count iterMax).  A live
// lane has cnt < lim, and no sum below can exceed lim, so nothing wraps even
// for iterMax near 2^32.
template <int STEPS>
__device__ __forceinline__ void resolve(LaneF32& L, double) {
  if (L.live) {
    if (L.esc) {
      float zr = L.szr, zi = L.szi;
      uint32_t c = L.cnt;
      for (int k = 0; k < STEPS * F32_ITERS; ++k) {
        bool e;
        f32_iter(zr, zi, L.cr, L.ci, L.r2, e);
        if (e) break;
        if (++c == L.lim) break;
      }
      L.cnt = c;
      L.live = false;
    } else if (L.lim - L.cnt <= (uint32_t)(STEPS * F32_ITERS)) {
      L.cnt = L.lim;
      L.live = false;
    } else {
      L.cnt += STEPS * F32_ITERS;
    }
  }
}

// ---- double-float --------------------------------------------------------

struct F2 {
  float h, l;
};

// Exact a + b = s + e (Knuth's two-sum).
__device__ __forceinline__ F2 two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bv = __fsub_rn(s, a);
  float av = __fsub_rn(s, bv);
  F2 r;
  r.h = s;
  r.l = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
  return r;
}

// Exact a + b = s + e for |a| >= |b| (Dekker's fast two-sum).
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  F2 r;
  r.h = s;
  r.l = __fsub_rn(b, __fsub_rn(s, a));
  return r;
}

__device__ __forceinline__ F2 f2_from(double x) {
  F2 r;
  r.h = __double2float_rn(x);
  r.l = __double2float_rn(__dsub_rn(x, (double)r.h));  // x - h is exact in binary64
  return r;
}

// Accurate double-word sum.
__device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
  F2 s = two_sum(x.h, y.h);
  F2 t = two_sum(x.l, y.l);
  F2 v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}

// Double-word product: exact high product, the three cross terms folded into
// its error with fused multiply-adds, one renormalisation.
__device__ __forceinline__ F2 f2_mul(F2 x, F2 y) {
  float ch = __fmul_rn(x.h, y.h);
  float cl1 = __fmaf_rn(x.h, y.h, -ch);
  float tl1 = __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.l));
  float cl2 = __fmaf_rn(x.l, y.h, tl1);
  return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}

struct LaneF2 {
  F2 zr, zi, cr, ci, r2;
  uint32_t cnt, lim;
  bool live;
};

__device__ __forceinline__ void lane_clear(LaneF2& L) {
  L.zr.h = L.zr.l = L.zi.h = L.zi.l = 0.0f;
  L.cr = L.zr;
  L.ci = L.zr;
  L.r2.h = 4.0f;
  L.r2.l = 0.0f;
  L.cnt = L.lim = 0;
  L.live = false;
}

__device__ __forceinline__ void lane_start(LaneF2& L, double cr, double ci, uint32_t lim, double r2) {
  L.cr = f2_from(cr);
  L.ci = f2_from(ci);
  L.r2 = f2_from(r2);
  L.zr.h = L.zr.l = L.zi.h = L.zi.l = 0.0f;
  L.cnt = 0;
  L.lim = lim;
  L.live = lim != 0u;
}

__device__ __forceinline__ void block_begin(LaneF2&) {}

template <bool FILT, bool EMUL>
__device__ __forceinline__ void step(LaneF2& L, double, EscThr, bool = false) {
  F2 zr2 = f2_mul(L.zr, L.zr);
  F2 zi2 = f2_mul(L.zi, L.zi);
  F2 s = f2_add(zr2, zi2);
  bool esc = s.h > L.r2.h || (s.h == L.r2.h && s.l > L.r2.l);
  L.live = L.live && !esc && L.cnt < L.lim;  // the budget each iteration: the count never passes iterMax
  L.cnt += L.live ? 1u : 0u;
  F2 twice_zr;
  twice_zr.h = __fadd_rn(L.zr.h, L.zr.h);
  twice_zr.l = __fadd_rn(L.zr.l, L.zr.l);
  L.zi = f2_add(f2_mul(twice_zr, L.zi), L.ci);
  F2 neg_zi2;
  neg_zi2.h = -zi2.h;
  neg_zi2.l = -zi2.l;
  L.zr = f2_add(f2_add(zr2, neg_zi2), L.cr);
}

template <int STEPS>
__device__ __forceinline__ void resolve(LaneF2& L, double) {
  if (L.cnt >= L.lim) {
    L.cnt = L.lim;
    L.live = false;
  }
}

// ---- lane type of each precision -------------------------------------------

template <int PREC>
struct LaneOf {
  using type = Lane;
};
template <>
struct LaneOf<PREC_F32> {
  using type = LaneF32;
};
template <>
struct LaneOf<PREC_F2> {
  using type = LaneF2;
};
template <>
struct LaneOf<PREC_F64_CYCLE> {
  using type = LaneCyc;
};

}  // namespace mb
