// escape_core.cuh -- the per-pixel escape-time step on sm_103a, bit-exact in binary64.
//
// One step of Eq. 1 (Sec. I) from state (zr, zi) and constant c = (cr, ci):
//     zr2 = zr*zr; zi2 = zi*zi; stop if zr2 + zi2 > R2;
//     zi <- (2*zr)*zi + ci;  zr <- (zr2 - zi2) + cr
// with every operation rounded to nearest-even on its own.
//
// GB300's FP64 pipe delivers about 1.7 lanes per clock per SM (measured),
// against 64-128 for the integer and FP32 pipes, and the pipes run
// concurrently.  So a step issues only six FP64 operations (three multiplies,
// three adds) and does the rest exactly on the other pipes, without a branch:
//  * 2*zr is formed by integer operations on its bit pattern (exponent + 1 for
//    normal numbers, a one-bit shift for zeros and subnormals, infinity past
//    the largest finite exponent) -- exactly the value the FP64 multiply by two
//    would give -- and (2*zr)*zi is then one FP64 multiply, as in the method.
//  * the escape test RN(zr2 + zi2) > R2 is decided from FP32 truncations of
//    zr2 and zi2 whenever their sum is more than 2^-16 (relative) away from R2;
//    the error bounds in filter_sure() make that decision exact.  Within the
//    band the lane carries on as if it had not escaped and saves the state of
//    that step; resolve() later replays the saved steps with the literal FP64
//    add and compare and corrects the count if the lane had in fact escaped.
// Measured on GB300: any branch or predicated FP64 instruction inside the step
// (even one that is almost never taken) costs about a quarter of the
// throughput, because the warp then waits for the FP64 results before it can
// issue the next step's independent work; the deferred replay keeps the step
// straight-line.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mb {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Truncate a non-negative binary64 to an FP32 value v with v <= x < v*(1 + 2^-20)
// for x in [2^-126, 2^128); smaller x map to 2^-126 (over-estimate by at most
// 2^-126), larger x and +inf to the largest finite FP32 value.
__device__ __forceinline__ float trunc_to_f32(double x) {
  int h = __double2hiint(x);
  h = max(h, 0x38100000);          // 2^-126
  h = min(h, 0x47EFFFFF);          // just below 2^128
  // float bits = (h << 3) - ((1023 - 127) << 23), taken mod 2^32
  return __int_as_float(h * 8 + 0x40000000);
}

// Float thresholds for the escape filter: lo <= R2 (1 - 2^-16), hi >= R2 (1 + 2^-16).
// Valid for R2 in [2^-100, 2^100]; see filter_sure().
struct EscThr {
  float lo, hi;
};

// Decides RN(a + b) > R2 for a, b >= 0 from their FP32 truncations.
// With fa, fb from trunc_to_f32 and s = RN32(fa + fb):
//   s > hi  =>  a + b >= s/(1+2^-24) - 2^-125 > R2 (1 + 2^-17)  =>  RN(a + b) > R2
//   s < lo  =>  a + b <  s (1+2^-24)(1+2^-20) < R2 (1 - 2^-17)  =>  RN(a + b) < R2
// (R2 >= 2^-100 makes the 2^-125 slack negligible.)  Otherwise `amb` is set and
// the caller must decide with the binary64 add.
__device__ __forceinline__ bool filter_sure(double a, double b, EscThr t, bool& amb) {
  float s = __fadd_rn(trunc_to_f32(a), trunc_to_f32(b));
  bool above = s > t.hi;
  amb = !(above || s < t.lo);
  return above;
}

// Exact 2*x for any binary64 x, with integer operations only: the exponent
// field is incremented for normal numbers below 2^1023, the magnitude is
// shifted left by one bit for zeros and subnormals (which lands on the right
// normal number when the top mantissa bit carries into the exponent), the
// result is infinity past the largest finite exponent, and infinities and NaNs
// are returned unchanged.  RN(2*x) is exact in binary64, so this is the value
// the FP64 multiply would produce.
__device__ __forceinline__ double twice(double x) {
  int h = __double2hiint(x), l = __double2loint(x);
  unsigned e = ((unsigned)h >> 20) & 0x7FFu;
  int sign = h & (int)0x80000000;
  int sub_h = (int)((((unsigned)h & 0x7FFFFFFFu) << 1) | ((unsigned)l >> 31)) | sign;
  int sub_l = (int)((unsigned)l << 1);
  int rh = e == 0 ? sub_h : (e < 0x7FEu ? h + 0x00100000 : (e == 0x7FEu ? (sign | 0x7FF00000) : h));
  int rl = e == 0 ? sub_l : (e == 0x7FEu ? 0 : l);
  return __hiloint2double(rh, rl);
}

// Binary64 operations that the compiler may not hoist out of the rare replay
// branch in resolve().
__device__ __forceinline__ double dadd_branch(double a, double b) {
  double r;
  asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
  return r;
}
__device__ __forceinline__ double dsub_branch(double a, double b) {
  double r;
  asm volatile("sub.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
  return r;
}
__device__ __forceinline__ double dmul_branch(double a, double b) {
  double r;
  asm volatile("mul.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
  return r;
}

// State of one lane's pixel.
struct Lane {
  double zr, zi, cr, ci;
  double szr, szi;  // state at the start of the first undecided escape test since the last resolve()
  uint32_t cnt;     // z-updates made so far
  uint32_t lim;     // iterMax of this pixel's view
  uint32_t scnt;    // cnt at that saved step
  bool live;        // still iterating (no escape seen, budget not spent)
  bool pend;        // a saved step awaits resolve()
};

// One step for one lane; straight-line code.  FILT selects the FP32 escape
// filter (R2 in [2^-100, 2^100]); otherwise the test is the literal binary64
// add and compare.
template <bool FILT>
__device__ __forceinline__ void step(Lane& L, double r2, EscThr thr) {
  double zr2 = __dmul_rn(L.zr, L.zr);
  double zi2 = __dmul_rn(L.zi, L.zi);
  double t = __dmul_rn(twice(L.zr), L.zi);
  bool esc;
  if (FILT) {
    bool amb;
    esc = filter_sure(zr2, zi2, thr, amb);
    bool first = amb && L.live && !L.pend;
    L.szr = first ? L.zr : L.szr;
    L.szi = first ? L.zi : L.szi;
    L.scnt = first ? L.cnt : L.scnt;
    L.pend = L.pend || first;
  } else {
    esc = __dadd_rn(zr2, zi2) > r2;
  }
  bool upd = L.live && !esc && (L.cnt < L.lim);
  L.live = upd;
  L.cnt += upd ? 1u : 0u;
  L.zi = __dadd_rn(t, L.ci);
  L.zr = __dadd_rn(__dsub_rn(zr2, zi2), L.cr);
}

// Settle a lane whose provisional run passed an undecided escape test: replay
// from the saved step with the literal binary64 test up to the provisional
// count; if an escape shows up earlier, that is the count.  Call
// warp-uniformly between blocks of step() calls.
__device__ __forceinline__ void resolve(Lane& L, double r2) {
  if (__any_sync(FULL_MASK, L.pend)) {
    if (L.pend) {
      double zr = L.szr, zi = L.szi;
      uint32_t c = L.scnt;
      while (c < L.cnt) {
        double zr2 = dmul_branch(zr, zr);
        double zi2 = dmul_branch(zi, zi);
        if (dadd_branch(zr2, zi2) > r2) break;
        double t = dmul_branch(twice(zr), zi);
        zi = dadd_branch(t, L.ci);
        zr = dadd_branch(dsub_branch(zr2, zi2), L.cr);
        ++c;
      }
      if (c < L.cnt) {
        L.cnt = c;
        L.live = false;
      }
      L.pend = false;
    }
  }
}

}  // namespace mb
