// escape_core.cuh -- the per-pixel escape-time step on sm_103a, bit-exact in binary64.
//
// One step of Eq. 1 (Sec. I) from state (zr, zi) and constant c = (cr, ci):
//     zr2 = zr*zr; zi2 = zi*zi; stop if zr2 + zi2 > R2;
//     zi <- (2*zr)*zi + ci;  zr <- (zr2 - zi2) + cr
// with every operation rounded to nearest-even on its own.
//
// GB300's FP64 pipe issues about 2 lanes per clock per SM (measured), against
// 64-128 for the integer and FP32 pipes, and the pipes run concurrently.  So
// a step issues only six FP64 operations (three multiplies, three adds) and
// does the rest exactly on the other pipes:
//  * (2*zr)*zi is formed as 2*(zr*zi) by adding one to the exponent field of
//    the product.  Scaling by two commutes with round-to-nearest whenever the
//    product is a normal number below 2^1023; zero products are kept as they
//    are (2*0 = 0 with the same sign), and the rare subnormal or huge products
//    fall back to the literal (zr+zr)*zi on the FP64 pipe.
//  * the escape test RN(zr2 + zi2) > R2 is decided from FP32 truncations of
//    zr2 and zi2 whenever their sum is more than 2^-16 (relative) away from R2,
//    which the error bounds in filter_sure() make exact; only sums within that
//    band (a few per million tests) take the literal binary64 add and compare.
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

// Exact 2*p for the product p = zr*zi when p is normal and below 2^1023.
// Returns false (and leaves t = p) when p is zero (then 2p = p exactly) or when
// p is subnormal / >= 2^1023 (then `slow` is set: the caller must recompute).
__device__ __forceinline__ double twice_product(double p, bool& slow) {
  int ph = __double2hiint(p);
  int pl = __double2loint(p);
  unsigned e = ((unsigned)ph >> 20) & 0x7FFu;
  bool ok = (e - 1u) < 0x7FDu;
  slow = !ok && (((ph & 0x7FFFFFFF) | pl) != 0);
  return ok ? __hiloint2double(ph + 0x00100000, pl) : p;
}

// State of one lane's pixel.
struct Lane {
  double zr, zi, cr, ci;
  uint32_t cnt;   // z-updates made so far
  uint32_t lim;   // iterMax of this pixel's view
  bool live;      // still iterating (has not escaped, budget not spent)
};

// One step for all lanes of the warp (must be called warp-uniformly).  FILT
// selects the FP32 escape filter (R2 in [2^-100, 2^100]); otherwise the test is
// the literal binary64 add and compare.
template <bool FILT>
__device__ __forceinline__ void step(Lane& L, double r2, EscThr thr) {
  double zr2 = __dmul_rn(L.zr, L.zr);
  double zi2 = __dmul_rn(L.zi, L.zi);
  double p = __dmul_rn(L.zr, L.zi);
  bool esc;
  if (FILT) {
    bool amb;
    esc = filter_sure(zr2, zi2, thr, amb);
    amb = amb && L.live;
    if (__any_sync(FULL_MASK, amb)) {
      if (amb) esc = __dadd_rn(zr2, zi2) > r2;
    }
  } else {
    esc = __dadd_rn(zr2, zi2) > r2;
  }
  bool upd = L.live && !esc && (L.cnt < L.lim);
  L.live = upd;
  L.cnt += upd ? 1u : 0u;
  bool slow;
  double t = twice_product(p, slow);
  slow = slow && upd;
  if (__any_sync(FULL_MASK, slow)) {
    if (slow) t = __dmul_rn(__dadd_rn(L.zr, L.zr), L.zi);
  }
  L.zi = __dadd_rn(t, L.ci);
  L.zr = __dadd_rn(__dsub_rn(zr2, zi2), L.cr);
}

}  // namespace mb
