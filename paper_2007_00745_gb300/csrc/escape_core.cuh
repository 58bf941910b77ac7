// escape_core.cuh -- the per-pixel escape-time step on sm_103a, bit-exact in binary64.
//
// One step of Eq. 1 (Sec. I) from state (zr, zi) and constant c = (cr, ci):
//     zr2 = zr*zr; zi2 = zi*zi; stop if zr2 + zi2 > R2;
//     zi <- (2*zr)*zi + ci;  zr <- (zr2 - zi2) + cr
// with every operation rounded to nearest-even on its own.
//
// GB300's FP64 pipe delivers about 1.7 lanes per clock per SM (measured),
// against 64 for the integer ALU and 64 for integer multiply-adds on the FMA
// pipe, and the pipes run concurrently.  A step therefore keeps at most three
// additions on the FP64 pipe and does everything else exactly on the other
// pipes, without a branch:
//  * the three products zr*zr, zi*zi and (2*zr)*zi are formed exactly with
//    integer multiply-adds (emul_sqr / emul_mul: 53 x 53-bit mantissa products
//    from three or four 32 x 32 -> 64-bit multiplies, rounded to nearest-even by
//    one carry add at the rounding position), valid whenever zr and zi are
//    normal numbers in a fixed exponent range -- then every product is normal;
//  * on every other step the subtraction zr2 - zi2 of two positive normal
//    numbers is also done exactly on the integer pipes (emul_psub), which takes
//    that step to two FP64-pipe additions; doing it on every step makes the
//    integer ALU the bottleneck instead (measured), so the two kinds alternate;
//  * the escape test RN(zr2 + zi2) > R2 is decided from FP32 truncations of
//    zr2 and zi2 whenever their sum is more than 2^-16 (relative) away from R2;
//    the error bounds in filter_sure() make that decision exact.
// A step that meets none of these conditions (a zero, a tiny or huge component,
// a sum within the band, a subtraction whose leading 32 bits cancel) marks the
// lane pending and carries on; every block of steps starts from a saved copy of
// the lane's state, and resolve() replays a pending lane's block with the
// literal FP64 operations, restoring the exact state and count.  Measured on
// GB300: a branch or predicated FP64 instruction inside the step costs about a
// quarter of the throughput, so the step stays straight-line and all exceptions
// go through the replay.
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

// Operand ranges of the integer products, as biased exponent fields:
//  * [513, 1533] (values in [2^-510, 2^511)): the three products of a step are
//    normal binary64 numbers;
//  * [960, 1086] (values in [2^-63, 2^64)), used with the escape filter: the
//    two squares then also lie in [2^-126, 2^128), the normal binary32 range,
//    so that their FP32 truncations need no clamping (trunc_to_f32_inrange).
// Checked on the high word h with its sign shifted out: (2h - 2*lo*2^20)
// compared unsigned against the range's width.
template <bool TIGHT>
__device__ __forceinline__ bool emul_ok_hi(uint32_t h) {
  if (TIGHT) return h * 2u - (960u << 21) < (127u << 21);
  return h * 2u - (513u << 21) < (1021u << 21);
}

__device__ __forceinline__ bool emul_ok(double x) { return emul_ok_hi<false>((uint32_t)__double2hiint(x)); }

// RN of the 106-bit mantissa product P = hi*2^64 + x*2^32 + l (2^104 <= P < 2^106)
// to 53 bits, packed into a binary64.  eterm holds sign and biased exponent
// minus one of the result for P < 2^105 in bits 20..31 of the high word (taken
// modulo 2^32: the sign falls out of the sum of the operands' sign bits); top =
// (P >= 2^105) adds one to the exponent and moves the rounding position s
// (within x) from bit 20 to bit 21.  Round to nearest-even: add
// 2^(s-1) - 1 + (lsb | sticky) at the rounding position and truncate, where lsb
// is the lowest kept bit and sticky = (l != 0) -- the bits of x below s are
// examined exactly by the carry; a mantissa that rounds up to 2^53 carries into
// the exponent field, which is the correct result.
__device__ __forceinline__ double emul_pack(uint64_t hi, uint32_t x, uint32_t l, uint32_t eterm) {
  uint32_t hh = (uint32_t)(hi >> 32);
  uint32_t top = hh >> 9;
  uint32_t s = 20u + top;
  uint32_t rb = ((x >> s) | min(l, 1u)) & 1u;
  uint64_t lo = (uint64_t)x + (0x7FFFFu + (top << 19) + rb);
  uint64_t mid = hi + (lo >> 32);
  uint32_t ml = (uint32_t)mid, mh = (uint32_t)(mid >> 32);
  uint32_t Mlo = __funnelshift_r((uint32_t)lo, ml, s);
  uint32_t Mhi = __funnelshift_r(ml, mh, s);
  return __hiloint2double((int)(Mhi + eterm + (top << 20)), (int)Mlo);
}

// RN(a*a) from the words of a (h = high, l = low); eterm = 2*(h & 0xFFF00000) - (1024 << 20).
__device__ __forceinline__ double emul_sqr_w(uint32_t h, uint32_t l, uint32_t eterm) {
  uint32_t A = (h & 0xFFFFFu) | 0x100000u;
  uint64_t bd = (uint64_t)l * l;
  uint64_t mid = (uint64_t)(A << 1) * l + (bd >> 32);
  uint64_t hi = (uint64_t)A * A + (mid >> 32);
  return emul_pack(hi, (uint32_t)mid, (uint32_t)bd, eterm);
}

// RN(a*b) * 2^e_add from the words of a and b;
// eterm = (ah & 0xFFF00000) + (bh & 0xFFF00000) - ((1024 - e_add) << 20).
__device__ __forceinline__ double emul_mul_w(uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl, uint32_t eterm) {
  uint32_t A = (ah & 0xFFFFFu) | 0x100000u, C = (bh & 0xFFFFFu) | 0x100000u;
  uint64_t bd = (uint64_t)al * bl;
  uint64_t mid = (uint64_t)A * bl + (bd >> 32);
  mid += (uint64_t)al * C;
  uint64_t hi = (uint64_t)A * C + (mid >> 32);
  return emul_pack(hi, (uint32_t)mid, (uint32_t)bd, eterm);
}

// RN(a*a), exact when a passes emul_ok().
__device__ __forceinline__ double emul_sqr(double a) {
  uint32_t h = (uint32_t)__double2hiint(a);
  return emul_sqr_w(h, (uint32_t)__double2loint(a), (h & 0xFFF00000u) * 2u - 0x40000000u);
}

// RN(a*b) * 2^e_add, e_add in {0, 1}, exact when a and b pass emul_ok().
__device__ __forceinline__ double emul_mul(double a, double b, int e_add) {
  uint32_t ah = (uint32_t)__double2hiint(a), bh = (uint32_t)__double2hiint(b);
  uint32_t et = (ah & 0xFFF00000u) + (bh & 0xFFF00000u) - ((1024u - (uint32_t)e_add) << 20);
  return emul_mul_w(ah, (uint32_t)__double2loint(a), bh, (uint32_t)__double2loint(b), et);
}

// RN(a - b) for positive normal binary64 a and b, with integer operations.
// The larger operand B and the smaller S (compared as bit patterns, which
// order like the values) have their 53-bit mantissas placed at bits 10..62 of
// a 64-bit word; S is shifted right by the exponent difference d with the bits
// shifted out jammed into bit 0 (a sticky bit: with at least two guard bits
// below the rounding position this leaves every rounding decision unchanged),
// the difference is normalised back to bit 62 with a count of leading zeros
// and rounded to nearest-even at bit 10 as in emul_pack.  `odd` is set, and the
// result is not to be used, when d > 31 or when the leading 32 bits cancel
// (which includes a == b); the caller replays those steps.
__device__ __forceinline__ double emul_psub(double a, double b, bool& odd) {
  uint32_t ah = (uint32_t)__double2hiint(a), al = (uint32_t)__double2loint(a);
  uint32_t bh = (uint32_t)__double2hiint(b), bl = (uint32_t)__double2loint(b);
  bool sw = (bh > ah) || (bh == ah && bl > al);
  uint32_t Bh = sw ? bh : ah, Bl = sw ? bl : al, Sh = sw ? ah : bh, Sl = sw ? al : bl;
  uint32_t EB = Bh >> 20;
  uint32_t d = EB - (Sh >> 20);
  uint32_t mBh = (__funnelshift_l(Bl, Bh, 10) & 0x3FFFFFFFu) | 0x40000000u, mBl = Bl << 10;
  uint32_t mSh = (__funnelshift_l(Sl, Sh, 10) & 0x3FFFFFFFu) | 0x40000000u, mSl = Sl << 10;
  uint32_t sSl = __funnelshift_r(mSl, mSh, d);
  uint32_t sSh = __funnelshift_r(mSh, 0u, d);
  uint32_t lost = __funnelshift_lc(0u, mSl, 32u - d);  // the low d bits of mSl (d <= 31), at the top
  sSl |= min(lost, 1u);
  uint64_t D = (((uint64_t)mBh << 32) | mBl) - (((uint64_t)sSh << 32) | sSl);
  uint32_t Dh = (uint32_t)(D >> 32), Dl = (uint32_t)D;
  odd = (Dh == 0u) | (d > 31u);
  uint32_t sh = __clz(Dh) - 1u;  // D < 2^63: the leading bit moves to bit 62
  uint32_t Nh = __funnelshift_l(Dl, Dh, sh), Nl = Dl << (sh & 31u);
  uint32_t rb = (Nl >> 10) & 1u;
  uint64_t R = ((((uint64_t)Nh << 32) | Nl) + (0x1FFu + rb)) >> 10;
  uint32_t rh = (uint32_t)(R >> 32) + ((EB - sh - 1u) << 20) + ((uint32_t)sw << 31);
  return __hiloint2double((int)rh, (int)(uint32_t)R);
}

// Whether step u of a block (0-based) takes its subtraction on the integer
// pipes: every other step (steps 0, 2, 4, ...).  Measured on the 8192^2 view:
// 1 of 2 steps 199 Giter/s, 3 of 8 196, 5 of 8 190, 3 of 4 183, all 171 (the
// integer ALU saturates), none 168.
__device__ __forceinline__ constexpr bool isub_step(int u) { return (u & 1) == 0; }

// FP32 truncation of x in [2^-126, 2^128) (no clamping): v <= x < v (1 + 2^-20).
__device__ __forceinline__ float trunc_to_f32_inrange(double x) {
  return __int_as_float(__double2hiint(x) * 8 + 0x40000000);
}

// RN(0 + x): the first step from z = 0 gives z = (RN(0 + cr), RN(0 + ci)), which
// is c itself except that -0 becomes +0.
__device__ __forceinline__ double plus_zero(double x) {
  return __double_as_longlong(x) == (long long)0x8000000000000000ull ? 0.0 : x;
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
  double szr, szi;  // state at the start of the current block of steps
  uint32_t cnt;     // z-updates made so far
  uint32_t lim;     // iterMax of this pixel's view
  uint32_t scnt;    // cnt at the start of the block
  bool live;        // still iterating (no escape seen, budget not spent)
  bool pend;        // a step of this block was not decided exactly: resolve() replays the block
};

// Start a pixel: the first step from z = 0 never escapes (R2 > 0) and leaves
// z = c (with -0 read as +0), so it is taken here.
__device__ __forceinline__ void lane_start(Lane& L, double cr, double ci, uint32_t lim) {
  L.cr = cr;
  L.ci = ci;
  L.lim = lim;
  L.cnt = lim ? 1u : 0u;
  L.live = lim != 0u;
  L.zr = plus_zero(cr);
  L.zi = plus_zero(ci);
  L.pend = false;
}

// Same, with the escape radius of the view (used by the reduced-precision lanes).
__device__ __forceinline__ void lane_start(Lane& L, double cr, double ci, uint32_t lim, double) {
  lane_start(L, cr, ci, lim);
}

// An idle lane.
__device__ __forceinline__ void lane_clear(Lane& L) {
  L.zr = L.zi = L.cr = L.ci = L.szr = L.szi = 0.0;
  L.cnt = L.lim = L.scnt = 0;
  L.live = false;
  L.pend = false;
}

// Checkpoint at the start of a block of steps.
__device__ __forceinline__ void block_begin(Lane& L) {
  L.szr = L.zr;
  L.szi = L.zi;
  L.scnt = L.cnt;
}

// A lane that also detects exactly periodic orbits.  If the binary64 state
// (zr, zi) at the start of a block is bit-identical to the state at an earlier
// block start, the map -- a fixed sequence of rounded operations on that state
// and the same c -- repeats the same steps forever; none of them escaped the
// first time, so none ever will, and the count is iterMax.  The state is
// compared at block starts (where it is exact: resolve() has run) against a
// copy saved at blocks 1, 2, 4, 8, ... of the pixel (Brent's power-of-two
// schedule), which finds any cycle within about twice its pre-period plus
// period.  Counts are unchanged; only steps are saved.
struct LaneCyc : Lane {
  double pzr, pzi;  // state saved at the last power-of-two block
  uint32_t blk;     // blocks begun since the pixel started
};

__device__ __forceinline__ void lane_clear(LaneCyc& L) {
  lane_clear(static_cast<Lane&>(L));
  L.pzr = L.pzi = 0.0;
  L.blk = 0;
}

__device__ __forceinline__ void lane_start(LaneCyc& L, double cr, double ci, uint32_t lim, double) {
  lane_start(static_cast<Lane&>(L), cr, ci, lim);
  L.pzr = L.zr;
  L.pzi = L.zi;
  L.blk = 0;
}

__device__ __forceinline__ void block_begin(LaneCyc& L) {
  bool rep = L.blk != 0u && __double_as_longlong(L.zr) == __double_as_longlong(L.pzr) &&
             __double_as_longlong(L.zi) == __double_as_longlong(L.pzi);
  if (rep && L.live) {
    L.cnt = L.lim;
    L.live = false;
  }
  L.blk += 1u;
  if ((L.blk & (L.blk - 1u)) == 0u) {
    L.pzr = L.zr;
    L.pzi = L.zi;
  }
  block_begin(static_cast<Lane&>(L));
}

// One step for one lane; straight-line code.  FILT selects the FP32 escape
// filter (R2 in [2^-100, 2^100]); otherwise the test is the literal binary64
// add and compare.  EMUL selects the integer-pipe products (else three FP64
// multiplies, 2*zr by twice()).  isub (a compile-time constant after the block
// loop is unrolled) takes zr2 - zi2 on the integer pipes too; it applies with
// FILT and EMUL, whose range check guarantees positive normal squares.
template <bool FILT, bool EMUL>
__device__ __forceinline__ void step(Lane& L, double r2, EscThr thr, bool isub = false) {
  double zr2, zi2, t;
  bool odd = false;
  if (EMUL) {
    uint32_t rh = (uint32_t)__double2hiint(L.zr), rl = (uint32_t)__double2loint(L.zr);
    uint32_t ih = (uint32_t)__double2hiint(L.zi), il = (uint32_t)__double2loint(L.zi);
    odd = !(emul_ok_hi<FILT>(rh) && emul_ok_hi<FILT>(ih));
    uint32_t er = rh & 0xFFF00000u, ei = ih & 0xFFF00000u;
    zr2 = emul_sqr_w(rh, rl, er * 2u - 0x40000000u);
    zi2 = emul_sqr_w(ih, il, ei * 2u - 0x40000000u);
    t = emul_mul_w(rh, rl, ih, il, er + ei - (1023u << 20));
  } else {
    zr2 = __dmul_rn(L.zr, L.zr);
    zi2 = __dmul_rn(L.zi, L.zi);
    t = __dmul_rn(twice(L.zr), L.zi);
  }
  bool esc;
  if (FILT) {
    bool amb;
    if (EMUL) {  // squares in [2^-126, 2^128) whenever the range check passed
      float s = __fadd_rn(trunc_to_f32_inrange(zr2), trunc_to_f32_inrange(zi2));
      esc = s > thr.hi;
      amb = !(esc || s < thr.lo);
    } else {
      esc = filter_sure(zr2, zi2, thr, amb);
    }
    odd = odd || amb;
  } else {
    esc = __dadd_rn(zr2, zi2) > r2;
  }
  double dz;
  if (FILT && EMUL && isub) {
    bool c;
    dz = emul_psub(zr2, zi2, c);
    odd = odd || c;
  } else {
    dz = __dsub_rn(zr2, zi2);
  }
  L.pend = L.pend || (odd && L.live);
  bool upd = L.live && !esc && (L.cnt < L.lim);
  L.live = upd;
  L.cnt += upd ? 1u : 0u;
  L.zi = __dadd_rn(t, L.ci);
  L.zr = __dadd_rn(dz, L.cr);
}

// Settle a pending lane: redo the whole block from its checkpoint with the
// literal binary64 operations -- STEPS exact steps, stopping at an escape or at
// the budget -- and take that state and count.  Every block therefore moves a
// lane STEPS steps forward or finishes it, whatever the provisional run did
// (a lane whose every step is undecided, e.g. zi = 0 on the real axis, still
// advances one exact block per block).  Call warp-uniformly between blocks.
template <int STEPS>
__device__ __forceinline__ void resolve(Lane& L, double r2) {
  if (__any_sync(FULL_MASK, L.pend)) {
    if (L.pend) {
      double zr = L.szr, zi = L.szi;
      uint32_t c = L.scnt;
      bool live = true;
      for (int k = 0; k < STEPS; ++k) {
        if (c >= L.lim) {
          live = false;
          break;
        }
        double zr2 = dmul_branch(zr, zr);
        double zi2 = dmul_branch(zi, zi);
        if (dadd_branch(zr2, zi2) > r2) {
          live = false;
          break;
        }
        double t = dmul_branch(twice(zr), zi);
        zi = dadd_branch(t, L.ci);
        zr = dadd_branch(dsub_branch(zr2, zi2), L.cr);
        ++c;
      }
      L.cnt = c;
      L.live = live;
      L.zr = zr;
      L.zi = zi;
      L.pend = false;
    }
  }
}

}  // namespace mb
