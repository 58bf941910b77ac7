/*
 * mb_oracle_lowp.c -- plain CPU oracle of the reduced-precision escape-time
 * variants (binary32, and double-float = an unevaluated sum of two binary32).
 * TEST INFRASTRUCTURE ONLY: nothing on the product path links or calls this
 * file; it shares no code, header or constant with the CUDA path.
 *
 * The paper computes in double precision only (Sec. I, Eq. 1-2).  These two
 * variants trade count accuracy for throughput; each is defined here by its
 * exact operation sequence, so that a GPU implementation can be checked bit for
 * bit against it, while its distance from the binary64 counts is a measured
 * property (a count tolerance), not a parity claim.
 *
 * Built with the binary64 oracle (oracle/build.py: -ffp-contract=off, no fast
 * math): every float operation below is one IEEE binary32 operation rounded to
 * nearest-even; fmaf() is the correctly rounded fused multiply-add of C99.
 *
 * Common to both variants:
 *   - c is the binary64 pixel map of the binary64 oracle (mbo_c_re / mbo_c_im),
 *     converted once; R2 is converted the same way;
 *   - the per-iteration order is the binary64 one:
 *       zr2 = zr*zr; zi2 = zi*zi; stop if zr2 + zi2 > R2;
 *       zi = (2*zr)*zi + ci; zr = (zr2 - zi2) + cr,
 *     and the count is the number of z-updates before the stop, else iterMax.
 *
 * Binary32: c32 = RN32(c), R2_32 = RN32(R2), each operation in binary32.
 *
 * Double-float: a value is (h, l) with h = RN32(h + l).  Conversion of a
 * binary64 x: h = RN32(x), l = RN32(x - h) (x - h is exact in binary64).
 * The arithmetic is the double-word algorithms of Joldes, Muller and Popescu
 * ("Tight and rigorous error bounds for basic building blocks of double-word
 * arithmetic", ACM TOMS 44(2), 2017):
 *   - sum: the accurate double-word + double-word algorithm (two exact
 *     two-sums of the high and low parts, renormalised twice by fast
 *     two-sums), relative error below 3u^2 (u = 2^-24);
 *   - product: the double-word x double-word algorithm with three fused
 *     multiply-adds (exact high product, then xh*yl + xl*yh + xl*yl folded
 *     into its error), relative error below 4u^2;
 *   - 2*x doubles both parts (exact unless it overflows);
 *   - the escape test compares (h, l) pairs lexicographically: s > R2 iff
 *     s.h > R2.h, or s.h == R2.h and s.l > R2.l.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The binary64 pixel map (Cx / Cy of Sec. III-A), from mb_oracle.c. */
double mbo_c_re(double xmin, double xmax, uint32_t n, uint32_t j);
double mbo_c_im(double ymin, double ymax, uint32_t m, uint32_t i);

/* ---- binary32 ------------------------------------------------------------- */

/* Eq. 1-2 in binary32 (not in the paper, which computes in double precision):
 * c and R^2 rounded once, then the binary64 operation order in binary32. */
uint32_t mbo_escape_f32(double cr64, double ci64, uint32_t iter_max, double r2_64) {
  float cr = (float)cr64, ci = (float)ci64, r2 = (float)r2_64;
  float zr = 0.0f, zi = 0.0f;
  uint32_t k = 0;
  while (k < iter_max) {
    float zr2 = zr * zr;
    float zi2 = zi * zi;
    if (zr2 + zi2 > r2) break;
    float two_zr = 2.0f * zr;
    zi = two_zr * zi + ci;
    zr = (zr2 - zi2) + cr;
    k = k + 1;
  }
  return k;
}

/* ---- double-float ----------------------------------------------------------- */

typedef struct {
  float h, l;
} mbo_df;

/* Exact sum a + b = s + e (Knuth's two-sum; six operations, no precondition). */
void mbo_two_sum(float a, float b, float* s, float* e) {
  float sum = a + b;
  float b_virtual = sum - a;
  float a_virtual = sum - b_virtual;
  float b_err = b - b_virtual;
  float a_err = a - a_virtual;
  *s = sum;
  *e = a_err + b_err;
}

/* Exact sum a + b = s + e when |a| >= |b| (Dekker's fast two-sum). */
void mbo_fast_two_sum(float a, float b, float* s, float* e) {
  float sum = a + b;
  float b_virtual = sum - a;
  *s = sum;
  *e = b - b_virtual;
}

/* Exact product a * b = p + e (the error term from one fused multiply-add; the
 * two-product of the double-word algorithms of Joldes, Muller and Popescu). */
void mbo_two_prod(float a, float b, float* p, float* e) {
  float prod = a * b;
  *p = prod;
  *e = fmaf(a, b, -prod);
}

/* A binary64 value as a double-float pair (the conversion described above). */
mbo_df mbo_df_from_f64(double x) {
  mbo_df r;
  r.h = (float)x;
  r.l = (float)(x - (double)r.h);
  return r;
}

/* Accurate double-word sum (Joldes-Muller-Popescu 2017). */
mbo_df mbo_df_add(mbo_df x, mbo_df y) {
  float sh, sl, th, tl, vh, vl;
  mbo_two_sum(x.h, y.h, &sh, &sl);
  mbo_two_sum(x.l, y.l, &th, &tl);
  float c = sl + th;
  mbo_fast_two_sum(sh, c, &vh, &vl);
  float w = tl + vl;
  mbo_df z;
  mbo_fast_two_sum(vh, w, &z.h, &z.l);
  return z;
}

/* Double-word product with three fused multiply-adds (Joldes-Muller-Popescu 2017). */
mbo_df mbo_df_mul(mbo_df x, mbo_df y) {
  float ch, cl1;
  mbo_two_prod(x.h, y.h, &ch, &cl1);
  float tl0 = x.l * y.l;
  float tl1 = fmaf(x.h, y.l, tl0);
  float cl2 = fmaf(x.l, y.h, tl1);
  float cl3 = cl1 + cl2;
  mbo_df z;
  mbo_fast_two_sum(ch, cl3, &z.h, &z.l);
  return z;
}

static mbo_df df_neg(mbo_df x) {
  mbo_df r;
  r.h = -x.h;
  r.l = -x.l;
  return r;
}

static mbo_df df_twice(mbo_df x) {
  mbo_df r;
  r.h = 2.0f * x.h;
  r.l = 2.0f * x.l;
  return r;
}

static int df_greater(mbo_df a, mbo_df b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }

/* Eq. 1-2 in double-float arithmetic (not in the paper): the binary64
 * operation order with the double-word sum and product above, 2*zr by doubling
 * both parts, and the lexicographic escape test. */
uint32_t mbo_escape_df(double cr64, double ci64, uint32_t iter_max, double r2_64) {
  mbo_df cr = mbo_df_from_f64(cr64), ci = mbo_df_from_f64(ci64), r2 = mbo_df_from_f64(r2_64);
  mbo_df zr = {0.0f, 0.0f}, zi = {0.0f, 0.0f};
  uint32_t k = 0;
  while (k < iter_max) {
    mbo_df zr2 = mbo_df_mul(zr, zr);
    mbo_df zi2 = mbo_df_mul(zi, zi);
    if (df_greater(mbo_df_add(zr2, zi2), r2)) break;
    mbo_df two_zr = df_twice(zr);
    zi = mbo_df_add(mbo_df_mul(two_zr, zi), ci);
    zr = mbo_df_add(mbo_df_add(zr2, df_neg(zi2)), cr);
    k = k + 1;
  }
  return k;
}

/* Flat wrappers of the double-float primitives (test infrastructure: the
 * pins check them against exact rationals and their published error bounds). */
void mbo_df_add4(float xh, float xl, float yh, float yl, float* zh, float* zl) {
  mbo_df x = {xh, xl}, y = {yh, yl};
  mbo_df z = mbo_df_add(x, y);
  *zh = z.h;
  *zl = z.l;
}

void mbo_df_mul4(float xh, float xl, float yh, float yl, float* zh, float* zl) {
  mbo_df x = {xh, xl}, y = {yh, yl};
  mbo_df z = mbo_df_mul(x, y);
  *zh = z.h;
  *zl = z.l;
}

/* ---- images ------------------------------------------------------------------ */

/* Eq. 2 over the image in the given precision (1 = binary32, 2 = double-float;
 * not in the paper), rows [row0, row0 + nrows) only, out[(i - row0) * n + j]. */
void mbo_render_rows_lowp(double xmin, double xmax, double ymin, double ymax, uint32_t m, uint32_t n,
                          uint32_t iter_max, double r2, int precision, uint32_t row0, uint32_t nrows,
                          uint32_t* out, int threads) {
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
#endif
  for (long r = 0; r < (long)nrows; r++) {
    uint32_t i = row0 + (uint32_t)r;
    double ci = mbo_c_im(ymin, ymax, m, i);
    for (uint32_t j = 0; j < n; j++) {
      double cr = mbo_c_re(xmin, xmax, n, j);
      out[(size_t)r * n + j] =
          precision == 1 ? mbo_escape_f32(cr, ci, iter_max, r2) : mbo_escape_df(cr, ci, iter_max, r2);
    }
  }
  (void)threads;
}
