/*
 * mb_oracle.c -- plain, slow, obviously correct CPU oracle for the escape-time
 * renderer.  TEST INFRASTRUCTURE ONLY: nothing on the product path links or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header or constant with the CUDA path.
 *
 * Build (see oracle/build.py): gcc -O2 -ffp-contract=off -fno-fast-math
 * -fopenmp -shared -fPIC.  -ffp-contract=off keeps every product and sum a
 * separately rounded IEEE binary64 operation (no fused multiply-add), on x86-64
 * (SSE2) and on aarch64 alike.
 *
 * What it computes (Sec. I, Eq. 1 and Eq. 2 of the paper): for every pixel
 * (i, j) of an m x n image, iterate f(z) = z^2 + c from z = 0 and record the
 * iteration at which |z|^2 first exceeds the escape radius, or iterationMax.
 * Readings of points the paper leaves open:
 *   - pixel -> c (Sec. I says only that c comes from m and n; Sec. III-A
 *     says every task precomputes the Cx and Cy arrays):
 *         c_re = xmin + (j * (xmax - xmin)) / n
 *         c_im = ymax - (i * (ymax - ymin)) / m        (row 0 = top)
 *     evaluated left to right, one rounding per operation;
 *   - "exceeds" is strict: escape when zr^2 + zi^2 > R2, with R2 passed in
 *     directly as the squared radius;
 *   - the recorded count k is the number of z-updates made before the first
 *     iterate whose squared modulus exceeds R2 (iterMax if none does);
 *   - evaluation order per iteration: zr2 = zr*zr; zi2 = zi*zi;
 *     test zr2 + zi2 > R2; zi = (2*zr)*zi + ci; zr = (zr2 - zi2) + cr.
 */
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif


/* Pixel -> c, real part (Sec. I; Cx array of Sec. III-A). */
double mbo_c_re(double xmin, double xmax, uint32_t n, uint32_t j) {
  double span = xmax - xmin;
  double num = (double)j * span;
  return xmin + num / (double)n;
}

/* Pixel -> c, imaginary part, row 0 at the top (Sec. I; Cy array of Sec. III-A). */
double mbo_c_im(double ymin, double ymax, uint32_t m, uint32_t i) {
  double span = ymax - ymin;
  double num = (double)i * span;
  return ymax - num / (double)m;
}

/* Boolean escape-time count of one point c (Eq. 1 iterated from z = 0; Eq. 2). */
uint32_t mbo_escape(double cr, double ci, uint32_t iter_max, double r2) {
  double zr = 0.0, zi = 0.0;
  uint32_t k = 0;
  while (k < iter_max) {
    double zr2 = zr * zr;
    double zi2 = zi * zi;
    if (zr2 + zi2 > r2) break;
    double two_zr = 2.0 * zr;
    zi = two_zr * zi + ci;
    zr = (zr2 - zi2) + cr;
    k = k + 1;
  }
  return k;
}

/* Fill the Cx (n entries) and Cy (m entries) arrays of Sec. III-A. */
void mbo_pixel_map(double xmin, double xmax, double ymin, double ymax, uint32_t m, uint32_t n,
                   double* cx, double* cy) {
  for (uint32_t j = 0; j < n; j++) cx[j] = mbo_c_re(xmin, xmax, n, j);
  for (uint32_t i = 0; i < m; i++) cy[i] = mbo_c_im(ymin, ymax, m, i);
}

/* Whole image I_{i,j} (Eq. 2), row-major uint32.  Rows are shared among host
 * threads first come, first served (OpenMP dynamic, one row at a time); the
 * result does not depend on the schedule (Bernstein's conditions, Sec. II-A). */
void mbo_render(double xmin, double xmax, double ymin, double ymax, uint32_t m, uint32_t n,
                uint32_t iter_max, double r2, uint32_t* out, int threads) {
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
#endif
  for (long i = 0; i < (long)m; i++) {
    double ci = mbo_c_im(ymin, ymax, m, (uint32_t)i);
    for (uint32_t j = 0; j < n; j++) {
      double cr = mbo_c_re(xmin, xmax, n, j);
      out[(size_t)i * n + j] = mbo_escape(cr, ci, iter_max, r2);
    }
  }
  (void)threads;
}

/* Rows [row0, row0 + nrows) of the image of Eq. 2 only (for bounded CPU samples). */
void mbo_render_rows(double xmin, double xmax, double ymin, double ymax, uint32_t m, uint32_t n,
                     uint32_t iter_max, double r2, uint32_t row0, uint32_t nrows, uint32_t* out,
                     int threads) {
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
#endif
  for (long r = 0; r < (long)nrows; r++) {
    uint32_t i = row0 + (uint32_t)r;
    double ci = mbo_c_im(ymin, ymax, m, i);
    for (uint32_t j = 0; j < n; j++) {
      double cr = mbo_c_re(xmin, xmax, n, j);
      out[(size_t)r * n + j] = mbo_escape(cr, ci, iter_max, r2);
    }
  }
  (void)threads;
}

/* Counts I_{i,j} (Eq. 2) of an arbitrary list of pixels, idx[t] = i * n + j. */
void mbo_render_pixels(double xmin, double xmax, double ymin, double ymax, uint32_t m, uint32_t n,
                       uint32_t iter_max, double r2, const uint64_t* idx, size_t count,
                       uint32_t* out, int threads) {
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads)
#endif
  for (long t = 0; t < (long)count; t++) {
    uint32_t i = (uint32_t)(idx[t] / n);
    uint32_t j = (uint32_t)(idx[t] % n);
    out[t] = mbo_escape(mbo_c_re(xmin, xmax, n, j), mbo_c_im(ymin, ymax, m, i), iter_max, r2);
  }
  (void)threads;
}

/* Sum of counts (z-updates, Eq. 2) over each tile_h x tile_w tile -- the per-tile
 * cost that the tile-cost model learns (not in the paper); tiles are numbered
 * row-major, the last tile row / column is cut at the image edge. */
void mbo_tile_totals(const uint32_t* counts, uint32_t m, uint32_t n, uint32_t tile_h,
                     uint32_t tile_w, uint64_t* totals) {
  uint32_t tiles_x = (n + tile_w - 1) / tile_w;
  uint32_t tiles_y = (m + tile_h - 1) / tile_h;
  for (uint32_t t = 0; t < tiles_x * tiles_y; t++) totals[t] = 0;
  for (uint32_t i = 0; i < m; i++)
    for (uint32_t j = 0; j < n; j++)
      totals[(i / tile_h) * tiles_x + (j / tile_w)] += counts[(size_t)i * n + j];
}

/* Low-resolution probe of Eq. 2 (the input of the tile-cost model; not in the
 * paper): in each tile x tile block, probe x probe samples, sample
 * (a, b) at pixel (ty*tile + a*s + s/2, tx*tile + b*s + s/2) with s = tile/probe,
 * clamped to the last row / column of the image.  Output layout:
 * out[((ty * tiles_x + tx) * probe + a) * probe + b]. */
void mbo_probe(double xmin, double xmax, double ymin, double ymax, uint32_t m, uint32_t n,
               uint32_t iter_max, double r2, uint32_t tile, uint32_t probe, uint32_t* out,
               int threads) {
  uint32_t tiles_x = (n + tile - 1) / tile;
  uint32_t tiles_y = (m + tile - 1) / tile;
  uint32_t s = tile / probe;
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
#endif
  for (long t = 0; t < (long)tiles_x * tiles_y; t++) {
    uint32_t ty = (uint32_t)(t / tiles_x), tx = (uint32_t)(t % tiles_x);
    for (uint32_t a = 0; a < probe; a++) {
      for (uint32_t b = 0; b < probe; b++) {
        uint32_t i = ty * tile + a * s + s / 2;
        uint32_t j = tx * tile + b * s + s / 2;
        if (i > m - 1) i = m - 1;
        if (j > n - 1) j = n - 1;
        out[((size_t)t * probe + a) * probe + b] =
            mbo_escape(mbo_c_re(xmin, xmax, n, j), mbo_c_im(ymin, ymax, m, i), iter_max, r2);
      }
    }
  }
  (void)threads;
}

/* Naive row partition (Sec. III-A): worker r of N computes rows [S_r, E_r],
 * S_r = (m / N) * r, E_r = (m / N) * (r + 1) - 1 with integer division; the
 * last worker also takes the m mod N remaining rows.  Returns S_r and the row
 * count. */
void mbo_naive_rows(uint32_t m, uint32_t workers, uint32_t r, uint32_t* first, uint32_t* count) {
  uint32_t per = m / workers;
  *first = per * r;
  *count = per + (r == workers - 1 ? m % workers : 0);
}

/* Alternating row partition (Sec. III-C): row i belongs to worker i mod N. */
uint32_t mbo_alternating_owner(uint32_t i, uint32_t workers) { return i % workers; }

/* Iteration -> pixel colour (Sec. I: the iteration determines the colour; the
 * paper gives no palette).  Reading taken: points that never escape are
 * black; otherwise each channel is a triangle wave of the count,
 * tri(x) = x < 256 ? x : 511 - x, with r = tri((7k) mod 512),
 * g = tri((5k) mod 512), b = tri((3k) mod 512).  Integers only. */
static unsigned tri(unsigned x) { return x < 256u ? x : 511u - x; }

/* Sec. I colouring of every count with the palette above. */
void mbo_colorize(const uint32_t* counts, uint64_t count, uint32_t iter_max, uint8_t* rgb) {
  for (uint64_t t = 0; t < count; t++) {
    uint32_t k = counts[t];
    uint8_t r = 0, g = 0, b = 0;
    if (k != iter_max) {
      r = (uint8_t)tri((uint32_t)(((uint64_t)k * 7u) % 512u));
      g = (uint8_t)tri((uint32_t)(((uint64_t)k * 5u) % 512u));
      b = (uint8_t)tri((uint32_t)(((uint64_t)k * 3u) % 512u));
    }
    rgb[3 * t] = r;
    rgb[3 * t + 1] = g;
    rgb[3 * t + 2] = b;
  }
}

/* Host threads the OpenMP loops above use (the core count reported with the CPU
 * baseline; not a step of the method). */
int mbo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
