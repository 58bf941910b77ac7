/*
 * c_abi_driver.c -- drives libmb.so through its C ABI alone (no Python, no
 * torch): renders a view with every scheduler, the reduced-precision variants
 * and cycle detection, and compares each image with the CPU oracle's
 * (test infrastructure: the oracle's functions are declared here, no header
 * is shared with the library).  Also checks mb_last_stats, an invalid call and
 * mb_strerror.  Exit status 0 when everything matches.
 *
 * Built by tests/test_c_driver.py:
 *   gcc -std=c99 -I include -I <cuda>/include tests/c_abi_driver.c -L <lib dirs> -lmb -lmb_oracle -lcudart
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "mb.h"

/* from oracle/mb_oracle.c and oracle/mb_oracle_lowp.c */
void mbo_render(double xmin, double xmax, double ymin, double ymax, uint32_t m, uint32_t n, uint32_t iter_max,
                double r2, uint32_t* out, int threads);
void mbo_render_rows_lowp(double xmin, double xmax, double ymin, double ymax, uint32_t m, uint32_t n,
                          uint32_t iter_max, double r2, int precision, uint32_t row0, uint32_t nrows, uint32_t* out,
                          int threads);

static int failures = 0;

static void check(int cond, const char* what) {
  if (!cond) {
    fprintf(stderr, "FAILED: %s\n", what);
    ++failures;
  }
}

static size_t differ(const uint32_t* a, const uint32_t* b, size_t count) {
  size_t d = 0;
  for (size_t k = 0; k < count; ++k) d += a[k] != b[k];
  return d;
}

int main(void) {
  const mb_window w = {-2.0, 1.0, -1.0, 1.0};
  const uint32_t m = 120, n = 160, iter_max = 1000;
  const double r2 = 4.0;
  const size_t count = (size_t)m * n;
  uint32_t* want = malloc(count * 4);
  uint32_t* want_lowp = malloc(count * 4);
  uint32_t* got = malloc(count * 4);
  uint32_t* d_out = NULL;
  if (!want || !want_lowp || !got || cudaMalloc((void**)&d_out, count * 4) != cudaSuccess) {
    fprintf(stderr, "allocation failed\n");
    return 2;
  }
  mbo_render(w.xmin, w.xmax, w.ymin, w.ymax, m, n, iter_max, r2, want, 0);
  uint64_t want_sum = 0;
  for (size_t k = 0; k < count; ++k) want_sum += want[k];

  for (int sched = MB_SCHED_NAIVE; sched <= MB_SCHED_FCFS_TILES; ++sched) {
    for (int variant = 0; variant < 4; ++variant) { /* binary64, cycle check, binary32, double-float */
      mb_opts o;
      memset(&o, 0, sizeof o);
      o.sched = sched;
      o.cycle_check = variant == 1;
      o.precision = variant == 2 ? MB_PREC_FP32 : variant == 3 ? MB_PREC_DFLOAT : MB_PREC_FP64;
      cudaMemset(d_out, 0xFF, count * 4);
      int rc = mb_render(&w, m, n, iter_max, r2, d_out, &o);
      check(rc == MB_OK, "mb_render returns MB_OK");
      check(cudaMemcpy(got, d_out, count * 4, cudaMemcpyDeviceToHost) == cudaSuccess, "copy back");
      const uint32_t* ref = want;
      if (variant >= 2) {
        mbo_render_rows_lowp(w.xmin, w.xmax, w.ymin, w.ymax, m, n, iter_max, r2, variant == 2 ? 1 : 2, 0, m,
                             want_lowp, 0);
        ref = want_lowp;
      }
      size_t d = differ(got, ref, count);
      if (d) fprintf(stderr, "sched %d variant %d: %zu pixels differ\n", sched, variant, d);
      check(d == 0, "image equals the oracle's");
      if (variant == 0) {
        mb_run_stats st;
        check(mb_last_stats(&st) == MB_OK, "mb_last_stats");
        check(st.iterations == want_sum, "mb_last_stats iterations equal the oracle's sum");
        check(st.ctas > 0 && st.makespan_ns > 0, "mb_last_stats has a makespan");
      }
    }
  }
  mb_window bad = {1.0, -1.0, -1.0, 1.0};
  check(mb_render(&bad, m, n, iter_max, r2, d_out, NULL) == MB_EINVAL, "an empty window is rejected");
  check(strcmp(mb_strerror(MB_EINVAL), "invalid argument") == 0, "mb_strerror names MB_EINVAL");
  cudaFree(d_out);
  free(want);
  free(want_lowp);
  free(got);
  if (failures) {
    fprintf(stderr, "%d checks failed\n", failures);
    return 1;
  }
  printf("c driver ok: %s\n", mb_version());
  return 0;
}
