// render_lowp.cu -- kernel table of the reduced-precision renders (binary32 and
// double-float lanes of escape_lowp.cuh under the same schedulers as binary64,
// and over the batched item list of mb_render_batch and the server).
#include "mb_internal.h"
#include "render_kernels.cuh"

namespace mb {

template <int KIND, int SCHED>
static RenderFn pick_prec(int prec, int unroll) {
  if (prec == PREC_F32)
    return unroll == 16 ? render_kernel<KIND, SCHED, false, 16, false, PREC_F32>
                        : render_kernel<KIND, SCHED, false, 8, false, PREC_F32>;
  return unroll == 16 ? render_kernel_f2<KIND, SCHED, 16> : render_kernel_f2<KIND, SCHED, 8>;
}

RenderFn render_fn_lowp(int kind, int sched, int prec, int unroll) {
  if (kind == KIND_ROWS) {
    if (sched == S_NAIVE) return pick_prec<KIND_ROWS, S_NAIVE>(prec, unroll);
    if (sched == S_ALT) return pick_prec<KIND_ROWS, S_ALT>(prec, unroll);
    return pick_prec<KIND_ROWS, S_FCFS>(prec, unroll);
  }
  if (kind == KIND_RASTER) return pick_prec<KIND_RASTER, S_FCFS>(prec, unroll);
  if (kind == KIND_LIST) return pick_prec<KIND_LIST, S_FCFS>(prec, unroll);
  if (kind == KIND_BATCH) return pick_prec<KIND_BATCH, S_FCFS>(prec, unroll);
  return nullptr;
}

}  // namespace mb
