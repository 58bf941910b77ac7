// render_cycle.cu -- kernel table of the binary64 renders with exact cycle
// detection (LaneCyc in escape_core.cuh): the mb_render schedulers, and the
// batched item list used by mb_render_batch and the server.
#include "mb_internal.h"
#include "render_kernels.cuh"

namespace mb {

template <int KIND, int SCHED, bool FILT>
static RenderFn pick_unroll_cycle(int unroll) {
  return unroll == 16 ? render_kernel<KIND, SCHED, FILT, 16, true, PREC_F64_CYCLE>
                      : render_kernel<KIND, SCHED, FILT, 8, true, PREC_F64_CYCLE>;
}

template <int KIND, int SCHED>
static RenderFn pick_filt_cycle(bool filt, int unroll) {
  return filt ? pick_unroll_cycle<KIND, SCHED, true>(unroll) : pick_unroll_cycle<KIND, SCHED, false>(unroll);
}

RenderFn render_fn_cycle(int kind, int sched, bool filt, int unroll) {
  if (kind == KIND_ROWS) {
    if (sched == S_NAIVE) return pick_filt_cycle<KIND_ROWS, S_NAIVE>(filt, unroll);
    if (sched == S_ALT) return pick_filt_cycle<KIND_ROWS, S_ALT>(filt, unroll);
    return pick_filt_cycle<KIND_ROWS, S_FCFS>(filt, unroll);
  }
  if (kind == KIND_RASTER) return pick_filt_cycle<KIND_RASTER, S_FCFS>(filt, unroll);
  if (kind == KIND_LIST) return pick_filt_cycle<KIND_LIST, S_FCFS>(filt, unroll);
  if (kind == KIND_BATCH) return pick_filt_cycle<KIND_BATCH, S_FCFS>(filt, unroll);
  return nullptr;
}

}  // namespace mb
