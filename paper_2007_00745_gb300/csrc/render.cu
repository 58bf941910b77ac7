// render.cu -- mb_render and its helpers: argument checks, workspace layout,
// kernel selection and launch.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "mb.h"
#include "mb_internal.h"
#include "render_kernels.cuh"

namespace mb {

static float f32_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = nextafterf(f, 0.0f);
  return f;
}
static float f32_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, INFINITY);
  return f;
}

bool filter_ok(double r2) { return r2 >= 0x1p-100 && r2 <= 0x1p100; }

EscThr make_thr(double r2) {
  EscThr t;
  if (filter_ok(r2)) {
    t.lo = f32_down(r2 * (1.0 - 0x1p-16));
    t.hi = f32_up(r2 * (1.0 + 0x1p-16));
  } else {
    t.lo = 0.0f;
    t.hi = 0.0f;
  }
  return t;
}

int check_view(const mb_window* w, uint32_t m, uint32_t n, double r2, const void* out) {
  if (!w || !out) return MB_EINVAL;
  if (m == 0 || n == 0 || m > MAX_SIDE || n > MAX_SIDE) return MB_EINVAL;
  if (!std::isfinite(w->xmin) || !std::isfinite(w->xmax) || !std::isfinite(w->ymin) || !std::isfinite(w->ymax))
    return MB_EINVAL;
  if (!(w->xmin < w->xmax) || !(w->ymin < w->ymax)) return MB_EINVAL;
  if (!std::isfinite(w->xmax - w->xmin) || !std::isfinite(w->ymax - w->ymin)) return MB_EINVAL;
  if (!std::isfinite(r2) || !(r2 > 0.0)) return MB_EINVAL;
  return MB_OK;
}

int check_device_access(const void* p) {
  if (!p) return MB_EINVAL;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return MB_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MB_ECUDA;
  switch (a.type) {
    case cudaMemoryTypeDevice:
      return a.device == dev ? MB_OK : MB_EINVAL;
    case cudaMemoryTypeManaged:
      return MB_OK;
    case cudaMemoryTypeHost:  // pinned or registered: usable when the device sees it at the same address
      return a.devicePointer == p ? MB_OK : MB_EINVAL;
    default: {                // ordinary host memory: only where the device can access pageable memory
      int pageable = 0;
      if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) return MB_ECUDA;
      return pageable ? MB_OK : MB_EINVAL;
    }
  }
}

int check_opts(const mb_opts* o, uint32_t* log2_tile, unsigned allow) {
  uint32_t tile = o && o->tile ? o->tile : DEFAULT_TILE;
  if (tile < 8 || tile > 256 || (tile & (tile - 1))) return MB_EINVAL;
  uint32_t l = 0;
  while ((1u << l) < tile) ++l;
  *log2_tile = l;
  uint32_t block = o && o->block ? o->block : DEFAULT_BLOCK;
  if (block < 32 || block > 512 || block % 32) return MB_EINVAL;
  if (o && (o->sched < MB_SCHED_NAIVE || o->sched > MB_SCHED_FCFS_ITEMS)) return MB_EINVAL;
  if (o && o->sched == MB_SCHED_FCFS_ITEMS && (!o->items || o->n_items == 0)) return MB_EINVAL;
  if (o && o->workspace && (((uintptr_t)o->workspace) & 255)) return MB_EINVAL;
  if (o && o->unroll && o->unroll != 4 && o->unroll != 8 && o->unroll != 16) return MB_EINVAL;
  if (o && o->precision != MB_PREC_FP64) {
    if (!(allow & ALLOW_PRECISION) || o->precision > MB_PREC_DFLOAT || o->fp64_products) return MB_EINVAL;
  }
  if (o && o->cycle_check) {
    if (!(allow & ALLOW_CYCLE) || o->cycle_check != 1 || o->precision != MB_PREC_FP64 || o->fp64_products)
      return MB_EINVAL;
  }
  return MB_OK;
}

// ---- kernel table -------------------------------------------------------

template <int KIND, int SCHED, bool FILT>
static RenderFn pick_unroll(int unroll) {
  switch (unroll) {
    case 4: return render_kernel<KIND, SCHED, FILT, 4, true>;
    case 16: return render_kernel<KIND, SCHED, FILT, 16, true>;
    default: return render_kernel<KIND, SCHED, FILT, 8, true>;
  }
}

template <int KIND, int SCHED>
static RenderFn pick_filt(bool filt, int unroll) {
  return filt ? pick_unroll<KIND, SCHED, true>(unroll) : pick_unroll<KIND, SCHED, false>(unroll);
}

RenderFn render_fn(int kind, int sched, bool filt, int unroll) {
  if (kind == KIND_ROWS) {
    if (sched == S_NAIVE) return pick_filt<KIND_ROWS, S_NAIVE>(filt, unroll);
    if (sched == S_ALT) return pick_filt<KIND_ROWS, S_ALT>(filt, unroll);
    return pick_filt<KIND_ROWS, S_FCFS>(filt, unroll);
  }
  if (kind == KIND_RASTER) return pick_filt<KIND_RASTER, S_FCFS>(filt, unroll);
  if (kind == KIND_PROBE) return pick_filt<KIND_PROBE, S_FCFS>(filt, unroll);
  if (kind == KIND_LIST) return pick_filt<KIND_LIST, S_FCFS>(filt, unroll);
  return pick_filt<KIND_BATCH, S_FCFS>(filt, unroll);
}

// All-FP64 products (three multiplies on the FP64 pipe): raster tiles only,
// kept as the measured baseline of the integer-pipe products.
RenderFn render_fn_fp64(bool filt) {
  return filt ? render_kernel<KIND_RASTER, S_FCFS, true, 8, false> : render_kernel<KIND_RASTER, S_FCFS, false, 8, false>;
}

static std::mutex g_occ_mu;
static std::unordered_map<uint64_t, int> g_occ;

int sm_count() {
  static int sms = 0;
  int dev = 0;
  if (!sms) {
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  }
  return sms;
}

int resident_ctas(const void* fn, int block) {
  std::lock_guard<std::mutex> g(g_occ_mu);
  uint64_t key = (uint64_t)(uintptr_t)fn ^ ((uint64_t)block << 48);
  auto it = g_occ.find(key);
  if (it != g_occ.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, 0) != cudaSuccess || n < 1) n = 1;
  g_occ[key] = n;
  return n;
}

// ---- workspace ------------------------------------------------------------

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SingleLayout {
  size_t view, counter, cx, cy, total;
};

static SingleLayout single_layout(uint32_t m, uint32_t n) {
  SingleLayout L;
  L.view = 0;
  L.counter = align256(sizeof(ViewDesc));
  L.cx = L.counter + 256;
  L.cy = L.cx + align256((size_t)n * 8);
  L.total = L.cy + align256((size_t)m * 8);
  return L;
}

int launch_render(const RenderFn fn, const RenderParams& P, uint32_t grid, uint32_t block, cudaStream_t st) {
  fn<<<grid, block, 0, st>>>(P);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

int launch_render_timed(const RenderFn fn, const RenderParams& P, uint32_t grid, uint32_t block, cudaStream_t st,
                        const mb_opts* opt) {
  if (opt && opt->ev_start && cudaEventRecord((cudaEvent_t)opt->ev_start, st) != cudaSuccess) return MB_ECUDA;
  int rc = launch_render(fn, P, grid, block, st);
  if (rc == MB_OK && opt && opt->ev_stop && cudaEventRecord((cudaEvent_t)opt->ev_stop, st) != cudaSuccess)
    rc = MB_ECUDA;
  return rc;
}

uint32_t default_grid(RenderFn fn, uint32_t block) {
  return (uint32_t)(sm_count() * resident_ctas((const void*)fn, (int)block));
}

}  // namespace mb

using namespace mb;

extern "C" size_t mb_render_workspace_size(uint32_t m, uint32_t n, const mb_opts* opt) {
  (void)opt;
  return single_layout(m, n).total;
}

extern "C" int mb_render(const mb_window* w, uint32_t m, uint32_t n, uint32_t iter_max, double escape_r2,
                         uint32_t* out, const mb_opts* opt) {
  int rc = check_view(w, m, n, escape_r2, out);
  if (rc) return rc;
  rc = check_device_access(out);
  if (rc) return rc;
  uint32_t log2_tile = 0;
  rc = check_opts(opt, &log2_tile, ALLOW_PRECISION | ALLOW_CYCLE);
  if (rc) return rc;
  const int sched = opt ? opt->sched : MB_SCHED_FCFS_TILES;
  const uint32_t block = opt && opt->block ? opt->block : DEFAULT_BLOCK;
  cudaStream_t st = opt ? (cudaStream_t)opt->stream : nullptr;
  const uint32_t tile = 1u << log2_tile;
  const uint32_t tiles_x = (n + tile - 1) / tile, tiles_y = (m + tile - 1) / tile;
  if ((uint64_t)tiles_x * tiles_y >= END_ITEM) return MB_EINVAL;

  SingleLayout lay = single_layout(m, n);
  char* ws = nullptr;
  bool owned = false;
  if (opt && opt->workspace) {
    if (opt->workspace_bytes < lay.total) return MB_EINVAL;
    ws = (char*)opt->workspace;
  } else {
    if (cudaMallocAsync((void**)&ws, lay.total, st) != cudaSuccess) {
      cudaGetLastError();
      return MB_ENOMEM;
    }
    owned = true;
  }

  ViewDesc V;
  std::memset(&V, 0, sizeof V);
  V.cx = (const double*)(ws + lay.cx);
  V.cy = (const double*)(ws + lay.cy);
  V.out = out;
  V.totals = opt ? opt->tile_totals : nullptr;
  V.xmin = w->xmin;
  V.xmax = w->xmax;
  V.ymin = w->ymin;
  V.ymax = w->ymax;
  V.r2 = escape_r2;
  V.thr = make_thr(escape_r2);
  V.m = m;
  V.n = n;
  V.iter_max = iter_max;
  V.tiles_x = tiles_x;
  V.tiles_y = tiles_y;

  RenderParams P;
  std::memset(&P, 0, sizeof P);
  P.views = (const ViewDesc*)(ws + lay.view);
  P.log2_tile = log2_tile;
  P.counter = (uint32_t*)(ws + lay.counter);
  P.status = opt ? opt->status : nullptr;
  P.trace = opt ? opt->trace : nullptr;
  P.trace_len = opt && opt->trace ? opt->trace_len : 0;
  P.deadline_ns = opt_deadline_ns(opt);

  int kind, s;
  switch (sched) {
    case MB_SCHED_NAIVE: kind = KIND_ROWS; s = S_NAIVE; P.n_items = m; break;
    case MB_SCHED_ALTERNATING: kind = KIND_ROWS; s = S_ALT; P.n_items = m; break;
    case MB_SCHED_FCFS_ROWS: kind = KIND_ROWS; s = S_FCFS; P.n_items = m; break;
    case MB_SCHED_FCFS_ITEMS: kind = KIND_LIST; s = S_FCFS; P.n_items = opt->n_items; P.items = opt->items; break;
    default: kind = KIND_RASTER; s = S_FCFS; P.n_items = tiles_x * tiles_y; break;
  }
  const int prec = opt ? (int)opt->precision : PREC_F64;
  RenderFn fn = prec != PREC_F64       ? render_fn_lowp(kind, s, prec, opt_unroll(opt))
                : opt && opt->cycle_check ? render_fn_cycle(kind, s, filter_ok(escape_r2), opt_unroll(opt))
                                          : render_fn(kind, s, filter_ok(escape_r2), opt_unroll(opt));
  if (opt && opt->fp64_products) {
    if (kind != KIND_RASTER) {
      if (owned) cudaFreeAsync(ws, st);
      return MB_EINVAL;
    }
    fn = render_fn_fp64(filter_ok(escape_r2));
  }
  uint32_t grid = opt && opt->grid ? opt->grid : default_grid(fn, block);

  uint32_t map_blocks = (m + n + 255) / 256;
  if (map_blocks > 1024) map_blocks = 1024;
  pixel_map_single_kernel<<<map_blocks, 256, 0, st>>>(V, (ViewDesc*)(ws + lay.view), P.counter);
  rc = cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
  if (rc == MB_OK) {
    stats_begin(P, grid, st, out, (uint64_t)m * n);
    rc = launch_render_timed(fn, P, grid, block, st, opt);
    if (rc != MB_OK) stats_cancel();
  }
  if (owned) cudaFreeAsync(ws, st);
  return rc;
}
