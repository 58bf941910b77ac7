// render_noalloc.cu -- mb_render_noalloc: the render of mb_render for callers
// that may not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaMallocAsync are not
// allowed or not wanted -- a host callback or a real-time loop that must not
// take the allocator's locks, a process whose memory pool is reserved in full
// by another framework, or an embedding that forbids allocation after start-up.
// Such a caller still passes its own output buffer; the temporary memory the
// render needs (the view descriptor, the FCFS work counter and the Cx / Cy
// arrays) lives in one fixed array below, part of the library's device image.
//
// Limits and sharing:
//  - m and n are each at most MB_NOALLOC_MAX_SIDE (16384); larger sizes are
//    rejected with MB_EINVAL.  The array is 512 + 2 * 16384 * 8 bytes
//    (262,656 bytes) and stays resident on every GPU that loads the library
//    until the process exits.
//  - All calls on a device use the same array, which keeps whatever the last
//    call left in it.  The pixel-map kernel rewrites every part a render reads
//    (and zeroes the work counter) before the render kernel runs, so nothing
//    from an earlier call leaks into a result.  Calls whose kernels overlap on
//    the GPU (different streams, or different host threads without ordering)
//    race on the array; order them on one stream.
//  - The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress and caches it; make that first call before any
//    stream capture begins.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "mb.h"
#include "mb_internal.h"
#include "render_kernels.cuh"

namespace mb {

constexpr uint32_t NOALLOC_MAX_SIDE = MB_NOALLOC_MAX_SIDE;
constexpr size_t NOALLOC_VIEW = 0;          // ViewDesc
constexpr size_t NOALLOC_COUNTER = 256;     // FCFS work counter
constexpr size_t NOALLOC_CX = 512;          // Cx, then Cy right after the n entries of Cx
constexpr size_t NOALLOC_BYTES = NOALLOC_CX + 2 * (size_t)NOALLOC_MAX_SIDE * sizeof(double);
static_assert(sizeof(ViewDesc) <= NOALLOC_COUNTER, "view descriptor must fit its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device.  In host code
// the name g_noalloc_scratch stands for a host-side shadow, not device memory,
// so the kernel gets this address instead.
static int noalloc_scratch(char** p) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    cudaGetLastError();
    return MB_ECUDA;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* a = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
    if (e != cudaSuccess || !a) {
      cudaGetLastError();
      return MB_ECUDA;
    }
    g_noalloc_addr[dev] = a;
  }
  *p = (char*)g_noalloc_addr[dev];
  return MB_OK;
}

}  // namespace mb

using namespace mb;

extern "C" int mb_render_noalloc(const mb_window* w, uint32_t m, uint32_t n, uint32_t iter_max, double escape_r2,
                                 uint32_t* out, const mb_opts* opt) {
  int rc = check_view(w, m, n, escape_r2, out);
  if (rc) return rc;
  if (m > NOALLOC_MAX_SIDE || n > NOALLOC_MAX_SIDE) return MB_EINVAL;
  rc = check_device_access(out);
  if (rc) return rc;
  uint32_t log2_tile = 0;
  rc = check_opts(opt, &log2_tile);  // rejects precision != binary64 and cycle_check
  if (rc) return rc;
  if (opt && opt->workspace) return MB_EINVAL;    // the fixed array is the workspace here
  if (opt && opt->fp64_products) return MB_EINVAL;  // the all-FP64 baseline kernel comes with mb_render only
  const int sched = opt ? opt->sched : MB_SCHED_FCFS_TILES;
  const uint32_t block = opt && opt->block ? opt->block : DEFAULT_BLOCK;
  cudaStream_t st = opt ? (cudaStream_t)opt->stream : nullptr;
  const uint32_t tile = 1u << log2_tile;
  const uint32_t tiles_x = (n + tile - 1) / tile, tiles_y = (m + tile - 1) / tile;

  char* ws = nullptr;
  rc = noalloc_scratch(&ws);
  if (rc) return rc;

  ViewDesc V;
  std::memset(&V, 0, sizeof V);
  V.cx = (const double*)(ws + NOALLOC_CX);
  V.cy = (const double*)(ws + NOALLOC_CX + (size_t)n * sizeof(double));
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
  P.views = (const ViewDesc*)(ws + NOALLOC_VIEW);
  P.log2_tile = log2_tile;
  P.counter = (uint32_t*)(ws + NOALLOC_COUNTER);
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
  RenderFn fn = render_fn(kind, s, filter_ok(escape_r2), opt_unroll(opt));
  uint32_t grid = opt && opt->grid ? opt->grid : default_grid(fn, block);

  uint32_t map_blocks = (m + n + 255) / 256;
  if (map_blocks > 1024) map_blocks = 1024;
  pixel_map_single_kernel<<<map_blocks, 256, 0, st>>>(V, (ViewDesc*)(ws + NOALLOC_VIEW), P.counter);
  if (cudaGetLastError() != cudaSuccess) return MB_ECUDA;
  return launch_render_timed(fn, P, grid, block, st, opt);
}
