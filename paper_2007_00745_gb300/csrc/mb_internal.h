// mb_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mb.h"

namespace mb {

constexpr uint32_t MAX_SIDE = 1u << 20;
constexpr uint32_t DEFAULT_TILE = 64;
constexpr uint32_t DEFAULT_BLOCK = 256;
constexpr uint32_t DEFAULT_UNROLL = 4;  // measured fastest with the alternating integer subtraction

enum ItemKind : int { KIND_ROWS = 0, KIND_RASTER = 1, KIND_LIST = 2, KIND_BATCH = 3, KIND_PROBE = 4 };

// Low-resolution probe: PROBE_SIDE x PROBE_SIDE samples per tile (sample (a, b) at
// tile-local pixel (a*s + s/2, b*s + s/2), s = tile / PROBE_SIDE, clamped to the image).
constexpr uint32_t PROBE_SIDE = 8;
enum SchedKind : int { S_NAIVE = 0, S_ALT = 1, S_FCFS = 2 };
// Arithmetic of the escape step: the values of mb_opts.precision, and binary64
// with exact cycle detection (mb_opts.cycle_check).
enum Precision : int { PREC_F64 = 0, PREC_F32 = 1, PREC_F2 = 2, PREC_F64_CYCLE = 3 };

struct RenderParams;
struct EscThr;
using RenderFn = void (*)(RenderParams);

bool filter_ok(double r2);
EscThr make_thr(double r2);
int check_view(const mb_window* w, uint32_t m, uint32_t n, double r2, const void* out);
// MB_OK when the kernels of the current device can write through p: device memory of this
// device, managed memory, pinned / registered host memory mapped at the same address, or
// ordinary host memory on a device with pageable memory access (e.g. over NVLink-C2C).
int check_device_access(const void* p);
// Options an entry point honours beyond the common ones (check_opts rejects the others when set).
enum OptAllow : unsigned { ALLOW_PRECISION = 1u, ALLOW_CYCLE = 2u };
int check_opts(const mb_opts* o, uint32_t* log2_tile, unsigned allow = 0u);
RenderFn render_fn(int kind, int sched, bool filt, int unroll);
RenderFn render_fn_fp64(bool filt);
// binary32 / double-float kernels (render_lowp.cu): KIND_ROWS, KIND_RASTER, KIND_LIST and KIND_BATCH
RenderFn render_fn_lowp(int kind, int sched, int prec, int unroll);
// binary64 kernels with exact cycle detection (render_cycle.cu): KIND_ROWS, KIND_RASTER, KIND_LIST
// and KIND_BATCH; unroll 16, else 8
RenderFn render_fn_cycle(int kind, int sched, bool filt, int unroll);
int launch_render(const RenderFn fn, const RenderParams& P, uint32_t grid, uint32_t block, cudaStream_t st);
// launch_render with the caller's optional timing events around it (opts->ev_start / ev_stop)
int launch_render_timed(const RenderFn fn, const RenderParams& P, uint32_t grid, uint32_t block, cudaStream_t st,
                        const mb_opts* opt);
uint32_t default_grid(RenderFn fn, uint32_t block);
int sm_count();
int resident_ctas(const void* fn, int block);

// mb_last_stats bookkeeping (stats.cu): called right before the main render launch of
// mb_render / mb_render_learned; gives P a trace buffer if the caller gave none.
// stats_cancel() forgets the launch (call it when the launch failed).
void stats_begin(RenderParams& P, uint32_t grid, cudaStream_t st, const uint32_t* counts, uint64_t npix);
void stats_cancel();

// Longest-first item list with splits (the rule of mb_order_split, every tile cut into at
// least min_strips strips) over `nt` tiles numbered
// 0..nt-1, from their predicted costs -- the network `params` on their features `feat`
// (tiles x MB_MLP_FEATURES), or, when params is NULL, the probe-sum estimate from their
// probe counts (tiles x 64) -- after the neighbourhood guard (mb_guard_costs) within each
// view: view v owns tiles goff[v] .. goff[v+1]-1, tx[v] per row (device arrays; goff NULL:
// one view, tx[0] on the host side is not read -- pass goff and tx for several views).
// Temporaries live in `ws` when given (order_tiles_ws_bytes(nt) bytes, 256-byte aligned,
// not in use by other work on other streams), else in stream-ordered allocations on `st`.
int order_tiles(const uint32_t* probe, const float* feat, uint32_t nt, const float* params, uint32_t tile,
                uint32_t grid, uint32_t split, uint32_t min_strips, const uint32_t* goff, const uint32_t* tx,
                uint32_t nviews, mb_item* items, uint32_t capacity, uint32_t* n_items, uint32_t* status,
                cudaStream_t st, void* ws = nullptr);
size_t order_tiles_ws_bytes(uint32_t nt);

// Smallest number of strips a tile is cut into by the learned order (mb_opts.min_strips):
// 0 -> 1; callers validate it with min_strips_ok().
inline uint32_t opt_min_strips(const mb_opts* o, uint32_t) { return o && o->min_strips ? o->min_strips : 1u; }
inline bool min_strips_ok(const mb_opts* o, uint32_t tile) {
  uint32_t s = o ? o->min_strips : 0u;
  return s == 0 || ((s & (s - 1)) == 0 && s <= 16 && s <= tile);
}

inline int opt_unroll(const mb_opts* o) { return o && o->unroll ? (int)o->unroll : (int)DEFAULT_UNROLL; }
inline uint64_t opt_deadline_ns(const mb_opts* o) { return o && o->max_seconds ? o->max_seconds * 1000000000ull : 0ull; }

}  // namespace mb
