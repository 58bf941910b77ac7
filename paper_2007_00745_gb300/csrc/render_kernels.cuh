// render_kernels.cuh -- pixel map and the scheduled escape-time render kernel.
//
// One kernel family serves every scheduler of the paper's Sec. III and the
// batched / served modes.  A worker is one CTA.  The CTA keeps one 64-bit
// word in shared memory, (current item id : next pixel offset); a warp with
// idle lanes claims that many pixels with one shared atomicAdd.  The warp whose
// claim reaches the end of the item fetches the CTA's next item -- statically
// for the naive (Sec. III-A) and alternating (Sec. III-C) partitions, from a
// global atomic counter for first-come-first-served (Sec. III-B) -- and
// publishes it with one atomicExch; warps that claimed past the end wait
// (bounded) for that word to change and claim again.  A lane whose pixel
// finishes stores its count and takes a fresh pixel at the next refill, so
// lanes stay busy although trip counts differ wildly between pixels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "escape_core.cuh"
#include "escape_lowp.cuh"
#include "mb.h"
#include "mb_internal.h"

namespace mb {

// Per-view constants, in device memory.
struct ViewDesc {
  const double* cx;     // n entries: c_re of each column
  const double* cy;     // m entries: c_im of each row
  uint32_t* out;        // m*n counts
  uint64_t* totals;     // per-tile sums of counts (may be null)
  double xmin, xmax, ymin, ymax;
  double r2;
  EscThr thr;
  uint32_t m, n, iter_max, tiles_x, tiles_y;
  uint32_t pad_;
  const uint32_t* order;  // batched items only: if set, item tile k stands for tile order[k] of the view
};

// Work item of the batched list: rows [row0, row0+rows) of tile `tile` of view `view`.
struct BatchItem {
  uint32_t view;
  uint32_t tile;
  uint16_t row0, rows;
};
// load_item() reads both item kinds as 32-bit words, rows above row0 in the last word
static_assert(sizeof(mb_item) == 8 && sizeof(BatchItem) == 12, "item layouts");


// status bits
constexpr uint32_t ST_SPIN_TIMEOUT = 1u;
constexpr uint32_t ST_BAD_ITEM = 2u;
constexpr uint32_t ST_DEADLINE = 4u;

constexpr uint32_t END_ITEM = 0xFFFFFFFFu;
constexpr int SPIN_LIMIT = 1 << 22;  // ~0.3 s at 64 ns per try: far above any real wait

struct RenderParams {
  const ViewDesc* views;
  const mb_item* items;        // KIND_LIST
  const BatchItem* bitems;     // KIND_BATCH
  uint32_t n_items;            // rows (KIND_ROWS), tiles (KIND_RASTER / KIND_PROBE) or list length
  const uint32_t* n_items_dev; // if set, the list length is read from device memory instead
  uint32_t* probe_out;         // KIND_PROBE: counts, [tile][PROBE_SIDE^2]
  uint32_t skip_probe;         // tile kinds: 1 = leave the probe's sample pixels alone (already written)
  uint32_t log2_tile;
  uint32_t* counter;           // FCFS work counter (zeroed before launch)
  uint32_t* status;            // error bits (may be null)
  mb_cta_trace* trace;         // per-CTA record (may be null)
  uint32_t trace_len;          // records available at `trace`
  uint64_t deadline_ns;        // 0 = none; else a CTA stops (status ST_DEADLINE) once it has run this long
};

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smid() {
  uint32_t s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

__device__ __forceinline__ void set_status(const RenderParams& P, uint32_t bits) {
  if (P.status) atomicOr(P.status, bits);
}

// The words of one listed work item, read once by the claiming lane and handed
// to the warp (KIND_LIST: mb_item; KIND_BATCH: BatchItem), so that refills do
// not wait on a second read of the same item from global memory.
struct ItemWords {
  uint32_t view, tile, rr;  // rr = row0 | rows << 16
};

template <int KIND>
__device__ __forceinline__ ItemWords load_item(const RenderParams& P, uint32_t it) {
  ItemWords w{0u, it, 0u};
  if (KIND == KIND_LIST) {
    const uint32_t* e = reinterpret_cast<const uint32_t*>(P.items + it);
    w.tile = e[0];
    w.rr = e[1];
  } else if (KIND == KIND_BATCH) {
    const uint32_t* e = reinterpret_cast<const uint32_t*>(P.bitems + it);
    w.view = e[0];
    w.tile = e[1];
    w.rr = e[2];
  }
  return w;
}

// Pixels in item `it` (before edge clipping); `w` holds its words for listed kinds.
template <int KIND>
__device__ __forceinline__ uint32_t item_pixels(const RenderParams& P, const ItemWords& w) {
  if (KIND == KIND_ROWS) return P.views[0].n;
  if (KIND == KIND_RASTER) return 1u << (2 * P.log2_tile);
  if (KIND == KIND_PROBE) return PROBE_SIDE * PROBE_SIDE;
  return (w.rr >> 16) << P.log2_tile;
}

// Number of items: the host's count, or the device count a previous kernel wrote.
__device__ __forceinline__ uint32_t item_count(const RenderParams& P) {
  return P.n_items_dev ? *(volatile const uint32_t*)P.n_items_dev : P.n_items;
}

// First item of CTA b, and the item after `it`, among N items.
template <int SCHED>
__device__ __forceinline__ uint32_t first_item(const RenderParams& P, uint32_t N) {
  uint32_t G = gridDim.x, b = blockIdx.x;
  if (SCHED == S_NAIVE) {  // S_b = (N/G) b; the last CTA also takes N mod G (Sec. III-A)
    uint32_t per = N / G;
    uint32_t cnt = per + (b == G - 1 ? N % G : 0);
    return cnt ? per * b : END_ITEM;
  }
  if (SCHED == S_ALT) return b < N ? b : END_ITEM;  // rows b, b+G, ... (Sec. III-C)
  uint32_t k = atomicAdd(P.counter, 1u);             // Sec. III-B
  return k < N ? k : END_ITEM;
}

template <int SCHED>
__device__ __forceinline__ uint32_t next_item(const RenderParams& P, uint32_t it, uint32_t N) {
  uint32_t G = gridDim.x, b = blockIdx.x;
  if (SCHED == S_NAIVE) {
    uint32_t per = N / G;
    uint32_t last = per * (b + 1) + (b == G - 1 ? N % G : 0);
    return it + 1 < last ? it + 1 : END_ITEM;
  }
  if (SCHED == S_ALT) return it + G < N ? it + G : END_ITEM;
  uint32_t k = atomicAdd(P.counter, 1u);
  return k < N ? k : END_ITEM;
}

// Claim up to `need` pixels for the calling warp (lane 0 only) among N items.
// Returns the number granted (0 = no work left), the item, its first offset
// and (listed kinds) its words.
template <int KIND, int SCHED>
__device__ uint32_t claim(const RenderParams& P, unsigned long long* word, uint32_t* taken, uint32_t need, uint32_t N,
                          uint32_t& item, uint32_t& off, ItemWords& iw) {
  int spins = 0;
  for (;;) {
    unsigned long long w = atomicAdd(word, (unsigned long long)need);
    uint32_t it = (uint32_t)(w >> 32), o = (uint32_t)w;
    if (it == END_ITEM) return 0;
    ItemWords e = load_item<KIND>(P, it);
    uint32_t Pn = item_pixels<KIND>(P, e);
    if (Pn == 0 && o == 0) {  // an empty item (rows = 0 in a list): its unique first claimer moves on
      uint32_t nx = next_item<SCHED>(P, it, N);
      if (nx != END_ITEM) atomicAdd(taken, 1u);
      atomicExch(word, (unsigned long long)nx << 32);
      continue;
    }
    if (o < Pn) {
      item = it;
      off = o;
      iw = e;
      if (o + need >= Pn) {  // this claim reaches the item's end: advance the CTA
        uint32_t nx = next_item<SCHED>(P, it, N);
        if (nx != END_ITEM) atomicAdd(taken, 1u);
        atomicExch(word, (unsigned long long)nx << 32);
        return Pn - o;
      }
      return need;
    }
    // Claimed past the end: another warp is fetching the next item.
    while ((uint32_t)(*(volatile unsigned long long*)word >> 32) == it) {
      if (++spins > SPIN_LIMIT) {
        set_status(P, ST_SPIN_TIMEOUT);
        return 0;
      }
      __nanosleep(64);
    }
  }
}

// Map pixel `pix` of item `it` to (view, row, col); false if it lies outside the image.
template <int KIND>
__device__ __forceinline__ bool decode(const RenderParams& P, uint32_t it, const ItemWords& e, uint32_t pix,
                                       uint32_t& v, uint32_t& row, uint32_t& col, uint32_t& tile) {
  if (KIND == KIND_ROWS) {
    v = 0;
    row = it;
    col = pix;
    tile = 0;
    return true;
  }
  if (KIND == KIND_PROBE) {
    const ViewDesc& V = P.views[0];
    uint32_t ty = it / V.tiles_x, tx = it - ty * V.tiles_x;
    uint32_t st = (1u << P.log2_tile) / PROBE_SIDE;
    v = 0;
    tile = it;
    row = min((ty << P.log2_tile) + (pix / PROBE_SIDE) * st + st / 2, V.m - 1);
    col = min((tx << P.log2_tile) + (pix % PROBE_SIDE) * st + st / 2, V.n - 1);
    return true;
  }
  uint32_t t, r0;
  if (KIND == KIND_RASTER) {
    v = 0;
    t = it;
    r0 = 0;
  } else {  // listed kinds: the words the claiming lane read
    v = KIND == KIND_BATCH ? e.view : 0u;
    t = e.tile;
    r0 = e.rr & 0xFFFFu;
  }
  if ((r0 + (pix >> P.log2_tile)) >> P.log2_tile) {  // item reaches past its tile
    if (P.status) atomicOr(P.status, ST_BAD_ITEM);
    return false;
  }
  const ViewDesc& V = P.views[v];
  if (KIND == KIND_BATCH && V.order) t = V.order[t];  // a served request's learned tile order
  uint32_t ty = t / V.tiles_x, tx = t - ty * V.tiles_x;
  uint32_t lr = r0 + (pix >> P.log2_tile), lc = pix & ((1u << P.log2_tile) - 1u);
  row = (ty << P.log2_tile) + lr;
  col = (tx << P.log2_tile) + lc;
  tile = t;
  if (P.skip_probe) {  // the probe kernel already wrote its in-image sample pixels
    uint32_t st = (1u << P.log2_tile) / PROBE_SIDE;
    if ((lr % st) == st / 2 && (lc % st) == st / 2) return false;
  }
  return ty < V.tiles_y && row < V.m && col < V.n;
}

// The worker loop of every render kernel.  PREC selects the lane arithmetic:
// the exact binary64 step (escape_core.cuh) or a reduced-precision one
// (escape_lowp.cuh; FILT and EMUL then unused).
template <int KIND, int SCHED, bool FILT, int UNROLL, bool EMUL, int PREC>
__device__ __forceinline__ void render_body(RenderParams P) {
  __shared__ unsigned long long s_word;
  __shared__ uint32_t s_taken, s_items;
  __shared__ uint64_t s_t0;
  const int lane = threadIdx.x & 31;
  uint64_t t_start = 0;
  if (threadIdx.x == 0) {
    t_start = globaltimer_ns();
    s_t0 = t_start;
    s_items = item_count(P);  // fixed for the launch: read once per CTA
    uint32_t it = first_item<SCHED>(P, s_items);
    s_word = (unsigned long long)it << 32;
    s_taken = it != END_ITEM ? 1u : 0u;
  }
  __syncthreads();
  const uint32_t n_items = s_items;

  typename LaneOf<PREC>::type L;
  lane_clear(L);
  bool has = false;
  bool drained = false;
  uint32_t* optr = nullptr;
  uint32_t* pptr = nullptr;
  uint64_t* tptr = nullptr;
  double r2 = 4.0;
  EscThr thr{3.99f, 4.01f};

  for (;;) {
    // Settle provisional escape decisions, then retire finished pixels.
    resolve<UNROLL>(L, r2);
    if (has && !L.live) {
      *optr = L.cnt;
      if (KIND == KIND_PROBE && pptr) *pptr = L.cnt;
      if (tptr) atomicAdd((unsigned long long*)tptr, (unsigned long long)L.cnt);
      has = false;
    }
    // Refill idle lanes.
    unsigned idle = __ballot_sync(FULL_MASK, !has);
    while (idle && !drained) {
      uint32_t need = __popc(idle), item = 0, off = 0, got = 0;
      ItemWords iw{0u, 0u, 0u};
      if (lane == 0) got = claim<KIND, SCHED>(P, &s_word, &s_taken, need, n_items, item, off, iw);
      got = __shfl_sync(FULL_MASK, got, 0);
      if (got == 0) {
        drained = true;
        break;
      }
      item = __shfl_sync(FULL_MASK, item, 0);
      off = __shfl_sync(FULL_MASK, off, 0);
      if (KIND == KIND_LIST || KIND == KIND_BATCH) {
        iw.tile = __shfl_sync(FULL_MASK, iw.tile, 0);
        iw.rr = __shfl_sync(FULL_MASK, iw.rr, 0);
        if (KIND == KIND_BATCH) iw.view = __shfl_sync(FULL_MASK, iw.view, 0);
      }
      uint32_t rank = __popc(idle & ((1u << lane) - 1u));
      if (!has && rank < got) {
        uint32_t v, row, col, tile;
        if (decode<KIND>(P, item, iw, off + rank, v, row, col, tile)) {
          const ViewDesc& V = P.views[v];
          lane_start(L, V.cx[col], V.cy[row], V.iter_max, V.r2);
          r2 = V.r2;
          thr = V.thr;
          optr = V.out ? V.out + (size_t)row * V.n + col : nullptr;
          tptr = V.totals ? V.totals + tile : nullptr;
          if (KIND == KIND_PROBE) {  // probe slot, plus the image pixel when an image is given
            uint32_t* slot = P.probe_out + (size_t)item * (PROBE_SIDE * PROBE_SIDE) + off + rank;
            pptr = optr ? slot : nullptr;
            optr = optr ? optr : slot;
            tptr = nullptr;
          }
          has = true;
        }
      }
      idle = __ballot_sync(FULL_MASK, !has);
    }
    if (__ballot_sync(FULL_MASK, has) == 0) break;
    if (P.deadline_ns && globaltimer_ns() - s_t0 > P.deadline_ns) {  // guard against a run-away launch
      if (lane == 0) set_status(P, ST_DEADLINE);
      break;
    }
    block_begin(L);
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) step<FILT, EMUL>(L, r2, thr, isub_step(u));
  }

  __syncthreads();
  if (threadIdx.x == 0 && P.trace && blockIdx.x < P.trace_len) {
    mb_cta_trace rec;
    rec.start_ns = t_start;
    rec.end_ns = globaltimer_ns();
    rec.smid = smid();
    rec.items = s_taken;
    P.trace[blockIdx.x] = rec;
  }
}

template <int KIND, int SCHED, bool FILT, int UNROLL, bool EMUL, int PREC = PREC_F64>
__global__ void __launch_bounds__(512) render_kernel(RenderParams P) {
  render_body<KIND, SCHED, FILT, UNROLL, EMUL, PREC>(P);
}

// Double-float lanes need about 50 registers; without a lower bound on resident
// CTAs the compiler keeps them to 32 and spills.  Two 512-thread CTAs per SM
// allow 64.
template <int KIND, int SCHED, int UNROLL>
__global__ void __launch_bounds__(512, 2) render_kernel_f2(RenderParams P) {
  render_body<KIND, SCHED, false, UNROLL, false, PREC_F2>(P);
}

// Cx / Cy arrays of one or more views (Sec. III-A: every task precomputes them),
// one view per blockIdx.y.  Also zeroes the FCFS counter.
static __global__ void pixel_map_kernel(const ViewDesc* views, uint32_t* counter) {
  const ViewDesc& V = views[blockIdx.y];
  if (counter && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *counter = 0;
  double sx = __dsub_rn(V.xmax, V.xmin);
  double sy = __dsub_rn(V.ymax, V.ymin);
  double dn = (double)V.n, dm = (double)V.m;
  double* cx = const_cast<double*>(V.cx);
  double* cy = const_cast<double*>(V.cy);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < V.n + V.m; k += gridDim.x * blockDim.x) {
    if (k < V.n) {
      cx[k] = __dadd_rn(V.xmin, __ddiv_rn(__dmul_rn((double)k, sx), dn));
    } else {
      uint32_t i = k - V.n;
      cy[i] = __dsub_rn(V.ymax, __ddiv_rn(__dmul_rn((double)i, sy), dm));
    }
  }
}

// Single-view form: takes the descriptor by value and also stores it for the
// render kernel that follows on the same stream.
static __global__ void pixel_map_single_kernel(ViewDesc V, ViewDesc* dst, uint32_t* counter) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *dst = V;
    if (counter) *counter = 0;
  }
  double sx = __dsub_rn(V.xmax, V.xmin);
  double sy = __dsub_rn(V.ymax, V.ymin);
  double dn = (double)V.n, dm = (double)V.m;
  double* cx = const_cast<double*>(V.cx);
  double* cy = const_cast<double*>(V.cy);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < V.n + V.m; k += gridDim.x * blockDim.x) {
    if (k < V.n) {
      cx[k] = __dadd_rn(V.xmin, __ddiv_rn(__dmul_rn((double)k, sx), dn));
    } else {
      uint32_t i = k - V.n;
      cy[i] = __dsub_rn(V.ymax, __ddiv_rn(__dmul_rn((double)i, sy), dm));
    }
  }
}

}  // namespace mb
