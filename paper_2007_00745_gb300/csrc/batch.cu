// batch.cu -- many viewports in one persistent launch, as a replayable CUDA graph.
//
// Every view gets its Cx / Cy arrays (Sec. III-A) in one pixel-map launch (one
// grid row per view); the render is one first-come-first-served launch
// (Sec. III-B) over a list of (view, tile) items.  By default views are queued
// in order of decreasing iteration budget (a cost bound known before
// rendering), tiles of a view in raster order.  With opts->learned_order the
// queue is built once, when the plan is made, from predicted tile costs: every
// view is probed (8 x 8 samples per tile), the tile-cost network (or the
// probe-sum estimate) predicts each tile's cost, and the tiles of all views are
// queued longest-first with heavy tiles split into row strips.  A plan owns
// its device memory and a captured graph of the two launches, so replaying a
// batch costs one cudaGraphLaunch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "mb.h"
#include "mb_internal.h"
#include "render_kernels.cuh"

struct mb_batch_plan {
  int device = 0;
  uint32_t count = 0, n_items = 0, tile = 64, block = 256, unroll = 8, grid = 0;
  char* dmem = nullptr;
  size_t bytes = 0;
  mb::ViewDesc* views = nullptr;
  mb::BatchItem* items = nullptr;
  mb::BatchItem* litems = nullptr;  // the learned queue (owned; items points to it when in use)
  uint32_t learned = 0;
  uint32_t* counter = nullptr;
  uint32_t* status = nullptr;
  mb::RenderFn fn = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t pixels = 0;
};

namespace mb {

static size_t b256(size_t x) { return (x + 255) & ~(size_t)255; }

// items of the batch: global tile g -> (view, tile); prefix[k] = first global tile of the k-th queued view
__global__ void batch_items_kernel(const uint32_t* __restrict__ prefix, const uint32_t* __restrict__ vorder,
                                   uint32_t nviews, uint32_t tile, BatchItem* __restrict__ items) {
  uint32_t total = prefix[nviews];
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = nviews;  // largest k with prefix[k] <= g
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) / 2;
      if (prefix[mid] <= g) lo = mid;
      else hi = mid;
    }
    BatchItem it;
    it.view = vorder[lo];
    it.tile = g - prefix[lo];
    it.row0 = 0;
    it.rows = (uint16_t)tile;
    items[g] = it;
  }
}

// Learned queue: global tile g of the batch (views in index order, goff[v] = first
// global tile of view v) -> (view, tile within the view), keeping the strip.
__global__ void batch_learned_items_kernel(const mb_item* __restrict__ in, uint32_t n, const uint32_t* __restrict__ goff,
                                           uint32_t nviews, BatchItem* __restrict__ out) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    mb_item e = in[k];
    uint32_t lo = 0, hi = nviews;  // largest v with goff[v] <= g
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) / 2;
      if (goff[mid] <= e.tile) lo = mid;
      else hi = mid;
    }
    BatchItem b;
    b.view = lo;
    b.tile = e.tile - goff[lo];
    b.row0 = e.row0;
    b.rows = e.rows;
    out[k] = b;
  }
}

// Build the learned queue of a plan (see the file comment).  Leaves the default
// queue in place when the list would not fit its capacity.
static int batch_learned_queue(const mb_view* views, uint32_t count, const mb_opts* opt, mb_batch_plan* P) {
  const uint32_t tile = P->tile;
  if (tile < 16 || !min_strips_ok(opt, tile)) return MB_EINVAL;
  const uint32_t smin = opt_min_strips(opt, tile);
  std::vector<uint32_t> goff(count + 1, 0), txs(count);
  for (uint32_t i = 0; i < count; ++i) {
    txs[i] = (views[i].n + tile - 1) / tile;
    goff[i + 1] = goff[i] + txs[i] * ((views[i].m + tile - 1) / tile);
  }
  const uint32_t nt = goff[count];
  const uint32_t split = opt->split ? (opt->split > 4096 ? 4096u : opt->split) : 4u;
  uint64_t cap64 = (smin + 1ull) * nt + 4ull * split * P->grid + 1024;
  if (cap64 > 16ull * nt) cap64 = 16ull * nt;
  if (cap64 >= 0xFFFFFFF0ull) return MB_EINVAL;
  const uint32_t cap = (uint32_t)cap64;
  size_t o_probe = 0, o_feat = b256((size_t)nt * 64 * 4);
  size_t o_items = o_feat + (opt->model ? b256((size_t)nt * MB_MLP_FEATURES * 4) : 0);
  size_t o_n = o_items + b256((size_t)cap * sizeof(mb_item));
  size_t o_goff = o_n + 256, o_tx = o_goff + b256((size_t)(count + 1) * 4), total = o_tx + b256((size_t)count * 4);
  char* tmp = nullptr;
  if (cudaMalloc((void**)&tmp, total) != cudaSuccess) {
    cudaGetLastError();
    return MB_ENOMEM;
  }
  uint32_t* probe = (uint32_t*)(tmp + o_probe);
  float* feat = opt->model ? (float*)(tmp + o_feat) : nullptr;
  mb_item* li = (mb_item*)(tmp + o_items);
  uint32_t* dn = (uint32_t*)(tmp + o_n);
  mb_opts po;
  std::memset(&po, 0, sizeof po);
  po.tile = tile;
  po.block = P->block;
  po.unroll = P->unroll;
  int rc = MB_OK;
  if (cudaMemcpy(tmp + o_goff, goff.data(), (count + 1) * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(tmp + o_tx, txs.data(), count * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    rc = MB_ECUDA;
  for (uint32_t i = 0; i < count && rc == MB_OK; ++i) {
    const mb_view& q = views[i];
    rc = mb_probe(&q.w, q.m, q.n, q.iter_max, q.escape_r2, probe + (size_t)goff[i] * 64, nullptr, &po);
    if (rc == MB_OK && feat)
      rc = mb_tile_features(probe + (size_t)goff[i] * 64, &q.w, q.m, q.n, q.iter_max, tile,
                            feat + (size_t)goff[i] * MB_MLP_FEATURES, nullptr);
  }
  if (rc == MB_OK)
    rc = order_tiles(probe, feat, nt, opt->model, tile, P->grid, split, smin, (const uint32_t*)(tmp + o_goff),
                     (const uint32_t*)(tmp + o_tx), count, li, cap, dn, nullptr, nullptr);
  uint32_t n = 0;
  if (rc == MB_OK && cudaMemcpy(&n, dn, 4, cudaMemcpyDeviceToHost) != cudaSuccess) rc = MB_ECUDA;
  if (rc == MB_OK && n > 0) {
    if (cudaMalloc((void**)&P->litems, (size_t)n * sizeof(BatchItem)) != cudaSuccess) {
      cudaGetLastError();
      rc = MB_ENOMEM;
    }
    if (rc == MB_OK) {
      uint32_t nb = (uint32_t)std::min<uint64_t>((n + 255) / 256, 4096);
      batch_learned_items_kernel<<<nb, 256>>>(li, n, (const uint32_t*)(tmp + o_goff), count, P->litems);
      if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = MB_ECUDA;
    }
    if (rc == MB_OK) {
      P->items = P->litems;
      P->n_items = n;
      P->learned = 1;
    }
  }
  cudaFree(tmp);
  return rc;
}

struct BatchLayout {
  size_t views, prefix, vorder, counter, status, cxy, items, total;
};

static int batch_prepare(const mb_view* views, uint32_t count, const mb_opts* opt, mb_batch_plan* P, bool graph) {
  if (!views || count == 0 || count > 65535) return MB_EINVAL;
  uint32_t log2_tile = 0;
  int rc = check_opts(opt, &log2_tile, ALLOW_CYCLE | ALLOW_PRECISION);
  if (rc) return rc;
  const uint32_t tile = 1u << log2_tile;
  bool filt = true;
  std::vector<uint32_t> tiles(count);
  uint64_t total_tiles = 0, cxy = 0;
  for (uint32_t i = 0; i < count; ++i) {
    rc = check_view(&views[i].w, views[i].m, views[i].n, views[i].escape_r2, views[i].out);
    if (rc) return rc;
    rc = check_device_access(views[i].out);
    if (rc) return rc;
    uint64_t t = (uint64_t)((views[i].n + tile - 1) / tile) * ((views[i].m + tile - 1) / tile);
    tiles[i] = (uint32_t)t;
    total_tiles += t;
    cxy += views[i].m + views[i].n;
    filt = filt && filter_ok(views[i].escape_r2);
    P->pixels += (uint64_t)views[i].m * views[i].n;
  }
  if (total_tiles >= 0xFFFFFFF0ull) return MB_EINVAL;
  // queue order: decreasing iteration budget, then view index
  std::vector<uint32_t> vorder(count);
  std::iota(vorder.begin(), vorder.end(), 0u);
  std::stable_sort(vorder.begin(), vorder.end(),
                   [&](uint32_t a, uint32_t b) { return views[a].iter_max > views[b].iter_max; });
  std::vector<uint32_t> prefix(count + 1, 0);
  for (uint32_t k = 0; k < count; ++k) prefix[k + 1] = prefix[k] + tiles[vorder[k]];

  BatchLayout L;
  L.views = 0;
  L.prefix = b256((size_t)count * sizeof(ViewDesc));
  L.vorder = L.prefix + b256((size_t)(count + 1) * 4);
  L.counter = L.vorder + b256((size_t)count * 4);
  L.status = L.counter + 256;
  L.cxy = L.status + 256;
  L.items = L.cxy + b256((size_t)cxy * 8);
  L.total = L.items + b256((size_t)total_tiles * sizeof(BatchItem));
  if (cudaGetDevice(&P->device) != cudaSuccess) return MB_ECUDA;
  if (cudaMalloc((void**)&P->dmem, L.total) != cudaSuccess) {
    cudaGetLastError();
    return MB_ENOMEM;
  }
  P->bytes = L.total;
  P->count = count;
  P->n_items = (uint32_t)total_tiles;
  P->tile = tile;
  P->block = opt && opt->block ? opt->block : DEFAULT_BLOCK;
  P->unroll = (uint32_t)opt_unroll(opt);
  P->views = (ViewDesc*)(P->dmem + L.views);
  P->items = (BatchItem*)(P->dmem + L.items);
  P->counter = (uint32_t*)(P->dmem + L.counter);
  P->status = opt && opt->status ? opt->status : (uint32_t*)(P->dmem + L.status);

  std::vector<ViewDesc> hv(count);
  uint64_t off = 0;
  for (uint32_t i = 0; i < count; ++i) {
    ViewDesc& V = hv[i];
    std::memset(&V, 0, sizeof V);
    const mb_view& q = views[i];
    V.cx = (const double*)(P->dmem + L.cxy) + off;
    V.cy = V.cx + q.n;
    off += q.m + q.n;
    V.out = q.out;
    V.xmin = q.w.xmin;
    V.xmax = q.w.xmax;
    V.ymin = q.w.ymin;
    V.ymax = q.w.ymax;
    V.r2 = q.escape_r2;
    V.thr = make_thr(q.escape_r2);
    V.m = q.m;
    V.n = q.n;
    V.iter_max = q.iter_max;
    V.tiles_x = (q.n + tile - 1) / tile;
    V.tiles_y = (q.m + tile - 1) / tile;
  }
  bool ok = cudaMemcpy(P->views, hv.data(), count * sizeof(ViewDesc), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(P->dmem + L.prefix, prefix.data(), (count + 1) * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(P->dmem + L.vorder, vorder.data(), count * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemset(P->dmem + L.status, 0, 256) == cudaSuccess;
  if (!ok) return MB_ECUDA;
  uint32_t ib = (uint32_t)std::min<uint64_t>((total_tiles + 255) / 256, 4096);
  batch_items_kernel<<<ib, 256>>>((const uint32_t*)(P->dmem + L.prefix), (const uint32_t*)(P->dmem + L.vorder),
                                  count, tile, P->items);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return MB_ECUDA;
  const int prec = opt ? (int)opt->precision : PREC_F64;
  P->fn = prec != PREC_F64              ? render_fn_lowp(KIND_BATCH, S_FCFS, prec, (int)P->unroll)
          : opt && opt->cycle_check ? render_fn_cycle(KIND_BATCH, S_FCFS, filt, (int)P->unroll)
                                    : render_fn(KIND_BATCH, S_FCFS, filt, (int)P->unroll);
  P->grid = opt && opt->grid ? opt->grid : default_grid(P->fn, P->block);
  (void)graph;
  if (opt && opt->learned_order) return batch_learned_queue(views, count, opt, P);
  return MB_OK;
}

// The two launches of a batch pass: pixel maps of all views (also zeroes the
// counter), then the FCFS render over the item list.
static int batch_enqueue(mb_batch_plan* P, cudaStream_t st, const mb_opts* opt) {
  dim3 g(64, P->count);
  pixel_map_kernel<<<g, 256, 0, st>>>(P->views, P->counter);
  if (cudaGetLastError() != cudaSuccess) return MB_ECUDA;
  RenderParams R;
  std::memset(&R, 0, sizeof R);
  R.views = P->views;
  R.bitems = P->items;
  R.n_items = P->n_items;
  R.log2_tile = 0;
  while ((1u << R.log2_tile) < P->tile) ++R.log2_tile;
  R.counter = P->counter;
  R.status = P->status;
  R.trace = opt ? opt->trace : nullptr;
  R.trace_len = opt && opt->trace ? opt->trace_len : 0;
  R.deadline_ns = opt_deadline_ns(opt);
  return launch_render_timed(P->fn, R, P->grid, P->block, st, opt);
}

static void plan_free(mb_batch_plan* P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  if (P->dmem) cudaFree(P->dmem);
  if (P->litems) cudaFree(P->litems);
  delete P;
}

}  // namespace mb

using namespace mb;

extern "C" int mb_render_batch(const mb_view* views, uint32_t count, const mb_opts* opt) {
  mb_batch_plan* P = new mb_batch_plan();
  int rc = batch_prepare(views, count, opt, P, false);
  cudaStream_t st = opt ? (cudaStream_t)opt->stream : nullptr;
  if (rc == MB_OK) rc = batch_enqueue(P, st, opt);
  if (rc == MB_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = MB_ECUDA;
  plan_free(P);
  return rc;
}

extern "C" int mb_batch_plan_create(const mb_view* views, uint32_t count, const mb_opts* opt, mb_batch_plan** plan) {
  if (!plan) return MB_EINVAL;
  *plan = nullptr;
  mb_batch_plan* P = new mb_batch_plan();
  int rc = batch_prepare(views, count, opt, P, true);
  if (rc == MB_OK && cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking) != cudaSuccess) rc = MB_ECUDA;
  if (rc == MB_OK) {
    if (cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = MB_ECUDA;
    int rc2 = rc == MB_OK ? batch_enqueue(P, P->cap_stream, opt) : rc;
    cudaGraph_t g = nullptr;
    if (rc == MB_OK) {
      if (cudaStreamEndCapture(P->cap_stream, &g) != cudaSuccess) rc = MB_ECUDA;
      P->graph = g;
      if (rc2 != MB_OK) rc = rc2;
    }
    if (rc == MB_OK && cudaGraphInstantiate(&P->exec, P->graph, 0) != cudaSuccess) rc = MB_ECUDA;
  }
  if (rc != MB_OK) {
    cudaGetLastError();
    plan_free(P);
    return rc;
  }
  *plan = P;
  return MB_OK;
}

extern "C" int mb_batch_plan_launch(mb_batch_plan* plan, void* stream) {
  if (!plan || !plan->exec) return MB_EINVAL;
  return cudaGraphLaunch(plan->exec, (cudaStream_t)stream) == cudaSuccess ? MB_OK : MB_ECUDA;
}

extern "C" int mb_batch_plan_info(const mb_batch_plan* plan, uint32_t* n_items, uint32_t* grid, uint64_t* pixels) {
  if (!plan) return MB_EINVAL;
  if (n_items) *n_items = plan->n_items;
  if (grid) *grid = plan->grid;
  if (pixels) *pixels = plan->pixels;
  return MB_OK;
}

extern "C" int mb_batch_plan_destroy(mb_batch_plan* plan) {
  if (!plan) return MB_EINVAL;
  cudaDeviceSynchronize();
  plan_free(plan);
  return MB_OK;
}

// ---- autotuner ------------------------------------------------------------------

namespace mb {

static std::mutex g_tune_mu;

static uint64_t fnv1a(const void* p, size_t n, uint64_t h) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

// key of a batch: its views (not their output pointers) and the sample stride
static uint64_t batch_key(const mb_view* views, uint32_t count, uint32_t stride, const mb_opts& base) {
  uint64_t h = 1469598103934665603ull;
  for (uint32_t i = 0; i < count; ++i) {
    h = fnv1a(&views[i].w, sizeof(mb_window), h);
    h = fnv1a(&views[i].m, 12, h);
    h = fnv1a(&views[i].escape_r2, 8, h);
  }
  h = fnv1a(&base.precision, 4, h);    // the arithmetic changes the best launch shape
  h = fnv1a(&base.cycle_check, 4, h);
  h = fnv1a(&base.learned_order, 4, h);
  return fnv1a(&stride, 4, h);
}

static bool cache_lookup(const char* path, uint64_t key, mb_opts* best, float* ms) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[256];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    unsigned long long k;
    unsigned t, b, u;
    float x;
    if (sscanf(line, "%llx %u %u %u %f", &k, &t, &b, &u, &x) == 5 && k == key) {
      best->tile = t;
      best->block = b;
      best->unroll = u;
      *ms = x;
      found = true;
    }
  }
  fclose(f);
  return found;
}

static void cache_store(const char* path, uint64_t key, const mb_opts* best, float ms) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%016llx %u %u %u %.4f\n", (unsigned long long)key, best->tile, best->block, best->unroll, ms);
  fclose(f);
}

}  // namespace mb

extern "C" int mb_batch_autotune(const mb_view* views, uint32_t count, const mb_opts* base, uint32_t sample_stride,
                                 const char* cache_path, mb_opts* best, float* best_ms) {
  if (!views || count == 0 || !best) return MB_EINVAL;
  if (sample_stride == 0) sample_stride = 1;
  std::lock_guard<std::mutex> g(g_tune_mu);
  mb_opts b;
  std::memset(&b, 0, sizeof b);
  if (base) b = *base;
  b.grid = 0;
  uint64_t key = batch_key(views, count, sample_stride, b);
  float ms = 0.0f;
  if (cache_lookup(cache_path, key, &b, &ms)) {
    *best = b;
    if (best_ms) *best_ms = ms;
    return MB_OK;
  }
  std::vector<mb_view> sample;
  for (uint32_t i = 0; i < count; i += sample_stride) sample.push_back(views[i]);
  const uint32_t tiles[] = {16, 32, 64};
  const uint32_t blocks[] = {256, 512};
  const uint32_t unrolls[] = {4, 8, 16};
  float best_t = 1e30f;
  mb_opts winner = b;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MB_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MB_ECUDA;
  }
  int first_error = MB_OK;  // a candidate that fails (e.g. out of memory) is skipped
  bool any = false;
  for (uint32_t t : tiles)
    for (uint32_t bl : blocks)
      for (uint32_t u : unrolls) {
        mb_opts o = b;
        o.tile = t;
        o.block = bl;
        o.unroll = u;
        o.trace = nullptr;
        mb_batch_plan* P = nullptr;
        int rc = mb_batch_plan_create(sample.data(), (uint32_t)sample.size(), &o, &P);
        float tm = 1e30f;
        for (int rep = 0; rep < 2 && rc == MB_OK; ++rep) {
          cudaEventRecord(e0, nullptr);
          rc = mb_batch_plan_launch(P, nullptr);
          cudaEventRecord(e1, nullptr);
          if (cudaEventSynchronize(e1) != cudaSuccess) rc = MB_ECUDA;
          float x = 0.0f;
          cudaEventElapsedTime(&x, e0, e1);
          if (rep > 0) tm = x;  // first launch warms up
        }
        if (P) mb_batch_plan_destroy(P);
        if (rc) {
          if (first_error == MB_OK) first_error = rc;
          continue;
        }
        any = true;
        if (tm < best_t) {
          best_t = tm;
          winner = o;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!any) return first_error;
  *best = winner;
  if (best_ms) *best_ms = best_t;
  cache_store(cache_path, key, &winner, best_t);
  return MB_OK;
}
