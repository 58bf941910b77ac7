// serve.cu -- continuous-batching render server.
//
// Requests (one view each) are admitted while their device memory (counts,
// Cx / Cy arrays) fits a byte budget; the rest wait in a bounded queue.  A
// worker thread keeps up to four rounds in flight on four streams: each round is
// one first-come-first-served launch (Sec. III-B) over the next tiles of every
// live request, oldest request first, so a request that arrives while others
// are on the GPU joins the very next round and shares the machine with them.
// When a round's event fires, its tiles are done; a request whose tiles are all
// done is complete.  All per-request state (view descriptor, Cx / Cy, counts)
// stays on the device; the host keeps only tile counters and timestamps.
// With opts->learned_order each admitted request is probed once (8 x 8
// samples per tile, written into its counts and skipped by the rounds), its
// tiles' costs are predicted (network or probe-sum estimate), guarded and
// ranked longest-first on the device; rounds then hand out its tiles by rank,
// and the render kernel reads the tile through that permutation.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mb.h"
#include "mb_internal.h"
#include "render_kernels.cuh"

namespace mb {

static uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

static size_t s256(size_t x) { return (x + 255) & ~(size_t)255; }

enum ReqState { RQ_QUEUED, RQ_LIVE, RQ_DONE, RQ_FAILED };

struct Req {
  uint64_t id = 0;
  mb_request rq{};
  ReqState state = RQ_QUEUED;
  int status = MB_OK;
  uint32_t slot = 0;
  size_t bytes = 0;
  char* dmem = nullptr;  // counts then Cx, Cy
  uint32_t tiles = 0, tiles_x = 0, next_tile = 0, done_tiles = 0;
  uint64_t submit_ns = 0, admit_ns = 0, start_ns = 0, done_ns = 0;
  bool released = false;
};

struct Round {
  cudaEvent_t ev = nullptr;
  std::vector<std::pair<uint64_t, uint32_t>> parts;  // (request id, tiles in this round)
  BatchItem* h_items = nullptr;                      // pinned
  BatchItem* d_items = nullptr;
  uint32_t* d_counter = nullptr;
  bool busy = false;
};

constexpr uint32_t SERVE_SLOTS = 4096;
// Rounds in flight: a round that ends on a heavy tile holds its stream for a
// while; with more rounds queued the other streams keep the GPU covered.
constexpr int SERVE_STREAMS = 4;
// Set-up streams of the learned order: each admitted request's probe and ranking run on one
// of them in turn, so that one large request's probe does not hold back the next ones'.
constexpr int SERVE_SETUP = 4;

}  // namespace mb

struct mb_server {
  int device = 0;
  size_t budget = 0, in_use = 0, peak = 0;
  uint32_t queue_limit = 0, tile = 32, block = 512, unroll = 16, grid = 0, round_tiles = 0;
  bool filt_all = true;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_idle;
  int waiters = 0;  // threads inside mb_serve_wait; destroy drains them first
  std::thread worker;
  bool stop = false;
  int failed = MB_OK;
  uint64_t next_id = 1;
  std::unordered_map<uint64_t, mb::Req> reqs;
  std::deque<uint64_t> queue;  // waiting for memory
  std::deque<uint64_t> live;   // admitted, tiles not all handed out yet (admission order)
  std::vector<uint32_t> free_slots;
  mb::ViewDesc* d_views = nullptr;
  mb::ViewDesc* h_view_stage = nullptr;  // pinned
  cudaStream_t setup = nullptr, streams[mb::SERVE_STREAMS] = {};
  std::vector<cudaEvent_t> slot_ev;  // per view slot: the admitted request's set-up work is done
  bool setup_pending = false;        // a live request's set-up was still running at the last round
  cudaMemPool_t pool = nullptr;  // the server's own pool: freed request memory stays reserved for the next ones
  mb::Round rounds[mb::SERVE_STREAMS];
  mb::RenderFn fn_filt = nullptr, fn_exact = nullptr, fn_probe_filt = nullptr, fn_probe_exact = nullptr;
  bool learned = false;         // opts->learned_order: rank each request's tiles by predicted cost
  const float* model = nullptr;  // the tile-cost network (may be null: probe-sum estimate)
  uint32_t* d_probe_counter = nullptr;  // one FCFS counter per learned set-up stream, 128 bytes apart
  cudaStream_t lsetup[mb::SERVE_SETUP] = {};
  uint32_t next_lsetup = 0;
  mb_serve_counters ctr{};
};

namespace mb {

// Device memory of a request: counts, Cx / Cy, and for a learned order the probe
// counts, features, ranked items, permutation and the view table of its ranking.
struct ReqLayout {
  size_t cx, probe, feat, items, perm, meta, ows, total;
};

static ReqLayout req_layout(const mb_request& r, uint32_t tile, bool learned, bool model) {
  ReqLayout L;
  const size_t nt = (size_t)((r.n + tile - 1) / tile) * ((r.m + tile - 1) / tile);
  L.cx = s256((size_t)r.m * r.n * 4);
  L.probe = L.cx + s256((size_t)(r.m + r.n) * 8);
  L.feat = L.probe + (learned ? s256(nt * 64 * 4) : 0);
  L.items = L.feat + (learned && model ? s256(nt * MB_MLP_FEATURES * 4) : 0);
  L.perm = L.items + (learned ? s256(nt * sizeof(mb_item)) : 0);
  L.meta = L.perm + (learned ? s256(nt * 4) : 0);
  L.ows = L.meta + (learned ? 256 : 0);  // the ranking's temporaries: no allocation at admission
  L.total = L.ows + (learned ? order_tiles_ws_bytes((uint32_t)nt) : 0);
  return L;
}

// meta = {goff = (0, nt), tx = (tiles_x), n_items}: the one-view table order_tiles reads
__global__ void serve_meta_kernel(uint32_t* meta, uint32_t nt, uint32_t tiles_x) {
  meta[0] = 0u;
  meta[1] = nt;
  meta[2] = tiles_x;
  meta[3] = 0u;
}

// perm[k] = tile of rank k; the identity if the ranking did not produce one item per tile
__global__ void serve_perm_kernel(const mb_item* __restrict__ items, uint32_t nt, const uint32_t* __restrict__ n_items,
                                  uint32_t* __restrict__ perm) {
  const bool ok = *n_items == nt;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nt; k += gridDim.x * blockDim.x)
    perm[k] = ok ? items[k].tile : k;
}

// Probe, predict, guard and rank one admitted request's tiles on the setup stream.
static int learn_order_locked(mb_server* S, Req& R, cudaStream_t st, uint32_t* counter) {
  ReqLayout L = req_layout(R.rq, S->tile, true, S->model != nullptr);
  const uint32_t nt = R.tiles;
  uint32_t* probe = (uint32_t*)(R.dmem + L.probe);
  float* feat = S->model ? (float*)(R.dmem + L.feat) : nullptr;
  mb_item* items = (mb_item*)(R.dmem + L.items);
  uint32_t* meta = (uint32_t*)(R.dmem + L.meta);
  uint32_t log2_tile = 0;
  while ((1u << log2_tile) < S->tile) ++log2_tile;
  if (cudaMemsetAsync(counter, 0, 4, st) != cudaSuccess) return MB_ECUDA;
  RenderParams PP;
  std::memset(&PP, 0, sizeof PP);
  PP.views = S->d_views + R.slot;
  PP.log2_tile = log2_tile;
  PP.counter = counter;
  PP.probe_out = probe;
  PP.n_items = nt;
  RenderFn fp = filter_ok(R.rq.escape_r2) ? S->fn_probe_filt : S->fn_probe_exact;
  // Narrow CTAs: one probe tile is 64 pixels, two warps' worth.  The probe runs beside the
  // rounds, and a full-width CTA holds a round-sized slot of registers for two busy warps until
  // its slowest sample ends; 64-thread CTAs fit beside the rounds' CTAs instead (measured at
  // saturation, 2000 req/s: 186.6 against 183.9 Giter/s with the rounds' launch shape).
  const uint32_t pgrid = std::min<uint32_t>(nt, (uint32_t)std::max(sm_count(), 1) * 4u);
  int rc = launch_render(fp, PP, pgrid, PROBE_SIDE * PROBE_SIDE, st);
  if (rc) return rc;
  serve_meta_kernel<<<1, 1, 0, st>>>(meta, nt, R.tiles_x);
  if (cudaGetLastError() != cudaSuccess) return MB_ECUDA;
  if (feat) {
    rc = mb_tile_features(probe, &R.rq.w, R.rq.m, R.rq.n, R.rq.iter_max, S->tile, feat, st);
    if (rc) return rc;
  }
  // one rank per tile: a work list without splits (one worker, split divisor 1)
  rc = order_tiles(probe, feat, nt, S->model, S->tile, 1u, 1u, 1u, meta, meta + 2, 1u, items, nt, meta + 3, nullptr,
                   st, R.dmem + L.ows);
  if (rc) return rc;
  serve_perm_kernel<<<(nt + 255) / 256 < 1024 ? (nt + 255) / 256 : 1024, 256, 0, st>>>(
      items, nt, meta + 3, (uint32_t*)(R.dmem + L.perm));
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

static size_t req_bytes(const mb_server* S, const mb_request& r) {
  return req_layout(r, S->tile, S->learned, S->model != nullptr).total;
}

// Admit queued requests that fit (caller holds the lock).  Device work is
// enqueued on the setup stream and followed by the request's slot event; a
// round takes a request's tiles only once that event has completed, so no
// round waits for another request's set-up (its probe, with the learned order).
static int admit_locked(mb_server* S, bool* capped) {
  // A learned admission enqueues a dozen launches; a burst of arrivals is taken a few at a
  // time so that the worker keeps launching rounds in between (*capped: more are waiting).
  int cap = S->learned ? 8 : 1 << 30;
  *capped = false;
  while (!S->queue.empty() && !S->free_slots.empty()) {
    if (cap-- == 0) {
      *capped = true;
      break;
    }
    Req& R = S->reqs[S->queue.front()];
    if (S->in_use + R.bytes > S->budget) break;
    cudaStream_t st = S->setup;
    uint32_t j = 0;
    if (S->learned) {
      j = S->next_lsetup++ % SERVE_SETUP;
      st = S->lsetup[j];
    }
    if (cudaMallocFromPoolAsync((void**)&R.dmem, R.bytes, S->pool, st) != cudaSuccess) {
      cudaGetLastError();
      return MB_ECUDA;
    }
    S->queue.pop_front();
    S->in_use += R.bytes;
    S->peak = std::max(S->peak, S->in_use);
    R.slot = S->free_slots.back();
    S->free_slots.pop_back();
    ViewDesc& V = S->h_view_stage[R.slot];
    std::memset(&V, 0, sizeof V);
    V.out = (uint32_t*)R.dmem;
    V.cx = (const double*)(R.dmem + s256((size_t)R.rq.m * R.rq.n * 4));
    V.cy = V.cx + R.rq.n;
    V.xmin = R.rq.w.xmin;
    V.xmax = R.rq.w.xmax;
    V.ymin = R.rq.w.ymin;
    V.ymax = R.rq.w.ymax;
    V.r2 = R.rq.escape_r2;
    V.thr = make_thr(R.rq.escape_r2);
    V.m = R.rq.m;
    V.n = R.rq.n;
    V.iter_max = R.rq.iter_max;
    V.tiles_x = (R.rq.n + S->tile - 1) / S->tile;
    V.tiles_y = (R.rq.m + S->tile - 1) / S->tile;
    if (S->learned) V.order = (const uint32_t*)(R.dmem + req_layout(R.rq, S->tile, true, S->model != nullptr).perm);
    if (cudaMemcpyAsync(S->d_views + R.slot, &V, sizeof V, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return MB_ECUDA;
    pixel_map_kernel<<<dim3(16, 1), 256, 0, st>>>(S->d_views + R.slot, nullptr);
    if (cudaGetLastError() != cudaSuccess) return MB_ECUDA;
    if (S->learned) {
      int rc = learn_order_locked(S, R, st, S->d_probe_counter + 32u * j);
      if (rc) return rc;
    }
    if (!S->slot_ev[R.slot] && cudaEventCreateWithFlags(&S->slot_ev[R.slot], cudaEventDisableTiming) != cudaSuccess)
      return MB_ECUDA;
    if (cudaEventRecord(S->slot_ev[R.slot], st) != cudaSuccess) return MB_ECUDA;
    R.state = RQ_LIVE;
    R.admit_ns = now_ns();
    S->live.push_back(R.id);
    S->ctr.admitted++;
  }
  return MB_OK;
}

// Fill and launch one round on stream k (caller holds the lock).  Returns false if there was no work.
static int launch_round_locked(mb_server* S, int k, bool* launched) {
  Round& Rd = S->rounds[k];
  *launched = false;
  uint32_t nit = 0;
  Rd.parts.clear();
  uint64_t t = now_ns();
  S->setup_pending = false;
  for (auto it = S->live.begin(); it != S->live.end() && nit < S->round_tiles;) {
    Req& R = S->reqs[*it];
    cudaError_t q = cudaEventQuery(S->slot_ev[R.slot]);
    if (q == cudaErrorNotReady) {  // its set-up is still running: it joins a later round
      S->setup_pending = true;
      ++it;
      continue;
    }
    if (q != cudaSuccess) {
      cudaGetLastError();
      return MB_ECUDA;
    }
    uint32_t take = std::min(R.tiles - R.next_tile, S->round_tiles - nit);
    for (uint32_t j = 0; j < take; ++j) {
      BatchItem b;
      b.view = R.slot;
      b.tile = R.next_tile + j;
      b.row0 = 0;
      b.rows = (uint16_t)S->tile;
      Rd.h_items[nit + j] = b;
    }
    if (take) {
      Rd.parts.emplace_back(R.id, take);
      if (R.next_tile == 0) R.start_ns = t;
    }
    R.next_tile += take;
    nit += take;
    if (R.next_tile == R.tiles) it = S->live.erase(it);
    else ++it;
  }
  if (nit == 0) return MB_OK;
  cudaStream_t st = S->streams[k];
  if (cudaMemcpyAsync(Rd.d_items, Rd.h_items, (size_t)nit * sizeof(BatchItem), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemsetAsync(Rd.d_counter, 0, 4, st) != cudaSuccess)
    return MB_ECUDA;
  RenderParams P;
  std::memset(&P, 0, sizeof P);
  P.views = S->d_views;
  P.bitems = Rd.d_items;
  P.n_items = nit;
  P.log2_tile = 0;
  while ((1u << P.log2_tile) < S->tile) ++P.log2_tile;
  P.counter = Rd.d_counter;
  P.skip_probe = S->learned ? 1u : 0u;  // the probe already wrote its samples
  int rc = launch_render(S->filt_all ? S->fn_filt : S->fn_exact, P, S->grid, S->block, st);
  if (rc) return rc;
  if (cudaEventRecord(Rd.ev, st) != cudaSuccess) return MB_ECUDA;
  Rd.busy = true;
  S->ctr.rounds++;
  *launched = true;
  return MB_OK;
}

static void fail_all_locked(mb_server* S, int code) {
  S->failed = code;
  for (auto& kv : S->reqs) {
    if (kv.second.state == RQ_QUEUED || kv.second.state == RQ_LIVE) {
      kv.second.state = RQ_FAILED;
      kv.second.status = code;
      kv.second.done_ns = now_ns();
    }
  }
  S->queue.clear();
  S->live.clear();
  S->setup_pending = false;
  S->cv_done.notify_all();
}

static void worker_main(mb_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  int next = 0;
  while (true) {
    bool capped = false;
    if (S->failed == MB_OK) {
      int rc = admit_locked(S, &capped);
      if (rc) fail_all_locked(S, rc);
    }
    // launch into every idle stream while there is work
    bool launched_any = false;
    for (int i = 0; i < SERVE_STREAMS && S->failed == MB_OK; ++i) {
      int k = (next + i) % SERVE_STREAMS;
      if (S->rounds[k].busy) continue;
      bool launched = false;
      int rc = launch_round_locked(S, k, &launched);
      if (rc) {
        fail_all_locked(S, rc);
        break;
      }
      if (launched) {
        launched_any = true;
        next = (k + 1) % SERVE_STREAMS;
      }
    }
    // retire finished rounds
    bool busy = false;
    for (int k = 0; k < SERVE_STREAMS; ++k) {
      Round& Rd = S->rounds[k];
      if (!Rd.busy) continue;
      cudaError_t q = cudaEventQuery(Rd.ev);
      if (q == cudaErrorNotReady) {
        busy = true;
        continue;
      }
      Rd.busy = false;
      if (q != cudaSuccess) {
        cudaGetLastError();
        fail_all_locked(S, MB_ECUDA);
        continue;
      }
      uint64_t t = now_ns();
      for (auto& pr : Rd.parts) {
        auto it = S->reqs.find(pr.first);
        if (it == S->reqs.end()) continue;
        Req& R = it->second;
        R.done_tiles += pr.second;
        if (R.done_tiles == R.tiles && R.state == RQ_LIVE) {
          R.state = RQ_DONE;
          R.done_ns = t;
          S->ctr.completed++;
        }
      }
      S->cv_done.notify_all();
    }
    if (S->stop && !busy && !launched_any && !S->setup_pending && !capped) break;
    if (busy || launched_any || S->setup_pending || capped) {
      // poll the in-flight rounds without holding the lock for long
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(100));
      lk.lock();
    } else {
      S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
  }
}

}  // namespace mb

using namespace mb;

extern "C" int mb_serve_create(size_t mem_budget_bytes, uint32_t queue_limit, const mb_opts* opt, mb_server** out) {
  if (!out || mem_budget_bytes == 0) return MB_EINVAL;
  *out = nullptr;
  uint32_t log2_tile = 0;
  mb_opts o;
  std::memset(&o, 0, sizeof o);
  if (opt) o = *opt;
  if (!o.tile) o.tile = 32;
  if (!o.block) o.block = 512;
  if (!o.unroll) o.unroll = 4;
  int rc = check_opts(&o, &log2_tile, ALLOW_CYCLE | ALLOW_PRECISION);
  if (rc) return rc;
  if (o.learned_order && o.tile < 16) return MB_EINVAL;  // the probe takes 8 x 8 samples per tile
  mb_server* S = new mb_server();
  S->budget = mem_budget_bytes;
  S->queue_limit = queue_limit ? queue_limit : 1024;
  S->tile = o.tile;
  S->block = o.block;
  S->unroll = o.unroll;
  cudaGetDevice(&S->device);
  if (o.precision != MB_PREC_FP64) {  // reduced-precision lanes take no escape filter
    S->fn_filt = S->fn_exact = render_fn_lowp(KIND_BATCH, S_FCFS, (int)o.precision, (int)S->unroll);
  } else {
    S->fn_filt = o.cycle_check ? render_fn_cycle(KIND_BATCH, S_FCFS, true, (int)S->unroll)
                               : render_fn(KIND_BATCH, S_FCFS, true, (int)S->unroll);
    S->fn_exact = o.cycle_check ? render_fn_cycle(KIND_BATCH, S_FCFS, false, (int)S->unroll)
                                : render_fn(KIND_BATCH, S_FCFS, false, (int)S->unroll);
  }
  S->grid = o.grid ? o.grid : default_grid(S->fn_filt, S->block);
  if (o.learned_order) {
    S->learned = true;
    S->model = o.model;
    S->fn_probe_filt = render_fn(KIND_PROBE, S_FCFS, true, (int)S->unroll);
    S->fn_probe_exact = render_fn(KIND_PROBE, S_FCFS, false, (int)S->unroll);
  }
  S->round_tiles = o.round_tiles ? o.round_tiles : 16 * S->grid;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof props);
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = S->device;
  uint64_t keep = ~0ull;
  bool ok = cudaMemPoolCreate(&S->pool, &props) == cudaSuccess &&
            cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess &&
            cudaMalloc((void**)&S->d_views, SERVE_SLOTS * sizeof(ViewDesc)) == cudaSuccess &&
            cudaMallocHost((void**)&S->h_view_stage, SERVE_SLOTS * sizeof(ViewDesc)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->setup, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc((void**)&S->d_probe_counter, 128 * SERVE_SETUP) == cudaSuccess;
  for (int j = 0; j < SERVE_SETUP && ok && o.learned_order; ++j)
    ok = cudaStreamCreateWithFlags(&S->lsetup[j], cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; k < SERVE_STREAMS && ok; ++k) {
    Round& Rd = S->rounds[k];
    ok = cudaStreamCreateWithFlags(&S->streams[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&Rd.ev, cudaEventDisableTiming) == cudaSuccess &&
         cudaMallocHost((void**)&Rd.h_items, (size_t)S->round_tiles * sizeof(BatchItem)) == cudaSuccess &&
         cudaMalloc((void**)&Rd.d_items, (size_t)S->round_tiles * sizeof(BatchItem)) == cudaSuccess &&
         cudaMalloc((void**)&Rd.d_counter, 256) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    mb_serve_destroy(S);
    return MB_ENOMEM;
  }
  for (uint32_t k = 0; k < SERVE_SLOTS; ++k) S->free_slots.push_back(SERVE_SLOTS - 1 - k);
  S->slot_ev.assign(SERVE_SLOTS, nullptr);
  S->worker = std::thread(worker_main, S);
  *out = S;
  return MB_OK;
}

extern "C" int mb_serve_submit(mb_server* S, const mb_request* rq, uint64_t* id) {
  if (!S || !rq || !id) return MB_EINVAL;
  int rc = check_view(&rq->w, rq->m, rq->n, rq->escape_r2, (const void*)1);
  if (rc) return rc;
  uint32_t tiles_x = (rq->n + S->tile - 1) / S->tile, tiles_y = (rq->m + S->tile - 1) / S->tile;
  if ((uint64_t)tiles_x * tiles_y >= 0xFFFFFFF0ull) return MB_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  if (S->failed != MB_OK) return S->failed;
  if (S->stop) return MB_EBUSY;
  size_t bytes = req_bytes(S, *rq);
  if (bytes > S->budget) {
    S->ctr.rejected++;
    return MB_ENOMEM;
  }
  if (S->queue.size() >= S->queue_limit) {
    S->ctr.rejected++;
    return MB_EBUSY;
  }
  if (!filter_ok(rq->escape_r2)) S->filt_all = false;
  Req R;
  R.id = S->next_id++;
  R.rq = *rq;
  R.bytes = bytes;
  R.tiles = tiles_x * tiles_y;
  R.tiles_x = tiles_x;
  R.submit_ns = now_ns();
  S->reqs[R.id] = R;
  S->queue.push_back(R.id);
  S->ctr.submitted++;
  *id = R.id;
  S->cv_work.notify_one();
  return MB_OK;
}

extern "C" int mb_serve_wait(mb_server* S, uint64_t id, uint32_t timeout_ms, mb_req_stats* st) {
  if (!S) return MB_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto pred = [&] {
    auto it = S->reqs.find(id);
    return it == S->reqs.end() || it->second.state == RQ_DONE || it->second.state == RQ_FAILED;
  };
  S->waiters++;
  bool ready = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
  if (--S->waiters == 0) S->cv_idle.notify_all();
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return MB_ENOTFOUND;
  if (!ready) return MB_ETIMEDOUT;
  const Req& R = it->second;
  if (st) {
    st->submit_ns = R.submit_ns;
    st->admit_ns = R.admit_ns;
    st->start_ns = R.start_ns;
    st->done_ns = R.done_ns;
    st->bytes = R.bytes;
    st->status = R.status;
  }
  return R.state == RQ_DONE ? MB_OK : R.status;
}

extern "C" int mb_serve_result(mb_server* S, uint64_t id, uint32_t** dev_out) {
  if (!S || !dev_out) return MB_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return MB_ENOTFOUND;
  if (it->second.state != RQ_DONE) return MB_EBUSY;
  *dev_out = (uint32_t*)it->second.dmem;
  return MB_OK;
}

extern "C" int mb_serve_read(mb_server* S, uint64_t id, uint32_t* dst, uint64_t count, void* stream) {
  if (!S || !dst) return MB_EINVAL;
  const uint32_t* src = nullptr;
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return MB_ENOTFOUND;
    if (it->second.state != RQ_DONE) return MB_EBUSY;
    if (count > (uint64_t)it->second.rq.m * it->second.rq.n) return MB_EINVAL;
    src = (const uint32_t*)it->second.dmem;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(dst, src, count * 4, cudaMemcpyDefault, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return MB_ECUDA;
  }
  return MB_OK;
}

extern "C" int mb_serve_release(mb_server* S, uint64_t id) {
  if (!S) return MB_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return MB_ENOTFOUND;
  Req& R = it->second;
  if (R.state == RQ_QUEUED || R.state == RQ_LIVE) return MB_EBUSY;
  if (R.dmem) {
    // Order the free after every round launched so far (a failed request may
    // still be read by a round in flight); no later round includes it.
    for (int k = 0; k < SERVE_STREAMS; ++k) cudaStreamWaitEvent(S->setup, S->rounds[k].ev, 0);
    if (S->slot_ev[R.slot]) cudaStreamWaitEvent(S->setup, S->slot_ev[R.slot], 0);  // its own set-up, too
    cudaFreeAsync(R.dmem, S->setup);
    S->in_use -= R.bytes;
    S->free_slots.push_back(R.slot);
  }
  S->reqs.erase(it);
  S->cv_work.notify_one();
  return MB_OK;
}

extern "C" int mb_serve_counters_get(mb_server* S, mb_serve_counters* c) {
  if (!S || !c) return MB_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  *c = S->ctr;
  c->bytes_in_use = S->in_use;
  c->peak_bytes = S->peak;
  c->queued = (uint32_t)S->queue.size();
  return MB_OK;
}

extern "C" int mb_serve_fail(mb_server* S, int code) {
  if (!S || code == MB_OK) return MB_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  fail_all_locked(S, code);
  return MB_OK;
}

extern "C" int mb_serve_destroy(mb_server* S) {
  if (!S) return MB_EINVAL;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
    // requests still waiting for memory are cancelled; admitted ones finish
    for (uint64_t id : S->queue) {
      Req& R = S->reqs[id];
      R.state = RQ_FAILED;
      R.status = MB_ECANCELED;
      R.done_ns = now_ns();
    }
    S->queue.clear();
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  {
    // every admitted request is now done: wake and drain the waiting threads
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.notify_all();
    S->cv_idle.wait(lk, [&] { return S->waiters == 0; });
  }
  for (int k = 0; k < SERVE_STREAMS; ++k)
    if (S->streams[k]) cudaStreamSynchronize(S->streams[k]);
  if (S->setup) cudaStreamSynchronize(S->setup);
  for (int j = 0; j < SERVE_SETUP; ++j)
    if (S->lsetup[j]) cudaStreamSynchronize(S->lsetup[j]);
  for (auto& kv : S->reqs)
    if (kv.second.dmem) cudaFree(kv.second.dmem);
  for (int k = 0; k < SERVE_STREAMS; ++k) {
    Round& Rd = S->rounds[k];
    if (Rd.ev) cudaEventDestroy(Rd.ev);
    if (Rd.h_items) cudaFreeHost(Rd.h_items);
    if (Rd.d_items) cudaFree(Rd.d_items);
    if (Rd.d_counter) cudaFree(Rd.d_counter);
    if (S->streams[k]) cudaStreamDestroy(S->streams[k]);
  }
  for (cudaEvent_t e : S->slot_ev)
    if (e) cudaEventDestroy(e);
  if (S->setup) cudaStreamDestroy(S->setup);
  for (int j = 0; j < SERVE_SETUP; ++j)
    if (S->lsetup[j]) cudaStreamDestroy(S->lsetup[j]);
  if (S->d_views) cudaFree(S->d_views);
  if (S->d_probe_counter) cudaFree(S->d_probe_counter);
  if (S->h_view_stage) cudaFreeHost(S->h_view_stage);
  if (S->pool) cudaMemPoolDestroy(S->pool);
  delete S;
  return MB_OK;
}
