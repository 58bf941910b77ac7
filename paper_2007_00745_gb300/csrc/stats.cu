// stats.cu -- mb_last_stats: makespan, per-SM activity and the iteration total
// of the calling thread's most recent render.
//
// mb_render and mb_render_learned give their main render launch a per-CTA trace
// buffer (the caller's opts->trace, else a small buffer this thread owns on the
// device) and note the launch here.  mb_last_stats waits for that launch's
// stream and reduces the records on the host; the iteration total is the sum of
// the counts in the output buffer, reduced on the device.
#include <algorithm>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "mb.h"
#include "mb_internal.h"
#include "render_kernels.cuh"

namespace mb {

__global__ void sum_counts_kernel(const uint32_t* __restrict__ c, uint64_t count, unsigned long long* total);

namespace {

struct OwnBuffer {
  mb_cta_trace* trace = nullptr;  // `cap` records, then one uint64 for the iteration total
  uint32_t cap = 0;
};

struct LastRun {
  bool valid = false;
  int device = 0;
  cudaStream_t stream = nullptr;
  const mb_cta_trace* trace = nullptr;
  uint32_t records = 0;
  const uint32_t* counts = nullptr;
  uint64_t npix = 0;
  unsigned long long* total = nullptr;  // device scratch of the owning thread
};

// Per host thread: one trace buffer per device (kept until the process exits)
// and the record of the last launch.
thread_local std::unordered_map<int, OwnBuffer> t_own;
thread_local LastRun t_last;

OwnBuffer* own_buffer(int dev, uint32_t need) {
  OwnBuffer& b = t_own[dev];
  if (b.cap >= need) return &b;
  uint32_t cap = std::max<uint32_t>(need, 1024u);
  void* p = nullptr;
  if (cudaMalloc(&p, (size_t)cap * sizeof(mb_cta_trace) + 8) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (b.trace) cudaFree(b.trace);  // cudaFree waits for work that may still use the old buffer
  b.trace = (mb_cta_trace*)p;
  b.cap = cap;
  return &b;
}

}  // namespace

void stats_begin(RenderParams& P, uint32_t grid, cudaStream_t st, const uint32_t* counts, uint64_t npix) {
  t_last.valid = false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  OwnBuffer* b = own_buffer(dev, P.trace ? 1u : grid);
  if (!b) return;  // no statistics for this launch; the render itself goes ahead
  if (!P.trace) {
    P.trace = b->trace;
    P.trace_len = b->cap;
  }
  // Every CTA below trace_len writes its record when it finishes, so the
  // records [0, min(grid, trace_len)) are all rewritten by the launch.
  t_last.valid = true;
  t_last.device = dev;
  t_last.stream = st;
  t_last.trace = P.trace;
  t_last.records = std::min(grid, P.trace_len);
  t_last.counts = counts;
  t_last.npix = npix;
  t_last.total = (unsigned long long*)(b->trace + b->cap);
}

void stats_cancel() { t_last.valid = false; }

}  // namespace mb

using namespace mb;

extern "C" int mb_last_stats(mb_run_stats* st) {
  if (!st) return MB_EINVAL;
  if (!t_last.valid) return MB_ENOTFOUND;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return MB_ECUDA;
  if (cur != t_last.device && cudaSetDevice(t_last.device) != cudaSuccess) return MB_ECUDA;
  int rc = MB_OK;
  std::vector<mb_cta_trace> rec(t_last.records);
  unsigned long long total = 0;
  if (cudaStreamSynchronize(t_last.stream) != cudaSuccess ||
      cudaMemcpy(rec.data(), t_last.trace, rec.size() * sizeof(mb_cta_trace), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(t_last.total, 0, 8) != cudaSuccess) {
    rc = MB_ECUDA;
  }
  if (rc == MB_OK) {
    uint32_t blocks = (uint32_t)std::min<uint64_t>((t_last.npix + 255) / 256, 4096);
    sum_counts_kernel<<<std::max(blocks, 1u), 256>>>(t_last.counts, t_last.npix, t_last.total);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&total, t_last.total, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = MB_ECUDA;
  }
  if (cur != t_last.device) cudaSetDevice(cur);
  if (rc != MB_OK) return rc;

  std::memset(st, 0, sizeof *st);
  st->iterations = total;
  uint64_t t0 = ~0ull, t1 = 0;
  for (const auto& r : rec) {
    if (r.end_ns == 0) continue;  // a CTA that wrote no record
    t0 = std::min(t0, r.start_ns);
    t1 = std::max(t1, r.end_ns);
    st->ctas += 1;
  }
  if (st->ctas == 0) return MB_OK;
  st->makespan_ns = t1 - t0;
  const double span = (double)std::max<uint64_t>(t1 - t0, 1);
  std::unordered_map<uint32_t, std::pair<uint64_t, uint64_t>> sm;  // smid -> (first start, last end)
  for (const auto& r : rec) {
    if (r.end_ns == 0) continue;
    auto it = sm.find(r.smid);
    if (it == sm.end()) {
      sm[r.smid] = {r.start_ns, r.end_ns};
    } else {
      it->second.first = std::min(it->second.first, r.start_ns);
      it->second.second = std::max(it->second.second, r.end_ns);
    }
  }
  int sms = sm_count();
  st->sms = (uint32_t)sm.size();
  double tail = 0.0, bmin = 1.0, bmax = 0.0, bsum = 0.0;
  for (const auto& kv : sm) {
    tail += (double)(t1 - kv.second.second);
    double busy = (double)(kv.second.second - kv.second.first) / span;
    bmin = std::min(bmin, busy);
    bmax = std::max(bmax, busy);
    bsum += busy;
  }
  uint32_t denom = std::max<uint32_t>((uint32_t)sms, st->sms);
  tail += (double)(denom - st->sms) * span;  // SMs that ran no CTA idle throughout
  st->idle_tail = tail / ((double)denom * span);
  st->sm_busy_min = denom > st->sms ? 0.0 : bmin;
  st->sm_busy_mean = bsum / (double)denom;
  st->sm_busy_max = bmax;
  return MB_OK;
}
