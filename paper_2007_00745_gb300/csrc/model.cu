// model.cu -- learned tile-cost model around the first-come-first-served queue.
//
// The paper's FCFS scheme (Sec. III-B) hands out rows in index order; here the
// work items are tiles and a small MLP predicts each tile's cost from a
// low-resolution probe, so that the queue runs longest-first and heavy tiles
// are split into row strips.  Scheduling only: the counts are the same as any
// other order (Bernstein's conditions, Sec. II-A).
//
// Features (70 per tile), network (70-64-64-1, ReLU, FP32), target
// log2(1 + tile total)/32, Adam, and the integer order-and-split rule are
// specified in include/mb.h next to the entry points.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mb.h"
#include "mb_internal.h"
#include "render_kernels.cuh"

namespace mb {

constexpr int NF = 70, HID = 64;
constexpr int OFF_W1 = 0, OFF_B1 = HID * NF, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID, P_COUNT = OFF_B3 + 1;
static_assert(P_COUNT == MB_MLP_PARAMS, "parameter count");

// ---- features ---------------------------------------------------------------

__global__ void features_kernel(const uint32_t* __restrict__ probe, uint32_t ntiles, uint32_t tiles_x,
                                uint32_t tiles_y, uint32_t iter_max, double xmin, double xmax, uint32_t n,
                                uint32_t tile, float* __restrict__ feat) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const double log_i = log2(1.0 + (double)iter_max);
  const float inv = (float)(1.0 / log_i);
  const uint32_t* p = probe + (size_t)t * 64;
  float* f = feat + (size_t)t * NF;
  unsigned long long sum = 0;
  uint32_t full = 0;
  for (int k = 0; k < 64; ++k) {
    uint32_t c = p[k];
    f[k] = __fmul_rn(log2f(1.0f + (float)c), inv);
    sum += c;
    full += c == iter_max ? 1u : 0u;
  }
  uint32_t tx = t % tiles_x, ty = t / tiles_x;
  f[64] = (float)((tx + 0.5) / tiles_x);
  f[65] = (float)((ty + 0.5) / tiles_y);
  f[66] = (float)(log_i / 17.0);
  f[67] = (float)(-log10((xmax - xmin) / (double)n) / 16.0);
  f[68] = (float)(log2(1.0 + (double)tile * tile / 64.0 * (double)sum) / 32.0);
  f[69] = (float)full / 64.0f;
}

// training label of a tile: log2(1 + total) / 32
__global__ void tile_targets_kernel(const unsigned long long* __restrict__ totals, uint32_t ntiles, float* __restrict__ y) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ntiles) y[t] = (float)(log2(1.0 + (double)totals[t]) / 32.0);
}

// ablation without the network: a tile's cost predicted from its probe alone,
// y = log2(1 + 64 * sum of the 64 probe counts) / 32 (the probe's estimate of the tile total)
__global__ void probe_sum_cost_kernel(const uint32_t* __restrict__ probe, uint32_t ntiles, uint32_t tile,
                                      float* __restrict__ y) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  unsigned long long s = 0;
  for (int k = 0; k < 64; ++k) s += probe[(size_t)t * 64 + k];
  double scale = (double)tile * tile / 64.0;
  y[t] = (float)(log2(1.0 + scale * (double)s) / 32.0);
}

// Neighbourhood guard of predicted costs: g[t] = the largest y over the 3 x 3
// tiles around t within its view (NaN ignored; NaN only if all nine are NaN).
// Views are consecutive runs of tiles: view v has tiles goff[v] .. goff[v+1]-1,
// tx[v] per row; goff == NULL means one view of width tx1.  Interior regions of the set are connected, so a tile whose
// probe missed them almost always borders tiles whose probe did not: with the
// guard such tiles cannot end up at the cheap end of the longest-first queue.
__global__ void guard_kernel(const float* __restrict__ y, uint32_t nt, const uint32_t* __restrict__ goff,
                             const uint32_t* __restrict__ tx, uint32_t nviews, uint32_t tx1, float* __restrict__ g) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    uint32_t base = 0, w = tx1, h = nt / tx1;
    if (goff) {
      uint32_t lo = 0, hi = nviews;  // largest v with goff[v] <= t
      while (hi - lo > 1) {
        uint32_t mid = (lo + hi) / 2;
        if (goff[mid] <= t) lo = mid;
        else hi = mid;
      }
      base = goff[lo];
      w = tx[lo];
      h = (goff[lo + 1] - base) / w;
    }
    const uint32_t r = (t - base) / w, c = (t - base) - r * w;
    float best = y[t];
    for (uint32_t rr = r ? r - 1 : 0; rr <= r + 1 && rr < h; ++rr)
      for (uint32_t cc = c ? c - 1 : 0; cc <= c + 1 && cc < w; ++cc) best = fmaxf(best, y[base + rr * w + cc]);
    g[t] = best;
  }
}

// ---- MLP forward --------------------------------------------------------------

constexpr int FWD_S = 16;  // samples per pass of a forward block (64 threads, one per hidden unit)

__global__ void __launch_bounds__(64) mlp_forward_kernel(const float* __restrict__ prm, const float* __restrict__ X,
                                                         const uint32_t* __restrict__ idx, uint32_t N,
                                                         float* __restrict__ y, float* __restrict__ h1o,
                                                         float* __restrict__ h2o) {
  __shared__ float W1T[NF][HID];
  __shared__ float W2T[HID][HID];
  __shared__ float xs[FWD_S][NF];
  __shared__ float h1s[FWD_S][HID];
  __shared__ float red[2][FWD_S];
  const int j = threadIdx.x;
  for (int e = j; e < HID * NF; e += HID) W1T[e % NF][e / NF] = prm[OFF_W1 + e];
  for (int e = j; e < HID * HID; e += HID) W2T[e % HID][e / HID] = prm[OFF_W2 + e];
  const float b1 = prm[OFF_B1 + j], b2 = prm[OFF_B2 + j], w3 = prm[OFF_W3 + j], b3 = prm[OFF_B3];
  __syncthreads();
  for (uint32_t base = blockIdx.x * FWD_S; base < N; base += gridDim.x * FWD_S) {
    for (int e = j; e < FWD_S * NF; e += HID) {
      int s = e / NF, k = e % NF;
      uint32_t r = base + s;
      xs[s][k] = r < N ? X[(size_t)(idx ? idx[r] : r) * NF + k] : 0.0f;
    }
    __syncthreads();
    for (int s = 0; s < FWD_S; ++s) {
      float a = b1;
      for (int k = 0; k < NF; ++k) a = fmaf(W1T[k][j], xs[s][k], a);
      a = fmaxf(a, 0.0f);
      h1s[s][j] = a;
      if (h1o && base + s < N) h1o[(size_t)(base + s) * HID + j] = a;
    }
    __syncthreads();
    for (int s = 0; s < FWD_S; ++s) {
      float a = b2;
      for (int k = 0; k < HID; ++k) a = fmaf(W2T[k][j], h1s[s][k], a);
      a = fmaxf(a, 0.0f);
      if (h2o && base + s < N) h2o[(size_t)(base + s) * HID + j] = a;
      float part = w3 * a;
      for (int o = 16; o; o >>= 1) part += __shfl_down_sync(FULL_MASK, part, o);
      if ((j & 31) == 0) red[j >> 5][s] = part;
    }
    __syncthreads();
    if (j < FWD_S && base + j < N) y[base + j] = xs[j][68] + b3 + red[0][j] + red[1][j];
    __syncthreads();
  }
}

// ---- MLP backward (one block per minibatch; deterministic) ----------------------

constexpr int BWD_T = 256, BWD_S = 16;
constexpr int W1_PER_T = (HID * NF + BWD_T - 1) / BWD_T;  // 18
constexpr int W2_PER_T = HID * HID / BWD_T;               // 16

__global__ void __launch_bounds__(BWD_T) mlp_backward_kernel(const float* __restrict__ prm, const float* __restrict__ X,
                                                             const uint32_t* __restrict__ idx, uint32_t B,
                                                             const float* __restrict__ h1g, const float* __restrict__ h2g,
                                                             const float* __restrict__ yp, const float* __restrict__ tgt,
                                                             float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float W2[HID][HID];
  __shared__ float W3[HID];
  __shared__ float xs[BWD_S][NF];
  __shared__ float h1s[BWD_S][HID];
  __shared__ float h2s[BWD_S][HID];
  __shared__ float g1s[BWD_S][HID];
  __shared__ float g2s[BWD_S][HID];
  __shared__ float gs[BWD_S];
  __shared__ float lred[BWD_T / 32];
  const int t = threadIdx.x;
  for (int e = t; e < HID * HID; e += BWD_T) W2[e / HID][e % HID] = prm[OFF_W2 + e];
  if (t < HID) W3[t] = prm[OFF_W3 + t];
  float a1[W1_PER_T], a2[W2_PER_T], asmall = 0.0f, lacc = 0.0f;
#pragma unroll
  for (int r = 0; r < W1_PER_T; ++r) a1[r] = 0.0f;
#pragma unroll
  for (int r = 0; r < W2_PER_T; ++r) a2[r] = 0.0f;
  const float scale = 2.0f / (float)B;
  __syncthreads();
  for (uint32_t base = 0; base < B; base += BWD_S) {
    for (int e = t; e < BWD_S * NF; e += BWD_T) {
      int s = e / NF, k = e % NF;
      uint32_t r = base + s;
      xs[s][k] = r < B ? X[(size_t)(idx ? idx[r] : r) * NF + k] : 0.0f;
    }
    for (int e = t; e < BWD_S * HID; e += BWD_T) {
      int s = e / HID, k = e % HID;
      uint32_t r = base + s;
      h1s[s][k] = r < B ? h1g[(size_t)r * HID + k] : 0.0f;
      h2s[s][k] = r < B ? h2g[(size_t)r * HID + k] : 0.0f;
    }
    if (t < BWD_S) {
      uint32_t r = base + t;
      float d = r < B ? yp[r] - tgt[idx ? idx[r] : r] : 0.0f;
      gs[t] = scale * d;
      lacc += d * d;
    }
    __syncthreads();
    for (int e = t; e < BWD_S * HID; e += BWD_T) {
      int s = e / HID, j = e % HID;
      g2s[s][j] = h2s[s][j] > 0.0f ? gs[s] * W3[j] : 0.0f;
    }
    __syncthreads();
    for (int e = t; e < BWD_S * HID; e += BWD_T) {
      int s = e / HID, k = e % HID;
      float a = 0.0f;
      for (int j = 0; j < HID; ++j) a = fmaf(g2s[s][j], W2[j][k], a);
      g1s[s][k] = h1s[s][k] > 0.0f ? a : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < W1_PER_T; ++r) {
      int e = t + BWD_T * r;
      if (e < HID * NF) {
        int k = e / NF, i = e % NF;
        float a = a1[r];
        for (int s = 0; s < BWD_S; ++s) a = fmaf(g1s[s][k], xs[s][i], a);
        a1[r] = a;
      }
    }
#pragma unroll
    for (int r = 0; r < W2_PER_T; ++r) {
      int e = t + BWD_T * r;
      int j = e / HID, k = e % HID;
      float a = a2[r];
      for (int s = 0; s < BWD_S; ++s) a = fmaf(g2s[s][j], h1s[s][k], a);
      a2[r] = a;
    }
    if (t < HID) {
      for (int s = 0; s < BWD_S; ++s) asmall += g1s[s][t];
    } else if (t < 2 * HID) {
      for (int s = 0; s < BWD_S; ++s) asmall += g2s[s][t - HID];
    } else if (t < 3 * HID) {
      for (int s = 0; s < BWD_S; ++s) asmall = fmaf(gs[s], h2s[s][t - 2 * HID], asmall);
    } else if (t == 3 * HID) {
      for (int s = 0; s < BWD_S; ++s) asmall += gs[s];
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < W1_PER_T; ++r) {
    int e = t + BWD_T * r;
    if (e < HID * NF) grad[OFF_W1 + e] = a1[r];
  }
#pragma unroll
  for (int r = 0; r < W2_PER_T; ++r) grad[OFF_W2 + t + BWD_T * r] = a2[r];
  if (t < HID) grad[OFF_B1 + t] = asmall;
  else if (t < 2 * HID) grad[OFF_B2 + t - HID] = asmall;
  else if (t < 3 * HID) grad[OFF_W3 + t - 2 * HID] = asmall;
  else if (t == 3 * HID) grad[OFF_B3] = asmall;
  if (loss) {
    for (int o = 16; o; o >>= 1) lacc += __shfl_down_sync(FULL_MASK, lacc, o);
    if ((t & 31) == 0) lred[t >> 5] = lacc;
    __syncthreads();
    if (t == 0) {
      float s = 0.0f;
      for (int w = 0; w < BWD_T / 32; ++w) s += lred[w];
      *loss = s / (float)B;
    }
  }
}

// ---- Adam ---------------------------------------------------------------------

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, uint32_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.0f - b1) * gi;
  float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// mean of `count` floats into *out (one block)
__global__ void mean_kernel(const float* __restrict__ x, uint32_t count, float* __restrict__ out) {
  __shared__ float red[32];
  float a = 0.0f;
  for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) a += x[i];
  for (int o = 16; o; o >>= 1) a += __shfl_down_sync(FULL_MASK, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (unsigned w = 0; w < (blockDim.x + 31) / 32; ++w) s += red[w];
    *out = s / (float)count;
  }
}

// ---- order and split (one block, stable, integer arithmetic) --------------------

constexpr int OS_T = 1024, OS_WARPS = OS_T / 32, Q_LEVELS = 192;

__device__ __forceinline__ uint32_t cost_level(float y) {
  if (!(y > 0.0f)) return 0;
  float prod = fminf(__fmul_rn(y, 128.0f), 4096.0f);
  uint32_t q = (uint32_t)prod;  // truncation
  return q < (uint32_t)(Q_LEVELS - 1) ? q : (uint32_t)(Q_LEVELS - 1);
}

__device__ __forceinline__ unsigned long long level_cost(uint32_t q) {
  const unsigned long long M[4] = {65536ull, 77936ull, 92682ull, 110218ull};
  return ((1ull << (q >> 2)) * M[q & 3]) >> 16;
}

__device__ __forceinline__ unsigned long long sat_add(unsigned long long a, unsigned long long b) {
  unsigned long long s = a + b;
  return s < a ? ~0ull : s;
}

__global__ void __launch_bounds__(OS_T) order_split_kernel(const float* __restrict__ y, uint32_t ntiles, uint32_t tile,
                                                           uint32_t grid, uint32_t split, uint32_t smin,
                                                           uint8_t* __restrict__ qbuf,
                                                           uint32_t* __restrict__ order, mb_item* __restrict__ items,
                                                           uint32_t capacity, uint32_t* __restrict__ n_items,
                                                           uint32_t* __restrict__ status) {
  __shared__ uint32_t hist[Q_LEVELS];
  __shared__ uint32_t start[Q_LEVELS];
  __shared__ uint32_t wcnt[OS_WARPS][Q_LEVELS];
  __shared__ unsigned long long csum[OS_WARPS];
  __shared__ uint32_t part[OS_T];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int k = t; k < Q_LEVELS; k += OS_T) hist[k] = 0;
  __syncthreads();
  // levels, histogram, saturating cost sum
  unsigned long long cs = 0;
  for (uint32_t i = t; i < ntiles; i += OS_T) {
    uint32_t q = cost_level(y[i]);
    qbuf[i] = (uint8_t)q;
    atomicAdd(&hist[q], 1u);
    cs = sat_add(cs, level_cost(q));
  }
  for (int o = 16; o; o >>= 1) cs = sat_add(cs, __shfl_down_sync(FULL_MASK, cs, o));
  if (lane == 0) csum[w] = cs;
  __syncthreads();
  if (t == 0) {  // bucket starts, q descending
    uint32_t acc = 0;
    for (int q = Q_LEVELS - 1; q >= 0; --q) {
      start[q] = acc;
      acc += hist[q];
    }
    unsigned long long s = 0;
    for (int k = 0; k < OS_WARPS; ++k) s = sat_add(s, csum[k]);
    csum[0] = s;
  }
  __syncthreads();
  // stable scatter in chunks of OS_T elements
  for (uint32_t base = 0; base < ntiles; base += OS_T) {
    for (int k = t; k < OS_WARPS * Q_LEVELS; k += OS_T) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    uint32_t i = base + t;
    bool valid = i < ntiles;
    uint32_t q = valid ? qbuf[i] : Q_LEVELS;  // Q_LEVELS never matches a real level
    unsigned peers = __match_any_sync(FULL_MASK, q);
    uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[w][q] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pos = start[q] + rank;
      for (int k = 0; k < w; ++k) pos += wcnt[k][q];
      order[pos] = i;
    }
    __syncthreads();
    for (int k = t; k < Q_LEVELS; k += OS_T) {
      uint32_t add = 0;
      for (int ww = 0; ww < OS_WARPS; ++ww) add += wcnt[ww][k];
      start[k] += add;
    }
    __syncthreads();
  }
  // strips per tile in sorted order, exclusive scan, items
  unsigned long long target = csum[0] / ((unsigned long long)split * grid);
  if (target < 1) target = 1;
  uint32_t smax = tile / 4 < 16 ? tile / 4 : 16;
  uint32_t per = (ntiles + OS_T - 1) / OS_T;
  uint32_t lo = t * per, hi = min(lo + per, ntiles);
  uint32_t mine = 0;
  for (uint32_t r = lo; r < hi; ++r) {
    unsigned long long c = level_cost(qbuf[order[r]]);
    unsigned long long need = (c + target - 1) / target;
    uint32_t s = smin;
    while (s < need && s < smax) s *= 2;
    mine += s;
  }
  part[t] = mine;
  __syncthreads();
  if (t == 0) {
    uint32_t acc = 0;
    for (int k = 0; k < OS_T; ++k) {
      uint32_t v = part[k];
      part[k] = acc;
      acc += v;
    }
    *n_items = acc <= capacity ? acc : 0;
    if (acc > capacity && status) atomicOr(status, 2u);
  }
  __syncthreads();
  uint32_t pos = part[t];
  uint32_t total = *(volatile uint32_t*)n_items;
  for (uint32_t r = lo; r < hi; ++r) {
    uint32_t tt = order[r];
    unsigned long long c = level_cost(qbuf[tt]);
    unsigned long long need = (c + target - 1) / target;
    uint32_t s = smin;
    while (s < need && s < smax) s *= 2;
    uint32_t rows = tile / s;
    for (uint32_t k = 0; k < s; ++k, ++pos) {
      if (pos < total) {
        mb_item it;
        it.tile = tt;
        it.row0 = (uint16_t)(k * rows);
        it.rows = (uint16_t)rows;
        items[pos] = it;
      }
    }
  }
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace mb

using namespace mb;

extern "C" int mb_tile_features(const uint32_t* probe, const mb_window* w, uint32_t m, uint32_t n, uint32_t iter_max,
                                uint32_t tile, float* feat, void* stream) {
  if (!probe || !w || !feat || m == 0 || n == 0 || tile < 16 || tile > 256 || (tile & (tile - 1))) return MB_EINVAL;
  uint32_t tx = (n + tile - 1) / tile, ty = (m + tile - 1) / tile, nt = tx * ty;
  features_kernel<<<(nt + 127) / 128, 128, 0, (cudaStream_t)stream>>>(probe, nt, tx, ty, iter_max, w->xmin, w->xmax, n,
                                                                       tile, feat);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

extern "C" int mb_tile_targets(const uint64_t* totals, uint32_t ntiles, float* y, void* stream) {
  if (!totals || !y) return MB_EINVAL;
  if (ntiles == 0) return MB_OK;
  tile_targets_kernel<<<(ntiles + 255) / 256, 256, 0, (cudaStream_t)stream>>>((const unsigned long long*)totals,
                                                                               ntiles, y);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

extern "C" int mb_mlp_forward(const float* params, const float* x, uint32_t count, float* y, void* stream) {
  if (!params || !x || !y) return MB_EINVAL;
  if (count == 0) return MB_OK;
  uint32_t blocks = (count + FWD_S - 1) / FWD_S;
  uint32_t cap = (uint32_t)(sm_count() > 0 ? sm_count() : 1) * 16;
  if (blocks > cap) blocks = cap;
  mlp_forward_kernel<<<blocks, HID, 0, (cudaStream_t)stream>>>(params, x, nullptr, count, y, nullptr, nullptr);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

namespace mb {
// Forward with saved activations, then backward, for one minibatch (rows idx[0..B) of x).
static int grad_launch(const float* params, const float* x, const uint32_t* idx, uint32_t B, const float* target,
                       float* grad, float* loss, float* h1, float* h2, float* yp, cudaStream_t st) {
  uint32_t blocks = (B + FWD_S - 1) / FWD_S;
  mlp_forward_kernel<<<blocks, HID, 0, st>>>(params, x, idx, B, yp, h1, h2);
  mlp_backward_kernel<<<1, BWD_T, 0, st>>>(params, x, idx, B, h1, h2, yp, target, grad, loss);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}
}  // namespace mb

extern "C" int mb_mlp_grad(const float* params, const float* x, const uint32_t* idx, uint32_t batch,
                           const float* target, float* grad, float* loss, void* stream) {
  if (!params || !x || !target || !grad || batch == 0) return MB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  size_t bytes = a256((size_t)batch * HID * 4) * 2 + a256((size_t)batch * 4);
  char* ws = nullptr;
  if (cudaMallocAsync((void**)&ws, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return MB_ENOMEM;
  }
  float* h1 = (float*)ws;
  float* h2 = (float*)(ws + a256((size_t)batch * HID * 4));
  float* yp = (float*)(ws + 2 * a256((size_t)batch * HID * 4));
  int rc = grad_launch(params, x, idx, batch, target, grad, loss, h1, h2, yp, st);
  cudaFreeAsync(ws, st);
  return rc;
}

extern "C" int mb_adam_step(float* params, const float* grad, float* m, float* v, uint32_t count, uint32_t t,
                            float lr, float beta1, float beta2, float eps, void* stream) {
  if (!params || !grad || !m || !v || t == 0) return MB_EINVAL;
  float c1 = (float)(1.0 / (1.0 - pow((double)beta1, (double)t)));
  float c2 = (float)(1.0 / (1.0 - pow((double)beta2, (double)t)));
  adam_kernel<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, count, lr, beta1, beta2,
                                                                       eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

extern "C" int mb_model_train(float* params, float* adam_m, float* adam_v, const float* x, const float* target,
                              uint32_t count, const uint32_t* order, uint32_t epochs, uint32_t batch, float lr,
                              float* epoch_loss, void* stream) {
  if (!params || !adam_m || !adam_v || !x || !target || !order || count == 0 || batch == 0 || batch > count)
    return MB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t steps = count / batch;
  size_t bytes = a256((size_t)batch * HID * 4) * 2 + a256((size_t)batch * 4) + a256((size_t)P_COUNT * 4) +
                 a256((size_t)steps * 4);
  char* ws = nullptr;
  if (cudaMallocAsync((void**)&ws, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return MB_ENOMEM;
  }
  float* h1 = (float*)ws;
  float* h2 = (float*)(ws + a256((size_t)batch * HID * 4));
  float* yp = (float*)(ws + 2 * a256((size_t)batch * HID * 4));
  float* grad = (float*)(ws + 2 * a256((size_t)batch * HID * 4) + a256((size_t)batch * 4));
  float* losses = (float*)((char*)grad + a256((size_t)P_COUNT * 4));
  int rc = MB_OK;
  uint32_t t = 0;
  for (uint32_t e = 0; e < epochs && rc == MB_OK; ++e) {
    for (uint32_t s = 0; s < steps && rc == MB_OK; ++s) {
      const uint32_t* idx = order + (size_t)e * count + (size_t)s * batch;
      rc = grad_launch(params, x, idx, batch, target, grad, losses + s, h1, h2, yp, st);
      if (rc == MB_OK) rc = mb_adam_step(params, grad, adam_m, adam_v, P_COUNT, ++t, lr, 0.9f, 0.999f, 1e-8f, st);
    }
    if (rc == MB_OK && epoch_loss) {
      mean_kernel<<<1, 256, 0, st>>>(losses, steps, epoch_loss + e);
      if (cudaGetLastError() != cudaSuccess) rc = MB_ECUDA;
    }
  }
  cudaFreeAsync(ws, st);
  return rc;
}

extern "C" int mb_order_split(const float* cost_pred, uint32_t ntiles, uint32_t tile, uint32_t grid, uint32_t split,
                              mb_item* items, uint32_t capacity, uint32_t* n_items, uint32_t* status, void* stream) {
  if (!cost_pred || !items || !n_items || ntiles == 0 || grid == 0 || tile < 8 || tile > 256 ||
      (tile & (tile - 1)) || split > 4096)
    return MB_EINVAL;
  if (split == 0) split = 4;
  cudaStream_t st = (cudaStream_t)stream;
  size_t bytes = a256(ntiles) + a256((size_t)ntiles * 4);
  char* ws = nullptr;
  if (cudaMallocAsync((void**)&ws, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return MB_ENOMEM;
  }
  order_split_kernel<<<1, OS_T, 0, st>>>(cost_pred, ntiles, tile, grid, split, 1u, (uint8_t*)ws,
                                         (uint32_t*)(ws + a256(ntiles)),
                                         items, capacity, n_items, status);
  int rc = cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
  cudaFreeAsync(ws, st);
  return rc;
}

extern "C" int mb_guard_costs(const float* cost_pred, uint32_t tiles_x, uint32_t tiles_y, float* guarded,
                              void* stream) {
  if (!cost_pred || !guarded || tiles_x == 0 || tiles_y == 0 || (uint64_t)tiles_x * tiles_y >= 0xFFFFFFFFull)
    return MB_EINVAL;
  const uint32_t nt = tiles_x * tiles_y;
  guard_kernel<<<min((nt + 255) / 256, 4096u), 256, 0, (cudaStream_t)stream>>>(cost_pred, nt, nullptr, nullptr, 1u,
                                                                             tiles_x, guarded);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

extern "C" int mb_model_save(const float* params, const char* path) {
  if (!params || !path) return MB_EINVAL;
  std::vector<float> h(P_COUNT);
  if (cudaMemcpy(h.data(), params, P_COUNT * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return MB_ECUDA;
  FILE* f = fopen(path, "wb");
  if (!f) return MB_EINVAL;
  const char magic[8] = {'M', 'B', 'M', 'L', 'P', '7', '0', '1'};
  uint32_t cnt = P_COUNT;
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&cnt, 4, 1, f) == 1 && fwrite(h.data(), 4, P_COUNT, f) == P_COUNT;
  ok = (fclose(f) == 0) && ok;
  return ok ? MB_OK : MB_EINVAL;
}

extern "C" int mb_model_load(const char* path, float* params) {
  if (!params || !path) return MB_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return MB_ENOTFOUND;
  char magic[8];
  uint32_t cnt = 0;
  std::vector<float> h(P_COUNT);
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "MBMLP701", 8) == 0 && fread(&cnt, 4, 1, f) == 1 &&
            cnt == (uint32_t)P_COUNT && fread(h.data(), 4, P_COUNT, f) == P_COUNT;
  fclose(f);
  if (!ok) return MB_EINVAL;
  return cudaMemcpy(params, h.data(), P_COUNT * 4, cudaMemcpyHostToDevice) == cudaSuccess ? MB_OK : MB_ECUDA;
}

// ---- probe and the learned render pipeline ----------------------------------------

namespace mb {

size_t order_tiles_ws_bytes(uint32_t nt) { return 2 * a256((size_t)nt * 4) + a256(nt) + a256((size_t)nt * 4); }

int order_tiles(const uint32_t* probe, const float* feat, uint32_t nt, const float* params, uint32_t tile,
                uint32_t grid, uint32_t split, uint32_t min_strips, const uint32_t* goff, const uint32_t* tx,
                uint32_t nviews, mb_item* items, uint32_t capacity, uint32_t* n_items, uint32_t* status,
                cudaStream_t st, void* ws_given) {
  if (!probe || !items || !n_items || nt == 0 || grid == 0 || (params && !feat) || !goff || !tx || nviews == 0)
    return MB_EINVAL;
  if (split == 0) split = 4;
  if (split > 4096) split = 4096;
  char* ws = (char*)ws_given;
  if (!ws && cudaMallocAsync((void**)&ws, order_tiles_ws_bytes(nt), st) != cudaSuccess) {
    cudaGetLastError();
    return MB_ENOMEM;
  }
  float* y = (float*)ws;
  float* yg = (float*)(ws + a256((size_t)nt * 4));
  uint8_t* qbuf = (uint8_t*)(ws + 2 * a256((size_t)nt * 4));
  uint32_t* order = (uint32_t*)(ws + 2 * a256((size_t)nt * 4) + a256(nt));
  int rc = MB_OK;
  if (params) {
    rc = mb_mlp_forward(params, feat, nt, y, st);
  } else {
    probe_sum_cost_kernel<<<(nt + 255) / 256, 256, 0, st>>>(probe, nt, tile, y);
    rc = cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
  }
  if (rc == MB_OK) {
    guard_kernel<<<min((nt + 255) / 256, 4096u), 256, 0, st>>>(y, nt, goff, tx, nviews, 0u, yg);
    order_split_kernel<<<1, OS_T, 0, st>>>(yg, nt, tile, grid, split, min_strips, qbuf, order, items, capacity,
                                           n_items, status);
    rc = cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
  }
  if (!ws_given) cudaFreeAsync(ws, st);
  return rc;
}

struct LearnedLayout {
  size_t view, counter, cx, cy, probe, feat, y, yg, items, nitems, qbuf, order, total;
};

static LearnedLayout learned_layout(uint32_t m, uint32_t n, uint32_t nt, uint32_t cap) {
  LearnedLayout L;
  L.view = 0;
  L.counter = a256(sizeof(ViewDesc));
  L.cx = L.counter + 256;
  L.cy = L.cx + a256((size_t)n * 8);
  L.probe = L.cy + a256((size_t)m * 8);
  L.feat = L.probe + a256((size_t)nt * 64 * 4);
  L.y = L.feat + a256((size_t)nt * NF * 4);
  L.yg = L.y + a256((size_t)nt * 4);
  L.items = L.yg + a256((size_t)nt * 4);
  L.nitems = L.items + a256((size_t)cap * sizeof(mb_item));
  L.qbuf = L.nitems + 256;
  L.order = L.qbuf + a256(nt);
  L.total = L.order + a256((size_t)nt * 4);
  return L;
}

static void fill_view(ViewDesc& V, const mb_window* w, uint32_t m, uint32_t n, uint32_t iter_max, double r2,
                      uint32_t* out, uint64_t* totals, char* ws, size_t cx, size_t cy, uint32_t tile) {
  std::memset(&V, 0, sizeof V);
  V.cx = (const double*)(ws + cx);
  V.cy = (const double*)(ws + cy);
  V.out = out;
  V.totals = totals;
  V.xmin = w->xmin;
  V.xmax = w->xmax;
  V.ymin = w->ymin;
  V.ymax = w->ymax;
  V.r2 = r2;
  V.thr = make_thr(r2);
  V.m = m;
  V.n = n;
  V.iter_max = iter_max;
  V.tiles_x = (n + tile - 1) / tile;
  V.tiles_y = (m + tile - 1) / tile;
}

}  // namespace mb

extern "C" int mb_probe(const mb_window* w, uint32_t m, uint32_t n, uint32_t iter_max, double escape_r2,
                        uint32_t* probe_out, uint32_t* image_out, const mb_opts* opt) {
  int rc = check_view(w, m, n, escape_r2, probe_out);
  if (rc) return rc;
  rc = check_device_access(probe_out);
  if (rc == MB_OK && image_out) rc = check_device_access(image_out);
  if (rc) return rc;
  uint32_t log2_tile = 0;
  rc = check_opts(opt, &log2_tile);
  if (rc) return rc;
  const uint32_t tile = 1u << log2_tile;
  if (tile < 16) return MB_EINVAL;
  const uint32_t block = opt && opt->block ? opt->block : DEFAULT_BLOCK;
  cudaStream_t st = opt ? (cudaStream_t)opt->stream : nullptr;
  LearnedLayout lay = learned_layout(m, n, 0, 0);
  char* ws = nullptr;
  if (cudaMallocAsync((void**)&ws, lay.probe, st) != cudaSuccess) {
    cudaGetLastError();
    return MB_ENOMEM;
  }
  ViewDesc V;
  fill_view(V, w, m, n, iter_max, escape_r2, image_out, nullptr, ws, lay.cx, lay.cy, tile);
  RenderParams P;
  std::memset(&P, 0, sizeof P);
  P.views = (const ViewDesc*)(ws + lay.view);
  P.log2_tile = log2_tile;
  P.counter = (uint32_t*)(ws + lay.counter);
  P.status = opt ? opt->status : nullptr;
  P.probe_out = probe_out;
  P.n_items = V.tiles_x * V.tiles_y;
  P.deadline_ns = opt_deadline_ns(opt);
  RenderFn fn = render_fn(KIND_PROBE, S_FCFS, filter_ok(escape_r2), opt_unroll(opt));
  uint32_t grid = opt && opt->grid ? opt->grid : default_grid(fn, block);
  uint32_t map_blocks = min((m + n + 255) / 256, 1024u);
  pixel_map_single_kernel<<<map_blocks, 256, 0, st>>>(V, (ViewDesc*)(ws + lay.view), P.counter);
  rc = cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
  if (rc == MB_OK) rc = launch_render(fn, P, grid, block, st);
  cudaFreeAsync(ws, st);
  return rc;
}

extern "C" int mb_render_learned(const mb_window* w, uint32_t m, uint32_t n, uint32_t iter_max, double escape_r2,
                                 uint32_t* out, const float* params, const mb_opts* opt) {
  int rc = check_view(w, m, n, escape_r2, out);
  if (rc) return rc;
  rc = check_device_access(out);
  if (rc) return rc;
  uint32_t log2_tile = 0;
  rc = check_opts(opt, &log2_tile);
  if (rc) return rc;
  const uint32_t tile = 1u << log2_tile;
  if (tile < 16 || !min_strips_ok(opt, tile)) return MB_EINVAL;
  const uint32_t block = opt && opt->block ? opt->block : DEFAULT_BLOCK;
  cudaStream_t st = opt ? (cudaStream_t)opt->stream : nullptr;
  const uint32_t tx = (n + tile - 1) / tile, ty = (m + tile - 1) / tile;
  if ((uint64_t)tx * ty * 16 >= 0xFFFFFFFFull) return MB_EINVAL;
  const uint32_t nt = tx * ty, cap = nt * 16;
  LearnedLayout lay = learned_layout(m, n, nt, cap);
  char* ws = nullptr;
  if (cudaMallocAsync((void**)&ws, lay.total, st) != cudaSuccess) {
    cudaGetLastError();
    return MB_ENOMEM;
  }
  ViewDesc V;
  fill_view(V, w, m, n, iter_max, escape_r2, out, opt ? opt->tile_totals : nullptr, ws, lay.cx, lay.cy, tile);
  const bool filt = filter_ok(escape_r2);
  RenderFn fprobe = render_fn(KIND_PROBE, S_FCFS, filt, opt_unroll(opt));
  RenderFn frender = render_fn(KIND_LIST, S_FCFS, filt, opt_unroll(opt));
  uint32_t grid = opt && opt->grid ? opt->grid : default_grid(frender, block);

  RenderParams P;
  std::memset(&P, 0, sizeof P);
  P.views = (const ViewDesc*)(ws + lay.view);
  P.log2_tile = log2_tile;
  P.counter = (uint32_t*)(ws + lay.counter);
  P.status = opt ? opt->status : nullptr;
  P.deadline_ns = opt_deadline_ns(opt);
  // 1. pixel map + probe (writes its samples into the image too)
  uint32_t map_blocks = min((m + n + 255) / 256, 1024u);
  pixel_map_single_kernel<<<map_blocks, 256, 0, st>>>(V, (ViewDesc*)(ws + lay.view), P.counter);
  RenderParams PP = P;
  PP.probe_out = (uint32_t*)(ws + lay.probe);
  PP.n_items = nt;
  rc = cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
  if (rc == MB_OK) rc = launch_render(fprobe, PP, default_grid(fprobe, block), block, st);
  // 2. features, 3. predicted cost, 4. longest-first items with splits
  if (params) {
    if (rc == MB_OK) rc = mb_tile_features(PP.probe_out, w, m, n, iter_max, tile, (float*)(ws + lay.feat), st);
    if (rc == MB_OK) rc = mb_mlp_forward(params, (const float*)(ws + lay.feat), nt, (float*)(ws + lay.y), st);
  } else if (rc == MB_OK) {
    probe_sum_cost_kernel<<<(nt + 255) / 256, 256, 0, st>>>(PP.probe_out, nt, tile, (float*)(ws + lay.y));
    rc = cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
  }
  if (rc == MB_OK) {
    uint32_t split = opt && opt->split ? opt->split : 4u;
    if (split > 4096) split = 4096;
    guard_kernel<<<min((nt + 255) / 256, 4096u), 256, 0, st>>>((const float*)(ws + lay.y), nt, nullptr, nullptr, 1u, tx,
                                                               (float*)(ws + lay.yg));
    order_split_kernel<<<1, OS_T, 0, st>>>((const float*)(ws + lay.yg), nt, tile, grid, split, opt_min_strips(opt, tile),
                                           (uint8_t*)(ws + lay.qbuf),
                                           (uint32_t*)(ws + lay.order), (mb_item*)(ws + lay.items), cap,
                                           (uint32_t*)(ws + lay.nitems), P.status);
    rc = cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
  }
  // 5. render the remaining pixels from the ordered queue; the counter is reset first
  if (rc == MB_OK) rc = cudaMemsetAsync(P.counter, 0, 4, st) == cudaSuccess ? MB_OK : MB_ECUDA;
  if (rc == MB_OK) {
    RenderParams PR = P;
    PR.items = (const mb_item*)(ws + lay.items);
    PR.n_items_dev = (const uint32_t*)(ws + lay.nitems);
    PR.skip_probe = 1;
    PR.trace = opt ? opt->trace : nullptr;
    PR.trace_len = opt && opt->trace ? opt->trace_len : 0;
    stats_begin(PR, grid, st, out, (uint64_t)m * n);
    rc = launch_render_timed(frender, PR, grid, block, st, opt);
    if (rc != MB_OK) stats_cancel();
  }
  cudaFreeAsync(ws, st);
  return rc;
}
