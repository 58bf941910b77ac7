// api.cu -- small entry points: version, error names, count reduction, device
// info and the FP64 issue-rate microbenchmark that defines "% of FP64 peak".
#include <cstdint>
#include <cstring>

#include "mb.h"
#include "mb_internal.h"
#include "escape_core.cuh"
#include "render_kernels.cuh"

namespace mb {

// Block-wide sum of uint32 counts into one uint64 (grid-stride, one atomic per block).
__global__ void sum_counts_kernel(const uint32_t* __restrict__ c, uint64_t count, unsigned long long* total) {
  unsigned long long acc = 0;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (uint64_t)gridDim.x * blockDim.x)
    acc += c[k];
  for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(FULL_MASK, acc, o);
  __shared__ unsigned long long part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0ull;
    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(FULL_MASK, acc, o);
    if (threadIdx.x == 0) atomicAdd(total, acc);
  }
}

// Independent dependency chains of one binary64 operation, written in PTX so
// that the compiler can neither fuse nor drop them.
constexpr int PEAK_CHAINS = 8;

template <int OP>
__global__ void fp64_peak_kernel(double* sink, double y, double z, int iters) {
  double x[PEAK_CHAINS];
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) {
      if (OP == 0) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(x[c]) : "d"(y));
      if (OP == 1) asm volatile("mul.rn.f64 %0, %0, %1;" : "+d"(x[c]) : "d"(y));
      if (OP == 2) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[c]) : "d"(y), "d"(z));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
  if (s == 12345.678) sink[blockIdx.x] = s;  // keeps the chains alive
}

__global__ void selftest_products_kernel(const double* __restrict__ a, const double* __restrict__ b, uint64_t n,
                                         double* __restrict__ sq, double* __restrict__ pr, uint8_t* __restrict__ ok) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    sq[i] = emul_sqr(a[i]);
    pr[i] = emul_mul(a[i], b[i], 1);
    ok[i] = (uint8_t)(emul_ok(a[i]) && emul_ok(b[i]));
  }
}

__global__ void selftest_psub_kernel(const double* __restrict__ a, const double* __restrict__ b, uint64_t n,
                                     double* __restrict__ d, uint8_t* __restrict__ ok) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    bool odd = false;
    d[i] = emul_psub(a[i], b[i], odd);
    ok[i] = (uint8_t)!odd;
  }
}

// Bounded-wait self-test of the CTA work-claiming protocol: the CTA's work word
// says its item (a 64-pixel raster tile) is already claimed past its end, and
// no worker will ever publish the next item -- the producer is gone.  Every warp
// then runs the real claim() wait, which must give up after its bounded spin,
// OR 1 into *status and report no work; got[warp] receives what claim()
// returned (0 expected).  Nothing is read or written outside status and got.
__global__ void selftest_wait_kernel(RenderParams P, uint32_t* got) {
  __shared__ unsigned long long s_word;
  __shared__ uint32_t s_taken;
  if (threadIdx.x == 0) {
    s_word = 65ull;  // item 0, next pixel 65 of 64
    s_taken = 1u;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    uint32_t item = 0, off = 0;
    ItemWords iw{0u, 0u, 0u};
    uint32_t n = claim<KIND_RASTER, S_FCFS>(P, &s_word, &s_taken, 32u, P.n_items, item, off, iw);
    got[blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)] = n;
  }
}

}  // namespace mb

using namespace mb;

extern "C" int mb_selftest_wait(uint32_t ctas, uint32_t* status, uint32_t* got, void* stream) {
  if (!status || !got || ctas == 0 || ctas > 1024) return MB_EINVAL;
  RenderParams P;
  memset(&P, 0, sizeof P);
  P.log2_tile = 3;  // raster items of 8 x 8 = 64 pixels; no view is read
  P.n_items = 1;
  P.status = status;
  selftest_wait_kernel<<<ctas, 128, 0, (cudaStream_t)stream>>>(P, got);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

extern "C" int mb_selftest_products(const double* a, const double* b, uint64_t n, double* sq, double* pr,
                                    uint8_t* ok, void* stream) {
  if (!a || !b || !sq || !pr || !ok) return MB_EINVAL;
  if (n == 0) return MB_OK;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  selftest_products_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(a, b, n, sq, pr, ok);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

extern "C" int mb_selftest_psub(const double* a, const double* b, uint64_t n, double* d, uint8_t* ok, void* stream) {
  if (!a || !b || !d || !ok) return MB_EINVAL;
  if (n == 0) return MB_OK;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  selftest_psub_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(a, b, n, d, ok);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

extern "C" const char* mb_version(void) { return "mb 0.1.0 (sm_103a)"; }

extern "C" const char* mb_strerror(int code) {
  switch (code) {
    case MB_OK: return "ok";
    case MB_EINVAL: return "invalid argument";
    case MB_ENOMEM: return "out of memory or over budget";
    case MB_ECUDA: return "CUDA runtime error";
    case MB_ETIMEDOUT: return "timed out";
    case MB_EBUSY: return "busy";
    case MB_ENOTFOUND: return "not found";
    case MB_EDEVICE: return "device-side error";
    case MB_ECANCELED: return "cancelled";
    default: return "unknown error";
  }
}

extern "C" int mb_sum_counts(const uint32_t* counts, uint64_t count, uint64_t* total, void* stream) {
  if (!counts || !total) return MB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(total, 0, sizeof(uint64_t), st) != cudaSuccess) return MB_ECUDA;
  if (count == 0) return MB_OK;
  uint64_t blocks = (count + 255) / 256;
  uint64_t cap = (uint64_t)(sm_count() > 0 ? sm_count() : 1) * 8;
  if (blocks > cap) blocks = cap;
  sum_counts_kernel<<<(unsigned)blocks, 256, 0, st>>>(counts, count, (unsigned long long*)total);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

extern "C" int mb_device_info(uint32_t block, uint32_t* sms, uint32_t* ctas_per_sm) {
  if (!sms || !ctas_per_sm) return MB_EINVAL;
  if (block == 0) block = DEFAULT_BLOCK;
  if (block < 32 || block > 512 || block % 32) return MB_EINVAL;
  int s = sm_count();
  if (s <= 0) return MB_ECUDA;
  *sms = (uint32_t)s;
  *ctas_per_sm = (uint32_t)resident_ctas((const void*)render_fn(KIND_RASTER, S_FCFS, true, DEFAULT_UNROLL), (int)block);
  return MB_OK;
}

extern "C" int mb_fp64_peak(int op, double* ops_per_s, double* seconds) {
  if (!ops_per_s || op < 0 || op > 2) return MB_EINVAL;
  int sms = sm_count();
  if (sms <= 0) return MB_ECUDA;
  const int block = 256, per_sm = 4, iters = 4096;
  const int grid = sms * per_sm;
  double* sink = nullptr;
  if (cudaMalloc(&sink, grid * sizeof(double)) != cudaSuccess) return MB_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  void (*fn)(double*, double, double, int) =
      op == 0 ? fp64_peak_kernel<0> : (op == 1 ? fp64_peak_kernel<1> : fp64_peak_kernel<2>);
  fn<<<grid, block>>>(sink, 1.0000001, 0.5, 64);  // warm-up
  cudaEventRecord(e0);
  fn<<<grid, block>>>(sink, 1.0000001, 0.5, iters);
  cudaEventRecord(e1);
  int rc = cudaEventSynchronize(e1) == cudaSuccess ? MB_OK : MB_ECUDA;
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (rc) return rc;
  double ops = (double)grid * block * PEAK_CHAINS * (double)iters;
  *ops_per_s = ops / (ms * 1e-3);
  if (seconds) *seconds = ms * 1e-3;
  return MB_OK;
}
