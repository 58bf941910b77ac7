// output.cu -- the paper's output stage: iteration -> pixel colour (Sec. I) on
// the GPU, and the image file the master node writes (a binary PPM, Sec. IV).
//
// Palette (the paper names none): points that never escape are black, other
// counts k map channel-wise through the triangle wave tri(x) = x < 256 ? x :
// 511 - x as r = tri(7k mod 512), g = tri(5k mod 512), b = tri(3k mod 512) --
// integer arithmetic, so every byte is reproducible.
#include <cstdint>
#include <cstdio>

#include "mb.h"
#include "mb_internal.h"

namespace mb {

__device__ __forceinline__ uint32_t tri(uint32_t x) { return x < 256u ? x : 511u - x; }

// One thread per 4 pixels: 12 output bytes as three 32-bit stores.
__global__ void colorize_kernel(const uint32_t* __restrict__ counts, uint64_t count, uint32_t iter_max,
                                uint8_t* __restrict__ rgb) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < count; t += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t k = counts[t];
    uint32_t r = 0, g = 0, b = 0;
    if (k != iter_max) {
      r = tri((uint32_t)(((uint64_t)k * 7u) & 511u));
      g = tri((uint32_t)(((uint64_t)k * 5u) & 511u));
      b = tri((uint32_t)(((uint64_t)k * 3u) & 511u));
    }
    rgb[3 * t] = (uint8_t)r;
    rgb[3 * t + 1] = (uint8_t)g;
    rgb[3 * t + 2] = (uint8_t)b;
  }
}

}  // namespace mb

using namespace mb;

extern "C" int mb_colorize(const uint32_t* counts, uint64_t count, uint32_t iter_max, uint8_t* rgb, void* stream) {
  if (!counts || !rgb) return MB_EINVAL;
  if (count == 0) return MB_OK;
  uint64_t blocks = (count + 255) / 256;
  uint64_t cap = (uint64_t)(sm_count() > 0 ? sm_count() : 1) * 16;
  if (blocks > cap) blocks = cap;
  colorize_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(counts, count, iter_max, rgb);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

extern "C" int mb_write_ppm(const char* path, const uint8_t* rgb, uint32_t m, uint32_t n) {
  if (!path || !rgb || m == 0 || n == 0) return MB_EINVAL;
  FILE* f = fopen(path, "wb");
  if (!f) return MB_EINVAL;
  bool ok = fprintf(f, "P6\n%u %u\n255\n", n, m) > 0;
  size_t bytes = (size_t)m * n * 3;
  ok = ok && fwrite(rgb, 1, bytes, f) == bytes;
  ok = (fclose(f) == 0) && ok;
  return ok ? MB_OK : MB_EINVAL;
}
