// gather.cu -- packing of rendered work items for the master gather (Sec. III-A/B).
//
// When one image is rendered across several GPUs, each worker renders the items
// it was dealt into its own image buffer; only those pixels travel to the
// master.  mb_pack_items copies the pixels of a list of items (rows row0 ..
// row0+rows-1 of tile `tile`, tile x tile pixels, tiles row-major over the
// image) into a dense buffer, one fixed slot of tile*tile counts per item, row
// by row; mb_unpack_items writes such a buffer back into an image.  Slot
// positions of rows past the item and of pixels outside the image are left
// unwritten by mb_pack_items and ignored by mb_unpack_items.  One CTA per item,
// threads along the tile's rows: plain coalesced copies, bound by HBM.
#include <cstdint>

#include "mb.h"
#include "mb_internal.h"

namespace mb {

__global__ void pack_items_kernel(const uint32_t* __restrict__ img, uint32_t m, uint32_t n, uint32_t log2_tile,
                                  const mb_item* __restrict__ items, uint32_t n_items, uint32_t* __restrict__ packed,
                                  int unpack, uint32_t* __restrict__ out, uint32_t* status) {
  const uint32_t tile = 1u << log2_tile, tiles_x = (n + tile - 1) >> log2_tile;
  for (uint32_t k = blockIdx.x; k < n_items; k += gridDim.x) {
    mb_item e = items[k];
    uint32_t ty = e.tile / tiles_x, tx = e.tile - ty * tiles_x;
    if ((uint32_t)e.row0 + e.rows > tile || (ty << log2_tile) >= m) {  // not an item of this image
      if (threadIdx.x == 0 && status) atomicOr(status, 2u);
      continue;
    }
    uint32_t r0 = (ty << log2_tile) + e.row0, c0 = tx << log2_tile;
    uint32_t cnt = (uint32_t)e.rows << log2_tile;
    uint64_t slot = (uint64_t)k << (2 * log2_tile);
    for (uint32_t p = threadIdx.x; p < cnt; p += blockDim.x) {
      uint32_t r = r0 + (p >> log2_tile), c = c0 + (p & (tile - 1));
      if (r >= m || c >= n) continue;
      uint64_t at = (uint64_t)r * n + c;
      uint64_t sp = slot + ((uint64_t)e.row0 << log2_tile) + p;
      if (unpack)
        out[at] = packed[sp];
      else
        packed[sp] = img[at];
    }
  }
}

static int pack_common(const uint32_t* img, uint32_t m, uint32_t n, uint32_t tile, const mb_item* items,
                       uint32_t n_items, uint32_t* packed, uint32_t* out, int unpack, uint32_t* status, void* stream) {
  if (!items || !packed || (unpack ? !out : !img)) return MB_EINVAL;
  if (m == 0 || n == 0 || m > MAX_SIDE || n > MAX_SIDE) return MB_EINVAL;
  if (tile < 8 || tile > 256 || (tile & (tile - 1))) return MB_EINVAL;
  if (n_items == 0) return MB_OK;
  uint32_t l = 0;
  while ((1u << l) < tile) ++l;
  uint32_t grid = n_items < 65535u ? n_items : 65535u;
  pack_items_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(img, m, n, l, items, n_items, packed, unpack, out,
                                                             status);
  return cudaGetLastError() == cudaSuccess ? MB_OK : MB_ECUDA;
}

}  // namespace mb

using namespace mb;

extern "C" int mb_pack_items(const uint32_t* img, uint32_t m, uint32_t n, uint32_t tile, const mb_item* items,
                             uint32_t n_items, uint32_t* packed, uint32_t* status, void* stream) {
  return pack_common(img, m, n, tile, items, n_items, packed, nullptr, 0, status, stream);
}

extern "C" int mb_unpack_items(const uint32_t* packed, uint32_t m, uint32_t n, uint32_t tile, const mb_item* items,
                               uint32_t n_items, uint32_t* img, uint32_t* status, void* stream) {
  return pack_common(nullptr, m, n, tile, items, n_items, const_cast<uint32_t*>(packed), img, 1, status, stream);
}
