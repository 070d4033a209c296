// Strided tile copies between pinned host memory (device-accessible over the
// host link) and dense device buffers, for the out-of-core driver: the
// columns [c0, c0 + w) of a row-major host array are gathered into a
// [rows][w] device tile (the bytes of a row past the copied width, up to
// dwidth, set to zero), or a tile is scattered back.  A kernel does the copy
// (every SM issues loads and stores across the link), in 16-byte units when
// the addresses, the pitches and the widths allow it, else in 4- or 1-byte units.
#include "spod_internal.cuh"

namespace spod {
namespace {

template <typename U>
__global__ void k_copy2d(const char* __restrict__ src, int64_t spitch, char* __restrict__ dst, int64_t dpitch,
                         int64_t width, int64_t dwidth, int64_t rows) {
  const int64_t per_row = dwidth / (int64_t)sizeof(U), ncopy = width / (int64_t)sizeof(U);
  const int64_t n = per_row * rows;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / per_row, c = e - r * per_row;
    U v;
    if (c < ncopy) v = *reinterpret_cast<const U*>(src + r * spitch + c * (int64_t)sizeof(U));
    else memset(&v, 0, sizeof(U));
    *reinterpret_cast<U*>(dst + r * dpitch + c * (int64_t)sizeof(U)) = v;
  }
}

}  // namespace

cudaError_t launch_copy2d(void* dst, int64_t dpitch, const void* src, int64_t spitch, int64_t width, int64_t dwidth,
                          int64_t rows, int num_sms, cudaStream_t s) {
  if (dwidth < width) dwidth = width;
  if (dwidth <= 0 || rows <= 0) return cudaSuccess;
  const uint64_t a = reinterpret_cast<uint64_t>(dst) | reinterpret_cast<uint64_t>(src) | (uint64_t)dpitch |
                     (uint64_t)spitch | (uint64_t)width | (uint64_t)dwidth;
  const unsigned grid = (unsigned)(4 * (num_sms > 0 ? num_sms : 148));
  const char* sc = static_cast<const char*>(src);
  char* dc = static_cast<char*>(dst);
  if (a % 16 == 0) k_copy2d<uint4><<<grid, 512, 0, s>>>(sc, spitch, dc, dpitch, width, dwidth, rows);
  else if (a % 4 == 0) k_copy2d<uint32_t><<<grid, 512, 0, s>>>(sc, spitch, dc, dpitch, width, dwidth, rows);
  else k_copy2d<unsigned char><<<grid, 512, 0, s>>>(sc, spitch, dc, dpitch, width, dwidth, rows);
  return cudaGetLastError();
}

}  // namespace spod
