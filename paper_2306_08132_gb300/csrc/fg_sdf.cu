// Per-object preprocessing of the SDF grid at creation: a min-pyramid used to
// prove that a chunk of hand points cannot touch the object (forward-sweep
// culling in the fused kernel).
//
// Level k (k >= 1) has one entry per block of 2^k x 2^k x 2^k cells: the minimum
// of the grid nodes of those cells.  The trilinear interpolant inside a cell is
// a convex combination of the cell's corners, so it never drops below the
// minimum of any block that contains the cell.
#include <cuda_runtime.h>

#include "fg_internal.h"

namespace fg {

namespace {

__global__ void pyr_level1_kernel(const float* __restrict__ G, int nx, int ny, int nz, float* __restrict__ out,
                                  int bx, int by, int bz) {
  const size_t total = (size_t)bx * by * bz;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(t % bx), J = (int)((t / bx) % by), K = (int)(t / ((size_t)bx * by));
    float m = 3.0e38f;
    for (int z = 2 * K; z <= min(2 * K + 2, nz - 1); ++z)
      for (int y = 2 * J; y <= min(2 * J + 2, ny - 1); ++y)
        for (int x = 2 * I; x <= min(2 * I + 2, nx - 1); ++x) m = fminf(m, G[((size_t)z * ny + y) * nx + x]);
    out[t] = m;
  }
}

__global__ void pyr_level_kernel(const float* __restrict__ in, int ix, int iy, int iz, float* __restrict__ out,
                                 int bx, int by, int bz) {
  const size_t total = (size_t)bx * by * bz;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(t % bx), J = (int)((t / bx) % by), K = (int)(t / ((size_t)bx * by));
    float m = 3.0e38f;
    for (int z = 2 * K; z <= min(2 * K + 1, iz - 1); ++z)
      for (int y = 2 * J; y <= min(2 * J + 1, iy - 1); ++y)
        for (int x = 2 * I; x <= min(2 * I + 1, ix - 1); ++x) m = fminf(m, in[((size_t)z * iy + y) * ix + x]);
    out[t] = m;
  }
}

inline int blocks_at(int n, int k) { return ((n - 1) + (1 << k) - 1) >> k; }

}  // namespace

size_t min_pyramid_floats(int nx, int ny, int nz, int* levels) {
  size_t total = 0;
  int k = 1;
  for (; k <= kMaxPyrLevels; ++k) {
    total += (size_t)blocks_at(nx, k) * blocks_at(ny, k) * blocks_at(nz, k);
    if (blocks_at(nx, k) == 1 && blocks_at(ny, k) == 1 && blocks_at(nz, k) == 1) break;
  }
  *levels = k > kMaxPyrLevels ? kMaxPyrLevels : k;
  return total;
}

cudaError_t build_min_pyramid(const float* grid, int nx, int ny, int nz, float* pyr, int levels, int* offsets) {
  size_t off = 0;
  const float* prev = nullptr;
  int px = 0, py = 0, pz = 0;
  for (int k = 1; k <= levels; ++k) {
    const int bx = blocks_at(nx, k), by = blocks_at(ny, k), bz = blocks_at(nz, k);
    offsets[k - 1] = (int)off;
    const size_t total = (size_t)bx * by * bz;
    size_t blocks = (total + 255) / 256;
    const size_t cap = (size_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    if (k == 1)
      pyr_level1_kernel<<<(int)blocks, 256>>>(grid, nx, ny, nz, pyr + off, bx, by, bz);
    else
      pyr_level_kernel<<<(int)blocks, 256>>>(prev, px, py, pz, pyr + off, bx, by, bz);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prev = pyr + off;
    px = bx;
    py = by;
    pz = bz;
    off += total;
  }
  return cudaDeviceSynchronize();
}

}  // namespace fg
