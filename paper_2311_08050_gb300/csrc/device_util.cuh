// Small device helpers shared by the kernel files (header-only, internal linkage).
#pragma once
#include <cuda_runtime.h>

namespace inla {

// deterministic sum of one value per thread over a 256-thread block (fixed tree order)
static __device__ __forceinline__ double block_sum_256(double v) {
  __shared__ double sh[256];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// linear index x -> (i, j), j <= i, of the lower triangle in row order
static __device__ __forceinline__ void tri_decode(int x, int& i, int& j) {
  int t = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
  while (t * (t + 1) / 2 > x) --t;
  while ((t + 1) * (t + 2) / 2 <= x) ++t;
  i = t;
  j = x - t * (t + 1) / 2;
}

}  // namespace inla
