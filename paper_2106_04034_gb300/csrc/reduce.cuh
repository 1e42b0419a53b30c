// Deterministic reductions used by the fitness and survival steps.
#pragma once

#include <math_constants.h>

#include "common.cuh"

namespace gsgp {

// RMSE from a sum of squared errors over n cases (Sec. 2.2, "Fitness
// computation"); a non-finite value becomes +inf, no cases give 0.
__device__ __forceinline__ double rmse_from_sse(double sse, int n) {
  if (n <= 0) return 0.0;
  const double v = sqrt(sse / (double)n);
  return isfinite(v) ? v : CUDART_INF;
}

// Sum of tiles [0, tiles) of one row of (train, test) partial sums by one
// warp, in a fixed order: lane k adds tiles k, k + 32, ... then a fixed
// butterfly; lane 0 holds the result.  Reads go to L2 (other CTAs wrote them).
__device__ __forceinline__ double2 warp_sum_partials(const double2 *row, int tiles, int lane) {
  double tr = 0.0, te = 0.0;
  for (int k = lane; k < tiles; k += 32) {
    const double2 v = __ldcg(row + k);
    tr += v.x;
    te += v.y;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    te += __shfl_xor_sync(0xffffffffu, te, o);
  }
  return make_double2(tr, te);
}

// (value, index) order used for arg-min / arg-max: the first index wins ties.
template <bool kMax>
__device__ __forceinline__ bool arg_better(double x, int i, double bx, int bi) {
  if (kMax) return x > bx || (x == bx && i < bi);
  return x < bx || (x == bx && i < bi);
}

// Block-wide arg-min (kMax = false) or arg-max of v[0, n) over blockDim.x
// threads (a power of two <= 1024).  s_v, s_i: blockDim.x scratch entries.
// Every thread returns the result.  Loads bypass L1.
template <bool kMax>
__device__ void block_arg(const double *v, int n, double *s_v, int *s_i, double &out_v,
                          int &out_i) {
  double bx = kMax ? -CUDART_INF : CUDART_INF;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = __ldcg(v + i);
    if (arg_better<kMax>(x, i, bx, bi)) {
      bx = x;
      bi = i;
    }
  }
  s_v[threadIdx.x] = bx;
  s_i[threadIdx.x] = bi;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      const double x = s_v[threadIdx.x + w];
      const int i = s_i[threadIdx.x + w];
      if (arg_better<kMax>(x, i, s_v[threadIdx.x], s_i[threadIdx.x])) {
        s_v[threadIdx.x] = x;
        s_i[threadIdx.x] = i;
      }
    }
    __syncthreads();
  }
  out_v = s_v[0];
  out_i = s_i[0];
  __syncthreads();
}

}  // namespace gsgp
