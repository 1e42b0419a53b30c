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

// The same sum for long rows (many 1024-case chunks): four loads are issued
// before their additions, which stay in the same order, so the result is
// identical and a row of 1221 chunks costs about a quarter of the L2 round
// trips.  Not inlined, so that the unrolled loop's registers do not count
// against the streaming code of the kernels that call it.
static __device__ __noinline__ double2 warp_sum_partials_long(const double2 *row, int tiles, int lane) {
  double tr = 0.0, te = 0.0;
#pragma unroll 4
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

// Fitness values are RMSEs: >= 0 or +inf, never NaN or -0.  For such
// doubles the IEEE bit pattern, read as an unsigned integer, orders exactly
// like the value, so arg-min / arg-max compare 64-bit integer keys instead of
// doubles (FP64 issue rate is a small fraction of the integer rate on this
// GPU, and these reductions sit on the per-generation critical path).
__device__ __forceinline__ unsigned long long fit_key(double x) {
  return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ double key_fit(unsigned long long k) {
  return __longlong_as_double((long long)k);
}

// (key, index) order used for arg-min / arg-max: the first index wins ties.
template <bool kMax>
__device__ __forceinline__ bool arg_better(unsigned long long x, int i, unsigned long long bx,
                                           int bi) {
  if (kMax) return x > bx || (x == bx && i < bi);
  return x < bx || (x == bx && i < bi);
}

constexpr unsigned long long kKeyAboveAll = 0x7FF0000000000001ull;   // above +inf
constexpr unsigned long long kKeyBelowAll = 0ull;                   // = +0.0 (ties by index)

// Block-wide arg-min (kMax = false) and arg-max (kMax = true) of keys, one
// (key, index) pair per thread in and the block's result out, first index
// on ties.  s_k, s_i: blockDim.x entries each (a power of two).
template <bool kMax>
__device__ void block_arg_keys(unsigned long long k, int i, unsigned long long *s_k, int *s_i,
                               unsigned long long &out_k, int &out_i) {
  s_k[threadIdx.x] = k;
  s_i[threadIdx.x] = i;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      const int o = threadIdx.x + w;
      if (arg_better<kMax>(s_k[o], s_i[o], s_k[threadIdx.x], s_i[threadIdx.x])) {
        s_k[threadIdx.x] = s_k[o];
        s_i[threadIdx.x] = s_i[o];
      }
    }
    __syncthreads();
  }
  out_k = s_k[0];
  out_i = s_i[0];
  __syncthreads();
}

// Block-wide arg-min or arg-max of fitness values v[0, n) (loads bypass L1).
template <bool kMax>
__device__ void block_arg(const double *v, int n, unsigned long long *s_k, int *s_i, double &out_v,
                          int &out_i) {
  unsigned long long bk = kMax ? kKeyBelowAll : kKeyAboveAll;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned long long k = fit_key(__ldcg(v + i));
    if (arg_better<kMax>(k, i, bk, bi)) {
      bk = k;
      bi = i;
    }
  }
  unsigned long long rk;
  block_arg_keys<kMax>(bk, bi, s_k, s_i, rk, out_i);
  out_v = key_fit(rk);
}

}  // namespace gsgp
