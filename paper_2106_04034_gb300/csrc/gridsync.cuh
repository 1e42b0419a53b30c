// Grid-wide barrier of the persistent cooperative kernels: bounded waits
// and a sticky error word (GridSync in kernels.cuh).
#pragma once

#include "kernels.cuh"

namespace gsgp {

constexpr unsigned kSpinLimit = kSpinLimitDefault;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait until *p >= target; false (and the sticky error word set)
// when `limit` naps have passed or another CTA already gave up.
__device__ __forceinline__ bool wait_at_least(const unsigned *p, unsigned target, GridSync *gs,
                                              unsigned limit = kSpinLimit) {
  unsigned spins = 0;
  while (ld_acquire_u32(p) < target) {
    if (ld_relaxed_s32(&gs->err) != 0) return false;
    if (++spins > limit) {
      atomicExch(&gs->err, 1);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

// Grid-wide barrier: every CTA adds one arrival to the counter and waits for
// epoch * grid arrivals (the counter is zeroed before each launch).  A
// two-level variant (groups of CTAs, one global arrival per group) measured
// slower here: each extra dependent round trip costs more than the
// contention it removes.  Returns false when the grid must stop.
__device__ __forceinline__ bool grid_sync(GridSync *gs, unsigned &epoch, int *s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    __threadfence();
    atomicAdd(&gs->count, 1u);
    const bool ok = wait_at_least(&gs->count, epoch * gridDim.x, gs);
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// grid_sync of the persistent kernels with the launch's wait bound (read by
// thread 0 only, from the kernel's parameter block).
__device__ __forceinline__ bool grid_sync_args(const PersistArgs &x, unsigned &epoch, int *s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    __threadfence();
    atomicAdd(&x.gs->count, 1u);
    const bool ok = wait_at_least(&x.gs->count, epoch * gridDim.x, x.gs,
                                  x.spin_limit ? x.spin_limit : kSpinLimit);
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

}  // namespace gsgp
