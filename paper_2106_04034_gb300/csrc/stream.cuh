// Pieces shared by the two implementations of a generation (the chained
// select/stream/final launches and the persistent cooperative kernel).
#pragma once

#include "common.cuh"
#include "reduce.cuh"

namespace gsgp {

constexpr int kGenThreads = 256;

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;"); }

// sigma(R) loads, widened to float (bf16 -> float is exact).
template <typename SigT>
struct SigLoad;

template <>
struct SigLoad<float> {
  static __device__ __forceinline__ float4 load(const float *base, int64_t off) {
    return __ldg(reinterpret_cast<const float4 *>(base + off));
  }
};

template <>
struct SigLoad<__nv_bfloat16> {
  static __device__ __forceinline__ float4 load(const __nv_bfloat16 *base, int64_t off) {
    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(base + off));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
  }
};

// Tournament selection and mutation draws of offspring slot i at generation
// g from its Philox stream (i, g): t candidates idx(w, m) (smallest training
// RMSE wins, the earliest drawn on ties; t = 0 keeps slot i), then the two
// random trees idx(w, r) and the step word.  fit(slot) returns the parent
// population's training RMSE and row(slot) the pool row holding the slot's
// semantics; both are issued for up to kBatch candidates at a time so that
// the tournament costs one memory round trip per kBatch candidates.
struct Draws {
  int parent, a, b, prow;
  float ms;
};

template <typename FitFn, typename RowFn>
__device__ __forceinline__ Draws draw_offspring(const GenParams &p, int i, int g, FitFn fit,
                                                RowFn row) {
  WordStream ws(p.key, (uint32_t)i, (uint32_t)g, p.run);
  Draws d;
  if (p.tsize == 0) {
    d.parent = i;
    d.prow = row(i);
  } else {
    unsigned long long best = 0;
    constexpr int kBatch = 4;
    for (int k0 = 0; k0 < p.tsize; k0 += kBatch) {
      int c[kBatch];
      unsigned long long f[kBatch];
      int r[kBatch];
      const int n = min(kBatch, p.tsize - k0);
#pragma unroll
      for (int k = 0; k < kBatch; ++k)
        if (k < n) c[k] = (int)draw_index(ws.next(), (uint32_t)p.m);
#pragma unroll
      for (int k = 0; k < kBatch; ++k)
        if (k < n) {
          f[k] = fit_key(fit(c[k]));
          r[k] = row(c[k]);
        }
#pragma unroll
      for (int k = 0; k < kBatch; ++k)
        if (k < n && (k0 + k == 0 || f[k] < best)) {   // strict: earliest drawn wins ties
          best = f[k];
          d.parent = c[k];
          d.prow = r[k];
        }
    }
  }
  d.a = (int)draw_index(ws.next(), (uint32_t)p.r);
  d.b = (int)draw_index(ws.next(), (uint32_t)p.r);
  const uint32_t wms = ws.next();
  d.ms = p.ms;
  if (p.ms_mode == 1) d.ms = __double2float_rn(__dmul_rn((double)p.ms, (double)draw_u24(wms)));
  return d;
}

// Mutation of 4 consecutive cases j0..j0+3 of one offspring (one fused
// multiply-add per case, s_O = s_T + ms (sR_a - sR_b)) and their squared
// errors, added to the training or test sum by case index.
template <typename SigT>
__device__ __forceinline__ void mutate4(const GenParams &p, const float *src, float *dst,
                                        const SigT *ra, const SigT *rb, int64_t j0, float step,
                                        float &str, float &ste) {
  const float4 s = __ldcg(reinterpret_cast<const float4 *>(src + j0));
  const float4 a4 = SigLoad<SigT>::load(ra, j0);
  const float4 b4 = SigLoad<SigT>::load(rb, j0);
  const float4 t4 = __ldg(reinterpret_cast<const float4 *>(p.target + j0));
  float4 o;
  o.x = fmaf(step, a4.x - b4.x, s.x);
  o.y = fmaf(step, a4.y - b4.y, s.y);
  o.z = fmaf(step, a4.z - b4.z, s.z);
  o.w = fmaf(step, a4.w - b4.w, s.w);
  *reinterpret_cast<float4 *>(dst + j0) = o;
  const float dd[4] = {o.x - t4.x, o.y - t4.y, o.z - t4.z, o.w - t4.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (j0 + q < p.n_train)
      str += dd[q] * dd[q];
    else if (j0 + q < p.n_cases)
      ste += dd[q] * dd[q];
  }
}

__device__ __forceinline__ void warp_sum2(float &a, float &b) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
}

// Canonical (train, test) squared-error sum of one 1024-case chunk.  The
// chunk is 8 sub-blocks of 128 cases, one per warp; lane l of sub-block k
// holds the float sum of its 4 cases (k * 128 + 4 l ... + 3, added in case
// order from 0).  A warp butterfly (xor 16, 8, 4, 2, 1) gives the sub-block
// total; every lane ends with the same value because each step adds the same
// two numbers on both partner lanes.  The 8 sub-block totals are then added
// in sub-block order (float, from 0) and the result is widened to double
// once.  Every kernel that computes squared errors (interpreter, chained and
// persistent generation kernels, allocation-free entry point) produces its
// chunk sums this way, so fitness values do not depend on which kernel or
// which work split computed them, and the float64 work per chunk is one
// conversion (float64 issue is scarce on this GPU).
__device__ __forceinline__ float2 subblock_sum(float lane_tr, float lane_te) {
  warp_sum2(lane_tr, lane_te);
  return make_float2(lane_tr, lane_te);
}

// Chunk sum from its 8 sub-block totals sub[0..7].
__device__ __forceinline__ double2 chunk_total(const float2 *sub) {
  float a = 0.f, b = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float2 v = sub[k];
    a += v.x;
    b += v.y;
  }
  return make_double2((double)a, (double)b);
}

}  // namespace gsgp
