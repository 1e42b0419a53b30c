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
  bool cross;          // geometric semantic crossover instead of mutation
  int parent2, prow2;  // its second parent (slot, row)
};

// The draws as the stream reads them: (parent row, offspring row, rt1, rt2)
// for a mutation, (parent row, offspring row, mask tree, -1 - second parent
// row) for a crossover; and as the trace records them: (parent, rt1, rt2,
// ms bits) for a mutation, (parent, mask tree, -2 - second parent, 0) for a
// crossover.
__device__ __forceinline__ int4 sel_entry(const Draws &d, int orow) {
  return make_int4(d.prow, orow, d.a, d.cross ? -1 - d.prow2 : d.b);
}
__device__ __forceinline__ int4 trace_entry(const Draws &d) {
  return d.cross ? make_int4(d.parent, d.a, -2 - d.parent2, 0)
                 : make_int4(d.parent, d.a, d.b, __float_as_int(d.ms));
}

// Tournament of t candidates drawn from the stream: the smallest training
// RMSE wins, the earliest drawn on ties; t = 0 keeps slot i.  Candidates'
// fitness and rows are fetched kBatch at a time, one memory round trip each.
template <typename FitFn, typename RowFn>
__device__ __forceinline__ void tournament(const GenParams &p, int i, WordStream &ws, FitFn fit,
                                           RowFn row, int &winner, int &winner_row) {
  if (p.tsize == 0) {
    winner = i;
    winner_row = row(i);
    return;
  }
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
        winner = c[k];
        winner_row = r[k];
      }
  }
}

// CROSS = false compiles the mutation-only draws (p_crossover must be 0).
template <bool CROSS, typename FitFn, typename RowFn>
__device__ __forceinline__ Draws draw_offspring(const GenParams &p, int i, int g, FitFn fit,
                                                RowFn row) {
  WordStream ws(p.key, (uint32_t)i, (uint32_t)g, p.run);
  Draws d;
  tournament(p, i, ws, fit, row, d.parent, d.prow);
  d.a = (int)draw_index(ws.next(), (uint32_t)p.r);
  d.b = (int)draw_index(ws.next(), (uint32_t)p.r);
  const uint32_t wms = ws.next();
  d.ms = p.ms;
  if (p.ms_mode == 1) d.ms = __double2float_rn(__dmul_rn((double)p.ms, (double)draw_u24(wms)));
  // geometric semantic crossover (only when enabled, so that mutation-only
  // runs draw exactly the words above): word t+3 decides, words t+4 .. 2t+3
  // are the second parent's tournament; the mask is random tree a
  d.cross = false;
  d.parent2 = d.parent;
  d.prow2 = d.prow;
  if (CROSS && p.p_crossover > 0.0f) {
    d.cross = draw_u24(ws.next()) < p.p_crossover;
    if (d.cross) tournament(p, i, ws, fit, row, d.parent2, d.prow2);
  }
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

// Geometric semantic crossover of 4 consecutive cases: with R = sigma of the
// mask tree, offspring = R T1 + (1 - R) T2, computed as T2 + R (T1 - T2)
// (one subtraction and one fused multiply-add per case), and the squared
// errors as in mutate4.
template <typename SigT>
__device__ __forceinline__ void crossover4(const GenParams &p, const float *src1,
                                           const float *src2, float *dst, const SigT *rm,
                                           int64_t j0, float &str, float &ste) {
  const float4 s1 = __ldcg(reinterpret_cast<const float4 *>(src1 + j0));
  const float4 s2 = __ldcg(reinterpret_cast<const float4 *>(src2 + j0));
  const float4 r4 = SigLoad<SigT>::load(rm, j0);
  const float4 t4 = __ldg(reinterpret_cast<const float4 *>(p.target + j0));
  float4 o;
  o.x = fmaf(r4.x, s1.x - s2.x, s2.x);
  o.y = fmaf(r4.y, s1.y - s2.y, s2.y);
  o.z = fmaf(r4.z, s1.z - s2.z, s2.z);
  o.w = fmaf(r4.w, s1.w - s2.w, s2.w);
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

// Selection of offspring slot i at generation g from the population of
// parity par whose tables are complete in memory (Algorithm 1, "Selection"
// and the draws of "GSM"): writes the draws used by the stream (parent row,
// offspring row, rt1, rt2, step) and the trace entry (parent slot, rt1, rt2,
// step bits).
template <bool CROSS>
__device__ __forceinline__ void select_offspring(const GenParams &p, int i, int g, int par) {
  const int m = p.m;
  const double *F = p.fit + (size_t)par * m;
  const int *perm = p.perm + (size_t)par * 2 * m;
  const int orow = __ldcg(perm + m + i);
  const Draws d = draw_offspring<CROSS>(
      p, i, g, [&](int slot) { return __ldcg(F + slot); },
      [&](int slot) { return __ldcg(perm + slot); });
  p.sel[i] = sel_entry(d, orow);
  p.sel_ms[i] = d.ms;
  p.trace[(size_t)g * m + i] = trace_entry(d);
}

// Sub-block totals of one stream item: [offspring][chunk][sub-block].
template <int VEC, int OPB>
using ItemSums = float2[OPB][VEC][kGenThreads / 32];

// Mutation stream of one item: offspring i0 .. i0 + cnt - 1 (cnt <= OPB) of
// run p over the cases [tile * 1024 VEC, (tile + 1) * 1024 VEC), all 256
// threads of the CTA taking part.  sel / ms are the draws of offspring i0;
// those of the next offspring are loaded while the current one streams.
// Warp w leaves the total of sub-block w of chunk v of offspring k in
// sum[k][v][w]; after a barrier item_partials finishes the chunk sums.
// CROSS = false compiles the mutation stream alone.
template <typename SigT, int VEC, int OPB, bool CROSS>
__device__ __forceinline__ void stream_item(const GenParams &p, int tile, int i0, int cnt,
                                            int4 sel, float ms, ItemSums<VEC, OPB> &sum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SigT *sig = static_cast<const SigT *>(p.sigma_r);
  const int64_t base = (int64_t)tile * (1024 * VEC);
  for (int k = 0; k < cnt; ++k) {
    const float *src = p.pool + (int64_t)sel.x * p.n_pad;
    float *dst = p.pool + (int64_t)sel.y * p.n_pad;
    const SigT *ra = sig + (int64_t)sel.z * p.n_pad;
    const int w = sel.w;                  // rt2, or -1 - second parent row
    const bool cross = CROSS && w < 0;
    const SigT *rb = sig + (int64_t)(cross ? 0 : w) * p.n_pad;
    const float step = ms;
    if (k + 1 < cnt) {
      sel = __ldcg(p.sel + i0 + k + 1);
      ms = __ldcg(p.sel_ms + i0 + k + 1);
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      // chunk v: sub-block = warp, 4 consecutive cases per lane
      const int64_t j0 = base + v * 1024 + tid * 4;
      float str = 0.f, ste = 0.f;
      if (j0 < p.n_pad) {
        if (cross)   // uniform across the CTA: one offspring at a time
          crossover4<SigT>(p, src, p.pool + (int64_t)(-1 - w) * p.n_pad, dst, ra, j0, str, ste);
        else
          mutate4<SigT>(p, src, dst, ra, rb, j0, step, str, ste);
      }
      const float2 t = subblock_sum(str, ste);
      if (lane == 0) sum[k][v][warp] = t;
    }
  }
}

// Stream of one item with 1024-case tiles (VEC = 1), software pipelined:
// the next offspring's three row loads are issued before the current
// offspring's arithmetic, store and reduction, and the targets are read
// once per item.  The item's draws come from shared memory (sels / mss,
// filled one item ahead), so no offspring waits for its draws.  A mutation
// loads its parent and two random-tree rows, a crossover (CROSS, entry
// w = -1 - second parent row) its two parents and the mask tree; the
// arithmetic and the sub-block sums are mutate4's / crossover4's and
// stream_item's.
template <typename SigT, int OPB, bool CROSS>
__device__ __forceinline__ void stream_item_pipe(const GenParams &p, int tile, int cnt,
                                                 const int4 *sels, const float *mss,
                                                 ItemSums<1, OPB> &sum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SigT *sig = static_cast<const SigT *>(p.sigma_r);
  const int64_t j0 = (int64_t)tile * 1024 + tid * 4;
  const bool in = j0 < p.n_pad;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  // x: parent row; y: random tree a (mutation) or mask tree (crossover);
  // z: random tree b (mutation) or second parent row (crossover)
  auto load = [&](const int4 e, float4 &x, float4 &y, float4 &z) {
    x = __ldcg(reinterpret_cast<const float4 *>(p.pool + (int64_t)e.x * p.n_pad + j0));
    y = SigLoad<SigT>::load(sig + (int64_t)e.z * p.n_pad, j0);
    if (CROSS && e.w < 0)
      z = __ldcg(reinterpret_cast<const float4 *>(p.pool + (int64_t)(-1 - e.w) * p.n_pad + j0));
    else
      z = SigLoad<SigT>::load(sig + (int64_t)e.w * p.n_pad, j0);
  };
  float4 t4 = zero, x = zero, y = zero, z = zero;
  if (in) {
    t4 = __ldg(reinterpret_cast<const float4 *>(p.target + j0));
    load(sels[0], x, y, z);
  }
  for (int k = 0; k < cnt; ++k) {
    const int4 e = sels[k];
    const float step = mss[k];
    float4 x2 = x, y2 = y, z2 = z;   // the next offspring's operands
    if (in && k + 1 < cnt) load(sels[k + 1], x2, y2, z2);
    float str = 0.f, ste = 0.f;
    if (in) {
      float4 o;
      if (CROSS && e.w < 0) {   // R T1 + (1 - R) T2 as T2 + R (T1 - T2)
        o.x = fmaf(y.x, x.x - z.x, z.x);
        o.y = fmaf(y.y, x.y - z.y, z.y);
        o.z = fmaf(y.z, x.z - z.z, z.z);
        o.w = fmaf(y.w, x.w - z.w, z.w);
      } else {
        o.x = fmaf(step, y.x - z.x, x.x);
        o.y = fmaf(step, y.y - z.y, x.y);
        o.z = fmaf(step, y.z - z.z, x.z);
        o.w = fmaf(step, y.w - z.w, x.w);
      }
      *reinterpret_cast<float4 *>(p.pool + (int64_t)e.y * p.n_pad + j0) = o;
      const float dd[4] = {o.x - t4.x, o.y - t4.y, o.z - t4.z, o.w - t4.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (j0 + q < p.n_train)
          str += dd[q] * dd[q];
        else if (j0 + q < p.n_cases)
          ste += dd[q] * dd[q];
      }
    }
    const float2 t = subblock_sum(str, ste);
    if (lane == 0) sum[k][0][warp] = t;
    x = x2;
    y = y2;
    z = z2;
  }
}

// The same pipelined stream for bf16 sigma and 2048-case tiles (VEC = 2),
// mutation only: the next offspring's parent row and raw bf16 pairs are
// loaded while the current offspring is computed (the bf16 values are
// widened only when used, which keeps two offspring's operands within the
// register budget).  Arithmetic and sums as mutate4 / stream_item.
template <int OPB>
__device__ __forceinline__ void stream_item_pipe_bf16x2(const GenParams &p, int tile, int cnt,
                                                        const int4 *sels, const float *mss,
                                                        ItemSums<2, OPB> &sum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const __nv_bfloat16 *sig = static_cast<const __nv_bfloat16 *>(p.sigma_r);
  const int64_t base = (int64_t)tile * 2048 + tid * 4;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const uint2 zero2 = make_uint2(0u, 0u);
  auto widen = [](const uint2 u) {
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
  };
  float4 t4[2], x[2];
  uint2 y[2], z[2];
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    t4[v] = x[v] = zero;
    y[v] = z[v] = zero2;
  }
  auto load = [&](const int4 e, float4 (&xx)[2], uint2 (&yy)[2], uint2 (&zz)[2]) {
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int64_t j0 = base + v * 1024;
      if (j0 < p.n_pad) {
        xx[v] = __ldcg(reinterpret_cast<const float4 *>(p.pool + (int64_t)e.x * p.n_pad + j0));
        yy[v] = __ldg(reinterpret_cast<const uint2 *>(sig + (int64_t)e.z * p.n_pad + j0));
        zz[v] = __ldg(reinterpret_cast<const uint2 *>(sig + (int64_t)e.w * p.n_pad + j0));
      }
    }
  };
#pragma unroll
  for (int v = 0; v < 2; ++v)
    if (base + v * 1024 < p.n_pad)
      t4[v] = __ldg(reinterpret_cast<const float4 *>(p.target + base + v * 1024));
  load(sels[0], x, y, z);
  for (int k = 0; k < cnt; ++k) {
    const int orow = sels[k].y;
    const float step = mss[k];
    float4 x2[2] = {x[0], x[1]};
    uint2 y2[2] = {y[0], y[1]}, z2[2] = {z[0], z[1]};
    if (k + 1 < cnt) load(sels[k + 1], x2, y2, z2);
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int64_t j0 = base + v * 1024;
      float str = 0.f, ste = 0.f;
      if (j0 < p.n_pad) {
        const float4 a = widen(y[v]), b = widen(z[v]);
        float4 o;
        o.x = fmaf(step, a.x - b.x, x[v].x);
        o.y = fmaf(step, a.y - b.y, x[v].y);
        o.z = fmaf(step, a.z - b.z, x[v].z);
        o.w = fmaf(step, a.w - b.w, x[v].w);
        *reinterpret_cast<float4 *>(p.pool + (int64_t)orow * p.n_pad + j0) = o;
        const float dd[4] = {o.x - t4[v].x, o.y - t4[v].y, o.z - t4[v].z, o.w - t4[v].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (j0 + q < p.n_train)
            str += dd[q] * dd[q];
          else if (j0 + q < p.n_cases)
            ste += dd[q] * dd[q];
        }
      }
      const float2 t = subblock_sum(str, ste);
      if (lane == 0) sum[k][v][warp] = t;
    }
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      x[v] = x2[v];
      y[v] = y2[v];
      z[v] = z2[v];
    }
  }
}

// Chunk partials of one stream item from its sub-block totals (after a
// barrier that follows stream_item).
template <int VEC, int OPB>
__device__ __forceinline__ void item_partials(const GenParams &p, int tile, int i0, int cnt,
                                              const ItemSums<VEC, OPB> &sum) {
  const int chunks = (int)((p.n_pad + 1023) >> 10);   // this context's chunks
  for (int e = threadIdx.x; e < cnt * VEC; e += kGenThreads) {
    const int k = e / VEC, v = e - k * VEC;
    const int chunk = tile * VEC + v;
    if (chunk < chunks)
      p.partial[(size_t)(i0 + k) * p.tiles + p.chunk0 + chunk] = chunk_total(sum[k][v]);
  }
}

// Survival with elitism (Algorithm 1, "Survival") of run p by the whole CTA
// (blockDim.x = 256), from the fitness tables in memory: b_P = argmin parent
// fitness, b_O = argmin offspring fitness, w = argmax offspring fitness
// (first index on ties).  If F_T[b_P] < F_O[b_O] slot w takes parent b_P's
// row, fitness and an elite trace entry.  No row is copied: population
// slots map to rows of a pool of 2m rows, and survival rewrites that map
// (the paper's pointer swap of S_T and S_O).  Writes the best-of-generation
// log and advances the run's generation counter and parity.
static __device__ void survive_population(const GenParams &p, int g, int par) {
  __shared__ unsigned long long s_v[kGenThreads];
  __shared__ int s_i[kGenThreads];
  const int m = p.m;
  const double *FT = p.fit + (size_t)par * m;
  const double *FO = p.fit + (size_t)(par ^ 1) * m;
  double fbp, fbo, fw;
  int bP, bO, w;
  block_arg<false>(FT, m, s_v, s_i, fbp, bP);
  block_arg<false>(FO, m, s_v, s_i, fbo, bO);
  block_arg<true>(FO, m, s_v, s_i, fw, w);
  const bool elite = p.elitism && fbp < fbo;
  const int *cur = p.perm + (size_t)par * 2 * m;
  int *nxt = p.perm + (size_t)(par ^ 1) * 2 * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int ph = __ldcg(cur + i), fr = __ldcg(cur + m + i);
    nxt[i] = fr;       // offspring i becomes population slot i
    nxt[m + i] = ph;   // the parents' rows are free for the next offspring
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double *fit_o = p.fit + (size_t)(par ^ 1) * m;
    double *fte_o = p.fit_te + (size_t)(par ^ 1) * m;
    int best = bO;
    double btr = fbo;
    double bte = __ldcg(fte_o + bO);
    if (elite) {
      nxt[w] = __ldcg(cur + bP);
      nxt[m + bP] = __ldcg(cur + m + w);
      const double te = __ldcg(p.fit_te + (size_t)par * m + bP);
      fit_o[w] = fbp;
      fte_o[w] = te;
      p.trace[(size_t)g * m + w] = make_int4(bP, -1, -1, 0);
      best = w;
      btr = fbp;
      bte = te;
    }
    p.best_log[g] = make_double2(btr, bte);
    p.state->best_slot = best;
    p.state->done = 0u;
    p.state->parity = par ^ 1;
    p.state->gen = g + 1;
  }
}

}  // namespace gsgp
