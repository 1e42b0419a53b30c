// One GSGP generation in one launch (Algorithm 1 loop body): tournament
// selection, geometric semantic mutation of every offspring fused with its
// training/test squared errors, the offspring RMSE and survival with
// elitism, plus the ancestry trace.
//
// Work decomposition.  The m x n offspring semantic matrix is cut into
// tiles of W = 1024 * VEC cases; a CTA owns one tile for OPB consecutive
// offspring.  CTA index = tile * groups + group, so the CTAs resident at any
// moment cover one or two case tiles: the sigma(R) columns of those tiles
// (r x W values) and the parents re-selected by several offspring are then
// read from L2 while the parent and offspring rows stream through HBM once.
//
// Per CTA:
//   1. prologue - thread k < OPB draws offspring i's Philox words of this
//      generation: tournament candidates (the smallest training RMSE wins,
//      the earliest drawn on ties), random trees a, b and the mutation step;
//      the CTA of tile 0 records (parent, a, b, ms) in the trace.
//   2. stream - for each offspring: s_O = s_T[parent] + ms (sR[a] - sR[b])
//      on 4 * VEC cases per thread (float4 loads/stores), squared errors
//      against the targets accumulated in float over train and test cases,
//      reduced with warp shuffles.
//   3. epilogue - per offspring one (train, test) double partial per tile;
//      the CTA that completes an offspring's last tile (atomic tile counter)
//      sums its partials in a fixed order into the RMSE; the CTA that
//      completes the last offspring runs survival for the whole population.
//
// Survival (Sec. 2.2, "Survival"): b_P = argmin parent fitness, b_O = argmin
// offspring fitness (first index); if F_T[b_P] < F_O[b_O] the first worst
// offspring w is replaced by parent b_P.  No row is copied: population slots
// map to rows of a pool of 2m rows, and replacement swaps two entries of
// that map, which keeps the paper's pointer swap of S_T and S_O.
#include "kernels.cuh"
#include "reduce.cuh"

namespace gsgp {

constexpr int kGenThreads = 256;

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

// Survival with elitism for the whole population, run by the last CTA.
__device__ void finalize_generation(const GenParams &p, int g, int par) {
  __shared__ double s_v[kGenThreads];
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
    const int ph = cur[i], fr = cur[m + i];
    nxt[i] = fr;       // offspring i becomes population slot i
    nxt[m + i] = ph;   // parents' rows are free for the next offspring
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double *fit_o = p.fit + (size_t)(par ^ 1) * m;
    double *fte_o = p.fit_te + (size_t)(par ^ 1) * m;
    int best = bO;
    double btr = fbo;
    double bte = __ldcg(fte_o + bO);
    if (elite) {
      nxt[w] = cur[bP];
      nxt[m + bP] = cur[m + w];
      const double te = p.fit_te[(size_t)par * m + bP];
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

template <typename SigT, int VEC, int OPB>
__global__ void __launch_bounds__(kGenThreads) generation_kernel(const GenParams p) {
  constexpr int W = kGenThreads * 4 * VEC;
  constexpr int NW = kGenThreads / 32;
  __shared__ int s_prow[OPB], s_orow[OPB], s_a[OPB], s_b[OPB];
  __shared__ float s_ms[OPB];
  __shared__ float s_red[OPB][NW][2];
  __shared__ int s_last[OPB];
  __shared__ int s_final;

  const int g = __ldcg(&p.state->gen);
  const int par = __ldcg(&p.state->parity);
  const int m = p.m;
  const int groups = (m + OPB - 1) / OPB;
  const int tile = blockIdx.x / groups;
  const int grp = blockIdx.x - tile * groups;
  const int i0 = grp * OPB;
  const int cnt = min(OPB, m - i0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int *perm = p.perm + (size_t)par * 2 * m;

  // 1. selection and mutation draws (stream (i, g) of run p.run)
  if (tid < cnt) {
    const int i = i0 + tid;
    const double *F = p.fit + (size_t)par * m;
    WordStream ws(p.key, (uint32_t)i, (uint32_t)g, p.run);
    int parent = i;
    if (p.tsize > 0) {
      parent = (int)draw_index(ws.next(), (uint32_t)m);
      double best = F[parent];
      for (int k = 1; k < p.tsize; ++k) {
        const int c = (int)draw_index(ws.next(), (uint32_t)m);
        const double f = F[c];
        if (f < best) {
          best = f;
          parent = c;
        }
      }
    }
    const int a = (int)draw_index(ws.next(), (uint32_t)p.r);
    const int b = (int)draw_index(ws.next(), (uint32_t)p.r);
    const uint32_t wms = ws.next();
    float ms = p.ms;
    if (p.ms_mode == 1) ms = __double2float_rn(__dmul_rn((double)p.ms, (double)draw_u24(wms)));
    s_prow[tid] = perm[parent];
    s_orow[tid] = perm[m + i];
    s_a[tid] = a;
    s_b[tid] = b;
    s_ms[tid] = ms;
    if (tile == 0) p.trace[(size_t)g * m + i] = make_int4(parent, a, b, __float_as_int(ms));
  }
  __syncthreads();

  // 2. stream the tile: targets once, then every offspring of the group
  const int64_t base = (int64_t)tile * W;
  const SigT *sig = static_cast<const SigT *>(p.sigma_r);
  float4 tv[VEC];
  bool ok[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const int64_t j = base + v * 1024 + tid * 4;
    ok[v] = j < p.n_pad;
    tv[v] = ok[v] ? __ldg(reinterpret_cast<const float4 *>(p.target + j))
                  : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int k = 0; k < cnt; ++k) {
    const float *src = p.pool + (int64_t)s_prow[k] * p.n_pad + base;
    float *dst = p.pool + (int64_t)s_orow[k] * p.n_pad + base;
    const SigT *ra = sig + (int64_t)s_a[k] * p.n_pad + base;
    const SigT *rb = sig + (int64_t)s_b[k] * p.n_pad + base;
    const float ms = s_ms[k];
    float str = 0.f, ste = 0.f;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      if (!ok[v]) continue;
      const int off = v * 1024 + tid * 4;
      const float4 s = *reinterpret_cast<const float4 *>(src + off);
      const float4 a4 = SigLoad<SigT>::load(ra, off);
      const float4 b4 = SigLoad<SigT>::load(rb, off);
      float4 o;
      o.x = fmaf(ms, a4.x - b4.x, s.x);
      o.y = fmaf(ms, a4.y - b4.y, s.y);
      o.z = fmaf(ms, a4.z - b4.z, s.z);
      o.w = fmaf(ms, a4.w - b4.w, s.w);
      *reinterpret_cast<float4 *>(dst + off) = o;
      const float ov[4] = {o.x, o.y, o.z, o.w};
      const float tt[4] = {tv[v].x, tv[v].y, tv[v].z, tv[v].w};
      const int64_t j0 = base + off;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float d = ov[q] - tt[q];
        if (j0 + q < p.n_train)
          str += d * d;
        else if (j0 + q < p.n_cases)
          ste += d * d;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      str += __shfl_xor_sync(0xffffffffu, str, o);
      ste += __shfl_xor_sync(0xffffffffu, ste, o);
    }
    if (lane == 0) {
      s_red[k][warp][0] = str;
      s_red[k][warp][1] = ste;
    }
  }
  __syncthreads();

  // 3. per-tile partials; detect the last tile of every offspring
  if (tid < cnt) {
    double tr = 0.0, te = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      tr += (double)s_red[tid][w][0];
      te += (double)s_red[tid][w][1];
    }
    const int i = i0 + tid;
    p.partial[(size_t)i * p.tiles + tile] = make_double2(tr, te);
    __threadfence();
    const unsigned prev = atomicAdd(&p.tile_count[i], 1u);
    s_last[tid] = prev == (unsigned)(p.tiles - 1);
    __threadfence();
  }
  __syncthreads();
  for (int k = warp; k < cnt; k += NW) {
    if (!s_last[k]) continue;
    const int i = i0 + k;
    const double2 sse = warp_sum_partials(p.partial + (size_t)i * p.tiles, p.tiles, lane);
    if (lane == 0) {
      p.fit[(size_t)(par ^ 1) * m + i] = rmse_from_sse(sse.x, p.n_train);
      p.fit_te[(size_t)(par ^ 1) * m + i] = rmse_from_sse(sse.y, p.n_cases - p.n_train);
      p.tile_count[i] = 0u;
      __threadfence();
    }
  }
  __syncthreads();
  if (tid == 0) {
    int nf = 0;
    for (int k = 0; k < cnt; ++k) nf += s_last[k];
    int fin = 0;
    if (nf) {
      __threadfence();
      const unsigned prev = atomicAdd(&p.state->done, (unsigned)nf);
      fin = prev + (unsigned)nf == (unsigned)m;
      __threadfence();
    }
    s_final = fin;
  }
  __syncthreads();
  if (s_final) finalize_generation(p, g, par);
}

int gen_tile_cases(const GenShape &sh) { return kGenThreads * 4 * sh.vec; }

bool gen_shape_supported(const GenShape &sh) {
  return (sh.vec == 1 || sh.vec == 2 || sh.vec == 4) && (sh.opb == 2 || sh.opb == 4 || sh.opb == 8);
}

template <typename SigT, int VEC>
static void launch_opb(const GenParams &p, int opb, unsigned grid, cudaStream_t s) {
  switch (opb) {
    case 2: generation_kernel<SigT, VEC, 2><<<grid, kGenThreads, 0, s>>>(p); break;
    case 4: generation_kernel<SigT, VEC, 4><<<grid, kGenThreads, 0, s>>>(p); break;
    default: generation_kernel<SigT, VEC, 8><<<grid, kGenThreads, 0, s>>>(p); break;
  }
}

template <typename SigT>
static void launch_vec(const GenParams &p, const GenShape &sh, unsigned grid, cudaStream_t s) {
  switch (sh.vec) {
    case 1: launch_opb<SigT, 1>(p, sh.opb, grid, s); break;
    case 2: launch_opb<SigT, 2>(p, sh.opb, grid, s); break;
    default: launch_opb<SigT, 4>(p, sh.opb, grid, s); break;
  }
}

cudaError_t launch_generation(const GenParams &p, int sigma_bf16, const GenShape &sh,
                              cudaStream_t s) {
  if (!gen_shape_supported(sh)) return cudaErrorInvalidValue;
  const int groups = (p.m + sh.opb - 1) / sh.opb;
  const unsigned grid = (unsigned)((int64_t)p.tiles * groups);
  if (sigma_bf16)
    launch_vec<__nv_bfloat16>(p, sh, grid, s);
  else
    launch_vec<float>(p, sh, grid, s);
  return cudaGetLastError();
}

}  // namespace gsgp
