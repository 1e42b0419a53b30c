// Persistent cooperative implementation of the GSGP generation loop: one
// launch runs G generations with every CTA resident for the whole launch,
// synchronised by a grid-wide barrier instead of kernel boundaries (the
// generation of the mid-size problem moves ~240 MB, about 35 us of HBM time,
// so per-launch overheads would otherwise dominate).
//
// Per generation g (parity par of the double-buffered tables):
//   S  selection: thread t of the grid draws offspring i = t, t + threads, ...
//      (tournament on training RMSE, two random trees, step) and records the
//      trace entry; parent rows / offspring rows come from the slot-to-row map.
//   -- barrier --
//   M  mutation stream: CTA b takes items b, b + grid, ... in tile-major order
//      (an item = one tile of 1024 * VEC cases for OPB offspring; the grid is
//      sized so that every CTA gets the same number of items), computes
//      s_O = s_T[parent] + ms (sR_a - sR_b) and the per-1024-case-chunk
//      (train, test) squared-error partials, summed in the same order as the
//      chained kernels and the interpreter.
//   -- barrier --
//   F1 fitness: warp w of the grid sums the partials of offspring w, w + warps,
//      ... in a fixed order into its RMSE; each CTA publishes the arg-min and
//      arg-max (value, first index) of the offspring it finished.
//   -- barrier --
//   F2 survival (every CTA, redundantly, from the per-CTA results): b_O, the
//      worst offspring w, and b_P = the best slot of the parents (known from
//      the previous survival).  If F_T[b_P] < F_O[b_O] slot w takes parent
//      b_P's row and fitness.  The new slot-to-row map, the elite's fitness and
//      trace entry and the best-of-generation log are written by the CTAs that
//      own them; the next selection applies the same decision to the old map
//      on the fly, so no fourth barrier is needed.
//
// The barrier is one arrival counter; every wait is a bounded spin and, when
// the bound is hit (a fault, never expected), sets a sticky error word, after
// which every CTA leaves the kernel.  Cooperative launch guarantees that all
// CTAs are co-resident.  The selection runs on the first CTAs and the
// persisting of the slot-to-row map on the last ones, so that CTAs arrive at
// the barriers spread out in time rather than all at once.
#include "kernels.cuh"
#include "reduce.cuh"
#include "stream.cuh"

namespace gsgp {

constexpr unsigned kSpinLimit = 1u << 24;   // ~1 s of 32-64 ns naps

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
// when the bound is hit or another CTA already gave up.
__device__ __forceinline__ bool wait_at_least(const unsigned *p, unsigned target, GridSync *gs) {
  unsigned spins = 0;
  while (ld_acquire_u32(p) < target) {
    if (ld_relaxed_s32(&gs->err) != 0) return false;
    if (++spins > kSpinLimit) {
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

// Warp-wide arg-min and arg-max of (key, index) pairs (first index on ties);
// every lane returns the warp's result.
__device__ __forceinline__ void warp_minmax(unsigned long long &mn, int &imn, unsigned long long &mx,
                                            int &imx) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long k1 = __shfl_xor_sync(0xffffffffu, mn, o);
    const int i1 = __shfl_xor_sync(0xffffffffu, imn, o);
    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, mx, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, imx, o);
    if (arg_better<false>(k1, i1, mn, imn)) {
      mn = k1;
      imn = i1;
    }
    if (arg_better<true>(k2, i2, mx, imx)) {
      mx = k2;
      imx = i2;
    }
  }
}

// Block-wide version: warps reduce with shuffles, then every thread reduces
// the per-warp results (one shared-memory round).
__device__ void block_minmax(unsigned long long mn, int imn, unsigned long long mx, int imx,
                             ulonglong2 *s_min, ulonglong2 *s_max, unsigned long long &omn,
                             int &oimn, unsigned long long &omx, int &oimx) {
  warp_minmax(mn, imn, mx, imx);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_min[warp] = make_ulonglong2(mn, (unsigned long long)(unsigned)imn);
    s_max[warp] = make_ulonglong2(mx, (unsigned long long)(unsigned)imx);
  }
  __syncthreads();
  omn = kKeyAboveAll;
  omx = kKeyBelowAll;
  oimn = oimx = 0x7fffffff;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    const ulonglong2 a = s_min[w], c = s_max[w];
    if (arg_better<false>(a.x, (int)a.y, omn, oimn)) {
      omn = a.x;
      oimn = (int)a.y;
    }
    if (arg_better<true>(c.x, (int)c.y, omx, oimx)) {
      omx = c.x;
      oimx = (int)c.y;
    }
  }
  __syncthreads();
}

// Per-CTA generation state, kept in shared memory so that the streaming
// phase has the registers to itself.  The survival decision of the previous
// generation is applied by the next selection to the old slot-to-row map and
// offspring fitness.
struct GenState {
  int g, par, best;
  double fbest, fbest_te;   // training / test RMSE of the best parent
  int active;               // 0: the tables of the current parity are complete in memory
  int old_par;              // parity whose map describes the previous population
  int elite, w, bP;
  double fbp;
};

// S: tournament selection and mutation draws; offspring i is drawn by thread
// i % 256 of CTA i / 256.
__device__ __forceinline__ void select_phase(const GenParams &p, const GenState &pd, int b,
                                             int nb) {
  const int m = p.m;
  const int tid = threadIdx.x;
  const int g = pd.g, par = pd.par;
  const double *F = p.fit + (size_t)par * m;
  const int *pm = p.perm + (size_t)(pd.active ? pd.old_par : par) * 2 * m;
  for (int i = b * kGenThreads + tid; i < m; i += nb * kGenThreads) {
    int orow;
    if (pd.active)   // rows of the population after the previous survival
      orow = (pd.elite && i == pd.bP) ? __ldcg(pm + m + pd.w) : __ldcg(pm + i);
    else
      orow = __ldcg(pm + m + i);
    const Draws d = draw_offspring(
        p, i, g,
        [&](int s) { return (pd.active && pd.elite && s == pd.w) ? pd.fbp : __ldcg(F + s); },
        [&](int s) {
          if (!pd.active) return __ldcg(pm + s);
          return (pd.elite && s == pd.w) ? __ldcg(pm + pd.bP) : __ldcg(pm + m + s);
        });
    p.sel[i] = make_int4(d.prow, orow, d.a, d.b);
    p.sel_ms[i] = d.ms;
    p.trace[(size_t)g * m + i] = make_int4(d.parent, d.a, d.b, __float_as_int(d.ms));
  }
}

// F1: offspring i is summed by warp (i / nb) % NW of CTA i % nb, which
// spreads the m offspring over all CTAs; each warp adds its partials in the
// fixed lane-strided order and one thread per offspring then takes the RMSE
// (the phase's only float64 division and square root).  Each CTA publishes
// the arg-min and arg-max (fitness key, first index) of its offspring.
__device__ __forceinline__ void fitness_phase(const GenParams &p, const PersistArgs &x, int par, int b,
                                           int nb, double2 *s_sse) {
  constexpr int NW = kGenThreads / 32;
  const int m = p.m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long mn = kKeyAboveAll, mx = kKeyBelowAll;
  int imn = 0x7fffffff, imx = 0x7fffffff;
  double *fo = p.fit + (size_t)(par ^ 1) * m;
  double *fo_te = p.fit_te + (size_t)(par ^ 1) * m;
  for (int r0 = 0; r0 < m; r0 += nb * NW) {
    const int i = r0 + warp * nb + b;
    if (i < m) {
      const double2 sse = warp_sum_partials(p.partial + (size_t)i * p.tiles, p.tiles, lane);
      if (lane == 0) s_sse[warp] = sse;
    }
    __syncthreads();
    if (tid < NW) {
      const int ii = r0 + tid * nb + b;
      if (ii < m) {
        const double2 sse = s_sse[tid];
        const double f = rmse_from_sse(sse.x, p.n_train);
        fo[ii] = f;
        fo_te[ii] = rmse_from_sse(sse.y, p.n_cases - p.n_train);
        const unsigned long long k = fit_key(f);
        if (arg_better<false>(k, ii, mn, imn)) {
          mn = k;
          imn = ii;
        }
        if (arg_better<true>(k, ii, mx, imx)) {
          mx = k;
          imx = ii;
        }
      }
    }
    __syncthreads();
  }
  if (warp == 0) {
    warp_minmax(mn, imn, mx, imx);
    if (lane == 0) {
      x.cta_min[b] = make_ulonglong2(mn, (unsigned long long)(unsigned)imn);
      x.cta_max[b] = make_ulonglong2(mx, (unsigned long long)(unsigned)imx);
    }
  }
}

template <typename SigT, int VEC, int OPB>
__global__ void __launch_bounds__(kGenThreads, 4) persist_kernel(const GenParams p, PersistArgs x) {
  constexpr int NW = kGenThreads / 32;
  constexpr int W = 1024 * VEC;
  __shared__ float s_red[2][OPB][VEC][NW][2];
  __shared__ ulonglong2 s_min[NW], s_max[NW];
  __shared__ double2 s_sse[NW];
  __shared__ int s_ok;
  __shared__ GenState st;

  GridSync *gs = x.gs;
  if (ld_relaxed_s32(&gs->err) != 0) return;   // an earlier launch failed
  const int m = p.m;
  const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int groups = (m + OPB - 1) / OPB;
  const int tiles = (int)((p.n_pad + W - 1) / W);
  const int items = tiles * groups;
  const SigT *sig = static_cast<const SigT *>(p.sigma_r);
  unsigned epoch = 0;

  if (tid == 0) {
    st.g = __ldcg(&p.state->gen);
    st.par = __ldcg(&p.state->parity);
    st.best = __ldcg(&p.state->best_slot);
    st.fbest = __ldcg(p.fit + (size_t)st.par * m + st.best);
    st.fbest_te = __ldcg(p.fit_te + (size_t)st.par * m + st.best);
    st.active = 0;
    st.old_par = st.elite = st.w = st.bP = 0;
    st.fbp = 0.0;
  }
  __syncthreads();

  for (int it = 0; it < x.G; ++it) {
    // ---------------- S: selection ----------------------------------------
    select_phase(p, st, b, nb);
    if (!grid_sync(gs, epoch, &s_ok)) return;

    // ---------------- M: mutation stream ----------------------------------
    // CTA b streams items b, b + grid, ... in tile-major order; the grid is
    // sized so that every CTA gets the same number of items.
    {
      int buf = 0;
      for (int item = b; item < items; item += nb, buf ^= 1) {
        const int tile = item / groups;
        const int i0 = (item - tile * groups) * OPB;
        const int cnt = min(OPB, m - i0);
        const int64_t base_case = (int64_t)tile * W;
        int4 sel = __ldcg(p.sel + i0);
        float ms = __ldcg(p.sel_ms + i0);
        for (int k = 0; k < cnt; ++k) {
          const float *src = p.pool + (int64_t)sel.x * p.n_pad;
          float *dst = p.pool + (int64_t)sel.y * p.n_pad;
          const SigT *ra = sig + (int64_t)sel.z * p.n_pad;
          const SigT *rb = sig + (int64_t)sel.w * p.n_pad;
          const float step = ms;
          if (k + 1 < cnt) {
            sel = __ldcg(p.sel + i0 + k + 1);
            ms = __ldcg(p.sel_ms + i0 + k + 1);
          }
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            const int64_t j0 = base_case + v * 1024 + tid * 4;
            float str = 0.f, ste = 0.f;
            if (j0 < p.n_pad) mutate4<SigT>(p, src, dst, ra, rb, j0, step, str, ste);
            warp_sum2(str, ste);
            if (lane == 0) {
              s_red[buf][k][v][warp][0] = str;
              s_red[buf][k][v][warp][1] = ste;
            }
          }
        }
        __syncthreads();
        const int chunk0 = tile * VEC;
        for (int e = tid; e < cnt * VEC; e += kGenThreads) {
          const int k = e / VEC, v = e - k * VEC;
          if (chunk0 + v >= p.tiles) continue;
          double tr = 0.0, te = 0.0;
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            tr += (double)s_red[buf][k][v][w][0];
            te += (double)s_red[buf][k][v][w][1];
          }
          p.partial[(size_t)(i0 + k) * p.tiles + chunk0 + v] = make_double2(tr, te);
        }
      }
    }
    if (!grid_sync(gs, epoch, &s_ok)) return;

    // ---------------- F1: offspring RMSE ----------------------------------
    fitness_phase(p, x, st.par, b, nb, s_sse);
    if (!grid_sync(gs, epoch, &s_ok)) return;

    // ---------------- F2: survival with elitism ---------------------------
    {
      unsigned long long mn = kKeyAboveAll, mx = kKeyBelowAll;
      int imn = 0x7fffffff, imx = 0x7fffffff;
      for (int k = tid; k < nb; k += kGenThreads) {
        const ulonglong2 a = __ldcg(x.cta_min + k);
        const ulonglong2 c = __ldcg(x.cta_max + k);
        if (arg_better<false>(a.x, (int)a.y, mn, imn)) {
          mn = a.x;
          imn = (int)a.y;
        }
        if (arg_better<true>(c.x, (int)c.y, mx, imx)) {
          mx = c.x;
          imx = (int)c.y;
        }
      }
      unsigned long long kbo, kw;
      int bO, w;
      block_minmax(mn, imn, mx, imx, s_min, s_max, kbo, bO, kw, w);
      const int g = st.g, par = st.par, bP = st.best;
      const double fbest = st.fbest, fbest_te = st.fbest_te;
      const bool elite = p.elitism && fit_key(fbest) < kbo;
      const int *cur = p.perm + (size_t)par * 2 * m;
      int *nxt = p.perm + (size_t)(par ^ 1) * 2 * m;
      // persist the new slot-to-row map: slot s by the (s / 256)-th CTA from the end
      for (int s = (nb - 1 - b) * kGenThreads + tid; s >= 0 && s < m; s += nb * kGenThreads) {
        nxt[s] = (elite && s == w) ? __ldcg(cur + bP) : __ldcg(cur + m + s);
        nxt[m + s] = (elite && s == bP) ? __ldcg(cur + m + w) : __ldcg(cur + s);
      }
      double *fo = p.fit + (size_t)(par ^ 1) * m;
      double *fo_te = p.fit_te + (size_t)(par ^ 1) * m;
      if (elite && b == w % nb && tid == 0) {
        fo[w] = fbest;
        fo_te[w] = fbest_te;
        p.trace[(size_t)g * m + w] = make_int4(bP, -1, -1, 0);
      }
      const int nbest = elite ? w : bO;
      const double nf = elite ? fbest : key_fit(kbo);
      // the test RMSE of the new best is needed only for the log; the last
      // CTA fetches it while the others move on
      double nfte = fbest_te;
      if (!elite && (b == nb - 1 || it + 1 < x.G)) nfte = __ldcg(fo_te + bO);
      if (b == nb - 1 && tid == 0) {
        p.best_log[g] = make_double2(nf, nfte);
        p.state->gen = g + 1;
        p.state->parity = par ^ 1;
        p.state->best_slot = nbest;
      }
      __syncthreads();   // every thread has read st
      if (tid == 0) {
        st.active = 1;
        st.old_par = par;
        st.elite = elite;
        st.w = w;
        st.bP = bP;
        st.fbp = fbest;
        st.best = nbest;
        st.fbest = nf;
        st.fbest_te = nfte;
        st.par = par ^ 1;
        st.g = g + 1;
      }
      __syncthreads();
    }
  }
}

template <typename SigT, int VEC, int OPB>
static const void *persist_fn() {
  return reinterpret_cast<const void *>(&persist_kernel<SigT, VEC, OPB>);
}

static const void *pick(int bf, const GenShape &sh) {
#define GSGP_P(V, O) \
  if (sh.vec == V && sh.opb == O) return bf ? persist_fn<__nv_bfloat16, V, O>() : persist_fn<float, V, O>();
  GSGP_P(1, 1) GSGP_P(1, 2) GSGP_P(1, 4) GSGP_P(2, 1) GSGP_P(2, 2) GSGP_P(2, 4)
#undef GSGP_P
  return nullptr;
}

bool persist_shape_supported(const GenShape &sh) {
  return (sh.vec == 1 || sh.vec == 2) && (sh.opb == 1 || sh.opb == 2 || sh.opb == 4);
}

int persist_max_grid(int sigma_bf16, const GenShape &sh) {
  const void *fn = pick(sigma_bf16, sh);
  if (!fn) return 0;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
    return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kGenThreads, 0) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

cudaError_t launch_persist(const GenParams &p, const PersistArgs &x, int sigma_bf16,
                           const GenShape &sh, int grid, cudaStream_t s) {
  const void *fn = pick(sigma_bf16, sh);
  if (!fn || grid <= 0) return cudaErrorInvalidValue;
  GenParams pp = p;
  PersistArgs xx = x;
  void *args[] = {&pp, &xx};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kGenThreads), args, 0, s);
}

}  // namespace gsgp
