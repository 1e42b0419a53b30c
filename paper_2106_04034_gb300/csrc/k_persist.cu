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
#include <type_traits>

#include "gridsync.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "stream.cuh"

namespace gsgp {

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
template <bool CROSS>
__device__ __forceinline__ void select_phase(const GenParams &p, const GenState &pd, int b,
                                             int nb) {
  const int m = p.m;
  const int tid = threadIdx.x;
  if (tid >= kGenThreads) return;   // a producer warp, if any, has no draws
  const int g = pd.g, par = pd.par;
  const double *F = p.fit + (size_t)par * m;
  const int *pm = p.perm + (size_t)(pd.active ? pd.old_par : par) * 2 * m;
  for (int i = b * kGenThreads + tid; i < m; i += nb * kGenThreads) {
    int orow;
    if (pd.active)   // rows of the population after the previous survival
      orow = (pd.elite && i == pd.bP) ? __ldcg(pm + m + pd.w) : __ldcg(pm + i);
    else
      orow = __ldcg(pm + m + i);
    const Draws d = draw_offspring<CROSS>(
        p, i, g,
        [&](int s) { return (pd.active && pd.elite && s == pd.w) ? pd.fbp : __ldcg(F + s); },
        [&](int s) {
          if (!pd.active) return __ldcg(pm + s);
          return (pd.elite && s == pd.w) ? __ldcg(pm + pd.bP) : __ldcg(pm + m + s);
        });
    p.sel[i] = sel_entry(d, orow);
    p.sel_ms[i] = d.ms;
    p.trace[(size_t)g * m + i] = trace_entry(d);
  }
}

// F1: offspring i is summed by warp (i / nb) % NW of CTA i % nb, which
// spreads the m offspring over all CTAs; each warp adds its partials in the
// fixed lane-strided order and one thread per offspring then takes the RMSE
// (the phase's only float64 division and square root).  Each CTA publishes
// the arg-min and arg-max (fitness key, first index) of its offspring.
// kLongRows: rows of more than 128 chunks are summed by the unrolled,
// not-inlined warp_sum_partials_long (same order, same result); only the
// kernels whose streaming code keeps its registers with that call use it.
template <bool kLongRows>
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
    if (warp < NW && i < m) {
      const double2 *row = p.partial + (size_t)i * p.tiles;
      const double2 sse = kLongRows && p.tiles > 128 ? warp_sum_partials_long(row, p.tiles, lane)
                                                     : warp_sum_partials(row, p.tiles, lane);
      if (lane == 0) s_sse[warp] = sse;
    }
    __syncthreads();
    if (tid < NW) {
      const int ii = r0 + tid * nb + b;
      if (ii < m) {
        const double2 sse = s_sse[tid];
        const double f = rmse_from_sse(sse.x, p.n_train_all);
        fo[ii] = f;
        fo_te[ii] = rmse_from_sse(sse.y, p.n_test_all);
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

// F2: survival with elitism, decided redundantly by every CTA from the
// per-CTA arg-min / arg-max of F1; the best parent b_P is the best slot the
// previous survival kept.  Updates the CTA's generation state.
__device__ __forceinline__ void survive_phase(const GenParams &p, const PersistArgs &x, GenState &st,
                                          int b, int nb, bool last_generation,
                                          ulonglong2 *s_min, ulonglong2 *s_max) {
  const int m = p.m;
  const int tid = threadIdx.x;
  const bool worker = tid < kGenThreads;

  unsigned long long mn = kKeyAboveAll, mx = kKeyBelowAll;
  int imn = 0x7fffffff, imx = 0x7fffffff;
  for (int k = tid; worker && k < nb; k += kGenThreads) {
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
  for (int s = (nb - 1 - b) * kGenThreads + tid; worker && s >= 0 && s < m;
       s += nb * kGenThreads) {
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
  if (!elite && (b == nb - 1 || !last_generation)) nfte = __ldcg(fo_te + bO);
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

// MINB: CTAs per SM the register budget is sized for (4: 64 registers a
// thread; 6: 40, the (2, 2) shape, which streams without the one-offspring-
// ahead pipelining and keeps more warps resident instead).
template <typename SigT, int VEC, int OPB, bool CROSS, int MINB = 4>
__global__ void __launch_bounds__(kGenThreads, MINB) persist_kernel(const GenParams p, PersistArgs x) {
  constexpr int NW = kGenThreads / 32;
  constexpr int W = 1024 * VEC;
  __shared__ ItemSums<VEC, OPB> s_sum[2];   // sub-block totals, double-buffered per item
  __shared__ int4 s_isel[2][OPB];           // draws of the current / next item (VEC = 1)
  __shared__ float s_ims[2][OPB];
  __shared__ ulonglong2 s_min[32], s_max[32];
  __shared__ double2 s_sse[NW];
  __shared__ int s_ok;
  __shared__ GenState st;

  GridSync *gs = x.gs;
  if (ld_relaxed_s32(&gs->err) != 0) return;   // an earlier launch failed
  const int m = p.m;
  const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int groups = (m + OPB - 1) / OPB;
  const int tiles = (int)((p.n_pad + W - 1) / W);
  const int items = tiles * groups;
  unsigned epoch = 0;
  auto barrier = [&]() { return grid_sync_args(x, epoch, &s_ok); };

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
    select_phase<CROSS>(p, st, b, nb);
    if (!barrier()) return;

    // ---------------- M: mutation stream ----------------------------------
    // CTA b streams items b, b + grid, ... in tile-major order; the grid is
    // sized so that every CTA gets the same number of items.
    constexpr bool kPipeBf16 = VEC == 2 && !CROSS && std::is_same<SigT, __nv_bfloat16>::value && MINB == 4;
    if constexpr ((VEC == 1 && MINB == 4) || kPipeBf16) {
      // 1024-case tiles (or bf16 sigma with 2048-case tiles): the draws of
      // each item in shared memory, one item ahead, and the row loads
      // pipelined one offspring ahead
      int buf = 0;
      if (tid < OPB && b < items) {
        const int i = (b % groups) * OPB + tid;
        if (i < m) {
          s_isel[0][tid] = __ldcg(p.sel + i);
          s_ims[0][tid] = __ldcg(p.sel_ms + i);
        }
      }
      __syncthreads();
      for (int item = b; item < items; item += nb, buf ^= 1) {
        const int tile = item / groups;
        const int i0 = (item - tile * groups) * OPB;
        const int cnt = min(OPB, m - i0);
        if (tid < OPB && item + nb < items) {
          const int i = ((item + nb) % groups) * OPB + tid;
          if (i < m) {
            s_isel[buf ^ 1][tid] = __ldcg(p.sel + i);
            s_ims[buf ^ 1][tid] = __ldcg(p.sel_ms + i);
          }
        }
        if constexpr (VEC == 1)
          stream_item_pipe<SigT, OPB, CROSS>(p, tile, cnt, s_isel[buf], s_ims[buf], s_sum[buf]);
        else
          stream_item_pipe_bf16x2<OPB>(p, tile, cnt, s_isel[buf], s_ims[buf], s_sum[buf]);
        // one barrier per item: it also publishes the next item's draws
        __syncthreads();
        item_partials<VEC, OPB>(p, tile, i0, cnt, s_sum[buf]);
      }
    } else {
      int buf = 0;   // alternates per item
      // the first draws of the next item are loaded one item ahead
      int4 sel_next = make_int4(0, 0, 0, 0);
      float ms_next = 0.f;
      if (b < items) {
        const int i0 = (b % groups) * OPB;
        sel_next = __ldcg(p.sel + i0);
        ms_next = __ldcg(p.sel_ms + i0);
      }
      for (int item = b; item < items; item += nb, buf ^= 1) {
        const int tile = item / groups;
        const int i0 = (item - tile * groups) * OPB;
        const int cnt = min(OPB, m - i0);
        const int4 sel = sel_next;
        const float ms = ms_next;
        if (item + nb < items) {
          const int i0n = ((item + nb) % groups) * OPB;
          sel_next = __ldcg(p.sel + i0n);
          ms_next = __ldcg(p.sel_ms + i0n);
        }
        stream_item<SigT, VEC, OPB, CROSS>(p, tile, i0, cnt, sel, ms, s_sum[buf]);
        // one barrier per item; the other buffer is written by the next item,
        // and this one again only after the next item's barrier
        __syncthreads();
        item_partials<VEC, OPB>(p, tile, i0, cnt, s_sum[buf]);
      }
    }
    if (!barrier()) return;

    // ---------------- F1: offspring RMSE ----------------------------------
    fitness_phase<VEC == 2>(p, x, st.par, b, nb, s_sse);
    if (!barrier()) return;

    // ---------------- F2: survival with elitism ---------------------------
    survive_phase(p, x, st, b, nb, it + 1 == x.G, s_min, s_max);
  }
}

// ---------------------------------------------------------------------------
// TMA-staged variant of the mutation stream.  A producer warp (warp 16) keeps
// up to S units in flight: for each unit (one offspring x one tile of
// W = 1024 * VEC cases) its lane 0 issues three bulk asynchronous copies
// (cp.async.bulk, global -> shared, completion counted in bytes on the
// unit's "full" mbarrier): the parent row segment and the two sigma(R) row
// segments, 4 KB * VEC each.  The 16 consumer warps take every unit in
// order: wait on "full", compute the offspring from shared memory (warp w
// takes sub-block w % 8 of chunks w / 8, w / 8 + 2, ..., 4 cases per lane,
// the targets read through L2 before the wait), store it, leave their
// sub-block totals in shared memory and arrive on the unit's "empty"
// mbarrier.  The producer warp then finishes the unit's chunk sums
// (canonical order) and reuses the slot.  A bulk copy streams HBM at the
// copy rate only when it is large (measured on this GPU: 1.7 TB/s with
// 4 KB copies from one producer lane per SM, 6.8 TB/s with 16 KB copies),
// so the useful shapes are VEC = 4 (16 KB copies) and VEC = 2.
// ---------------------------------------------------------------------------
constexpr int kTmaConsumerWarps = 16;
constexpr int kTmaThreads = kTmaConsumerWarps * 32 + 32;      // + producer warp
constexpr int kTmaSmemBudget = 200 * 1024;   // stage buffers; the rest is static smem

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait on an mbarrier phase; false when it gives up (then the error
// word is set) or when another thread already gave up.
constexpr unsigned kMbarSpinLimit = 1u << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, GridSync *gs,
                                          volatile int *s_fail) {
  unsigned spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    ++spins;
    if ((spins & 1023u) == 0 && (*s_fail || ld_relaxed_s32(&gs->err) != 0)) return false;
    if (spins > kMbarSpinLimit) {
      atomicExch(&gs->err, 1);
      return false;
    }
  }
  return true;
}

// Stages S: every consumer warp consumes every unit, in order, so no
// mbarrier wait (by phase parity, which only tells the current phase from
// the one before) is ever issued more than one phase ahead.
template <typename SigT, int VEC>
struct TmaCfg {
  static constexpr int W = 1024 * VEC;
  // parent row segment (float), two sigma(R) row segments
  static constexpr int kStageBytes = W * (int)(sizeof(float) + 2 * sizeof(SigT));
  static constexpr int S0 = kTmaSmemBudget / kStageBytes;
  static constexpr int S = S0 > 16 ? 16 : S0;   // stages
  static constexpr int kSmem = S * kStageBytes;
  static_assert(S >= 2, "stage layout");
};

struct UnitMeta {
  int i;      // offspring slot
  int tile;   // case tile
  int orow;   // pool row the offspring is written to
  float ms;
};

template <typename SigT, int VEC>
__global__ void __launch_bounds__(kTmaThreads, 1) persist_tma_kernel(const GenParams p, PersistArgs x) {
  using C = TmaCfg<SigT, VEC>;
  constexpr int W = C::W, S = C::S, NW = kTmaConsumerWarps;
  extern __shared__ __align__(128) unsigned char stage_mem[];
  __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S];
  __shared__ UnitMeta meta[S];
  __shared__ float2 s_sub[S][VEC][8];    // per unit and chunk: sub-block totals
  __shared__ ulonglong2 s_min[32], s_max[32];
  __shared__ double2 s_sse[kGenThreads / 32];
  __shared__ int s_ok;
  __shared__ volatile int s_fail;
  __shared__ int s_issued;   // units issued by the producer in this generation
  __shared__ GenState st;

  GridSync *gs = x.gs;
  if (ld_relaxed_s32(&gs->err) != 0) return;   // an earlier launch failed
  const int m = p.m;
  const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tiles = (int)((p.n_pad + W - 1) / W);
  const int items = tiles * m;                  // one unit = (tile, offspring); < 2^31 (host)
  const int nunits = b < items ? (items - 1 - b) / nb + 1 : 0;
  const SigT *sig = static_cast<const SigT *>(p.sigma_r);
  unsigned epoch = 0;
  unsigned u0 = 0;   // units this CTA has run in earlier generations of the launch
  auto barrier = [&]() { return grid_sync_args(x, epoch, &s_ok); };

  if (tid == 0) {
    for (int k = 0; k < S; ++k) {
      mbar_init(&full_bar[k], 1);
      mbar_init(&empty_bar[k], NW);   // every consumer warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
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
    select_phase<false>(p, st, b, nb);
    if (!barrier()) return;

    // ---------------- M: TMA-staged mutation stream -----------------------
    bool ok = true;
    if (tid == 0) s_issued = 0;
    __syncthreads();
    if (warp == NW) {
      // producer warp: retires consumed units (chunk sums from the consumers'
      // sub-block totals, lane v for chunk v) and lane 0 issues the copies;
      // the draws of units are loaded 32 at a time, one per lane, a batch ahead
      int4 bs_cur = make_int4(0, 0, 0, 0), bs_nxt = make_int4(0, 0, 0, 0);
      float bm_cur = 0.f, bm_nxt = 0.f;
      auto load_batch = [&](int q_first, int4 &s4, float &sm) {
        const int qq = q_first + lane;
        if (qq < nunits) {
          const int i = (b + qq * nb) % m;
          s4 = __ldcg(p.sel + i);
          sm = __ldcg(p.sel_ms + i);
        }
      };
      load_batch(0, bs_cur, bm_cur);
      load_batch(32, bs_nxt, bm_nxt);
      for (int q = 0; q < nunits + S && ok; ++q) {
        if (q >= S) {   // retire unit q - S (its slot is reused next, or drained)
          const unsigned u = u0 + q - S;
          const int slot = (int)(u % S);
          ok = __all_sync(0xffffffffu, mbar_wait(&empty_bar[slot], (u / S) & 1u, gs, &s_fail));
          if (!ok) break;   // warp-uniform
          if (lane < VEC) {   // lane v finishes chunk v
            const UnitMeta mt = meta[slot];
            const int chunk = mt.tile * VEC + lane;
            if (chunk < (int)((p.n_pad + 1023) >> 10))
              p.partial[(size_t)mt.i * p.tiles + p.chunk0 + chunk] =
                  chunk_total(s_sub[slot][lane]);
          }
          __syncwarp();
        }
        if (q < nunits && q > 0 && (q & 31) == 0) {   // next batch of draws
          bs_cur = bs_nxt;
          bm_cur = bm_nxt;
          load_batch(q + 32, bs_nxt, bm_nxt);
        }
        int4 sl;
        float ms_u = 0.f;
        if (q < nunits) {   // warp-uniform: every lane joins the shuffles
          const int src = q & 31;
          sl.x = __shfl_sync(0xffffffffu, bs_cur.x, src);
          sl.y = __shfl_sync(0xffffffffu, bs_cur.y, src);
          sl.z = __shfl_sync(0xffffffffu, bs_cur.z, src);
          sl.w = __shfl_sync(0xffffffffu, bs_cur.w, src);
          ms_u = __shfl_sync(0xffffffffu, bm_cur, src);
        }
        if (q < nunits && lane == 0) {   // issue unit q
          const unsigned u = u0 + q;
          const int slot = (int)(u % S);
          const int item = b + q * nb;
          const int tile = item / m;
          const int i = item - tile * m;
          meta[slot] = UnitMeta{i, tile, sl.y, ms_u};
          const int64_t base = (int64_t)tile * W;
          const int64_t rem = p.n_pad - base;
          const int n = (int)(rem < W ? rem : W);
          unsigned char *st_p = stage_mem + (size_t)slot * C::kStageBytes;
          SigT *st_a = reinterpret_cast<SigT *>(st_p + (size_t)W * sizeof(float));
          SigT *st_b = st_a + W;
          mbar_arrive_expect_tx(&full_bar[slot],
                                (unsigned)n * (unsigned)(sizeof(float) + 2 * sizeof(SigT)));
          bulk_copy_g2s(st_p, p.pool + (int64_t)sl.x * p.n_pad + base, (unsigned)n * 4u,
                        &full_bar[slot]);
          bulk_copy_g2s(st_a, sig + (int64_t)sl.z * p.n_pad + base, (unsigned)(n * sizeof(SigT)),
                        &full_bar[slot]);
          bulk_copy_g2s(st_b, sig + (int64_t)sl.w * p.n_pad + base, (unsigned)(n * sizeof(SigT)),
                        &full_bar[slot]);
          s_issued = q + 1;
        }
        __syncwarp();
      }
      if (!ok) s_fail = 1;
    } else {
      // consumer warps: every warp takes every unit, in order; warp w handles
      // sub-block w % 8 (128 cases) of chunks w / 8, w / 8 + 2, ... of each
      // unit, 4 cases per lane, the same cases per lane as the 256-thread
      // CTAs of the other kernels; the targets come through L2, requested
      // before the wait for the unit's rows
      const int sb = warp & 7, v0 = warp >> 3;
      constexpr int kMyChunks = (VEC + 1) / 2;   // chunks v0, v0 + 2, ... below VEC
      for (int q = 0; q < nunits && ok; ++q) {
        const unsigned u = u0 + q;
        const int slot = (int)(u % S);
        const int item = b + q * nb;
        const int64_t base = (int64_t)(item / m) * W;
        float4 t4[kMyChunks];
#pragma unroll
        for (int c = 0; c < kMyChunks; ++c) {
          const int jl = (v0 + 2 * c) * 1024 + sb * 128 + lane * 4;
          t4[c] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (v0 + 2 * c < VEC && base + jl < p.n_pad)
            t4[c] = __ldg(reinterpret_cast<const float4 *>(p.target + base + jl));
        }
        ok = __all_sync(0xffffffffu, mbar_wait(&full_bar[slot], (u / S) & 1u, gs, &s_fail));
        if (!ok) {   // warp-uniform
          s_fail = 1;
          break;
        }
        const UnitMeta mt = meta[slot];
        const unsigned char *st_p = stage_mem + (size_t)slot * C::kStageBytes;
        const float *sp = reinterpret_cast<const float *>(st_p);
        const SigT *sa = reinterpret_cast<const SigT *>(sp + W);
        const SigT *sbb = sa + W;
        float *dst = p.pool + (int64_t)mt.orow * p.n_pad + base;
#pragma unroll
        for (int c = 0; c < kMyChunks; ++c) {
          const int v = v0 + 2 * c;
          if (v >= VEC) break;   // warp-uniform
          const int jl = v * 1024 + sb * 128 + lane * 4;
          float str = 0.f, ste = 0.f;
          if (base + jl < p.n_pad) {
            const float4 s4 = *reinterpret_cast<const float4 *>(sp + jl);
            float4 a4, b4;
            if (sizeof(SigT) == 4) {
              a4 = *reinterpret_cast<const float4 *>(sa + jl);
              b4 = *reinterpret_cast<const float4 *>(sbb + jl);
            } else {
              const uint2 ua = *reinterpret_cast<const uint2 *>(sa + jl);
              const uint2 ub = *reinterpret_cast<const uint2 *>(sbb + jl);
              a4 = make_float4(__uint_as_float(ua.x << 16), __uint_as_float(ua.x & 0xffff0000u),
                               __uint_as_float(ua.y << 16), __uint_as_float(ua.y & 0xffff0000u));
              b4 = make_float4(__uint_as_float(ub.x << 16), __uint_as_float(ub.x & 0xffff0000u),
                               __uint_as_float(ub.y << 16), __uint_as_float(ub.y & 0xffff0000u));
            }
            const int64_t j0 = base + jl;
            float4 o;
            o.x = fmaf(mt.ms, a4.x - b4.x, s4.x);
            o.y = fmaf(mt.ms, a4.y - b4.y, s4.y);
            o.z = fmaf(mt.ms, a4.z - b4.z, s4.z);
            o.w = fmaf(mt.ms, a4.w - b4.w, s4.w);
            *reinterpret_cast<float4 *>(dst + jl) = o;
            const float dd[4] = {o.x - t4[c].x, o.y - t4[c].y, o.z - t4[c].z, o.w - t4[c].w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if (j0 + k < p.n_train)
                str += dd[k] * dd[k];
              else if (j0 + k < p.n_cases)
                ste += dd[k] * dd[k];
            }
          }
          const float2 sub = subblock_sum(str, ste);
          if (lane == 0) s_sub[slot][v][sb] = sub;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_bar[slot]);
      }
    }
    __syncthreads();
    if (s_fail) {
      // a wait gave up: let every bulk copy this CTA issued land (each unit
      // issued is one phase of its slot's full barrier; bounded), then leave
      if (tid == 0) {
        const int issued = s_issued;
        for (int q = issued > S ? issued - S : 0; q < issued; ++q) {
          const unsigned u = u0 + q;
          unsigned spins = 0;
          while (!mbar_try_wait(&full_bar[u % S], (u / S) & 1u) && ++spins < kMbarSpinLimit) {
          }
        }
      }
      __syncthreads();
      return;
    }
    u0 += (unsigned)nunits;
    if (!barrier()) return;

    fitness_phase<false>(p, x, st.par, b, nb, s_sse);
    if (!barrier()) return;

    survive_phase(p, x, st, b, nb, it + 1 == x.G, s_min, s_max);
  }
}

template <typename SigT, int VEC, int OPB, int MINB = 4>
static const void *persist_fn(bool cross) {
  return cross ? reinterpret_cast<const void *>(&persist_kernel<SigT, VEC, OPB, true, MINB>)
               : reinterpret_cast<const void *>(&persist_kernel<SigT, VEC, OPB, false, MINB>);
}


template <typename SigT, int VEC>
static const void *persist_tma_fn() {
  return reinterpret_cast<const void *>(&persist_tma_kernel<SigT, VEC>);
}

// (vec, opb) with opb in {1, 2, 4}: register stream, 256 threads; opb == 0:
// TMA-staged stream, 288 threads, dynamic shared memory for the stages.
struct PersistKernel {
  const void *fn;
  int threads;
  int smem;
};

// cross: the register-stream variant with crossover (the TMA variant has none).
static PersistKernel pick(int bf, const GenShape &sh, bool cross = false) {
  // (2, 2) is the shape sized for six CTAs per SM (40 registers a thread):
  // more warps to hide the row loads' latency, fewer loads in flight each
  if (sh.vec == 2 && sh.opb == 2)
    return {bf ? persist_fn<__nv_bfloat16, 2, 2, 6>(cross) : persist_fn<float, 2, 2, 6>(cross),
            kGenThreads, 0};
#define GSGP_P(V, O)                                                                      \
  if (sh.vec == V && sh.opb == O)                                                         \
    return {bf ? persist_fn<__nv_bfloat16, V, O>(cross) : persist_fn<float, V, O>(cross), \
            kGenThreads, 0};
  GSGP_P(1, 1) GSGP_P(1, 2) GSGP_P(1, 4) GSGP_P(1, 8) GSGP_P(1, 16) GSGP_P(2, 1) GSGP_P(2, 4)
  GSGP_P(2, 8) GSGP_P(2, 16)
#undef GSGP_P
#define GSGP_T(V)                                                                             \
  if (sh.vec == V && sh.opb == 0)                                                             \
    return bf ? PersistKernel{persist_tma_fn<__nv_bfloat16, V>(), kTmaThreads,                \
                              TmaCfg<__nv_bfloat16, V>::kSmem}                                \
              : PersistKernel{persist_tma_fn<float, V>(), kTmaThreads, TmaCfg<float, V>::kSmem};
  if (!cross) {
    GSGP_T(1) GSGP_T(2) GSGP_T(4)
  }
#undef GSGP_T
  return {nullptr, 0, 0};
}

bool persist_shape_supported(const GenShape &sh) {
  if (sh.opb == 0) return sh.vec == 1 || sh.vec == 2 || sh.vec == 4;
  return ((sh.vec == 1 || sh.vec == 2) && (sh.opb == 8 || sh.opb == 16)) ||
         ((sh.vec == 1 || sh.vec == 2) && (sh.opb == 1 || sh.opb == 2 || sh.opb == 4));
}

// Co-resident CTAs; for the register stream the smaller of the two variants
// (with and without crossover), should they differ.
int persist_max_grid(int sigma_bf16, const GenShape &sh) {
  const PersistKernel k = pick(sigma_bf16, sh);
  if (!k.fn) return 0;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
    return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (k.smem > 0 &&
      cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, k.threads, k.smem) !=
      cudaSuccess)
    return 0;
  if (sh.opb > 0) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick(sigma_bf16, sh, true).fn, k.threads,
                                                      k.smem) != cudaSuccess)
      return 0;
    per_sm = n < per_sm ? n : per_sm;
  }
  return per_sm * sms;
}

cudaError_t launch_persist(const GenParams &p, const PersistArgs &x, int sigma_bf16,
                           const GenShape &sh, int grid, cudaStream_t s) {
  const PersistKernel k = pick(sigma_bf16, sh, p.p_crossover > 0.0f);
  if (!k.fn || grid <= 0) return cudaErrorInvalidValue;
  if (k.smem > 0) {
    const cudaError_t e =
        cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem);
    if (e != cudaSuccess) return e;
  }
  GenParams pp = p;
  PersistArgs xx = x;
  void *args[] = {&pp, &xx};
  return cudaLaunchCooperativeKernel(k.fn, dim3((unsigned)grid), dim3((unsigned)k.threads), args,
                                     (size_t)k.smem, s);
}

}  // namespace gsgp
