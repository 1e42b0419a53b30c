// Batched persistent generation kernel: R independent GSGP runs, each with
// its own fitness cases, sizes, parameters, random trees and state, advance
// G generations together in one cooperative launch.  The paper runs one
// evolution at a time and repeats runs in a loop on the host; here the
// generation loop of Algorithm 1 is the same for every run and the work of
// all runs is one flat list per phase:
//
//   S  selection: the offspring of all runs, concatenated (run r owns the
//      global indices [m_off[r], m_off[r+1])), thread t of the grid takes
//      t, t + threads, ...  -- barrier --
//   M  mutation stream: the items of all runs, concatenated (an item = one
//      tile of 1024 * VEC cases for OPB offspring of one run, tile-major
//      within a run, so the CTAs resident at a time share a few sigma(R)
//      tiles of one run in L2); CTA b takes items b, b + grid, ...
//      -- barrier --
//   F1 fitness: one warp per offspring of all runs sums its chunk partials
//      in the fixed order and writes its RMSE.  -- barrier --
//   F2 survival with elitism: CTA b decides runs b, b + grid, ... from the
//      fitness tables and rewrites their slot-to-row maps, logs and
//      counters.  -- barrier --
//
// Every per-run value is computed by the same device code, in the same
// order, as the single-run kernels (select_offspring, stream_item,
// item_partials, warp_sum_partials, survive_population), so a run evolved in
// a batch is bit-identical to the same run evolved alone.
#include "gridsync.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "stream.cuh"

namespace gsgp {

// Advance r to the run holding global index x (offsets ascending; x only
// grows within a phase for a given thread or CTA).
__device__ __forceinline__ int advance_run(const int *off, int r, int x) {
  while (off[r + 1] <= x) ++r;
  return r;
}

template <typename SigT, int VEC, int OPB, bool CROSS>
__global__ void __launch_bounds__(kGenThreads, 4) batch_kernel(const __grid_constant__ BatchArgs a) {
  constexpr int NW = kGenThreads / 32;
  __shared__ ItemSums<VEC, OPB> s_sum[2];
  __shared__ int4 s_isel[2][OPB];   // draws of the current / next item (VEC = 1)
  __shared__ float s_ims[2][OPB];
  __shared__ int s_ok;

  GridSync *gs = a.gs;
  if (ld_relaxed_s32(&gs->err) != 0) return;   // an earlier launch failed
  const int R = a.R;
  const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int M = a.m_off[R], items = a.item_off[R];
  unsigned epoch = 0;

  for (int it = 0; it < a.G; ++it) {
    // ---------------- S: selection ----------------------------------------
    {
      int r = 0;
      for (int gi = b * kGenThreads + tid; gi < M; gi += nb * kGenThreads) {
        r = advance_run(a.m_off, r, gi);
        const GenParams &p = a.runs[r];
        select_offspring<CROSS>(p, gi - a.m_off[r], __ldcg(&p.state->gen), __ldcg(&p.state->parity));
      }
    }
    if (!grid_sync(gs, epoch, &s_ok)) return;

    // ---------------- M: mutation stream ----------------------------------
    // The CTA's items of one run form a segment: the run's parameters and
    // its item-to-(tile, offspring group) division are taken once per
    // segment, and the position then advances by nb items without a
    // division.  The next item's draws are fetched one item ahead: from the
    // advanced position within the segment, through a run lookup across it.
    if constexpr (VEC == 1) {
      // 1024-case tiles: each item's draws staged in shared memory one item
      // ahead, the row loads pipelined one offspring ahead
      int buf = 0, r = 0, rn = 0;
      auto stage_from = [&](const GenParams &q, int i0, int to) {
        const int i = i0 + tid;
        if (tid < OPB && i < q.m) {
          s_isel[to][tid] = __ldcg(q.sel + i);
          s_ims[to][tid] = __ldcg(q.sel_ms + i);
        }
      };
      auto stage = [&](int item, int to) {   // an item of another run
        rn = advance_run(a.item_off, rn, item);
        const GenParams &q = a.runs[rn];
        const int groups = (q.m + OPB - 1) / OPB;
        stage_from(q, ((item - a.item_off[rn]) % groups) * OPB, to);
      };
      if (b < items) stage(b, 0);
      __syncthreads();
      for (int item = b; item < items;) {
        r = advance_run(a.item_off, r, item);
        const GenParams &p = a.runs[r];
        const int groups = (p.m + OPB - 1) / OPB;
        const int seg_end = a.item_off[r + 1];
        const int step_t = nb / groups, step_g = nb - step_t * groups;
        const int local = item - a.item_off[r];
        int tile = local / groups;
        int grp = local - tile * groups;
        for (; item < seg_end; item += nb, buf ^= 1) {
          const int t = tile, i0 = grp * OPB;
          const int cnt = min(OPB, p.m - i0);
          tile += step_t;
          grp += step_g;
          if (grp >= groups) {
            grp -= groups;
            ++tile;
          }
          if (item + nb < seg_end)
            stage_from(p, grp * OPB, buf ^ 1);
          else if (item + nb < items)
            stage(item + nb, buf ^ 1);
          stream_item_pipe<SigT, OPB, CROSS>(p, t, cnt, s_isel[buf], s_ims[buf], s_sum[buf]);
          __syncthreads();   // one barrier per item; it also publishes the next item's draws
          item_partials<VEC, OPB>(p, t, i0, cnt, s_sum[buf]);
        }
      }
    } else {
      // the first draws of the next item are loaded one item ahead
      int buf = 0, r = 0, rn = 0;
      int4 sel_next = make_int4(0, 0, 0, 0);
      float ms_next = 0.f;
      auto prefetch = [&](int item) {   // an item of another run
        rn = advance_run(a.item_off, rn, item);
        const GenParams &q = a.runs[rn];
        const int groups = (q.m + OPB - 1) / OPB;
        const int i0 = ((item - a.item_off[rn]) % groups) * OPB;
        sel_next = __ldcg(q.sel + i0);
        ms_next = __ldcg(q.sel_ms + i0);
      };
      if (b < items) prefetch(b);
      for (int item = b; item < items;) {
        r = advance_run(a.item_off, r, item);
        const GenParams &p = a.runs[r];
        const int groups = (p.m + OPB - 1) / OPB;
        const int seg_end = a.item_off[r + 1];
        const int step_t = nb / groups, step_g = nb - step_t * groups;
        const int local = item - a.item_off[r];
        int tile = local / groups;
        int grp = local - tile * groups;
        for (; item < seg_end; item += nb, buf ^= 1) {
          const int t = tile, i0 = grp * OPB;
          const int cnt = min(OPB, p.m - i0);
          const int4 sel = sel_next;
          const float ms = ms_next;
          tile += step_t;
          grp += step_g;
          if (grp >= groups) {
            grp -= groups;
            ++tile;
          }
          if (item + nb < seg_end) {
            sel_next = __ldcg(p.sel + grp * OPB);
            ms_next = __ldcg(p.sel_ms + grp * OPB);
          } else if (item + nb < items) {
            prefetch(item + nb);
          }
          stream_item<SigT, VEC, OPB, CROSS>(p, t, i0, cnt, sel, ms, s_sum[buf]);
          __syncthreads();   // one barrier per item (s_sum is double-buffered)
          item_partials<VEC, OPB>(p, t, i0, cnt, s_sum[buf]);
        }
      }
    }
    if (!grid_sync(gs, epoch, &s_ok)) return;

    // ---------------- F1: offspring RMSE ----------------------------------
    {
      int r = 0;
      for (int gw = b * NW + warp; gw < M; gw += nb * NW) {
        r = advance_run(a.m_off, r, gw);
        const GenParams &p = a.runs[r];
        const int i = gw - a.m_off[r];
        const double2 *row = p.partial + (size_t)i * p.tiles;
        const double2 sse = VEC == 2 && p.tiles > 128 ? warp_sum_partials_long(row, p.tiles, lane)
                                                      : warp_sum_partials(row, p.tiles, lane);
        if (lane == 0) {
          const int par = __ldcg(&p.state->parity);
          p.fit[(size_t)(par ^ 1) * p.m + i] = rmse_from_sse(sse.x, p.n_train_all);
          p.fit_te[(size_t)(par ^ 1) * p.m + i] = rmse_from_sse(sse.y, p.n_test_all);
        }
      }
    }
    if (!grid_sync(gs, epoch, &s_ok)) return;

    // ---------------- F2: survival, one CTA per run -----------------------
    for (int r = b; r < R; r += nb) {
      const GenParams &p = a.runs[r];
      const int g = __ldcg(&p.state->gen), par = __ldcg(&p.state->parity);
      __syncthreads();   // every thread has read the counters before thread 0 advances them
      survive_population(p, g, par);
    }
    if (!grid_sync(gs, epoch, &s_ok)) return;
  }
}

template <typename SigT, int VEC, int OPB>
static const void *batch_fn(bool cross) {
  return cross ? reinterpret_cast<const void *>(&batch_kernel<SigT, VEC, OPB, true>)
               : reinterpret_cast<const void *>(&batch_kernel<SigT, VEC, OPB, false>);
}

// The crossover variant when any run of the launch has p_crossover > 0.
static const void *batch_pick(int sigma_bf16, const GenShape &sh, bool cross = false) {
#define GSGP_BATCH_CASE(V, O)                                                        \
  if (sh.vec == V && sh.opb == O)                                                    \
    return sigma_bf16 ? batch_fn<__nv_bfloat16, V, O>(cross) : batch_fn<float, V, O>(cross);
  GSGP_BATCH_CASE(1, 1)
  GSGP_BATCH_CASE(1, 2)
  GSGP_BATCH_CASE(1, 4)
  GSGP_BATCH_CASE(1, 8)
  GSGP_BATCH_CASE(2, 1)
  GSGP_BATCH_CASE(2, 2)
  GSGP_BATCH_CASE(2, 4)
#undef GSGP_BATCH_CASE
  return nullptr;
}

bool batch_shape_supported(const GenShape &sh) { return batch_pick(0, sh) != nullptr; }

// Co-resident CTAs of both variants (the smaller, should they differ).
int batch_max_grid(int sigma_bf16, const GenShape &sh) {
  if (!batch_pick(sigma_bf16, sh)) return 0;
  int dev = 0, coop = 0, sms = 0, per_sm = 1 << 30;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
    return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  for (const bool cross : {false, true}) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_pick(sigma_bf16, sh, cross),
                                                      kGenThreads, 0) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    per_sm = n < per_sm ? n : per_sm;
  }
  return per_sm * sms;
}

cudaError_t launch_batch(const BatchArgs &a, int sigma_bf16, const GenShape &sh, int grid,
                         cudaStream_t s) {
  if (a.R < 1 || a.R > kBatchRunsPerLaunch) return cudaErrorInvalidValue;
  bool cross = false;
  for (int r = 0; r < a.R; ++r) cross |= a.runs[r].p_crossover > 0.0f;
  const void *fn = batch_pick(sigma_bf16, sh, cross);
  if (!fn || grid <= 0) return cudaErrorInvalidValue;
  void *args[] = {const_cast<BatchArgs *>(&a)};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kGenThreads), args, 0, s);
}

}  // namespace gsgp
