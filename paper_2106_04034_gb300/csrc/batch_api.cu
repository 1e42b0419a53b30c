// C ABI of batched runs: several initialised run contexts advanced together
// by the batched persistent kernel (k_batch.cu), one cooperative launch per
// up to 64 generations and block of up to kBatchRunsPerLaunch runs, replayed
// from a CUDA graph.  The runs keep their own state in device memory; the
// batch owns only the launch arguments (the runs' generation parameters and
// work-list offsets) and its barrier words.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"

struct gsgp_batch {
  std::vector<gsgp_ctx *> runs;
  std::string err;
  int device = -1;
  cudaStream_t stream = nullptr;       // runs[0]'s stream: all batch work
  cudaStream_t cap_stream = nullptr;   // private stream for graph capture
  int bf = 0;                          // sigma(R) stored as bf16
  GenShape forced{0, 0};               // {0, 0}: autotune
  GenShape shape{0, 0};
  bool shape_ready = false;
  int64_t items = 0, offspring = 0, updates = 0;

  // launch arguments, one block of at most kBatchRunsPerLaunch runs per
  // launch (G is set per launch), and the barrier words they share
  std::vector<BatchArgs> groups;
  std::vector<int> group_grid;
  GridSync *gs = nullptr;

  // CUDA graph of kBatchGenerations generations (one launch per group),
  // valid while the groups' arguments equal the captured ones
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<BatchArgs> graph_groups;
  std::vector<int> graph_grid;
  GenShape graph_shape{0, 0};
  bool graph_unsupported = false;   // capture of the cooperative launch failed once

  cudaEvent_t ev_join = nullptr;
  bool timing = false;
  std::vector<cudaEvent_t> ev0, ev1;
  int ev_used = 0;
  int64_t launches = 0;
};

namespace {

constexpr int kBatchGenerations = 64;   // generations per launch
constexpr int kMaxBatchRuns = 1024;     // runs per batch (public limit)

gsgp_status bfail(gsgp_batch *b, gsgp_status st, const char *fmt, ...) {
  if (b) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    b->err = buf;
  }
  return st;
}

gsgp_status bcuda(gsgp_batch *b, cudaError_t e, const char *what, int line) {
  cudaGetLastError();
  return bfail(b, e == cudaErrorMemoryAllocation ? GSGP_E_OOM : GSGP_E_CUDA,
               "%s (batch_api.cu:%d): %s", what, line, cudaGetErrorString(e));
}

// A run-level helper failed: its message moves to the batch.
gsgp_status brun(gsgp_batch *b, int k, gsgp_status st) {
  return bfail(b, st, "run %d: %s", k, b->runs[(size_t)k]->err.c_str());
}

#define BCK(call)                                                    \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call, __LINE__);     \
  } while (0)

#define BTRY(expr)                                                   \
  do {                                                               \
    gsgp_status s_ = (expr);                                         \
    if (s_ != GSGP_OK) return s_;                                    \
  } while (0)

void free_graph(gsgp_batch *b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->graph_groups.clear();
  b->graph_grid.clear();
}

// GenParams has no padding, so launch arguments built from zeroed storage
// compare equal byte for byte exactly when their values are equal.
static_assert(sizeof(GenParams) == 12 * sizeof(void *) + 8 + 8 * 4 + 8 + 8 + 8 + 8,
              "GenParams padding");

int64_t run_items(const gsgp_ctx *c, const GenShape &sh) {
  const int64_t tiles = (c->n_pad + 1024 * sh.vec - 1) / (1024 * sh.vec);
  return tiles * ((c->cfg.pop_size + sh.opb - 1) / sh.opb);
}

// Every run initialised, on the batch's device; grow each run's trace for
// `generations` more and refresh the work-list sizes.
gsgp_status check_runs(gsgp_batch *b, int generations) {
  int64_t M = 0, upd = 0;
  for (size_t k = 0; k < b->runs.size(); ++k) {
    gsgp_ctx *c = b->runs[k];
    if (c->state != 2) return bfail(b, GSGP_E_STATE, "run %d is not initialised", (int)k);
    if (c->device != b->device) return bfail(b, GSGP_E_INVALID, "run %d changed device", (int)k);
    if ((int64_t)c->gen + generations > 0x7fffffff)
      return bfail(b, GSGP_E_INVALID, "run %d: too many generations", (int)k);
    if (generations > 0) {
      const gsgp_status st = ensure_trace(c, c->gen + generations);
      if (st != GSGP_OK) return brun(b, (int)k, st);
    }
    M += c->cfg.pop_size;
    upd += (int64_t)c->cfg.pop_size * c->N;
  }
  if (M >= ((int64_t)1 << 31)) return bfail(b, GSGP_E_INVALID, "too many offspring in the batch");
  b->offspring = M;
  b->updates = upd;
  return GSGP_OK;
}

// Balanced grid of one launch: at most the co-resident count, and no more
// CTAs than needed to give every CTA the same number of stream items.
int balanced_grid(int max_grid, int64_t items) {
  if (max_grid <= 0 || items <= 0) return 0;
  const int64_t rounds = (items + max_grid - 1) / max_grid;
  const int64_t grid = (items + rounds - 1) / rounds;
  return (int)(grid < max_grid ? grid : max_grid);
}

// Launch arguments of shape sh: the runs in blocks of kBatchRunsPerLaunch,
// each with its offsets and grid (G is set per launch).
gsgp_status build_groups(gsgp_batch *b, const GenShape &sh, std::vector<BatchArgs> &groups,
                         std::vector<int> &grids, int64_t *items_out) {
  const int R = (int)b->runs.size();
  const int max_grid = batch_max_grid(b->bf, sh);
  if (max_grid <= 0)
    return bfail(b, GSGP_E_CUDA, "cooperative launch of the batched kernel is not available");
  const int ng = (R + kBatchRunsPerLaunch - 1) / kBatchRunsPerLaunch;
  groups.resize((size_t)ng);
  grids.assign((size_t)ng, 0);
  int64_t total = 0;
  for (int q = 0; q < ng; ++q) {
    BatchArgs &a = groups[(size_t)q];
    memset(&a, 0, sizeof a);
    const int r0 = q * kBatchRunsPerLaunch;
    const int n = R - r0 < kBatchRunsPerLaunch ? R - r0 : kBatchRunsPerLaunch;
    int64_t m_acc = 0, it_acc = 0;
    for (int k = 0; k < n; ++k) {
      gsgp_ctx *c = b->runs[(size_t)(r0 + k)];
      a.runs[k] = gen_params(c);
      a.m_off[k] = (int)m_acc;
      a.item_off[k] = (int)it_acc;
      m_acc += c->cfg.pop_size;
      it_acc += run_items(c, sh);
    }
    if (it_acc >= ((int64_t)1 << 31))
      return bfail(b, GSGP_E_INVALID, "too many stream items in one launch of the batch");
    a.m_off[n] = (int)m_acc;
    a.item_off[n] = (int)it_acc;
    a.gs = b->gs;
    a.R = n;
    a.G = 0;
    grids[(size_t)q] = balanced_grid(max_grid, it_acc);
    total += it_acc;
  }
  *items_out = total;
  return GSGP_OK;
}

// G generations of every run: one launch per block of runs, each after
// zeroing the barrier counter.
gsgp_status launch_all(gsgp_batch *b, const GenShape &sh, std::vector<BatchArgs> &groups,
                       const std::vector<int> &grids, int G, cudaStream_t s) {
  for (size_t q = 0; q < groups.size(); ++q) {
    groups[q].G = G;
    BCK(cudaMemsetAsync(&b->gs->count, 0, sizeof(GridSync) - offsetof(GridSync, count), s));
    BCK(launch_batch(groups[q], b->bf, sh, grids[q], s));
    b->launches += 1;
  }
  return GSGP_OK;
}

bool same_groups(const std::vector<BatchArgs> &x, const std::vector<BatchArgs> &y) {
  if (x.size() != y.size()) return false;
  for (size_t q = 0; q < x.size(); ++q) {
    BatchArgs u = x[q], v = y[q];
    u.G = v.G = 0;
    if (memcmp(&u, &v, sizeof u) != 0) return false;
  }
  return true;
}

// Capture the launches of kBatchGenerations generations; a device or driver
// that cannot capture a cooperative launch leaves the batch on direct
// launches (graph_unsupported).
gsgp_status build_graph(gsgp_batch *b) {
  free_graph(b);
  if (!b->cap_stream) BCK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int64_t launches = b->launches;
  gsgp_status st = launch_all(b, b->shape, b->groups, b->group_grid, kBatchGenerations,
                              b->cap_stream);
  b->launches = launches;   // captured, not launched
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(b->cap_stream, &graph);
  cudaError_t ie = cudaErrorUnknown;
  if (st == GSGP_OK && ee == cudaSuccess && graph) ie = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGetLastError();
  b->err.clear();
  if (ie != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    b->gexec = nullptr;
    b->graph_unsupported = true;
    return GSGP_OK;
  }
  b->graph = graph;
  b->graph_groups = b->groups;
  b->graph_grid = b->group_grid;
  b->graph_shape = b->shape;
  return GSGP_OK;
}

const GenShape kBatchShapes[] = {{1, 1}, {1, 2}, {1, 4}, {1, 8}, {2, 1}, {2, 2}, {2, 4}};

// One generation of the whole batch in shape sh, timed, with every run's
// state restored afterwards (the trial rewrites only what the real
// generation rewrites identically: free rows, draws, partials, this
// generation's trace and log entries).
gsgp_status time_shape(gsgp_batch *b, const GenShape &sh, float *out_ms) {
  std::vector<BatchArgs> groups;
  std::vector<int> grids;
  int64_t items = 0;
  BTRY(build_groups(b, sh, groups, grids, &items));
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  gsgp_status st = GSGP_OK;
  float best = 1e30f;
  for (size_t k = 0; k < b->runs.size() && st == GSGP_OK; ++k) {
    st = snapshot(b->runs[k], true, b->stream);
    if (st != GSGP_OK) st = brun(b, (int)k, st);
  }
  for (int rep = 0; rep < 3 && st == GSGP_OK; ++rep) {
    cudaError_t e = cudaEventRecord(e0, b->stream);
    if (e == cudaSuccess) st = launch_all(b, sh, groups, grids, 1, b->stream);
    if (st == GSGP_OK && e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    for (size_t k = 0; k < b->runs.size() && st == GSGP_OK && e == cudaSuccess; ++k) {
      st = snapshot(b->runs[k], false, b->stream);
      if (st != GSGP_OK) st = brun(b, (int)k, st);
    }
    if (st == GSGP_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (st == GSGP_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (st == GSGP_OK && e != cudaSuccess) st = bcuda(b, e, "batch autotune", __LINE__);
    if (rep > 0 && ms > 0.f && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *out_ms = best;
  return st;
}

gsgp_status check_error(gsgp_batch *b) {
  int err = 0;
  BCK(cudaMemcpyAsync(&err, &b->gs->err, sizeof err, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (err)
    return bfail(b, GSGP_E_TIMEOUT,
                 "a grid barrier of the batched generation kernel gave up waiting; re-run "
                 "gsgp_init on every run of the batch");
  return GSGP_OK;
}

gsgp_status choose_shape(gsgp_batch *b) {
  if (b->shape_ready) return GSGP_OK;
  if (b->forced.vec) {
    b->shape = b->forced;
  } else {
    for (size_t k = 0; k < b->runs.size(); ++k) {
      const gsgp_status st = ensure_backup(b->runs[k]);
      if (st != GSGP_OK) return brun(b, (int)k, st);
    }
    // the backups were allocated on the runs' streams
    for (gsgp_ctx *c : b->runs) {
      BCK(cudaEventRecord(b->ev_join, c->stream));
      BCK(cudaStreamWaitEvent(b->stream, b->ev_join, 0));
    }
    float best_ms = 1e30f;
    GenShape best = kBatchShapes[0];
    for (const GenShape &sh : kBatchShapes) {
      float ms = 1e30f;
      BTRY(time_shape(b, sh, &ms));
      if (ms < best_ms * 0.99f) {   // near-ties keep the earlier shape
        best_ms = ms;
        best = sh;
      }
    }
    BTRY(check_error(b));
    b->shape = best;
  }
  b->shape_ready = true;
  return GSGP_OK;
}

gsgp_status ensure_events(gsgp_batch *b, int need) {
  while ((int)b->ev0.size() < need) {
    cudaEvent_t x, y;
    BCK(cudaEventCreate(&x));
    BCK(cudaEventCreate(&y));
    b->ev0.push_back(x);
    b->ev1.push_back(y);
  }
  return GSGP_OK;
}

}  // namespace

#define BATCH_GUARD(b)                                                       \
  if (!(b)) return GSGP_E_INVALID;                                           \
  (b)->err.clear();                                                          \
  try {
#define BATCH_END(b)                                                         \
  }                                                                          \
  catch (const std::bad_alloc &) {                                           \
    return bfail((b), GSGP_E_OOM, "host allocation failed");                 \
  }                                                                          \
  catch (...) {                                                              \
    return bfail((b), GSGP_E_INVALID, "unexpected host exception");          \
  }

extern "C" gsgp_status gsgp_batch_create(gsgp_ctx *const *runs, int32_t count, gsgp_batch **out) {
  if (!out) return GSGP_E_INVALID;
  *out = nullptr;
  if (!runs || count < 1 || count > kMaxBatchRuns) return GSGP_E_INVALID;
  for (int32_t k = 0; k < count; ++k) {
    if (!runs[k]) return GSGP_E_INVALID;
    for (int32_t q = 0; q < k; ++q)
      if (runs[q] == runs[k]) return GSGP_E_INVALID;   // a run appears once
  }
  for (int32_t k = 0; k < count; ++k)
    if (runs[k]->state != 2 || runs[k]->sharded) return GSGP_E_STATE;
  const int dev = runs[0]->device;
  const int32_t dtype = runs[0]->cfg.sigma_dtype;
  for (int32_t k = 1; k < count; ++k)
    if (runs[k]->device != dev || runs[k]->cfg.sigma_dtype != dtype) return GSGP_E_INVALID;
  gsgp_batch *b = new (std::nothrow) gsgp_batch();
  if (!b) return GSGP_E_OOM;
  try {
    b->runs.assign(runs, runs + count);
  } catch (...) {
    delete b;
    return GSGP_E_OOM;
  }
  b->device = dev;
  b->stream = runs[0]->stream;
  b->bf = dtype == GSGP_SIGMA_BF16;
  cudaError_t e = cudaSetDevice(dev);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->gs), sizeof(GridSync));
  if (e == cudaSuccess) e = cudaMemset(b->gs, 0, sizeof(GridSync));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    gsgp_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? GSGP_E_OOM : GSGP_E_CUDA;
  }
  *out = b;
  return GSGP_OK;
}

extern "C" gsgp_status gsgp_batch_set_shape(gsgp_batch *b, int32_t vec, int32_t opb) {
  BATCH_GUARD(b)
  const bool autotune = vec == 0 && opb == 0;
  if (!autotune && !batch_shape_supported(GenShape{vec, opb}))
    return bfail(b, GSGP_E_INVALID,
                 "batch shape must have vec in {1,2} and opb in {1,2,4}, or vec 1 and opb 8");
  b->forced = autotune ? GenShape{0, 0} : GenShape{vec, opb};
  b->shape_ready = false;
  return GSGP_OK;
  BATCH_END(b)
}

extern "C" gsgp_status gsgp_batch_evolve(gsgp_batch *b, int32_t generations,
                                         double *best_train, double *best_test) {
  BATCH_GUARD(b)
  if (generations < 0) return bfail(b, GSGP_E_INVALID, "generations must be >= 0");
  BCK(cudaSetDevice(b->device));
  BTRY(check_runs(b, generations));
  if (generations == 0) return GSGP_OK;
  const int R = (int)b->runs.size();
  std::vector<int> g0((size_t)R);
  for (int k = 0; k < R; ++k) g0[(size_t)k] = b->runs[(size_t)k]->gen;
  // the batch's work follows everything already queued on the runs' streams
  for (gsgp_ctx *c : b->runs) {
    if (c->stream == b->stream) continue;
    BCK(cudaEventRecord(b->ev_join, c->stream));
    BCK(cudaStreamWaitEvent(b->stream, b->ev_join, 0));
  }
  BTRY(choose_shape(b));
  // the runs' parameters and sizes are read afresh: a run may have been
  // re-loaded, re-initialised or grown its trace since the last call
  BTRY(build_groups(b, b->shape, b->groups, b->group_grid, &b->items));
  if (b->timing) BTRY(ensure_events(b, b->ev_used + (generations + kBatchGenerations - 1) /
                                                       kBatchGenerations));
  int left = generations;
  while (left > 0) {
    const int G = left < kBatchGenerations ? left : kBatchGenerations;
    if (b->timing) BCK(cudaEventRecord(b->ev0[(size_t)b->ev_used], b->stream));
    if (G == kBatchGenerations && !b->graph_unsupported &&
        (!b->gexec || b->graph_shape.vec != b->shape.vec || b->graph_shape.opb != b->shape.opb ||
         b->graph_grid != b->group_grid || !same_groups(b->graph_groups, b->groups)))
      BTRY(build_graph(b));
    if (G == kBatchGenerations && b->gexec) {
      BCK(cudaGraphLaunch(b->gexec, b->stream));
      b->launches += (int64_t)b->groups.size();
    } else {
      BTRY(launch_all(b, b->shape, b->groups, b->group_grid, G, b->stream));
    }
    if (b->timing) {
      BCK(cudaEventRecord(b->ev1[(size_t)b->ev_used], b->stream));
      ++b->ev_used;
    }
    left -= G;
  }
  for (gsgp_ctx *c : b->runs) {
    c->gen += generations;
    c->model_gen = -1;
  }
  // later work on the runs' streams follows the batch
  BCK(cudaEventRecord(b->ev_join, b->stream));
  for (gsgp_ctx *c : b->runs)
    if (c->stream != b->stream) BCK(cudaStreamWaitEvent(c->stream, b->ev_join, 0));
  if (best_train || best_test) {
    std::vector<double2> h((size_t)generations);
    for (int k = 0; k < R; ++k) {
      gsgp_ctx *c = b->runs[(size_t)k];
      BCK(cudaMemcpyAsync(h.data(), c->best_log + g0[(size_t)k],
                          sizeof(double2) * (size_t)generations, cudaMemcpyDeviceToHost,
                          b->stream));
      BTRY(check_error(b));   // synchronises the batch stream
      for (int q = 0; q < generations; ++q) {
        if (best_train) best_train[(size_t)k * generations + q] = h[(size_t)q].x;
        if (best_test) best_test[(size_t)k * generations + q] = h[(size_t)q].y;
      }
    }
  }
  return GSGP_OK;
  BATCH_END(b)
}

extern "C" gsgp_status gsgp_batch_set_kernel_timing(gsgp_batch *b, int32_t enabled) {
  BATCH_GUARD(b)
  b->timing = enabled != 0;
  return GSGP_OK;
  BATCH_END(b)
}

extern "C" gsgp_status gsgp_batch_kernel_times(gsgp_batch *b, float *ms, int32_t cap,
                                               int32_t *n_out) {
  BATCH_GUARD(b)
  if (cap < 0 || (cap > 0 && !ms)) return bfail(b, GSGP_E_INVALID, "bad output buffer");
  BCK(cudaSetDevice(b->device));
  BCK(cudaStreamSynchronize(b->stream));
  BTRY(check_error(b));
  const int n = b->ev_used;
  const int k0 = n > cap ? n - cap : 0;
  for (int k = k0; k < n; ++k) {
    float t = 0.f;
    BCK(cudaEventElapsedTime(&t, b->ev0[(size_t)k], b->ev1[(size_t)k]));
    ms[k - k0] = t;
  }
  if (n_out) *n_out = n - k0;
  b->ev_used = 0;
  return GSGP_OK;
  BATCH_END(b)
}

extern "C" gsgp_status gsgp_batch_get_info(gsgp_batch *b, gsgp_batch_info *out) {
  BATCH_GUARD(b)
  if (!out || out->struct_size != sizeof(gsgp_batch_info))
    return bfail(b, GSGP_E_INVALID, "out must be a gsgp_batch_info with struct_size set");
  int64_t M = 0, upd = 0;
  for (gsgp_ctx *c : b->runs) {
    M += c->cfg.pop_size;
    upd += (int64_t)c->cfg.pop_size * c->N;
  }
  out->runs = (int32_t)b->runs.size();
  out->tile_cases = b->shape_ready ? 1024 * b->shape.vec : 0;
  out->offspring_per_cta = b->shape_ready ? b->shape.opb : 0;
  int grid = 0;
  for (int g : b->group_grid) grid = g > grid ? g : grid;
  out->grid = b->shape_ready ? grid : 0;
  out->generations_per_launch = kBatchGenerations;
  out->graph = b->gexec != nullptr;
  out->offspring = M;
  out->updates_per_generation = upd;
  out->items_per_generation = b->shape_ready ? b->items : 0;
  out->kernel_launches = b->launches;
  return GSGP_OK;
  BATCH_END(b)
}

extern "C" const char *gsgp_batch_last_error(const gsgp_batch *b) {
  return b ? b->err.c_str() : "";
}

extern "C" void gsgp_batch_destroy(gsgp_batch *b) {
  if (!b) return;
  if (b->device >= 0) {
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    free_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (cudaEvent_t e : b->ev0) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev1) cudaEventDestroy(e);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->gs) cudaFree(b->gs);
    cudaGetLastError();
  }
  delete b;
}
