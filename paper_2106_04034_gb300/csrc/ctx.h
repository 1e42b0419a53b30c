// Internal to the library: the run context behind the opaque gsgp_ctx of
// the C ABI, and the helpers that api.cu shares with batch_api.cu.
#pragma once

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "gsgp.h"
#include "kernels.cuh"

using namespace gsgp;

struct gsgp_ctx {
  gsgp_config cfg{};
  std::string err;
  int state = 0;   // 0 created, 1 loaded, 2 initialised
  int device = -1;
  cudaStream_t stream = nullptr;
  // stream-ordered pool of the context's own device allocations (without a
  // caller allocator): memory freed by one call stays mapped for the next
  cudaMemPool_t mem_pool = nullptr;
  cudaStream_t cap_stream = nullptr;

  // fitness cases
  int l = 0;
  int64_t n_tr = 0, n_te = 0, N = 0, n_pad = 0;
  float *X = nullptr;   // [l][n_pad]
  float *t = nullptr;   // [n_pad]

  // case sharding (gsgp_shard_configure): this context holds the problem's
  // cases [shard_case0, shard_case0 + N) of n_train_all + n_test_all
  bool sharded = false;
  int64_t shard_case0 = 0, n_train_all = 0, n_test_all = 0;
  int shard_pending = 0;   // 1: initial fitness, 2: a generation's survival awaits the exchange

  // run state
  int Kp = 0, Kr = 0;
  int tiles_interp = 0;   // 1024-case chunks of the whole problem: row stride of partial
  // generation loop: path 1 = persistent cooperative kernel, 2 = chained
  // select/stream/final launches; shape = (float4 chunks per thread,
  // offspring per CTA); grid = CTAs of the persistent kernel
  int path = 1;
  GenShape shape{1, 2};
  int grid = 0;
  int forced_path = 0;       // gsgp_set_evolve_shape: 0 = choose
  GenShape forced{0, 0};     // {0, 0} = autotune within the path
  bool shape_ready = false;
  GridSync *gs = nullptr;
  ulonglong2 *cta_min = nullptr, *cta_max = nullptr;
  // armed by gsgp_arm_barrier_fault for the next persistent launch only
  unsigned fault_spin_limit = 0;   // 0: not armed
  int cta_cap = 0;
  int *bk_perm = nullptr;    // state snapshot used while autotuning
  double *bk_fit = nullptr, *bk_fit_te = nullptr;
  DevState *bk_state = nullptr;
  int64_t layout_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int *P_genes = nullptr, *P_len = nullptr, *R_genes = nullptr, *R_len = nullptr;
  float *P_consts = nullptr, *R_consts = nullptr;
  // the programs the interpreter and the model evaluate: the live code of
  // linear genomes (own buffers), or the programs themselves (aliases)
  int *Pc_genes = nullptr, *Pc_len = nullptr, *Rc_genes = nullptr, *Rc_len = nullptr;
  float *Pc_consts = nullptr, *Rc_consts = nullptr;
  float *pool = nullptr;
  void *sigR = nullptr;
  int *perm = nullptr;
  double *fit = nullptr, *fit_te = nullptr;
  double2 *partial = nullptr;
  int4 *sel = nullptr;
  float *sel_ms = nullptr;
  DevState *dstate = nullptr;
  int4 *trace = nullptr;
  double2 *best_log = nullptr;
  int gcap = 0;
  int4 *lineage = nullptr;
  int lineage_cap = 0;
  int *lin_jump = nullptr;    // scratch of the segmented lineage walk
  int *lin_start = nullptr;
  int64_t lin_jump_cap = 0;
  int lin_start_cap = 0;
  int *d_anc = nullptr;
  int *d_stack = nullptr;     // [2] deepest interpreter stack of P and R (linear genomes)
  int64_t eval_genes[2] = {0, 0};   // genes evaluated per case over P and R
  unsigned *d_flag = nullptr;
  int gen = 0;

  // CUDA graph of `graph_u` generations, replayed by gsgp_evolve; when built
  // for timing it records an event before and after every stream launch
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_u = 0;
  bool graph_timed = false;
  bool graph_dirty = true;
  std::vector<cudaGraphNode_t> ev_nodes;   // [2 * graph_u] start/stop record nodes
  std::vector<cudaEvent_t> ev_marks;       // events the nodes were captured with

  // stream-kernel timing
  bool timing = false;
  std::vector<cudaEvent_t> ev0, ev1;
  cudaEvent_t ev_init[4] = {nullptr, nullptr, nullptr, nullptr};   // around the interpreter
  bool init_timed = false;                                          // launches of the last init
  int ev_used = 0;

  // rebuilt best model (valid while model_gen == gen)
  int model_gen = -1;
  int best_slot = 0, ancestor = 0;
  double best_tr = 0.0, best_te = 0.0;
  std::vector<int4> h_lineage;
  std::vector<double> coef;
  int *d_terms = nullptr;
  double *d_coef = nullptr;
  int terms_cap = 0;
  int n_terms = 0;

  int64_t launches = 0;
  int64_t dev_bytes = 0;
  std::unordered_map<void *, size_t> allocs;
};

// Errors: set the context's message and return the status.
gsgp_status fail(gsgp_ctx *c, gsgp_status st, const char *fmt, ...);
gsgp_status cuda_fail(gsgp_ctx *c, cudaError_t e, const char *what, int line);

#define CK(call)                                                      \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call, __LINE__);  \
  } while (0)

#define LAUNCH(n, call)      \
  do {                       \
    CK(call);                \
    c->launches += (n);      \
  } while (0)

#define TRY(expr)                                  \
  do {                                             \
    gsgp_status s_ = (expr);                       \
    if (s_ != GSGP_OK) return s_;                  \
  } while (0)

#define API_GUARD(c)                                                                   \
  if (!(c)) return GSGP_E_INVALID;                                                     \
  (c)->err.clear();                                                                    \
  try {
#define API_END(c)                                                                     \
  }                                                                                    \
  catch (const std::bad_alloc &) {                                                     \
    return fail((c), GSGP_E_OOM, "host allocation failed");                            \
  }                                                                                    \
  catch (...) {                                                                        \
    return fail((c), GSGP_E_INVALID, "unexpected host exception");                     \
  }


// Shared run helpers (api.cu).
gsgp_status use_device(gsgp_ctx *c);
GenParams gen_params(gsgp_ctx *c);
// Grow the trace and best-of-generation log to hold `need` generations.
gsgp_status ensure_trace(gsgp_ctx *c, int need);
// Save (save = true) or restore the per-generation state of the run
// (slot-to-row map, fitness, counters) on stream s; ensure_backup allocates
// the backup buffers (on the run's stream) ahead of the first snapshot.
gsgp_status ensure_backup(gsgp_ctx *c);
gsgp_status snapshot(gsgp_ctx *c, bool save, cudaStream_t s);
// GSGP_E_TIMEOUT when a bounded wait of the generation kernel gave up
// (synchronises the run's stream).
gsgp_status check_device_error(gsgp_ctx *c);
