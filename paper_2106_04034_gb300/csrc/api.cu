// C ABI of the GSGP library: context, state machine, device memory, stream
// ordering, CUDA-graph replay of the generation loop and host-side model
// reconstruction.  Every step of the method runs in the kernels of
// k_init.cu, k_generation.cu and k_predict.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "ctx.h"

using namespace gsgp;

// ---------------------------------------------------------------- errors --
gsgp_status fail(gsgp_ctx *c, gsgp_status st, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return st;
}

gsgp_status cuda_fail(gsgp_ctx *c, cudaError_t e, const char *what, int line) {
  cudaGetLastError();
  return fail(c, e == cudaErrorMemoryAllocation ? GSGP_E_OOM : GSGP_E_CUDA, "%s (api.cu:%d): %s",
              what, line, cudaGetErrorString(e));
}

// ---------------------------------------------------------------- memory --
// Without a caller allocator the context allocates stream-ordered from a
// pool of its own whose release threshold keeps freed memory: the staging
// buffers of a load or a prediction and the temporaries of an init are
// freed at the end of each call, and a pool that returned them to the
// driver at every synchronisation (the default pool's behaviour) would map
// fresh physical memory for each call -- measured at 27-33 ms instead of
// 5 ms for the large workload's 773 MB load once the GPU's memory had been
// used by other processes.  The pool is destroyed with the context.
static gsgp_status context_pool(gsgp_ctx *c) {
  if (c->mem_pool) return GSGP_OK;
  if (c->device < 0) CK(cudaGetDevice(&c->device));
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = c->device;
  CK(cudaMemPoolCreate(&c->mem_pool, &props));
  uint64_t keep = ~(uint64_t)0;
  CK(cudaMemPoolSetAttribute(c->mem_pool, cudaMemPoolAttrReleaseThreshold, &keep));
  return GSGP_OK;
}

static gsgp_status dalloc(gsgp_ctx *c, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (c->cfg.alloc) {
    *p = c->cfg.alloc(c->cfg.alloc_user, bytes, c->stream);
    if (!*p) return fail(c, GSGP_E_OOM, "device allocator returned NULL for %zu bytes", bytes);
  } else {
    TRY(context_pool(c));
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, c->mem_pool, c->stream);
    if (e != cudaSuccess) {
      *p = nullptr;
      cudaGetLastError();
      return fail(c, e == cudaErrorMemoryAllocation ? GSGP_E_OOM : GSGP_E_CUDA,
                  "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
  }
  c->allocs[*p] = bytes;
  c->dev_bytes += (int64_t)bytes;
  return GSGP_OK;
}

template <typename T>
static gsgp_status dalloc_n(gsgp_ctx *c, T **p, size_t count) {
  void *v = nullptr;
  gsgp_status s = dalloc(c, &v, count * sizeof(T));
  *p = static_cast<T *>(v);
  return s;
}

template <typename T>
static void dfree(gsgp_ctx *c, T *&p) {
  if (!p) return;
  void *v = (void *)p;
  auto it = c->allocs.find(v);
  if (it != c->allocs.end()) {
    c->dev_bytes -= (int64_t)it->second;
    c->allocs.erase(it);
  }
  if (c->cfg.alloc)
    c->cfg.free(c->cfg.alloc_user, v, c->stream);
  else
    cudaFreeAsync(v, c->stream);
  p = nullptr;
}

static void free_run_buffers(gsgp_ctx *c) {
  dfree(c, c->P_genes);
  dfree(c, c->P_consts);
  dfree(c, c->P_len);
  dfree(c, c->R_genes);
  dfree(c, c->R_consts);
  dfree(c, c->R_len);
  if (c->Pc_genes) {   // owned only for linear genomes; otherwise aliases
    dfree(c, c->Pc_genes);
    dfree(c, c->Pc_consts);
    dfree(c, c->Pc_len);
    dfree(c, c->Rc_genes);
    dfree(c, c->Rc_consts);
    dfree(c, c->Rc_len);
  }
  dfree(c, c->pool);
  dfree(c, c->sigR);
  dfree(c, c->perm);
  dfree(c, c->fit);
  dfree(c, c->fit_te);
  dfree(c, c->partial);
  dfree(c, c->sel);
  dfree(c, c->sel_ms);
  dfree(c, c->dstate);
  dfree(c, c->d_stack);
  dfree(c, c->gs);
  dfree(c, c->cta_min);
  dfree(c, c->cta_max);
  dfree(c, c->bk_perm);
  dfree(c, c->bk_fit);
  dfree(c, c->bk_fit_te);
  dfree(c, c->bk_state);
  c->cta_cap = 0;
  dfree(c, c->trace);
  dfree(c, c->best_log);
  dfree(c, c->lineage);
  dfree(c, c->lin_jump);
  dfree(c, c->lin_start);
  c->lin_jump_cap = 0;
  c->lin_start_cap = 0;
  dfree(c, c->d_anc);
  dfree(c, c->d_terms);
  dfree(c, c->d_coef);
  c->gcap = 0;
  c->lineage_cap = 0;
  c->terms_cap = 0;
  memset(c->layout_key, 0, sizeof c->layout_key);
  c->graph_dirty = true;
}

static void free_graph(gsgp_ctx *c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
  c->graph_u = 0;
  c->ev_nodes.clear();
}

// ---------------------------------------------------------------- config --
extern "C" void gsgp_config_default(gsgp_config *cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof *cfg);
  cfg->struct_size = sizeof(gsgp_config);
  cfg->seed = 1;
  cfg->run = 0;
  cfg->pop_size = 1024;
  cfg->n_random_trees = 1024;
  cfg->pop_min_depth = 2;
  cfg->pop_max_depth = 6;
  cfg->rt_min_depth = 2;
  cfg->rt_max_depth = 6;
  cfg->const_lo = -1.0f;
  cfg->const_hi = 1.0f;
  cfg->p_grow_function = 0.5f;
  cfg->p_feature_given_terminal = (float)(0.14 / 0.18);   /* 7/9 rounded once */
  cfg->protect_eps = 1e-3f;
  cfg->ms = 0.1f;
  cfg->ms_mode = 0;
  cfg->tournament_size = 4;
  cfg->elitism = 1;
  cfg->sigma_dtype = GSGP_SIGMA_F32;
  cfg->init_mode = GSGP_INIT_RHH;
  cfg->max_genes = 127;
  cfg->p_crossover = 0.0f;
}

static bool prob_ok(float p) { return std::isfinite(p) && p >= 0.0f && p <= 1.0f; }

static const char *check_config(const gsgp_config *cfg) {
  if (cfg->struct_size != sizeof(gsgp_config)) return "struct_size does not match this library";
  if (cfg->pop_size < 2 || cfg->pop_size > 65536) return "pop_size must be in [2, 65536]";
  if (cfg->n_random_trees < 1 || cfg->n_random_trees > 65536)
    return "n_random_trees must be in [1, 65536]";
  if (cfg->pop_min_depth < 0 || cfg->pop_max_depth > kMaxDepth ||
      cfg->pop_min_depth > cfg->pop_max_depth)
    return "population depths must satisfy 0 <= min <= max <= 10";
  if (cfg->rt_min_depth < 0 || cfg->rt_max_depth > kMaxDepth ||
      cfg->rt_min_depth > cfg->rt_max_depth)
    return "random-tree depths must satisfy 0 <= min <= max <= 10";
  if (!std::isfinite(cfg->const_lo) || !std::isfinite(cfg->const_hi) ||
      cfg->const_lo > cfg->const_hi)
    return "constant range must be finite with lo <= hi";
  if (!prob_ok(cfg->p_grow_function) || !prob_ok(cfg->p_feature_given_terminal) ||
      !prob_ok(cfg->p_crossover))
    return "probabilities must be in [0, 1]";
  if (!std::isfinite(cfg->protect_eps) || cfg->protect_eps < 0.0f)
    return "protect_eps must be finite and >= 0";
  if (!std::isfinite(cfg->ms)) return "ms must be finite";
  if (cfg->ms_mode != 0 && cfg->ms_mode != 1) return "ms_mode must be 0 or 1";
  if (cfg->tournament_size < 0 || cfg->tournament_size > 64)
    return "tournament_size must be in [0, 64]";
  if (cfg->elitism != 0 && cfg->elitism != 1) return "elitism must be 0 or 1";
  if (cfg->sigma_dtype != GSGP_SIGMA_F32 && cfg->sigma_dtype != GSGP_SIGMA_BF16)
    return "sigma_dtype must be GSGP_SIGMA_F32 or GSGP_SIGMA_BF16";
  if ((cfg->alloc == nullptr) != (cfg->free == nullptr))
    return "alloc and free must be given together";
  if (cfg->init_mode != GSGP_INIT_RHH && cfg->init_mode != GSGP_INIT_LINEAR)
    return "init_mode must be GSGP_INIT_RHH or GSGP_INIT_LINEAR";
  if (cfg->init_mode == GSGP_INIT_LINEAR &&
      (cfg->max_genes < 1 || cfg->max_genes > kMaxGenomeGenes))
    return "max_genes must be in [1, 4095] for linear genomes";
  return nullptr;
}

extern "C" gsgp_status gsgp_create(const gsgp_config *cfg, gsgp_ctx **out) {
  if (!out) return GSGP_E_INVALID;
  *out = nullptr;
  if (!cfg) return GSGP_E_INVALID;
  if (check_config(cfg)) return GSGP_E_INVALID;
  gsgp_ctx *c = new (std::nothrow) gsgp_ctx();
  if (!c) return GSGP_E_OOM;
  c->cfg = *cfg;
  c->stream = static_cast<cudaStream_t>(cfg->stream);
  *out = c;
  return GSGP_OK;
}

// Same check with a message for the caller that kept a context.
extern "C" const char *gsgp_config_error(const gsgp_config *cfg) {
  if (!cfg) return "NULL config";
  const char *e = check_config(cfg);
  return e ? e : "";
}

extern "C" const char *gsgp_last_error(const gsgp_ctx *c) { return c ? c->err.c_str() : ""; }

gsgp_status use_device(gsgp_ctx *c) {
  if (c->device < 0) CK(cudaGetDevice(&c->device));
  CK(cudaSetDevice(c->device));
  return GSGP_OK;
}

// Host input of `bytes` bytes to device memory on the context's stream.
// Page-locked (pinned or registered) host memory that is 16-byte aligned is
// read by a kernel through its device-mapped address (launch_host_read:
// no copy-engine stall after long kernels); any other host memory is copied
// with cudaMemcpyAsync.
static gsgp_status stage_h2d(gsgp_ctx *c, void *dst, const void *src, size_t bytes) {
  if (bytes == 0) return GSGP_OK;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, src) != cudaSuccess) {
    cudaGetLastError();   // not a pointer CUDA knows: ordinary host memory
    at.type = cudaMemoryTypeUnregistered;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer &&
      (((uintptr_t)at.devicePointer | (uintptr_t)dst | bytes) & 15u) == 0) {
    LAUNCH(1, launch_host_read(at.devicePointer, dst, bytes, c->stream));
  } else {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
  }
  return GSGP_OK;
}

// ------------------------------------------------------------------ load --
static gsgp_status check_shapes(gsgp_ctx *c, const float *Xtr, const float *ytr, int64_t ntr,
                                int32_t l, const float *Xte, const float *yte, int64_t nte) {
  if (nte < 0) return fail(c, GSGP_E_INVALID, "n_test must be >= 0");
  if (c->sharded) {
    // the shard's cases are the problem's cases [case0, case0 + n), training
    // cases first: its training cases are those below n_train_all
    const int64_t n = ntr + nte, all = c->n_train_all + c->n_test_all;
    const int64_t want_tr = std::min(std::max(c->n_train_all - c->shard_case0, (int64_t)0), n);
    if (n < 1 || c->shard_case0 + n > all)
      return fail(c, GSGP_E_INVALID, "a shard holds 1 .. n_train_all + n_test_all - case0 cases");
    if (c->shard_case0 + n < all && n % 1024 != 0)
      return fail(c, GSGP_E_INVALID,
                  "every shard but the last holds a multiple of 1024 cases");
    if (ntr != want_tr)
      return fail(c, GSGP_E_INVALID, "shard at case %lld must hold %lld training cases",
                  (long long)c->shard_case0, (long long)want_tr);
  } else if (ntr < 1) {
    return fail(c, GSGP_E_INVALID, "n_train must be >= 1");
  }
  if (l < 1 || l > 65535) return fail(c, GSGP_E_INVALID, "n_features must be in [1, 65535]");
  if ((ntr > 0 && (!Xtr || !ytr)) || (!c->sharded && (!Xtr || !ytr)))
    return fail(c, GSGP_E_INVALID, "training data pointers must not be NULL");
  if (nte > 0 && (!Xte || !yte)) return fail(c, GSGP_E_INVALID, "test data pointers are NULL");
  if (ntr + nte > (int64_t)0x7fffff00) return fail(c, GSGP_E_INVALID, "too many fitness cases");
  return GSGP_OK;
}

static gsgp_status prepare_data(gsgp_ctx *c, int64_t ntr, int32_t l, int64_t nte) {
  TRY(use_device(c));
  const int64_t N = ntr + nte;
  const int64_t n_pad = (N + 63) / 64 * 64;
  if (c->X && (c->l != l || c->n_pad != n_pad)) {
    dfree(c, c->X);
    dfree(c, c->t);
  }
  if (c->n_pad != n_pad) free_run_buffers(c);
  c->l = l;
  c->n_tr = ntr;
  c->n_te = nte;
  c->N = N;
  c->n_pad = n_pad;
  if (!c->X) TRY(dalloc_n(c, &c->X, (size_t)l * n_pad + kXTailFloats));
  if (!c->t) TRY(dalloc_n(c, &c->t, (size_t)n_pad));
  CK(cudaMemsetAsync(c->X, 0, sizeof(float) * ((size_t)l * n_pad + kXTailFloats), c->stream));
  CK(cudaMemsetAsync(c->t, 0, sizeof(float) * (size_t)n_pad, c->stream));
  c->state = 1;
  c->model_gen = -1;
  return GSGP_OK;
}

extern "C" gsgp_status gsgp_load(gsgp_ctx *c, const float *Xtr, const float *ytr, int64_t ntr,
                                 int32_t l, const float *Xte, const float *yte, int64_t nte) {
  API_GUARD(c)
  TRY(check_shapes(c, Xtr, ytr, ntr, l, Xte, yte, nte));
  TRY(use_device(c));
  // stage every input on the device and check it there (a scan on the GPU
  // instead of the host), before the context's data is touched
  const size_t nx_tr = (size_t)ntr * l, nx_te = (size_t)nte * l;
  float *stage = nullptr;
  TRY(dalloc_n(c, &stage, nx_tr + nx_te + (size_t)ntr + (size_t)nte));
  struct Free {
    gsgp_ctx *c;
    float *&p;
    ~Free() { dfree(c, p); }
  } guard{c, stage};
  float *sXtr = stage, *sXte = stage + nx_tr, *sy = stage + nx_tr + nx_te;
  if (ntr > 0) {   // a case shard may hold test cases only
    TRY(stage_h2d(c, sXtr, Xtr, sizeof(float) * nx_tr));
    TRY(stage_h2d(c, sy, ytr, sizeof(float) * (size_t)ntr));
  }
  if (nte > 0) {
    TRY(stage_h2d(c, sXte, Xte, sizeof(float) * nx_te));
    TRY(stage_h2d(c, sy + ntr, yte, sizeof(float) * (size_t)nte));
  }
  if (!c->d_flag) TRY(dalloc_n(c, &c->d_flag, 1));
  CK(cudaMemsetAsync(c->d_flag, 0, sizeof(unsigned), c->stream));
  LAUNCH(1, launch_nonfinite_check(stage, (int64_t)(nx_tr + nx_te + ntr + nte), c->d_flag,
                                   c->stream));
  unsigned bad = 0;
  CK(cudaMemcpyAsync(&bad, c->d_flag, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (bad) return fail(c, GSGP_E_INVALID, "non-finite value in the fitness cases");
  TRY(prepare_data(c, ntr, l, nte));
  if (ntr > 0) LAUNCH(1, launch_transpose(sXtr, ntr, l, c->X, c->n_pad, 0, c->stream));
  CK(cudaMemcpyAsync(c->t, sy, sizeof(float) * (size_t)(ntr + nte), cudaMemcpyDeviceToDevice,
                     c->stream));
  if (nte > 0) LAUNCH(1, launch_transpose(sXte, nte, l, c->X, c->n_pad, ntr, c->stream));
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_load_device(gsgp_ctx *c, const float *Xtr, const float *ytr,
                                        int64_t ntr, int32_t l, const float *Xte,
                                        const float *yte, int64_t nte) {
  API_GUARD(c)
  TRY(check_shapes(c, Xtr, ytr, ntr, l, Xte, yte, nte));
  TRY(use_device(c));
  if (!c->d_flag) TRY(dalloc_n(c, &c->d_flag, 1));
  CK(cudaMemsetAsync(c->d_flag, 0, sizeof(unsigned), c->stream));
  if (ntr > 0) {
    LAUNCH(1, launch_nonfinite_check(Xtr, ntr * l, c->d_flag, c->stream));
    LAUNCH(1, launch_nonfinite_check(ytr, ntr, c->d_flag, c->stream));
  }
  if (nte > 0) {
    LAUNCH(1, launch_nonfinite_check(Xte, nte * l, c->d_flag, c->stream));
    LAUNCH(1, launch_nonfinite_check(yte, nte, c->d_flag, c->stream));
  }
  unsigned bad = 0;
  CK(cudaMemcpyAsync(&bad, c->d_flag, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (bad) return fail(c, GSGP_E_INVALID, "non-finite value in the fitness cases");
  TRY(prepare_data(c, ntr, l, nte));
  if (ntr > 0) {
    LAUNCH(1, launch_transpose(Xtr, ntr, l, c->X, c->n_pad, 0, c->stream));
    CK(cudaMemcpyAsync(c->t, ytr, sizeof(float) * (size_t)ntr, cudaMemcpyDeviceToDevice,
                       c->stream));
  }
  if (nte > 0) {
    LAUNCH(1, launch_transpose(Xte, nte, l, c->X, c->n_pad, ntr, c->stream));
    CK(cudaMemcpyAsync(c->t + ntr, yte, sizeof(float) * (size_t)nte, cudaMemcpyDeviceToDevice,
                       c->stream));
  }
  return GSGP_OK;
  API_END(c)
}

// ------------------------------------------------------------------ init --
// Programs as evaluated: the live code of linear genomes, else the programs.
static const int *prog_genes(const gsgp_ctx *c, bool pop) {
  if (c->Pc_genes) return pop ? c->Pc_genes : c->Rc_genes;
  return pop ? c->P_genes : c->R_genes;
}
static const float *prog_consts(const gsgp_ctx *c, bool pop) {
  if (c->Pc_genes) return pop ? c->Pc_consts : c->Rc_consts;
  return pop ? c->P_consts : c->R_consts;
}
static const int *prog_len(const gsgp_ctx *c, bool pop) {
  if (c->Pc_genes) return pop ? c->Pc_len : c->Rc_len;
  return pop ? c->P_len : c->R_len;
}

GenParams gen_params(gsgp_ctx *c) {
  GenParams p{};
  p.target = c->t;
  p.pool = c->pool;
  p.sigma_r = c->sigR;
  p.perm = c->perm;
  p.fit = c->fit;
  p.fit_te = c->fit_te;
  p.partial = c->partial;
  p.sel = c->sel;
  p.sel_ms = c->sel_ms;
  p.trace = c->trace;
  p.best_log = c->best_log;
  p.state = c->dstate;
  p.n_pad = c->n_pad;
  p.m = c->cfg.pop_size;
  p.r = c->cfg.n_random_trees;
  p.tsize = c->cfg.tournament_size;
  p.n_train = (int)c->n_tr;
  p.n_cases = (int)c->N;
  p.tiles = c->tiles_interp;   // 1024-case chunks, whatever the stream shape
  p.chunk0 = c->sharded ? (int)(c->shard_case0 / 1024) : 0;
  p.n_train_all = c->sharded ? (int)c->n_train_all : (int)c->n_tr;
  p.n_test_all = c->sharded ? (int)c->n_test_all : (int)(c->N - c->n_tr);
  p.ms_mode = c->cfg.ms_mode;
  p.ms = c->cfg.ms;
  p.key = make_uint2((uint32_t)(c->cfg.seed & 0xffffffffu), (uint32_t)(c->cfg.seed >> 32));
  p.run = c->cfg.run;
  p.elitism = c->cfg.elitism;
  p.p_crossover = c->cfg.p_crossover;
  return p;
}

gsgp_status ensure_trace(gsgp_ctx *c, int need) {
  if (need <= c->gcap) return GSGP_OK;
  const int m = c->cfg.pop_size;
  int cap = c->gcap ? c->gcap : 64;
  while (cap < need) cap *= 2;
  int4 *tr = nullptr;
  double2 *bl = nullptr;
  TRY(dalloc_n(c, &tr, (size_t)cap * m));
  TRY(dalloc_n(c, &bl, (size_t)cap));
  if (c->gen > 0 && c->trace) {
    CK(cudaMemcpyAsync(tr, c->trace, sizeof(int4) * (size_t)c->gen * m, cudaMemcpyDeviceToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(bl, c->best_log, sizeof(double2) * (size_t)c->gen,
                       cudaMemcpyDeviceToDevice, c->stream));
  }
  dfree(c, c->trace);
  dfree(c, c->best_log);
  c->trace = tr;
  c->best_log = bl;
  c->gcap = cap;
  c->graph_dirty = true;
  return GSGP_OK;
}

static gsgp_status finish_init(gsgp_ctx *c);

extern "C" gsgp_status gsgp_init(gsgp_ctx *c) {
  API_GUARD(c)
  if (c->state < 1) return fail(c, GSGP_E_STATE, "gsgp_init before gsgp_load");
  TRY(use_device(c));
  c->state = 1;   // until this initialisation completes
  const gsgp_config &cf = c->cfg;
  const int m = cf.pop_size, r = cf.n_random_trees;
  const bool linear = cf.init_mode == GSGP_INIT_LINEAR;
  const int Kp = linear ? cf.max_genes : (1 << (cf.pop_max_depth + 1)) - 1;
  const int Kr = linear ? cf.max_genes : (1 << (cf.rt_max_depth + 1)) - 1;
  // chunks of the whole problem (all shards): the partial sums' row stride
  const int64_t n_all = c->sharded ? c->n_train_all + c->n_test_all : c->N;
  const int64_t chunks_all = (c->sharded ? n_all : c->n_pad) / 1024 +
                             ((c->sharded ? n_all : c->n_pad) % 1024 != 0);
  const int64_t key[8] = {m, r, c->n_pad, Kp, Kr, cf.sigma_dtype, cf.init_mode, chunks_all};
  if (memcmp(key, c->layout_key, sizeof key) != 0) {
    free_run_buffers(c);
    c->Kp = Kp;
    c->Kr = Kr;
    // partial sums per 1024-case chunk (interpreter and stream kernels)
    c->tiles_interp = (int)chunks_all;
    const int tiles_max = c->tiles_interp;
    TRY(dalloc_n(c, &c->P_genes, (size_t)m * Kp));
    TRY(dalloc_n(c, &c->P_consts, (size_t)m * Kp));
    TRY(dalloc_n(c, &c->P_len, (size_t)m));
    TRY(dalloc_n(c, &c->R_genes, (size_t)r * Kr));
    TRY(dalloc_n(c, &c->R_consts, (size_t)r * Kr));
    TRY(dalloc_n(c, &c->R_len, (size_t)r));
    if (linear) {
      TRY(dalloc_n(c, &c->Pc_genes, (size_t)m * Kp));
      TRY(dalloc_n(c, &c->Pc_consts, (size_t)m * Kp));
      TRY(dalloc_n(c, &c->Pc_len, (size_t)m));
      TRY(dalloc_n(c, &c->Rc_genes, (size_t)r * Kr));
      TRY(dalloc_n(c, &c->Rc_consts, (size_t)r * Kr));
      TRY(dalloc_n(c, &c->Rc_len, (size_t)r));
    }
    TRY(dalloc_n(c, &c->pool, (size_t)2 * m * c->n_pad));
    const size_t sbytes = cf.sigma_dtype == GSGP_SIGMA_BF16 ? 2 : 4;
    TRY(dalloc(c, &c->sigR, sbytes * (size_t)r * c->n_pad));
    TRY(dalloc_n(c, &c->perm, (size_t)4 * m));
    TRY(dalloc_n(c, &c->fit, (size_t)2 * m));
    TRY(dalloc_n(c, &c->fit_te, (size_t)2 * m));
    TRY(dalloc_n(c, &c->partial, (size_t)m * tiles_max));
    TRY(dalloc_n(c, &c->sel, (size_t)m));
    TRY(dalloc_n(c, &c->sel_ms, (size_t)m));
    TRY(dalloc_n(c, &c->dstate, 1));
    TRY(dalloc_n(c, &c->d_anc, 1));
    TRY(dalloc_n(c, &c->d_stack, 2));
    memcpy(c->layout_key, key, sizeof key);
    c->graph_dirty = true;
    c->shape_ready = false;
  }
  c->gen = 0;
  c->model_gen = -1;
  TRY(ensure_trace(c, 64));
  const uint2 k2 = make_uint2((uint32_t)(cf.seed & 0xffffffffu), (uint32_t)(cf.seed >> 32));
  // interpreter stack entries below the top: a tree of depth d needs d + 1
  int slots_p = cf.pop_max_depth + 1, slots_r = cf.rt_max_depth + 1;
  int max_len_p = Kp, max_len_r = Kr;   // longest program of each pool
  if (linear) max_len_p = max_len_r = 1;
  if (linear) {
    LAUNCH(1, launch_genomes(m, Kp, c->l, k2, cf.run, kPurposePop, cf.const_lo, cf.const_hi,
                             c->P_genes, c->P_consts, c->P_len, c->stream));
    LAUNCH(1, launch_genomes(r, Kr, c->l, k2, cf.run, kPurposeRt, cf.const_lo, cf.const_hi,
                             c->R_genes, c->R_consts, c->R_len, c->stream));
    // the live code of each genome, then the deepest stack of each pool,
    // which sizes the interpreter's stack
    LAUNCH(1, launch_compact(c->P_genes, c->P_consts, c->P_len, m, Kp, c->Pc_genes, c->Pc_consts,
                             c->Pc_len, c->stream));
    LAUNCH(1, launch_compact(c->R_genes, c->R_consts, c->R_len, r, Kr, c->Rc_genes, c->Rc_consts,
                             c->Rc_len, c->stream));
    CK(cudaMemsetAsync(c->d_stack, 0, 2 * sizeof(int), c->stream));
    LAUNCH(1, launch_max_stack(c->Pc_genes, c->Pc_len, m, Kp, c->d_stack, c->stream));
    LAUNCH(1, launch_max_stack(c->Rc_genes, c->Rc_len, r, Kr, c->d_stack + 1, c->stream));
    int h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, c->d_stack, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    std::vector<int> lp((size_t)m), lr((size_t)r);
    CK(cudaMemcpyAsync(lp.data(), c->Pc_len, sizeof(int) * lp.size(), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaMemcpyAsync(lr.data(), c->Rc_len, sizeof(int) * lr.size(), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->eval_genes[0] = c->eval_genes[1] = 0;
    for (int v : lp) {
      c->eval_genes[0] += v;
      max_len_p = v > max_len_p ? v : max_len_p;
    }
    for (int v : lr) {
      c->eval_genes[1] += v;
      max_len_r = v > max_len_r ? v : max_len_r;
    }
    if (h[0] > kMaxStack || h[1] > kMaxStack)
      return fail(c, GSGP_E_INVALID,
                  "a generated genome needs a stack of %d entries (limit %d); use a shorter "
                  "max_genes or another seed", h[0] > h[1] ? h[0] : h[1], kMaxStack);
    slots_p = h[0] > 1 ? h[0] : 1;
    slots_r = h[1] > 1 ? h[1] : 1;
  } else {
    c->Pc_genes = nullptr;   // the trees are evaluated as generated
    c->eval_genes[0] = c->eval_genes[1] = -1;   // counted on request (gsgp_get_info)
    LAUNCH(1, launch_treegen(m, cf.pop_min_depth, cf.pop_max_depth, Kp, c->l, k2, cf.run,
                             kPurposePop, cf.p_grow_function, cf.p_feature_given_terminal,
                             cf.const_lo, cf.const_hi, c->P_genes, c->P_consts, c->P_len,
                             c->stream));
    LAUNCH(1, launch_treegen(r, cf.rt_min_depth, cf.rt_max_depth, Kr, c->l, k2, cf.run,
                             kPurposeRt, cf.p_grow_function, cf.p_feature_given_terminal,
                             cf.const_lo, cf.const_hi, c->R_genes, c->R_consts, c->R_len,
                             c->stream));
  }
  // the interpreter runs the programs with their "terminal, function" pairs
  // fused, from buffers that live for this call
  struct Fused {
    gsgp_ctx *c;
    int *genes[2] = {nullptr, nullptr}, *len[2] = {nullptr, nullptr};
    float *consts[2] = {nullptr, nullptr};
    int *need = nullptr, *order = nullptr;
    ~Fused() {
      for (int q = 0; q < 2; ++q) {
        dfree(c, genes[q]);
        dfree(c, consts[q]);
        dfree(c, len[q]);
      }
      dfree(c, need);
      dfree(c, order);
    }
  } fz{c};
  for (int q = 0; q < 2; ++q) {
    const size_t cnt = q == 0 ? (size_t)m : (size_t)r, K = q == 0 ? (size_t)Kp : (size_t)Kr;
    TRY(dalloc_n(c, &fz.genes[q], cnt * K));
    TRY(dalloc_n(c, &fz.consts[q], cnt * K));
    TRY(dalloc_n(c, &fz.len[q], cnt));
  }
  LAUNCH(1, launch_fuse(prog_genes(c, true), prog_consts(c, true), prog_len(c, true), m, Kp,
                        fz.genes[0], fz.consts[0], fz.len[0], c->stream));
  LAUNCH(1, launch_fuse(prog_genes(c, false), prog_consts(c, false), prog_len(c, false), r, Kr,
                        fz.genes[1], fz.consts[1], fz.len[1], c->stream));
  // Interpreter launches: one per group of programs, shared memory sized for
  // the group's deepest stack.  Linear genomes are grouped by the stack
  // entries each needs (most need a few; the deepest of a large pool needs
  // about twice as many, and sizing every CTA for it costs occupancy; a
  // group needing at most 3 also runs at six CTAs per SM instead of five);
  // a pool of trees is one group sized by its depth.
  struct Group {
    int first, count, slots;   // first < 0: programs 0 .. count - 1 in order
  };
  std::vector<Group> groups[2];
  if (linear) {
    TRY(dalloc_n(c, &fz.need, (size_t)(m + r)));
    TRY(dalloc_n(c, &fz.order, (size_t)(m + r)));
    LAUNCH(1, launch_stack_need(fz.genes[0], fz.len[0], m, Kp, fz.need, c->stream));
    LAUNCH(1, launch_stack_need(fz.genes[1], fz.len[1], r, Kr, fz.need + m, c->stream));
    std::vector<int> need((size_t)(m + r)), order;
    order.reserve((size_t)(m + r));
    CK(cudaMemcpyAsync(need.data(), fz.need, sizeof(int) * need.size(), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    static const int kSlotBounds[] = {2, 3, 4, 6, 8, 12, 16, 24, kMaxStack};
    for (int q = 0; q < 2; ++q) {
      const int base = q == 0 ? 0 : m, cnt = q == 0 ? m : r;
      int lo = -1;
      for (const int hi : kSlotBounds) {
        Group gq{(int)order.size(), 0, 1};
        for (int i = 0; i < cnt; ++i) {
          const int v = need[(size_t)(base + i)];
          if (v > lo && v <= hi) {
            order.push_back(i);
            gq.slots = v > gq.slots ? v : gq.slots;
          }
        }
        gq.count = (int)order.size() - gq.first;
        if (gq.count > 0) groups[q].push_back(gq);
        lo = hi;
      }
    }
    if ((int)order.size() != m + r)
      return fail(c, GSGP_E_INVALID, "interpreter groups cover %d of %d programs",
                  (int)order.size(), m + r);
    CK(cudaMemcpyAsync(fz.order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice,
                       c->stream));
  } else {
    groups[0].push_back(Group{-1, m, slots_p});
    groups[1].push_back(Group{-1, r, slots_r});
  }
  InterpParams ip{};
  ip.X = c->X;
  ip.target = c->t;
  ip.n_pad = c->n_pad;
  ip.n_train = (int)c->n_tr;
  ip.n_cases = (int)c->N;
  ip.tiles = c->tiles_interp;
  ip.chunk0 = c->sharded ? (int)(c->shard_case0 / 1024) : 0;
  if (c->sharded)   // the other shards' chunks stay zero until the exchange
    CK(cudaMemsetAsync(c->partial, 0, sizeof(double2) * (size_t)m * c->tiles_interp, c->stream));
  ip.protect_eps = cf.protect_eps;
  ip.n_features = c->l;
  // population semantics + squared errors (rows 0..m-1 of the pool)
  ip.genes = fz.genes[0];
  ip.consts = fz.consts[0];
  ip.lengths = fz.len[0];
  ip.K = Kp;
  ip.max_len = max_len_p;
  ip.out = c->pool;
  ip.partial = c->partial;
  c->init_timed = false;
  if (c->timing && !c->ev_init[0])
    for (auto &e : c->ev_init) CK(cudaEventCreate(&e));
  if (c->timing) CK(cudaEventRecord(c->ev_init[0], c->stream));
  for (const Group &gq : groups[0]) {
    ip.order = gq.first < 0 ? nullptr : fz.order + gq.first;
    ip.stack_slots = gq.slots;
    LAUNCH(1, launch_interpret(0, ip, gq.count, c->stream));
  }
  if (c->timing) CK(cudaEventRecord(c->ev_init[1], c->stream));
  // random-tree semantics wrapped by the logistic function
  ip.genes = fz.genes[1];
  ip.consts = fz.consts[1];
  ip.lengths = fz.len[1];
  ip.K = Kr;
  ip.max_len = max_len_r;
  ip.out = c->sigR;
  ip.partial = nullptr;
  if (c->timing) CK(cudaEventRecord(c->ev_init[2], c->stream));
  for (const Group &gq : groups[1]) {
    ip.order = gq.first < 0 ? nullptr : fz.order + gq.first;
    ip.stack_slots = gq.slots;
    LAUNCH(1, launch_interpret(cf.sigma_dtype == GSGP_SIGMA_BF16 ? 2 : 1, ip, gq.count, c->stream));
  }
  if (c->timing) {
    CK(cudaEventRecord(c->ev_init[3], c->stream));
    c->init_timed = true;
  }
  c->shard_pending = 0;
  if (c->sharded) {   // the fitness waits for the other shards' chunk sums
    c->shard_pending = 1;
    return GSGP_OK;
  }
  return finish_init(c);
  API_END(c)
}

// ComputeFitness of the initial population from the complete chunk sums,
// and the generation-0 state.
static gsgp_status finish_init(gsgp_ctx *c) {
  const int m = c->cfg.pop_size;
  const int n_tr = c->sharded ? (int)c->n_train_all : (int)c->n_tr;
  const int n_te = c->sharded ? (int)c->n_test_all : (int)c->n_te;
  LAUNCH(1, launch_fitness_finalize(c->partial, c->tiles_interp, m, n_tr, n_te, c->fit,
                                    c->fit_te, c->stream));
  LAUNCH(1, launch_init_state(m, c->perm, c->fit, c->dstate, c->stream));
  if (c->gs) CK(cudaMemsetAsync(&c->gs->err, 0, sizeof(int), c->stream));
  c->shard_pending = 0;
  c->state = 2;
  return GSGP_OK;
}

// ---------------------------------------------------------------- evolve --
static gsgp_status launch_generation(gsgp_ctx *c, const GenParams &p, cudaStream_t s,
                                     cudaEvent_t ev_start, cudaEvent_t ev_stop, bool external) {
  const int bf = c->cfg.sigma_dtype == GSGP_SIGMA_BF16;
  LAUNCH(1, launch_select(p, s, true));
  if (ev_start)
    CK(external ? cudaEventRecordWithFlags(ev_start, s, cudaEventRecordExternal)
                : cudaEventRecord(ev_start, s));
  LAUNCH(1, launch_stream(p, bf, c->shape, s, ev_start == nullptr));
  if (ev_stop)
    CK(external ? cudaEventRecordWithFlags(ev_stop, s, cudaEventRecordExternal)
                : cudaEventRecord(ev_stop, s));
  LAUNCH(1, launch_final(p, s, ev_stop == nullptr));
  return GSGP_OK;
}

// Shapes the autotuner tries: chained path (vec in {1,2,4}, opb in {2,4,8})
// and persistent path (vec in {1,2}, opb in {1,2,4}, the register stream);
// the choice is cached per problem layout for the process.  The TMA-staged
// stream (opb = 0) is selectable with gsgp_set_evolve_shape but not a
// candidate: its one-generation trials can come out ahead while it is slower
// over whole launches on every measured workload (one CTA per SM, a start-up
// cost that a one-generation trial hides).
static const GenShape kChainShapes[] = {{1, 2}, {1, 4}, {1, 8}, {2, 2}, {2, 4},
                                        {2, 8}, {4, 2}, {4, 4}, {4, 8}};
static const GenShape kPersistShapes[] = {{1, 1}, {1, 2}, {1, 4}, {1, 8}, {1, 16},
                                          {2, 1}, {2, 2}, {2, 4}, {2, 8}, {2, 16}};
struct Tuned {
  int path;
  GenShape shape;
};
static std::unordered_map<std::string, Tuned> g_tuned;

static std::string shape_key(gsgp_ctx *c) {
  char buf[192];
  snprintf(buf, sizeof buf, "%d:%d:%d:%lld:%d:%lld:%d:%d:%d", c->device, c->cfg.pop_size,
           c->cfg.n_random_trees, (long long)c->n_pad, c->cfg.sigma_dtype, (long long)c->n_tr,
           c->forced_path, c->forced.vec, c->forced.opb);
  return buf;
}

// CTAs of the persistent kernel: at most the co-resident count, and no more
// than needed to give every CTA the same number of stream items (a partly
// filled last round of items would leave most CTAs idle at the barrier).
static int persist_grid(gsgp_ctx *c, const GenShape &sh) {
  const int max_grid = persist_max_grid(c->cfg.sigma_dtype == GSGP_SIGMA_BF16, sh);
  if (max_grid <= 0) return 0;
  const int64_t tiles = (c->n_pad + 1024 * sh.vec - 1) / (1024 * sh.vec);
  const int opb = sh.opb > 0 ? sh.opb : 1;   // the TMA variant streams one offspring per unit
  const int64_t groups = (c->cfg.pop_size + opb - 1) / opb;
  const int64_t items = tiles * groups;
  if (items >= ((int64_t)1 << 31)) return 0;   // item indices are 32-bit in the kernels
  const int64_t rounds = (items + max_grid - 1) / max_grid;
  const int64_t grid = (items + rounds - 1) / rounds;
  return (int)(grid < max_grid ? grid : max_grid);
}

static gsgp_status ensure_cta_arrays(gsgp_ctx *c, int grid) {
  if (grid <= c->cta_cap && c->gs) return GSGP_OK;
  int err = 0;
  if (c->gs) {   // keep the sticky error word across the reallocation
    CK(cudaMemcpyAsync(&err, &c->gs->err, sizeof err, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  dfree(c, c->cta_min);
  dfree(c, c->cta_max);
  dfree(c, c->gs);
  TRY(dalloc_n(c, &c->cta_min, (size_t)grid));
  TRY(dalloc_n(c, &c->cta_max, (size_t)grid));
  void *g = nullptr;
  TRY(dalloc(c, &g, grid_sync_bytes(grid)));
  c->gs = static_cast<GridSync *>(g);
  CK(cudaMemsetAsync(c->gs, 0, grid_sync_bytes(grid), c->stream));
  if (err) CK(cudaMemcpyAsync(&c->gs->err, &err, sizeof err, cudaMemcpyHostToDevice, c->stream));
  c->cta_cap = grid;
  return GSGP_OK;
}

static gsgp_status launch_persist_chunk(gsgp_ctx *c, int G) {
  const GenParams p = gen_params(c);
  PersistArgs x{c->gs, c->cta_min, c->cta_max, G, kSpinLimitDefault};
  CK(cudaMemsetAsync(&c->gs->count, 0, grid_sync_bytes(c->grid) - offsetof(GridSync, count),
                     c->stream));
  if (c->fault_spin_limit) {
    // the timeout test (one launch only): the arrival counter starts one
    // arrival short (2^32 - 1: the first arrival wraps it to 0), so after
    // every CTA has arrived at the first barrier the count is grid - 1 and
    // every wait runs out after fault_spin_limit naps; no CTA passes it
    x.spin_limit = c->fault_spin_limit;
    CK(cudaMemsetAsync(&c->gs->count, 0xff, sizeof(unsigned), c->stream));
    c->fault_spin_limit = 0;
  }
  LAUNCH(1, launch_persist(p, x, c->cfg.sigma_dtype == GSGP_SIGMA_BF16, c->shape, c->grid,
                           c->stream));
  return GSGP_OK;
}

// Save / restore the per-generation state (slot-to-row map, fitness,
// counters) around autotuning trials of whole generations.  A trial of one
// generation writes only free rows of the pool, the draws, the partials and
// this generation's trace and log entries, all of which the real generation
// rewrites identically.
gsgp_status ensure_backup(gsgp_ctx *c) {
  const size_t m = (size_t)c->cfg.pop_size;
  if (!c->bk_perm) {
    TRY(dalloc_n(c, &c->bk_perm, 4 * m));
    TRY(dalloc_n(c, &c->bk_fit, 2 * m));
    TRY(dalloc_n(c, &c->bk_fit_te, 2 * m));
    TRY(dalloc_n(c, &c->bk_state, 1));
  }
  return GSGP_OK;
}

gsgp_status snapshot(gsgp_ctx *c, bool save, cudaStream_t s) {
  const size_t m = (size_t)c->cfg.pop_size;
  TRY(ensure_backup(c));
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  if (save) {
    CK(cudaMemcpyAsync(c->bk_perm, c->perm, sizeof(int) * 4 * m, k, s));
    CK(cudaMemcpyAsync(c->bk_fit, c->fit, sizeof(double) * 2 * m, k, s));
    CK(cudaMemcpyAsync(c->bk_fit_te, c->fit_te, sizeof(double) * 2 * m, k, s));
    CK(cudaMemcpyAsync(c->bk_state, c->dstate, sizeof(DevState), k, s));
  } else {
    CK(cudaMemcpyAsync(c->perm, c->bk_perm, sizeof(int) * 4 * m, k, s));
    CK(cudaMemcpyAsync(c->fit, c->bk_fit, sizeof(double) * 2 * m, k, s));
    CK(cudaMemcpyAsync(c->fit_te, c->bk_fit_te, sizeof(double) * 2 * m, k, s));
    CK(cudaMemcpyAsync(c->dstate, c->bk_state, sizeof(DevState), k, s));
  }
  return GSGP_OK;
}

static gsgp_status time_shape(gsgp_ctx *c, int path, const GenShape &sh, float *out_ms) {
  const int bf = c->cfg.sigma_dtype == GSGP_SIGMA_BF16;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  c->path = path;
  c->shape = sh;
  gsgp_status st = GSGP_OK;
  cudaError_t e = cudaSuccess;
  float best = 1e30f;
  if (path == 2) {
    const GenParams p = gen_params(c);
    e = launch_select(p, c->stream, false);
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
      if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
      if (e == cudaSuccess) e = launch_stream(p, bf, sh, c->stream, false);
      if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
      c->launches += 1;
    }
    c->launches += 1;
  } else {
    c->grid = persist_grid(c, sh);
    st = ensure_cta_arrays(c, c->grid);
    if (st == GSGP_OK) st = snapshot(c, true, c->stream);
    for (int rep = 0; rep < 4 && st == GSGP_OK && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, c->stream);
      if (e == cudaSuccess) st = launch_persist_chunk(c, 1);
      if (st == GSGP_OK && e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
      if (st == GSGP_OK && e == cudaSuccess) st = snapshot(c, false, c->stream);
      if (st == GSGP_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (st == GSGP_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms > 0.f && ms < best) best = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GSGP_OK) return st;
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune", __LINE__);
  *out_ms = best;
  return GSGP_OK;
}

// Choose the generation path and shape: forced, cached for this layout, or
// timed.  The persistent path is used whenever the device supports
// cooperative launch (it removes the per-generation launch chain); a forced
// path may still autotune its shape.
static gsgp_status choose_shape(gsgp_ctx *c) {
  if (c->shape_ready) return GSGP_OK;
  const int bf = c->cfg.sigma_dtype == GSGP_SIGMA_BF16;
  int path = c->forced_path;
  if (path == 0) path = persist_max_grid(bf, GenShape{1, 2}) > 0 ? 1 : 2;
  if (c->forced.vec) {
    c->path = path;
    c->shape = c->forced;
  } else {
    const std::string key = shape_key(c);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      c->path = it->second.path;
      c->shape = it->second.shape;
    } else {
      float best_ms = 1e30f;
      Tuned best{path, path == 1 ? kPersistShapes[0] : kChainShapes[0]};
      const GenShape *cand = path == 1 ? kPersistShapes : kChainShapes;
      const int nc = path == 1 ? (int)(sizeof kPersistShapes / sizeof kPersistShapes[0])
                               : (int)(sizeof kChainShapes / sizeof kChainShapes[0]);
      for (int k = 0; k < nc; ++k) {
        if (path == 1 && persist_max_grid(bf, cand[k]) <= 0) continue;
        float ms = 0.f;
        TRY(time_shape(c, path, cand[k], &ms));
        // a later shape must win by more than 1% (trial noise): near-ties
        // keep the earlier shape, so the choice repeats from run to run
        if (ms < best_ms * 0.99f) {
          best_ms = ms;
          best = Tuned{path, cand[k]};
        }
      }
      g_tuned[key] = best;
      c->path = best.path;
      c->shape = best.shape;
    }
  }
  if (c->path == 1) {
    c->grid = persist_grid(c, c->shape);
    if (c->grid <= 0) return fail(c, GSGP_E_CUDA, "cooperative launch is not available");
    TRY(ensure_cta_arrays(c, c->grid));
  }
  c->shape_ready = true;
  c->graph_dirty = true;
  return GSGP_OK;
}

// Sticky device error of the persistent kernel's barrier (after a sync).
gsgp_status check_device_error(gsgp_ctx *c) {
  if (!c->gs) return GSGP_OK;
  int err = 0;
  CK(cudaMemcpyAsync(&err, &c->gs->err, sizeof err, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (err)
    return fail(c, GSGP_E_TIMEOUT,
                "a grid barrier of the generation kernel gave up waiting; re-run gsgp_init");
  return GSGP_OK;
}

static gsgp_status build_graph(gsgp_ctx *c, int u, bool timed) {
  free_graph(c);
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  while (timed && (int)c->ev_marks.size() < 2 * u) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    c->ev_marks.push_back(e);
  }
  const GenParams p = gen_params(c);
  CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  gsgp_status st = GSGP_OK;
  for (int k = 0; k < u && st == GSGP_OK; ++k)
    st = launch_generation(c, p, c->cap_stream, timed ? c->ev_marks[2 * k] : nullptr,
                           timed ? c->ev_marks[2 * k + 1] : nullptr, true);
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &graph);
  if (st != GSGP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ee != cudaSuccess) return cuda_fail(c, ee, "cudaStreamEndCapture", __LINE__);
  c->graph = graph;
  if (timed) {
    // locate the event-record nodes by the event each was captured with
    c->ev_nodes.assign((size_t)2 * u, nullptr);
    size_t n = 0;
    CK(cudaGraphGetNodes(graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    CK(cudaGraphGetNodes(graph, nodes.data(), &n));
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType ty;
      CK(cudaGraphNodeGetType(nd, &ty));
      if (ty != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t ev;
      CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
      for (int k = 0; k < 2 * u; ++k)
        if (c->ev_marks[(size_t)k] == ev) c->ev_nodes[(size_t)k] = nd;
    }
    for (auto nd : c->ev_nodes)
      if (!nd) return fail(c, GSGP_E_CUDA, "timing node missing from the captured graph");
  }
  cudaError_t ie = cudaGraphInstantiate(&c->gexec, graph, 0);
  if (ie != cudaSuccess) {
    c->gexec = nullptr;
    return cuda_fail(c, ie, "cudaGraphInstantiate", __LINE__);
  }
  c->graph_u = u;
  c->graph_timed = timed;
  c->graph_dirty = false;
  return GSGP_OK;
}

static gsgp_status ensure_events(gsgp_ctx *c, int need) {
  while ((int)c->ev0.size() < need) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    c->ev0.push_back(a);
    c->ev1.push_back(b);
  }
  return GSGP_OK;
}

static constexpr int kGraphGenerations = 8;      // chained path: generations per graph
static constexpr int kPersistGenerations = 64;   // persistent path: generations per launch

extern "C" gsgp_status gsgp_evolve(gsgp_ctx *c, int32_t generations, double *best_train,
                                   double *best_test) {
  API_GUARD(c)
  if (c->state != 2) return fail(c, GSGP_E_STATE, "gsgp_evolve before gsgp_init");
  if (c->sharded)
    return fail(c, GSGP_E_STATE,
                "a case shard evolves by gsgp_shard_generation and gsgp_shard_finish");
  if (generations < 0) return fail(c, GSGP_E_INVALID, "generations must be >= 0");
  if (generations == 0) return GSGP_OK;
  if ((int64_t)c->gen + generations > 0x7fffffff) return fail(c, GSGP_E_INVALID, "too many generations");
  TRY(use_device(c));
  TRY(ensure_trace(c, c->gen + generations));
  TRY(choose_shape(c));
  const int g0 = c->gen;
  int left = generations;
  if (c->timing) TRY(ensure_events(c, c->ev_used + generations));
  if (c->path == 1) {
    while (left > 0) {
      const int G = left < kPersistGenerations ? left : kPersistGenerations;
      if (c->timing) CK(cudaEventRecord(c->ev0[(size_t)c->ev_used], c->stream));
      TRY(launch_persist_chunk(c, G));
      if (c->timing) {
        CK(cudaEventRecord(c->ev1[(size_t)c->ev_used], c->stream));
        ++c->ev_used;
      }
      left -= G;
    }
  }
  if (left >= kGraphGenerations) {
    if (c->graph_dirty || !c->gexec || c->graph_u != kGraphGenerations ||
        c->graph_timed != c->timing)
      TRY(build_graph(c, kGraphGenerations, c->timing));
    while (left >= kGraphGenerations) {
      if (c->timing) {
        for (int k = 0; k < kGraphGenerations; ++k) {
          CK(cudaGraphExecEventRecordNodeSetEvent(c->gexec, c->ev_nodes[(size_t)2 * k],
                                                  c->ev0[(size_t)c->ev_used + k]));
          CK(cudaGraphExecEventRecordNodeSetEvent(c->gexec, c->ev_nodes[(size_t)2 * k + 1],
                                                  c->ev1[(size_t)c->ev_used + k]));
        }
        c->ev_used += kGraphGenerations;
      }
      CK(cudaGraphLaunch(c->gexec, c->stream));
      c->launches += 3 * kGraphGenerations;
      left -= kGraphGenerations;
    }
  }
  if (left > 0) {
    const GenParams p = gen_params(c);
    for (int k = 0; k < left; ++k) {
      cudaEvent_t a = nullptr, b = nullptr;
      if (c->timing) {
        a = c->ev0[(size_t)c->ev_used];
        b = c->ev1[(size_t)c->ev_used];
        ++c->ev_used;
      }
      TRY(launch_generation(c, p, c->stream, a, b, false));
    }
  }
  c->gen += generations;
  c->model_gen = -1;
  if (best_train || best_test) {
    std::vector<double2> h((size_t)generations);
    CK(cudaMemcpyAsync(h.data(), c->best_log + g0, sizeof(double2) * (size_t)generations,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    TRY(check_device_error(c));
    for (int k = 0; k < generations; ++k) {
      if (best_train) best_train[k] = h[k].x;
      if (best_test) best_test[k] = h[k].y;
    }
  }
  return GSGP_OK;
  API_END(c)
}

// ------------------------------------------------------- case sharding --
extern "C" gsgp_status gsgp_shard_configure(gsgp_ctx *c, int64_t case0, int64_t n_train_all,
                                            int64_t n_test_all) {
  API_GUARD(c)
  if (c->state != 0) return fail(c, GSGP_E_STATE, "gsgp_shard_configure after gsgp_load");
  if (n_train_all < 1 || n_test_all < 0 || n_train_all + n_test_all > (int64_t)0x7fffff00)
    return fail(c, GSGP_E_INVALID, "need n_train_all >= 1, n_test_all >= 0");
  if (case0 < 0 || case0 % 1024 != 0 || case0 >= n_train_all + n_test_all)
    return fail(c, GSGP_E_INVALID, "case0 must be a multiple of 1024 below the case count");
  c->sharded = true;
  c->shard_case0 = case0;
  c->n_train_all = n_train_all;
  c->n_test_all = n_test_all;
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_shard_partials(gsgp_ctx *c, double **partials, int64_t *rows,
                                           int64_t *chunks) {
  API_GUARD(c)
  if (!c->sharded) return fail(c, GSGP_E_STATE, "not a case shard");
  if (!c->shard_pending)
    return fail(c, GSGP_E_STATE, "no exchange is pending (after gsgp_init or a generation)");
  if (partials) *partials = reinterpret_cast<double *>(c->partial);
  if (rows) *rows = c->cfg.pop_size;
  if (chunks) *chunks = c->tiles_interp;
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_shard_generation(gsgp_ctx *c) {
  API_GUARD(c)
  if (!c->sharded) return fail(c, GSGP_E_STATE, "not a case shard");
  if (c->state != 2 || c->shard_pending)
    return fail(c, GSGP_E_STATE, "gsgp_shard_generation needs a finished init or generation");
  if (c->gen == 0x7fffffff) return fail(c, GSGP_E_INVALID, "too many generations");
  TRY(use_device(c));
  TRY(ensure_trace(c, c->gen + 1));
  const GenParams p = gen_params(c);
  // this shard's chunk columns are rewritten by the stream; the others must
  // be zero, so that summing the shards' arrays assembles the whole
  CK(cudaMemsetAsync(c->partial, 0, sizeof(double2) * (size_t)p.m * c->tiles_interp, c->stream));
  LAUNCH(1, launch_select(p, c->stream, false));
  LAUNCH(1, launch_stream(p, c->cfg.sigma_dtype == GSGP_SIGMA_BF16, GenShape{1, 8}, c->stream,
                          false));
  c->shard_pending = 2;
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_shard_finish(gsgp_ctx *c) {
  API_GUARD(c)
  if (!c->sharded) return fail(c, GSGP_E_STATE, "not a case shard");
  if (!c->shard_pending) return fail(c, GSGP_E_STATE, "no exchange is pending");
  TRY(use_device(c));
  if (c->shard_pending == 1) return finish_init(c);
  const GenParams p = gen_params(c);
  LAUNCH(1, launch_final(p, c->stream, false));
  c->gen += 1;
  c->model_gen = -1;
  c->shard_pending = 0;
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_arm_barrier_fault(gsgp_ctx *c, uint32_t spin_limit) {
  API_GUARD(c)
  if (spin_limit < 1024 || spin_limit > kSpinLimitDefault)
    return fail(c, GSGP_E_INVALID, "spin_limit must be in [1024, 2^24]");
  c->fault_spin_limit = spin_limit;
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_set_evolve_shape(gsgp_ctx *c, int32_t path, int32_t vec,
                                             int32_t opb) {
  API_GUARD(c)
  if (path < 0 || path > 2) return fail(c, GSGP_E_INVALID, "path must be 0, 1 or 2");
  const bool autotune = vec == 0 && opb == 0;   // (vec, 0) with vec > 0 is the TMA variant
  if (!autotune) {
    const GenShape sh{vec, opb};
    if (path == 0) return fail(c, GSGP_E_INVALID, "a shape needs an explicit path");
    if (path == 1 && !persist_shape_supported(sh))
      return fail(c, GSGP_E_INVALID,
                  "persistent shape: vec in {1,2} with opb in {1,2,4,8,16}, "
                  "or vec in {1,2,4} with opb 0");
    if (path == 1 && opb == 0 && c->cfg.p_crossover > 0.0f)
      return fail(c, GSGP_E_INVALID, "the TMA-staged stream does not support crossover");
    if (path == 2 && !gen_shape_supported(sh))
      return fail(c, GSGP_E_INVALID, "chained shape must have vec in {1,2,4}, opb in {2,4,8}");
  }
  c->forced_path = path;
  c->forced = autotune ? GenShape{0, 0} : GenShape{vec, opb};
  c->shape_ready = false;
  c->graph_dirty = true;
  return GSGP_OK;
  API_END(c)
}

// ------------------------------------------------------- best individual --
// Runs with crossover keep no ancestor-plus-coefficients model.
static bool with_crossover(const gsgp_ctx *c) { return c->cfg.p_crossover > 0.0f; }

static gsgp_status build_model(gsgp_ctx *c) {
  if (c->model_gen == c->gen) return GSGP_OK;
  const int m = c->cfg.pop_size, r = c->cfg.n_random_trees;
  const int G = c->gen;
  if (G > c->lineage_cap) {
    dfree(c, c->lineage);
    int cap = 64;
    while (cap < G) cap *= 2;
    TRY(dalloc_n(c, &c->lineage, (size_t)cap));
    c->lineage_cap = cap;
  }
  if (!c->lineage) {
    TRY(dalloc_n(c, &c->lineage, 64));
    c->lineage_cap = 64;
  }
  const int L = lineage_segment(G > 0 ? G : 1);
  const int nseg = G > 0 ? (G + L - 1) / L : 1;
  if ((int64_t)nseg * m > c->lin_jump_cap) {
    dfree(c, c->lin_jump);
    TRY(dalloc_n(c, &c->lin_jump, (size_t)nseg * m));
    c->lin_jump_cap = (int64_t)nseg * m;
  }
  if (nseg > c->lin_start_cap) {
    dfree(c, c->lin_start);
    TRY(dalloc_n(c, &c->lin_start, (size_t)nseg));
    c->lin_start_cap = nseg;
  }
  LAUNCH(3, launch_lineage(c->trace, m, G, c->dstate, c->lineage, c->d_anc, c->lin_jump,
                           c->lin_start, c->stream));
  c->h_lineage.resize((size_t)G);
  DevState st{};
  if (G > 0)
    CK(cudaMemcpyAsync(c->h_lineage.data(), c->lineage, sizeof(int4) * (size_t)G,
                       cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&c->ancestor, c->d_anc, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&st, c->dstate, sizeof st, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  TRY(check_device_error(c));
  c->best_slot = st.best_slot;
  const size_t par = (size_t)(G & 1);
  CK(cudaMemcpyAsync(&c->best_tr, c->fit + par * m + c->best_slot, sizeof(double),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&c->best_te, c->fit_te + par * m + c->best_slot, sizeof(double),
                     cudaMemcpyDeviceToHost, c->stream));
  // coefficients: walk generations G-1 .. 0 (+ms on rt1, -ms on rt2)
  c->coef.assign((size_t)r, 0.0);
  for (int g = G - 1; g >= 0; --g) {
    const int4 e = c->h_lineage[(size_t)g];
    if (e.y >= 0) {
      float ms;
      memcpy(&ms, &e.w, sizeof ms);
      c->coef[(size_t)e.y] += (double)ms;
      c->coef[(size_t)e.z] -= (double)ms;
    }
  }
  std::vector<int> terms;
  std::vector<double> tc;
  for (int k = 0; k < r; ++k)
    if (c->coef[(size_t)k] != 0.0) {
      terms.push_back(k);
      tc.push_back(c->coef[(size_t)k]);
    }
  c->n_terms = (int)terms.size();
  if (c->n_terms > c->terms_cap || !c->d_terms) {
    dfree(c, c->d_terms);
    dfree(c, c->d_coef);
    const int cap = c->n_terms > 16 ? c->n_terms : 16;
    TRY(dalloc_n(c, &c->d_terms, (size_t)cap));
    TRY(dalloc_n(c, &c->d_coef, (size_t)cap));
    c->terms_cap = cap;
  }
  if (c->n_terms > 0) {
    CK(cudaMemcpyAsync(c->d_terms, terms.data(), sizeof(int) * terms.size(),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_coef, tc.data(), sizeof(double) * tc.size(), cudaMemcpyHostToDevice,
                       c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  c->model_gen = c->gen;
  return GSGP_OK;
}

extern "C" gsgp_status gsgp_best_trace(gsgp_ctx *c, gsgp_trace *out) {
  API_GUARD(c)
  if (!out || out->struct_size != sizeof(gsgp_trace))
    return fail(c, GSGP_E_INVALID, "gsgp_trace NULL or struct_size mismatch");
  if (c->state != 2) return fail(c, GSGP_E_STATE, "gsgp_best_trace before gsgp_init");
  if (with_crossover(c))
    return fail(c, GSGP_E_STATE,
                "a run with crossover has no ancestor-plus-coefficients model; gsgp_predict "
                "replays its trace");
  TRY(use_device(c));
  TRY(build_model(c));
  const int G = c->gen;
  out->best_slot = c->best_slot;
  out->best_train_rmse = c->best_tr;
  out->best_test_rmse = c->best_te;
  out->ancestor = c->ancestor;
  out->max_genes = c->Kp;
  out->n_generations = G;
  out->n_random_trees = c->cfg.n_random_trees;
  out->rt_max_genes = c->Kr;
  out->sigma_dtype = c->cfg.sigma_dtype;
  out->n_features = c->l;
  out->protect_eps = c->cfg.protect_eps;
  out->init_mode = c->cfg.init_mode;
  CK(cudaMemcpyAsync(&out->ancestor_length, c->P_len + c->ancestor, sizeof(int),
                     cudaMemcpyDeviceToHost, c->stream));
  if (out->ancestor_genes)
    CK(cudaMemcpyAsync(out->ancestor_genes, c->P_genes + (size_t)c->ancestor * c->Kp,
                       sizeof(int) * c->Kp, cudaMemcpyDeviceToHost, c->stream));
  if (out->ancestor_consts)
    CK(cudaMemcpyAsync(out->ancestor_consts, c->P_consts + (size_t)c->ancestor * c->Kp,
                       sizeof(float) * c->Kp, cudaMemcpyDeviceToHost, c->stream));
  const size_t r = (size_t)c->cfg.n_random_trees;
  if (out->rt_genes)
    CK(cudaMemcpyAsync(out->rt_genes, c->R_genes, sizeof(int) * r * c->Kr, cudaMemcpyDeviceToHost,
                       c->stream));
  if (out->rt_consts)
    CK(cudaMemcpyAsync(out->rt_consts, c->R_consts, sizeof(float) * r * c->Kr,
                       cudaMemcpyDeviceToHost, c->stream));
  if (out->rt_lengths)
    CK(cudaMemcpyAsync(out->rt_lengths, c->R_len, sizeof(int) * r, cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int g = 0; g < G; ++g) {
    const int4 e = c->h_lineage[(size_t)g];
    if (out->lineage_parent) out->lineage_parent[g] = e.x;
    if (out->lineage_rt1) out->lineage_rt1[g] = e.y;
    if (out->lineage_rt2) out->lineage_rt2[g] = e.z;
    if (out->lineage_ms) memcpy(&out->lineage_ms[g], &e.w, sizeof(float));
  }
  if (out->coef) memcpy(out->coef, c->coef.data(), sizeof(double) * r);
  return GSGP_OK;
  API_END(c)
}

static gsgp_status run_predict(gsgp_ctx *c, const float *X_dev_rows, int64_t n, double *y_dev) {
  const int64_t n_pad = (n + 3) / 4 * 4;
  float *Xt = nullptr;
  TRY(dalloc_n(c, &Xt, (size_t)c->l * n_pad));
  LAUNCH(1, launch_transpose(X_dev_rows, n, c->l, Xt, n_pad, 0, c->stream));
  PredictParams p{};
  p.X = Xt;
  p.n_pad = n_pad;
  p.n = n;
  p.anc_genes = prog_genes(c, true) + (size_t)c->ancestor * c->Kp;
  p.anc_consts = prog_consts(c, true) + (size_t)c->ancestor * c->Kp;
  int anc_len = 0;
  CK(cudaMemcpyAsync(&anc_len, prog_len(c, true) + c->ancestor, sizeof(int), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  p.anc_len = anc_len;
  p.rt_genes = prog_genes(c, false);
  p.rt_consts = prog_consts(c, false);
  p.rt_len = prog_len(c, false);
  p.Kr = c->Kr;
  p.terms = c->d_terms;
  p.coef = c->d_coef;
  p.nk = c->n_terms;
  p.y = y_dev;
  p.protect_eps = c->cfg.protect_eps;
  p.sigma_bf16 = c->cfg.sigma_dtype == GSGP_SIGMA_BF16;
  LAUNCH(1, launch_predict(p, c->stream));
  dfree(c, Xt);
  return GSGP_OK;
}

// Runs with crossover: replay the generations on the new cases (float64).
// Only the ancestors of the best slot are replayed: a backward pass over the
// trace (host) lists, for every generation, the slots whose values a later
// listed slot reads (one parent for a mutation or copy, two for a
// crossover); under tournament selection that is about a quarter of the
// population, and a handful of slots in the last generations.
static gsgp_status run_predict_replay(gsgp_ctx *c, const float *X_dev_rows, int64_t n,
                                      double *y_dev) {
  const int m = c->cfg.pop_size, r = c->cfg.n_random_trees, G = c->gen;
  const int64_t n_pad = (n + 3) / 4 * 4;
  if ((int64_t)G * m > (int64_t)INT32_MAX)   // slot lists are indexed with 32 bits
    return fail(c, GSGP_E_INVALID, "trace of %d generations x %d slots too long to replay", G, m);
  struct Bufs {
    gsgp_ctx *c;
    float *Xt = nullptr;
    double *S0 = nullptr, *S1 = nullptr, *Sr = nullptr;
    int *slots = nullptr, *off = nullptr;
    ~Bufs() {
      dfree(c, Xt);
      dfree(c, S0);
      dfree(c, S1);
      dfree(c, Sr);
      dfree(c, slots);
      dfree(c, off);
    }
  } b{c};
  DevState st{};
  std::vector<int4> tr((size_t)G * m);
  CK(cudaMemcpyAsync(&st, c->dstate, sizeof st, cudaMemcpyDeviceToHost, c->stream));
  if (G > 0)
    CK(cudaMemcpyAsync(tr.data(), c->trace, sizeof(int4) * tr.size(), cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (st.best_slot < 0 || st.best_slot >= m) return fail(c, GSGP_E_STATE, "no best slot");
  // backward: need[i] = slot i's value at generation g is read later
  std::vector<std::vector<int>> lists((size_t)G);
  std::vector<char> need((size_t)m, 0), prev((size_t)m);
  need[(size_t)st.best_slot] = 1;
  for (int g = G - 1; g >= 0; --g) {
    std::fill(prev.begin(), prev.end(), 0);
    std::vector<int> &lg = lists[(size_t)g];
    for (int i = 0; i < m; ++i) {
      if (!need[(size_t)i]) continue;
      lg.push_back(i);
      const int4 e = tr[(size_t)g * m + i];
      const int p2 = (e.y >= 0 && e.z <= -2) ? -2 - e.z : -1;
      if (e.x < 0 || e.x >= m || (e.y >= r) || (e.y >= 0 && p2 < 0 && (e.z < 0 || e.z >= r)) ||
          p2 >= m)
        return fail(c, GSGP_E_STATE, "corrupt trace entry at generation %d, slot %d", g, i);
      prev[(size_t)e.x] = 1;
      if (p2 >= 0) prev[(size_t)p2] = 1;
    }
    need.swap(prev);
  }
  std::vector<int> flat, off((size_t)G + 1, 0);
  for (int g = 0; g < G; ++g) {
    flat.insert(flat.end(), lists[(size_t)g].begin(), lists[(size_t)g].end());
    off[(size_t)g + 1] = (int)flat.size();
  }
  TRY(dalloc_n(c, &b.Xt, (size_t)c->l * n_pad));
  TRY(dalloc_n(c, &b.S0, (size_t)m * n_pad));
  TRY(dalloc_n(c, &b.Sr, (size_t)r * n_pad));
  TRY(dalloc_n(c, &b.slots, flat.size() ? flat.size() : 1));
  TRY(dalloc_n(c, &b.off, off.size()));
  if (!flat.empty())
    CK(cudaMemcpyAsync(b.slots, flat.data(), sizeof(int) * flat.size(), cudaMemcpyHostToDevice,
                       c->stream));
  CK(cudaMemcpyAsync(b.off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice,
                     c->stream));
  LAUNCH(1, launch_transpose(X_dev_rows, n, c->l, b.Xt, n_pad, 0, c->stream));
  LAUNCH(1, launch_eval_pool(prog_genes(c, true), prog_consts(c, true), prog_len(c, true), c->Kp,
                             m, b.Xt, n_pad, n, b.S0, c->cfg.protect_eps, 0, c->stream));
  LAUNCH(1, launch_eval_pool(prog_genes(c, false), prog_consts(c, false), prog_len(c, false),
                             c->Kr, r, b.Xt, n_pad, n, b.Sr, c->cfg.protect_eps,
                             c->cfg.sigma_dtype == GSGP_SIGMA_BF16 ? 2 : 1, c->stream));
  // one case per CTA measured fastest (more CTAs resident per SM; 2-8 cases
  // per CTA were 1-4% slower on 1024-slot pools)
  const int lt = replay_tile_log2(m, r) >= 0 ? 0 : -1;
  if (lt >= 0) {   // every generation in one launch, the values in shared memory
    LAUNCH(1, launch_replay_tiles(c->trace, b.slots, b.off, G, m, r, b.S0, b.Sr, n_pad, n,
                                  st.best_slot, y_dev, lt, c->stream));
  } else {   // pools too large for shared memory: one launch per generation
    TRY(dalloc_n(c, &b.S1, (size_t)m * n_pad));
    double *cur = b.S0, *nxt = b.S1;
    for (int g = 0; g < G; ++g) {
      LAUNCH(1, launch_replay(c->trace + (size_t)g * m, b.slots + off[(size_t)g],
                              off[(size_t)g + 1] - off[(size_t)g], cur, nxt, b.Sr, n_pad, n,
                              c->stream));
      std::swap(cur, nxt);
    }
    CK(cudaMemcpyAsync(y_dev, cur + (size_t)st.best_slot * n_pad, sizeof(double) * (size_t)n,
                       cudaMemcpyDeviceToDevice, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));   // the host lists above are read by the copies
  return GSGP_OK;
}

extern "C" gsgp_status gsgp_predict(gsgp_ctx *c, const float *X, int64_t n, double *y_out) {
  API_GUARD(c)
  if (c->state != 2) return fail(c, GSGP_E_STATE, "gsgp_predict before gsgp_init");
  if (n < 0 || (n > 0 && (!X || !y_out))) return fail(c, GSGP_E_INVALID, "bad predict arguments");
  if (n == 0) return GSGP_OK;
  TRY(use_device(c));
  struct Bufs {
    gsgp_ctx *c;
    float *Xd = nullptr;
    double *yd = nullptr;
    ~Bufs() {
      dfree(c, Xd);
      dfree(c, yd);
    }
  } b{c};
  TRY(dalloc_n(c, &b.Xd, (size_t)n * c->l));
  TRY(dalloc_n(c, &b.yd, (size_t)n));
  TRY(stage_h2d(c, b.Xd, X, sizeof(float) * (size_t)n * c->l));
  // the cases are checked on the device once copied
  if (!c->d_flag) TRY(dalloc_n(c, &c->d_flag, 1));
  CK(cudaMemsetAsync(c->d_flag, 0, sizeof(unsigned), c->stream));
  LAUNCH(1, launch_nonfinite_check(b.Xd, n * c->l, c->d_flag, c->stream));
  unsigned bad = 0;
  CK(cudaMemcpyAsync(&bad, c->d_flag, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (bad) return fail(c, GSGP_E_INVALID, "non-finite value in X");
  if (!with_crossover(c)) TRY(build_model(c));
  if (with_crossover(c))
    TRY(run_predict_replay(c, b.Xd, n, b.yd));
  else
    TRY(run_predict(c, b.Xd, n, b.yd));
  CK(cudaMemcpyAsync(y_out, b.yd, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_predict_device(gsgp_ctx *c, const float *X, int64_t n,
                                           double *y_out) {
  API_GUARD(c)
  if (c->state != 2) return fail(c, GSGP_E_STATE, "gsgp_predict_device before gsgp_init");
  if (n < 0 || (n > 0 && (!X || !y_out))) return fail(c, GSGP_E_INVALID, "bad predict arguments");
  if (n == 0) return GSGP_OK;
  TRY(use_device(c));
  if (with_crossover(c)) {
    TRY(run_predict_replay(c, X, n, y_out));
    return GSGP_OK;
  }
  TRY(build_model(c));
  TRY(run_predict(c, X, n, y_out));
  return GSGP_OK;
  API_END(c)
}

// ---------------------------------------------------------- introspection --
extern "C" gsgp_status gsgp_get_info(gsgp_ctx *c, gsgp_info *out) {
  API_GUARD(c)
  if (!out || out->struct_size != sizeof(gsgp_info))
    return fail(c, GSGP_E_INVALID, "gsgp_info NULL or struct_size mismatch");
  out->state = c->state;
  out->n_features = c->l;
  out->n_train = c->n_tr;
  out->n_test = c->n_te;
  out->n_cases = c->N;
  out->n_cases_padded = c->n_pad;
  out->pop_size = c->cfg.pop_size;
  out->n_random_trees = c->cfg.n_random_trees;
  // row lengths of the program arrays: the genome length for linear genomes,
  // the full-tree size of the maximum depth for ramped half-and-half trees
  const bool linear = c->cfg.init_mode == GSGP_INIT_LINEAR;
  out->pop_max_genes = linear ? c->cfg.max_genes : (1 << (c->cfg.pop_max_depth + 1)) - 1;
  out->rt_max_genes = linear ? c->cfg.max_genes : (1 << (c->cfg.rt_max_depth + 1)) - 1;
  out->generation = c->gen;
  out->evolve_tile_cases = c->shape_ready ? gen_tile_cases(c->shape) : 0;
  out->evolve_offspring_per_cta = c->shape_ready ? c->shape.opb : 0;
  out->evolve_path = c->shape_ready ? c->path : 0;
  out->evolve_grid = c->shape_ready && c->path == 1 ? c->grid : 0;
  out->evolve_generations_per_launch =
      c->shape_ready ? (c->path == 1 ? kPersistGenerations : 1) : 0;
  out->kernel_launches = c->launches;
  out->device_bytes = c->dev_bytes;
  if (c->state == 2 && c->eval_genes[0] < 0) {   // trees: their lengths, counted once
    TRY(use_device(c));
    std::vector<int> lp((size_t)c->cfg.pop_size), lr((size_t)c->cfg.n_random_trees);
    CK(cudaMemcpyAsync(lp.data(), c->P_len, sizeof(int) * lp.size(), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaMemcpyAsync(lr.data(), c->R_len, sizeof(int) * lr.size(), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->eval_genes[0] = c->eval_genes[1] = 0;
    for (int v : lp) c->eval_genes[0] += v;
    for (int v : lr) c->eval_genes[1] += v;
  }
  out->pop_evaluated_genes = c->state == 2 ? c->eval_genes[0] : 0;
  out->rt_evaluated_genes = c->state == 2 ? c->eval_genes[1] : 0;
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_get_programs(gsgp_ctx *c, int32_t pool, int32_t *genes, float *consts,
                                         int32_t *lengths) {
  API_GUARD(c)
  if (c->state != 2) return fail(c, GSGP_E_STATE, "programs exist after gsgp_init");
  if (pool != GSGP_POOL_POPULATION && pool != GSGP_POOL_RANDOM)
    return fail(c, GSGP_E_INVALID, "unknown pool");
  TRY(use_device(c));
  const bool P = pool == GSGP_POOL_POPULATION;
  const size_t cnt = (size_t)(P ? c->cfg.pop_size : c->cfg.n_random_trees);
  const size_t K = (size_t)(P ? c->Kp : c->Kr);
  if (genes)
    CK(cudaMemcpyAsync(genes, P ? c->P_genes : c->R_genes, sizeof(int) * cnt * K,
                       cudaMemcpyDeviceToHost, c->stream));
  if (consts)
    CK(cudaMemcpyAsync(consts, P ? c->P_consts : c->R_consts, sizeof(float) * cnt * K,
                       cudaMemcpyDeviceToHost, c->stream));
  if (lengths)
    CK(cudaMemcpyAsync(lengths, P ? c->P_len : c->R_len, sizeof(int) * cnt,
                       cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_get_semantics(gsgp_ctx *c, int32_t pool, int32_t row0, int32_t rows,
                                          float *out) {
  API_GUARD(c)
  if (c->state != 2) return fail(c, GSGP_E_STATE, "semantics exist after gsgp_init");
  const bool P = pool == GSGP_POOL_POPULATION;
  if (!P && pool != GSGP_POOL_RANDOM) return fail(c, GSGP_E_INVALID, "unknown pool");
  const int cnt = P ? c->cfg.pop_size : c->cfg.n_random_trees;
  if (row0 < 0 || rows < 0 || row0 + rows > cnt || (rows > 0 && !out))
    return fail(c, GSGP_E_INVALID, "row range out of bounds");
  if (rows == 0) return GSGP_OK;
  TRY(use_device(c));
  const size_t N = (size_t)c->N;
  if (P) {
    const int m = c->cfg.pop_size;
    std::vector<int> rowmap((size_t)rows);
    const size_t par = (size_t)(c->gen & 1);
    CK(cudaMemcpyAsync(rowmap.data(), c->perm + par * 2 * m + row0, sizeof(int) * rows,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < rows; ++k)
      CK(cudaMemcpyAsync(out + (size_t)k * N, c->pool + (size_t)rowmap[(size_t)k] * c->n_pad,
                         sizeof(float) * N, cudaMemcpyDeviceToHost, c->stream));
  } else if (c->cfg.sigma_dtype == GSGP_SIGMA_F32) {
    CK(cudaMemcpy2DAsync(out, sizeof(float) * N, static_cast<float *>(c->sigR) + (size_t)row0 * c->n_pad,
                         sizeof(float) * c->n_pad, sizeof(float) * N, (size_t)rows,
                         cudaMemcpyDeviceToHost, c->stream));
  } else {
    std::vector<uint16_t> h((size_t)rows * N);
    CK(cudaMemcpy2DAsync(h.data(), 2 * N,
                         static_cast<uint16_t *>(c->sigR) + (size_t)row0 * c->n_pad, 2 * c->n_pad,
                         2 * N, (size_t)rows, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k < h.size(); ++k) {
      const uint32_t bits = (uint32_t)h[k] << 16;
      memcpy(out + k, &bits, sizeof(float));
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_get_fitness(gsgp_ctx *c, double *train, double *test) {
  API_GUARD(c)
  if (c->state != 2) return fail(c, GSGP_E_STATE, "fitness exists after gsgp_init");
  TRY(use_device(c));
  const size_t m = (size_t)c->cfg.pop_size;
  const size_t par = (size_t)(c->gen & 1);
  if (train)
    CK(cudaMemcpyAsync(train, c->fit + par * m, sizeof(double) * m, cudaMemcpyDeviceToHost,
                       c->stream));
  if (test)
    CK(cudaMemcpyAsync(test, c->fit_te + par * m, sizeof(double) * m, cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_get_trace(gsgp_ctx *c, int32_t g0, int32_t count, int32_t *parent,
                                      int32_t *rt1, int32_t *rt2, float *ms) {
  API_GUARD(c)
  if (c->state != 2) return fail(c, GSGP_E_STATE, "trace exists after gsgp_init");
  if (g0 < 0 || count < 0 || g0 + count > c->gen)
    return fail(c, GSGP_E_INVALID, "generation range out of bounds");
  if (count == 0) return GSGP_OK;
  TRY(use_device(c));
  const size_t m = (size_t)c->cfg.pop_size;
  std::vector<int4> h((size_t)count * m);
  CK(cudaMemcpyAsync(h.data(), c->trace + (size_t)g0 * m, sizeof(int4) * h.size(),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (size_t k = 0; k < h.size(); ++k) {
    if (parent) parent[k] = h[k].x;
    if (rt1) rt1[k] = h[k].y;
    if (rt2) rt2[k] = h[k].z;
    if (ms) memcpy(ms + k, &h[k].w, sizeof(float));
  }
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_set_kernel_timing(gsgp_ctx *c, int32_t enabled) {
  API_GUARD(c)
  c->timing = enabled != 0;
  c->ev_used = 0;
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_kernel_times(gsgp_ctx *c, float *ms, int32_t cap, int32_t *n_out) {
  API_GUARD(c)
  if (cap < 0 || (cap > 0 && !ms)) return fail(c, GSGP_E_INVALID, "bad output buffer");
  int n = 0;
  if (c->ev_used > 0) {
    TRY(use_device(c));
    CK(cudaStreamSynchronize(c->stream));
    const int first = c->ev_used > cap ? c->ev_used - cap : 0;
    for (int k = first; k < c->ev_used; ++k) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, c->ev0[(size_t)k], c->ev1[(size_t)k]));
      ms[n++] = t;
    }
  }
  c->ev_used = 0;
  if (n_out) *n_out = n;
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_init_kernel_times(gsgp_ctx *c, float *ms) {
  API_GUARD(c)
  if (!ms) return fail(c, GSGP_E_INVALID, "ms must hold 2 floats");
  if (!c->init_timed)
    return fail(c, GSGP_E_STATE, "the last gsgp_init ran without kernel timing");
  TRY(use_device(c));
  CK(cudaEventSynchronize(c->ev_init[3]));
  CK(cudaEventElapsedTime(&ms[0], c->ev_init[0], c->ev_init[1]));
  CK(cudaEventElapsedTime(&ms[1], c->ev_init[2], c->ev_init[3]));
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_rng_words(uint64_t seed, uint32_t run, uint32_t gp,
                                      uint32_t individual, int32_t n_words, uint32_t *out,
                                      void *stream) {
  if (n_words < 0 || (n_words > 0 && !out)) return GSGP_E_INVALID;
  if (n_words == 0) return GSGP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t *d = nullptr;
  if (cudaMallocAsync((void **)&d, sizeof(uint32_t) * (size_t)n_words, s) != cudaSuccess) {
    cudaGetLastError();
    return GSGP_E_OOM;
  }
  cudaError_t e = launch_rng_words(make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)),
                                   run, gp, individual, n_words, d, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, d, sizeof(uint32_t) * (size_t)n_words, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GSGP_E_CUDA;
  }
  return GSGP_OK;
}

extern "C" void gsgp_destroy(gsgp_ctx *c) {
  if (!c) return;
  if (c->device >= 0) {
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_graph(c);
    free_run_buffers(c);
    dfree(c, c->X);
    dfree(c, c->t);
    dfree(c, c->d_flag);
    // anything an interrupted call left behind (an error between its
    // allocation and its release)
    for (const auto &kv : c->allocs) {
      if (c->cfg.alloc)
        c->cfg.free(c->cfg.alloc_user, kv.first, c->stream);
      else
        cudaFreeAsync(kv.first, c->stream);
    }
    c->allocs.clear();
    for (auto e : c->ev0) cudaEventDestroy(e);
    for (auto e : c->ev_marks) cudaEventDestroy(e);
    for (auto e : c->ev1) cudaEventDestroy(e);
    for (auto e : c->ev_init)
      if (e) cudaEventDestroy(e);
    cudaStreamSynchronize(c->stream);
    if (c->mem_pool) cudaMemPoolDestroy(c->mem_pool);   // every block is back: its memory goes too
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    cudaGetLastError();
  }
  delete c;
}
