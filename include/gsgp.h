/*
 * gsgp.h - C ABI of the GB300 (sm_103a) Geometric Semantic GP library.
 *
 * The library runs the data-parallel hot path of GSGP for symbolic
 * regression (Trujillo et al., "GSGP-CUDA: a CUDA framework for Geometric
 * Semantic Genetic Programming", Sec. 2 and Algorithm 1) on one GPU:
 *   - program generation for the population P and the random-tree pool R,
 *   - interpretation of every program over all fitness cases (semantics),
 *   - per generation: tournament selection, geometric semantic mutation
 *     offspring = parent + ms * (sigma(R_a) - sigma(R_b)) over the semantic
 *     vectors, fused with the training and test RMSE of every offspring,
 *     survival with elitism and an ancestry trace on the device,
 *   - reconstruction of the best individual from the trace and its
 *     evaluation on new cases.
 *
 * Conventions shared by every call:
 *   - Every call returns a gsgp_status; nothing throws or aborts across the
 *     ABI.  On failure the context keeps a message (gsgp_last_error) and
 *     stays destroyable.  GSGP_E_CUDA means a CUDA runtime error.
 *   - Inputs are copied: the caller keeps ownership of every pointer it
 *     passes.  Outputs go to caller-allocated buffers.
 *   - Host pointers are ordinary (pageable or pinned) CPU memory.  Device
 *     pointers are CUDA global memory of the context's device.
 *   - All device work is ordered on config.stream (a cudaStream_t; NULL
 *     means the legacy default stream).  Calls that return host data
 *     synchronise that stream before returning.
 *   - Call order: create -> load -> init -> evolve* -> best_trace / predict.
 *     init may be called again to restart the run; load again to replace
 *     the data (then init).  Out-of-order calls return GSGP_E_STATE.
 *   - A context is not thread-safe; distinct contexts are independent.
 *
 * Randomness: Philox4x32-10 (Salmon et al., SC'11), key = (seed low 32 bits,
 * seed high 32 bits), counter = (block, individual, generation-or-purpose,
 * run).  Initialisation streams use 0x80000000 | purpose (1 = population,
 * 2 = random trees); generation g uses g.  Identical draws are reproduced by
 * an independent CPU implementation.
 */
#ifndef GSGP_H
#define GSGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsgp_ctx gsgp_ctx;

typedef enum {
  GSGP_OK = 0,
  GSGP_E_INVALID = 1,  /* bad argument, size, configuration or non-finite input */
  GSGP_E_STATE = 2,    /* call out of order (e.g. evolve before init) */
  GSGP_E_OOM = 3,      /* device or host allocation failed */
  GSGP_E_CUDA = 4,     /* CUDA runtime error; message in gsgp_last_error */
  GSGP_E_TIMEOUT = 5,  /* a bounded device-side wait gave up */
  GSGP_E_NUMERIC = 6   /* numerical failure (reserved) */
} gsgp_status;

/* Gene encoding of the linear (postfix) program representation (Sec. 2.2,
 * "Initialization"): function set {+, -, x, protected /}; terminals are
 * input features and ephemeral random constants.  A gene is an int32:
 * GSGP_OP_ADD..GSGP_OP_DIV are functions; GSGP_OP_CONST takes its value from
 * the parallel float array; GSGP_OP_VAR | (f << 8) reads feature f;
 * GSGP_GENE_PAD (-1) fills a program's row after its last gene. */
enum {
  GSGP_OP_ADD = 0,
  GSGP_OP_SUB = 1,
  GSGP_OP_MUL = 2,
  GSGP_OP_DIV = 3,   /* protected: |b| < protect_eps gives 1 */
  GSGP_OP_CONST = 4,
  GSGP_OP_VAR = 5,
  GSGP_GENE_PAD = -1
};

enum { GSGP_SIGMA_F32 = 0, GSGP_SIGMA_BF16 = 1 };

/* Program representation of P and R.
 *   GSGP_INIT_RHH: ramped half-and-half trees emitted in postfix order,
 *     depths from the config (the default).
 *   GSGP_INIT_LINEAR: the paper's fixed-length linear genomes (Sec. 2.2,
 *     "Initialization"): max_genes genes, each independently a function,
 *     a feature or a constant with weights 0.8 : 0.14 : 0.04.  The
 *     interpreter skips a function that finds fewer than two operands and
 *     returns register Out, the last function output ("Interpreter"); a
 *     genome whose stack would exceed 32 entries is rejected by gsgp_init
 *     (GSGP_E_INVALID). */
enum { GSGP_INIT_RHH = 0, GSGP_INIT_LINEAR = 1 };

/* Geometric semantic crossover (the GSGP crossover the paper names beside
 * mutation, Sec. 2; its experiments use probability 0, the default): with
 * probability p_crossover an offspring is R * T1 + (1 - R) * T2 case by case,
 * R = sigma of a random tree, T1 and T2 two tournament winners, computed as
 * T2 + R (T1 - T2) in float32.  Its trace entry is (parent 1, mask tree,
 * -2 - parent 2, 0).  Runs with crossover have no ancestor-plus-coefficients
 * model (gsgp_best_trace returns GSGP_E_STATE); gsgp_predict then replays
 * the trace on the new cases in float64, for the ancestors of the best slot
 * only (the trace is copied to the host once per call to list them).  The
 * TMA-staged stream shapes do not support crossover. */
enum { GSGP_POOL_POPULATION = 0, GSGP_POOL_RANDOM = 1 };

/* Optional device allocator.  alloc returns device memory of at least
 * `bytes` bytes usable on `stream` (NULL on failure -> GSGP_E_OOM); free
 * releases it.  When NULL the library allocates stream-ordered
 * (cudaMallocFromPoolAsync / cudaFreeAsync) from a memory pool the context
 * creates on its device: memory the context frees (the staging buffers of
 * gsgp_load and gsgp_predict, the temporaries of gsgp_init) stays mapped in
 * that pool for its later calls, and the pool with all of its memory goes
 * at gsgp_destroy. */
typedef void *(*gsgp_alloc_fn)(void *user, size_t bytes, void *stream);
typedef void (*gsgp_free_fn)(void *user, void *ptr, void *stream);

typedef struct {
  uint32_t struct_size;        /* = sizeof(gsgp_config); ABI versioning */
  uint64_t seed;               /* Philox key */
  uint32_t run;                /* Philox counter word 3: independent runs */
  int32_t pop_size;            /* m, 2 .. 65536 */
  int32_t n_random_trees;      /* r, 1 .. 65536 */
  int32_t pop_min_depth, pop_max_depth;  /* ramped half-and-half depths, 0..10 */
  int32_t rt_min_depth, rt_max_depth;
  float const_lo, const_hi;    /* ephemeral random constants in [lo, hi) */
  float p_grow_function;       /* grow method: P(function) below the root */
  float p_feature_given_terminal; /* P(feature) for a terminal; else constant */
  float protect_eps;           /* protected division threshold (strict <) */
  float ms;                    /* mutation step */
  int32_t ms_mode;             /* 0: fixed ms; 1: ms * U[0,1) per mutation */
  int32_t tournament_size;     /* 0: slot i mutates parent i (no selection) */
  int32_t elitism;             /* 1: keep the best of parents and offspring */
  int32_t sigma_dtype;         /* GSGP_SIGMA_F32 or GSGP_SIGMA_BF16 storage of sigma(R) */
  int32_t init_mode;           /* GSGP_INIT_RHH or GSGP_INIT_LINEAR (see below) */
  int32_t max_genes;           /* GSGP_INIT_LINEAR: genome length k, 1 .. 4095 */
  float p_crossover;           /* probability of geometric semantic crossover (see below) */
  void *stream;                /* cudaStream_t for all device work */
  gsgp_alloc_fn alloc;         /* optional device allocator (see above) */
  gsgp_free_fn free;
  void *alloc_user;
} gsgp_config;

/* Fill *cfg with defaults: seed 1, run 0, m = 1024, r = 1024, depths 2-6,
 * constants in [-1, 1), p_grow 0.5, p_feature 7/9, protect_eps 1e-3,
 * ms 0.1 fixed, tournament 4, elitism on, float32 sigma, ramped
 * half-and-half programs (max_genes 127 for linear genomes), no crossover,
 * NULL stream and allocator.  No CUDA call. */
void gsgp_config_default(gsgp_config *cfg);

/* Reason *cfg would be rejected by gsgp_create, or "" when it is valid.
 * Static string; no CUDA call. */
const char *gsgp_config_error(const gsgp_config *cfg);

/* Validate *cfg and create a context (host memory only; no CUDA call).
 * Errors: GSGP_E_INVALID (NULL pointers, struct_size mismatch, sizes or
 * probabilities out of range), GSGP_E_OOM. */
gsgp_status gsgp_create(const gsgp_config *cfg, gsgp_ctx **out);

/* Fitness cases (Sec. 2: fc_j = (x_j, t_j), x_j in R^l) from HOST memory in
 * the paper's file layout (Sec. 3.3): X_* row-major (cases x n_features)
 * float32, y_* one float32 target per case.  Training cases drive selection;
 * test cases (n_test may be 0, pointers then NULL) are evaluated for every
 * individual.  The library copies them to the device, stored feature-major.
 * Values are checked for NaN / Inf on the device after the copy; a rejected
 * call leaves the previously loaded data in place.  Synchronises the stream.
 * Errors: GSGP_E_INVALID (n_train < 1, n_features < 1 or > 65535,
 * NULL data, any non-finite value), GSGP_E_OOM, GSGP_E_CUDA. */
gsgp_status gsgp_load(gsgp_ctx *ctx, const float *X_train, const float *y_train,
                      int64_t n_train, int32_t n_features, const float *X_test,
                      const float *y_test, int64_t n_test);

/* As gsgp_load with DEVICE pointers (same layouts).  Non-finite values are
 * detected on the device (GSGP_E_INVALID). */
gsgp_status gsgp_load_device(gsgp_ctx *ctx, const float *X_train, const float *y_train,
                             int64_t n_train, int32_t n_features, const float *X_test,
                             const float *y_test, int64_t n_test);

/* Initialisation of Algorithm 1: CreatePopulation for P (m programs) and R
 * (r programs), ComputeSemantics of both over all cases (random trees
 * wrapped by the logistic function, Sec. 2), ComputeFitness of P.  Resets
 * the generation counter and the trace.  Diagnostic: with the environment
 * variable GSGP_INTERP_GENERAL set to a nonzero integer, the interpreter
 * evaluates every program with its general loop (stack pointer and skip
 * rule) instead of the precomputed stack schedule; the results are the same
 * bit for bit.  Errors: GSGP_E_STATE (no data), GSGP_E_OOM, GSGP_E_CUDA. */
gsgp_status gsgp_init(gsgp_ctx *ctx);

/* Errors of every call that synchronises after device work also include
 * GSGP_E_TIMEOUT: a bounded wait of the persistent generation kernel gave up
 * (never expected; the run must be restarted with gsgp_init). */

/* ---- Case sharding -----------------------------------------------------------
 *
 * The paper notes that large datasets need the semantic matrix partitioned
 * (Sec. 2.2, "Fitness computation"); every step of a generation is
 * independent per fitness case except the squared-error sums of the RMSE.
 * A problem of n_train_all + n_test_all cases (training cases first, as in
 * gsgp_load) can therefore be split into K shard contexts, one per GPU or
 * several on one GPU, each holding a contiguous slice of the cases:
 *
 *   shard k holds cases [case0_k, case0_(k+1)); case0_0 = 0; every case0 is
 *   a multiple of 1024 and every shard but the last holds a multiple of 1024
 *   cases.  Its gsgp_load gets exactly its slice: the slice's training cases
 *   (those below n_train_all) as X_train / y_train (possibly none) and its
 *   test cases as X_test / y_test.
 *
 * All shards share one gsgp_config (seed, run, sizes), so they generate the
 * same programs and draw the same selections and random trees.  Each shard
 * writes the (train, test) squared-error sum of every individual and every
 * 1024-case chunk it holds into a partial-sum array of pop_size x chunks
 * (double pairs, chunk c of the whole problem at column c), with zeros in
 * the other shards' columns.  Between a step and its completion the caller
 * replaces every shard's array by the element-wise sum over all shards (an
 * all-reduce; exact, since each element has one non-zero term).  The
 * completion then sums the chunks in the library's fixed order, so fitness,
 * every selection and survival decision, the trace and the semantics equal,
 * bit for bit, those of one unsharded context over all the cases.
 *
 *   gsgp_shard_configure (before gsgp_load) -> gsgp_load (the slice)
 *   -> gsgp_init -> [exchange] -> gsgp_shard_finish
 *   -> { gsgp_shard_generation -> [exchange] -> gsgp_shard_finish } * G
 *
 * The exchange must be ordered after the preceding call's work on the
 * context's stream and must complete before the next call's work starts
 * (e.g. an all-reduce queued on the same stream).  gsgp_evolve, checkpoints
 * and batches refuse shard contexts; gsgp_best_trace and gsgp_predict work
 * on any shard (the trace is the same on all). */

/* Make ctx (created, no data loaded yet) shard `case0` of a problem of
 * n_train_all training and n_test_all test cases.  Errors: GSGP_E_STATE
 * (data already loaded), GSGP_E_INVALID (case0 not a multiple of 1024 or
 * not below the case count, n_train_all < 1, n_test_all < 0). */
gsgp_status gsgp_shard_configure(gsgp_ctx *ctx, int64_t case0, int64_t n_train_all,
                                 int64_t n_test_all);

/* The device partial-sum array of the pending exchange: *partials receives
 * a DEVICE pointer to rows x chunks pairs of doubles (row-major, (train,
 * test) per chunk), owned by the context and valid until its next
 * gsgp_init; *rows = pop_size, *chunks = 1024-case chunks of the whole
 * problem.  Each output pointer may be NULL.  Errors: GSGP_E_STATE (not a
 * shard, or no exchange pending). */
gsgp_status gsgp_shard_partials(gsgp_ctx *ctx, double **partials, int64_t *rows,
                                int64_t *chunks);

/* Queue one generation's selection and mutation stream (Algorithm 1: GSM
 * and the squared errors of the offspring) on the shard's cases and leave
 * the partial sums for the exchange.  Does not synchronise.  Errors:
 * GSGP_E_STATE (not a shard, not initialised, or an exchange pending),
 * GSGP_E_OOM, GSGP_E_CUDA. */
gsgp_status gsgp_shard_generation(gsgp_ctx *ctx);

/* Complete the pending step from the exchanged partial sums: after
 * gsgp_init, the initial population's fitness; after gsgp_shard_generation,
 * the offspring's RMSE and survival with elitism (the generation counts from
 * here).  Does not synchronise.  Errors: GSGP_E_STATE (not a shard or
 * nothing pending), GSGP_E_CUDA. */
gsgp_status gsgp_shard_finish(gsgp_ctx *ctx);

/* Test hook of the GSGP_E_TIMEOUT path (the paper has no counterpart).  Arms,
 * for the next launch of the persistent generation kernel only (the next
 * gsgp_evolve on that path, after its shape was chosen), a bound of
 * spin_limit naps (1024 .. 2^24; the default bound is 2^24, about a second)
 * on every grid-barrier wait, and starts that launch's barrier arrival
 * counter one arrival short, as if one CTA never arrived at the first
 * barrier.  Every CTA's bounded wait there runs out, the sticky error word is
 * set, every CTA leaves the kernel (none passes the barrier), later launches
 * return at once, and the next call that synchronises (gsgp_evolve with a
 * log, gsgp_best_trace, ...) returns GSGP_E_TIMEOUT; gsgp_init clears it and
 * the context is usable again.  No kernel faults, traps or waits without
 * bound.  Errors: GSGP_E_INVALID (spin_limit out of range). */
gsgp_status gsgp_arm_barrier_fault(gsgp_ctx *ctx, uint32_t spin_limit);

/* Run `generations` generations of the loop of Algorithm 1 (GSM, fitness of
 * the offspring, survival with elitism), continuing from the current one.
 * best_train_rmse / best_test_rmse (nullable HOST arrays of `generations`
 * doubles) receive, per generation, the training and test RMSE of the best
 * individual after survival (the paper's two output series, Sec. 3.3);
 * when both are NULL the call does not synchronise.
 * Errors: GSGP_E_STATE (before init), GSGP_E_INVALID (generations < 0),
 * GSGP_E_OOM, GSGP_E_CUDA. */
gsgp_status gsgp_evolve(gsgp_ctx *ctx, int32_t generations, double *best_train_rmse,
                        double *best_test_rmse);

/* The best individual ("Return: best individual found", Algorithm 1) as a
 * model: its generation-0 ancestor in P plus one coefficient per random
 * tree, obtained by walking the ancestry trace back from the best slot
 * (each mutation adds +ms to rt1's coefficient and -ms to rt2's).  The model
 * is y(x) = P_ancestor(x) + sum_k coef[k] * q(sigma(R_k(x))), evaluated by
 * gsgp_predict in float64; with BF16 storage, q(sigma(R_k(x))) is the value
 * training used (R_k and the logistic in float32, rounded to bfloat16), with
 * float32 storage q is the identity.
 * Size query: set the pointer fields to NULL to receive only the sizes.
 * All pointers are HOST buffers owned by the caller. */
typedef struct {
  uint32_t struct_size;     /* in: sizeof(gsgp_trace) */
  int32_t best_slot;        /* out: population slot of the best individual */
  double best_train_rmse;   /* out */
  double best_test_rmse;    /* out */
  int32_t ancestor;         /* out: index of the ancestor in P */
  int32_t ancestor_length;  /* out: genes of the ancestor */
  int32_t max_genes;        /* out: row length of P programs */
  int32_t *ancestor_genes;  /* in/out, nullable: max_genes int32 */
  float *ancestor_consts;   /* in/out, nullable: max_genes float */
  int32_t n_generations;    /* out: length of the lineage (generations run) */
  int32_t *lineage_parent;  /* in/out, nullable: per generation g, the slot at g-1 */
  int32_t *lineage_rt1;     /* in/out, nullable: -1 for an elite copy */
  int32_t *lineage_rt2;
  float *lineage_ms;
  int32_t n_random_trees;   /* out: r */
  double *coef;             /* in/out, nullable: r coefficients */
  int32_t rt_max_genes;     /* out: row length of R programs */
  int32_t *rt_genes;        /* in/out, nullable: r * rt_max_genes */
  float *rt_consts;         /* in/out, nullable: r * rt_max_genes */
  int32_t *rt_lengths;      /* in/out, nullable: r */
  int32_t sigma_dtype;      /* out */
  int32_t n_features;       /* out: features of a case */
  float protect_eps;        /* out: protected division threshold */
  int32_t init_mode;        /* out: GSGP_INIT_RHH or GSGP_INIT_LINEAR */
} gsgp_trace;

/* Errors: GSGP_E_STATE (before init), GSGP_E_INVALID, GSGP_E_CUDA. */
gsgp_status gsgp_best_trace(gsgp_ctx *ctx, gsgp_trace *out);

/* Evaluate the best model (see gsgp_trace) in float64 on n new cases:
 * X row-major (n x n_features) float32 HOST, y_out n doubles HOST.
 * Errors: GSGP_E_STATE (before init), GSGP_E_INVALID (n < 0, NULL with
 * n > 0, non-finite X), GSGP_E_OOM, GSGP_E_CUDA. */
gsgp_status gsgp_predict(gsgp_ctx *ctx, const float *X, int64_t n, double *y_out);

/* As gsgp_predict with DEVICE pointers; does not synchronise. */
gsgp_status gsgp_predict_device(gsgp_ctx *ctx, const float *X, int64_t n, double *y_out);

/* Evaluate a model given as a filled gsgp_trace (as returned by
 * gsgp_best_trace, possibly saved and loaded again) on n new cases, with no
 * context: y = ancestor(x) + sum_k coef[k] * q(sigma(R_k(x))) in float64,
 * q as in gsgp_trace.  Uses ancestor_genes/consts/length, coef, rt_genes,
 * rt_consts, rt_lengths, max_genes, rt_max_genes, n_random_trees,
 * sigma_dtype, n_features and protect_eps of *model.  X is row-major
 * (n x n_features) float32 HOST, y_out n doubles HOST; device work runs on
 * `stream` (cudaStream_t, NULL = legacy default) of the current device and
 * the call synchronises it.  err_msg (nullable, err_cap bytes) receives a
 * message on failure.  Errors: GSGP_E_INVALID (NULL or inconsistent fields,
 * non-finite X, a program needing more than 32 stack entries), GSGP_E_OOM,
 * GSGP_E_CUDA. */
gsgp_status gsgp_model_predict(const gsgp_trace *model, const float *X, int64_t n, double *y_out,
                               void *stream, char *err_msg, size_t err_cap);

/* Checkpoint of a run after any number of generations: the current
 * population's semantics and fitness, the generation counter and best slot,
 * the trace and the best-of-generation log, with the configuration fields
 * that shape the search and a hash of the targets.  buf (HOST, cap bytes)
 * receives it; buf = NULL only reports the size in *size_out.
 * Errors: GSGP_E_STATE (before init), GSGP_E_INVALID (cap too small),
 * GSGP_E_CUDA, GSGP_E_TIMEOUT. */
gsgp_status gsgp_checkpoint(gsgp_ctx *ctx, void *buf, size_t cap, size_t *size_out);

/* Resume a checkpointed run in ctx, which holds the same configuration and
 * the same loaded data: re-runs the initialisation (programs and random-tree
 * semantics are functions of the configuration and data) and installs the
 * saved state, so that further gsgp_evolve calls continue bit for bit as the
 * original run would have.  Errors: GSGP_E_STATE (no data loaded),
 * GSGP_E_INVALID (not a checkpoint, another configuration or other data,
 * corrupt sizes), GSGP_E_OOM, GSGP_E_CUDA. */
gsgp_status gsgp_restore(gsgp_ctx *ctx, const void *buf, size_t size);

/* Last error message of ctx ("" if none); valid until the next call. */
const char *gsgp_last_error(const gsgp_ctx *ctx);

/* Release every resource of ctx (NULL is ignored).  Synchronises its stream. */
void gsgp_destroy(gsgp_ctx *ctx);

/* ---- Introspection: sizes, programs, semantics, fitness, trace ----------- */

typedef struct {
  uint32_t struct_size;     /* in: sizeof(gsgp_info) */
  int32_t state;            /* 0 created, 1 loaded, 2 initialised */
  int32_t n_features;
  int64_t n_train, n_test, n_cases;   /* n_cases = n_train + n_test */
  int64_t n_cases_padded;             /* row stride of semantic matrices */
  int32_t pop_size, n_random_trees;
  int32_t pop_max_genes, rt_max_genes;
  int32_t generation;                 /* generations run since init */
  int32_t evolve_tile_cases;          /* cases per tile of the mutation stream (0 before
                                         the first gsgp_evolve chose a shape) */
  int32_t evolve_offspring_per_cta;
  int32_t evolve_path;                /* GSGP_PATH_PERSISTENT or GSGP_PATH_CHAINED */
  int32_t evolve_grid;                /* CTAs of the persistent kernel */
  int32_t evolve_generations_per_launch;
  int64_t kernel_launches;            /* library kernels launched since create */
  int64_t device_bytes;               /* device memory held by the context */
  int64_t pop_evaluated_genes;        /* genes the interpreter applies per case over P and R: */
  int64_t rt_evaluated_genes;         /* the live code of linear genomes, else all genes */
} gsgp_info;

gsgp_status gsgp_get_info(gsgp_ctx *ctx, gsgp_info *out);

/* Programs of a pool (GSGP_POOL_POPULATION or GSGP_POOL_RANDOM) as
 * generated by init: genes/consts HOST (count x max_genes), lengths HOST
 * (count).  Any pointer may be NULL. */
gsgp_status gsgp_get_programs(gsgp_ctx *ctx, int32_t pool, int32_t *genes, float *consts,
                              int32_t *lengths);

/* Semantic vectors of rows [row0, row0 + rows) over all n_cases cases, as
 * float32 into HOST out (rows x n_cases): the current population
 * (GSGP_POOL_POPULATION, slot order) or the sigma-wrapped random trees
 * (GSGP_POOL_RANDOM; BF16 storage is widened exactly). */
gsgp_status gsgp_get_semantics(gsgp_ctx *ctx, int32_t pool, int32_t row0, int32_t rows,
                               float *out);

/* Training and test RMSE of the current population (HOST, m doubles each;
 * either may be NULL). */
gsgp_status gsgp_get_fitness(gsgp_ctx *ctx, double *train, double *test);

/* Trace entries of generations [g0, g0 + count): HOST arrays of count * m,
 * generation-major; rt1 = rt2 = -1 and ms = 0 mark an elite copy. */
gsgp_status gsgp_get_trace(gsgp_ctx *ctx, int32_t g0, int32_t count, int32_t *parent,
                           int32_t *rt1, int32_t *rt2, float *ms);

/* How generations run on the device.
 *   GSGP_PATH_PERSISTENT: one cooperative kernel runs up to 64 generations
 *     per launch, its CTAs resident throughout and synchronised by grid-wide
 *     barriers (3 per generation); the default where cooperative launch is
 *     available.
 *   GSGP_PATH_CHAINED: three launches per generation (selection, mutation
 *     stream, fitness + survival) chained with programmatic dependent launch
 *     and replayed from a CUDA graph.
 * Both produce bit-identical results.  The shape of the mutation stream is
 * (vec, opb): a tile of 1024 * vec cases for opb offspring per CTA
 * (persistent: vec in {1,2} with opb in {1,2,4,8,16} streams through
 * registers -- with vec 1, and with vec 2 and bf16 sigma, the next
 * offspring's rows are loaded while the current one is computed; (2, 2) is
 * sized for six CTAs per SM instead of four --, vec in {1,2,4} with opb = 0
 * stages rows in shared memory with TMA bulk
 * copies, one offspring per unit; chained: vec in {1,2,4}, opb in {2,4,8}).
 * path 0 chooses the path; vec = opb = 0 (the default)
 * times every register-stream shape of the path (one generation each) on
 * the first gsgp_evolve of a problem layout and keeps the fastest for the
 * process; the TMA-staged shapes run only when set explicitly.  Results do
 * not depend on the path or the shape.  Errors: GSGP_E_INVALID. */
enum { GSGP_PATH_AUTO = 0, GSGP_PATH_PERSISTENT = 1, GSGP_PATH_CHAINED = 2 };
gsgp_status gsgp_set_evolve_shape(gsgp_ctx *ctx, int32_t path, int32_t vec, int32_t opb);

/* Timing of the generation kernel.  When enabled, gsgp_evolve records CUDA
 * events on config.stream right before and after every launch of the
 * dominant kernel: the persistent kernel (one launch per up to 64
 * generations, see gsgp_info.evolve_generations_per_launch) or, on the
 * chained path, the mutation stream kernel of each generation.
 * gsgp_kernel_times then synchronises and returns the durations (ms) of the
 * most recent min(cap, n) launches, oldest first, and clears them.  *n_out
 * receives the count. */
gsgp_status gsgp_set_kernel_timing(gsgp_ctx *ctx, int32_t enabled);
gsgp_status gsgp_kernel_times(gsgp_ctx *ctx, float *ms, int32_t cap, int32_t *n_out);

/* With kernel timing enabled, gsgp_init also records events around its two
 * interpreter launches (ComputeSemantics of P, then of R);
 * gsgp_init_kernel_times synchronises and writes their durations in ms to
 * HOST ms[0], ms[1].  Errors: GSGP_E_STATE (the last init was not timed),
 * GSGP_E_INVALID. */
gsgp_status gsgp_init_kernel_times(gsgp_ctx *ctx, float *ms);

/* Philox4x32-10 words [0, n_words) of the stream (individual,
 * gen_or_purpose, run) under key `seed`, computed on the GPU on `stream` and
 * copied to HOST `out`.  Errors: GSGP_E_INVALID, GSGP_E_CUDA. */
gsgp_status gsgp_rng_words(uint64_t seed, uint32_t run, uint32_t gen_or_purpose,
                           uint32_t individual, int32_t n_words, uint32_t *out,
                           void *stream);

/* ---- Batched runs ----------------------------------------------------------
 *
 * Several independent runs, each its own context (data, sizes, parameters,
 * random trees, state), evolved together.  The paper evolves one run at a
 * time and repeats runs from a host loop (Sec. 3.3); a batch advances all of
 * its runs by the same number of generations with one persistent cooperative
 * kernel launch per up to 64 generations (captured once in a CUDA graph and
 * replayed) over the flattened work of all runs: selection of every run's
 * offspring, the mutation stream over every run's case tiles, every
 * offspring's RMSE, then survival per run.  A run evolved in a batch is
 * bit-identical to the same run evolved alone with gsgp_evolve, and every
 * single-run call (evolve, best_trace, predict, get_*) keeps working on it
 * between batch calls.
 *
 * The batch does not own its runs: they must outlive it.  A run may be
 * re-loaded or re-initialised between batch calls (the batch reads each
 * run's sizes and buffers at every gsgp_batch_evolve), but must then be
 * initialised again before the next one. */
typedef struct gsgp_batch gsgp_batch;

/* Group `count` (1 .. 1024) distinct initialised runs on one device, all
 * with the same sigma_dtype.  The batch's device work is ordered on
 * runs[0]'s config.stream; each gsgp_batch_evolve first waits for the work
 * already queued on every run's stream and then makes every run's stream
 * wait for the batch.  Allocates a few bytes of device memory per run.
 * Errors: GSGP_E_INVALID (NULL, count out of range, a run given twice,
 * mixed devices or sigma dtypes), GSGP_E_STATE (a run not initialised),
 * GSGP_E_OOM, GSGP_E_CUDA. */
gsgp_status gsgp_batch_create(gsgp_ctx *const *runs, int32_t count, gsgp_batch **out);

/* Advance every run of the batch by `generations` generations, each from its
 * own current generation.  best_train_rmse / best_test_rmse (nullable HOST
 * arrays of count * generations doubles, run-major) receive per run what
 * gsgp_evolve would return; when both are NULL the call does not
 * synchronise.  The first call times every supported shape on one
 * generation of the whole batch (state restored) unless a shape was set.
 * Errors: GSGP_E_STATE (a run not initialised), GSGP_E_INVALID, GSGP_E_OOM,
 * GSGP_E_CUDA, GSGP_E_TIMEOUT (then every run must be re-initialised). */
gsgp_status gsgp_batch_evolve(gsgp_batch *batch, int32_t generations, double *best_train_rmse,
                              double *best_test_rmse);

/* Shape of the batch's mutation stream: tiles of 1024 * vec cases for opb
 * offspring per CTA, vec in {1, 2} with opb in {1, 2, 4}, or vec 1 with opb 8;
 * (0, 0), the default, autotunes.  Results do not depend on the shape.
 * Errors: GSGP_E_INVALID. */
gsgp_status gsgp_batch_set_shape(gsgp_batch *batch, int32_t vec, int32_t opb);

/* Kernel timing of the batch, as gsgp_set_kernel_timing / gsgp_kernel_times:
 * one duration per launch (up to 64 generations of every run). */
gsgp_status gsgp_batch_set_kernel_timing(gsgp_batch *batch, int32_t enabled);
gsgp_status gsgp_batch_kernel_times(gsgp_batch *batch, float *ms, int32_t cap, int32_t *n_out);

typedef struct {
  uint32_t struct_size;            /* in: sizeof(gsgp_batch_info) */
  int32_t runs;
  int32_t tile_cases;              /* 1024 * vec (0 before the first evolve chose a shape) */
  int32_t offspring_per_cta;       /* opb */
  int32_t grid;                    /* CTAs of the batched kernel */
  int32_t generations_per_launch;
  int32_t graph;                   /* 1: full launches replay a captured CUDA graph */
  int64_t offspring;               /* sum over runs of m */
  int64_t updates_per_generation;  /* sum over runs of m * n_cases */
  int64_t items_per_generation;    /* stream items of all runs in the chosen shape */
  int64_t kernel_launches;         /* batched-kernel launches since create */
} gsgp_batch_info;

gsgp_status gsgp_batch_get_info(gsgp_batch *batch, gsgp_batch_info *out);

/* Last error message of the batch ("" if none). */
const char *gsgp_batch_last_error(const gsgp_batch *batch);

/* Release the batch (NULL is ignored); its runs are not touched.
 * Synchronises the batch's stream. */
void gsgp_batch_destroy(gsgp_batch *batch);

/* ---- Allocation-free mutation + fitness -----------------------------------
 *
 * The paper has no counterpart to this call; it exists for callers that can
 * not allocate device memory (code running while a framework captures a CUDA
 * graph and forbids cudaMalloc, plug-ins given a fixed device budget by their
 * host application, request paths that must not touch the allocator).  It
 * applies one generation's geometric semantic mutation to m offspring and
 * returns their RMSE, using only the caller's buffers plus a built-in scratch
 * area (per-chunk partial sums) that the library keeps in a static device
 * array of 2 MiB, held by every GPU that loads the library until exit.
 *
 *   offspring[i][j] = parents[parent[i]][j] + ms[i] * (sigma_r[rt1[i]][j] - sigma_r[rt2[i]][j])
 *   rmse_train[i]   = RMSE over cases [0, n_train), rmse_test[i] over the next n_test
 *
 * All pointers are DEVICE memory of the current device.  Row-major matrices
 * share the row stride ld (floats; a multiple of 4, >= n_train + n_test); the
 * row buffers and target are 16-byte aligned and target holds ld floats.
 * parent / rt1 / rt2 index rows of parents / sigma_r (not checked).  Work is
 * queued on `stream` (cudaStream_t; NULL = legacy default stream); the call
 * does not synchronise.  It calls no cudaMalloc/cudaFree and no allocating
 * library routine.  Limit: m * ceil((n_train + n_test) / 1024) <= 131072 and
 * m, ceil(n / 1024) <= 65535; larger sizes return GSGP_E_INVALID.
 *
 * offspring must not overlap parents, sigma_r or target: the call reads those
 * while it writes the offspring, so an in-place call (offspring == parents)
 * would race; an input that starts inside the m offspring rows is refused.
 *
 * The first call on a device, and the first call in a context the library has
 * not seen on that device (for example after cudaDeviceReset), looks up the
 * scratch array's device address (cudaGetSymbolAddress) with that device
 * current and caches it per context; make that first call before any stream
 * capture.  Every call shares the one scratch array: calls that overlap on
 * the GPU (for example on two streams) race and must be serialised by the
 * caller.  Nothing in the scratch needs clearing between calls: each call
 * writes every partial it reads.  The offspring and RMSE equal bit for bit
 * what gsgp_evolve computes for the same draws (same per-case arithmetic,
 * same summation order).
 *
 * err_msg (nullable, err_cap bytes) receives a message on failure.
 * Errors: GSGP_E_INVALID (sizes, NULL, misaligned or overlapping pointers),
 * GSGP_E_CUDA. */
gsgp_status gsgp_mutate_noalloc(const float *parents, const float *sigma_r, int64_t ld,
                                const float *target, int64_t n_train, int64_t n_test,
                                const int32_t *parent, const int32_t *rt1, const int32_t *rt2,
                                const float *ms, int32_t m, float *offspring, double *rmse_train,
                                double *rmse_test, void *stream, char *err_msg, size_t err_cap);

#ifdef __cplusplus
}
#endif

#endif /* GSGP_H */
