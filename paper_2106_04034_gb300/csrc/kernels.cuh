// Host-side launchers of the GSGP kernels (each returns the CUDA launch error).
#pragma once

#include "common.cuh"

namespace gsgp {

// Block-wide arg-min / arg-max with the first index winning ties.
constexpr int kFinalThreads = 256;

cudaError_t launch_treegen(int count, int dmin, int dmax, int K, int n_features, uint2 key,
                           uint32_t run, uint32_t purpose, float p_grow, float p_feature,
                           float const_lo, float const_hi, int *genes, float *consts,
                           int *lengths, cudaStream_t s);

// The paper's linear genomes (fixed length K) for a pool, and the deepest
// stack any program of a pool reaches (atomicMax into *out).
cudaError_t launch_genomes(int count, int K, int n_features, uint2 key, uint32_t run,
                           uint32_t purpose, float const_lo, float const_hi, int *genes,
                           float *consts, int *lengths, cudaStream_t s);
cudaError_t launch_max_stack(const int *genes, const int *lengths, int count, int K, int *out,
                             cudaStream_t s);
// The live genes of each linear genome (the expression under register Out),
// in order: a postfix program with the same value, bit for bit.
cudaError_t launch_compact(const int *genes, const float *consts, const int *lengths, int count,
                           int K, int *out_genes, float *out_consts, int *out_len,
                           cudaStream_t s);

// Each "terminal, function" pair of a postfix program as one fused gene
// (kOpFusedConst / kOpFusedVar + function): the form the interpreter runs.
cudaError_t launch_fuse(const int *genes, const float *consts, const int *lengths, int count,
                        int K, int *out_genes, float *out_consts, int *out_len, cudaStream_t s);

// Stack entries each fused program needs below the cached top (need[i]).
cudaError_t launch_stack_need(const int *genes, const int *lengths, int count, int K, int *need,
                              cudaStream_t s);

cudaError_t launch_transpose(const float *in, int64_t n, int l, float *out, int64_t n_pad,
                             int64_t col0, cudaStream_t s);

cudaError_t launch_nonfinite_check(const float *v, int64_t n, unsigned *flag, cudaStream_t s);
// Device copy of page-locked host memory by kernel loads (src_mapped: the
// buffer's device-mapped address); both 16-byte aligned, bytes % 16 == 0.
cudaError_t launch_host_read(const void *src_mapped, void *dst, size_t bytes, cudaStream_t s);

// Floats of padding after the last feature row of X: the interpreter reads
// the second 1024-case chunk of a tile 4 KB after the first, also past the
// end of a row for a partial last tile (values it does not use).
constexpr int kXTailFloats = 1024;

// mode 0: population (float semantics + per-tile squared errors);
// mode 1: random trees, sigma stored float; mode 2: sigma stored bf16.
cudaError_t launch_interpret(int mode, const InterpParams &p, int count, cudaStream_t s);

cudaError_t launch_fitness_finalize(const double2 *partial, int tiles, int count, int n_train,
                                    int n_test, double *fit, double *fit_te, cudaStream_t s);

cudaError_t launch_init_state(int m, int *perm, const double *fit, DevState *state,
                              cudaStream_t s);

// Cases per tile and offspring per CTA of the stream kernel.
struct GenShape {
  int vec;   // float4 chunks per thread; tile = 1024 * vec cases
  int opb;   // offspring per CTA
};
int gen_tile_cases(const GenShape &sh);
bool gen_shape_supported(const GenShape &sh);
// One generation = select, stream, final on stream s; with pdl the launches
// may overlap their predecessor's tail (programmatic dependent launch).
cudaError_t launch_select(const GenParams &p, cudaStream_t s, bool pdl);
cudaError_t launch_stream(const GenParams &p, int sigma_bf16, const GenShape &sh, cudaStream_t s,
                          bool pdl);
cudaError_t launch_final(const GenParams &p, cudaStream_t s, bool pdl);

// Persistent cooperative generation kernel (k_persist.cu).
// Synchronisation words of the persistent kernel, each on its own 128-byte
// line: the sticky error word and the barrier arrival counter (zeroed before
// every launch).
constexpr int kSyncStride = 32;   // unsigned words per 128-byte line
struct GridSync {
  int err;                        // sticky: nonzero once a barrier wait gave up
  unsigned pad0[kSyncStride - 1];
  unsigned count;                 // barrier arrivals of the running launch
  unsigned pad1[kSyncStride - 1];
};
inline size_t grid_sync_bytes(int /*grid*/) { return sizeof(GridSync); }
// Naps (__nanosleep(64) plus one L2 round trip each) a barrier wait may
// spend before it gives up: about a second.
constexpr unsigned kSpinLimitDefault = 1u << 24;
struct PersistArgs {
  GridSync *gs;
  ulonglong2 *cta_min;   // [grid] (fitness key, index) arg-min of each CTA's offspring
  ulonglong2 *cta_max;   // [grid] (fitness key, index) arg-max
  int G;              // generations this launch runs
  unsigned spin_limit;   // bound of every barrier wait (kSpinLimitDefault)
};
bool persist_shape_supported(const GenShape &sh);
// Co-resident CTAs of the persistent kernel for this shape (0: no cooperative launch).
int persist_max_grid(int sigma_bf16, const GenShape &sh);
cudaError_t launch_persist(const GenParams &p, const PersistArgs &x, int sigma_bf16,
                           const GenShape &sh, int grid, cudaStream_t s);

// Batched persistent kernel (k_batch.cu): up to kBatchRunsPerLaunch
// independent runs advance G generations in one cooperative launch.  The
// runs' generation parameters and the offsets of their offspring and stream
// items (tiles of 1024 * vec cases x groups of opb offspring) in the
// flattened work lists travel in the kernel's parameter block, so that the
// kernel reads them, as the single-run kernel reads its GenParams, through
// the constant cache (uniform per CTA) instead of holding them in registers.
constexpr int kBatchRunsPerLaunch = 160;   // keeps the parameter block under 32 KB
struct BatchArgs {
  GenParams runs[kBatchRunsPerLaunch];
  int m_off[kBatchRunsPerLaunch + 1];      // ascending, m_off[0] = 0
  int item_off[kBatchRunsPerLaunch + 1];   // ascending, item_off[0] = 0
  GridSync *gs;
  int R;
  int G;
};
static_assert(sizeof(BatchArgs) < 32000, "kernel parameter block limit");
bool batch_shape_supported(const GenShape &sh);
int batch_max_grid(int sigma_bf16, const GenShape &sh);
cudaError_t launch_batch(const BatchArgs &a, int sigma_bf16, const GenShape &sh, int grid,
                         cudaStream_t s);

// Lineage of the best slot over G generations (k_predict.cu); jump holds
// ceil(G / lineage_segment(G)) * m ints and start ceil(G / L) ints of scratch.
int lineage_segment(int G);
cudaError_t launch_lineage(const int4 *trace, int m, int G, const DevState *state, int4 *lineage,
                           int *ancestor, int *jump, int *start, cudaStream_t s);

struct PredictParams {
  const float *X;      // [l][n_pad] feature-major new cases
  int64_t n_pad;
  int64_t n;
  const int *anc_genes;
  const float *anc_consts;
  int anc_len;
  const int *rt_genes;   // [r][Kr]
  const float *rt_consts;
  const int *rt_len;
  int Kr;
  const int *terms;      // [nk] random-tree indices with a nonzero coefficient
  const double *coef;    // [nk]
  int nk;
  double *y;             // [n]
  float protect_eps;
  int sigma_bf16;
};
cudaError_t launch_predict(const PredictParams &p, cudaStream_t s);

// Prediction by replaying the trace (k_predict.cu): float64 values of every
// program of a pool on new cases (mode 0 plain, 1 logistic, 2 the bf16
// sigma of training), and one generation's recorded operations on every slot.
cudaError_t launch_eval_pool(const int *genes, const float *consts, const int *lengths, int K,
                             int count, const float *X, int64_t n_pad, int64_t n, double *out,
                             float eps, int mode, cudaStream_t s);
// One generation's entries applied to the slots slots[0 .. count).
cudaError_t launch_replay(const int4 *entries, const int *slots, int count, const double *prev,
                          double *next, const double *sig, int64_t n_pad, int64_t n,
                          cudaStream_t s);
// All G generations in one launch, 2^lt cases per CTA held in shared memory,
// generation g computing slots[off[g] .. off[g + 1]); replay_tile_log2 gives
// the largest lt (at most 5) that fits, or -1.
int replay_tile_log2(int m, int r);
cudaError_t launch_replay_tiles(const int4 *entries, const int *slots, const int *off, int G,
                                int m, int r, const double *S0, const double *Sr, int64_t n_pad,
                                int64_t n, int best, double *y, int lt, cudaStream_t s);

cudaError_t launch_rng_words(uint2 key, uint32_t run, uint32_t gp, uint32_t individual,
                             int n_words, uint32_t *out, cudaStream_t s);

}  // namespace gsgp
