// Returning the best individual (Algorithm 1, "Return: best individual
// found"): the ancestry walk over the device trace and the float64
// evaluation of the rebuilt model on new cases.
#include "kernels.cuh"

namespace gsgp {

// Walk the trace back from the best slot: entry (g, slot) names the slot of
// generation g-1 it came from, so lineage[g] = trace[g][slot_g] with
// slot_{G-1} = best and slot_{g-1} = lineage[g].parent; the slot left after
// generation 0 is the ancestor in P.  The walk is a chain of G dependent
// loads; it is split into segments of L generations:
//   1. jump: for every segment s and every slot, the slot L generations
//      back (nseg * m independent walks of L steps);
//   2. one thread follows the jumps from the best slot (nseg steps) and
//      records the slot each segment starts from;
//   3. one thread per segment walks it (L steps) writing its lineage entries.
// Three chains of about sqrt(G) loads instead of one of G.
__global__ void lineage_jump_kernel(const int4 *__restrict__ trace, int m, int G, int L, int nseg,
                                    int *__restrict__ jump) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nseg * m) return;
  const int seg = (int)(t / m);
  int slot = (int)(t - (int64_t)seg * m);
  const int g0 = G - 1 - seg * L;
  const int g1 = g0 - L + 1 > 0 ? g0 - L + 1 : 0;
  for (int g = g0; g >= g1; --g) slot = __ldg(&trace[(size_t)g * m + slot]).x;
  jump[t] = slot;
}

__global__ void lineage_follow_kernel(const int *__restrict__ jump, int m, int nseg,
                                      const DevState *__restrict__ state, int *__restrict__ start,
                                      int *__restrict__ ancestor) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int slot = state->best_slot;
  for (int s = 0; s < nseg; ++s) {
    start[s] = slot;
    slot = jump[(size_t)s * m + slot];
  }
  *ancestor = slot;
}

__global__ void lineage_walk_kernel(const int4 *__restrict__ trace, int m, int G, int L, int nseg,
                                    const int *__restrict__ start, int4 *__restrict__ lineage) {
  const int seg = blockIdx.x * blockDim.x + threadIdx.x;
  if (seg >= nseg) return;
  int slot = start[seg];
  const int g0 = G - 1 - seg * L;
  const int g1 = g0 - L + 1 > 0 ? g0 - L + 1 : 0;
  for (int g = g0; g >= g1; --g) {
    const int4 e = __ldg(&trace[(size_t)g * m + slot]);
    lineage[g] = e;
    slot = e.x;
  }
}

int lineage_segment(int G) {
  int L = 8;
  while (L * L < G && L < 256) L *= 2;
  return L;
}

cudaError_t launch_lineage(const int4 *trace, int m, int G, const DevState *state, int4 *lineage,
                           int *ancestor, int *jump, int *start, cudaStream_t s) {
  if (G <= 0) {   // no generation: the ancestor is the best slot itself
    lineage_follow_kernel<<<1, 32, 0, s>>>(jump, m, 0, state, start, ancestor);
    return cudaGetLastError();
  }
  const int L = lineage_segment(G);
  const int nseg = (G + L - 1) / L;
  const int64_t jobs = (int64_t)nseg * m;
  lineage_jump_kernel<<<(unsigned)((jobs + 255) / 256), 256, 0, s>>>(trace, m, G, L, nseg, jump);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  lineage_follow_kernel<<<1, 32, 0, s>>>(jump, m, nseg, state, start, ancestor);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  lineage_walk_kernel<<<(nseg + 127) / 128, 128, 0, s>>>(trace, m, G, L, nseg, start, lineage);
  return cudaGetLastError();
}

// Evaluation of one program on case j with the interpreter's rules: a
// function short of operands is skipped, the value is register Out (the last
// function output), else the stack top, else 0.  Programs are checked at
// initialisation to need at most kMaxStack stack entries.
template <typename T>
__device__ __forceinline__ T eval_program(const int *__restrict__ genes,
                                          const float *__restrict__ consts, int len,
                                          const float *__restrict__ X, int64_t n_pad, int64_t j,
                                          T eps) {
  T st[kMaxStack];
  T out = T(0);
  bool applied = false;
  int sp = 0;
  for (int k = 0; k < len; ++k) {
    const int g = genes[k];
    const int op = g & 0xFF;
    if (op == kOpVar) {
      if (sp < kMaxStack) st[sp++] = (T)X[(int64_t)(g >> 8) * n_pad + j];
    } else if (op == kOpConst) {
      if (sp < kMaxStack) st[sp++] = (T)consts[k];
    } else if (sp >= 2) {
      const T b = st[sp - 1];
      const T a = st[sp - 2];
      T r;
      switch (op) {
        case kOpAdd: r = a + b; break;
        case kOpSub: r = a - b; break;
        case kOpMul: r = a * b; break;
        default: r = fabs(b) < eps ? T(1) : a / b; break;
      }
      st[sp - 2] = r;
      --sp;
      out = r;
      applied = true;
    }
  }
  return applied ? out : (sp ? st[sp - 1] : T(0));
}

// float64: the model's arithmetic.  float32: the interpreter's arithmetic
// (one rounding per operation, protected division on the float divisor), so
// that sigma of a random tree comes out bit-identical to the stored value.
__device__ double eval_program64(const int *genes, const float *consts, int len, const float *X,
                                 int64_t n_pad, int64_t j, double eps) {
  return eval_program<double>(genes, consts, len, X, n_pad, j, eps);
}
__device__ float eval_program32(const int *genes, const float *consts, int len, const float *X,
                                int64_t n_pad, int64_t j, float eps) {
  return eval_program<float>(genes, consts, len, X, n_pad, j, eps);
}

// y(x) = ancestor(x) + sum_k coef_k * q(sigma(R_k(x))) in float64.  With
// float32 storage q is the identity and the programs are evaluated in
// float64.  With bf16 storage q(sigma(R_k(x))) is the value training used:
// R_k evaluated in float32, the logistic in float32, rounded to bf16
// (nearest-even), so the rebuilt model reproduces the training semantics.
//
// A CTA takes 32 cases (one per lane) and its kPredWarps warps split the
// terms: warp w adds terms w, w + kPredWarps, ... in order, so every warp
// evaluates one program at a time for its 32 cases (uniform gene stream).
// The last warp also evaluates the ancestor.  The case's value is then the
// ancestor plus the warps' sums, added in warp order (a fixed order).
constexpr int kPredWarps = 16;

__global__ void __launch_bounds__(kPredWarps * 32) predict_kernel(const PredictParams p) {
  __shared__ double s_acc[kPredWarps][32];
  __shared__ double s_anc[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  const bool valid = j < p.n;
  const int64_t jj = valid ? j : 0;   // padding lanes evaluate case 0 and store nothing
  const double eps = (double)p.protect_eps;
  double acc = 0.0;
  for (int q = warp; q < p.nk; q += kPredWarps) {
    const int k = p.terms[q];
    double sg;
    if (p.sigma_bf16) {
      const float v = eval_program32(p.rt_genes + (size_t)k * p.Kr, p.rt_consts + (size_t)k * p.Kr,
                                     p.rt_len[k], p.X, p.n_pad, jj, p.protect_eps);
      sg = (double)__bfloat162float(__float2bfloat16_rn(1.0f / (1.0f + expf(-v))));
    } else {
      const double v = eval_program64(p.rt_genes + (size_t)k * p.Kr,
                                      p.rt_consts + (size_t)k * p.Kr, p.rt_len[k], p.X, p.n_pad, jj,
                                      eps);
      sg = 1.0 / (1.0 + exp(-v));
    }
    acc += p.coef[q] * sg;
  }
  if (warp == kPredWarps - 1)
    s_anc[lane] = eval_program64(p.anc_genes, p.anc_consts, p.anc_len, p.X, p.n_pad, jj, eps);
  s_acc[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && valid) {
    double y = s_anc[lane];
#pragma unroll
    for (int w = 0; w < kPredWarps; ++w) y += s_acc[w][lane];
    p.y[j] = y;
  }
}

// ---------------------------------------------------------------------------
// Prediction by replaying the trace (runs with crossover, whose model is not
// an ancestor plus coefficients): every program of a pool evaluated on the
// new cases in float64 (random trees wrapped by the logistic, or by the
// training's bf16 rounding), then each generation's recorded operation
// applied to every slot: copy (rt1 < 0), crossover (rt2 <= -2: R T1 +
// (1 - R) T2 with R = sigma(rt1)) or mutation (T + ms (sigma_a - sigma_b)).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
    eval_pool_kernel(const int *__restrict__ genes, const float *__restrict__ consts,
                     const int *__restrict__ lengths, int K, int count,
                     const float *__restrict__ X, int64_t n_pad, int64_t n,
                     double *__restrict__ out, float eps, int mode) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int prog = blockIdx.y; prog < count; prog += gridDim.y) {
    const int *g = genes + (size_t)prog * K;
    const float *c = consts + (size_t)prog * K;
    double v;
    if (mode == 2) {   // the training's bf16 sigma
      const float f = eval_program32(g, c, lengths[prog], X, n_pad, j, eps);
      v = (double)__bfloat162float(__float2bfloat16_rn(1.0f / (1.0f + expf(-f))));
    } else {
      v = eval_program64(g, c, lengths[prog], X, n_pad, j, (double)eps);
      if (mode == 1) v = 1.0 / (1.0 + exp(-v));
    }
    out[(size_t)prog * n_pad + j] = v;
  }
}

__global__ void __launch_bounds__(128)
    replay_kernel(const int4 *__restrict__ entries, const int *__restrict__ slots, int count,
                  const double *__restrict__ prev, double *__restrict__ next,
                  const double *__restrict__ sig, int64_t n_pad, int64_t n) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int k = blockIdx.y; k < count; k += gridDim.y) {
    const int i = slots[k];
    const int4 e = entries[i];
    const double t1 = prev[(size_t)e.x * n_pad + j];
    double v;
    if (e.y < 0) {
      v = t1;
    } else if (e.z <= -2) {
      const double rm = sig[(size_t)e.y * n_pad + j];
      v = __fma_rn(rm, t1, (1.0 - rm) * prev[(size_t)(-2 - e.z) * n_pad + j]);
    } else {
      const double ms = (double)__int_as_float(e.w);
      v = __fma_rn(ms, sig[(size_t)e.y * n_pad + j] - sig[(size_t)e.z * n_pad + j], t1);
    }
    next[(size_t)i * n_pad + j] = v;
  }
}

// The whole replay for a tile of 2^lt consecutive new cases in one CTA: the
// population's values ([slot][case], two buffers that alternate by
// generation) and the random trees' values of the tile stay in shared
// memory for all G generations; the slot lists and trace entries come from
// L2, where every CTA reads the same ones.  Generation g computes only the
// slots slots[off[g] .. off[g + 1]), the ancestors of the final slot `best`
// (a slot left out keeps a stale value that no later listed slot reads).
// The arithmetic is replay_kernel's, so both give the same bits.
__global__ void __launch_bounds__(256)
    replay_tile_kernel(const int4 *__restrict__ entries, const int *__restrict__ slots,
                       const int *__restrict__ off, int G, int m, int r,
                       const double *__restrict__ S0, const double *__restrict__ Sr,
                       int64_t n_pad, int64_t n, int best, double *__restrict__ y, int lt) {
  extern __shared__ double s_val[];
  const int T = 1 << lt, tm = T - 1;
  double *cur = s_val, *nxt = s_val + (size_t)m * T;
  double *sig = s_val + (size_t)2 * m * T;
  const int64_t j0 = (int64_t)blockIdx.x * T;
  const int tc = (int)(n - j0 < T ? n - j0 : T);   // cases of this tile
  for (int e = threadIdx.x; e < m * T; e += blockDim.x) {
    const int q = e & tm;
    cur[e] = q < tc ? S0[(size_t)(e >> lt) * n_pad + j0 + q] : 0.0;
  }
  for (int e = threadIdx.x; e < r * T; e += blockDim.x) {
    const int q = e & tm;
    sig[e] = q < tc ? Sr[(size_t)(e >> lt) * n_pad + j0 + q] : 0.0;
  }
  __syncthreads();
  for (int g = 0; g < G; ++g) {
    const int4 *eg = entries + (size_t)g * m;
    const int *lg = slots + __ldg(off + g);
    const int cnt = __ldg(off + g + 1) - __ldg(off + g);
    for (int e = threadIdx.x; e < (cnt << lt); e += blockDim.x) {
      const int q = e & tm;
      const int i = __ldg(lg + (e >> lt));
      const int4 en = __ldg(eg + i);
      const double t1 = cur[(en.x << lt) + q];
      double v;
      if (en.y < 0) {
        v = t1;
      } else if (en.z <= -2) {
        const double rm = sig[(en.y << lt) + q];
        v = __fma_rn(rm, t1, (1.0 - rm) * cur[((-2 - en.z) << lt) + q]);
      } else {
        const double ms = (double)__int_as_float(en.w);
        v = __fma_rn(ms, sig[(en.y << lt) + q] - sig[(en.z << lt) + q], t1);
      }
      nxt[(i << lt) + q] = v;
    }
    __syncthreads();
    double *t = cur;
    cur = nxt;
    nxt = t;
  }
  for (int q = threadIdx.x; q < tc; q += blockDim.x) y[j0 + q] = cur[(best << lt) + q];
}

int replay_tile_log2(int m, int r) {
  int dev = 0, smem = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return -1;
  const size_t per_case = (size_t)(2 * m + r) * sizeof(double);
  int lt = -1;
  while (lt < 5 && per_case << (lt + 1) <= (size_t)smem) ++lt;
  return lt;   // -1: not even one case fits
}

cudaError_t launch_replay_tiles(const int4 *entries, const int *slots, const int *off, int G,
                                int m, int r, const double *S0, const double *Sr, int64_t n_pad,
                                int64_t n, int best, double *y, int lt, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (lt < 0 || lt > 5) return cudaErrorInvalidValue;
  const size_t smem = ((size_t)(2 * m + r) * sizeof(double)) << lt;
  cudaError_t e = cudaFuncSetAttribute(replay_tile_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + (1 << lt) - 1) >> lt;
  replay_tile_kernel<<<(unsigned)tiles, 256, smem, s>>>(entries, slots, off, G, m, r, S0, Sr,
                                                        n_pad, n, best, y, lt);
  return cudaGetLastError();
}

cudaError_t launch_eval_pool(const int *genes, const float *consts, const int *lengths, int K,
                             int count, const float *X, int64_t n_pad, int64_t n, double *out,
                             float eps, int mode, cudaStream_t s) {
  if (count <= 0 || n <= 0) return cudaSuccess;
  const unsigned gy = (unsigned)(count < 65535 ? count : 65535);
  eval_pool_kernel<<<dim3((unsigned)((n + 127) / 128), gy), 128, 0, s>>>(
      genes, consts, lengths, K, count, X, n_pad, n, out, eps, mode);
  return cudaGetLastError();
}

cudaError_t launch_replay(const int4 *entries, const int *slots, int count, const double *prev,
                          double *next, const double *sig, int64_t n_pad, int64_t n,
                          cudaStream_t s) {
  if (count <= 0 || n <= 0) return cudaSuccess;
  const unsigned gy = (unsigned)(count < 65535 ? count : 65535);
  replay_kernel<<<dim3((unsigned)((n + 127) / 128), gy), 128, 0, s>>>(entries, slots, count, prev,
                                                                     next, sig, n_pad, n);
  return cudaGetLastError();
}

cudaError_t launch_predict(const PredictParams &p, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  predict_kernel<<<(unsigned)((p.n + 31) / 32), kPredWarps * 32, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace gsgp
