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
                     const int *__restrict__ lengths, int K, const float *__restrict__ X,
                     int64_t n_pad, int64_t n, double *__restrict__ out, float eps, int mode) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int prog = blockIdx.y;
  if (j >= n) return;
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

__global__ void __launch_bounds__(128)
    replay_kernel(const int4 *__restrict__ entries, const double *__restrict__ prev,
                  double *__restrict__ next, const double *__restrict__ sig, int64_t n_pad,
                  int64_t n) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= n) return;
  const int4 e = entries[i];
  const double t1 = prev[(size_t)e.x * n_pad + j];
  double v;
  if (e.y < 0) {
    v = t1;
  } else if (e.z <= -2) {
    const double rm = sig[(size_t)e.y * n_pad + j];
    v = rm * t1 + (1.0 - rm) * prev[(size_t)(-2 - e.z) * n_pad + j];
  } else {
    const double ms = (double)__int_as_float(e.w);
    v = t1 + ms * (sig[(size_t)e.y * n_pad + j] - sig[(size_t)e.z * n_pad + j]);
  }
  next[(size_t)i * n_pad + j] = v;
}

cudaError_t launch_eval_pool(const int *genes, const float *consts, const int *lengths, int K,
                             int count, const float *X, int64_t n_pad, int64_t n, double *out,
                             float eps, int mode, cudaStream_t s) {
  if (count <= 0 || n <= 0) return cudaSuccess;
  eval_pool_kernel<<<dim3((unsigned)((n + 127) / 128), (unsigned)count), 128, 0, s>>>(
      genes, consts, lengths, K, X, n_pad, n, out, eps, mode);
  return cudaGetLastError();
}

cudaError_t launch_replay(const int4 *entries, int m, const double *prev, double *next,
                          const double *sig, int64_t n_pad, int64_t n, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  replay_kernel<<<dim3((unsigned)((n + 127) / 128), (unsigned)m), 128, 0, s>>>(entries, prev, next,
                                                                            sig, n_pad, n);
  return cudaGetLastError();
}

cudaError_t launch_predict(const PredictParams &p, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  predict_kernel<<<(unsigned)((p.n + 31) / 32), kPredWarps * 32, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace gsgp
