// Returning the best individual (Algorithm 1, "Return: best individual
// found"): the ancestry walk over the device trace and the float64
// evaluation of the rebuilt model on new cases.
#include "kernels.cuh"

namespace gsgp {

// Walk the trace back from the best slot: entry (g, slot) names the slot of
// generation g-1 it came from.  One thread; the trace of a run is small and
// L2-resident.
__global__ void lineage_kernel(const int4 *__restrict__ trace, int m, int G,
                               const DevState *__restrict__ state, int4 *__restrict__ lineage,
                               int *__restrict__ ancestor) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int slot = state->best_slot;
  for (int g = G - 1; g >= 0; --g) {
    const int4 e = trace[(size_t)g * m + slot];
    lineage[g] = e;
    slot = e.x;
  }
  *ancestor = slot;
}

cudaError_t launch_lineage(const int4 *trace, int m, int G, const DevState *state, int4 *lineage,
                           int *ancestor, cudaStream_t s) {
  lineage_kernel<<<1, 32, 0, s>>>(trace, m, G, state, lineage, ancestor);
  return cudaGetLastError();
}

// Float64 postfix evaluation of one program on case j (protected division:
// |b| < eps gives 1; a function short of operands is skipped).
__device__ double eval_program64(const int *__restrict__ genes, const float *__restrict__ consts,
                                 int len, const float *__restrict__ X, int64_t n_pad, int64_t j,
                                 double eps) {
  double st[kMaxDepth + 2];
  int sp = 0;
  for (int k = 0; k < len; ++k) {
    const int g = genes[k];
    const int op = g & 0xFF;
    if (op == kOpVar) {
      if (sp < kMaxDepth + 2) st[sp++] = (double)X[(int64_t)(g >> 8) * n_pad + j];
    } else if (op == kOpConst) {
      if (sp < kMaxDepth + 2) st[sp++] = (double)consts[k];
    } else if (sp >= 2) {
      const double b = st[sp - 1];
      const double a = st[sp - 2];
      double r;
      switch (op) {
        case kOpAdd: r = a + b; break;
        case kOpSub: r = a - b; break;
        case kOpMul: r = a * b; break;
        default: r = fabs(b) < eps ? 1.0 : a / b; break;
      }
      st[sp - 2] = r;
      --sp;
    }
  }
  return sp ? st[sp - 1] : 0.0;
}

// Float32 evaluation of one program on case j with the interpreter's
// arithmetic (one rounding per operation, protected division on the float
// divisor), so that sigma of a random tree comes out bit-identical to the
// value the interpreter stored during initialisation.
__device__ float eval_program32(const int *__restrict__ genes, const float *__restrict__ consts,
                                int len, const float *__restrict__ X, int64_t n_pad, int64_t j,
                                float eps) {
  float st[kMaxDepth + 2];
  int sp = 0;
  for (int k = 0; k < len; ++k) {
    const int g = genes[k];
    const int op = g & 0xFF;
    if (op == kOpVar) {
      if (sp < kMaxDepth + 2) st[sp++] = X[(int64_t)(g >> 8) * n_pad + j];
    } else if (op == kOpConst) {
      if (sp < kMaxDepth + 2) st[sp++] = consts[k];
    } else if (sp >= 2) {
      const float b = st[sp - 1];
      const float a = st[sp - 2];
      float r;
      switch (op) {
        case kOpAdd: r = a + b; break;
        case kOpSub: r = a - b; break;
        case kOpMul: r = a * b; break;
        default: r = fabsf(b) < eps ? 1.0f : a / b; break;
      }
      st[sp - 2] = r;
      --sp;
    }
  }
  return sp ? st[sp - 1] : 0.0f;
}

// y(x) = ancestor(x) + sum_k coef_k * q(sigma(R_k(x))) in float64.  With
// float32 storage q is the identity and the programs are evaluated in
// float64.  With bf16 storage q(sigma(R_k(x))) is the value training used:
// R_k evaluated in float32, the logistic in float32, rounded to bf16
// (nearest-even), so the rebuilt model reproduces the training semantics.
__global__ void __launch_bounds__(128) predict_kernel(const PredictParams p) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.n) return;
  const double eps = (double)p.protect_eps;
  double y = eval_program64(p.anc_genes, p.anc_consts, p.anc_len, p.X, p.n_pad, j, eps);
  for (int q = 0; q < p.nk; ++q) {
    const int k = p.terms[q];
    double sg;
    if (p.sigma_bf16) {
      const float v = eval_program32(p.rt_genes + (size_t)k * p.Kr, p.rt_consts + (size_t)k * p.Kr,
                                     p.rt_len[k], p.X, p.n_pad, j, p.protect_eps);
      sg = (double)__bfloat162float(__float2bfloat16_rn(1.0f / (1.0f + expf(-v))));
    } else {
      const double v = eval_program64(p.rt_genes + (size_t)k * p.Kr,
                                      p.rt_consts + (size_t)k * p.Kr, p.rt_len[k], p.X, p.n_pad, j,
                                      eps);
      sg = 1.0 / (1.0 + exp(-v));
    }
    y += p.coef[q] * sg;
  }
  p.y[j] = y;
}

cudaError_t launch_predict(const PredictParams &p, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  predict_kernel<<<(unsigned)((p.n + 127) / 128), 128, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace gsgp
