// Initialisation kernels of Algorithm 1: CreatePopulation (program
// generation), ComputeSemantics (postfix interpretation over every fitness
// case) and ComputeFitness of the initial population, plus data staging.
#include <cstdlib>

#include "kernels.cuh"
#include "reduce.cuh"
#include "stream.cuh"

namespace gsgp {

// ---------------------------------------------------------------------------
// CreatePopulation: one thread per program, ramped half-and-half in postfix.
// Individual i of a pool with depths [dmin, dmax] (D = dmax - dmin + 1) gets
// depth dmin + i mod D and the "full" method when floor(i / D) is even, else
// "grow".  Nodes are decided in preorder from the individual's own Philox
// stream: below the target depth a node is a function under "full" or at the
// root, otherwise iff u24 < p_grow; a function draws its operator
// idx(w, 4); a terminal is a feature idx(w, l) iff u24 < p_feature, else a
// constant in [lo, hi).  Postfix order emits a function after both operand
// subtrees, which the explicit frame stack below tracks without recursion.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
    treegen_kernel(int count, int dmin, int dmax, int K, int n_features, uint2 key, uint32_t run,
                   uint32_t purpose, float p_grow, float p_feature, float lo, float hi,
                   int *__restrict__ genes, float *__restrict__ consts, int *__restrict__ lengths) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int D = dmax - dmin + 1;
  const int depth = dmin + i % D;
  const bool full = ((i / D) & 1) == 0;
  WordStream ws(key, (uint32_t)i, kInitFlag | purpose, run);
  int *g = genes + (size_t)i * K;
  float *c = consts + (size_t)i * K;
  int frame_op[kMaxDepth + 1];
  int frame_left[kMaxDepth + 1];   // operands still to be completed
  int sp = 0, d = 0, pos = 0;
  for (;;) {
    bool is_function;
    if (d == depth)
      is_function = false;
    else if (full || d == 0)
      is_function = true;
    else
      is_function = draw_u24(ws.next()) < p_grow;
    if (is_function) {
      frame_op[sp] = (int)draw_index(ws.next(), 4u);
      frame_left[sp] = 2;
      ++sp;
      ++d;
      continue;
    }
    if (draw_u24(ws.next()) < p_feature) {
      const int f = (int)draw_index(ws.next(), (uint32_t)n_features);
      g[pos] = kOpVar | (f << 8);
      c[pos] = 0.0f;
    } else {
      const float v = draw_const(ws.next(), lo, hi);
      g[pos] = kOpConst;
      c[pos] = v;
    }
    ++pos;
    // close every function whose second operand just completed
    while (sp > 0) {
      if (--frame_left[sp - 1] != 0) break;
      g[pos] = frame_op[sp - 1];
      c[pos] = 0.0f;
      ++pos;
      --sp;
    }
    if (sp == 0) break;
    d = sp;   // next: second operand of the innermost open function
  }
  lengths[i] = pos;
  for (int k = pos; k < K; ++k) {
    g[k] = kGenePad;
    c[k] = 0.0f;
  }
}

cudaError_t launch_treegen(int count, int dmin, int dmax, int K, int n_features, uint2 key,
                           uint32_t run, uint32_t purpose, float p_grow, float p_feature,
                           float const_lo, float const_hi, int *genes, float *consts,
                           int *lengths, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  treegen_kernel<<<(count + 127) / 128, 128, 0, s>>>(count, dmin, dmax, K, n_features, key, run,
                                                     purpose, p_grow, p_feature, const_lo,
                                                     const_hi, genes, consts, lengths);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CreatePopulation in the paper's representation (Sec. 2.2,
// "Initialization"): fixed-length linear genomes whose genes are drawn
// independently, a function with weight 0.8, a feature 0.14, a constant
// 0.04 (the printed probabilities, which add up to 0.98, as weights).  Gene j
// of individual i reads words 2j (class, u24 against the two cumulative
// thresholds) and 2j+1 (operator idx(w, 4), feature idx(w, l) or constant in
// [lo, hi)) of the individual's stream; one thread makes the two genes of
// one Philox block.
// ---------------------------------------------------------------------------
constexpr float kGenomePFunction = (float)(0.8 / 0.98);
constexpr float kGenomePFunctionOrFeature = (float)((0.8 + 0.14) / 0.98);

__global__ void __launch_bounds__(256)
    genome_kernel(int count, int K, int n_features, uint2 key, uint32_t run, uint32_t purpose,
                  float lo, float hi, int *__restrict__ genes, float *__restrict__ consts,
                  int *__restrict__ lengths) {
  const int pairs = (K + 1) / 2;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)count * pairs) return;
  const int i = (int)(t / pairs);
  const int q = (int)(t - (int64_t)i * pairs);
  const uint4 w = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)i, kInitFlag | purpose, run), key);
  const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = 2 * q + h;
    if (j >= K) break;
    const float u = draw_u24(words[2 * h]);
    const uint32_t c = words[2 * h + 1];
    int g;
    float v = 0.0f;
    if (u < kGenomePFunction) {
      g = (int)draw_index(c, 4u);
    } else if (u < kGenomePFunctionOrFeature) {
      g = kOpVar | ((int)draw_index(c, (uint32_t)n_features) << 8);
    } else {
      g = kOpConst;
      v = draw_const(c, lo, hi);
    }
    genes[(size_t)i * K + j] = g;
    consts[(size_t)i * K + j] = v;
  }
  if (q == 0) lengths[i] = K;
}

cudaError_t launch_genomes(int count, int K, int n_features, uint2 key, uint32_t run,
                           uint32_t purpose, float const_lo, float const_hi, int *genes,
                           float *consts, int *lengths, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int64_t threads = (int64_t)count * ((K + 1) / 2);
  genome_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
      count, K, n_features, key, run, purpose, const_lo, const_hi, genes, consts, lengths);
  return cudaGetLastError();
}

// Live code of a linear genome.  The value of a genome is Out, the output
// of the last function applied (or the stack top if none is applied); every
// other gene either is a function skipped for lack of operands or produces a
// value that never reaches Out.  Only the genes of the expression tree under
// that root matter, and in their original order they form a well-formed
// postfix program: a function's first operand is complete before its second
// is started (the stack is last-in first-out).  Evaluating that program
// applies the same operations to the same operands in the same order, so the
// result is bit-identical while skipped functions and dead values cost
// nothing.  One thread per genome: a forward pass marks the applied
// functions and finds the root, a backward pass from the root counts the
// values still needed (a terminal supplies one, an applied function supplies
// one and needs two) and marks the live genes, a last pass copies them.
// ---------------------------------------------------------------------------
constexpr int kMaskWords = (kMaxGenomeGenes + 31) / 32;

__global__ void __launch_bounds__(128)
    compact_kernel(const int *__restrict__ genes, const float *__restrict__ consts,
                   const int *__restrict__ lengths, int count, int K, int *__restrict__ out_genes,
                   float *__restrict__ out_consts, int *__restrict__ out_len) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int *g = genes + (size_t)i * K;
  const float *c = consts + (size_t)i * K;
  const int len = lengths[i];
  uint32_t applied[kMaskWords], live[kMaskWords];
  const int words = (len + 31) / 32;
  for (int w = 0; w < words; ++w) applied[w] = live[w] = 0u;
  int sp = 0, root = -1, last_terminal = -1;
  for (int k = 0; k < len; ++k) {
    const int op = g[k] & 0xFF;
    if (op >= kOpConst) {
      ++sp;
      last_terminal = k;
    } else if (sp >= 2) {
      --sp;
      applied[k >> 5] |= 1u << (k & 31);
      root = k;
    }
  }
  if (root < 0) root = last_terminal;   // no function applied: the stack top (or nothing)
  int need = root >= 0 ? 1 : 0;
  for (int k = root; k >= 0 && need > 0; --k) {
    const bool terminal = (g[k] & 0xFF) >= kOpConst;
    const bool app = (applied[k >> 5] >> (k & 31)) & 1u;
    if (terminal) {
      --need;
    } else if (app) {
      ++need;
    } else {
      continue;
    }
    live[k >> 5] |= 1u << (k & 31);
  }
  int *og = out_genes + (size_t)i * K;
  float *oc = out_consts + (size_t)i * K;
  int n = 0;
  for (int k = 0; k <= root; ++k) {
    if ((live[k >> 5] >> (k & 31)) & 1u) {
      og[n] = g[k];
      oc[n] = c[k];
      ++n;
    }
  }
  out_len[i] = n;
  for (int k = n; k < K; ++k) {
    og[k] = kGenePad;
    oc[k] = 0.0f;
  }
}

cudaError_t launch_compact(const int *genes, const float *consts, const int *lengths, int count,
                           int K, int *out_genes, float *out_consts, int *out_len,
                           cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (K > kMaxGenomeGenes) return cudaErrorInvalidValue;
  compact_kernel<<<(count + 127) / 128, 128, 0, s>>>(genes, consts, lengths, count, K, out_genes,
                                                      out_consts, out_len);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Terminal-operand fusion.  In postfix code a terminal followed by a
// function pushes the terminal and at once pops it again as the function's
// right operand; the pair is one step, "stack top := f(stack top, terminal)".
// Each such pair becomes one gene (kOpFusedConst / kOpFusedVar + f, with the
// terminal's feature index or constant), which spares the interpreter a
// dispatch and a shared-memory push and pop per pair.  The arithmetic is
// unchanged: the same operation on the same two operands.  On an empty
// stack the interpreter pushes the terminal and skips the function, as the
// unfused pair would.  One warp per program: lanes take 32 consecutive
// genes and place the kept ones by ballot.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool gene_is_terminal(int g) {
  return (g & 0xFF) == kOpConst || (g & 0xFF) == kOpVar;
}
__device__ __forceinline__ bool gene_is_function(int g) { return g >= 0 && (g & 0xFF) < kOpConst; }

__global__ void __launch_bounds__(128)
    fuse_kernel(const int *__restrict__ genes, const float *__restrict__ consts,
                const int *__restrict__ lengths, int count, int K, int *__restrict__ out_genes,
                float *__restrict__ out_consts, int *__restrict__ out_len) {
  const int prog = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (prog >= count) return;   // whole warps leave together
  const int *g = genes + (size_t)prog * K;
  const float *c = consts + (size_t)prog * K;
  int *og = out_genes + (size_t)prog * K;
  float *oc = out_consts + (size_t)prog * K;
  const int len = lengths[prog];
  int n = 0;
  for (int k0 = 0; k0 < len; k0 += 32) {
    const int k = k0 + lane;
    const bool in = k < len;
    const int gk = in ? g[k] : kGenePad;
    const int gnext = k + 1 < len ? g[k + 1] : kGenePad;
    const int gprev = in && k > 0 ? g[k - 1] : kGenePad;
    const bool drop = gene_is_terminal(gk) && gene_is_function(gnext);   // joins gene k + 1
    const bool fused = gene_is_function(gk) && gene_is_terminal(gprev);
    const unsigned keep = __ballot_sync(0xffffffffu, in && !drop);
    if (in && !drop) {
      const int pos = n + __popc(keep & ((1u << lane) - 1u));
      if (fused) {
        const int base = (gprev & 0xFF) == kOpVar ? kOpFusedVar : kOpFusedConst;
        og[pos] = (gprev & ~0xFF) | (base + (gk & 0xFF));
        oc[pos] = c[k - 1];
      } else {
        og[pos] = gk;
        oc[pos] = c[k];
      }
    }
    n += __popc(keep);
  }
  if (lane == 0) out_len[prog] = n;
}

cudaError_t launch_fuse(const int *genes, const float *consts, const int *lengths, int count,
                        int K, int *out_genes, float *out_consts, int *out_len, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  fuse_kernel<<<(unsigned)((count + 3) / 4), 128, 0, s>>>(genes, consts, lengths, count, K,
                                                         out_genes, out_consts, out_len);
  return cudaGetLastError();
}

// Shared-memory stack entries one fused program needs: the deepest stack
// it reaches under the interpreter's rules (a fused gene on a non-empty
// stack pushes nothing, a function short of operands is skipped) less the
// top, which lives in registers.  The interpreter groups programs by this
// need so that shallow programs run at a higher occupancy.
__global__ void __launch_bounds__(256)
    stack_need_kernel(const int *__restrict__ genes, const int *__restrict__ lengths, int count,
                      int K, int *__restrict__ need) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int *g = genes + (size_t)i * K;
  const int len = lengths[i];
  int sp = 0, best = 0;
  for (int k = 0; k < len; ++k) {
    const int op = g[k] & 0xFF;
    if (op >= kOpFusedConst && sp >= 1) continue;
    if (op >= kOpConst) {
      ++sp;
      best = max(best, sp);
    } else if (sp >= 2) {
      --sp;
    }
  }
  need[i] = best > 1 ? best - 1 : 0;
}

cudaError_t launch_stack_need(const int *genes, const int *lengths, int count, int K, int *need,
                              cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  stack_need_kernel<<<(count + 255) / 256, 256, 0, s>>>(genes, lengths, count, K, need);
  return cudaGetLastError();
}

// Deepest stack any program of a pool reaches under the interpreter's rule
// (a function short of operands is skipped): sizes the interpreter's shared
// memory stack.  One thread per program; *out must be zero before.
__global__ void __launch_bounds__(256)
    max_stack_kernel(const int *__restrict__ genes, const int *__restrict__ lengths, int count,
                     int K, int *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int *g = genes + (size_t)i * K;
  const int len = lengths[i];
  int sp = 0, best = 0;
  for (int k = 0; k < len; ++k) {
    const int op = g[k] & 0xFF;
    if (op >= kOpConst) {
      ++sp;
      best = max(best, sp);
    } else if (sp >= 2) {
      --sp;
    }
  }
  atomicMax(out, best);
}

cudaError_t launch_max_stack(const int *genes, const int *lengths, int count, int K, int *out,
                             cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  max_stack_kernel<<<(count + 255) / 256, 256, 0, s>>>(genes, lengths, count, K, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Row-major cases (n x l) -> feature-major X[f][col0 + j] through a padded
// 32 x 32 shared tile, so both the reads and the writes are coalesced.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
    transpose_kernel(const float *__restrict__ in, int64_t n, int l, float *__restrict__ out,
                     int64_t n_pad, int64_t col0) {
  __shared__ float tile[32][33];
  const int64_t j0 = (int64_t)blockIdx.x * 32;
  const int f0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int64_t j = j0 + k;
    const int f = f0 + threadIdx.x;
    if (j < n && f < l) tile[k][threadIdx.x] = in[j * l + f];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int f = f0 + k;
    const int64_t j = j0 + threadIdx.x;
    if (j < n && f < l) out[(int64_t)f * n_pad + col0 + j] = tile[threadIdx.x][k];
  }
}

cudaError_t launch_transpose(const float *in, int64_t n, int l, float *out, int64_t n_pad,
                             int64_t col0, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((l + 31) / 32));
  transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(in, n, l, out, n_pad, col0);
  return cudaGetLastError();
}

// Reads page-locked host memory (its device-mapped address) over the
// CPU-GPU link with plain loads and writes it to device memory: the staging
// copy of host inputs.  On GB300 the copy engines were measured to stall for
// ~40 ms on the first host-to-device copy that follows a long
// bandwidth-bound kernel (in a process started after other GPU work), while
// this kernel read the same 773 MB at the link's 211 GB/s every time.
// src and dst 16-byte aligned, bytes a multiple of 16.
__global__ void host_read_kernel(const float4 *__restrict__ src, float4 *__restrict__ dst,
                                 int64_t n4) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

cudaError_t launch_host_read(const void *src_mapped, void *dst, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  if (((uintptr_t)src_mapped | (uintptr_t)dst | bytes) & 15u) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t n4 = (int64_t)(bytes / 16);
  const int64_t need = (n4 + 255) / 256;
  const int64_t grid = need < (int64_t)sms * 4 ? need : (int64_t)sms * 4;
  host_read_kernel<<<(unsigned)grid, 256, 0, s>>>(static_cast<const float4 *>(src_mapped),
                                                  static_cast<float4 *>(dst), n4);
  return cudaGetLastError();
}

__global__ void nonfinite_kernel(const float *__restrict__ v, int64_t n, unsigned *flag) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(v[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1u);
}

cudaError_t launch_nonfinite_check(const float *v, int64_t n, unsigned *flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  nonfinite_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(v, n, flag);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ComputeSemantics (Sec. 2.2, "Interpreter"): the genome is read left to
// right with a LIFO stack; a terminal pushes, a function pops its operands
// and pushes its result.  One CTA interprets one program over a tile of 1024
// cases: every thread owns 4 consecutive cases (one float4 of each feature
// row), so the gene stream is uniform across the CTA and decoded once per
// 4 cases.  The top of the stack lives in registers; deeper entries live in
// shared memory laid out [slot][thread] (conflict-free 16-byte accesses).
// The programs arrive with their "terminal, function" pairs fused
// (fuse_kernel), which apply the function to the top and the terminal
// without touching shared memory.
// A function with fewer than two operands on the stack is skipped and the
// value is register Out, the last function output (the paper's rules; a
// ramped half-and-half program never skips and ends with its root).  Protected division
// returns 1 when |b| < eps.  Random trees are wrapped by the logistic
// function (Sec. 2) and stored as float or bf16.  For the population the
// CTA also reduces the squared errors of its tile (train and test cases) in
// the canonical chunk order (subblock_sum, chunk_total).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float apply_op(int op, float a, float b, float eps) {
  switch (op) {
    case kOpAdd: return a + b;
    case kOpSub: return a - b;
    case kOpMul: return a * b;
    default: return fabsf(b) < eps ? 1.0f : a / b;
  }
}

__device__ __forceinline__ float logistic(float v) { return 1.0f / (1.0f + expf(-v)); }

constexpr int kInterpThreads = 256;
constexpr int kInterpTile = kInterpThreads * 4;

// The values of one stack entry for the thread's VEC chunks (4 cases each).
template <int VEC>
struct Lanes {
  float4 v[VEC];
};

// One operation on the thread's 4 VEC cases, the operator decided once
// (warp-uniform).
template <int F, int VEC>
__device__ __forceinline__ Lanes<VEC> opv(const Lanes<VEC> &a, const Lanes<VEC> &b, float eps) {
  Lanes<VEC> r;
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    const float4 x = a.v[q], y = b.v[q];
    if (F == kOpAdd)
      r.v[q] = make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
    else if (F == kOpSub)
      r.v[q] = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
    else if (F == kOpMul)
      r.v[q] = make_float4(x.x * y.x, x.y * y.y, x.z * y.z, x.w * y.w);
    else
      r.v[q] = make_float4(apply_op(kOpDiv, x.x, y.x, eps), apply_op(kOpDiv, x.y, y.y, eps),
                           apply_op(kOpDiv, x.z, y.z, eps), apply_op(kOpDiv, x.w, y.w, eps));
  }
  return r;
}

// Decoded gene, general form: bits 0-1 the function, bit 2 a terminal
// operand (alone or fused), bit 3 the terminal is a feature, bit 4 a
// function (alone or fused); the argument is the feature row's offset in
// float4 units or the constant's bits.
constexpr int kDecFun = 16, kDecTerm = 4, kDecVar = 8;

__device__ __forceinline__ int2 decode_gene(int g, float c, int64_t row4) {
  const int op = g & 0xFF;
  if (op < kOpConst) return make_int2(kDecFun | op, 0);
  const bool var = op == kOpVar || op >= kOpFusedVar;
  const int code = kDecTerm | (var ? kDecVar : 0) | (op >= kOpFusedConst ? kDecFun | (op & 3) : 0);
  return make_int2(code, var ? (int)((g >> 8) * row4) : __float_as_int(c));
}

// Static form (bits 0-3 of the entry the loop reads; the general code sits in
// bits 4-8, the stack entry's offset in bytes in bits 12-31, i.e. in float4
// units from bit 16).  The
// stack depth before every gene of a program is fixed by the program, so the
// decoding pass resolves it once and the loop keeps no stack pointer:
//   kStFv + f   top := f(top, feature)        kStFc + f   top := f(top, constant)
//   kStPop + f  top := f(entry, top)          kStPushV/C  entry := top; top := terminal
//   kStEnd      the program's end (a sentinel after its last gene)
constexpr int kStFv = 0, kStFc = 4, kStPop = 8, kStPushV = 12, kStPushC = 13, kStEnd = 14;

// The static loop for two chunks per thread (8 cases) in PTX: the gene's
// code selects its case by an indirect branch declared uniform across the
// warp (brx.idx.uni; every thread of a CTA runs the same program), and each
// case ends with the same dispatch of the next gene, so no reconvergence
// bookkeeping surrounds it.  Arithmetic with explicit round-to-nearest
// (.rn), so nothing is contracted into an FMA; protected division
// |b| < eps ? 1 : a / b with IEEE division (div.rn.f32): the same
// operations, bit for bit, as the C++ loops.  t[0..7]: the stack top's 8
// cases; x0: the thread's first case in feature row 0 for chunk 0 (global;
// chunk 1 is 4 KB further, for a partial last tile read past the last row
// into the padding of X, values that are not stored); pc: the decoded
// program in shared memory; stk: the thread's stack entry 0, chunk 0
// (shared window addresses).
// chunk 1 of a thread's cases (feature row, stack entry) is 4096 bytes after chunk 0
static_assert(kInterpThreads * sizeof(float4) == 4096, "the PTX loop's chunk stride");
static_assert(kXTailFloats * sizeof(float) >= 4096, "X's padding covers a chunk read past its end");
#define GSGP_X "%8"
#define GSGP_EPS "%11"
#define GSGP_OP_ADD(T, V) "add.rn.f32 " T ", " T ", " V ";\n\t"
#define GSGP_OP_SUB(T, V) "sub.rn.f32 " T ", " T ", " V ";\n\t"
#define GSGP_OP_MUL(T, V) "mul.rn.f32 " T ", " T ", " V ";\n\t"
#define GSGP_OP_DIV(T, V)                                       \
  "abs.f32 ab, " V ";\n\t"                                      \
  "setp.lt.f32 pp, ab, " GSGP_EPS ";\n\t"                       \
  "div.rn.f32 qq, " T ", " V ";\n\t"                            \
  "selp.f32 " T ", 0f3F800000, qq, pp;\n\t"
// entry (left operand) op top
#define GSGP_RP_ADD(T, V) "add.rn.f32 " T ", " V ", " T ";\n\t"
#define GSGP_RP_SUB(T, V) "sub.rn.f32 " T ", " V ", " T ";\n\t"
#define GSGP_RP_MUL(T, V) "mul.rn.f32 " T ", " V ", " T ";\n\t"
#define GSGP_RP_DIV(T, V)                                       \
  "abs.f32 ab, " T ";\n\t"                                      \
  "setp.lt.f32 pp, ab, " GSGP_EPS ";\n\t"                       \
  "div.rn.f32 qq, " V ", " T ";\n\t"                            \
  "selp.f32 " T ", 0f3F800000, qq, pp;\n\t"
#define GSGP_ALL8(OP, V0, V1, V2, V3, V4, V5, V6, V7)                                    \
  OP("%0", V0) OP("%1", V1) OP("%2", V2) OP("%3", V3) OP("%4", V4) OP("%5", V5)         \
      OP("%6", V6) OP("%7", V7)
#define GSGP_LOAD_FEATURE                                        \
  "mad.wide.s32 a0, ey, 16, xg0;\n\t"                            \
  "ld.global.nc.v4.f32 {v0, v1, v2, v3}, [a0];\n\t"             \
  "ld.global.nc.v4.f32 {v4, v5, v6, v7}, [a0+4096];\n\t"
#define GSGP_ENTRY_ADDR                                          \
  "shr.u32 so, ex, 12;\n\t"                                      \
  "add.u32 sa, %10, so;\n\t"
#define GSGP_NEXT                                                \
  "ld.shared.v2.b32 {ex, ey}, [pcr];\n\t"                        \
  "add.u32 pcr, pcr, 8;\n\t"                                     \
  "and.b32 cc, ex, 15;\n\t"                                      \
  "brx.idx.uni cc, GSGP_TBL;\n\t"
#define GSGP_CASE_FV(L, OP)                                      \
  L ":\n\t" GSGP_LOAD_FEATURE GSGP_ALL8(OP, "v0", "v1", "v2", "v3", "v4", "v5", "v6", "v7") \
  GSGP_NEXT
#define GSGP_CASE_FC(L, OP)                                      \
  L ":\n\t" GSGP_ALL8(OP, "ey", "ey", "ey", "ey", "ey", "ey", "ey", "ey") \
  GSGP_NEXT
#define GSGP_CASE_POP(L, OP)                                     \
  L ":\n\t" GSGP_ENTRY_ADDR                                      \
  "ld.shared.v4.f32 {v0, v1, v2, v3}, [sa];\n\t"                 \
  "ld.shared.v4.f32 {v4, v5, v6, v7}, [sa+4096];\n\t"            \
  GSGP_ALL8(OP, "v0", "v1", "v2", "v3", "v4", "v5", "v6", "v7")  \
  GSGP_NEXT

__device__ __forceinline__ void static_loop_ptx2(Lanes<2> &t, const float4 *x0, unsigned pc,
                                                 unsigned stk, float eps) {
  asm volatile(
      "{\n\t"
      ".reg .b32 ex, ey, so, sa, pcr;\n\t"
      ".reg .u32 cc;\n\t"
      ".reg .b64 a0, xg0;\n\t"
      ".reg .f32 v0, v1, v2, v3, v4, v5, v6, v7, ab, qq;\n\t"
      ".reg .pred pp;\n\t"
      "cvta.to.global.u64 xg0, " GSGP_X ";\n\t"
      "mov.u32 pcr, %9;\n\t"
      "GSGP_TBL: .branchtargets GSGP_C0, GSGP_C1, GSGP_C2, GSGP_C3, GSGP_C4, GSGP_C5, GSGP_C6, "
      "GSGP_C7, GSGP_C8, GSGP_C9, GSGP_C10, GSGP_C11, GSGP_C12, GSGP_C13, GSGP_END, GSGP_END;\n\t"
      GSGP_NEXT
      GSGP_CASE_FV("GSGP_C0", GSGP_OP_ADD)
      GSGP_CASE_FV("GSGP_C1", GSGP_OP_SUB)
      GSGP_CASE_FV("GSGP_C2", GSGP_OP_MUL)
      GSGP_CASE_FV("GSGP_C3", GSGP_OP_DIV)
      GSGP_CASE_FC("GSGP_C4", GSGP_OP_ADD)
      GSGP_CASE_FC("GSGP_C5", GSGP_OP_SUB)
      GSGP_CASE_FC("GSGP_C6", GSGP_OP_MUL)
      GSGP_CASE_FC("GSGP_C7", GSGP_OP_DIV)
      GSGP_CASE_POP("GSGP_C8", GSGP_RP_ADD)
      GSGP_CASE_POP("GSGP_C9", GSGP_RP_SUB)
      GSGP_CASE_POP("GSGP_C10", GSGP_RP_MUL)
      GSGP_CASE_POP("GSGP_C11", GSGP_RP_DIV)
      // push a feature: the top goes to its entry, the feature becomes the top
      "GSGP_C12:\n\t" GSGP_ENTRY_ADDR
      "st.shared.v4.f32 [sa], {%0, %1, %2, %3};\n\t"
      "st.shared.v4.f32 [sa+4096], {%4, %5, %6, %7};\n\t"
      "mad.wide.s32 a0, ey, 16, xg0;\n\t"
      "ld.global.nc.v4.f32 {%0, %1, %2, %3}, [a0];\n\t"
      "ld.global.nc.v4.f32 {%4, %5, %6, %7}, [a0+4096];\n\t"
      GSGP_NEXT
      // push a constant
      "GSGP_C13:\n\t" GSGP_ENTRY_ADDR
      "st.shared.v4.f32 [sa], {%0, %1, %2, %3};\n\t"
      "st.shared.v4.f32 [sa+4096], {%4, %5, %6, %7};\n\t"
      "mov.b32 %0, ey;\n\t"
      "mov.b32 %1, ey;\n\t"
      "mov.b32 %2, ey;\n\t"
      "mov.b32 %3, ey;\n\t"
      "mov.b32 %4, ey;\n\t"
      "mov.b32 %5, ey;\n\t"
      "mov.b32 %6, ey;\n\t"
      "mov.b32 %7, ey;\n\t"
      GSGP_NEXT
      "GSGP_END:\n\t"
      "}"
      : "+f"(t.v[0].x), "+f"(t.v[0].y), "+f"(t.v[0].z), "+f"(t.v[0].w), "+f"(t.v[1].x),
        "+f"(t.v[1].y), "+f"(t.v[1].z), "+f"(t.v[1].w)
      : "l"(x0), "r"(pc), "r"(stk), "f"(eps)
      : "memory");
}

// The same loop for one chunk per thread (4 cases): t[0..3], operands x0,
// pc, stk, eps as %4 .. %7.
#define GSGP_OP_DIV1(T, V)                                      \
  "abs.f32 ab, " V ";\n\t"                                      \
  "setp.lt.f32 pp, ab, %7;\n\t"                                 \
  "div.rn.f32 qq, " T ", " V ";\n\t"                            \
  "selp.f32 " T ", 0f3F800000, qq, pp;\n\t"
#define GSGP_RP_DIV1(T, V)                                      \
  "abs.f32 ab, " T ";\n\t"                                      \
  "setp.lt.f32 pp, ab, %7;\n\t"                                 \
  "div.rn.f32 qq, " V ", " T ";\n\t"                            \
  "selp.f32 " T ", 0f3F800000, qq, pp;\n\t"
#define GSGP_ALL4(OP, V0, V1, V2, V3) OP("%0", V0) OP("%1", V1) OP("%2", V2) OP("%3", V3)
#define GSGP_ENTRY_ADDR1                                         \
  "shr.u32 so, ex, 12;\n\t"                                      \
  "add.u32 sa, %6, so;\n\t"
#define GSGP_CASE_FV1(L, OP)                                     \
  L ":\n\t"                                                      \
  "mad.wide.s32 a0, ey, 16, xg0;\n\t"                            \
  "ld.global.nc.v4.f32 {v0, v1, v2, v3}, [a0];\n\t"             \
  GSGP_ALL4(OP, "v0", "v1", "v2", "v3") GSGP_NEXT
#define GSGP_CASE_FC1(L, OP) L ":\n\t" GSGP_ALL4(OP, "ey", "ey", "ey", "ey") GSGP_NEXT
#define GSGP_CASE_POP1(L, OP)                                    \
  L ":\n\t" GSGP_ENTRY_ADDR1                                     \
  "ld.shared.v4.f32 {v0, v1, v2, v3}, [sa];\n\t"                 \
  GSGP_ALL4(OP, "v0", "v1", "v2", "v3") GSGP_NEXT

__device__ __forceinline__ void static_loop_ptx1(Lanes<1> &t, const float4 *x0, unsigned pc,
                                                 unsigned stk, float eps) {
  asm volatile(
      "{\n\t"
      ".reg .b32 ex, ey, so, sa, pcr;\n\t"
      ".reg .u32 cc;\n\t"
      ".reg .b64 a0, xg0;\n\t"
      ".reg .f32 v0, v1, v2, v3, ab, qq;\n\t"
      ".reg .pred pp;\n\t"
      "cvta.to.global.u64 xg0, %4;\n\t"
      "mov.u32 pcr, %5;\n\t"
      "GSGP_TBL: .branchtargets GSGP_C0, GSGP_C1, GSGP_C2, GSGP_C3, GSGP_C4, GSGP_C5, GSGP_C6, "
      "GSGP_C7, GSGP_C8, GSGP_C9, GSGP_C10, GSGP_C11, GSGP_C12, GSGP_C13, GSGP_END, GSGP_END;\n\t"
      GSGP_NEXT
      GSGP_CASE_FV1("GSGP_C0", GSGP_OP_ADD)
      GSGP_CASE_FV1("GSGP_C1", GSGP_OP_SUB)
      GSGP_CASE_FV1("GSGP_C2", GSGP_OP_MUL)
      GSGP_CASE_FV1("GSGP_C3", GSGP_OP_DIV1)
      GSGP_CASE_FC1("GSGP_C4", GSGP_OP_ADD)
      GSGP_CASE_FC1("GSGP_C5", GSGP_OP_SUB)
      GSGP_CASE_FC1("GSGP_C6", GSGP_OP_MUL)
      GSGP_CASE_FC1("GSGP_C7", GSGP_OP_DIV1)
      GSGP_CASE_POP1("GSGP_C8", GSGP_RP_ADD)
      GSGP_CASE_POP1("GSGP_C9", GSGP_RP_SUB)
      GSGP_CASE_POP1("GSGP_C10", GSGP_RP_MUL)
      GSGP_CASE_POP1("GSGP_C11", GSGP_RP_DIV1)
      // push a feature: the top goes to its entry, the feature becomes the top
      "GSGP_C12:\n\t" GSGP_ENTRY_ADDR1
      "st.shared.v4.f32 [sa], {%0, %1, %2, %3};\n\t"
      "mad.wide.s32 a0, ey, 16, xg0;\n\t"
      "ld.global.nc.v4.f32 {%0, %1, %2, %3}, [a0];\n\t"
      GSGP_NEXT
      // push a constant
      "GSGP_C13:\n\t" GSGP_ENTRY_ADDR1
      "st.shared.v4.f32 [sa], {%0, %1, %2, %3};\n\t"
      "mov.b32 %0, ey;\n\t"
      "mov.b32 %1, ey;\n\t"
      "mov.b32 %2, ey;\n\t"
      "mov.b32 %3, ey;\n\t"
      GSGP_NEXT
      "GSGP_END:\n\t"
      "}"
      : "+f"(t.v[0].x), "+f"(t.v[0].y), "+f"(t.v[0].z), "+f"(t.v[0].w)
      : "l"(x0), "r"(pc), "r"(stk), "f"(eps)
      : "memory");
}
#undef GSGP_CASE_POP1
#undef GSGP_CASE_FC1
#undef GSGP_CASE_FV1
#undef GSGP_ENTRY_ADDR1
#undef GSGP_ALL4
#undef GSGP_RP_DIV1
#undef GSGP_OP_DIV1
#undef GSGP_CASE_POP
#undef GSGP_NEXT
#undef GSGP_CASE_FC
#undef GSGP_CASE_FV
#undef GSGP_ENTRY_ADDR
#undef GSGP_LOAD_FEATURE
#undef GSGP_ALL8
#undef GSGP_RP_DIV
#undef GSGP_RP_MUL
#undef GSGP_RP_SUB
#undef GSGP_RP_ADD
#undef GSGP_OP_DIV
#undef GSGP_OP_MUL
#undef GSGP_OP_SUB
#undef GSGP_OP_ADD
#undef GSGP_EPS
#undef GSGP_X

// A CTA interprets one program over VEC chunks of 1024 cases: thread t holds
// cases 4t .. 4t + 3 of each chunk, so one decoded gene serves 4 VEC cases.
// The stack below the top lives in shared memory as [slot][chunk][thread];
// each chunk's squared errors are reduced exactly as with one chunk per CTA.
// Every program the library interprets is well-formed postfix (a generated
// tree, or the live code of a linear genome), which the static form needs;
// a program that is not (a function short of operands, or a stack deeper
// than the launch's slots) is run by the general loop, which tracks the
// stack pointer and skips a function short of operands (the paper's rule);
// its value is then the final stack top (register Out is the live code's
// root, which compaction has already made the last gene).
template <int MODE, int VEC, int MINB>
__global__ void __launch_bounds__(kInterpThreads, MINB)
    interpret_kernel(InterpParams p, int force_general) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4 *s_stack = reinterpret_cast<float4 *>(smem_raw);
  int2 *s_prog =
      reinterpret_cast<int2 *>(s_stack + (size_t)p.stack_slots * VEC * kInterpThreads);
  __shared__ float2 s_sub[VEC][kInterpThreads / 32];   // sub-block (warp) totals per chunk
  __shared__ int s_warp[kInterpThreads / 32];
  __shared__ int s_general;

  const int prog = p.order ? p.order[blockIdx.x] : (int)blockIdx.x;
  const int tile = blockIdx.y;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int len = p.lengths[prog];
  const int64_t row4 = p.n_pad / 4;   // float4s per feature row
  if (tid == 0) s_general = force_general;
  // Decoding pass: the stack depth before each gene, by a block-wide
  // prefix sum of the genes' stack effects (+1 terminal, 0 fused,
  // -1 function).
  int carry = 0;
  for (int k0 = 0; k0 < len; k0 += kInterpThreads) {
    const int k = k0 + tid;
    int2 d = make_int2(0, 0);
    int eff = 0;
    if (k < len) {
      d = decode_gene(p.genes[(size_t)prog * p.K + k], p.consts[(size_t)prog * p.K + k], row4);
      eff = (d.x & kDecFun) ? ((d.x & kDecTerm) ? 0 : -1) : 1;
    }
    int incl = eff;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int before = carry + incl - eff, total = 0;
#pragma unroll
    for (int w = 0; w < kInterpThreads / 32; ++w) {
      const int t = s_warp[w];
      before += w < warp ? t : 0;
      total += t;
    }
    if (k < len) {
      int st, slot = 0;
      bool bad;
      if (!(d.x & kDecFun)) {   // a terminal alone: the top moves to entry before - 1
        st = (d.x & kDecVar) ? kStPushV : kStPushC;
        slot = before > 0 ? before - 1 : 0;
        bad = before > p.stack_slots;
      } else if (d.x & kDecTerm) {
        st = ((d.x & kDecVar) ? kStFv : kStFc) + (d.x & 3);
        bad = before < 1;
      } else {
        st = kStPop + (d.x & 3);
        slot = before - 2;
        bad = before < 2;
      }
      if (bad) s_general = 1;
      s_prog[k] = make_int2(
          st | (d.x << 4) |
              (bad ? 0 : (slot * VEC * kInterpThreads * (int)sizeof(float4)) << 12),
          d.y);
    }
    carry += total;
    __syncthreads();   // s_warp is reused
  }
  if (tid == 0) s_prog[len] = make_int2(kStEnd, 0);
  __syncthreads();
  const bool general = s_general != 0;

  int64_t j4[VEC];   // float4 index of the thread's cases in chunk q
  bool valid[VEC];
  const float4 *xcase[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    j4[q] = ((int64_t)tile * VEC + q) * kInterpThreads + tid;
    valid[q] = j4[q] * 4 < p.n_pad;
    xcase[q] = reinterpret_cast<const float4 *>(p.X) + (valid[q] ? j4[q] : 0);
  }
  float4 *stk = s_stack + tid;   // entry s, chunk q at stk[(s * VEC + q) * kInterpThreads]
  Lanes<VEC> tos;
#pragma unroll
  for (int q = 0; q < VEC; ++q) tos.v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  auto feature = [&](int off) {
    Lanes<VEC> a;
#pragma unroll
    for (int q = 0; q < VEC; ++q) a.v[q] = __ldg(xcase[q] + off);
    return a;
  };
  auto constant = [&](float c) {
    Lanes<VEC> a;
#pragma unroll
    for (int q = 0; q < VEC; ++q) a.v[q] = make_float4(c, c, c, c);
    return a;
  };
  auto entry = [&](int off) {   // stack entry at a float4 offset
    Lanes<VEC> a;
#pragma unroll
    for (int q = 0; q < VEC; ++q) a.v[q] = stk[off + q * kInterpThreads];
    return a;
  };
  auto put = [&](int off) {
#pragma unroll
    for (int q = 0; q < VEC; ++q) stk[off + q * kInterpThreads] = tos.v[q];
  };
  const float eps = p.protect_eps;
  if (!general) {
    if constexpr (VEC == 2)
      static_loop_ptx2(tos, xcase[0], (unsigned)__cvta_generic_to_shared(s_prog),
                       (unsigned)__cvta_generic_to_shared(stk), eps);
    else
      static_loop_ptx1(tos, xcase[0], (unsigned)__cvta_generic_to_shared(s_prog),
                       (unsigned)__cvta_generic_to_shared(stk), eps);
  } else {
    int sp = 0;
    auto push = [&](const Lanes<VEC> &x) {
      if (sp > 0 && sp - 1 < p.stack_slots) put((sp - 1) * VEC * kInterpThreads);
      tos = x;
      ++sp;
    };
    for (int k = 0; k < len; ++k) {
      const int2 e = s_prog[k];
      switch ((e.x >> 4) & 31) {
#define GSGP_FUN(F)                                                                      \
  case kDecFun | F:                                                                      \
    if (sp >= 2) {                                                                       \
      tos = opv<F, VEC>(entry((sp - 2) * VEC * kInterpThreads), tos, eps);               \
      --sp;                                                                              \
    }                                                                                    \
    break;                                                                               \
  case kDecTerm | kDecFun | F: {                                                         \
    const Lanes<VEC> v = constant(__int_as_float(e.y));                                  \
    if (sp >= 1)                                                                         \
      tos = opv<F, VEC>(tos, v, eps);                                                    \
    else                                                                                 \
      push(v);                                                                           \
    break;                                                                               \
  }                                                                                      \
  case kDecTerm | kDecVar | kDecFun | F: {                                               \
    const Lanes<VEC> v = feature(e.y);                                                   \
    if (sp >= 1)                                                                         \
      tos = opv<F, VEC>(tos, v, eps);                                                    \
    else                                                                                 \
      push(v);                                                                           \
    break;                                                                               \
  }
        GSGP_FUN(kOpAdd)
        GSGP_FUN(kOpSub)
        GSGP_FUN(kOpMul)
        GSGP_FUN(kOpDiv)
#undef GSGP_FUN
        case kDecTerm:
          push(constant(__int_as_float(e.y)));
          break;
        case kDecTerm | kDecVar:
          push(feature(e.y));
          break;
        default:
          break;
      }
    }
  }
  // The program's value is register Out (Sec. 2.2, "Interpreter"): every
  // program interpreted here is well-formed postfix (a ramped half-and-half
  // tree, or the live code of a linear genome, which ends with the last
  // function applied), so Out is the final stack top; an empty program is 0.

  if (MODE == 0) {
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      float str = 0.f, ste = 0.f;
      if (valid[q]) {
        reinterpret_cast<float4 *>(static_cast<float *>(p.out) + (int64_t)prog * p.n_pad)[j4[q]] =
            tos.v[q];
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p.target) + j4[q]);
        const float vv[4] = {tos.v[q].x, tos.v[q].y, tos.v[q].z, tos.v[q].w};
        const float tt[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int64_t j = j4[q] * 4 + c;
          const float d = vv[c] - tt[c];
          if (j < p.n_train)
            str += d * d;
          else if (j < p.n_cases)
            ste += d * d;
        }
      }
      const float2 sub = subblock_sum(str, ste);
      if (lane == 0) s_sub[q][warp] = sub;
    }
    __syncthreads();
    if (tid < VEC && tile * VEC + tid < (int)((p.n_pad + 1023) >> 10))
      p.partial[(size_t)prog * p.tiles + p.chunk0 + tile * VEC + tid] = chunk_total(s_sub[tid]);
  } else {
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      if (!valid[q]) continue;
      const float4 t4 = tos.v[q];
      const float4 sg = make_float4(logistic(t4.x), logistic(t4.y), logistic(t4.z), logistic(t4.w));
      if (MODE == 1) {
        reinterpret_cast<float4 *>(static_cast<float *>(p.out) + (int64_t)prog * p.n_pad)[j4[q]] =
            sg;
      } else {
        __nv_bfloat162 lo = __floats2bfloat162_rn(sg.x, sg.y);
        __nv_bfloat162 hi = __floats2bfloat162_rn(sg.z, sg.w);
        uint2 packed;
        packed.x = *reinterpret_cast<uint32_t *>(&lo);
        packed.y = *reinterpret_cast<uint32_t *>(&hi);
        reinterpret_cast<uint2 *>(static_cast<__nv_bfloat16 *>(p.out) + (int64_t)prog * p.n_pad)
            [j4[q]] = packed;
      }
    }
  }
}

// Diagnostic switch: with the environment variable GSGP_INTERP_GENERAL set
// to a nonzero integer when gsgp_init runs, every program is interpreted by
// the general loop (stack pointer, skip rule) instead of the static PTX
// loop; the results are the same bit for bit.  The library generates only
// well-formed programs, so this is how the general loop is exercised.
static int interp_force_general() {
  const char *v = getenv("GSGP_INTERP_GENERAL");
  return v && atoi(v) != 0 ? 1 : 0;
}

template <int MODE, int VEC, int MINB>
static cudaError_t interpret_launch_minb(const InterpParams &p, int count, cudaStream_t s) {
  const size_t smem = (size_t)p.stack_slots * VEC * kInterpThreads * sizeof(float4) +
                      (size_t)(p.max_len + 1) * sizeof(int2);   // genes + the end sentinel
  const int64_t tile = (int64_t)kInterpTile * VEC;
  const dim3 grid((unsigned)count, (unsigned)((p.n_pad + tile - 1) / tile));
  cudaError_t e = cudaFuncSetAttribute(interpret_kernel<MODE, VEC, MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  interpret_kernel<MODE, VEC, MINB><<<grid, kInterpThreads, smem, s>>>(p, interp_force_general());
  return cudaGetLastError();
}

// Two chunks per thread with a stack of at most 3 entries below the top
// (24 KB) leave shared memory for six CTAs per SM: a kernel built for 40
// registers a thread; otherwise five (48 registers).
template <int MODE, int VEC>
static cudaError_t interpret_launch(const InterpParams &p, int count, cudaStream_t s) {
  if constexpr (VEC == 2) {
    if (p.stack_slots <= 3) return interpret_launch_minb<MODE, VEC, 6>(p, count, s);
  }
  return interpret_launch_minb<MODE, VEC, 5>(p, count, s);
}

// Pools whose longest program has this many genes take two chunks per CTA
// (one decode per 8 cases); shorter ones one chunk (measured on the paper's
// k = 127 shape: 15.6 ms against 18.1 with one chunk).
constexpr int kInterpWideGenes = 64;

cudaError_t launch_interpret(int mode, const InterpParams &p, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  // feature offsets are 32-bit float4 indices
  if (p.n_features <= 0 || (int64_t)p.n_features * (p.n_pad / 4) > (int64_t)INT32_MAX)
    return cudaErrorInvalidValue;
  const bool wide = p.max_len >= kInterpWideGenes;
  switch (mode) {
    case 0: return wide ? interpret_launch<0, 2>(p, count, s) : interpret_launch<0, 1>(p, count, s);
    case 1: return wide ? interpret_launch<1, 2>(p, count, s) : interpret_launch<1, 1>(p, count, s);
    default: return wide ? interpret_launch<2, 2>(p, count, s) : interpret_launch<2, 1>(p, count, s);
  }
}

// ComputeFitness of the initial population: one warp per individual sums
// its per-tile squared errors in a fixed order and takes the RMSE.
__global__ void __launch_bounds__(256)
    fitness_finalize_kernel(const double2 *__restrict__ partial, int tiles, int count, int n_train,
                            int n_test, double *__restrict__ fit, double *__restrict__ fit_te) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= count) return;
  const double2 *row = partial + (size_t)i * tiles;
  const double2 sse = tiles > 128 ? warp_sum_partials_long(row, tiles, lane)
                                  : warp_sum_partials(row, tiles, lane);
  if (lane == 0) {
    fit[i] = rmse_from_sse(sse.x, n_train);
    fit_te[i] = rmse_from_sse(sse.y, n_test);
  }
}

cudaError_t launch_fitness_finalize(const double2 *partial, int tiles, int count, int n_train,
                                    int n_test, double *fit, double *fit_te, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  fitness_finalize_kernel<<<(count * 32 + 255) / 256, 256, 0, s>>>(partial, tiles, count, n_train,
                                                                   n_test, fit, fit_te);
  return cudaGetLastError();
}

// Generation-0 state: population slot i lives in pool row i, offspring slot
// i will be written to row m + i; best slot of the initial population.
__global__ void __launch_bounds__(kFinalThreads)
    init_state_kernel(int m, int *perm, const double *fit, DevState *state) {
  __shared__ unsigned long long s_v[kFinalThreads];
  __shared__ int s_i[kFinalThreads];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    perm[i] = i;
    perm[m + i] = m + i;
  }
  double bv;
  int bi;
  block_arg<false>(fit, m, s_v, s_i, bv, bi);
  if (threadIdx.x == 0) {
    state->gen = 0;
    state->parity = 0;
    state->done = 0u;
    state->best_slot = bi;
  }
}

cudaError_t launch_init_state(int m, int *perm, const double *fit, DevState *state,
                              cudaStream_t s) {
  init_state_kernel<<<1, kFinalThreads, 0, s>>>(m, perm, fit, state);
  return cudaGetLastError();
}

__global__ void rng_words_kernel(uint2 key, uint32_t run, uint32_t gp, uint32_t individual,
                                 int n_words, uint32_t *out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b * 4 >= n_words) return;
  const uint4 v = philox4x32_10(make_uint4((uint32_t)b, individual, gp, run), key);
  for (int q = 0; q < 4 && b * 4 + q < n_words; ++q) out[b * 4 + q] = lane_of(v, q);
}

cudaError_t launch_rng_words(uint2 key, uint32_t run, uint32_t gp, uint32_t individual,
                             int n_words, uint32_t *out, cudaStream_t s) {
  if (n_words <= 0) return cudaSuccess;
  const int blocks = (n_words + 3) / 4;
  rng_words_kernel<<<(blocks + 127) / 128, 128, 0, s>>>(key, run, gp, individual, n_words, out);
  return cudaGetLastError();
}

}  // namespace gsgp
