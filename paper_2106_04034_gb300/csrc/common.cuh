// Device-side building blocks shared by the GSGP kernels: the Philox4x32-10
// counter-based generator, the integer-only draw mappings, gene decoding and
// the parameter blocks handed to every kernel launch.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gsgp {

// ---- gene encoding (linear postfix genome, Sec. 2.2 "Initialization") ----
constexpr int kOpAdd = 0, kOpSub = 1, kOpMul = 2, kOpDiv = 3, kOpConst = 4, kOpVar = 5;
constexpr int kGenePad = -1;
// Interpreter-only codes written by the terminal-operand fusion pass: a
// terminal and the function right after it as one gene, base + function
// (the feature index in the upper bits as for kOpVar).
constexpr int kOpFusedConst = 8, kOpFusedVar = 12;
constexpr int kMaxDepth = 10;                    // deepest tree a pool may hold
constexpr int kMaxGenes = (1 << (kMaxDepth + 1)) - 1;
constexpr int kMaxGenomeGenes = 4095;             // longest linear genome
constexpr int kMaxStack = 32;                     // deepest interpreter stack a program may use

// Purposes of the initialisation streams (counter word 2 = 0x80000000 | p).
constexpr uint32_t kInitFlag = 0x80000000u;
constexpr uint32_t kPurposePop = 1, kPurposeRt = 2;

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) -------------------
// Ten rounds of: multiply counter words 0 and 2 by two odd 32-bit constants,
// cross the 64-bit products' halves with words 1 and 3 and the round key,
// then bump the key by the two Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ uint32_t lane_of(const uint4 &v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

// Sequential reader of the stream (individual, gen_or_purpose, run): word w
// is lane w & 3 of block w >> 2 (counter word 0 = block).
struct WordStream {
  uint4 ctr;
  uint2 key;
  uint4 buf;
  uint32_t pos;
  __device__ WordStream(uint2 key_, uint32_t individual, uint32_t gen_or_purpose, uint32_t run)
      : ctr(make_uint4(0u, individual, gen_or_purpose, run)), key(key_), buf(), pos(0) {}
  __device__ __forceinline__ uint32_t next() {
    if ((pos & 3u) == 0u) {
      ctr.x = pos >> 2;
      buf = philox4x32_10(ctr, key);
    }
    const uint32_t w = lane_of(buf, pos & 3u);
    ++pos;
    return w;
  }
};

// idx(w, n) = floor(w * n / 2^32): the high word of the 32x32 product.
__device__ __forceinline__ uint32_t draw_index(uint32_t w, uint32_t n) { return __umulhi(w, n); }

// u24(w) = (w >> 8) * 2^-24, exact in float.
__device__ __forceinline__ float draw_u24(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

// Ephemeral random constant lo + (hi - lo) * u24(w): each double operation
// rounded separately (no contraction), then rounded to float once.
__device__ __forceinline__ float draw_const(uint32_t w, float lo, float hi) {
  const double lo64 = (double)lo, hi64 = (double)hi;
  const double span = __dadd_rn(hi64, -lo64);
  const double prod = __dmul_rn(span, (double)draw_u24(w));
  return __double2float_rn(__dadd_rn(lo64, prod));
}

// ---- per-generation device state -----------------------------------------
struct DevState {
  int gen;            // generations completed since init
  int parity;         // which half of the double-buffered tables is current
  unsigned done;      // offspring finalised in the running generation
  int best_slot;      // best individual after the last survival
};

// Parameters of the generation kernels (passed by value).
struct GenParams {
  const float *target;       // [n_pad] targets, train cases first then test
  float *pool;               // [2m][n_pad] semantic rows (population + offspring)
  const void *sigma_r;       // [r][n_pad] sigma(R) as float or bf16
  int *perm;                 // [2][2m]: rows of population slots, then free rows
  double *fit;               // [2][m] training RMSE
  double *fit_te;            // [2][m] test RMSE
  double2 *partial;          // [m][tiles] per-chunk (train, test) squared errors
  int4 *sel;                 // [m] (parent row, offspring row, rt1, rt2) of this generation
  float *sel_ms;             // [m] mutation step of this generation
  int4 *trace;               // [gcap][m] (parent slot, rt1, rt2, ms bits)
  double2 *best_log;         // [gcap] (train, test) RMSE of the best
  DevState *state;
  int64_t n_pad;
  int m, r, tsize;
  int n_train, n_cases;      // cases held by this context (train first)
  int tiles;                 // 1024-case chunks of the whole problem: row stride of partial
  int ms_mode;
  float ms;
  uint2 key;
  uint32_t run;
  int elitism;
  float p_crossover;         // probability of geometric semantic crossover (0: mutation only)
  // Case sharding: this context's cases are the problem's cases from chunk
  // chunk0 on (its chunk c is column chunk0 + c of partial); the RMSE
  // divides by the whole problem's training / test case counts.  Unsharded:
  // chunk0 = 0, n_train_all = n_train, n_test_all = n_cases - n_train.
  int chunk0;
  int n_train_all, n_test_all;
};

// Parameters of the interpreter (ComputeSemantics) kernel.
struct InterpParams {
  const float *X;            // [l][n_pad] feature-major cases
  const float *target;       // [n_pad]
  const int *genes;          // [count][K]
  const float *consts;       // [count][K]
  const int *lengths;        // [count]
  int K;                     // row stride of genes / consts
  int max_len;               // longest program of the pool (sizes shared memory)
  void *out;                 // [count][n_pad] float (population) or sigma (random)
  double2 *partial;          // [count][tiles] (population only); chunk c at column chunk0 + c
  int64_t n_pad;
  int n_train, n_cases;
  int tiles;
  int stack_slots;           // shared-memory stack depth below the cached top
  float protect_eps;
  const int *order;          // programs of this launch (CTA column x runs order[x]), or null
  int n_features;            // rows of X
  int chunk0;                // first chunk of partial this context writes (case sharding)
};

}  // namespace gsgp
