// Allocation-free mutation + fitness entry point.
//
// Some callers cannot allocate device memory at all: code that runs while a
// framework is capturing a CUDA graph and forbids cudaMalloc, plug-ins
// handed a fixed device budget by their host application, or services that
// must not touch the allocator on their request path.  gsgp_mutate_noalloc
// gives them one generation's mutation stream (offspring = parent +
// ms * (sigma_a - sigma_b)) with the offspring's training and test RMSE,
// using only the caller's input and output buffers.  Its one piece of
// scratch, the per-chunk squared-error partial sums, lives in the
// file-scope device array below instead of a cudaMalloc'd buffer.
//
// The per-chunk summation order is the library's canonical one (chunk_total)
// and chunks are added in the same fixed lane-strided order, so the offspring
// and their RMSE equal, bit for bit, the ones the library computes for the
// same draws.
#include <cuda.h>

#include <mutex>

#include "gsgp.h"
#include "kernels.cuh"
#include "reduce.cuh"
#include "stream.cuh"

namespace gsgp {

// Maximum (offspring x 1024-case chunks) of one call: 2 MiB of double2,
// held by every GPU that loads the library until the process exits.
constexpr int64_t kNoAllocMaxPartials = 1 << 17;
static __device__ __align__(256) double2 g_noalloc_partials[kNoAllocMaxPartials];

struct NoAllocArgs {
  const float *parents;   // parent semantic rows, row stride ld
  const float *sigma_r;   // sigma(R) rows, row stride ld
  float *offspring;       // offspring rows, row stride ld
  const int *parent, *rt1, *rt2;
  const float *ms;
  double *rmse_train, *rmse_test;
  double2 *partial;       // device address of g_noalloc_partials
  int64_t ld;
  int chunks;
};

// One CTA = one offspring x one 1024-case chunk.
__global__ void __launch_bounds__(kGenThreads) noalloc_mutate_kernel(const GenParams p,
                                                                     const NoAllocArgs a) {
  __shared__ float2 s_sub[kGenThreads / 32];   // sub-block (warp) totals
  const int chunk = blockIdx.x;
  const int i = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float *src = a.parents + (int64_t)a.parent[i] * a.ld;
  const float *ra = a.sigma_r + (int64_t)a.rt1[i] * a.ld;
  const float *rb = a.sigma_r + (int64_t)a.rt2[i] * a.ld;
  float *dst = a.offspring + (int64_t)i * a.ld;
  const int64_t j0 = (int64_t)chunk * 1024 + tid * 4;
  float str = 0.f, ste = 0.f;
  if (j0 < p.n_cases) mutate4<float>(p, src, dst, ra, rb, j0, a.ms[i], str, ste);
  const float2 sub = subblock_sum(str, ste);
  if (lane == 0) s_sub[warp] = sub;
  __syncthreads();
  if (tid == 0) a.partial[(size_t)i * a.chunks + chunk] = chunk_total(s_sub);
}

// One warp per offspring: fixed-order sum of its chunk partials, RMSE.
__global__ void __launch_bounds__(256) noalloc_rmse_kernel(const GenParams p, const NoAllocArgs a,
                                                           int m) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  const double2 sse = warp_sum_partials(a.partial + (size_t)i * a.chunks, a.chunks, lane);
  if (lane == 0) {
    a.rmse_train[i] = rmse_from_sse(sse.x, p.n_train);
    a.rmse_test[i] = rmse_from_sse(sse.y, p.n_cases - p.n_train);
  }
}

// Device address of the scratch array.  The host-side symbol is only a
// stand-in for it, so the address is looked up with cudaGetSymbolAddress
// once per device with that device current, and cached.  The address
// belongs to the module loaded into one CUDA context; after a
// cudaDeviceReset (or under another context) the same device has a new
// module and a new address.  The cache is therefore keyed by the current
// context's unique id (cuCtxGetCurrent + cuCtxGetId, reached through the
// runtime's driver entry points, so the library needs no link against
// libcuda), and a context it has not seen triggers a fresh lookup.
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
struct ScratchEntry {
  unsigned long long ctx_id;   // 0: empty
  double2 *addr;
};
static ScratchEntry g_noalloc_addr[kMaxDevices];

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (0 if none is current
// yet); resolves the two driver entry points on first use.
static cudaError_t current_ctx_id(unsigned long long *id) {
  static PfnCtxGetCurrent get_current = nullptr;
  static PfnCtxGetId get_id = nullptr;
  if (!get_current || !get_id) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                     cudaEnableDefault, &q1);
    if (e != cudaSuccess) return e;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorSymbolNotFound;
    get_current = reinterpret_cast<PfnCtxGetCurrent>(f1);
    get_id = reinterpret_cast<PfnCtxGetId>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
  *id = 0;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
  return cudaSuccess;
}

static cudaError_t noalloc_scratch(double2 **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  unsigned long long id = 0;
  e = current_ctx_id(&id);
  if (e != cudaSuccess) return e;
  if (id != 0 && g_noalloc_addr[dev].ctx_id == id) {
    *out = g_noalloc_addr[dev].addr;
    return cudaSuccess;
  }
  // set-up on this device and context: the lookup also makes the device's
  // primary context current if no context was yet
  void *ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
  if (e != cudaSuccess) return e;
  e = current_ctx_id(&id);
  if (e != cudaSuccess) return e;
  g_noalloc_addr[dev] = ScratchEntry{id, static_cast<double2 *>(ptr)};
  *out = static_cast<double2 *>(ptr);
  return cudaSuccess;
}

}  // namespace gsgp

using namespace gsgp;

static gsgp_status noalloc_fail(char *msg, size_t cap, gsgp_status st, const char *text) {
  if (msg && cap) {
    size_t k = 0;
    for (; text[k] && k + 1 < cap; ++k) msg[k] = text[k];
    msg[k] = '\0';
  }
  return st;
}

extern "C" gsgp_status gsgp_mutate_noalloc(const float *parents, const float *sigma_r, int64_t ld,
                                           const float *target, int64_t n_train, int64_t n_test,
                                           const int32_t *parent, const int32_t *rt1,
                                           const int32_t *rt2, const float *ms, int32_t m,
                                           float *offspring, double *rmse_train,
                                           double *rmse_test, void *stream, char *err_msg,
                                           size_t err_cap) {
  if (err_msg && err_cap) err_msg[0] = '\0';
  if (m < 1 || n_train < 1 || n_test < 0)
    return noalloc_fail(err_msg, err_cap, GSGP_E_INVALID, "need m >= 1, n_train >= 1, n_test >= 0");
  const int64_t n = n_train + n_test;
  if (n > (int64_t)0x7fffff00 || ld < n || ld % 4 != 0)
    return noalloc_fail(err_msg, err_cap, GSGP_E_INVALID,
                        "ld must be a multiple of 4 and at least n_train + n_test");
  if (!parents || !sigma_r || !target || !parent || !rt1 || !rt2 || !ms || !offspring ||
      !rmse_train || !rmse_test)
    return noalloc_fail(err_msg, err_cap, GSGP_E_INVALID, "NULL pointer argument");
  const uintptr_t align = (uintptr_t)parents | (uintptr_t)sigma_r | (uintptr_t)target |
                          (uintptr_t)offspring;
  if (align % 16 != 0)
    return noalloc_fail(err_msg, err_cap, GSGP_E_INVALID, "row buffers must be 16-byte aligned");
  // offspring is written while parents, sigma_r and target are read: an
  // input that starts inside the offspring rows (an in-place call) races
  const uintptr_t o0 = (uintptr_t)offspring, o1 = o0 + (uintptr_t)m * (uintptr_t)ld * 4u;
  for (const void *in : {(const void *)parents, (const void *)sigma_r, (const void *)target})
    if ((uintptr_t)in >= o0 && (uintptr_t)in < o1)
      return noalloc_fail(err_msg, err_cap, GSGP_E_INVALID,
                          "offspring must not overlap parents, sigma_r or target");
  const int64_t chunks = (n + 1023) / 1024;
  if ((int64_t)m * chunks > kNoAllocMaxPartials)
    return noalloc_fail(err_msg, err_cap, GSGP_E_INVALID,
                        "m * ceil((n_train + n_test) / 1024) exceeds the 131072 partial sums "
                        "of the built-in scratch");
  if (chunks > 65535 || m > 65535)
    return noalloc_fail(err_msg, err_cap, GSGP_E_INVALID, "m and the chunk count must be <= 65535");
  double2 *scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(err_msg, err_cap, GSGP_E_CUDA, cudaGetErrorString(e));
  }
  GenParams p{};
  p.target = target;
  p.n_pad = ld;
  p.n_train = (int)n_train;
  p.n_cases = (int)n;
  NoAllocArgs a{parents, sigma_r, offspring, parent, rt1, rt2, ms, rmse_train, rmse_test,
                scratch, ld, (int)chunks};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  noalloc_mutate_kernel<<<dim3((unsigned)chunks, (unsigned)m), kGenThreads, 0, s>>>(p, a);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    noalloc_rmse_kernel<<<(unsigned)((m * 32 + 255) / 256), 256, 0, s>>>(p, a, m);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return noalloc_fail(err_msg, err_cap, GSGP_E_CUDA, cudaGetErrorString(e));
  return GSGP_OK;
}
