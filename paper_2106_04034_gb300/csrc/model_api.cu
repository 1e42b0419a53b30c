// Context-free evaluation of a rebuilt model (Algorithm 1, "Return: best
// individual found", applied to new data): the ancestor program and the
// random trees with a nonzero coefficient are uploaded from a gsgp_trace,
// compacted to their live code on the device (the interpreter's rule makes
// every program's value the expression under its last applied function), and
// evaluated by the same float64 model kernel as gsgp_predict.
#include <cmath>
#include <cstring>
#include <vector>

#include "gsgp.h"
#include "kernels.cuh"

using namespace gsgp;

namespace {

gsgp_status model_fail(char *msg, size_t cap, gsgp_status st, const char *text) {
  if (msg && cap) {
    size_t k = 0;
    for (; text[k] && k + 1 < cap; ++k) msg[k] = text[k];
    msg[k] = '\0';
  }
  return st;
}

// Device buffers of one call, released in the destructor (stream-ordered).
struct Scratch {
  cudaStream_t s;
  std::vector<void *> ptrs;
  cudaError_t err = cudaSuccess;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <typename T>
  T *alloc(size_t count) {
    void *p = nullptr;
    if (err != cudaSuccess) return nullptr;
    err = cudaMallocAsync(&p, count ? count * sizeof(T) : 16, s);
    if (err != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<T *>(p);
  }
  ~Scratch() {
    for (void *p : ptrs) cudaFreeAsync(p, s);
  }
};

}  // namespace

extern "C" gsgp_status gsgp_model_predict(const gsgp_trace *t, const float *X, int64_t n,
                                          double *y_out, void *stream, char *err_msg,
                                          size_t err_cap) {
  if (err_msg && err_cap) err_msg[0] = '\0';
  if (!t || t->struct_size != sizeof(gsgp_trace))
    return model_fail(err_msg, err_cap, GSGP_E_INVALID, "model NULL or struct_size mismatch");
  if (n < 0 || (n > 0 && (!X || !y_out)))
    return model_fail(err_msg, err_cap, GSGP_E_INVALID, "need n >= 0 and X, y_out for n > 0");
  const int l = t->n_features, K = t->max_genes, Kr = t->rt_max_genes, r = t->n_random_trees;
  if (l < 1 || K < 1 || K > kMaxGenomeGenes || Kr < 1 || Kr > kMaxGenomeGenes || r < 0 ||
      t->ancestor_length < 0 || t->ancestor_length > K || !t->ancestor_genes ||
      !t->ancestor_consts || (r > 0 && (!t->coef || !t->rt_genes || !t->rt_consts ||
                                        !t->rt_lengths)) ||
      !std::isfinite(t->protect_eps) ||
      (t->sigma_dtype != GSGP_SIGMA_F32 && t->sigma_dtype != GSGP_SIGMA_BF16))
    return model_fail(err_msg, err_cap, GSGP_E_INVALID, "inconsistent model fields");
  for (int64_t k = 0; k < n * (int64_t)l; ++k)
    if (!std::isfinite(X[k]))
      return model_fail(err_msg, err_cap, GSGP_E_INVALID, "non-finite input");
  if (n == 0) return GSGP_OK;
  // the terms: random trees with a nonzero coefficient, packed in order
  std::vector<int> terms;
  std::vector<double> coef;
  for (int k = 0; k < r; ++k)
    if (t->coef[k] != 0.0) {
      if (t->rt_lengths[k] < 0 || t->rt_lengths[k] > Kr)
        return model_fail(err_msg, err_cap, GSGP_E_INVALID, "random-tree length out of range");
      terms.push_back(k);
      coef.push_back(t->coef[k]);
    }
  const int nk = (int)terms.size();
  std::vector<int> rg((size_t)(nk ? nk : 1) * Kr), rl((size_t)(nk ? nk : 1)), idx((size_t)(nk ? nk : 1));
  std::vector<float> rc(rg.size());
  for (int q = 0; q < nk; ++q) {
    memcpy(&rg[(size_t)q * Kr], t->rt_genes + (size_t)terms[q] * Kr, sizeof(int) * Kr);
    memcpy(&rc[(size_t)q * Kr], t->rt_consts + (size_t)terms[q] * Kr, sizeof(float) * Kr);
    rl[(size_t)q] = t->rt_lengths[terms[q]];
    idx[(size_t)q] = q;
  }
  // programs use genes < 6 (and features below l)
  auto check = [&](const int *g, int len) {
    for (int k = 0; k < len; ++k) {
      const int op = g[k] & 0xFF;
      if (g[k] < 0 || op > kOpVar || (op == kOpVar && (g[k] >> 8) >= l)) return false;
    }
    return true;
  };
  if (!check(t->ancestor_genes, t->ancestor_length))
    return model_fail(err_msg, err_cap, GSGP_E_INVALID, "bad gene in the ancestor");
  for (int q = 0; q < nk; ++q)
    if (!check(&rg[(size_t)q * Kr], rl[(size_t)q]))
      return model_fail(err_msg, err_cap, GSGP_E_INVALID, "bad gene in a random tree");

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n_pad = (n + 3) / 4 * 4;
  gsgp_status st = GSGP_OK;
  {
    Scratch m(s);
    float *xr = m.alloc<float>((size_t)n * l);
    float *xt = m.alloc<float>((size_t)l * n_pad);
    int *ag = m.alloc<int>((size_t)K), *agc = m.alloc<int>((size_t)K);
    float *ac = m.alloc<float>((size_t)K), *acc = m.alloc<float>((size_t)K);
    int *al = m.alloc<int>(1), *alc = m.alloc<int>(1);
    int *dg = m.alloc<int>(rg.size()), *dgc = m.alloc<int>(rg.size());
    float *dc = m.alloc<float>(rc.size()), *dcc = m.alloc<float>(rc.size());
    int *dl = m.alloc<int>(rl.size()), *dlc = m.alloc<int>(rl.size());
    int *dterms = m.alloc<int>(idx.size());
    double *dcoef = m.alloc<double>(idx.size());
    int *dstack = m.alloc<int>(1);
    double *dy = m.alloc<double>((size_t)n);
    cudaError_t e = m.err;
    auto h2d = [&](void *d, const void *h, size_t b) {
      if (e == cudaSuccess) e = cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, s);
    };
    h2d(xr, X, sizeof(float) * (size_t)n * l);
    h2d(ag, t->ancestor_genes, sizeof(int) * (size_t)K);
    h2d(ac, t->ancestor_consts, sizeof(float) * (size_t)K);
    const int alen = t->ancestor_length;
    h2d(al, &alen, sizeof(int));
    h2d(dg, rg.data(), sizeof(int) * rg.size());
    h2d(dc, rc.data(), sizeof(float) * rc.size());
    h2d(dl, rl.data(), sizeof(int) * rl.size());
    h2d(dterms, idx.data(), sizeof(int) * idx.size());
    if (nk) h2d(dcoef, coef.data(), sizeof(double) * coef.size());
    if (e == cudaSuccess) e = cudaMemsetAsync(dstack, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_transpose(xr, n, l, xt, n_pad, 0, s);
    // live code of every program, and the deepest stack it needs
    if (e == cudaSuccess) e = launch_compact(ag, ac, al, 1, K, agc, acc, alc, s);
    if (e == cudaSuccess && nk) e = launch_compact(dg, dc, dl, nk, Kr, dgc, dcc, dlc, s);
    if (e == cudaSuccess) e = launch_max_stack(agc, alc, 1, K, dstack, s);
    if (e == cudaSuccess && nk) e = launch_max_stack(dgc, dlc, nk, Kr, dstack, s);
    int hstack = 0, hlen = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hstack, dstack, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hlen, alc, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && hstack > kMaxStack) {
      st = model_fail(err_msg, err_cap, GSGP_E_INVALID,
                      "a program of the model needs more than 32 stack entries");
    } else if (e == cudaSuccess) {
      PredictParams p{};
      p.X = xt;
      p.n_pad = n_pad;
      p.n = n;
      p.anc_genes = agc;
      p.anc_consts = acc;
      p.anc_len = hlen;
      p.rt_genes = dgc;
      p.rt_consts = dcc;
      p.rt_len = dlc;
      p.Kr = Kr;
      p.terms = dterms;
      p.coef = dcoef;
      p.nk = nk;
      p.y = dy;
      p.protect_eps = t->protect_eps;
      p.sigma_bf16 = t->sigma_dtype == GSGP_SIGMA_BF16;
      e = launch_predict(p, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(y_out, dy, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      st = model_fail(err_msg, err_cap,
                      e == cudaErrorMemoryAllocation ? GSGP_E_OOM : GSGP_E_CUDA,
                      cudaGetErrorString(e));
    }
  }
  if (st == GSGP_OK && cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    st = model_fail(err_msg, err_cap, GSGP_E_CUDA, "stream error while releasing scratch");
  }
  return st;
}
