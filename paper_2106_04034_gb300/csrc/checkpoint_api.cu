// Checkpoint and restore of a run: everything later generations depend on
// that initialisation does not rebuild, i.e. the current population's
// semantics and fitness, the generation counter and best slot, and the
// trace and best-of-generation log so far.  Programs, random-tree semantics
// and the initial state are deterministic functions of the configuration and
// the data, so a restore re-runs the initialisation on the loaded data and
// then installs the saved state; evolution continues bit for bit as if the
// run had never stopped.
#include <cstring>
#include <vector>

#include "ctx.h"

namespace {

constexpr char kMagic[8] = {'G', 'S', 'G', 'P', 'C', 'K', 'P', '1'};

// Fixed-layout header of a checkpoint (host byte order).
struct Header {
  char magic[8];
  uint32_t header_bytes;
  uint32_t reserved;
  // identity of the run: configuration fields that shape the search
  uint64_t seed;
  uint32_t run;
  int32_t pop_size, n_random_trees, n_features;
  int64_t n_train, n_test;
  int32_t pop_min_depth, pop_max_depth, rt_min_depth, rt_max_depth;
  int32_t init_mode, max_genes, sigma_dtype, tournament_size, elitism, ms_mode;
  float const_lo, const_hi, p_grow_function, p_feature_given_terminal, protect_eps, ms,
      p_crossover;
  uint64_t target_hash;   // FNV-1a of the targets' bytes
  // state
  int32_t generation, best_slot;
  uint64_t payload_bytes;
};

uint64_t fnv1a(const void *data, size_t n) {
  const unsigned char *p = static_cast<const unsigned char *>(data);
  uint64_t h = 1469598103934665603ull;
  for (size_t k = 0; k < n; ++k) {
    h ^= p[k];
    h *= 1099511628211ull;
  }
  return h;
}

void fill_identity(const gsgp_ctx *c, Header &h) {
  const gsgp_config &f = c->cfg;
  h.seed = f.seed;
  h.run = f.run;
  h.pop_size = f.pop_size;
  h.n_random_trees = f.n_random_trees;
  h.n_features = c->l;
  h.n_train = c->n_tr;
  h.n_test = c->n_te;
  h.pop_min_depth = f.pop_min_depth;
  h.pop_max_depth = f.pop_max_depth;
  h.rt_min_depth = f.rt_min_depth;
  h.rt_max_depth = f.rt_max_depth;
  h.init_mode = f.init_mode;
  h.max_genes = f.init_mode == GSGP_INIT_LINEAR ? f.max_genes : 0;
  h.sigma_dtype = f.sigma_dtype;
  h.tournament_size = f.tournament_size;
  h.elitism = f.elitism;
  h.ms_mode = f.ms_mode;
  h.const_lo = f.const_lo;
  h.const_hi = f.const_hi;
  h.p_grow_function = f.p_grow_function;
  h.p_feature_given_terminal = f.p_feature_given_terminal;
  h.protect_eps = f.protect_eps;
  h.ms = f.ms;
  h.p_crossover = f.p_crossover;
}

bool same_identity(const Header &a, const Header &b) {
  return a.seed == b.seed && a.run == b.run && a.pop_size == b.pop_size &&
         a.n_random_trees == b.n_random_trees && a.n_features == b.n_features &&
         a.n_train == b.n_train && a.n_test == b.n_test && a.pop_min_depth == b.pop_min_depth &&
         a.pop_max_depth == b.pop_max_depth && a.rt_min_depth == b.rt_min_depth &&
         a.rt_max_depth == b.rt_max_depth && a.init_mode == b.init_mode &&
         a.max_genes == b.max_genes && a.sigma_dtype == b.sigma_dtype &&
         a.tournament_size == b.tournament_size && a.elitism == b.elitism &&
         a.ms_mode == b.ms_mode && !memcmp(&a.const_lo, &b.const_lo, 7 * sizeof(float)) &&
         a.target_hash == b.target_hash;
}

// payload: semantics [m][N] float (slot order), fit [m] double, fit_te [m]
// double, trace [gen][m] int4, best_log [gen] double2
uint64_t payload_bytes(const gsgp_ctx *c, int gen) {
  const uint64_t m = (uint64_t)c->cfg.pop_size;
  return m * (uint64_t)c->N * sizeof(float) + 2 * m * sizeof(double) +
         (uint64_t)gen * m * sizeof(int4) + (uint64_t)gen * sizeof(double2);
}

gsgp_status target_hash(gsgp_ctx *c, uint64_t *out) {
  std::vector<float> t((size_t)c->N);
  CK(cudaMemcpyAsync(t.data(), c->t, sizeof(float) * t.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *out = fnv1a(t.data(), sizeof(float) * t.size());
  return GSGP_OK;
}

}  // namespace

extern "C" gsgp_status gsgp_checkpoint(gsgp_ctx *c, void *buf, size_t cap, size_t *size_out) {
  API_GUARD(c)
  if (c->state != 2) return fail(c, GSGP_E_STATE, "gsgp_checkpoint before gsgp_init");
  if (c->sharded) return fail(c, GSGP_E_STATE, "checkpoints of case shards are not supported");
  const int gen = c->gen;
  const size_t total = sizeof(Header) + payload_bytes(c, gen);
  if (size_out) *size_out = total;
  if (!buf) return GSGP_OK;   // size query
  if (cap < total) return fail(c, GSGP_E_INVALID, "buffer of %zu bytes, %zu needed", cap, total);
  TRY(use_device(c));
  Header h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, kMagic, sizeof kMagic);
  h.header_bytes = sizeof(Header);
  fill_identity(c, h);
  TRY(target_hash(c, &h.target_hash));
  const int m = c->cfg.pop_size;
  const size_t par = (size_t)(gen & 1);
  DevState st{};
  CK(cudaMemcpyAsync(&st, c->dstate, sizeof st, cudaMemcpyDeviceToHost, c->stream));
  std::vector<int> rowmap((size_t)m);
  CK(cudaMemcpyAsync(rowmap.data(), c->perm + par * 2 * m, sizeof(int) * m,
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  TRY(check_device_error(c));
  h.generation = gen;
  h.best_slot = st.best_slot;
  h.payload_bytes = payload_bytes(c, gen);
  unsigned char *p = static_cast<unsigned char *>(buf);
  memcpy(p, &h, sizeof h);
  p += sizeof h;
  const size_t N = (size_t)c->N;
  for (int i = 0; i < m; ++i, p += sizeof(float) * N)
    CK(cudaMemcpyAsync(p, c->pool + (size_t)rowmap[(size_t)i] * c->n_pad, sizeof(float) * N,
                       cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(p, c->fit + par * m, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream));
  p += sizeof(double) * m;
  CK(cudaMemcpyAsync(p, c->fit_te + par * m, sizeof(double) * m, cudaMemcpyDeviceToHost,
                     c->stream));
  p += sizeof(double) * m;
  if (gen > 0) {
    CK(cudaMemcpyAsync(p, c->trace, sizeof(int4) * (size_t)gen * m, cudaMemcpyDeviceToHost,
                       c->stream));
    p += sizeof(int4) * (size_t)gen * m;
    CK(cudaMemcpyAsync(p, c->best_log, sizeof(double2) * (size_t)gen, cudaMemcpyDeviceToHost,
                       c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return GSGP_OK;
  API_END(c)
}

extern "C" gsgp_status gsgp_restore(gsgp_ctx *c, const void *buf, size_t size) {
  API_GUARD(c)
  if (c->state < 1) return fail(c, GSGP_E_STATE, "gsgp_restore before gsgp_load");
  if (c->sharded) return fail(c, GSGP_E_STATE, "checkpoints of case shards are not supported");
  if (!buf || size < sizeof(Header)) return fail(c, GSGP_E_INVALID, "checkpoint too short");
  Header h;
  memcpy(&h, buf, sizeof h);
  if (memcmp(h.magic, kMagic, sizeof kMagic) != 0 || h.header_bytes != sizeof(Header))
    return fail(c, GSGP_E_INVALID, "not a checkpoint of this library version");
  Header mine;
  memset(&mine, 0, sizeof mine);
  fill_identity(c, mine);
  TRY(use_device(c));
  TRY(target_hash(c, &mine.target_hash));
  if (!same_identity(h, mine))
    return fail(c, GSGP_E_INVALID,
                "the checkpoint belongs to another configuration or other data");
  const int m = c->cfg.pop_size;
  if (h.generation < 0 || h.best_slot < 0 || h.best_slot >= m ||
      h.payload_bytes != payload_bytes(c, h.generation) ||
      size != sizeof(Header) + h.payload_bytes)
    return fail(c, GSGP_E_INVALID, "corrupt checkpoint (sizes)");
  // the deterministic part: programs, random-tree semantics, initial state
  TRY(gsgp_init(c));
  c->state = 1;   // until the saved state is installed
  const int gen = h.generation;
  TRY(ensure_trace(c, gen > 64 ? gen : 64));
  // install the saved population as slots 0..m-1 in rows 0..m-1 of the
  // tables of parity gen & 1
  const size_t par = (size_t)(gen & 1);
  std::vector<int> ident((size_t)(2 * m));
  for (int i = 0; i < 2 * m; ++i) ident[(size_t)i] = i;
  CK(cudaMemcpyAsync(c->perm + par * 2 * m, ident.data(), sizeof(int) * 2 * m,
                     cudaMemcpyHostToDevice, c->stream));
  const unsigned char *p = static_cast<const unsigned char *>(buf) + sizeof(Header);
  const size_t N = (size_t)c->N;
  CK(cudaMemcpy2DAsync(c->pool, sizeof(float) * c->n_pad, p, sizeof(float) * N,
                       sizeof(float) * N, (size_t)m, cudaMemcpyHostToDevice, c->stream));
  p += sizeof(float) * N * m;
  CK(cudaMemcpyAsync(c->fit + par * m, p, sizeof(double) * m, cudaMemcpyHostToDevice, c->stream));
  p += sizeof(double) * m;
  CK(cudaMemcpyAsync(c->fit_te + par * m, p, sizeof(double) * m, cudaMemcpyHostToDevice,
                     c->stream));
  p += sizeof(double) * m;
  if (gen > 0) {
    CK(cudaMemcpyAsync(c->trace, p, sizeof(int4) * (size_t)gen * m, cudaMemcpyHostToDevice,
                       c->stream));
    p += sizeof(int4) * (size_t)gen * m;
    CK(cudaMemcpyAsync(c->best_log, p, sizeof(double2) * (size_t)gen, cudaMemcpyHostToDevice,
                       c->stream));
  }
  DevState st{};
  st.gen = gen;
  st.parity = (int)par;
  st.done = 0u;
  st.best_slot = h.best_slot;
  CK(cudaMemcpyAsync(c->dstate, &st, sizeof st, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));   // the host buffers above are the caller's / local
  c->gen = gen;
  c->model_gen = -1;
  c->state = 2;
  return GSGP_OK;
  API_END(c)
}
