// C ABI entry points of include/sph.h: argument checks, context allocation
// and the sequencing of the device passes.
#include <string.h>

#include <algorithm>
#include <utility>

#include "sph_internal.cuh"

namespace sph {
void scan_counts(sph_ctx *c, const int32_t *in, int32_t *out, int64_t m, cudaStream_t st);
void export_nodes(sph_ctx *c, int64_t cap, int32_t *level, int64_t *cell, int64_t *count, double *mass, double *com,
                  cudaStream_t st);
}  // namespace sph

using namespace sph;

namespace sph {
std::atomic<int64_t> g_launches{0};

int prof_begin(sph_ctx *c, cudaStream_t st, int phase) {
  if (!c->prof || c->prof_used >= kMaxProfEvents) return -1;
  int i = c->prof_used++;
  c->prof_phase[i] = phase;
  cudaEventRecord(c->prof_ev[2 * i], st);
  return i;
}

void prof_end(sph_ctx *c, cudaStream_t st, int idx) {
  if (idx >= 0) cudaEventRecord(c->prof_ev[2 * idx + 1], st);
}
}  // namespace sph

static sph_status fail(sph_ctx *c, sph_status s, const char *msg) {
  if (c) snprintf(c->err, sizeof(c->err), "%s", msg);
  return s;
}

static sph_status cuda_check(sph_ctx *c, const char *where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (c) snprintf(c->err, sizeof(c->err), "%s: %s", where, cudaGetErrorString(e));
    return SPH_ERR_CUDA;
  }
  return SPH_OK;
}

template <class T>
static T *ctx_alloc(sph_ctx *c, int64_t count, bool &ok) {
  constexpr int kMaxAllocs = (int)(sizeof(c->allocs) / sizeof(c->allocs[0]));
  if (!ok || c->nallocs >= kMaxAllocs) {
    ok = false;
    return nullptr;
  }
  void *p = nullptr;
  size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    ok = false;
    return nullptr;
  }
  c->allocs[c->nallocs++] = p;
  c->bytes += (int64_t)bytes;
  return (T *)p;
}

extern "C" {

sph_status sph_create(sph_ctx **out, int32_t dim, int64_t max_particles, int32_t max_instances,
                      int32_t max_neighbours, int32_t leaf_size, void *stream) {
  (void)stream;
  if (!out) return SPH_ERR_INVALID;
  *out = nullptr;
  if ((dim != 2 && dim != 3) || max_particles < 1 || max_particles > ((int64_t)1 << 31) - 64 ||
      max_instances < 1 || max_neighbours < 1 || leaf_size < 1 || leaf_size > kMaxLeaf)
    return SPH_ERR_INVALID;
  sph_ctx *c = new sph_ctx();
  memset(c, 0, sizeof(*c));
  cudaGetDevice(&c->device);
  c->dim = dim;
  c->cap_n = max_particles;
  c->cap_inst = max_instances;
  c->kmax = max_neighbours;
  c->leaf_default = leaf_size;
  c->tune.walk_leaf = 64;
  c->tune.walk_blocks_per_sm = 16;
  c->tune.pass_threads = 128;
  c->tune.walk_every_eval = 0;
  c->tune.iter_cap = 0;
  c->tune.plain_forms = 0;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (c->num_sms < 1) c->num_sms = 1;
  const int64_t N = max_particles;
  bool ok = true;
  c->d_err = ctx_alloc<int32_t>(c, 1, ok);
  if (cudaMallocHost(&c->h_err, sizeof(int32_t)) != cudaSuccess) ok = false;
  Tree &T = c->tree;
  for (int k = 0; k < 2; ++k) {
    T.keys[k] = ctx_alloc<unsigned long long>(c, N, ok);
    T.vals[k] = ctx_alloc<int32_t>(c, N, ok);
  }
  T.hist_cap = (int64_t)256 * ((N + 4095) / 4096 + 1);
  T.hist = ctx_alloc<uint32_t>(c, T.hist_cap, ok);
  T.ncount = ctx_alloc<int32_t>(c, N + 1, ok);
  T.nstart = ctx_alloc<int32_t>(c, N + 1, ok);
  T.cap_nodes = std::max<int64_t>(4096, leaf_size <= 2 ? 4 * N : 2 * N);
  T.scan_tmp = ctx_alloc<int32_t>(c, (std::max(N, T.cap_nodes) + 1) / 4096 + 2, ok);
  const int64_t cn = T.cap_nodes;
  T.nnodes = ctx_alloc<int32_t>(c, 1, ok);
  T.nleaf = ctx_alloc<int32_t>(c, 1, ok);
  T.first = ctx_alloc<int32_t>(c, cn, ok);
  T.end = ctx_alloc<int32_t>(c, cn, ok);
  T.skip = ctx_alloc<int32_t>(c, cn, ok);
  T.parent = ctx_alloc<int32_t>(c, cn, ok);
  T.nchild = ctx_alloc<int32_t>(c, cn, ok);
  T.arrived = ctx_alloc<int32_t>(c, cn, ok);
  T.child = ctx_alloc<int32_t>(c, 8 * cn, ok);
  T.nrec = ctx_alloc<int4>(c, cn, ok);
  T.level = ctx_alloc<int32_t>(c, cn, ok);
  T.cell = ctx_alloc<unsigned long long>(c, cn, ok);
  T.mass = ctx_alloc<double>(c, cn, ok);
  T.com = ctx_alloc<double>(c, 3 * cn, ok);
  T.bblo = ctx_alloc<double>(c, 3 * cn, ok);
  T.bbhi = ctx_alloc<double>(c, 3 * cn, ok);
  T.hmax = ctx_alloc<double>(c, cn, ok);
  T.fbox_lo = ctx_alloc<float4>(c, cn, ok);
  T.fbox_hi = ctx_alloc<float4>(c, cn, ok);
  T.fcom_hi = ctx_alloc<float4>(c, cn, ok);
  T.fcom_lo = ctx_alloc<float4>(c, cn, ok);
  const int64_t ci = max_instances;
  T.inst_bb = ctx_alloc<unsigned long long>(c, 6 * ci, ok);
  T.inst_lo = ctx_alloc<double>(c, 3 * ci, ok);
  T.inst_s0 = ctx_alloc<double>(c, ci, ok);
  T.inst_rs0 = ctx_alloc<double>(c, ci, ok);
  T.inst_root = ctx_alloc<int32_t>(c, ci, ok);
  T.gcnt = ctx_alloc<int32_t>(c, cn + 1, ok);
  T.gstart = ctx_alloc<int32_t>(c, cn + 1, ok);
  T.cap_groups = N + ci + 1;
  T.grp_start = ctx_alloc<int32_t>(c, T.cap_groups, ok);
  T.grp_end = ctx_alloc<int32_t>(c, T.cap_groups, ok);
  T.grp_inst = ctx_alloc<int32_t>(c, T.cap_groups, ok);
  T.ngroups = ctx_alloc<int32_t>(c, 1, ok);
  c->pk.px_ = ctx_alloc<float4>(c, N, ok);
  c->pk.pxl_ = ctx_alloc<float4>(c, N, ok);
  c->pk.pv_ = ctx_alloc<float4>(c, N, ok);
  c->pk.pvl_ = ctx_alloc<float4>(c, N, ok);
  c->nb_idx = ctx_alloc<int32_t>(c, (int64_t)max_neighbours * N, ok);
  c->nb_cnt = ctx_alloc<int32_t>(c, N, ok);
  c->nb_alt = ctx_alloc<int32_t>(c, (int64_t)max_neighbours * N, ok);
  c->nb_cnt_alt = ctx_alloc<int32_t>(c, N, ok);
  c->sh_idx = ctx_alloc<int32_t>(c, (int64_t)kMaxShell * N, ok);
  c->sh_cnt = ctx_alloc<int32_t>(c, N, ok);
  c->sh_in = ctx_alloc<int32_t>(c, N, ok);
  c->need_walk = ctx_alloc<int32_t>(c, 1, ok);
  c->csr_total = ctx_alloc<int64_t>(c, 1, ok);
  c->hflags = ctx_alloc<int32_t>(c, kMaxHIter + 3, ok);
  c->T = ctx_alloc<double>(c, 8 * N, ok);
  c->zeta = ctx_alloc<double>(c, 8 * N, ok);
  c->cs = ctx_alloc<double>(c, N, ok);
  c->p = ctx_alloc<double>(c, N, ok);
  c->ag = ctx_alloc<double>(c, 3 * N, ok);
  c->units = ctx_alloc<Units>(c, 1, ok);
  c->d_ctr = ctx_alloc<unsigned long long>(c, kNumCounters, ok);
  c->adj_inter = ctx_alloc<double>(c, 22 * N, ok);
  c->adj32 = ctx_alloc<float4>(c, 7 * N, ok);
  c->adj_sums = ctx_alloc<float>(c, 16 * N, ok);
  c->vscale = 1.0;
  StepBufs &S = c->st;
  for (int k = 0; k < 3; ++k) {
    S.x[k] = ctx_alloc<double>(c, N, ok);
    S.v[k] = ctx_alloc<double>(c, N, ok);
  }
  S.rho = ctx_alloc<double>(c, N, ok);
  S.u = ctx_alloc<double>(c, N, ok);
  S.S = ctx_alloc<double>(c, 6 * N, ok);
  S.dmg = ctx_alloc<double>(c, N, ok);
  for (int s = 0; s < 3; ++s) {
    for (int k = 0; k < 3; ++k) {
      S.d_x[s][k] = ctx_alloc<double>(c, N, ok);
      S.d_v[s][k] = ctx_alloc<double>(c, N, ok);
    }
    S.d_rho[s] = ctx_alloc<double>(c, N, ok);
    S.d_u[s] = ctx_alloc<double>(c, N, ok);
    S.d_S[s] = ctx_alloc<double>(c, 6 * N, ok);
    S.d_dmg[s] = ctx_alloc<double>(c, N, ok);
    S.d_cs[s] = ctx_alloc<double>(c, N, ok);
    S.d_nact[s] = ctx_alloc<int32_t>(c, N, ok);
  }
  S.dt_enc = ctx_alloc<unsigned long long>(c, ci, ok);
  S.rk_err = ctx_alloc<unsigned long long>(c, ci, ok);
  S.rk_acc = ctx_alloc<int32_t>(c, ci, ok);
  S.dmove = ctx_alloc<unsigned long long>(c, 1, ok);
  S.dbuild = ctx_alloc<unsigned long long>(c, 1, ok);
  S.dgrow = ctx_alloc<unsigned long long>(c, 1, ok);
  S.dt = ctx_alloc<double>(c, ci, ok);
  S.gather = ctx_alloc<double>(c, N, ok);
  S.gather_i = ctx_alloc<int32_t>(c, N, ok);
  for (int k = 0; k < 4; ++k) S.snap[k] = ctx_alloc<double>(c, N, ok);
  S.differ = ctx_alloc<int32_t>(c, 1, ok);
  FlawBufs &F = c->fl;
  F.cap_groups = (int64_t)ci * SPH_MAX_MATERIALS;
  F.cap_plan = (int)F.cap_groups;
  F.goff = ctx_alloc<int32_t>(c, F.cap_groups + 1, ok);
  F.kv = ctx_alloc<double>(c, F.cap_groups, ok);
  F.invm = ctx_alloc<double>(c, F.cap_groups, ok);
  F.J = ctx_alloc<uint32_t>(c, F.cap_groups, ok);
  F.unc = ctx_alloc<int32_t>(c, F.cap_groups, ok);
  F.plan_grp = ctx_alloc<int32_t>(c, F.cap_groups, ok);
  F.plan_b0 = ctx_alloc<int64_t>(c, F.cap_groups, ok);
  F.plan_pre = ctx_alloc<int64_t>(c, F.cap_groups + 1, ok);
  F.bad = ctx_alloc<int32_t>(c, 1, ok);
  F.cap_chunks = (int)(N / 4096 + F.cap_groups + 1);  // chunks of 4096 members
  F.ck_g = ctx_alloc<int32_t>(c, F.cap_chunks, ok);
  F.ck_lo = ctx_alloc<int32_t>(c, F.cap_chunks, ok);
  F.ck_hi = ctx_alloc<int32_t>(c, F.cap_chunks, ok);
  F.ck_sum = ctx_alloc<double>(c, F.cap_chunks, ok);
  F.g_ck = ctx_alloc<int32_t>(c, F.cap_groups + 1, ok);
  if (ok) ok = cudaMemset(c->d_err, 0, sizeof(int32_t)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    sph_destroy(c);
    return SPH_ERR_CUDA;
  }
  *out = c;
  return SPH_OK;
}

void sph_destroy(sph_ctx *c) {
  if (!c) return;
  if (c->prof_ev) {
    for (int i = 0; i < 2 * kMaxProfEvents; ++i) cudaEventDestroy(c->prof_ev[i]);
    delete[] c->prof_ev;
    delete[] c->prof_phase;
  }
  for (int i = 0; i < c->nallocs; ++i) cudaFree(c->allocs[i]);
  if (c->h_err) cudaFreeHost(c->h_err);
  delete c;
}

const char *sph_last_error(const sph_ctx *c) { return c ? c->err : "no context"; }

int64_t sph_ctx_bytes(const sph_ctx *c) { return c ? c->bytes : 0; }

sph_status sph_sync_status(sph_ctx *c, void *stream) {
  if (!c) return SPH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(c, SPH_ERR_CUDA, cudaGetErrorString(e));
  int32_t w = *c->h_err;
  cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), st);
  if (w & ERR_NONFINITE) return fail(c, SPH_ERR_NONFINITE, "non-finite input, or h <= 0 or rho <= 0");
  if (w & (ERR_NB_OVERFLOW | ERR_NODE_OVERFLOW | ERR_CSR_OVERFLOW))
    return fail(c, SPH_ERR_CAPACITY,
                (w & ERR_NB_OVERFLOW) ? "a particle has more partners than max_neighbours"
                : (w & ERR_NODE_OVERFLOW) ? "octree node capacity exceeded"
                                          : "partner list longer than nb_capacity");
  if (w & ERR_TIMEOUT) return fail(c, SPH_ERR_TIMEOUT, "a bounded device loop hit its iteration limit");
  return SPH_OK;
}

}  // extern "C"

static sph_status check_state(sph_ctx *c, const sph_state *s) {
  if (!c || !s) return SPH_ERR_INVALID;
  // any call may rebuild the tree or rewrite the partner lists: the window a
  // previous sph_step left is only kept for an sph_step that continues it
  c->win_was = c->win_valid;
  c->win_valid = false;
  if (s->dim != c->dim) return fail(c, SPH_ERR_INVALID, "state dim differs from the context's");
  if (s->n < 0 || s->n > c->cap_n) return fail(c, SPH_ERR_INVALID, "n exceeds the context capacity");
  int ninst = s->ninst > 0 ? s->ninst : 1;
  if (ninst > c->cap_inst) return fail(c, SPH_ERR_INVALID, "ninst exceeds the context capacity");
  if (ninst > 1 && !s->inst_off) return fail(c, SPH_ERR_INVALID, "inst_off is required when ninst > 1");
  if (s->n > 0) {
    for (int ax = 0; ax < s->dim; ++ax)
      if (!s->x[ax] || !s->v[ax]) return fail(c, SPH_ERR_INVALID, "missing position or velocity array");
    if (!s->rho || !s->u || !s->m || !s->h) return fail(c, SPH_ERR_INVALID, "missing rho, u, m or h");
  }
  return SPH_OK;
}

static sph_status check_tree_args(sph_ctx *c, const sph_state *s, int leaf, int depth) {
  if (leaf < 1 || leaf > kMaxLeaf) return fail(c, SPH_ERR_INVALID, "leaf_size must be in 1..32");
  int ninst = s->ninst > 0 ? s->ninst : 1;
  int ibits = 0;
  while ((1 << ibits) < ninst) ++ibits;
  if (depth < 1 || depth > 21 || s->dim * depth + ibits > 64)
    return fail(c, SPH_ERR_INVALID, "max_depth must be in 1..21 with dim * max_depth + log2(ninst) <= 64");
  return SPH_OK;
}

static sph_status check_params(sph_ctx *c, const sph_state *s, const sph_material *mats, int nmat,
                               const sph_params *p, MatTable &mt) {
  if (!p || !mats || nmat < 1 || nmat > SPH_MAX_MATERIALS)
    return fail(c, SPH_ERR_INVALID, "params and 1..8 materials are required");
  if (p->dim != s->dim) return fail(c, SPH_ERR_INVALID, "params.dim differs from the state's");
  if (p->precision != SPH_FP64 && p->precision != SPH_MIXED) return fail(c, SPH_ERR_INVALID, "bad precision");
  if (p->eps_s > 0.0 && !(p->dmpd > 0.0)) return fail(c, SPH_ERR_INVALID, "artificial stress needs dmpd > 0");
  if (p->tree_reuse < 0) return fail(c, SPH_ERR_INVALID, "tree_reuse must be >= 0");
  if (p->n_des > 0.0 && (p->h_tol < 0 || p->h_iter < 0 || p->h_iter > kMaxHIter))
    return fail(c, SPH_ERR_INVALID, "variable h needs h_tol >= 0 and 0 <= h_iter <= 64");
  memset(&mt, 0, sizeof(mt));
  for (int i = 0; i < nmat; ++i) {
    mt.m[i] = mats[i];
    if (mats[i].damage && (!s->flaw_off || !s->flaw_eps) && s->dmg)
      return fail(c, SPH_ERR_INVALID, "damage needs flaw_off and flaw_eps");
    if (!(mats[i].rho0 > 0.0)) return fail(c, SPH_ERR_INVALID, "material rho0 must be positive");
  }
  mt.nmat = nmat;
  return check_tree_args(c, s, p->leaf_size, p->max_depth);
}

namespace sph {
// Velocity scale of the materials (sound speed, or sqrt(K / rho0)), for the
// time unit of the FP32 views.
double velocity_scale(const MatTable &mt) {
  double v = 0.0;
  for (int i = 0; i < mt.nmat; ++i) {
    const sph_material &m = mt.m[i];
    double c = m.cs;
    double K = std::max(m.K0, std::max(m.A_T, m.B_T));
    if (!(c > 0.0) && K > 0.0 && m.rho0 > 0.0) c = sqrt(K / m.rho0);
    if (c > v) v = c;
  }
  return v > 0.0 ? v : 1.0;
}
}  // namespace sph

static void set_materials(sph_ctx *c, const MatTable *mt) {
  if (mt) {
    c->mt = *mt;
    c->vscale = velocity_scale(*mt);
  } else {
    memset(&c->mt, 0, sizeof(c->mt));
    c->vscale = 1.0;
  }
}

static sph_status finish(sph_ctx *c, const sph_params *p, cudaStream_t st, const char *where) {
  sph_status r = cuda_check(c, where);
  if (r != SPH_OK) return r;
  if (p && p->check) return sph_sync_status(c, st);
  return SPH_OK;
}

// One full right-hand side on state s into out (tree + partners + passes).
static void timed_tree(sph_ctx *c, const sph_state *s, const sph_params &p, cudaStream_t st) {
  int pr = prof_begin(c, st, PH_TREE);
  tree_build(c, s, p.leaf_size, p.max_depth, st);
  prof_end(c, st, pr);
}

// grow: displacement bound since the tree build (NULL: built at s);
// greuse: gravity from the pseudo-particles of an earlier build;
// shell: the walk also records the partner shells (for a later refine);
// move: refine the partners from the lists and shells of the last walk, which
// every particle has left by at most *move per axis (NULL: walk)
static void partners_gravity_passes(sph_ctx *c, sph_state *s, const MatTable &mt, const sph_params &p,
                                    const sph_derivs &out, cudaStream_t st,
                                    const unsigned long long *grow = nullptr, bool greuse = false,
                                    bool shell = false, const unsigned long long *move = nullptr) {
  int pr;
  if (move) {
    pr = prof_begin(c, st, PH_REFINE);
    refine_partners(c, s, move, grow, st);
    prof_end(c, st, pr);
    std::swap(c->nb_idx, c->nb_alt);  // the passes read the refined lists
    std::swap(c->nb_cnt, c->nb_cnt_alt);
  } else {
    pr = prof_begin(c, st, PH_PARTNERS);
    find_partners(c, s, st, grow, shell);
    prof_end(c, st, pr);
  }
  if (p.gravity) {
    pr = prof_begin(c, st, PH_GRAVITY);
    gravity_walk(c, s, p, c->ag, c->ag + c->cap_n, c->ag + 2 * c->cap_n, st, greuse);
    prof_end(c, st, pr);
  }
  rhs_passes(c, s, mt, p, out, st);
  if (move) {  // the walk's lists, counts and shells stay for the next refine
    std::swap(c->nb_idx, c->nb_alt);
    std::swap(c->nb_cnt, c->nb_cnt_alt);
  }
}

static void rhs_all(sph_ctx *c, sph_state *s, const MatTable &mt, const sph_params &p, const sph_derivs &out,
                    cudaStream_t st) {
  timed_tree(c, s, p, st);
  partners_gravity_passes(c, s, mt, p, out, st);
}

extern "C" {

sph_status sph_build_tree(sph_ctx *c, sph_state *s, int32_t leaf_size, int32_t max_depth, int32_t reorder,
                          int32_t *perm, void *stream) {
  sph_status r = check_state(c, s);
  if (r != SPH_OK) return r;
  if ((r = check_tree_args(c, s, leaf_size, max_depth)) != SPH_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  set_materials(c, nullptr);
  tree_build(c, s, leaf_size, max_depth, st);
  if (perm && s->n > 0)
    cudaMemcpyAsync(perm, c->tree.perm, sizeof(int32_t) * s->n, cudaMemcpyDeviceToDevice, st);
  if (reorder) tree_reorder_state(c, s, st);
  return cuda_check(c, "sph_build_tree");
}

sph_status sph_tree_nodes(sph_ctx *c, int64_t cap, int32_t *level, int64_t *cell, int64_t *count, double *mass,
                          double *com, int64_t *nnodes, void *stream) {
  if (!c || !nnodes) return SPH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t nn = 0;
  cudaMemcpyAsync(&nn, c->tree.nnodes, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(c, "sph_tree_nodes");
  *nnodes = nn;
  if (nn > cap) return fail(c, SPH_ERR_CAPACITY, "node list longer than cap");
  if (nn > 0) export_nodes(c, nn, level, cell, count, mass, com, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(c, "sph_tree_nodes");
  return sph_sync_status(c, stream);
}

sph_status sph_neighbours(sph_ctx *c, const sph_state *s, int32_t leaf_size, int32_t max_depth, int64_t *nb_offset,
                          int32_t *nb_index, int64_t nb_capacity, void *stream) {
  sph_status r = check_state(c, s);
  if (r != SPH_OK) return r;
  if ((r = check_tree_args(c, s, leaf_size, max_depth)) != SPH_OK) return r;
  if (!nb_offset || (!nb_index && nb_capacity > 0)) return fail(c, SPH_ERR_INVALID, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  set_materials(c, nullptr);
  tree_build(c, s, leaf_size, max_depth, st);
  find_partners(c, s, st);
  partners_to_csr(c, s, nb_offset, nb_index, nb_capacity, st);
  if ((r = cuda_check(c, "sph_neighbours")) != SPH_OK) return r;
  return sph_sync_status(c, stream);
}

sph_status sph_adapt_h(sph_ctx *c, sph_state *s, int32_t leaf_size, int32_t max_depth, double n_des, int32_t tol,
                       int32_t max_iter, int32_t *counts, int32_t *updates, void *stream) {
  sph_status r = check_state(c, s);
  if (r != SPH_OK) return r;
  if ((r = check_tree_args(c, s, leaf_size, max_depth)) != SPH_OK) return r;
  if (!(n_des > 0.0) || tol < 0 || max_iter < 0 || max_iter > kMaxHIter)
    return fail(c, SPH_ERR_INVALID, "need n_des > 0, tol >= 0 and 0 <= max_iter <= 64");
  cudaStream_t st = (cudaStream_t)stream;
  set_materials(c, nullptr);
  tree_build(c, s, leaf_size, max_depth, st);  // positions only: the counts use the current h
  adapt_h(c, s, n_des, tol, max_iter, c->hflags, st);
  if (counts && s->n > 0) cudaMemcpyAsync(counts, c->nb_cnt, sizeof(int32_t) * s->n, cudaMemcpyDeviceToDevice, st);
  int32_t u = 0;
  cudaMemcpyAsync(&u, c->hflags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if ((r = cuda_check(c, "sph_adapt_h")) != SPH_OK) return r;
  if ((r = sph_sync_status(c, stream)) != SPH_OK) return r;
  if (updates) *updates = u;
  return SPH_OK;
}

sph_status sph_flaws(sph_ctx *c, const sph_state *s, const sph_material *mats, int32_t nmat, const double *weibull_k,
                     const double *weibull_m, uint64_t seed, int64_t *flaw_off, float *flaw_eps,
                     int64_t eps_capacity, int64_t *nflaws, void *stream) {
  if (!c || !s) return SPH_ERR_INVALID;
  c->win_valid = false;  // its sort runs on the tree's scratch
  if (s->n < 0 || s->n > c->cap_n) return fail(c, SPH_ERR_INVALID, "n exceeds the context capacity");
  const int ninst = s->ninst > 0 ? s->ninst : 1;
  if (ninst > c->cap_inst) return fail(c, SPH_ERR_INVALID, "ninst exceeds the context capacity");
  if (ninst > 1 && !s->inst_off) return fail(c, SPH_ERR_INVALID, "inst_off is required when ninst > 1");
  if (!mats || nmat < 1 || nmat > SPH_MAX_MATERIALS || !weibull_k || !weibull_m || !nflaws)
    return fail(c, SPH_ERR_INVALID, "need materials (1..8), weibull_k, weibull_m and nflaws");
  if (s->n > 0 && (!s->mat || !s->id || !s->m)) return fail(c, SPH_ERR_INVALID, "need mat, id and m");
  if (eps_capacity < 0 || (flaw_eps && !flaw_off)) return fail(c, SPH_ERR_INVALID, "bad flaw output");
  for (int k = 0; k < nmat; ++k)
    if (mats[k].damage && weibull_k[k] > 0.0 && weibull_m[k] > 0.0 && !(mats[k].rho0 > 0.0))
      return fail(c, SPH_ERR_INVALID, "a brittle material needs rho0 > 0");
  cudaStream_t st = (cudaStream_t)stream;
  sph_status r = flaws_generate(c, s, mats, nmat, weibull_k, weibull_m, seed, flaw_off, flaw_eps, eps_capacity,
                                nflaws, st);
  if (r == SPH_ERR_CUDA) {
    const sph_status e = cuda_check(c, "sph_flaws");
    return e != SPH_OK ? e : fail(c, r, "sph_flaws: stream synchronisation failed");
  }
  if (r != SPH_OK) return r;
  if ((r = cuda_check(c, "sph_flaws")) != SPH_OK) return r;
  return sph_sync_status(c, stream);
}

sph_status sph_fragments(sph_ctx *c, const sph_state *s, const double *h0, double link, double d_remove,
                         int32_t min_size, int32_t leaf_size, int32_t max_depth, int32_t *label, int32_t *frag_count,
                         double *frag_mass, int64_t frag_capacity, int64_t *nfrag, void *stream) {
  sph_status r = check_state(c, s);
  if (r != SPH_OK) return r;
  if ((r = check_tree_args(c, s, leaf_size, max_depth)) != SPH_OK) return r;
  if (!(link > 0.0) || min_size < 1 || frag_capacity < 0 || !nfrag || (s->n > 0 && !label))
    return fail(c, SPH_ERR_INVALID, "need link > 0, min_size >= 1, label and nfrag");
  cudaStream_t st = (cudaStream_t)stream;
  set_materials(c, nullptr);
  fragments_fof(c, s, h0, link, d_remove, min_size, leaf_size, max_depth, label, frag_count, frag_mass,
                frag_capacity, nfrag, st);
  if ((r = cuda_check(c, "sph_fragments")) != SPH_OK) return r;
  if ((r = sph_sync_status(c, stream)) != SPH_OK) return r;
  if (*nfrag > frag_capacity)
    return fail(c, SPH_ERR_CAPACITY, "more fragments than frag_capacity (labels and nfrag are complete)");
  return SPH_OK;
}

sph_status sph_rhs(sph_ctx *c, sph_state *s, const sph_material *mats, int32_t nmat, const sph_params *p,
                   sph_derivs *out, void *stream) {
  sph_status r = check_state(c, s);
  if (r != SPH_OK) return r;
  MatTable mt;
  if ((r = check_params(c, s, mats, nmat, p, mt)) != SPH_OK) return r;
  if (!out) return fail(c, SPH_ERR_INVALID, "null derivs");
  for (int ax = 0; ax < s->dim && s->n > 0; ++ax)
    if (!out->dx[ax] || !out->dv[ax]) return fail(c, SPH_ERR_INVALID, "dx and dv outputs are required");
  if (s->n > 0 && (!out->drho || !out->du)) return fail(c, SPH_ERR_INVALID, "drho and du outputs are required");
  if (s->n > 0 && s->S && !out->dS) return fail(c, SPH_ERR_INVALID, "dS output required when S is given");
  if (s->n > 0 && s->dmg && !out->ddmg) return fail(c, SPH_ERR_INVALID, "ddmg output required when dmg is given");
  cudaStream_t st = (cudaStream_t)stream;
  set_materials(c, &mt);
  rhs_all(c, s, mt, *p, *out, st);
  return finish(c, p, st, "sph_rhs");
}

sph_status sph_gravity(sph_ctx *c, const sph_state *s, const sph_params *p, double *ax, double *ay, double *az,
                       void *stream) {
  sph_status r = check_state(c, s);
  if (r != SPH_OK) return r;
  if (!p) return fail(c, SPH_ERR_INVALID, "null params");
  if ((r = check_tree_args(c, s, p->leaf_size, p->max_depth)) != SPH_OK) return r;
  if (!ax || !ay || (s->dim == 3 && !az)) return fail(c, SPH_ERR_INVALID, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  set_materials(c, nullptr);
  int pr = prof_begin(c, st, PH_TREE);
  tree_build(c, s, p->leaf_size, p->max_depth, st);
  prof_end(c, st, pr);
  pr = prof_begin(c, st, PH_GRAVITY);
  gravity_walk(c, s, *p, ax, ay, az, st);
  prof_end(c, st, pr);
  return finish(c, p, st, "sph_gravity");
}

// *differ = 1 when a position or h of the state differs (bit for bit) from
// the copy the last sph_step call kept (s0..s3: x, y, z or unused, h)
__global__ void k_differs(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                          const double *__restrict__ h, const double *__restrict__ s0, const double *__restrict__ s1,
                          const double *__restrict__ s2, const double *__restrict__ s3, int dim, int64_t n,
                          int32_t *differ) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  bool d = __double_as_longlong(x[a]) != __double_as_longlong(s0[a]) ||
           __double_as_longlong(y[a]) != __double_as_longlong(s1[a]) ||
           __double_as_longlong(h[a]) != __double_as_longlong(s3[a]);
  if (dim == 3) d = d || __double_as_longlong(z[a]) != __double_as_longlong(s2[a]);
  if (d) *differ = 1;
}

// Checks the promise of params.tree_continue: the previous call on c was an
// sph_step that left a tree window with the same settings, and the state's
// positions and h are those it returned.  Blocks on the stream.
static sph_status check_continue(sph_ctx *c, const sph_state *s, const sph_params *p, cudaStream_t st) {
  const int ninst = s->ninst > 0 ? s->ninst : 1;
  if (!c->win_was || c->win_R != p->tree_reuse || c->win_n != s->n || c->win_ninst != ninst ||
      c->win_leaf != p->leaf_size || c->win_depth != p->max_depth || c->win_gravity != (p->gravity != 0))
    return fail(c, SPH_ERR_INVALID,
                "tree_continue: the previous call on this context was not an sph_step with the same tree_reuse, "
                "n, instances, leaf_size, max_depth and gravity setting");
  if (s->n == 0) return SPH_OK;
  StepBufs &B = c->st;
  cudaMemsetAsync(B.differ, 0, sizeof(int32_t), st);
  { k_differs<<<nblk(s->n, 256), 256, 0, st>>>(s->x[0], s->x[1], s->dim == 3 ? s->x[2] : s->x[0], s->h, B.snap[0],
                                              B.snap[1], B.snap[2], B.snap[3], s->dim, s->n, B.differ); ++g_launches; }
  int32_t d = 0;
  cudaMemcpyAsync(&d, B.differ, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(c, "sph_step");
  if (d) return fail(c, SPH_ERR_INVALID, "tree_continue: positions or h differ from those the previous sph_step returned");
  return SPH_OK;
}

// Keeps what a later call needs to continue the tree window of this one.
static void keep_window(sph_ctx *c, const sph_state *s, const sph_params *p, int age, cudaStream_t st) {
  StepBufs &B = c->st;
  const int64_t n = s->n;
  for (int k = 0; k < s->dim; ++k) cudaMemcpyAsync(B.snap[k], s->x[k], sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(B.snap[3], s->h, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  c->win_valid = true;
  c->win_age = age;
  c->win_R = p->tree_reuse;
  c->win_n = n;
  c->win_ninst = s->ninst > 0 ? s->ninst : 1;
  c->win_leaf = p->leaf_size;
  c->win_depth = p->max_depth;
  c->win_gravity = p->gravity != 0;
}

sph_status sph_step(sph_ctx *c, sph_state *s, const sph_material *mats, int32_t nmat, const sph_params *p, double *dt,
                    int32_t nsteps, void *stream) {
  sph_status r = check_state(c, s);
  if (r != SPH_OK) return r;
  MatTable mt;
  if ((r = check_params(c, s, mats, nmat, p, mt)) != SPH_OK) return r;
  if (nsteps < 0) return fail(c, SPH_ERR_INVALID, "nsteps < 0");
  cudaStream_t st = (cudaStream_t)stream;
  set_materials(c, &mt);
  StepBufs &B = c->st;
  const int ninst = s->ninst > 0 ? s->ninst : 1;
  // predicted state shares m, h, mat, id, flaws and instances with s
  sph_state q = *s;
  for (int k = 0; k < 3; ++k) {
    q.x[k] = s->x[k] ? B.x[k] : nullptr;
    q.v[k] = s->v[k] ? B.v[k] : nullptr;
  }
  q.rho = B.rho;
  q.u = B.u;
  q.S = s->S ? B.S : nullptr;
  q.dmg = s->dmg ? B.dmg : nullptr;
  sph_derivs d[2];
  for (int j = 0; j < 2; ++j) {
    memset(&d[j], 0, sizeof(sph_derivs));
    for (int k = 0; k < 3; ++k) {
      d[j].dx[k] = B.d_x[j][k];
      d[j].dv[k] = B.d_v[j][k];
    }
    d[j].drho = B.d_rho[j];
    d[j].du = B.d_u[j];
    d[j].dS = B.d_S[j];
    d[j].ddmg = B.d_dmg[j];
    d[j].cs = B.d_cs[j];
    d[j].n_act = B.d_nact[j];
  }
  // Trees: without gravity the tree only serves the partner search, whose
  // result is exact for any tree, so the predicted state keeps the slots of s
  // and reuses its tree, the walk widening its boxes by the displacement
  // since the build.  Gravity's multipole sums depend on the tree: each
  // evaluation builds one, unless tree_reuse = R > 0 (the gravity/hydro
  // decoupling of Sect. 6.3), when the tree of a step start serves every
  // evaluation of R consecutive steps with its pseudo-particles (and, for the
  // partner search, boxes widened by the summed displacement bounds).
  const int R = p->tree_reuse > 0 ? p->tree_reuse : 0;
  const bool reuse_pred = !p->gravity || R > 0;
  // Later evaluations' partners: refined from the lists and shells of the
  // last walk, the step's first one or, on a reused tree, the build step's
  // (a walk follows only where the particles moved too far since it)
  const bool refine = reuse_pred && c->tune.walk_every_eval == 0;
  // a window of R steps on one tree may span calls (params.tree_continue)
  const bool window = R > 0 && !(p->n_des > 0.0);
  int age = 0;
  if (window && p->tree_continue) {
    if ((r = check_continue(c, s, p, st)) != SPH_OK) return r;
    age = c->win_age;
  }
  // the FP32 views hold s already: the last corrector wrote them (the first
  // step of a call packs, as the state may have been changed between calls)
  bool packed = false;
  const bool fuse = c->tune.plain_forms == 0;  // the update may write the views
  for (int it = 0; it < nsteps; ++it) {
    const bool vh = p->n_des > 0.0;
    if (vh) {  // variable smoothing length from the last step's h (Sect. 4.2)
      int pa = prof_begin(c, st, PH_PARTNERS);
      tree_build(c, s, p->leaf_size, p->max_depth, st);
      adapt_h(c, s, p->n_des, p->h_tol, p->h_iter, c->hflags, st);
      prof_end(c, st, pa);
    }
    const bool build = R == 0 || age == 0 || vh;  // h changes invalidate the node boxes
    int pr;
    if (build) {
      // order the state along the tree once per build (coalesced partner gathers)
      timed_tree(c, s, *p, st);
      pr = prof_begin(c, st, PH_REORDER);
      tree_reorder_state(c, s, st);
      prof_end(c, st, pr);
      if (R > 0) cudaMemsetAsync(B.dbuild, 0, sizeof(unsigned long long), st);
      partners_gravity_passes(c, s, mt, *p, d[0], st, nullptr, false, refine);
    } else {
      if (!packed) {
        pr = prof_begin(c, st, PH_TREE);
        pack_f32(c, s, st);
        prof_end(c, st, pr);
      }
      // the lists and shells of the build step's walk stay in place: while
      // the displacement since that walk is within the shell's bound, the
      // partners are refined from them (else a walk over the widened boxes)
      partners_gravity_passes(c, s, mt, *p, d[0], st, B.dbuild, p->gravity, false, refine ? B.dbuild : nullptr);
    }
    pr = prof_begin(c, st, PH_INTEGRATE);
    timestep_reduce(c, s, *p, d[0], st);
    if (reuse_pred) cudaMemsetAsync(B.dmove, 0, sizeof(unsigned long long), st);
    // on a kept tree the update also writes the predicted state's FP32 views
    pc_update(c, s, &q, d[0], 0.5, mt, *p, st, reuse_pred ? B.dmove : nullptr, reuse_pred && fuse);
    if (reuse_pred && !build) bound_add(B.dgrow, B.dbuild, B.dmove, st);
    prof_end(c, st, pr);
    if (reuse_pred) {
      if (!fuse) {
        pr = prof_begin(c, st, PH_TREE);
        pack_f32(c, &q, st);
        prof_end(c, st, pr);
      }
      // displacement since the walk whose lists are refined: this step's walk
      // at a build, the build step's walk otherwise
      const unsigned long long *since = build ? B.dmove : B.dgrow;
      partners_gravity_passes(c, &q, mt, *p, d[1], st, since, p->gravity, false, refine ? since : nullptr);
    } else {
      rhs_all(c, &q, mt, *p, d[1], st);
    }
    pr = prof_begin(c, st, PH_INTEGRATE);
    packed = false;
    if (R > 0) {  // the corrector's displacement joins the bound of the reused tree
      // views of the new state for the next step of this call, if it keeps the tree
      const bool keep = fuse && it + 1 < nsteps && !vh && (age + 1) % R != 0;
      cudaMemsetAsync(B.dmove, 0, sizeof(unsigned long long), st);
      pc_update(c, s, s, d[1], 1.0, mt, *p, st, B.dmove, keep);
      bound_add(B.dbuild, B.dbuild, B.dmove, st);
      age = (age + 1) % R;
      packed = keep;
    } else {
      pc_update(c, s, s, d[1], 1.0, mt, *p, st);
    }
    prof_end(c, st, pr);
  }
  if (dt && nsteps > 0) cudaMemcpyAsync(dt, B.dt, sizeof(double) * ninst, cudaMemcpyDeviceToDevice, st);
  if (window) keep_window(c, s, p, age, st);
  return finish(c, p, st, "sph_step");
}

sph_status sph_step_rk3(sph_ctx *c, sph_state *s, const sph_material *mats, int32_t nmat, const sph_params *p,
                        double eps_des, double *dt, double *t, int32_t nsteps, double *err_log, int32_t *acc_log,
                        void *stream) {
  sph_status r = check_state(c, s);
  if (r != SPH_OK) return r;
  MatTable mt;
  if ((r = check_params(c, s, mats, nmat, p, mt)) != SPH_OK) return r;
  if (nsteps < 0 || !dt || !(eps_des > 0.0)) return fail(c, SPH_ERR_INVALID, "need dt, eps_des > 0, nsteps >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  set_materials(c, &mt);
  StepBufs &B = c->st;
  const int ninst = s->ninst > 0 ? s->ninst : 1;
  // stage states share m, h, mat, id, flaws and instances with s
  sph_state q = *s;
  for (int k = 0; k < 3; ++k) {
    q.x[k] = s->x[k] ? B.x[k] : nullptr;
    q.v[k] = s->v[k] ? B.v[k] : nullptr;
  }
  q.rho = B.rho;
  q.u = B.u;
  q.S = s->S ? B.S : nullptr;
  q.dmg = s->dmg ? B.dmg : nullptr;
  sph_derivs d[3];
  for (int j = 0; j < 3; ++j) {
    memset(&d[j], 0, sizeof(sph_derivs));
    for (int k = 0; k < 3; ++k) {
      d[j].dx[k] = B.d_x[j][k];
      d[j].dv[k] = B.d_v[j][k];
    }
    d[j].drho = B.d_rho[j];
    d[j].du = B.d_u[j];
    d[j].dS = B.d_S[j];
    d[j].ddmg = B.d_dmg[j];
    d[j].cs = B.d_cs[j];
    d[j].n_act = B.d_nact[j];
  }
  const sph_derivs *k1[1] = {&d[0]}, *k12[2] = {&d[0], &d[1]}, *k123[3] = {&d[0], &d[1], &d[2]};
  const double c2[1] = {0.5}, c3[2] = {-1.0, 2.0}, cf[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};
  const bool reuse = !p->gravity;  // stage states keep the slots of s and use its tree (as in sph_step)
  const bool refine = reuse && c->tune.walk_every_eval == 0;  // stage partners refined from k1's walk
  auto stage = [&](const sph_derivs *const *k, const double *coef, int nd, sph_derivs &out) {
    int pr = prof_begin(c, st, PH_INTEGRATE);
    if (reuse) cudaMemsetAsync(B.dmove, 0, sizeof(unsigned long long), st);
    combine_update(c, s, &q, k, coef, nd, nullptr, mt, *p, st, reuse ? B.dmove : nullptr);
    prof_end(c, st, pr);
    if (reuse) {
      pr = prof_begin(c, st, PH_TREE);
      pack_f32(c, &q, st);
      prof_end(c, st, pr);
      partners_gravity_passes(c, &q, mt, *p, out, st, B.dmove, false, false, refine ? B.dmove : nullptr);
    } else {
      rhs_all(c, &q, mt, *p, out, st);
    }
  };
  for (int it = 0; it < nsteps; ++it) {
    if (p->n_des > 0.0) {  // variable smoothing length from the last step's h (Sect. 4.2)
      int pa = prof_begin(c, st, PH_PARTNERS);
      tree_build(c, s, p->leaf_size, p->max_depth, st);
      adapt_h(c, s, p->n_des, p->h_tol, p->h_iter, c->hflags, st);
      prof_end(c, st, pa);
    }
    timed_tree(c, s, *p, st);
    int pr = prof_begin(c, st, PH_REORDER);
    tree_reorder_state(c, s, st);
    prof_end(c, st, pr);
    partners_gravity_passes(c, s, mt, *p, d[0], st, nullptr, false, refine);  // k1
    pr = prof_begin(c, st, PH_INTEGRATE);
    timestep_reduce(c, s, *p, d[0], st);  // the limit, for a first step size
    rk_set_dt(c, s, dt, st);
    prof_end(c, st, pr);
    stage(k1, c2, 1, d[1]);    // k2 = f(q + dt/2 k1)
    stage(k12, c3, 2, d[2]);   // k3 = f(q - dt k1 + 2 dt k2)
    pr = prof_begin(c, st, PH_INTEGRATE);
    rk_error_control(c, s, k123, *p, eps_des, dt, t, err_log ? err_log + (int64_t)it * ninst : nullptr,
                     acc_log ? acc_log + (int64_t)it * ninst : nullptr, st);
    combine_update(c, s, s, k123, cf, 3, B.rk_acc, mt, *p, st);  // q + dt (k1 + 4 k2 + k3)/6 where accepted
    prof_end(c, st, pr);
  }
  return finish(c, p, st, "sph_step_rk3");
}

sph_status sph_rhs_adjoint(sph_ctx *c, sph_state *s, const sph_material *mats, int32_t nmat, const sph_params *p,
                           const sph_derivs *dbar, sph_state *sbar, double *param_bar, void *stream) {
  sph_status r = check_state(c, s);
  if (r != SPH_OK) return r;
  MatTable mt;
  if ((r = check_params(c, s, mats, nmat, p, mt)) != SPH_OK) return r;
  if (!dbar || !sbar) return fail(c, SPH_ERR_INVALID, "null cotangents");
  if (p->density_sum || p->gravity || p->eps_s > 0.0)
    return fail(c, SPH_ERR_INVALID, "adjoint needs continuity density, no gravity and no artificial stress");
  if (s->n > 0) {
    for (int ax = 0; ax < s->dim; ++ax)
      if (!sbar->x[ax] || !sbar->v[ax]) return fail(c, SPH_ERR_INVALID, "state_bar x and v are required");
    if (!sbar->rho || !sbar->u || (s->S && !sbar->S)) return fail(c, SPH_ERR_INVALID, "state_bar rho, u, S required");
  }
  cudaStream_t st = (cudaStream_t)stream;
  set_materials(c, &mt);
  sph_params q = *p;
  // forward evaluation in the requested precision: partner lists, T = sigma /
  // rho^2 and c_s (FP64 arrays, or the FP32 code-unit views of the mixed form)
  StepBufs &B = c->st;
  sph_derivs fwd;
  memset(&fwd, 0, sizeof(fwd));
  for (int k = 0; k < 3; ++k) {
    fwd.dx[k] = B.d_x[0][k];
    fwd.dv[k] = B.d_v[0][k];
  }
  fwd.drho = B.d_rho[0];
  fwd.du = B.d_u[0];
  fwd.dS = B.d_S[0];
  fwd.ddmg = B.d_dmg[0];
  fwd.n_act = B.d_nact[0];
  tree_build(c, s, q.leaf_size, q.max_depth, st);
  find_partners(c, s, st);
  rhs_passes(c, s, mt, q, fwd, st, q.precision == SPH_MIXED ? c->adj_sums : nullptr);
  rhs_adjoint(c, s, mt, q, *dbar, sbar, param_bar, st);
  return finish(c, p, st, "sph_rhs_adjoint");
}

sph_status sph_pc_update(sph_ctx *c, const sph_state *base, const sph_derivs *d, const sph_material *mats,
                         int32_t nmat, const sph_params *p, const double *dt, double frac, sph_state *out,
                         void *stream) {
  sph_status r = check_state(c, base);
  if (r != SPH_OK) return r;
  MatTable mt;
  if ((r = check_params(c, base, mats, nmat, p, mt)) != SPH_OK) return r;
  if (!d || !dt || !out) return fail(c, SPH_ERR_INVALID, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int ninst = base->ninst > 0 ? base->ninst : 1;
  cudaMemcpyAsync(c->st.dt, dt, sizeof(double) * ninst, cudaMemcpyDeviceToDevice, st);
  pc_update(c, base, out, *d, frac, mt, *p, st);
  return finish(c, p, st, "sph_pc_update");
}

sph_status sph_pc_update_adjoint(sph_ctx *c, const sph_state *base, const sph_derivs *d, const sph_material *mats,
                                 int32_t nmat, const sph_params *p, const double *dt, double frac,
                                 const sph_state *out_bar, sph_state *base_bar, sph_derivs *d_bar, double *param_bar,
                                 void *stream) {
  sph_status r = check_state(c, base);
  if (r != SPH_OK) return r;
  MatTable mt;
  if ((r = check_params(c, base, mats, nmat, p, mt)) != SPH_OK) return r;
  if (!d || !dt || !out_bar || !base_bar || !d_bar) return fail(c, SPH_ERR_INVALID, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  pc_update_adjoint(c, base, *d, dt, frac, mt, *p, out_bar, base_bar, d_bar, param_bar, st);
  return finish(c, p, st, "sph_pc_update_adjoint");
}

sph_status sph_get_tuning(const sph_ctx *c, sph_tuning *out) {
  if (!c || !out) return SPH_ERR_INVALID;
  *out = c->tune;
  return SPH_OK;
}

sph_status sph_set_tuning(sph_ctx *c, const sph_tuning *t) {
  if (!c || !t) return SPH_ERR_INVALID;
  const int pt = t->pass_threads;
  if (t->walk_leaf < 8 || t->walk_leaf > 1024 || t->walk_blocks_per_sm < 1 || t->walk_blocks_per_sm > 32 ||
      !(pt == 64 || pt == 128) || (t->walk_every_eval != 0 && t->walk_every_eval != 1) || t->iter_cap < 0 ||
      (t->plain_forms != 0 && t->plain_forms != 1))
    return fail(c, SPH_ERR_INVALID, "tuning out of range");
  c->tune = *t;
  c->tree.iter_cap = t->iter_cap;
  return SPH_OK;
}

sph_status sph_profile_enable(sph_ctx *c, int32_t on) {
  if (!c) return SPH_ERR_INVALID;
  if (on && !c->prof_ev) {
    c->prof_ev = new cudaEvent_t[2 * kMaxProfEvents];
    c->prof_phase = new int32_t[kMaxProfEvents];
    for (int i = 0; i < 2 * kMaxProfEvents; ++i)
      if (cudaEventCreate(&c->prof_ev[i]) != cudaSuccess) return cuda_check(c, "sph_profile_enable");
  }
  if (on && !c->prof) cudaMemset(c->d_ctr, 0, sizeof(unsigned long long) * kNumCounters);
  c->prof = on ? 1 : 0;
  c->prof_used = 0;
  return cuda_check(c, "sph_profile_enable");
}

sph_status sph_profile_counters(sph_ctx *c, int64_t *out, int32_t n, void *stream) {
  if (!c || !out || n < 1) return SPH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long h[kNumCounters];
  cudaMemcpyAsync(h, c->d_ctr, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(c, "sph_profile_counters");
  for (int k = 0; k < n; ++k) out[k] = k < kNumCounters ? (int64_t)h[k] : 0;
  cudaMemsetAsync(c->d_ctr, 0, sizeof(h), st);
  return cuda_check(c, "sph_profile_counters");
}

sph_status sph_profile_read(sph_ctx *c, double *ms, int32_t *calls, int32_t nphase) {
  if (!c || !ms || !calls || nphase < 1) return SPH_ERR_INVALID;
  for (int k = 0; k < nphase; ++k) {
    ms[k] = 0.0;
    calls[k] = 0;
  }
  for (int i = 0; i < c->prof_used; ++i) {
    if (cudaEventSynchronize(c->prof_ev[2 * i + 1]) != cudaSuccess) return cuda_check(c, "sph_profile_read");
    float t = 0.f;
    cudaEventElapsedTime(&t, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]);
    int ph = c->prof_phase[i];
    if (ph < nphase) {
      ms[ph] += t;
      calls[ph] += 1;
    }
  }
  c->prof_used = 0;
  return cuda_check(c, "sph_profile_read");
}

int64_t sph_launch_count(void) { return sph::g_launches.load(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// FMA throughput probe
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fma_loop(T *out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = fma(x0, a, b);
      x1 = fma(x1, a, b);
      x2 = fma(x2, a, b);
      x3 = fma(x3, a, b);
      x4 = fma(x4, a, b);
      x5 = fma(x5, a, b);
      x6 = fma(x6, a, b);
      x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
static double fma_rate(int iters) {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_loop<T><<<blocks, threads>>>(out, 8, (T)0.999999, (T)1e-7);
  double best = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    k_fma_loop<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
    best = std::max(best, flops / (ms * 1e-3));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return best;
}

extern "C" sph_status sph_measure_fma_peak(int32_t precision, double *flops) {
  if (!flops) return SPH_ERR_INVALID;
  double r = precision == SPH_FP64 ? fma_rate<double>(100) : fma_rate<float>(4000);
  *flops = r;
  return (r > 0 && cudaGetLastError() == cudaSuccess) ? SPH_OK : SPH_ERR_CUDA;
}


