// Internal declarations of the GB300 SPH library: the context, device
// helpers and the kernels' host launchers.  Not part of the public ABI
// (include/sph.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>

#include "sph.h"

namespace sph {

// Kernels launched by this library in this process (every launch site adds 1).
extern std::atomic<int64_t> g_launches;

// Phases timed by the optional profiler (CUDA events on the launch stream).
enum { PH_TREE = 0, PH_REORDER, PH_PARTNERS, PH_DENSITY, PH_PASSA, PH_PASSB, PH_GRAVITY, PH_INTEGRATE,
       PH_FLAW_DRAWS, PH_FLAW_FILL, PH_FOF_LINKS, PH_REFINE, PH_COUNT };
constexpr int kMaxProfEvents = 8192;

// ---------------------------------------------------------------------------
// Device error word bits (OR-ed by kernels, read by sph_sync_status).
// ---------------------------------------------------------------------------
enum : int32_t {
  ERR_NB_OVERFLOW = 1,     // a particle has more partners than max_neighbours
  ERR_NODE_OVERFLOW = 2,   // octree needs more nodes than the context holds
  ERR_NONFINITE = 4,       // NaN/Inf coordinate or velocity, h <= 0, rho <= 0
  ERR_TIMEOUT = 8,         // a bounded loop hit its iteration limit
  ERR_CSR_OVERFLOW = 16,   // CSR output longer than the caller's capacity
};

constexpr int kWarp = 32;
constexpr int kMaxLeaf = 32;
constexpr int kMaxHIter = 64;  // most updates of one variable smoothing length iteration
// Partner shells: a walk may also record, per particle, the candidates with
// (1 - kSkin) h_ab <= r_ab < (1 + kSkin) h_ab (at most kMaxShell of them),
// partners and non-partners alike, from which the partners at positions
// moved by less than kSkin h / (4 sqrt D) follow without a walk: a partner
// outside the shell stays one, a non-partner outside it stays none, and only
// the shell is tested again (neighbours.cu).
constexpr double kSkin = 1.0 / 64.0;
constexpr int kMaxShell = 24;

// Per-particle FP32 views used by the walks and the mixed-precision passes.
// Positions are split X = x - corner into hi = float(X), lo = float(X - hi)
// so that differences of neighbours keep ~48 bits; velocities likewise.
// Four separate arrays (structure of arrays): the lanes of a warp gather
// nearby neighbours, whose words then share few 128-byte lines per load; an
// interleaved 64-byte record per particle measured slower in the passes
// (more lines, i.e. L1 wavefronts, per gather instruction).
struct PackedF32 {
  float4 *px_, *pxl_, *pv_, *pvl_;
  __host__ __device__ float4 &px(int64_t i) const { return px_[i]; }    // (x_hi, y_hi, z_hi, h)
  __host__ __device__ float4 &pxl(int64_t i) const { return pxl_[i]; }  // (x_lo, y_lo, z_lo, m)
  __host__ __device__ float4 &pv(int64_t i) const { return pv_[i]; }    // (vx_hi, vy_hi, vz_hi, rho)
  __host__ __device__ float4 &pvl(int64_t i) const { return pvl_[i]; }  // (vx_lo, vy_lo, vz_lo, m/rho)
};

// Largest skip index of the packed node word of the gravity walk (26 bits).
constexpr int64_t kPackedSkip = (1LL << 26) - 1;

struct Tree {
  // sort
  unsigned long long *keys[2];
  int32_t *vals[2];
  uint32_t *hist;
  int64_t hist_cap;
  int32_t *perm;       // sorted slot -> state index (points into vals[*])
  unsigned long long *skey;  // sorted keys (points into keys[*])
  // per-slot node emission counts and their exclusive scan; after the scan
  // ncount holds the list of leaf ids (nleaf of them, in no fixed order)
  int32_t *ncount;
  int32_t *nleaf;      // device scalar
  int32_t *nstart;
  int32_t *scan_tmp;
  // nodes (pre-order)
  int64_t cap_nodes;
  int packed_walk;     // fcom_lo.w holds the packed node word (cap_nodes <= kPackedSkip + 1)
  int32_t *nnodes;     // device scalar
  int32_t *first, *end, *skip, *parent, *nchild, *arrived, *level;
  int32_t *child;      // up to 8 child ids per node, in arrival order
  int4 *nrec;          // (first, end, skip, level) per node, for the walks
  unsigned long long *cell;  // level prefix of the key (instance bits included)
  double *mass, *com;  // com: 3 * cap_nodes, component-major
  double *bblo, *bbhi; // tight particle box, 3 * cap_nodes each
  double *hmax;
  float4 *fbox_lo;     // (lo xyz relative to instance corner, rounded down; +-hmax rounded up, negative
                       //  where the partner walk stops: at most max(leaf_size, walk_leaf) particles or depth B)
  float4 *fbox_hi;     // (hi xyz, rounded up; skip[] as int bits)
  float4 *fcom_hi;     // (com hi xyz relative to instance corner, mass)
  float4 *fcom_lo;     // (com lo xyz, w): w = the edge s0 / 2^level, or, where packed_walk, the word
                       // skip | level << 26 | leaf << 31 as int bits (leaf: at most leaf_size
                       // particles or level max_depth), the edge then being s0 / 2^level
  // per instance
  unsigned long long *inst_bb;  // 6 per instance: encoded min xyz, encoded max xyz
  double *inst_lo;     // 3 per instance
  double *inst_s0;
  double *inst_rs0;    // 1 / s0, correctly rounded
  int32_t *inst_root;
  // walk groups: up to 32 consecutive slots inside one tree cell
  int32_t *gcnt, *gstart;  // per node: groups it starts, and their exclusive scan (cap_nodes + 1)
  int32_t *grp_start, *grp_end, *grp_inst;
  int32_t *ngroups;    // device scalar
  int64_t cap_groups;
  int leaf_size, max_depth, dim, ninst;
  int64_t n;
  int perm_identity;   // host flag: the state is in tree order (perm[i] = i)
  int iter_cap;        // > 0: node visits of one walk are bounded by this instead of the node count
};

struct MatTable {
  sph_material m[SPH_MAX_MATERIALS];
  int32_t nmat;
};

// Code units of the FP32 views.  Every factor is a power of two, so the
// scaling is exact and FP32 arithmetic in code units rounds exactly as it
// would in SI, but without overflow or underflow: L from h of particle 0,
// M from its mass, T from L over a material sound speed.
struct Units {
  double L, M, T;                 // base units (SI per code unit)
  double invL, invM, invT;
  double rho, invrho;             // M / L^D
  double V, invV;                 // L / T
  double sig, invsig;             // rho V^2: stress, pressure
  double E, invE;                 // V^2: specific energy
  double acc;                     // L / T^2
  double Gs;                      // gravity constant in code units (set per call)
  float matf[SPH_MAX_MATERIALS][16];  // materials in code units (see k_units)
};

struct StepBufs {
  // predicted state
  double *x[3], *v[3], *rho, *u, *S, *dmg;
  // three derivative sets (two for the predictor-corrector, three for the
  // embedded Runge-Kutta step)
  double *d_x[3][3], *d_v[3][3], *d_rho[3], *d_u[3], *d_S[3], *d_dmg[3], *d_cs[3];
  int32_t *d_nact[3];
  unsigned long long *rk_err;  // per instance, bits of the error estimate (non-negative)
  int32_t *rk_acc;             // per instance, step accepted
  unsigned long long *dt_enc;  // per instance, ordered encoding for atomicMin
  unsigned long long *dmove;   // bits of the predictor's largest per-axis displacement
  unsigned long long *dbuild;  // bits of a bound on every displacement since the last tree build
  unsigned long long *dgrow;   // dbuild + dmove
  double *dt;                  // per instance
  double *gather;              // reorder scratch (n doubles)
  int32_t *gather_i;
  double *snap[4];             // positions and h an sph_step call returned (tree_continue check)
  int32_t *differ;             // device flag of that check
};

// Per-group scratch of the flaw generator (group = instance x material).
struct FlawBufs {
  int64_t cap_groups;
  int32_t *goff;       // cap_groups + 1: first sorted position of each group
  double *kv, *invm;   // log2(k V) and 1/m per group
  uint32_t *J;         // number of flaws per group
  int32_t *unc;        // members not yet hit
  int32_t *plan_grp;   // draw plan of one round
  int64_t *plan_b0, *plan_pre;
  int cap_plan;
  int32_t *bad;        // set when an id or material index is out of range
  // volume chunks: group, member range, partial sum; first chunk of each group
  int32_t *ck_g, *ck_lo, *ck_hi, *g_ck;
  double *ck_sum;
  int cap_chunks;
};

}  // namespace sph

struct sph_ctx {
  int dim;
  int device;
  int64_t cap_n;
  int32_t cap_inst;
  int32_t kmax;
  int32_t leaf_default;
  int64_t bytes;
  char err[512];
  int32_t *d_err;       // device error word
  int32_t *h_err;       // pinned host copy
  sph::Tree tree;
  sph::PackedF32 pk;
  // partners, column-major: nb_idx[k * cap_n + a]
  int32_t *nb_idx;
  int32_t *nb_cnt;
  int32_t *nb_alt;      // second lists and counts (partners refined from nb_idx)
  int32_t *nb_cnt_alt;
  int32_t *sh_idx;      // shell candidates, column-major, kMaxShell per particle
  int32_t *sh_cnt;      // their number, -1 when more than kMaxShell
  int32_t *sh_in;       // bit j set when shell entry j was a partner at the walk
  int32_t *need_walk;   // device flag: some particle could not refine its list
  int64_t *csr_total;   // device scalar for sph_neighbours
  int32_t *hflags;      // variable-h iteration: done, updates, off-target count per pass
  // pass A -> pass B per-particle data
  void *T;              // nsym * cap_n of double (FP64) or float (mixed)
  void *zeta;
  double *cs;
  double *p;
  double *ag;           // gravity acceleration, 3 * cap_n
  double *adj_inter;    // adjoint scratch, 22 * cap_n
  float4 *adj32;        // mixed adjoint scratch, 7 * cap_n float4
  float *adj_sums;      // mixed adjoint: the forward pass A's pair sums, 16 * cap_n
  sph::Units *units;    // device
  double vscale;        // host: velocity scale for the time unit
  sph::MatTable mt;     // host copy of the materials of the current call
  sph_tuning tune;      // launch shapes and walk granularity
  int num_sms;
  // profiler
  unsigned long long *d_ctr;  // device interaction counters (kNumCounters), summed while profiling
  int prof;
  int prof_used;
  cudaEvent_t *prof_ev;       // 2 * kMaxProfEvents
  int32_t *prof_phase;        // kMaxProfEvents
  sph::StepBufs st;
  sph::FlawBufs fl;
  // tree window of sph_step (tree_reuse) that a later call may continue:
  // valid only while no other call has touched the tree or the lists
  bool win_valid, win_was;
  int win_age, win_R, win_ninst, win_leaf, win_depth, win_gravity;
  int64_t win_n;
  // allocation list
  void *allocs[256];
  int nallocs;
};

namespace sph {

// ---------------------------------------------------------------------------
// Small device helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline int nsym(int dim) { return dim == 3 ? 6 : 3; }

// symmetric component index: 3D (xx,yy,zz,xy,xz,yz), 2D (xx,yy,xy)
__host__ __device__ inline int symk(int dim, int a, int b) {
  if (a == b) return a;
  if (dim == 2) return 2;
  int s = a + b;  // (0,1)->1, (0,2)->2, (1,2)->3
  return s + 2;
}

// Order-preserving map of doubles to unsigned 64-bit integers, so that
// atomicMin/atomicMax on the integers give the min/max of the doubles.
__device__ __forceinline__ unsigned long long dbl_to_ord(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double ord_to_dbl(unsigned long long o) {
  unsigned long long b = (o & 0x8000000000000000ULL) ? (o & 0x7fffffffffffffffULL) : ~o;
  return __longlong_as_double((long long)b);
}

// Instance of particle i (instances are contiguous ranges).
__device__ __forceinline__ int inst_of(const int64_t *inst_off, int ninst, int64_t i) {
  if (ninst <= 1 || inst_off == nullptr) return 0;
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (inst_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void raise_err(int32_t *err, int32_t bit) { atomicOr(err, bit); }

// Cubic B-spline kernel of Sect. 3.1.1 with support radius h.
template <class R>
__device__ __forceinline__ R kernel_sigma(int dim) {
  return dim == 3 ? R(2.5464790894703255) : R(1.8189136353359467);  // 8/pi, 40/(7 pi)
}

template <class R>
__device__ __forceinline__ R kern_W(R q, R norm) {  // norm = s / h^D
  if (q < R(0.5)) return norm * (R(6) * q * q * q - R(6) * q * q + R(1));
  if (q <= R(1)) {
    R t = R(1) - q;
    return norm * R(2) * t * t * t;
  }
  return R(0);
}

template <class R>
__device__ __forceinline__ R kern_dW(R q, R gnorm) {  // gnorm = 6 s / h^(D+1)
  if (q < R(0.5)) return gnorm * (R(3) * q * q - R(2) * q);
  if (q <= R(1)) {
    R t = R(1) - q;
    return -gnorm * t * t;
  }
  return R(0);
}

template <class R>
__device__ __forceinline__ R hpow(R h, int k) {
  R r = h;
  for (int i = 1; i < k; ++i) r *= h;
  return r;
}

// Kahan-compensated accumulator (plain sum in double).
template <class R>
struct KahanT {
  R s = R(0), c = R(0);
  __device__ __forceinline__ void add(R v) {
    R y = v - c;
    R t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <>
struct KahanT<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};

// Host-side launch helpers ---------------------------------------------------
inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

// Material constants in code units, indices into Units::matf
enum { MF_RHO0, MF_CS, MF_K0, MF_NM, MF_AT, MF_BT, MF_E0, MF_EIV, MF_ECV, MF_AA, MF_BB, MF_ALPHA, MF_BETA,
       MF_RHOCUT, MF_MU, MF_Y0 };

double velocity_scale(const MatTable &mt);
// Interaction counters, accumulated while the profiler is enabled
enum { CTR_GRAV_NODES, CTR_GRAV_TERMS, CTR_GRAV_VISITS, CTR_WALK_TESTS, CTR_WALK_PARTNERS, kNumCounters };
inline unsigned long long *counters(const sph_ctx *c) { return c->prof ? c->d_ctr : nullptr; }

// Sum of v over the warp, added to *ctr by lane 0 (every lane must arrive)
__device__ __forceinline__ void warp_count(unsigned long long *ctr, unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(ctr, v);
}

// api.cu: profiler hooks (no-ops unless enabled)
int prof_begin(sph_ctx *c, cudaStream_t st, int phase);
void prof_end(sph_ctx *c, cudaStream_t st, int idx);
// tree.cu
void tree_build(sph_ctx *c, const sph_state *s, int leaf_size, int max_depth, cudaStream_t st);
void tree_reorder_state(sph_ctx *c, sph_state *s, cudaStream_t st);
void pack_f32(sph_ctx *c, const sph_state *s, cudaStream_t st);
// neighbours.cu
// grow (device, may be NULL): bits of a displacement bound by which every
// particle may have left the node boxes of the current tree, per axis
// shell: also record the shell candidates of every particle (sh_idx, sh_cnt)
void find_partners(sph_ctx *c, const sph_state *s, cudaStream_t st, const unsigned long long *grow = nullptr,
                   bool shell = false);
// Partners of s into c->nb_alt / nb_cnt_alt from the lists and shells of the
// last walk (nb_idx, nb_cnt, sh_idx, sh_cnt; left unchanged), whose positions
// every particle of s left by at most `move` per axis (device bits); a walk
// with boxes grown by `grow` recomputes every list when some particle cannot
// refine its own.  The caller swaps the two list buffers (and the two count
// arrays) for the passes that read the result.
void refine_partners(sph_ctx *c, const sph_state *s, const unsigned long long *move, const unsigned long long *grow,
                     cudaStream_t st);
// variable smoothing length iteration; flags: device int32[max_iter + 3]
void adapt_h(sph_ctx *c, sph_state *s, double n_des, int tol, int max_iter, int32_t *flags, cudaStream_t st);
void partners_to_csr(sph_ctx *c, const sph_state *s, int64_t *off, int32_t *idx, int64_t cap, cudaStream_t st);
// rhs.cu
// sums: NULL, or (mixed) where pass A also stores its pair sums for the
// adjoint (16 * cap_n floats, the layout of k_passA's KEEP_SUMS form)
void rhs_passes(sph_ctx *c, sph_state *s, const MatTable &mt, const sph_params &p, const sph_derivs &out,
                cudaStream_t st, float *sums = nullptr);
// gravity.cu
// reuse: the tree was built at earlier positions (pseudo-particles reused)
void gravity_walk(sph_ctx *c, const sph_state *s, const sph_params &p, double *ax, double *ay, double *az,
                  cudaStream_t st, bool reuse = false);
// adjoint.cu
void rhs_adjoint(sph_ctx *c, const sph_state *s, const MatTable &mt, const sph_params &p, const sph_derivs &dbar,
                 sph_state *sbar, double *param_bar, cudaStream_t st);
void pc_update_adjoint(sph_ctx *c, const sph_state *base, const sph_derivs &d, const double *dt, double frac,
                       const MatTable &mt, const sph_params &p, const sph_state *obar, sph_state *gbar,
                       sph_derivs *fbar, double *param_bar, cudaStream_t st);
// flaws.cu: Weibull thresholds (Sect. 3.2); *total receives the number of flaws
sph_status flaws_generate(sph_ctx *c, const sph_state *s, const sph_material *mats, int nmat, const double *wk,
                          const double *wm, uint64_t seed, int64_t *flaw_off, float *flaw_eps, int64_t cap,
                          int64_t *total, cudaStream_t st);
// fof.cu: friends-of-friends fragments (Sect. 4); blocking (*nfrag on return)
void fragments_fof(sph_ctx *c, const sph_state *s, const double *h0, double b, double d_remove, int min_size,
                   int leaf_size, int max_depth, int32_t *label, int32_t *frag_count, double *frag_mass, int64_t cap,
                   int64_t *nfrag, cudaStream_t st);
// step.cu
void timestep_reduce(sph_ctx *c, const sph_state *s, const sph_params &p, const sph_derivs &d, cudaStream_t st);
// dmove (device, may be NULL): receives the bits of max over particles and
// axes of |out.x - base.x|; non-finite output or rho <= 0 then raises the
// non-finite error bit, as a tree build over `out` would.  pack: also write
// the FP32 views of out (c->pk, in the units and instance corners of the
// current tree), as pack_f32 would.
void pc_update(sph_ctx *c, const sph_state *base, sph_state *out, const sph_derivs &d, double frac,
               const MatTable &mt, const sph_params &p, cudaStream_t st, unsigned long long *dmove = nullptr,
               bool pack = false);
// out = base + dt (coef_0 d_0 + ...), nd <= 3 sets, where mask[inst] (NULL: all)
void combine_update(sph_ctx *c, const sph_state *base, sph_state *out, const sph_derivs *const *d, const double *coef,
                    int nd, const int32_t *mask, const MatTable &mt, const sph_params &p, cudaStream_t st,
                    unsigned long long *dmove = nullptr, bool pack = false);
// embedded Runge-Kutta: step size of the attempt (c->st.dt), error and control
void rk_set_dt(sph_ctx *c, const sph_state *s, double *dt_io, cudaStream_t st);
// *out = a + b rounded up (bits of non-negative doubles)
void bound_add(unsigned long long *out, const unsigned long long *a, const unsigned long long *b, cudaStream_t st);
void rk_error_control(sph_ctx *c, const sph_state *s, const sph_derivs *const *k, const sph_params &p, double eps_des,
                      double *dt_io, double *t_io, double *err_log, int32_t *acc_log, cudaStream_t st);

}  // namespace sph
