// Interaction partners (Sect. 3.5.2), GB300 form.
//
// The paper walks the tree once per particle from the root.  Here a warp
// walks it once for 32 consecutive sorted particles (one "group"): the tree
// is stored in pre-order, so the walk is a single loop over node ids that
// either enters a node (id + 1) or jumps over its subtree (skip[id]) - no
// stack, and every lane follows the same path.  A node is entered when its
// particle box comes within (h_group + h_node,max)/2 of the group's box,
// which can only keep more candidates than the paper's test; the set itself
// is decided per lane by the exact predicate.
//
// Predicate: b is a partner of a iff ((dx^2 + dy^2) + dz^2) < h_ab^2 with
// h_ab = (h_a + h_b)/2, all in FP64 without fused multiply-add.  On GB300
// FP64 runs at 1/62 of the FP32 rate, so each candidate is first classified
// in FP32 from positions relative to the group (formed from hi/lo split
// coordinates); only candidates whose squared distance lies within a
// relative band of 6e-5 around h_ab^2 - far wider than the FP32 error of
// about 2e-6 - are decided by the FP64 expression.  The result is therefore
// bit-identical to the FP64 definition.
#include "fpbits.cuh"
#include "sph_internal.cuh"

namespace sph {

// Warps (particle groups) per block; the grid keeps the warp count of 4-warp
// blocks.  1, 2 and 4 measured within 3 % of each other on GB300.
#ifndef SPH_WALK_WARPS
#define SPH_WALK_WARPS 4
#endif
constexpr int kNbWarps = SPH_WALK_WARPS;
// resident blocks per SM the walk is compiled for: 8 (64 registers) was the
// fastest of 4..12 on GB300, the walk being latency- and issue-bound
#ifndef SPH_WALK_MIN_BLOCKS
#define SPH_WALK_MIN_BLOCKS 8
#endif
#define SPH_WALK_BOUNDS __launch_bounds__(kNbWarps * 32, SPH_WALK_MIN_BLOCKS)
constexpr float kBand = 6e-5f;

__device__ __forceinline__ bool exact_partner(const double *__restrict__ x, const double *__restrict__ y,
                                              const double *__restrict__ z, const double *__restrict__ h, int dim,
                                              int64_t a, int64_t b) {
  double dx = __dsub_rn(x[a], x[b]);
  double dy = __dsub_rn(y[a], y[b]);
  double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  if (dim == 3) {
    double dz = __dsub_rn(z[a], z[b]);
    r2 = __dadd_rn(r2, __dmul_rn(dz, dz));
  }
  double hab = __dmul_rn(0.5, __dadd_rn(h[a], h[b]));
  return r2 < __dmul_rn(hab, hab);
}

// The same predicate with the particle's own support radius, for the
// variable smoothing length iteration: ((dx^2 + dy^2) + dz^2) < h_a^2.
__device__ __forceinline__ bool exact_within_own_h(const double *__restrict__ x, const double *__restrict__ y,
                                                   const double *__restrict__ z, const double *__restrict__ h,
                                                   int dim, int64_t a, int64_t b) {
  double dx = __dsub_rn(x[a], x[b]);
  double dy = __dsub_rn(y[a], y[b]);
  double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  if (dim == 3) {
    double dz = __dsub_rn(z[a], z[b]);
    r2 = __dadd_rn(r2, __dmul_rn(dz, dz));
  }
  return r2 < __dmul_rn(h[a], h[a]);
}

// Shells (SHELL = true): the walk also records, in ascending order, every b
// with (1 - kSkin) h_ab <= r_ab < (1 + kSkin) h_ab (FP32 tests with the band's
// margin on both sides, so possibly a few more): the partners near the
// support radius and the non-partners just beyond it, for k_partners_refine.
constexpr float kSkinF = (float)kSkin;
constexpr float kShell2 = (1.0f + kSkinF) * (1.0f + kSkinF) * (1.0f + kBand);
constexpr float kInner2 = (1.0f - kSkinF) * (1.0f - kSkinF) * (1.0f - kBand);

// OWN_H = false: interaction partners (h_ab), lists and counts, skipped when
// the flag `done` is given and is 0 (it is then a run-if flag).  OWN_H = true:
// only the number of particles within each particle's own h (the current h of
// the state, not the packed one), plus the count of particles whose number
// lies farther than tol from n_des (*unconverged); the walk is skipped once
// *done is set.
template <bool OWN_H, bool SHELL>
__global__ void SPH_WALK_BOUNDS k_partners(Tree T, PackedF32 pk, const double *__restrict__ x,
                                           const double *__restrict__ y, const double *__restrict__ z,
                                           const double *__restrict__ h, int dim, int kmax,
                                           int32_t *__restrict__ nb_idx, int32_t *__restrict__ nb_cnt, int64_t ld,
                                           int32_t *err, const unsigned long long *__restrict__ grow,
                                           const Units *__restrict__ U, const int32_t *__restrict__ done,
                                           int32_t *__restrict__ unconverged, double n_des, int tol,
                                           int32_t *__restrict__ sh_idx, int32_t *__restrict__ sh_cnt,
                                           int32_t *__restrict__ sh_in, unsigned long long *ctr) {
  static_assert(!(OWN_H && SHELL), "shells are partner candidates");
  if constexpr (OWN_H) {
    if (*done) return;
  } else {
    if (done && *done == 0) return;  // done is run_if here
  }
  // the shell widens every test by the factor (1 + kSkin) of its radius
  const float wide = SHELL ? 1.0f + kSkinF : 1.0f;
  __shared__ float4 sc[kNbWarps][kMaxLeaf];
  __shared__ int32_t sb[kNbWarps][kMaxLeaf];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngroups = *T.ngroups;
  // The walk stops at nodes flagged in their box word (at most
  // max(leaf_size, walk_leaf) particles, or depth B; set by the tree build)
  // and culls their whole particle range: any stopping rule gives the same set.
  const int nnodes = T.iter_cap > 0 ? min(*T.nnodes, T.iter_cap) : *T.nnodes;
  // Node boxes are those of the tree the walk runs on; when the particles have
  // moved since it was built (by at most `grow` per axis), widening the
  // group's box by that much keeps every node that may hold a partner.
  float gw = 0.f;
  if (grow) gw = to_f32_dir_scaled(bitsd(*grow), pow2_exp(U->invL), true, U->invL);
  for (int g = blockIdx.x * kNbWarps + w; g < ngroups; g += gridDim.x * kNbWarps) {
    const int32_t s0 = T.grp_start[g], s1 = T.grp_end[g], inst = T.grp_inst[g];
    const int32_t slot = s0 + lane;
    const bool act = slot < s1;
    const int32_t a = act ? (T.perm_identity ? slot : T.perm[slot]) : -1;
    float4 P = act ? pk.px(a) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 Q = act ? pk.pxl(a) : make_float4(0.f, 0.f, 0.f, 0.f);
    // reference point: lane 0's position
    const float cx = __shfl_sync(0xffffffffu, P.x, 0), cy = __shfl_sync(0xffffffffu, P.y, 0),
                cz = __shfl_sync(0xffffffffu, P.z, 0);
    const float lx = __shfl_sync(0xffffffffu, Q.x, 0), ly = __shfl_sync(0xffffffffu, Q.y, 0),
                lz = __shfl_sync(0xffffffffu, Q.z, 0);
    const float rax = (P.x - cx) + (Q.x - lx), ray = (P.y - cy) + (Q.y - ly), raz = (P.z - cz) + (Q.z - lz);
    const float hha = 0.5f * P.w;
    // own support radius in code units (OWN_H): from the state's current h
    float hown = 0.f;
    if constexpr (OWN_H) hown = act ? to_f32_scaled(h[a], pow2_exp(U->invL), U->invL) : 0.f;
    // group box (hi coordinates, for the node test) and largest h
    float gl[3] = {act ? P.x : 3e38f, act ? P.y : 3e38f, act ? P.z : 3e38f};
    float gh[3] = {act ? P.x : -3e38f, act ? P.y : -3e38f, act ? P.z : -3e38f};
    float hg = act ? (OWN_H ? hown : P.w) : 0.f;
    // the same box relative to the reference point, for culling candidates
    float rl[3] = {act ? rax : 3e38f, act ? ray : 3e38f, act ? raz : 3e38f};
    float rh[3] = {act ? rax : -3e38f, act ? ray : -3e38f, act ? raz : -3e38f};
    for (int o = 16; o > 0; o >>= 1) {
      for (int ax = 0; ax < 3; ++ax) {
        gl[ax] = fminf(gl[ax], __shfl_xor_sync(0xffffffffu, gl[ax], o));
        gh[ax] = fmaxf(gh[ax], __shfl_xor_sync(0xffffffffu, gh[ax], o));
        rl[ax] = fminf(rl[ax], __shfl_xor_sync(0xffffffffu, rl[ax], o));
        rh[ax] = fmaxf(rh[ax], __shfl_xor_sync(0xffffffffu, rh[ax], o));
      }
      hg = fmaxf(hg, __shfl_xor_sync(0xffffffffu, hg, o));
    }
    float mag = fmaxf(fmaxf(fabsf(gh[0]), fabsf(gh[1])), fabsf(gh[2]));
    float slack = 1e-6f * mag + gw * (1.0f + 1e-6f);
    for (int ax = 0; ax < 3; ++ax) {
      gl[ax] -= slack;
      gh[ax] += slack;
    }
    // relative coordinates carry an error of a few 1e-7 of the group's extent + h
    const float rslack = 1e-5f * (fmaxf(fmaxf(rh[0] - rl[0], rh[1] - rl[1]), rh[2] - rl[2]) + hg);
    const unsigned lt_mask = (1u << lane) - 1u;
    const int32_t root = T.inst_root[inst];
    const int32_t stop = root >= 0 ? T.skip[root] : root;
    int cnt = 0, scnt = 0;
    uint32_t sin = 0;  // shell entries that are partners (bit per entry)
    int iter = 0;
    unsigned ntest = 0;  // candidates this lane tested (counters)
    // Stackless pre-order walk over the node box words: (lo, +-hmax) and
    // (hi, skip), the sign of hmax marking the nodes where the walk stops.
    for (int32_t nd = root; nd < stop && iter <= nnodes; ++iter) {
      const float4 bl = __ldg(&T.fbox_lo[nd]), bh = __ldg(&T.fbox_hi[nd]);
      const float hw = fabsf(bl.w);
      float gx = fmaxf(0.f, fmaxf(bl.x - gh[0], gl[0] - bh.x));
      float gy = fmaxf(0.f, fmaxf(bl.y - gh[1], gl[1] - bh.y));
      float gz = fmaxf(0.f, fmaxf(bl.z - gh[2], gl[2] - bh.z));
      float d2 = gx * gx + gy * gy + gz * gz;
      float thr = (OWN_H ? hg : 0.5f * (hg + hw)) * (1.0f + 1e-5f) * wide;
      bool enter = false;
      if (d2 <= thr * thr) {
        if (__float_as_uint(bl.w) >> 31) {  // the walk stops here: cull its particles
          const int4 nr = __ldg(&T.nrec[nd]);
          const int32_t f = nr.x, e = nr.y;
          for (int32_t base = f; base < e; base += kMaxLeaf) {  // leaves at full depth may exceed 32
            // stage the candidates that come within reach of the group's box
            bool keep = false;
            float4 cand = make_float4(0.f, 0.f, 0.f, 0.f);
            int32_t b = -1;
            if (base + lane < e) {
              b = T.perm_identity ? base + lane : __ldg(&T.perm[base + lane]);
              float4 Pb = __ldg(&pk.px(b)), Qb = __ldg(&pk.pxl(b));
              cand = make_float4((Pb.x - cx) + (Qb.x - lx), (Pb.y - cy) + (Qb.y - ly), (Pb.z - cz) + (Qb.z - lz),
                                 0.5f * Pb.w);  // half support radius: h_ab = h_a / 2 + h_b / 2
              float qx = fmaxf(0.f, fmaxf(rl[0] - cand.x, cand.x - rh[0]));
              float qy = fmaxf(0.f, fmaxf(rl[1] - cand.y, cand.y - rh[1]));
              float qz = fmaxf(0.f, fmaxf(rl[2] - cand.z, cand.z - rh[2]));
              float reach = (OWN_H ? hg : 0.5f * hg + cand.w) * (1.0f + 1e-5f) * wide + rslack;
              keep = qx * qx + qy * qy + qz * qz <= reach * reach;
            }
            const unsigned km = __ballot_sync(0xffffffffu, keep);
            const int c = __popc(km);
            if (keep) {
              const int pos = __popc(km & lt_mask);
              sc[w][pos] = cand;
              sb[w][pos] = b;
            }
            __syncwarp();
            if (act) {
              ntest += c;
              for (int k = 0; k < c; ++k) {
                const float4 cb = sc[w][k];
                const int32_t b = sb[w][k];
                float dx = rax - cb.x, dy = ray - cb.y, dz = raz - cb.z;
                float r2 = dx * dx + dy * dy + dz * dz;
                float hab = OWN_H ? hown : hha + cb.w;
                float h2 = hab * hab;
                bool in;
                if (r2 < h2 * (1.0f - kBand)) in = true;
                else if (r2 > h2 * (1.0f + kBand)) in = false;
                else in = OWN_H ? exact_within_own_h(x, y, z, h, dim, a, b) : exact_partner(x, y, z, h, dim, a, b);
                if (in && b != a) {
                  if constexpr (!OWN_H)
                    if (cnt < kmax) nb_idx[(int64_t)cnt * ld + a] = b;
                  ++cnt;
                  if constexpr (SHELL) {
                    if (r2 >= h2 * kInner2) {  // a partner near the support radius
                      if (scnt < kMaxShell) {
                        sh_idx[(int64_t)scnt * ld + a] = b;
                        sin |= 1u << scnt;
                      }
                      ++scnt;
                    }
                  }
                } else if constexpr (SHELL) {
                  if (b != a && r2 <= h2 * kShell2) {
                    if (scnt < kMaxShell) sh_idx[(int64_t)scnt * ld + a] = b;
                    ++scnt;
                  }
                }
              }
            }
            __syncwarp();
          }
        } else {
          enter = true;
        }
      }
      nd = enter ? nd + 1 : __float_as_int(bh.w);
    }
    if (iter > nnodes) raise_err(err, ERR_TIMEOUT);
    if (ctr) {
      warp_count(ctr + CTR_WALK_TESTS, ntest);
      warp_count(ctr + CTR_WALK_PARTNERS, act && !OWN_H ? (unsigned)cnt : 0u);
    }
    if constexpr (OWN_H) {
      if (act) {
        nb_cnt[a] = cnt;
        if (fabs((double)cnt - n_des) > (double)tol) atomicAdd(unconverged, 1);
      }
    } else if (act) {
      nb_cnt[a] = min(cnt, kmax);
      if (cnt > kmax) raise_err(err, ERR_NB_OVERFLOW);
      if constexpr (SHELL) {
        sh_cnt[a] = scnt <= kMaxShell ? scnt : -1;
        sh_in[a] = (int32_t)sin;
      }
    }
  }
}

// Partners at moved positions from the lists and shells of an earlier walk
// (the Verlet-list idea).  When every particle moved by at most `move` per
// axis since that walk, a pair's distance changed by at most 2 sqrt(D) move;
// with 4 sqrt(D) move <= kSkin h_a that is at most kSkin h_ab (h_ab >= h_a / 2).
// So a partner of the walk closer than (1 - kSkin) h_ab is still one, a
// non-partner farther than (1 + kSkin) h_ab is still none, and only the shell
// between the two can change.  The old list and the shell are both ascending,
// and the shell's partners are also in the list: merged, the candidates are
// visited in ascending order, the list's members outside the shell are kept
// as they are (no gather), and each shell member is decided by the walk's
// predicate (FP32 outside the band, the FP64 definition inside it), so the new
// list equals that of a walk at the new positions bit for bit.  A particle
// whose bound does not hold, or whose shell overflowed, sets *need_walk
// instead, and a walk follows.
constexpr int kRefineThreads = 128;
__global__ void __launch_bounds__(kRefineThreads)
    k_partners_refine(PackedF32 pk, const double *__restrict__ x, const double *__restrict__ y,
                      const double *__restrict__ z, const double *__restrict__ h, int dim, int64_t n, int64_t ld,
                      int kmax, const int32_t *__restrict__ old_idx, const int32_t *__restrict__ old_cnt,
                      const int32_t *__restrict__ sh_idx, const int32_t *__restrict__ sh_cnt,
                      const int32_t *__restrict__ sh_in, int32_t *__restrict__ new_idx,
                      int32_t *__restrict__ new_cnt,
                      const unsigned long long *__restrict__ move, int32_t *__restrict__ need_walk, int32_t *err) {
  // the shell of each thread's particle, staged for the merge
  __shared__ int32_t shs[kMaxShell][kRefineThreads];
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const int ns = sh_cnt[a];
  const double sqd = dim == 3 ? 1.7320508075688772 : 1.4142135623730951;  // sqrt(D)
  const double bound = __dmul_ru(__dmul_ru(4.0 * sqd, bitsd(*move)), 1.0 + 1e-6);
  if (ns < 0 || !(bound <= __dmul_rd(kSkin, h[a]))) {
    *need_walk = 1;
    return;
  }
  const int t = threadIdx.x;
  // 1. decide every shell member at the new positions (bit j of `in`)
  uint32_t in = 0;
  {
    const float4 P = pk.px(a), Q = pk.pxl(a);
    const float hha = 0.5f * P.w;
    for (int j = 0; j < ns; ++j) {
      const int32_t b = sh_idx[(int64_t)j * ld + a];
      shs[j][t] = b;
      const float4 Pb = pk.px(b), Qb = pk.pxl(b);
      const float dx = (P.x - Pb.x) + (Q.x - Qb.x), dy = (P.y - Pb.y) + (Q.y - Qb.y),
                  dz = (P.z - Pb.z) + (Q.z - Qb.z);
      const float r2 = dx * dx + dy * dy + dz * dz;
      const float hab = hha + 0.5f * Pb.w;
      const float h2 = hab * hab;
      bool ok;
      if (r2 < h2 * (1.0f - kBand)) ok = true;
      else if (r2 > h2 * (1.0f + kBand)) ok = false;
      else ok = exact_partner(x, y, z, h, dim, a, b);
      in |= (uint32_t)ok << j;
    }
  }
  // 2a. no shell member changed sides: the list is the walk's, and a count of
  // -1 tells the passes to read that list (nothing is copied)
  if (in == (uint32_t)sh_in[a]) {
    new_cnt[a] = -1;
    return;
  }
  // 2b. merge: list members outside the shell are kept, shell members that are
  // in are emitted once (in the list or inserted), the others dropped; the
  // list is read 8 entries at a time so that its loads overlap
  const int nl = old_cnt[a];
  int j = 0, cnt = 0;
  int32_t bs = ns > 0 ? shs[0][t] : INT_MAX;
  auto emit = [&](int32_t b) {
    if (cnt < kmax) new_idx[(int64_t)cnt * ld + a] = b;
    ++cnt;
  };
  for (int base = 0; base < nl; base += 8) {
    int32_t buf[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) buf[u] = base + u < nl ? old_idx[(int64_t)(base + u) * ld + a] : INT_MAX;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int32_t b = buf[u];
      if (b != INT_MAX) {
        while (bs < b) {  // shell members below b that are not in the list
          if ((in >> j) & 1u) emit(bs);
          ++j;
          bs = j < ns ? shs[j][t] : INT_MAX;
        }
        if (bs == b) {  // a list member in the shell: kept if still in
          if ((in >> j) & 1u) emit(b);
          ++j;
          bs = j < ns ? shs[j][t] : INT_MAX;
        } else {
          emit(b);
        }
      }
    }
  }
  for (; j < ns; ++j)
    if ((in >> j) & 1u) emit(shs[j][t]);
  new_cnt[a] = min(cnt, kmax);
  if (cnt > kmax) raise_err(err, ERR_NB_OVERFLOW);
}

static void walk(sph_ctx *c, const sph_state *s, cudaStream_t st, const unsigned long long *grow, int32_t *idx,
                 int32_t *cnt, bool shell, const int32_t *run_if) {
  const int blocks = c->num_sms * c->tune.walk_blocks_per_sm * (4 / kNbWarps);
  if (shell)
    k_partners<false, true><<<blocks, kNbWarps * 32, 0, st>>>(
        c->tree, c->pk, s->x[0], s->x[1], s->x[2], s->h, s->dim, c->kmax, idx, cnt, c->cap_n, c->d_err, grow,
        c->units, run_if, nullptr, 0.0, 0, c->sh_idx, c->sh_cnt, c->sh_in, counters(c));
  else
    k_partners<false, false><<<blocks, kNbWarps * 32, 0, st>>>(
        c->tree, c->pk, s->x[0], s->x[1], s->x[2], s->h, s->dim, c->kmax, idx, cnt, c->cap_n, c->d_err, grow,
        c->units, run_if, nullptr, 0.0, 0, nullptr, nullptr, nullptr, counters(c));
  ++sph::g_launches;
}

void find_partners(sph_ctx *c, const sph_state *s, cudaStream_t st, const unsigned long long *grow, bool shell) {
  if (s->n == 0) return;
  walk(c, s, st, grow, c->nb_idx, c->nb_cnt, shell && c->sh_idx != nullptr, nullptr);
}

void refine_partners(sph_ctx *c, const sph_state *s, const unsigned long long *move, const unsigned long long *grow,
                     cudaStream_t st) {
  const int64_t n = s->n;
  if (n == 0) return;
  cudaMemsetAsync(c->need_walk, 0, sizeof(int32_t), st);
  { k_partners_refine<<<nblk(n, kRefineThreads), kRefineThreads, 0, st>>>(c->pk, s->x[0], s->x[1], s->x[2], s->h, s->dim, n, c->cap_n,
                                                   c->kmax, c->nb_idx, c->nb_cnt, c->sh_idx, c->sh_cnt, c->sh_in, c->nb_alt,
                                                   c->nb_cnt_alt, move, c->need_walk, c->d_err); ++sph::g_launches; }
  // returns at once unless a particle set the flag
  walk(c, s, st, grow, c->nb_alt, c->nb_cnt_alt, false, c->need_walk);
}

// ---------------------------------------------------------------------------
// Variable smoothing length (Sect. 4.2): count with the own h, then
// h <- (h / 2) (1 + (n_des / n_a)^(1/D)) for every particle when any count lies
// farther than tol from n_des (else the iteration is done)
// ---------------------------------------------------------------------------
__global__ void k_h_update(double *__restrict__ h, const int32_t *__restrict__ cnt, int64_t n, int dim,
                           double n_des, const int32_t *__restrict__ unconverged, int32_t *__restrict__ done,
                           int32_t *__restrict__ updates) {
  if (*done) return;
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (*unconverged == 0) {
    if (a == 0) *done = 1;
    return;
  }
  if (a == 0) atomicAdd(updates, 1);
  if (a >= n) return;
  const int32_t na = cnt[a];
  if (na == 0) {
    h[a] = 2.0 * h[a];
  } else {
    const double q = n_des / (double)na;
    const double r = dim == 3 ? cbrt(q) : (dim == 2 ? sqrt(q) : q);
    h[a] = h[a] * 0.5 * (1.0 + r);
  }
}

void adapt_h(sph_ctx *c, sph_state *s, double n_des, int tol, int max_iter, int32_t *flags, cudaStream_t st) {
  // flags: [0] done, [1] updates, [2 + i] particles off target at count i
  const int64_t n = s->n;
  cudaMemsetAsync(flags, 0, sizeof(int32_t) * (max_iter + 3), st);
  if (n == 0) return;
  const int blocks = c->num_sms * c->tune.walk_blocks_per_sm * (4 / kNbWarps);
  for (int i = 0; i <= max_iter; ++i) {
    { k_partners<true, false><<<blocks, kNbWarps * 32, 0, st>>>(c->tree, c->pk, s->x[0], s->x[1], s->x[2], s->h,
                                                               s->dim, c->kmax, c->nb_idx, c->nb_cnt, c->cap_n,
                                                               c->d_err, nullptr, c->units, flags, flags + 2 + i,
                                                               n_des, tol, nullptr, nullptr, nullptr, nullptr); ++sph::g_launches; }
    if (i == max_iter) break;
    { k_h_update<<<nblk(n, 256), 256, 0, st>>>(s->h, c->nb_cnt, n, s->dim, n_des, flags + 2 + i, flags,
                                             flags + 1); ++sph::g_launches; }
  }
}

// ---------------------------------------------------------------------------
// CSR export (ascending within a particle)
// ---------------------------------------------------------------------------
__global__ void k_cnt_copy(const int32_t *cnt, int32_t *out, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = cnt[i];
  if (i == n) out[n] = 0;
}

__global__ void k_csr_fill(const int32_t *__restrict__ nb_idx, const int32_t *__restrict__ nb_cnt, int64_t ld,
                           const int32_t *__restrict__ start, int64_t n, int64_t *off, int32_t *idx, int64_t cap,
                           int32_t *err) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a > n) return;
  off[a] = start[a];
  if (a == n) {
    if ((int64_t)start[n] > cap) raise_err(err, ERR_CSR_OVERFLOW);
    return;
  }
  int64_t o = start[a];
  int k = nb_cnt[a];
  if (o + k > cap) return;
  for (int i = 0; i < k; ++i) {  // insertion sort while copying
    int32_t v = nb_idx[(int64_t)i * ld + a];
    int j = i;
    while (j > 0 && idx[o + j - 1] > v) {
      idx[o + j] = idx[o + j - 1];
      --j;
    }
    idx[o + j] = v;
  }
}

void scan_counts(sph_ctx *c, const int32_t *in, int32_t *out, int64_t m, cudaStream_t st);

void partners_to_csr(sph_ctx *c, const sph_state *s, int64_t *off, int32_t *idx, int64_t cap, cudaStream_t st) {
  int64_t n = s->n;
  { k_cnt_copy<<<nblk(n + 1, 256), 256, 0, st>>>(c->nb_cnt, c->tree.ncount, n); ++sph::g_launches; }
  scan_counts(c, c->tree.ncount, c->tree.nstart, n + 1, st);
  { k_csr_fill<<<nblk(n + 1, 128), 128, 0, st>>>(c->nb_idx, c->nb_cnt, c->cap_n, c->tree.nstart, n, off, idx, cap,
                                               c->d_err); ++sph::g_launches; }
}

}  // namespace sph
