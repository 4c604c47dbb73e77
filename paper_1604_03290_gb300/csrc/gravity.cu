// Barnes-Hut self-gravity (Sect. 3.3), GB300 form.
//
// A warp walks the pre-order tree for 32 consecutive sorted particles.
// Acceptance stays per particle, exactly as in a per-particle walk: a lane
// that uses node n as a pseudo-particle ignores the rest of n's subtree
// (ids below skip[n]); the warp enters n's children if any lane rejected
// n.  Leaves rejected by a lane are summed particle by particle (self
// skipped), staged through shared memory.  The accepted set of every
// particle - hence the sum - is the one of the per-particle definition:
//   node used iff its cube does not contain a and s / r < theta
//   (s = s0 / 2^level, r = |x_a - com|, evaluated as s < theta * r);
//   a_a = -G sum m_p (x_a - x_p) / (r^2 + eps_a^2)^1.5, eps_a = eps_grav h_a
// (the paper's Eq. gravitational_force read as attractive, with Plummer
// softening).
//
// Reused tree (gravity/hydro decoupling, Sect. 6.3): the pseudo-particles,
// node cubes and leaf membership are those of the build, the particle's cell
// is recomputed from its current position in the build's root cube, and
// leaves are summed at the members' current positions (the packed views are
// refreshed before the walk).
//
// Mixed precision: distances from hi/lo split coordinates in FP32, the
// acceptance test in FP32 with a relative band of 1e-4 around the threshold
// inside which the FP64 expression decides, FP32 monopole terms summed with
// Kahan compensation.
#include <type_traits>

#include "morton.cuh"
#include "sph_internal.cuh"

namespace sph {

// One warp (one particle group at a time) per block, 32 resident blocks per
// SM at 64 registers: measured on GB300 (2M cloud) 33.1 ms per step against
// 34.5 (4 warps x 8 blocks), 34.8 (8 x 4) and 36.1 (2 x 16).
#ifndef SPH_GRAV_WARPS
#define SPH_GRAV_WARPS 1
#endif
constexpr int kGrWarps = SPH_GRAV_WARPS;  // warps (particle groups) per block
// resident blocks per SM the walk is compiled for (register budget)
#ifndef SPH_GRAV_MIN_BLOCKS
#define SPH_GRAV_MIN_BLOCKS 32
#endif
constexpr float kMacBand = 1e-4f;
constexpr int kFlushTerms = 16;
// A leaf summed directly by few lanes: rather than each of them looping over
// the members while the others wait, the warp takes the lanes one at a time,
// every member lane evaluates its term for that lane, and a butterfly sum
// over the warp gives the leaf's contribution (mixed precision).  Chosen when
// (lanes summing the leaf) x kTransposedCost < (members) x kSerialCost, the
// instruction counts of the two forms per lane and per member.
constexpr int kTransposedCost = 66, kSerialCost = 29;

// Sum of the FP32 terms of one particle: a plain partial sum, added into a
// compensated (Kahan) sum every kFlushTerms terms, so that the error stays
// near that of a compensated sum (the partial sums are short) at a fraction
// of its cost per term.
struct GravSumF {
  float px = 0.f, py = 0.f, pz = 0.f;
  int n = 0;
  KahanT<float> kx, ky, kz;
  __device__ __forceinline__ void flush() {
    kx.add(px);
    ky.add(py);
    kz.add(pz);
    px = py = pz = 0.f;
    n = 0;
  }
  __device__ __forceinline__ void add(float fx, float fy, float fz) {
    px += fx;
    py += fy;
    pz += fz;
    if (++n == kFlushTerms) flush();
  }
  __device__ __forceinline__ void value(double &x, double &y, double &z) {
    flush();
    x = kx.value();
    y = ky.value();
    z = kz.value();
  }
};

struct GravSumD {
  double sx = 0.0, sy = 0.0, sz = 0.0;
  __device__ __forceinline__ void add(double fx, double fy, double fz) {
    sx += fx;
    sy += fy;
    sz += fz;
  }
  __device__ __forceinline__ void value(double &x, double &y, double &z) {
    x = sx;
    y = sy;
    z = sz;
  }
};

// 1 / q^(3/2): from the reciprocal square root in FP32 (a few ulps, far below
// the mixed form's tolerance), correctly rounded operations in FP64
__device__ __forceinline__ float inv_q32(float q) {
  const float r = rsqrtf(q);
  return r * r * r;
}
__device__ __forceinline__ double inv_q32(double q) { return 1.0 / (q * sqrt(q)); }

struct GravArgs {
  Tree T;
  PackedF32 pk;
  const double *x[3], *m, *h;
  int dim;
  double G, theta, eps;
  double *out[3];
  const Units *U;
  int32_t *err;
  int reuse;  // the tree was built at earlier positions: locate each particle anew
  unsigned long long *ctr;  // NULL, or the interaction counters
};

template <int DIM>
__device__ __forceinline__ double r2_fp64(const double xa[3], double cx, double cy, double cz) {
  double dx = __dsub_rn(xa[0], cx);
  double dy = __dsub_rn(xa[1], cy);
  double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  if (DIM == 3) {
    double dz = __dsub_rn(xa[2], cz);
    r2 = __dadd_rn(r2, __dmul_rn(dz, dz));
  }
  return r2;
}

// PACKED (mixed, Tree::packed_walk): a node's skip, level and leaf flag come
// from the w word of its second COM view, so that a visit loads two float4
// (the node's member range only when some lane sums it directly), and the
// node edge s0 / 2^level is the instance's FP32 edge shifted by the level:
// the same value k_node_finish stores otherwise.
template <bool MIXED, int DIM, bool PACKED>
__global__ void __launch_bounds__(kGrWarps * 32, SPH_GRAV_MIN_BLOCKS) k_gravity(GravArgs A) {
  static_assert(MIXED || !PACKED, "the packed word is read by the mixed walk");
  using R = typename std::conditional<MIXED, float, double>::type;
  __shared__ float4 sh_hi[kGrWarps][kMaxLeaf];  // (x_hi, y_hi, z_hi, G m_b) of leaf members
  __shared__ float4 sh_lo[kGrWarps][kMaxLeaf];
  __shared__ int32_t sh_b[kGrWarps][kMaxLeaf];
  const Tree &T = A.T;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Warps take groups of particles; acceptance is per particle, so any
  // grouping gives the same sums.  One instance: full chunks of 32
  // consecutive slots (Morton order keeps them close); several: the tree's
  // groups, which never span instances.
  const bool chunks = T.ninst <= 1;
  const int ngroups = chunks ? (int)((T.n + 31) >> 5) : *T.ngroups;
  constexpr int dim = DIM;
  const int L = T.leaf_size, B = T.max_depth;
  const int nnodes = T.iter_cap > 0 ? min(*T.nnodes, T.iter_cap) : *T.nnodes;
  const int64_t cap = T.cap_nodes;
  const double Gs = MIXED ? A.G * A.U->M * A.U->T * A.U->T * A.U->invL * A.U->invL * A.U->invL : A.G;
  const R G = (R)Gs;
  for (int g = blockIdx.x * kGrWarps + w; g < ngroups; g += gridDim.x * kGrWarps) {
    const int32_t s0 = chunks ? g * 32 : T.grp_start[g];
    const int32_t s1 = chunks ? (int32_t)(((int64_t)s0 + 32 < T.n) ? (int64_t)s0 + 32 : T.n) : T.grp_end[g];
    const int inst = chunks ? 0 : T.grp_inst[g];
    const int32_t slot = s0 + lane;
    const bool act = slot < s1;
    const int32_t a = act ? (T.perm_identity ? slot : T.perm[slot]) : 0;  // identity: state in tree order
    double xa[3] = {0, 0, 0};
    for (int ax = 0; ax < dim; ++ax) xa[ax] = A.x[ax][a];
    // the cell of the particle's current position (the key of the build
    // unless the tree is reused); node cubes are those of the build
    const unsigned long long ka =
        !act ? 0ULL
             : (A.reuse ? morton_key(xa, dim, B, inst, T.inst_lo, T.inst_s0[inst], T.inst_rs0[inst]) : T.skey[slot]);
    const float4 Pa = A.pk.px(a), Qa = A.pk.pxl(a);
    const double e = MIXED ? A.eps * (double)Pa.w : A.eps * A.h[a];
    const R eps2 = (R)(e * e);
    const double s0r = T.inst_s0[inst];
    // the instance's root edge in FP32 code units (PACKED: shifted by the level per node)
    const float s0f = PACKED ? to_f32_scaled(s0r, pow2_exp(A.U->invL), A.U->invL) : 0.f;
    const double th = A.theta;
    const float th2f = (float)(th * th);
    // A node whose cube holds the particle also holds its centre of mass, so
    // r <= sqrt(D) s there; with D theta^2 < 1 (by a margin far above the
    // rounding of either test) the opening criterion already rejects it and
    // the containment test can be skipped: the accepted set is the same.
    const bool test_inside = (double)dim * th * th >= 0.99;
    typename std::conditional<MIXED, GravSumF, GravSumD>::type acc;
    int32_t skip_until = -1;
    const int32_t root = T.inst_root[inst];
    const int32_t stop = root >= 0 ? T.skip[root] : root;
    int iter = 0;
    unsigned nacc = 0, nterm = 0;  // this lane's accepted nodes and particle terms (counters)
    for (int32_t nd = root; nd < stop && iter <= nnodes; ++iter) {
      int32_t f = 0, e1 = 0, sk;
      int lev;
      bool leaf;
      float4 ch, cl;
      if constexpr (PACKED) {
        ch = T.fcom_hi[nd];
        cl = T.fcom_lo[nd];
        const uint32_t wd = __float_as_uint(cl.w);
        sk = (int32_t)(wd & (uint32_t)kPackedSkip);
        lev = (int)((wd >> 26) & 31u);
        leaf = (wd >> 31) != 0u;
      } else {
        const int4 rec = T.nrec[nd];  // (first, end, skip, level)
        f = rec.x;
        e1 = rec.y;
        sk = rec.z;
        lev = rec.w;
        leaf = (e1 - f <= L) || lev == B;
      }
      bool open = false, direct = false;
      if (act && nd >= skip_until) {
        const bool inside = test_inside && (ka >> (dim * (B - lev))) == T.cell[nd];
        bool accept = false;
        float mpf = 0.f;
        R d[3] = {R(0), R(0), R(0)}, r2 = R(0);
        if (!inside) {
          if constexpr (MIXED) {
            if constexpr (!PACKED) {
              ch = T.fcom_hi[nd];
              cl = T.fcom_lo[nd];
            }
            d[0] = (Pa.x - ch.x) + (Qa.x - cl.x);
            d[1] = (Pa.y - ch.y) + (Qa.y - cl.y);
            d[2] = (Pa.z - ch.z) + (Qa.z - cl.z);
            r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            mpf = ch.w;
            const float sf = PACKED ? __int_as_float(__float_as_int(s0f) - (lev << 23)) : cl.w;
            const float lhs = sf * sf, rhs = th2f * r2;
            if (lhs < rhs * (1.0f - kMacBand)) accept = true;
            else if (lhs > rhs * (1.0f + kMacBand)) accept = false;
            else {
              // rare: the FP64 decision, from values reloaded here rather than kept live in the loop
              const double xr[3] = {A.x[0][a], A.x[1][a], DIM == 3 ? A.x[2][a] : 0.0};
              accept = ldexp(T.inst_s0[inst], -lev) <
                       A.theta * sqrt(r2_fp64<DIM>(xr, T.com[nd], T.com[cap + nd], DIM == 3 ? T.com[2 * cap + nd] : 0.0));
            }
          } else {
            const double s = ldexp(s0r, -lev);
            const double cx = T.com[nd], cy = T.com[cap + nd], cz = DIM == 3 ? T.com[2 * cap + nd] : 0.0;
            d[0] = xa[0] - cx;
            d[1] = xa[1] - cy;
            d[2] = DIM == 3 ? xa[2] - cz : 0.0;
            r2 = r2_fp64<DIM>(xa, cx, cy, cz);
            accept = s < th * sqrt(r2);
          }
        }
        if (accept) {
          const R mp = MIXED ? (R)mpf : (R)T.mass[nd];
          const R gq = -G * mp * inv_q32(r2 + eps2);
          acc.add(gq * d[0], gq * d[1], dim == 3 ? gq * d[2] : R(0));
          skip_until = sk;
          ++nacc;
        } else if (leaf) {
          direct = true;
          skip_until = sk;
        } else {
          open = true;
        }
      }
      const bool any_open = __any_sync(0xffffffffu, open);
      const unsigned dmask = __ballot_sync(0xffffffffu, direct);
      if (dmask) {
        if constexpr (PACKED) {
          const int4 rec = T.nrec[nd];
          f = rec.x;
          e1 = rec.y;
        }
        for (int32_t base = f; base < e1; base += kMaxLeaf) {
          const int c = min(e1 - base, kMaxLeaf);
          int32_t bm = -1;
          float4 pb = make_float4(0.f, 0.f, 0.f, 0.f), qb = pb;
          if (lane < c) {
            bm = T.perm_identity ? base + lane : T.perm[base + lane];
            pb = A.pk.px(bm);
            qb = A.pk.pxl(bm);
            sh_hi[w][lane] = make_float4(pb.x, pb.y, pb.z, -(float)G * qb.w);  // qb.w = m as float
            sh_lo[w][lane] = make_float4(qb.x, qb.y, qb.z, qb.w);
            sh_b[w][lane] = bm;
          }
          __syncwarp();
          bool transposed = false;
          if constexpr (MIXED) transposed = __popc(dmask) * kTransposedCost < c * kSerialCost;
          if (transposed) {
            const float gmk = -(float)G * qb.w;
            unsigned mm = dmask;
            while (mm) {
              const int i = __ffs(mm) - 1;
              mm &= mm - 1;
              // lane i's particle, against member `lane`
              const float ax = __shfl_sync(0xffffffffu, Pa.x, i), ay = __shfl_sync(0xffffffffu, Pa.y, i),
                          az = __shfl_sync(0xffffffffu, Pa.z, i);
              const float lx = __shfl_sync(0xffffffffu, Qa.x, i), ly = __shfl_sync(0xffffffffu, Qa.y, i),
                          lz = __shfl_sync(0xffffffffu, Qa.z, i);
              const float e2i = __shfl_sync(0xffffffffu, (float)eps2, i);
              const int32_t ai = __shfl_sync(0xffffffffu, a, i);
              float fx = 0.f, fy = 0.f, fz = 0.f;
              bool ok = false;
              if (lane < c && bm != ai) {
                const float dx = (ax - pb.x) + (lx - qb.x), dy = (ay - pb.y) + (ly - qb.y),
                            dz = (az - pb.z) + (lz - qb.z);
                const float q = dx * dx + dy * dy + dz * dz + e2i;
                if (q > 0.f) {
                  const float gq = gmk * inv_q32(q);
                  fx = gq * dx;
                  fy = gq * dy;
                  fz = gq * dz;
                  ok = true;
                }
              }
              for (int o = 16; o > 0; o >>= 1) {
                fx += __shfl_xor_sync(0xffffffffu, fx, o);
                fy += __shfl_xor_sync(0xffffffffu, fy, o);
                fz += __shfl_xor_sync(0xffffffffu, fz, o);
              }
              const unsigned okm = __ballot_sync(0xffffffffu, ok);
              if (lane == i) {
                acc.add((R)fx, (R)fy, dim == 3 ? (R)fz : R(0));
                nterm += __popc(okm);
              }
            }
          } else if (direct) {
            for (int k = 0; k < c; ++k) {
              const int32_t b = sh_b[w][k];
              if (b == a) continue;
              R d[3], gm;  // gm = -G m_b
              if constexpr (MIXED) {
                const float4 ph = sh_hi[w][k], pl = sh_lo[w][k];
                d[0] = (Pa.x - ph.x) + (Qa.x - pl.x);
                d[1] = (Pa.y - ph.y) + (Qa.y - pl.y);
                d[2] = (Pa.z - ph.z) + (Qa.z - pl.z);
                gm = ph.w;
              } else {
                for (int ax = 0; ax < 3; ++ax) d[ax] = ax < dim ? xa[ax] - A.x[ax][b] : 0.0;
                gm = -G * A.m[b];
              }
              const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
              const R q = r2 + eps2;
              if (!(q > R(0))) continue;
              const R gq = gm * inv_q32(q);
              acc.add(gq * d[0], gq * d[1], dim == 3 ? gq * d[2] : R(0));
              ++nterm;
            }
          }
          __syncwarp();
        }
      }
      nd = any_open ? nd + 1 : sk;
    }
    if (iter > nnodes) raise_err(A.err, ERR_TIMEOUT);
    if (A.ctr) {
      warp_count(A.ctr + CTR_GRAV_NODES, nacc);
      warp_count(A.ctr + CTR_GRAV_TERMS, nterm);
      if (lane == 0) atomicAdd(A.ctr + CTR_GRAV_VISITS, (unsigned long long)iter);
    }
    if (act) {
      double gx, gy, gz;
      acc.value(gx, gy, gz);
      const double osc = MIXED ? A.U->acc : 1.0;
      A.out[0][a] = gx * osc;
      A.out[1][a] = gy * osc;
      if (DIM == 3) A.out[2][a] = gz * osc;
    }
  }
}

void gravity_walk(sph_ctx *c, const sph_state *s, const sph_params &p, double *ax, double *ay, double *az,
                  cudaStream_t st, bool reuse) {
  if (s->n == 0) return;
  GravArgs A;
  memset(&A, 0, sizeof(A));
  A.T = c->tree;
  A.pk = c->pk;
  for (int k = 0; k < 3; ++k) A.x[k] = s->x[k];
  A.m = s->m;
  A.h = s->h;
  A.dim = s->dim;
  A.G = p.G;
  A.theta = p.theta;
  A.eps = p.eps_grav;
  A.out[0] = ax;
  A.out[1] = ay;
  A.out[2] = az;
  A.U = c->units;
  A.err = c->d_err;
  A.reuse = reuse ? 1 : 0;
  A.ctr = counters(c);
  int blocks = c->num_sms * SPH_GRAV_MIN_BLOCKS;  // persistent: the resident blocks, looping over groups
  const bool mixed = p.precision == SPH_MIXED;
  const bool packed = mixed && c->tree.packed_walk;
  if (s->dim == 3) {
    if (packed) { k_gravity<true, 3, true><<<blocks, kGrWarps * 32, 0, st>>>(A); ++sph::g_launches; }
    else if (mixed) { k_gravity<true, 3, false><<<blocks, kGrWarps * 32, 0, st>>>(A); ++sph::g_launches; }
    else { k_gravity<false, 3, false><<<blocks, kGrWarps * 32, 0, st>>>(A); ++sph::g_launches; }
  } else {
    if (packed) { k_gravity<true, 2, true><<<blocks, kGrWarps * 32, 0, st>>>(A); ++sph::g_launches; }
    else if (mixed) { k_gravity<true, 2, false><<<blocks, kGrWarps * 32, 0, st>>>(A); ++sph::g_launches; }
    else { k_gravity<false, 2, false><<<blocks, kGrWarps * 32, 0, st>>>(A); ++sph::g_launches; }
  }
}

}  // namespace sph
