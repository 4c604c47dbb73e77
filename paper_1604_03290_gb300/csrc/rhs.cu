// SPH right-hand side (Sect. 3.1-3.2), GB300 form: two gather passes over
// the partner lists, one thread per particle, particles in Morton order so
// that a warp's partners share cache lines.
//
//   pass A  (Sects. 3.1.2, 3.1.5, 3.1.6): continuity sum, the correction
//           tensor L, the velocity-gradient sum G, XSPH; then, in the same
//           thread, the per-particle constitutive update: EOS (Sect. 2.5),
//           Hooke + Jaumann (Sect. 2.4), von Mises (Sect. 2.6), damage
//           (Sects. 2.7, 3.2) and artificial stress (Sect. 3.1.4);
//   pass B  (Eqs. accel_artvisc, energy_sph): momentum and energy with the
//           stress bracket of both particles and artificial viscosity.
//
// Readings of the paper used here (same as the CPU oracle's):
//   - momentum / energy: dv_a/dt = sum m_b [T_a + T_b + (zeta_a+zeta_b) f^n
//     - Pi* I] grad_a W, du_a/dt = -1/2 sum m_b v_ab.[T_a + T_b - Pi* I]
//     grad_a W, with T = sigma / rho^2 (the printed d/dx_b form with +Pi
//     would make pressure attractive);
//   - L^{ag} = sum (m_b/rho_b) (x_b - x_a)^a d_g W (the form in which
//     L C = I holds), C = L^-1 unless det L is tiny or there are fewer than
//     D + 1 partners;
//   - Jaumann terms R S - S R (co-rotational), deviator in D dimensions;
//   - XSPH with the mean density (rho_a + rho_b)/2;
//   - artificial stress built in the principal frame of sigma;
//   - Tillotson sound speed c^2 = max(A/rho0, dp/drho + p/rho^2 dp/du);
//   - crack speed c_g = 0.4 sqrt((K + 4/3 (1-d) mu)/rho), R_s = h.
//
// Precision.  FP64 mode: everything in double.  Mixed mode: pair arithmetic
// in FP32 on differences of hi/lo-split positions and velocities (so a
// difference keeps ~48 bits before it is rounded to FP32), Kahan-compensated
// FP32 sums for density, momentum and energy, FP32 constitutive update except
// that rho - rho0 (the cold-expansion cancellation) is formed in FP64.
#include <type_traits>

#include "eos.cuh"
#include "fpbits.cuh"
#include "sph_internal.cuh"

namespace sph {

struct RhsArgs {
  int dim;
  int64_t n, ld;
  const double *x[3], *v[3];
  const double *rho, *u, *m, *h, *S, *dmg;
  const int32_t *mat, *id;
  const int64_t *flaw_off;
  const float *flaw_eps;
  const int32_t *nb_idx, *nb_cnt;
  // a count of -1 (a refined list left as it was) means: the list and count
  // of the walk it was refined from, here
  const int32_t *nb_idx2, *nb_cnt2;
  PackedF32 pk;
  double *dx[3], *dv[3], *drho, *du, *dS, *ddmg, *p_out, *cs_out;
  int32_t *nact, *nnb;
  double *Td, *Zd, *csd;    // FP64 pass-A -> pass-B data, component-major with stride ld
  float4 *Tf, *Zf;          // mixed: 2 float4 per particle each (stride ld)
  const double *ag;         // gravity (3 * ld) or NULL
  double *rho_out;          // density-sum output
  const Units *U;           // code units of the FP32 views (mixed mode)
  float *sums;              // mixed, KEEP_SUMS: pass A's pair sums (16 rows of stride ld)
  MatTable mt;
  sph_params prm;
  int32_t *err;
};

template <class R>
__device__ __forceinline__ R rsqrt_or_zero(R r2);
template <>
__device__ __forceinline__ float rsqrt_or_zero<float>(float r2) {
  return r2 > 0.f ? rsqrtf(r2) : 0.f;
}
template <>
__device__ __forceinline__ double rsqrt_or_zero<double>(double r2) {
  return r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
}

// Resident blocks per SM the neighbour passes are compiled for (register
// budget).  Measured on GB300 with the partner prefetch below: pass A is
// fastest at 7 (capped registers, positions alone prefetched) in mixed
// precision, pass B with the compiler's own choice.
#ifndef SPH_PASSA_MIN_BLOCKS
#define SPH_PASSA_MIN_BLOCKS 7
#endif
#define SPH_PASSA_BOUNDS __launch_bounds__(128, MIXED ? SPH_PASSA_MIN_BLOCKS : 1)  // FP64: uncapped
#ifdef SPH_PASSB_MIN_BLOCKS
#define SPH_PASSB_BOUNDS __launch_bounds__(128, SPH_PASSB_MIN_BLOCKS)
#else
#define SPH_PASSB_BOUNDS __launch_bounds__(128)
#endif

// 1 / x, correctly rounded: the same value as the division
template <class R>
__device__ __forceinline__ R rcp_rn(R x);
template <>
__device__ __forceinline__ float rcp_rn<float>(float x) {
  return __frcp_rn(x);
}
template <>
__device__ __forceinline__ double rcp_rn<double>(double x) {
  return __drcp_rn(x);
}

// Reciprocal and quotient inside the pair loops.  Mixed: the hardware's
// approximations (relative error below 2^-22, a few FP32 roundings of a pair
// term, well inside the mixed tolerance; operands are in code units, far from
// the subnormal range).  FP64: correctly rounded, as everywhere else.
#ifndef SPH_FAST_PAIR_MATH
#define SPH_FAST_PAIR_MATH 1
#endif
template <class R>
__device__ __forceinline__ R pair_rcp(R x);
template <>
__device__ __forceinline__ float pair_rcp<float>(float x) {
#if SPH_FAST_PAIR_MATH
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return __frcp_rn(x);
#endif
}
template <>
__device__ __forceinline__ double pair_rcp<double>(double x) {
  return __drcp_rn(x);
}
template <class R>
__device__ __forceinline__ R pair_div(R a, R b);
template <>
__device__ __forceinline__ float pair_div<float>(float a, float b) {
#if SPH_FAST_PAIR_MATH
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
template <>
__device__ __forceinline__ double pair_div<double>(double a, double b) {
  return a / b;
}

// ---------------------------------------------------------------------------
// Pair geometry: a - b differences of position and velocity, b's scalars.
// ---------------------------------------------------------------------------
template <bool MIXED>
struct Own;

template <>
struct Own<false> {
  double x[3], v[3], h, rho, m;
  __device__ void load(const RhsArgs &A, int64_t a) {
    for (int ax = 0; ax < 3; ++ax) {
      x[ax] = ax < A.dim ? A.x[ax][a] : 0.0;
      v[ax] = ax < A.dim ? A.v[ax][a] : 0.0;
    }
    h = A.h[a];
    rho = A.rho[a];
    m = A.m[a];
  }
  // d = x_a - x_b, w = v_a - v_b
  __device__ __forceinline__ void pair(const RhsArgs &A, int32_t b, double d[3], double w[3], double &hb,
                                       double &rhob, double &mb, double &vol) const {
    for (int ax = 0; ax < 3; ++ax) {
      d[ax] = ax < A.dim ? x[ax] - A.x[ax][b] : 0.0;
      w[ax] = ax < A.dim ? v[ax] - A.v[ax][b] : 0.0;
    }
    hb = A.h[b];
    rhob = A.rho[b];
    mb = A.m[b];
    vol = mb / rhob;
  }
  // the same split into the loads of b (issued ahead) and the arithmetic
  struct Raw {
    int32_t b;
  };
  using RawPos = Raw;
  __device__ __forceinline__ Raw fetch(const RhsArgs &, int32_t b) const { return Raw{b}; }
  __device__ __forceinline__ Raw fetch_pos(const RhsArgs &, int32_t b) const { return Raw{b}; }
  __device__ __forceinline__ void from(const RhsArgs &A, const Raw &r, double d[3], double w[3], double &hb,
                                       double &rhob, double &mb, double &vol) const {
    pair(A, r.b, d, w, hb, rhob, mb, vol);
  }
};

template <>
struct Own<true> {
  float4 P, Q, V, W;
  float h, rho, m;
  __device__ void load(const RhsArgs &A, int64_t a) {
    P = A.pk.px(a);
    Q = A.pk.pxl(a);
    V = A.pk.pv(a);
    W = A.pk.pvl(a);
    h = P.w;
    rho = V.w;
    m = Q.w;
  }
  struct Raw {
    float4 P, Q, V, W;
  };
  // the positions alone, the velocity views loaded when the pair is evaluated
  struct RawPos {
    float4 P, Q;
    int32_t b;
  };
  __device__ __forceinline__ Raw fetch(const RhsArgs &A, int32_t b) const {
    return Raw{A.pk.px(b), A.pk.pxl(b), A.pk.pv(b), A.pk.pvl(b)};
  }
  __device__ __forceinline__ RawPos fetch_pos(const RhsArgs &A, int32_t b) const {
    return RawPos{A.pk.px(b), A.pk.pxl(b), b};
  }
  __device__ __forceinline__ void from(const RhsArgs &, const Raw &r, float d[3], float w[3], float &hb,
                                       float &rhob, float &mb, float &vol) const {
    unpack(r.P, r.Q, r.V, r.W, d, w, hb, rhob, mb, vol);
  }
  __device__ __forceinline__ void from(const RhsArgs &A, const RawPos &r, float d[3], float w[3], float &hb,
                                       float &rhob, float &mb, float &vol) const {
    unpack(r.P, r.Q, A.pk.pv(r.b), A.pk.pvl(r.b), d, w, hb, rhob, mb, vol);
  }
  __device__ __forceinline__ void pair(const RhsArgs &A, int32_t b, float d[3], float w[3], float &hb, float &rhob,
                                       float &mb, float &vol) const {
    unpack(A.pk.px(b), A.pk.pxl(b), A.pk.pv(b), A.pk.pvl(b), d, w, hb, rhob, mb, vol);
  }
  __device__ __forceinline__ void unpack(const float4 Pb, const float4 Qb, const float4 Vb, const float4 Wb, float d[3],
                                         float w[3], float &hb, float &rhob, float &mb, float &vol) const {
    d[0] = (P.x - Pb.x) + (Q.x - Qb.x);
    d[1] = (P.y - Pb.y) + (Q.y - Qb.y);
    d[2] = (P.z - Pb.z) + (Q.z - Qb.z);
    w[0] = (V.x - Vb.x) + (W.x - Wb.x);
    w[1] = (V.y - Vb.y) + (W.y - Wb.y);
    w[2] = (V.z - Vb.z) + (W.z - Wb.z);
    hb = Pb.w;
    rhob = Vb.w;
    mb = Qb.w;
    vol = Wb.w;
  }
};

// ---------------------------------------------------------------------------
// Partner cursor: the column-major list of particle a, read with the index
// two pairs ahead and the neighbour's data one pair ahead, so that the
// gathers of pair k + 1 are in flight while pair k is evaluated.
// ---------------------------------------------------------------------------
#ifndef SPH_PASS_PREFETCH
#define SPH_PASS_PREFETCH 1
#endif

// Particle a's partner column and count (see RhsArgs::nb_idx2)
__device__ __forceinline__ int partner_list(const RhsArgs &A, int64_t a, const int32_t *&col) {
  int cnt = A.nb_cnt[a];
  col = A.nb_idx + a;
  if (cnt < 0) {
    cnt = A.nb_cnt2[a];
    col = A.nb_idx2 + a;
  }
  return cnt;
}

// POS: only the partner's position views are loaded ahead (pass A, whose
// registers then allow 7 resident blocks per SM: 4 % faster on GB300); pass B
// loads positions and velocities ahead (its stress pack in the loop body:
// prefetching that too took three more registers and made it 6 % slower).
template <bool MIXED, bool POS = false>
struct PartnerCursor {
  using Raw = typename std::conditional<POS, typename Own<MIXED>::RawPos, typename Own<MIXED>::Raw>::type;
  __device__ __forceinline__ static Raw get(const RhsArgs &A, const Own<MIXED> &o, int32_t b) {
    if constexpr (POS) return o.fetch_pos(A, b);
    else return o.fetch(A, b);
  }
  const int32_t *col;
  int64_t ld;
  int cnt;
  int32_t b1, b2;
  Raw r1;
  __device__ __forceinline__ void start(const RhsArgs &A, const Own<MIXED> &o, const int32_t *list, int n) {
    col = list;
    ld = A.ld;
    cnt = n;
    b1 = n > 0 ? col[0] : 0;
    b2 = n > 1 ? col[ld] : 0;
    if (n > 0) r1 = get(A, o, b1);
  }
  // the pair k: its index and its raw data
  __device__ __forceinline__ int32_t next(const RhsArgs &A, const Own<MIXED> &o, int k, Raw &cur) {
    const int32_t b = b1;
    cur = r1;
    b1 = b2;
    if (k + 2 < cnt) b2 = col[(int64_t)(k + 2) * ld];
    if (k + 1 < cnt) r1 = get(A, o, b1);
    return b;
  }
};

// ---------------------------------------------------------------------------
// Density by kernel sum (Eq. density_by_kernel_sum) including m_a W(0; h_a).
// ---------------------------------------------------------------------------
template <bool MIXED, int DIM>
__global__ void __launch_bounds__(128) k_density_sum(RhsArgs A) {
  using R = typename std::conditional<MIXED, float, double>::type;
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A.n) return;
  Own<MIXED> o;
  o.load(A, a);
  constexpr int dim = DIM;
  const R sig = kernel_sigma<R>(dim);
  KahanT<R> sum;
  {
    R hinv = rcp_rn((R)o.h);
    sum.add((R)o.m * sig * hpow(hinv, dim));
  }
  const int32_t *list;
  const int cnt = partner_list(A, a, list);
  for (int k = 0; k < cnt; ++k) {
    const int32_t b = list[(int64_t)k * A.ld];
    R d[3], w[3], hb, rhob, mb, vol;
    o.pair(A, b, d, w, hb, rhob, mb, vol);
    R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    R r = r2 * rsqrt_or_zero(r2);
    R hinv = pair_rcp(R(0.5) * ((R)o.h + hb));
    sum.add(mb * kern_W(r * hinv, sig * hpow(hinv, dim)));
  }
  A.rho_out[a] = sum.value() * (MIXED ? A.U->rho : 1.0);
}

// ---------------------------------------------------------------------------
// Per-particle helpers
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R det_of(int dim, const R M[3][3]) {
  if (dim == 2) return M[0][0] * M[1][1] - M[0][1] * M[1][0];
  return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
         M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

// C = L^-1 by cofactors; identity when L is (nearly) singular.
template <class R>
__device__ __forceinline__ void correction_tensor(int dim, const R L[3][3], bool enable, R C[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i][j] = i == j ? R(1) : R(0);
  if (!enable) return;
  R det = det_of(dim, L);
  R diag = R(1);
  for (int i = 0; i < dim; ++i) diag *= fabs(L[i][i]);
  if (!(fabs(det) > R(1e-8) * diag) || !(diag > R(0))) return;
  R inv = rcp_rn(det);
  if (dim == 2) {
    C[0][0] = L[1][1] * inv;
    C[0][1] = -L[0][1] * inv;
    C[1][0] = -L[1][0] * inv;
    C[1][1] = L[0][0] * inv;
    return;
  }
  C[0][0] = (L[1][1] * L[2][2] - L[1][2] * L[2][1]) * inv;
  C[0][1] = (L[0][2] * L[2][1] - L[0][1] * L[2][2]) * inv;
  C[0][2] = (L[0][1] * L[1][2] - L[0][2] * L[1][1]) * inv;
  C[1][0] = (L[1][2] * L[2][0] - L[1][0] * L[2][2]) * inv;
  C[1][1] = (L[0][0] * L[2][2] - L[0][2] * L[2][0]) * inv;
  C[1][2] = (L[0][2] * L[1][0] - L[0][0] * L[1][2]) * inv;
  C[2][0] = (L[1][0] * L[2][1] - L[1][1] * L[2][0]) * inv;
  C[2][1] = (L[0][1] * L[2][0] - L[0][0] * L[2][1]) * inv;
  C[2][2] = (L[0][0] * L[1][1] - L[0][1] * L[1][0]) * inv;
}

// Symmetric eigen-decomposition by cyclic Jacobi rotations: A is overwritten
// by its (diagonal) spectral form, V accumulates the rotations (columns are
// eigenvectors).  Each rotation zeroes A[p][q] with t = tan of the angle,
// t = sign(tau)/(|tau| + sqrt(1 + tau^2)), tau = (A_qq - A_pp)/(2 A_pq).
template <class R>
__device__ __forceinline__ void jacobi_rotate(int p, int q, R A[3][3], R V[3][3], int dim) {
  R apq = A[p][q];
  if (apq == R(0)) return;
  R tau = (A[q][q] - A[p][p]) / (R(2) * apq);
  R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
  R c = R(1) / sqrt(R(1) + t * t), s = t * c;
  A[p][p] -= t * apq;
  A[q][q] += t * apq;
  A[p][q] = A[q][p] = R(0);
  for (int r = 0; r < dim; ++r) {
    if (r != p && r != q) {
      R arp = A[r][p], arq = A[r][q];
      A[r][p] = A[p][r] = c * arp - s * arq;
      A[r][q] = A[q][r] = s * arp + c * arq;
    }
    R vrp = V[r][p], vrq = V[r][q];
    V[r][p] = c * vrp - s * vrq;
    V[r][q] = s * vrp + c * vrq;
  }
}

template <class R>
__device__ __forceinline__ void sym_eigen(int dim, R A[3][3], R w[3], R V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = i == j ? R(1) : R(0);
  if (dim == 2) {
    jacobi_rotate(0, 1, A, V, 2);
  } else {
    const R tiny = sizeof(R) == 4 ? R(1e-14) : R(1e-30);
    for (int sweep = 0; sweep < 12; ++sweep) {
      R off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
      R dg = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
      if (!(off > tiny * dg)) break;
      jacobi_rotate(0, 1, A, V, 3);
      jacobi_rotate(0, 2, A, V, 3);
      jacobi_rotate(1, 2, A, V, 3);
    }
  }
  for (int i = 0; i < 3; ++i) w[i] = i < dim ? A[i][i] : R(0);
}

// ---------------------------------------------------------------------------
// Pass A + per-particle update
// ---------------------------------------------------------------------------
// KEEP_SUMS (mixed, for the adjoint): also store the pair sums in A.sums,
// rows of stride ld: 0 the continuity sum sum_b V_b (v_a - v_b).grad W (code
// units 1/T), 1..6 the lower triangle of L (00, 10, 11, 20, 21, 22), 7..15 G
// row by row (1/T).
template <bool MIXED, int DIM, bool KEEP_SUMS = false>
__global__ void SPH_PASSA_BOUNDS k_passA(RhsArgs A) {
  using R = typename std::conditional<MIXED, float, double>::type;
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A.n) return;
  constexpr int dim = DIM;
  const sph_params &P = A.prm;
  Own<MIXED> o;
  o.load(A, a);
  const R sig = kernel_sigma<R>(dim);
  const R ha = (R)o.h, rhoa = (R)o.rho;
  const bool xsph = P.xsph != 0.0;
  KahanT<R> drho;
  R L[3][3], G[3][3], xs[3] = {R(0), R(0), R(0)};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) L[i][j] = G[i][j] = R(0);
  const int32_t *list;
  const int cnt = partner_list(A, a, list);
#if SPH_PASS_PREFETCH
  PartnerCursor<MIXED, true> cur;
  cur.start(A, o, list, cnt);
#endif
  for (int k = 0; k < cnt; ++k) {
    R d[3], w[3], hb, rhob, mb, vol;
#if SPH_PASS_PREFETCH
    typename PartnerCursor<MIXED, true>::Raw raw;
    cur.next(A, o, k, raw);
    o.from(A, raw, d, w, hb, rhob, mb, vol);
#else
    const int32_t b = list[(int64_t)k * A.ld];
    o.pair(A, b, d, w, hb, rhob, mb, vol);
#endif
    const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const R rinv = rsqrt_or_zero(r2);
    const R r = r2 * rinv;
    const R hinv = pair_rcp(R(0.5) * (ha + hb));
    const R q = r * hinv;
    const R hD = hpow(hinv, dim);
    const R fr = kern_dW(q, R(6) * sig * hD * hinv) * rinv;
    R g[3] = {fr * d[0], fr * d[1], fr * d[2]};
    drho.add(vol * (w[0] * g[0] + w[1] * g[1] + w[2] * g[2]));
    // L is symmetric (grad W is parallel to d): its lower triangle only
    for (int i = 0; i < 3; ++i) {
      if (i >= dim) break;
      const R vd = vol * d[i], vw = vol * w[i];
      for (int j = 0; j < 3; ++j) {
        if (j >= dim) break;
        if (j <= i) L[i][j] -= vd * g[j];
        G[i][j] -= vw * g[j];
      }
    }
    if (xsph) {
      const R c = pair_div(R(2) * mb, rhoa + rhob) * kern_W(q, sig * hD);
      for (int i = 0; i < 3; ++i) xs[i] -= c * w[i];
    }
  }
  // ---- per-particle update ----
  const int mi0 = A.mat ? A.mat[a] : 0;
  const int mi = (mi0 >= 0 && mi0 < A.mt.nmat) ? mi0 : 0;
  const sph_material &M = A.mt.m[mi];
  const float *mf = MIXED ? A.U->matf[mi] : nullptr;
  const EosC<R> K = eos_consts<R>(M, mf, A.U);
  // SI <-> R-unit factors (1 in FP64 mode)
  const double f_sig = MIXED ? A.U->invsig : 1.0;
  const R mu_r = MIXED ? (R)mf[MF_MU] : (R)M.mu;
  const R Y0_r = MIXED ? (R)mf[MF_Y0] : (R)M.Y0;
  const R K0_r = MIXED ? (R)mf[MF_K0] : (R)M.K0;
  const double rho_d = A.rho[a];
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j) L[i][j] = L[j][i];
  R C[3][3];
  correction_tensor<R>(dim, L, P.consistency && cnt >= dim + 1, C);
  R gv[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      R s = R(0);
      for (int k = 0; k < dim; ++k) s += G[i][k] * C[k][j];
      gv[i][j] = (i < dim && j < dim) ? s : R(0);
    }
  R p, cs;
  eos_eval<R>(M, K, rho_d, A.u[a], p, cs);
  const int ns = nsym(dim);
  R S[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[i][j] = R(0);
  const bool strength = A.S != nullptr && M.strength;
  if (strength) {
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) {
        const double sv = A.S[(int64_t)symk(dim, i, j) * A.n + a];
        if constexpr (MIXED)
          S[i][j] = to_f32_scaled(sv, pow2_exp(f_sig), f_sig);
        else
          S[i][j] = sv;
      }
    // von Mises: f_Y = min(Y0^2 / (3 J2), 1)
    if (M.Y0 > 0.0) {
      R J2 = R(0);
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) J2 += S[i][j] * S[i][j];
      J2 *= R(0.5);
      if (J2 > R(0)) {
        R fY = Y0_r * Y0_r / (R(3) * J2);
        if (fY < R(1))
          for (int i = 0; i < dim; ++i)
            for (int j = 0; j < dim; ++j) S[i][j] *= fY;
      }
    }
    // Hooke + Jaumann: dS = 2 mu (eps_dot - tr/D I) + R S - S R
    R tr = R(0);
    for (int i = 0; i < dim; ++i) tr += gv[i][i];
    const R mu2 = R(2) * mu_r;
    for (int i = 0; i < dim; ++i)
      for (int j = i; j < dim; ++j) {
        R ed = R(0.5) * (gv[i][j] + gv[j][i]) - (i == j ? tr / R(dim) : R(0));
        R rot = R(0);
        for (int k = 0; k < dim; ++k) {
          R Rik = R(0.5) * (gv[i][k] - gv[k][i]);
          R Rkj = R(0.5) * (gv[k][j] - gv[j][k]);
          rot += Rik * S[k][j] - S[i][k] * Rkj;
        }
        if constexpr (MIXED) {
          const double us = A.U->sig * A.U->invT;
          A.dS[(int64_t)symk(dim, i, j) * A.n + a] = to_f64_scaled(mu2 * ed + rot, pow2_exp(us), us);
        } else {
          A.dS[(int64_t)symk(dim, i, j) * A.n + a] = mu2 * ed + rot;
        }
      }
  } else if (A.S != nullptr && A.dS != nullptr) {
    for (int k = 0; k < ns; ++k) A.dS[(int64_t)k * A.n + a] = 0.0;
  }
  // damage-reduced stress sigma_d = -p_hat I + (1 - d) S
  const bool damage = A.dmg != nullptr && M.damage;
  R dd = R(0);
  if (damage) {
    R del = (R)A.dmg[a];
    dd = del * del * del;
  }
  const R phat = p >= R(0) ? p : (R(1) - dd) * p;
  R sd[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) sd[i][j] = (R(1) - dd) * S[i][j];
  // principal frame of the deviatoric part (sigma_d shares its axes)
  R lam[3] = {R(0), R(0), R(0)}, Q[3][3];
  const bool need_eig = (damage || P.eps_s > 0.0);
  if (need_eig) {
    R E[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) E[i][j] = sd[i][j];
    sym_eigen<R>(dim, E, lam, Q);
    for (int i = 0; i < dim; ++i) lam[i] -= phat;
  }
  int nact = 0;
  R ddel = R(0);
  if (damage) {
    R smax = lam[0];
    for (int i = 1; i < dim; ++i) smax = lam[i] > smax ? lam[i] : smax;
    const R Em = R(9) * K0_r * mu_r / (R(3) * K0_r + mu_r);
    const R den = (R(1) - dd) * Em;
    const R eps = den > R(0) ? smax / den : R(0);
    const int64_t idp = A.id ? A.id[a] : a;
    const int64_t f0 = A.flaw_off[idp], f1 = A.flaw_off[idp + 1];
    const int64_t ntot = f1 - f0;
    if (eps > R(0) && ntot > 0) {
      int64_t lo = f0, hi = f1;  // count of thresholds strictly below eps
      while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((R)A.flaw_eps[mid] < eps) lo = mid + 1; else hi = mid;
      }
      nact = (int)(lo - f0);
    }
    if (nact > 0 && dd < (R)nact / (R)ntot) {
      R cg = R(0.4) * sqrt((K0_r + R(4) / R(3) * (R(1) - dd) * mu_r) / rhoa);
      ddel = (R)nact * cg / ha;
    }
  }
  // artificial stress in the principal frame
  R Z[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Z[i][j] = R(0);
  const R rr = rhoa * rhoa;
  if (P.eps_s > 0.0) {
    R zl[3];
    for (int k = 0; k < 3; ++k) zl[k] = (k < dim && lam[k] > R(0)) ? -(R)P.eps_s * lam[k] / rr : R(0);
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) {
        R s = R(0);
        for (int k = 0; k < dim; ++k) s += Q[i][k] * zl[k] * Q[j][k];
        Z[i][j] = s;
      }
  }
  // outputs
  const R irr = rcp_rn(rr);
  R T[6], Zc[6];
  for (int i = 0; i < dim; ++i)
    for (int j = i; j < dim; ++j) {
      int k = symk(dim, i, j);
      T[k] = (sd[i][j] - (i == j ? phat : R(0))) * irr;
      Zc[k] = Z[i][j];
    }
  if constexpr (MIXED) {
    float t[6] = {0, 0, 0, 0, 0, 0}, z[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < ns; ++k) {
      t[k] = T[k];
      z[k] = Zc[k];
    }
    A.Tf[a] = make_float4(t[0], t[1], t[2], t[3]);
    A.Tf[A.ld + a] = make_float4(t[4], t[5], cs, 0.f);
    if (P.eps_s > 0.0) {
      A.Zf[a] = make_float4(z[0], z[1], z[2], z[3]);
      A.Zf[A.ld + a] = make_float4(z[4], z[5], 0.f, 0.f);
    }
  } else {
    for (int k = 0; k < ns; ++k) {
      A.Td[(int64_t)k * A.ld + a] = T[k];
      if (P.eps_s > 0.0) A.Zd[(int64_t)k * A.ld + a] = Zc[k];
    }
    A.csd[a] = cs;
  }
  if constexpr (MIXED) {
    // back to SI by exponent shifts (the code units are powers of two); the
    // product rho_a * sum is formed exactly as a float pair
    const double u_drho = A.U->rho * A.U->invT, u_v = A.U->V, u_t = A.U->invT, u_sig = A.U->sig;
    const int k_drho = pow2_exp(u_drho), k_v = pow2_exp(u_v), k_t = pow2_exp(u_t), k_sig = pow2_exp(u_sig);
    if (A.drho) {
      const float sum = drho.value(), hi = rhoa * sum, lo = fmaf(rhoa, sum, -hi);
      A.drho[a] = P.density_sum ? 0.0 : to_f64_scaled(hi, k_drho, u_drho) + to_f64_scaled(lo, k_drho, u_drho);
    }
    for (int ax = 0; ax < dim; ++ax)
      if (A.dx[ax]) A.dx[ax][a] = A.v[ax][a] + P.xsph * to_f64_scaled(xs[ax], k_v, u_v);
    if (A.ddmg) A.ddmg[a] = to_f64_scaled(ddel, k_t, u_t);
    if (A.p_out) A.p_out[a] = to_f64_scaled(p, k_sig, u_sig);
    if (A.cs_out) A.cs_out[a] = to_f64_scaled(cs, k_v, u_v);
  } else {
    if (A.drho) A.drho[a] = P.density_sum ? 0.0 : rhoa * drho.value();
    for (int ax = 0; ax < dim; ++ax)
      if (A.dx[ax]) A.dx[ax][a] = A.v[ax][a] + P.xsph * xs[ax];
    if (A.ddmg) A.ddmg[a] = ddel;
    if (A.p_out) A.p_out[a] = p;
    if (A.cs_out) A.cs_out[a] = cs;
  }
  if (A.nact) A.nact[a] = nact;
  if (A.nnb) A.nnb[a] = cnt;
  if constexpr (MIXED && KEEP_SUMS) {
    float *o = A.sums;
    const int64_t ld = A.ld;
    o[a] = drho.value();
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j <= i; ++j) o[(int64_t)(1 + i * (i + 1) / 2 + j) * ld + a] = L[i][j];
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) o[(int64_t)(7 + 3 * i + j) * ld + a] = G[i][j];
  }
}

// ---------------------------------------------------------------------------
// Pass B: momentum and energy
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void sym_mv(int dim, const R t[6], const R g[3], R out[3]) {
  if (dim == 3) {
    out[0] = t[0] * g[0] + t[3] * g[1] + t[4] * g[2];
    out[1] = t[3] * g[0] + t[1] * g[1] + t[5] * g[2];
    out[2] = t[4] * g[0] + t[5] * g[1] + t[2] * g[2];
  } else {
    out[0] = t[0] * g[0] + t[2] * g[1];
    out[1] = t[2] * g[0] + t[1] * g[1];
    out[2] = R(0);
  }
}

template <bool MIXED>
__device__ __forceinline__ void load_T(const RhsArgs &A, int64_t b, int ns,
                                       typename std::conditional<MIXED, float, double>::type t[6],
                                       typename std::conditional<MIXED, float, double>::type &cs) {
  if constexpr (MIXED) {
    const float4 t0 = A.Tf[b], t1 = A.Tf[A.ld + b];
    t[0] = t0.x;
    t[1] = t0.y;
    t[2] = t0.z;
    t[3] = t0.w;
    t[4] = t1.x;
    t[5] = t1.y;
    cs = t1.z;
  } else {
    for (int k = 0; k < 6; ++k) t[k] = k < ns ? A.Td[(int64_t)k * A.ld + b] : 0.0;
    cs = A.csd[b];
  }
}

template <bool MIXED>
__device__ __forceinline__ void load_Z(const RhsArgs &A, int64_t b, int ns,
                                       typename std::conditional<MIXED, float, double>::type z[6]) {
  if constexpr (MIXED) {
    const float4 z0 = A.Zf[b], z1 = A.Zf[A.ld + b];
    z[0] = z0.x;
    z[1] = z0.y;
    z[2] = z0.z;
    z[3] = z0.w;
    z[4] = z1.x;
    z[5] = z1.y;
  } else {
    for (int k = 0; k < 6; ++k) z[k] = k < ns ? A.Zd[(int64_t)k * A.ld + b] : 0.0;
  }
}

template <class R>
__device__ __forceinline__ R ipow(R f, R n) {
  if (n == R(4)) {
    R f2 = f * f;
    return f2 * f2;
  }
  return pow(f, n);
}

template <bool MIXED, bool AS, int DIM>
__global__ void SPH_PASSB_BOUNDS k_passB(RhsArgs A) {
  using R = typename std::conditional<MIXED, float, double>::type;
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A.n) return;
  constexpr int dim = DIM;
  const int ns = nsym(dim);
  const sph_params &P = A.prm;
  Own<MIXED> o;
  o.load(A, a);
  const R sig = kernel_sigma<R>(dim);
  const R ha = (R)o.h, rhoa = (R)o.rho;
  R Ta[6], Za[6], csa;
  load_T<MIXED>(A, a, ns, Ta, csa);
  if (AS) load_Z<MIXED>(A, a, ns, Za);
  const R alpha = (R)P.alpha, beta = (R)P.beta, epsv = (R)P.eps_v, nas = (R)P.n_as;
  const R dmpd = (R)(P.dmpd * (MIXED ? A.U->invL : 1.0));
  KahanT<R> acc[3], du;
  const int32_t *list;
  const int cnt = partner_list(A, a, list);
#if SPH_PASS_PREFETCH
  PartnerCursor<MIXED> cur;
  cur.start(A, o, list, cnt);
#endif
  for (int k = 0; k < cnt; ++k) {
    R d[3], w[3], hb, rhob, mb, vol;
    R Tb[6], csb;
#if SPH_PASS_PREFETCH
    typename Own<MIXED>::Raw raw;
    const int32_t b = cur.next(A, o, k, raw);
    o.from(A, raw, d, w, hb, rhob, mb, vol);
    load_T<MIXED>(A, b, ns, Tb, csb);
#else
    const int32_t b = list[(int64_t)k * A.ld];
    o.pair(A, b, d, w, hb, rhob, mb, vol);
    load_T<MIXED>(A, b, ns, Tb, csb);
#endif
    const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const R rinv = rsqrt_or_zero(r2);
    const R r = r2 * rinv;
    const R hab = R(0.5) * (ha + hb);
    const R hinv = pair_rcp(hab);
    const R q = r * hinv;
    const R hD = hpow(hinv, dim);
    const R fr = kern_dW(q, R(6) * sig * hD * hinv) * rinv;
    const R g[3] = {fr * d[0], fr * d[1], fr * d[2]};
    // artificial viscosity for approaching pairs
    const R vx = w[0] * d[0] + w[1] * d[1] + w[2] * d[2];
    R Pi = R(0);
    if (vx < R(0)) {
      const R nu = pair_div(hab * vx, r2 + epsv * hab * hab);
      Pi = pair_div(-alpha * R(0.5) * (csa + csb) * nu + beta * nu * nu, R(0.5) * (rhoa + rhob));
    }
    R tsum[6];
    for (int c = 0; c < 6; ++c) tsum[c] = Ta[c] + Tb[c];
    R tg[3];
    sym_mv(dim, tsum, g, tg);
    R su[3] = {tg[0] - Pi * g[0], tg[1] - Pi * g[1], tg[2] - Pi * g[2]};
    R sv[3] = {su[0], su[1], su[2]};
    if (AS) {
      R Zb[6];
      load_Z<MIXED>(A, b, ns, Zb);
      const R fn = ipow(kern_W(q, R(1)) / kern_W(dmpd * hinv, R(1)), nas);
      R zs[6];
      for (int c = 0; c < 6; ++c) zs[c] = (Za[c] + Zb[c]) * fn;
      R zg[3];
      sym_mv(dim, zs, g, zg);
      for (int i = 0; i < 3; ++i) sv[i] += zg[i];
    }
    for (int i = 0; i < dim; ++i) acc[i].add(mb * sv[i]);
    du.add(R(-0.5) * mb * (w[0] * su[0] + w[1] * su[1] + w[2] * su[2]));
  }
  if constexpr (MIXED) {
    const double u_acc = A.U->acc, u_du = A.U->E * A.U->invT;
    const int k_acc = pow2_exp(u_acc), k_du = pow2_exp(u_du);
    for (int ax = 0; ax < dim; ++ax) {
      double v = to_f64_scaled(acc[ax].value(), k_acc, u_acc);
      if (A.ag) v += A.ag[(int64_t)ax * A.ld + a];
      A.dv[ax][a] = v;
    }
    if (A.du) A.du[a] = to_f64_scaled(du.value(), k_du, u_du);
  } else {
    for (int ax = 0; ax < dim; ++ax) {
      double v = acc[ax].value();
      if (A.ag) v += A.ag[(int64_t)ax * A.ld + a];
      A.dv[ax][a] = v;
    }
    if (A.du) A.du[a] = du.value();
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
__global__ void k_repack_rho(const double *__restrict__ rho, const double *__restrict__ m, PackedF32 pk, int64_t n,
                             const Units *__restrict__ U) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 v = pk.pv(i), w = pk.pvl(i);
  // as in the packing after the tree build: rho scaled by its power-of-two
  // unit, and the volume m / rho from the FP32 views
  const float rf = to_f32_scaled(rho[i], pow2_exp(U->invrho), U->invrho);
  v.w = rf;
  w.w = __fdiv_rn(pk.pxl(i).w, rf);
  pk.pv(i) = v;
  pk.pvl(i) = w;
}

void rhs_passes(sph_ctx *c, sph_state *s, const MatTable &mt, const sph_params &p, const sph_derivs &out,
                cudaStream_t st, float *sums) {
  const int64_t n = s->n;
  if (n == 0) return;
  RhsArgs A;
  memset(&A, 0, sizeof(A));
  A.dim = s->dim;
  A.n = n;
  A.ld = c->cap_n;
  for (int ax = 0; ax < 3; ++ax) {
    A.x[ax] = s->x[ax];
    A.v[ax] = s->v[ax];
    A.dx[ax] = out.dx[ax];
    A.dv[ax] = out.dv[ax];
  }
  A.rho = s->rho;
  A.u = s->u;
  A.m = s->m;
  A.h = s->h;
  A.S = s->S;
  A.dmg = s->dmg;
  A.mat = s->mat;
  A.id = s->id;
  A.flaw_off = s->flaw_off;
  A.flaw_eps = s->flaw_eps;
  A.nb_idx = c->nb_idx;
  A.nb_cnt = c->nb_cnt;
  A.nb_idx2 = c->nb_alt;
  A.nb_cnt2 = c->nb_cnt_alt;
  A.pk = c->pk;
  A.drho = out.drho;
  A.du = out.du;
  A.dS = out.dS;
  A.ddmg = out.ddmg;
  A.p_out = out.p;
  A.cs_out = out.cs;
  A.nact = out.n_act;
  A.nnb = out.nnb;
  A.Td = (double *)c->T;
  A.Zd = (double *)c->zeta;
  A.Tf = (float4 *)c->T;
  A.Zf = (float4 *)c->zeta;
  A.csd = c->cs;
  A.ag = p.gravity ? c->ag : nullptr;
  A.rho_out = s->rho;
  A.U = c->units;
  A.mt = mt;
  A.prm = p;
  A.err = c->d_err;
  const bool mixed = p.precision == SPH_MIXED;
  A.sums = mixed ? sums : nullptr;
  const int T = c->tune.pass_threads;
  int pr = -1;
  const bool d3 = s->dim == 3;
#define SPH_LAUNCH(kern, ...)                                                     \
  do {                                                                            \
    if (d3) kern<__VA_ARGS__, 3><<<nblk(n, T), T, 0, st>>>(A);                   \
    else kern<__VA_ARGS__, 2><<<nblk(n, T), T, 0, st>>>(A);                      \
    ++sph::g_launches;                                                            \
  } while (0)
  if (p.density_sum) {
    pr = prof_begin(c, st, PH_DENSITY);
    if (mixed) SPH_LAUNCH(k_density_sum, true);
    else SPH_LAUNCH(k_density_sum, false);
    { k_repack_rho<<<nblk(n, 256), 256, 0, st>>>(s->rho, s->m, c->pk, n, c->units); ++sph::g_launches; }
    prof_end(c, st, pr);
  }
  pr = prof_begin(c, st, PH_PASSA);
  if (mixed && A.sums) {
    if (d3) k_passA<true, 3, true><<<nblk(n, T), T, 0, st>>>(A);
    else k_passA<true, 2, true><<<nblk(n, T), T, 0, st>>>(A);
    ++sph::g_launches;
  } else if (mixed) {
    SPH_LAUNCH(k_passA, true);
  } else {
    SPH_LAUNCH(k_passA, false);
  }
  prof_end(c, st, pr);
  const bool as = p.eps_s > 0.0;
  pr = prof_begin(c, st, PH_PASSB);
  if (mixed) {
    if (as) SPH_LAUNCH(k_passB, true, true);
    else SPH_LAUNCH(k_passB, true, false);
  } else {
    if (as) SPH_LAUNCH(k_passB, false, true);
    else SPH_LAUNCH(k_passB, false, false);
  }
#undef SPH_LAUNCH
  prof_end(c, st, pr);
}

}  // namespace sph
