// Reverse-mode derivative (adjoint) of the right-hand side (Sect. 3.1) and of
// the predictor-corrector update (Sect. 3.4.1), in FP64, with the partner
// lists and the damage of the forward evaluation held fixed.
//
// Given cotangents of the right-hand side's outputs (dx/dt, dv/dt, drho/dt,
// du/dt, dS/dt) the kernels accumulate the cotangents of the state (x, v,
// rho, u, S) and of the material parameters (shear modulus mu, yield stress
// Y0, bulk modulus K: a common scale of K0, A_T and B_T).  Every pair term of
// particle a depends on both a and its partner b; because the lists are
// symmetric (b in N(a) iff a in N(b)) each particle gathers, over its own
// list, both the derivatives of its own terms and the derivatives of its
// partners' terms with respect to itself.  No atomics, deterministic order.
//
//   k_adj_passB   reverse of the momentum / energy pass -> x, v, T, c_s, rho
//   k_adj_update  pass-A sums recomputed, reverse of the constitutive update
//                 (T = sigma/rho^2, damage-reduced stress, Hooke + Jaumann,
//                 von Mises, EOS, grad v = G C with C = L^-1) -> S, u, rho,
//                 parameters, and the cotangents of the pass-A sums
//   k_adj_passA   reverse of the continuity / L / G / XSPH sums -> x, v, rho
//
// Not covered (argument error): artificial stress, density by kernel sum,
// gravity.  Branch switches (viscosity on/off, yield on/off, EOS branches,
// C = I fallback) are held at the forward evaluation's side.
#include "eos.cuh"
#include "sph_internal.cuh"

namespace sph {

struct AdjArgs {
  int dim;
  int64_t n, ld;
  const double *x[3], *v[3], *rho, *u, *m, *h, *S, *dmg;
  const int32_t *mat;
  const int32_t *nb_idx, *nb_cnt;
  const double *T, *cs;               // forward pass A (FP64, stride ld)
  const double *bdx[3], *bdv[3], *bdrho, *bdu, *bdS;  // output cotangents
  double *gx[3], *gv[3], *grho, *gu, *gS;             // accumulated state cotangents
  double *Tbar, *csbar;               // scratch: 6 * ld, ld
  double *inter;                      // scratch: 22 * ld (sum_rho_bar, Lbar 9, Gbar 9, xsph_bar 3)
  double *pbar;                       // scratch: 3 * ld (mu, Y0, K per particle)
  MatTable mt;
  sph_params prm;
  // mixed mode: FP32 views and code units of the forward evaluation
  PackedF32 pk;
  const float4 *Tf;                   // forward pass A: (T0..T3), (T4, T5, c_s, 0) in code units
  float4 *Bpk;                        // output cotangents of dv and du in code units (ld)
  float4 *Apk;                        // cotangents of the pass-A sums in code units (6 * ld)
  const Units *U;
  const float *sums;  // mixed: the forward pass A's pair sums (16 rows of stride ld)
};

__device__ __forceinline__ int sidx(int dim, int i, int j) { return symk(dim, i, j); }

// Partner list of particle c in the mixed pair kernels: the index read two
// pairs ahead and the partner's position views one pair ahead (as in the
// forward pass A), so that their loads are in flight during the pair before.
struct AdjCursor {
  const int32_t *col;
  int64_t ld;
  int cnt;
  int32_t e1, e2;
  float4 P1, Q1;
  __device__ __forceinline__ void start(const AdjArgs &A, int64_t c, int n) {
    col = A.nb_idx + c;
    ld = A.ld;
    cnt = n;
    e1 = n > 0 ? col[0] : 0;
    e2 = n > 1 ? col[ld] : 0;
    if (n > 0) {
      P1 = A.pk.px(e1);
      Q1 = A.pk.pxl(e1);
    }
  }
  __device__ __forceinline__ int32_t next(const AdjArgs &A, int k, float4 &P, float4 &Q) {
    const int32_t e = e1;
    P = P1;
    Q = Q1;
    e1 = e2;
    if (k + 2 < cnt) e2 = col[(int64_t)(k + 2) * ld];
    if (k + 1 < cnt) {
      P1 = A.pk.px(e1);
      Q1 = A.pk.pxl(e1);
    }
    return e;
  }
};

// Kernel radial factors for a pair: phi = dW/dr / r and phi'(r)/r, W, dW/dr.
template <class R>
struct KPair {
  R phi, dphi_r, W, dWdr;
};
using KernelPair = KPair<double>;

template <class R>
__device__ __forceinline__ KPair<R> kernel_pair(int dim, R r, R hab) {
  const R sig = kernel_sigma<R>(dim);
  const R hinv = R(1.0) / hab;
  const R hD = hpow(hinv, dim);
  const R gnorm = R(6.0) * sig * hD * hinv;
  const R q = r * hinv;
  R s = R(0.0), sp = R(0.0), w = R(0.0);
  if (q < R(0.5)) {
    s = R(3.0) * q * q - R(2.0) * q;
    sp = R(6.0) * q - R(2.0);
    w = R(6.0) * q * q * q - R(6.0) * q * q + R(1.0);
  } else if (q <= R(1.0)) {
    const R t = R(1.0) - q;
    s = -t * t;
    sp = R(2.0) * t;
    w = R(2.0) * t * t * t;
  }
  KPair<R> k;
  k.dWdr = gnorm * s;
  k.W = sig * hD * w;
  const R d2W = gnorm * sp * hinv;
  if (r > R(0.0)) {
    const R ir = R(1.0) / r;
    k.phi = k.dWdr * ir;
    k.dphi_r = (d2W - k.phi) * ir * ir;
  } else {
    k.phi = -R(2.0) * gnorm * hinv;  // limit of dW/dr / r at r = 0
    k.dphi_r = R(0.0);
  }
  return k;
}

// ---------------------------------------------------------------------------
// Reverse of one momentum/energy pair term of particle a with partner b:
//   dv_a += m_b B g,  du_a += -1/2 m_b w.(B g),  B = T_a + T_b - Pi I,  g = phi d
// Given the cotangents vb (of dv_a) and ub (of du_a), returns the cotangents
// of d = x_a - x_b, w = v_a - v_b, of B (symmetrised; it goes to T_a and T_b),
// and half the cotangents of the pair's mean sound speed and density.
// ---------------------------------------------------------------------------
// Artificial viscosity of a pair and its partial derivatives; symmetric in
// the two particles (v.r, the mean sound speed and density do not change when
// they swap), so computed once for both terms of the pair.
template <class R>
struct VPair {
  R vx, Pi, dPi_dnu, dnu_dvx, dnu_dr2, dPi_dc, dPi_drb;
};
using ViscPair = VPair<double>;

template <class R>
__device__ __forceinline__ VPair<R> visc_pair(int dim, const R d[3], const R w[3], R r2, R hab,
                                              R rho_a, R rho_b, R cs_a, R cs_b,
                                              const sph_params &P) {
  VPair<R> V;
  V.vx = R(0.0);
  for (int i = 0; i < dim; ++i) V.vx += w[i] * d[i];
  V.Pi = V.dPi_dnu = V.dnu_dvx = V.dnu_dr2 = V.dPi_dc = V.dPi_drb = R(0.0);
  if (V.vx < R(0.0)) {
    const R iQ = R(1.0) / (r2 + R(P.eps_v) * hab * hab);
    const R nu = hab * V.vx * iQ;
    const R cb = R(0.5) * (cs_a + cs_b), irb = R(1.0) / (R(0.5) * (rho_a + rho_b));
    V.Pi = (-R(P.alpha) * cb * nu + R(P.beta) * nu * nu) * irb;
    V.dPi_dnu = (-R(P.alpha) * cb + R(2.0) * R(P.beta) * nu) * irb;
    V.dnu_dvx = hab * iQ;
    V.dnu_dr2 = -nu * iQ;
    V.dPi_dc = -R(P.alpha) * nu * irb;
    V.dPi_drb = -V.Pi * irb;
  }
  return V;
}

// K: the kernel factors of the pair (the same for both of its terms); Vs: its
// artificial viscosity (the same for both terms: v.r is unchanged when d and
// w change sign together).
template <class R>
__device__ void pairB_adj(int dim, const R d[3], const R w[3], const KPair<R> &K, const VPair<R> &Vs,
                          const R Ta[6], const R Tb[6], R mb, const R vb[3], R ub,
                          R dbar[3], R wbar[3], R Bsym[6], R &cs_half, R &rho_half) {
  const int ns = nsym(dim);
  R g[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i) g[i] = K.phi * d[i];
  const R vx = Vs.vx, Pi = Vs.Pi, dPi_dnu = Vs.dPi_dnu, dnu_dvx = Vs.dnu_dvx, dnu_dr2 = Vs.dnu_dr2,
               dPi_dc = Vs.dPi_dc, dPi_drb = Vs.dPi_drb;
  R B[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      if (i < dim && j < dim) {
        const int k = sidx(dim, i, j);
        B[i][j] = Ta[k] + Tb[k] - (i == j ? Pi : R(0.0));
      } else {
        B[i][j] = R(0.0);
      }
    }
  R Bg[3] = {0, 0, 0}, Bw[3] = {0, 0, 0}, Bv[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j) {
      Bg[i] += B[i][j] * g[j];
      Bw[i] += B[i][j] * w[j];
      Bv[i] += B[i][j] * vb[j];
    }
  // cotangents of B (general matrix), g and w
  R Bbar[3][3];
  R trB = R(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Bbar[i][j] = (i < dim && j < dim) ? mb * vb[i] * g[j] - R(0.5) * mb * ub * w[i] * g[j] : R(0.0);
      if (i == j) trB += Bbar[i][j];
    }
  R gbar[3] = {0, 0, 0};
  for (int i = 0; i < 3; ++i) {
    gbar[i] = mb * Bv[i] - R(0.5) * mb * ub * Bw[i];
    wbar[i] = -R(0.5) * mb * ub * Bg[i];
    dbar[i] = R(0.0);
  }
  for (int i = 0; i < dim; ++i)
    for (int j = i; j < dim; ++j) Bsym[sidx(dim, i, j)] = R(0.5) * (Bbar[i][j] + Bbar[j][i]);
  for (int k = ns; k < 6; ++k) Bsym[k] = R(0.0);
  cs_half = R(0.0);
  rho_half = R(0.0);
  if (vx < R(0.0)) {
    const R Pibar = -trB;
    const R nubar = Pibar * dPi_dnu;
    const R vxbar = nubar * dnu_dvx;
    const R r2bar = nubar * dnu_dr2;
    cs_half = R(0.5) * Pibar * dPi_dc;
    rho_half = R(0.5) * Pibar * dPi_drb;
    for (int i = 0; i < dim; ++i) {
      wbar[i] += vxbar * d[i];
      dbar[i] += vxbar * w[i] + R(2.0) * r2bar * d[i];
    }
  }
  R gd = R(0.0);
  for (int i = 0; i < dim; ++i) gd += gbar[i] * d[i];
  for (int i = 0; i < dim; ++i) dbar[i] += K.phi * gbar[i] + K.dphi_r * gd * d[i];
}

__device__ __forceinline__ void load_T64(const AdjArgs &A, int64_t a, double t[6]) {
  const int ns = nsym(A.dim);
  for (int k = 0; k < 6; ++k) t[k] = k < ns ? A.T[(int64_t)k * A.ld + a] : 0.0;
}

// The kernels are instantiated per dimension, so that every small-matrix loop
// has a compile-time bound and the matrices stay in registers.
template <int DIM>
__global__ void k_adj_passB(AdjArgs A) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.n) return;
  constexpr int dim = DIM;
  const int ns = nsym(dim);
  double xc[3] = {0, 0, 0}, vc[3] = {0, 0, 0}, vbc[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i) {
    xc[i] = A.x[i][c];
    vc[i] = A.v[i][c];
    vbc[i] = A.bdv[i] ? A.bdv[i][c] : 0.0;
  }
  const double ubc = A.bdu ? A.bdu[c] : 0.0;
  double Tc[6];
  load_T64(A, c, Tc);
  const double hc = A.h[c], rc = A.rho[c], csc = A.cs[c], mc = A.m[c];
  double gx[3] = {0, 0, 0}, gv[3] = {0, 0, 0}, Tb_acc[6] = {0, 0, 0, 0, 0, 0};
  double csbar = 0.0, rhobar = 0.0;
  const int cnt = A.nb_cnt[c];
  for (int k = 0; k < cnt; ++k) {
    const int32_t e = A.nb_idx[(int64_t)k * A.ld + c];
    double d[3] = {0, 0, 0}, w[3] = {0, 0, 0}, vbe[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) {
      d[i] = xc[i] - A.x[i][e];
      w[i] = vc[i] - A.v[i][e];
      vbe[i] = A.bdv[i] ? A.bdv[i][e] : 0.0;
    }
    const double ube = A.bdu ? A.bdu[e] : 0.0;
    double Te[6];
    load_T64(A, e, Te);
    const double he = A.h[e], re = A.rho[e], cse = A.cs[e], me = A.m[e];
    const double hab = 0.5 * (hc + he);
    double r2 = 0.0;
    for (int i = 0; i < dim; ++i) r2 += d[i] * d[i];
    const KernelPair K = kernel_pair(dim, sqrt(r2), hab);
    const ViscPair Vs = visc_pair(dim, d, w, r2, hab, rc, re, csc, cse, A.prm);
    double db[3], wb[3], Bs[6], csh, rh;
    // c's own term with partner e
    pairB_adj(dim, d, w, K, Vs, Tc, Te, me, vbc, ubc, db, wb, Bs, csh, rh);
    for (int i = 0; i < dim; ++i) {
      gx[i] += db[i];
      gv[i] += wb[i];
    }
    for (int q = 0; q < ns; ++q) Tb_acc[q] += Bs[q];
    csbar += csh;
    rhobar += rh;
    // e's term with partner c, differentiated with respect to c
    double dn[3] = {-d[0], -d[1], -d[2]}, wn[3] = {-w[0], -w[1], -w[2]};
    pairB_adj(dim, dn, wn, K, Vs, Te, Tc, mc, vbe, ube, db, wb, Bs, csh, rh);
    for (int i = 0; i < dim; ++i) {
      gx[i] -= db[i];
      gv[i] -= wb[i];
    }
    for (int q = 0; q < ns; ++q) Tb_acc[q] += Bs[q];
    csbar += csh;
    rhobar += rh;
  }
  for (int i = 0; i < dim; ++i) {
    A.gx[i][c] += gx[i];
    A.gv[i][c] += gv[i];
  }
  A.grho[c] += rhobar;
  for (int q = 0; q < 6; ++q) A.Tbar[(int64_t)q * A.ld + c] = q < ns ? Tb_acc[q] : 0.0;
  A.csbar[c] = csbar;
}

// ---------------------------------------------------------------------------
// Constitutive update, recomputed and reversed
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ bool invert_L(int dim, const R L[3][3], R C[3][3]) {
  R det;
  if (dim == 2) det = L[0][0] * L[1][1] - L[0][1] * L[1][0];
  else
    det = L[0][0] * (L[1][1] * L[2][2] - L[1][2] * L[2][1]) - L[0][1] * (L[1][0] * L[2][2] - L[1][2] * L[2][0]) +
          L[0][2] * (L[1][0] * L[2][1] - L[1][1] * L[2][0]);
  R diag = R(1);
  for (int i = 0; i < dim; ++i) diag *= fabs(L[i][i]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i][j] = i == j ? R(1) : R(0);
  if (!(fabs(det) > R(1e-8) * diag) || !(diag > R(0))) return false;
  const R inv = R(1) / det;
  if (dim == 2) {
    C[0][0] = L[1][1] * inv;
    C[0][1] = -L[0][1] * inv;
    C[1][0] = -L[1][0] * inv;
    C[1][1] = L[0][0] * inv;
    return true;
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
  return true;
}

// p and c_s of a material whose bulk-modulus constants are scaled by s.
__device__ void eos_scaled(const sph_material &M0, double s, double rho, double u, double &p, double &cs, double *pr,
                           double *pu) {
  sph_material M = M0;
  M.K0 *= s;
  M.A_T *= s;
  M.B_T *= s;
  const EosC<double> K = eos_consts<double>(M, nullptr, nullptr);
  eos_eval<double>(M, K, rho, u, p, cs, pr, pu);
}

// MIXED: the pass-A sums are the forward pass A's own (FP32, code units, kept
// by it for this kernel), the equation of state is differentiated in FP32
// dual numbers, and the rest of the reverse runs in FP32 in SI units.  The
// reverse is linear in the cotangents it is given (of T, c_s and dS/dt), so
// each particle's are scaled by a power of two to order one first and its
// results scaled back exactly: FP32's exponent range then limits only the
// state, whose SI values it holds.  FP64: the sums are recomputed here, and
// the reverse is FP64 throughout (F = double, no scaling).
template <bool MIXED, int DIM>
__global__ void k_adj_update(AdjArgs A) {
  using F = typename std::conditional<MIXED, float, double>::type;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.n) return;
  constexpr int dim = DIM;
  const int ns = nsym(dim);
  const sph_params &P = A.prm;
  const int64_t ld = A.ld;
  // ---- pass-A sums ----
  const double rc = A.rho[c];
  double srho = 0.0;
  F L[3][3], G[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) L[i][j] = G[i][j] = F(0);
  const int cnt = A.nb_cnt[c];
  if constexpr (MIXED) {
    // k_passA's KEEP_SUMS layout; the continuity sum and G are rates (code
    // unit 1/T, a power of two: the conversion is exact), L is a number
    const float *sm = A.sums;
    const float it = (float)A.U->invT;
    srho = (double)sm[c] * A.U->invT;
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j <= i; ++j) L[i][j] = L[j][i] = sm[(int64_t)(1 + i * (i + 1) / 2 + j) * ld + c];
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) G[i][j] = sm[(int64_t)(7 + 3 * i + j) * ld + c] * it;
  } else {
    double xc[3] = {0, 0, 0}, vc[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) {
      xc[i] = A.x[i][c];
      vc[i] = A.v[i][c];
    }
    const double hc = A.h[c];
    for (int k = 0; k < cnt; ++k) {
      const int32_t e = A.nb_idx[(int64_t)k * A.ld + c];
      double d[3] = {0, 0, 0}, w[3] = {0, 0, 0}, r2 = 0.0;
      for (int i = 0; i < dim; ++i) {
        d[i] = xc[i] - A.x[i][e];
        w[i] = vc[i] - A.v[i][e];
        r2 += d[i] * d[i];
      }
      const KernelPair K = kernel_pair(dim, sqrt(r2), 0.5 * (hc + A.h[e]));
      const double vol = A.m[e] / A.rho[e];
      double wg = 0.0;
      for (int i = 0; i < dim; ++i) wg += w[i] * K.phi * d[i];
      srho += vol * wg;
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
          L[i][j] -= vol * d[i] * K.phi * d[j];
          G[i][j] -= vol * w[i] * K.phi * d[j];
        }
    }
  }
  F C[3][3];
  const bool corr = P.consistency && cnt >= dim + 1 && invert_L<F>(dim, L, C);
  if (!corr)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) C[i][j] = i == j ? F(1) : F(0);
  F gv[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      F s = F(0);
      for (int k = 0; k < dim; ++k) s += G[i][k] * C[k][j];
      gv[i][j] = (i < dim && j < dim) ? s : F(0);
    }
  // ---- constitutive state ----
  const int mi0 = A.mat ? A.mat[c] : 0;
  const int mi = (mi0 >= 0 && mi0 < A.mt.nmat) ? mi0 : 0;
  const sph_material &M = A.mt.m[mi];
  const double uc = A.u[c];
  const F mu = (F)M.mu, Y0 = (F)M.Y0;
  F p, pr, pu;
  // MIXED: one evaluation in FP32 dual numbers, in the forward's code units,
  // gives p, dp/drho, dp/du and the exact derivatives of c_s in rho and u and
  // of p and c_s in the bulk-modulus scale (code units to SI by powers of
  // two); FP64: the analytic derivatives of p here, those of c_s and the
  // scale by central differences below.
  F dcr = F(0), dcu = F(0), dps = F(0), dcs = F(0);
  if constexpr (MIXED) {
    const Units *U = A.U;
    const EosC<ad::Dual3> K = eos_consts<ad::Dual3>(M, U->matf[mi], U);
    ad::Dual3 p3, c3, pr3, pu3;
    eos_eval<ad::Dual3>(M, K, rc, uc, p3, c3, &pr3, &pu3);
    p = p3.v * (float)U->sig;
    pr = pr3.v * (float)(U->sig * U->invrho);
    pu = pu3.v * (float)(U->sig * U->invE);
    dcr = c3.d[0] * (float)(U->V * U->invrho);
    dcu = c3.d[1] * (float)(U->V * U->invE);
    dps = p3.d[2] * (float)U->sig;
    dcs = c3.d[2] * (float)U->V;
  } else {
    double cs;
    eos_scaled(M, 1.0, rc, uc, p, cs, &pr, &pu);
  }
  const bool strength = A.S != nullptr && M.strength;
  F S[3][3], St[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      S[i][j] = (strength && i < dim && j < dim) ? (F)A.S[(int64_t)sidx(dim, i, j) * A.n + c] : F(0);
  F J2 = F(0);
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j) J2 += S[i][j] * S[i][j];
  J2 *= F(0.5);
  F fY = F(1);
  if (strength && M.Y0 > 0.0 && J2 > F(0)) {
    const F q = Y0 * Y0 / (F(3) * J2);
    fY = q < F(1) ? q : F(1);
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) St[i][j] = fY * S[i][j];
  const bool damage = A.dmg != nullptr && M.damage;
  F dd = F(0);
  if (damage) {
    const F del = (F)A.dmg[c];
    dd = del * del * del;
  }
  // ---- the cotangents (of T, c_s, dS/dt), scaled (MIXED) ----
  double sc = 1.0, isc = 1.0;
  if constexpr (MIXED) {
    double mx = fabs(A.csbar[c]);
    for (int k = 0; k < ns; ++k) mx = fmax(mx, fabs(A.Tbar[(int64_t)k * ld + c]));
    if (A.bdS && strength)
      for (int k = 0; k < ns; ++k) mx = fmax(mx, fabs(A.bdS[(int64_t)k * A.n + c]));
    if (mx > 0.0 && mx < INFINITY) {
      int e;
      frexp(mx, &e);
      sc = ldexp(1.0, -e);
      isc = ldexp(1.0, e);
    }
  }
  // ---- reverse: T = sigma / rho^2 ----
  F Tb[3][3], Tc[6];
  {
    double t64[6];
    load_T64(A, c, t64);
    for (int k = 0; k < 6; ++k) Tc[k] = (F)t64[k];
  }
  F TbT = F(0), trSig = F(0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Tb[i][j] = (i < dim && j < dim) ? (F)(A.Tbar[(int64_t)sidx(dim, i, j) * A.ld + c] * sc) : F(0);
      if (i < dim && j < dim) TbT += Tb[i][j] * Tc[sidx(dim, i, j)];
    }
  const F rcf = (F)rc;
  F rhobar = F(-2) * TbT / rcf;
  const F irc2 = F(1) / (rcf * rcf);  // one division for the nine components below
  F sigbar[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) sigbar[i][j] = Tb[i][j] * irc2;
  for (int i = 0; i < dim; ++i) trSig += sigbar[i][i];
  // sigma = -p_hat I + (1 - d) S_tilde
  const F phatbar = -trSig;
  const F pbar = p >= F(0) ? phatbar : (F(1) - dd) * phatbar;
  F Stbar[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Stbar[i][j] = (F(1) - dd) * sigbar[i][j];
  // ---- reverse: dS = 2 mu (eps_dot - tr/D I) + R S_t - S_t R ----
  F Sdb[3][3];  // full-matrix cotangent of dS (symmetric)
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const F cst = (A.bdS && strength && i < dim && j < dim) ? (F)(A.bdS[(int64_t)sidx(dim, i, j) * A.n + c] * sc)
                                                               : F(0);
      Sdb[i][j] = (i == j) ? cst : F(0.5) * cst;
    }
  F ed[3][3], Rr[3][3], tr = F(0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      ed[i][j] = F(0.5) * (gv[i][j] + gv[j][i]);
      Rr[i][j] = F(0.5) * (gv[i][j] - gv[j][i]);
    }
  for (int i = 0; i < dim; ++i) tr += ed[i][i];
  F mubar = F(0), trSdb = F(0);
  for (int i = 0; i < dim; ++i) trSdb += Sdb[i][i];
  const F tr_d = tr / F(dim), trSdb_d = trSdb / F(dim);
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j) mubar += F(2) * (ed[i][j] - (i == j ? tr_d : F(0))) * Sdb[i][j];
  F edbar[3][3], Rbar[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      edbar[i][j] = (i < dim && j < dim) ? F(2) * mu * (Sdb[i][j] - (i == j ? trSdb_d : F(0))) : F(0);
      F a1 = F(0), a2 = F(0), b1 = F(0), b2 = F(0);
      for (int k = 0; k < dim; ++k) {
        a1 += Sdb[i][k] * St[k][j];  // Z S_t
        a2 += St[i][k] * Sdb[k][j];  // S_t Z
        b1 += Rr[i][k] * Sdb[k][j];  // R Z
        b2 += Sdb[i][k] * Rr[k][j];  // Z R
      }
      Rbar[i][j] = (i < dim && j < dim) ? a1 - a2 : F(0);
      if (i < dim && j < dim) Stbar[i][j] += -b1 + b2;
    }
  if (!strength)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) edbar[i][j] = Rbar[i][j] = F(0);
  F gvbar[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      gvbar[i][j] = F(0.5) * (edbar[i][j] + edbar[j][i]) + F(0.5) * (Rbar[i][j] - Rbar[j][i]);
  // ---- reverse: S_t = f_Y S (stored components) ----
  F Y0bar = F(0);
  if (strength && A.gS) {
    F Stb_st[6], S_st[6];
    for (int i = 0; i < dim; ++i)
      for (int j = i; j < dim; ++j) {
        const int k = sidx(dim, i, j);
        Stb_st[k] = (i == j) ? Stbar[i][i] : Stbar[i][j] + Stbar[j][i];
        S_st[k] = S[i][j];
      }
    F proj = F(0);
    for (int k = 0; k < ns; ++k) proj += Stb_st[k] * S_st[k];
    const bool yielding = M.Y0 > 0.0 && J2 > F(0) && Y0 * Y0 / (F(3) * J2) < F(1);
    const F fjp = yielding ? fY / J2 * proj : F(0);
    for (int k = 0; k < ns; ++k) {
      F sb = Stb_st[k];
      if (yielding) {
        const F wk = k < dim ? F(1) : F(2);
        sb = fY * Stb_st[k] - fjp * wk * S_st[k];
      }
      A.gS[(int64_t)k * A.n + c] += (double)sb * isc;
    }
    if (yielding) Y0bar = proj * F(2) * fY / Y0;
  }
  // ---- reverse: EOS ----
  const F csbar = (F)(A.csbar[c] * sc);
  F ubar = pbar * pu;
  rhobar += pbar * pr;
  F Kbar = F(0);
  if constexpr (MIXED) {
    const float Kref = (float)fmax(fmax(M.K0, M.A_T), M.B_T);
    rhobar += csbar * dcr;
    ubar += csbar * dcu;
    if (Kref > 0.f) Kbar = (pbar * dps + csbar * dcs) / Kref;
  } else {
    const double er = 1e-6 * rc, eu = 1e-6 * (fabs(uc) + 1e-3 * fabs(M.E0) + 1e-30), es = 1e-6;
    const double Kref = fmax(fmax(M.K0, M.A_T), M.B_T);
    // the six evaluations of the central differences (rho +-, u +-, scale +-)
    // in one loop, so that the equation of state is emitted once here: six
    // inlined copies overflowed the instruction cache.  c+ + (-c-) from zero is
    // the same value as c+ - c-.
#pragma unroll 1
    for (int k = 0; k < 6; ++k) {
      if (k < 4 ? csbar == 0.0 : !(Kref > 0.0)) continue;
      const double sg = (k & 1) ? -1.0 : 1.0;
      const double r1 = k == 0 ? rc + er : (k == 1 ? rc - er : rc);
      const double u1 = k == 2 ? uc + eu : (k == 3 ? uc - eu : uc);
      const double s1 = k == 4 ? 1.0 + es : (k == 5 ? 1.0 - es : 1.0);
      double p1, c1;
      eos_scaled(M, s1, r1, u1, p1, c1, nullptr, nullptr);
      if (k < 2) {
        dcr += sg * c1;
      } else if (k < 4) {
        dcu += sg * c1;
      } else {
        dps += sg * p1;
        dcs += sg * c1;
      }
    }
    if (csbar != 0.0) {
      rhobar += csbar * dcr / (2.0 * er);
      ubar += csbar * dcu / (2.0 * eu);
    }
    if (Kref > 0.0) Kbar = (pbar * dps + csbar * dcs) / (2.0 * es * Kref);
  }
  // ---- reverse: grad v = G C, C = L^-1 ----
  F Gbar[3][3], Lbar[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      F s = F(0);
      for (int k = 0; k < dim; ++k) s += gvbar[i][k] * C[j][k];  // gvbar C^T
      Gbar[i][j] = (i < dim && j < dim) ? s : F(0);
      Lbar[i][j] = F(0);
    }
  if (corr) {
    F Cbar[3][3], T1[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        F s = F(0);
        for (int k = 0; k < dim; ++k) s += G[k][i] * gvbar[k][j];  // G^T gvbar
        Cbar[i][j] = s;
      }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        F s = F(0);
        for (int k = 0; k < dim; ++k) s += Cbar[i][k] * C[j][k];  // Cbar C^T
        T1[i][j] = s;
      }
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) {
        F s = F(0);
        for (int k = 0; k < dim; ++k) s += C[k][i] * T1[k][j];  // C^T (Cbar C^T)
        Lbar[i][j] = -s;
      }
  }
  // ---- reverse: drho = rho * sum_rho ; dx = v + xsph * xs (FP64, unscaled) ----
  const double bdr = A.bdrho ? A.bdrho[c] : 0.0;
  A.grho[c] += (double)rhobar * isc + bdr * srho;
  A.gu[c] += (double)ubar * isc;
  for (int i = 0; i < dim; ++i)
    if (A.bdx[i]) A.gv[i][c] += A.bdx[i][c];
  double *I = A.inter;
  I[c] = rc * bdr;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      I[(1 + 3 * i + j) * ld + c] = (double)Lbar[i][j] * isc;
      I[(10 + 3 * i + j) * ld + c] = (double)Gbar[i][j] * isc;
    }
  for (int i = 0; i < 3; ++i) I[(19 + i) * ld + c] = (i < dim && A.bdx[i]) ? P.xsph * A.bdx[i][c] : 0.0;
  A.pbar[c] = strength ? (double)mubar * isc : 0.0;
  A.pbar[ld + c] = (double)Y0bar * isc;
  A.pbar[2 * ld + c] = (double)Kbar * isc;
}

// ---------------------------------------------------------------------------
// Reverse of one pass-A pair term of particle a with partner b:
//   sum_rho += vol_b w.g,  L -= vol_b d (x) g,  G -= vol_b w (x) g,
//   xs -= 2 m_b/(rho_a + rho_b) W w,   vol_b = m_b / rho_b
// ---------------------------------------------------------------------------
// Cotangents of the pass-A sums of one particle: continuity sum, L, G, XSPH.
template <class R>
struct ACot {
  R sr, Lb[3][3], Gb[3][3], xb[3];
};

__device__ __forceinline__ ACot<double> load_acot64(const double *I, int64_t ld, int64_t a) {
  ACot<double> c;
  c.sr = I[a];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      c.Lb[i][j] = I[(1 + 3 * i + j) * ld + a];
      c.Gb[i][j] = I[(10 + 3 * i + j) * ld + a];
    }
    c.xb[i] = I[(19 + i) * ld + a];
  }
  return c;
}

// K: the kernel factors of the pair, r = |d|; Ct: the cotangents of the sums
// of the particle whose term this is.
template <class R>
__device__ void pairA_adj(int dim, const R d[3], const R w[3], R r, const KPair<R> &K, R mb, R rho_a, R rho_b,
                          const ACot<R> &Ct, R dbar[3], R wbar[3], R &rho_a_bar, R &rho_b_bar) {
  const R vol = mb / rho_b;
  R g[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i) g[i] = K.phi * d[i];
  const R sr = Ct.sr;
  R gbar[3] = {0, 0, 0}, wg = R(0);
  for (int i = 0; i < 3; ++i) {
    dbar[i] = R(0);
    wbar[i] = R(0);
  }
  for (int i = 0; i < dim; ++i) wg += w[i] * g[i];
  R volbar = sr * wg;
  for (int i = 0; i < dim; ++i) {
    gbar[i] += sr * vol * w[i];
    wbar[i] += sr * vol * g[i];
  }
  // L and G
  for (int i = 0; i < dim; ++i) {
    R Lg = R(0), Gg = R(0), LTd = R(0), GTw = R(0);
    for (int j = 0; j < dim; ++j) {
      Lg += Ct.Lb[i][j] * g[j];
      Gg += Ct.Gb[i][j] * g[j];
      LTd += Ct.Lb[j][i] * d[j];
      GTw += Ct.Gb[j][i] * w[j];
    }
    dbar[i] += -vol * Lg;
    wbar[i] += -vol * Gg;
    gbar[i] += -vol * (LTd + GTw);
    volbar += -d[i] * Lg - w[i] * Gg;
  }
  // XSPH
  rho_a_bar = R(0);
  rho_b_bar = R(0);
  R wx = R(0);
  for (int i = 0; i < dim; ++i) wx += w[i] * Ct.xb[i];
  if (wx != R(0)) {
    const R cc = R(2) * mb / (rho_a + rho_b);
    for (int i = 0; i < dim; ++i) wbar[i] += -cc * K.W * Ct.xb[i];
    const R Wbar = -cc * wx;
    const R ccbar = -K.W * wx;
    const R dcc = -cc / (rho_a + rho_b);
    rho_a_bar += ccbar * dcc;
    rho_b_bar += ccbar * dcc;
    if (r > R(0))
      for (int i = 0; i < dim; ++i) dbar[i] += Wbar * K.phi * d[i];  // dW/dr d / r
  }
  R gd = R(0);
  for (int i = 0; i < dim; ++i) gd += gbar[i] * d[i];
  for (int i = 0; i < dim; ++i) dbar[i] += K.phi * gbar[i] + K.dphi_r * gd * d[i];
  rho_b_bar += -volbar * vol / rho_b;
}

template <int DIM>
__global__ void k_adj_passA(AdjArgs A) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.n) return;
  constexpr int dim = DIM;
  double xc[3] = {0, 0, 0}, vc[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i) {
    xc[i] = A.x[i][c];
    vc[i] = A.v[i][c];
  }
  const double hc = A.h[c], rc = A.rho[c], mc = A.m[c];
  const ACot<double> Cc = load_acot64(A.inter, A.ld, c);
  double gx[3] = {0, 0, 0}, gv[3] = {0, 0, 0}, grho = 0.0;
  const int cnt = A.nb_cnt[c];
  for (int k = 0; k < cnt; ++k) {
    const int32_t e = A.nb_idx[(int64_t)k * A.ld + c];
    double d[3] = {0, 0, 0}, w[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) {
      d[i] = xc[i] - A.x[i][e];
      w[i] = vc[i] - A.v[i][e];
    }
    const double he = A.h[e], re = A.rho[e], me = A.m[e];
    const double hab = 0.5 * (hc + he);
    double r2 = 0.0;
    for (int i = 0; i < dim; ++i) r2 += d[i] * d[i];
    const double r = sqrt(r2);
    const KernelPair K = kernel_pair(dim, r, hab);
    double db[3], wb[3], ra, rb;
    pairA_adj(dim, d, w, r, K, me, rc, re, Cc, db, wb, ra, rb);  // c's own term
    for (int i = 0; i < dim; ++i) {
      gx[i] += db[i];
      gv[i] += wb[i];
    }
    grho += ra;
    double dn[3] = {-d[0], -d[1], -d[2]}, wn[3] = {-w[0], -w[1], -w[2]};
    const ACot<double> Ce = load_acot64(A.inter, A.ld, e);
    pairA_adj(dim, dn, wn, r, K, mc, re, rc, Ce, db, wb, ra, rb);  // e's term, w.r.t. c
    for (int i = 0; i < dim; ++i) {
      gx[i] -= db[i];
      gv[i] -= wb[i];
    }
    grho += rb;
  }
  for (int i = 0; i < dim; ++i) {
    A.gx[i][c] += gx[i];
    A.gv[i][c] += gv[i];
  }
  A.grho[c] += grho;
}

// Per-instance, per-material sums of the particle parameter cotangents,
// param_bar[(inst * nmat + mat) * 3 + k], in a fixed order.  Block (inst, j)
// sums the j-th of gy equal chunks of its instance (a strided loop, then a
// tree in shared memory); with part set it stores that partial sum, and
// k_adj_params_final adds the gy partials of each entry in chunk order.  With
// part NULL (gy = 1) the block adds its instance's sum to out itself.
constexpr int kParamThreads = 256;
constexpr int64_t kParamChunk = 4096;  // particles per block, about
__global__ void __launch_bounds__(kParamThreads) k_adj_params(const double *__restrict__ pbar, int64_t ld,
                                                              const int32_t *__restrict__ mat,
                                                              const int64_t *__restrict__ inst_off, int ninst,
                                                              int64_t n, int nmat, int gy, double *part, double *out) {
  const int inst = blockIdx.x, j = blockIdx.y;
  const int64_t lo0 = (ninst > 1 && inst_off) ? inst_off[inst] : 0;
  const int64_t hi0 = (ninst > 1 && inst_off) ? inst_off[inst + 1] : n;
  const int64_t len = hi0 - lo0, ch = (len + gy - 1) / gy;
  const int64_t lo = lo0 + min(len, (int64_t)j * ch), hi = lo0 + min(len, (int64_t)(j + 1) * ch);
  __shared__ double sh[kParamThreads][3];
  for (int mm = 0; mm < nmat; ++mm) {
    double acc[3] = {0, 0, 0};
    for (int64_t i = lo + threadIdx.x; i < hi; i += kParamThreads) {
      const int mi0 = mat ? mat[i] : 0;
      const int mi = (mi0 >= 0 && mi0 < nmat) ? mi0 : 0;
      if (mi != mm) continue;
      for (int k = 0; k < 3; ++k) acc[k] += pbar[k * ld + i];
    }
    for (int k = 0; k < 3; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = kParamThreads / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s)
        for (int k = 0; k < 3; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + s][k];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const int64_t q = (int64_t)inst * nmat + mm;
      for (int k = 0; k < 3; ++k) {
        if (part) part[(q * gy + j) * 3 + k] = sh[0][k];
        else out[q * 3 + k] += sh[0][k];
      }
    }
    __syncthreads();
  }
}

__global__ void k_adj_params_final(const double *__restrict__ part, int64_t m, int gy, double *out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // entry (inst * nmat + mat) * 3 + k
  if (t >= m) return;
  const int64_t q = t / 3;
  const int k = (int)(t - 3 * q);
  double s = 0.0;
  for (int j = 0; j < gy; ++j) s += part[(q * gy + j) * 3 + k];
  out[t] += s;
}

// The parameter cotangents of all particles (c->ag, 3 x cap_n) summed into
// param_bar; the adjoint's intermediate buffer holds the partial sums (it is
// free once pass A's reverse has read it).
static void adj_params_sum(sph_ctx *c, const int32_t *mat, const int64_t *inst_off, int ninst, int64_t n, int nmat,
                           double *param_bar, cudaStream_t st) {
  int64_t g = (n / ninst + kParamChunk - 1) / kParamChunk;
  int gy = (int)std::max<int64_t>(1, std::min<int64_t>(1024, g));
  if ((int64_t)ninst * nmat * gy * 3 > (int64_t)22 * c->cap_n) gy = 1;
  double *part = gy > 1 ? c->adj_inter : nullptr;
  { k_adj_params<<<dim3(ninst, gy), kParamThreads, 0, st>>>(c->ag, c->cap_n, mat, inst_off, ninst, n, nmat, gy, part,
                                                          param_bar); ++sph::g_launches; }
  if (part) {
    const int64_t m = (int64_t)ninst * nmat * 3;
    { k_adj_params_final<<<nblk(m, 256), 256, 0, st>>>(part, m, gy, param_bar); ++sph::g_launches; }
  }
}

// ---------------------------------------------------------------------------
// Mixed precision (requested precision SPH_MIXED): the pair terms of passes B
// and A are differentiated in FP32, in the code units of the forward
// evaluation (powers of two, so every conversion is exact), on differences of
// the hi/lo-split positions and velocities as in the forward pass, with
// Kahan-compensated FP32 sums; the constitutive update (k_adj_update) stays
// FP64.  A quantity q in SI is q_code * U_q, so its cotangent in SI is the
// code-unit cotangent divided by U_q, and a given output cotangent enters in
// code units multiplied by U_q.
// ---------------------------------------------------------------------------
// Forward T and c_s back to FP64 SI for k_adj_update; output cotangents of
// dv/dt and du/dt into code units for pass B.
__global__ void k_adj_unpack32(AdjArgs A, double *T64, double *cs64) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.n) return;
  const Units &U = *A.U;
  const double uT = U.sig * U.invrho * U.invrho;  // T = sigma / rho^2
  const float4 t0 = A.Tf[c], t1 = A.Tf[A.ld + c];
  const float t[6] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y};
  const int ns = nsym(A.dim);
  for (int k = 0; k < 6; ++k) T64[(int64_t)k * A.ld + c] = k < ns ? (double)t[k] * uT : 0.0;
  cs64[c] = (double)t1.z * U.V;
  float vb[3] = {0.f, 0.f, 0.f};
  for (int i = 0; i < A.dim; ++i)
    if (A.bdv[i]) vb[i] = (float)(A.bdv[i][c] * U.acc);
  const float ub = A.bdu ? (float)(A.bdu[c] * (U.E * U.invT)) : 0.f;
  A.Bpk[c] = make_float4(vb[0], vb[1], vb[2], ub);
}

__device__ __forceinline__ void load_T32(const AdjArgs &A, int64_t b, float t[6], float &cs) {
  const float4 t0 = A.Tf[b], t1 = A.Tf[A.ld + b];
  t[0] = t0.x;
  t[1] = t0.y;
  t[2] = t0.z;
  t[3] = t0.w;
  t[4] = t1.x;
  t[5] = t1.y;
  cs = t1.z;
}

template <int DIM>
__global__ void k_adj_passB32(AdjArgs A) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.n) return;
  constexpr int dim = DIM;
  const int ns = nsym(dim);
  const float4 Pc = A.pk.px(c), Qc = A.pk.pxl(c), Vc = A.pk.pv(c), Wc = A.pk.pvl(c);
  float Tc[6], csc;
  load_T32(A, c, Tc, csc);
  const float4 bc = A.Bpk[c];
  const float vbc[3] = {bc.x, bc.y, bc.z};
  KahanT<float> gx[3], gv[3], Tb[6], csb, rhb;
  const int cnt = A.nb_cnt[c];
  AdjCursor cur;
  cur.start(A, c, cnt);
  for (int k = 0; k < cnt; ++k) {
    float4 Pe, Qe;
    const int32_t e = cur.next(A, k, Pe, Qe);
    const float4 Ve = A.pk.pv(e), We = A.pk.pvl(e);
    float d[3] = {(Pc.x - Pe.x) + (Qc.x - Qe.x), (Pc.y - Pe.y) + (Qc.y - Qe.y),
                  DIM == 3 ? (Pc.z - Pe.z) + (Qc.z - Qe.z) : 0.f};
    float w[3] = {(Vc.x - Ve.x) + (Wc.x - We.x), (Vc.y - Ve.y) + (Wc.y - We.y),
                  DIM == 3 ? (Vc.z - Ve.z) + (Wc.z - We.z) : 0.f};
    float Te[6], cse;
    load_T32(A, e, Te, cse);
    const float4 be = A.Bpk[e];
    const float vbe[3] = {be.x, be.y, be.z};
    const float hab = 0.5f * (Pc.w + Pe.w);
    float r2 = 0.f;
    for (int i = 0; i < dim; ++i) r2 += d[i] * d[i];
    const KPair<float> K = kernel_pair<float>(dim, sqrtf(r2), hab);
    const VPair<float> Vs = visc_pair<float>(dim, d, w, r2, hab, Vc.w, Ve.w, csc, cse, A.prm);
    float db[3], wb[3], Bs[6], csh, rh;
    pairB_adj<float>(dim, d, w, K, Vs, Tc, Te, Qe.w, vbc, bc.w, db, wb, Bs, csh, rh);  // c's own term
    for (int i = 0; i < dim; ++i) {
      gx[i].add(db[i]);
      gv[i].add(wb[i]);
    }
    for (int q = 0; q < ns; ++q) Tb[q].add(Bs[q]);
    csb.add(csh);
    rhb.add(rh);
    const float dn[3] = {-d[0], -d[1], -d[2]}, wn[3] = {-w[0], -w[1], -w[2]};
    pairB_adj<float>(dim, dn, wn, K, Vs, Te, Tc, Qc.w, vbe, be.w, db, wb, Bs, csh, rh);  // e's term, w.r.t. c
    for (int i = 0; i < dim; ++i) {
      gx[i].add(-db[i]);
      gv[i].add(-wb[i]);
    }
    for (int q = 0; q < ns; ++q) Tb[q].add(Bs[q]);
    csb.add(csh);
    rhb.add(rh);
  }
  const Units &U = *A.U;
  for (int i = 0; i < dim; ++i) {
    A.gx[i][c] += gx[i].value() * U.invL;
    A.gv[i][c] += gv[i].value() * U.invV;
  }
  A.grho[c] += rhb.value() * U.invrho;
  const double uTinv = U.rho * U.rho * U.invsig;
  for (int q = 0; q < 6; ++q) A.Tbar[(int64_t)q * A.ld + c] = q < ns ? Tb[q].value() * uTinv : 0.0;
  A.csbar[c] = csb.value() * U.invV;
}

// Cotangents of the pass-A sums (FP64 SI, from k_adj_update) into code units:
// the continuity sum and G are rates (1/T), L is a number, XSPH a velocity.
__global__ void k_adj_pack_acot32(AdjArgs A) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.n) return;
  const Units &U = *A.U;
  const double *I = A.inter;
  const int64_t ld = A.ld;
  float v[24];
  v[0] = (float)(I[c] * U.invT);
  for (int k = 0; k < 9; ++k) {
    v[1 + k] = (float)I[(1 + k) * ld + c];
    v[10 + k] = (float)(I[(10 + k) * ld + c] * U.invT);
  }
  for (int i = 0; i < 3; ++i) v[19 + i] = (float)(I[(19 + i) * ld + c] * U.V);
  v[22] = v[23] = 0.f;
  for (int q = 0; q < 6; ++q) A.Apk[(int64_t)q * ld + c] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__device__ __forceinline__ ACot<float> load_acot32(const AdjArgs &A, int64_t a) {
  float v[24];
  for (int q = 0; q < 6; ++q) {
    const float4 t = A.Apk[(int64_t)q * A.ld + a];
    v[4 * q] = t.x;
    v[4 * q + 1] = t.y;
    v[4 * q + 2] = t.z;
    v[4 * q + 3] = t.w;
  }
  ACot<float> c;
  c.sr = v[0];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      c.Lb[i][j] = v[1 + 3 * i + j];
      c.Gb[i][j] = v[10 + 3 * i + j];
    }
    c.xb[i] = v[19 + i];
  }
  return c;
}

template <int DIM>
__global__ void k_adj_passA32(AdjArgs A) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.n) return;
  constexpr int dim = DIM;
  const float4 Pc = A.pk.px(c), Qc = A.pk.pxl(c), Vc = A.pk.pv(c), Wc = A.pk.pvl(c);
  const ACot<float> Cc = load_acot32(A, c);
  KahanT<float> gx[3], gv[3], grho;
  const int cnt = A.nb_cnt[c];
  AdjCursor cur;
  cur.start(A, c, cnt);
  for (int k = 0; k < cnt; ++k) {
    float4 Pe, Qe;
    const int32_t e = cur.next(A, k, Pe, Qe);
    const float4 Ve = A.pk.pv(e), We = A.pk.pvl(e);
    float d[3] = {(Pc.x - Pe.x) + (Qc.x - Qe.x), (Pc.y - Pe.y) + (Qc.y - Qe.y),
                  DIM == 3 ? (Pc.z - Pe.z) + (Qc.z - Qe.z) : 0.f};
    float w[3] = {(Vc.x - Ve.x) + (Wc.x - We.x), (Vc.y - Ve.y) + (Wc.y - We.y),
                  DIM == 3 ? (Vc.z - Ve.z) + (Wc.z - We.z) : 0.f};
    const float hab = 0.5f * (Pc.w + Pe.w);
    float r2 = 0.f;
    for (int i = 0; i < dim; ++i) r2 += d[i] * d[i];
    const float r = sqrtf(r2);
    const KPair<float> K = kernel_pair<float>(dim, r, hab);
    float db[3], wb[3], ra, rb;
    pairA_adj<float>(dim, d, w, r, K, Qe.w, Vc.w, Ve.w, Cc, db, wb, ra, rb);  // c's own term
    for (int i = 0; i < dim; ++i) {
      gx[i].add(db[i]);
      gv[i].add(wb[i]);
    }
    grho.add(ra);
    const ACot<float> Ce = load_acot32(A, e);
    const float dn[3] = {-d[0], -d[1], -d[2]}, wn[3] = {-w[0], -w[1], -w[2]};
    pairA_adj<float>(dim, dn, wn, r, K, Qc.w, Ve.w, Vc.w, Ce, db, wb, ra, rb);  // e's term, w.r.t. c
    for (int i = 0; i < dim; ++i) {
      gx[i].add(-db[i]);
      gv[i].add(-wb[i]);
    }
    grho.add(rb);
  }
  const Units &U = *A.U;
  for (int i = 0; i < dim; ++i) {
    A.gx[i][c] += gx[i].value() * U.invL;
    A.gv[i][c] += gv[i].value() * U.invV;
  }
  A.grho[c] += grho.value() * U.invrho;
}

void rhs_adjoint(sph_ctx *c, const sph_state *s, const MatTable &mt, const sph_params &p, const sph_derivs &dbar,
                 sph_state *sbar, double *param_bar, cudaStream_t st) {
  const int64_t n = s->n;
  if (n == 0) return;
  AdjArgs A;
  memset(&A, 0, sizeof(A));
  A.dim = s->dim;
  A.n = n;
  A.ld = c->cap_n;
  for (int k = 0; k < 3; ++k) {
    A.x[k] = s->x[k];
    A.v[k] = s->v[k];
    A.bdx[k] = dbar.dx[k];
    A.bdv[k] = dbar.dv[k];
    A.gx[k] = sbar->x[k];
    A.gv[k] = sbar->v[k];
  }
  A.rho = s->rho;
  A.u = s->u;
  A.m = s->m;
  A.h = s->h;
  A.S = s->S;
  A.dmg = s->dmg;
  A.mat = s->mat;
  A.nb_idx = c->nb_idx;
  A.nb_cnt = c->nb_cnt;
  A.T = (const double *)c->T;
  A.cs = c->cs;
  A.bdrho = dbar.drho;
  A.bdu = dbar.du;
  A.bdS = dbar.dS;
  A.grho = sbar->rho;
  A.gu = sbar->u;
  A.gS = sbar->S;
  // scratch: the step buffers of the second derivative set are free here
  A.Tbar = c->st.d_S[1];
  A.csbar = c->st.d_cs[1];
  A.inter = c->adj_inter;
  A.pbar = c->ag;
  A.mt = mt;
  A.prm = p;
  const int T = 128;
  if (p.precision == SPH_MIXED) {
    A.pk = c->pk;
    A.Tf = (const float4 *)c->T;
    A.Bpk = c->adj32;
    A.Apk = c->adj32 + c->cap_n;
    A.U = c->units;
    A.sums = c->adj_sums;
    // FP64 SI copies of T and c_s for the constitutive reverse (the third
    // derivative set of the step buffers is free here)
    double *T64 = c->st.d_S[2], *cs64 = c->st.d_cs[2];
    A.T = T64;
    A.cs = cs64;
    { k_adj_unpack32<<<nblk(n, 256), 256, 0, st>>>(A, T64, cs64); ++sph::g_launches; }
    if (s->dim == 3) {
      { k_adj_passB32<3><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
      { k_adj_update<true, 3><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
    } else {
      { k_adj_passB32<2><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
      { k_adj_update<true, 2><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
    }
    { k_adj_pack_acot32<<<nblk(n, 256), 256, 0, st>>>(A); ++sph::g_launches; }
    if (s->dim == 3) { k_adj_passA32<3><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
    else { k_adj_passA32<2><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
  } else if (s->dim == 3) {
    { k_adj_passB<3><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
    { k_adj_update<false, 3><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
    { k_adj_passA<3><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
  } else {
    { k_adj_passB<2><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
    { k_adj_update<false, 2><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
    { k_adj_passA<2><<<nblk(n, T), T, 0, st>>>(A); ++sph::g_launches; }
  }
  const int ninst = s->ninst > 0 ? s->ninst : 1;
  if (param_bar) adj_params_sum(c, s->mat, s->inst_off, ninst, n, mt.nmat, param_bar, st);
}

// ---------------------------------------------------------------------------
// Reverse of out = Y(base + frac dt d): the state cotangent passes to base,
// frac dt times it to the derivatives, through the yield map for S.
// ---------------------------------------------------------------------------
struct PcAdjArgs {
  int dim;
  int64_t n;
  const double *bS, *dS;
  const int32_t *mat;
  const int64_t *inst_off;
  int ninst;
  const double *dt;
  double frac;
  MatTable mt;
  const double *ox[3], *ov[3], *orho, *ou, *oS;   // cotangent of out
  double *gx[3], *gv[3], *grho, *gu, *gS;         // base cotangent (+=)
  double *fx[3], *fv[3], *frho, *fu, *fS;         // derivative cotangent (=)
  double *pY;                                     // per-particle Y0 cotangent (=)
  int density_sum;
};

__global__ void k_pc_adj(PcAdjArgs A) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A.n) return;
  const int inst = inst_of(A.inst_off, A.ninst, a);
  const double h = A.frac * A.dt[inst];
  for (int ax = 0; ax < A.dim; ++ax) {
    const double lx = A.ox[ax][a], lv = A.ov[ax][a];
    A.gx[ax][a] += lx;
    A.gv[ax][a] += lv;
    A.fx[ax][a] = h * lx;
    A.fv[ax][a] = h * lv;
  }
  A.grho[a] += A.orho[a];
  A.frho[a] = A.density_sum ? 0.0 : h * A.orho[a];
  A.gu[a] += A.ou[a];
  A.fu[a] = h * A.ou[a];
  double yb = 0.0;
  if (A.bS) {
    const int ns = nsym(A.dim);
    const int mi0 = A.mat ? A.mat[a] : 0;
    const sph_material &M = A.mt.m[(mi0 >= 0 && mi0 < A.mt.nmat) ? mi0 : 0];
    double Sp[6], lo[6], J2 = 0.0, proj = 0.0;
    for (int k = 0; k < ns; ++k) {
      Sp[k] = A.bS[(int64_t)k * A.n + a] + h * A.dS[(int64_t)k * A.n + a];
      lo[k] = A.oS[(int64_t)k * A.n + a];
      J2 += (k < A.dim ? 1.0 : 2.0) * Sp[k] * Sp[k];
      proj += lo[k] * Sp[k];
    }
    J2 *= 0.5;
    const bool yielding = M.strength && M.Y0 > 0.0 && J2 > 0.0 && M.Y0 * M.Y0 / (3.0 * J2) < 1.0;
    const double f = yielding ? M.Y0 * M.Y0 / (3.0 * J2) : 1.0;
    for (int k = 0; k < ns; ++k) {
      double sb = lo[k];
      if (yielding) sb = f * lo[k] - f / J2 * proj * (k < A.dim ? 1.0 : 2.0) * Sp[k];
      A.gS[(int64_t)k * A.n + a] += sb;
      A.fS[(int64_t)k * A.n + a] = h * sb;
    }
    if (yielding) yb = proj * 2.0 * f / M.Y0;
  }
  A.pY[a] = yb;
}

void pc_update_adjoint(sph_ctx *c, const sph_state *base, const sph_derivs &d, const double *dt, double frac,
                       const MatTable &mt, const sph_params &p, const sph_state *obar, sph_state *gbar,
                       sph_derivs *fbar, double *param_bar, cudaStream_t st) {
  const int64_t n = base->n;
  if (n == 0) return;
  PcAdjArgs A;
  memset(&A, 0, sizeof(A));
  A.dim = base->dim;
  A.n = n;
  A.bS = base->S;
  A.dS = d.dS;
  A.mat = base->mat;
  A.inst_off = base->inst_off;
  A.ninst = base->ninst > 0 ? base->ninst : 1;
  A.dt = dt;
  A.frac = frac;
  A.mt = mt;
  for (int k = 0; k < 3; ++k) {
    A.ox[k] = obar->x[k];
    A.ov[k] = obar->v[k];
    A.gx[k] = gbar->x[k];
    A.gv[k] = gbar->v[k];
    A.fx[k] = fbar->dx[k];
    A.fv[k] = fbar->dv[k];
  }
  A.orho = obar->rho;
  A.ou = obar->u;
  A.oS = obar->S;
  A.grho = gbar->rho;
  A.gu = gbar->u;
  A.gS = gbar->S;
  A.frho = fbar->drho;
  A.fu = fbar->du;
  A.fS = fbar->dS;
  // per-particle Y0 cotangent in the parameter scratch (mu and K stay zero)
  cudaMemsetAsync(c->ag, 0, sizeof(double) * 3 * c->cap_n, st);
  A.pY = c->ag + c->cap_n;
  A.density_sum = p.density_sum;
  { k_pc_adj<<<nblk(n, 256), 256, 0, st>>>(A); ++sph::g_launches; }
  const int ninst = base->ninst > 0 ? base->ninst : 1;
  if (param_bar) adj_params_sum(c, base->mat, base->inst_off, ninst, n, mt.nmat, param_bar, st);
}

}  // namespace sph
