// Equations of state shared by the right-hand side and its adjoint.
#pragma once

#include <type_traits>

#include "fpbits.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace ad {
// Forward-mode dual number in FP32 with three tangent directions: the value v
// and d[k] = dv/dx_k.  The mixed adjoint evaluates the equation of state once
// in it (directions: density, specific energy, bulk-modulus scale) for the
// derivatives of p and c_s.  Its functions live in this namespace, so that
// only argument-dependent lookup finds them and the float and double
// overloads of the same names are unaffected.
struct Dual3 {
  float v, d[3];
  __device__ Dual3() : v(0.f), d{0.f, 0.f, 0.f} {}
  __device__ Dual3(int x) : v((float)x), d{0.f, 0.f, 0.f} {}
  __device__ Dual3(float x) : v(x), d{0.f, 0.f, 0.f} {}
  __device__ explicit Dual3(double x) : v((float)x), d{0.f, 0.f, 0.f} {}
  __device__ Dual3(float x, float d0, float d1, float d2) : v(x), d{d0, d1, d2} {}
};
__device__ __forceinline__ Dual3 operator+(const Dual3 &a, const Dual3 &b) {
  return Dual3(a.v + b.v, a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]);
}
__device__ __forceinline__ Dual3 operator-(const Dual3 &a, const Dual3 &b) {
  return Dual3(a.v - b.v, a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]);
}
__device__ __forceinline__ Dual3 operator-(const Dual3 &a) { return Dual3(-a.v, -a.d[0], -a.d[1], -a.d[2]); }
__device__ __forceinline__ Dual3 operator*(const Dual3 &a, const Dual3 &b) {
  return Dual3(a.v * b.v, a.d[0] * b.v + a.v * b.d[0], a.d[1] * b.v + a.v * b.d[1], a.d[2] * b.v + a.v * b.d[2]);
}
__device__ __forceinline__ Dual3 operator/(const Dual3 &a, const Dual3 &b) {
  const float q = a.v / b.v, ib = 1.f / b.v;
  return Dual3(q, (a.d[0] - q * b.d[0]) * ib, (a.d[1] - q * b.d[1]) * ib, (a.d[2] - q * b.d[2]) * ib);
}
__device__ __forceinline__ bool operator<(const Dual3 &a, const Dual3 &b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>(const Dual3 &a, const Dual3 &b) { return a.v > b.v; }
// f(a) with f'(a) = g
__device__ __forceinline__ Dual3 chain(const Dual3 &a, float f, float g) {
  return Dual3(f, g * a.d[0], g * a.d[1], g * a.d[2]);
}
__device__ __forceinline__ Dual3 exp(const Dual3 &a) {
  const float e = expf(a.v);
  return chain(a, e, e);
}
__device__ __forceinline__ Dual3 expm1(const Dual3 &a) { return chain(a, expm1f(a.v), expf(a.v)); }
__device__ __forceinline__ Dual3 log1p(const Dual3 &a) { return chain(a, log1pf(a.v), 1.f / (1.f + a.v)); }
__device__ __forceinline__ Dual3 sqrt(const Dual3 &a) {
  const float s = sqrtf(a.v);
  return chain(a, s, s > 0.f ? 0.5f / s : 0.f);
}
}  // namespace ad

// Equation of state (Sect. 2.5) -> pressure and sound speed, in R and in the
// units of the constants (SI in FP64 mode, code units in mixed mode).
// Branch decisions and rho - rho0 (the cold-expansion cancellation) use the
// SI doubles in every mode.
template <class R>
struct EosC {
  R rho0, cs, K0, nM, A, B, E0, a, b, alpha, beta;
  double iE, irho;  // SI -> code for specific energy and density
};

template <class R>
__device__ __forceinline__ EosC<R> eos_consts(const sph_material &M, const float *mf, const Units *U);

template <>
__device__ __forceinline__ EosC<double> eos_consts<double>(const sph_material &M, const float *, const Units *) {
  return EosC<double>{M.rho0, M.cs, M.K0, M.n_M, M.A_T, M.B_T, M.E0, M.a_T, M.b_T, M.alpha_T, M.beta_T, 1.0, 1.0};
}
template <>
__device__ __forceinline__ EosC<float> eos_consts<float>(const sph_material &, const float *f, const Units *U) {
  return EosC<float>{f[MF_RHO0], f[MF_CS], f[MF_K0], f[MF_NM], f[MF_AT], f[MF_BT], f[MF_E0], f[MF_AA], f[MF_BB],
                     f[MF_ALPHA], f[MF_BETA], U->invE, U->invrho};
}

// The code-unit constants of the mixed form as dual numbers: the bulk-modulus
// constants (K0, A, B) carry their derivative with respect to a common scale
// factor of all three (third direction).
template <>
__device__ __forceinline__ EosC<ad::Dual3> eos_consts<ad::Dual3>(const sph_material &, const float *f,
                                                                  const Units *U) {
  using D = ad::Dual3;
  return EosC<D>{D(f[MF_RHO0]), D(f[MF_CS]), D(f[MF_K0], 0.f, 0.f, f[MF_K0]), D(f[MF_NM]),
                 D(f[MF_AT], 0.f, 0.f, f[MF_AT]), D(f[MF_BT], 0.f, 0.f, f[MF_BT]), D(f[MF_E0]), D(f[MF_AA]),
                 D(f[MF_BB]), D(f[MF_ALPHA]), D(f[MF_BETA]), U->invE, U->invrho};
}

// R = ad::Dual3: the mixed form's code units and decisions, with density and
// specific energy as the first two directions (derivatives with respect to
// their code-unit values).
template <class R>
__device__ void eos_eval(const sph_material &M, const EosC<R> &K, double rho_d, double u_d, R &p, R &cs,
                         R *pr_out = nullptr, R *pu_out = nullptr) {
  constexpr bool F32 = std::is_same<R, float>::value;
  constexpr bool DUAL = std::is_same<R, ad::Dual3>::value;
  constexpr bool BITS = F32 || DUAL;  // branch decisions from the bit patterns of the SI doubles
  const double drho = rho_d - M.rho0;
  R chi, rho, u;
  const R rho0 = K.rho0;
  int kE = 0;
  if constexpr (F32) {
    // code-unit views by exponent shifts (the units are powers of two); chi
    // from the FP64 difference, in FP32
    const int kr = pow2_exp(K.irho);
    kE = pow2_exp(K.iE);
    rho = to_f32_scaled(rho_d, kr, K.irho);
    u = to_f32_scaled(u_d, kE, K.iE);
    chi = __fdiv_rn(to_f32_scaled(drho, kr, K.irho), rho0);
  } else if constexpr (DUAL) {
    const int kr = pow2_exp(K.irho);
    kE = pow2_exp(K.iE);
    rho = R(to_f32_scaled(rho_d, kr, K.irho), 1.f, 0.f, 0.f);
    u = R(to_f32_scaled(u_d, kE, K.iE), 0.f, 1.f, 0.f);
    chi = R(__fdiv_rn(to_f32_scaled(drho, kr, K.irho), rho0.v), __frcp_rn(rho0.v), 0.f, 0.f);
  } else {
    chi = (R)(drho / M.rho0);
    rho = (R)(rho_d * K.irho);
    u = (R)(u_d * K.iE);
  }
  switch (M.eos) {
    case SPH_EOS_LINEAR: {
      R dr;
      if constexpr (DUAL) dr = chi * rho0;
      else dr = (R)(drho * K.irho);
      p = K.cs * K.cs * dr;
      R pr = K.cs * K.cs;
      if (M.rho_cut > 0.0 && rho_d / M.rho0 < M.rho_cut) {
        p = R(0);
        pr = R(0);
      }
      cs = K.cs;
      if (pr_out) *pr_out = pr;
      if (pu_out) *pu_out = R(0);
      return;
    }
    case SPH_EOS_MURNAGHAN: {
      // K0/n ((rho/rho0)^n - 1) = K0/n expm1(n log1p(chi)), accurate near rho0
      R lg = log1p(chi);
      p = K.K0 / K.nM * expm1(K.nM * lg);
      const R c2 = K.K0 / rho0 * exp((K.nM - R(1)) * lg);
      cs = sqrt(c2);
      if (pr_out) *pr_out = c2;
      if (pu_out) *pu_out = R(0);
      return;
    }
    case SPH_EOS_ISOTHERMAL: {
      p = K.cs * K.cs * rho;
      cs = K.cs;
      if (pr_out) *pr_out = K.cs * K.cs;
      if (pu_out) *pu_out = R(0);
      return;
    }
    default:
      break;
  }
  // Tillotson (Eqs. tillo1, tillo2)
  const R A = K.A, B = K.B, E0 = K.E0, a = K.a, b = K.b;
  const R eta = R(1) + chi;
  const R w = R(1) + u / (E0 * eta * eta);
  const R dw_drho = -R(2) * u / (E0 * eta * eta * eta * rho0);
  const R dw_du = R(1) / (E0 * eta * eta);
  // compressed / cold branch
  const R kc = a + b / w;
  const R pc = kc * rho * u + A * chi + B * chi * chi;
  const R pcr = kc * u - b / (w * w) * dw_drho * rho * u + (A + R(2) * B * chi) / rho0;
  const R pcu = kc * rho - b / (w * w) * dw_du * rho * u;
  R pr, pu;
  const bool cold = BITS ? (nonneg_bits(drho) || le_bits(u_d, M.E_iv)) : (drho >= 0.0 || u_d <= M.E_iv);
  if (cold) {
    p = pc;
    pr = pcr;
    pu = pcu;
  } else {
    // expanded branch; z = rho0/rho - 1 = -chi/eta (density floored at 1e-3 rho0 inside the exponentials)
    const bool floored = BITS ? le_bits(rho_d, 1e-3 * M.rho0) : !(rho_d > 1e-3 * M.rho0);
    const R z = floored ? R(999) : -chi / eta;
    const R dz = floored ? R(0) : -rho0 / (rho * rho);
    const R eb = exp(-K.beta * z), ea = exp(-K.alpha * z * z);
    const R X = b * rho * u / w + A * chi * eb;
    const R dX = b * u / w - b * rho * u / (w * w) * dw_drho + A / rho0 * eb + A * chi * eb * (-K.beta) * dz;
    const R dY = ea * (-R(2) * K.alpha * z) * dz;
    const R pe = a * rho * u + X * ea;
    const R per = a * u + dX * ea + X * dY;
    const R peu = a * rho + (b * rho / w - b * rho * u / (w * w) * dw_du) * ea;
    if (BITS ? le_bits(M.E_cv, u_d) : u_d >= M.E_cv) {
      p = pe;
      pr = per;
      pu = peu;
    } else {
      R dE, wu, wl;
      if constexpr (F32) {
        dE = to_f32_scaled(M.E_cv - M.E_iv, kE, K.iE);
        wu = to_f32_scaled(u_d - M.E_iv, kE, K.iE);
        wl = to_f32_scaled(M.E_cv - u_d, kE, K.iE);
      } else if constexpr (DUAL) {
        dE = R(to_f32_scaled(M.E_cv - M.E_iv, kE, K.iE));
        wu = R(to_f32_scaled(u_d - M.E_iv, kE, K.iE), 0.f, 1.f, 0.f);
        wl = R(to_f32_scaled(M.E_cv - u_d, kE, K.iE), 0.f, -1.f, 0.f);
      } else {
        dE = (R)((M.E_cv - M.E_iv) * K.iE);
        wu = (R)((u_d - M.E_iv) * K.iE);
        wl = (R)((M.E_cv - u_d) * K.iE);
      }
      p = (wu * pe + wl * pc) / dE;
      pr = (wu * per + wl * pcr) / dE;
      pu = ((pe - pc) + wu * peu + wl * pcu) / dE;
    }
  }
  R c2 = pr + p / (rho * rho) * pu;
  const R cmin = A / rho0;
  cs = sqrt(c2 > cmin ? c2 : cmin);
  if (pr_out) *pr_out = pr;
  if (pu_out) *pu_out = pu;
}

}  // namespace sph
