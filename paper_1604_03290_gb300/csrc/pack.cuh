// FP32 views of one particle (see PackedF32), shared by the packing kernel of
// the tree build and the predictor-corrector update, which writes the views
// of the state it produces.
#pragma once

#include "fpbits.cuh"
#include "sph_internal.cuh"

namespace sph {

// Particle i of instance corner ilo (3 doubles), in code units.  The code
// units are powers of two: scaling is an exponent shift, and the conversions
// and hi/lo splits run on the integer pipe (fpbits.cuh); only the corner
// subtraction needs the FP64 unit.
__device__ __forceinline__ void pack_particle(const PackedF32 &pk, int64_t i, int dim, double x, double y, double z,
                                              double vx, double vy, double vz, double h, double m, double rho,
                                              const double *ilo, const Units *U) {
  const int kL = pow2_exp(U->invL), kV = pow2_exp(U->invV), kM = pow2_exp(U->invM), kR = pow2_exp(U->invrho);
  const double X[3] = {__dsub_rn(x, ilo[0]), __dsub_rn(y, ilo[1]), dim == 3 ? __dsub_rn(z, ilo[2]) : 0.0};
  const double V[3] = {vx, vy, dim == 3 ? vz : 0.0};
  float xh[3], xl[3], vh[3], vl[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    to_f32_split_scaled(X[ax], kL, U->invL, xh[ax], xl[ax]);
    to_f32_split_scaled(V[ax], kV, U->invV, vh[ax], vl[ax]);
  }
  const float hf = to_f32_scaled(h, kL, U->invL), mf = to_f32_scaled(m, kM, U->invM);
  const float rf = to_f32_scaled(rho, kR, U->invrho);
  pk.px(i) = make_float4(xh[0], xh[1], xh[2], hf);
  pk.pxl(i) = make_float4(xl[0], xl[1], xl[2], mf);
  pk.pv(i) = make_float4(vh[0], vh[1], vh[2], rf);
  pk.pvl(i) = make_float4(vl[0], vl[1], vl[2], __fdiv_rn(mf, rf));
}

}  // namespace sph
