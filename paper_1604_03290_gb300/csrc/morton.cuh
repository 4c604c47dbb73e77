// Morton keys and cell indices (Sect. 3.5.1), shared by the tree build and
// the walks that locate a particle in an existing tree.
#pragma once

#include <stdint.h>

#include "fpbits.cuh"

namespace sph {

__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}
__device__ __forceinline__ unsigned long long compact3(unsigned long long v) {
  v &= 0x1249249249249249ULL;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ULL;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00fULL;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffULL;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffULL;
  v = (v ^ (v >> 32)) & 0x1fffffULL;
  return v;
}
__device__ __forceinline__ unsigned long long spread2(unsigned long long v) {
  v &= 0xffffffffULL;
  v = (v | (v << 16)) & 0x0000ffff0000ffffULL;
  v = (v | (v << 8)) & 0x00ff00ff00ff00ffULL;
  v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0fULL;
  v = (v | (v << 2)) & 0x3333333333333333ULL;
  v = (v | (v << 1)) & 0x5555555555555555ULL;
  return v;
}
__device__ __forceinline__ unsigned long long compact2(unsigned long long v) {
  v &= 0x5555555555555555ULL;
  v = (v ^ (v >> 1)) & 0x3333333333333333ULL;
  v = (v ^ (v >> 2)) & 0x0f0f0f0f0f0f0f0fULL;
  v = (v ^ (v >> 4)) & 0x00ff00ff00ff00ffULL;
  v = (v ^ (v >> 8)) & 0x0000ffff0000ffffULL;
  v = (v ^ (v >> 16)) & 0xffffffffULL;
  return v;
}

// Cell index along one axis, evaluated in the same operation order as the
// definition: floor(((x - min) / s0) * 2^B), clamped to [0, 2^B - 1].
__device__ __forceinline__ unsigned long long cell_index(double v, double lo, double s0, int B) {
  double t = __ddiv_rn(__dsub_rn(v, lo), s0);
  double f = floor(__dmul_rn(t, (double)(1ULL << B)));
  long long kmax = (1LL << B) - 1;
  long long k = f < 0.0 ? 0 : (f > (double)kmax ? kmax : (long long)f);
  return (unsigned long long)k;
}

// The same cell index with the quotient taken as (x - min) * (1/s0): within
// 2 ulps of the correctly rounded quotient, so the floor can differ only when
// the scaled value lies within a few ulps of an integer; those rare cases
// take the division.  The floor and that test read the bits of the scaled
// value (integer pipe); two FP64 operations remain per axis.
__device__ __forceinline__ unsigned long long cell_index_fast(double v, double lo, double s0, double rs0, int B) {
  const double t = __dmul_rn(__dsub_rn(v, lo), rs0);
  const uint64_t tb = dbits(t);
  const int et = (int)((tb >> 52) & 0x7ff);
  if ((int64_t)tb <= 0 || et == 0) return (int64_t)tb < 0 ? cell_index(v, lo, s0, B) : 0ULL;  // 0, tiny or negative
  const int E = et - 1023 + B;  // exponent of f = t * 2^B
  const unsigned long long kmax = (1ULL << B) - 1;
  if (E >= B) return kmax;
  const uint64_t mant = (tb & ((1ULL << 52) - 1)) | (1ULL << 52);
  bool near;
  unsigned long long k;
  if (E < 0) {
    k = 0;
    near = E == -1 && (mant & ((1ULL << 52) - 1)) >= (1ULL << 52) - 4;  // within 4 ulps below 1
  } else {
    const int sh = 52 - E;
    k = mant >> sh;
    const uint64_t frac = mant & ((1ULL << sh) - 1);
    near = frac <= 4 || frac >= (1ULL << sh) - 4;
  }
  return near ? cell_index(v, lo, s0, B) : k;
}


// Morton key of a position in instance `inst` of a tree: the interleaved
// cell indices at depth B below the instance bits (as the tree build forms it).
__device__ __forceinline__ unsigned long long morton_key(const double *xa, int dim, int B, int inst,
                                                         const double *ilo, double s0, double rs0) {
  const unsigned long long kx = cell_index_fast(xa[0], ilo[3 * inst + 0], s0, rs0, B);
  const unsigned long long ky = cell_index_fast(xa[1], ilo[3 * inst + 1], s0, rs0, B);
  unsigned long long key;
  if (dim == 3) {
    const unsigned long long kz = cell_index_fast(xa[2], ilo[3 * inst + 2], s0, rs0, B);
    key = spread3(kx) | (spread3(ky) << 1) | (spread3(kz) << 2);
  } else {
    key = spread2(kx) | (spread2(ky) << 1);
  }
  return key | ((unsigned long long)inst << (dim * B));
}

}  // namespace sph
