// FP64 <-> FP32 conversions, scalings by powers of two and orderings done
// from the IEEE-754 bit patterns on the integer pipe.
//
// On GB300 every FP64 instruction (add, multiply, min/max, compare and the
// double <-> float conversions) issues to the FP64 unit, which runs at 1/64
// of the FP32 rate; element-wise kernels that only convert, scale by the
// (power-of-two) code units, or compare doubles are bound by that unit.  The
// helpers below produce the same results as the FP64 instructions they
// replace (round to nearest even, or the stated directed rounding) for
// results in FP32's normal range and report failure otherwise, so callers
// keep the FP64 instruction as a fallback for the rare out-of-range case.
#pragma once

#include <stdint.h>
#include <string.h>

namespace sph {

__host__ __device__ __forceinline__ uint64_t dbits(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  memcpy(&b, &v, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ double bitsd(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  memcpy(&v, &b, 8);
  return v;
#endif
}
__host__ __device__ __forceinline__ uint32_t fbits(float v) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(v);
#else
  uint32_t b;
  memcpy(&b, &v, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ float bitsf(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float v;
  memcpy(&v, &b, 4);
  return v;
#endif
}

// Binary exponent k of a power of two p = 2^k (normal doubles).
__host__ __device__ __forceinline__ int pow2_exp(double p) { return (int)((dbits(p) >> 52) & 0x7ff) - 1023; }

// float(v * 2^k) rounded to nearest even.  False if v is subnormal, inf or
// NaN, or the result is not a normal float (or zero, for v = 0).
__host__ __device__ __forceinline__ bool f32_rn_scaled(double v, int k, float &out) {
  const uint64_t b = dbits(v);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b, sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e == 0) {
    if ((b << 1) != 0) return false;
    out = bitsf(sign);
    return true;
  }
  const int ef = e - 1023 + k + 127;
  if (e == 0x7ff || ef < 1 || ef > 254) return false;
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 fraction bits
  const uint32_t rest = lo & 0x1fffffffu, half = 0x10000000u;  // 29 dropped bits
  uint32_t r = ((uint32_t)ef << 23) | m;
  if (rest > half || (rest == half && (m & 1u))) ++r;  // a fraction carry moves into the exponent
  if ((r >> 23) > 254u) return false;
  out = bitsf(sign | r);
  return true;
}

// float(v * 2^k) rounded toward -inf (up = false) or +inf (up = true); same
// domain as f32_rn_scaled.
__host__ __device__ __forceinline__ bool f32_dir_scaled(double v, int k, bool up, float &out) {
  const uint64_t b = dbits(v);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b, sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e == 0) {
    if ((b << 1) != 0) return false;
    out = bitsf(sign);
    return true;
  }
  const int ef = e - 1023 + k + 127;
  if (e == 0x7ff || ef < 1 || ef > 254) return false;
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1fffffffu;
  uint32_t r = ((uint32_t)ef << 23) | m;
  if (rest != 0 && (up == (sign == 0))) ++r;  // away from zero: up for positive, down for negative
  if ((r >> 23) > 254u) return false;
  out = bitsf(sign | r);
  return true;
}

// X = v * 2^k split as hi = float(X), lo = float(X - hi), both rounded to
// nearest even (X - hi is exact in FP64).  False outside the domain of
// f32_rn_scaled or when lo would not be a normal float (or zero).
__host__ __device__ __forceinline__ bool f32_split_scaled(double v, int k, float &hi_out, float &lo_out) {
  const uint64_t b = dbits(v);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b, sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e == 0) {
    if ((b << 1) != 0) return false;
    hi_out = lo_out = bitsf(sign);
    return true;
  }
  const int ef = e - 1023 + k + 127;
  if (e == 0x7ff || ef < 1 || ef > 254) return false;
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1fffffffu, half = 0x10000000u;
  uint32_t r = ((uint32_t)ef << 23) | m;
  int32_t res = (int32_t)rest;  // X - hi in units of 2^(e - 1075 + k)
  if (rest > half || (rest == half && (m & 1u))) {
    ++r;
    res -= (int32_t)0x20000000;
  }
  if ((r >> 23) > 254u) return false;
  hi_out = bitsf(sign | r);
  if (res == 0) {
    lo_out = bitsf(sign);
    return true;
  }
  const int es = e - 1075 + k + 127;  // biased exponent of the residual's unit
  if (es < 1) return false;
  // |res| < 2^29: the int -> float conversion rounds to nearest even, and the
  // power-of-two factor is exact while the result stays normal
  const float fr = (float)(sign ? -res : res);
  const uint32_t fb = fbits(fr);
  const int er = (int)((fb >> 23) & 0xffu) + (es - 127);
  if (er < 1) return false;
  lo_out = bitsf((fb & 0x807fffffu) | ((uint32_t)er << 23));
  return true;
}

// (double)f * 2^k, exact.  False for zero-exponent (subnormal), inf or NaN
// f, or if the result leaves the normal double range.
__host__ __device__ __forceinline__ bool f64_scaled(float f, int k, double &out) {
  const uint32_t b = fbits(f);
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  const int e = (int)((b >> 23) & 0xffu);
  if (e == 0) {
    if ((b << 1) != 0) return false;
    out = bitsd(sign);
    return true;
  }
  const int ed = e - 127 + 1023 + k;
  if (e == 0xff || ed < 1 || ed > 2046) return false;
  out = bitsd(sign | ((uint64_t)ed << 52) | ((uint64_t)(b & 0x7fffffu) << 29));
  return true;
}

// Order-preserving map of finite doubles (and +-inf) to unsigned integers.
__host__ __device__ __forceinline__ uint64_t ord_of(double v) {
  const uint64_t b = dbits(v);
  return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}
__host__ __device__ __forceinline__ double of_ord(uint64_t o) {
  return bitsd((o & 0x8000000000000000ULL) ? (o & 0x7fffffffffffffffULL) : ~o);
}
// v is neither inf nor NaN
__host__ __device__ __forceinline__ bool finite_bits(double v) { return ((dbits(v) >> 52) & 0x7ff) != 0x7ff; }
// v > 0 and finite
__host__ __device__ __forceinline__ bool positive_finite_bits(double v) {
  const uint64_t b = dbits(v);
  return (int64_t)b > 0 && ((b >> 52) & 0x7ff) != 0x7ff;
}

#ifdef __CUDACC__
// FP64 fallbacks for values outside the helpers' domain.  They are kept out
// of line: inlined, the compiler would evaluate them unconditionally (as
// predicated code) and the FP64 unit would be busy for every value again.
static __device__ __noinline__ float f32_rn_slow(double v, double scale) { return __double2float_rn(v * scale); }
static __device__ __noinline__ float f32_rd_slow(double v, double scale) { return __double2float_rd(v * scale); }
static __device__ __noinline__ float f32_ru_slow(double v, double scale) { return __double2float_ru(v * scale); }
static __device__ __noinline__ float2 f32_split_slow(double v, double scale) {
  const double X = v * scale;
  const float hi = __double2float_rn(X);
  return make_float2(hi, __double2float_rn(X - (double)hi));
}
static __device__ __noinline__ double f64_slow(float f, double scale) { return (double)f * scale; }

// v * 2^k as a float (nearest even); `scale` = 2^k for the FP64 fallback.
__device__ __forceinline__ float to_f32_scaled(double v, int k, double scale) {
  float f;
  if (!f32_rn_scaled(v, k, f)) f = f32_rn_slow(v, scale);
  return f;
}
// float(v * 2^k) rounded down (up = false) or up
__device__ __forceinline__ float to_f32_dir_scaled(double v, int k, bool up, double scale) {
  float f;
  if (!f32_dir_scaled(v, k, up, f)) f = up ? f32_ru_slow(v, scale) : f32_rd_slow(v, scale);
  return f;
}
// hi = float(v * 2^k), lo = float(v * 2^k - hi)
__device__ __forceinline__ void to_f32_split_scaled(double v, int k, double scale, float &hi, float &lo) {
  if (!f32_split_scaled(v, k, hi, lo)) {
    const float2 r = f32_split_slow(v, scale);
    hi = r.x;
    lo = r.y;
  }
}
// (double)f * 2^k, exact; `scale` = 2^k for the fallback.
__device__ __forceinline__ double to_f64_scaled(float f, int k, double scale) {
  double d;
  if (!f64_scaled(f, k, d)) d = f64_slow(f, scale);
  return d;
}
// a <= b and a >= 0 for doubles that are not NaN, on the integer pipe
__device__ __forceinline__ bool le_bits(double a, double b) {
  return ord_of(a) <= ord_of(b) || ((dbits(a) | dbits(b)) << 1) == 0;
}
__device__ __forceinline__ bool nonneg_bits(double a) {
  const uint64_t b = dbits(a);
  return (b >> 63) == 0 || (b << 1) == 0;
}
#endif

}  // namespace sph
