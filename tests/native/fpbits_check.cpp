// Checks the integer-pipe conversions of fpbits.cuh against the C library's
// own FP64 -> FP32 conversions (round to nearest even, and the directed
// modes through fesetround), ldexp, and ordering, on random and edge inputs.
#define __host__
#define __device__
#define __forceinline__ inline
#include <cfenv>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>

#include "fpbits.cuh"

using namespace sph;

static bool normal_or_zero(float f) { return f == 0.0f || std::fpclassify(f) == FP_NORMAL; }

static float cvt(double v, int mode) {
  std::fesetround(mode);
  volatile double vv = v;
  volatile float r = (float)vv;
  std::fesetround(FE_TONEAREST);
  return r;
}

int main(int argc, char **argv) {
  long iters = argc > 1 ? atol(argv[1]) : 2000000;
  std::mt19937_64 g(12345);
  long checked = 0, fails = 0, fallbacks = 0;
  auto report = [&](const char *what, double v, int k) {
    if (++fails < 20) printf("FAIL %s v=%.17g (%016llx) k=%d\n", what, v, (unsigned long long)dbits(v), k);
  };
  const double edge[] = {0.0, -0.0, 1.0, -1.0, 0.5, 1.5, 3.0, 1e-30, 1e30, 3.4028234e38, 1.1754944e-38,
                         1.0000000596046448, 1.0000001788139343, 0.99999997, 16777217.0, -16777217.0,
                         33554435.0, 1e-300, 1e300, INFINITY, -INFINITY, NAN, 5e-324};
  for (long it = 0; it < iters + (long)(sizeof(edge) / sizeof(edge[0])); ++it) {
    double v;
    int k;
    if (it < (long)(sizeof(edge) / sizeof(edge[0]))) {
      v = edge[it];
      k = 0;
    } else {
      uint64_t r = g();
      int mode = (int)(r & 3);
      if (mode == 0) {
        v = bitsd(g());  // any bit pattern
      } else if (mode == 1) {  // near float rounding boundaries
        float f = bitsf((uint32_t)(g() >> 8) & 0x7fffffffu);
        if (!std::isfinite(f)) continue;
        int64_t d = (int64_t)(g() % 7) - 3;
        v = bitsd(dbits((double)f) + ((uint64_t)d << 28) + (uint64_t)(g() % 3) - 1);
      } else {
        std::uniform_real_distribution<double> u(-1e4, 1e4);
        v = u(g) * std::ldexp(1.0, (int)(g() % 120) - 60);
      }
      k = (int)(g() % 41) - 20;
    }
    const double X = std::ldexp(v, k);  // exact unless it leaves the range
    float a;
    if (f32_rn_scaled(v, k, a)) {
      ++checked;
      float ref = cvt(X, FE_TONEAREST);
      if (!(std::isfinite(v) && normal_or_zero(ref) && fbits(a) == fbits(ref))) report("rn", v, k);
    } else {
      ++fallbacks;
      float ref = cvt(X, FE_TONEAREST);
      if (std::isfinite(v) && std::fpclassify(v) != FP_SUBNORMAL && std::fpclassify(X) == FP_NORMAL &&
          normal_or_zero(ref) && ref != 0.0f && std::fabs(X) < 3.0e38)
        report("rn-declined", v, k);
    }
    for (int up = 0; up < 2; ++up)
      if (f32_dir_scaled(v, k, up != 0, a)) {
        float ref = cvt(X, up ? FE_UPWARD : FE_DOWNWARD);
        if (!(normal_or_zero(ref) && fbits(a) == fbits(ref))) report(up ? "ru" : "rd", v, k);
      }
    float h, l;
    if (f32_split_scaled(v, k, h, l)) {
      float rh = cvt(X, FE_TONEAREST);
      float rl = cvt(X - (double)rh, FE_TONEAREST);
      if (fbits(h) != fbits(rh) || (fbits(l) != fbits(rl) && !(l == 0.0f && rl == 0.0f))) report("split", v, k);
    }
    double o;
    float f = bitsf((uint32_t)g());
    if (f64_scaled(f, k, o)) {
      if (dbits(o) != dbits(std::ldexp((double)f, k))) report("f64", (double)f, k);
    }
    double w = bitsd(g());
    if (std::isfinite(v) && std::isfinite(w) && !(v == 0.0 && w == 0.0)) {
      if ((v < w) != (ord_of(v) < ord_of(w))) report("ord", v, k);
      if (dbits(of_ord(ord_of(v))) != dbits(v)) report("ord-inverse", v, k);
    }
    if (finite_bits(v) != (bool)std::isfinite(v)) report("finite", v, k);
    if (positive_finite_bits(v) != (std::isfinite(v) && v > 0.0)) report("positive", v, k);
  }
  printf("checked %ld fallbacks %ld fails %ld\n", checked, fallbacks, fails);
  return fails ? 1 : 0;
}
