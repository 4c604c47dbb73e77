// Predictor-corrector integrator (Sect. 3.4.1): time-step limits reduced on
// the device (no host round trip, so a step can run inside a CUDA graph) and
// a fused element-wise update of every integrated field.
//
// dt per instance = min over its particles of
//   c_courant h / c_s,   c_accel sqrt(h / |dv/dt|),
//   c_quantity (|q| + floor_q) / |dq/dt| for rho (continuity), u, each S
//   component and d^1/3 (the paper's sqrt(q^2 / dq^2) with a floor so that a
//   quantity starting at zero does not force dt = 0), capped at dt_max.
// The acceleration limit takes the square root that makes it a time.
#include <cmath>

#include "fpbits.cuh"
#include "pack.cuh"
#include "sph_internal.cuh"

namespace sph {

__global__ void k_dt_init(unsigned long long *enc, int ninst, double dtmax) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ninst) enc[i] = dbl_to_ord(dtmax);
}

struct DtArgs {
  int dim;
  int64_t n;
  const double *rho, *u, *h, *S, *dmg;
  const double *dv[3], *drho, *du, *dS, *ddmg, *cs;
  const int64_t *inst_off;
  int ninst;
  sph_params prm;
  unsigned long long *enc;
  // FP32 copies of the constants, for the screening below
  float f_courant, f_accel, f_quantity, f_u_floor, f_S_floor, f_dmg_floor, f_dt_max;
};

// FP32 view of a double for screening, built from its bits on the integer
// pipe: the top 23 mantissa bits (truncated: relative error below 2^-23).
// Outside 2^-60 <= |v| <= 2^60 (zero excepted) the view is not trusted and
// `risky` is set; squares and quotients of trusted views stay in FP32's
// normal range.
__device__ __forceinline__ float screen_f32(double v, bool &risky) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if ((b << 1) == 0ULL) return 0.f;
  const unsigned hi = (unsigned)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e < 1023 - 60 || e > 1023 + 60) {
    risky = true;
    return 0.f;
  }
  const unsigned mant = ((hi & 0xfffffu) << 3) | ((unsigned)b >> 29);
  return __uint_as_float((hi & 0x80000000u) | ((unsigned)(e - 1023 + 127) << 23) | mant);
}

__device__ __forceinline__ bool bits_nonzero(double v) { return ((unsigned long long)__double_as_longlong(v) << 1) != 0ULL; }

// c_accel sqrt(h / |dv/dt|), or `none` for zero acceleration.  Out of line
// so that the compiler branches around it rather than predicating it.
static __device__ __noinline__ double accel_limit(int dim, double h, double a0, double a1, double a2v, double c,
                                           double none) {
  double a2 = a0 * a0;
  a2 += a1 * a1;
  if (dim == 3) a2 += a2v * a2v;
  return a2 > 0.0 ? c * sqrt(h / sqrt(a2)) : none;
}

// The limits of one particle, called by every thread of a block.  Every limit
// is first estimated in FP32 (within about 1e-6 relative); the FP64 expression
// is then evaluated only for limits whose estimate lies within 2^-12 of the
// smallest estimate of the block (of the warp or the lane, when those span
// several instances: `scope` 2, 1, 0), or whose inputs the FP32 view does not
// trust.  Any limit skipped is larger than the one that attains that minimum,
// so the minimum over the scope equals the all-FP64 minimum bit for bit, at
// about one FP64 division per block.  The result for one thread is only
// meaningful through that minimum.
__device__ double particle_dt(const DtArgs &A, int64_t a_in, bool valid, int scope) {
  const sph_params &P = A.prm;
  const int64_t a = valid ? a_in : A.n - 1;  // lanes past the end read the last particle, then drop out
  const float inf = __int_as_float(0x7f800000);
  float est[11];
  unsigned risky = 0;
  const double h = A.h[a], cs = A.cs[a];
  bool r = false;
  const float hf = screen_f32(h, r);
  {
    bool rc = r;
    const float csf = screen_f32(cs, rc);
    est[0] = (long long)__double_as_longlong(cs) > 0 ? A.f_courant * hf * __frcp_rn(csf) : inf;
    if (rc) risky |= 1u;
  }
  double dvd[3] = {0.0, 0.0, 0.0};
  {
    bool ra = r, any = false;
    float a2 = 0.f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if (ax >= A.dim) break;
      dvd[ax] = A.dv[ax][a];
      const float f = screen_f32(dvd[ax], ra);
      a2 += f * f;
      any |= bits_nonzero(dvd[ax]);
    }
    est[1] = any ? A.f_accel * sqrtf(hf) * rsqrtf(sqrtf(a2)) : inf;
    if (ra) risky |= 2u;
  }
  const double drho = A.drho[a], rho = A.rho[a];
  {
    bool rr = false;
    const float q = fabsf(screen_f32(rho, rr)), d = fabsf(screen_f32(drho, rr));
    est[2] = (!P.density_sum && bits_nonzero(drho)) ? A.f_quantity * q * __frcp_rn(d) : inf;
    if (rr) risky |= 4u;
  }
  const double du = A.du[a], u = A.u[a];
  {
    bool rr = false;
    const float q = fabsf(screen_f32(u, rr)), d = fabsf(screen_f32(du, rr));
    est[3] = bits_nonzero(du) ? A.f_quantity * (q + A.f_u_floor) * __frcp_rn(d) : inf;
    if (rr) risky |= 8u;
  }
  const int ns = nsym(A.dim);
  const bool has_S = A.S && A.dS;
  for (int k = 0; k < 6; ++k) {
    est[4 + k] = inf;
    if (has_S && k < ns) {
      bool rr = false;
      const double q = A.S[(int64_t)k * A.n + a], dq = A.dS[(int64_t)k * A.n + a];
      const float qf = fabsf(screen_f32(q, rr)), df = fabsf(screen_f32(dq, rr));
      if (bits_nonzero(dq)) est[4 + k] = A.f_quantity * (qf + A.f_S_floor) * __frcp_rn(df);
      if (rr) risky |= 16u << k;
    }
  }
  est[10] = inf;
  const bool has_d = A.dmg && A.ddmg;
  double dd = 0.0, dq = 0.0;
  if (has_d) {
    bool rr = false;
    dq = A.ddmg[a];
    dd = A.dmg[a];
    const float qf = fabsf(screen_f32(dd, rr)), df = screen_f32(dq, rr);
    if ((long long)__double_as_longlong(dq) > 0) est[10] = A.f_quantity * (qf + A.f_dmg_floor) * __frcp_rn(df);
    if (rr) risky |= 1024u;
  }
  if (!valid) {
    risky = 0;
#pragma unroll
    for (int i = 0; i < 11; ++i) est[i] = inf;
  }
  float best = A.f_dt_max;
#pragma unroll
  for (int i = 0; i < 11; ++i)
    if (!((risky >> i) & 1u)) best = fminf(best, est[i]);
  if (scope >= 1)
    for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (scope == 2) {
    __shared__ float bmin[32];
    if ((threadIdx.x & 31) == 0) bmin[threadIdx.x >> 5] = best;
    __syncthreads();
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) best = fminf(best, bmin[k]);
  }
  const float thr = best * (1.f + 1.f / 4096.f);
  unsigned pick = risky;
#pragma unroll
  for (int i = 0; i < 11; ++i)
    if (est[i] <= thr) pick |= 1u << i;
  // FP64, exactly as the limits are defined.  Every limit except the
  // acceleration one has the form c (|q| + floor) / den (floor = 0 for the
  // Courant and density limits, where |q| + 0 = |q|); the picked ones are
  // evaluated in a loop with one division per pass, usually a single pass.
  double dt = P.dt_max;
  const unsigned avail = 0xfu | (has_S ? ((1u << ns) - 1u) << 4 : 0u) | (has_d ? 1024u : 0u);
  pick &= avail;
  unsigned rem = pick & ~2u;
  while (rem) {
    const int i = __ffs(rem) - 1;
    rem &= rem - 1;
    double q, d, c = P.c_quantity, fl = 0.0;
    bool ok = true, absd = true;
    if (i == 0) {
      q = h;
      d = cs;
      c = P.c_courant;
      absd = false;
    } else if (i == 2) {
      q = rho;
      d = drho;
      ok = !P.density_sum;
    } else if (i == 3) {
      q = u;
      d = du;
      fl = P.u_floor;
    } else if (i < 10) {
      q = A.S[(int64_t)(i - 4) * A.n + a];
      d = A.dS[(int64_t)(i - 4) * A.n + a];
      fl = P.S_floor;
    } else {
      q = dd;
      d = dq;
      fl = P.dmg_floor;
      absd = false;
    }
    const uint64_t db = dbits(d) & (absd ? 0x7fffffffffffffffULL : ~0ULL);
    const uint64_t qb = dbits(q) & 0x7fffffffffffffffULL;
    if (ok && (int64_t)db > 0 && db <= 0x7ff0000000000000ULL)  // den > 0 (NaN excluded)
      dt = fmin(dt, c * (bitsd(qb) + fl) / bitsd(db));
  }
  if (pick & 2u) dt = fmin(dt, accel_limit(A.dim, h, dvd[0], dvd[1], dvd[2], P.c_accel, dt));
  return dt;
}

__device__ __forceinline__ unsigned long long warp_min_ord(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

__global__ void k_dt(DtArgs A) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const sph_params &P = A.prm;
  const bool valid = a < A.n;
  const int inst = valid ? inst_of(A.inst_off, A.ninst, a) : 0;
  // the widest scope lying in one instance: block (2), warp (1) or lane (0)
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ int binst;
  if (threadIdx.x == 0) binst = inst;
  __syncthreads();
  const int inst0 = __shfl_sync(full, inst, 0);
  const bool wsame = __all_sync(full, inst == inst0 || !valid);
  const bool bsame = __syncthreads_and(inst == binst || !valid);
  const int scope = bsame ? 2 : (wsame ? 1 : 0);
  const double dt = particle_dt(A, a, valid, scope);
  // minima as order-preserving integers (integer pipe): per lane when the warp
  // spans instances, else per warp, then one atomic per run of equal instances
  // among the block's warps
  unsigned long long o = valid ? dbl_to_ord(dt) : dbl_to_ord(P.dt_max);
  __shared__ unsigned long long wmin[32];
  __shared__ int winst[32];
  if (wsame) {
    o = warp_min_ord(o);
  } else {
    if (valid) atomicMin(&A.enc[inst], o);
    o = dbl_to_ord(P.dt_max);  // already reported
  }
  if (lane == 0) {
    wmin[w] = o;
    winst[w] = inst0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long none = dbl_to_ord(P.dt_max);
    const int nw = blockDim.x >> 5;
    unsigned long long cur = wmin[0];
    int ci = winst[0];
    for (int k = 1; k < nw; ++k) {
      if (winst[k] == ci) {
        cur = wmin[k] < cur ? wmin[k] : cur;
      } else {
        if (cur < none) atomicMin(&A.enc[ci], cur);
        cur = wmin[k];
        ci = winst[k];
      }
    }
    if (cur < none) atomicMin(&A.enc[ci], cur);
  }
}

__global__ void k_dt_final(const unsigned long long *enc, double *dt, int ninst, double dt_fixed, double *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  double v = dt_fixed > 0.0 ? dt_fixed : ord_to_dbl(enc[i]);
  dt[i] = v;
  if (out) out[i] = v;
}

void timestep_reduce(sph_ctx *c, const sph_state *s, const sph_params &p, const sph_derivs &d, cudaStream_t st) {
  const int ninst = s->ninst > 0 ? s->ninst : 1;
  { k_dt_init<<<nblk(ninst, 128), 128, 0, st>>>(c->st.dt_enc, ninst, p.dt_max); ++sph::g_launches; }
  if (p.dt_fixed <= 0.0 && s->n > 0) {
    DtArgs A;
    memset(&A, 0, sizeof(A));
    A.dim = s->dim;
    A.n = s->n;
    A.rho = s->rho;
    A.u = s->u;
    A.h = s->h;
    A.S = s->S;
    A.dmg = s->dmg;
    for (int k = 0; k < 3; ++k) A.dv[k] = d.dv[k];
    A.drho = d.drho;
    A.du = d.du;
    A.dS = d.dS;
    A.ddmg = d.ddmg;
    A.cs = d.cs;
    A.inst_off = s->inst_off;
    A.ninst = ninst;
    A.prm = p;
    A.enc = c->st.dt_enc;
    A.f_courant = (float)p.c_courant;
    A.f_accel = (float)p.c_accel;
    A.f_quantity = (float)p.c_quantity;
    A.f_u_floor = (float)p.u_floor;
    A.f_S_floor = (float)p.S_floor;
    A.f_dmg_floor = (float)p.dmg_floor;
    A.f_dt_max = (float)p.dt_max;
    { k_dt<<<nblk(s->n, 256), 256, 0, st>>>(A); ++sph::g_launches; }
  }
  { k_dt_final<<<nblk(ninst, 128), 128, 0, st>>>(c->st.dt_enc, c->st.dt, ninst, p.dt_fixed, nullptr); ++sph::g_launches; }
}

// ---------------------------------------------------------------------------
// out = base + frac * dt * deriv, then S <- f_Y S and the damage cap
// ---------------------------------------------------------------------------
// One derivative set (device arrays, layout of sph_derivs)
struct DSet {
  const double *dx[3], *dv[3], *drho, *du, *dS, *ddmg;
};

// out = base + dt_inst (c_0 d_0 + c_1 d_1 + c_2 d_2), nd sets (the
// predictor-corrector: one set, c_0 = 1/2 or 1; the Runge-Kutta stages:
// up to three), then the yield and damage limits.
struct PcArgs {
  int dim;
  int64_t n;
  const double *bx[3], *bv[3], *brho, *bu, *bS, *bdmg;
  double *ox[3], *ov[3], *orho, *ou, *oS, *odmg;
  DSet d[3];
  double coef[3];
  int pow2;  // one derivative set whose coefficient is a power of two
  int nd;
  const int32_t *mask;  // per instance: update only where set (NULL: all)
  const int32_t *nact, *mat, *id;  // nact: of the last set
  const int64_t *flaw_off;
  const int64_t *inst_off;
  int ninst;
  const double *dt;
  MatTable mt;
  int density_sum;
  unsigned long long *dmove;  // NULL, or max |out.x - base.x| (bits of a non-negative double)
  int32_t *err;
  // pack: also write the FP32 views of out (those k_pack would write)
  int pack;
  PackedF32 pk;
  const double *ilo, *h, *m;
  const Units *U;
};

// The combined derivative c_0 d_0[i] + c_1 d_1[i] + c_2 d_2[i], in that
// order (for one set, c_0 = 1/2 or 1 scales exactly)
__device__ __forceinline__ double comb(const PcArgs &A, const double *p0, const double *p1, const double *p2,
                                       int64_t i) {
  double v = A.coef[0] * p0[i];
  if (A.nd > 1) v += A.coef[1] * p1[i];
  if (A.nd > 2) v += A.coef[2] * p2[i];
  return v;
}

// b + dt (c_0 d_0[i] + ...).  With one set and c_0 a power of two,
// (c_0 dt) d_0[i] is the same exact product as dt (c_0 d_0[i]), so the update
// is one fused multiply-add with the same rounding.
__device__ __forceinline__ double upd(const PcArgs &A, double b, double dt, double dtc, const double *p0,
                                      const double *p1, const double *p2, int64_t i) {
  if (A.pow2) return b + dtc * p0[i];
  return b + dt * comb(A, p0, p1, p2, i);
}

// The exact difference, for the rare operands outside FP32's range (kept out
// of line, as the FP64 fallbacks of fpbits.cuh)
static __device__ __noinline__ uint64_t move_bits_slow(double ox, double bx) {
  return dbits(ox - bx) & 0x7fffffffffffffffULL;
}

// Bits of an upper bound of |ox - bx| for ox = fl(bx + dtc d) (one rounding):
// |dtc d| + ulp(ox) / 2 <= fl_up(fl_up(|dtc|) fl_up(|d|)) + ulp(ox), taken in
// FP32 with upward rounding from the bit patterns, so that no FP64
// instruction is spent on the displacement bound.
__device__ __forceinline__ uint64_t move_bound_bits(double dtc, double d, double ox, double bx) {
  const uint64_t mag = 0x7fffffffffffffffULL;
  float fa, fb;
  const int e = (int)((dbits(ox) >> 52) & 0x7ff);
  const int ef = e - 1075 + 127;  // float exponent field of ulp(ox) = 2^(e - 1075)
  if (ef <= 254 && f32_dir_scaled(bitsd(dbits(dtc) & mag), 0, true, fa) &&
      f32_dir_scaled(bitsd(dbits(d) & mag), 0, true, fb)) {
    const float ulp = bitsf((uint32_t)(ef >= 1 ? ef : 1) << 23);  // 2^-126 bounds the smaller ulps
    double out;
    if (f64_scaled(__fadd_ru(__fmul_ru(fa, fb), ulp), 0, out)) return dbits(out);
  }
  return move_bits_slow(ox, bx);
}

// Update of particle a; returns the bits of an upper bound of
// max_axis |out.x - base.x| when A.dmove is set (else 0).
__device__ __forceinline__ unsigned long long pc_particle(const PcArgs &A, int64_t a) {
  const int inst = inst_of(A.inst_off, A.ninst, a);
  if (A.mask && !A.mask[inst]) return 0ULL;
  const double dt = A.dt[inst];
  const double dtc = dt * A.coef[0];
  unsigned long long mv = 0ULL;  // bits of max |ox - bx| (non-negative doubles order as integers)
  bool bad = false;
  double xo[3] = {0.0, 0.0, 0.0}, vo[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (ax >= A.dim) continue;  // a constant trip count keeps xo, vo in registers
    const double bx = A.bx[ax][a];
    const double ox = upd(A, bx, dt, dtc, A.d[0].dx[ax], A.d[1].dx[ax], A.d[2].dx[ax], a);
    const double ov = upd(A, A.bv[ax][a], dt, dtc, A.d[0].dv[ax], A.d[1].dv[ax], A.d[2].dv[ax], a);
    A.ox[ax][a] = ox;
    A.ov[ax][a] = ov;
    xo[ax] = ox;
    vo[ax] = ov;
    if (A.dmove) {
      const unsigned long long m =
          A.pow2 ? move_bound_bits(dtc, A.d[0].dx[ax][a], ox, bx) : (dbits(ox - bx) & 0x7fffffffffffffffULL);
      mv = m > mv ? m : mv;
      bad |= !finite_bits(ox) || !finite_bits(ov);
    }
  }
  const double rho_o =
      A.density_sum ? A.brho[a] : upd(A, A.brho[a], dt, dtc, A.d[0].drho, A.d[1].drho, A.d[2].drho, a);
  A.orho[a] = rho_o;
  if (A.dmove) {
    bad |= !positive_finite_bits(rho_o);
    if (bad) raise_err(A.err, ERR_NONFINITE);
  }
  if (A.pack)
    pack_particle(A.pk, a, A.dim, xo[0], xo[1], xo[2], vo[0], vo[1], vo[2], A.h[a], A.m[a], rho_o, A.ilo + 3 * inst,
                  A.U);
  A.ou[a] = upd(A, A.bu[a], dt, dtc, A.d[0].du, A.d[1].du, A.d[2].du, a);
  const int mi = A.mat ? A.mat[a] : 0;
  const sph_material &M = A.mt.m[(mi >= 0 && mi < A.mt.nmat) ? mi : 0];
  if (A.bS) {
    const int ns = nsym(A.dim);
    double S[6];
    for (int k = 0; k < ns; ++k) {
      int64_t i = (int64_t)k * A.n + a;
      S[k] = upd(A, A.bS[i], dt, dtc, A.d[0].dS, A.d[1].dS, A.d[2].dS, i);
    }
    // f_Y = min(Y0^2 / (3 J2), 1) differs from 1 only if Y0^2 < 3 J2 (both
    // rounded as in the quotient), so the division runs for yielding
    // particles only; the result is the same bit for bit.  An FP32 screen
    // from the bit patterns (relative error below 2^-20) first excludes the
    // particles clearly inside the yield surface, 3 J2 < Y0^2 (1 - 2^-12),
    // without FP64 instructions.
    if (M.strength && M.Y0 > 0.0) {
      bool inside = false;
      {
        float s2 = 0.f, y0f;
        bool ok = f32_rn_scaled(M.Y0, 0, y0f);
        for (int k = 0; k < ns; ++k) {
          float f;
          ok = ok && f32_rn_scaled(S[k], 0, f);
          s2 += (k < A.dim ? 1.f : 2.f) * f * f;
        }
        inside = ok && 1.5f * s2 < y0f * y0f * (1.f - 1.f / 4096.f);
      }
      if (!inside) {
        double J2 = 0.0;
        for (int k = 0; k < ns; ++k) J2 += (k < A.dim ? 1.0 : 2.0) * S[k] * S[k];  // off-diagonals twice in S:S
        J2 *= 0.5;
        const double y2 = M.Y0 * M.Y0, j3 = 3.0 * J2;
        if (J2 > 0.0 && y2 < j3) {
          const double fY = fmin(y2 / j3, 1.0);
          for (int k = 0; k < ns; ++k) S[k] *= fY;
        }
      }
    }
    for (int k = 0; k < ns; ++k) A.oS[(int64_t)k * A.n + a] = S[k];
  }
  if (A.bdmg) {
    // with one set of coefficient c_0 > 0, dd > 0 iff its derivative is
    // positive (a test of the bits)
    const double d0 = A.d[0].ddmg[a];
    const double dd = A.pow2 ? d0 : comb(A, A.d[0].ddmg, A.d[1].ddmg, A.d[2].ddmg, a);
    double nd = A.pow2 ? A.bdmg[a] + dtc * d0 : A.bdmg[a] + dt * dd;
    const bool grows = A.pow2 ? (int64_t)dbits(d0) > 0 : dd > 0.0;
    if (grows) {
      const int64_t idp = A.id ? A.id[a] : a;
      const int64_t ntot = A.flaw_off[idp + 1] - A.flaw_off[idp];
      // the cap (n_act / n_tot)^(1/3) binds only if nd^3 n_tot >= n_act; an
      // FP32 test with a 2^-12 margin skips the cube root where it cannot
      float ndf;
      const bool below = f32_rn_scaled(nd, 0, ndf) && ndf >= 0.f &&
                         ndf * ndf * ndf * (float)ntot < (float)A.nact[a] * (1.f - 1.f / 4096.f);
      if (!below) nd = fmin(nd, cbrt((double)A.nact[a] / (double)ntot));
    }
    A.odmg[a] = (ord_of(nd) <= ord_of(1.0) && finite_bits(nd)) ? nd : 1.0;  // min(nd, 1) on the integer pipe
  }
  return mv;
}

__global__ void k_pc(PcArgs A) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long mv = 0ULL;
  if (a < A.n) mv = pc_particle(A, a);
  if (A.dmove) {  // every lane of the warp arrives here
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, mv, o);
      mv = w > mv ? w : mv;
    }
    if ((threadIdx.x & 31) == 0 && mv != 0ULL) atomicMax(A.dmove, mv);
  }
}

static DSet dset_of(const sph_derivs &d) {
  DSet r;
  for (int k = 0; k < 3; ++k) {
    r.dx[k] = d.dx[k];
    r.dv[k] = d.dv[k];
  }
  r.drho = d.drho;
  r.du = d.du;
  r.dS = d.dS;
  r.ddmg = d.ddmg;
  return r;
}

void combine_update(sph_ctx *c, const sph_state *base, sph_state *out, const sph_derivs *const *d, const double *coef,
                    int nd, const int32_t *mask, const MatTable &mt, const sph_params &p, cudaStream_t st,
                    unsigned long long *dmove, bool pack) {
  if (base->n == 0) return;
  PcArgs A;
  memset(&A, 0, sizeof(A));
  A.dim = base->dim;
  A.n = base->n;
  for (int k = 0; k < 3; ++k) {
    A.bx[k] = base->x[k];
    A.bv[k] = base->v[k];
    A.ox[k] = out->x[k];
    A.ov[k] = out->v[k];
  }
  A.brho = base->rho;
  A.bu = base->u;
  A.bS = base->S;
  A.bdmg = base->dmg;
  A.orho = out->rho;
  A.ou = out->u;
  A.oS = out->S;
  A.odmg = out->dmg;
  A.nd = nd;
  for (int j = 0; j < nd; ++j) {
    A.d[j] = dset_of(*d[j]);
    A.coef[j] = coef[j];
  }
  int e2 = 0;
  A.pow2 = nd == 1 && std::frexp(coef[0], &e2) == 0.5;
  A.nact = d[nd - 1]->n_act;
  A.mask = mask;
  A.mat = base->mat;
  A.id = base->id;
  A.flaw_off = base->flaw_off;
  A.inst_off = base->inst_off;
  A.ninst = base->ninst > 0 ? base->ninst : 1;
  A.dt = c->st.dt;
  A.mt = mt;
  A.density_sum = p.density_sum;
  A.dmove = dmove;
  A.err = c->d_err;
  A.pack = pack ? 1 : 0;
  if (pack) {
    A.pk = c->pk;
    A.ilo = c->tree.inst_lo;
    A.h = out->h;
    A.m = out->m;
    A.U = c->units;
  }
  { k_pc<<<nblk(base->n, 256), 256, 0, st>>>(A); ++sph::g_launches; }
}

void pc_update(sph_ctx *c, const sph_state *base, sph_state *out, const sph_derivs &d, double frac,
               const MatTable &mt, const sph_params &p, cudaStream_t st, unsigned long long *dmove, bool pack) {
  const sph_derivs *dd[1] = {&d};
  combine_update(c, base, out, dd, &frac, 1, nullptr, mt, p, st, dmove, pack);
}

// ---------------------------------------------------------------------------
// Embedded Runge-Kutta step (Sect. 3.4.2): error estimate and step control
// ---------------------------------------------------------------------------
struct RkErrArgs {
  int dim;
  int64_t n;
  const double *x[3], *v[3], *rho, *u, *S, *dmg, *h;
  DSet k[3];
  const double *cs;  // of k1
  const int64_t *inst_off;
  int ninst;
  const double *dt;
  double u_floor, S_floor, dmg_floor;
  int density_sum;
  unsigned long long *err;  // per instance
};

// largest |2 k2 - k1 - k3| / (|q + dt k1| + floor) of one particle, tracked as
// a (numerator, denominator) pair by cross-multiplication so that only the
// winner is divided
__device__ __forceinline__ void rk_track(double q, double k1, double k2, double k3, double dt, double fl, double &bn,
                                         double &bd) {
  const double num = fabs(2.0 * k2 - k1 - k3), den = fabs(q + dt * k1) + fl;
  if (num * bd > bn * den) {
    bn = num;
    bd = den;
  }
}

__global__ void k_rk_error(RkErrArgs A) {
  const int64_t a_in = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = a_in < A.n;
  const int64_t a = valid ? a_in : A.n - 1;  // lanes past the end read the last particle, then drop out
  const int inst = inst_of(A.inst_off, A.ninst, a);
  const double dt = A.dt[inst];
  double bn = 0.0, bd = 1.0;
  for (int ax = 0; ax < A.dim; ++ax) {
    rk_track(A.x[ax][a], A.k[0].dx[ax][a], A.k[1].dx[ax][a], A.k[2].dx[ax][a], dt, A.h[a], bn, bd);
    rk_track(A.v[ax][a], A.k[0].dv[ax][a], A.k[1].dv[ax][a], A.k[2].dv[ax][a], dt, A.cs[a], bn, bd);
  }
  if (!A.density_sum) rk_track(A.rho[a], A.k[0].drho[a], A.k[1].drho[a], A.k[2].drho[a], dt, 0.0, bn, bd);
  rk_track(A.u[a], A.k[0].du[a], A.k[1].du[a], A.k[2].du[a], dt, A.u_floor, bn, bd);
  if (A.S)
    for (int k = 0; k < nsym(A.dim); ++k) {
      const int64_t i = (int64_t)k * A.n + a;
      rk_track(A.S[i], A.k[0].dS[i], A.k[1].dS[i], A.k[2].dS[i], dt, A.S_floor, bn, bd);
    }
  if (A.dmg) rk_track(A.dmg[a], A.k[0].ddmg[a], A.k[1].ddmg[a], A.k[2].ddmg[a], dt, A.dmg_floor, bn, bd);
  const double num = bn * dt / 6.0;
  const double e = bd > 0.0 ? num / bd : (num > 0.0 ? __longlong_as_double(0x7ff0000000000000LL) : 0.0);
  // non-negative doubles order as their bits: a warp maximum when the warp lies
  // in one instance, then one atomic
  unsigned long long o = valid ? (unsigned long long)__double_as_longlong(e) : 0ULL;
  const int inst0 = __shfl_sync(0xffffffffu, inst, 0);
  if (__all_sync(0xffffffffu, inst == inst0)) {
    for (int k = 16; k > 0; k >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, o, k);
      o = w > o ? w : o;
    }
    if ((threadIdx.x & 31) == 0 && o != 0ULL) atomicMax(&A.err[inst0], o);
  } else if (o != 0ULL) {
    atomicMax(&A.err[inst], o);
  }
}

// per instance: accept where err < eps_des (t += dt), then the new step size
__global__ void k_rk_control(const unsigned long long *__restrict__ err, int32_t *__restrict__ acc,
                             double *__restrict__ dt_io, const double *__restrict__ dt_used, double *__restrict__ t_io,
                             int ninst, double eps_des, double dt_max, double *__restrict__ err_log,
                             int32_t *__restrict__ acc_log) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  const double e = __longlong_as_double((long long)err[i]), dt = dt_used[i];
  const int ok = e < eps_des;
  acc[i] = ok;
  if (t_io && ok) t_io[i] += dt;
  double dn;
  if (ok) dn = e > 0.0 ? dt * pow(eps_des / e, 0.3) : dt_max;
  else dn = 0.9 * dt * pow(eps_des / e, 0.25);
  dt_io[i] = dn < dt_max ? dn : dt_max;
  if (err_log) err_log[i] = e;
  if (acc_log) acc_log[i] = ok;
}

// the step size of this attempt: the caller's where positive, else the
// predictor-corrector limit just computed into dt_used
__global__ void k_rk_dt(double *__restrict__ dt_io, double *__restrict__ dt_used, int ninst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  const double v = dt_io[i] > 0.0 ? dt_io[i] : dt_used[i];
  dt_io[i] = v;
  dt_used[i] = v;
}

void rk_error_control(sph_ctx *c, const sph_state *s, const sph_derivs *const *k, const sph_params &p, double eps_des,
                      double *dt_io, double *t_io, double *err_log, int32_t *acc_log, cudaStream_t st) {
  const int ninst = s->ninst > 0 ? s->ninst : 1;
  cudaMemsetAsync(c->st.rk_err, 0, sizeof(unsigned long long) * ninst, st);
  if (s->n > 0) {
    RkErrArgs A;
    memset(&A, 0, sizeof(A));
    A.dim = s->dim;
    A.n = s->n;
    for (int ax = 0; ax < 3; ++ax) {
      A.x[ax] = s->x[ax];
      A.v[ax] = s->v[ax];
    }
    A.rho = s->rho;
    A.u = s->u;
    A.S = s->S;
    A.dmg = s->dmg;
    A.h = s->h;
    for (int j = 0; j < 3; ++j) A.k[j] = dset_of(*k[j]);
    A.cs = k[0]->cs;
    A.inst_off = s->inst_off;
    A.ninst = ninst;
    A.dt = c->st.dt;
    A.u_floor = p.u_floor;
    A.S_floor = p.S_floor;
    A.dmg_floor = p.dmg_floor;
    A.density_sum = p.density_sum;
    A.err = c->st.rk_err;
    { k_rk_error<<<nblk(s->n, 256), 256, 0, st>>>(A); ++sph::g_launches; }
  }
  { k_rk_control<<<nblk(ninst, 128), 128, 0, st>>>(c->st.rk_err, c->st.rk_acc, dt_io, c->st.dt, t_io, ninst, eps_des,
                                                  p.dt_max, err_log, acc_log); ++sph::g_launches; }
}

void rk_set_dt(sph_ctx *c, const sph_state *s, double *dt_io, cudaStream_t st) {
  const int ninst = s->ninst > 0 ? s->ninst : 1;
  { k_rk_dt<<<nblk(ninst, 128), 128, 0, st>>>(dt_io, c->st.dt, ninst); ++sph::g_launches; }
}

// Displacement bounds of a reused tree: the sum of per-update maxima, rounded
// up, bounds every particle's displacement since the build.
__global__ void k_bound_add(unsigned long long *out, const unsigned long long *a, const unsigned long long *b) {
  *out = dbits(__dadd_ru(bitsd(*a), bitsd(*b)));
}

void bound_add(unsigned long long *out, const unsigned long long *a, const unsigned long long *b, cudaStream_t st) {
  { k_bound_add<<<1, 1, 0, st>>>(out, a, b); ++g_launches; }
}

}  // namespace sph
