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
};

__global__ void k_dt(DtArgs A) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const sph_params &P = A.prm;
  double dt = P.dt_max;
  int inst = 0;
  if (a < A.n) {
    inst = inst_of(A.inst_off, A.ninst, a);
    const double h = A.h[a];
    const double cs = A.cs[a];
    if (cs > 0.0) dt = fmin(dt, P.c_courant * h / cs);
    double a2 = 0.0;
    for (int ax = 0; ax < A.dim; ++ax) a2 += A.dv[ax][a] * A.dv[ax][a];
    if (a2 > 0.0) dt = fmin(dt, P.c_accel * sqrt(h / sqrt(a2)));
    if (!P.density_sum && fabs(A.drho[a]) > 0.0) dt = fmin(dt, P.c_quantity * fabs(A.rho[a]) / fabs(A.drho[a]));
    if (fabs(A.du[a]) > 0.0) dt = fmin(dt, P.c_quantity * (fabs(A.u[a]) + P.u_floor) / fabs(A.du[a]));
    if (A.S && A.dS) {
      const int ns = nsym(A.dim);
      for (int k = 0; k < ns; ++k) {
        double q = A.S[(int64_t)k * A.n + a], dq = A.dS[(int64_t)k * A.n + a];
        if (fabs(dq) > 0.0) dt = fmin(dt, P.c_quantity * (fabs(q) + P.S_floor) / fabs(dq));
      }
    }
    if (A.dmg && A.ddmg && A.ddmg[a] > 0.0)
      dt = fmin(dt, P.c_quantity * (fabs(A.dmg[a]) + P.dmg_floor) / A.ddmg[a]);
  }
  // warp-level min when the warp lies in one instance, else per lane; then one
  // atomic per run of equal instances among the block's warps
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ double wmin[32];
  __shared__ int winst[32];
  int inst0 = __shfl_sync(full, inst, 0);
  bool same = __all_sync(full, inst == inst0 || a >= A.n);
  if (same) {
    for (int o = 16; o > 0; o >>= 1) dt = fmin(dt, __shfl_xor_sync(full, dt, o));
  } else {
    if (a < A.n) atomicMin(&A.enc[inst], dbl_to_ord(dt));
    dt = P.dt_max;  // already reported
  }
  if (lane == 0) {
    wmin[w] = dt;
    winst[w] = inst0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    double cur = wmin[0];
    int ci = winst[0];
    for (int k = 1; k < nw; ++k) {
      if (winst[k] == ci) {
        cur = fmin(cur, wmin[k]);
      } else {
        if (cur < P.dt_max) atomicMin(&A.enc[ci], dbl_to_ord(cur));
        cur = wmin[k];
        ci = winst[k];
      }
    }
    if (cur < P.dt_max) atomicMin(&A.enc[ci], dbl_to_ord(cur));
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
    { k_dt<<<nblk(s->n, 256), 256, 0, st>>>(A); ++sph::g_launches; }
  }
  { k_dt_final<<<nblk(ninst, 128), 128, 0, st>>>(c->st.dt_enc, c->st.dt, ninst, p.dt_fixed, nullptr); ++sph::g_launches; }
}

// ---------------------------------------------------------------------------
// out = base + frac * dt * deriv, then S <- f_Y S and the damage cap
// ---------------------------------------------------------------------------
struct PcArgs {
  int dim;
  int64_t n;
  const double *bx[3], *bv[3], *brho, *bu, *bS, *bdmg;
  double *ox[3], *ov[3], *orho, *ou, *oS, *odmg;
  const double *dx[3], *dv[3], *drho, *du, *dS, *ddmg;
  const int32_t *nact, *mat, *id;
  const int64_t *flaw_off;
  const int64_t *inst_off;
  int ninst;
  const double *dt;
  double frac;
  MatTable mt;
  int density_sum;
};

__global__ void k_pc(PcArgs A) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A.n) return;
  const int inst = inst_of(A.inst_off, A.ninst, a);
  const double dt = A.frac * A.dt[inst];
  for (int ax = 0; ax < A.dim; ++ax) {
    A.ox[ax][a] = A.bx[ax][a] + dt * A.dx[ax][a];
    A.ov[ax][a] = A.bv[ax][a] + dt * A.dv[ax][a];
  }
  A.orho[a] = A.density_sum ? A.brho[a] : A.brho[a] + dt * A.drho[a];
  A.ou[a] = A.bu[a] + dt * A.du[a];
  const int mi = A.mat ? A.mat[a] : 0;
  const sph_material &M = A.mt.m[(mi >= 0 && mi < A.mt.nmat) ? mi : 0];
  if (A.bS) {
    const int ns = nsym(A.dim);
    double S[6];
    double J2 = 0.0;
    for (int k = 0; k < ns; ++k) {
      int64_t i = (int64_t)k * A.n + a;
      S[k] = A.bS[i] + dt * A.dS[i];
      J2 += (k < A.dim ? 1.0 : 2.0) * S[k] * S[k];  // off-diagonal terms appear twice in S:S
    }
    J2 *= 0.5;
    double fY = 1.0;
    if (M.strength && M.Y0 > 0.0 && J2 > 0.0) fY = fmin(M.Y0 * M.Y0 / (3.0 * J2), 1.0);
    for (int k = 0; k < ns; ++k) A.oS[(int64_t)k * A.n + a] = S[k] * fY;
  }
  if (A.bdmg) {
    double nd = A.bdmg[a] + dt * A.ddmg[a];
    if (A.ddmg[a] > 0.0) {
      const int64_t idp = A.id ? A.id[a] : a;
      const int64_t ntot = A.flaw_off[idp + 1] - A.flaw_off[idp];
      nd = fmin(nd, cbrt((double)A.nact[a] / (double)ntot));
    }
    A.odmg[a] = fmin(nd, 1.0);
  }
}

void pc_update(sph_ctx *c, const sph_state *base, sph_state *out, const sph_derivs &d, double frac,
               const MatTable &mt, const sph_params &p, cudaStream_t st) {
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
    A.dx[k] = d.dx[k];
    A.dv[k] = d.dv[k];
  }
  A.brho = base->rho;
  A.bu = base->u;
  A.bS = base->S;
  A.bdmg = base->dmg;
  A.orho = out->rho;
  A.ou = out->u;
  A.oS = out->S;
  A.odmg = out->dmg;
  A.drho = d.drho;
  A.du = d.du;
  A.dS = d.dS;
  A.ddmg = d.ddmg;
  A.nact = d.n_act;
  A.mat = base->mat;
  A.id = base->id;
  A.flaw_off = base->flaw_off;
  A.inst_off = base->inst_off;
  A.ninst = base->ninst > 0 ? base->ninst : 1;
  A.dt = c->st.dt;
  A.frac = frac;
  A.mt = mt;
  A.density_sum = p.density_sum;
  { k_pc<<<nblk(base->n, 256), 256, 0, st>>>(A); ++sph::g_launches; }
}

}  // namespace sph
