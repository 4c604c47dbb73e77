/*
 * FP64 CPU oracle for the solid-body SPH right-hand side of Schaefer et al. (2016),
 * "A smooth particle hydrodynamics code to model collisions between solid,
 * self-gravitating objects".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, helper or constant with the CUDA library; every formula here is
 * written from the paper's equations (cited per function in sph_oracle.c).
 *
 * Everything is double precision, sums over neighbours run in ascending
 * neighbour index, and the file is compiled with -ffp-contract=off so that no
 * multiply-add is fused.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_EOS_LINEAR = 0, ORC_EOS_MURNAGHAN = 1, ORC_EOS_TILLOTSON = 2, ORC_EOS_ISOTHERMAL = 3 };

typedef struct {
  int32_t eos;
  int32_t strength; /* 1: evolve the deviatoric stress S (Hooke + Jaumann) */
  int32_t damage;   /* 1: Grady-Kipp damage with per-particle flaws       */
  int32_t pad;
  double rho0, cs;  /* reference density; sound speed (linear, isothermal) */
  double K0, n_M;   /* bulk modulus (Murnaghan; also the K in E and c_g)   */
  double A_T, B_T, E0, E_iv, E_cv, a_T, b_T, alpha_T, beta_T; /* Tillotson */
  double rho_cut;   /* linear EOS: p = 0 when rho/rho0 < rho_cut (0: off)  */
  double mu, Y0;    /* shear modulus; von Mises yield stress (<= 0: none)  */
} orc_material;

typedef struct {
  int32_t dim;
  int32_t density_sum;  /* 1: rho by kernel sum, 0: continuity equation   */
  int32_t consistency;  /* 1: apply the linear-consistency tensor C = L^-1 */
  int32_t gravity;      /* 1: add Barnes-Hut self-gravity                  */
  int32_t leaf_size;    /* max particles in a tree leaf                   */
  int32_t max_depth;    /* octree depth (bits per axis of the cell index)  */
  double alpha, beta, eps_v;      /* artificial viscosity                  */
  double eps_s, n_as, dmpd;       /* artificial stress (eps_s = 0: off)    */
  double xsph;                    /* XSPH factor (0: off)                  */
  double G, theta, eps_grav;      /* gravity constant, opening angle, softening / h */
  double c_courant, c_accel, c_quantity;
  double u_floor, S_floor, dmg_floor, dt_max, dt_fixed;
  double n_des;                   /* > 0: variable h (Sect. 4.2) at the start of each step */
  int32_t h_tol, h_iter;          /* its count tolerance and most updates   */
  int32_t tree_reuse;             /* > 0: with gravity, one tree (and its pseudo-particles) serves the
                                     evaluations of this many consecutive steps (Sect. 6.3); 0: a tree per
                                     evaluation */
  int32_t pad2;
} orc_params;

/* Particle state, structure of arrays.  Tensors S are symmetric and stored
 * component-major: 3D (xx, yy, zz, xy, xz, yz), 2D (xx, yy, xy); S + k*n is
 * component k.  S and dmg may be NULL (no strength / no damage).  Flaws are
 * indexed by id[a]: thresholds flaw_eps[flaw_off[id]..flaw_off[id+1]) sorted
 * ascending.  Instances: inst_off[0..ninst], particles of instance i occupy
 * [inst_off[i], inst_off[i+1]); no pair crosses an instance. */
typedef struct {
  int64_t n;
  double *x, *y, *z, *vx, *vy, *vz;
  double *rho, *u, *m, *h;
  double *S, *dmg;
  int32_t *mat;
  const int64_t *flaw_off;
  const float *flaw_eps;
  int32_t *id;
  int32_t ninst;
  int32_t pad;
  const int64_t *inst_off;
} orc_state;

/* Time derivatives and per-particle diagnostics.  Any pointer may be NULL. */
typedef struct {
  double *dxdt, *dydt, *dzdt;
  double *dvx, *dvy, *dvz;
  double *drho, *du, *dS, *ddmg;
  double *p, *cs;          /* pressure and sound speed                       */
  int32_t *n_act;          /* activated flaws                                 */
  int32_t *nnb;            /* neighbour count                                 */
  /* Per-particle magnitude sums sum_b |term_b| used as error scales:        */
  double *mag_drho, *mag_dv, *mag_du, *mag_gradv;
  /* The same sums with each term weighted by its conditioning at the       */
  /* kernel's support edge, kappa = q/(1-q) for q >= 1/2 (else 1): a       */
  /* relative error e in q changes a term by about 2 e kappa |term|.       */
  double *mag1_drho, *mag1_dv, *mag1_du, *mag1_gradv, *mag_rho, *mag1_rho;
  double *gradv;           /* corrected velocity gradient, D*D per particle,  component-major */
  double *agx, *agy, *agz; /* gravitational acceleration alone               */
  double *eps_t;           /* local strain of the damage model, sigma_max / ((1 - d) E); 0 without damage */
} orc_derivs;

/* Kernel (Sect. 3.1.1) */
double orc_W(double r, double h, int32_t dim);
double orc_dWdr(double r, double h, int32_t dim);

/* Neighbour sets N(a) = {b != a : r_ab^2 < h_ab^2}, h_ab = (h_a + h_b)/2,
 * sorted ascending.  Return the total count, or -1 if it exceeds cap. */
int64_t orc_neighbours_brute(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                             const double *h, int64_t *off, int32_t *idx, int64_t cap);
int64_t orc_neighbours_grid(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                            const double *h, int64_t *off, int32_t *idx, int64_t cap);
int32_t orc_neighbours_one(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                           const double *h, int64_t a, int32_t *out, int32_t cap);

/* Variable smoothing length (Sect. 4.2): h <- h (1 + (n_des/n_a)^(1/D)) / 2 for all
 * particles at once, n_a = #{b != a in a's instance : r_ab^2 < h_a^2}; repeated until
 * every |n_a - n_des| <= tol or max_iter updates.  n_a = 0 doubles h.  h in place;
 * counts[n] = the last n_a; returns the number of updates.  inst_off may be NULL. */
int32_t orc_adapt_h(int32_t dim, int64_t n, const double *x, const double *y, const double *z, double *h,
                    const int64_t *inst_off, int32_t ninst, double n_des, int32_t tol, int32_t max_iter,
                    int32_t *counts);

/* Embedded Runge-Kutta steps (Sect. 3.4.2), nsteps attempts: k1 = f(q), k2 = f(q + dt/2 k1),
 * k3 = f(q - dt k1 + 2 dt k2); error per instance = max over particles and components of
 * dt |2 k2 - k1 - k3| / 6 / (|q + dt k1| + floor) (floors: h for x, c_s for v, 0 for rho,
 * u_floor, S_floor, dmg_floor); err < eps_des accepts q + dt (k1 + 4 k2 + k3)/6 and sets
 * dt <- dt (eps_des/err)^0.3 (dt_max for err = 0), else q is kept and dt <- 0.9 dt
 * (eps_des/err)^(1/4); dt <= dt_max.  dt_inst[ninst] in/out (<= 0: the predictor-corrector
 * limit of k1); t_inst (may be NULL) += dt of accepted steps; err_log, acc_log (may be NULL):
 * [nsteps][ninst]. */
int32_t orc_step_rk3(orc_state *s, const orc_material *mats, int32_t nmat, const orc_params *P, double eps_des,
                     int32_t nsteps, double *dt_inst, double *t_inst, double *err_log, int32_t *acc_log);

/* Barnes-Hut accelerations at positions (x, y, z) with the tree and pseudo-particles built at
 * (xb, yb, zb): containment by the particle's current cell in the build's root cube, leaves summed
 * over their members' current positions.  xb = x gives orc_gravity_bh. */
int32_t orc_gravity_bh_reuse(int32_t dim, int64_t n, const double *xb, const double *yb, const double *zb,
                             const double *x, const double *y, const double *z, const double *m, const double *h,
                             double G, double theta, double eps_grav, int32_t leaf_size, int32_t max_depth,
                             const int64_t *sample, int64_t nsample, double *ax, double *ay, double *az);

/* Octree (Sect. 3.5.1 root cube and subdivision; bucket leaves of <= leaf_size).
 * Writes per node: level, integer cell coordinates, particle count, mass, COM.
 * Returns the node count, or -1 if it exceeds cap. */
int64_t orc_tree_nodes(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                       const double *m, int32_t leaf_size, int32_t max_depth, int64_t cap,
                       int32_t *level, int64_t *cell, int64_t *count, double *mass, double *com);
/* Integer cell coordinates of each particle at max_depth (3 per particle). */
void orc_cell_coords(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                     int32_t max_depth, int64_t *k);

/* Gravity (Sect. 3.3).  Direct O(N^2) sum and Barnes-Hut walk.  sample:
 * optional list of nsample target particles (NULL: all). */
void orc_gravity_direct(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                        const double *m, const double *h, double G, double eps_grav,
                        double *ax, double *ay, double *az);
int32_t orc_gravity_bh(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                       const double *m, const double *h, double G, double theta, double eps_grav,
                       int32_t leaf_size, int32_t max_depth, const int64_t *sample, int64_t nsample,
                       double *ax, double *ay, double *az);

/* Equation of state (Sect. 2.5): pressure, partial derivatives, sound speed. */
void orc_eos(const orc_material *mat, double rho, double u, double *p, double *dpdrho, double *dpdu,
             double *cs);

/* Symmetric eigen-solve by cyclic Jacobi rotations (dim 2 or 3); A row-major
 * dim x dim, eigenvalues w ascending, eigenvectors as columns of V. */
void orc_sym_eig(int32_t dim, const double *A, double *w, double *V);

/* One right-hand-side evaluation (Sect. 3.1.2 - 3.3).  In density-sum mode
 * rho is recomputed and written into the state.  Returns 0, or a negative
 * code when a capacity is exceeded. */
int32_t orc_rhs(orc_state *s, const orc_material *mats, int32_t nmat, const orc_params *prm,
                orc_derivs *d);

/* Time step limit (Sect. 3.4.1), per instance. */
void orc_timestep(const orc_state *s, const orc_material *mats, int32_t nmat, const orc_params *prm,
                  const orc_derivs *d, double *dt_inst);

/* nsteps predictor-corrector steps (Sect. 3.4.1).  dt_inst[ninst] receives
 * the last step's time steps; dt_log (NULL or nsteps*ninst) all of them. */
int32_t orc_step(orc_state *s, const orc_material *mats, int32_t nmat, const orc_params *prm,
                 int32_t nsteps, double *dt_inst, double *dt_log);

/* Philox4x64-10 block: out = the ten-round cipher of ctr under key. */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Weibull activation thresholds (Sect. 3.2): per group of the brittle particles of one instance and
 * material (damage set, weibull_k > 0, weibull_m > 0; group g = instance * nmat + material, members in
 * ascending id, volume V = sum m / rho0), flaw j = 1, 2, ... goes to member floor(w_j N / 2^64), w_j the
 * draw (word (j-1) mod 4 of Philox4x64-10 with counter ((j-1)/4, 0, 0, 0) and key (seed, g)), with
 * threshold (j / (k V))^(1/m) as float, until every member holds one.  flaw_off[n+1] by id; flaw_eps
 * (ascending per particle) written when the total fits in cap.  Returns the total, -1 for invalid ids. */
int64_t orc_flaws(int64_t n, const int32_t *id, const int32_t *mat, const double *m, const int64_t *inst_off,
                  int32_t ninst, const orc_material *mats, int32_t nmat, const double *weibull_k,
                  const double *weibull_m, uint64_t seed, int64_t *flaw_off, float *flaw_eps, int64_t cap);

/* Friends-of-friends fragments (Sect. 4): particles with dmg >= d_remove removed (dmg may be NULL);
 * friends = partners (same instance) with smoothing lengths b h0; fragments = connected components of
 * at least min_size particles, numbered by decreasing count, ties by smallest member index; label[n]
 * = fragment or -1; frag_count, frag_mass up to cap.  Returns the number of fragments. */
int64_t orc_fof(int32_t dim, int64_t n, const double *x, const double *y, const double *z, const double *h0,
                const double *dmg, const double *m, const int64_t *inst_off, int32_t ninst, double b,
                double d_remove, int32_t min_size, int32_t *label, int32_t *frag_count, double *frag_mass,
                int64_t cap);

void orc_set_threads(int32_t nthreads);
int32_t orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
