/*
 * sph.h - C ABI of the GB300 (sm_103a) solid-body SPH right-hand-side library.
 *
 * The library evaluates, on one GPU, the per-time-step right-hand side of the
 * SPH method of Schaefer et al. (2016), "A smooth particle hydrodynamics code
 * to model collisions between solid, self-gravitating objects":
 *   octree over Morton-sorted particles (Sect. 3.5.1), interaction partners
 *   (Sect. 3.5.2), kernel sums for continuity, momentum with the full stress
 *   tensor and internal energy (Sect. 3.1.2, Eqs. continuity_equation_sph,
 *   accel_artvisc, energy_sph), equations of state (Sect. 2.5), Hooke's law
 *   with Jaumann rotation (Sect. 2.4, Eqs. stresstensor_evolution,
 *   rotation_terms), von Mises yield (Sect. 2.6), Grady-Kipp damage
 *   (Sects. 2.7, 3.2), artificial viscosity and stress (Sects. 3.1.3, 3.1.4),
 *   XSPH (Sect. 3.1.5), the linear-consistency tensor (Sect. 3.1.6, Eq.
 *   ext_sph), Barnes-Hut self-gravity (Sect. 3.3, Eq. gravitational_force)
 *   and the predictor-corrector integrator (Sect. 3.4.1).
 *
 * Conventions shared by every entry point
 *  - All particle arrays are caller-owned DEVICE memory; the library never
 *    frees or reallocates them.  Host pointers are only the sph_material
 *    array, sph_params, sph_state/sph_derivs structs themselves (their
 *    fields point to device memory) and the ctx handle.
 *  - Particle data is structure-of-arrays, FP64 unless stated.  Symmetric
 *    tensors are stored component-major: 3D (xx, yy, zz, xy, xz, yz), 2D
 *    (xx, yy, xy); component k of particle a is at S[k*n + a].
 *  - h is the kernel's support radius: W(r; h) = 0 for r > h (Sect. 3.1.1).
 *    Pairs use h_ab = (h_a + h_b) / 2 (Sect. 4.2).
 *  - A context (sph_ctx) owns all scratch, sized once by sph_create; no
 *    other call allocates device memory.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = legacy default stream).  Argument errors are reported at once
 *    (SPH_ERR_INVALID); errors found by kernels (capacity exceeded,
 *    non-finite input) set a device error word that sph_sync_status reads,
 *    and that blocking calls (params.check = 1) read before returning.
 *  - No call traps, asserts or spins without a bound on the device.
 *  - Not thread-safe per context; different contexts are independent.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPH_OK = 0,
  SPH_ERR_INVALID = 1,   /* bad argument (checked on the host)                 */
  SPH_ERR_CAPACITY = 2,  /* a list or node capacity of the context was exceeded */
  SPH_ERR_NONFINITE = 3, /* NaN/Inf in the input, or h <= 0, rho <= 0           */
  SPH_ERR_TIMEOUT = 4,   /* a bounded device loop reached its iteration limit  */
  SPH_ERR_CUDA = 5       /* a CUDA runtime call failed; see sph_last_error     */
} sph_status;

enum { SPH_EOS_LINEAR = 0, SPH_EOS_MURNAGHAN = 1, SPH_EOS_TILLOTSON = 2, SPH_EOS_ISOTHERMAL = 3 };
enum { SPH_FP64 = 0, SPH_MIXED = 1 };
enum { SPH_MAX_MATERIALS = 8 };

/* Material (Sect. 2.5-2.7).  K0 is the bulk modulus used in Young's modulus
 * E = 9 K mu / (3K + mu) and the crack speed c_g (Sect. 3.2, 2.7). */
typedef struct {
  int32_t eos;       /* SPH_EOS_*                                           */
  int32_t strength;  /* 1: evolve deviatoric stress S                       */
  int32_t damage;    /* 1: Grady-Kipp damage (needs state.dmg and flaws)     */
  int32_t pad;
  double rho0, cs;   /* reference density; sound speed (linear, isothermal) */
  double K0, n_M;    /* bulk modulus; Murnaghan exponent                    */
  double A_T, B_T, E0, E_iv, E_cv, a_T, b_T, alpha_T, beta_T; /* Tillotson  */
  double rho_cut;    /* linear EOS: p = 0 below rho/rho0 < rho_cut (0: off)  */
  double mu, Y0;     /* shear modulus; von Mises yield stress (<= 0: none)   */
} sph_material;

/* Run parameters. */
typedef struct {
  int32_t dim;          /* 2 or 3                                              */
  int32_t density_sum;  /* 1: rho = sum m W (Eq. density_by_kernel_sum)        */
  int32_t consistency;  /* 1: velocity gradient with C = L^-1 (Eq. ext_sph)     */
  int32_t gravity;      /* 1: add Barnes-Hut self-gravity to dv/dt             */
  int32_t leaf_size;    /* tree leaves hold at most this many particles (<=32) */
  int32_t max_depth;    /* octree depth B: cell index bits per axis (<= 21)     */
  int32_t precision;    /* SPH_FP64 or SPH_MIXED                                */
  int32_t check;        /* 1: synchronise and report device errors per call    */
  double alpha, beta, eps_v;      /* artificial viscosity (Sect. 3.1.3)          */
  double eps_s, n_as, dmpd;       /* artificial stress eps_s (0: off), n, Delta mpd */
  double xsph;                    /* XSPH factor (0: off)                          */
  double G, theta, eps_grav;      /* gravity constant; opening angle; softening/h  */
  double c_courant, c_accel, c_quantity;          /* time step factors (Sect. 3.4.1) */
  double u_floor, S_floor, dmg_floor, dt_max, dt_fixed;
  double n_des;         /* > 0: sph_step adapts h at the start of each step to
                           about n_des partners (sph_adapt_h, Sect. 4.2)      */
  int32_t h_tol, h_iter;  /* its count tolerance and most updates (<= 64)     */
  int32_t tree_reuse;     /* sph_step: > 0 lets the tree built at a step start
                             serve every evaluation of this many consecutive
                             steps (gravity from its pseudo-particles: the
                             gravity/hydro decoupling of Sect. 6.3; partners stay
                             exact, refined from the build step's walk
                             while the displacement bound allows, see
                             sph_tuning); the state is reordered only at a
                             build.  0: with gravity, a tree per evaluation;
                             without, a tree per step.  Variable h builds
                             every step; each call starts with a build,
                             unless tree_continue.                          */
  int32_t tree_continue;  /* sph_step with tree_reuse > 0: 1 continues the
                             window of R steps that the previous call on the
                             context left (its age, tree, partner lists and
                             displacement bound), so a window may span calls.
                             The state must hold the positions and h that
                             call returned, in the same slots (as after
                             copying the state out and back); the call checks
                             them bit for bit (blocking on the stream) and
                             returns SPH_ERR_INVALID if they differ or if
                             another call used the context in between.
                             Ignored when tree_reuse = 0 or n_des > 0.      */
} sph_params;

/* Particle state (device pointers).  S and dmg may be NULL.  Flaw thresholds
 * of particle a are flaw_eps[flaw_off[id[a]] .. flaw_off[id[a]+1]) (FP32,
 * ascending; Sect. 3.2), so flaws need not move when particles are reordered.
 * Instances: ninst >= 1; when ninst > 1, inst_off[0..ninst] (device, int64)
 * delimits independent problems that never interact; they must be listed in
 * particle order and stay contiguous (reordering keeps them so). */
typedef struct {
  int32_t dim;
  int32_t ninst;
  int64_t n;
  double *x[3];
  double *v[3];
  double *rho, *u, *m, *h;
  double *S, *dmg;
  int32_t *mat, *id;
  const int64_t *flaw_off;
  const float *flaw_eps;
  const int64_t *inst_off;
} sph_state;

/* Time derivatives (device pointers; optional ones may be NULL). */
typedef struct {
  double *dx[3];     /* dx/dt: v plus the XSPH term                        */
  double *dv[3];     /* dv/dt, gravity included                             */
  double *drho;      /* d rho/dt (0 in density-sum mode)                     */
  double *du;        /* du/dt                                                */
  double *dS;        /* dS/dt, component-major like S                        */
  double *ddmg;      /* d(d^1/3)/dt                                          */
  double *cs;        /* optional: sound speed                               */
  double *p;         /* optional: pressure                                  */
  int32_t *n_act;    /* optional: activated flaws                           */
  int32_t *nnb;      /* optional: number of interaction partners            */
} sph_derivs;

typedef struct sph_ctx sph_ctx;

/* Launch shapes and walk granularity of a context.  None of them changes a
 * result: the partner set, the sums and their order are the same for every
 * value.  walk_leaf: the partner walk stops descending at nodes of at most
 * this many particles and tests their whole particle range (8..1024).
 * walk_blocks_per_sm: resident blocks per SM of the persistent walk grids
 * (1..32).  pass_threads: threads per block of the neighbour passes (64 or 128).
 * walk_every_eval: 0 (default) lets the evaluations that reuse a tree take
 * their partners from the last walk on it (within one sph_step or
 * sph_step_rk3 step, the step's first walk; across the steps that share a
 * tree under tree_reuse, the walk of the step that built it), which also
 * records each particle's candidates with (1 - 1/64) h_ab <= r_ab <
 * (1 + 1/64) h_ab (only those are tested again), as long as the
 * summed bound on the largest per-axis displacement of any particle since
 * that walk is at most h_a / (256 sqrt D) for every particle a and no
 * particle has more than 24 such candidates (else they walk); the lists are
 * the same either way.  1 walks the tree at every evaluation
 * (Sect. 3.5.2 as printed).  iter_cap: 0 (default) bounds each tree walk
 * (partner search and gravity) by the number of tree nodes and each find of
 * the friends-of-friends union by 2^24 pointer steps; a positive value lowers
 * both bounds to iter_cap.  A walk or find that reaches its bound stops and
 * the call returns SPH_ERR_TIMEOUT; a positive value exists to make that
 * happen on purpose (tests of the timeout report).  plain_forms: 0 (default)
 * lets the predictor-corrector update write the FP32 views of the state it
 * produces on a kept tree, and the mixed Barnes-Hut walk read its node's skip,
 * level and leaf flag packed into one word (while the node capacity fits 26
 * bits); 1 packs the views in a separate launch at every evaluation and reads
 * the node records unpacked.  Results are the same bit for bit either way; 1
 * exists to test that. */
typedef struct {
  int32_t walk_leaf;
  int32_t walk_blocks_per_sm;
  int32_t pass_threads;
  int32_t walk_every_eval;
  int32_t iter_cap;
  int32_t plain_forms;
} sph_tuning;

/* Creates a context for up to max_particles particles in up to
 * max_instances instances, max_neighbours partners per particle and tree
 * leaves of up to leaf_size (1..32) particles; allocates all scratch on the
 * current device.  Returns SPH_ERR_INVALID for bad sizes, SPH_ERR_CUDA when
 * the allocation fails (ctx is then NULL). */
sph_status sph_create(sph_ctx **ctx, int32_t dim, int64_t max_particles, int32_t max_instances,
                      int32_t max_neighbours, int32_t leaf_size, void *stream);
void sph_destroy(sph_ctx *ctx);
/* Text of the last error on this context (static storage of the context). */
const char *sph_last_error(const sph_ctx *ctx);
/* Waits for `stream`, reads and clears the device error word. */
sph_status sph_sync_status(sph_ctx *ctx, void *stream);
/* Bytes of device memory the context holds. */
int64_t sph_ctx_bytes(const sph_ctx *ctx);

/* Octree of Sect. 3.5.1 over the state: root cube per instance (lower corner
 * at the per-axis minimum, edge s0 = max extent * (1 + 2^-20)), particles
 * ordered by Morton key of the cell index floor((x - min)/s0 * 2^B), nodes
 * = every cell whose parent holds more than leaf_size particles (leaves: at
 * most leaf_size particles, or depth B).  Node mass and centre of mass.
 * reorder = 1 permutes every state array in place into that order (the
 * flaws stay indexed by id).  perm (device int32[n], may be NULL) receives,
 * for each sorted slot, the state index (before any reorder). */
sph_status sph_build_tree(sph_ctx *ctx, sph_state *state, int32_t leaf_size, int32_t max_depth, int32_t reorder,
                          int32_t *perm, void *stream);

/* Copies the tree of the last sph_build_tree out (device buffers, capacity
 * `cap` nodes, pre-order): level, cell index at that level (3 int64 per node,
 * instance bits stripped), particle count, mass, centre of mass (3 per node).
 * *nnodes (host) receives the node count; returns SPH_ERR_CAPACITY if > cap.
 * Blocks on `stream`. */
sph_status sph_tree_nodes(sph_ctx *ctx, int64_t cap, int32_t *level, int64_t *cell, int64_t *count, double *mass,
                          double *com, int64_t *nnodes, void *stream);

/* Interaction partners (Sect. 3.5.2): N(a) = {b != a, same instance :
 * ((dx^2 + dy^2) + dz^2) < h_ab^2} evaluated exactly in FP64 (no fused
 * multiply-add).  Builds the tree itself (no reorder).  Writes CSR lists in
 * state order, ascending within a particle: nb_offset (device int64[n+1]),
 * nb_index (device int32[nb_capacity]).  Returns SPH_ERR_CAPACITY if a
 * particle has more than max_neighbours partners or the total exceeds
 * nb_capacity (checked by blocking on `stream`). */
sph_status sph_neighbours(sph_ctx *ctx, const sph_state *state, int32_t leaf_size, int32_t max_depth,
                          int64_t *nb_offset, int32_t *nb_index, int64_t nb_capacity, void *stream);

/* Bytes of the fixed device scratch behind sph_neighbours_static (64 MiB). */
#define SPH_STATIC_SCRATCH_BYTES (64LL << 20)

/* sph_neighbours without a context, for callers that may not allocate
 * device memory: a plug-in whose host application owns the device memory
 * and hands libraries only the buffers they work on, or a real-time loop
 * with a memory budget fixed at start-up, where cudaMalloc can fail or
 * cudaFree would stall every stream of the device.  The paper has no
 * counterpart; this is a packaging of the partner search above.
 *
 * Same state, leaf_size, max_depth, outputs (nb_offset, nb_index,
 * nb_capacity), partner lists and error codes as sph_neighbours, with
 * max_neighbours the per-particle limit a context would hold.  The tree,
 * packed positions and partner columns live in one array of
 * SPH_STATIC_SCRATCH_BYTES bytes inside the library's device code; every
 * device that loads the library holds it until the process exits.  A call
 * needs about 600 + 4 * max_neighbours bytes per particle and at least
 * 1 MiB, so the array holds about 60 000 particles at max_neighbours = 128;
 * larger n returns SPH_ERR_CAPACITY, before touching the device, with a
 * message that gives the bytes needed.  The call itself allocates nothing:
 * no cudaMalloc, cudaFree or other allocating routine.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the life
 * of the process; make that first call before any stream capture.  After
 * cudaDeviceReset the array may move: calls after a reset are not supported.  All calls on a device share the
 * array and it keeps the last call's contents (each call clears its own error
 * word): calls whose work overlaps on the GPU, from two streams or two host
 * threads, race and corrupt each other's results, so serialise them.  Blocks
 * on `stream` at the end to read the error word.  msg (host, msg_len bytes,
 * may be NULL) receives the error message, or "" on success. */
sph_status sph_neighbours_static(const sph_state *state, int32_t leaf_size, int32_t max_depth,
                                 int32_t max_neighbours, int64_t *nb_offset, int32_t *nb_index,
                                 int64_t nb_capacity, char *msg, int32_t msg_len, void *stream);

/* Variable smoothing length (Sect. 4.2, after Hernquist & Katz): starting
 * from state->h, every particle's support radius is replaced by
 * h (1 + (n_des / n_a)^(1/D)) / 2, with n_a = #{b != a in a's instance :
 * ((dx^2 + dy^2) + dz^2) < h_a^2} evaluated exactly in FP64 (the particle's
 * own h), all particles at once, until every |n_a - n_des| <= tol or
 * max_iter (<= 64) updates have been made; n_a = 0 doubles h.  state->h is
 * updated in place.  counts (device int32[n], may be NULL) receives n_a of the
 * last count; *updates (host, may be NULL) the number of updates made.  Builds
 * the tree itself (no reorder); blocks on `stream` at the end. */
sph_status sph_adapt_h(sph_ctx *ctx, sph_state *state, int32_t leaf_size, int32_t max_depth, double n_des,
                       int32_t tol, int32_t max_iter, int32_t *counts, int32_t *updates, void *stream);

/* One right-hand side: tree, partners, (density sum), the neighbour pass for
 * continuity / velocity gradient / XSPH, the per-particle constitutive update
 * (EOS, Hooke + Jaumann, yield, damage, artificial stress), the momentum and
 * energy pass, and gravity if params->gravity.  In density-sum mode rho is
 * overwritten with the kernel sum.  mats: host array of nmat materials
 * indexed by state->mat. */
sph_status sph_rhs(sph_ctx *ctx, sph_state *state, const sph_material *mats, int32_t nmat, const sph_params *params,
                   sph_derivs *out, void *stream);

/* Barnes-Hut self-gravity alone (Sect. 3.3): a_a = -G sum m_p (x_a - x_p) /
 * (r^2 + eps_a^2)^1.5, eps_a = eps_grav h_a; a node is a pseudo-particle when
 * s/r < theta and its cube does not contain a.  theta = 0 gives the direct
 * sum.  Builds the tree itself (no reorder).  Writes ax, ay, az (device; az
 * ignored in 2D). */
sph_status sph_gravity(sph_ctx *ctx, const sph_state *state, const sph_params *params, double *ax, double *ay,
                       double *az, void *stream);

/* nsteps predictor-corrector steps (Sect. 3.4.1) in place:
 *   q^p = q + dt/2 dq/dt(q),  q^c = q + dt dq/dt(q^p)
 * for x, v, rho (continuity mode), u, S, d^1/3, then S <- f_Y S and the
 * damage cap.  dt per instance = params->dt_fixed if > 0, else the minimum of
 * the Courant, acceleration and quantity limits, computed on the device.
 * dt (device double[ninst], may be NULL) receives the last step's time
 * steps.  At the start of every step the state is reordered along the
 * octree, so particle order changes; id follows the particles. */
sph_status sph_step(sph_ctx *ctx, sph_state *state, const sph_material *mats, int32_t nmat, const sph_params *params,
                    double *dt, int32_t nsteps, void *stream);

/* Embedded Runge-Kutta steps with adaptive step size (Sect. 3.4.2), nsteps
 * attempts: k1 = f(q), k2 = f(q + dt/2 k1), k3 = f(q - dt k1 + 2 dt k2) with
 * each stage state limited as in the predictor-corrector (yield, damage
 * cap); per instance the error estimate is the largest
 * dt |2 k2 - k1 - k3| / 6 / (|q + dt k1| + floor) over its particles and
 * integrated components (floors: h for positions, c_s of k1 for velocities,
 * 0 for rho, params u_floor, S_floor, dmg_floor), the difference of the
 * midpoint and third-order values relative to the Euler value.  err < eps_des
 * accepts q + dt (k1 + 4 k2 + k3)/6 (limited) and sets dt <- dt
 * (eps_des/err)^0.3 (dt_max for err = 0); otherwise the instance keeps its
 * state and dt <- 0.9 dt (eps_des/err)^(1/4); dt <= dt_max.
 * dt: device double[ninst], in/out (<= 0: start from the predictor-corrector
 * limit of k1); t (device double[ninst], may be NULL) += dt of accepted steps;
 * err_log, acc_log (device double / int32 [nsteps][ninst], may be NULL).
 * State reordered along the tree as in sph_step.  Variable h (params.n_des)
 * as in sph_step. */
sph_status sph_step_rk3(sph_ctx *ctx, sph_state *state, const sph_material *mats, int32_t nmat,
                        const sph_params *params, double eps_des, double *dt, double *t, int32_t nsteps,
                        double *err_log, int32_t *acc_log, void *stream);

/* Weibull activation thresholds (Sect. 3.2, after Benz & Asphaug): the
 * brittle particles (mats[mat].damage set, weibull_k[mat] > 0 and
 * weibull_m[mat] > 0) of each instance and material form a group of N
 * particles, listed by ascending id, with volume V = sum m / rho0.  Flaw
 * j = 1, 2, ... goes to member floor(w_j N / 2^64) with threshold strain
 * (j / (k V))^(1/m), until every member holds one; w_j is word (j-1) mod 4
 * of the Philox4x64-10 block (Salmon et al. 2011) with counter
 * ((j-1)/4, 0, 0, 0) and key (seed, instance * nmat + material).
 * state: n, ninst/inst_off, mat, id (a permutation of 0..n-1) and m are
 * read.  weibull_k, weibull_m: host double[nmat].
 * flaw_off: device int64[n+1] (may be NULL: count only), CSR offsets by id,
 * as sph_state.flaw_off expects; flaw_eps: device float[eps_capacity] (may
 * be NULL), thresholds ascending per particle.  *nflaws (host) receives
 * the total.  Blocking.  SPH_ERR_CAPACITY when the total exceeds
 * eps_capacity (offsets and *nflaws are still written) or 2^31;
 * SPH_ERR_INVALID for an id or material index out of range.  The result
 * depends only on seed and the state, not on the particle order within an
 * instance; it equals the sequential procedure's up to the rounding of V
 * (a sum in a different order) and of pow. */
sph_status sph_flaws(sph_ctx *ctx, const sph_state *state, const sph_material *mats, int32_t nmat,
                     const double *weibull_k, const double *weibull_m, uint64_t seed, int64_t *flaw_off,
                     float *flaw_eps, int64_t eps_capacity, int64_t *nflaws, void *stream);

/* Fragments by friends-of-friends (Sect. 4, fragment analysis of an
 * impact): particles with dmg >= d_remove are removed (state.dmg NULL:
 * none); two remaining particles of one instance are friends when
 * r_ab^2 < ((h'_a + h'_b)/2)^2 with h' = link * h0 (the partner rule of
 * sph_neighbours at smoothing lengths h'; the paper links at 1.01 times the
 * original smoothing length); fragments are the connected components with
 * at least min_size particles (the paper drops those below 3), numbered by
 * decreasing particle count, ties by smallest member index.
 * h0: device double[n], the original smoothing lengths (NULL: state.h).
 * label: device int32[n], fragment number or -1 (removed, or in a smaller
 * component).  frag_count (int32), frag_mass (double, sum of m): device
 * arrays of frag_capacity entries (may be NULL); masses are summed with
 * atomics, so their last bits may differ between runs.  *nfrag (host)
 * receives the number of fragments.  Blocking.  Uses the context's partner
 * lists: SPH_ERR_CAPACITY when a particle has more than max_neighbours
 * friends, or more fragments than frag_capacity (labels and *nfrag are
 * complete then). */
sph_status sph_fragments(sph_ctx *ctx, const sph_state *state, const double *h0, double link, double d_remove,
                         int32_t min_size, int32_t leaf_size, int32_t max_depth, int32_t *label,
                         int32_t *frag_count, double *frag_mass, int64_t frag_capacity, int64_t *nfrag,
                         void *stream);

/* Reverse-mode derivative of sph_rhs at `state`, with the partner lists and
 * the damage of
 * that evaluation held fixed and every branch (artificial viscosity on/off,
 * yield on/off, EOS branch, C = I fallback) at its forward side.  Given the
 * cotangents dbar of the outputs dx/dt, dv/dt, drho/dt, du/dt, dS/dt (device,
 * layout of sph_derivs; NULL entries count as zero), it ADDS the cotangents of
 * x, v, rho, u and S to the matching arrays of `state_bar` (device, layout of
 * sph_state; its other fields are ignored) and ADDS to param_bar (device,
 * ninst * nmat * 3 doubles, may be NULL) the cotangents of the shear modulus
 * mu, the yield stress Y0 and the bulk modulus K of each material and
 * instance; K scales K0, A_T and B_T together and is measured in units of the
 * largest of them.  Requires continuity density, no artificial stress and no
 * gravity (SPH_ERR_INVALID otherwise).  Builds the tree and partners itself.
 * Precision: SPH_FP64 evaluates the forward pass and every derivative in
 * FP64; SPH_MIXED evaluates the forward pass in mixed precision and the pair
 * terms of the derivative in FP32 (in the power-of-two code units of the
 * forward pass, on hi/lo position and velocity differences, compensated sums),
 * and the constitutive reverse in FP32: the forward pass A's own sums, the
 * equation of state differentiated exactly by one dual-number evaluation, the
 * rest in SI units with each particle's cotangents scaled by a power of two
 * (within ~3e-6 of the FP64 form, which takes the derivatives of c_s and of
 * the bulk scale by central differences). */
sph_status sph_rhs_adjoint(sph_ctx *ctx, sph_state *state, const sph_material *mats, int32_t nmat,
                           const sph_params *params, const sph_derivs *dbar, sph_state *state_bar, double *param_bar,
                           void *stream);

/* One predictor or corrector update without reordering (Sect. 3.4.1):
 * out = Y(base + frac * dt * d) for x, v, rho (continuity), u and S, Y the von
 * Mises limiter, damage and its cap as in sph_step.  dt: device, one per
 * instance.  out may alias base. */
sph_status sph_pc_update(sph_ctx *ctx, const sph_state *base, const sph_derivs *d, const sph_material *mats,
                         int32_t nmat, const sph_params *params, const double *dt, double frac, sph_state *out,
                         void *stream);

/* Reverse of sph_pc_update with damage held fixed: given the cotangent of
 * out (out_bar: x, v, rho, u, S), ADDS the cotangent of base to base_bar,
 * WRITES frac * dt times the pre-limiter cotangent to d_bar (dx, dv, drho,
 * du, dS) and ADDS the yield-stress cotangent to param_bar (as in
 * sph_rhs_adjoint; may be NULL).  out_bar must not alias base_bar. */
sph_status sph_pc_update_adjoint(sph_ctx *ctx, const sph_state *base, const sph_derivs *d,
                                 const sph_material *mats, int32_t nmat, const sph_params *params, const double *dt,
                                 double frac, const sph_state *out_bar, sph_state *base_bar, sph_derivs *d_bar,
                                 double *param_bar, void *stream);

/* Reads / replaces the tuning of a context (defaults: 64, 16, 128, 0). */
sph_status sph_get_tuning(const sph_ctx *ctx, sph_tuning *out);
sph_status sph_set_tuning(sph_ctx *ctx, const sph_tuning *t);

/* Optional per-phase timing.  When enabled, every phase of sph_rhs and
 * sph_step is bracketed by CUDA events recorded on the call's stream (at most
 * 8192 phases between reads; later ones go untimed).  Phases, in order:
 * 0 tree build, 1 state reorder, 2 partner search (tree walk), 3 density sum,
 * 4 neighbour pass A with the constitutive update, 5 momentum/energy pass B,
 * 6 gravity, 7 integrator (time step and updates), 8 flaw draws and 9 flaw
 * thresholds (sph_flaws), 10 friends-of-friends links (sph_fragments),
 * 11 partners refined from the step's first walk (see walk_every_eval). */
sph_status sph_profile_enable(sph_ctx *ctx, int32_t on);
/* Milliseconds and call counts per phase since the last read (nphase
 * entries of each); synchronises on the recorded events, then resets. */
sph_status sph_profile_read(sph_ctx *ctx, double *ms, int32_t *calls, int32_t nphase);
/* Interaction counters summed on the device by the walks that ran while the
 * profiler was enabled (since it was enabled or last read), for the
 * instruction and FP32 rooflines of the walks: 0 nodes used as
 * pseudo-particles by the Barnes-Hut walk (Sect. 3.3), 1 particle-particle
 * terms it summed, 2 tree nodes its warps visited, 3 candidates the partner
 * walk (Sect. 3.5.2) tested against the partner predicate, 4 partners it
 * found.  Writes n entries of `out` (host int64; entries beyond 5 are 0),
 * blocking on `stream`, then resets the counters. */
sph_status sph_profile_counters(sph_ctx *ctx, int64_t *out, int32_t n, void *stream);
/* Number of kernels this library has launched in this process. */
int64_t sph_launch_count(void);

/* Peak FMA throughput of this device, measured by a register-resident loop
 * (precision SPH_FP64 or SPH_MIXED = FP32); returns FLOP/s (2 per FMA) in
 * *flops.  Blocks. */
sph_status sph_measure_fma_peak(int32_t precision, double *flops);

#ifdef __cplusplus
}
#endif
#endif
