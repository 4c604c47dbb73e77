/*
 * FP64 CPU oracle of the solid-body SPH right-hand side and predictor-corrector
 * step of Schaefer et al. (2016), "A smooth particle hydrodynamics code to model
 * collisions between solid, self-gravitating objects".
 *
 * TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file's library; the product path
 * never does.  No code is shared with the CUDA library.
 *
 * Plain and slow on purpose: every particle loops over its neighbours in
 * ascending index order, every formula is written as the paper states it
 * (with the readings listed next to the code where the paper is silent or
 * misprinted), everything is double precision, and the build uses
 * -ffp-contract=off.  OpenMP only splits the outer loop over particles.
 *
 * Parity pins: every function here is checked in tests/test_oracle_*.py
 * against closed forms, invariants, brute force or an independent library
 * routine; none is "parity unpinned".
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static int g_threads = 1;
void orc_set_threads(int32_t t) { g_threads = t < 1 ? 1 : t; }
int32_t orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* Symmetric tensor storage: 3D (xx, yy, zz, xy, xz, yz), 2D (xx, yy, xy).    */
/* ------------------------------------------------------------------------ */
static int nsym(int dim) { return dim == 3 ? 6 : 3; }

static int symk(int dim, int a, int b) {
  if (a == b) return a;
  if (dim == 2) return 2;
  if ((a == 0 && b == 1) || (a == 1 && b == 0)) return 3;
  if ((a == 0 && b == 2) || (a == 2 && b == 0)) return 4;
  return 5;
}

static void sym_load(int dim, const double *S, int64_t n, int64_t a, double M[3][3]) {
  memset(M, 0, 9 * sizeof(double));
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j) M[i][j] = S[(int64_t)symk(dim, i, j) * n + a];
}

static void sym_store(int dim, double M[3][3], double *S, int64_t n, int64_t a) {
  for (int i = 0; i < dim; ++i)
    for (int j = i; j < dim; ++j) S[(int64_t)symk(dim, i, j) * n + a] = M[i][j];
}

/* ------------------------------------------------------------------------ */
/* Cubic B-spline kernel, Sect. 3.1.1.  h is the support radius: W = 0 for   */
/* r > h.  Normalisation s = 4/3, 40/(7 pi), 8/pi for D = 1, 2, 3.           */
/* ------------------------------------------------------------------------ */
static double kernel_norm(int dim) {
  if (dim == 1) return 4.0 / 3.0;
  if (dim == 2) return 40.0 / (7.0 * M_PI);
  return 8.0 / M_PI;
}

static double hpow(double h, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r = r * h;
  return r;
}

double orc_W(double r, double h, int32_t dim) {
  double q = r / h;
  double f = kernel_norm(dim) / hpow(h, dim);
  if (q < 0.5) return f * (6.0 * q * q * q - 6.0 * q * q + 1.0);
  if (q <= 1.0) return f * 2.0 * (1.0 - q) * (1.0 - q) * (1.0 - q);
  return 0.0;
}

double orc_dWdr(double r, double h, int32_t dim) {
  double q = r / h;
  double g = 6.0 * kernel_norm(dim) / hpow(h, dim + 1);
  if (q < 0.5) return g * (3.0 * q * q - 2.0 * q);
  if (q <= 1.0) return -g * (1.0 - q) * (1.0 - q);
  return 0.0;
}

/* ------------------------------------------------------------------------ */
/* Interaction partners, Sect. 3.5.2: b is a partner of a if b != a and      */
/* r_ab < h_ab, with h_ab = (h_a + h_b)/2 (Sect. 4.2, mean smoothing length; */
/* equal to h for a uniform h).  The distance is squared in a fixed order,   */
/* ((dx dx + dy dy) + dz dz), and compared with h_ab * h_ab.                 */
/* ------------------------------------------------------------------------ */
static int is_partner(int dim, const double *x, const double *y, const double *z, const double *h,
                      int64_t a, int64_t b) {
  double dx = x[a] - x[b];
  double dy = y[a] - y[b];
  double r2 = dx * dx + dy * dy;
  if (dim == 3) {
    double dz = z[a] - z[b];
    r2 = r2 + dz * dz;
  }
  double hab = 0.5 * (h[a] + h[b]);
  return r2 < hab * hab;
}

int32_t orc_neighbours_one(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                           const double *h, int64_t a, int32_t *out, int32_t cap) {
  int32_t c = 0;
  for (int64_t b = 0; b < n; ++b) {
    if (b == a || !is_partner(dim, x, y, z, h, a, b)) continue;
    if (c < cap) out[c] = (int32_t)b;
    ++c;
  }
  return c;
}

int64_t orc_neighbours_brute(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                             const double *h, int64_t *off, int32_t *idx, int64_t cap) {
  off[0] = 0;
  for (int64_t a = 0; a < n; ++a) {
    int64_t c = 0;
    for (int64_t b = 0; b < n; ++b)
      if (b != a && is_partner(dim, x, y, z, h, a, b)) ++c;
    off[a + 1] = off[a] + c;
  }
  if (off[n] > cap) return -1;
  for (int64_t a = 0; a < n; ++a) {
    int64_t c = off[a];
    for (int64_t b = 0; b < n; ++b)
      if (b != a && is_partner(dim, x, y, z, h, a, b)) idx[c++] = (int32_t)b;
  }
  return off[n];
}

/* Cell list with cells no smaller than max h: the same partner definition,  */
/* candidates restricted to the 3^D surrounding cells.                       */
typedef struct {
  int dim;
  int64_t nc[3];
  double lo[3], cell;
  int64_t *start; /* ncell + 1 */
  int64_t *items; /* particles sorted by cell, ascending index within a cell */
} cellgrid;

static int64_t grid_coord(const cellgrid *g, int ax, double v) {
  int64_t c = (int64_t)floor((v - g->lo[ax]) / g->cell);
  if (c < 0) c = 0;
  if (c >= g->nc[ax]) c = g->nc[ax] - 1;
  return c;
}

static void grid_build(cellgrid *g, int dim, int64_t n, const double *x, const double *y, const double *z,
                       const double *h) {
  const double *X[3] = {x, y, z};
  double hmax = 0.0, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int ax = 0; ax < dim; ++ax) {
    lo[ax] = hi[ax] = n > 0 ? X[ax][0] : 0.0;
  }
  for (int64_t a = 0; a < n; ++a) {
    if (h[a] > hmax) hmax = h[a];
    for (int ax = 0; ax < dim; ++ax) {
      if (X[ax][a] < lo[ax]) lo[ax] = X[ax][a];
      if (X[ax][a] > hi[ax]) hi[ax] = X[ax][a];
    }
  }
  g->dim = dim;
  g->cell = hmax > 0 ? hmax : 1.0;
  for (;;) {
    double ncell = 1.0;
    for (int ax = 0; ax < 3; ++ax) {
      g->nc[ax] = ax < dim ? (int64_t)floor((hi[ax] - lo[ax]) / g->cell) + 1 : 1;
      ncell *= (double)g->nc[ax];
    }
    if (ncell <= 4.0 * (double)n + 64.0) break;
    g->cell *= 2.0;
  }
  for (int ax = 0; ax < 3; ++ax) g->lo[ax] = ax < dim ? lo[ax] : 0.0;
  int64_t ncell = g->nc[0] * g->nc[1] * g->nc[2];
  g->start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
  g->items = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t *cid = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  for (int64_t a = 0; a < n; ++a) {
    int64_t c[3] = {0, 0, 0};
    for (int ax = 0; ax < dim; ++ax) c[ax] = grid_coord(g, ax, X[ax][a]);
    cid[a] = (c[2] * g->nc[1] + c[1]) * g->nc[0] + c[0];
    g->start[cid[a] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) g->start[c + 1] += g->start[c];
  int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t) + 8);
  memcpy(fill, g->start, (size_t)ncell * sizeof(int64_t));
  for (int64_t a = 0; a < n; ++a) g->items[fill[cid[a]]++] = a;
  free(fill);
  free(cid);
}

static void grid_free(cellgrid *g) {
  free(g->start);
  free(g->items);
}

static int cmp_i32(const void *p, const void *q) {
  int32_t a = *(const int32_t *)p, b = *(const int32_t *)q;
  return (a > b) - (a < b);
}

/* Partners of a from the grid, sorted ascending; returns the count (writes at
 * most cap entries). */
static int64_t grid_partners(const cellgrid *g, const double *x, const double *y, const double *z,
                             const double *h, int64_t a, int32_t *out, int64_t cap) {
  const double *X[3] = {x, y, z};
  int dim = g->dim;
  int64_t c0[3] = {0, 0, 0};
  for (int ax = 0; ax < dim; ++ax) c0[ax] = grid_coord(g, ax, X[ax][a]);
  int64_t cnt = 0;
  int zr = dim == 3 ? 1 : 0;
  for (int64_t dz = -zr; dz <= zr; ++dz)
    for (int64_t dy = -1; dy <= 1; ++dy)
      for (int64_t dx = -1; dx <= 1; ++dx) {
        int64_t cx = c0[0] + dx, cy = c0[1] + dy, cz = c0[2] + dz;
        if (cx < 0 || cy < 0 || cz < 0 || cx >= g->nc[0] || cy >= g->nc[1] || cz >= g->nc[2]) continue;
        int64_t c = (cz * g->nc[1] + cy) * g->nc[0] + cx;
        for (int64_t k = g->start[c]; k < g->start[c + 1]; ++k) {
          int64_t b = g->items[k];
          if (b == a || !is_partner(dim, x, y, z, h, a, b)) continue;
          if (cnt < cap) out[cnt] = (int32_t)b;
          ++cnt;
        }
      }
  if (cnt <= cap) qsort(out, (size_t)cnt, sizeof(int32_t), cmp_i32);
  return cnt;
}

int64_t orc_neighbours_grid(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                            const double *h, int64_t *off, int32_t *idx, int64_t cap) {
  cellgrid g;
  grid_build(&g, dim, n, x, y, z, h);
  int64_t *cnt = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
#pragma omp parallel num_threads(g_threads)
  {
    int32_t *tmp = (int32_t *)malloc(4096 * sizeof(int32_t));
#pragma omp for schedule(static)
    for (int64_t a = 0; a < n; ++a) cnt[a] = grid_partners(&g, x, y, z, h, a, tmp, 0);
    free(tmp);
  }
  off[0] = 0;
  for (int64_t a = 0; a < n; ++a) off[a + 1] = off[a] + cnt[a];
  int64_t total = off[n];
  if (total <= cap) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t a = 0; a < n; ++a) grid_partners(&g, x, y, z, h, a, idx + off[a], cnt[a]);
  }
  free(cnt);
  grid_free(&g);
  return total <= cap ? total : -1;
}

/* ------------------------------------------------------------------------ */
/* Variable smoothing length, Sect. 4.2 (after Hernquist & Katz 1989): every */
/* particle's h is replaced by h (1 + (n_des / n_a)^(1/D)) / 2, where n_a is  */
/* the number of other particles of its instance closer than its own h,      */
/* ((dx dx + dy dy) + dz dz) < h_a h_a; all particles at once, repeated until */
/* every |n_a - n_des| <= tol or max_iter updates have been made.  A particle */
/* without partners doubles its h.  Returns the number of updates; counts    */
/* receives n_a of the last count.                                           */
/* ------------------------------------------------------------------------ */
static int within_own_h(int dim, const double *x, const double *y, const double *z, const double *h, int64_t a,
                        int64_t b) {
  double dx = x[a] - x[b];
  double dy = y[a] - y[b];
  double r2 = dx * dx + dy * dy;
  if (dim == 3) {
    double dz = z[a] - z[b];
    r2 = r2 + dz * dz;
  }
  return r2 < h[a] * h[a];
}

/* n_a for every particle of one instance (arrays offset to its first particle) */
static void count_own_h(int dim, int64_t n, const double *x, const double *y, const double *z, const double *h,
                        int32_t *counts) {
  if (n == 0) return;
  cellgrid g;
  grid_build(&g, dim, n, x, y, z, h); /* cells no smaller than max h >= h_a */
  const double *X[3] = {x, y, z};
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t a = 0; a < n; ++a) {
    int64_t c0[3] = {0, 0, 0};
    for (int ax = 0; ax < dim; ++ax) c0[ax] = grid_coord(&g, ax, X[ax][a]);
    int32_t cnt = 0;
    int zr = dim == 3 ? 1 : 0;
    for (int64_t dz = -zr; dz <= zr; ++dz)
      for (int64_t dy = -1; dy <= 1; ++dy)
        for (int64_t dx = -1; dx <= 1; ++dx) {
          int64_t cx = c0[0] + dx, cy = c0[1] + dy, cz = c0[2] + dz;
          if (cx < 0 || cy < 0 || cz < 0 || cx >= g.nc[0] || cy >= g.nc[1] || cz >= g.nc[2]) continue;
          int64_t c = (cz * g.nc[1] + cy) * g.nc[0] + cx;
          for (int64_t k = g.start[c]; k < g.start[c + 1]; ++k) {
            int64_t b = g.items[k];
            if (b != a && within_own_h(dim, x, y, z, h, a, b)) ++cnt;
          }
        }
    counts[a] = cnt;
  }
  grid_free(&g);
}

int32_t orc_adapt_h(int32_t dim, int64_t n, const double *x, const double *y, const double *z, double *h,
                    const int64_t *inst_off, int32_t ninst, double n_des, int32_t tol, int32_t max_iter,
                    int32_t *counts) {
  int32_t it = 0;
  if (ninst < 1 || !inst_off) ninst = 1;
  for (;;) {
    for (int32_t i = 0; i < ninst; ++i) {
      int64_t lo = ninst > 1 ? inst_off[i] : 0, hi = ninst > 1 ? inst_off[i + 1] : n;
      count_own_h(dim, hi - lo, x + lo, y + lo, z ? z + lo : NULL, h + lo, counts + lo);
    }
    int done = 1;
    for (int64_t a = 0; a < n; ++a)
      if (fabs((double)counts[a] - n_des) > (double)tol) done = 0;
    if (done || it >= max_iter) return it;
    for (int64_t a = 0; a < n; ++a) {
      if (counts[a] == 0) {
        h[a] = 2.0 * h[a];
      } else {
        double q = n_des / (double)counts[a];
        double r = dim == 3 ? cbrt(q) : (dim == 2 ? sqrt(q) : q);
        h[a] = h[a] * 0.5 * (1.0 + r);
      }
    }
    ++it;
  }
}

/* ------------------------------------------------------------------------ */
/* Octree, Sect. 3.5.1.  Root cube: lower corner at the per-axis minimum,    */
/* edge s0 = max_axis(extent) * (1 + 2^-20) so the particle at the maximum   */
/* lies inside; a node at depth d has edge s0 / 2^d.  Cell index of a        */
/* particle at full depth B: k = floor((x - min) / s0 * 2^B), clamped.  A    */
/* node with more than leaf_size particles (and depth < B) splits into its   */
/* non-empty octants, visited in the order ox + 2 oy + 4 oz.                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  double lo[3], s0;
} rootcube;

static rootcube root_cube(int dim, int64_t n, const double *x, const double *y, const double *z) {
  const double *X[3] = {x, y, z};
  rootcube rc;
  double ext = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    rc.lo[ax] = 0.0;
    if (ax >= dim || n == 0) continue;
    double lo = X[ax][0], hi = X[ax][0];
    for (int64_t a = 1; a < n; ++a) {
      if (X[ax][a] < lo) lo = X[ax][a];
      if (X[ax][a] > hi) hi = X[ax][a];
    }
    rc.lo[ax] = lo;
    if (hi - lo > ext) ext = hi - lo;
  }
  rc.s0 = ext * (1.0 + ldexp(1.0, -20));
  if (!(rc.s0 > 0.0)) rc.s0 = 1.0; /* one particle, or all coincident */
  return rc;
}

static int64_t cell_index(const rootcube *rc, int ax, double v, int B) {
  double t = (v - rc->lo[ax]) / rc->s0;
  double f = floor(ldexp(t, B));
  int64_t k = (int64_t)f;
  int64_t kmax = ((int64_t)1 << B) - 1;
  if (f < 0.0) k = 0;
  if (k > kmax) k = kmax;
  return k;
}

void orc_cell_coords(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                     int32_t max_depth, int64_t *k) {
  const double *X[3] = {x, y, z};
  rootcube rc = root_cube(dim, n, x, y, z);
  for (int64_t a = 0; a < n; ++a)
    for (int ax = 0; ax < 3; ++ax) k[3 * a + ax] = ax < dim ? cell_index(&rc, ax, X[ax][a], max_depth) : 0;
}

typedef struct {
  int level, leaf, nchild;
  int64_t cell[3];
  int64_t first, count; /* range in the tree's particle order */
  int64_t child[8];
  double mass, com[3];
} onode;

typedef struct {
  int dim, B, L;
  rootcube rc;
  int64_t n, nnodes, cap;
  onode *nodes;
  int64_t *ord; /* particle indices, grouped by node */
  int64_t *k;   /* cell indices at full depth, 3 per particle */
} otree;

static int64_t tree_new_node(otree *t) {
  if (t->nnodes == t->cap) {
    t->cap = t->cap ? 2 * t->cap : 1024;
    t->nodes = (onode *)realloc(t->nodes, (size_t)t->cap * sizeof(onode));
  }
  return t->nnodes++;
}

/* Builds node `id` over ord[first .. first+count) at `level`; children are  */
/* appended in pre-order (a node, then each child subtree in octant order).  */
static void tree_split(otree *t, int64_t id, int64_t *scratch) {
  onode *nd = &t->nodes[id];
  int level = nd->level;
  int64_t first = nd->first, count = nd->count;
  nd->nchild = 0;
  nd->leaf = (count <= t->L || level == t->B);
  if (nd->leaf) return;
  int shift = t->B - level - 1;
  int64_t bucket[8] = {0};
  for (int64_t i = first; i < first + count; ++i) {
    int64_t a = t->ord[i];
    int o = 0;
    for (int ax = 0; ax < t->dim; ++ax) o |= (int)((t->k[3 * a + ax] >> shift) & 1) << ax;
    bucket[o]++;
  }
  int64_t start[8];
  int64_t s = first;
  for (int o = 0; o < 8; ++o) {
    start[o] = s;
    s += bucket[o];
  }
  int64_t fill[8];
  memcpy(fill, start, sizeof(fill));
  for (int64_t i = first; i < first + count; ++i) {
    int64_t a = t->ord[i];
    int o = 0;
    for (int ax = 0; ax < t->dim; ++ax) o |= (int)((t->k[3 * a + ax] >> shift) & 1) << ax;
    scratch[fill[o]++] = a;
  }
  memcpy(t->ord + first, scratch + first, (size_t)count * sizeof(int64_t));
  int noct = 1 << t->dim;
  for (int o = 0; o < noct; ++o) {
    if (bucket[o] == 0) continue;
    int64_t c = tree_new_node(t);
    nd = &t->nodes[id]; /* realloc may move the array */
    onode *ch = &t->nodes[c];
    memset(ch, 0, sizeof(*ch));
    ch->level = level + 1;
    for (int ax = 0; ax < 3; ++ax) ch->cell[ax] = ax < t->dim ? 2 * nd->cell[ax] + ((o >> ax) & 1) : 0;
    ch->first = start[o];
    ch->count = bucket[o];
    nd->child[nd->nchild++] = c;
    tree_split(t, c, scratch);
    nd = &t->nodes[id];
  }
}

/* Node mass and centre of mass straight from the node's particles. */
static void tree_moments(otree *t, const double *x, const double *y, const double *z, const double *m) {
  const double *X[3] = {x, y, z};
  for (int64_t id = 0; id < t->nnodes; ++id) {
    onode *nd = &t->nodes[id];
    double M = 0.0, mx[3] = {0, 0, 0};
    for (int64_t i = nd->first; i < nd->first + nd->count; ++i) {
      int64_t a = t->ord[i];
      M += m[a];
      for (int ax = 0; ax < t->dim; ++ax) mx[ax] += m[a] * X[ax][a];
    }
    nd->mass = M;
    for (int ax = 0; ax < 3; ++ax) nd->com[ax] = (ax < t->dim && M > 0.0) ? mx[ax] / M : 0.0;
  }
}

static void tree_build(otree *t, int dim, int64_t n, const double *x, const double *y, const double *z,
                       const double *m, int L, int B) {
  memset(t, 0, sizeof(*t));
  t->dim = dim;
  t->B = B;
  t->L = L < 1 ? 1 : L;
  t->n = n;
  t->rc = root_cube(dim, n, x, y, z);
  t->k = (int64_t *)malloc((size_t)(3 * n + 3) * sizeof(int64_t));
  t->ord = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
  int64_t *scratch = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
  const double *X[3] = {x, y, z};
  for (int64_t a = 0; a < n; ++a) {
    t->ord[a] = a;
    for (int ax = 0; ax < 3; ++ax) t->k[3 * a + ax] = ax < dim ? cell_index(&t->rc, ax, X[ax][a], B) : 0;
  }
  int64_t r = tree_new_node(t);
  memset(&t->nodes[r], 0, sizeof(onode));
  t->nodes[r].first = 0;
  t->nodes[r].count = n;
  tree_split(t, r, scratch);
  free(scratch);
  if (m) tree_moments(t, x, y, z, m);
}

static void tree_free(otree *t) {
  free(t->nodes);
  free(t->ord);
  free(t->k);
}

int64_t orc_tree_nodes(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                       const double *m, int32_t leaf_size, int32_t max_depth, int64_t cap,
                       int32_t *level, int64_t *cell, int64_t *count, double *mass, double *com) {
  otree t;
  tree_build(&t, dim, n, x, y, z, m, leaf_size, max_depth);
  int64_t nn = t.nnodes;
  if (nn <= cap) {
    for (int64_t i = 0; i < nn; ++i) {
      level[i] = t.nodes[i].level;
      count[i] = t.nodes[i].count;
      if (mass) mass[i] = t.nodes[i].mass;
      for (int ax = 0; ax < 3; ++ax) {
        cell[3 * i + ax] = t.nodes[i].cell[ax];
        if (com) com[3 * i + ax] = t.nodes[i].com[ax];
      }
    }
  }
  tree_free(&t);
  return nn <= cap ? nn : -1;
}

/* ------------------------------------------------------------------------ */
/* Self-gravity, Sect. 3.3, Eq. (gravitational_force), read as attractive   */
/* and Plummer-softened: a_a = -G sum_p m_p (x_a - x_p) / (r^2 + eps_a^2)^1.5 */
/* with eps_a = eps_grav * h_a.                                              */
/* ------------------------------------------------------------------------ */
static void grav_term(int dim, const double xa[3], const double xp[3], double mp, double eps2, double G,
                      double acc[3]) {
  double d[3] = {0, 0, 0};
  double r2 = 0.0;
  for (int ax = 0; ax < dim; ++ax) {
    d[ax] = xa[ax] - xp[ax];
    r2 = r2 + d[ax] * d[ax];
  }
  double q = r2 + eps2;
  if (!(q > 0.0)) return; /* coincident and unsoftened: no defined direction */
  double inv = 1.0 / (q * sqrt(q));
  for (int ax = 0; ax < dim; ++ax) acc[ax] -= G * mp * d[ax] * inv;
}

void orc_gravity_direct(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                        const double *m, const double *h, double G, double eps_grav,
                        double *ax, double *ay, double *az) {
  const double *X[3] = {x, y, z};
  double *A[3] = {ax, ay, az};
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t a = 0; a < n; ++a) {
    double xa[3] = {0, 0, 0}, acc[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) xa[k] = X[k][a];
    double e = eps_grav * h[a];
    for (int64_t b = 0; b < n; ++b) {
      if (b == a) continue;
      double xb[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) xb[k] = X[k][b];
      grav_term(dim, xa, xb, m[b], e * e, G, acc);
    }
    for (int k = 0; k < dim; ++k) A[k][a] = acc[k];
  }
}

/* Barnes-Hut walk for particle a.  A node is used as a pseudo-particle when */
/* its edge s satisfies s / r < theta (evaluated as s < theta * r, r the     */
/* distance to the node's centre of mass) and its cube does not contain a;   */
/* otherwise a leaf is summed particle by particle (self skipped) and an     */
/* inner node is opened.                                                     */
static void bh_walk(const otree *t, int64_t id, int64_t a, const int64_t ka[3], const double *const X[3],
                    const double *m, double G, double theta, double eps2, double acc[3]) {
  const onode *nd = &t->nodes[id];
  int dim = t->dim;
  int inside = 1;
  for (int ax = 0; ax < dim; ++ax)
    if ((ka[ax] >> (t->B - nd->level)) != nd->cell[ax]) inside = 0;
  double xa[3] = {0, 0, 0};
  for (int ax = 0; ax < dim; ++ax) xa[ax] = X[ax][a];
  if (!inside) {
    double r2 = 0.0;
    for (int ax = 0; ax < dim; ++ax) {
      double d = xa[ax] - nd->com[ax];
      r2 = r2 + d * d;
    }
    double s = ldexp(t->rc.s0, -nd->level);
    if (s < theta * sqrt(r2)) {
      grav_term(dim, xa, nd->com, nd->mass, eps2, G, acc);
      return;
    }
  }
  if (nd->leaf) {
    for (int64_t i = nd->first; i < nd->first + nd->count; ++i) {
      int64_t b = t->ord[i];
      if (b == a) continue;
      double xb[3] = {0, 0, 0};
      for (int ax = 0; ax < dim; ++ax) xb[ax] = X[ax][b];
      grav_term(dim, xa, xb, m[b], eps2, G, acc);
    }
    return;
  }
  for (int c = 0; c < nd->nchild; ++c) bh_walk(t, nd->child[c], a, ka, X, m, G, theta, eps2, acc);
}

/* Barnes-Hut accelerations at positions (x, y, z) from the tree built at    */
/* (xb, yb, zb): the pseudo-particles (node mass and centre of mass), node   */
/* cubes and leaf membership are those of the build; each particle's cell   */
/* comes from its current position in the build's root cube (clamped, as in */
/* the build), and leaves are summed over their members' current positions. */
/* With xb = x this is the plain Barnes-Hut sum.                             */
static void gravity_bh_at(int32_t dim, int64_t n, const double *xb, const double *yb, const double *zb,
                          const double *x, const double *y, const double *z, const double *m, const double *h,
                          double G, double theta, double eps_grav, int32_t leaf_size, int32_t max_depth,
                          const int64_t *sample, int64_t nsample, double *ax, double *ay, double *az) {
  otree t;
  tree_build(&t, dim, n, xb, yb, zb, m, leaf_size, max_depth);
  const double *X[3] = {x, y, z};
  double *A[3] = {ax, ay, az};
  int64_t cnt = sample ? nsample : n;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 64)
  for (int64_t i = 0; i < cnt; ++i) {
    int64_t a = sample ? sample[i] : i;
    double acc[3] = {0, 0, 0};
    int64_t ka[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) ka[k] = cell_index(&t.rc, k, X[k][a], max_depth);
    double e = eps_grav * h[a];
    if (n > 0) bh_walk(&t, 0, a, ka, X, m, G, theta, e * e, acc);
    for (int k = 0; k < dim; ++k) A[k][i] = acc[k];
  }
  tree_free(&t);
}

int32_t orc_gravity_bh(int32_t dim, int64_t n, const double *x, const double *y, const double *z,
                       const double *m, const double *h, double G, double theta, double eps_grav,
                       int32_t leaf_size, int32_t max_depth, const int64_t *sample, int64_t nsample,
                       double *ax, double *ay, double *az) {
  gravity_bh_at(dim, n, x, y, z, x, y, z, m, h, G, theta, eps_grav, leaf_size, max_depth, sample, nsample, ax, ay,
                az);
  return 0;
}

int32_t orc_gravity_bh_reuse(int32_t dim, int64_t n, const double *xb, const double *yb, const double *zb,
                             const double *x, const double *y, const double *z, const double *m, const double *h,
                             double G, double theta, double eps_grav, int32_t leaf_size, int32_t max_depth,
                             const int64_t *sample, int64_t nsample, double *ax, double *ay, double *az) {
  gravity_bh_at(dim, n, xb, yb, zb, x, y, z, m, h, G, theta, eps_grav, leaf_size, max_depth, sample, nsample, ax,
                ay, az);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Equations of state, Sect. 2.5.                                            */
/*  linear (2.5.1):  p = cs^2 (rho - rho0); p = 0 when rho/rho0 < rho_cut.   */
/*  Murnaghan (2.5.2): p = K0/n [ (rho/rho0)^n - 1 ], c^2 = dp/drho.         */
/*  isothermal ideal gas (Sect. 4.2): p = cs^2 rho.                          */
/*  Tillotson (2.5.3), Eqs. (tillo1, tillo2): compressed form p_c for        */
/*  rho >= rho0 or u <= E_iv, expanded form p_e for u >= E_cv, linear        */
/*  interpolation in u in between.  Sound speed (not given in the paper):    */
/*  c^2 = max(A_T/rho0, dp/drho|_u + p/rho^2 dp/du|_rho).                    */
/* ------------------------------------------------------------------------ */
static void tillotson_compressed(const orc_material *M, double rho, double u, double *p, double *pr,
                                 double *pu) {
  double eta = rho / M->rho0, chi = eta - 1.0;
  double w = 1.0 + u / (M->E0 * eta * eta);
  double dw_drho = -2.0 * u / (M->E0 * eta * eta * eta * M->rho0);
  double dw_du = 1.0 / (M->E0 * eta * eta);
  double k = M->a_T + M->b_T / w;
  *p = k * rho * u + M->A_T * chi + M->B_T * chi * chi;
  *pr = k * u - M->b_T / (w * w) * dw_drho * rho * u + (M->A_T + 2.0 * M->B_T * chi) / M->rho0;
  *pu = k * rho - M->b_T / (w * w) * dw_du * rho * u;
}

static void tillotson_expanded(const orc_material *M, double rho, double u, double *p, double *pr,
                               double *pu) {
  double eta = rho / M->rho0, chi = eta - 1.0;
  double w = 1.0 + u / (M->E0 * eta * eta);
  double dw_drho = -2.0 * u / (M->E0 * eta * eta * eta * M->rho0);
  double dw_du = 1.0 / (M->E0 * eta * eta);
  double rf = rho > 1e-3 * M->rho0 ? rho : 1e-3 * M->rho0; /* floor inside the exponentials only */
  double zz = M->rho0 / rf - 1.0;
  double dz = rho > 1e-3 * M->rho0 ? -M->rho0 / (rho * rho) : 0.0;
  double eb = exp(-M->beta_T * zz);
  double ea = exp(-M->alpha_T * zz * zz);
  double X = M->b_T * rho * u / w + M->A_T * chi * eb;
  double dX = M->b_T * u / w - M->b_T * rho * u / (w * w) * dw_drho + M->A_T / M->rho0 * eb +
              M->A_T * chi * eb * (-M->beta_T) * dz;
  double dY = ea * (-2.0 * M->alpha_T * zz) * dz;
  *p = M->a_T * rho * u + X * ea;
  *pr = M->a_T * u + dX * ea + X * dY;
  *pu = M->a_T * rho + (M->b_T * rho / w - M->b_T * rho * u / (w * w) * dw_du) * ea;
}

void orc_eos(const orc_material *M, double rho, double u, double *p_out, double *dpdrho, double *dpdu,
             double *cs_out) {
  double p = 0.0, pr = 0.0, pu = 0.0, c2 = 0.0;
  switch (M->eos) {
    case ORC_EOS_LINEAR:
      p = M->cs * M->cs * (rho - M->rho0);
      pr = M->cs * M->cs;
      if (M->rho_cut > 0.0 && rho / M->rho0 < M->rho_cut) {
        p = 0.0;
        pr = 0.0;
      }
      c2 = M->cs * M->cs;
      break;
    case ORC_EOS_MURNAGHAN: {
      double eta = rho / M->rho0;
      p = M->K0 / M->n_M * (pow(eta, M->n_M) - 1.0);
      pr = M->K0 / M->rho0 * pow(eta, M->n_M - 1.0);
      c2 = pr;
      break;
    }
    case ORC_EOS_ISOTHERMAL:
      p = M->cs * M->cs * rho;
      pr = M->cs * M->cs;
      c2 = M->cs * M->cs;
      break;
    case ORC_EOS_TILLOTSON: {
      double pc, pcr, pcu;
      tillotson_compressed(M, rho, u, &pc, &pcr, &pcu);
      if (rho >= M->rho0 || u <= M->E_iv) {
        p = pc;
        pr = pcr;
        pu = pcu;
      } else {
        double pe, per, peu;
        tillotson_expanded(M, rho, u, &pe, &per, &peu);
        if (u >= M->E_cv) {
          p = pe;
          pr = per;
          pu = peu;
        } else {
          double dE = M->E_cv - M->E_iv;
          p = ((u - M->E_iv) * pe + (M->E_cv - u) * pc) / dE;
          pr = ((u - M->E_iv) * per + (M->E_cv - u) * pcr) / dE;
          pu = ((pe - pc) + (u - M->E_iv) * peu + (M->E_cv - u) * pcu) / dE;
        }
      }
      c2 = pr + p / (rho * rho) * pu;
      if (c2 < M->A_T / M->rho0) c2 = M->A_T / M->rho0;
      break;
    }
    default:
      break;
  }
  if (p_out) *p_out = p;
  if (dpdrho) *dpdrho = pr;
  if (dpdu) *dpdu = pu;
  if (cs_out) *cs_out = sqrt(c2);
}

/* ------------------------------------------------------------------------ */
/* Principal axes of a symmetric D x D matrix by the cyclic Jacobi method    */
/* (each sweep zeroes every off-diagonal entry once by a plane rotation      */
/* J = [[c, s], [-s, c]] with t = tan = sign(tau)/(|tau| + sqrt(1 + tau^2)),  */
/* tau = (a_qq - a_pp)/(2 a_pq); A <- J^T A J, V <- V J).                    */
/* ------------------------------------------------------------------------ */
void orc_sym_eig(int32_t dim, const double *Ain, double *w, double *Vout) {
  double A[3][3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      A[i][j] = (i < dim && j < dim) ? Ain[i * dim + j] : 0.0;
      V[i][j] = i == j ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < dim; ++p)
      for (int q = p + 1; q < dim; ++q) off += A[p][q] * A[p][q];
    if (off == 0.0) break;
    for (int p = 0; p < dim; ++p)
      for (int q = p + 1; q < dim; ++q) {
        if (A[p][q] == 0.0) continue;
        double tau = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        J[p][p] = c;
        J[q][q] = c;
        J[p][q] = s;
        J[q][p] = -s;
        double B[3][3], C[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            B[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) B[i][j] += A[i][k] * J[k][j];
          }
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            C[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) C[i][j] += J[k][i] * B[k][j];
          }
        memcpy(A, C, sizeof(A));
        A[p][q] = A[q][p] = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            B[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) B[i][j] += V[i][k] * J[k][j];
          }
        memcpy(V, B, sizeof(V));
      }
  }
  /* ascending order, eigenvectors as columns */
  int ord[3] = {0, 1, 2};
  for (int i = 0; i < dim; ++i)
    for (int j = i + 1; j < dim; ++j)
      if (A[ord[j]][ord[j]] < A[ord[i]][ord[i]]) {
        int tmp = ord[i];
        ord[i] = ord[j];
        ord[j] = tmp;
      }
  for (int i = 0; i < dim; ++i) {
    w[i] = A[ord[i]][ord[i]];
    if (Vout)
      for (int r = 0; r < dim; ++r) Vout[r * dim + i] = V[r][ord[i]];
  }
}

/* ------------------------------------------------------------------------ */
/* Right-hand side of one instance.                                          */
/* ------------------------------------------------------------------------ */
static const orc_material *mat_of(const orc_state *s, const orc_material *mats, int nmat, int64_t a) {
  int k = s->mat ? s->mat[a] : 0;
  if (k < 0 || k >= nmat) k = 0;
  return &mats[k];
}

static double det3(int dim, double M[3][3]) {
  if (dim == 2) return M[0][0] * M[1][1] - M[0][1] * M[1][0];
  return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
         M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* Inverse by the adjugate; returns 0 when L is treated as singular. */
static int invert(int dim, double L[3][3], double C[3][3]) {
  double det = det3(dim, L);
  double diag = 1.0;
  for (int i = 0; i < dim; ++i) diag *= fabs(L[i][i]);
  if (!(fabs(det) > 1e-8 * diag) || !(diag > 0.0)) return 0;
  memset(C, 0, 9 * sizeof(double));
  if (dim == 2) {
    C[0][0] = L[1][1] / det;
    C[0][1] = -L[0][1] / det;
    C[1][0] = -L[1][0] / det;
    C[1][1] = L[0][0] / det;
    return 1;
  }
  C[0][0] = (L[1][1] * L[2][2] - L[1][2] * L[2][1]) / det;
  C[0][1] = (L[0][2] * L[2][1] - L[0][1] * L[2][2]) / det;
  C[0][2] = (L[0][1] * L[1][2] - L[0][2] * L[1][1]) / det;
  C[1][0] = (L[1][2] * L[2][0] - L[1][0] * L[2][2]) / det;
  C[1][1] = (L[0][0] * L[2][2] - L[0][2] * L[2][0]) / det;
  C[1][2] = (L[0][2] * L[1][0] - L[0][0] * L[1][2]) / det;
  C[2][0] = (L[1][0] * L[2][1] - L[1][1] * L[2][0]) / det;
  C[2][1] = (L[0][1] * L[2][0] - L[0][0] * L[2][1]) / det;
  C[2][2] = (L[0][0] * L[1][1] - L[0][1] * L[1][0]) / det;
  return 1;
}

/* Per-particle quantities passed from the update to the momentum pass. */
typedef struct {
  double T[3][3];    /* sigma_d / rho^2                                    */
  double zeta[3][3]; /* artificial stress of the particle                  */
  double cs;
} pstate;

/* von Mises limiter, Sect. 2.6: f_Y = min(Y0^2 / (3 J2), 1), J2 = S:S / 2. */
static double yield_factor(int dim, const orc_material *M, double S[3][3]) {
  if (!(M->Y0 > 0.0)) return 1.0;
  double J2 = 0.0;
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j) J2 += S[i][j] * S[i][j];
  J2 = 0.5 * J2;
  if (!(J2 > 0.0)) return 1.0;
  double f = M->Y0 * M->Y0 / (3.0 * J2);
  return f < 1.0 ? f : 1.0;
}

static int flaw_count_below(const float *eps, int64_t n, double e) {
  int c = 0;
  for (int64_t j = 0; j < n; ++j)
    if ((double)eps[j] < e) ++c;
  return c;
}

/* Conditioning of a kernel term at the support edge (see oracle.h). */
static double edge_kappa(double q) { return q >= 0.5 ? q / (1.0 - q) : 1.0; }

/* xb (may be NULL): positions at which the gravity tree was built, when its */
/* pseudo-particles are reused (tree_reuse); NULL builds it at s's positions. */
static int rhs_instance(orc_state *s, const orc_material *mats, int nmat, const orc_params *P, orc_derivs *d,
                        const double *const *xb) {
  const int dim = P->dim;
  const int64_t n = s->n;
  if (n == 0) return 0;
  double *X[3] = {s->x, s->y, s->z};
  double *V[3] = {s->vx, s->vy, s->vz};

  /* Interaction partners, Sect. 3.5.2 */
  int64_t *off = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
  int64_t cap = 64 * n + 1024;
  int32_t *nb = NULL;
  for (;;) {
    nb = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    if (orc_neighbours_grid(dim, n, s->x, s->y, s->z, s->h, off, nb, cap) >= 0) break;
    free(nb);
    cap = off[n] + 1;
  }

  /* Density by kernel sum, Eq. (density_by_kernel_sum), with the particle's */
  /* own contribution m_a W(0; h_a) and W_ab = W(r_ab; (h_a + h_b)/2).       */
  if (P->density_sum) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t a = 0; a < n; ++a) {
      double sum = s->m[a] * orc_W(0.0, s->h[a], dim), m1 = 0.0;
      for (int64_t k = off[a]; k < off[a + 1]; ++k) {
        int64_t b = nb[k];
        double r2 = 0.0;
        for (int ax = 0; ax < dim; ++ax) {
          double dd = X[ax][a] - X[ax][b];
          r2 = r2 + dd * dd;
        }
        double hab = 0.5 * (s->h[a] + s->h[b]);
        double t = s->m[b] * orc_W(sqrt(r2), hab, dim);
        sum += t;
        m1 += t * edge_kappa(sqrt(r2) / hab);
      }
      s->rho[a] = sum;
      if (d->mag_rho) d->mag_rho[a] = sum;
      if (d->mag1_rho) d->mag1_rho[a] = m1;
    }
  }

  pstate *ps = (pstate *)calloc((size_t)n, sizeof(pstate));
  int any_strength = s->S != NULL;

  /* Pass over neighbours for continuity, velocity gradient, XSPH, then the */
  /* per-particle constitutive update.                                      */
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t a = 0; a < n; ++a) {
    const orc_material *M = mat_of(s, mats, nmat, a);
    double drho = 0.0, magdrho = 0.0, maggv = 0.0, m1drho = 0.0, m1gv = 0.0;
    double L[3][3] = {{0}}, Gt[3][3] = {{0}}, xs[3] = {0, 0, 0};
    for (int64_t k = off[a]; k < off[a + 1]; ++k) {
      int64_t b = nb[k];
      double dx[3] = {0, 0, 0}, dv[3] = {0, 0, 0}, r2 = 0.0;
      for (int ax = 0; ax < dim; ++ax) {
        dx[ax] = X[ax][a] - X[ax][b];
        dv[ax] = V[ax][a] - V[ax][b];
        r2 = r2 + dx[ax] * dx[ax];
      }
      double r = sqrt(r2), hab = 0.5 * (s->h[a] + s->h[b]);
      double g[3] = {0, 0, 0};
      if (r > 0.0) {
        double f = orc_dWdr(r, hab, dim) / r;
        for (int ax = 0; ax < dim; ++ax) g[ax] = f * dx[ax]; /* grad_a W_ab */
      }
      double vol = s->m[b] / s->rho[b];
      /* Eq. (continuity_equation_sph): (v_a - v_b) . grad_a W_ab */
      double vg = 0.0, vga = 0.0;
      for (int ax = 0; ax < dim; ++ax) {
        vg += dv[ax] * g[ax];
        vga += fabs(dv[ax] * g[ax]);
      }
      double kap = edge_kappa(r / hab);
      drho += vol * vg;
      magdrho += vol * vga;
      m1drho += vol * vga * kap;
      /* Sect. 3.1.6: L^{ag} = sum vol (x_b - x_a)^a d_g W, same with v for G */
      double sdv = 0.0, sg = 0.0;
      for (int i = 0; i < dim; ++i) {
        sdv += fabs(dv[i]);
        sg += fabs(g[i]);
        for (int j = 0; j < dim; ++j) {
          L[i][j] += vol * (-dx[i]) * g[j];
          Gt[i][j] += vol * (-dv[i]) * g[j];
        }
      }
      maggv += vol * sdv * sg;
      m1gv += vol * sdv * sg * kap;
      /* Sect. 3.1.5: XSPH with the mean density (rho_a + rho_b)/2 */
      if (P->xsph != 0.0) {
        double w = orc_W(r, hab, dim);
        double c = 2.0 * s->m[b] / (s->rho[a] + s->rho[b]);
        for (int ax = 0; ax < dim; ++ax) xs[ax] += c * (-dv[ax]) * w;
      }
    }
    drho = s->rho[a] * drho;
    magdrho = fabs(s->rho[a]) * magdrho;
    m1drho = fabs(s->rho[a]) * m1drho;

    /* Linear consistency, Eq. (ext_sph): grad v = G C with C = L^-1, or I */
    double C[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    int nnb = (int)(off[a + 1] - off[a]);
    if (P->consistency && nnb >= dim + 1) {
      double Ci[3][3];
      if (invert(dim, L, Ci)) memcpy(C, Ci, sizeof(C));
    }
    double gv[3][3] = {{0}};
    double cmax = 0.0;
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) {
        if (fabs(C[i][j]) > cmax) cmax = fabs(C[i][j]);
        for (int k = 0; k < dim; ++k) gv[i][j] += Gt[i][k] * C[k][j];
      }
    maggv = maggv * cmax * dim;
    m1gv = m1gv * cmax * dim;

    /* Equation of state, Sect. 2.5 */
    double p, cs;
    orc_eos(M, s->rho[a], s->u[a], &p, NULL, NULL, &cs);

    /* Deviatoric stress, Sects. 2.4 and 2.6 */
    double S[3][3] = {{0}}, dS[3][3] = {{0}};
    int strength = any_strength && M->strength;
    if (strength) {
      sym_load(dim, s->S, n, a, S);
      double fY = yield_factor(dim, M, S);
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) S[i][j] *= fY;
      /* Eqs. (strain_rate_tensor, rotation_terms): eps_dot and R from grad v */
      double ed[3][3], R[3][3], tr = 0.0;
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
          ed[i][j] = 0.5 * (gv[i][j] + gv[j][i]);
          R[i][j] = 0.5 * (gv[i][j] - gv[j][i]);
        }
      for (int i = 0; i < dim; ++i) tr += ed[i][i];
      /* Eq. (stresstensor_evolution): Hooke's law with the Jaumann terms   */
      /* R S - S R (the co-rotational sign; deviator taken in D dimensions) */
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
          double rot = 0.0;
          for (int k = 0; k < dim; ++k) rot += R[i][k] * S[k][j] - S[i][k] * R[k][j];
          dS[i][j] = 2.0 * M->mu * (ed[i][j] - (i == j ? tr / dim : 0.0)) + rot;
        }
    }

    /* Damage, Sects. 2.7 and 3.2: sigma_d = -p_hat I + (1 - d) S */
    double dmgd = 0.0, dd = 0.0, eps_t = 0.0;
    int nact = 0;
    int damage = s->dmg != NULL && M->damage;
    if (damage) {
      double delta = s->dmg[a];
      dmgd = delta * delta * delta;
    }
    double sig[3][3] = {{0}};
    double phat = (p >= 0.0) ? p : (1.0 - dmgd) * p;
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) sig[i][j] = (i == j ? -phat : 0.0) + (1.0 - dmgd) * S[i][j];

    double lam[3] = {0, 0, 0}, Q[9] = {0};
    int need_eig = damage || P->eps_s > 0.0;
    if (need_eig) {
      double A[9];
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) A[i * dim + j] = sig[i][j];
      orc_sym_eig(dim, A, lam, Q);
    }
    if (damage) {
      /* local scalar strain eps = sigma_max / ((1 - d) E), E = 9 K mu / (3K + mu) */
      double E = 9.0 * M->K0 * M->mu / (3.0 * M->K0 + M->mu);
      double smax = lam[dim - 1];
      double den = (1.0 - dmgd) * E;
      double eps = den > 0.0 ? smax / den : 0.0;
      eps_t = eps;
      int64_t id = s->id ? s->id[a] : a;
      int64_t f0 = s->flaw_off ? s->flaw_off[id] : 0, f1 = s->flaw_off ? s->flaw_off[id + 1] : 0;
      int64_t ntot = f1 - f0;
      nact = (eps > 0.0 && ntot > 0) ? flaw_count_below(s->flaw_eps + f0, ntot, eps) : 0;
      /* d(d^1/3)/dt = n_act c_g / R_s while d < n_act / n_tot;            */
      /* c_g = 0.4 sqrt((K + 4/3 (1 - d) mu) / rho), R_s = h_a.            */
      if (nact > 0 && dmgd < (double)nact / (double)ntot) {
        double cg = 0.4 * sqrt((M->K0 + 4.0 / 3.0 * (1.0 - dmgd) * M->mu) / s->rho[a]);
        dd = nact * cg / s->h[a];
      }
    }

    /* Artificial stress, Sect. 3.1.4, in the principal frame of sigma */
    double zeta[3][3] = {{0}};
    if (P->eps_s > 0.0) {
      double rr = s->rho[a] * s->rho[a];
      double zl[3] = {0, 0, 0};
      for (int i = 0; i < dim; ++i) zl[i] = lam[i] > 0.0 ? -P->eps_s * lam[i] / rr : 0.0;
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
          double v = 0.0;
          for (int k = 0; k < dim; ++k) v += Q[i * dim + k] * zl[k] * Q[j * dim + k];
          zeta[i][j] = v;
        }
    }

    double rr = s->rho[a] * s->rho[a];
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) {
        ps[a].T[i][j] = sig[i][j] / rr;
        ps[a].zeta[i][j] = zeta[i][j];
      }
    ps[a].cs = cs;

    if (d->drho) d->drho[a] = P->density_sum ? 0.0 : drho;
    if (d->mag_drho) d->mag_drho[a] = magdrho;
    if (d->mag_gradv) d->mag_gradv[a] = maggv;
    if (d->mag1_drho) d->mag1_drho[a] = m1drho;
    if (d->mag1_gradv) d->mag1_gradv[a] = m1gv;
    if (d->gradv)
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) d->gradv[(int64_t)(i * dim + j) * n + a] = gv[i][j];
    if (d->dS && any_strength) sym_store(dim, dS, d->dS, n, a);
    if (d->ddmg) d->ddmg[a] = dd;
    if (d->n_act) d->n_act[a] = nact;
    if (d->eps_t) d->eps_t[a] = eps_t;
    if (d->p) d->p[a] = p;
    if (d->cs) d->cs[a] = cs;
    if (d->nnb) d->nnb[a] = nnb;
    double *DX[3] = {d->dxdt, d->dydt, d->dzdt};
    for (int ax = 0; ax < dim; ++ax)
      if (DX[ax]) DX[ax][a] = V[ax][a] + P->xsph * xs[ax];
  }

  /* Momentum and energy, Eqs. (accel_artvisc) and (energy_sph), read with   */
  /* grad_a W and -Pi* I added to the stress bracket:                        */
  /*   dv_a/dt = sum_b m_b [T_a + T_b + (zeta_a + zeta_b) f^n - Pi* I] grad_a W */
  /*   du_a/dt = -1/2 sum_b m_b (v_a - v_b) . [T_a + T_b - Pi* I] grad_a W   */
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t a = 0; a < n; ++a) {
    double acc[3] = {0, 0, 0}, du = 0.0, magdv = 0.0, magdu = 0.0, m1dv = 0.0, m1du = 0.0;
    for (int64_t k = off[a]; k < off[a + 1]; ++k) {
      int64_t b = nb[k];
      double dx[3] = {0, 0, 0}, dv[3] = {0, 0, 0}, r2 = 0.0;
      for (int ax = 0; ax < dim; ++ax) {
        dx[ax] = X[ax][a] - X[ax][b];
        dv[ax] = V[ax][a] - V[ax][b];
        r2 = r2 + dx[ax] * dx[ax];
      }
      double r = sqrt(r2), hab = 0.5 * (s->h[a] + s->h[b]);
      double g[3] = {0, 0, 0};
      if (r > 0.0) {
        double f = orc_dWdr(r, hab, dim) / r;
        for (int ax = 0; ax < dim; ++ax) g[ax] = f * dx[ax];
      }
      /* Artificial viscosity, Sect. 3.1.3, approaching pairs only */
      double vx = 0.0;
      for (int ax = 0; ax < dim; ++ax) vx += dv[ax] * dx[ax];
      double Pi = 0.0;
      if (vx < 0.0) {
        double nu = hab * vx / (r2 + P->eps_v * hab * hab);
        double cbar = 0.5 * (ps[a].cs + ps[b].cs);
        double rbar = 0.5 * (s->rho[a] + s->rho[b]);
        Pi = (-P->alpha * cbar * nu + P->beta * nu * nu) / rbar;
      }
      double fn = 0.0;
      if (P->eps_s > 0.0) {
        double f = orc_W(r, hab, dim) / orc_W(P->dmpd, hab, dim);
        fn = pow(f, P->n_as);
      }
      for (int i = 0; i < dim; ++i) {
        double sv = 0.0, sva = 0.0, su = 0.0, sua = 0.0;
        for (int j = 0; j < dim; ++j) {
          double Bij = ps[a].T[i][j] + ps[b].T[i][j] - (i == j ? Pi : 0.0);
          double Mij = Bij + (ps[a].zeta[i][j] + ps[b].zeta[i][j]) * fn;
          sv += Mij * g[j];
          sva += fabs(Mij * g[j]);
          su += Bij * g[j];
          sua += fabs(dv[i] * Bij * g[j]);
        }
        double kap = edge_kappa(r / hab);
        acc[i] += s->m[b] * sv;
        magdv += s->m[b] * sva;
        m1dv += s->m[b] * sva * kap;
        du += -0.5 * s->m[b] * dv[i] * su;
        magdu += 0.5 * s->m[b] * sua;
        m1du += 0.5 * s->m[b] * sua * kap;
      }
    }
    double *DV[3] = {d->dvx, d->dvy, d->dvz};
    for (int ax = 0; ax < dim; ++ax)
      if (DV[ax]) DV[ax][a] = acc[ax];
    if (d->du) d->du[a] = du;
    if (d->mag_dv) d->mag_dv[a] = magdv;
    if (d->mag_du) d->mag_du[a] = magdu;
    if (d->mag1_dv) d->mag1_dv[a] = m1dv;
    if (d->mag1_du) d->mag1_du[a] = m1du;
  }

  /* Self-gravity, Sect. 3.3 */
  if (P->gravity) {
    double *ag[3];
    for (int ax = 0; ax < 3; ++ax) ag[ax] = (double *)calloc((size_t)n, sizeof(double));
    if (xb)
      orc_gravity_bh_reuse(dim, n, xb[0], xb[1], xb[2], s->x, s->y, s->z, s->m, s->h, P->G, P->theta, P->eps_grav,
                           P->leaf_size, P->max_depth, NULL, 0, ag[0], ag[1], ag[2]);
    else
      orc_gravity_bh(dim, n, s->x, s->y, s->z, s->m, s->h, P->G, P->theta, P->eps_grav, P->leaf_size,
                     P->max_depth, NULL, 0, ag[0], ag[1], ag[2]);
    double *DV[3] = {d->dvx, d->dvy, d->dvz};
    double *AG[3] = {d->agx, d->agy, d->agz};
    for (int ax = 0; ax < dim; ++ax)
      for (int64_t a = 0; a < n; ++a) {
        if (DV[ax]) DV[ax][a] += ag[ax][a];
        if (AG[ax]) AG[ax][a] = ag[ax][a];
      }
    for (int ax = 0; ax < 3; ++ax) free(ag[ax]);
  }

  free(ps);
  free(nb);
  free(off);
  return 0;
}

/* Views of one instance: every per-particle pointer shifted by lo. */
#define SHIFT(p, lo) ((p) ? (p) + (lo) : NULL)

static orc_state state_view(const orc_state *s, int64_t lo, int64_t hi) {
  orc_state v = *s;
  v.n = hi - lo;
  v.x = SHIFT(s->x, lo);
  v.y = SHIFT(s->y, lo);
  v.z = SHIFT(s->z, lo);
  v.vx = SHIFT(s->vx, lo);
  v.vy = SHIFT(s->vy, lo);
  v.vz = SHIFT(s->vz, lo);
  v.rho = SHIFT(s->rho, lo);
  v.u = SHIFT(s->u, lo);
  v.m = SHIFT(s->m, lo);
  v.h = SHIFT(s->h, lo);
  v.dmg = SHIFT(s->dmg, lo);
  v.mat = SHIFT(s->mat, lo);
  v.id = SHIFT(s->id, lo);
  v.S = NULL;
  v.ninst = 1;
  v.inst_off = NULL;
  return v;
}

static orc_derivs derivs_view(const orc_derivs *d, int64_t lo) {
  orc_derivs v = *d;
  v.dxdt = SHIFT(d->dxdt, lo);
  v.dydt = SHIFT(d->dydt, lo);
  v.dzdt = SHIFT(d->dzdt, lo);
  v.dvx = SHIFT(d->dvx, lo);
  v.dvy = SHIFT(d->dvy, lo);
  v.dvz = SHIFT(d->dvz, lo);
  v.drho = SHIFT(d->drho, lo);
  v.du = SHIFT(d->du, lo);
  v.ddmg = SHIFT(d->ddmg, lo);
  v.p = SHIFT(d->p, lo);
  v.cs = SHIFT(d->cs, lo);
  v.n_act = SHIFT(d->n_act, lo);
  v.nnb = SHIFT(d->nnb, lo);
  v.mag_drho = SHIFT(d->mag_drho, lo);
  v.mag_dv = SHIFT(d->mag_dv, lo);
  v.mag_du = SHIFT(d->mag_du, lo);
  v.mag_gradv = SHIFT(d->mag_gradv, lo);
  v.mag1_drho = SHIFT(d->mag1_drho, lo);
  v.mag1_dv = SHIFT(d->mag1_dv, lo);
  v.mag1_du = SHIFT(d->mag1_du, lo);
  v.mag1_gradv = SHIFT(d->mag1_gradv, lo);
  v.mag_rho = SHIFT(d->mag_rho, lo);
  v.mag1_rho = SHIFT(d->mag1_rho, lo);
  v.agx = SHIFT(d->agx, lo);
  v.agy = SHIFT(d->agy, lo);
  v.agz = SHIFT(d->agz, lo);
  v.eps_t = SHIFT(d->eps_t, lo);
  v.dS = NULL;
  v.gradv = NULL;
  return v;
}

/* Component-major tensors cannot be shifted by a pointer offset, so an      */
/* instance's tensors are copied into and out of contiguous scratch.         */
static int32_t rhs_at(orc_state *s, const orc_material *mats, int32_t nmat, const orc_params *P, orc_derivs *d,
                      const double *const *xb) {
  int32_t ninst = s->ninst > 0 ? s->ninst : 1;
  if (ninst == 1 || !s->inst_off) return rhs_instance(s, mats, nmat, P, d, xb);
  const int ns = nsym(P->dim);
  const int nd2 = P->dim * P->dim;
  int64_t N = s->n;
  for (int32_t i = 0; i < ninst; ++i) {
    int64_t lo = s->inst_off[i], hi = s->inst_off[i + 1], n = hi - lo;
    if (n <= 0) continue;
    orc_state v = state_view(s, lo, hi);
    orc_derivs dv = derivs_view(d, lo);
    double *S = NULL, *dS = NULL, *gv = NULL;
    if (s->S) {
      S = (double *)malloc((size_t)(ns * n) * sizeof(double));
      for (int k = 0; k < ns; ++k) memcpy(S + k * n, s->S + k * N + lo, (size_t)n * sizeof(double));
      v.S = S;
    }
    if (d->dS) {
      dS = (double *)calloc((size_t)(ns * n), sizeof(double));
      dv.dS = dS;
    }
    if (d->gradv) {
      gv = (double *)calloc((size_t)(nd2 * n), sizeof(double));
      dv.gradv = gv;
    }
    const double *xbv[3] = {NULL, NULL, NULL};
    if (xb)
      for (int k = 0; k < 3; ++k) xbv[k] = xb[k] ? xb[k] + lo : NULL;
    int rc = rhs_instance(&v, mats, nmat, P, &dv, xb ? xbv : NULL);
    if (dS)
      for (int k = 0; k < ns; ++k) memcpy(d->dS + k * N + lo, dS + k * n, (size_t)n * sizeof(double));
    if (gv)
      for (int k = 0; k < nd2; ++k) memcpy(d->gradv + k * N + lo, gv + k * n, (size_t)n * sizeof(double));
    free(S);
    free(dS);
    free(gv);
    if (rc) return rc;
  }
  return 0;
}

int32_t orc_rhs(orc_state *s, const orc_material *mats, int32_t nmat, const orc_params *P, orc_derivs *d) {
  return rhs_at(s, mats, nmat, P, d, NULL);
}

/* ------------------------------------------------------------------------ */
/* Time step, Sect. 3.4.1: the minimum over particles of                    */
/*   c_courant h / c_s,  c_accel sqrt(h / |dv/dt|)  (the square root makes   */
/*   the acceleration limit a time), and c_quantity (|q| + floor) / |dq/dt|  */
/*   for rho (continuity), u, each stored S component and d^1/3,            */
/* capped at dt_max; dt_fixed > 0 overrides.                                 */
/* ------------------------------------------------------------------------ */
static double dt_particle(const orc_state *s, const orc_params *P, const orc_derivs *d, int64_t a) {
  const int dim = P->dim;
  double dt = P->dt_max;
  double cs = d->cs ? d->cs[a] : 0.0;
  if (cs > 0.0) {
    double t = P->c_courant * s->h[a] / cs;
    if (t < dt) dt = t;
  }
  double a2 = 0.0;
  const double *DV[3] = {d->dvx, d->dvy, d->dvz};
  for (int ax = 0; ax < dim; ++ax) a2 += DV[ax][a] * DV[ax][a];
  if (a2 > 0.0) {
    double t = P->c_accel * sqrt(s->h[a] / sqrt(a2));
    if (t < dt) dt = t;
  }
  if (!P->density_sum && d->drho && fabs(d->drho[a]) > 0.0) {
    double t = P->c_quantity * fabs(s->rho[a]) / fabs(d->drho[a]);
    if (t < dt) dt = t;
  }
  if (d->du && fabs(d->du[a]) > 0.0) {
    double t = P->c_quantity * (fabs(s->u[a]) + P->u_floor) / fabs(d->du[a]);
    if (t < dt) dt = t;
  }
  return dt;
}

void orc_timestep(const orc_state *s, const orc_material *mats, int32_t nmat, const orc_params *P,
                  const orc_derivs *d, double *dt_inst) {
  (void)mats;
  (void)nmat;
  int32_t ninst = s->ninst > 0 ? s->ninst : 1;
  const int ns = nsym(P->dim);
  for (int32_t i = 0; i < ninst; ++i) {
    int64_t lo = (ninst == 1 || !s->inst_off) ? 0 : s->inst_off[i];
    int64_t hi = (ninst == 1 || !s->inst_off) ? s->n : s->inst_off[i + 1];
    double dt = P->dt_max;
    for (int64_t a = lo; a < hi; ++a) {
      double t = dt_particle(s, P, d, a);
      if (t < dt) dt = t;
      if (s->S && d->dS)
        for (int k = 0; k < ns; ++k) {
          double q = s->S[(int64_t)k * s->n + a], dq = d->dS[(int64_t)k * s->n + a];
          if (fabs(dq) > 0.0) {
            double tq = P->c_quantity * (fabs(q) + P->S_floor) / fabs(dq);
            if (tq < dt) dt = tq;
          }
        }
      if (s->dmg && d->ddmg && d->ddmg[a] > 0.0) {
        double tq = P->c_quantity * (fabs(s->dmg[a]) + P->dmg_floor) / d->ddmg[a];
        if (tq < dt) dt = tq;
      }
    }
    dt_inst[i] = P->dt_fixed > 0.0 ? P->dt_fixed : dt;
  }
}

/* ------------------------------------------------------------------------ */
/* Predictor-corrector, Sect. 3.4.1:                                         */
/*   q^p = q + dt/2 dq/dt(q),   q^c = q + dt dq/dt(q^p)                      */
/* for x (with the XSPH velocity), v, rho (continuity), u, S and d^1/3.      */
/* After each update S is replaced by f_Y S (Sect. 2.6) and a growing d^1/3  */
/* is capped at (n_act / n_tot)^1/3 (Sect. 3.2), with n_act from the         */
/* right-hand side that produced the derivative.                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  double *buf;
  orc_derivs d;
} dstore;

static void dstore_alloc(dstore *ds, int dim, int64_t n) {
  int ns = nsym(dim);
  int64_t tot = (int64_t)(3 + 3 + 4 + ns + 2) * n;
  ds->buf = (double *)calloc((size_t)tot + 1, sizeof(double));
  memset(&ds->d, 0, sizeof(ds->d));
  double *p = ds->buf;
  ds->d.dxdt = p; p += n;
  ds->d.dydt = p; p += n;
  ds->d.dzdt = p; p += n;
  ds->d.dvx = p; p += n;
  ds->d.dvy = p; p += n;
  ds->d.dvz = p; p += n;
  ds->d.drho = p; p += n;
  ds->d.du = p; p += n;
  ds->d.ddmg = p; p += n;
  ds->d.cs = p; p += n;
  ds->d.dS = p; p += ns * n;
  ds->d.p = p; p += n;
  ds->d.n_act = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
}

static void dstore_free(dstore *ds) {
  free(ds->buf);
  free(ds->d.n_act);
}

static int64_t inst_of(const orc_state *s, int64_t a) {
  if (s->ninst <= 1 || !s->inst_off) return 0;
  int64_t lo = 0, hi = s->ninst - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) / 2;
    if (s->inst_off[mid] <= a)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

/* out = base + f * dt_inst * deriv, then the limiters. */
static void pc_update(const orc_state *base, orc_state *out, const orc_derivs *d, const double *dt_inst,
                      double f, const orc_material *mats, int nmat, const orc_params *P) {
  const int dim = P->dim;
  const int64_t n = base->n;
  const int ns = nsym(dim);
  double *Xb[3] = {base->x, base->y, base->z}, *Xo[3] = {out->x, out->y, out->z};
  double *Vb[3] = {base->vx, base->vy, base->vz}, *Vo[3] = {out->vx, out->vy, out->vz};
  double *DX[3] = {d->dxdt, d->dydt, d->dzdt}, *DV[3] = {d->dvx, d->dvy, d->dvz};
  for (int64_t a = 0; a < n; ++a) {
    double dt = f * dt_inst[inst_of(base, a)];
    for (int ax = 0; ax < dim; ++ax) {
      Xo[ax][a] = Xb[ax][a] + dt * DX[ax][a];
      Vo[ax][a] = Vb[ax][a] + dt * DV[ax][a];
    }
    if (!P->density_sum) out->rho[a] = base->rho[a] + dt * d->drho[a];
    else out->rho[a] = base->rho[a];
    out->u[a] = base->u[a] + dt * d->du[a];
    const orc_material *M = mat_of(base, mats, nmat, a);
    if (base->S) {
      double S[3][3];
      for (int k = 0; k < ns; ++k) {
        int64_t i = (int64_t)k * n + a;
        out->S[i] = base->S[i] + dt * d->dS[i];
      }
      if (M->strength) {
        sym_load(dim, out->S, n, a, S);
        double fY = yield_factor(dim, M, S);
        for (int k = 0; k < ns; ++k) out->S[(int64_t)k * n + a] *= fY;
      }
    }
    if (base->dmg) {
      double nd = base->dmg[a] + dt * d->ddmg[a];
      if (d->ddmg[a] > 0.0) {
        int64_t id = base->id ? base->id[a] : a;
        int64_t ntot = base->flaw_off[id + 1] - base->flaw_off[id];
        double cap = cbrt((double)d->n_act[a] / (double)ntot);
        if (nd > cap) nd = cap;
      }
      if (nd > 1.0) nd = 1.0;
      out->dmg[a] = nd;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Embedded Runge-Kutta step, Sect. 3.4.2.  k1 = f(q), k2 = f(q + dt/2 k1),  */
/* k3 = f(q - dt k1 + 2 dt k2); q_rk3 = q + dt (k1 + 4 k2 + k3)/6 and the    */
/* midpoint value q + dt k2 differ by dt (2 k2 - k1 - k3)/6.  The error of   */
/* an instance is the largest ratio of that difference to the Euler value    */
/* |q + dt k1| over its particles and integrated components; a floor is      */
/* added to the denominator (h for positions, c_s for velocities, the        */
/* limiter floors for u, S and d^1/3, none for rho).  err < eps_des accepts  */
/* the step (q <- q_rk3, t += dt, dt <- dt (eps_des/err)^0.3, or dt_max for  */
/* err = 0); otherwise the instance keeps q and dt <- 0.9 dt                 */
/* (eps_des/err)^(1/4).  dt never exceeds dt_max.  Every state formed (the  */
/* two stage states and q_rk3) gets the yield and damage limits of the       */
/* predictor-corrector update, with n_act of the last derivative used.       */
/* ------------------------------------------------------------------------ */
static void rk_combine(const orc_state *base, orc_state *out, const orc_derivs *k[3], const double c[3],
                       const double *dt_inst, const int32_t *mask, const orc_material *mats, int nmat,
                       const orc_params *P) {
  const int dim = P->dim;
  const int64_t n = base->n;
  const int ns = nsym(dim);
  int last = 0;
  for (int j = 0; j < 3; ++j)
    if (c[j] != 0.0) last = j;
  /* D = c1 k1 + c2 k2 + c3 k3, in that order */
#define RK_D(field, i) ((c[0] * k[0]->field[i] + c[1] * (c[1] != 0.0 ? k[1]->field[i] : 0.0)) + \
                        c[2] * (c[2] != 0.0 ? k[2]->field[i] : 0.0))
  double *Xb[3] = {base->x, base->y, base->z}, *Xo[3] = {out->x, out->y, out->z};
  double *Vb[3] = {base->vx, base->vy, base->vz}, *Vo[3] = {out->vx, out->vy, out->vz};
  for (int64_t a = 0; a < n; ++a) {
    const int32_t ii = inst_of(base, a);
    if (mask && !mask[ii]) continue;
    const double dt = dt_inst[ii];
    for (int ax = 0; ax < dim; ++ax) {
      double dX = ax == 0 ? RK_D(dxdt, a) : (ax == 1 ? RK_D(dydt, a) : RK_D(dzdt, a));
      double dV = ax == 0 ? RK_D(dvx, a) : (ax == 1 ? RK_D(dvy, a) : RK_D(dvz, a));
      Xo[ax][a] = Xb[ax][a] + dt * dX;
      Vo[ax][a] = Vb[ax][a] + dt * dV;
    }
    if (!P->density_sum) out->rho[a] = base->rho[a] + dt * RK_D(drho, a);
    else out->rho[a] = base->rho[a];
    out->u[a] = base->u[a] + dt * RK_D(du, a);
    const orc_material *M = mat_of(base, mats, nmat, a);
    if (base->S) {
      double S[3][3];
      for (int kk = 0; kk < ns; ++kk) {
        int64_t i = (int64_t)kk * n + a;
        out->S[i] = base->S[i] + dt * RK_D(dS, i);
      }
      if (M->strength) {
        sym_load(dim, out->S, n, a, S);
        double fY = yield_factor(dim, M, S);
        for (int kk = 0; kk < ns; ++kk) out->S[(int64_t)kk * n + a] *= fY;
      }
    }
    if (base->dmg) {
      const double dd = RK_D(ddmg, a);
      double nd = base->dmg[a] + dt * dd;
      if (dd > 0.0) {
        int64_t id = base->id ? base->id[a] : a;
        int64_t ntot = base->flaw_off[id + 1] - base->flaw_off[id];
        double cap = cbrt((double)k[last]->n_act[a] / (double)ntot);
        if (nd > cap) nd = cap;
      }
      if (nd > 1.0) nd = 1.0;
      out->dmg[a] = nd;
    }
  }
#undef RK_D
}

static double rk_ratio(double q, double k1, double k2, double k3, double dt, double floor) {
  double num = fabs(2.0 * k2 - k1 - k3) * dt / 6.0;
  double den = fabs(q + dt * k1) + floor;
  return den > 0.0 ? num / den : (num > 0.0 ? INFINITY : 0.0);
}

int32_t orc_step_rk3(orc_state *s, const orc_material *mats, int32_t nmat, const orc_params *P, double eps_des,
                     int32_t nsteps, double *dt_inst, double *t_inst, double *err_log, int32_t *acc_log) {
  const int dim = P->dim;
  const int64_t n = s->n;
  const int ns = nsym(dim);
  int32_t ninst = s->ninst > 0 ? s->ninst : 1;
  orc_state q = *s;
  double *buf = (double *)calloc((size_t)((8 + ns + 2) * n) + 1, sizeof(double));
  double *p = buf;
  q.x = p; p += n;
  q.y = p; p += n;
  q.z = p; p += n;
  q.vx = p; p += n;
  q.vy = p; p += n;
  q.vz = p; p += n;
  q.rho = p; p += n;
  q.u = p; p += n;
  q.S = s->S ? p : NULL; p += ns * n;
  q.dmg = s->dmg ? p : NULL; p += n;
  if (dim == 2) {
    q.z = NULL;
    q.vz = NULL;
  }
  dstore d[3];
  for (int j = 0; j < 3; ++j) dstore_alloc(&d[j], dim, n);
  const orc_derivs *k[3] = {&d[0].d, &d[1].d, &d[2].d};
  double *lim = (double *)malloc((size_t)ninst * sizeof(double));
  double *err = (double *)malloc((size_t)ninst * sizeof(double));
  int32_t *acc = (int32_t *)malloc((size_t)ninst * sizeof(int32_t));
  int rc = 0;
  int32_t *hcnt = P->n_des > 0.0 ? (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t)) : NULL;
  for (int32_t st = 0; st < nsteps && rc == 0; ++st) {
    /* variable smoothing length at the start of each attempt, from the current */
    /* h (Sect. 4.2); a rejected attempt keeps the adapted h                     */
    if (hcnt)
      orc_adapt_h(dim, n, s->x, s->y, s->z, s->h, s->inst_off, ninst, P->n_des, P->h_tol, P->h_iter, hcnt);
    rc = orc_rhs(s, mats, nmat, P, &d[0].d);
    if (rc) break;
    orc_timestep(s, mats, nmat, P, &d[0].d, lim); /* first step size where none is given */
    for (int32_t i = 0; i < ninst; ++i)
      if (!(dt_inst[i] > 0.0)) dt_inst[i] = lim[i];
    const double c2[3] = {0.5, 0.0, 0.0}, c3[3] = {-1.0, 2.0, 0.0}, cf[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};
    rk_combine(s, &q, k, c2, dt_inst, NULL, mats, nmat, P);
    rc = orc_rhs(&q, mats, nmat, P, &d[1].d);
    if (rc) break;
    rk_combine(s, &q, k, c3, dt_inst, NULL, mats, nmat, P);
    rc = orc_rhs(&q, mats, nmat, P, &d[2].d);
    if (rc) break;
    /* error of each instance */
    for (int32_t i = 0; i < ninst; ++i) err[i] = 0.0;
    const double *Xs[3] = {s->x, s->y, s->z}, *Vs[3] = {s->vx, s->vy, s->vz};
    for (int64_t a = 0; a < n; ++a) {
      const int32_t ii = inst_of(s, a);
      const double dt = dt_inst[ii];
      double e = 0.0, r;
      const double *K1x[3] = {k[0]->dxdt, k[0]->dydt, k[0]->dzdt}, *K2x[3] = {k[1]->dxdt, k[1]->dydt, k[1]->dzdt},
                   *K3x[3] = {k[2]->dxdt, k[2]->dydt, k[2]->dzdt};
      const double *K1v[3] = {k[0]->dvx, k[0]->dvy, k[0]->dvz}, *K2v[3] = {k[1]->dvx, k[1]->dvy, k[1]->dvz},
                   *K3v[3] = {k[2]->dvx, k[2]->dvy, k[2]->dvz};
      for (int ax = 0; ax < dim; ++ax) {
        r = rk_ratio(Xs[ax][a], K1x[ax][a], K2x[ax][a], K3x[ax][a], dt, s->h[a]);
        if (r > e) e = r;
        r = rk_ratio(Vs[ax][a], K1v[ax][a], K2v[ax][a], K3v[ax][a], dt, k[0]->cs[a]);
        if (r > e) e = r;
      }
      if (!P->density_sum) {
        r = rk_ratio(s->rho[a], k[0]->drho[a], k[1]->drho[a], k[2]->drho[a], dt, 0.0);
        if (r > e) e = r;
      }
      r = rk_ratio(s->u[a], k[0]->du[a], k[1]->du[a], k[2]->du[a], dt, P->u_floor);
      if (r > e) e = r;
      if (s->S)
        for (int kk = 0; kk < ns; ++kk) {
          int64_t i = (int64_t)kk * n + a;
          r = rk_ratio(s->S[i], k[0]->dS[i], k[1]->dS[i], k[2]->dS[i], dt, P->S_floor);
          if (r > e) e = r;
        }
      if (s->dmg) {
        r = rk_ratio(s->dmg[a], k[0]->ddmg[a], k[1]->ddmg[a], k[2]->ddmg[a], dt, P->dmg_floor);
        if (r > e) e = r;
      }
      if (e > err[ii]) err[ii] = e;
    }
    for (int32_t i = 0; i < ninst; ++i) acc[i] = err[i] < eps_des;
    rk_combine(s, s, k, cf, dt_inst, acc, mats, nmat, P);
    for (int32_t i = 0; i < ninst; ++i) {
      if (t_inst && acc[i]) t_inst[i] += dt_inst[i];
      double dn;
      if (acc[i]) dn = err[i] > 0.0 ? dt_inst[i] * pow(eps_des / err[i], 0.3) : P->dt_max;
      else dn = 0.9 * dt_inst[i] * pow(eps_des / err[i], 0.25);
      dt_inst[i] = dn < P->dt_max ? dn : P->dt_max;
      if (err_log) err_log[(int64_t)st * ninst + i] = err[i];
      if (acc_log) acc_log[(int64_t)st * ninst + i] = acc[i];
    }
  }
  for (int j = 0; j < 3; ++j) dstore_free(&d[j]);
  free(buf);
  free(lim);
  free(err);
  free(acc);
  free(hcnt);
  return rc;
}

int32_t orc_step(orc_state *s, const orc_material *mats, int32_t nmat, const orc_params *P, int32_t nsteps,
                 double *dt_inst, double *dt_log) {
  const int dim = P->dim;
  const int64_t n = s->n;
  const int ns = nsym(dim);
  int32_t ninst = s->ninst > 0 ? s->ninst : 1;
  /* predicted state */
  orc_state q = *s;
  double *buf = (double *)calloc((size_t)((8 + ns + 2) * n) + 1, sizeof(double));
  double *p = buf;
  q.x = p; p += n;
  q.y = p; p += n;
  q.z = p; p += n;
  q.vx = p; p += n;
  q.vy = p; p += n;
  q.vz = p; p += n;
  q.rho = p; p += n;
  q.u = p; p += n;
  q.S = s->S ? p : NULL; p += ns * n;
  q.dmg = s->dmg ? p : NULL; p += n;
  if (dim == 2) {
    q.z = NULL;
    q.vz = NULL;
  }
  dstore d0, d1;
  dstore_alloc(&d0, dim, n);
  dstore_alloc(&d1, dim, n);
  int rc = 0;
  int32_t *hcnt = P->n_des > 0.0 ? (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t)) : NULL;
  /* Decoupled self-gravity (tree_reuse = R > 0, Sect. 6.3): the tree built at */
  /* the start of a step serves every evaluation of R consecutive steps; its */
  /* pseudo-particles are reused (positions of the build kept in xb).  With  */
  /* variable h every step builds.  A call starts with a build.             */
  const int reuse = P->gravity && P->tree_reuse > 0;
  double *xbuf = reuse ? (double *)malloc((size_t)(3 * n + 1) * sizeof(double)) : NULL;
  const double *xb[3] = {NULL, NULL, NULL};
  if (reuse) {
    for (int k = 0; k < dim; ++k) xb[k] = xbuf + k * n;
  }
  int32_t age = 0;
  for (int32_t st = 0; st < nsteps && rc == 0; ++st) {
    /* variable smoothing length: iterate from the last step's h (Sect. 4.2) */
    if (hcnt)
      orc_adapt_h(dim, n, s->x, s->y, s->z, s->h, s->inst_off, ninst, P->n_des, P->h_tol, P->h_iter, hcnt);
    if (reuse && (age == 0 || hcnt)) {
      const double *X[3] = {s->x, s->y, s->z};
      for (int k = 0; k < dim; ++k) memcpy(xbuf + k * n, X[k], (size_t)n * sizeof(double));
      age = 0;
    }
    rc = rhs_at(s, mats, nmat, P, &d0.d, reuse ? xb : NULL);
    if (rc) break;
    orc_timestep(s, mats, nmat, P, &d0.d, dt_inst);
    if (dt_log) memcpy(dt_log + (int64_t)st * ninst, dt_inst, (size_t)ninst * sizeof(double));
    pc_update(s, &q, &d0.d, dt_inst, 0.5, mats, nmat, P);
    rc = rhs_at(&q, mats, nmat, P, &d1.d, reuse ? xb : NULL);
    if (rc) break;
    pc_update(s, s, &d1.d, dt_inst, 1.0, mats, nmat, P);
    if (reuse) age = (age + 1) % P->tree_reuse;
  }
  dstore_free(&d0);
  dstore_free(&d1);
  free(buf);
  free(hcnt);
  free(xbuf);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: Philox4x64-10 (Salmon, Moraes, Dror and     */
/* Shaw 2011, "Parallel random numbers: as easy as 1, 2, 3").  Each of the   */
/* ten rounds multiplies counter words 0 and 2 by the two round multipliers  */
/* (full 128-bit products); the new counter is (hi(2)^c1^k0, lo(2),           */
/* hi(0)^c3^k1, lo(0)); the key gains the two Weyl increments (golden ratio  */
/* and sqrt(3) - 1 in 64-bit fixed point) before every round but the first.  */
/* ------------------------------------------------------------------------ */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B97F4A7C15ULL;
      k1 += 0xBB67AE8584CAA73BULL;
    }
    unsigned __int128 p0 = (unsigned __int128)0xD2E7470EE14C6C93ULL * c0;
    unsigned __int128 p2 = (unsigned __int128)0xCA5A826395121157ULL * c2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi2 = (uint64_t)(p2 >> 64), lo2 = (uint64_t)p2;
    c0 = hi2 ^ c1 ^ k0;
    c1 = lo2;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* Draw j >= 1 of group g: word (j - 1) mod 4 of the block with counter   */
/* ((j - 1) / 4, 0, 0, 0) and key (seed, g); a member index in [0, N) is     */
/* the high word of draw * N (multiply-shift).                               */
static uint64_t flaw_draw(uint64_t seed, uint64_t g, uint64_t j) {
  uint64_t ctr[4] = {(j - 1) >> 2, 0, 0, 0}, key[2] = {seed, g}, out[4];
  orc_philox4x64(ctr, key, out);
  return out[(j - 1) & 3];
}

typedef struct {
  int32_t id;
  int64_t a;
} id_idx;

static int cmp_id_idx(const void *p, const void *q) {
  int32_t a = ((const id_idx *)p)->id, b = ((const id_idx *)q)->id;
  return (a > b) - (a < b);
}

/* ------------------------------------------------------------------------ */
/* Weibull activation thresholds, Sect. 3.2 (after Benz & Asphaug 1995).    */
/* The brittle particles of each instance and material form a group of N    */
/* particles (ascending id) with volume V = sum m / rho0.  Flaw j = 1, 2, ... */
/* goes to a uniformly drawn member and has the threshold strain             */
/* (j / (k V))^(1/m); flaws are handed out until every member holds one.     */
/* Group g = instance * nmat + material; brittle: damage set, k > 0, m > 0.  */
/* flaw_off[0..n] (indexed by id, ids a permutation of 0..n-1) receives the  */
/* CSR offsets; flaw_eps the thresholds (float, ascending per particle) when */
/* the total fits in cap.  Returns the total, or -1 for invalid ids.         */
/* ------------------------------------------------------------------------ */
int64_t orc_flaws(int64_t n, const int32_t *id, const int32_t *mat, const double *m, const int64_t *inst_off,
                  int32_t ninst, const orc_material *mats, int32_t nmat, const double *weibull_k,
                  const double *weibull_m, uint64_t seed, int64_t *flaw_off, float *flaw_eps, int64_t cap) {
  if (ninst < 1) ninst = 1;
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t *owner = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t)); /* id -> index */
  for (int64_t a = 0; a < n; ++a) owner[a] = -1;
  for (int64_t a = 0; a < n; ++a) {
    if (id[a] < 0 || id[a] >= n || owner[id[a]] >= 0) {
      free(cnt);
      free(owner);
      return -1;
    }
    owner[id[a]] = a;
  }
  /* draws of every group, in order: (member particle index, j) */
  int64_t ndraw = 0, capd = 1024;
  int64_t *dpart = (int64_t *)malloc((size_t)capd * sizeof(int64_t));
  uint64_t *dj = (uint64_t *)malloc((size_t)capd * sizeof(uint64_t));
  double *dkv = (double *)malloc((size_t)capd * sizeof(double)), *dinvm = (double *)malloc((size_t)capd * sizeof(double));
  id_idx *mem = (id_idx *)malloc((size_t)(n > 0 ? n : 1) * sizeof(id_idx));
  char *covered = (char *)malloc((size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < ninst; ++i) {
    int64_t b0 = (ninst > 1 && inst_off) ? inst_off[i] : 0, b1 = (ninst > 1 && inst_off) ? inst_off[i + 1] : n;
    for (int32_t mt = 0; mt < nmat; ++mt) {
      if (!mats[mt].damage || !(weibull_k[mt] > 0.0) || !(weibull_m[mt] > 0.0)) continue;
      int64_t N = 0;
      for (int64_t a = b0; a < b1; ++a)
        if (mat[a] == mt) {
          mem[N].id = id[a];
          mem[N].a = a;
          ++N;
        }
      if (N <= 0) continue;
      qsort(mem, (size_t)N, sizeof(id_idx), cmp_id_idx);
      double V = 0.0;
      for (int64_t k = 0; k < N; ++k) V = V + m[mem[k].a] / mats[mt].rho0;
      const double kV = weibull_k[mt] * V, invm = 1.0 / weibull_m[mt];
      const uint64_t g = (uint64_t)i * (uint64_t)nmat + (uint64_t)mt;
      memset(covered, 0, (size_t)N);
      int64_t left = N;
      for (uint64_t j = 1; left > 0; ++j) {
        uint64_t w = flaw_draw(seed, g, j);
        int64_t k = (int64_t)(((unsigned __int128)w * (uint64_t)N) >> 64);
        if (!covered[k]) {
          covered[k] = 1;
          --left;
        }
        if (ndraw == capd) {
          capd *= 2;
          dpart = (int64_t *)realloc(dpart, (size_t)capd * sizeof(int64_t));
          dj = (uint64_t *)realloc(dj, (size_t)capd * sizeof(uint64_t));
          dkv = (double *)realloc(dkv, (size_t)capd * sizeof(double));
          dinvm = (double *)realloc(dinvm, (size_t)capd * sizeof(double));
        }
        dpart[ndraw] = mem[k].a;
        dj[ndraw] = j;
        dkv[ndraw] = kV;
        dinvm[ndraw] = invm;
        ++ndraw;
        cnt[id[mem[k].a] + 1]++;
      }
    }
  }
  for (int64_t k = 0; k < n; ++k) cnt[k + 1] += cnt[k];
  memcpy(flaw_off, cnt, (size_t)(n + 1) * sizeof(int64_t));
  if (ndraw <= cap) {
    /* draws are in ascending j within a group, so each particle's list stays ascending */
    int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    memcpy(fill, cnt, (size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t d = 0; d < ndraw; ++d) {
      double eps = pow((double)dj[d] / dkv[d], dinvm[d]);
      flaw_eps[fill[id[dpart[d]]]++] = (float)eps;
    }
    free(fill);
  }
  free(cnt);
  free(owner);
  free(dpart);
  free(dj);
  free(dkv);
  free(dinvm);
  free(mem);
  free(covered);
  return ndraw;
}

/* ------------------------------------------------------------------------ */
/* Fragments by friends-of-friends (Sect. 4, fragment analysis of the       */
/* impact experiment): particles with dmg >= d_remove are removed; two of    */
/* the rest in the same instance are friends when they would be interaction  */
/* partners with smoothing lengths b h0 (r_ab^2 < h'_ab^2, h' = b h0 rounded */
/* to double); fragments are the connected components of the friendship     */
/* graph with at least min_size particles, numbered by decreasing particle  */
/* count, ties by smallest member index.  label[n]: fragment or -1.         */
/* frag_count, frag_mass (sum of m in ascending index) up to cap entries.    */
/* dmg may be NULL (nothing removed).  Returns the number of fragments.     */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t count, first;
} frag_key;

static int cmp_frag(const void *p, const void *q) {
  const frag_key *a = (const frag_key *)p, *b = (const frag_key *)q;
  if (a->count != b->count) return a->count > b->count ? -1 : 1;
  return (a->first > b->first) - (a->first < b->first);
}

int64_t orc_fof(int32_t dim, int64_t n, const double *x, const double *y, const double *z, const double *h0,
                const double *dmg, const double *m, const int64_t *inst_off, int32_t ninst, double b,
                double d_remove, int32_t min_size, int32_t *label, int32_t *frag_count, double *frag_mass,
                int64_t cap) {
  if (ninst < 1) ninst = 1;
  double *hb = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  for (int64_t a = 0; a < n; ++a) hb[a] = b * h0[a];
  int64_t *comp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t)); /* smallest member index */
  int64_t *stack = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  for (int64_t a = 0; a < n; ++a) comp[a] = -1;
  for (int32_t i = 0; i < ninst; ++i) {
    int64_t b0 = (ninst > 1 && inst_off) ? inst_off[i] : 0, b1 = (ninst > 1 && inst_off) ? inst_off[i + 1] : n;
    int64_t ni = b1 - b0;
    if (ni <= 0) continue;
    const double *xi = x + b0, *yi = y + b0, *zi = dim == 3 ? z + b0 : NULL;
    int64_t *off = (int64_t *)malloc((size_t)(ni + 1) * sizeof(int64_t));
    int64_t capn = 64 * ni + 1024;
    int32_t *nb = NULL;
    for (;;) {
      nb = (int32_t *)malloc((size_t)capn * sizeof(int32_t));
      if (orc_neighbours_grid(dim, ni, xi, yi, zi, hb + b0, off, nb, capn) >= 0) break;
      free(nb);
      capn = off[ni] + 1;
    }
    /* depth-first search from each unvisited surviving particle, in index order */
    for (int64_t s0 = 0; s0 < ni; ++s0) {
      int64_t a0 = b0 + s0;
      if (comp[a0] >= 0 || (dmg && dmg[a0] >= d_remove)) continue;
      int64_t top = 0;
      stack[top++] = s0;
      comp[a0] = a0;
      while (top > 0) {
        int64_t s = stack[--top];
        for (int64_t k = off[s]; k < off[s + 1]; ++k) {
          int64_t t = nb[k], at = b0 + t;
          if (comp[at] >= 0 || (dmg && dmg[at] >= d_remove)) continue;
          comp[at] = a0;
          stack[top++] = t;
        }
      }
    }
    free(off);
    free(nb);
  }
  /* sizes of the components, keyed by their smallest member */
  int64_t *size = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  for (int64_t a = 0; a < n; ++a)
    if (comp[a] >= 0) size[comp[a]]++;
  int64_t nf = 0;
  for (int64_t a = 0; a < n; ++a)
    if (comp[a] == a && size[a] >= min_size) ++nf;
  frag_key *fk = (frag_key *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(frag_key));
  nf = 0;
  for (int64_t a = 0; a < n; ++a)
    if (comp[a] == a && size[a] >= min_size) {
      fk[nf].count = size[a];
      fk[nf].first = a;
      ++nf;
    }
  qsort(fk, (size_t)nf, sizeof(frag_key), cmp_frag);
  int64_t *rank = stack; /* reuse: rank of a component by its smallest member */
  for (int64_t a = 0; a < n; ++a) rank[a] = -1;
  for (int64_t f = 0; f < nf; ++f) rank[fk[f].first] = f;
  for (int64_t f = 0; f < nf && f < cap; ++f) {
    frag_count[f] = (int32_t)fk[f].count;
    frag_mass[f] = 0.0;
  }
  for (int64_t a = 0; a < n; ++a) {
    int64_t f = comp[a] >= 0 ? rank[comp[a]] : -1;
    label[a] = (int32_t)f;
    if (f >= 0 && f < cap) frag_mass[f] = frag_mass[f] + m[a];
  }
  free(hb);
  free(comp);
  free(stack);
  free(size);
  free(fk);
  return nf;
}
