// Octree over Morton-sorted particles (Sect. 3.5.1), GB300 form.
//
// Instead of the paper's lock-based insertion (atomicCAS on child slots) the
// tree is derived from sorted keys, with no locks and no waits:
//   1. per-instance bounding box -> root cube (lower corner = per-axis min,
//      edge s0 = max extent * (1 + 2^-20));
//   2. key = instance bits | Morton interleave of the cell index
//      k = floor((x - min) / s0 * 2^B) (B bits per axis);
//   3. LSD radix sort of (key, particle) pairs, 8-bit digits, stable;
//   4. every slot i that starts a cell at some level emits that cell as a
//      node if its parent cell holds more than L particles; slot order then
//      level order is exactly pre-order, so the subtree of a node is the
//      contiguous id range [id, skip[id]) and walks need no stack;
//   5. node mass, centre of mass and tight box bottom-up: the last child to
//      arrive (atomic counter) combines its siblings in child order, so the
//      result does not depend on arrival order.
#include <climits>

#include "sph_internal.cuh"
#include "fpbits.cuh"
#include "morton.cuh"
#include "pack.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// Bounding boxes and validity
// ---------------------------------------------------------------------------
__global__ void k_bbox_init(unsigned long long *bb, int ninst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ninst) {
    for (int ax = 0; ax < 3; ++ax) {
      bb[6 * i + ax] = dbl_to_ord(__longlong_as_double(0x7ff0000000000000LL));       // +inf
      bb[6 * i + 3 + ax] = dbl_to_ord(__longlong_as_double((long long)0xfff0000000000000ULL));  // -inf
    }
  }
}

// min / max of order-preserving encodings (integer pipe)
__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// One block per instance when several instances are given; otherwise a
// grid-stride pass.  Also flags non-finite positions/velocities and h, rho
// that are not positive.
__global__ void k_bbox(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                       const double *__restrict__ vx, const double *__restrict__ vy, const double *__restrict__ vz,
                       const double *__restrict__ h, const double *__restrict__ rho, int64_t n, int dim,
                       const int64_t *__restrict__ inst_off, int ninst, unsigned long long *bb, int32_t *err) {
  // extrema as order-preserving integers: comparisons stay off the FP64 unit
  unsigned long long lo[3] = {~0ULL, ~0ULL, ~0ULL}, hi[3] = {0ULL, 0ULL, 0ULL};
  int64_t i0, i1, stride;
  int inst;
  if (ninst > 1 && inst_off) {
    inst = blockIdx.x;
    i0 = inst_off[inst] + threadIdx.x;
    i1 = inst_off[inst + 1];
    stride = blockDim.x;
  } else {
    inst = 0;
    i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    i1 = n;
    stride = (int64_t)gridDim.x * blockDim.x;
  }
  bool bad = false;
  for (int64_t i = i0; i < i1; i += stride) {
    const double p[3] = {x[i], y[i], dim == 3 ? z[i] : 0.0};
    bad |= !finite_bits(p[0]) || !finite_bits(p[1]) || !finite_bits(p[2]) || !finite_bits(vx[i]) ||
           !finite_bits(vy[i]) || (dim == 3 && !finite_bits(vz[i])) || !positive_finite_bits(h[i]) ||
           !positive_finite_bits(rho[i]);
    for (int ax = 0; ax < 3; ++ax) {
      const unsigned long long o = ord_of(p[ax]);
      lo[ax] = o < lo[ax] ? o : lo[ax];
      hi[ax] = o > hi[ax] ? o : hi[ax];
    }
  }
  if (bad) raise_err(err, ERR_NONFINITE);
  __shared__ unsigned long long s[6][32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int ax = 0; ax < 3; ++ax) {
    unsigned long long a = warp_min_u64(lo[ax]), b = warp_max_u64(hi[ax]);
    if (lane == 0) {
      s[ax][w] = a;
      s[3 + ax][w] = b;
    }
  }
  __syncthreads();
  if (w == 0) {
    for (int ax = 0; ax < 3; ++ax) {
      unsigned long long a = lane < nw ? s[ax][lane] : ~0ULL;
      unsigned long long b = lane < nw ? s[3 + ax][lane] : 0ULL;
      a = warp_min_u64(a);
      b = warp_max_u64(b);
      if (lane == 0) {
        atomicMin(&bb[6 * inst + ax], a);
        atomicMax(&bb[6 * inst + 3 + ax], b);
      }
    }
  }
}

// Root cube per instance (Sect. 3.5.1): corner = per-axis minimum, edge
// s0 = max over axes of the extent, enlarged by 2^-20 so that the particle
// at the maximum falls inside; a zero extent (one particle) gives s0 = 1.
__global__ void k_root(const unsigned long long *bb, int ninst, int dim, double *lo_out, double *s0_out,
                       double *rs0_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  double ext = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    double lo = ord_to_dbl(bb[6 * i + ax]), hi = ord_to_dbl(bb[6 * i + 3 + ax]);
    if (ax >= dim || !(hi >= lo)) {  // unused axis or empty instance
      lo = 0.0;
      hi = 0.0;
    }
    lo_out[3 * i + ax] = lo;
    ext = fmax(ext, __dsub_rn(hi, lo));
  }
  double s0 = __dmul_rn(ext, 1.0 + 0x1p-20);
  s0 = s0 > 0.0 ? s0 : 1.0;
  s0_out[i] = s0;
  rs0_out[i] = __drcp_rn(s0);
}

__global__ void k_keys(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                       int64_t n, int dim, int B, const int64_t *__restrict__ inst_off, int ninst,
                       const double *__restrict__ ilo, const double *__restrict__ is0,
                       const double *__restrict__ irs0, unsigned long long *keys, int32_t *vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int inst = inst_of(inst_off, ninst, i);
  const double s0 = is0[inst], rs0 = irs0[inst];
  unsigned long long kx = cell_index_fast(x[i], ilo[3 * inst + 0], s0, rs0, B);
  unsigned long long ky = cell_index_fast(y[i], ilo[3 * inst + 1], s0, rs0, B);
  unsigned long long key;
  if (dim == 3) {
    unsigned long long kz = cell_index_fast(z[i], ilo[3 * inst + 2], s0, rs0, B);
    key = spread3(kx) | (spread3(ky) << 1) | (spread3(kz) << 2);
  } else {
    key = spread2(kx) | (spread2(ky) << 1);
  }
  key |= (unsigned long long)inst << (dim * B);
  keys[i] = key;
  vals[i] = (int32_t)i;
}

// Code units from particle 0 (see Units).
__device__ __forceinline__ double pow2_floor(double v) { return (v > 0.0 && isfinite(v)) ? ldexp(1.0, ilogb(v)) : 1.0; }

__global__ void k_units(const double *__restrict__ h, const double *__restrict__ m, int64_t n, int dim,
                        double vscale, MatTable mt, Units *U) {
  // every lane forms the (power-of-two) base units; lane i converts material i
  const double L = pow2_floor(n > 0 ? h[0] : 1.0), M = pow2_floor(n > 0 ? m[0] : 1.0);
  const double T = pow2_floor(L / (vscale > 0.0 ? vscale : 1.0));
  Units u;
  u.L = L;
  u.M = M;
  u.T = T;
  u.invL = 1.0 / L;
  u.invM = 1.0 / M;
  u.invT = 1.0 / T;
  u.rho = dim == 3 ? M / (L * L * L) : M / (L * L);  // density: mass per L^D
  u.invrho = 1.0 / u.rho;
  u.V = L / T;
  u.invV = 1.0 / u.V;
  u.sig = dim == 3 ? M / (L * T * T) : M / (T * T);  // stress: rho V^2
  u.invsig = 1.0 / u.sig;
  u.E = u.V * u.V;
  u.invE = 1.0 / u.E;
  u.acc = L / (T * T);
  u.Gs = 0.0;
  const int i = threadIdx.x;
  if (i < SPH_MAX_MATERIALS) {
    const sph_material &a = mt.m[i < mt.nmat ? i : 0];
    float *f = U->matf[i];
    f[MF_RHO0] = (float)(a.rho0 * u.invrho);
    f[MF_CS] = (float)(a.cs * u.invV);
    f[MF_K0] = (float)(a.K0 * u.invsig);
    f[MF_NM] = (float)a.n_M;
    f[MF_AT] = (float)(a.A_T * u.invsig);
    f[MF_BT] = (float)(a.B_T * u.invsig);
    f[MF_E0] = (float)(a.E0 * u.invE);
    f[MF_EIV] = (float)(a.E_iv * u.invE);
    f[MF_ECV] = (float)(a.E_cv * u.invE);
    f[MF_AA] = (float)a.a_T;
    f[MF_BB] = (float)a.b_T;
    f[MF_ALPHA] = (float)a.alpha_T;
    f[MF_BETA] = (float)a.beta_T;
    f[MF_RHOCUT] = (float)a.rho_cut;
    f[MF_MU] = (float)(a.mu * u.invsig);
    f[MF_Y0] = (float)(a.Y0 * u.invsig);
  }
  if (threadIdx.x == 0) {
    // base fields only: the material rows are written by their lanes
    U->L = u.L;
    U->M = u.M;
    U->T = u.T;
    U->invL = u.invL;
    U->invM = u.invM;
    U->invT = u.invT;
    U->rho = u.rho;
    U->invrho = u.invrho;
    U->V = u.V;
    U->invV = u.invV;
    U->sig = u.sig;
    U->invsig = u.invsig;
    U->E = u.E;
    U->invE = u.invE;
    U->acc = u.acc;
    U->Gs = u.Gs;
  }
}

// FP32 views of the state (see PackedF32), in code units.
__global__ void k_pack(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                       const double *__restrict__ vx, const double *__restrict__ vy, const double *__restrict__ vz,
                       const double *__restrict__ h, const double *__restrict__ m, const double *__restrict__ rho,
                       int64_t n, int dim, const int64_t *__restrict__ inst_off, int ninst,
                       const double *__restrict__ ilo, const Units *__restrict__ U, PackedF32 pk) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int inst = inst_of(inst_off, ninst, i);
  pack_particle(pk, i, dim, x[i], y[i], dim == 3 ? z[i] : 0.0, vx[i], vy[i], dim == 3 ? vz[i] : 0.0, h[i], m[i],
                rho[i], ilo + 3 * inst, U);
}

// ---------------------------------------------------------------------------
// LSD radix sort of (u64 key, i32 value), 8-bit digits, stable.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const unsigned long long *__restrict__ keys, int64_t n,
                                                             int shift, uint32_t *hist, int nblocks) {
  __shared__ uint32_t hs[256];
  hs[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = base + it * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&hs[(keys[i] >> shift) & 255], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = hs[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const unsigned long long *__restrict__ kin,
                                                                const int32_t *__restrict__ vin,
                                                                unsigned long long *__restrict__ kout,
                                                                int32_t *__restrict__ vout, int64_t n, int shift,
                                                                const uint32_t *__restrict__ hist, int nblocks) {
  __shared__ uint32_t off[256];
  __shared__ uint32_t wc[kSortThreads / 32][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  off[threadIdx.x] = hist[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  const unsigned lt = (1u << lane) - 1u;
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = base + it * kSortThreads + threadIdx.x;
    bool valid = i < n;
    unsigned long long key = valid ? kin[i] : 0ULL;
    int32_t val = valid ? vin[i] : 0;
    int d = valid ? (int)((key >> shift) & 255) : 256;
#pragma unroll
    for (int ww = 0; ww < kSortThreads / 32; ++ww) wc[ww][threadIdx.x] = 0;
    __syncthreads();
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank = __popc(peers & lt);
    if (valid && rank == 0) wc[w][d] = __popc(peers);
    __syncthreads();
    uint32_t tot = 0;
    {
      int dd = threadIdx.x;
#pragma unroll
      for (int ww = 0; ww < kSortThreads / 32; ++ww) {
        uint32_t t = wc[ww][dd];
        wc[ww][dd] = tot;
        tot += t;
      }
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = off[d] + wc[w][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    off[threadIdx.x] += tot;
    __syncthreads();
  }
}

static void scan_excl_i32(const int32_t *in, int32_t *out, int64_t m, int32_t *tmp, cudaStream_t st);

static void radix_sort(sph_ctx *c, int64_t n, int bits, cudaStream_t st) {
  Tree &T = c->tree;
  int nblocks = nblk(n, kSortTile);
  int passes = (bits + 7) / 8;
  int src = 0;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    { k_radix_hist<<<nblocks, kSortThreads, 0, st>>>(T.keys[src], n, shift, T.hist, nblocks); ++sph::g_launches; }
    scan_excl_i32((const int32_t *)T.hist, (int32_t *)T.hist, (int64_t)256 * nblocks, T.scan_tmp, st);
    { k_radix_scatter<<<nblocks, kSortThreads, 0, st>>>(T.keys[src], T.vals[src], T.keys[src ^ 1], T.vals[src ^ 1], n,
                                                     shift, T.hist, nblocks); ++sph::g_launches; }
    src ^= 1;
  }
  T.skey = T.keys[src];
  T.perm = T.vals[src];
}

// Sorts (keys[0], vals[0]) of the tree's sort buffers; the result is left
// in (skey, perm).  Used outside the tree build by the flaw generator and the
// fragment finder, which do not need the tree afterwards.
void sort_pairs(sph_ctx *c, int64_t n, int bits, cudaStream_t st) {
  if (n > 0) {
    radix_sort(c, n, bits, st);
  } else {
    c->tree.skey = c->tree.keys[0];
    c->tree.perm = c->tree.vals[0];
  }
}

// ---------------------------------------------------------------------------
// Exclusive scan of int32 counts (length m), three phases.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256, kScanItems = 16, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *total) {
  __shared__ int32_t ws[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t s = v;
  for (int o = 1; o < 32; o <<= 1) {
    int32_t t = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) s += t;
  }
  if (lane == 31) ws[w] = s;
  __syncthreads();
  if (w == 0) {
    int32_t t = lane < nw ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    ws[lane] = t;
  }
  __syncthreads();
  int32_t res = s - v + (w > 0 ? ws[w - 1] : 0);
  *total = ws[nw - 1];
  __syncthreads();
  return res;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int32_t *__restrict__ in, int32_t *__restrict__ out,
                                                             int64_t m, int32_t *tile_sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < m) ? in[base + k] : 0;
    s += v[k];
  }
  int32_t tot;
  int32_t off = block_excl_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < m) out[base + k] = off;
    off += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_tops(int32_t *t, int m) {
  int chunk = (m + 1023) / 1024;
  int b = threadIdx.x * chunk, e = min(m, b + chunk);
  int32_t s = 0;
  for (int i = b; i < e; ++i) s += t[i];
  int32_t tot;
  int32_t off = block_excl_scan(s, &tot);
  for (int i = b; i < e; ++i) {
    int32_t x = t[i];
    t[i] = off;
    off += x;
  }
}

__global__ void k_scan_add(int32_t *out, int64_t m, const int32_t *tile_sums) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] += tile_sums[i / kScanTile];
}

static void scan_excl_i32(const int32_t *in, int32_t *out, int64_t m, int32_t *tmp, cudaStream_t st) {
  int tiles = nblk(m, kScanTile);
  { k_scan_tiles<<<tiles, kScanThreads, 0, st>>>(in, out, m, tmp); ++sph::g_launches; }
  { k_scan_tops<<<1, 1024, 0, st>>>(tmp, tiles); ++sph::g_launches; }
  { k_scan_add<<<nblk(m, 256), 256, 0, st>>>(out, m, tmp); ++sph::g_launches; }
}

void scan_counts(sph_ctx *c, const int32_t *in, int32_t *out, int64_t m, cudaStream_t st) {
  scan_excl_i32(in, out, m, c->tree.scan_tmp, st);
}

// ---------------------------------------------------------------------------
// Node emission
// ---------------------------------------------------------------------------
struct KeyLevels {
  const unsigned long long *key;
  int dim, B;
  __device__ __forceinline__ unsigned long long prefix(int64_t i, int l) const { return key[i] >> (dim * (B - l)); }
  // deepest level at which slots i-1 and i share a cell; -1 if they lie in
  // different instances
  __device__ __forceinline__ int common(int64_t i) const {
    unsigned long long d = key[i] ^ key[i - 1];
    if (d == 0) return B;
    int hb = 63 - __clzll((long long)d);
    if (hb >= dim * B) return -1;
    return B - 1 - hb / dim;
  }
  // first slot in [lo, hi) whose level-l prefix exceeds p
  __device__ __forceinline__ int64_t upper(unsigned long long p, int l, int64_t lo, int64_t hi) const {
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (prefix(mid, l) <= p) lo = mid + 1; else hi = mid;
    }
    return lo;
  }
  // first slot in [lo, hi) whose level-l prefix is >= p
  __device__ __forceinline__ int64_t lower(unsigned long long p, int l, int64_t lo, int64_t hi) const {
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (prefix(mid, l) < p) lo = mid + 1; else hi = mid;
    }
    return lo;
  }
};

__device__ __forceinline__ void slot_segment(const int64_t *inst_off, int ninst, int64_t n, int64_t i, int64_t &lo,
                                             int64_t &hi) {
  if (ninst > 1 && inst_off) {
    int k = inst_of(inst_off, ninst, i);
    lo = inst_off[k];
    hi = inst_off[k + 1];
  } else {
    lo = 0;
    hi = n;
  }
}

// First level at which slot i starts a cell that is a node, or B+1 if none.
__device__ __forceinline__ int first_node_level(const KeyLevels &K, int64_t i, int64_t seg_lo, int64_t seg_hi,
                                                int L) {
  int c = (i == seg_lo) ? -1 : K.common(i);
  int l0 = c + 1;
  if (l0 > K.B) return K.B + 1;
  if (l0 > 0) {
    unsigned long long pp = K.prefix(i, l0 - 1);
    int64_t lo = K.lower(pp, l0 - 1, max(seg_lo, i - L), i);
    int64_t hi = K.upper(pp, l0 - 1, i + 1, min(seg_hi, i + L + 1));
    if (hi - lo <= L) return K.B + 1;  // the parent cell is a leaf (or lies below one)
  }
  return l0;
}

__global__ void k_node_count(KeyLevels K, int64_t n, int L, const int64_t *__restrict__ inst_off, int ninst,
                             int32_t *cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) {
    cnt[n] = 0;
    return;
  }
  int64_t seg_lo, seg_hi;
  slot_segment(inst_off, ninst, n, i, seg_lo, seg_hi);
  int l0 = first_node_level(K, i, seg_lo, seg_hi, L);
  int k = 0;
  int64_t e = seg_hi;
  for (int l = l0; l <= K.B; ++l) {
    int64_t end = K.upper(K.prefix(i, l), l, i + 1, e);
    ++k;
    if (end - i <= L || l == K.B) break;
    e = end;
  }
  cnt[i] = k;
}

__global__ void k_node_emit(KeyLevels K, int64_t n, int L, const int64_t *__restrict__ inst_off, int ninst,
                            const int32_t *__restrict__ nstart, Tree T, int32_t *err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) {
    *T.nnodes = nstart[n] <= T.cap_nodes ? nstart[n] : (int32_t)T.cap_nodes;
    if (nstart[n] > T.cap_nodes) raise_err(err, ERR_NODE_OVERFLOW);
    return;
  }
  if (nstart[i + 1] == nstart[i]) return;
  int64_t seg_lo, seg_hi;
  slot_segment(inst_off, ninst, n, i, seg_lo, seg_hi);
  int l0 = first_node_level(K, i, seg_lo, seg_hi, L);
  int32_t parent = -1;
  if (l0 > 0) {
    // the parent cell starts at slot p; its node is the (l0-1 - l0(p))-th of p's chain
    unsigned long long pp = K.prefix(i, l0 - 1);
    int64_t p = K.lower(pp, l0 - 1, seg_lo, i);
    int lp = (p == seg_lo) ? 0 : K.common(p) + 1;
    parent = nstart[p] + (l0 - 1 - lp);
  }
  int64_t e = seg_hi;
  int32_t id = nstart[i];
  for (int l = l0; l <= K.B; ++l, ++id) {
    int64_t end = K.upper(K.prefix(i, l), l, i + 1, e);
    if (id < T.cap_nodes) {
      T.first[id] = (int32_t)i;
      T.end[id] = (int32_t)end;
      T.level[id] = l;
      T.cell[id] = K.prefix(i, l);
      T.skip[id] = min((int64_t)nstart[end], T.cap_nodes);
      T.nrec[id] = make_int4((int32_t)i, (int32_t)end, T.skip[id], l);
      T.parent[id] = parent;
      if (parent >= 0) {
        const int r = atomicAdd(&T.nchild[parent], 1);
        if (r < 8) T.child[8 * (int64_t)parent + r] = id;
      }
    }
    parent = id;
    if (end - i <= L || l == K.B) break;
    e = end;
  }
  // the chain ends at a leaf: list it for the moments pass
  if (id < T.cap_nodes) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(T.nleaf, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    T.ncount[base + __popc(mask & ((1u << lane) - 1u))] = id;
  }
}

__global__ void k_inst_roots(const int64_t *__restrict__ inst_off, int ninst, int64_t n, const int32_t *nstart,
                             Tree T) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  int64_t lo = 0, hi = n;
  if (ninst > 1 && inst_off) {
    lo = inst_off[i];
    hi = inst_off[i + 1];
  }
  T.inst_root[i] = (hi > lo) ? nstart[lo] : -1;
}

// Walk groups: runs of consecutive sibling cells that each hold at most 32
// particles, packed greedily up to 32 particles by their parent (a node with
// more than 32); a root with at most 32 particles is one group, and a leaf at
// full depth with more than 32 is cut into runs of 32.  Siblings are adjacent
// in Morton order, so a group is a compact block of space, and together the
// groups partition the particles in slot order.
__device__ __forceinline__ int node_count(const Tree &T, int32_t id) { return T.end[id] - T.first[id]; }

template <bool EMIT>
__device__ int group_runs(const Tree &T, int32_t id, int32_t g0, int inst) {
  const int c = node_count(T, id);
  const bool leaf = c <= T.leaf_size || T.level[id] == T.max_depth;
  int g = 0;
  if (c <= kWarp) {
    if (T.parent[id] >= 0) return 0;  // packed by its parent
    if (EMIT && g0 < T.cap_groups) {
      T.grp_start[g0] = T.first[id];
      T.grp_end[g0] = T.end[id];
      T.grp_inst[g0] = inst;
    }
    return 1;
  }
  if (leaf) {
    const int32_t f = T.first[id], e = T.end[id];
    for (int32_t s = f; s < e; s += kWarp, ++g)
      if (EMIT && g0 + g < T.cap_groups) {
        T.grp_start[g0 + g] = s;
        T.grp_end[g0 + g] = min(s + kWarp, e);
        T.grp_inst[g0 + g] = inst;
      }
    return g;
  }
  int32_t run_s = -1, run_e = -1;
  int run = 0;
  const int32_t stop = T.skip[id];
  int guard = 0;
  for (int32_t ch = id + 1; ch < stop && guard < 64; ch = T.skip[ch], ++guard) {
    const int cc = node_count(T, ch);
    if (cc <= kWarp && run + cc <= kWarp) {
      if (run == 0) run_s = T.first[ch];
      run += cc;
      run_e = T.end[ch];
      continue;
    }
    if (run > 0) {  // close the current run
      if (EMIT && g0 + g < T.cap_groups) {
        T.grp_start[g0 + g] = run_s;
        T.grp_end[g0 + g] = run_e;
        T.grp_inst[g0 + g] = inst;
      }
      ++g;
      run = 0;
    }
    if (cc <= kWarp) {  // starts a new run
      run_s = T.first[ch];
      run_e = T.end[ch];
      run = cc;
    }
  }
  if (run > 0) {
    if (EMIT && g0 + g < T.cap_groups) {
      T.grp_start[g0 + g] = run_s;
      T.grp_end[g0 + g] = run_e;
      T.grp_inst[g0 + g] = inst;
    }
    ++g;
  }
  return g;
}

__global__ void k_group_count(Tree T, int32_t *gcnt) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id > T.cap_nodes) return;
  const int nn = *T.nnodes;
  gcnt[id] = id < nn ? group_runs<false>(T, (int32_t)id, 0, 0) : 0;
}

__global__ void k_group_emit(Tree T, const int32_t *__restrict__ gstart, const int64_t *__restrict__ inst_off,
                             int ninst) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = *T.nnodes;
  if (id == 0) *T.ngroups = min(gstart[nn], (int32_t)T.cap_groups);
  if (id >= nn || gstart[id + 1] == gstart[id]) return;
  group_runs<true>(T, (int32_t)id, gstart[id], inst_of(inst_off, ninst, T.first[id]));
}

// ---------------------------------------------------------------------------
// Node moments, bottom-up
// ---------------------------------------------------------------------------

// Bottom-up sums, one thread per leaf: mass, the mass-weighted position sum
// (kept in T.com until k_node_finish divides it), the particle box and h_max.
// The last child to arrive combines its parent's children in id order, so the
// sums are deterministic.  Extrema are kept as order-preserving integers and
// h_max as the bits of a positive double: only the sums use the FP64 unit.
__global__ void k_moments(Tree T, const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ z, const double *__restrict__ m, const double *__restrict__ h,
                          int dim) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= *T.nleaf) return;
  const int64_t id = T.ncount[tid];  // one thread per leaf
  int32_t f = T.first[id], e = T.end[id];
  const double *X[3] = {x, y, z};
  const int64_t cap = T.cap_nodes;
  double M = 0.0, mx[3] = {0, 0, 0};
  unsigned long long lo[3] = {~0ULL, ~0ULL, ~0ULL}, hi[3] = {0ULL, 0ULL, 0ULL};
  unsigned long long hm = 0ULL;
  for (int32_t j = f; j < e; ++j) {
    int32_t a = T.perm[j];
    double ma = m[a];
    M += ma;
    const unsigned long long hb = dbits(h[a]);
    hm = hb > hm ? hb : hm;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if (ax >= dim) break;
      double v = X[ax][a];
      mx[ax] += ma * v;
      const unsigned long long o = ord_of(v);
      lo[ax] = o < lo[ax] ? o : lo[ax];
      hi[ax] = o > hi[ax] ? o : hi[ax];
    }
  }
  int64_t node = id;
  for (int depth = 0; depth < 64; ++depth) {
    T.mass[node] = M;
    T.hmax[node] = bitsd(hm);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const bool use = ax < dim;
      T.com[ax * cap + node] = use ? mx[ax] : 0.0;
      T.bblo[ax * cap + node] = use ? of_ord(lo[ax]) : 0.0;
      T.bbhi[ax * cap + node] = use ? of_ord(hi[ax]) : 0.0;
    }
    int32_t p = T.parent[node];
    if (p < 0) return;
    __threadfence();
    int old = atomicAdd(&T.arrived[p], 1);
    if (old != T.nchild[p] - 1) return;
    __threadfence();
    // last child in: combine all children of p, in ascending id (= child) order
    M = 0.0;
    hm = 0ULL;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      mx[ax] = 0.0;
      lo[ax] = ~0ULL;
      hi[ax] = 0ULL;
    }
    const int nc = min(T.nchild[p], 8);
    int32_t ch[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) ch[k] = k < nc ? __ldcg(&T.child[8 * (int64_t)p + k]) : INT_MAX;
    // odd-even transposition sort of the 8 slots (unused slots sort last)
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int k = r & 1; k + 1 < 8; k += 2) {
        const int32_t a = min(ch[k], ch[k + 1]), b = max(ch[k], ch[k + 1]);
        ch[k] = a;
        ch[k + 1] = b;
      }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (k >= nc) break;
      const int32_t cc = ch[k];
      M += __ldcg(&T.mass[cc]);
      const unsigned long long hb = dbits(__ldcg(&T.hmax[cc]));
      hm = hb > hm ? hb : hm;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        if (ax >= dim) break;
        mx[ax] += __ldcg(&T.com[ax * cap + cc]);
        const unsigned long long ol = ord_of(__ldcg(&T.bblo[ax * cap + cc]));
        const unsigned long long oh = ord_of(__ldcg(&T.bbhi[ax * cap + cc]));
        lo[ax] = ol < lo[ax] ? ol : lo[ax];
        hi[ax] = oh > hi[ax] ? oh : hi[ax];
      }
    }
    node = p;
  }
}

// Per node, all warps full: centre of mass from the sums, and the FP32 words
// of the walks in code units relative to the instance corner - the box rounded
// outwards with +-h_max (negative where the partner walk stops: at most
// max(L, walk_leaf) particles or depth B) and skip[], and the COM as hi + lo
// with the mass and the cell edge s0 / 2^level.
__global__ void k_node_finish(Tree T, int dim, int L, const int64_t *__restrict__ inst_off, int ninst,
                              const Units *__restrict__ U, int walk_leaf) {
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= *T.nnodes) return;
  const int Lw = max(L, walk_leaf);
  const int64_t cap = T.cap_nodes;
  const int32_t nf = T.first[node], ne = T.end[node];
  const int inst = inst_of(inst_off, ninst, nf);
  const int kL = pow2_exp(U->invL), kM = pow2_exp(U->invM);
  const double M = T.mass[node], iM = 1.0 / M, hmax = T.hmax[node];
  float bl[3] = {0.f, 0.f, 0.f}, bh[3] = {0.f, 0.f, 0.f}, chi[3] = {0.f, 0.f, 0.f}, clo[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (ax >= dim) break;
    const double ilo = T.inst_lo[3 * inst + ax];
    const double com = T.com[ax * cap + node] * iM;
    T.com[ax * cap + node] = com;
    const double dl = __dsub_rn(T.bblo[ax * cap + node], ilo), dh = __dsub_rn(T.bbhi[ax * cap + node], ilo);
    bl[ax] = to_f32_dir_scaled(dl, kL, false, U->invL);
    bh[ax] = to_f32_dir_scaled(dh, kL, true, U->invL);
    to_f32_split_scaled(__dsub_rn(com, ilo), kL, U->invL, chi[ax], clo[ax]);
  }
  const float hf = to_f32_dir_scaled(hmax, kL, true, U->invL), mf = to_f32_scaled(M, kM, U->invM);
  const int lev = T.level[node];
  // edge s0 / 2^level: one exponent shift (the fallback's scale 2^(kL - level)
  // is built from its bits)
  const float ef = to_f32_scaled(T.inst_s0[inst], kL - lev, bitsd((uint64_t)(1023 + kL - lev) << 52));
  const bool stop = ne - nf <= Lw || lev == T.max_depth;
  // the gravity walk's word: skip, level and whether the walk sums the node's
  // members directly (its leaf test); the edge follows from the level
  const bool gleaf = ne - nf <= L || lev == T.max_depth;
  const float wf = T.packed_walk ? __uint_as_float((uint32_t)T.skip[node] | ((uint32_t)lev << 26) |
                                                   (gleaf ? 0x80000000u : 0u))
                                 : ef;
  T.fbox_lo[node] = make_float4(bl[0], bl[1], bl[2], stop ? -hf : hf);
  T.fbox_hi[node] = make_float4(bh[0], bh[1], bh[2], __int_as_float(T.skip[node]));
  T.fcom_hi[node] = make_float4(chi[0], chi[1], chi[2], mf);
  T.fcom_lo[node] = make_float4(clo[0], clo[1], clo[2], wf);
}

// ---------------------------------------------------------------------------
// Host orchestration
// ---------------------------------------------------------------------------
void pack_f32(sph_ctx *c, const sph_state *s, cudaStream_t st) {
  int64_t n = s->n;
  if (n == 0) return;
  { k_pack<<<nblk(n, 256), 256, 0, st>>>(s->x[0], s->x[1], s->x[2], s->v[0], s->v[1], s->v[2], s->h, s->m, s->rho, n,
                                       s->dim, s->inst_off, s->ninst, c->tree.inst_lo, c->units, c->pk); ++sph::g_launches; }
}

void tree_build(sph_ctx *c, const sph_state *s, int leaf_size, int max_depth, cudaStream_t st) {
  Tree &T = c->tree;
  const int64_t n = s->n;
  const int ninst = s->ninst > 0 ? s->ninst : 1;
  const int dim = s->dim;
  T.leaf_size = leaf_size;
  T.max_depth = max_depth;
  T.packed_walk = (c->tune.plain_forms == 0 && T.cap_nodes <= kPackedSkip && max_depth <= 31) ? 1 : 0;
  T.perm_identity = 0;
  T.dim = dim;
  T.ninst = ninst;
  T.n = n;
  { k_bbox_init<<<nblk(ninst, 128), 128, 0, st>>>(T.inst_bb, ninst); ++sph::g_launches; }
  if (n > 0) {
    if (ninst > 1)
      { k_bbox<<<ninst, 256, 0, st>>>(s->x[0], s->x[1], s->x[2], s->v[0], s->v[1], s->v[2], s->h, s->rho, n, dim,
                                   s->inst_off, ninst, T.inst_bb, c->d_err); ++sph::g_launches; }
    else
      { k_bbox<<<min(nblk(n, 256), 152 * 8), 256, 0, st>>>(s->x[0], s->x[1], s->x[2], s->v[0], s->v[1], s->v[2], s->h,
                                                        s->rho, n, dim, nullptr, 1, T.inst_bb, c->d_err); ++sph::g_launches; }
  }
  { k_root<<<nblk(ninst, 128), 128, 0, st>>>(T.inst_bb, ninst, dim, T.inst_lo, T.inst_s0, T.inst_rs0); ++sph::g_launches; }
  { k_units<<<1, 32, 0, st>>>(s->h, s->m, n, dim, c->vscale, c->mt, c->units); ++sph::g_launches; }
  if (n > 0) {
    { k_keys<<<nblk(n, 256), 256, 0, st>>>(s->x[0], s->x[1], s->x[2], n, dim, max_depth, s->inst_off, ninst,
                                         T.inst_lo, T.inst_s0, T.inst_rs0, T.keys[0], T.vals[0]); ++sph::g_launches; }
    int ibits = 0;
    while ((1 << ibits) < ninst) ++ibits;
    radix_sort(c, n, dim * max_depth + ibits, st);
  } else {
    T.skey = T.keys[0];
    T.perm = T.vals[0];
  }
  pack_f32(c, s, st);
  KeyLevels K{T.skey, dim, max_depth};
  { k_node_count<<<nblk(n + 1, 256), 256, 0, st>>>(K, n, leaf_size, s->inst_off, ninst, T.ncount); ++sph::g_launches; }
  scan_excl_i32(T.ncount, T.nstart, n + 1, T.scan_tmp, st);
  cudaMemsetAsync(T.nchild, 0, sizeof(int32_t) * T.cap_nodes, st);
  cudaMemsetAsync(T.arrived, 0, sizeof(int32_t) * T.cap_nodes, st);
  cudaMemsetAsync(T.nleaf, 0, sizeof(int32_t), st);
  { k_node_emit<<<nblk(n + 1, 256), 256, 0, st>>>(K, n, leaf_size, s->inst_off, ninst, T.nstart, T, c->d_err); ++sph::g_launches; }
  { k_moments<<<nblk(std::max<int64_t>(n, 1), 256), 256, 0, st>>>(T, s->x[0], s->x[1], s->x[2], s->m, s->h,
                                                                   dim); ++sph::g_launches; }
  { k_node_finish<<<nblk(T.cap_nodes, 256), 256, 0, st>>>(T, dim, leaf_size, s->inst_off, ninst, c->units,
                                                        c->tune.walk_leaf); ++sph::g_launches; }
  { k_inst_roots<<<nblk(ninst, 128), 128, 0, st>>>(s->inst_off, ninst, n, T.nstart, T); ++sph::g_launches; }
  { k_group_count<<<nblk(T.cap_nodes + 1, 256), 256, 0, st>>>(T, T.gcnt); ++sph::g_launches; }
  scan_excl_i32(T.gcnt, T.gstart, T.cap_nodes + 1, T.scan_tmp, st);
  { k_group_emit<<<nblk(T.cap_nodes, 256), 256, 0, st>>>(T, T.gstart, s->inst_off, ninst); ++sph::g_launches; }
}

// ---------------------------------------------------------------------------
// In-place reorder of the caller's state along the tree
// ---------------------------------------------------------------------------
__global__ void k_iota(int32_t *p, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int32_t)i;
}

// All fields at once: dst_f[i] = src_f[perm[i]] (gather) or dst_f[i] = src_f[i]
// (copy back), doubles then ints.
constexpr int kMaxFields = 20;
struct FieldSet {
  const double *dsrc[kMaxFields];
  double *ddst[kMaxFields];
  const int32_t *isrc[2];
  int32_t *idst[2];
  int nd, ni;
};

__global__ void k_gather_fields(FieldSet F, const int32_t *__restrict__ perm, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t j = perm ? perm[i] : i;
#pragma unroll 4
  for (int f = 0; f < F.nd; ++f) F.ddst[f][i] = F.dsrc[f][j];
  for (int f = 0; f < F.ni; ++f) F.idst[f][i] = F.isrc[f][j];
}

void tree_reorder_state(sph_ctx *c, sph_state *s, cudaStream_t st) {
  const int64_t n = s->n;
  if (n == 0) return;
  // scratch: the predicted-state and derivative buffers, free at this point
  StepBufs &B = c->st;
  double *scratch[kMaxFields] = {B.x[0], B.x[1], B.x[2], B.v[0], B.v[1], B.v[2], B.rho, B.u, B.dmg,
                                 B.d_x[0][0], B.d_x[0][1], B.d_x[0][2], B.d_v[0][0], B.d_v[0][1],
                                 B.d_v[0][2], B.d_rho[0], B.d_u[0], B.d_dmg[0], B.d_cs[0], B.gather};
  FieldSet G, R;
  memset(&G, 0, sizeof(G));
  auto add = [&](double *f) {
    if (!f) return;
    G.dsrc[G.nd] = f;
    G.ddst[G.nd] = scratch[G.nd];
    ++G.nd;
  };
  for (int ax = 0; ax < s->dim; ++ax) {
    add(s->x[ax]);
    add(s->v[ax]);
  }
  add(s->rho);
  add(s->u);
  add(s->m);
  add(s->h);
  add(s->dmg);
  if (s->S)
    for (int k = 0; k < nsym(s->dim); ++k) add(s->S + (int64_t)k * n);
  int32_t *iscr[2] = {B.gather_i, B.d_nact[0]};
  if (s->mat) {
    G.isrc[G.ni] = s->mat;
    G.idst[G.ni] = iscr[G.ni];
    ++G.ni;
  }
  if (s->id) {
    G.isrc[G.ni] = s->id;
    G.idst[G.ni] = iscr[G.ni];
    ++G.ni;
  }
  R = G;
  for (int f = 0; f < G.nd; ++f) {
    R.dsrc[f] = G.ddst[f];
    R.ddst[f] = const_cast<double *>(G.dsrc[f]);
  }
  for (int f = 0; f < G.ni; ++f) {
    R.isrc[f] = G.idst[f];
    R.idst[f] = const_cast<int32_t *>(G.isrc[f]);
  }
  { k_gather_fields<<<nblk(n, 256), 256, 0, st>>>(G, c->tree.perm, n); ++sph::g_launches; }
  { k_gather_fields<<<nblk(n, 256), 256, 0, st>>>(R, nullptr, n); ++sph::g_launches; }
  { k_iota<<<nblk(n, 256), 256, 0, st>>>(c->tree.perm, n); ++sph::g_launches; }
  c->tree.perm_identity = 1;
  pack_f32(c, s, st);
}

// ---------------------------------------------------------------------------
// Node export (tests)
// ---------------------------------------------------------------------------
__global__ void k_export_nodes(Tree T, int64_t cap, int dim, int32_t *level, int64_t *cell, int64_t *count,
                               double *mass, double *com) {
  int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int nn = *T.nnodes;
  if (id >= nn || id >= cap) return;
  int l = T.level[id];
  unsigned long long pre = T.cell[id] & ((l * dim >= 64) ? ~0ULL : ((1ULL << (l * dim)) - 1ULL));
  level[id] = l;
  count[id] = T.end[id] - T.first[id];
  mass[id] = T.mass[id];
  if (dim == 3) {
    cell[3 * id] = (int64_t)compact3(pre);
    cell[3 * id + 1] = (int64_t)compact3(pre >> 1);
    cell[3 * id + 2] = (int64_t)compact3(pre >> 2);
  } else {
    cell[3 * id] = (int64_t)compact2(pre);
    cell[3 * id + 1] = (int64_t)compact2(pre >> 1);
    cell[3 * id + 2] = 0;
  }
  for (int ax = 0; ax < 3; ++ax) com[3 * id + ax] = T.com[ax * T.cap_nodes + id];
}

void export_nodes(sph_ctx *c, int64_t cap, int32_t *level, int64_t *cell, int64_t *count, double *mass, double *com,
                  cudaStream_t st) {
  { k_export_nodes<<<nblk(cap, 256), 256, 0, st>>>(c->tree, cap, c->tree.dim, level, cell, count, mass, com); ++sph::g_launches; }
}

}  // namespace sph
