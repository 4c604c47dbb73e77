// Weibull activation thresholds on the device (Sect. 3.2, after Benz and
// Asphaug 1995).  For every group of brittle particles (one material in one
// instance) the sequential procedure hands flaw j = 1, 2, ... to a randomly
// drawn member, with threshold strain (j / (k V))^(1/m), until every member
// holds one.  Draw j is a counter-based random number (Philox4x64-10 with
// counter (j-1)/4 and key (seed, group)), so any draw can be made by any
// thread in any order, and the sequential result follows from two facts:
// the procedure stops at J = the largest, over members, of the first draw
// that hits the member, and the flaws are exactly draws 1..J.  So:
//   1. sort the particles by (group, id): the members of group g are the
//      sorted positions goff[g] .. goff[g+1];
//   2. V_g = sum m / rho0 over the members (chunks of members, one block
//      each, then each group's chunks in order: the same sum every run);
//   3. coverage rounds: make a batch of draws of every group that is not
//      yet covered and record, per member, the smallest j that hit it
//      (atomicMin); repeat for the groups with members still unhit;
//   4. J_g = the largest first hit; count the draws j <= J_g per particle,
//      scan the counts (indexed by id) into the CSR offsets, fill the
//      thresholds, and sort each particle's (short) list.
#include <math.h>

#include <algorithm>
#include <vector>

#include "sph_internal.cuh"

namespace sph {

void sort_pairs(sph_ctx *c, int64_t n, int bits, cudaStream_t st);
void scan_counts(sph_ctx *c, const int32_t *in, int32_t *out, int64_t m, cudaStream_t st);

namespace {

// Philox4x64-10 (Salmon, Moraes, Dror and Shaw 2011): ten rounds, each
// multiplying counter words 0 and 2 by the round multipliers into 128-bit
// products and recombining with the key; the key gains the Weyl increments
// before every round after the first.
__device__ __forceinline__ void philox4x64(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B97F4A7C15ULL;
      k1 += 0xBB67AE8584CAA73BULL;
    }
    const uint64_t m0 = 0xD2E7470EE14C6C93ULL, m1 = 0xCA5A826395121157ULL;
    const uint64_t hi0 = __umul64hi(m0, c[0]), lo0 = m0 * c[0];
    const uint64_t hi2 = __umul64hi(m1, c[2]), lo2 = m1 * c[2];
    const uint64_t n0 = hi2 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo2;
    c[2] = n2;
    c[3] = lo0;
  }
}

constexpr uint32_t kNoHit = 0xffffffffu;
constexpr int kIdBits = 31;
constexpr int kMaxRounds = 64;

struct FlawMats {
  double rho0[SPH_MAX_MATERIALS], k[SPH_MAX_MATERIALS], m[SPH_MAX_MATERIALS];
  int32_t brittle;  // bit per material
  int32_t nmat;
};

// (group, id) keys; particles that are not brittle sort last (group G)
__global__ void k_flaw_keys(const int32_t *__restrict__ mat, const int32_t *__restrict__ id, int64_t n,
                            const int64_t *__restrict__ inst_off, int ninst, FlawMats M, unsigned long long *keys,
                            int32_t *vals, int32_t *bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t G = (uint64_t)ninst * (uint64_t)M.nmat;
  const int32_t mt = mat[i], d = id[i];
  uint64_t g = G;
  if (d < 0 || (int64_t)d >= n || mt < 0 || mt >= M.nmat) {
    atomicOr(bad, 1);
  } else if ((M.brittle >> mt) & 1) {
    g = (uint64_t)inst_of(inst_off, ninst, i) * (uint64_t)M.nmat + (uint64_t)mt;
  }
  keys[i] = (g << kIdBits) | (uint64_t)(d < 0 ? 0 : d);
  vals[i] = (int32_t)i;
}

// goff[g] = first sorted position of group g (g = 0..G; goff[G] = number of
// brittle particles)
__global__ void k_flaw_bounds(const unsigned long long *__restrict__ skey, int64_t n, int64_t G, int32_t *goff) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > n) return;
  const int64_t g = p < n ? (int64_t)(skey[p] >> kIdBits) : G;
  const int64_t gp = p > 0 ? (int64_t)(skey[p - 1] >> kIdBits) : -1;
  for (int64_t q = gp + 1; q <= g && q <= G; ++q) goff[q] = (int32_t)p;
}

// V = sum over the members of m / rho0, in two deterministic steps: chunks
// of kVolChunk consecutive members (one block each, fixed reduction shape),
// then the chunks of a group in order.  log2(k V) and 1/m per group.
constexpr int kVolChunk = 4096;

__global__ void __launch_bounds__(256) k_flaw_vol_chunks(const int32_t *__restrict__ ck_g,
                                                         const int32_t *__restrict__ ck_lo,
                                                         const int32_t *__restrict__ ck_hi,
                                                         const int32_t *__restrict__ perm,
                                                         const double *__restrict__ m, FlawMats M, double *ck_sum) {
  const int k = blockIdx.x;
  const double rho0 = M.rho0[ck_g[k] % M.nmat];
  double s = 0.0;
  for (int32_t p = ck_lo[k] + threadIdx.x; p < ck_hi[k]; p += blockDim.x) s += m[perm[p]] / rho0;
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) ck_sum[k] = red[0];
}

__global__ void k_flaw_vol_groups(const int32_t *__restrict__ g_ck, const double *__restrict__ ck_sum, int64_t G,
                                  FlawMats M, double *lkv, double *invm) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int mt = (int)(g % M.nmat);
  double V = 0.0;
  for (int32_t k = g_ck[g]; k < g_ck[g + 1]; ++k) V += ck_sum[k];
  lkv[g] = log2(M.k[mt] * V);
  invm[g] = M.m[mt] > 0.0 ? 1.0 / M.m[mt] : 0.0;
}

// One batch of Philox blocks per listed group: entry e covers blocks
// b0[e] .. b0[e] + (pre[e+1] - pre[e]) of group grp[e] (four draws each).
struct DrawPlan {
  const int32_t *grp;
  const int64_t *b0;
  const int64_t *pre;  // exclusive prefix of block counts, nplan + 1
  int nplan;
};

__device__ __forceinline__ int plan_entry(const DrawPlan &P, int64_t t) {
  int lo = 0, hi = P.nplan - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.pre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

enum { DRAW_COVER = 0, DRAW_COUNT = 1, DRAW_FILL = 2 };

// MODE cover: first_hit[member] = min j.  count: cnt[id] += 1 for j <= J.
// fill: threshold of draw j <= J into the particle's next slot.
template <int MODE>
__global__ void k_flaw_draws(DrawPlan P, uint64_t seed, const int32_t *__restrict__ goff,
                             const uint32_t *__restrict__ J, const int32_t *__restrict__ perm,
                             const int32_t *__restrict__ id, uint32_t *first_hit, int32_t *cnt,
                             const int32_t *__restrict__ start, float *eps, const double *__restrict__ lkv,
                             const double *__restrict__ invm) {
  const int64_t total = P.pre[P.nplan];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int e = plan_entry(P, t);
    const int g = P.grp[e];
    const uint64_t b = (uint64_t)(P.b0[e] + (t - P.pre[e]));
    const int32_t base = goff[g];
    const uint64_t N = (uint64_t)(goff[g + 1] - base);
    uint64_t w[4] = {b, 0, 0, 0};
    philox4x64(w, seed, (uint64_t)g);
    const uint64_t jlim = MODE == DRAW_COVER ? ~0ULL : (uint64_t)J[g];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const uint64_t j = 4 * b + l + 1;
      if (j > jlim) break;
      const int32_t p = base + (int32_t)__umul64hi(w[l], N);
      if (MODE == DRAW_COVER) {
        atomicMin(&first_hit[p], (uint32_t)j);
      } else {
        const int32_t d = id[perm[p]];
        if (MODE == DRAW_COUNT) {
          atomicAdd(&cnt[d], 1);
        } else {
          const int32_t slot = start[d] + atomicAdd(&cnt[d], 1);
          // (j / (k V))^(1/m) as 2^((log2 j - log2(k V)) / m): within ~1e-15 of
          // the power in FP64, so the float rounds as the power's does except
          // at near-ties
          eps[slot] = (float)exp2(invm[g] * (log2((double)j) - lkv[g]));
        }
      }
    }
  }
}

// per group: members not yet hit, and the largest first hit.  Members of
// a group are consecutive, so the lanes of a warp mostly share it: they
// combine first and one lane per group does the atomics.
__global__ void k_flaw_cover_stats(const unsigned long long *__restrict__ skey, const uint32_t *__restrict__ first_hit,
                                   int32_t nb, int32_t *unc, uint32_t *J) {
  const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = p < nb;
  const int g = valid ? (int)(skey[p] >> kIdBits) : -1;
  const uint32_t f = valid ? first_hit[p] : 0u;
  const unsigned peers = __match_any_sync(0xffffffffu, g);
  const unsigned nun = __reduce_add_sync(peers, (valid && f == kNoHit) ? 1u : 0u);
  const unsigned mx = __reduce_max_sync(peers, (valid && f != kNoHit) ? f : 0u);
  if (valid && (threadIdx.x & 31) == __ffs(peers) - 1) {
    if (nun) atomicAdd(&unc[g], (int32_t)nun);
    if (mx) atomicMax(&J[g], mx);
  }
}

__global__ void k_flaw_offsets(const int32_t *__restrict__ start, int64_t n, int64_t *off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) off[i] = start[i];
}

// thresholds of one particle in ascending order (lists are short: ~ln N)
__global__ void k_flaw_sort(const int32_t *__restrict__ start, int64_t n, float *eps) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const int32_t b = start[d], e = start[d + 1];
  for (int32_t i = b + 1; i < e; ++i) {
    const float v = eps[i];
    int32_t j = i;
    while (j > b && eps[j - 1] > v) {
      eps[j] = eps[j - 1];
      --j;
    }
    eps[j] = v;
  }
}

int draw_blocks(sph_ctx *c) { return c->num_sms * 8; }

}  // namespace

// Host driver; returns SPH_OK or an error status (message in c->err).
sph_status flaws_generate(sph_ctx *c, const sph_state *s, const sph_material *mats, int nmat, const double *wk,
                          const double *wm, uint64_t seed, int64_t *flaw_off, float *flaw_eps, int64_t cap,
                          int64_t *total, cudaStream_t st) {
  const int64_t n = s->n;
  const int ninst = s->ninst > 0 ? s->ninst : 1;
  const int64_t G = (int64_t)ninst * nmat;
  FlawBufs &F = c->fl;
  FlawMats M;
  memset(&M, 0, sizeof(M));
  M.nmat = nmat;
  for (int k = 0; k < nmat; ++k) {
    M.rho0[k] = mats[k].rho0;
    M.k[k] = wk[k];
    M.m[k] = wm[k];
    if (mats[k].damage && wk[k] > 0.0 && wm[k] > 0.0) M.brittle |= 1 << k;
  }
  *total = 0;
  if (n == 0 || M.brittle == 0) {
    if (flaw_off) cudaMemsetAsync(flaw_off, 0, sizeof(int64_t) * (n + 1), st);
    return SPH_OK;
  }
  int gbits = 0;
  while ((int64_t{1} << gbits) <= G) ++gbits;
  Tree &T = c->tree;
  cudaMemsetAsync(F.bad, 0, sizeof(int32_t), st);
  { k_flaw_keys<<<nblk(n, 256), 256, 0, st>>>(s->mat, s->id, n, s->inst_off, ninst, M, T.keys[0], T.vals[0],
                                              F.bad); ++g_launches; }
  sort_pairs(c, n, kIdBits + gbits, st);
  { k_flaw_bounds<<<nblk(n + 1, 256), 256, 0, st>>>(T.skey, n, G, F.goff); ++g_launches; }
  std::vector<int32_t> goff(G + 1);
  int32_t bad = 0;
  cudaMemcpyAsync(goff.data(), F.goff, sizeof(int32_t) * (G + 1), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&bad, F.bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPH_ERR_CUDA;
  if (bad) {
    snprintf(c->err, sizeof(c->err), "sph_flaws: id outside 0..n-1 or material outside 0..nmat-1");
    return SPH_ERR_INVALID;
  }
  // group volumes from chunks of members
  std::vector<int32_t> ck_g, ck_lo, ck_hi, g_ck(G + 1, 0);
  for (int64_t g = 0; g < G; ++g) {
    g_ck[g] = (int32_t)ck_g.size();
    for (int32_t lo = goff[g]; lo < goff[g + 1]; lo += kVolChunk) {
      ck_g.push_back((int32_t)g);
      ck_lo.push_back(lo);
      ck_hi.push_back(std::min(lo + kVolChunk, goff[g + 1]));
    }
  }
  g_ck[G] = (int32_t)ck_g.size();
  const int nck = (int)ck_g.size();
  if (nck > F.cap_chunks) {
    snprintf(c->err, sizeof(c->err), "sph_flaws: too many volume chunks");
    return SPH_ERR_CAPACITY;
  }
  cudaMemcpyAsync(F.ck_g, ck_g.data(), sizeof(int32_t) * nck, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(F.ck_lo, ck_lo.data(), sizeof(int32_t) * nck, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(F.ck_hi, ck_hi.data(), sizeof(int32_t) * nck, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(F.g_ck, g_ck.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, st);
  if (nck > 0)
    { k_flaw_vol_chunks<<<nck, 256, 0, st>>>(F.ck_g, F.ck_lo, F.ck_hi, T.perm, s->m, M, F.ck_sum); ++g_launches; }
  { k_flaw_vol_groups<<<nblk(G, 128), 128, 0, st>>>(F.g_ck, F.ck_sum, G, M, F.kv, F.invm); ++g_launches; }
  const int32_t nb = goff[G];  // brittle particles
  uint32_t *first_hit = reinterpret_cast<uint32_t *>(c->st.gather_i);
  cudaMemsetAsync(first_hit, 0xff, sizeof(uint32_t) * nb, st);
  cudaMemsetAsync(F.J, 0, sizeof(uint32_t) * G, st);

  // coverage rounds: the groups still uncovered, each with a batch of blocks
  std::vector<int64_t> done_blocks(G, 0);
  std::vector<int32_t> unc(G);
  for (int64_t g = 0; g < G; ++g) unc[g] = goff[g + 1] - goff[g];
  std::vector<int32_t> pg;
  std::vector<int64_t> pb0, ppre;
  int rounds = 0;
  for (;;) {
    pg.clear();
    pb0.clear();
    ppre.assign(1, 0);
    for (int64_t g = 0; g < G; ++g) {
      if (unc[g] == 0) continue;
      const double N = goff[g + 1] - goff[g];
      // expected draws to hit the u members still missing: about N (ln u + 0.58); ask for a few more
      const double want = N * (log((double)unc[g]) + 4.0) + 64.0;
      const int64_t blocks = (int64_t)(want / 4.0) + 1;
      if ((done_blocks[g] + blocks) * 4 >= (int64_t)kNoHit) {
        snprintf(c->err, sizeof(c->err), "sph_flaws: a group needs more than 2^32 draws");
        return SPH_ERR_CAPACITY;
      }
      pg.push_back((int32_t)g);
      pb0.push_back(done_blocks[g]);
      ppre.push_back(ppre.back() + blocks);
      done_blocks[g] += blocks;
    }
    if (pg.empty()) break;
    if (++rounds > kMaxRounds) {
      snprintf(c->err, sizeof(c->err), "sph_flaws: coverage did not complete in %d rounds", kMaxRounds);
      return SPH_ERR_TIMEOUT;
    }
    const int np = (int)pg.size();
    if (np > F.cap_plan) {
      snprintf(c->err, sizeof(c->err), "sph_flaws: too many groups");
      return SPH_ERR_CAPACITY;
    }
    cudaMemcpyAsync(F.plan_grp, pg.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(F.plan_b0, pb0.data(), sizeof(int64_t) * np, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(F.plan_pre, ppre.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice, st);
    DrawPlan P{F.plan_grp, F.plan_b0, F.plan_pre, np};
    const int pr = prof_begin(c, st, PH_FLAW_DRAWS);
    { k_flaw_draws<DRAW_COVER><<<draw_blocks(c), 256, 0, st>>>(P, seed, F.goff, nullptr, nullptr, nullptr, first_hit,
                                                               nullptr, nullptr, nullptr, nullptr, nullptr); ++g_launches; }
    cudaMemsetAsync(F.unc, 0, sizeof(int32_t) * G, st);
    { k_flaw_cover_stats<<<nblk(nb, 256), 256, 0, st>>>(T.skey, first_hit, nb, F.unc, F.J); ++g_launches; }
    prof_end(c, st, pr);
    cudaMemcpyAsync(unc.data(), F.unc, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return SPH_ERR_CUDA;
  }
  std::vector<uint32_t> J(G);
  cudaMemcpyAsync(J.data(), F.J, sizeof(uint32_t) * G, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPH_ERR_CUDA;
  int64_t tot = 0;
  for (int64_t g = 0; g < G; ++g) tot += J[g];
  *total = tot;
  if (tot > INT32_MAX) {
    snprintf(c->err, sizeof(c->err), "sph_flaws: more than 2^31 flaws");
    return SPH_ERR_CAPACITY;
  }
  if (!flaw_off) return SPH_OK;

  // draws 1..J of every group
  pg.clear();
  pb0.clear();
  ppre.assign(1, 0);
  for (int64_t g = 0; g < G; ++g) {
    if (J[g] == 0) continue;
    pg.push_back((int32_t)g);
    pb0.push_back(0);
    ppre.push_back(ppre.back() + ((int64_t)J[g] + 3) / 4);
  }
  const int np = (int)pg.size();
  cudaMemcpyAsync(F.plan_grp, pg.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(F.plan_b0, pb0.data(), sizeof(int64_t) * np, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(F.plan_pre, ppre.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice, st);
  DrawPlan P{F.plan_grp, F.plan_b0, F.plan_pre, np};
  int32_t *cnt = T.ncount, *start = T.nstart;
  int pr = prof_begin(c, st, PH_FLAW_DRAWS);
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), st);
  { k_flaw_draws<DRAW_COUNT><<<draw_blocks(c), 256, 0, st>>>(P, seed, F.goff, F.J, T.perm, s->id, nullptr, cnt,
                                                             nullptr, nullptr, nullptr, nullptr); ++g_launches; }
  scan_counts(c, cnt, start, n + 1, st);
  { k_flaw_offsets<<<nblk(n + 1, 256), 256, 0, st>>>(start, n, flaw_off); ++g_launches; }
  prof_end(c, st, pr);
  if (!flaw_eps || tot > cap) {
    // the host vectors above must outlive the copies
    if (cudaStreamSynchronize(st) != cudaSuccess) return SPH_ERR_CUDA;
    if (flaw_eps && tot > cap) {
      snprintf(c->err, sizeof(c->err), "sph_flaws: %lld flaws exceed the capacity %lld", (long long)tot,
               (long long)cap);
      return SPH_ERR_CAPACITY;
    }
    return SPH_OK;
  }
  pr = prof_begin(c, st, PH_FLAW_FILL);
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), st);
  { k_flaw_draws<DRAW_FILL><<<draw_blocks(c), 256, 0, st>>>(P, seed, F.goff, F.J, T.perm, s->id, nullptr, cnt, start,
                                                            flaw_eps, F.kv, F.invm); ++g_launches; }
  { k_flaw_sort<<<nblk(n, 128), 128, 0, st>>>(start, n, flaw_eps); ++g_launches; }
  prof_end(c, st, pr);
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPH_ERR_CUDA;
  return SPH_OK;
}

}  // namespace sph
