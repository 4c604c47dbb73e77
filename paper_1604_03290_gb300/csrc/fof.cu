// Fragments by friends-of-friends on the device (Sect. 4, fragment analysis
// of the impact experiment).  Particles with dmg >= d_remove are removed;
// two remaining particles of one instance are friends when they would be
// interaction partners with smoothing lengths b h0, so the partner walk of
// the tree (with h' = b h0) lists every friend pair.  Components come from a
// lock-free union-find over those lists: a root is hooked under the smaller
// of two roots by compare-and-swap, so every root is the smallest index of
// its tree and the final partition, with its roots, does not depend on the
// order in which threads ran.  Fragments (components with at least min_size
// particles) are ordered by decreasing count, then smallest member, with the
// radix sort of the tree build.
#include "sph_internal.cuh"

namespace sph {

void sort_pairs(sph_ctx *c, int64_t n, int bits, cudaStream_t st);
void scan_counts(sph_ctx *c, const int32_t *in, int32_t *out, int64_t m, cudaStream_t st);

namespace {

constexpr int kFindLimit = 1 << 24;  // bound on the pointer chases of one find or union

__global__ void k_fof_init(const double *__restrict__ h0, const double *__restrict__ dmg, int64_t n, double b,
                           double d_remove, double *hq, int32_t *parent) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  hq[i] = b * h0[i];
  // removed particles are marked -1 and never join
  parent[i] = (dmg != nullptr && !(dmg[i] < d_remove)) ? -1 : (int32_t)i;
}

// Representative of x, halving the path on the way (every pointer only ever
// moves to an ancestor, and roots are only changed by the hook below).
__device__ __forceinline__ int32_t fof_rep(int32_t *parent, int32_t x, int &steps, int limit) {
  int32_t cur = __ldcg(parent + x);
  if (cur == x) return x;
  int32_t prev = x;
  for (;;) {
    const int32_t next = __ldcg(parent + cur);
    if (next == cur || ++steps > limit) break;
    parent[prev] = next;
    prev = cur;
    cur = next;
  }
  return cur;
}

__global__ void k_fof_union(int32_t *parent, const int32_t *__restrict__ nb_idx, const int32_t *__restrict__ nb_cnt,
                            int64_t ld, int64_t n, int limit, int32_t *err) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n || __ldcg(parent + a) < 0) return;
  const int k = nb_cnt[a];
  int steps = 0;
  // a's representative is kept across its pairs.  It may go stale (hooked
  // by another thread); a hook on it then fails and it is found again, and
  // hooking a root under it is still a union with a's set.
  int32_t ra = fof_rep(parent, (int32_t)a, steps, limit);
  for (int i = 0; i < k; ++i) {
    const int32_t b = nb_idx[(int64_t)i * ld + a];
    if (b <= a || __ldcg(parent + b) < 0) continue;  // each pair once, survivors only
    int32_t rb = fof_rep(parent, b, steps, limit);
    while (ra != rb && steps <= limit) {
      const int32_t hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
      const int32_t old = atomicCAS(parent + hi, hi, lo);
      if (old == hi) {  // hooked: lo now represents both sets
        ra = lo;
        break;
      }
      // hi was hooked elsewhere meanwhile: continue from its new representative
      ++steps;
      if (hi == ra) ra = fof_rep(parent, old, steps, limit);
      else rb = fof_rep(parent, old, steps, limit);
    }
    if (steps > limit) {
      raise_err(err, ERR_TIMEOUT);
      return;
    }
  }
}

// parent[i] <- root, and the component's count and mass (no hooks run now,
// so the reads only ever see ancestors; each thread writes its own entry)
__global__ void k_fof_roots(int32_t *parent, const double *__restrict__ m, int64_t n, int32_t *cnt, double *mass,
                            int limit, int32_t *err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t r = __ldcg(parent + i);
  if (r < 0) return;
  for (int s = 0; s < limit; ++s) {
    const int32_t p = __ldcg(parent + r);
    if (p == r) break;
    r = p;
  }
  if (__ldcg(parent + r) != r) {
    raise_err(err, ERR_TIMEOUT);
    return;
  }
  parent[i] = r;
  atomicAdd(cnt + r, 1);
  atomicAdd(mass + r, m[i]);
}

__device__ __forceinline__ bool is_fragment(const int32_t *parent, const int32_t *cnt, int64_t r, int min_size) {
  return __ldcg(parent + r) == (int32_t)r && cnt[r] >= min_size;
}

__global__ void k_fof_flag(const int32_t *parent, const int32_t *__restrict__ cnt, int64_t n, int min_size,
                           int32_t *flag) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > n) return;
  flag[r] = (r < n && is_fragment(parent, cnt, r, min_size)) ? 1 : 0;
}

// sort key: (2^31 - 1 - count, root): ascending = count descending, then root
__global__ void k_fof_compact(const int32_t *parent, const int32_t *__restrict__ cnt, const int32_t *__restrict__ pos,
                              int64_t n, int min_size, unsigned long long *keys, int32_t *vals) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n || !is_fragment(parent, cnt, r, min_size)) return;
  const int32_t k = pos[r];
  keys[k] = ((unsigned long long)(0x7fffffff - cnt[r]) << 31) | (unsigned long long)r;
  vals[k] = (int32_t)r;
}

__global__ void k_fof_rank(const int32_t *__restrict__ sorted_roots, int64_t nf, const int32_t *__restrict__ cnt,
                           const double *__restrict__ mass, int32_t *rank, int32_t *frag_count, double *frag_mass,
                           int64_t cap) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  const int32_t r = sorted_roots[k];
  rank[r] = (int32_t)k;
  if (k < cap) {
    if (frag_count) frag_count[k] = cnt[r];
    if (frag_mass) frag_mass[k] = mass[r];
  }
}

__global__ void k_fof_label(const int32_t *parent, const int32_t *__restrict__ cnt, const int32_t *__restrict__ rank,
                            int64_t n, int min_size, int32_t *label) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t r = parent[i];
  label[i] = (r >= 0 && cnt[r] >= min_size) ? rank[r] : -1;
}

}  // namespace

void fragments_fof(sph_ctx *c, const sph_state *s, const double *h0, double b, double d_remove, int min_size,
                   int leaf_size, int max_depth, int32_t *label, int32_t *frag_count, double *frag_mass, int64_t cap,
                   int64_t *nfrag, cudaStream_t st) {
  const int64_t n = s->n;
  *nfrag = 0;
  if (n == 0) return;
  double *hq = c->st.gather;
  int32_t *parent = c->st.gather_i;
  int32_t *cnt = c->tree.ncount, *pos = c->tree.nstart;
  double *mass = c->cs;
  { k_fof_init<<<nblk(n, 256), 256, 0, st>>>(h0 ? h0 : s->h, s->dmg, n, b, d_remove, hq, parent); ++g_launches; }
  sph_state q = *s;
  q.h = hq;
  const int limit = c->tune.iter_cap > 0 ? c->tune.iter_cap : kFindLimit;
  int pr = prof_begin(c, st, PH_TREE);
  tree_build(c, &q, leaf_size, max_depth, st);
  prof_end(c, st, pr);
  pr = prof_begin(c, st, PH_PARTNERS);
  find_partners(c, &q, st);
  prof_end(c, st, pr);
  pr = prof_begin(c, st, PH_FOF_LINKS);
  { k_fof_union<<<nblk(n, 128), 128, 0, st>>>(parent, c->nb_idx, c->nb_cnt, c->cap_n, n, limit, c->d_err); ++g_launches; }
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), st);
  cudaMemsetAsync(mass, 0, sizeof(double) * n, st);
  { k_fof_roots<<<nblk(n, 256), 256, 0, st>>>(parent, s->m, n, cnt, mass, limit, c->d_err); ++g_launches; }
  { k_fof_flag<<<nblk(n + 1, 256), 256, 0, st>>>(parent, cnt, n, min_size, pos); ++g_launches; }
  scan_counts(c, pos, pos, n + 1, st);
  int32_t nf = 0;
  cudaMemcpyAsync(&nf, pos + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  prof_end(c, st, pr);
  { k_fof_compact<<<nblk(n, 256), 256, 0, st>>>(parent, cnt, pos, n, min_size, c->tree.keys[0], c->tree.vals[0]); ++g_launches; }
  cudaStreamSynchronize(st);
  *nfrag = nf;
  int32_t *rank = pos;  // positions are no longer needed
  if (nf > 0) {
    sort_pairs(c, nf, 62, st);
    { k_fof_rank<<<nblk(nf, 256), 256, 0, st>>>(c->tree.perm, nf, cnt, mass, rank, frag_count, frag_mass, cap); ++g_launches; }
  }
  { k_fof_label<<<nblk(n, 256), 256, 0, st>>>(parent, cnt, rank, n, min_size, label); ++g_launches; }
}

}  // namespace sph
