// sph_neighbours_static: the partner search of sph_neighbours for callers
// that may not allocate device memory.  The tree, the packed FP32 views and
// the partner columns are carved from one fixed array in the library's own
// device memory instead of from a context; the kernels are the same ones.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "sph_internal.cuh"

using namespace sph;

// The scratch.  Every device that loads this module holds it until the
// process exits.  In host code this name only stands for the symbol: its
// device address comes from cudaGetSymbolAddress (static_scratch_base).
static __device__ __align__(256) unsigned char g_static_scratch[SPH_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_base[kMaxDevices];

// Device address of the scratch on device `dev`, which must be current.
// Looked up on the first call per device and cached.
cudaError_t static_scratch_base(int dev, unsigned char **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_base[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_base[dev] = (unsigned char *)p;
  }
  *out = g_scratch_base[dev];
  return cudaSuccess;
}

// Bump allocation over the scratch, 256-byte aligned.  With base == nullptr
// it only adds up the bytes a layout needs.
struct Carve {
  unsigned char *base;
  int64_t used;
  template <class T>
  T *take(int64_t count) {
    int64_t bytes = ((std::max<int64_t>(count, 1) * (int64_t)sizeof(T) + 255) / 256) * 256;
    T *p = base ? (T *)(base + used) : nullptr;
    used += bytes;
    return p;
  }
};

// Points every buffer the tree build, the partner walk and the CSR export
// use into the scratch, sized for exactly n particles in ninst instances.
void layout(sph_ctx *c, Carve &k, int64_t n, int ninst, int leaf_size, int kmax) {
  const int64_t N = std::max<int64_t>(n, 1);
  c->d_err = k.take<int32_t>(1);
  c->units = k.take<Units>(1);
  Tree &T = c->tree;
  for (int i = 0; i < 2; ++i) {
    T.keys[i] = k.take<unsigned long long>(N);
    T.vals[i] = k.take<int32_t>(N);
  }
  T.hist_cap = (int64_t)256 * ((N + 4095) / 4096 + 1);
  T.hist = k.take<uint32_t>(T.hist_cap);
  T.ncount = k.take<int32_t>(N + 1);
  T.nstart = k.take<int32_t>(N + 1);
  T.cap_nodes = std::max<int64_t>(4096, leaf_size <= 2 ? 4 * N : 2 * N);
  const int64_t cn = T.cap_nodes;
  T.scan_tmp = k.take<int32_t>((std::max(N, cn) + 1) / 4096 + 2);
  T.nnodes = k.take<int32_t>(1);
  T.nleaf = k.take<int32_t>(1);
  T.first = k.take<int32_t>(cn);
  T.end = k.take<int32_t>(cn);
  T.skip = k.take<int32_t>(cn);
  T.parent = k.take<int32_t>(cn);
  T.nchild = k.take<int32_t>(cn);
  T.arrived = k.take<int32_t>(cn);
  T.child = k.take<int32_t>(8 * cn);
  T.nrec = k.take<int4>(cn);
  T.level = k.take<int32_t>(cn);
  T.cell = k.take<unsigned long long>(cn);
  T.mass = k.take<double>(cn);
  T.com = k.take<double>(3 * cn);
  T.bblo = k.take<double>(3 * cn);
  T.bbhi = k.take<double>(3 * cn);
  T.hmax = k.take<double>(cn);
  T.fbox_lo = k.take<float4>(cn);
  T.fbox_hi = k.take<float4>(cn);
  T.fcom_hi = k.take<float4>(cn);
  T.fcom_lo = k.take<float4>(cn);
  T.inst_bb = k.take<unsigned long long>(6 * (int64_t)ninst);
  T.inst_lo = k.take<double>(3 * (int64_t)ninst);
  T.inst_s0 = k.take<double>(ninst);
  T.inst_rs0 = k.take<double>(ninst);
  T.inst_root = k.take<int32_t>(ninst);
  T.gcnt = k.take<int32_t>(cn + 1);
  T.gstart = k.take<int32_t>(cn + 1);
  T.cap_groups = N + ninst + 1;
  T.grp_start = k.take<int32_t>(T.cap_groups);
  T.grp_end = k.take<int32_t>(T.cap_groups);
  T.grp_inst = k.take<int32_t>(T.cap_groups);
  T.ngroups = k.take<int32_t>(1);
  c->pk.px_ = k.take<float4>(N);
  c->pk.pxl_ = k.take<float4>(N);
  c->pk.pv_ = k.take<float4>(N);
  c->pk.pvl_ = k.take<float4>(N);
  c->nb_idx = k.take<int32_t>((int64_t)kmax * N);
  c->nb_cnt = k.take<int32_t>(N);
  c->cap_n = N;
  c->cap_inst = ninst;
  c->kmax = kmax;
}

sph_status report(sph_ctx *c, char *msg, int32_t msg_len, sph_status s, const char *text) {
  snprintf(c->err, sizeof(c->err), "%s", text);
  if (msg && msg_len > 0) snprintf(msg, (size_t)msg_len, "%s", c->err);
  return s;
}

}  // namespace

extern "C" sph_status sph_neighbours_static(const sph_state *s, int32_t leaf_size, int32_t max_depth,
                                            int32_t max_neighbours, int64_t *nb_offset, int32_t *nb_index,
                                            int64_t nb_capacity, char *msg, int32_t msg_len, void *stream) {
  sph_ctx c;
  memset(&c, 0, sizeof(c));
  if (msg && msg_len > 0) msg[0] = 0;
  if (!s) return report(&c, msg, msg_len, SPH_ERR_INVALID, "null state");
  if (s->dim != 2 && s->dim != 3) return report(&c, msg, msg_len, SPH_ERR_INVALID, "dim must be 2 or 3");
  if (s->n < 0 || s->n > ((int64_t)1 << 31) - 64) return report(&c, msg, msg_len, SPH_ERR_INVALID, "bad n");
  const int ninst = s->ninst > 0 ? s->ninst : 1;
  if (ninst > 1 && !s->inst_off)
    return report(&c, msg, msg_len, SPH_ERR_INVALID, "inst_off is required when ninst > 1");
  if (s->n > 0) {
    for (int ax = 0; ax < s->dim; ++ax)
      if (!s->x[ax] || !s->v[ax]) return report(&c, msg, msg_len, SPH_ERR_INVALID, "missing position or velocity");
    if (!s->rho || !s->u || !s->m || !s->h)
      return report(&c, msg, msg_len, SPH_ERR_INVALID, "missing rho, u, m or h");
  }
  if (leaf_size < 1 || leaf_size > kMaxLeaf)
    return report(&c, msg, msg_len, SPH_ERR_INVALID, "leaf_size must be in 1..32");
  // bits of the instance id in a key; 64-bit shifts, so any int32 ninst ends
  // the loop (at most 31 bits)
  int ibits = 0;
  while (((int64_t)1 << ibits) < (int64_t)ninst) ++ibits;
  if (max_depth < 1 || max_depth > 21 || s->dim * max_depth + ibits > 64)
    return report(&c, msg, msg_len, SPH_ERR_INVALID,
                  "max_depth must be in 1..21 with dim * max_depth + log2(ninst) <= 64");
  if (max_neighbours < 1) return report(&c, msg, msg_len, SPH_ERR_INVALID, "max_neighbours must be positive");
  if (!nb_offset || (!nb_index && nb_capacity > 0))
    return report(&c, msg, msg_len, SPH_ERR_INVALID, "null output");

  Carve dry{nullptr, 0};
  layout(&c, dry, s->n, ninst, leaf_size, max_neighbours);
  if (dry.used > (int64_t)SPH_STATIC_SCRATCH_BYTES) {
    char text[256];
    snprintf(text, sizeof(text),
             "n = %lld with max_neighbours = %d needs %lld bytes of scratch; the static scratch holds %lld",
             (long long)s->n, max_neighbours, (long long)dry.used, (long long)SPH_STATIC_SCRATCH_BYTES);
    return report(&c, msg, msg_len, SPH_ERR_CAPACITY, text);
  }

  cudaGetDevice(&c.device);
  if (c.device < 0 || c.device >= kMaxDevices) return report(&c, msg, msg_len, SPH_ERR_INVALID, "device id >= 64");
  unsigned char *base = nullptr;
  cudaError_t e = static_scratch_base(c.device, &base);
  if (e != cudaSuccess) return report(&c, msg, msg_len, SPH_ERR_CUDA, cudaGetErrorString(e));
  Carve carve{base, 0};
  layout(&c, carve, s->n, ninst, leaf_size, max_neighbours);
  c.dim = s->dim;
  c.leaf_default = leaf_size;
  c.vscale = 1.0;
  c.tune.walk_leaf = 64;
  c.tune.walk_blocks_per_sm = 16;
  c.tune.pass_threads = 128;
  cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device);
  if (c.num_sms < 1) c.num_sms = 1;

  cudaStream_t st = (cudaStream_t)stream;
  // the scratch keeps the previous call's contents: clear the error word
  cudaMemsetAsync(c.d_err, 0, sizeof(int32_t), st);
  tree_build(&c, s, leaf_size, max_depth, st);
  find_partners(&c, s, st);
  partners_to_csr(&c, s, nb_offset, nb_index, nb_capacity, st);
  int32_t w = 0;
  cudaMemcpyAsync(&w, c.d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return report(&c, msg, msg_len, SPH_ERR_CUDA, cudaGetErrorString(e));
  if (w & ERR_NONFINITE) return report(&c, msg, msg_len, SPH_ERR_NONFINITE, "non-finite input, or h <= 0 or rho <= 0");
  if (w & ERR_NB_OVERFLOW)
    return report(&c, msg, msg_len, SPH_ERR_CAPACITY, "a particle has more partners than max_neighbours");
  if (w & ERR_NODE_OVERFLOW) return report(&c, msg, msg_len, SPH_ERR_CAPACITY, "octree node capacity exceeded");
  if (w & ERR_CSR_OVERFLOW) return report(&c, msg, msg_len, SPH_ERR_CAPACITY, "partner list longer than nb_capacity");
  if (w & ERR_TIMEOUT) return report(&c, msg, msg_len, SPH_ERR_TIMEOUT, "a bounded device loop hit its iteration limit");
  return SPH_OK;
}
