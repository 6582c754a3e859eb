// C ABI entry points (include/pbng.h): argument checks, host/device
// marshalling, and the disjoint-union batch.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"

namespace pbng {
extern thread_local char g_detail[512];

namespace {

template <class F>
int guarded(F &&f) {
  g_detail[0] = 0;
  try {
    f();
    return PBNG_OK;
  } catch (Error &e) {
    return e.code;
  } catch (std::bad_alloc &) {
    snprintf(g_detail, sizeof(g_detail), "host allocation failed");
    return PBNG_ENOMEM;
  } catch (...) {
    snprintf(g_detail, sizeof(g_detail), "unexpected internal exception");
    return PBNG_ECUDA;
  }
}

pbng_opts defaults() {
  pbng_opts o;
  pbng_opts_init(&o);
  return o;
}

// host-side checks that need no device
void check_graph(const pbng_bigraph *g) {
  if (!g) fail(PBNG_EINVAL, "null graph");
  if (!g->u_off) fail(PBNG_EINVAL, "null u_off");
  if (g->m && !g->u_adj) fail(PBNG_EINVAL, "null u_adj with m > 0");
  if ((uint64_t)g->nu + g->nv >= (1ull << 31) || g->m >= (1ull << 31))
    fail(PBNG_EINVAL, "graph exceeds the size limits (nu+nv < 2^31, m < 2^31)");
}

// Device view of the caller's graph: copies host arrays when mem == HOST.
pbng_bigraph device_graph(Arena &a, const pbng_bigraph *g, int mem) {
  check_graph(g);
  pbng_bigraph d = *g;
  if (mem == PBNG_MEM_HOST) {
    uint64_t *off = a.alloc<uint64_t>((size_t)g->nu + 1);
    CK(cudaMemcpyAsync(off, g->u_off, ((size_t)g->nu + 1) * 8, cudaMemcpyHostToDevice, a.st));
    uint32_t *adj = a.alloc<uint32_t>(g->m ? g->m : 1);
    if (g->m) CK(cudaMemcpyAsync(adj, g->u_adj, g->m * 4, cudaMemcpyHostToDevice, a.st));
    d.u_off = off;
    d.u_adj = adj;
  }
  return d;
}

struct OutBuf {  // device output buffer, copied back to host memory if needed
  uint64_t *user = nullptr, *dev = nullptr;
  size_t n = 0;
  int mem = 0;
  void init(Arena &a, uint64_t *p, size_t count, int m) {
    user = p;
    n = count;
    mem = m;
    if (!p) return;
    dev = mem == PBNG_MEM_HOST ? a.alloc<uint64_t>(n ? n : 1) : p;
  }
  void finish(Arena &a) {
    if (user && mem == PBNG_MEM_HOST && n) CK(cudaMemcpyAsync(user, dev, n * 8, cudaMemcpyDeviceToHost, a.st));
  }
};

__global__ void k_gather_lab(const unsigned long long *cnt_lab, const uint32_t *g2lab, uint32_t off, uint32_t n,
                             uint64_t *out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = cnt_lab[g2lab[off + i]];
}

TipParams tip_params(uint32_t P, const pbng_opts &o) {
  if (P == 0) fail(PBNG_EINVAL, "P must be >= 1");
  if (o.bounds_mode != PBNG_BOUNDS_ESTIMATOR && o.bounds_mode != PBNG_BOUNDS_EXPLICIT &&
      o.bounds_mode != PBNG_BOUNDS_LEARNED)
    fail(PBNG_EINVAL, "unknown bounds_mode %d", o.bounds_mode);
  if (o.bounds_mode == PBNG_BOUNDS_LEARNED && (!o.mlp_params || !o.mlp_hidden || !o.mlp_out))
    fail(PBNG_EINVAL, "learned bounds need mlp_params, mlp_hidden and mlp_out");
  if (o.bounds_mode == PBNG_BOUNDS_EXPLICIT) {
    if (o.n_bounds && !o.bounds) fail(PBNG_EINVAL, "null bounds with n_bounds > 0");
    for (uint32_t i = 1; i < o.n_bounds; i++)
      if (o.bounds[i] <= o.bounds[i - 1]) fail(PBNG_EBOUNDS, "bounds must be strictly increasing (index %u)", i);
  }
  TipParams p{};
  p.P = P;
  p.bounds_mode = o.bounds_mode;
  p.bounds = o.bounds;
  p.n_bounds = o.bounds_mode == PBNG_BOUNDS_EXPLICIT ? o.n_bounds : 0;
  p.recount = o.recount;
  p.compact = o.compact;
  p.graph_rounds = o.graph_rounds;
  if (o.bucket_shift && (o.bucket_shift < 14 || o.bucket_shift > 30)) fail(PBNG_EINVAL, "bucket_shift must be 0 or 14..30");
  p.bucket_shift = o.bucket_shift;
  {
    uint32_t wm = o.warp_max_w ? o.warp_max_w : 512, gm = o.group_max_w ? o.group_max_w : 2048;
    if (wm > 512 || gm > 2048 || gm < wm) fail(PBNG_EINVAL, "need warp_max_w <= group_max_w, warp_max_w <= 512, group_max_w <= 2048");
    if (o.item_w && o.item_w < 4096) fail(PBNG_EINVAL, "item_w must be 0 or at least 4096");
    p.warp_max_w = wm;
    p.group_max_w = gm;
    p.item_w = o.item_w;
  }
  p.fd_cluster_min = o.fd_cluster_min ? o.fd_cluster_min : 32768u;
  if (o.count_scratch > PBNG_SCRATCH_DENSE32) fail(PBNG_EINVAL, "unknown count_scratch %u", o.count_scratch);
  p.count_scratch = (int)o.count_scratch;
  if (o.learned_vet != o.learned_vet) fail(PBNG_EINVAL, "learned_vet is NaN");
  p.learned_vet = o.learned_vet == 0.0f ? 2.0 : (o.learned_vet < 0.0f ? 0.0 : (double)o.learned_vet);
  p.timeout_ns = o.timeout_ns ? o.timeout_ns : 10000000000ull;
  p.mlp_params = o.mlp_params;
  p.mlp_hidden = o.mlp_hidden;
  p.mlp_out = o.mlp_out;
  p.bounds_used = nullptr;
  return p;
}

// Turn on kernel-span profiling for a call that asked for statistics.
struct ProfScope {
  pbng_stats *st;
  uint64_t l0;
  ProfScope(pbng_stats *s, cudaStream_t stream) : st(s), l0(g_launches) {
    g_prof = Prof();
    g_prof.on = s != nullptr;
    g_prof.st = stream;
  }
  void fill() {
    if (!st) return;
    uint64_t ns[PROF_NGROUPS];
    g_prof.collect(ns);
    st->launches = g_launches - l0;
    st->ns_k_count = ns[PROF_COUNT];
    st->ns_k_peel = ns[PROF_PEEL];
    st->ns_k_fd = ns[PROF_FD];
    st->n_k_count = g_prof.launches[PROF_COUNT];
    st->n_k_peel = g_prof.launches[PROF_PEEL];
    st->n_k_fd = g_prof.launches[PROF_FD];
  }
  ~ProfScope() {
    uint64_t ns[PROF_NGROUPS];
    g_prof.collect(ns);
    g_prof.on = false;
  }
};

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  uint64_t ns() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    return (uint64_t)(ms * 1e6);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

}  // namespace
}  // namespace pbng

using namespace pbng;

extern "C" {

void pbng_opts_init(pbng_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->bounds_mode = PBNG_BOUNDS_ESTIMATOR;
  o->recount = 1;
  o->compact = 1;
  o->mem = PBNG_MEM_DEVICE;
}

const char *pbng_strerror(int s) {
  switch (s) {
    case PBNG_OK: return "ok";
    case PBNG_EINVAL: return "invalid argument";
    case PBNG_ENOMEM: return "out of device memory";
    case PBNG_ECUDA: return "CUDA error";
    case PBNG_ETIMEOUT: return "device wait timed out";
    case PBNG_EOVERFLOW: return "count overflow";
    case PBNG_EBOUNDS: return "bounds not strictly increasing";
    default: return "unknown status";
  }
}

const char *pbng_last_error_detail(void) { return g_detail; }

int pbng_version(void) { return 100; }

int pbng_count(const pbng_bigraph *g, uint64_t *out_u, uint64_t *out_v, uint64_t *out_e, const pbng_opts *opts,
               pbng_stats *stats) {
  pbng_opts o = opts ? *opts : defaults();
  return guarded([&] {
    check_graph(g);
    init_device_pool();
    Arena a((cudaStream_t)o.stream);
    ProfScope ps(stats, a.st);
    Timer tm(a.st);
    pbng_bigraph d = device_graph(a, g, o.mem);
    Graph G;
    build_graph(a, d, true, out_e != nullptr, G);
    OutBuf bu, bv, be;
    bu.init(a, out_u, G.nu, o.mem);
    bv.init(a, out_v, G.nv, o.mem);
    be.init(a, out_e, G.m, o.mem);
    uint64_t *cnt = a.zeros<uint64_t>((size_t)G.n + 1);
    if (be.dev && G.m) CK(cudaMemsetAsync(be.dev, 0, (size_t)G.m * 8, a.st));
    uint64_t *wd = a.zeros<uint64_t>(3);
    if (o.count_scratch > PBNG_SCRATCH_DENSE32) fail(PBNG_EINVAL, "unknown count_scratch %u", o.count_scratch);
    CountOut co;
    co.cnt_lab = cnt;
    co.cnt_e = be.dev;
    co.wedges = wd;
    co.scratch = (int)o.count_scratch;
    count_butterflies(a, G, co);
    if (bu.dev && G.nu)
      k_gather_lab<<<grid_for(G.nu, 256, 16 * num_sms()), 256, 0, a.st>>>((unsigned long long *)cnt, G.g2lab, 0, G.nu, bu.dev);
    if (bv.dev && G.nv)
      k_gather_lab<<<grid_for(G.nv, 256, 16 * num_sms()), 256, 0, a.st>>>((unsigned long long *)cnt, G.g2lab, G.nu, G.nv, bv.dev);
    CK_LAUNCH();
    bu.finish(a);
    bv.finish(a);
    be.finish(a);
    uint64_t w[3];
    CK(cudaMemcpyAsync(w, wd, sizeof(w), cudaMemcpyDeviceToHost, a.st));
    CK(cudaStreamSynchronize(a.st));
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      stats->wedges_count = w[0];
      stats->updates = w[2];
      stats->bytes_count = 4 * w[0] + 12 * w[1] + 16 * w[2];
      stats->wedge_bound = G.wedge_bound;
      stats->ns_total = tm.ns();
      ps.fill();
    }
  });
}

int pbng_tip_decompose(const pbng_bigraph *g, pbng_side side, uint32_t P, uint64_t *out_tip, const pbng_opts *opts,
                       pbng_stats *stats) {
  pbng_opts o = opts ? *opts : defaults();
  return guarded([&] {
    if (side != PBNG_SIDE_U && side != PBNG_SIDE_V) fail(PBNG_EINVAL, "side must be PBNG_SIDE_U or PBNG_SIDE_V");
    if (!out_tip) fail(PBNG_EINVAL, "null out_tip");
    TipParams p = tip_params(P, o);
    check_graph(g);
    init_device_pool();
    Arena a((cudaStream_t)o.stream);
    ProfScope ps(stats, a.st);
    Timer tm(a.st);
    pbng_bigraph d = device_graph(a, g, o.mem);
    Graph G;
    build_graph(a, d, true, false, G);
    OutBuf out;
    out.init(a, out_tip, side == PBNG_SIDE_U ? G.nu : G.nv, o.mem);
    pbng_stats st;
    memset(&st, 0, sizeof(st));
    uint64_t t_setup = 0;
    {
      CK(cudaStreamSynchronize(a.st));
      t_setup = tm.ns();
    }
    std::vector<uint64_t> used;
    p.bounds_used = &used;
    tip_decompose(a, G, side == PBNG_SIDE_U ? 0 : 1, p, out.dev, stats ? &st : nullptr);
    out.finish(a);
    CK(cudaStreamSynchronize(a.st));
    if (o.bounds_out)
      for (size_t i = 0; i < used.size() && i < o.n_bounds_out; i++) o.bounds_out[i] = used[i];
    if (stats) {
      *stats = st;
      stats->ns_setup = t_setup;
      stats->ns_total = tm.ns();
      ps.fill();
    }
  });
}

int pbng_tip_components(const pbng_bigraph *g, pbng_side side, const uint64_t *theta, uint64_t k, uint32_t *out_comp,
                        const pbng_opts *opts, pbng_stats *stats) {
  pbng_opts o = opts ? *opts : defaults();
  return guarded([&] {
    if (side != PBNG_SIDE_U && side != PBNG_SIDE_V) fail(PBNG_EINVAL, "side must be PBNG_SIDE_U or PBNG_SIDE_V");
    check_graph(g);
    uint32_t n = side == PBNG_SIDE_U ? g->nu : g->nv;
    if (n && (!theta || !out_comp)) fail(PBNG_EINVAL, "null theta or out_comp");
    init_device_pool();
    Arena a((cudaStream_t)o.stream);
    Timer tm(a.st);
    pbng_bigraph d = device_graph(a, g, o.mem);
    Graph G;
    build_graph(a, d, false, false, G);
    const uint64_t *th = theta;
    uint32_t *out = out_comp;
    if (o.mem == PBNG_MEM_HOST && n) {
      uint64_t *t = a.alloc<uint64_t>(n);
      CK(cudaMemcpyAsync(t, theta, (size_t)n * 8, cudaMemcpyHostToDevice, a.st));
      th = t;
      out = a.alloc<uint32_t>(n);
    }
    uint64_t wedges = 0, joins = 0;
    tip_components(a, G, side == PBNG_SIDE_U ? 0 : 1, th, k, out, &wedges, &joins);
    if (o.mem == PBNG_MEM_HOST && n) CK(cudaMemcpyAsync(out_comp, out, (size_t)n * 4, cudaMemcpyDeviceToHost, a.st));
    CK(cudaStreamSynchronize(a.st));
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      stats->wedges_fd = wedges;  // wedges of the members' subgraph
      stats->updates = joins;     // pairs found in a common butterfly
      stats->ns_total = tm.ns();
    }
  });
}

int pbng_wing_components(const pbng_bigraph *g, const uint64_t *theta, uint64_t k, uint32_t *out_comp,
                         const pbng_opts *opts, pbng_stats *stats) {
  pbng_opts o = opts ? *opts : defaults();
  return guarded([&] {
    check_graph(g);
    uint64_t m = g->m;
    if (m && (!theta || !out_comp)) fail(PBNG_EINVAL, "null theta or out_comp");
    init_device_pool();
    Arena a((cudaStream_t)o.stream);
    Timer tm(a.st);
    pbng_bigraph d = device_graph(a, g, o.mem);
    Graph G;
    build_graph(a, d, false, false, G);
    const uint64_t *th = theta;
    uint32_t *out = out_comp;
    if (o.mem == PBNG_MEM_HOST && m) {
      uint64_t *t = a.alloc<uint64_t>(m);
      CK(cudaMemcpyAsync(t, theta, (size_t)m * 8, cudaMemcpyHostToDevice, a.st));
      th = t;
      out = a.alloc<uint32_t>(m);
    }
    uint64_t wedges = 0, joins = 0;
    wing_components(a, G, th, k, out, &wedges, &joins);
    if (o.mem == PBNG_MEM_HOST && m) CK(cudaMemcpyAsync(out_comp, out, (size_t)m * 4, cudaMemcpyDeviceToHost, a.st));
    CK(cudaStreamSynchronize(a.st));
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      stats->wedges_fd = wedges;
      stats->updates = joins;
      stats->ns_total = tm.ns();
    }
  });
}

int pbng_wing_decompose(const pbng_bigraph *g, uint32_t P, uint64_t *out_wing, const pbng_opts *opts, pbng_stats *stats) {
  pbng_opts o = opts ? *opts : defaults();
  return guarded([&] {
    if (!out_wing && g && g->m) fail(PBNG_EINVAL, "null out_wing");
    TipParams p = tip_params(P, o);
    check_graph(g);
    init_device_pool();
    Arena a((cudaStream_t)o.stream);
    ProfScope ps(stats, a.st);
    Timer tm(a.st);
    pbng_bigraph d = device_graph(a, g, o.mem);
    Graph G;
    build_graph(a, d, true, true, G);
    OutBuf out;
    out.init(a, out_wing, G.m, o.mem);
    pbng_stats st;
    memset(&st, 0, sizeof(st));
    CK(cudaStreamSynchronize(a.st));
    uint64_t t_setup = tm.ns();
    std::vector<uint64_t> used;
    p.bounds_used = &used;
    wing_decompose(a, G, p, out.dev, stats ? &st : nullptr);
    out.finish(a);
    CK(cudaStreamSynchronize(a.st));
    if (o.bounds_out)
      for (size_t i = 0; i < used.size() && i < o.n_bounds_out; i++) o.bounds_out[i] = used[i];
    if (stats) {
      *stats = st;
      stats->ns_setup = t_setup;
      stats->ns_total = tm.ns();
      ps.fill();
    }
  });
}

int pbng_be_index_sums(const pbng_bigraph *g, uint64_t *out_e, uint64_t *out_total, const pbng_opts *opts,
                       pbng_stats *stats) {
  pbng_opts o = opts ? *opts : defaults();
  return guarded([&] {
    if (!out_total) fail(PBNG_EINVAL, "null out_total");
    if (!out_e && g && g->m) fail(PBNG_EINVAL, "null out_e");
    check_graph(g);
    init_device_pool();
    Arena a((cudaStream_t)o.stream);
    Timer tm(a.st);
    pbng_bigraph d = device_graph(a, g, o.mem);
    Graph G;
    build_graph(a, d, true, true, G);
    OutBuf out;
    out.init(a, out_e, G.m, o.mem);
    pbng_stats st;
    memset(&st, 0, sizeof(st));
    uint64_t total = 0;
    be_index_sums(a, G, out.dev, &total, &st);
    out.finish(a);
    CK(cudaStreamSynchronize(a.st));
    *out_total = total;
    if (stats) {
      *stats = st;
      stats->ns_total = tm.ns();
    }
  });
}

int pbng_propose_bounds(const pbng_bigraph *g, pbng_side side, uint32_t P, uint64_t *out_bounds,
                        const pbng_opts *opts) {
  pbng_opts o = opts ? *opts : defaults();
  return guarded([&] {
    if (side != PBNG_SIDE_U && side != PBNG_SIDE_V) fail(PBNG_EINVAL, "side must be PBNG_SIDE_U or PBNG_SIDE_V");
    if (!out_bounds) fail(PBNG_EINVAL, "null out_bounds");
    TipParams p = tip_params(P, o);
    check_graph(g);
    init_device_pool();
    Arena a((cudaStream_t)o.stream);
    pbng_bigraph d = device_graph(a, g, o.mem);
    Graph G;
    build_graph(a, d, true, false, G);
    std::vector<uint64_t> used;
    p.bounds_used = &used;
    p.coarse_only = true;
    tip_decompose(a, G, side == PBNG_SIDE_U ? 0 : 1, p, nullptr, nullptr);
    CK(cudaStreamSynchronize(a.st));
    // theta(1) = 0, the bounds of the ranges used, then +inf (UINT64_MAX)
    out_bounds[0] = 0;
    for (uint32_t i = 1; i <= P; i++) out_bounds[i] = i - 1 < used.size() ? used[i - 1] : ~0ull;
  });
}

int pbng_bound_features(const pbng_bigraph *g, pbng_side side, float *out, const pbng_opts *opts) {
  pbng_opts o = opts ? *opts : defaults();
  return guarded([&] {
    if (side != PBNG_SIDE_U && side != PBNG_SIDE_V) fail(PBNG_EINVAL, "side must be PBNG_SIDE_U or PBNG_SIDE_V");
    if (!out) fail(PBNG_EINVAL, "null output");
    check_graph(g);
    init_device_pool();
    Arena a((cudaStream_t)o.stream);
    pbng_bigraph d = device_graph(a, g, o.mem);
    Graph G;
    build_graph(a, d, true, false, G);
    uint32_t nx = side == PBNG_SIDE_U ? G.nu : G.nv;
    uint64_t *cnt = a.zeros<uint64_t>((size_t)G.n + 1), *sup = a.alloc<uint64_t>((size_t)nx + 1);
    CountOut co;
    co.cnt_lab = cnt;
    count_butterflies(a, G, co);
    if (nx) {
      k_gather_lab<<<grid_for(nx, 256, 16 * num_sms()), 256, 0, a.st>>>((unsigned long long *)cnt, G.g2lab,
                                                                          side == PBNG_SIDE_U ? 0 : G.nu, nx, sup);
      CK_LAUNCH();
    }
    bound_features(a, sup, side == PBNG_SIDE_U ? G.u_off : G.v_off, nx, out);
    CK(cudaStreamSynchronize(a.st));
  });
}

int pbng_wing_bound_features(const pbng_bigraph *g, float *out, const pbng_opts *opts) {
  pbng_opts o = opts ? *opts : defaults();
  return guarded([&] {
    if (!out) fail(PBNG_EINVAL, "null output");
    check_graph(g);
    init_device_pool();
    Arena a((cudaStream_t)o.stream);
    pbng_bigraph d = device_graph(a, g, o.mem);
    Graph G;
    build_graph(a, d, true, true, G);
    uint64_t *cnt = a.zeros<uint64_t>((size_t)G.n + 1), *cnt_e = a.zeros<uint64_t>((size_t)G.m + 1);
    uint32_t *edeg = a.alloc<uint32_t>((size_t)G.m + 1);
    CountOut co;
    co.cnt_lab = cnt;
    co.cnt_e = cnt_e;
    count_butterflies(a, G, co);
    edge_min_degrees(a, G, edeg);
    bound_features(a, cnt_e, nullptr, G.m, out, edeg);
    CK(cudaStreamSynchronize(a.st));
  });
}

}  // extern "C"

// ------------------------------------------------------------------ batch
namespace pbng {
namespace {
struct BatchDesc {
  const uint64_t *u_off;
  const uint32_t *u_adj;
  uint32_t nu, nv;
  uint32_t m;
  uint32_t u_base, v_base;  // offsets of this graph's vertices in the union
  uint32_t e_base;          // offset of this graph's edges in the union
};

enum { BERR_OFFSETS = 1, BERR_RANGE = 2, BERR_ORDER = 4 };

// One block per graph, one warp per row: each graph's own CSR must be valid
// on its own (u_off[0] = 0, u_off[nu] = m, non-decreasing offsets, ids below
// its own nv, rows strictly increasing).  The union would otherwise shift a
// bad id or offset into a neighbouring graph.  Records the smallest failing
// graph index and the kinds of failure.  Offsets are checked before any
// neighbour id of their row is read.
__global__ void k_batch_validate(const BatchDesc *ds, uint32_t n, unsigned *bad_graph, unsigned *flags) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (uint32_t gi = blockIdx.x; gi < n; gi += gridDim.x) {
    BatchDesc d = ds[gi];
    unsigned bad = 0;
    for (uint32_t u = warp; u <= d.nu; u += nwarps) {
      uint64_t b = d.u_off[u];
      if (u == d.nu) {
        if (b != d.m) bad |= BERR_OFFSETS;
        continue;
      }
      uint64_t e = d.u_off[u + 1];
      if (b > e || e > d.m || (u == 0 && b != 0)) {
        bad |= BERR_OFFSETS;
        continue;
      }
      for (uint64_t i = b + lane; i < e; i += 32) {
        uint32_t x = d.u_adj[i];
        if (x >= d.nv) bad |= BERR_RANGE;
        if (i + 1 < e && d.u_adj[i + 1] <= x) bad |= BERR_ORDER;
      }
    }
    if (bad) {
      atomicMin(bad_graph, gi);
      atomicOr(flags, bad);
    }
  }
}

// one block per graph: union offsets and neighbour ids shifted into place
__global__ void k_union(const BatchDesc *ds, uint32_t n, uint64_t *uoff, uint32_t *uadj) {
  for (uint32_t gi = blockIdx.x; gi < n; gi += gridDim.x) {
    BatchDesc d = ds[gi];
    for (uint32_t u = threadIdx.x; u < d.nu; u += blockDim.x) uoff[d.u_base + u] = d.e_base + d.u_off[u];
    for (uint32_t e = threadIdx.x; e < d.m; e += blockDim.x) uadj[d.e_base + e] = d.v_base + d.u_adj[e];
  }
}

// per-edge numbers of graph gi: its edges are [e_base, e_base + m) of the union's U-CSR order
__global__ void k_scatter_edges(const uint64_t *wing, const BatchDesc *ds, uint32_t n, uint64_t *const *outs) {
  for (uint32_t gi = blockIdx.x; gi < n; gi += gridDim.x) {
    BatchDesc d = ds[gi];
    uint64_t *o = outs[gi];
    for (uint32_t e = threadIdx.x; e < d.m; e += blockDim.x) o[e] = wing[d.e_base + e];
  }
}

__global__ void k_scatter_out(const uint64_t *theta, const BatchDesc *ds, uint32_t n, uint64_t *const *outs, int side) {
  for (uint32_t gi = blockIdx.x; gi < n; gi += gridDim.x) {
    BatchDesc d = ds[gi];
    uint64_t *o = outs[gi];
    uint32_t cnt = side == 0 ? d.nu : d.nv, base = side == 0 ? d.u_base : d.v_base;
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) o[i] = theta[base + i];
  }
}

// The disjoint union of a batch of graphs on the device (shared by both
// batch calls): host checks, copies of host graphs, the per-graph CSR check,
// then the union's U-side CSR (graph i's vertices and edges shifted by the
// sizes of graphs 0..i-1).
struct BatchUnion {
  std::vector<BatchDesc> hd;
  BatchDesc *dd = nullptr;
  pbng_bigraph ug{};
};

void batch_union(Arena &a, const pbng_bigraph *gs, uint32_t n, int mem, BatchUnion &B) {
  B.hd.resize(n);
  uint64_t nu = 0, nv = 0, m = 0;
  for (uint32_t i = 0; i < n; i++) {
    const pbng_bigraph &g = gs[i];
    if (!g.u_off || (g.m && !g.u_adj)) fail(PBNG_EINVAL, "graph %u: null pointer", i);
    if ((uint64_t)g.nu + g.nv >= (1ull << 31) || g.m >= (1ull << 31)) fail(PBNG_EINVAL, "graph %u exceeds the size limits", i);
    B.hd[i].nu = g.nu;
    B.hd[i].nv = g.nv;
    B.hd[i].m = (uint32_t)g.m;
    B.hd[i].u_base = (uint32_t)nu;
    B.hd[i].e_base = (uint32_t)m;
    nu += g.nu;
    m += g.m;
    if (nu >= (1ull << 31) || m >= (1ull << 31)) fail(PBNG_EINVAL, "batch exceeds the size limits");
  }
  for (uint32_t i = 0; i < n; i++) {
    B.hd[i].v_base = (uint32_t)nv;
    nv += gs[i].nv;
  }
  if (nu + nv >= (1ull << 31)) fail(PBNG_EINVAL, "batch exceeds the size limits");
  for (uint32_t i = 0; i < n; i++) {  // inputs on the device (copy host graphs first)
    if (mem == PBNG_MEM_HOST) {
      uint64_t *off = a.alloc<uint64_t>((size_t)gs[i].nu + 1);
      uint32_t *adj = a.alloc<uint32_t>(gs[i].m ? gs[i].m : 1);
      CK(cudaMemcpyAsync(off, gs[i].u_off, ((size_t)gs[i].nu + 1) * 8, cudaMemcpyHostToDevice, a.st));
      if (gs[i].m) CK(cudaMemcpyAsync(adj, gs[i].u_adj, gs[i].m * 4, cudaMemcpyHostToDevice, a.st));
      B.hd[i].u_off = off;
      B.hd[i].u_adj = adj;
    } else {
      B.hd[i].u_off = gs[i].u_off;
      B.hd[i].u_adj = gs[i].u_adj;
    }
  }
  B.dd = a.alloc<BatchDesc>(n);
  CK(cudaMemcpyAsync(B.dd, B.hd.data(), n * sizeof(BatchDesc), cudaMemcpyHostToDevice, a.st));
  unsigned *chk = a.alloc<unsigned>(2);
  const unsigned init[2] = {0xffffffffu, 0u};
  CK(cudaMemcpyAsync(chk, init, sizeof(init), cudaMemcpyHostToDevice, a.st));
  k_batch_validate<<<std::min<uint32_t>(n, 8 * num_sms()), 256, 0, a.st>>>(B.dd, n, chk, chk + 1);
  CK_LAUNCH();
  unsigned hchk[2];
  CK(cudaMemcpyAsync(hchk, chk, sizeof(hchk), cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  if (hchk[0] != 0xffffffffu)
    fail(PBNG_EINVAL, "graph %u: malformed CSR (%s%s%s)", hchk[0], (hchk[1] & BERR_OFFSETS) ? "bad offsets " : "",
         (hchk[1] & BERR_RANGE) ? "neighbour id out of range " : "",
         (hchk[1] & BERR_ORDER) ? "row not strictly increasing" : "");
  uint64_t *uoff = a.alloc<uint64_t>(nu + 1);
  uint32_t *uadj = a.alloc<uint32_t>(m ? m : 1);
  k_union<<<std::min<uint32_t>(n, 8 * num_sms()), 256, 0, a.st>>>(B.dd, n, uoff, uadj);
  CK_LAUNCH();
  CK(cudaMemcpyAsync(uoff + nu, &m, 8, cudaMemcpyHostToDevice, a.st));
  CK(cudaStreamSynchronize(a.st));
  B.ug.nu = (uint32_t)nu;
  B.ug.nv = (uint32_t)nv;
  B.ug.m = m;
  B.ug.u_off = uoff;
  B.ug.u_adj = uadj;
  check_graph(&B.ug);
}

void copy_bounds_out(const pbng_opts &o, const std::vector<uint64_t> &used) {
  if (o.bounds_out)
    for (size_t i = 0; i < used.size() && i < o.n_bounds_out; i++) o.bounds_out[i] = used[i];
}
}  // namespace
}  // namespace pbng

extern "C" int pbng_tip_decompose_batch(const pbng_bigraph *gs, uint32_t n, pbng_side side, uint32_t P,
                                        uint64_t *const *outs, const pbng_opts *opts, pbng_stats *stats) {
  pbng_opts o = opts ? *opts : defaults();
  return guarded([&] {
    if (n == 0) return;
    if (!gs || !outs) fail(PBNG_EINVAL, "null graph or output array");
    if (side != PBNG_SIDE_U && side != PBNG_SIDE_V) fail(PBNG_EINVAL, "side must be PBNG_SIDE_U or PBNG_SIDE_V");
    TipParams p = tip_params(P, o);
    for (uint32_t i = 0; i < n; i++)
      if (!outs[i]) fail(PBNG_EINVAL, "graph %u: null output", i);
    init_device_pool();
    Arena a((cudaStream_t)o.stream);
    ProfScope ps(stats, a.st);
    Timer tm(a.st);
    BatchUnion B;
    batch_union(a, gs, n, o.mem, B);
    Graph G;
    build_graph(a, B.ug, true, false, G);
    CK(cudaStreamSynchronize(a.st));
    uint64_t t_setup = tm.ns();
    uint32_t nx = side == PBNG_SIDE_U ? G.nu : G.nv;
    uint64_t *theta = a.alloc<uint64_t>(nx ? nx : 1);
    pbng_stats st;
    memset(&st, 0, sizeof(st));
    std::vector<uint64_t> used;
    p.bounds_used = &used;
    tip_decompose(a, G, side == PBNG_SIDE_U ? 0 : 1, p, theta, stats ? &st : nullptr);
    // per-graph outputs
    std::vector<uint64_t *> douts(n);
    for (uint32_t i = 0; i < n; i++) {
      if (o.mem == PBNG_MEM_HOST) {
        uint32_t cnt = side == PBNG_SIDE_U ? gs[i].nu : gs[i].nv;
        douts[i] = a.alloc<uint64_t>(cnt ? cnt : 1);
      } else {
        douts[i] = outs[i];
      }
    }
    uint64_t **dptr = a.alloc<uint64_t *>(n);
    CK(cudaMemcpyAsync(dptr, douts.data(), n * sizeof(uint64_t *), cudaMemcpyHostToDevice, a.st));
    k_scatter_out<<<std::min<uint32_t>(n, 8 * num_sms()), 256, 0, a.st>>>(theta, B.dd, n, dptr, side == PBNG_SIDE_U ? 0 : 1);
    CK_LAUNCH();
    if (o.mem == PBNG_MEM_HOST)
      for (uint32_t i = 0; i < n; i++) {
        uint32_t cnt = side == PBNG_SIDE_U ? gs[i].nu : gs[i].nv;
        if (cnt) CK(cudaMemcpyAsync(outs[i], douts[i], (size_t)cnt * 8, cudaMemcpyDeviceToHost, a.st));
      }
    CK(cudaStreamSynchronize(a.st));
    copy_bounds_out(o, used);
    if (stats) {
      *stats = st;
      stats->ns_setup = t_setup;
      stats->ns_total = tm.ns();
      ps.fill();
    }
  });
}

extern "C" int pbng_wing_decompose_batch(const pbng_bigraph *gs, uint32_t n, uint32_t P, uint64_t *const *outs,
                                         const pbng_opts *opts, pbng_stats *stats) {
  pbng_opts o = opts ? *opts : defaults();
  return guarded([&] {
    if (n == 0) return;
    if (!gs || !outs) fail(PBNG_EINVAL, "null graph or output array");
    TipParams p = tip_params(P, o);
    for (uint32_t i = 0; i < n; i++)
      if (gs[i].m && !outs[i]) fail(PBNG_EINVAL, "graph %u: null output", i);
    init_device_pool();
    Arena a((cudaStream_t)o.stream);
    ProfScope ps(stats, a.st);
    Timer tm(a.st);
    BatchUnion B;
    batch_union(a, gs, n, o.mem, B);
    const uint64_t m = B.ug.m;
    Graph G;
    build_graph(a, B.ug, true, true, G);
    CK(cudaStreamSynchronize(a.st));
    uint64_t t_setup = tm.ns();
    uint64_t *wing = a.alloc<uint64_t>(m ? m : 1);
    pbng_stats st;
    memset(&st, 0, sizeof(st));
    std::vector<uint64_t> used;
    p.bounds_used = &used;
    if (m) pbng::wing_decompose(a, G, p, wing, stats ? &st : nullptr);
    std::vector<uint64_t *> douts(n);
    for (uint32_t i = 0; i < n; i++)
      douts[i] = (o.mem == PBNG_MEM_HOST && gs[i].m) ? a.alloc<uint64_t>(gs[i].m) : outs[i];
    uint64_t **dptr = a.alloc<uint64_t *>(n);
    CK(cudaMemcpyAsync(dptr, douts.data(), n * sizeof(uint64_t *), cudaMemcpyHostToDevice, a.st));
    if (m) {
      k_scatter_edges<<<std::min<uint32_t>(n, 8 * num_sms()), 256, 0, a.st>>>(wing, B.dd, n, dptr);
      CK_LAUNCH();
    }
    if (o.mem == PBNG_MEM_HOST)
      for (uint32_t i = 0; i < n; i++)
        if (gs[i].m) CK(cudaMemcpyAsync(outs[i], douts[i], (size_t)gs[i].m * 8, cudaMemcpyDeviceToHost, a.st));
    CK(cudaStreamSynchronize(a.st));
    copy_bounds_out(o, used);
    if (stats) {
      *stats = st;
      stats->ns_setup = t_setup;
      stats->ns_total = tm.ns();
      ps.fill();
    }
  });
}
