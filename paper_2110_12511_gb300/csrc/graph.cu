// Graph setup: CSR validation, V-side CSR, degree-priority relabelling and
// the labelled adjacency of Alg. 1 (Sec. 2.1, Alg. 1 lines 2-4): vertices of
// U u V ranked by decreasing degree (ties: U before V, then smaller id), every
// neighbour list sorted by increasing label so that the wedge scan of a
// start vertex can stop at the first neighbour whose label is too large.
#include "internal.cuh"

namespace pbng {
namespace {

enum { ERR_OFFSETS = 1, ERR_RANGE = 2, ERR_ORDER = 4 };

// One warp per row: check offsets, range and strict order; write 32-bit
// offsets, degrees and the owner of each edge.
__global__ void k_validate(const uint64_t *off, const uint32_t *adj, uint32_t nu, uint32_t nv, uint64_t m,
                           uint32_t *off32, uint32_t *eu, unsigned *err) {
  int lane = threadIdx.x & 31;
  size_t w = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t u = w; u <= nu; u += nw) {
    uint64_t b = off[u];
    if (lane == 0) off32[u] = (uint32_t)b;
    if (u == nu) {
      if (lane == 0 && b != m) atomicOr(err, ERR_OFFSETS);
      continue;
    }
    uint64_t e = off[u + 1];
    if (b > e || e > m || (u == 0 && b != 0)) {
      if (lane == 0) atomicOr(err, ERR_OFFSETS);
      continue;
    }
    unsigned bad = 0;
    for (uint64_t i = b + lane; i < e; i += 32) {
      uint32_t x = adj[i];
      if (x >= nv) bad |= ERR_RANGE;
      if (i + 1 < e && adj[i + 1] <= x) bad |= ERR_ORDER;
      eu[i] = (uint32_t)u;
    }
    if (bad) atomicOr(err, bad);
  }
}

__global__ void k_vdeg(const uint32_t *adj, uint32_t m, uint32_t *dv) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
    atomicAdd(&dv[adj[i]], 1u);
}

__global__ void k_iota_keys(const uint32_t *adj, uint32_t m, uint64_t *key, uint32_t *val) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    key[i] = adj[i];
    val[i] = (uint32_t)i;
  }
}

__global__ void k_vcsr_fill(const uint32_t *v_eid, const uint32_t *eu, uint32_t m, uint32_t *v_adj) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
    v_adj[i] = eu[v_eid[i]];
}

// degree of global index x (x < nu: U vertex x; else V vertex x-nu)
__device__ __forceinline__ uint32_t gdeg(const uint32_t *u_off, const uint32_t *v_off, uint32_t nu, uint32_t x) {
  return x < nu ? u_off[x + 1] - u_off[x] : v_off[x - nu + 1] - v_off[x - nu];
}

__global__ void k_deg_keys(const uint32_t *u_off, const uint32_t *v_off, uint32_t nu, uint32_t n, uint32_t maxdeg,
                           uint64_t *key, uint32_t *val) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
    key[x] = maxdeg - gdeg(u_off, v_off, nu, (uint32_t)x);
    val[x] = (uint32_t)x;
  }
}

__global__ void k_label_maps(const uint32_t *lab2g, const uint32_t *u_off, const uint32_t *v_off, uint32_t nu, uint32_t n,
                             uint32_t *g2lab, uint32_t *ldeg) {
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < n; r += (size_t)gridDim.x * blockDim.x) {
    uint32_t x = lab2g[r];
    g2lab[x] = (uint32_t)r;
    ldeg[r] = gdeg(u_off, v_off, nu, x);
  }
}

// directed entries of the labelled adjacency: both orientations of each edge
__global__ void k_lab_entries(const uint32_t *eu, const uint32_t *u_adj, const uint32_t *g2lab, uint32_t nu, uint32_t m,
                              int bn, uint64_t *key, uint32_t *val) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < m; e += (size_t)gridDim.x * blockDim.x) {
    uint64_t a = g2lab[eu[e]], b = g2lab[nu + u_adj[e]];
    key[2 * e] = (a << bn) | b;
    val[2 * e] = (uint32_t)e;
    key[2 * e + 1] = (b << bn) | a;
    val[2 * e + 1] = (uint32_t)e;
  }
}

__global__ void k_lab_split(const uint64_t *key, uint32_t n2, uint64_t mask, uint32_t *lab_adj) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x)
    lab_adj[i] = (uint32_t)(key[i] & mask);
}

__global__ void k_wedge_bound(const uint32_t *eu, const uint32_t *u_adj, const uint32_t *u_off, const uint32_t *v_off,
                              uint32_t m, unsigned long long *out) {
  unsigned long long s = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < m; e += (size_t)gridDim.x * blockDim.x) {
    uint32_t u = eu[e], v = u_adj[e];
    uint32_t du = u_off[u + 1] - u_off[u], dv = v_off[v + 1] - v_off[v];
    s += min(du, dv);
  }
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

__global__ void k_diff(const uint32_t *off, uint32_t n, uint32_t *out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = off[i + 1] - off[i];
}

__global__ void k_side_flags(const uint32_t *lab2g, uint32_t nu, uint32_t n, uint8_t *isU) {
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < n; r += (size_t)gridDim.x * blockDim.x)
    isU[r] = lab2g[r] < nu;
}

}  // namespace

uint8_t *label_sides(Arena &a, const Graph &G) {
  uint8_t *isU = a.alloc<uint8_t>(G.n);
  k_side_flags<<<grid_for(G.n, 256, 8 * num_sms()), 256, 0, a.st>>>(G.lab2g, G.nu, G.n, isU);
  CK_LAUNCH();
  return isU;
}

void build_graph(Arena &a, const pbng_bigraph &g, bool want_labels, bool want_eid, Graph &G) {
  if (!g.u_off || (g.m && !g.u_adj)) fail(PBNG_EINVAL, "null CSR pointer");
  if ((uint64_t)g.nu + g.nv >= (1ull << 31)) fail(PBNG_EINVAL, "nu+nv=%llu exceeds the 2^31 limit", (unsigned long long)g.nu + g.nv);
  if (g.m >= (1ull << 31)) fail(PBNG_EINVAL, "m=%llu exceeds the 2^31 limit", (unsigned long long)g.m);
  G.nu = g.nu;
  G.nv = g.nv;
  G.m = (uint32_t)g.m;
  const int T = 256, cap = 16 * num_sms();
  uint32_t m = G.m;

  // ---- validate and convert the U-side CSR
  G.u_off = a.alloc<uint32_t>((size_t)G.nu + 1);
  G.u_adj = const_cast<uint32_t *>(g.u_adj);  // read-only use
  uint32_t *eu = a.alloc<uint32_t>(m ? m : 1);
  unsigned *err = a.zeros<unsigned>(1);
  k_validate<<<grid_for(((size_t)G.nu + 1) * 32, T, cap), T, 0, a.st>>>(g.u_off, g.u_adj, G.nu, G.nv, g.m, G.u_off, eu, err);
  CK_LAUNCH();
  unsigned e = fetch(a, err);
  if (e & ERR_OFFSETS) fail(PBNG_EINVAL, "CSR offsets are not a valid non-decreasing 0..m sequence");
  if (e & ERR_RANGE) fail(PBNG_EINVAL, "neighbour id out of range [0, nv)");
  if (e & ERR_ORDER) fail(PBNG_EINVAL, "CSR rows must be strictly increasing (sorted, no duplicate edges)");

  // ---- V-side CSR: stable sort of edge ids by v keeps u ascending within rows
  uint32_t *dv = a.zeros<uint32_t>((size_t)G.nv + 1);
  if (m) {
    k_vdeg<<<grid_for(m, T, cap), T, 0, a.st>>>(g.u_adj, m, dv);
    CK_LAUNCH();
  }
  G.v_off = a.alloc<uint32_t>((size_t)G.nv + 1);
  exclusive_scan_u32(a, dv, G.v_off, G.nv);
  G.v_adj = a.alloc<uint32_t>(m ? m : 1);
  G.v_eid = a.alloc<uint32_t>(m ? m : 1);
  if (m) {
    uint64_t *key = a.alloc<uint64_t>(m);
    k_iota_keys<<<grid_for(m, T, cap), T, 0, a.st>>>(g.u_adj, m, key, G.v_eid);
    CK_LAUNCH();
    sort_pairs(a, key, G.v_eid, m, bits_for(G.nv));
    k_vcsr_fill<<<grid_for(m, T, cap), T, 0, a.st>>>(G.v_eid, eu, m, G.v_adj);
    CK_LAUNCH();
    a.free(key);
  }
  a.free(dv);

  // ---- degree bound checks (Sec. 2.1 counts stay below 2^64)
  {
    uint32_t *du = a.alloc<uint32_t>((size_t)G.nu + 1), *dd = a.alloc<uint32_t>((size_t)G.nv + 1);
    auto diff = [&](const uint32_t *off, uint32_t n, uint32_t *out) {
      if (n) {
        k_diff<<<grid_for(n, T, cap), T, 0, a.st>>>(off, n, out);
        CK_LAUNCH();
      }
    };
    diff(G.u_off, G.nu, du);
    diff(G.v_off, G.nv, dd);
    uint32_t mu = G.nu ? reduce_max_u32(a, du, G.nu) : 0, mv = G.nv ? reduce_max_u32(a, dd, G.nv) : 0;
    G.maxdeg = mu > mv ? mu : mv;
    unsigned __int128 bu = (unsigned __int128)mu * (mu > 0 ? mu - 1 : 0) / 2 * (mv > 0 ? mv - 1 : 0);
    unsigned __int128 bv = (unsigned __int128)mv * (mv > 0 ? mv - 1 : 0) / 2 * (mu > 0 ? mu - 1 : 0);
    if ((bu >> 64) || (bv >> 64)) fail(PBNG_EOVERFLOW, "butterfly counts may exceed 2^64 (max degrees %u, %u)", mu, mv);
    a.free(du);
    a.free(dd);
  }
  {
    unsigned long long *wb = a.zeros<unsigned long long>(1);
    if (m) {
      k_wedge_bound<<<grid_for(m, T, cap), T, 0, a.st>>>(eu, g.u_adj, G.u_off, G.v_off, m, wb);
      CK_LAUNCH();
    }
    G.wedge_bound = fetch(a, (const uint64_t *)wb);
  }

  G.n = G.nu + G.nv;
  if (want_labels) {
    uint32_t n = G.n;
    // ---- priority: stable sort of global indices by decreasing degree
    uint64_t *key = a.alloc<uint64_t>(n ? n : 1);
    G.lab2g = a.alloc<uint32_t>(n ? n : 1);
    G.g2lab = a.alloc<uint32_t>(n ? n : 1);
    uint32_t *ldeg = a.alloc<uint32_t>((size_t)n + 1);
    if (n) {
      k_deg_keys<<<grid_for(n, T, cap), T, 0, a.st>>>(G.u_off, G.v_off, G.nu, n, G.maxdeg, key, G.lab2g);
      CK_LAUNCH();
      sort_pairs(a, key, G.lab2g, n, bits_for(G.maxdeg));
      k_label_maps<<<grid_for(n, T, cap), T, 0, a.st>>>(G.lab2g, G.u_off, G.v_off, G.nu, n, G.g2lab, ldeg);
      CK_LAUNCH();
    }
    a.free(key);
    G.lab_off = a.alloc<uint32_t>((size_t)n + 1);
    exclusive_scan_u32(a, ldeg, G.lab_off, n);
    a.free(ldeg);
    // ---- labelled adjacency: (src label, dst label) sorted, value = edge id
    size_t n2 = 2 * (size_t)m;
    G.lab_adj = a.alloc<uint32_t>(n2 ? n2 : 1);
    G.lab_eid = a.alloc<uint32_t>(n2 ? n2 : 1);
    if (m) {
      int bn = bits_for(n);
      uint64_t *k2 = a.alloc<uint64_t>(n2);
      k_lab_entries<<<grid_for(m, T, cap), T, 0, a.st>>>(eu, g.u_adj, G.g2lab, G.nu, m, bn, k2, G.lab_eid);
      CK_LAUNCH();
      sort_pairs(a, k2, G.lab_eid, n2, 2 * bn);
      k_lab_split<<<grid_for(n2, T, cap), T, 0, a.st>>>(k2, (uint32_t)n2, (1ull << bn) - 1, G.lab_adj);
      CK_LAUNCH();
      a.free(k2);
    }
    if (!want_eid) {
      a.free(G.lab_eid);
      G.lab_eid = nullptr;
    }
    G.has_labels = true;
  }
  a.free(eu);
  a.free(err);
}

}  // namespace pbng
