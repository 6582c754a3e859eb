// k-tip retrieval from tip numbers (Def. 2 and the remark after it: tip
// numbers index every level of the k-tip hierarchy).
//
// For side X and level k, the k-tips are the maximal butterfly-connected sets
// of X_k = {x : theta_x >= k} in the subgraph induced on (X_k, Y).  Two
// vertices of X_k lie in a common butterfly exactly when they share at least
// two neighbours (all of Y is in the subgraph), so the k-tips are the
// connected components of the graph on X_k joining x, x' with c(x, x') >= 2.
//
// GPU: the other side's lists are restricted to X_k (warp per list, stable);
// every member x aggregates c(x, x') over members x' > x - one warp with a
// shared hash when x has few wedges, else one block with dense counters in
// global memory - and joins x and x' in a lock-free union-find whose roots
// are the smallest ids (a root is only ever hooked under a smaller root).
// A component is labelled by its smallest member.
#include "internal.cuh"
#include "wedge.cuh"

namespace pbng {
namespace {

using ull = unsigned long long;
constexpr uint32_t NONE = 0xffffffffu;
constexpr uint32_t HW_MAXW = 256, HW_CAP = 512;  // warp class: wedges, shared hash slots
constexpr int HWT = 256, HBT = 512;
constexpr uint32_t UF_LIMIT = 1u << 22;  // retries of one union before the call reports an error

template <int N>
struct HMid {
  uint32_t lo[N];
  uint32_t len[N];
  uint32_t pre[N + 1];
};

struct HArgs {
  const uint32_t *p_off, *p_adj;  // X -> Y
  const uint32_t *f_off, *f_adj;  // Y -> members of X_k
  uint32_t *par;                  // union-find parents over X
  ull *ctr;                       // [0] wedges, [1] joins
  unsigned *err;                  // set when a union exceeded UF_LIMIT retries
};

__device__ __forceinline__ uint32_t uf_find(uint32_t *par, uint32_t x) {
  volatile uint32_t *vp = par;
  for (;;) {
    uint32_t p = vp[x];
    if (p == x) return x;
    uint32_t gp = vp[p];
    if (gp != p) atomicCAS(&par[x], p, gp);  // path halving
    x = gp;
  }
}

// join the components of a and b: the larger root is hooked under the smaller
__device__ __forceinline__ void uf_unite(const HArgs &A, uint32_t a, uint32_t b) {
  for (uint32_t it = 0; it < UF_LIMIT; it++) {
    a = uf_find(A.par, a);
    b = uf_find(A.par, b);
    if (a == b) return;
    if (a > b) {
      uint32_t t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(&A.par[b], b, a) == b) return;
  }
  atomicExch(A.err, 1u);
}

__global__ void k_members(const ull *theta, uint32_t nx, ull k, uint8_t *mem, uint32_t *par) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < nx; x += (size_t)gridDim.x * blockDim.x) {
    mem[x] = theta[x] >= k;
    par[x] = (uint32_t)x;
  }
}

// warp per Y list: members in it (pass 0) or the members copied in order (pass 1)
__global__ void k_filter(const uint32_t *o_off, const uint32_t *o_adj, uint32_t ny, const uint8_t *mem, uint32_t *cnt,
                         const uint32_t *f_off, uint32_t *f_adj, int fill) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t y = gw; y < ny; y += nw) {
    uint32_t lo = o_off[y], len = o_off[y + 1] - lo, out = fill ? f_off[y] : 0;
    for (uint32_t k = 0; k < len; k += 32) {
      uint32_t x = 0;
      bool keep = false;
      if (k + lane < len) {
        x = o_adj[lo + k + lane];
        keep = mem[x] != 0;
      }
      unsigned b = __ballot_sync(0xffffffffu, keep);
      if (fill && keep) f_adj[out + __popc(b & ((1u << lane) - 1u))] = x;
      out += __popc(b);
    }
    if (!fill && lane == 0) cnt[y] = out;
  }
}

// members by wedge count W = sum of their neighbours' restricted lists
__global__ void k_hclassify(const HArgs A, uint32_t nx, const uint8_t *mem, uint32_t *lists, unsigned *counts) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t x = gw; x < nx; x += nw) {
    if (!mem[x]) continue;
    uint32_t xo = A.p_off[x], xd = A.p_off[x + 1] - xo;
    ull W = 0;
    for (uint32_t k = lane; k < xd; k += 32) {
      uint32_t y = A.p_adj[xo + k];
      W += A.f_off[y + 1] - A.f_off[y];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) W += __shfl_xor_sync(0xffffffffu, W, o);
    if (lane == 0 && W >= 2) {
      int c = W <= HW_MAXW ? 0 : 1;
      lists[(size_t)c * nx + atomicAdd(&counts[c], 1u)] = (uint32_t)x;
    }
  }
}

// restricted lists of N(x)[base, base + N) into mb; returns their chunks
template <class Grp, int N>
__device__ __forceinline__ uint32_t h_load(const HArgs &A, uint32_t xo, uint32_t xd, uint32_t base, const Grp &g,
                                           HMid<N> &mb) {
  int r = g.rank();
  uint32_t lo = 0, len = 0;
  if (base + r < xd) {
    uint32_t y = A.p_adj[xo + base + r];
    lo = A.f_off[y];
    len = A.f_off[y + 1] - lo;
  }
  mb.lo[r] = lo;
  mb.len[r] = len;
  return g.scan(nchunks(len), mb.pre);
}

__global__ void __launch_bounds__(HWT) k_hwarp(HArgs A, const uint32_t *list, const unsigned *count) {
  __shared__ uint32_t keys[HWT / 32][HW_CAP], vals[HWT / 32][HW_CAP];
  __shared__ HMid<32> mids[HWT / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint32_t i = lane; i < HW_CAP; i += 32) keys[w][i] = EMPTY_KEY, vals[w][i] = 0;
  __syncwarp();
  WarpGrp g;
  SmemHash h{keys[w], vals[w], HW_CAP - 1};
  ull wedges = 0, joins = 0;
  const unsigned n = *count;
  for (size_t it = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5; it < n; it += ((size_t)gridDim.x * blockDim.x) >> 5) {
    const uint32_t x = list[it], xo = A.p_off[x], xd = A.p_off[x + 1] - xo;
    for (uint32_t base = 0; base < xd; base += 32) {
      uint32_t C = h_load(A, xo, xd, base, g, mids[w]);
      walk_chunks<32>(A.f_adj, lane, mids[w].lo, mids[w].len, mids[w].pre, (int)min(32u, xd - base), C,
                      [&](int, uint32_t, uint32_t xp) {
                        wedges++;
                        if (xp > x) h.inc(xp);
                      });
      __syncwarp();
    }
    for (uint32_t i = lane; i < HW_CAP; i += 32) {
      uint32_t k = keys[w][i];
      if (k != EMPTY_KEY) {
        if (vals[w][i] >= 2) uf_unite(A, x, k), joins++;
        keys[w][i] = EMPTY_KEY;
        vals[w][i] = 0;
      }
    }
    __syncwarp();
  }
  for (int o = 16; o; o >>= 1) {
    wedges += __shfl_xor_sync(0xffffffffu, wedges, o);
    joins += __shfl_xor_sync(0xffffffffu, joins, o);
  }
  if (lane == 0) {
    if (wedges) atomicAdd(&A.ctr[0], wedges);
    if (joins) atomicAdd(&A.ctr[1], joins);
  }
}

// block per member with many wedges; dense counters over X in global memory
// (one zeroed array per block, cleared again by the second walk)
__global__ void __launch_bounds__(HBT) k_hblock(HArgs A, const uint32_t *list, const unsigned *count, uint32_t *gcnt,
                                                uint32_t nx) {
  __shared__ HMid<HBT> mb;
  __shared__ uint32_t ws[HBT / 32 + 1];
  __shared__ ull ws64[HBT / 32];
  BlockGrp<HBT> g{ws, ws64};
  uint32_t *cnt = gcnt + (size_t)blockIdx.x * nx;
  ull wedges = 0, joins = 0;
  const unsigned n = *count;
  for (size_t it = blockIdx.x; it < n; it += gridDim.x) {
    const uint32_t x = list[it], xo = A.p_off[x], xd = A.p_off[x + 1] - xo;
    for (uint32_t base = 0; base < xd; base += HBT) {
      uint32_t C = h_load(A, xo, xd, base, g, mb);
      walk_chunks<HBT>(A.f_adj, threadIdx.x, mb.lo, mb.len, mb.pre, (int)min((uint32_t)HBT, xd - base), C,
                       [&](int, uint32_t, uint32_t xp) {
                         wedges++;
                         if (xp > x) atomicAdd(&cnt[xp], 1u);
                       });
      __syncthreads();
    }
    for (uint32_t base = 0; base < xd; base += HBT) {
      uint32_t C = h_load(A, xo, xd, base, g, mb);
      walk_chunks<HBT>(A.f_adj, threadIdx.x, mb.lo, mb.len, mb.pre, (int)min((uint32_t)HBT, xd - base), C,
                       [&](int, uint32_t, uint32_t xp) {
                         if (xp <= x) return;
                         uint32_t c = atomicExch(&cnt[xp], 0u);  // the first visitor takes the count
                         if (c >= 2) uf_unite(A, x, xp), joins++;
                       });
      __syncthreads();
    }
  }
  for (int o = 16; o; o >>= 1) {
    wedges += __shfl_xor_sync(0xffffffffu, wedges, o);
    joins += __shfl_xor_sync(0xffffffffu, joins, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (wedges) atomicAdd(&A.ctr[0], wedges);
    if (joins) atomicAdd(&A.ctr[1], joins);
  }
}

__global__ void k_hlabels(uint32_t *par, const uint8_t *mem, uint32_t nx, uint32_t *out) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < nx; x += (size_t)gridDim.x * blockDim.x)
    out[x] = mem[x] ? uf_find(par, (uint32_t)x) : NONE;
}

// ------------------------------------------------------------ k-wings
// E_k = {e : theta_e >= k}.  Two edges of E_k lie in a common butterfly inside
// E_k exactly when both belong to the edge set of one vertex pair (u, u') with
// at least two common neighbours over E_k (for v1 != v2 the butterfly
// (u, u', v1, v2) holds them; for (u, v) and (u', v) any second common v2
// gives one).  So every pair with two or more common neighbours joins all its
// E_k edges: each is united with one representative edge of the pair (the
// smallest id of its (u, v) edges).
struct WArgs {
  const uint32_t *u_off, *u_adj;           // U-side CSR, edge id = position
  const uint32_t *v_off, *v_adj, *v_eid;   // V-side CSR with edge ids
  const uint8_t *emem;                     // edge in E_k
  uint32_t *par;                           // union-find over edges
  ull *ctr;                                // [0] wedges, [1] joins
  unsigned *err;
};

__device__ __forceinline__ void uf_unite_e(const WArgs &W, uint32_t a, uint32_t b) {
  HArgs A;
  A.par = W.par;
  A.err = W.err;
  uf_unite(A, a, b);
}

__global__ void k_wmembers(const ull *theta, uint32_t m, ull k, uint8_t *emem, uint32_t *par) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < m; e += (size_t)gridDim.x * blockDim.x) {
    emem[e] = theta[e] >= k;
    par[e] = (uint32_t)e;
  }
}

// U vertices by wedge bound W = sum over their E_k edges (u, v) of d(v)
__global__ void k_wclassify(const WArgs A, uint32_t nu, uint32_t *lists, unsigned *counts, uint32_t warp_max) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t u = gw; u < nu; u += nw) {
    uint32_t uo = A.u_off[u], ud = A.u_off[u + 1] - uo;
    ull W = 0;
    for (uint32_t k = lane; k < ud; k += 32)
      if (A.emem[uo + k]) {
        uint32_t v = A.u_adj[uo + k];
        W += A.v_off[v + 1] - A.v_off[v];
      }
#pragma unroll
    for (int o = 16; o; o >>= 1) W += __shfl_xor_sync(0xffffffffu, W, o);
    if (lane == 0 && W >= 2) {
      int c = W <= warp_max ? 0 : 1;
      lists[(size_t)c * nu + atomicAdd(&counts[c], 1u)] = (uint32_t)u;
    }
  }
}

// V lists of u's E_k edges [base, base + N) into mb (slice i <-> edge uo + base + i)
template <class Grp, int N>
__device__ __forceinline__ uint32_t w_load(const WArgs &A, uint32_t uo, uint32_t ud, uint32_t base, const Grp &g,
                                           HMid<N> &mb) {
  int r = g.rank();
  uint32_t lo = 0, len = 0;
  if (base + r < ud && A.emem[uo + base + r]) {
    uint32_t v = A.u_adj[uo + base + r];
    lo = A.v_off[v];
    len = A.v_off[v + 1] - lo;
  }
  mb.lo[r] = lo;
  mb.len[r] = len;
  return g.scan(nchunks(len), mb.pre);
}

constexpr int WWT = 128;                           // 4 warps: three 512-slot tables each
constexpr uint32_t WW_MAXW = 256, WW_CAP = 512;

__global__ void __launch_bounds__(WWT) k_wwarp(WArgs A, const uint32_t *list, const unsigned *count) {
  __shared__ uint32_t keys[WWT / 32][WW_CAP], cnts[WWT / 32][WW_CAP], reps[WWT / 32][WW_CAP];
  __shared__ HMid<32> mids[WWT / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t *key = keys[w], *cnt = cnts[w], *rep = reps[w];
  for (uint32_t i = lane; i < WW_CAP; i += 32) key[i] = EMPTY_KEY, cnt[i] = 0, rep[i] = NONE;
  __syncwarp();
  WarpGrp g;
  ull wedges = 0, joins = 0;
  auto slot = [&](uint32_t k, bool insert) -> int {  // linear probing; -1 when absent
    uint32_t h = hash32(k) & (WW_CAP - 1);
    for (uint32_t probe = 0; probe < WW_CAP; probe++) {
      uint32_t cur = ((volatile uint32_t *)key)[h];
      if (cur == k) return (int)h;
      if (cur == EMPTY_KEY) {
        if (!insert) return -1;
        uint32_t prev = atomicCAS(&key[h], EMPTY_KEY, k);
        if (prev == EMPTY_KEY || prev == k) return (int)h;
      }
      h = (h + 1) & (WW_CAP - 1);
    }
    return -1;
  };
  const unsigned n = *count;
  for (size_t it = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5; it < n; it += ((size_t)gridDim.x * blockDim.x) >> 5) {
    const uint32_t u = list[it], uo = A.u_off[u], ud = A.u_off[u + 1] - uo;
    for (int pass = 0; pass < 2; pass++) {
      for (uint32_t base = 0; base < ud; base += 32) {
        uint32_t C = w_load(A, uo, ud, base, g, mids[w]);
        walk_chunks<32>(A.v_adj, lane, mids[w].lo, mids[w].len, mids[w].pre, (int)min(32u, ud - base), C,
                        [&](int i, uint32_t q, uint32_t up) {
                          if (up <= u) return;
                          uint32_t e2 = A.v_eid[q];
                          if (!A.emem[e2]) return;
                          uint32_t e = uo + base + i;
                          if (pass == 0) {
                            wedges++;
                            int h = slot(up, true);  // at most W <= WW_CAP / 2 distinct targets
                            if (h < 0) return;
                            atomicAdd(&cnt[h], 1u);
                            atomicMin(&rep[h], e);
                          } else {
                            int h = slot(up, false);
                            if (h >= 0 && cnt[h] >= 2) {
                              uf_unite_e(A, e, rep[h]);
                              uf_unite_e(A, e2, rep[h]);
                              joins++;
                            }
                          }
                        });
        __syncwarp();
      }
    }
    for (uint32_t i = lane; i < WW_CAP; i += 32) key[i] = EMPTY_KEY, cnt[i] = 0, rep[i] = NONE;
    __syncwarp();
  }
  for (int o = 16; o; o >>= 1) {
    wedges += __shfl_xor_sync(0xffffffffu, wedges, o);
    joins += __shfl_xor_sync(0xffffffffu, joins, o);
  }
  if (lane == 0) {
    if (wedges) atomicAdd(&A.ctr[0], wedges);
    if (joins) atomicAdd(&A.ctr[1], joins);
  }
}

// block per heavy U vertex; per-block dense arrays over U in global memory:
// pair counts and the complement of the representative edge (max of ~e is
// the smallest e; zero = none), cleared by a third walk
__global__ void __launch_bounds__(HBT) k_wblock(WArgs A, const uint32_t *list, const unsigned *count, uint32_t *gcnt,
                                                uint32_t *grep, uint32_t nu) {
  __shared__ HMid<HBT> mb;
  __shared__ uint32_t ws[HBT / 32 + 1];
  __shared__ ull ws64[HBT / 32];
  BlockGrp<HBT> g{ws, ws64};
  uint32_t *cnt = gcnt + (size_t)blockIdx.x * nu, *repc = grep + (size_t)blockIdx.x * nu;
  ull wedges = 0, joins = 0;
  const unsigned n = *count;
  for (size_t it = blockIdx.x; it < n; it += gridDim.x) {
    const uint32_t u = list[it], uo = A.u_off[u], ud = A.u_off[u + 1] - uo;
    for (int pass = 0; pass < 3; pass++) {
      for (uint32_t base = 0; base < ud; base += HBT) {
        uint32_t C = w_load(A, uo, ud, base, g, mb);
        walk_chunks<HBT>(A.v_adj, threadIdx.x, mb.lo, mb.len, mb.pre, (int)min((uint32_t)HBT, ud - base), C,
                         [&](int i, uint32_t q, uint32_t up) {
                           if (up <= u) return;
                           uint32_t e2 = A.v_eid[q];
                           if (!A.emem[e2]) return;
                           uint32_t e = uo + base + i;
                           if (pass == 0) {
                             wedges++;
                             atomicAdd(&cnt[up], 1u);
                             atomicMax(&repc[up], ~e);
                           } else if (pass == 1) {
                             if (__ldcg(&cnt[up]) >= 2) {
                               uint32_t r = ~__ldcg(&repc[up]);
                               uf_unite_e(A, e, r);
                               uf_unite_e(A, e2, r);
                               joins++;
                             }
                           } else {
                             cnt[up] = 0;
                             repc[up] = 0;
                           }
                         });
        __syncthreads();
      }
    }
  }
  for (int o = 16; o; o >>= 1) {
    wedges += __shfl_xor_sync(0xffffffffu, wedges, o);
    joins += __shfl_xor_sync(0xffffffffu, joins, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (wedges) atomicAdd(&A.ctr[0], wedges);
    if (joins) atomicAdd(&A.ctr[1], joins);
  }
}

__global__ void k_wlabels(uint32_t *par, const uint8_t *emem, uint32_t m, uint32_t *out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < m; e += (size_t)gridDim.x * blockDim.x)
    out[e] = emem[e] ? uf_find(par, (uint32_t)e) : NONE;
}

}  // namespace

void wing_components(Arena &a, Graph &G, const uint64_t *theta, uint64_t k, uint32_t *out, uint64_t *wedges,
                     uint64_t *joins) {
  const int T = 256;
  const unsigned sms = num_sms(), cap = 16 * sms;
  const uint32_t m = G.m, nu = G.nu;
  if (m == 0) return;
  WArgs A;
  A.u_off = G.u_off;
  A.u_adj = G.u_adj;
  A.v_off = G.v_off;
  A.v_adj = G.v_adj;
  A.v_eid = G.v_eid;
  uint8_t *emem = a.alloc<uint8_t>(m);
  A.emem = emem;
  A.par = a.alloc<uint32_t>(m);
  A.ctr = a.zeros<ull>(2);
  A.err = a.zeros<unsigned>(1);
  k_wmembers<<<grid_for(m, T, cap), T, 0, a.st>>>((const ull *)theta, m, (ull)k, emem, A.par);
  CK_LAUNCH();
  uint32_t *lists = a.alloc<uint32_t>((size_t)2 * nu);
  unsigned *counts = a.zeros<unsigned>(2);
  k_wclassify<<<grid_for((size_t)nu * 32, T, cap), T, 0, a.st>>>(A, nu, lists, counts, WW_MAXW);
  CK_LAUNCH();
  unsigned hc[2];
  CK(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  if (hc[0]) {
    k_wwarp<<<grid_for((size_t)hc[0] * 32, WWT, 8 * sms), WWT, 0, a.st>>>(A, lists, counts);
    CK_LAUNCH();
  }
  if (hc[1]) {
    unsigned grid = std::min<unsigned>(hc[1], 2 * sms);
    uint32_t *gcnt = a.zeros<uint32_t>((size_t)grid * nu), *grep = a.zeros<uint32_t>((size_t)grid * nu);
    k_wblock<<<grid, HBT, 0, a.st>>>(A, lists + nu, counts + 1, gcnt, grep, nu);
    CK_LAUNCH();
    a.free(grep);
    a.free(gcnt);
  }
  k_wlabels<<<grid_for(m, T, cap), T, 0, a.st>>>(A.par, emem, m, out);
  CK_LAUNCH();
  ull h[2];
  unsigned herr = 0;
  CK(cudaMemcpyAsync(h, A.ctr, sizeof(h), cudaMemcpyDeviceToHost, a.st));
  CK(cudaMemcpyAsync(&herr, A.err, 4, cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  if (herr) fail(PBNG_ETIMEOUT, "union-find retries exceeded their limit");
  if (wedges) *wedges = h[0];
  if (joins) *joins = h[1];
}

void tip_components(Arena &a, Graph &G, int side, const uint64_t *theta, uint64_t k, uint32_t *out, uint64_t *wedges,
                    uint64_t *joins) {
  const int T = 256;
  const unsigned sms = num_sms(), cap = 16 * sms;
  const uint32_t nx = side == 0 ? G.nu : G.nv, ny = side == 0 ? G.nv : G.nu;
  if (nx == 0) return;
  const uint32_t *p_off = side == 0 ? G.u_off : G.v_off, *p_adj = side == 0 ? G.u_adj : G.v_adj;
  const uint32_t *o_off = side == 0 ? G.v_off : G.u_off, *o_adj = side == 0 ? G.v_adj : G.u_adj;
  uint8_t *mem = a.alloc<uint8_t>(nx);
  uint32_t *par = a.alloc<uint32_t>(nx);
  k_members<<<grid_for(nx, T, cap), T, 0, a.st>>>((const ull *)theta, nx, (ull)k, mem, par);
  CK_LAUNCH();
  // lists of the other side restricted to X_k
  uint32_t *fcnt = a.zeros<uint32_t>((size_t)ny + 1), *f_off = a.alloc<uint32_t>((size_t)ny + 1);
  k_filter<<<grid_for((size_t)ny * 32, T, cap), T, 0, a.st>>>(o_off, o_adj, ny, mem, fcnt, nullptr, nullptr, 0);
  CK_LAUNCH();
  exclusive_scan_u32(a, fcnt, f_off, ny);
  uint32_t fm = fetch(a, f_off + ny);
  uint32_t *f_adj = a.alloc<uint32_t>(fm ? fm : 1);
  k_filter<<<grid_for((size_t)ny * 32, T, cap), T, 0, a.st>>>(o_off, o_adj, ny, mem, nullptr, f_off, f_adj, 1);
  CK_LAUNCH();
  HArgs A;
  A.p_off = p_off;
  A.p_adj = p_adj;
  A.f_off = f_off;
  A.f_adj = f_adj;
  A.par = par;
  A.ctr = a.zeros<ull>(2);
  A.err = a.zeros<unsigned>(1);
  uint32_t *lists = a.alloc<uint32_t>((size_t)2 * nx);
  unsigned *counts = a.zeros<unsigned>(2);
  k_hclassify<<<grid_for((size_t)nx * 32, T, cap), T, 0, a.st>>>(A, nx, mem, lists, counts);
  CK_LAUNCH();
  unsigned hc[2];
  CK(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  if (hc[0]) {
    k_hwarp<<<grid_for((size_t)hc[0] * 32, HWT, 4 * sms), HWT, 0, a.st>>>(A, lists, counts);
    CK_LAUNCH();
  }
  if (hc[1]) {
    unsigned grid = std::min<unsigned>(hc[1], 2 * sms);
    uint32_t *gcnt = a.zeros<uint32_t>((size_t)grid * nx);
    k_hblock<<<grid, HBT, 0, a.st>>>(A, lists + nx, counts + 1, gcnt, nx);
    CK_LAUNCH();
    a.free(gcnt);
  }
  k_hlabels<<<grid_for(nx, T, cap), T, 0, a.st>>>(par, mem, nx, out);
  CK_LAUNCH();
  ull h[2];
  unsigned herr = 0;
  CK(cudaMemcpyAsync(h, A.ctr, sizeof(h), cudaMemcpyDeviceToHost, a.st));
  CK(cudaMemcpyAsync(&herr, A.err, 4, cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  if (herr) fail(PBNG_ETIMEOUT, "union-find retries exceeded their limit");
  if (wedges) *wedges = h[0];
  if (joins) *joins = h[1];
}

}  // namespace pbng
