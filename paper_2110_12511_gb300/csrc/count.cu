// Per-vertex and per-edge butterfly counting (Sec. 2.1, Alg. 1 "pveBcnt").
//
// Vertex-priority wedge traversal over the labelled adjacency (label 0 =
// highest degree): from every start s, each wedge s-mid-last with
// last < min(s, mid) is expanded once, and wedge_count[last] counts the mids
// shared by s and last.  Then
//   start and last gain C(wc, 2) each,
//   every mid of a wedge to last gains wc - 1,
//   both edges (s, mid) and (mid, last) of such a wedge gain wc - 1.
//
// GPU design (replacing the paper's per-thread n-element wedge_count array):
// starts are bucketed by a bound B_s on their wedges (sum over mids of
// min(d_mid, min(s, mid))), which also bounds the distinct "last" vertices:
//   B_s <= 256            one warp per start, shared-memory hash (<= 512 slots)
//   s < 16384             one block per start, dense shared-memory counters
//   B_s <= 4096           one block per start, shared-memory hash (<= 8192 slots)
//   otherwise             one block per start, dense counters in global memory
// The wedges of a start are walked in flattened order (mids in chunks of the
// group size, an exclusive scan of their valid prefix lengths, then a
// strided walk so consecutive lanes read consecutive neighbour entries).
// Supports and edge counts are accumulated with 64-bit atomics.
#include "internal.cuh"
#include "wedge.cuh"

namespace pbng {
namespace {

constexpr uint32_t WARP_MAXW = 256, WARP_CAP = 512;
constexpr uint32_t DENSE_CAP = 16384;
constexpr uint32_t BHASH_MAXW = 4096, BHASH_CAP = 8192;
constexpr int BT = 512;  // threads of the block-per-start kernels
constexpr int WT = 256;  // threads of the warp-per-start kernel
enum { C_WARP = 0, C_DENSE = 1, C_BHASH = 2, C_GLOBAL = 3, NCLASS = 4 };

struct CArgs {
  const uint32_t *off, *adj, *eid;
  uint32_t n;
  unsigned long long *cnt, *cnt_e;
  const uint8_t *alive, *isU;
  int want_side;
  unsigned long long *ctr;  // [0] wedges, [1] (start, mid) expansions, [2] support updates
  unsigned long long *be_nb, *be_np;  // per start: blooms (lasts with wc >= 2) and their twin pairs
};

__device__ __forceinline__ bool want(const CArgs &A, uint32_t x) {
  return A.want_side < 0 || ((A.isU[x] != 0) == (A.want_side == 0));
}

template <int N>
struct MidBuf {
  uint32_t mid[N];
  uint32_t lo[N];
  uint32_t len[N];
  uint32_t pre[N + 1];  // exclusive prefix of the slices' 32-entry chunk counts
  unsigned long long acc[N];
};

template <class Grp, int N>
__device__ __forceinline__ uint32_t load_mids(const CArgs &A, uint32_t s, uint32_t so, uint32_t sd, uint32_t base,
                                              const Grp &g, MidBuf<N> &mb) {
  int r = g.rank();
  uint32_t mid = 0, lo = 0, len = 0;
  if (base + r < sd) {
    mid = A.adj[so + base + r];
    if (!A.alive || A.alive[mid]) {
      uint32_t b = min(s, mid);
      lo = A.off[mid];
      uint32_t d = A.off[mid + 1] - lo;
      len = lower_bound_u32(A.adj + lo, min(d, b), b);
    }
  }
  mb.mid[r] = mid;
  mb.lo[r] = lo;
  mb.len[r] = len;
  return g.scan(nchunks(len), mb.pre);  // chunks
}

// the wedges of the mids in mb (C chunks, mids [base, base + N) of sd)
template <class Grp, int N, class F>
__device__ __forceinline__ void walk(const CArgs &A, const Grp &g, const MidBuf<N> &mb, uint32_t sd, uint32_t base,
                                     uint32_t C, F &&f) {
  walk_chunks<N>(A.adj, g.rank(), mb.lo, mb.len, mb.pre, (int)min((uint32_t)N, sd - base), C, f);
}

// Table policies --------------------------------------------------------
struct HashPolicy {
  SmemHash h;
  uint32_t cap;
  __device__ void inc(uint32_t k) const { h.inc(k); }
  __device__ uint32_t get(uint32_t k) const { return h.get(k); }
  template <class Grp, int N>
  __device__ uint64_t drain(const CArgs &A, uint32_t, uint32_t, uint32_t, bool sl, const Grp &g, MidBuf<N> &,
                            uint64_t &nat, uint64_t &nb, uint64_t &np) const {
    uint64_t ss = 0;
    for (uint32_t i = g.rank(); i < cap; i += N) {
      uint32_t k = h.key[i];
      if (k != EMPTY_KEY) {
        uint32_t c = h.val[i];
        if (c >= 2) {
          uint64_t bc = choose2(c);
          if (sl) atomicAdd(&A.cnt[k], (unsigned long long)bc), nat++;
          ss += bc;
          nb++;
          np += c;
        }
        h.key[i] = EMPTY_KEY;
        h.val[i] = 0;
      }
    }
    return ss;
  }
};

struct DensePolicy {  // counters for labels [0, s) in shared memory
  uint32_t *c;
  __device__ void inc(uint32_t k) const { atomicAdd(&c[k], 1u); }
  __device__ uint32_t get(uint32_t k) const { return c[k]; }
  template <class Grp, int N>
  __device__ uint64_t drain(const CArgs &A, uint32_t s, uint32_t, uint32_t, bool sl, const Grp &g, MidBuf<N> &,
                            uint64_t &nat, uint64_t &nb, uint64_t &np) const {
    uint64_t ss = 0;
    for (uint32_t i = g.rank(); i < s; i += N) {
      uint32_t x = c[i];
      if (x) {
        if (x >= 2) {
          uint64_t bc = choose2(x);
          if (sl) atomicAdd(&A.cnt[i], (unsigned long long)bc), nat++;
          ss += bc;
          nb++;
          np += x;
        }
        c[i] = 0;
      }
    }
    return ss;
  }
};

struct GlobalPolicy {  // per-block dense counters over all labels in global memory
  uint32_t *c;
  __device__ void inc(uint32_t k) const { atomicAdd(&c[k], 1u); }
  __device__ uint32_t get(uint32_t k) const { return __ldcg(&c[k]); }
  template <class Grp, int N>
  __device__ uint64_t drain(const CArgs &A, uint32_t s, uint32_t so, uint32_t sd, bool sl, const Grp &g,
                            MidBuf<N> &mb, uint64_t &nat, uint64_t &nb, uint64_t &np) const {
    uint64_t ss = 0;
    for (uint32_t base = 0; base < sd; base += N) {
      uint32_t C = load_mids(A, s, so, sd, base, g, mb);
      walk(A, g, mb, sd, base, C, [&](int, uint32_t, uint32_t last) {
        if (A.alive && !A.alive[last]) return;
        uint32_t x = atomicExch(&c[last], 0u);  // first visitor of last takes its count
        if (x >= 2) {
          uint64_t bc = choose2(x);
          if (sl) atomicAdd(&A.cnt[last], (unsigned long long)bc), nat++;
          ss += bc;
          nb++;
          np += x;
        }
      });
      g.sync();
    }
    return ss;
  }
};

template <class Grp, int N, class Tbl>
__device__ void count_start(const CArgs &A, uint32_t s, const Grp &g, MidBuf<N> &mb, const Tbl &tbl) {
  uint32_t so = A.off[s], sd = A.off[s + 1] - so;
  bool sl = want(A, s);
  bool md = A.want_side < 0 || !sl;
  uint64_t wc = 0, nat = 0;
  // pass 1: wedge_count[last]++ for every valid wedge (Alg. 1 l.9-13)
  for (uint32_t base = 0; base < sd; base += N) {
    uint32_t C = load_mids(A, s, so, sd, base, g, mb);
    walk(A, g, mb, sd, base, C, [&](int, uint32_t, uint32_t last) {
      if (A.alive && !A.alive[last]) return;
      tbl.inc(last);
      wc++;
    });
    g.sync();
  }
  // pass 2: mids and edges of wedges whose endpoint pair closes butterflies
  // (Alg. 1 l.18-19 and l.21-23)
  if (md || A.cnt_e) {
    for (uint32_t base = 0; base < sd; base += N) {
      uint32_t C = load_mids(A, s, so, sd, base, g, mb);
      walk(A, g, mb, sd, base, C, [&](int i, uint32_t pos, uint32_t last) {
        if (A.alive && !A.alive[last]) return;
        uint32_t c = tbl.get(last);
        if (c >= 2) {
          atomicAdd(&mb.acc[i], (unsigned long long)(c - 1));
          if (A.cnt_e) atomicAdd(&A.cnt_e[A.eid[pos]], (unsigned long long)(c - 1)), nat++;
        }
      });
      g.sync();
      int r = g.rank();
      unsigned long long x = mb.acc[r];
      if (x && base + r < sd) {
        if (md) atomicAdd(&A.cnt[mb.mid[r]], x), nat++;
        if (A.cnt_e) atomicAdd(&A.cnt_e[A.eid[so + base + r]], x), nat++;
      }
      mb.acc[r] = 0;
      g.sync();
    }
  }
  // pass 3: start and last gain C(wc, 2) (Alg. 1 l.15-17); clears the table
  uint64_t nb = 0, np = 0;
  uint64_t ss = tbl.drain(A, s, so, sd, sl, g, mb, nat, nb, np);
  g.sync();
  uint64_t tot = g.sum64(ss), wt = g.sum64(wc), at = g.sum64(nat);
  if (A.be_nb) {
    uint64_t tb = g.sum64(nb), tp = g.sum64(np);
    if (g.rank() == 0) {
      A.be_nb[s] = tb;
      A.be_np[s] = tp;
    }
  }
  if (g.rank() == 0) {
    if (sl && tot) atomicAdd(&A.cnt[s], (unsigned long long)tot), at++;
    if (A.ctr) {
      if (wt) atomicAdd(&A.ctr[0], (unsigned long long)wt);
      atomicAdd(&A.ctr[1], (unsigned long long)sd);
      if (at) atomicAdd(&A.ctr[2], (unsigned long long)at);
    }
  }
  g.sync();
}

// ---------------------------------------------------------------- kernels
__global__ void k_classify(CArgs A, unsigned long long *lists, unsigned *counts) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t s = gw; s < A.n; s += nw) {
    if (A.alive && !A.alive[s]) continue;
    uint32_t so = A.off[s], sd = A.off[s + 1] - so;
    uint64_t B = 0;
    for (uint32_t k = lane; k < sd; k += 32) {
      uint32_t mid = A.adj[so + k];
      if (A.alive && !A.alive[mid]) continue;
      uint32_t d = A.off[mid + 1] - A.off[mid];
      B += min(d, min((uint32_t)s, mid));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) B += __shfl_xor_sync(0xffffffffu, B, o);
    if (lane == 0 && B >= 2) {
      int c = B <= WARP_MAXW ? C_WARP : (s < DENSE_CAP ? C_DENSE : (B <= BHASH_MAXW ? C_BHASH : C_GLOBAL));
      unsigned p = atomicAdd(&counts[c], 1u);
      lists[(size_t)c * A.n + p] = (unsigned long long)s | ((unsigned long long)min(B, (uint64_t)0xffffffffu) << 32);
    }
  }
}

__global__ void __launch_bounds__(WT) k_count_warp(CArgs A, const unsigned long long *list, const unsigned *count) {
  extern __shared__ __align__(16) uint8_t sm[];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr size_t per = align16(WARP_CAP * 8 + sizeof(MidBuf<32>));
  uint8_t *base = sm + w * per;
  uint32_t *key = (uint32_t *)base, *val = key + WARP_CAP;
  MidBuf<32> &mb = *(MidBuf<32> *)(base + WARP_CAP * 8);
  for (uint32_t i = lane; i < WARP_CAP; i += 32) key[i] = EMPTY_KEY, val[i] = 0;
  mb.acc[lane] = 0;
  __syncwarp();
  WarpGrp g;
  unsigned n = *count;
  for (size_t it = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5; it < n; it += ((size_t)gridDim.x * blockDim.x) >> 5) {
    unsigned long long item = list[it];
    uint32_t s = (uint32_t)item, B = (uint32_t)(item >> 32);
    uint32_t cap = pow2_at_least(max(2u * B, 32u));
    HashPolicy hp{SmemHash{key, val, cap - 1}, cap};
    count_start(A, s, g, mb, hp);
  }
}

template <int KIND>
__global__ void __launch_bounds__(BT) k_count_block(CArgs A, const unsigned long long *list, const unsigned *count,
                                                     uint32_t *gscratch) {
  extern __shared__ __align__(16) uint8_t sm[];
  MidBuf<BT> &mb = *(MidBuf<BT> *)sm;
  constexpr size_t o1 = align16(sizeof(MidBuf<BT>));
  uint32_t *ws = (uint32_t *)(sm + o1);
  unsigned long long *ws64 = (unsigned long long *)(sm + o1 + 128);
  uint8_t *tb = sm + o1 + 256;
  BlockGrp<BT> g{ws, ws64};
  mb.acc[threadIdx.x] = 0;
  if (KIND == C_DENSE) {
    uint32_t *c = (uint32_t *)tb;
    for (uint32_t i = threadIdx.x; i < DENSE_CAP; i += BT) c[i] = 0;
  } else if (KIND == C_BHASH) {
    uint32_t *key = (uint32_t *)tb, *val = key + BHASH_CAP;
    for (uint32_t i = threadIdx.x; i < BHASH_CAP; i += BT) key[i] = EMPTY_KEY, val[i] = 0;
  }
  __syncthreads();
  unsigned n = *count;
  for (size_t it = blockIdx.x; it < n; it += gridDim.x) {
    unsigned long long item = list[it];
    uint32_t s = (uint32_t)item, B = (uint32_t)(item >> 32);
    if (KIND == C_DENSE) {
      DensePolicy p{(uint32_t *)tb};
      count_start(A, s, g, mb, p);
    } else if (KIND == C_BHASH) {
      uint32_t cap = pow2_at_least(max(2u * B, 64u));
      uint32_t *key = (uint32_t *)tb;
      HashPolicy p{SmemHash{key, key + BHASH_CAP, cap - 1}, cap};
      count_start(A, s, g, mb, p);
    } else {
      GlobalPolicy p{gscratch + (size_t)blockIdx.x * A.n};
      count_start(A, s, g, mb, p);
    }
  }
}

size_t block_smem(int kind) {
  size_t s = align16(sizeof(MidBuf<BT>)) + 256;
  if (kind == C_DENSE) s += DENSE_CAP * 4;
  if (kind == C_BHASH) s += BHASH_CAP * 8;
  return s;
}

}  // namespace

void count_butterflies(Arena &a, const Graph &G, const CountOut &o) {
  if (!G.has_labels) fail(PBNG_EINVAL, "internal: labelled adjacency missing");
  if (G.m == 0 || G.n == 0) return;
  CArgs A{};
  A.off = G.lab_off;
  A.adj = G.lab_adj;
  A.eid = G.lab_eid;
  A.n = G.n;
  A.cnt = (unsigned long long *)o.cnt_lab;
  A.cnt_e = (unsigned long long *)o.cnt_e;
  A.alive = o.lab_alive;
  A.isU = o.lab_isU;
  A.want_side = o.want_side;
  A.ctr = (unsigned long long *)o.wedges;
  A.be_nb = (unsigned long long *)o.be_nb;
  A.be_np = (unsigned long long *)o.be_np;
  if (o.cnt_e && !G.lab_eid) fail(PBNG_EINVAL, "internal: edge ids missing for per-edge counts");

  static bool attr = false;
  if (!attr) {
    CK(cudaFuncSetAttribute(k_count_block<C_DENSE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)block_smem(C_DENSE)));
    CK(cudaFuncSetAttribute(k_count_block<C_BHASH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)block_smem(C_BHASH)));
    CK(cudaFuncSetAttribute(k_count_block<C_GLOBAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)block_smem(C_GLOBAL)));
    attr = true;
  }
  unsigned long long *lists = a.alloc<unsigned long long>((size_t)NCLASS * G.n);
  unsigned *counts = a.zeros<unsigned>(NCLASS);
  int sms = num_sms();
  k_classify<<<grid_for((size_t)G.n * 32, 256, 16 * sms), 256, 0, a.st>>>(A, lists, counts);
  CK_LAUNCH();
  unsigned hc[NCLASS];
  CK(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));

  g_prof.begin(PROF_COUNT);
  if (hc[C_WARP]) {
    size_t smem = (WT / 32) * align16(WARP_CAP * 8 + sizeof(MidBuf<32>));
    static bool wa = false;
    if (!wa) {
      CK(cudaFuncSetAttribute(k_count_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      wa = true;
    }
    unsigned grid = grid_for((size_t)hc[C_WARP] * 32, WT, 6 * sms);
    k_count_warp<<<grid, WT, smem, a.st>>>(A, lists + (size_t)C_WARP * G.n, counts + C_WARP);
    CK_LAUNCH();
  }
  if (hc[C_DENSE]) {
    k_count_block<C_DENSE><<<std::min<unsigned>(hc[C_DENSE], 2 * sms), BT, block_smem(C_DENSE), a.st>>>(
        A, lists + (size_t)C_DENSE * G.n, counts + C_DENSE, nullptr);
    CK_LAUNCH();
  }
  if (hc[C_BHASH]) {
    k_count_block<C_BHASH><<<std::min<unsigned>(hc[C_BHASH], 2 * sms), BT, block_smem(C_BHASH), a.st>>>(
        A, lists + (size_t)C_BHASH * G.n, counts + C_BHASH, nullptr);
    CK_LAUNCH();
  }
  if (hc[C_GLOBAL]) {
    unsigned grid = std::min<unsigned>(hc[C_GLOBAL], 2 * sms);
    uint32_t *scr = a.zeros<uint32_t>((size_t)grid * G.n);
    k_count_block<C_GLOBAL><<<grid, BT, block_smem(C_GLOBAL), a.st>>>(A, lists + (size_t)C_GLOBAL * G.n,
                                                                       counts + C_GLOBAL, scr);
    CK_LAUNCH();
    g_prof.end();
    a.free(scr);
  } else {
    g_prof.end();
  }
  a.free(lists);
  a.free(counts);
}

}  // namespace pbng
