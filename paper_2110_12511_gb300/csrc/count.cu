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
// starts are bucketed by their wedge count B_s (the valid prefix lengths of
// their mids' lists), which also bounds the distinct "last" vertices:
//   B_s <= 256            one warp per start, shared-memory hash (<= 512 slots)
//   s < 16384             one block per start, dense shared-memory counters
//   B_s <= 1024           one 128-thread group per start (four per block,
//                         named barriers), shared-memory hash (<= 2048 slots)
//   B_s <= 4096           one block per start, shared-memory hash (<= 8192 slots)
//   otherwise             one block per start, dense counters over all labels
//                         in global memory (one array per block)
// A caller may ask for dense shared counters instead of the hashes and the
// global arrays (count_scratch): the lasts (labels below s) are then counted
// in chunks of 32768 consecutive labels with 16-bit counters in 64 KB of
// shared memory (16384 labels with 32-bit counters), the mids' slices inside
// a chunk found by binary search in their label-sorted lists.
// The wedges of a start are walked in flattened order (mids in chunks of the
// group size, an exclusive scan of their valid prefix lengths, then a
// strided walk so consecutive lanes read consecutive neighbour entries).
// Supports and edge counts are accumulated with 64-bit atomics.
#include <cstdio>
#include <cstdlib>

#include "internal.cuh"
#include "wedge.cuh"

namespace pbng {
namespace {

constexpr uint32_t WARP_MAXW = 256, WARP_CAP = 512;
constexpr uint32_t DENSE_CAP = 16384;
constexpr uint32_t GRP_MAXW = 1024, GRP_CAP = 2048;
constexpr uint32_t BHASH_MAXW = 4096, BHASH_CAP = 8192;
constexpr uint32_t CH_WORDS = 16384;  // counters of the chunked class (64 KB)
constexpr int BT = 512;  // threads of the block-per-start kernels
constexpr int WT = 256;  // threads of the warp-per-start kernel
constexpr int GT = 128;  // threads of a group (GPB per block)
constexpr int GPB = 4;
enum { C_WARP = 0, C_DENSE = 1, C_GRP = 2, C_BHASH = 3, C_GLOBAL = 4, C_CHUNK = 5, NCLASS = 6 };
const char *const CLASS_NAME[NCLASS] = {"warp", "dense", "group", "hash", "global", "chunk"};

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
  __device__ uint64_t drain(const CArgs &A, uint32_t, uint32_t, uint32_t, bool sl, const Grp &g, MidBuf<N> &, uint32_t,
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
  __device__ uint64_t drain(const CArgs &A, uint32_t s, uint32_t, uint32_t, bool sl, const Grp &g, MidBuf<N> &, uint32_t,
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
  // C1: the chunk count of the slices still in mb when all mids fit one load
  template <class Grp, int N>
  __device__ uint64_t drain(const CArgs &A, uint32_t s, uint32_t so, uint32_t sd, bool sl, const Grp &g,
                            MidBuf<N> &mb, uint32_t C1, uint64_t &nat, uint64_t &nb, uint64_t &np) const {
    uint64_t ss = 0;
    for (uint32_t base = 0; base < sd; base += N) {
      uint32_t C = sd <= (uint32_t)N ? C1 : load_mids(A, s, so, sd, base, g, mb);
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

// end of one start: s gains the sum of C(wc, 2) over its lasts, the
// BE-Index sizes of s, and the counters.  The five sums of the group are
// formed in one round: warp shuffles, then (groups of several warps) shared
// 64-bit atomics into mb.acc[0..4], which is zero between passes and is left
// zero; one barrier.  The caller's last barrier (after the drain) already
// orders the table for the next start.
template <class Grp, int N>
__device__ void count_finish(const CArgs &A, uint32_t s, uint32_t sd, bool sl, uint64_t ss, uint64_t wc, uint64_t nat,
                             uint64_t nb, uint64_t np, const Grp &g, MidBuf<N> &mb) {
  uint64_t v[5] = {ss, wc, nat, nb, np};
#pragma unroll
  for (int k = 0; k < 5; k++)
#pragma unroll
    for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if constexpr (N > 32) {
    if ((g.rank() & 31) == 0)
#pragma unroll
      for (int k = 0; k < 5; k++)
        if (v[k]) atomicAdd(&mb.acc[k], (unsigned long long)v[k]);
    g.sync();
    if (g.rank() == 0)
#pragma unroll
      for (int k = 0; k < 5; k++) {
        v[k] = mb.acc[k];
        mb.acc[k] = 0;
      }
  }
  if (g.rank() == 0) {
    const uint64_t tot = v[0], wt = v[1], tb = v[3], tp = v[4];
    uint64_t at = v[2];
    if (A.be_nb) {
      A.be_nb[s] = tb;
      A.be_np[s] = tp;
    }
    if (sl && tot) atomicAdd(&A.cnt[s], (unsigned long long)tot), at++;
    if (A.ctr) {
      if (wt) atomicAdd(&A.ctr[0], (unsigned long long)wt);
      atomicAdd(&A.ctr[1], (unsigned long long)sd);
      if (at) atomicAdd(&A.ctr[2], (unsigned long long)at);
    }
  }
  if constexpr (N == 32) g.sync();
}

template <class Grp, int N, class Tbl>
__device__ void count_start(const CArgs &A, uint32_t s, const Grp &g, MidBuf<N> &mb, const Tbl &tbl) {
  uint32_t so = A.off[s], sd = A.off[s + 1] - so;
  bool sl = want(A, s);
  bool md = A.want_side < 0 || !sl;
  uint64_t wc = 0, nat = 0;
  // a start whose mids fit one load keeps its slices in mb for passes 2-3
  uint32_t C1 = 0;
  // pass 1: wedge_count[last]++ for every valid wedge (Alg. 1 l.9-13)
  for (uint32_t base = 0; base < sd; base += N) {
    uint32_t C = load_mids(A, s, so, sd, base, g, mb);
    C1 = C;
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
      uint32_t C = sd <= (uint32_t)N ? C1 : load_mids(A, s, so, sd, base, g, mb);
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
  uint64_t ss = tbl.drain(A, s, so, sd, sl, g, mb, C1, nat, nb, np);
  g.sync();
  count_finish(A, s, sd, sl, ss, wc, nat, nb, np, g, mb);
}

// the slices of the mids in [base, base + N) holding lasts with labels in
// [L0, min(L1, s, mid)) (binary searches in the label-sorted lists)
template <class Grp, int N>
__device__ __forceinline__ uint32_t load_mids_range(const CArgs &A, uint32_t s, uint32_t so, uint32_t sd, uint32_t base,
                                                    uint32_t L0, uint32_t L1, const Grp &g, MidBuf<N> &mb) {
  int r = g.rank();
  uint32_t mid = 0, lo = 0, len = 0;
  if (base + r < sd) {
    mid = A.adj[so + base + r];
    if (!A.alive || A.alive[mid]) {
      const uint32_t hi = min(L1, min(s, mid));
      if (hi > L0) {
        const uint32_t o = A.off[mid], d = min(A.off[mid + 1] - o, hi);  // labels below hi sit in the first hi
        const uint32_t a = lower_bound_u32(A.adj + o, d, L0);
        lo = o + a;
        len = lower_bound_u32(A.adj + lo, d - a, hi);
      }
    }
  }
  mb.mid[r] = mid;
  mb.lo[r] = lo;
  mb.len[r] = len;
  return g.scan(nchunks(len), mb.pre);
}

// Alg. 1 for one start whose lasts are counted chunk by chunk of labels:
// the three passes of count_start run on every chunk [L0, L1) that holds
// wedges, with 16-bit counters packed two per word (label offset o counts in
// word o mod CH_WORDS, half o / CH_WORDS) or 32-bit ones.
template <int N>
__device__ void count_start_chunked(const CArgs &A, uint32_t s, const BlockGrp<N> &g, MidBuf<N> &mb, uint32_t *tab,
                                    bool w16) {
  const uint32_t so = A.off[s], sd = A.off[s + 1] - so;
  const bool sl = want(A, s), md = A.want_side < 0 || !sl;
  const uint32_t width = w16 ? 2 * CH_WORDS : CH_WORDS;
  const int r = g.rank();
  uint64_t wc = 0, nat = 0, ss = 0, nb = 0, np = 0;
  for (uint32_t L0 = 0; L0 < s; L0 += width) {
    const uint32_t L1 = min(s, L0 + width);
    uint32_t any = 0;
    // pass 1: wedge_count[last]++ (Alg. 1 l.9-13)
    for (uint32_t base = 0; base < sd; base += N) {
      const uint32_t C = load_mids_range(A, s, so, sd, base, L0, L1, g, mb);
      any |= C;
      walk(A, g, mb, sd, base, C, [&](int, uint32_t, uint32_t last) {
        if (A.alive && !A.alive[last]) return;
        const uint32_t o = last - L0;
        if (w16) atomicAdd(&tab[o & (CH_WORDS - 1)], 1u << ((o / CH_WORDS) * 16));
        else atomicAdd(&tab[o], 1u);
        wc++;
      });
      g.sync();
    }
    if (!any) continue;  // (block-uniform: the scans' totals)
    auto get = [&](uint32_t last) -> uint32_t {
      const uint32_t o = last - L0;
      return w16 ? (tab[o & (CH_WORDS - 1)] >> ((o / CH_WORDS) * 16)) & 0xffffu : tab[o];
    };
    // pass 2: mids and edges of wedges whose endpoint pair closes butterflies
    if (md || A.cnt_e) {
      for (uint32_t base = 0; base < sd; base += N) {
        const uint32_t C = load_mids_range(A, s, so, sd, base, L0, L1, g, mb);
        walk(A, g, mb, sd, base, C, [&](int i, uint32_t pos, uint32_t last) {
          if (A.alive && !A.alive[last]) return;
          const uint32_t c = get(last);
          if (c >= 2) {
            atomicAdd(&mb.acc[i], (unsigned long long)(c - 1));
            if (A.cnt_e) atomicAdd(&A.cnt_e[A.eid[pos]], (unsigned long long)(c - 1)), nat++;
          }
        });
        g.sync();
        unsigned long long x = mb.acc[r];
        if (x && base + r < sd) {
          if (md) atomicAdd(&A.cnt[mb.mid[r]], x), nat++;
          if (A.cnt_e) atomicAdd(&A.cnt_e[A.eid[so + base + r]], x), nat++;
        }
        mb.acc[r] = 0;
        g.sync();
      }
    }
    // pass 3: the chunk's lasts gain C(wc, 2); counters read 16 bytes at a
    // time and zeroed where touched
    const uint32_t words = w16 ? min(L1 - L0, CH_WORDS) : L1 - L0;
    uint4 *v = (uint4 *)tab;
    for (uint32_t i = r; i * 4 < words; i += N) {
      const uint4 q = v[i];
      if ((q.x | q.y | q.z | q.w) == 0u) continue;
      v[i] = make_uint4(0u, 0u, 0u, 0u);
      const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int k = 0; k < 4; k++) {
        if (!wv[k]) continue;
#pragma unroll
        for (int h = 0; h < 2; h++) {
          if (h && !w16) break;
          const uint32_t c = w16 ? (wv[k] >> (16 * h)) & 0xffffu : wv[k];
          if (c < 2) continue;
          const uint32_t last = L0 + i * 4 + k + h * CH_WORDS;
          const uint64_t bc = choose2(c);
          if (sl) atomicAdd(&A.cnt[last], (unsigned long long)bc), nat++;
          ss += bc;
          nb++;
          np += c;
        }
      }
    }
    g.sync();
  }
  count_finish(A, s, sd, sl, ss, wc, nat, nb, np, g, mb);
}

// ---------------------------------------------------------------- kernels
__global__ void k_classify(CArgs A, unsigned long long *lists, unsigned *counts, int mode) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t s = gw; s < A.n; s += nw) {
    if (A.alive && !A.alive[s]) continue;
    uint32_t so = A.off[s], sd = A.off[s + 1] - so;
    uint64_t B = 0;  // the start's wedges exactly: the valid prefix of every mid's list
    for (uint32_t k = lane; k < sd; k += 32) {
      uint32_t mid = A.adj[so + k];
      if (A.alive && !A.alive[mid]) continue;
      const uint32_t b = min((uint32_t)s, mid), lo = A.off[mid], d = A.off[mid + 1] - lo;
      B += lower_bound_u32(A.adj + lo, min(d, b), b);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) B += __shfl_xor_sync(0xffffffffu, B, o);
    if (lane == 0 && B >= 2) {
      const bool dense = mode >= PBNG_SCRATCH_DENSE, hash = mode == PBNG_SCRATCH_HASH;
      int c = B <= WARP_MAXW                ? C_WARP
              : s < DENSE_CAP && !hash      ? C_DENSE
              : B <= GRP_MAXW && !dense     ? C_GRP
              : B <= BHASH_MAXW && !dense   ? C_BHASH
              : dense                       ? C_CHUNK
                                             : C_GLOBAL;
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

__host__ __device__ constexpr size_t group_bytes(uint32_t cap) {
  return align16(cap * 8 + align16(sizeof(MidBuf<GT>)) + (GT / 32) * 8 + (GT / 32 + 2) * 4);
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

// four 128-thread groups per block, each with its own shared hash of CAP
// slots and named barrier, one start per group
template <uint32_t CAP>
__global__ void __launch_bounds__(GPB * GT) k_count_group(CArgs A, const unsigned long long *list, const unsigned *count) {
  extern __shared__ __align__(16) uint8_t sm[];
  const int sub = threadIdx.x / GT;
  uint8_t *base = sm + sub * group_bytes(CAP);
  uint32_t *key = (uint32_t *)base, *val = key + CAP;
  MidBuf<GT> &mb = *(MidBuf<GT> *)(base + CAP * 8);
  unsigned long long *ws64 = (unsigned long long *)(base + CAP * 8 + align16(sizeof(MidBuf<GT>)));
  uint32_t *ws = (uint32_t *)(ws64 + GT / 32);
  SubGrp<GT> g{sub * GT, 1 + sub, ws, ws64};
  for (uint32_t i = g.rank(); i < CAP; i += GT) key[i] = EMPTY_KEY, val[i] = 0;
  mb.acc[g.rank()] = 0;
  g.sync();
  unsigned n = *count;
  for (size_t it = (size_t)blockIdx.x * GPB + sub; it < n; it += (size_t)gridDim.x * GPB) {
    unsigned long long item = list[it];
    uint32_t s = (uint32_t)item, B = (uint32_t)(item >> 32);
    uint32_t cap = pow2_at_least(max(2u * B, 64u));
    HashPolicy hp{SmemHash{key, val, cap - 1}, cap};
    count_start(A, s, g, mb, hp);
  }
}

// one block per start, lasts counted label chunk by label chunk
__global__ void __launch_bounds__(BT) k_count_chunk(CArgs A, const unsigned long long *list, const unsigned *count, int w16) {
  extern __shared__ __align__(16) uint8_t sm[];
  MidBuf<BT> &mb = *(MidBuf<BT> *)sm;
  constexpr size_t o1 = align16(sizeof(MidBuf<BT>));
  uint32_t *ws = (uint32_t *)(sm + o1);
  unsigned long long *ws64 = (unsigned long long *)(sm + o1 + 128);
  uint32_t *tab = (uint32_t *)(sm + o1 + 256);
  BlockGrp<BT> g{ws, ws64};
  mb.acc[threadIdx.x] = 0;
  for (uint32_t i = threadIdx.x; i < CH_WORDS; i += BT) tab[i] = 0;
  __syncthreads();
  unsigned n = *count;
  for (size_t it = blockIdx.x; it < n; it += gridDim.x) count_start_chunked(A, (uint32_t)list[it], g, mb, tab, w16 != 0);
}

size_t block_smem(int kind) {
  size_t s = align16(sizeof(MidBuf<BT>)) + 256;
  if (kind == C_DENSE) s += DENSE_CAP * 4;
  if (kind == C_BHASH) s += BHASH_CAP * 8;
  if (kind == C_CHUNK) s += CH_WORDS * 4;
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
    CK(cudaFuncSetAttribute(k_count_chunk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)block_smem(C_CHUNK)));
    CK(cudaFuncSetAttribute(k_count_block<C_GLOBAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)block_smem(C_GLOBAL)));
    CK(cudaFuncSetAttribute(k_count_group<GRP_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(GPB * group_bytes(GRP_CAP))));
    attr = true;
  }
  unsigned long long *lists = a.alloc<unsigned long long>((size_t)NCLASS * G.n);
  unsigned *counts = a.zeros<unsigned>(NCLASS);
  int sms = num_sms();
  k_classify<<<grid_for((size_t)G.n * 32, 256, 16 * sms), 256, 0, a.st>>>(A, lists, counts, o.scratch);
  CK_LAUNCH();
  unsigned hc[NCLASS];
  CK(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));

  // trace (env PBNG_TRACE=<file>): one line per class: name, starts, ms
  FILE *trace = nullptr;
  cudaEvent_t tev[NCLASS + 1] = {};
  if (const char *tp = getenv("PBNG_TRACE")) {
    trace = fopen(tp, "a");
    if (trace)
      for (auto &e : tev) CK(cudaEventCreate(&e));
  }
  auto mark = [&](int c) {
    if (trace) CK(cudaEventRecord(tev[c], a.st));
  };
  g_prof.begin(PROF_COUNT);
  mark(0);
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
  mark(1);
  if (hc[C_DENSE]) {
    k_count_block<C_DENSE><<<std::min<unsigned>(hc[C_DENSE], 2 * sms), BT, block_smem(C_DENSE), a.st>>>(
        A, lists + (size_t)C_DENSE * G.n, counts + C_DENSE, nullptr);
    CK_LAUNCH();
  }
  mark(2);
  if (hc[C_GRP]) {
    k_count_group<GRP_CAP><<<std::min<unsigned>((hc[C_GRP] + GPB - 1) / GPB, 2 * sms), GPB * GT,
                             GPB * group_bytes(GRP_CAP), a.st>>>(A, lists + (size_t)C_GRP * G.n, counts + C_GRP);
    CK_LAUNCH();
  }
  mark(3);
  if (hc[C_BHASH]) {
    k_count_block<C_BHASH><<<std::min<unsigned>(hc[C_BHASH], 2 * sms), BT, block_smem(C_BHASH), a.st>>>(
        A, lists + (size_t)C_BHASH * G.n, counts + C_BHASH, nullptr);
    CK_LAUNCH();
  }
  mark(4);
  uint32_t *gscr = nullptr;
  if (hc[C_GLOBAL]) {
    unsigned grid = std::min<unsigned>(hc[C_GLOBAL], 2 * sms);
    gscr = a.zeros<uint32_t>((size_t)grid * G.n);
    k_count_block<C_GLOBAL><<<grid, BT, block_smem(C_GLOBAL), a.st>>>(A, lists + (size_t)C_GLOBAL * G.n,
                                                                       counts + C_GLOBAL, gscr);
    CK_LAUNCH();
  }
  mark(5);
  if (hc[C_CHUNK]) {
    // 16-bit counters unless a count (at most the smaller degree) could reach 2^16
    k_count_chunk<<<std::min<unsigned>(hc[C_CHUNK], 3 * sms), BT, block_smem(C_CHUNK), a.st>>>(
        A, lists + (size_t)C_CHUNK * G.n, counts + C_CHUNK,
        (G.maxdeg < 65536 && o.scratch != PBNG_SCRATCH_DENSE32) ? 1 : 0);
    CK_LAUNCH();
  }
  mark(6);
  g_prof.end();
  if (trace) {
    CK(cudaEventSynchronize(tev[NCLASS]));
    for (int c = 0; c < NCLASS; c++) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, tev[c], tev[c + 1]));
      fprintf(trace, "C %s %u %.4f\n", CLASS_NAME[c], hc[c], ms);
    }
    for (auto &e : tev) cudaEventDestroy(e);
    fclose(trace);
  }
  if (gscr) a.free(gscr);
  a.free(lists);
  a.free(counts);
}

}  // namespace pbng
