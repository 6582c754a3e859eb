// Tip decomposition with two-phase peeling (Sec. 3.1, adapted to tips in
// Sec. 3.2).  X = the peeled vertex side, Y = the other side (never peeled).
//
// Coarse phase (Sec. 3.1.1, Alg. 4 with the tip adaptation of Sec. 3.2):
//  for each range i: theta(i+1) from find_range (Sec. 3.1.3) or an explicit
//  bound; snapshot supports into init (the support initialisation vector);
//  then peel rounds: the active set is every unpeeled vertex with support
//  below theta(i+1).  A round either
//   - peels the active set: every wedge x -> y -> x' from an active x to an
//     unpeeled x' is counted per pair, and support(x') -= C(c(x,x'), 2)
//     (updates from different active vertices are disjoint butterflies and
//     are summed atomically, Sec. 3.2), or
//   - re-counts the butterflies of all remaining vertices when the active
//     set's wedges exceed the counting bound (batch processing, Sec. 5.1).
//  Edges to peeled vertices are removed from the Y-side lists after each
//  round (dynamic graph updates, Sec. 5.2).  Supports are kept exact
//  (unclamped); the clamp of Alg. 2 only matters when a number is recorded.
// Fine phase (Sec. 3.1.2, 3.1.4, 3.2): partition i is peeled bottom-up from
//  init on the subgraph induced on (X_i, Y): one thread block per partition,
//  partitions handed out heaviest first (LPT) from a device queue; each step
//  peels every vertex whose support equals the running minimum (ties receive
//  the same number, exactly as one-at-a-time peeling with the clamp).
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "fdwin.cuh"
#include "internal.cuh"
#include "wedge.cuh"

namespace pbng {
namespace {

enum : uint8_t { ST_ALIVE = 0, ST_ACTIVE = 1, ST_PEELED = 2 };

constexpr uint32_t PW_MAXW = 256, PW_CAP = 512;  // fine phase: warp-per-vertex shared hash
constexpr uint32_t FEW_VERTICES = 8, WARP_FEW_W = 192;  // fine phase: few peeled vertices -> team-wide above this
constexpr uint32_t HW_KEEP = 4;
constexpr int FGT = 128;                           // fine phase: threads of a group (four per block)
constexpr uint32_t FG_CAP = 2048, FG_MAXW = 1024;  // group hash slots (in the dense counters' memory), most wedges
constexpr uint32_t FG_MIN_BIG = 8;                 // heavy vertices of a step from which groups take them
constexpr uint32_t FB_MAXW = 4096;                 // cluster teams: most wedges of a vertex one block takes  // fine phase, team path: wedges a thread keeps between its two passes
constexpr uint32_t QW_MAXW = 512, QW_CAP = 1024;  // coarse peel: warp-per-vertex shared hash
constexpr uint32_t QG_MAXW = 2048, QG_CAP = 4096; // coarse peel: 256-thread group per vertex
constexpr int QGT = 256;                          // threads of a group
constexpr uint32_t PB_CAP = 8192;                // block-class shared hash slots (64 KB)
constexpr uint32_t P_CHUNK = 2 * PB_CAP;         // block-class dense counters (same 64 KB)
constexpr uint32_t BK_SHIFT_MIN = 14;            // target buckets are at least P_CHUNK ids wide
constexpr uint64_t BOFF_BUDGET = 2ull << 30;     // most bytes of bucket offsets
constexpr uint64_t ITEM_W = 32768;               // wedges per block-class work item (at least)
constexpr int PB_PER_SM = 3;                     // resident blocks per SM (shared memory bound)
constexpr uint32_t P_DENSE = 16384;              // fine phase: dense shared counters when |X_p| <= this
constexpr int PBT = 512, PWT = 256;
enum { PC_WARP = 0, PC_GROUP = 1, PC_BLOCK = 2, PNCLASS = 3 };
static_assert(P_CHUNK <= 2 * PB_CAP, "dense counters share the hash table memory");
static_assert(P_CHUNK == 1u << BK_SHIFT_MIN, "a narrow bucket fits the dense counters");

using ull = unsigned long long;

// ------------------------------------------------------------ peel kernels
// Target buckets: the X ids are cut into NB buckets of 2^bshift ids, and for
// every Y vertex boff[y][b] is the position in its current (sorted) list of
// the first entry in bucket b, so that the slice of a list holding the
// targets of buckets [bs, be) is two loads away.  Lists shrink by stable
// compaction, which rewrites the offsets of the lists it touches.
struct PeelArgs {
  const uint32_t *p_off, *p_adj;  // X -> Y
  const uint32_t *o_off, *o_adj, *o_len;  // Y -> X (current)
  const uint32_t *boff;  // ny x (nb + 1) bucket offsets, null when nb == 1
  uint32_t nb, bshift;
  ull *sup;
  ull *updates;
  uint32_t nx;
  ull *bstat;  // block-class statistics (BS_*), null unless tracing
};

// block-class statistics of a round, gathered when tracing in a build with
// PBNG_PEEL_STATS=1 (off by default: the counters cost registers): items, SM
// cycles of the phases, passes, wedges, walked lanes, drains
#ifndef PBNG_PEEL_STATS
#define PBNG_PEEL_STATS 0
#endif
enum {
  BS_ITEMS = 0, BS_CYC_PLAN, BS_CYC_WALK, BS_CYC_DRAIN, BS_CYC_REWALK, BS_PASS_HASH, BS_PASS_DENSE, BS_WEDGES,
  BS_LANES, BS_DRAIN_DENSE, BS_DRAIN_SPARSE, BS_CYC_ITEM, BSTAT
};

// slices of the current lists being walked: start, length, and the
// exclusive prefix of their 32-wedge chunk counts
template <int N>
struct PMid {
  uint32_t lo[N];
  uint32_t len[N];
  uint32_t pre[N + 1];
};

// support(x') -= dec.  No return value is needed (the next active set is
// found by a scan), so this is a fire-and-forget reduction.  Targets that are
// active or peeled may receive it too: their supports are never read again.
__device__ __forceinline__ void sub_support(const PeelArgs &A, uint32_t xp, uint64_t dec) {
  atomicAdd(&A.sup[xp], (ull)(0ull - dec));
}

// wedge walk over the slices in mb (see walk_chunks in wedge.cuh); f(x')
template <int N, class F>
__device__ __forceinline__ void walk_slices(const PeelArgs &A, int rank, const PMid<N> &mb, int nseg, uint32_t C,
                                            F &&f) {
  walk_chunks<N>(A.o_adj, rank, mb.lo, mb.len, mb.pre, nseg, C, [&](int, uint32_t, uint32_t v) { f(v); });
}

// whole current lists of N(x)[base, base + N): slices into mb, returns their chunks
template <class Grp, int N>
__device__ __forceinline__ uint32_t peel_load(const PeelArgs &A, uint32_t xo, uint32_t xd, uint32_t base, const Grp &g,
                                              PMid<N> &mb) {
  int r = g.rank();
  uint32_t lo = 0, len = 0;
  if (base + r < xd) {
    uint32_t y = A.p_adj[xo + base + r];
    lo = A.o_off[y];
    len = A.o_len[y];
  }
  mb.lo[r] = lo;
  mb.len[r] = len;
  return g.scan(nchunks(len), mb.pre);
}

struct PHash {
  SmemHash h;
  uint32_t cap;
  __device__ void inc(uint32_t k) const { h.inc(k); }
  template <class Grp>
  __device__ uint64_t drain(const PeelArgs &A, const Grp &g) const {
    uint64_t nup = 0;
    for (uint32_t i = g.rank(); i < cap; i += Grp::N) {
      uint32_t k = h.key[i];
      if (k != EMPTY_KEY) {
        uint32_t c = h.val[i];
        if (c >= 2) {
          sub_support(A, k, choose2(c));
          nup++;
        }
        h.key[i] = EMPTY_KEY;
        h.val[i] = 0;
      }
    }
    return nup;
  }
};

// whole vertex through one shared hash (warp and group classes); returns
// this thread's number of support updates
template <class Grp, int N, class Tbl>
__device__ uint64_t peel_vertex(const PeelArgs &A, uint32_t x, const Grp &g, PMid<N> &mb, const Tbl &tbl) {
  uint32_t xo = A.p_off[x], xd = A.p_off[x + 1] - xo;
  for (uint32_t base = 0; base < xd; base += N) {
    uint32_t C = peel_load(A, xo, xd, base, g, mb);
    walk_slices(A, g.rank(), mb, (int)min((uint32_t)N, xd - base), C, [&](uint32_t xp) { tbl.inc(xp); });
    g.sync();
  }
  uint64_t nup = tbl.drain(A, g);
  g.sync();
  return nup;
}

__device__ __forceinline__ void add_updates(const PeelArgs &A, uint64_t nup) {
  for (int o = 16; o; o >>= 1) nup += __shfl_xor_sync(0xffffffffu, nup, o);
  if ((threadIdx.x & 31) == 0 && nup && A.updates) atomicAdd(A.updates, (ull)nup);
}

__global__ void __launch_bounds__(PWT) k_peel_warp(PeelArgs A, const uint64_t *list, const unsigned *count) {
  extern __shared__ __align__(16) uint8_t sm[];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr size_t per = align16(QW_CAP * 8 + sizeof(PMid<32>));
  uint32_t *key = (uint32_t *)(sm + w * per), *val = key + QW_CAP;
  PMid<32> &mb = *(PMid<32> *)(sm + w * per + QW_CAP * 8);
  for (uint32_t i = lane; i < QW_CAP; i += 32) key[i] = EMPTY_KEY, val[i] = 0;
  __syncwarp();
  WarpGrp g;
  uint64_t nup = 0;
  unsigned n = *count;
  for (size_t it = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5; it < n; it += ((size_t)gridDim.x * blockDim.x) >> 5) {
    uint64_t item = list[it];
    uint32_t x = (uint32_t)item, W = (uint32_t)(item >> 32);
    uint32_t cap = pow2_at_least(max(2u * W, 32u));
    PHash p{SmemHash{key, val, cap - 1}, cap};
    nup += peel_vertex(A, x, g, mb, p);
  }
  add_updates(A, nup);
}

// two 256-thread groups per block, each with its own shared hash and named
// barrier, one active vertex per group
__global__ void __launch_bounds__(2 * QGT) k_peel_group(PeelArgs A, const uint64_t *list, const unsigned *count) {
  if ((size_t)blockIdx.x * 2 >= *count) return;  // fixed grids of graph-captured rounds
  extern __shared__ __align__(16) uint8_t sm[];
  int sub = threadIdx.x / QGT;
  constexpr size_t per = align16(QG_CAP * 8 + sizeof(PMid<QGT>) + (QGT / 32 + 2) * 4);
  uint8_t *base = sm + sub * per;
  uint32_t *key = (uint32_t *)base, *val = key + QG_CAP;
  PMid<QGT> &mb = *(PMid<QGT> *)(base + QG_CAP * 8);
  uint32_t *ws = (uint32_t *)(base + QG_CAP * 8 + sizeof(PMid<QGT>));
  SubGrp<QGT> g{sub * QGT, 1 + sub, ws, nullptr};
  for (uint32_t i = g.rank(); i < QG_CAP; i += QGT) key[i] = EMPTY_KEY, val[i] = 0;
  g.sync();
  uint64_t nup = 0;
  unsigned n = *count;
  for (size_t it = (size_t)blockIdx.x * 2 + sub; it < n; it += (size_t)gridDim.x * 2) {
    uint64_t item = list[it];
    uint32_t x = (uint32_t)item, W = (uint32_t)(item >> 32);
    uint32_t cap = pow2_at_least(max(2u * W, 64u));
    PHash p{SmemHash{key, val, cap - 1}, cap};
    nup += peel_vertex(A, x, g, mb, p);
  }
  add_updates(A, nup);
}

size_t peel_group_smem() { return 2 * align16(QG_CAP * 8 + sizeof(PMid<QGT>) + (QGT / 32 + 2) * 4); }

// Shared hash with one 64-bit slot per target: (id + 1) << 32 | count, zero
// = empty, so that an insert is a single compare-and-swap and a repeat a
// single add, and an all-zero table doubles as zeroed dense counters.
struct WHash {
  unsigned long long *slot;
  uint32_t mask;
  __device__ __forceinline__ void inc(uint32_t id) const {
    const uint32_t tag = id + 1;
    uint32_t h = hash32(id) & mask;
    for (;;) {  // claim first: one shared operation for a new target
      unsigned long long cur = atomicCAS(&slot[h], 0ull, ((unsigned long long)tag << 32) | 1ull);
      if (cur == 0) return;
      if ((uint32_t)(cur >> 32) == tag) {
        atomicAdd(&slot[h], 1ull);
        return;
      }
      h = (h + 1) & mask;
    }
  }
};

// Shared hash with 32-bit slots (id - c0 + 1) << cb | count, for passes whose
// id range and counts fit together in 32 bits: twice the slots of WHash.
struct PHash32 {
  uint32_t *slot;
  uint32_t mask, c0, cb;
  __device__ __forceinline__ void inc(uint32_t id) const {
    const uint32_t tag = id - c0 + 1;
    uint32_t h = hash32(id) & mask;
    for (;;) {  // claim first: one shared operation for a new target
      uint32_t cur = atomicCAS(&slot[h], 0u, (tag << cb) | 1u);
      if (cur == 0) return;
      if ((cur >> cb) == tag) {
        atomicAdd(&slot[h], 1u);  // the count stays below 2^cb
        return;
      }
      h = (h + 1) & mask;
    }
  }
};

__device__ __forceinline__ uint32_t bit_len(uint64_t v) { return v ? 64 - __clzll(v) : 0; }

// slice of y's current list holding the targets of buckets [bs, be)
__device__ __forceinline__ void bucket_slice(const PeelArgs &A, uint32_t y, uint32_t bs, uint32_t be, uint32_t &lo,
                                             uint32_t &len) {
  uint32_t s0 = A.o_off[y];
  if (bs == 0 && be >= A.nb) {
    lo = s0;
    len = A.o_len[y];
    return;
  }
  const uint32_t *bo = A.boff + (size_t)y * (A.nb + 1);
  uint32_t a = bo[bs], b = bo[be];
  lo = s0 + a;
  len = b - a;
}

// Block-class work item: one active vertex x and a range of target buckets
// [b0, b1) (a heavy vertex is split into several items that run on
// different blocks; their targets are disjoint).  The block
//  1. sums, per bucket, the wedges of x landing in it (slice lengths),
//  2. cuts the buckets greedily into passes: a bucket with more than G
//     wedges starts a dense pass (16-bit counters over 32K ids when x has
//     fewer than 2^16 neighbours, else 32-bit counters over 16K ids), the
//     others are grouped while their wedges stay within G,
//  3. runs each pass: its slices are walked once into 64 KB of shared memory
//     - an open-addressing hash for a group (load at most 1/2), dense
//     counters for a heavy range (a bucket wider than the counters is cut
//     into sub-ranges found by binary search inside its slices) - and every
//     aggregated target x' loses C(c(x,x'), 2).
constexpr uint32_t BK_G = PB_CAP / 2;  // most wedges (hence targets) of a hash pass
constexpr uint32_t NB_MAX = PBT;      // buckets per item: one per thread

struct BPlan {
  uint32_t a[NB_MAX + 1];  // per-bucket wedges, then pass starts
  uint32_t b[NB_MAX + 1];  // prefix of the wedges, then per-pass wedges
  uint32_t np;
};

// drain of dense counters over ids [d0, d0 + n): 32-bit counters, or 16-bit
// halves (offset o in word o mod 2^14, half o / 2^14); 16-byte vector reads,
// zeroed where touched
template <bool W16>
__device__ __forceinline__ uint64_t drain_dense(const PeelArgs &A, uint32_t *tab, uint32_t d0, uint32_t n, int t, int N) {
  uint64_t nup = 0;
  uint4 *v = (uint4 *)tab;
  const uint32_t words = W16 ? min(n, P_CHUNK) : n;
  for (uint32_t i = t; i * 4 < words; i += N) {
    uint4 q = v[i];
    if ((q.x | q.y | q.z | q.w) == 0u) continue;
    v[i] = make_uint4(0u, 0u, 0u, 0u);
    uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (!w[k]) continue;
      uint32_t id = d0 + i * 4 + k;
      if (W16) {
        uint32_t lo = w[k] & 0xffffu, hi = w[k] >> 16;
        if (lo >= 2) sub_support(A, id, choose2(lo)), nup++;
        if (hi >= 2) sub_support(A, id + P_CHUNK, choose2(hi)), nup++;
      } else if (w[k] >= 2) {
        sub_support(A, id, choose2(w[k]));
        nup++;
      }
    }
  }
  return nup;
}

template <int N>
__device__ uint64_t peel_item_block(const PeelArgs &A, uint32_t x, uint32_t b0, uint32_t b1, const BlockGrp<N> &g,
                                    PMid<N> &mb, BPlan &pl, uint32_t *tab) {
  const uint32_t xo = A.p_off[x], xd = A.p_off[x + 1] - xo, nbi = b1 - b0;
  const int t = threadIdx.x;
  uint64_t nup = 0;
  const bool stat = PBNG_PEEL_STATS && A.bstat && t == 0;  // (a few global atomics per pass)
  long long c_item = stat ? clock64() : 0, c_mark = c_item;
  auto add = [&](int k, ull v) {
    if (stat) atomicAdd(&A.bstat[k], v);
  };
  auto mark = [&](int k) {
    if (stat) {
      long long c = clock64();
      atomicAdd(&A.bstat[k], (ull)(c - c_mark));
      c_mark = c;
    }
  };
  // this thread's neighbour (items of vertices with at most N neighbours)
  const bool cached = xd <= (uint32_t)N;
  uint32_t my_s0 = 0, my_len = 0;
  const uint32_t *my_bo = nullptr;
  if (cached && t < (int)xd) {
    uint32_t y = A.p_adj[xo + t];
    my_s0 = A.o_off[y];
    my_len = A.o_len[y];
    if (A.boff) my_bo = A.boff + (size_t)y * (A.nb + 1);
  }
  // 1. wedges per bucket
  if (t < (int)nbi) pl.a[t] = 0;
  __syncthreads();
  if (nbi == 1) {
    uint32_t s = 0;
    if (cached) {
      if (t < (int)xd) s = my_bo ? my_bo[b1] - my_bo[b0] : my_len;
    } else {
      for (uint32_t k = t; k < xd; k += N) {
        uint32_t lo, len;
        bucket_slice(A, A.p_adj[xo + k], b0, b1, lo, len);
        s += len;
      }
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((t & 31) == 0 && s) atomicAdd(&pl.a[0], s);
  } else {  // warps over neighbours, lanes over buckets (one row of offsets per neighbour)
    const uint32_t lane = t & 31, wid = t >> 5;
    for (uint32_t j = 0; j < nbi; j += 32) {
      uint32_t b = j + lane, s = 0;
      if (b < nbi)
        for (uint32_t k = wid; k < xd; k += N / 32) {
          const uint32_t *bo = A.boff + (size_t)A.p_adj[xo + k] * (A.nb + 1) + b0 + b;
          s += bo[1] - bo[0];
        }
      if (s) atomicAdd(&pl.a[b], s);
    }
  }
  __syncthreads();
  // 2. passes (greedy, one thread; pass starts into a, pass wedges into b)
  g.scan(t < (int)nbi ? pl.a[t] : 0u, pl.b);
  const bool w16 = xd < 65536u;  // a count never exceeds the number of neighbours
  const uint32_t dcap = w16 ? 2 * P_CHUNK : P_CHUNK;  // ids of one dense pass
  // 32-bit hash slots when every pass's id offsets and x's counts fit in them
  const uint32_t cb = bit_len(xd);
  const bool packed = bit_len((uint64_t)nbi << A.bshift) + cb <= 32;
  const uint32_t G = packed ? 2 * BK_G : BK_G;  // most wedges of a hash pass (load <= 1/2)
  const uint32_t width = 1u << A.bshift;
  const uint32_t dspan = width <= dcap ? dcap >> A.bshift : 1u;
  if (t == 0) {
    uint32_t s = 0, q = 0;
    while (s < nbi) {
      uint32_t e;
      if (pl.b[s + 1] - pl.b[s] > G) {
        e = min(nbi, s + dspan);
      } else {  // largest e with wedges(s..e) <= G
        uint32_t lo = s + 1, hi = nbi, lim = pl.b[s] + G;
        while (lo < hi) {
          uint32_t mid = (lo + hi + 1) >> 1;
          if (pl.b[mid] <= lim) lo = mid;
          else hi = mid - 1;
        }
        e = lo;
      }
      uint32_t T = pl.b[e] - pl.b[s];
      pl.a[q] = s;
      pl.b[q] = T;  // q <= s: no later read of the prefix looks at or below q
      q++;
      s = e;
    }
    pl.a[q] = nbi;
    pl.np = q;
  }
  __syncthreads();
  const uint32_t np = pl.np;
  mark(BS_CYC_PLAN);
  // 3. passes
  for (uint32_t qi = 0; qi < np; qi++) {
    const uint32_t bs = b0 + pl.a[qi], be = b0 + pl.a[qi + 1], Tq = pl.b[qi];
    if (Tq == 0) continue;
    const bool hash = Tq <= G;
    const uint32_t c0 = bs << A.bshift;
    const uint32_t cend = (uint32_t)min((uint64_t)A.nx, (uint64_t)be << A.bshift);
    const bool narrow = hash || width <= dcap;
    for (uint32_t d0 = c0; d0 < cend; d0 += narrow ? (cend - c0) : dcap) {
      const uint32_t d1 = narrow ? cend : min(cend, d0 + dcap);
      uint32_t cap = hash ? pow2_at_least(max(2u * Tq, 64u)) : 0u;
      WHash h{(unsigned long long *)tab, cap - 1};
      PHash32 h32{tab, cap - 1, c0, cb};
      auto load = [&](uint32_t base) -> uint32_t {  // slices of N(x)[base, base + N); returns chunks
        uint32_t lo = 0, len = 0;
        if (cached) {
          if (t < (int)xd) {
            if (bs == 0 && be >= A.nb) lo = 0, len = my_len;
            else lo = my_bo[bs], len = my_bo[be] - lo;
            lo += my_s0;
          }
        } else if (base + t < xd) {
          bucket_slice(A, A.p_adj[xo + base + t], bs, be, lo, len);
        }
        if (!narrow && len) {
          uint32_t a0 = lower_bound_u32(A.o_adj + lo, len, d0);
          uint32_t a1 = a0 + lower_bound_u32(A.o_adj + lo + a0, len - a0, d1);
          lo += a0;
          len = a1 - a0;
        }
        mb.lo[t] = lo;
        mb.len[t] = len;
        return g.scan(nchunks(len), mb.pre);
      };
      auto walk_all = [&](auto &&f) -> uint32_t {
        uint32_t Cw = 0;
        for (uint32_t base = 0; base < xd; base += N) {
          uint32_t C = (base == 0 || !cached) ? load(base) : 0u;
          Cw += C;
          walk_slices(A, t, mb, (int)min((uint32_t)N, xd - base), C, f);
          __syncthreads();
          if (cached) break;
        }
        return Cw;
      };
      bool rewalk = false;
      add(hash ? BS_PASS_HASH : BS_PASS_DENSE, 1);
      add(BS_WEDGES, Tq);
      if (hash && packed) {
        add(BS_LANES, 32ull * walk_all([&](uint32_t xp) { h32.inc(xp); }));
        mark(BS_CYC_WALK);
        const uint32_t cmask = (1u << cb) - 1u;
        for (uint32_t i = 4 * t; i < cap; i += 4 * N) {  // drain four slots at a time
          uint4 q = *(uint4 *)&tab[i];
          if ((q.x | q.y | q.z | q.w) == 0u) continue;
          uint32_t v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int u = 0; u < 4; u++) {
            uint32_t c = v[u] & cmask;
            if (c >= 2) sub_support(A, c0 + (v[u] >> cb) - 1, choose2(c)), nup++;
          }
          *(uint4 *)&tab[i] = make_uint4(0u, 0u, 0u, 0u);
        }
      } else if (hash) {
        add(BS_LANES, 32ull * walk_all([&](uint32_t xp) { h.inc(xp); }));
        mark(BS_CYC_WALK);
        for (uint32_t i = 2 * t; i < cap; i += 2 * N) {  // drain two slots at a time
          uint4 q = *(uint4 *)&tab[2 * i];  // slots i, i + 1: (count, tag) words
          if ((q.x | q.y | q.z | q.w) == 0u) continue;
          if (q.x >= 2) sub_support(A, q.y - 1, choose2(q.x)), nup++;
          if (q.z >= 2) sub_support(A, q.w - 1, choose2(q.z)), nup++;
          *(uint4 *)&tab[2 * i] = make_uint4(0u, 0u, 0u, 0u);
        }
      } else if (w16) {  // offset o counts in word o mod 2^14, half o / 2^14 (consecutive ids, distinct words)
        const uint32_t Cw = walk_all([&](uint32_t xp) {
          uint32_t o = xp - d0;
          atomicAdd(&tab[o & (P_CHUNK - 1)], 1u << ((o >> 14) * 16));
        });
        add(BS_LANES, 32ull * Cw);
        mark(BS_CYC_WALK);
        const uint64_t Tw = narrow ? (uint64_t)Tq : (uint64_t)Cw * 32;
        if (Tw >= (d1 - d0) / 2 || !cached) {  // crowded (or slices not kept): scan the counters
          add(BS_DRAIN_DENSE, 1);
          nup += drain_dense<true>(A, tab, d0, d1 - d0, t, N);
        } else {  // sparse: walk the wedges again, the first visitor takes the count
          add(BS_DRAIN_SPARSE, 1);
          rewalk = true;
          walk_slices(A, t, mb, (int)xd, Cw, [&](uint32_t xp) {
            uint32_t o = xp - d0, sh = (o >> 14) * 16;
            uint32_t c = (atomicAnd(&tab[o & (P_CHUNK - 1)], ~(0xffffu << sh)) >> sh) & 0xffffu;
            if (c >= 2) sub_support(A, xp, choose2(c)), nup++;
          });
        }
      } else {
        const uint32_t Cw = walk_all([&](uint32_t xp) { atomicAdd(&tab[xp - d0], 1u); });
        add(BS_LANES, 32ull * Cw);
        mark(BS_CYC_WALK);
        const uint64_t Tw = narrow ? (uint64_t)Tq : (uint64_t)Cw * 32;
        if (Tw >= (d1 - d0) / 2 || !cached) {
          add(BS_DRAIN_DENSE, 1);
          nup += drain_dense<false>(A, tab, d0, d1 - d0, t, N);
        } else {
          add(BS_DRAIN_SPARSE, 1);
          rewalk = true;
          walk_slices(A, t, mb, (int)xd, Cw, [&](uint32_t xp) {
            uint32_t c = atomicExch(&tab[xp - d0], 0u);
            if (c >= 2) sub_support(A, xp, choose2(c)), nup++;
          });
        }
      }
      __syncthreads();
      mark(rewalk ? BS_CYC_REWALK : BS_CYC_DRAIN);
    }
  }
  __syncthreads();  // the plan arrays are rewritten by the next item
  add(BS_ITEMS, 1);
  if (stat) add(BS_CYC_ITEM, (ull)(clock64() - c_item));
  return nup;
}

__global__ void __launch_bounds__(PBT, PB_PER_SM) k_peel_block(PeelArgs A, const uint64_t *list, const unsigned *count) {
  if (blockIdx.x >= *count) return;  // fixed grids of graph-captured rounds
  extern __shared__ __align__(16) uint8_t sm[];
  PMid<PBT> &mb = *(PMid<PBT> *)sm;
  constexpr size_t o1 = align16(sizeof(PMid<PBT>));
  constexpr size_t o2 = o1 + 256;
  constexpr size_t o3 = o2 + align16(sizeof(BPlan));
  uint32_t *ws = (uint32_t *)(sm + o1);
  ull *ws64 = (ull *)(sm + o1 + 128);
  BPlan &pl = *(BPlan *)(sm + o2);
  uint32_t *tab = (uint32_t *)(sm + o3);  // PB_CAP keys + PB_CAP values, or P_CHUNK counters
  BlockGrp<PBT> g{ws, ws64};
  for (uint32_t i = threadIdx.x; i < 2 * PB_CAP; i += PBT) tab[i] = 0;  // empty hash == zero counters
  __syncthreads();
  uint64_t nup = 0;
  unsigned n = *count;
  for (size_t it = blockIdx.x; it < n; it += gridDim.x) {
    uint64_t item = list[it];
    uint32_t x = (uint32_t)item, b0 = (uint32_t)(item >> 32) & 0xffffu, b1 = (uint32_t)(item >> 48);
    nup += peel_item_block(A, x, b0, b1, g, mb, pl, tab);
  }
  add_updates(A, nup);
}

size_t peel_block_smem() { return align16(sizeof(PMid<PBT>)) + 256 + align16(sizeof(BPlan)) + (size_t)PB_CAP * 8; }

// bucket offsets of one list (warp): bo[b] = first position whose id is in
// bucket >= b, for b = 0..nb
__device__ __forceinline__ void fill_boff(const uint32_t *list, uint32_t len, uint32_t *bo, uint32_t nb, uint32_t bshift,
                                          int lane) {
  for (uint32_t k = 0; k < len; k += 32) {
    uint32_t p = k + lane;
    if (p < len) {
      uint32_t bp = list[p] >> bshift;
      uint32_t bq = p == 0 ? 0u : (list[p - 1] >> bshift) + 1;
      for (uint32_t b = bq; b <= bp; b++) bo[b] = p;
    }
  }
  uint32_t bl = len == 0 ? 0u : (list[len - 1] >> bshift) + 1;
  for (uint32_t b = bl + lane; b <= nb; b += 32) bo[b] = len;
}

__global__ void k_boff_build(const uint32_t *o_off, const uint32_t *o_adj, uint32_t ny, uint32_t *boff, uint32_t nb,
                             uint32_t bshift) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t y = gw; y < ny; y += nw)
    fill_boff(o_adj + o_off[y], o_off[y + 1] - o_off[y], boff + y * (size_t)(nb + 1), nb, bshift, lane);
}

// sum over Y of len^2 = the wedges of all X vertices together
__global__ void k_sum_sq(const uint32_t *o_off, uint32_t ny, ull *out) {
  ull s = 0;
  for (size_t y = blockIdx.x * (size_t)blockDim.x + threadIdx.x; y < ny; y += (size_t)gridDim.x * blockDim.x) {
    ull d = o_off[y + 1] - o_off[y];
    s += d * d;
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// ------------------------------------------------------- round bookkeeping
struct PrepArgs {
  const uint32_t *frontier;
  uint32_t nf;
  const uint32_t *p_off, *p_adj, *o_len;
  uint32_t *part;
  uint32_t pi;
  uint8_t *state;
  ull *sum_w;  // [0] wedges of the active set, [1] its (vertex, mid) expansions, [2] largest W
  uint64_t *lists;  // warp and group classes, nx entries each: x | W << 32
  uint64_t *blist;  // block class work items: x | b0 << 32 | b1 << 48
  unsigned *counts;
  uint32_t nx, nb;
  uint64_t item_w;  // wedges per block-class item (at least)
  uint32_t warp_max_w, group_max_w;  // class limits (at most QW_MAXW, QG_MAXW)
  uint8_t *lab_alive;  // re-count labels (Sec. 5.1), or null
  const uint32_t *x2lab;
  // dynamic graph updates (Sec. 5.2): the active vertices' entries die this
  // round; a Y list is queued for compaction once a quarter of it is dead
  int compact;
  uint32_t *dead, *ytouch, *touched;
  unsigned *touched_n;
  const unsigned *nf_dev = nullptr, *pi_dev = nullptr;  // device-resident sizes (graph-captured rounds)
};

// one warp per active vertex: partition id, wedge count, class, touched Y lists
__global__ void k_prep(PrepArgs A) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  if (A.nf_dev) {
    A.nf = *A.nf_dev;
    A.pi = *A.pi_dev;
  }
  for (size_t j = gw; j < A.nf; j += nw) {
    uint32_t x = A.frontier[j];
    uint32_t xo = A.p_off[x], xd = A.p_off[x + 1] - xo;
    uint64_t W = 0;
    for (uint32_t k = lane; k < xd; k += 32) {
      uint32_t y = A.p_adj[xo + k], len = A.o_len[y];
      W += len;
      if (A.compact) {
        uint32_t d = atomicAdd(&A.dead[y], 1u) + 1;
        if (4 * d >= len && atomicExch(&A.ytouch[y], 1u) == 0u) A.touched[atomicAdd(A.touched_n, 1u)] = y;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) W += __shfl_xor_sync(0xffffffffu, W, o);
    if (lane == 0) {
      A.part[x] = A.pi;
      A.state[x] = ST_ACTIVE;  // leaves the remaining graph this round
      if (A.lab_alive) A.lab_alive[A.x2lab[x]] = 0;
      atomicAdd(&A.sum_w[0], (ull)W);
      atomicAdd(&A.sum_w[1], (ull)xd);
      atomicMax(&A.sum_w[2], (ull)W);
      if (W >= 2) {
        if (W <= A.group_max_w) {
          int c = W <= A.warp_max_w ? PC_WARP : PC_GROUP;
          unsigned p = atomicAdd(&A.counts[c], 1u);
          A.lists[(size_t)c * A.nx + p] = (uint64_t)x | (W << 32);
        } else {  // K items over equal shares of the target buckets
          uint32_t K = (uint32_t)min((uint64_t)A.nb, (W + A.item_w - 1) / A.item_w);
          unsigned p = atomicAdd(&A.counts[PC_BLOCK], K);
          for (uint32_t k = 0; k < K; k++) {
            uint64_t b0 = (uint64_t)k * A.nb / K, b1 = (uint64_t)(k + 1) * A.nb / K;
            A.blist[p + k] = (uint64_t)x | (b0 << 32) | (b1 << 48);
          }
        }
      }
    }
  }
}

// device-resident state of the graph-captured coarse rounds
struct RoundDev {
  unsigned nf, nn, touched_n, pi, na, pad_;
  unsigned counts[4];
  ull sum_w[3];
  ull tot_wedges, tot_exp, tot_front, rounds, part_work, iters;
};

__global__ void k_round_reset(RoundDev *R) {
  R->nn = 0;
  R->touched_n = 0;
  for (int i = 0; i < 4; i++) R->counts[i] = 0;
  R->sum_w[0] = R->sum_w[1] = R->sum_w[2] = 0;
}

// end of one round: totals, next frontier size, and (last round of the body)
// the loop condition of the conditional node
__global__ void k_round_end(RoundDev *R, cudaGraphConditionalHandle h, int set_cond) {
  if (R->nf) {
    R->rounds++;
    R->tot_wedges += R->sum_w[0];
    R->tot_exp += R->sum_w[1];
    R->tot_front += R->nf;
    R->part_work += R->sum_w[0];
  }
  R->nf = R->nn;
  if (set_cond) {
    R->iters++;
    cudaGraphSetConditional(h, R->nn > 0 ? 1u : 0u);
  }
}

// warp per touched Y vertex: stable in-place removal of peeled X entries
__global__ void k_compact(const uint32_t *touched, const unsigned *tn, const uint32_t *o_off, uint32_t *o_adj, uint32_t *o_len,
                          uint32_t *ytouch, uint32_t *dead, const uint8_t *state, uint32_t *boff, uint32_t nb,
                          uint32_t bshift) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  unsigned n = *tn;
  for (size_t j = gw; j < n; j += nw) {
    uint32_t y = touched[j];
    uint32_t lo = o_off[y], len = o_len[y], out = 0;
    for (uint32_t k = 0; k < len; k += 32) {
      uint32_t x = 0;
      bool keep = false;
      if (k + lane < len) {
        x = o_adj[lo + k + lane];
        keep = state[x] == ST_ALIVE;
      }
      unsigned b = __ballot_sync(0xffffffffu, keep);
      __syncwarp();
      if (keep) o_adj[lo + out + __popc(b & ((1u << lane) - 1u))] = x;
      out += __popc(b);
      __syncwarp();
    }
    if (boff) {  // the list's bucket offsets
      __syncwarp();
      fill_boff(o_adj + lo, out, boff + (size_t)y * (nb + 1), nb, bshift, lane);
    }
    if (lane == 0) {
      o_len[y] = out;
      ytouch[y] = 0;
      dead[y] = 0;
    }
  }
}

// -------------------------------------------------- partition bookkeeping
// keep alive entries of the remaining list
__global__ void k_compact_list(const uint32_t *in, uint32_t n, const uint8_t *state, uint32_t *out, unsigned *on) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    uint32_t x = in[j];
    bool keep = state[x] == ST_ALIVE;
    unsigned b = __ballot_sync(__activemask(), keep);
    int lane = threadIdx.x & 31, leader = __ffs(__activemask()) - 1;
    unsigned base = 0;
    if (lane == leader && b) base = atomicAdd(on, __popc(b));
    base = __shfl_sync(__activemask(), base, leader);
    if (keep) out[base + __popc(b & ((1u << lane) - 1u))] = x;
  }
}

// work proxy of the remaining vertices with support below a bound
__global__ void k_work_below(const uint32_t *alist, uint32_t na, const ull *sup, const ull *wl, ull bound, ull *out) {
  ull s = 0;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < na; j += (size_t)gridDim.x * blockDim.x)
    if (sup[alist[j]] < bound) s += wl[j];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// key range of the remaining vertices only (no work proxy)
__global__ void k_keyrange(const uint32_t *alist, uint32_t na, const ull *sup, RangeState *rs) {
  ull mn = ~0ull, mx = 0;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < na; j += (size_t)gridDim.x * blockDim.x) {
    ull s = sup[alist[j]];
    mn = min(mn, s);
    mx = max(mx, s);
  }
  for (int o = 16; o; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&rs->kmin, mn);
    atomicMax(&rs->kmax, mx);
  }
}

// warp per remaining vertex: work proxy w = wedges of x on the current graph
// (Sec. 3.2), key range and total work
__global__ void k_weights(const uint32_t *alist, uint32_t na, const uint32_t *p_off, const uint32_t *p_adj,
                          const uint32_t *o_len, const ull *sup, ull *wl, RangeState *rs) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  ull mn = ~0ull, mx = 0, ws = 0;
  for (size_t j = gw; j < na; j += nw) {
    uint32_t x = alist[j];
    uint32_t xo = p_off[x], xd = p_off[x + 1] - xo;
    ull W = 0;
    for (uint32_t k = lane; k < xd; k += 32) W += o_len[p_adj[xo + k]];
#pragma unroll
    for (int o = 16; o; o >>= 1) W += __shfl_xor_sync(0xffffffffu, W, o);
    if (lane == 0) {
      wl[j] = W;
      ull s = sup[x];
      mn = min(mn, s);
      mx = max(mx, s);
      ws += W;
    }
  }
  if (lane == 0) {
    atomicMin(&rs->kmin, mn);
    atomicMax(&rs->kmax, mx);
    if (ws) atomicAdd(&rs->wsum, ws);
  }
}

// start of a range (snapshot = 1): init <- support; any pass: the active set
// is every unpeeled vertex with support below theta_hi
// Next active set: every remaining vertex still alive with support below the
// range's upper bound (also the first active set of a range, with the
// snapshot of the supports into init).
__global__ void k_scan_frontier(const uint32_t *alist, uint32_t na, uint8_t *state, const ull *sup, ull *init,
                                const ull *theta_hi, int snapshot, uint32_t *f, unsigned *fn,
                                const unsigned *na_dev = nullptr) {
  ull thi = *theta_hi;
  if (na_dev) na = *na_dev;
  int lane = threadIdx.x & 31;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t j0 = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) & ~(size_t)31; j0 < na; j0 += stride) {
    size_t j = j0 + lane;
    bool take = false;
    uint32_t x = 0;
    if (j < na) {
      x = alist[j];
      if (state[x] == ST_ALIVE) {
        ull s = sup[x];
        if (snapshot) init[x] = s;
        take = s < thi;
      }
    }
    unsigned b = __ballot_sync(0xffffffffu, take);
    unsigned base = 0;
    if (lane == 0 && b) base = atomicAdd(fn, (unsigned)__popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (take) {
      state[x] = ST_ACTIVE;
      f[base + __popc(b & ((1u << lane) - 1u))] = x;
    }
  }
}

__global__ void k_gather_counts(const uint32_t *alist, uint32_t na, const uint8_t *state, const uint32_t *x2lab,
                                const ull *cnt_lab, ull *sup) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < na; j += (size_t)gridDim.x * blockDim.x) {
    uint32_t x = alist[j];
    if (state[x] == ST_ALIVE) sup[x] = cnt_lab[x2lab[x]];
  }
}

__global__ void k_degrees(const uint32_t *off, uint32_t n, uint32_t *len) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    len[i] = off[i + 1] - off[i];
}

__global__ void k_init_side(uint32_t nx, const uint32_t *x2lab, const ull *cnt_lab, ull *sup, uint32_t *alist) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < nx; x += (size_t)gridDim.x * blockDim.x) {
    sup[x] = cnt_lab[x2lab[x]];
    alist[x] = (uint32_t)x;
  }
}

__global__ void k_x2lab(const uint32_t *g2lab, uint32_t off, uint32_t nx, uint32_t *x2lab) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < nx; x += (size_t)gridDim.x * blockDim.x)
    x2lab[x] = g2lab[off + x];
}

// ------------------------------------------------------------ fine phase
struct FDArgs {
  const uint32_t *p_off, *p_adj;  // X -> Y
  const uint32_t *o_off;          // Y segments in the partitioned adjacency
  const uint32_t *fd_adj, *fd_part;  // Y -> X grouped by (y, part(x)), x ascending
  const uint32_t *xs, *ps, *loc;  // X ids grouped by partition; partition offsets; local index
  const uint32_t *order;          // partitions, heaviest first
  uint32_t nparts;
  uint8_t *state;
  ull *sup;  // starts as init
  ull *theta;
  uint32_t *buf_a, *buf_b, *buf_c, *buf_d, *buf_f, *buf_big;  // per-partition regions (offset ps[p])
  uint32_t *buf_huge;                                        // heavy vertices left by the groups (offset ps[p])
  uint32_t *gcnt;                             // per-partition dense counters (offset ps[p]), zeroed
  unsigned *queue;
  ull *wedges, *steps, *updates;
  ull *pstat;  // per partition: steps, SM cycles
  const uint32_t *seg_lo, *seg_len;  // per X-side edge: slice of (y, part(x)) in fd_adj
  const uint32_t *w_fd;              // per vertex: wedges in its partition's subgraph
  const uint32_t *seg_n;             // per vertex: its non-empty slices (from its first edge position)
};

constexpr int FT = 512, FW = FT / 32;
constexpr int TFD_PSTAT = 9;  // per-partition statistics of the fine phase

template <int N>
struct FMid {
  uint32_t lo[N];
  uint32_t pre[N + 1];
};

// segment of y's partitioned list holding partition p
__device__ __forceinline__ void fd_seg(const FDArgs &A, uint32_t y, uint32_t p, uint32_t &lo, uint32_t &len) {
  uint32_t b = A.o_off[y], e = A.o_off[y + 1];
  uint32_t l0 = b + lower_bound_u32(A.fd_part + b, e - b, p);
  uint32_t l1 = l0 + lower_bound_u32(A.fd_part + l0, e - l0, p + 1);
  lo = l0;
  len = l1 - l0;
}

template <class Grp, int N>
__device__ __forceinline__ uint32_t fd_load(const FDArgs &A, uint32_t p, uint32_t xo, uint32_t xd, uint32_t base,
                                            const Grp &g, FMid<N> &mb) {
  int r = g.rank();
  uint32_t lo = 0, len = 0;
  if (base + r < xd) {
    lo = A.seg_lo[xo + base + r];
    len = A.seg_len[xo + base + r];
  }
  mb.lo[r] = lo;
  return g.scan(len, mb.pre);
}

// once per call: every x gets the non-empty slices of its neighbours'
// partitioned lists that hold partition part(x) - compacted to the front of
// its own edge range, seg_n[x] of them - and its wedge count in G_part(x)
// (a neighbour with no vertex of the partition costs nothing later)
__global__ void k_fd_segs(FDArgs A, uint32_t nx, const uint32_t *part, uint32_t *seg_lo, uint32_t *seg_len, uint32_t *w_fd,
                          uint32_t *seg_n) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t x = gw; x < nx; x += nw) {
    uint32_t xo = A.p_off[x], xd = A.p_off[x + 1] - xo, p = part[x], W = 0, out = 0;
    for (uint32_t k0 = 0; k0 < xd; k0 += 32) {
      uint32_t lo = 0, len = 0;
      if (k0 + lane < xd) fd_seg(A, A.p_adj[xo + k0 + lane], p, lo, len);
      const unsigned b = __ballot_sync(0xffffffffu, len > 0);
      if (len) {
        const uint32_t at = xo + out + __popc(b & ((1u << lane) - 1u));
        seg_lo[at] = lo;
        seg_len[at] = len;
      }
      out += __popc(b);
      W += len;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) W += __shfl_xor_sync(0xffffffffu, W, o);
    if (lane == 0) {
      w_fd[x] = W;
      seg_n[x] = out;
    }
  }
}

// the T wedges of the slices in mb in flattened order (the partitioned slices
// are short, so one lane per wedge beats whole-warp chunks here)
template <class Grp, int N, class F>
__device__ __forceinline__ void fd_walk(const FDArgs &A, const Grp &g, const FMid<N> &mb, uint32_t T, F &&f) {
  uint32_t w = g.rank();
  for (; w + N < T; w += 2 * N) {  // two wedges in flight
    int i0 = seg_of(mb.pre, N, w), i1 = seg_of(mb.pre, N, w + N);
    uint32_t a0 = A.fd_adj[mb.lo[i0] + (w - mb.pre[i0])], a1 = A.fd_adj[mb.lo[i1] + (w + N - mb.pre[i1])];
    f(a0);
    f(a1);
  }
  if (w < T) {
    int i = seg_of(mb.pre, N, w);
    f(A.fd_adj[mb.lo[i] + (w - mb.pre[i])]);
  }
}

// Dense counters of the partition being peeled, indexed by the local index
// of a vertex: in the team's shared memory (a cluster spreads them over its
// blocks, index loc in block loc mod size at loc / size), or in global memory
// when the partition is larger than that.
struct FDCounters {
  uint32_t *dense;   // this block's shared array (P_DENSE entries)
  uint32_t *global;  // the partition's global array, or null
  uint32_t lg;       // log2 of the team's blocks
  template <bool CL>
  __device__ __forceinline__ uint32_t *at(uint32_t loc) const {
    if (global) return global + loc;
    if (!CL) return dense + loc;
    return cooperative_groups::this_cluster().map_shared_rank(dense, loc & ((1u << lg) - 1u)) + (loc >> lg);
  }
};

// per-group scratch of the fine phase's group tier: slices and scan words
__host__ __device__ constexpr size_t fd_group_bytes() { return align16(sizeof(FMid<FGT>)) + 32; }
static_assert((FT / FGT) * FG_CAP * 8 <= P_DENSE * 4, "group hashes fit the dense counters' memory");
static_assert(2 * FB_MAXW * 8 <= P_DENSE * 4, "a block hash fits the dense counters' memory");
static_assert((FT / FGT) <= 15, "named barriers 1..groups");

// Count the alive targets of x's wedges in G_p into a shared hash of 64-bit
// slots ((id + 1) << 32 | count, zero = empty) held by group g, then drain it
// (decrements C(c, 2), crossings into cand) leaving it zeroed; returns updates
template <class Grp, int N>
__device__ __forceinline__ uint64_t fd_hash_vertex(const FDArgs &A, const Grp &g, FMid<N> &mb, uint32_t p, uint32_t x,
                                                   uint32_t W, unsigned long long *slot, unsigned *nc, uint32_t *cand,
                                                   ull hi) {
  const uint32_t xo = A.p_off[x], xd = A.seg_n[x];
  const uint32_t capg = pow2_at_least(max(2u * W, 64u));
  WHash h{slot, capg - 1};
  for (uint32_t b0 = 0; b0 < xd; b0 += N) {
    const uint32_t Tw = fd_load(A, p, xo, xd, b0, g, mb);
    fd_walk(A, g, mb, Tw, [&](uint32_t xp) {
      if (ldt(&A.state[xp]) == ST_ALIVE) h.inc(xp);
    });
    g.sync();
  }
  uint64_t nup = 0;
  for (uint32_t i = g.rank(); i < capg; i += N) {
    const unsigned long long v = slot[i];
    if (!v) continue;
    slot[i] = 0;
    const uint32_t c = (uint32_t)v;
    if (c >= 2) {
      const uint32_t xp = (uint32_t)(v >> 32) - 1;
      const ull dec = choose2(c);
      fd_crossing(nc, cand, hi, xp, atomicAdd(&A.sup[xp], (ull)(0ull - dec)), dec);
      nup++;
    }
  }
  g.sync();
  return nup;
}

// Fine phase of the partitions handed out by A.queue / A.order (Sec. 3.1.2,
// 3.2): bottom-up peeling of G_p from init, one partition at a time per team.
// Each step: the selection (fd_select), then the updates of the peeled
// vertices - a warp per vertex with few wedges in G_p (shared hash); when a
// step has many heavier ones, 128-thread groups with shared hashes, then (in a
// cluster) single blocks with larger hashes, take those that fit; the whole
// team takes the rest (dense counters over the partition).  A step after
// which nothing remains in the partition does no updates: they could reach no
// remaining vertex.
template <class Team>
__device__ void tip_fd_run(const FDArgs &A, const Team &T, uint32_t cap, uint8_t *sm, size_t warp_bytes,
                           FMid<FT> &bmb, uint32_t *dense, uint8_t *gsm, const BlockGrp<FT> &bg) {
  constexpr bool CL = Team::kCluster;
  FDShared *S = T.S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t *wkey = (uint32_t *)(sm + warp * warp_bytes), *wval = wkey + PW_CAP;
  FMid<32> &wmb = *(FMid<32> *)(sm + warp * warp_bytes + PW_CAP * 8);
  for (uint32_t i = lane; i < PW_CAP; i += 32) wkey[i] = EMPTY_KEY, wval[i] = 0;
  for (uint32_t i = threadIdx.x; i < P_DENSE; i += FT) dense[i] = 0;
  const uint32_t nthr = T.nthr(), csize = nthr / FT;
  uint32_t lg = 0;
  while ((1u << lg) < csize) lg++;
  const uint32_t rank = T.tid() / FT;
  T.sync();
  WarpGrp wg;
  ull my_wedges = 0, my_updates = 0, my_steps = 0;
  for (;;) {
    if (T.leader()) {
      unsigned q = atomicAdd(A.queue, 1u);
      S->p = q < A.nparts ? A.order[q] : 0xffffffffu;
    }
    T.sync();
    const uint32_t p = *(volatile uint32_t *)&S->p;
    T.sync();  // every block has read p before it can change, or before the team exits
    if (p == 0xffffffffu) break;
    const uint32_t base = A.ps[p], np = A.ps[p + 1] - base;
    uint32_t *lf = A.buf_f + base, *lbig = A.buf_big + base;
    FDLists L{{A.buf_a + base, A.buf_b + base}, {A.buf_c + base, A.buf_d + base}, lf};
    const FDCounters cnt{dense, np <= P_DENSE * csize ? nullptr : A.gcnt + base, lg};
    for (uint32_t j = T.tid(); j < np; j += nthr) L.a[0][j] = A.xs[base + j];
    if (T.leader()) {
      S->na = np;
      S->wn = 0;
      S->ws = 0;
      S->nc = 0;
      S->pa = 0;
      S->pc = 0;
      S->level = 0;
    }
    long long t_part = clock64();
    ull p_steps = 0, cyc[3] = {0, 0, 0}, rescans = 0, nbigs = 0, nblkv = 0, nteamv = 0;
    T.sync();
    for (;;) {
      if (*(volatile uint32_t *)&S->na + *(volatile uint32_t *)&S->nc == 0) break;
      p_steps++;
      long long t0 = clock64();
      rescans += *(volatile uint32_t *)&S->nc == 0;
      // every vertex at the running minimum is peeled with tip number = level
      const uint32_t nf = fd_select(T, L, A.sup, A.theta, A.state, ST_PEELED, ST_PEELED, cap);
      long long t1 = clock64();
      cyc[0] += t1 - t0;
      my_steps++;
      // (uniform: crossings can only raise nc while something remains)
      if (*(volatile uint32_t *)&S->na + *(volatile uint32_t *)&S->nc == 0) break;
      uint32_t *cand = L.c[*(volatile uint32_t *)&S->pc];
      const ull hi = *(volatile ull *)&S->hi;
      // warp-per-vertex updates for vertices with few wedges in G_p (S->nt:
      // next vertex, S->ncq: heavy vertices, both reset by the selection).
      // When the step peels few vertices most warps would idle, so a vertex
      // with more than WARP_FEW_W wedges goes to the team-wide path instead
      const uint32_t big_w = nf <= FEW_VERTICES ? WARP_FEW_W : PW_MAXW;
      for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(&S->nt, 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= nf) break;
        uint32_t x = ldt(&lf[k]);
        uint32_t xo = A.p_off[x], xd = A.seg_n[x];
        uint32_t W = A.w_fd[x];
        if (W < 2) continue;
        if (W > big_w) {
          if (lane == 0) lbig[atomicAdd(&S->ncq, 1u)] = x;
          continue;
        }
        my_wedges += lane == 0 ? W : 0;
        uint32_t capw = pow2_at_least(max(2u * W, 32u));
        SmemHash h{wkey, wval, capw - 1};
        for (uint32_t b0 = 0; b0 < xd; b0 += 32) {
          uint32_t Tw = fd_load(A, p, xo, xd, b0, wg, wmb);
          fd_walk(A, wg, wmb, Tw, [&](uint32_t xp) {
            if (ldt(&A.state[xp]) == ST_ALIVE) h.inc(xp);
          });
          __syncwarp();
        }
        for (uint32_t i = lane; i < capw; i += 32) {
          uint32_t kk = wkey[i];
          if (kk != EMPTY_KEY) {
            uint32_t c = wval[i];
            if (c >= 2) {
              ull dec = choose2(c);
              fd_crossing(&S->nc, cand, hi, kk, atomicAdd(&A.sup[kk], (ull)(0ull - dec)), dec);
              my_updates++;
            }
            wkey[i] = EMPTY_KEY;
            wval[i] = 0;
          }
        }
        __syncwarp();
      }
      T.sync();
      long long t2 = clock64();
      cyc[1] += t2 - t1;
      // heavy vertices: the whole team, dense counters over the partition;
      // block r of the team walks neighbour chunks r, r + size, ...
      const uint32_t nbig = *(volatile uint32_t *)&S->ncq;
      nbigs += nbig;
      uint32_t nteam = nbig;
      const uint32_t *lteam = lbig;
      if (nbig >= FG_MIN_BIG) {
        // many heavy vertices: 128-thread groups (four per block, named
        // barriers 1-4) take one each with a 2K-slot hash in the dense
        // counters' memory (zero between uses); heavier ones are listed
        const int sub = threadIdx.x / FGT;
        uint8_t *gb = gsm + sub * fd_group_bytes();
        FMid<FGT> &gmb = *(FMid<FGT> *)gb;
        uint32_t *gws = (uint32_t *)(gb + align16(sizeof(FMid<FGT>)));
        SubGrp<FGT> sg{sub * FGT, 1 + sub, gws, nullptr};
        unsigned long long *gslot = (unsigned long long *)dense + (size_t)sub * FG_CAP;
        uint32_t *lhuge = A.buf_huge + base;
        for (;;) {
          if (sg.rank() == 0) gws[FGT / 32 + 1] = atomicAdd(&S->ng, 1u);
          sg.sync();
          const uint32_t k = gws[FGT / 32 + 1];
          sg.sync();
          if (k >= nbig) break;
          const uint32_t x = ldt(&lbig[k]);
          const uint32_t W = A.w_fd[x];
          if (W > FG_MAXW) {
            if (sg.rank() == 0) lhuge[atomicAdd(&S->nh, 1u)] = x;
            continue;
          }
          if (sg.rank() == 0) my_wedges += W;
          my_updates += fd_hash_vertex(A, sg, gmb, p, x, W, gslot, &S->nc, cand, hi);
        }
        T.sync();
        nteam = *(volatile uint32_t *)&S->nh;
        lteam = lhuge;
        if (CL && nteam >= 2) {
          // a cluster: its blocks take the vertices left one each (8K-slot
          // hash over the block's dense counters) with block barriers only;
          // the heaviest go on to the whole team, listed in lbig (read in
          // full by now)
          __shared__ uint32_t blk_k;
          for (;;) {
            if (threadIdx.x == 0) blk_k = atomicAdd(&S->nbq, 1u);
            __syncthreads();
            const uint32_t k = blk_k;
            __syncthreads();
            if (k >= nteam) break;
            const uint32_t x = ldt(&lhuge[k]);
            const uint32_t W = A.w_fd[x];
            if (W > FB_MAXW) {
              if (threadIdx.x == 0) lbig[atomicAdd(&S->nbh, 1u)] = x;
              continue;
            }
            if (threadIdx.x == 0) my_wedges += W;
            my_updates += fd_hash_vertex(A, bg, bmb, p, x, W, (unsigned long long *)dense, &S->nc, cand, hi);
          }
          T.sync();
          const uint32_t nleft = *(volatile uint32_t *)&S->nbh;
          nblkv += nteam - nleft;
          nteam = nleft;
          lteam = lbig;
        }
      }
      nteamv += nteam;
      for (uint32_t bi = 0; bi < nteam; bi++) {
        const uint32_t x = ldt(&lteam[bi]);
        const uint32_t xo = A.p_off[x], xd = A.seg_n[x];
        if (T.leader()) my_wedges += A.w_fd[x];
        if (xd <= csize * FT) {
          // one chunk of slices per block at most: a thread keeps the
          // alive targets of its (at most HW_KEEP) wedges from the counting
          // pass and takes their counts without a second walk
          uint32_t keep[HW_KEEP], tgt[HW_KEEP];
          const uint32_t b0 = rank * FT;
          const uint32_t Tw = fd_load(A, p, xo, xd, min(b0, xd), bg, bmb);  // (empty past xd)
          const bool cached = Tw <= HW_KEEP * FT;  // uniform in the block
          if (cached) {
#pragma unroll
            for (uint32_t r = 0; r < HW_KEEP; r++) {  // loads of all kept wedges first
              const uint32_t w = threadIdx.x + r * FT;
              tgt[r] = EMPTY_KEY;
              if (w < Tw) {
                int i = seg_of(bmb.pre, FT, w);
                tgt[r] = A.fd_adj[bmb.lo[i] + (w - bmb.pre[i])];
              }
            }
#pragma unroll
            for (uint32_t r = 0; r < HW_KEEP; r++) {
              keep[r] = EMPTY_KEY;
              if (tgt[r] != EMPTY_KEY && ldt(&A.state[tgt[r]]) == ST_ALIVE) {
                keep[r] = A.loc[tgt[r]];
                atomicAdd(cnt.at<CL>(keep[r]), 1u);
              }
            }
          } else {
            fd_walk(A, bg, bmb, Tw, [&](uint32_t xp) {
              if (ldt(&A.state[xp]) == ST_ALIVE) atomicAdd(cnt.at<CL>(A.loc[xp]), 1u);
            });
          }
          T.sync();
          if (cached) {
#pragma unroll
            for (uint32_t r = 0; r < HW_KEEP; r++) {
              const uint32_t l = keep[r];
              if (l == EMPTY_KEY) continue;
              uint32_t c = atomicExch(cnt.at<CL>(l), 0u);  // the first visitor takes the count
              if (c >= 2) {
                const uint32_t xp = tgt[r];
                ull dec = choose2(c);
                fd_crossing(&S->nc, cand, hi, xp, atomicAdd(&A.sup[xp], (ull)(0ull - dec)), dec);
                my_updates++;
              }
            }
          } else {
            fd_walk(A, bg, bmb, Tw, [&](uint32_t xp) {
              if (ldt(&A.state[xp]) != ST_ALIVE) return;
              uint32_t c = atomicExch(cnt.at<CL>(A.loc[xp]), 0u);
              if (c >= 2) {
                ull dec = choose2(c);
                fd_crossing(&S->nc, cand, hi, xp, atomicAdd(&A.sup[xp], (ull)(0ull - dec)), dec);
                my_updates++;
              }
            });
          }
          __syncthreads();  // the chunk arrays are reused by the next vertex
          T.sync();
          continue;
        }
        for (uint32_t b0 = rank * FT; b0 < xd; b0 += csize * FT) {
          uint32_t Tw = fd_load(A, p, xo, xd, b0, bg, bmb);
          fd_walk(A, bg, bmb, Tw, [&](uint32_t xp) {
            if (ldt(&A.state[xp]) == ST_ALIVE) atomicAdd(cnt.at<CL>(A.loc[xp]), 1u);
          });
          __syncthreads();
        }
        T.sync();
        for (uint32_t b0 = rank * FT; b0 < xd; b0 += csize * FT) {
          uint32_t Tw = fd_load(A, p, xo, xd, b0, bg, bmb);
          fd_walk(A, bg, bmb, Tw, [&](uint32_t xp) {
            if (ldt(&A.state[xp]) != ST_ALIVE) return;
            uint32_t c = atomicExch(cnt.at<CL>(A.loc[xp]), 0u);  // the first visitor takes the count
            if (c >= 2) {
              ull dec = choose2(c);
              fd_crossing(&S->nc, cand, hi, xp, atomicAdd(&A.sup[xp], (ull)(0ull - dec)), dec);
              my_updates++;
            }
          });
          __syncthreads();
        }
        T.sync();
      }
      T.sync();
      cyc[2] += clock64() - t2;
    }
    if (T.leader() && A.pstat) {
      // steps, cycles; then select, warp path, heavy-vertex path; rescans;
      // heavy vertices, those taken by single blocks, by the whole team
      ull *ps = A.pstat + (size_t)TFD_PSTAT * p;
      ps[0] = p_steps;
      ps[1] = (ull)(clock64() - t_part);
      for (int k = 0; k < 3; k++) ps[2 + k] = cyc[k];
      ps[5] = rescans;
      ps[6] = nbigs;
      ps[7] = nblkv;
      ps[8] = nteamv;
    }
  }
  my_wedges = bg.sum64(my_wedges);
  my_updates = bg.sum64(my_updates);
  if (threadIdx.x == 0) {
    if (A.wedges) atomicAdd(A.wedges, my_wedges);
    if (A.updates) atomicAdd(A.updates, my_updates);
  }
  if (T.leader() && A.steps) atomicAdd(A.steps, my_steps);
}

// one block per partition
__global__ void __launch_bounds__(FT, 1) k_fd_tip(FDArgs A, size_t warp_bytes, size_t dense_off, uint32_t cap) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ FDShared S;
  __shared__ TeamMin tmin;
  __shared__ uint32_t ws[FT / 32 + 2];
  __shared__ ull ws64[FT / 32];
  BlockGrp<FT> bg{ws, ws64};
  BlockTeam T{&S, S.hist, &tmin};
  tip_fd_run(A, T, cap, sm, warp_bytes, *(FMid<FT> *)(sm + FW * warp_bytes), (uint32_t *)(sm + dense_off),
             sm + dense_off + P_DENSE * 4, bg);
}

// one thread-block cluster per heavy partition (step state in the first
// block's shared memory, dense counters spread over the blocks)
__global__ void __launch_bounds__(FT, 1) k_fd_tip_cluster(FDArgs A, size_t warp_bytes, size_t dense_off, uint32_t cap) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ FDShared S;
  __shared__ TeamMin tmin;
  __shared__ uint32_t lhist[65];
  __shared__ uint32_t ws[FT / 32 + 2];
  __shared__ ull ws64[FT / 32];
  BlockGrp<FT> bg{ws, ws64};
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  ClusterTeam T{cl.map_shared_rank(&S, 0), lhist, &tmin, cl.block_rank(), cl.num_blocks()};
  tip_fd_run(A, T, cap, sm, warp_bytes, *(FMid<FT> *)(sm + FW * warp_bytes), (uint32_t *)(sm + dense_off),
             sm + dense_off + P_DENSE * 4, bg);
}

size_t fd_warp_bytes() { return align16(PW_CAP * 8 + sizeof(FMid<32>)); }
size_t fd_dense_off() { return align16(FW * fd_warp_bytes() + sizeof(FMid<FT>)); }
size_t fd_smem() { return fd_dense_off() + P_DENSE * 4 + (FT / FGT) * fd_group_bytes(); }

// FD adjacency keys: (y, part(x)) for every Y-side entry
__global__ void k_fd_keys(const uint32_t *o_off, const uint32_t *o_adj0, uint32_t ny, const uint32_t *part, int bp,
                          uint64_t *key, uint32_t *val) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t y = gw; y < ny; y += nw)
    for (uint32_t k = o_off[y] + lane; k < o_off[y + 1]; k += 32) {
      uint32_t x = o_adj0[k];
      key[k] = ((uint64_t)y << bp) | part[x];
      val[k] = x;
    }
}

__global__ void k_fd_part_of(const uint32_t *fd_adj, uint32_t m, const uint32_t *part, uint32_t *fd_part) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x)
    fd_part[k] = part[fd_adj[k]];
}

// work of partition p: wedges of G_p with both endpoints in X_p (Sec. 3.2),
// sum over groups (y, p) of size*(size-1)
__global__ void k_fd_work(const uint32_t *o_off, uint32_t ny, const uint32_t *fd_part, ull *work) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t y = gw; y < ny; y += nw) {
    uint32_t b = o_off[y], e = o_off[y + 1];
    for (uint32_t k = b + lane; k < e; k += 32) {
      if (k == b || fd_part[k] != fd_part[k - 1]) {  // group head
        uint32_t p = fd_part[k];
        uint32_t len = lower_bound_u32(fd_part + k, e - k, p + 1);
        if (len >= 2) atomicAdd(&work[p], (ull)len * (len - 1));
      }
    }
  }
}

__global__ void k_part_hist(const uint32_t *part, uint32_t nx, uint32_t *cnt) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < nx; x += (size_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[part[x]], 1u);
}

__global__ void k_part_keys(const uint32_t *part, uint32_t nx, uint64_t *key, uint32_t *val) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < nx; x += (size_t)gridDim.x * blockDim.x) {
    key[x] = part[x];
    val[x] = (uint32_t)x;
  }
}

__global__ void k_loc(const uint32_t *xs, uint32_t nx, const uint32_t *part, const uint32_t *ps, uint32_t *loc, uint8_t *state) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < nx; j += (size_t)gridDim.x * blockDim.x) {
    uint32_t x = xs[j];
    loc[x] = (uint32_t)(j - ps[part[x]]);
    state[x] = ST_ALIVE;
  }
}

}  // namespace

// --------------------------------------------------------------- driver
void tip_decompose(Arena &a, Graph &G, int side, const TipParams &prm, uint64_t *theta_out, pbng_stats *st) {
  const int T = 256;
  const int sms = num_sms();
  const unsigned cap = 16 * sms;
  uint32_t nx = side == 0 ? G.nu : G.nv, ny = side == 0 ? G.nv : G.nu;
  if (nx == 0) return;
  if (G.m == 0) {
    if (theta_out) CK(cudaMemsetAsync(theta_out, 0, (size_t)nx * 8, a.st));
    return;
  }
  const uint32_t *p_off = side == 0 ? G.u_off : G.v_off, *p_adj = side == 0 ? G.u_adj : G.v_adj;
  const uint32_t *o_off = side == 0 ? G.v_off : G.u_off, *o_adj0 = side == 0 ? G.v_adj : G.u_adj;
  cudaEvent_t ev[6];
  for (auto &e : ev) CK(cudaEventCreate(&e));
  CK(cudaEventRecord(ev[0], a.st));

  // ---- initial supports by Alg. 1 (counts of the peeled side only)
  // [0..2] initial count (wedges, expansions, updates), [3..5] re-counts,
  // [6] fd wedges, [7] fd steps, [8] coarse updates, [9] fine updates
  ull *dwedge = a.zeros<ull>(16);
  uint8_t *isU = label_sides(a, G);
  ull *cnt_lab = a.zeros<ull>(G.n);
  CountOut co;
  co.cnt_lab = (uint64_t *)cnt_lab;
  co.lab_isU = isU;
  co.want_side = side;
  co.wedges = (uint64_t *)dwedge;
  co.scratch = prm.count_scratch;
  count_butterflies(a, G, co);
  uint32_t *x2lab = a.alloc<uint32_t>(nx);
  k_x2lab<<<grid_for(nx, T, cap), T, 0, a.st>>>(G.g2lab, side == 0 ? 0 : G.nu, nx, x2lab);
  CK_LAUNCH();
  ull *sup = a.alloc<ull>(nx), *init = a.alloc<ull>(nx);
  uint32_t *alist = a.alloc<uint32_t>(nx), *alist2 = a.alloc<uint32_t>(nx);
  k_init_side<<<grid_for(nx, T, cap), T, 0, a.st>>>(nx, x2lab, cnt_lab, sup, alist);
  CK_LAUNCH();
  CK(cudaEventRecord(ev[1], a.st));

  // ---- coarse phase state
  uint8_t *state = a.zeros<uint8_t>(nx);
  uint8_t *lab_alive = nullptr;
  if (prm.recount) {
    lab_alive = a.alloc<uint8_t>(G.n);
    CK(cudaMemsetAsync(lab_alive, 1, G.n, a.st));
  }
  uint32_t *part = a.alloc<uint32_t>(nx);
  uint32_t *o_adj = a.alloc<uint32_t>(G.m), *o_len = a.alloc<uint32_t>(ny + 1);
  CK(cudaMemcpyAsync(o_adj, o_adj0, (size_t)G.m * 4, cudaMemcpyDeviceToDevice, a.st));
  k_degrees<<<grid_for(ny, T, cap), T, 0, a.st>>>(o_off, ny, o_len);
  CK_LAUNCH();
  uint32_t *ytouch = a.zeros<uint32_t>(ny + 1), *touched = a.alloc<uint32_t>(ny + 1), *dead = a.zeros<uint32_t>(ny + 1);
  uint32_t *front = a.alloc<uint32_t>(nx), *front2 = a.alloc<uint32_t>(nx);
  uint64_t *plists = a.alloc<uint64_t>((size_t)2 * nx);
  // target buckets and their offsets in every Y list
  // automatic: 2^15 ids (one 16-bit dense pass per bucket), at least 2^14
  uint32_t bshift = prm.bucket_shift ? std::max(BK_SHIFT_MIN, prm.bucket_shift) : BK_SHIFT_MIN + 1;
  while (bshift < 31 && (((uint64_t)nx + (1ull << bshift) - 1) >> bshift > NB_MAX ||
                         (uint64_t)ny * ((((uint64_t)nx + (1ull << bshift) - 1) >> bshift) + 1) * 4 > BOFF_BUDGET))
    bshift++;
  const uint32_t nb = (uint32_t)(((uint64_t)nx + (1ull << bshift) - 1) >> bshift);
  uint32_t *boff = nullptr;
  if (nb > 1) {
    boff = a.alloc<uint32_t>((size_t)ny * (nb + 1));
    k_boff_build<<<grid_for((size_t)ny * 32, T, 8 * cap), T, 0, a.st>>>(o_off, o_adj, ny, boff, nb, bshift);
    CK_LAUNCH();
  }
  // block-class items: at most one per active vertex plus one per item_w of
  // its wedges; the wedges of all X vertices together bound a round's
  uint64_t item_w = prm.item_w ? prm.item_w : ITEM_W, wtot = 0;
  {
    ull *d = a.zeros<ull>(1);
    k_sum_sq<<<grid_for(ny, T, cap), T, 0, a.st>>>(o_off, ny, d);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(&wtot, d, 8, cudaMemcpyDeviceToHost, a.st));
    CK(cudaStreamSynchronize(a.st));
    a.free(d);
  }
  item_w = std::max<uint64_t>(item_w, wtot / (4ull * nx) + 1);
  const uint64_t bcap = (uint64_t)nx + wtot / item_w + 1;
  uint64_t *blist = a.alloc<uint64_t>(bcap);
  // small device counters: [0] frontier size, [1] next size, [2] touched, [3..6] class counts, [7] alist size
  unsigned *dc = a.zeros<unsigned>(16);
  ull *sumw = a.zeros<ull>(4);
  // per-round trace (env PBNG_TRACE=<file>): one line per coarse round
  struct Trace {
    FILE *f = nullptr;
    cudaEvent_t ev[7] = {};
    ~Trace() {
      if (f) fclose(f);
      for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    }
  } tr;
  if (const char *tp = getenv("PBNG_TRACE")) {
    tr.f = fopen(tp, "a");
    if (tr.f)
      for (auto &e : tr.ev) CK(cudaEventCreate(&e));
  }
  FILE *trace = tr.f;
  cudaEvent_t *tev = tr.ev;
  uint64_t exp_cd = 0, front_cd = 0;
  RangeState *rs = a.zeros<RangeState>(1);
  ull *wl = a.alloc<ull>(nx);

  PeelArgs PA{};
  PA.p_off = p_off;
  PA.p_adj = p_adj;
  PA.o_off = o_off;
  PA.o_adj = o_adj;
  PA.o_len = o_len;
  PA.boff = boff;
  PA.nb = nb;
  PA.bshift = bshift;
  PA.sup = sup;
  PA.updates = dwedge + 8;
  PA.nx = nx;
  PA.bstat = trace && PBNG_PEEL_STATS ? a.zeros<ull>(BSTAT) : nullptr;

  static bool attr = false;
  size_t wsm = (PWT / 32) * align16(QW_CAP * 8 + sizeof(PMid<32>));
  if (!attr) {
    CK(cudaFuncSetAttribute(k_peel_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm));
    CK(cudaFuncSetAttribute(k_peel_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)peel_block_smem()));
    CK(cudaFuncSetAttribute(k_peel_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)peel_group_smem()));
    CK(cudaFuncSetAttribute(k_fd_tip, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fd_smem()));
    CK(cudaFuncSetAttribute(k_fd_tip_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fd_smem()));
    attr = true;
  }

  // graph-captured coarse rounds: the rounds of one range run as a CUDA graph
  // with a conditional WHILE node (two rounds per body, ping-pong frontier
  // buffers); every size is read from device memory, so there is no host
  // round trip per round.  The re-count branch needs host-side bucketing of
  // its starts, so this mode peels every round.
  struct GraphHold {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    ~GraphHold() {
      if (e) cudaGraphExecDestroy(e);
      if (g) cudaGraphDestroy(g);
    }
  } gh;
  // hc: host copies of the class sizes (grids sized to them, empty classes
  // skipped), or null for the fixed grids of graph-captured rounds
  // (ev: optional events recorded after the warp and the group class)
  auto launch_classes = [&](cudaStream_t st, unsigned *cnt, const unsigned *hc, cudaEvent_t *ev) {
    if (!hc || hc[PC_WARP]) {
      unsigned gw = hc ? grid_for((size_t)hc[PC_WARP] * 32, PWT, 6 * sms) : 6 * sms;
      k_peel_warp<<<gw, PWT, wsm, st>>>(PA, plists + (size_t)PC_WARP * nx, cnt + PC_WARP);
      CK_LAUNCH();
    }
    if (ev) CK(cudaEventRecord(ev[0], st));
    if (!hc || hc[PC_GROUP]) {
      unsigned gg = hc ? std::min<unsigned>((hc[PC_GROUP] + 1) / 2, 3 * sms) : 3 * sms;
      k_peel_group<<<gg, 2 * QGT, peel_group_smem(), st>>>(PA, plists + (size_t)PC_GROUP * nx, cnt + PC_GROUP);
      CK_LAUNCH();
    }
    if (ev) CK(cudaEventRecord(ev[1], st));
    if (!hc || hc[PC_BLOCK]) {
      unsigned gb = hc ? std::min<unsigned>(hc[PC_BLOCK], PB_PER_SM * sms) : PB_PER_SM * sms;
      k_peel_block<<<gb, PBT, peel_block_smem(), st>>>(PA, blist, cnt + PC_BLOCK);
      CK_LAUNCH();
    }
  };
  auto prep_args = [&](const uint32_t *F, uint32_t nf, uint32_t pi, ull *sum_w, unsigned *counts, unsigned *touched_n) {
    PrepArgs R{};
    R.frontier = F;
    R.nf = nf;
    R.p_off = p_off;
    R.p_adj = p_adj;
    R.o_len = o_len;
    R.part = part;
    R.pi = pi;
    R.state = state;
    R.sum_w = sum_w;
    R.lists = plists;
    R.blist = blist;
    R.counts = counts;
    R.nx = nx;
    R.nb = nb;
    R.item_w = item_w;
    R.warp_max_w = std::min(prm.warp_max_w ? prm.warp_max_w : QW_MAXW, QW_MAXW);
    R.group_max_w = std::min(prm.group_max_w ? prm.group_max_w : QG_MAXW, QG_MAXW);
    R.lab_alive = lab_alive;
    R.x2lab = x2lab;
    R.compact = prm.compact;
    R.dead = dead;
    R.ytouch = ytouch;
    R.touched = touched;
    R.touched_n = touched_n;
    return R;
  };
  bool use_graph = prm.graph_rounds != 0;
  RoundDev *Rd = use_graph ? a.zeros<RoundDev>(1) : nullptr;
  auto build_round_graph = [&]() {
    CK(cudaGraphCreate(&gh.g, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, gh.g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, gh.g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // capture on a private stream (the caller's may be the legacy default stream)
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const uint64_t launches0 = g_launches;  // captured launches are counted per execution
    for (int half = 0; half < 2; half++) {
      uint32_t *F = half == 0 ? front : front2, *Nx = half == 0 ? front2 : front;
      k_round_reset<<<1, 1, 0, cs>>>(Rd);
      PrepArgs R = prep_args(F, 0, 0, Rd->sum_w, Rd->counts, &Rd->touched_n);
      R.nf_dev = &Rd->nf;
      R.pi_dev = &Rd->pi;
      k_prep<<<16 * sms, T, 0, cs>>>(R);
      launch_classes(cs, Rd->counts, nullptr, nullptr);
      if (prm.compact)
        k_compact<<<4 * sms, T, 0, cs>>>(touched, &Rd->touched_n, o_off, o_adj, o_len, ytouch, dead, state, boff, nb, bshift);
      k_scan_frontier<<<cap, T, 0, cs>>>(alist, 0, state, sup, init, &rs->theta_hi, 0, Nx, &Rd->nn, &Rd->na);
      k_round_end<<<1, 1, 0, cs>>>(Rd, h, half == 1);
    }
    g_launches = launches0;
    cudaGraph_t captured = nullptr;
    cudaError_t le = cudaGetLastError(), ce = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    CK(le);
    CK(ce);
    CK(cudaGraphInstantiate(&gh.e, gh.g, 0));
  };

  // learned bounds: features of the initial supports -> MLP -> explicit bounds
  std::vector<uint64_t> learned;
  const uint64_t *bounds = prm.bounds;
  uint32_t n_bounds = prm.n_bounds;
  bool explicit_bounds = prm.bounds_mode == PBNG_BOUNDS_EXPLICIT;
  if (prm.bounds_mode == PBNG_BOUNDS_LEARNED) {
    float *feat = a.alloc<float>(128);
    uint64_t K = bound_features(a, (const uint64_t *)sup, p_off, nx, feat);
    learned = propose_bounds(a, prm.mlp_params, prm.mlp_hidden, prm.mlp_out, feat, K);
    a.free(feat);
    bounds = learned.data();
    n_bounds = (uint32_t)learned.size();
    explicit_bounds = true;
  }
  uint32_t na = nx;
  uint32_t pi = 0;
  double scale = 1.0;
  uint64_t prev_init_est = 0, cur_final = 0;
  uint64_t rounds = 0, recounts = 0, wedges_cd = 0;
  uint64_t wbound = G.wedge_bound;
  uint32_t P = prm.P;
  while (na > 0) {
    // ---- remaining list (drop peeled vertices)
    auto rwall0 = std::chrono::steady_clock::now();
    if (pi > 0) {
      CK(cudaMemsetAsync(dc + 7, 0, 4, a.st));
      k_compact_list<<<grid_for(na, T, cap), T, 0, a.st>>>(alist, na, state, alist2, dc + 7);
      CK_LAUNCH();
      na = fetch(a, dc + 7);
      if (use_graph)  // the captured rounds read the remaining list at a fixed address
        CK(cudaMemcpyAsync(alist, alist2, (size_t)na * 4, cudaMemcpyDeviceToDevice, a.st));
      else
        std::swap(alist, alist2);
      if (na == 0) break;
    }
    // ---- range [theta(i), theta(i+1)) (Alg. 4 l.8, Sec. 3.1.3)
    bool last = pi + 1 >= P;
    CK(cudaMemsetAsync(rs, 0, sizeof(RangeState), a.st));
    set_u64(a, (uint64_t *)&rs->kmin, ~0ull);
    // the work proxy is only needed when find_range will run, or when the
    // estimator vets a learned bound
    const bool vetted = prm.bounds_mode == PBNG_BOUNDS_LEARNED && !last && prm.learned_vet > 0;
    bool given = last || (explicit_bounds && pi < n_bounds);
    ull hk[3];
    if (given && !vetted) {
      k_keyrange<<<grid_for(na, T, cap), T, 0, a.st>>>(alist, na, sup, rs);
      CK_LAUNCH();
      CK(cudaMemcpyAsync(hk, &rs->kmin, sizeof(hk), cudaMemcpyDeviceToHost, a.st));
      CK(cudaStreamSynchronize(a.st));
      given = last || bounds[pi] > hk[0];
    }
    if (!given || vetted) {
      CK(cudaMemsetAsync(rs, 0, sizeof(RangeState), a.st));
      set_u64(a, (uint64_t *)&rs->kmin, ~0ull);
      k_weights<<<grid_for((size_t)na * 32, T, cap), T, 0, a.st>>>(alist, na, p_off, p_adj, o_len, sup, wl, rs);
      CK_LAUNCH();
      CK(cudaMemcpyAsync(hk, &rs->kmin, sizeof(hk), cudaMemcpyDeviceToHost, a.st));
      CK(cudaStreamSynchronize(a.st));
    }
    ull kmin = hk[0], kmax = hk[1], wsum = hk[2];
    // adaptive target (Sec. 3.1.3): remaining work over remaining partitions,
    // scaled by how far the previous partition overshot its estimate
    if (pi > 0 && cur_final > 0) {
      scale = (double)prev_init_est / (double)cur_final;
      if (scale > 1.0) scale = 1.0;
      if (scale <= 0.0) scale = 1.0;
    }
    ull thi;
    bool use_est = true;
    if (last) {
      thi = ~0ull;
      use_est = false;
    } else if (explicit_bounds && pi < n_bounds && bounds[pi] > kmin) {
      thi = bounds[pi];
      use_est = false;
    }
    uint64_t init_est = 0;
    if (!use_est && vetted && wsum > 0) {
      // the plain estimator vets a learned bound: its range may hold at
      // most learned_vet times the estimator's target work, else the
      // estimator's own bound is used
      double t = (double)wsum * scale / (double)(P - pi);
      ull *d = a.zeros<ull>(1), wb = 0;
      k_work_below<<<grid_for(na, T, cap), T, 0, a.st>>>(alist, na, sup, wl, thi, d);
      CK_LAUNCH();
      CK(cudaMemcpyAsync(&wb, d, 8, cudaMemcpyDeviceToHost, a.st));
      CK(cudaStreamSynchronize(a.st));
      a.free(d);
      if ((double)wb > prm.learned_vet * std::max(t, 1.0)) use_est = true;
      else init_est = wb;
    }
    if (use_est) {
      if (wsum == 0 || kmin == kmax) {
        thi = kmin + 1;
        init_est = wsum;
        set_u64(a, (uint64_t *)&rs->theta_hi, thi);
      } else {
        double t = (double)wsum * scale / (double)(P - pi);
        ull tgt = t < 1.0 ? 1 : (t >= (double)wsum ? wsum : (ull)t);
        thi = range_select(a, rs, alist, na, (const uint64_t *)sup, (const uint64_t *)wl, kmin, kmax, tgt, &init_est);
      }
    } else {
      set_u64(a, (uint64_t *)&rs->theta_hi, thi);
    }
    prev_init_est = init_est;
    cur_final = 0;
    if (prm.bounds_used && !last) prm.bounds_used->push_back(thi);
    // ---- snapshot + first active set (Alg. 4 l.6-9)
    if (use_graph) {
      // this range's rounds run entirely on the device; the host reads the
      // totals once the range is done (its work feeds the next target)
      RoundDev hr;
      CK(cudaMemsetAsync(&Rd->nf, 0, 8, a.st));  // nf, nn
      CK(cudaMemsetAsync(&Rd->part_work, 0, 8, a.st));
      CK(cudaMemcpyAsync(&Rd->pi, &pi, 4, cudaMemcpyHostToDevice, a.st));
      CK(cudaMemcpyAsync(&Rd->na, &na, 4, cudaMemcpyHostToDevice, a.st));
      k_scan_frontier<<<grid_for(na, T, cap), T, 0, a.st>>>(alist, na, state, sup, init, &rs->theta_hi, 1, front, &Rd->nf);
      CK_LAUNCH();
      if (!gh.e) build_round_graph();
      ull it0 = 0;
      CK(cudaMemcpyAsync(&it0, &Rd->iters, 8, cudaMemcpyDeviceToHost, a.st));
      g_prof.begin(PROF_PEEL);
      CK(cudaGraphLaunch(gh.e, a.st));
      g_prof.end();
      CK(cudaMemcpyAsync(&hr, Rd, sizeof(RoundDev), cudaMemcpyDeviceToHost, a.st));
      CK(cudaStreamSynchronize(a.st));
      cur_final = hr.part_work;
      g_launches += (hr.iters - it0) * 2 * (7 + (prm.compact ? 1 : 0));
      rounds = hr.rounds;
      wedges_cd = hr.tot_wedges;
      exp_cd = hr.tot_exp;
      front_cd = hr.tot_front;
      pi++;
      continue;
    }
    CK(cudaMemsetAsync(dc, 0, 4, a.st));
    k_scan_frontier<<<grid_for(na, T, cap), T, 0, a.st>>>(alist, na, state, sup, init, &rs->theta_hi, 1, front, dc);
    CK_LAUNCH();
    uint32_t nf = fetch(a, dc);
    if (trace)  // range line: side range |remaining| |first active set| ms to pick the range
      fprintf(trace, "R %d %u %u %u %.4f\n", side, pi, na, nf,
              std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - rwall0).count());
    // ---- peeling rounds (Alg. 4 l.10-13)
    while (nf > 0) {
      rounds++;
      auto wall0 = std::chrono::steady_clock::now();
      if (trace) CK(cudaEventRecord(tev[4], a.st));
      CK(cudaMemsetAsync(dc + 1, 0, 6 * 4, a.st));
      CK(cudaMemsetAsync(sumw, 0, 24, a.st));
      PrepArgs R = prep_args(front, nf, pi, sumw, dc + 3, dc + 2);
      k_prep<<<grid_for((size_t)nf * 32, T, cap), T, 0, a.st>>>(R);
      CK_LAUNCH();
      unsigned hc[6];
      ull hw2[3];
      CK(cudaMemcpyAsync(hc, dc + 1, sizeof(hc), cudaMemcpyDeviceToHost, a.st));
      CK(cudaMemcpyAsync(hw2, sumw, 24, cudaMemcpyDeviceToHost, a.st));
      CK(cudaStreamSynchronize(a.st));
      ull hw = hw2[0];
      cur_final += hw;
      bool do_recount = prm.recount && hw > wbound;
      if (do_recount) {
        // Sec. 5.1: re-count the remaining vertices instead of peeling
        recounts++;
        CK(cudaMemsetAsync(cnt_lab, 0, (size_t)G.n * 8, a.st));
        CountOut rc;
        rc.cnt_lab = (uint64_t *)cnt_lab;
        rc.lab_isU = isU;
        rc.want_side = side;
        rc.lab_alive = lab_alive;
        rc.wedges = (uint64_t *)(dwedge + 3);
        rc.scratch = prm.count_scratch;
        count_butterflies(a, G, rc);
        k_gather_counts<<<grid_for(na, T, cap), T, 0, a.st>>>(alist, na, state, x2lab, cnt_lab, sup);
        CK_LAUNCH();
      } else {
        wedges_cd += hw;
        exp_cd += hw2[1];
        front_cd += nf;
        if (trace) CK(cudaEventRecord(tev[0], a.st));
        g_prof.begin(PROF_PEEL);
        launch_classes(a.st, dc + 3, hc + 2, trace ? tev + 2 : nullptr);
        g_prof.end();
      }
      if (trace) CK(cudaEventRecord(tev[1], a.st));  // (re-count rounds: end of the re-count)
      if (prm.compact) {
        k_compact<<<4 * sms, T, 0, a.st>>>(touched, dc + 2, o_off, o_adj, o_len, ytouch, dead, state, boff, nb, bshift);
        CK_LAUNCH();
      }
      if (trace) CK(cudaEventRecord(tev[5], a.st));
      // next active set (dc[1] was cleared with the class counters)
      k_scan_frontier<<<grid_for(na, T, cap), T, 0, a.st>>>(alist, na, state, sup, init, &rs->theta_hi, 0, front2, dc + 1);
      CK_LAUNCH();
      if (trace) CK(cudaEventRecord(tev[6], a.st));
      uint32_t nf_next = fetch(a, dc + 1);
      if (trace) {
        float ms = 0.f, m1 = 0.f, m2 = 0.f, mp = 0.f, mc = 0.f, mf = 0.f;
        if (!do_recount) {
          CK(cudaEventElapsedTime(&ms, tev[0], tev[1]));
          CK(cudaEventElapsedTime(&m1, tev[0], tev[2]));
          CK(cudaEventElapsedTime(&m2, tev[2], tev[3]));
          CK(cudaEventElapsedTime(&mp, tev[4], tev[0]));
        }
        CK(cudaEventElapsedTime(&mc, tev[1], tev[5]));
        CK(cudaEventElapsedTime(&mf, tev[5], tev[6]));
        double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
        // side range round |active| items(warp group block) wedges maxW recount
        // ms: peel (warp group block) prep+sync compact scan wall
        fprintf(trace, "%d %u %llu %u %u %u %u %llu %llu %d %.4f %.4f %.4f %.4f %.4f %.4f %.4f %.4f\n", side, pi,
                (unsigned long long)rounds, nf, hc[2 + PC_WARP], hc[2 + PC_GROUP], hc[2 + PC_BLOCK], hw, hw2[2],
                (int)do_recount, ms, m1, m2, ms - m1 - m2, mp, mc, mf, wall);
        if (PA.bstat && !do_recount && hc[2 + PC_BLOCK]) {  // block class: "B" side range round, then BS_*
          ull hb[BSTAT];
          CK(cudaMemcpy(hb, PA.bstat, sizeof(hb), cudaMemcpyDeviceToHost));
          CK(cudaMemset(PA.bstat, 0, sizeof(hb)));
          fprintf(trace, "B %d %u %llu", side, pi, (unsigned long long)rounds);
          for (int k = 0; k < BSTAT; k++) fprintf(trace, " %llu", hb[k]);
          fprintf(trace, "\n");
        }
      }
      nf = nf_next;
      std::swap(front, front2);
    }
    pi++;
  }
  uint32_t nparts = pi;
  CK(cudaEventRecord(ev[2], a.st));
  if (prm.coarse_only) {  // the bounds were all that was asked for
    CK(cudaStreamSynchronize(a.st));
    for (auto &e : ev) cudaEventDestroy(e);
    return;
  }

  // ---- fine phase: partitions, induced subgraphs, LPT queue
  uint32_t *pcnt = a.zeros<uint32_t>(nparts + 1), *ps = a.alloc<uint32_t>(nparts + 1);
  k_part_hist<<<grid_for(nx, T, cap), T, 0, a.st>>>(part, nx, pcnt);
  CK_LAUNCH();
  exclusive_scan_u32(a, pcnt, ps, nparts);
  uint32_t *xs = a.alloc<uint32_t>(nx), *loc = a.alloc<uint32_t>(nx);
  {
    uint64_t *key = a.alloc<uint64_t>(nx);
    k_part_keys<<<grid_for(nx, T, cap), T, 0, a.st>>>(part, nx, key, xs);
    CK_LAUNCH();
    sort_pairs(a, key, xs, nx, bits_for(nparts));
    a.free(key);
  }
  k_loc<<<grid_for(nx, T, cap), T, 0, a.st>>>(xs, nx, part, ps, loc, state);
  CK_LAUNCH();
  int bp = bits_for(nparts);
  uint32_t *fd_adj = a.alloc<uint32_t>(G.m), *fd_part = a.alloc<uint32_t>(G.m);
  {
    uint64_t *key = a.alloc<uint64_t>(G.m);
    k_fd_keys<<<grid_for((size_t)ny * 32, T, cap), T, 0, a.st>>>(o_off, o_adj0, ny, part, bp, key, fd_adj);
    CK_LAUNCH();
    sort_pairs(a, key, fd_adj, G.m, bits_for(ny) + bp);
    a.free(key);
  }
  k_fd_part_of<<<grid_for(G.m, T, cap), T, 0, a.st>>>(fd_adj, G.m, part, fd_part);
  CK_LAUNCH();
  ull *work = a.zeros<ull>(nparts);
  k_fd_work<<<grid_for((size_t)ny * 32, T, cap), T, 0, a.st>>>(o_off, ny, fd_part, work);
  CK_LAUNCH();
  std::vector<ull> hwork(nparts);
  CK(cudaMemcpyAsync(hwork.data(), work, nparts * 8, cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  std::vector<uint32_t> ord(nparts);
  for (uint32_t i = 0; i < nparts; i++) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) { return hwork[x] > hwork[y]; });
  uint32_t *dord = a.alloc<uint32_t>(nparts);
  CK(cudaMemcpyAsync(dord, ord.data(), nparts * 4, cudaMemcpyHostToDevice, a.st));
  CK(cudaEventRecord(ev[3], a.st));

  // support initialisation vector (Sec. 3.1.1) -> fine-phase supports
  CK(cudaMemcpyAsync(sup, init, (size_t)nx * 8, cudaMemcpyDeviceToDevice, a.st));
  FDArgs F{};
  F.p_off = p_off;
  F.p_adj = p_adj;
  F.o_off = o_off;
  F.fd_adj = fd_adj;
  F.fd_part = fd_part;
  F.xs = xs;
  F.ps = ps;
  F.loc = loc;
  F.order = dord;
  F.nparts = nparts;
  F.state = state;
  F.sup = sup;
  F.theta = (ull *)theta_out;
  F.buf_a = alist;
  F.buf_b = alist2;
  F.buf_c = a.alloc<uint32_t>(nx);
  F.buf_d = a.alloc<uint32_t>(nx);
  F.buf_f = front;
  F.buf_big = front2;
  F.buf_huge = a.alloc<uint32_t>(nx);
  F.gcnt = a.zeros<uint32_t>(nx);
  F.queue = dc + 8;
  F.wedges = dwedge + 6;
  F.steps = dwedge + 7;
  F.updates = dwedge + 9;
  ull *pstat = a.zeros<ull>((size_t)TFD_PSTAT * nparts);
  F.pstat = pstat;
  uint32_t *seg_lo = a.alloc<uint32_t>(G.m), *seg_len = a.alloc<uint32_t>(G.m), *w_fd = a.alloc<uint32_t>(nx);
  uint32_t *seg_n = a.alloc<uint32_t>(nx);
  k_fd_segs<<<grid_for((size_t)nx * 32, T, cap), T, 0, a.st>>>(F, nx, part, seg_lo, seg_len, w_fd, seg_n);
  CK_LAUNCH();
  F.seg_lo = seg_lo;
  F.seg_len = seg_len;
  F.w_fd = w_fd;
  F.seg_n = seg_n;
  // heavy partitions (many vertices, or far more work than the mean) on
  // clusters of blocks on a side stream; the rest one block each, concurrently
  const FDClusterShape fc = fd_cluster_shape((const void *)k_fd_tip_cluster, FT, fd_smem());
  std::vector<uint32_t> heavy, light;
  {
    std::vector<uint32_t> hps(nparts + 1);
    CK(cudaMemcpy(hps.data(), ps, hps.size() * 4, cudaMemcpyDeviceToHost));
    double mean = 0;
    for (uint32_t i = 0; i < nparts; i++) mean += (double)hwork[i];
    mean /= std::max<uint32_t>(nparts, 1);
    for (uint32_t i : ord)
      (fc.size > 1 && (hps[i + 1] - hps[i] >= prm.fd_cluster_min || (double)hwork[i] > 4.0 * mean) ? heavy : light)
          .push_back(i);
    std::vector<uint32_t> both(heavy);
    both.insert(both.end(), light.begin(), light.end());
    CK(cudaMemcpyAsync(dord, both.data(), nparts * 4, cudaMemcpyHostToDevice, a.st));
  }
  CK(cudaMemsetAsync(dc + 8, 0, 8, a.st));  // queues of the light and heavy partitions
  g_prof.begin(PROF_FD);
  {
    const uint32_t nh = (uint32_t)heavy.size(), nl = (uint32_t)light.size();
    const uint32_t ncl = std::min<uint32_t>(nh, fc.max_clusters);
    SideLaunch side(a.st, ncl > 0);
    if (ncl) {
      FDArgs FH = F;
      FH.order = dord;
      FH.nparts = nh;
      FH.queue = dc + 9;
      CK(launch_cluster((const void *)k_fd_tip_cluster, ncl, fc.size, FT, fd_smem(), side.st, FH, fd_warp_bytes(),
                        fd_dense_off(), 4 * WIN_CAP_BIG));
      CK_LAUNCH();
    }
    if (nl) {
      FDArgs FL = F;
      FL.order = dord + nh;
      FL.nparts = nl;
      unsigned fgrid = std::max<unsigned>(1u, std::min<unsigned>(nl, sms - ncl * fc.size));
      k_fd_tip<<<fgrid, FT, fd_smem(), a.st>>>(FL, fd_warp_bytes(), fd_dense_off(), 4 * WIN_CAP);
      CK_LAUNCH();
    }
  }
  g_prof.end();
  CK(cudaEventRecord(ev[4], a.st));
  CK(cudaStreamSynchronize(a.st));
  if (trace) {  // fine-phase line per partition: side partition |X_p| work steps cycles
    std::vector<ull> pst((size_t)TFD_PSTAT * nparts);
    std::vector<uint32_t> hps(nparts + 1);
    CK(cudaMemcpy(pst.data(), pstat, pst.size() * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hps.data(), ps, hps.size() * 4, cudaMemcpyDeviceToHost));
    // side partition |X_p| work steps cycles | cycles of select, warp path, heavy path | rescans
    // heavy-vertices (of which by single blocks, by the whole team)
    for (uint32_t i = 0; i < nparts; i++) {
      const ull *q = &pst[(size_t)TFD_PSTAT * i];
      fprintf(trace, "F %d %u %u %llu %llu %llu %llu %llu %llu %llu %llu %llu %llu\n", side, i, hps[i + 1] - hps[i],
              (unsigned long long)hwork[i], q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], q[8]);
    }
  }
  if (st) {
    ull hd[10];
    CK(cudaMemcpy(hd, dwedge, sizeof(hd), cudaMemcpyDeviceToHost));
    float t01, t12, t23, t34;
    cudaEventElapsedTime(&t01, ev[0], ev[1]);
    cudaEventElapsedTime(&t12, ev[1], ev[2]);
    cudaEventElapsedTime(&t23, ev[2], ev[3]);
    cudaEventElapsedTime(&t34, ev[3], ev[4]);
    st->wedges_count += hd[0];
    st->wedges_cd += wedges_cd + hd[3];
    st->wedges_fd += hd[6];
    st->fd_steps += hd[7];
    st->updates += hd[8] + hd[9];
    // algorithmic bytes (per-unit figures documented in pbng.h)
    st->bytes_count += 4 * (hd[0] + hd[3]) + 12 * (hd[1] + hd[4]) + 16 * (hd[2] + hd[5]);
    st->bytes_peel += 4 * wedges_cd + 12 * exp_cd + 16 * hd[8] + 8 * front_cd;
    st->bytes_fd += 4 * hd[6] + 12 * (uint64_t)G.m + 16 * hd[9] + 8 * (uint64_t)nx;
    st->rounds += rounds;
    st->recounts += recounts;
    st->wedge_bound = G.wedge_bound;
    st->ns_count += (uint64_t)(t01 * 1e6);
    st->ns_cd += (uint64_t)(t12 * 1e6);
    st->ns_part += (uint64_t)(t23 * 1e6);
    st->ns_fd += (uint64_t)(t34 * 1e6);
    st->parts_used = nparts;
    for (uint32_t i = 0; i < nparts; i++) {
      st->fd_work_sum += hwork[i];
      if (hwork[i] > st->fd_work_max) st->fd_work_max = hwork[i];
    }
    std::vector<ull> ps_h((size_t)TFD_PSTAT * nparts);
    CK(cudaMemcpy(ps_h.data(), pstat, ps_h.size() * 8, cudaMemcpyDeviceToHost));
    for (uint32_t i = 0; i < nparts; i++) {
      st->fd_part_steps_max = std::max<uint64_t>(st->fd_part_steps_max, ps_h[(size_t)TFD_PSTAT * i]);
      st->fd_part_cycles_max = std::max<uint64_t>(st->fd_part_cycles_max, ps_h[(size_t)TFD_PSTAT * i + 1]);
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
}

}  // namespace pbng
