// Fine-phase step selection with a candidate window (shared by the tip and
// wing fine-phase kernels).
//
// Bottom-up peeling of a partition needs, at every step, the remaining
// entities at the running minimum support.  Scanning every remaining entity
// per step costs O(steps x entities).  Instead a scan picks a support window
// [min, hi) holding at most `cap` entities (the min level is always taken
// whole); steps then scan only those candidates, and an entity whose support
// drops below hi during an update joins the candidates (detected from the
// atomic's old value, so exactly once).  A new window is chosen when the
// candidates run out.  Peeling order and recorded numbers are unchanged.
// The window size adapts: a window of C candidates costs one scan of the n
// remaining entities plus two scans of C per step, so with r steps per
// entity (measured on the previous window) about sqrt(1.5 n / r) entities
// per window balance the two (bounded by the caller's cap).
// An entity that joined the candidates also stays in the non-candidate list;
// it is peeled through the candidates, and later windows drop it.
//
// A partition is peeled by a team: one thread block (BlockTeam), or the
// thread blocks of one thread-block cluster (ClusterTeam) for partitions too
// large for one block.  The team's step state lives in the shared memory of
// its first block; the other blocks of a cluster reach it through
// distributed shared memory, and the team barrier is the cluster's hardware
// barrier (release / acquire at cluster scope).  Nothing spins.
#pragma once
#include <cooperative_groups.h>
#include <stdint.h>

#include "wedge.cuh"

namespace pbng {

constexpr uint32_t WIN_CAP = 4096;    // largest window of a one-block team
constexpr uint32_t WIN_CAP_BIG = 65536;  // and of a cluster team (per cluster)

struct FDLists {
  uint32_t *a[2];  // remaining non-candidates (double buffer)
  uint32_t *c[2];  // candidates (double buffer)
  uint32_t *f;     // entities peeled this step
};

struct FDShared {
  uint32_t na, nc, nf, nn, pa, pc;
  unsigned long long level, mn, hi;
  uint32_t hist[65];
  uint32_t p;        // partition being peeled
  uint32_t nt, ncq;  // per-step work lists of the kernels (touched groups, compaction queue)
  uint32_t wn, ws;   // entities of the current window when it was chosen, steps taken since
  uint32_t ng, nh;   // per-step group queue and its overflow list (tip kernels)
  uint32_t nbq, nbh; // per-step block queue and its overflow list (tip cluster kernels)
};

// per-block scratch of a team's minimum reduction
struct TeamMin {
  unsigned long long warp[32];  // one per warp
  unsigned long long block;     // this block's minimum (read by the other blocks of a cluster)
  unsigned long long team;      // the team's minimum
};

struct BlockTeam {
  FDShared *S;      // the block's own step state
  uint32_t *lhist;  // == S->hist
  TeamMin *tm;
  __device__ __forceinline__ uint32_t tid() const { return threadIdx.x; }
  __device__ __forceinline__ uint32_t nthr() const { return blockDim.x; }
  __device__ __forceinline__ bool leader() const { return threadIdx.x == 0; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  // minimum of v over every thread of the team (all threads call it)
  __device__ unsigned long long reduce_min(unsigned long long v) const {
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) tm->warp[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = ~0ull;
      for (uint32_t w = 0; w < (blockDim.x >> 5); w++) m = min(m, tm->warp[w]);
      tm->team = m;
    }
    __syncthreads();
    return *(volatile unsigned long long *)&tm->team;
  }
  static constexpr bool kCluster = false;
};

// cluster barrier: release / acquire at cluster scope, and a compiler fence
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct ClusterTeam {
  FDShared *S;      // step state in the first block of the cluster (distributed shared memory)
  uint32_t *lhist;  // this block's own histogram
  TeamMin *tm;      // this block's reduction scratch
  uint32_t rank, size;
  __device__ __forceinline__ uint32_t tid() const { return rank * blockDim.x + threadIdx.x; }
  __device__ __forceinline__ uint32_t nthr() const { return size * blockDim.x; }
  __device__ __forceinline__ bool leader() const { return rank == 0 && threadIdx.x == 0; }
  __device__ __forceinline__ void sync() const { cluster_barrier(); }
  // minimum over the team: warp shuffles, the block's warps in shared memory,
  // then every block reads the other blocks' minima (plain loads of
  // distributed shared memory; no remote atomics)
  __device__ unsigned long long reduce_min(unsigned long long v) const {
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) tm->warp[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = ~0ull;
      for (uint32_t w = 0; w < (blockDim.x >> 5); w++) m = min(m, tm->warp[w]);
      tm->block = m;
    }
    cluster_barrier();
    if (threadIdx.x == 0) {
      cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
      unsigned long long m = ~0ull;
      for (uint32_t r = 0; r < size; r++) m = min(m, *(volatile unsigned long long *)&cl.map_shared_rank(tm, r)->block);
      tm->team = m;
    }
    __syncthreads();
    return *(volatile unsigned long long *)&tm->team;
  }
  static constexpr bool kCluster = true;
};

// values written by other blocks of the team during the kernel are read
// from L2, never from this SM's L1 (every such value is written in an
// earlier phase, before a team barrier, except pass 1's pair flags, whose
// racing reads only skip pairs the twin rule would skip anyway)
template <class T>
__device__ __forceinline__ T ldt(const T *p) {
  return __ldcg(p);
}

// append e to the candidates if its support fell below the window hi
// (nc, cand: the team's candidate counter and current candidate list)
__device__ __forceinline__ void fd_crossing(unsigned *nc, uint32_t *cand, unsigned long long hi, uint32_t e,
                                            unsigned long long old, unsigned long long dec) {
  if (old >= hi && old - dec < hi) cand[atomicAdd(nc, 1u)] = e;
}

// warp-aggregated append: every lane with `take` gets a distinct slot of
// the list counted by *ctr (all 32 lanes of the warp must call it)
__device__ __forceinline__ uint32_t warp_slot(unsigned *ctr, bool take) {
  const unsigned lane = threadIdx.x & 31, b = __ballot_sync(0xffffffffu, take);
  unsigned base = 0;
  if (lane == 0 && b) base = atomicAdd(ctr, (unsigned)__popc(b));
  base = __shfl_sync(0xffffffffu, base, 0);
  return base + __popc(b & ((1u << lane) - 1u));
}

// One selection step of a team; returns the number of entities peeled
// (written to L.f, their number recorded as the running level and their
// state set).  cap: largest window of candidates.
template <class Team>
__device__ uint32_t fd_select(const Team &T, const FDLists &L, unsigned long long *sup, unsigned long long *theta,
                              uint8_t *state, uint8_t active, uint8_t peeled, uint32_t cap) {
  FDShared *S = T.S;
  const uint32_t lane = threadIdx.x & 31, wbase = T.tid() & ~31u, nthr = T.nthr();
  if (*(volatile uint32_t *)&S->nc == 0) {  // choose a new window from the remaining entities
    const uint32_t na = *(volatile uint32_t *)&S->na, pa = *(volatile uint32_t *)&S->pa,
                   pc = *(volatile uint32_t *)&S->pc;
    uint32_t *la = L.a[pa], *lb = L.a[pa ^ 1], *lc = L.c[pc];
    if (T.leader()) S->nn = 0;
    for (uint32_t i = threadIdx.x; i < 65; i += blockDim.x) T.lhist[i] = 0;
    if (Team::kCluster && T.leader())
      for (uint32_t i = 0; i < 65; i++) S->hist[i] = 0;
    unsigned long long mn = ~0ull;
    for (uint32_t j = T.tid(); j < na; j += nthr) {
      uint32_t e = ldt(&la[j]);
      if (ldt(&state[e]) != peeled) mn = min(mn, ldt(&sup[e]));
    }
    mn = T.reduce_min(mn);  // (its barriers also order the resets above)
    for (uint32_t j = T.tid(); j < na; j += nthr) {
      uint32_t e = ldt(&la[j]);
      if (ldt(&state[e]) == peeled) continue;
      unsigned long long d = ldt(&sup[e]) - mn;
      atomicAdd(&T.lhist[d ? 64 - __clzll(d) : 0], 1u);
    }
    if (Team::kCluster) {  // merge the blocks' histograms into the team's
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < 65; i += blockDim.x)
        if (T.lhist[i]) atomicAdd(&S->hist[i], T.lhist[i]);
    }
    T.sync();
    if (T.leader()) {
      // window size from the previous window's steps per entity (1 for the first)
      const float r = S->wn ? fmaxf((float)S->ws, 1.0f) / (float)S->wn : 1.0f;
      const uint32_t w = (uint32_t)fminf((float)cap, fmaxf(64.0f, sqrtf(1.5f * (float)na / r)));
      uint32_t cum = 0, b = 0;
      for (uint32_t i = 0; i < 65; i++) {
        uint32_t h = *(volatile uint32_t *)&S->hist[i];
        if (i > 0 && cum + h > w) break;
        cum += h;
        b = i;
      }
      S->hi = b >= 64 ? ~0ull : mn + (1ull << b);  // buckets 0..b hold d < 2^b
    }
    T.sync();
    const unsigned long long hi = *(volatile unsigned long long *)&S->hi;
    for (uint32_t j0 = wbase; j0 < na; j0 += nthr) {
      const uint32_t j = j0 + lane;
      uint32_t e = 0;
      bool live = false, cand = false;
      if (j < na) {
        e = ldt(&la[j]);
        live = ldt(&state[e]) != peeled;
        cand = live && ldt(&sup[e]) < hi;
      }
      const uint32_t sc = warp_slot(&S->nc, cand);
      const uint32_t sn = warp_slot(&S->nn, live && !cand);
      if (cand) lc[sc] = e;
      else if (live) lb[sn] = e;
    }
    T.sync();
    if (T.leader()) {
      S->na = *(volatile uint32_t *)&S->nn;
      S->pa ^= 1;
      S->wn = *(volatile uint32_t *)&S->nc;
      S->ws = 0;
    }
    T.sync();
  }
  const uint32_t nc = *(volatile uint32_t *)&S->nc, pc = *(volatile uint32_t *)&S->pc;
  uint32_t *lc = L.c[pc], *ld = L.c[pc ^ 1];
  unsigned long long mn = ~0ull;
  for (uint32_t j = T.tid(); j < nc; j += nthr) mn = min(mn, ldt(&sup[ldt(&lc[j])]));
  mn = T.reduce_min(mn);
  if (T.leader()) {
    S->ws++;
    S->level = max(*(volatile unsigned long long *)&S->level, mn);
    S->nf = 0;
    S->nn = 0;
    S->nt = 0;  // the kernels' per-step lists start empty
    S->ncq = 0;
    S->ng = 0;
    S->nh = 0;
    S->nbq = 0;
    S->nbh = 0;
  }
  T.sync();
  const unsigned long long level = *(volatile unsigned long long *)&S->level;
  for (uint32_t j0 = wbase; j0 < nc; j0 += nthr) {
    const uint32_t j = j0 + lane;
    uint32_t e = 0;
    bool in = false, take = false;
    if (j < nc) {
      e = ldt(&lc[j]);
      in = true;
      take = ldt(&sup[e]) <= level;
    }
    const uint32_t sf = warp_slot(&S->nf, take);
    const uint32_t sn = warp_slot(&S->nn, in && !take);
    if (take) {
      L.f[sf] = e;
      theta[e] = level;
      state[e] = active;
    } else if (in) {
      ld[sn] = e;
    }
  }
  T.sync();
  if (T.leader()) {
    S->nc = *(volatile uint32_t *)&S->nn;
    S->pc ^= 1;
  }
  T.sync();
  return *(volatile uint32_t *)&S->nf;
}

}  // namespace pbng
