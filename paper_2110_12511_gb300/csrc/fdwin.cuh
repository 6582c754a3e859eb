// Fine-phase step selection with a candidate window (shared by the tip and
// wing fine-phase kernels; one thread block works on one partition).
//
// Bottom-up peeling of a partition needs, at every step, the remaining
// entities at the running minimum support.  Scanning every remaining entity
// per step costs O(steps x entities).  Instead a scan picks a support window
// [min, hi) holding at most WIN_CAP entities (the min level is always taken
// whole); steps then scan only those candidates, and an entity whose support
// drops below hi during an update joins the candidates (detected from the
// atomic's old value, so exactly once).  A new window is chosen when the
// candidates run out.  Peeling order and recorded numbers are unchanged.
// An entity that joined the candidates also stays in the non-candidate list;
// it is peeled through the candidates, and later windows drop it.
#pragma once
#include <stdint.h>

#include "wedge.cuh"

namespace pbng {

constexpr uint32_t WIN_CAP = 4096;

struct FDLists {
  uint32_t *a[2];  // remaining non-candidates (double buffer)
  uint32_t *c[2];  // candidates (double buffer)
  uint32_t *f;     // entities peeled this step
};

struct FDShared {
  uint32_t na, nc, nf, nn, pa, pc;
  unsigned long long level, mn, hi;
  uint32_t hist[65];
};

// append e to the candidates if its support fell below the window
__device__ __forceinline__ void fd_crossing(FDShared &S, const FDLists &L, uint32_t e, unsigned long long old,
                                            unsigned long long dec) {
  unsigned long long hi = S.hi;
  if (old >= hi && old - dec < hi) L.c[S.pc][atomicAdd(&S.nc, 1u)] = e;
}

// One selection step; returns the number of entities peeled (written to
// L.f, their number recorded as the running level and their state set).
template <int NT>
__device__ uint32_t fd_select(FDShared &S, const FDLists &L, unsigned long long *sup, unsigned long long *theta,
                              uint8_t *state, uint8_t active, uint8_t peeled) {
  int lane = threadIdx.x & 31;
  if (S.nc == 0) {  // choose a new window from the remaining entities
    uint32_t na = S.na, *la = L.a[S.pa], *lb = L.a[S.pa ^ 1], *lc = L.c[S.pc];
    if (threadIdx.x == 0) S.mn = ~0ull;
    for (uint32_t i = threadIdx.x; i < 65; i += NT) S.hist[i] = 0;
    __syncthreads();
    unsigned long long mn = ~0ull;
    for (uint32_t j = threadIdx.x; j < na; j += NT)
      if (state[la[j]] != peeled) mn = min(mn, __ldcg(&sup[la[j]]));
    for (int o = 16; o; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if (lane == 0) atomicMin(&S.mn, mn);
    __syncthreads();
    mn = S.mn;
    for (uint32_t j = threadIdx.x; j < na; j += NT) {
      if (state[la[j]] == peeled) continue;
      unsigned long long d = __ldcg(&sup[la[j]]) - mn;
      atomicAdd(&S.hist[d ? 64 - __clzll(d) : 0], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t cum = 0, b = 0;
      for (uint32_t i = 0; i < 65; i++) {
        if (i > 0 && cum + S.hist[i] > WIN_CAP) break;
        cum += S.hist[i];
        b = i;
      }
      S.hi = b >= 64 ? ~0ull : mn + (1ull << b);  // buckets 0..b hold d < 2^b
      S.nn = 0;
    }
    __syncthreads();
    unsigned long long hi = S.hi;
    for (uint32_t j = threadIdx.x; j < na; j += NT) {
      uint32_t e = la[j];
      if (state[e] == peeled) continue;
      if (__ldcg(&sup[e]) < hi) lc[atomicAdd(&S.nc, 1u)] = e;
      else lb[atomicAdd(&S.nn, 1u)] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      S.na = S.nn;
      S.pa ^= 1;
    }
    __syncthreads();
  }
  uint32_t nc = S.nc, *lc = L.c[S.pc], *ld = L.c[S.pc ^ 1];
  if (threadIdx.x == 0) S.mn = ~0ull;
  __syncthreads();
  unsigned long long mn = ~0ull;
  for (uint32_t j = threadIdx.x; j < nc; j += NT) mn = min(mn, __ldcg(&sup[lc[j]]));
  for (int o = 16; o; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if (lane == 0) atomicMin(&S.mn, mn);
  __syncthreads();
  if (threadIdx.x == 0) {
    S.level = max(S.level, S.mn);
    S.nf = 0;
    S.nn = 0;
  }
  __syncthreads();
  unsigned long long level = S.level;
  for (uint32_t j = threadIdx.x; j < nc; j += NT) {
    uint32_t e = lc[j];
    if (__ldcg(&sup[e]) <= level) {
      L.f[atomicAdd(&S.nf, 1u)] = e;
      theta[e] = level;
      state[e] = active;
    } else {
      ld[atomicAdd(&S.nn, 1u)] = e;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    S.nc = S.nn;
    S.pc ^= 1;
  }
  __syncthreads();
  return S.nf;
}

}  // namespace pbng
