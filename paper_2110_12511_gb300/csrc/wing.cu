// Wing decomposition with the Bloom-Edge-Index (Sec. 2.3, 3.3; Alg. 3-6).
//
// BE-Index (Sec. 2.3): every pair {start, last} of wedge endpoints found by
// the vertex-priority traversal of Alg. 1 with wedge_count >= 2 is the
// dominant set of one maximal priority bloom B with bloom number
// k_B = wedge_count; for each middle vertex the edges (start, mid) and
// (mid, last) are twins in B.  Stored bloom-major as twin pairs
// (pe1[q], pe2[q]) with bloom pbloom[q], plus the edge -> pair lists.
// Per-edge butterfly counts come from the same counting pass.
//
// Coarse phase (Alg. 4 with the batch update of Alg. 6): ranges from
// find_range with support as work proxy; each round peels the active set A
// of edges with support below theta(i+1):
//  pass 1, per active e and live pair q = (e, e_t) of bloom B: e acts iff
//    e_t is not active or edgeID(e_t) < edgeID(e) (Alg. 4 conflict rule);
//    an acting e removes the pair, counts it in count[B], and when e_t is not
//    active lowers support(e_t) by k_B - 1 (all butterflies e_t has in B);
//  pass 2, per bloom with count[B] > 0: k_B -= count[B], and every edge of
//    a remaining pair loses count[B] butterflies.
//  Alg. 6 as printed lowers the twin by k_B; Alg. 3, Alg. 4, Property 1 and
//  Lemma 2 all give k_B - 1, which is what is applied here.  Supports stay
//  exact (unclamped); pair lists of touched blooms are compacted in pass 2
//  (dynamic updates, Sec. 5.2).
// partition_BE_Index (Alg. 5): pair q belongs to the index of partition
//  pmin(q) = min(p(e1), p(e2)); its link (e, B) is kept for the edge(s) in
//  that partition, and k_B(I_i) = number of pairs of B with pmin >= i.
// Fine phase (Alg. 5): one thread block per partition, heaviest first;
//  every step peels all edges at the minimum support together, applying the
//  same two-pass update restricted to I_i.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "fdwin.cuh"
#include "internal.cuh"
#include "wedge.cuh"

namespace pbng {
namespace {

using ull = unsigned long long;
enum : uint8_t { ST_ALIVE = 0, ST_ACTIVE = 1, ST_PEELED = 2 };
constexpr uint32_t FW_MAXW = 256, FW_CAP = 512;
constexpr int FBT = 512, FWT = 256;
constexpr uint32_t NO_CUR = 0xffffffffu;

// ------------------------------------------------------------ BE-Index fill
struct FillArgs {
  const uint32_t *off, *adj, *eid;
  uint32_t n;
  const ull *bb, *pb;  // bloom and pair bases per start (exclusive scans)
  uint32_t *k0, *boff, *pe1, *pe2;
};

template <int N>
struct FMid {
  uint32_t mid[N];
  uint32_t lo[N];
  uint32_t pre[N + 1];
};

// chunk of mids of start s and their prefixes of valid lasts (labels below
// min(s, mid)), as in the counting traversal
template <class Grp, int N>
__device__ __forceinline__ uint32_t fill_load(const FillArgs &A, uint32_t s, uint32_t so, uint32_t sd, uint32_t base,
                                              const Grp &g, FMid<N> &mb) {
  int r = g.rank();
  uint32_t lo = 0, len = 0;
  if (base + r < sd) {
    uint32_t mid = A.adj[so + base + r];
    uint32_t b = min(s, mid);
    lo = A.off[mid];
    uint32_t d = A.off[mid + 1] - lo;
    len = lower_bound_u32(A.adj + lo, min(d, b), b);
  }
  mb.lo[r] = lo;
  return g.scan(len, mb.pre);
}

// f(i, pos, last): i = mid slot in the chunk, pos = position of last in N_mid
template <class Grp, int N, class F>
__device__ __forceinline__ void fill_walk(const FillArgs &A, const Grp &g, const FMid<N> &mb, uint32_t T, F &&f) {
  for (uint32_t w = g.rank(); w < T; w += N) {
    int i = seg_of(mb.pre, N, w);
    uint32_t pos = mb.lo[i] + (w - mb.pre[i]);
    f(i, pos, A.adj[pos]);
  }
}

__global__ void k_fill_classify(const uint32_t *off, const uint32_t *adj, uint32_t n, const ull *be_np, ull *lists,
                                unsigned *counts) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t s = gw; s < n; s += nw) {
    if (be_np[s] == 0) continue;
    uint32_t so = off[s], sd = off[s + 1] - so;
    uint64_t B = 0;
    for (uint32_t k = lane; k < sd; k += 32) {
      uint32_t mid = adj[so + k];
      B += min(off[mid + 1] - off[mid], min((uint32_t)s, mid));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) B += __shfl_xor_sync(0xffffffffu, B, o);
    if (lane == 0) {
      int c = B <= FW_MAXW ? 0 : 1;
      unsigned p = atomicAdd(&counts[c], 1u);
      lists[(size_t)c * n + p] = (ull)s | ((ull)min(B, (uint64_t)0xffffffffu) << 32);
    }
  }
}

// warp per start: shared hash of wedge counts per last, then number the
// blooms (packed counter: blooms in the high half, pairs in the low half so
// that bloom ids and pair ranges are handed out together), then write every
// wedge of a bloom as a twin pair
__global__ void __launch_bounds__(FWT) k_fill_warp(FillArgs A, const ull *list, const unsigned *count) {
  extern __shared__ __align__(16) uint8_t sm[];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr size_t per = align16(FW_CAP * 12 + sizeof(FMid<32>) + 16);
  uint8_t *base_p = sm + w * per;
  uint32_t *key = (uint32_t *)base_p, *val = key + FW_CAP, *cur = val + FW_CAP;
  FMid<32> &mb = *(FMid<32> *)(base_p + FW_CAP * 12);
  ull *ctr = (ull *)(base_p + align16(FW_CAP * 12 + sizeof(FMid<32>)));
  for (uint32_t i = lane; i < FW_CAP; i += 32) key[i] = EMPTY_KEY, val[i] = 0;
  if (lane == 0) *ctr = 0;
  __syncwarp();
  WarpGrp g;
  unsigned n = *count;
  for (size_t it = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5; it < n; it += ((size_t)gridDim.x * blockDim.x) >> 5) {
    ull item = list[it];
    uint32_t s = (uint32_t)item, B = (uint32_t)(item >> 32);
    uint32_t cap = pow2_at_least(max(2u * B, 32u));
    SmemHash h{key, val, cap - 1};
    uint32_t so = A.off[s], sd = A.off[s + 1] - so;
    for (uint32_t base = 0; base < sd; base += 32) {
      uint32_t T = fill_load(A, s, so, sd, base, g, mb);
      fill_walk(A, g, mb, T, [&](int, uint32_t, uint32_t last) { h.inc(last); });
      __syncwarp();
    }
    for (uint32_t i = lane; i < cap; i += 32) {
      uint32_t c = val[i];
      cur[i] = NO_CUR;
      if (key[i] != EMPTY_KEY && c >= 2) {
        ull p = atomicAdd(ctr, (1ull << 32) | c);
        uint32_t b = (uint32_t)(A.bb[s] + (p >> 32));
        uint32_t q0 = (uint32_t)(A.pb[s] + (uint32_t)p);
        A.k0[b] = c;
        A.boff[b] = q0;
        cur[i] = q0;
      }
    }
    __syncwarp();
    for (uint32_t base = 0; base < sd; base += 32) {
      uint32_t T = fill_load(A, s, so, sd, base, g, mb);
      fill_walk(A, g, mb, T, [&](int i, uint32_t pos, uint32_t last) {
        uint32_t hh = hash32(last) & h.mask;
        while (key[hh] != last) hh = (hh + 1) & h.mask;
        if (cur[hh] != NO_CUR) {
          uint32_t q = atomicAdd(&cur[hh], 1u);
          A.pe1[q] = A.eid[so + base + i];  // edge (start, mid)
          A.pe2[q] = A.eid[pos];            // its twin (mid, last)
        }
      });
      __syncwarp();
    }
    for (uint32_t i = lane; i < cap; i += 32) key[i] = EMPTY_KEY, val[i] = 0;
    if (lane == 0) *ctr = 0;
    __syncwarp();
  }
}

size_t fill_warp_smem() { return (FWT / 32) * align16(FW_CAP * 12 + sizeof(FMid<32>) + 16); }

// block per start with per-block dense counters and cursors over all labels
// in global memory (both zero between starts)
__global__ void __launch_bounds__(FBT) k_fill_block(FillArgs A, const ull *list, const unsigned *count, uint32_t *scr) {
  __shared__ FMid<FBT> mb;
  __shared__ uint32_t ws[FBT / 32 + 2];
  __shared__ ull ws64[FBT / 32];
  __shared__ ull ctr;
  BlockGrp<FBT> g{ws, ws64};
  uint32_t *cnt = scr + (size_t)blockIdx.x * 2 * A.n, *cur = cnt + A.n;
  if (threadIdx.x == 0) ctr = 0;
  __syncthreads();
  unsigned n = *count;
  for (size_t it = blockIdx.x; it < n; it += gridDim.x) {
    uint32_t s = (uint32_t)list[it];
    uint32_t so = A.off[s], sd = A.off[s + 1] - so;
    for (int pass = 0; pass < 4; pass++) {
      for (uint32_t base = 0; base < sd; base += FBT) {
        uint32_t T = fill_load(A, s, so, sd, base, g, mb);
        fill_walk(A, g, mb, T, [&](int i, uint32_t pos, uint32_t last) {
          if (pass == 0) {
            atomicAdd(&cnt[last], 1u);
          } else if (pass == 1) {  // number each bloom once
            uint32_t c = __ldcg(&cnt[last]);
            if (c >= 2 && atomicCAS(&cur[last], 0u, NO_CUR) == 0u) {
              ull p = atomicAdd(&ctr, (1ull << 32) | c);
              uint32_t b = (uint32_t)(A.bb[s] + (p >> 32));
              uint32_t q0 = (uint32_t)(A.pb[s] + (uint32_t)p);
              A.k0[b] = c;
              A.boff[b] = q0;
              atomicExch(&cur[last], q0 + 1);  // cursor, stored plus one
            }
          } else if (pass == 2) {
            uint32_t c = __ldcg(&cnt[last]);
            if (c >= 2) {
              uint32_t q = atomicAdd(&cur[last], 1u) - 1;
              A.pe1[q] = A.eid[so + base + i];
              A.pe2[q] = A.eid[pos];
            }
          } else {
            cnt[last] = 0;
            cur[last] = 0;
          }
        });
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) ctr = 0;
    __syncthreads();
  }
}

__global__ void k_pair_bloom(const uint32_t *k0, const uint32_t *boff, uint32_t nb, uint32_t *pbloom) {
  for (size_t b = blockIdx.x * (size_t)blockDim.x + threadIdx.x; b < nb; b += (size_t)gridDim.x * blockDim.x)
    for (uint32_t q = boff[b]; q < boff[b] + k0[b]; q++) pbloom[q] = (uint32_t)b;
}

__global__ void k_link_deg(const uint32_t *pe1, const uint32_t *pe2, size_t np, uint32_t *deg) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < np; q += (size_t)gridDim.x * blockDim.x) {
    atomicAdd(&deg[pe1[q]], 1u);
    atomicAdd(&deg[pe2[q]], 1u);
  }
}

__global__ void k_link_fill(const uint32_t *pe1, const uint32_t *pe2, size_t np, const uint32_t *eoff, uint32_t *ecur,
                            uint32_t *elink) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < np; q += (size_t)gridDim.x * blockDim.x) {
    uint32_t a = pe1[q], b = pe2[q];
    elink[eoff[a] + atomicAdd(&ecur[a], 1u)] = (uint32_t)q;
    elink[eoff[b] + atomicAdd(&ecur[b], 1u)] = (uint32_t)q;
  }
}

// ------------------------------------------------------------ coarse phase
struct CDArgs {
  const uint32_t *pe1, *pe2, *pbloom, *eoff, *elink, *boff;
  uint32_t *kcur, *cntB, *bq, *blen;
  uint8_t *palive, *state;
  ull *sup;
  const ull *theta_hi;
  uint32_t *next;
  unsigned *next_n;
  uint32_t *touched;
  unsigned *touched_n;
  ull *ctr;  // [0] links traversed, [1] updates, [3] support of peeled edges (work of the partition)
};

__device__ __forceinline__ void wdec(const CDArgs &A, uint32_t e, uint64_t dec, ull thi) {
  ull old = atomicAdd(&A.sup[e], (ull)(0ull - dec));
  if (old >= thi && old - dec < thi) {
    unsigned p = atomicAdd(A.next_n, 1u);
    A.next[p] = e;
  }
}

// pass 1: warp per active edge (Alg. 6 lines 3-9 with the k_B - 1 reading)
__global__ void k_wing_pass1(CDArgs A, const uint32_t *front, uint32_t nf, uint32_t *part, uint32_t pi) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  ull thi = *A.theta_hi, links = 0, ups = 0, work = 0;
  for (size_t j = gw; j < nf; j += nw) {
    uint32_t e = front[j];
    if (lane == 0) {
      part[e] = pi;
      work += A.sup[e];
    }
    uint32_t lo = A.eoff[e], hi = A.eoff[e + 1];
    for (uint32_t k = lo + lane; k < hi; k += 32) {
      uint32_t q = A.elink[k];
      links++;
      if (!A.palive[q]) continue;
      uint32_t a = A.pe1[q], b = A.pe2[q];
      uint32_t et = a == e ? b : a;
      uint8_t st = A.state[et];
      if (st == ST_ACTIVE && et > e) continue;  // the twin with the higher id acts
      uint32_t B = A.pbloom[q];
      A.palive[q] = 0;
      if (st == ST_ALIVE) {
        uint32_t kb = A.kcur[B];
        if (kb >= 2) wdec(A, et, kb - 1, thi), ups++;
      }
      if (atomicAdd(&A.cntB[B], 1u) == 0u) {
        unsigned p = atomicAdd(A.touched_n, 1u);
        A.touched[p] = B;
      }
    }
  }
  for (int o = 16; o; o >>= 1) links += __shfl_xor_sync(0xffffffffu, links, o), ups += __shfl_xor_sync(0xffffffffu, ups, o);
  if (lane == 0) {
    if (links) atomicAdd(&A.ctr[0], links);
    if (ups) atomicAdd(&A.ctr[1], ups);
    if (work) atomicAdd(&A.ctr[3], work);
  }
}

// pass 2: warp per touched bloom (Alg. 6 lines 10-13): k_B -= count[B];
// every edge of a remaining pair loses count[B]; the pair list is compacted
__global__ void k_wing_pass2(CDArgs A, int compact) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  ull thi = *A.theta_hi, links = 0, ups = 0;
  unsigned nt = *A.touched_n;
  for (size_t j = gw; j < nt; j += nw) {
    uint32_t B = A.touched[j];
    uint32_t c = A.cntB[B];
    uint32_t lo = A.boff[B], len = A.blen[B], out = 0;
    for (uint32_t k = 0; k < len; k += 32) {
      uint32_t q = 0;
      bool live = false;
      if (k + lane < len) {
        q = A.bq[lo + k + lane];
        live = A.palive[q];
        links++;
        if (live) {
          wdec(A, A.pe1[q], c, thi);
          wdec(A, A.pe2[q], c, thi);
          ups += 2;
        }
      }
      if (compact) {
        unsigned bal = __ballot_sync(0xffffffffu, live);
        __syncwarp();
        if (live) A.bq[lo + out + __popc(bal & ((1u << lane) - 1u))] = q;
        out += __popc(bal);
        __syncwarp();
      }
    }
    if (lane == 0) {
      A.kcur[B] -= c;
      A.cntB[B] = 0;
      if (compact) A.blen[B] = out;
    }
  }
  for (int o = 16; o; o >>= 1) links += __shfl_xor_sync(0xffffffffu, links, o), ups += __shfl_xor_sync(0xffffffffu, ups, o);
  if (lane == 0) {
    if (links) atomicAdd(&A.ctr[0], links);
    if (ups) atomicAdd(&A.ctr[1], ups);
  }
}

__global__ void k_wing_mark(const uint32_t *f, uint32_t nf, uint8_t *state, uint8_t st) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < nf; j += (size_t)gridDim.x * blockDim.x)
    state[f[j]] = st;
}

__global__ void k_iota(uint32_t *a, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) a[i] = (uint32_t)i;
}

__global__ void k_copy_u32(const uint32_t *a, uint32_t *b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}

// key range and total work of the remaining edges; work proxy = support
// (Sec. 3.3.2: peeling an edge costs O(support) in the BE-Index)
__global__ void k_wing_weights(const uint32_t *alist, uint32_t na, const ull *sup, ull *wl, RangeState *rs) {
  ull mn = ~0ull, mx = 0, ws = 0;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < na; j += (size_t)gridDim.x * blockDim.x) {
    ull s = sup[alist[j]];
    wl[j] = s;
    mn = min(mn, s);
    mx = max(mx, s);
    ws += s;
  }
  for (int o = 16; o; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    ws += __shfl_xor_sync(0xffffffffu, ws, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&rs->kmin, mn);
    atomicMax(&rs->kmax, mx);
    if (ws) atomicAdd(&rs->wsum, ws);
  }
}

__global__ void k_wing_scan(const uint32_t *alist, uint32_t na, uint8_t *state, const ull *sup, ull *init, const ull *theta_hi,
                            uint32_t *f, unsigned *fn) {
  ull thi = *theta_hi;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < na; j += (size_t)gridDim.x * blockDim.x) {
    uint32_t e = alist[j];
    if (state[e] != ST_ALIVE) continue;
    ull s = sup[e];
    init[e] = s;
    if (s < thi) {
      state[e] = ST_ACTIVE;
      f[atomicAdd(fn, 1u)] = e;
    }
  }
}

__global__ void k_wing_compact_list(const uint32_t *in, uint32_t n, const uint8_t *state, uint32_t *out, unsigned *on) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    uint32_t e = in[j];
    if (state[e] == ST_ALIVE) out[atomicAdd(on, 1u)] = e;
  }
}

// ------------------------------------------------------------ fine phase
__global__ void k_pmin(const uint32_t *pe1, const uint32_t *pe2, const uint32_t *pbloom, size_t np, const uint32_t *part,
                       int bp, uint64_t *key, uint32_t *val, uint32_t *pmin) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < np; q += (size_t)gridDim.x * blockDim.x) {
    uint32_t p = min(part[pe1[q]], part[pe2[q]]);
    pmin[q] = p;
    key[q] = ((uint64_t)pbloom[q] << bp) | p;
    val[q] = (uint32_t)q;
  }
}

__global__ void k_group_heads(const uint64_t *key, size_t np, uint32_t *head) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < np; k += (size_t)gridDim.x * blockDim.x)
    head[k] = (k == 0 || key[k] != key[k - 1]) ? 1u : 0u;
}

// groups (B, i) of the (bloom, pmin)-sorted pairs: start position, bloom
// number k_B(I_i) = pairs of B with pmin >= i, partition, pair -> group
__global__ void k_groups(const uint64_t *key, const uint32_t *order, size_t np, const uint32_t *gidx, const uint32_t *head,
                         const uint32_t *k0, const uint32_t *boff, int bp, uint32_t *gstart, uint32_t *gk, uint32_t *gpart,
                         uint32_t *pb_of) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < np; k += (size_t)gridDim.x * blockDim.x) {
    uint32_t g = gidx[k];  // exclusive scan of heads: group of position k is gidx[k] + head[k] - 1
    g = g + head[k] - 1;
    if (head[k]) {
      uint32_t B = (uint32_t)(key[k] >> bp);
      gstart[g] = (uint32_t)k;
      gk[g] = boff[B] + k0[B] - (uint32_t)k;
      gpart[g] = (uint32_t)(key[k] & ((1ull << bp) - 1));
    }
    pb_of[order[k]] = g;
  }
}

__global__ void k_edge_keys(const uint32_t *part, uint32_t m, uint64_t *key, uint32_t *val) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < m; e += (size_t)gridDim.x * blockDim.x) {
    key[e] = part[e];
    val[e] = (uint32_t)e;
  }
}

__global__ void k_hist_u32(const uint32_t *x, size_t n, uint32_t *cnt) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[x[i]], 1u);
}

__global__ void k_part_work(const uint32_t *part, const ull *init, uint32_t m, ull *work) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < m; e += (size_t)gridDim.x * blockDim.x)
    if (init[e]) atomicAdd(&work[part[e]], init[e]);
}

__global__ void k_fd_reset(uint8_t *palive, size_t np, uint8_t *state, uint32_t m) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < np || i < m; i += (size_t)gridDim.x * blockDim.x) {
    if (i < np) palive[i] = 1;
    if (i < m) state[i] = ST_ALIVE;
  }
}

// links (e, B) kept in the index of e's own partition: pmin(q) == part(e)
__global__ void k_flink_count(const uint32_t *eoff, const uint32_t *elink, const uint32_t *pmin, const uint32_t *part,
                              uint32_t m, uint32_t *fdeg) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t e = gw; e < m; e += nw) {
    uint32_t p = part[e], c = 0;
    for (uint32_t k = eoff[e] + lane; k < eoff[e + 1]; k += 32) c += pmin[elink[k]] == p;
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) fdeg[e] = c;
  }
}

__global__ void k_flink_fill(const uint32_t *eoff, const uint32_t *elink, const uint32_t *pmin, const uint32_t *part,
                             uint32_t m, const uint32_t *foff, uint32_t *flink) {
  int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t e = gw; e < m; e += nw) {
    uint32_t p = part[e], out = foff[e];
    for (uint32_t k = eoff[e]; k < eoff[e + 1]; k += 32) {
      uint32_t q = 0;
      bool keep = false;
      if (k + lane < eoff[e + 1]) {
        q = elink[k + lane];
        keep = pmin[q] == p;
      }
      unsigned b = __ballot_sync(0xffffffffu, keep);
      if (keep) flink[out + __popc(b & ((1u << lane) - 1u))] = q;
      out += __popc(b);
    }
  }
}

__global__ void k_group_len(const uint32_t *gstart, uint32_t ng, uint32_t *glen) {
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < ng; g += (size_t)gridDim.x * blockDim.x)
    glen[g] = gstart[g + 1] - gstart[g];
}

struct WFDArgs {
  const uint32_t *pe1, *pe2, *eoff, *elink, *pmin, *pb_of, *order, *gstart, *gps;
  const uint32_t *part, *es, *ps, *orderp;  // edges grouped by partition, partition offsets, LPT order
  uint32_t *gk, *gcnt;
  uint8_t *palive, *state;
  ull *sup, *theta;
  uint32_t *buf_a, *buf_b, *buf_c, *buf_d, *buf_f, *gtouch;  // per-partition regions
  uint32_t nparts;
  unsigned *queue;
  ull *ctr;  // [0] links, [1] updates, [2] steps
  ull *pstat;  // per partition: steps, SM cycles
  const uint32_t *foff, *flink;  // per edge: its links in its own partition's index
  uint32_t *glen;                // live prefix of each group's pair list in order
  uint32_t *order_w;             // writable alias of order (compaction)
};

constexpr int WFT = 512;
constexpr int WFD_PSTAT = 7;  // per-partition statistics of the fine phase

// Fine phase of the partitions handed out by A.queue / A.orderp (Alg. 5 lines
// 1-11 with the batch rule of Sec. 5.1), one partition at a time per team.
// Every step: the selection (fd_select), pass 1 over the links of the peeled
// edges inside I_p, pass 2 over the touched groups' live pairs, the groups'
// bloom numbers and lazy compaction, then the peeled state.  A cluster team
// splits every phase across its blocks (each block computes the same scan of
// a chunk and takes an interleaved share of its flattened work).
template <class Team>
__device__ void wing_fd_run(const WFDArgs &A, const Team &T, uint32_t cap, uint32_t *s_itm, uint32_t *s_lo,
                            uint32_t *s_pre, const BlockGrp<WFT> &bg) {
  FDShared *S = T.S;
  const int lane = threadIdx.x & 31;
  const uint32_t nthr = T.nthr();
  ull links = 0, ups = 0, steps = 0;
  for (;;) {
    if (T.leader()) {
      unsigned q = atomicAdd(A.queue, 1u);
      S->p = q < A.nparts ? A.orderp[q] : 0xffffffffu;
    }
    T.sync();
    const uint32_t p = *(volatile uint32_t *)&S->p;
    T.sync();  // every block has read p before it can change, or before the team exits
    if (p == 0xffffffffu) break;
    const uint32_t base = A.ps[p], np = A.ps[p + 1] - base;
    uint32_t *lf = A.buf_f + base, *gt = A.gtouch + 2 * A.gps[p];
    FDLists L{{A.buf_a + base, A.buf_b + base}, {A.buf_c + base, A.buf_d + base}, lf};
    for (uint32_t j = T.tid(); j < np; j += nthr) L.a[0][j] = A.es[base + j];
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
    ull p_steps = 0, cyc[4] = {0, 0, 0, 0}, rescans = 0;
    T.sync();
    for (;;) {
      if (*(volatile uint32_t *)&S->na + *(volatile uint32_t *)&S->nc == 0) break;
      p_steps++;
      long long t0 = clock64();
      rescans += *(volatile uint32_t *)&S->nc == 0;
      const uint32_t nf = fd_select(T, L, A.sup, A.theta, A.state, ST_ACTIVE, ST_PEELED, cap);
      long long t1 = clock64();
      uint32_t *cand = L.c[*(volatile uint32_t *)&S->pc];
      const ull hi = *(volatile ull *)&S->hi;
      steps++;
      // pass 1 restricted to I_p, flattened over (peeled edge, link) so the
      // whole team shares a few long link lists
      for (uint32_t c0 = 0; c0 < nf; c0 += WFT) {
        uint32_t r = threadIdx.x, lo = 0, len = 0;
        if (c0 + r < nf) {
          uint32_t e = ldt(&lf[c0 + r]);
          s_itm[r] = e;
          lo = A.foff[e];
          len = A.foff[e + 1] - lo;
        }
        s_lo[r] = lo;
        const uint32_t Tw = bg.scan(len, s_pre);
        for (uint32_t w = T.tid(); w < Tw; w += nthr) {
          int i = seg_of(s_pre, WFT, w);
          uint32_t e = s_itm[i], q = A.flink[s_lo[i] + (w - s_pre[i])];  // a link of e in I_p
          links++;
          if (!ldt(&A.palive[q])) continue;
          uint32_t a = A.pe1[q], b = A.pe2[q];
          uint32_t et = a == e ? b : a;
          bool in_p = A.part[et] == p;
          uint8_t st = in_p ? ldt(&A.state[et]) : (uint8_t)ST_ALIVE;
          if (st == ST_ACTIVE && et > e) continue;
          uint32_t g = A.pb_of[q];
          A.palive[q] = 0;
          if (in_p && st == ST_ALIVE) {
            uint32_t kb = ldt(&A.gk[g]);
            if (kb >= 2) {
              ull old = atomicAdd(&A.sup[et], (ull)(0ull - (ull)(kb - 1)));
              fd_crossing(&S->nc, cand, hi, et, old, kb - 1);
              ups++;
            }
          }
          if (atomicAdd(&A.gcnt[g], 1u) == 0u) gt[atomicAdd(&S->nt, 1u)] = g;
        }
        __syncthreads();  // the chunk arrays are rewritten by the next chunk
      }
      T.sync();
      long long t2 = clock64();
      // pass 2 restricted to I_p (Alg. 6, second loop) with the bloom numbers:
      // a warp per touched group walks its pair list in 32-pair chunks
      // (coalesced), lowers both edges of every live pair by count[g], and
      // compacts the list in the same walk
      const uint32_t nt = *(volatile uint32_t *)&S->nt;
      for (uint32_t j = T.tid() >> 5; j < nt; j += nthr >> 5) {
        const uint32_t g = ldt(&gt[j]);
        const uint32_t c = ldt(&A.gcnt[g]), lo = A.gstart[g], len = ldt(&A.glen[g]);
        uint32_t out = 0;
        for (uint32_t k = 0; k < len; k += 32) {
          uint32_t q = 0;
          bool live = false;
          if (k + lane < len) {
            q = ldt(&A.order_w[lo + k + lane]);
            live = ldt(&A.palive[q]);
            links++;
          }
          if (live) {
            const uint32_t ea = A.pe1[q], eb = A.pe2[q];
            if (A.part[ea] == p && ldt(&A.state[ea]) == ST_ALIVE)
              fd_crossing(&S->nc, cand, hi, ea, atomicAdd(&A.sup[ea], (ull)(0ull - c)), c), ups++;
            if (A.part[eb] == p && ldt(&A.state[eb]) == ST_ALIVE)
              fd_crossing(&S->nc, cand, hi, eb, atomicAdd(&A.sup[eb], (ull)(0ull - c)), c), ups++;
          }
          const unsigned bal = __ballot_sync(0xffffffffu, live);
          if (live) A.order_w[lo + out + __popc(bal & ((1u << lane) - 1u))] = q;
          out += __popc(bal);
          __syncwarp();
        }
        if (lane == 0) {
          A.glen[g] = out;
          A.gk[g] = ldt(&A.gk[g]) - c;
          A.gcnt[g] = 0;
        }
      }
      T.sync();
      long long t3 = clock64();
      for (uint32_t j = T.tid(); j < nf; j += nthr) A.state[ldt(&lf[j])] = ST_PEELED;
      T.sync();
      long long t4 = clock64();
      cyc[0] += t1 - t0;
      cyc[1] += t2 - t1;
      cyc[2] += t3 - t2;
      cyc[3] += t4 - t3;
    }
    if (T.leader() && A.pstat) {  // steps, cycles; then select, pass 1, pass 2, rest, window rescans
      ull *ps = A.pstat + (size_t)WFD_PSTAT * p;
      ps[0] = p_steps;
      ps[1] = (ull)(clock64() - t_part);
      for (int k = 0; k < 4; k++) ps[2 + k] = cyc[k];
      ps[6] = rescans;
    }
  }
  for (int o = 16; o; o >>= 1) links += __shfl_xor_sync(0xffffffffu, links, o), ups += __shfl_xor_sync(0xffffffffu, ups, o);
  if (lane == 0) {
    if (links) atomicAdd(&A.ctr[0], links);
    if (ups) atomicAdd(&A.ctr[1], ups);
  }
  if (T.leader()) atomicAdd(&A.ctr[2], steps);
}

// one block per partition
__global__ void __launch_bounds__(WFT) k_wing_fd(WFDArgs A, uint32_t cap) {
  __shared__ FDShared S;
  __shared__ uint32_t s_itm[WFT], s_lo[WFT], s_pre[WFT + 1];
  __shared__ uint32_t ws[WFT / 32 + 2];
  __shared__ ull ws64[WFT / 32];
  __shared__ TeamMin tmin;
  BlockGrp<WFT> bg{ws, ws64};
  BlockTeam T{&S, S.hist, &tmin};
  wing_fd_run(A, T, cap, s_itm, s_lo, s_pre, bg);
}

// one thread-block cluster per (heavy) partition; the step state lives in
// the shared memory of the cluster's first block
__global__ void __launch_bounds__(WFT) k_wing_fd_cluster(WFDArgs A, uint32_t cap) {
  __shared__ FDShared S;
  __shared__ uint32_t lhist[65];
  __shared__ uint32_t s_itm[WFT], s_lo[WFT], s_pre[WFT + 1];
  __shared__ uint32_t ws[WFT / 32 + 2];
  __shared__ ull ws64[WFT / 32];
  BlockGrp<WFT> bg{ws, ws64};
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  __shared__ TeamMin tmin;
  ClusterTeam T{cl.map_shared_rank(&S, 0), lhist, &tmin, cl.block_rank(), cl.num_blocks()};
  wing_fd_run(A, T, cap, s_itm, s_lo, s_pre, bg);
}

}  // namespace

// BE-Index of G (Sec. 2.3, "Construction of BE-Index"): per-edge butterfly
// counts into sup (zeroed by the caller; Alg. 1) and counters into cctr[0..2],
// then the blooms (k0, first pair boff), their twin pairs (pe1, pe2, pbloom)
// and the edge -> pair lists (eoff, elink).
void be_index_build(Arena &a, const Graph &G, unsigned long long *sup, uint64_t *cctr, BEIndex &I, int scratch) {
  const int T = 256;
  const int sms = num_sms();
  const unsigned cap = 16 * sms;
  const uint32_t m = G.m, n = G.n;
  uint64_t *cnt_lab = a.zeros<uint64_t>(n);
  ull *be_nb = a.zeros<ull>((size_t)n + 1), *be_np = a.zeros<ull>((size_t)n + 1);
  CountOut co;
  co.cnt_lab = cnt_lab;
  co.cnt_e = (uint64_t *)sup;
  co.wedges = cctr;
  co.be_nb = (uint64_t *)be_nb;
  co.be_np = (uint64_t *)be_np;
  co.scratch = scratch;
  count_butterflies(a, G, co);
  a.free(cnt_lab);
  ull *bb = a.alloc<ull>((size_t)n + 1), *pb = a.alloc<ull>((size_t)n + 1);
  exclusive_scan_u64(a, (const uint64_t *)be_nb, (uint64_t *)bb, n);
  exclusive_scan_u64(a, (const uint64_t *)be_np, (uint64_t *)pb, n);
  ull tot[2];
  CK(cudaMemcpyAsync(&tot[0], bb + n, 8, cudaMemcpyDeviceToHost, a.st));
  CK(cudaMemcpyAsync(&tot[1], pb + n, 8, cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  uint64_t nblooms = tot[0], npairs = tot[1];
  if (nblooms >= (1ull << 32) || 2 * npairs >= (1ull << 32))
    fail(PBNG_EOVERFLOW, "BE-Index with %llu blooms and %llu twin pairs exceeds the 32-bit index limit",
         (unsigned long long)nblooms, (unsigned long long)npairs);
  const uint32_t nb = (uint32_t)nblooms;
  const size_t np = (size_t)npairs;
  uint32_t *k0 = a.alloc<uint32_t>((size_t)nb + 1), *boff = a.alloc<uint32_t>((size_t)nb + 1);
  uint32_t *pe1 = a.alloc<uint32_t>(np + 1), *pe2 = a.alloc<uint32_t>(np + 1), *pbloom = a.alloc<uint32_t>(np + 1);
  if (np) {
    FillArgs F{};
    F.off = G.lab_off;
    F.adj = G.lab_adj;
    F.eid = G.lab_eid;
    F.n = n;
    F.bb = bb;
    F.pb = pb;
    F.k0 = k0;
    F.boff = boff;
    F.pe1 = pe1;
    F.pe2 = pe2;
    ull *lists = a.alloc<ull>(2 * (size_t)n);
    unsigned *cnts = a.zeros<unsigned>(2);
    k_fill_classify<<<grid_for((size_t)n * 32, T, cap), T, 0, a.st>>>(G.lab_off, G.lab_adj, n, be_np, lists, cnts);
    CK_LAUNCH();
    unsigned hc[2];
    CK(cudaMemcpyAsync(hc, cnts, sizeof(hc), cudaMemcpyDeviceToHost, a.st));
    CK(cudaStreamSynchronize(a.st));
    static bool attr = false;
    if (!attr) {
      CK(cudaFuncSetAttribute(k_fill_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fill_warp_smem()));
      attr = true;
    }
    if (hc[0]) {
      k_fill_warp<<<grid_for((size_t)hc[0] * 32, FWT, 6 * sms), FWT, fill_warp_smem(), a.st>>>(F, lists, cnts);
      CK_LAUNCH();
    }
    if (hc[1]) {
      unsigned grid = std::min<unsigned>(hc[1], 2 * sms);
      uint32_t *scr = a.zeros<uint32_t>((size_t)grid * 2 * n);
      k_fill_block<<<grid, FBT, 0, a.st>>>(F, lists + n, cnts + 1, scr);
      CK_LAUNCH();
      a.free(scr);
    }
    a.free(lists);
    a.free(cnts);
  }
  {
    uint32_t npu = (uint32_t)np;
    CK(cudaMemcpyAsync(boff + nb, &npu, 4, cudaMemcpyHostToDevice, a.st));
  }
  if (nb) {
    k_pair_bloom<<<grid_for(nb, T, cap), T, 0, a.st>>>(k0, boff, nb, pbloom);
    CK_LAUNCH();
  }
  // edge -> pair lists
  uint32_t *deg = a.zeros<uint32_t>((size_t)m + 1), *eoff = a.alloc<uint32_t>((size_t)m + 1);
  uint32_t *elink = a.alloc<uint32_t>(2 * np + 1);
  if (np) {
    k_link_deg<<<grid_for(np, T, cap), T, 0, a.st>>>(pe1, pe2, np, deg);
    CK_LAUNCH();
  }
  exclusive_scan_u32(a, deg, eoff, m);
  if (np) {
    CK(cudaMemsetAsync(deg, 0, (size_t)m * 4, a.st));
    k_link_fill<<<grid_for(np, T, cap), T, 0, a.st>>>(pe1, pe2, np, eoff, deg, elink);
    CK_LAUNCH();
  }
  a.free(deg);
  a.free(bb);
  a.free(pb);
  a.free(be_nb);
  a.free(be_np);
  I.nb = nb;
  I.np = np;
  I.k0 = k0;
  I.boff = boff;
  I.pe1 = pe1;
  I.pe2 = pe2;
  I.pbloom = pbloom;
  I.eoff = eoff;
  I.elink = elink;
}

namespace {
// Prop. 1-2 sums of the BE-Index: per edge, sum over its blooms of (k_B - 1);
// over all blooms, sum of C(k_B, 2)
__global__ void k_be_edge_sums(const uint32_t *pe1, const uint32_t *pe2, const uint32_t *pbloom, const uint32_t *k0,
                               size_t np, ull *out_e) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < np; q += (size_t)gridDim.x * blockDim.x) {
    ull k = k0[pbloom[q]] - 1ull;
    atomicAdd(&out_e[pe1[q]], k);
    atomicAdd(&out_e[pe2[q]], k);
  }
}

__global__ void k_be_bloom_sum(const uint32_t *k0, uint32_t nb, ull *out) {
  ull s = 0;
  for (size_t b = blockIdx.x * (size_t)blockDim.x + threadIdx.x; b < nb; b += (size_t)gridDim.x * blockDim.x) {
    ull k = k0[b];
    s += k * (k - 1) / 2;
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}
}  // namespace

void be_index_sums(Arena &a, const Graph &G, uint64_t *out_e, uint64_t *total, pbng_stats *st) {
  const int T = 256;
  const unsigned cap = 16 * num_sms();
  const uint32_t m = G.m;
  *total = 0;
  if (m == 0) return;
  ull *sup = a.zeros<ull>(m);
  uint64_t *cctr = a.zeros<uint64_t>(4);
  BEIndex I;
  be_index_build(a, G, sup, cctr, I, PBNG_SCRATCH_AUTO);
  CK(cudaMemsetAsync(out_e, 0, (size_t)m * 8, a.st));
  ull *tot = a.zeros<ull>(1);
  if (I.np) {
    k_be_edge_sums<<<grid_for(I.np, T, cap), T, 0, a.st>>>(I.pe1, I.pe2, I.pbloom, I.k0, I.np, (ull *)out_e);
    CK_LAUNCH();
  }
  if (I.nb) {
    k_be_bloom_sum<<<grid_for(I.nb, T, cap), T, 0, a.st>>>(I.k0, I.nb, tot);
    CK_LAUNCH();
  }
  CK(cudaMemcpyAsync(total, tot, 8, cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  if (st) {
    st->links = 2 * (uint64_t)I.np;
    st->blooms = I.nb;
  }
}

// --------------------------------------------------------------- driver
namespace {
// warp per U vertex: min(d_u, d_v) for each of its edges
__global__ void k_edge_min_deg(const uint32_t *u_off, const uint32_t *u_adj, const uint32_t *v_off, uint32_t nu,
                               uint32_t *out) {
  const int lane = threadIdx.x & 31;
  size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5, nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t u = gw; u < nu; u += nw) {
    const uint32_t o = u_off[u], du = u_off[u + 1] - o;
    for (uint32_t k = lane; k < du; k += 32) {
      const uint32_t v = u_adj[o + k];
      out[o + k] = min(du, v_off[v + 1] - v_off[v]);
    }
  }
}

// work proxy (support) of the remaining edges with support below a bound
__global__ void k_wing_work_below(const uint32_t *alist, uint32_t na, const ull *sup, ull bound, ull *out) {
  ull s = 0;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < na; j += (size_t)gridDim.x * blockDim.x) {
    const ull v = sup[alist[j]];
    if (v < bound) s += v;
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}
}  // namespace

void edge_min_degrees(Arena &a, const Graph &G, uint32_t *out) {
  if (!G.m) return;
  const int T = 256;
  k_edge_min_deg<<<grid_for((size_t)G.nu * 32, T, 16 * num_sms()), T, 0, a.st>>>(G.u_off, G.u_adj, G.v_off, G.nu, out);
  CK_LAUNCH();
}

void wing_decompose(Arena &a, Graph &G, const TipParams &prm, uint64_t *theta_out, pbng_stats *st) {
  const int T = 256;
  const int sms = num_sms();
  const unsigned cap = 16 * sms;
  uint32_t m = G.m, n = G.n;
  if (m == 0) return;
  cudaEvent_t ev[5];
  for (auto &e : ev) CK(cudaEventCreate(&e));
  CK(cudaEventRecord(ev[0], a.st));

  // ---- per-edge counts and the BE-Index (Alg. 1 + Sec. 2.3 construction)
  ull *sup = a.zeros<ull>(m), *init = a.alloc<ull>(m);
  uint64_t *cctr = a.zeros<uint64_t>(4);
  BEIndex I;
  be_index_build(a, G, sup, cctr, I, prm.count_scratch);
  const uint32_t nb = I.nb;
  const size_t np = I.np;
  uint32_t *k0 = I.k0, *boff = I.boff, *pe1 = I.pe1, *pe2 = I.pe2, *pbloom = I.pbloom, *eoff = I.eoff,
           *elink = I.elink;
  CK(cudaEventRecord(ev[1], a.st));

  // ---- coarse phase
  uint8_t *state = a.zeros<uint8_t>(m), *palive = a.alloc<uint8_t>(np + 1);
  CK(cudaMemsetAsync(palive, 1, np + 1, a.st));
  uint32_t *part = a.alloc<uint32_t>(m);
  uint32_t *kcur = a.alloc<uint32_t>((size_t)nb + 1), *cntB = a.zeros<uint32_t>((size_t)nb + 1);
  uint32_t *blen = a.alloc<uint32_t>((size_t)nb + 1), *bq = a.alloc<uint32_t>(np + 1);
  CK(cudaMemcpyAsync(kcur, k0, ((size_t)nb + 1) * 4, cudaMemcpyDeviceToDevice, a.st));
  CK(cudaMemcpyAsync(blen, k0, ((size_t)nb + 1) * 4, cudaMemcpyDeviceToDevice, a.st));
  if (np) {
    k_iota<<<grid_for(np, T, cap), T, 0, a.st>>>(bq, np);
    CK_LAUNCH();
  }
  uint32_t *alist = a.alloc<uint32_t>(m), *alist2 = a.alloc<uint32_t>(m);
  k_iota<<<grid_for(m, T, cap), T, 0, a.st>>>(alist, m);
  CK_LAUNCH();
  uint32_t *front = a.alloc<uint32_t>(m), *front2 = a.alloc<uint32_t>(m);
  uint32_t *touched = a.alloc<uint32_t>((size_t)nb + 1);
  unsigned *dc = a.zeros<unsigned>(16);
  ull *wctr = a.zeros<ull>(8);  // [0] CD links, [1] CD updates, [4] FD links, [5] FD updates, [6] FD steps
  RangeState *rs = a.zeros<RangeState>(1);
  ull *wl = a.alloc<ull>(m);
  CDArgs A{};
  A.pe1 = pe1;
  A.pe2 = pe2;
  A.pbloom = pbloom;
  A.eoff = eoff;
  A.elink = elink;
  A.boff = boff;
  A.kcur = kcur;
  A.cntB = cntB;
  A.bq = bq;
  A.blen = blen;
  A.palive = palive;
  A.state = state;
  A.sup = sup;
  A.theta_hi = (const ull *)&rs->theta_hi;
  A.touched = touched;
  A.touched_n = dc + 2;
  A.ctr = wctr;

  // learned bounds: features of the initial supports and edge degrees ->
  // MLP -> bounds, each judged by the estimator in its range
  std::vector<uint64_t> learned;
  const uint64_t *bounds = prm.bounds;
  uint32_t n_bounds = prm.bounds_mode == PBNG_BOUNDS_EXPLICIT ? prm.n_bounds : 0;
  const bool is_learned = prm.bounds_mode == PBNG_BOUNDS_LEARNED;
  if (is_learned) {
    float *feat = a.alloc<float>(128);
    uint32_t *edeg = a.alloc<uint32_t>(m);
    edge_min_degrees(a, G, edeg);
    const uint64_t K = bound_features(a, (const uint64_t *)sup, nullptr, m, feat, edeg);
    learned = propose_bounds(a, prm.mlp_params, prm.mlp_hidden, prm.mlp_out, feat, K);
    a.free(edeg);
    a.free(feat);
    bounds = learned.data();
    n_bounds = (uint32_t)learned.size();
  }
  uint32_t na = m, pi = 0, P = prm.P;
  double scale = 1.0;
  uint64_t prev_init_est = 0, rounds = 0, front_total = 0;
  ull cur_final = 0;
  while (na > 0) {
    if (pi > 0) {
      CK(cudaMemsetAsync(dc + 7, 0, 4, a.st));
      k_wing_compact_list<<<grid_for(na, T, cap), T, 0, a.st>>>(alist, na, state, alist2, dc + 7);
      CK_LAUNCH();
      na = fetch(a, dc + 7);
      std::swap(alist, alist2);
      if (na == 0) break;
    }
    bool last = pi + 1 >= P;
    CK(cudaMemsetAsync(rs, 0, sizeof(RangeState), a.st));
    set_u64(a, (uint64_t *)&rs->kmin, ~0ull);
    k_wing_weights<<<grid_for(na, T, cap), T, 0, a.st>>>(alist, na, sup, wl, rs);
    CK_LAUNCH();
    ull hk[3];
    CK(cudaMemcpyAsync(hk, &rs->kmin, sizeof(hk), cudaMemcpyDeviceToHost, a.st));
    CK(cudaMemcpyAsync(&cur_final, wctr + 3, 8, cudaMemcpyDeviceToHost, a.st));
    CK(cudaStreamSynchronize(a.st));
    CK(cudaMemsetAsync(wctr + 3, 0, 8, a.st));
    ull kmin = hk[0], kmax = hk[1], wsum = hk[2];
    if (pi > 0 && cur_final > 0) {
      scale = (double)prev_init_est / (double)cur_final;
      if (scale > 1.0 || scale <= 0.0) scale = 1.0;
    }
    ull thi = 0;
    uint64_t init_est = 0;
    bool use_est = true;
    if (last) {
      thi = ~0ull;
      use_est = false;
    } else if (pi < n_bounds && bounds[pi] > kmin) {
      thi = bounds[pi];
      use_est = false;
      if (is_learned && prm.learned_vet > 0 && wsum > 0) {
        // the plain estimator judges a learned bound: its range may hold at
        // most learned_vet times the estimator's target work
        const double t = (double)wsum * scale / (double)(P - pi);
        ull *d = a.zeros<ull>(1), wb = 0;
        k_wing_work_below<<<grid_for(na, T, cap), T, 0, a.st>>>(alist, na, sup, thi, d);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(&wb, d, 8, cudaMemcpyDeviceToHost, a.st));
        CK(cudaStreamSynchronize(a.st));
        a.free(d);
        if ((double)wb > prm.learned_vet * std::max(t, 1.0)) use_est = true;
        else init_est = wb;
      }
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
    if (prm.bounds_used && !last) prm.bounds_used->push_back(thi);
    CK(cudaMemsetAsync(dc, 0, 4, a.st));
    k_wing_scan<<<grid_for(na, T, cap), T, 0, a.st>>>(alist, na, state, sup, init, (const ull *)&rs->theta_hi, front, dc);
    CK_LAUNCH();
    uint32_t nf = fetch(a, dc);
    while (nf > 0) {
      rounds++;
      front_total += nf;
      CK(cudaMemsetAsync(dc + 1, 0, 8, a.st));  // next frontier size, touched blooms
      A.next = front2;
      A.next_n = dc + 1;
      // the whole active set must be visible before the twin rule is applied
      k_wing_mark<<<grid_for(nf, T, cap), T, 0, a.st>>>(front, nf, state, ST_ACTIVE);
      CK_LAUNCH();
      g_prof.begin(PROF_PEEL);
      k_wing_pass1<<<grid_for((size_t)nf * 32, T, cap), T, 0, a.st>>>(A, front, nf, part, pi);
      CK_LAUNCH();
      k_wing_pass2<<<8 * sms, T, 0, a.st>>>(A, prm.compact);
      CK_LAUNCH();
      g_prof.end();
      k_wing_mark<<<grid_for(nf, T, cap), T, 0, a.st>>>(front, nf, state, ST_PEELED);
      CK_LAUNCH();
      nf = fetch(a, dc + 1);
      std::swap(front, front2);
    }
    pi++;
  }
  uint32_t nparts = pi;
  CK(cudaEventRecord(ev[2], a.st));

  // ---- partition_BE_Index (Alg. 5 lines 12-25)
  int bp = bits_for(nparts);
  uint32_t *pcnt = a.zeros<uint32_t>((size_t)nparts + 1), *ps = a.alloc<uint32_t>((size_t)nparts + 1);
  k_hist_u32<<<grid_for(m, T, cap), T, 0, a.st>>>(part, m, pcnt);
  CK_LAUNCH();
  exclusive_scan_u32(a, pcnt, ps, nparts);
  uint32_t *es = a.alloc<uint32_t>(m);
  {
    uint64_t *key = a.alloc<uint64_t>(m);
    k_edge_keys<<<grid_for(m, T, cap), T, 0, a.st>>>(part, m, key, es);
    CK_LAUNCH();
    sort_pairs(a, key, es, m, bp);
    a.free(key);
  }
  uint32_t *pmin = a.alloc<uint32_t>(np + 1), *order = a.alloc<uint32_t>(np + 1), *pb_of = a.alloc<uint32_t>(np + 1);
  uint32_t ngroups = 0;
  uint32_t *gstart = nullptr, *gk = nullptr, *gpart = nullptr;
  if (np) {
    uint64_t *key = a.alloc<uint64_t>(np);
    k_pmin<<<grid_for(np, T, cap), T, 0, a.st>>>(pe1, pe2, pbloom, np, part, bp, key, order, pmin);
    CK_LAUNCH();
    sort_pairs(a, key, order, np, bits_for(nb) + bp);
    uint32_t *head = a.alloc<uint32_t>(np + 1), *gidx = a.alloc<uint32_t>(np + 1);
    k_group_heads<<<grid_for(np, T, cap), T, 0, a.st>>>(key, np, head);
    CK_LAUNCH();
    exclusive_scan_u32(a, head, gidx, np);
    ngroups = fetch(a, gidx + np);
    gstart = a.alloc<uint32_t>((size_t)ngroups + 1);
    gk = a.alloc<uint32_t>((size_t)ngroups + 1);
    gpart = a.alloc<uint32_t>((size_t)ngroups + 1);
    k_groups<<<grid_for(np, T, cap), T, 0, a.st>>>(key, order, np, gidx, head, k0, boff, bp, gstart, gk, gpart, pb_of);
    CK_LAUNCH();
    uint32_t npu = (uint32_t)np;
    CK(cudaMemcpyAsync(gstart + ngroups, &npu, 4, cudaMemcpyHostToDevice, a.st));
    a.free(head);
    a.free(gidx);
    a.free(key);
  } else {
    gstart = a.zeros<uint32_t>(1);
    gk = a.zeros<uint32_t>(1);
    gpart = a.zeros<uint32_t>(1);
  }
  uint32_t *gpc = a.zeros<uint32_t>((size_t)nparts + 1), *gps = a.alloc<uint32_t>((size_t)nparts + 1);
  if (ngroups) {
    k_hist_u32<<<grid_for(ngroups, T, cap), T, 0, a.st>>>(gpart, ngroups, gpc);
    CK_LAUNCH();
  }
  exclusive_scan_u32(a, gpc, gps, nparts);
  ull *work = a.zeros<ull>(nparts);
  k_part_work<<<grid_for(m, T, cap), T, 0, a.st>>>(part, init, m, work);
  CK_LAUNCH();
  std::vector<ull> hwork(nparts);
  CK(cudaMemcpyAsync(hwork.data(), work, (size_t)nparts * 8, cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  // LPT order (heaviest first), split into partitions large enough for a
  // cluster of blocks and the rest (one block each)
  std::vector<uint32_t> hps(nparts + 1);
  CK(cudaMemcpyAsync(hps.data(), ps, ((size_t)nparts + 1) * 4, cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  std::vector<uint32_t> ord(nparts);
  for (uint32_t i = 0; i < nparts; i++) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) { return hwork[x] > hwork[y]; });
  const FDClusterShape fc = fd_cluster_shape((const void *)k_wing_fd_cluster, WFT, 0);
  std::vector<uint32_t> heavy, light;
  for (uint32_t i : ord) (fc.size > 1 && hps[i + 1] - hps[i] >= prm.fd_cluster_min ? heavy : light).push_back(i);
  std::vector<uint32_t> both(heavy);
  both.insert(both.end(), light.begin(), light.end());
  uint32_t *dord = a.alloc<uint32_t>(nparts);
  CK(cudaMemcpyAsync(dord, both.data(), (size_t)nparts * 4, cudaMemcpyHostToDevice, a.st));
  CK(cudaEventRecord(ev[3], a.st));

  // ---- fine phase (Alg. 5 lines 1-11)
  CK(cudaMemcpyAsync(sup, init, (size_t)m * 8, cudaMemcpyDeviceToDevice, a.st));
  k_fd_reset<<<grid_for(std::max(np, (size_t)m), T, cap), T, 0, a.st>>>(palive, np, state, m);
  CK_LAUNCH();
  uint32_t *gcnt = a.zeros<uint32_t>((size_t)ngroups + 1), *gtouch = a.alloc<uint32_t>(2 * (size_t)ngroups + 2);
  WFDArgs W{};
  W.pe1 = pe1;
  W.pe2 = pe2;
  W.eoff = eoff;
  W.elink = elink;
  W.pmin = pmin;
  W.pb_of = pb_of;
  W.order = order;
  W.gstart = gstart;
  W.gps = gps;
  W.part = part;
  W.es = es;
  W.ps = ps;
  W.orderp = dord;
  W.gk = gk;
  W.gcnt = gcnt;
  W.palive = palive;
  W.state = state;
  W.sup = sup;
  W.theta = (ull *)theta_out;
  W.buf_a = alist;
  W.buf_b = alist2;
  W.buf_c = a.alloc<uint32_t>(m);
  W.buf_d = a.alloc<uint32_t>(m);
  W.buf_f = front;
  W.gtouch = gtouch;
  W.nparts = nparts;
  W.queue = dc + 8;
  CK(cudaMemsetAsync(dc + 8, 0, 8, a.st));  // queues of the light and heavy partitions
  W.ctr = wctr + 4;
  ull *pstat = a.zeros<ull>((size_t)WFD_PSTAT * nparts);
  W.pstat = pstat;
  {
    uint32_t *fdeg = a.zeros<uint32_t>((size_t)m + 1), *foff = a.alloc<uint32_t>((size_t)m + 1);
    k_flink_count<<<grid_for((size_t)m * 32, T, cap), T, 0, a.st>>>(eoff, elink, pmin, part, m, fdeg);
    CK_LAUNCH();
    exclusive_scan_u32(a, fdeg, foff, m);
    uint32_t nfl = fetch(a, foff + m);
    uint32_t *flink = a.alloc<uint32_t>((size_t)nfl + 1);
    k_flink_fill<<<grid_for((size_t)m * 32, T, cap), T, 0, a.st>>>(eoff, elink, pmin, part, m, foff, flink);
    CK_LAUNCH();
    a.free(fdeg);
    W.foff = foff;
    W.flink = flink;
    uint32_t *glen = a.alloc<uint32_t>((size_t)ngroups + 1);
    if (ngroups) {
      k_group_len<<<grid_for(ngroups, T, cap), T, 0, a.st>>>(gstart, ngroups, glen);
      CK_LAUNCH();
    }
    W.glen = glen;
    W.order_w = order;
  }
  g_prof.begin(PROF_FD);
  {
    // heavy partitions: clusters of fc.size blocks on a side stream; the rest:
    // one block each on the call's stream, concurrently
    const uint32_t nh = (uint32_t)heavy.size(), nl = (uint32_t)light.size();
    const uint32_t ncl = std::min<uint32_t>(nh, fc.max_clusters);
    SideLaunch side(a.st, ncl > 0);
    if (ncl) {
      WFDArgs WH = W;
      WH.orderp = dord;
      WH.nparts = nh;
      WH.queue = dc + 9;
      CK(launch_cluster((const void *)k_wing_fd_cluster, ncl, fc.size, WFT, 0, side.st, WH, WIN_CAP_BIG));
      CK_LAUNCH();
    }
    if (nl) {
      WFDArgs WL = W;
      WL.orderp = dord + nh;
      WL.nparts = nl;
      unsigned blocks = std::max<unsigned>(1u, std::min<unsigned>(nl, 2 * sms - ncl * fc.size));
      k_wing_fd<<<blocks, WFT, 0, a.st>>>(WL, 4 * WIN_CAP);
      CK_LAUNCH();
    }
  }
  g_prof.end();
  CK(cudaEventRecord(ev[4], a.st));
  CK(cudaStreamSynchronize(a.st));
  if (const char *tp = getenv("PBNG_TRACE")) {  // fine-phase line per partition: partition |E_p| work steps cycles
    if (FILE *f = fopen(tp, "a")) {
      std::vector<ull> pst((size_t)WFD_PSTAT * nparts);
      CK(cudaMemcpy(pst.data(), pstat, pst.size() * 8, cudaMemcpyDeviceToHost));
      // partition |E_p| work steps cycles | cycles of select, pass 1, pass 2, rest | rescans
      for (uint32_t i = 0; i < nparts; i++) {
        const ull *q = &pst[(size_t)WFD_PSTAT * i];
        fprintf(f, "W %u %u %llu %llu %llu %llu %llu %llu %llu %llu\n", i, hps[i + 1] - hps[i],
                (unsigned long long)hwork[i], q[0], q[1], q[2], q[3], q[4], q[5], q[6]);
      }
      fclose(f);
    }
  }
  if (st) {
    ull hw[8];
    uint64_t hcc[3];
    CK(cudaMemcpy(hw, wctr, sizeof(hw), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hcc, cctr, sizeof(hcc), cudaMemcpyDeviceToHost));
    float t01, t12, t23, t34;
    cudaEventElapsedTime(&t01, ev[0], ev[1]);
    cudaEventElapsedTime(&t12, ev[1], ev[2]);
    cudaEventElapsedTime(&t23, ev[2], ev[3]);
    cudaEventElapsedTime(&t34, ev[3], ev[4]);
    st->wedges_count += hcc[0];
    st->wedges_cd += hw[0];  // wing: bloom-edge links traversed
    st->wedges_fd += hw[4];
    st->updates += hw[1] + hw[5];
    st->links += 2 * np;
    st->blooms += nb;
    st->rounds += rounds;
    st->fd_steps += hw[6];
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
    std::vector<ull> ps_h((size_t)WFD_PSTAT * nparts);
    CK(cudaMemcpy(ps_h.data(), pstat, ps_h.size() * 8, cudaMemcpyDeviceToHost));
    for (uint32_t i = 0; i < nparts; i++) {
      st->fd_part_steps_max = std::max<uint64_t>(st->fd_part_steps_max, ps_h[(size_t)WFD_PSTAT * i]);
      st->fd_part_cycles_max = std::max<uint64_t>(st->fd_part_cycles_max, ps_h[(size_t)WFD_PSTAT * i + 1]);
    }
    st->bytes_count += 4 * hcc[0] + 12 * hcc[1] + 16 * hcc[2];
    st->bytes_peel += 8 * hw[0] + 16 * hw[1] + 8 * front_total;
    st->bytes_fd += 8 * hw[4] + 16 * hw[5] + 8 * (uint64_t)m;
  }
  for (auto &e : ev) cudaEventDestroy(e);
}

}  // namespace pbng
