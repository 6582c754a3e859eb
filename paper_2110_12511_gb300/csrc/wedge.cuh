// Device building blocks for wedge traversal: a cooperative group (one warp
// or one thread block) that walks the wedges of one vertex in flattened
// order, and the per-vertex counter tables that aggregate wedges by endpoint
// (shared-memory hash, shared-memory dense array, global dense array).
#pragma once
#include <stdint.h>

namespace pbng {

constexpr uint32_t EMPTY_KEY = 0xffffffffu;

constexpr __host__ __device__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__device__ __forceinline__ uint64_t choose2(uint64_t c) { return c * (c - 1) / 2; }

__device__ __forceinline__ uint32_t hash32(uint32_t k) { return k * 0x9E3779B1u; }

// number of entries < b among a[0..len) (a sorted ascending)
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *a, uint32_t len, uint32_t b) {
  uint32_t lo = 0, hi = len;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < b) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// largest i in [0, n) with pre[i] <= w, for pre non-decreasing, pre[0] = 0
__device__ __forceinline__ int seg_of(const uint32_t *pre, int n, uint32_t w) {
  int lo = 0, hi = n;  // invariant: pre[lo] <= w, answer < hi
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pre[mid] <= w) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t nchunks(uint32_t len) { return (len + 31) >> 5; }

// Wedge walk over nseg slices of an adjacency array (slice i starts at lo[i]
// and holds len[i] entries); pre is the exclusive prefix of the slices'
// 32-entry chunk counts (pre[nseg] = C, the total).  The NT/32 warps of the
// group take contiguous runs of chunks: a warp finds the slice of its first
// chunk by binary search and then advances slice by slice, so a chunk costs a
// few warp instructions and its 32 reads are coalesced; four chunks are in
// flight per warp.  f(i, pos, v) is called for every entry, v = adj[pos].
template <int NT, class F>
__device__ __forceinline__ void walk_chunks(const uint32_t *__restrict__ adj, int rank, const uint32_t *lo,
                                            const uint32_t *len, const uint32_t *pre, int nseg, uint32_t C, F &&f) {
  constexpr uint32_t NW = NT / 32;
  const uint32_t lane = rank & 31, wid = rank >> 5;
  const uint32_t per = (C + NW - 1) / NW;
  uint32_t c = wid * per;
  const uint32_t ce = min(C, c + per);
  if (c >= ce) return;
  int i = seg_of(pre, nseg, c);
  for (; c + 3 < ce; c += 4) {
    uint32_t a[4];
    int si[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      while (pre[i + 1] <= c + u) i++;
      uint32_t off = ((c + u - pre[i]) << 5) + lane;
      si[u] = i;
      ok[u] = off < len[i];
      a[u] = lo[i] + off;
    }
    uint32_t v[4];
#pragma unroll
    for (int u = 0; u < 4; u++) v[u] = ok[u] ? __ldg(&adj[a[u]]) : 0u;
#pragma unroll
    for (int u = 0; u < 4; u++)
      if (ok[u]) f(si[u], a[u], v[u]);
  }
  for (; c < ce; c++) {
    while (pre[i + 1] <= c) i++;
    uint32_t off = ((c - pre[i]) << 5) + lane;
    if (off < len[i]) f(i, lo[i] + off, __ldg(&adj[lo[i] + off]));
  }
}

// ------------------------------------------------------------ groups
struct WarpGrp {
  static constexpr int N = 32;
  __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  // exclusive scan into pre[0..N], pre[N] = total; returns total
  __device__ __forceinline__ uint32_t scan(uint32_t x, uint32_t *pre) const {
    int l = rank();
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (l >= o) inc += y;
    }
    pre[l] = inc - x;
    if (l == 31) pre[32] = inc;
    __syncwarp();
    return __shfl_sync(0xffffffffu, inc, 31);
  }
  __device__ __forceinline__ uint64_t sum64(uint64_t x) const {
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  }
};

template <int NT>
struct BlockGrp {
  static constexpr int N = NT;
  uint32_t *ws;            // NT/32 + 1 words of shared scratch
  unsigned long long *ws64;  // NT/32 words
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ uint32_t scan(uint32_t x, uint32_t *pre) const {
    int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (l >= o) inc += y;
    }
    if (l == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
      uint32_t s = l < NT / 32 ? ws[l] : 0u, si = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, si, o);
        if (l >= o) si += y;
      }
      if (l < NT / 32) ws[l] = si - s;
      if (l == NT / 32 - 1) ws[NT / 32] = si;
    }
    __syncthreads();
    pre[threadIdx.x] = inc - x + ws[w];
    if (threadIdx.x == 0) pre[NT] = ws[NT / 32];
    __syncthreads();
    return pre[NT];
  }
  __device__ __forceinline__ uint64_t sum64(uint64_t x) const {
    int l = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (l == 0) ws64[w] = x;
    __syncthreads();
    uint64_t t = 0;
    if (threadIdx.x == 0)
      for (int i = 0; i < NT / 32; i++) t += ws64[i];
    __syncthreads();
    return t;  // valid in thread 0 only
  }
};

// NT threads of a block (warps base/32 ..) synchronised by named barrier
// `bar` (1..15; barrier 0 is __syncthreads)
template <int NT>
struct SubGrp {
  static constexpr int N = NT;
  int base, bar;
  uint32_t *ws;              // NT/32 + 2 words of shared scratch
  unsigned long long *ws64;  // NT/32 words (sum64 only)
  __device__ __forceinline__ int rank() const { return (int)threadIdx.x - base; }
  __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(NT) : "memory"); }
  __device__ __forceinline__ uint32_t scan(uint32_t x, uint32_t *pre) const {
    int r = rank(), l = r & 31, w = r >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (l >= o) inc += y;
    }
    if (l == 31) ws[w] = inc;
    sync();
    if (w == 0) {
      uint32_t s = l < NT / 32 ? ws[l] : 0u, si = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, si, o);
        if (l >= o) si += y;
      }
      if (l < NT / 32) ws[l] = si - s;
      if (l == NT / 32 - 1) ws[NT / 32] = si;
    }
    sync();
    pre[r] = inc - x + ws[w];
    if (r == 0) pre[NT] = ws[NT / 32];
    sync();
    return pre[NT];
  }
  __device__ __forceinline__ uint64_t sum64(uint64_t x) const {
    int r = rank(), l = r & 31, w = r >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (l == 0) ws64[w] = x;
    sync();
    uint64_t t = 0;
    if (r == 0)
      for (int i = 0; i < NT / 32; i++) t += ws64[i];
    sync();
    return t;  // valid in rank 0 only
  }
};

// --------------------------------------------------------------- tables
// Open-addressing hash of uint32 keys with uint32 counts in shared memory.
struct SmemHash {
  uint32_t *key, *val;
  uint32_t mask;  // capacity - 1 (power of two)
  __device__ __forceinline__ void inc(uint32_t k) const {
    uint32_t h = hash32(k) & mask;
    volatile uint32_t *vk = key;
    for (;;) {
      uint32_t cur = vk[h];
      if (cur == k) break;
      if (cur == EMPTY_KEY) {
        uint32_t prev = atomicCAS(&key[h], EMPTY_KEY, k);
        if (prev == EMPTY_KEY || prev == k) break;
      }
      h = (h + 1) & mask;
    }
    atomicAdd(&val[h], 1u);
  }
  __device__ __forceinline__ uint32_t get(uint32_t k) const {
    uint32_t h = hash32(k) & mask;
    for (;;) {
      uint32_t cur = key[h];
      if (cur == k) return val[h];
      if (cur == EMPTY_KEY) return 0;
      h = (h + 1) & mask;
    }
  }
};

static inline __host__ __device__ uint32_t pow2_at_least(uint32_t x) {
  uint32_t c = 1;
  while (c < x) c <<= 1;
  return c;
}

}  // namespace pbng
