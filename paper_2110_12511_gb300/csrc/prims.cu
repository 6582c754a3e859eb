// Device primitives: errors, stream-ordered arena, exclusive scans, stable
// LSD radix sort of (uint64 key, uint32 value) pairs, reductions.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <algorithm>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace pbng {

// ------------------------------------------------------------------ errors
thread_local char g_detail[512];
thread_local uint64_t g_launches = 0;
thread_local Prof g_prof;

// --------------------------------------------------------------- profiling
void Prof::begin(int group) {
  if (!on) return;
  Span s;
  s.group = group;
  cudaEventCreate(&s.a);
  cudaEventCreate(&s.b);
  cudaEventRecord(s.a, st);
  spans.push_back(s);
  cur = group;
  l0 = g_launches;
}

void Prof::end() {
  if (!on || cur < 0) return;
  cudaEventRecord(spans.back().b, st);
  launches[cur] += g_launches - l0;
  cur = -1;
}

void Prof::collect(uint64_t ns[PROF_NGROUPS]) {
  for (int i = 0; i < PROF_NGROUPS; i++) ns[i] = 0;
  if (!spans.empty()) cudaEventSynchronize(spans.back().b);
  for (auto &s : spans) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, s.a, s.b) == cudaSuccess) ns[s.group] += (uint64_t)((double)ms * 1e6);
    cudaEventDestroy(s.a);
    cudaEventDestroy(s.b);
  }
  cudaGetLastError();
  spans.clear();
}

void fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
  va_end(ap);
  throw Error{code};
}

void cuda_check(cudaError_t e, const char *what, const char *file, int line) {
  if (e == cudaSuccess) return;
  cudaGetLastError();  // clear a sticky-free error so the next call starts clean
  const char *f = strrchr(file, '/');
  if (e == cudaErrorMemoryAllocation)
    fail(PBNG_ENOMEM, "%s: %s (%s:%d)", what, cudaGetErrorString(e), f ? f + 1 : file, line);
  fail(PBNG_ECUDA, "%s: %s (%s:%d)", what, cudaGetErrorString(e), f ? f + 1 : file, line);
}

// ------------------------------------------------------------------- arena
void *Arena::raw(size_t nbytes) {
  void *p = nullptr;
  size_t nb = nbytes ? (nbytes + 255) & ~size_t(255) : 256;
  cudaError_t e = cudaMallocAsync(&p, nb, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(PBNG_ENOMEM, "device allocation of %zu bytes failed (%s)", nb, cudaGetErrorString(e));
  }
  ptrs.push_back(p);
  bytes += nb;
  if (bytes > peak) peak = bytes;
  return p;
}

void Arena::free(void *p) {
  for (size_t i = 0; i < ptrs.size(); i++)
    if (ptrs[i] == p) {
      cudaFreeAsync(p, st);
      ptrs[i] = ptrs.back();
      ptrs.pop_back();
      return;
    }
}

Arena::~Arena() {
  for (void *p : ptrs) cudaFreeAsync(p, st);
  ptrs.clear();
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

void init_device_pool() {
  static int done_dev = -1;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (done_dev == dev) return;
  cudaMemPool_t pool;
  CK(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t thr = UINT64_MAX;  // keep freed blocks for reuse by later calls
  CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  done_dev = dev;
}

// -------------------------------------------------------------------- scan
namespace {
constexpr int SCAN_T = 256, SCAN_I = 16, SCAN_TILE = SCAN_T * SCAN_I;

template <class T>
__device__ T warp_incl_scan(T x) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// exclusive scan of one value per thread across the block; returns the
// block total in *total
template <class T>
__device__ T block_excl_scan(T x, T *total) {
  __shared__ T wsum[SCAN_T / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = warp_incl_scan(x);
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    T s = lane < SCAN_T / 32 ? wsum[lane] : T(0);
    T si = warp_incl_scan(s);
    if (lane < SCAN_T / 32) wsum[lane] = si - s;
    if (lane == SCAN_T / 32 - 1) *total = si;
  }
  __syncthreads();
  T r = inc - x + wsum[w];
  __syncthreads();
  return r;
}

template <class Tin, class Tout>
__global__ void k_tile_sums(const Tin *in, size_t n, Tout *sums) {
  size_t base = (size_t)blockIdx.x * SCAN_TILE;
  Tout s = 0;
  for (int j = 0; j < SCAN_I; j++) {
    size_t i = base + (size_t)j * SCAN_T + threadIdx.x;
    if (i < n) s += (Tout)in[i];
  }
  __shared__ Tout tot;
  block_excl_scan<Tout>(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// each thread owns SCAN_I consecutive items of the tile
template <class Tin, class Tout>
__global__ void k_tile_scan(const Tin *in, size_t n, Tout *out, const Tout *tile_off) {
  size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_I;
  Tout v[SCAN_I];
  Tout s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_I; j++) {
    size_t i = base + j;
    v[j] = i < n ? (Tout)in[i] : Tout(0);
    s += v[j];
  }
  __shared__ Tout tot;
  Tout pre = block_excl_scan<Tout>(s, &tot) + (tile_off ? tile_off[blockIdx.x] : Tout(0));
#pragma unroll
  for (int j = 0; j < SCAN_I; j++) {
    size_t i = base + j;
    if (i < n) out[i] = pre;
    pre += v[j];
  }
  if (base <= n && n < base + SCAN_I) out[n] = pre;  // total goes to out[n]
  if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

template <class Tin, class Tout>
void scan_impl(Arena &a, const Tin *in, Tout *out, size_t n) {
  size_t tiles = (n + SCAN_TILE) / SCAN_TILE;  // covers index n
  if (tiles <= 1) {
    k_tile_scan<Tin, Tout><<<1, SCAN_T, 0, a.st>>>(in, n, out, nullptr);
    CK_LAUNCH();
    return;
  }
  Tout *sums = a.alloc<Tout>(tiles + 1);
  k_tile_sums<Tin, Tout><<<(unsigned)tiles, SCAN_T, 0, a.st>>>(in, n, sums);
  CK_LAUNCH();
  scan_impl<Tout, Tout>(a, sums, sums, tiles);  // in-place is safe: each tile reads before writing
  k_tile_scan<Tin, Tout><<<(unsigned)tiles, SCAN_T, 0, a.st>>>(in, n, out, sums);
  CK_LAUNCH();
  a.free(sums);
}
}  // namespace

void exclusive_scan_u32(Arena &a, const uint32_t *in, uint32_t *out, size_t n) { scan_impl<uint32_t, uint32_t>(a, in, out, n); }
void exclusive_scan_u32_to_u64(Arena &a, const uint32_t *in, uint64_t *out, size_t n) {
  scan_impl<uint32_t, uint64_t>(a, in, out, n);
}
void exclusive_scan_u64(Arena &a, const uint64_t *in, uint64_t *out, size_t n) { scan_impl<uint64_t, uint64_t>(a, in, out, n); }

// -------------------------------------------------------------- radix sort
namespace {
constexpr int RS_T = 256, RS_I = 16, RS_TILE = RS_T * RS_I, RS_W = RS_T / 32;

__global__ void k_rs_hist(const uint64_t *keys, size_t n, int shift, uint32_t *hist, uint32_t ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  size_t base = (size_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int j = 0; j < RS_I; j++) {
    size_t i = base + (size_t)j * RS_T + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: items are ranked in position order (rounds of
// RS_T items, warps in order, lanes in order).
__global__ void k_rs_scatter(const uint64_t *kin, const uint32_t *vin, uint64_t *kout, uint32_t *vout, size_t n,
                             int shift, const uint32_t *hscan, uint32_t ntiles) {
  __shared__ uint32_t s_off[256];
  __shared__ uint32_t s_w[RS_W][256];
  int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  s_off[tid] = hscan[(size_t)tid * ntiles + blockIdx.x];
  size_t base = (size_t)blockIdx.x * RS_TILE;
  for (int j = 0; j < RS_I; j++) {
#pragma unroll
    for (int w = 0; w < RS_W; w++) s_w[w][tid] = 0;
    __syncthreads();
    size_t i = base + (size_t)j * RS_T + tid;
    bool valid = i < n;
    uint64_t k = valid ? kin[i] : 0;
    uint32_t v = valid ? vin[i] : 0;
    uint32_t d = valid ? (uint32_t)((k >> shift) & 255u) : 256u;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lane == __ffs(peers) - 1) s_w[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = s_off[tid];
#pragma unroll
      for (int w = 0; w < RS_W; w++) {
        uint32_t c = s_w[w][tid];
        s_w[w][tid] = run;
        run += c;
      }
      s_off[tid] = run;
    }
    __syncthreads();
    if (valid) {
      uint32_t dst = s_w[warp][d] + rank;
      kout[dst] = k;
      vout[dst] = v;
    }
    __syncthreads();
  }
}
}  // namespace

void sort_pairs(Arena &a, uint64_t *keys, uint32_t *vals, size_t n, int key_bits) {
  if (n <= 1 || key_bits <= 0) return;
  if (n >= (1ull << 32)) fail(PBNG_EINVAL, "sort of %zu items exceeds 2^32", n);
  int passes = (key_bits + 7) / 8;
  uint32_t ntiles = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
  uint64_t *k2 = a.alloc<uint64_t>(n);
  uint32_t *v2 = a.alloc<uint32_t>(n);
  uint32_t *hist = a.alloc<uint32_t>((size_t)256 * ntiles + 1);
  uint64_t *ks = keys, *kd = k2;
  uint32_t *vs = vals, *vd = v2;
  for (int p = 0; p < passes; p++) {
    int shift = 8 * p;
    k_rs_hist<<<ntiles, RS_T, 0, a.st>>>(ks, n, shift, hist, ntiles);
    CK_LAUNCH();
    exclusive_scan_u32(a, hist, hist, (size_t)256 * ntiles);
    k_rs_scatter<<<ntiles, RS_T, 0, a.st>>>(ks, vs, kd, vd, n, shift, hist, ntiles);
    CK_LAUNCH();
    uint64_t *tk = ks; ks = kd; kd = tk;
    uint32_t *tv = vs; vs = vd; vd = tv;
  }
  if (ks != keys) {
    CK(cudaMemcpyAsync(keys, ks, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, a.st));
    CK(cudaMemcpyAsync(vals, vs, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, a.st));
  }
  a.free(k2);
  a.free(v2);
  a.free(hist);
}

// --------------------------------------------------------------- reductions
namespace {
__global__ void k_sum_u64(const uint64_t *in, size_t n, unsigned long long *out) {
  unsigned long long s = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) s += in[i];
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}
__global__ void k_max_u32(const uint32_t *in, size_t n, unsigned *out) {
  unsigned s = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s = max(s, in[i]);
  for (int o = 16; o; o >>= 1) s = max(s, __shfl_down_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, s);
}
}  // namespace

uint64_t reduce_sum_u64(Arena &a, const uint64_t *in, size_t n) {
  unsigned long long *d = a.zeros<unsigned long long>(1);
  k_sum_u64<<<grid_for(n, 256, 4 * num_sms()), 256, 0, a.st>>>(in, n, d);
  CK_LAUNCH();
  uint64_t r = fetch(a, (const uint64_t *)d);
  a.free(d);
  return r;
}

uint32_t reduce_max_u32(Arena &a, const uint32_t *in, size_t n) {
  unsigned *d = a.zeros<unsigned>(1);
  k_max_u32<<<grid_for(n, 256, 4 * num_sms()), 256, 0, a.st>>>(in, n, d);
  CK_LAUNCH();
  uint32_t r = fetch(a, (const uint32_t *)d);
  a.free(d);
  return r;
}

FDClusterShape fd_cluster_shape(const void *kernel, int threads, size_t smem) {
  static std::vector<std::pair<const void *, FDClusterShape>> cache;
  for (auto &c : cache)
    if (c.first == kernel) return c.second;
  FDClusterShape fc;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) cudaGetLastError();
  for (uint32_t cs : {16u, 8u}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) == cudaSuccess && n > 0) {
      fc.size = cs;
      fc.max_clusters = std::max<uint32_t>(1u, std::min<uint32_t>((uint32_t)n, (uint32_t)num_sms() / (2 * cs)));
      break;
    }
    cudaGetLastError();
  }
  cache.push_back({kernel, fc});
  return fc;
}

SideLaunch::SideLaunch(cudaStream_t m, bool on) : main(m) {
  if (!on) return;
  CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CK(cudaEventRecord(ev, main));
  CK(cudaStreamWaitEvent(st, ev, 0));
}

SideLaunch::~SideLaunch() {
  if (!st) return;
  // (no throwing here: a failure shows up in the caller's next check)
  if (cudaEventRecord(ev, st) == cudaSuccess) cudaStreamWaitEvent(main, ev, 0);
  cudaEventDestroy(ev);
  cudaStreamDestroy(st);
}

}  // namespace pbng
