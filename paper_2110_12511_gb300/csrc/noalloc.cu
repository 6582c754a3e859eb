// Per-vertex butterfly counts of one side without any device allocation.
//
// For callers that cannot allocate device memory themselves or through the
// library: code running under an allocator that must not grow, inside a
// pre-sized memory budget, or in a process whose allocations are owned by
// another framework.  The kernel is the dense-counter variant of the coarse
// peel kernel: one thread block per vertex u walks every wedge u -> v -> u',
// counts the common neighbours c(u, u') in a block-private slice of dense
// counters, then walks again, taking each counter back to zero with an
// atomic exchange, and sums C(c, 2) into the count of u.  The counters live
// in a file-scope device array of fixed size, shared by every call.
#include <cstdio>
#include <cstring>

#include "pbng.h"
#include "wedge.cuh"

namespace {

constexpr size_t NOALLOC_WORDS = size_t(16) << 20;  // 16 Mi uint32 counters = 64 MiB
constexpr int NT = 512;
constexpr int MAX_DEVICES = 64;

// Scratch of every call on a device: per-block dense counter slices.
// Host code must not use the name as an address (it is a host-side stand-in);
// the device address comes from cudaGetSymbolAddress at set-up.
static __device__ __align__(256) uint32_t g_noalloc_scratch[NOALLOC_WORDS];
static __device__ unsigned g_noalloc_err;

uint32_t *g_scratch_addr[MAX_DEVICES];
unsigned *g_err_addr[MAX_DEVICES];

}  // namespace

namespace pbng {
extern thread_local char g_detail[512];  // read by pbng_last_error_detail()
}

namespace {

int fail_with(int code, const char *msg) {
  snprintf(pbng::g_detail, sizeof(pbng::g_detail), "%s", msg);
  return code;
}

// bounds of both CSRs, so the counting kernel never reads out of range
__global__ void k_noalloc_validate(const uint64_t *u_off, const uint32_t *u_adj, uint32_t nu, const uint64_t *v_off,
                                   const uint32_t *v_adj, uint32_t nv, uint64_t m, unsigned *err) {
  size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
  for (size_t i = tid; i <= nu; i += nt) {
    uint64_t a = u_off[i];
    if ((i == 0 && a != 0) || (i == nu && a != m) || (i < nu && u_off[i + 1] < a) || a > m) atomicOr(err, 1u);
  }
  for (size_t i = tid; i <= nv; i += nt) {
    uint64_t a = v_off[i];
    if ((i == 0 && a != 0) || (i == nv && a != m) || (i < nv && v_off[i + 1] < a) || a > m) atomicOr(err, 1u);
  }
  for (size_t e = tid; e < m; e += nt) {
    if (u_adj[e] >= nv) atomicOr(err, 2u);
    if (v_adj[e] >= nu) atomicOr(err, 2u);
  }
}

// one block per vertex u; cnt = this block's slice of nu counters (all zero
// on entry and on exit)
__global__ void __launch_bounds__(NT) k_vertex_counts_noalloc(const uint64_t *u_off, const uint32_t *u_adj,
                                                               const uint64_t *v_off, const uint32_t *v_adj,
                                                               uint32_t nu, uint64_t *out, uint32_t *scratch) {
  __shared__ uint32_t lo[NT], pre[NT + 1];
  __shared__ uint32_t ws[NT / 32 + 2];
  __shared__ unsigned long long ws64[NT / 32];
  pbng::BlockGrp<NT> g{ws, ws64};
  uint32_t *cnt = scratch + (size_t)blockIdx.x * nu;
  for (uint32_t u = blockIdx.x; u < nu; u += gridDim.x) {
    uint64_t uo = u_off[u];
    uint32_t ud = (uint32_t)(u_off[u + 1] - uo);
    uint64_t sum = 0;
    for (int pass = 0; pass < 2; pass++) {
      for (uint32_t base = 0; base < ud; base += NT) {
        uint32_t r = threadIdx.x, l0 = 0, len = 0;
        if (base + r < ud) {
          uint32_t v = u_adj[uo + base + r];
          l0 = (uint32_t)v_off[v];
          len = (uint32_t)(v_off[v + 1] - v_off[v]);
        }
        lo[r] = l0;
        uint32_t T = g.scan(len, pre);
        for (uint32_t w = r; w < T; w += NT) {
          int i = pbng::seg_of(pre, NT, w);
          uint32_t up = v_adj[lo[i] + (w - pre[i])];
          if (up == u) continue;
          if (pass == 0) {
            atomicAdd(&cnt[up], 1u);
          } else {
            uint32_t c = atomicExch(&cnt[up], 0u);  // first visitor takes the count
            if (c >= 2) sum += (uint64_t)c * (c - 1) / 2;
          }
        }
        __syncthreads();
      }
    }
    uint64_t t = g.sum64(sum);
    if (threadIdx.x == 0) out[u] = t;
    __syncthreads();
  }
}

}  // namespace

extern "C" int pbng_vertex_counts_noalloc(uint32_t nu, uint32_t nv, uint64_t m, const uint64_t *u_off,
                                          const uint32_t *u_adj, const uint64_t *v_off, const uint32_t *v_adj,
                                          uint64_t *out_u, void *stream) {
  pbng::g_detail[0] = 0;
  if (!u_off || !v_off || !out_u || (m && (!u_adj || !v_adj))) return fail_with(PBNG_EINVAL, "null pointer");
  if ((uint64_t)nu + nv >= (1ull << 31) || m >= (1ull << 31))
    return fail_with(PBNG_EINVAL, "graph exceeds the size limits (nu+nv < 2^31, m < 2^31)");
  if (nu > NOALLOC_WORDS)
    return fail_with(PBNG_EINVAL, "nu exceeds the no-allocation limit of 16777216 vertices on the counted side");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    return fail_with(PBNG_ECUDA, "no usable current device");
  }
  // one-time set-up on this device: device addresses of the static arrays
  if (!g_scratch_addr[dev]) {
    void *p = nullptr, *q = nullptr;
    cudaError_t e1 = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    cudaError_t e2 = cudaGetSymbolAddress(&q, g_noalloc_err);
    if (e1 != cudaSuccess || e2 != cudaSuccess || !p || !q) {
      cudaGetLastError();
      return fail_with(PBNG_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
    }
    g_err_addr[dev] = (unsigned *)q;
    g_scratch_addr[dev] = (uint32_t *)p;
  }
  if (nu == 0) return PBNG_OK;
  uint32_t *scr = g_scratch_addr[dev];
  unsigned *err = g_err_addr[dev];
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  size_t blocks = NOALLOC_WORDS / nu;
  if (blocks > (size_t)2 * sms) blocks = (size_t)2 * sms;
  if (blocks > nu) blocks = nu;
  if (blocks < 1) blocks = 1;
  unsigned herr = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) {
    k_noalloc_validate<<<(unsigned)(2 * sms), 256, 0, st>>>(u_off, u_adj, nu, v_off, v_adj, nv, m, err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail_with(PBNG_ECUDA, cudaGetErrorString(e));
  }
  if (herr & 1u) return fail_with(PBNG_EINVAL, "CSR offsets are not a valid non-decreasing 0..m sequence");
  if (herr & 2u) return fail_with(PBNG_EINVAL, "neighbour id out of range");
  // counters start at zero whatever an earlier call left behind
  e = cudaMemsetAsync(scr, 0, blocks * nu * sizeof(uint32_t), st);
  if (e == cudaSuccess) {
    k_vertex_counts_noalloc<<<(unsigned)blocks, NT, 0, st>>>(u_off, u_adj, v_off, v_adj, nu, out_u, scr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail_with(PBNG_ECUDA, cudaGetErrorString(e));
  }
  return PBNG_OK;
}
