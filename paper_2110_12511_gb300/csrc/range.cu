// find_range of the coarse phase (Sec. 3.1.3; Alg. 4, find_range): the
// upper bound theta(i+1) = K + 1 for the smallest support value K such that
// the work of the remaining entities with support <= K reaches the target.
// The paper bins supports in a hash map and sorts the keys (Sec. 4.2: tip
// supports can be cubic in |V|); here the same K is found by a weighted
// radix selection over the 64-bit supports, 8 bits per pass from the highest
// bit in which the remaining supports differ, with the work histogram of
// each digit built in shared memory.  Selection state stays on the device.
#include "internal.cuh"

namespace pbng {
namespace {

using ull = unsigned long long;

// One digit of the selection: the work histogram of the digit over the keys
// that match the prefix so far, then (last block to finish) the digit at
// which the cumulative work first reaches the target.
__global__ void __launch_bounds__(256) k_range_pass(const uint32_t *alist, uint32_t na, const ull *sup, const ull *wl,
                                                    RangeState *rs, int shift, int last) {
  __shared__ ull h[256];
  __shared__ ull wtot[8];
  __shared__ ull s_cum, s_hd, s_h255;
  __shared__ int s_d;
  __shared__ bool s_last;
  const int t = threadIdx.x;
  h[t] = 0;
  __syncthreads();
  const ull prefix = rs->prefix;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + t; j < na; j += (size_t)gridDim.x * blockDim.x) {
    ull key = sup[alist[j]];
    if (shift + 8 >= 64 || ((key ^ prefix) >> (shift + 8)) == 0) {
      ull w = wl[j];
      if (w) atomicAdd(&h[(key >> shift) & 255u], w);
    }
  }
  __syncthreads();
  if (h[t]) atomicAdd(&rs->hist[t], h[t]);
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&rs->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // inclusive scan of the 256 bins
  const ull v = __ldcg(&rs->hist[t]);
  const int lane = t & 31, w = t >> 5;
  ull inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    ull y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wtot[w] = inc;
  if (t == 0) s_d = 256;
  if (t == 255) s_h255 = v;
  __syncthreads();
  ull off = 0, total = 0;
  for (int k = 0; k < 8; k++) {
    if (k < w) off += wtot[k];
    total += wtot[k];
  }
  inc += off;
  const ull below = rs->below, tgt = rs->tgt, excl = inc - v;
  if (below + inc >= tgt && (t == 0 || below + excl < tgt)) {  // the first bin reaching the target
    s_d = t;
    s_cum = below + excl;
    s_hd = v;
  }
  __syncthreads();
  rs->hist[t] = 0;
  if (t == 0) {
    int d = s_d;
    ull cum = s_cum, hd = s_hd;
    if (d == 256) {  // the target is not reached: take the last digit
      d = 255;
      cum = below + total;
      hd = s_h255;
    }
    rs->below = cum;
    rs->prefix = (prefix & ~(255ull << shift)) | ((ull)d << shift);
    rs->done = 0;
    if (last) {
      rs->est = cum + hd;
      rs->theta_hi = rs->prefix + 1;
    }
  }
}

__global__ void k_range_init(RangeState *rs, ull tgt, ull prefix) {
  rs->tgt = tgt;
  rs->prefix = prefix;
  rs->below = 0;
  rs->done = 0;
}

__global__ void k_set_u64(ull *p, ull v) { *p = v; }

}  // namespace

void set_u64(Arena &a, uint64_t *p, uint64_t v) {
  k_set_u64<<<1, 1, 0, a.st>>>((ull *)p, (ull)v);
  CK_LAUNCH();
}

uint64_t range_select(Arena &a, RangeState *rs, const uint32_t *alist, uint32_t na, const uint64_t *sup, const uint64_t *wl,
                      uint64_t kmin, uint64_t kmax, uint64_t tgt, uint64_t *est) {
  if (kmin == kmax) {
    set_u64(a, (uint64_t *)&rs->theta_hi, kmin + 1);
    return kmin + 1;
  }
  int hb = 64 - __builtin_clzll(kmin ^ kmax);  // low bits in which keys differ
  uint64_t low = hb >= 64 ? ~0ull : ((1ull << hb) - 1);
  k_range_init<<<1, 1, 0, a.st>>>(rs, tgt, kmin & ~low);
  CK_LAUNCH();
  int top = ((hb - 1) / 8) * 8;
  for (int shift = top; shift >= 0; shift -= 8) {
    k_range_pass<<<grid_for(na, 256, 4 * num_sms()), 256, 0, a.st>>>(alist, na, (const ull *)sup, (const ull *)wl, rs,
                                                                      shift, shift == 0);
    CK_LAUNCH();
  }
  uint64_t he[2];
  CK(cudaMemcpyAsync(he, &rs->est, sizeof(he), cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  if (est) *est = he[0];
  return he[1];
}

}  // namespace pbng
