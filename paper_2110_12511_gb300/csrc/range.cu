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

__global__ void k_range_hist(const uint32_t *alist, uint32_t na, const ull *sup, const ull *wl, RangeState *rs, int shift) {
  __shared__ ull h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  ull prefix = rs->prefix;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < na; j += (size_t)gridDim.x * blockDim.x) {
    ull key = sup[alist[j]];
    if (shift + 8 >= 64 || ((key ^ prefix) >> (shift + 8)) == 0) {
      ull w = wl[j];
      if (w) atomicAdd(&h[(key >> shift) & 255u], w);
    }
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&rs->hist[threadIdx.x], h[threadIdx.x]);
}

// the digit at which the cumulative work first reaches the target
__global__ void k_range_select(RangeState *rs, int shift, int last) {
  if (threadIdx.x != 0) return;
  ull cum = rs->below;
  int d = 255;
  for (int i = 0; i < 256; i++) {
    if (cum + rs->hist[i] >= rs->tgt) {
      d = i;
      break;
    }
    cum += rs->hist[i];
  }
  ull est = cum + rs->hist[d];
  rs->below = cum;
  rs->prefix = (rs->prefix & ~(255ull << shift)) | ((ull)d << shift);
  for (int i = 0; i < 256; i++) rs->hist[i] = 0;
  if (last) {
    rs->est = est;
    rs->theta_hi = rs->prefix + 1;
  }
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
  set_u64(a, (uint64_t *)&rs->tgt, tgt);
  set_u64(a, (uint64_t *)&rs->prefix, kmin & ~low);
  set_u64(a, (uint64_t *)&rs->below, 0);
  int top = ((hb - 1) / 8) * 8;
  for (int shift = top; shift >= 0; shift -= 8) {
    k_range_hist<<<grid_for(na, 256, 4 * num_sms()), 256, 0, a.st>>>(alist, na, (const ull *)sup, (const ull *)wl, rs, shift);
    CK_LAUNCH();
    k_range_select<<<1, 32, 0, a.st>>>(rs, shift, shift == 0);
    CK_LAUNCH();
  }
  uint64_t he[2];
  CK(cudaMemcpyAsync(he, &rs->est, sizeof(he), cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  if (est) *est = he[0];
  return he[1];
}

}  // namespace pbng
