// Learned coarse-phase bounds: a small MLP (FP32) from histogram features of
// a graph to partition upper bounds, with its own forward, backward and Adam
// kernels, and the feature extraction.
//
// Any strictly increasing bounds give the same tip and wing numbers
// (Sec. 4.1, Th. 2: partitions are correct for every range sequence), so the
// network can only change how fast the decomposition runs; bounds that would
// peel nothing fall back to find_range.
//
// Network: x (in) -> relu(x W1 + b1) (hidden) -> relu(h1 W2 + b2) (hidden)
//          -> h2 W3 + b3 (out); parameters packed as
//          [W1 (in x hidden), b1, W2 (hidden x hidden), b2, W3 (hidden x out), b3],
//          row-major, float32.  Loss: mean squared error over batch x out.
// Features (in = 128): 64-bin half-octave histogram of the degrees of the
// peeled side (bin 0: d = 0, 1: d = 1, else 2 L - 2 + second-highest bit of d
// with L = bit length) and 64-bin histogram of how many bits below the
// largest initial support each support's bit length is, each normalised to
// fractions (integer binning, no rounding).  Outputs are relative to the
// largest initial support K: y_i = log2(1 + b_i) / log2(1 + K) for the upper
// bounds b_1 < b_2 < ... (theta(2), theta(3), ...), so the same network
// serves graphs of different scales.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace pbng {
namespace {

// out[b][j] = act(sum_k in[b][k] W[k][j] + bias[j]); one thread per (b, j)
__global__ void k_dense(const float *in, const float *W, const float *bias, float *out, uint32_t B, uint32_t nin, uint32_t nout,
                        int relu) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)B * nout) return;
  uint32_t b = (uint32_t)(t / nout), j = (uint32_t)(t % nout);
  float s = bias[j];
  const float *x = in + (size_t)b * nin;
  for (uint32_t k = 0; k < nin; k++) s += x[k] * W[(size_t)k * nout + j];
  out[t] = relu ? fmaxf(s, 0.f) : s;
}

// dY = 2 (Y - T) / (B * out); loss partial sums
__global__ void k_mse(const float *Y, const float *T, float *dY, size_t n, float scale, float *loss) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  float l = 0.f;
  if (t < n) {
    float d = Y[t] - T[t];
    dY[t] = 2.f * d * scale;
    l = d * d * scale;
  }
  for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

// dW[k][j] = sum_b in[b][k] dout[b][j]; db[j] = sum_b dout[b][j]
__global__ void k_wgrad(const float *in, const float *dout, float *dW, float *db, uint32_t B, uint32_t nin, uint32_t nout) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < (size_t)nin * nout) {
    uint32_t k = (uint32_t)(t / nout), j = (uint32_t)(t % nout);
    float s = 0.f;
    for (uint32_t b = 0; b < B; b++) s += in[(size_t)b * nin + k] * dout[(size_t)b * nout + j];
    dW[t] = s;
  }
  if (t < nout) {
    float s = 0.f;
    for (uint32_t b = 0; b < B; b++) s += dout[(size_t)b * nout + t];
    db[t] = s;
  }
}

// din[b][k] = (sum_j W[k][j] dout[b][j]) * (h[b][k] > 0)
__global__ void k_bgrad(const float *W, const float *dout, const float *h, float *din, uint32_t B, uint32_t nin, uint32_t nout) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)B * nin) return;
  uint32_t b = (uint32_t)(t / nin), k = (uint32_t)(t % nin);
  float s = 0.f;
  for (uint32_t j = 0; j < nout; j++) s += W[(size_t)k * nout + j] * dout[(size_t)b * nout + j];
  din[t] = h[t] > 0.f ? s : 0.f;
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  float gi = g[t];
  float mi = b1 * m[t] + (1.f - b1) * gi, vi = b2 * v[t] + (1.f - b2) * gi * gi;
  m[t] = mi;
  v[t] = vi;
  p[t] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

struct Layout {
  size_t w1, b1, w2, b2, w3, b3, n;
  Layout(uint32_t in, uint32_t h, uint32_t out) {
    w1 = 0;
    b1 = w1 + (size_t)in * h;
    w2 = b1 + h;
    b2 = w2 + (size_t)h * h;
    w3 = b2 + h;
    b3 = w3 + (size_t)h * out;
    n = b3 + out;
  }
};

void forward(Arena &a, const float *P, uint32_t in, uint32_t h, uint32_t out, const float *X, uint32_t B, float *H1, float *H2,
             float *Y) {
  Layout L(in, h, out);
  const int T = 128;
  k_dense<<<grid_for((size_t)B * h, T), T, 0, a.st>>>(X, P + L.w1, P + L.b1, H1, B, in, h, 1);
  CK_LAUNCH();
  k_dense<<<grid_for((size_t)B * h, T), T, 0, a.st>>>(H1, P + L.w2, P + L.b2, H2, B, h, h, 1);
  CK_LAUNCH();
  k_dense<<<grid_for((size_t)B * out, T), T, 0, a.st>>>(H2, P + L.w3, P + L.b3, Y, B, h, out, 0);
  CK_LAUNCH();
}

__global__ void k_max_u64(const unsigned long long *x, uint32_t n, unsigned long long *mx) {
  unsigned long long m = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) m = max(m, x[i]);
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

// degree of entity x: from the CSR offsets (vertices) or given (edges)
__global__ void k_features(const unsigned long long *sup, const uint32_t *p_off, const uint32_t *deg, uint32_t nx,
                           const unsigned long long *mx, float *hist) {
  __shared__ unsigned int h[128];
  if (threadIdx.x < 128) h[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long K = *mx;
  int kb = K ? 64 - __clzll(K) : 0;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < nx; x += (size_t)gridDim.x * blockDim.x) {
    uint32_t d = deg ? deg[x] : p_off[x + 1] - p_off[x];
    int db = d;
    if (d >= 2) {
      int L = 32 - __clz(d);
      db = 2 * L - 2 + (int)((d >> (L - 2)) & 1u);
    }
    atomicAdd(&h[db < 63 ? db : 63], 1u);
    unsigned long long s = sup[x];
    int sb = kb - (s ? 64 - __clzll(s) : 0);  // bits below the largest support
    atomicAdd(&h[64 + (sb < 63 ? sb : 63)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 128 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (float)h[threadIdx.x] / (float)nx);
}

}  // namespace

// features of the peeled entities from their initial supports and degrees
// (device arrays; deg null: degrees from p_off); returns the largest support
uint64_t bound_features(Arena &a, const uint64_t *sup, const uint32_t *p_off, uint32_t nx, float *out128,
                        const uint32_t *deg) {
  CK(cudaMemsetAsync(out128, 0, 128 * sizeof(float), a.st));
  if (!nx) return 0;
  unsigned long long *mx = a.zeros<unsigned long long>(1);
  k_max_u64<<<grid_for(nx, 256, 4 * num_sms()), 256, 0, a.st>>>((const unsigned long long *)sup, nx, mx);
  CK_LAUNCH();
  k_features<<<grid_for(nx, 256, 4 * num_sms()), 256, 0, a.st>>>((const unsigned long long *)sup, p_off, deg, nx, mx,
                                                                   out128);
  CK_LAUNCH();
  uint64_t K = fetch(a, (const uint64_t *)mx);
  a.free(mx);
  return K;
}

// run the proposer on device features; returns strictly increasing bounds
std::vector<uint64_t> propose_bounds(Arena &a, const float *params, uint32_t hidden, uint32_t out, const float *feat,
                                     uint64_t K) {
  float *H1 = a.alloc<float>(hidden), *H2 = a.alloc<float>(hidden), *Y = a.alloc<float>(out);
  forward(a, params, 128, hidden, out, feat, 1, H1, H2, Y);
  std::vector<float> y(out);
  CK(cudaMemcpyAsync(y.data(), Y, out * sizeof(float), cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  std::vector<uint64_t> b;
  double scale = std::log2(1.0 + (double)K);
  for (uint32_t i = 0; i < out; i++) {
    double e = (double)y[i] * scale;
    if (!(e > 0.0)) e = 0.0;
    if (e > 63.0) e = 63.0;
    uint64_t v = (uint64_t)std::llround(std::exp2(e)) ;  // 1 + b_i
    v = v > 0 ? v - 1 : 0;
    if (v == 0) v = 1;
    if (!b.empty() && v <= b.back()) continue;  // keep them strictly increasing
    b.push_back(v);
  }
  a.free(H1);
  a.free(H2);
  a.free(Y);
  return b;
}

}  // namespace pbng

using namespace pbng;

namespace {
template <class F>
int mlp_guard(F &&f) {
  try {
    f();
    return PBNG_OK;
  } catch (Error &e) {
    return e.code;
  } catch (...) {
    return PBNG_ECUDA;
  }
}
}  // namespace

extern "C" int pbng_mlp_forward(const float *params, uint32_t in, uint32_t hidden, uint32_t out, const float *X, uint32_t B,
                                float *Y, void *stream) {
  return mlp_guard([&] {
    if (!params || !X || !Y || !in || !hidden || !out) fail(PBNG_EINVAL, "invalid MLP arguments");
    Arena a((cudaStream_t)stream);
    float *H1 = a.alloc<float>((size_t)B * hidden), *H2 = a.alloc<float>((size_t)B * hidden);
    if (B) forward(a, params, in, hidden, out, X, B, H1, H2, Y);
    CK(cudaStreamSynchronize(a.st));
  });
}

extern "C" int pbng_mlp_grad(const float *params, uint32_t in, uint32_t hidden, uint32_t out, const float *X, const float *Tg,
                             uint32_t B, float *grad, float *loss, void *stream) {
  return mlp_guard([&] {
    if (!params || !X || !Tg || !grad || !loss || !in || !hidden || !out || !B) fail(PBNG_EINVAL, "invalid MLP arguments");
    Arena a((cudaStream_t)stream);
    Layout L(in, hidden, out);
    size_t bh = (size_t)B * hidden, bo = (size_t)B * out;
    float *H1 = a.alloc<float>(bh), *H2 = a.alloc<float>(bh), *Y = a.alloc<float>(bo);
    float *dY = a.alloc<float>(bo), *dH2 = a.alloc<float>(bh), *dH1 = a.alloc<float>(bh);
    forward(a, params, in, hidden, out, X, B, H1, H2, Y);
    CK(cudaMemsetAsync(loss, 0, sizeof(float), a.st));
    const int T = 128;
    k_mse<<<grid_for(bo, T), T, 0, a.st>>>(Y, Tg, dY, bo, 1.f / (float)bo, loss);
    CK_LAUNCH();
    k_wgrad<<<grid_for((size_t)hidden * out, T), T, 0, a.st>>>(H2, dY, grad + L.w3, grad + L.b3, B, hidden, out);
    CK_LAUNCH();
    k_bgrad<<<grid_for(bh, T), T, 0, a.st>>>(params + L.w3, dY, H2, dH2, B, hidden, out);
    CK_LAUNCH();
    k_wgrad<<<grid_for((size_t)hidden * hidden, T), T, 0, a.st>>>(H1, dH2, grad + L.w2, grad + L.b2, B, hidden, hidden);
    CK_LAUNCH();
    k_bgrad<<<grid_for(bh, T), T, 0, a.st>>>(params + L.w2, dH2, H1, dH1, B, hidden, hidden);
    CK_LAUNCH();
    k_wgrad<<<grid_for((size_t)in * hidden, T), T, 0, a.st>>>(X, dH1, grad + L.w1, grad + L.b1, B, in, hidden);
    CK_LAUNCH();
    CK(cudaStreamSynchronize(a.st));
  });
}

extern "C" int pbng_mlp_adam(float *params, const float *grad, float *m, float *v, uint64_t n, float lr, float beta1,
                             float beta2, float eps, uint32_t step, void *stream) {
  return mlp_guard([&] {
    if (!params || !grad || !m || !v || step == 0) fail(PBNG_EINVAL, "invalid Adam arguments");
    cudaStream_t st = (cudaStream_t)stream;
    float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adam<<<grid_for(n, 256), 256, 0, st>>>(params, grad, m, v, n, lr, beta1, beta2, eps, c1, c2);
    CK_LAUNCH();
    CK(cudaStreamSynchronize(st));
  });
}
