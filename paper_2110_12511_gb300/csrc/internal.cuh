// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pbng.h"

namespace pbng {

// ------------------------------------------------------------------ errors
struct Error {
  int code;
};
[[noreturn]] void fail(int code, const char *fmt, ...);
void cuda_check(cudaError_t e, const char *what, const char *file, int line);
#define CK(x) ::pbng::cuda_check((x), #x, __FILE__, __LINE__)
#define CK_LAUNCH() (::pbng::g_launches++, ::pbng::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__))
extern thread_local uint64_t g_launches;

// ------------------------------------------------------------- profiling
// Event spans around groups of kernel launches, collected when a caller
// asks for statistics.
enum { PROF_COUNT = 0, PROF_PEEL = 1, PROF_FD = 2, PROF_NGROUPS = 3 };
struct Prof {
  bool on = false;
  cudaStream_t st = nullptr;
  struct Span {
    cudaEvent_t a, b;
    int group;
  };
  std::vector<Span> spans;
  uint64_t launches[PROF_NGROUPS] = {0, 0, 0};
  uint64_t bytes[PROF_NGROUPS] = {0, 0, 0};
  uint64_t l0 = 0;
  int cur = -1;
  void begin(int group);
  void end();
  // sum the spans per group (synchronises on the last event) and reset
  void collect(uint64_t ns[PROF_NGROUPS]);
};
extern thread_local Prof g_prof;

// -------------------------------------------------------------- allocation
// Per-call arena of stream-ordered allocations, released when the call ends.
struct Arena {
  cudaStream_t st = nullptr;
  std::vector<void *> ptrs;
  size_t bytes = 0, peak = 0;
  explicit Arena(cudaStream_t s) : st(s) {}
  ~Arena();
  void *raw(size_t nbytes);
  template <class T>
  T *alloc(size_t n) {
    return static_cast<T *>(raw(n * sizeof(T)));
  }
  template <class T>
  T *zeros(size_t n) {
    T *p = alloc<T>(n);
    CK(cudaMemsetAsync(p, 0, (n ? n : 1) * sizeof(T), st));
    return p;
  }
  void free(void *p);
};

int num_sms();
void init_device_pool();

// ------------------------------------------------------------ primitives
// out[i] = sum_{j<i} in[j] for i in [0, n]; out has n+1 entries.
void exclusive_scan_u32(Arena &a, const uint32_t *in, uint32_t *out, size_t n);
void exclusive_scan_u32_to_u64(Arena &a, const uint32_t *in, uint64_t *out, size_t n);
void exclusive_scan_u64(Arena &a, const uint64_t *in, uint64_t *out, size_t n);
// Stable LSD radix sort of (key, value) pairs on the low key_bits bits.
// keys / vals are sorted in place (temporary buffers from the arena).
void sort_pairs(Arena &a, uint64_t *keys, uint32_t *vals, size_t n, int key_bits);
// device reductions to a host value (synchronises the stream)
uint64_t reduce_sum_u64(Arena &a, const uint64_t *in, size_t n);
uint32_t reduce_max_u32(Arena &a, const uint32_t *in, size_t n);
// read one device value (synchronises)
template <class T>
T fetch(Arena &a, const T *p) {
  T v;
  CK(cudaMemcpyAsync(&v, p, sizeof(T), cudaMemcpyDeviceToHost, a.st));
  CK(cudaStreamSynchronize(a.st));
  return v;
}

static inline int bits_for(uint64_t x) {  // bits needed to represent x (>= 1)
  int b = 1;
  while (b < 64 && (x >> b)) b++;
  return b;
}
static inline unsigned grid_for(size_t n, unsigned threads, unsigned cap = 1u << 30) {
  size_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// ------------------------------------------------------ cluster launches
// Thread-block clusters for the fine phase's heavy partitions: the cluster
// size (16 blocks where the device can hold such clusters for `kernel`, else
// 8, else 1 = none) and how many run at once (at most half of the SMs, so
// that one-block teams keep the rest).  Cached per kernel.
struct FDClusterShape {
  uint32_t size = 1, max_clusters = 0;
};
FDClusterShape fd_cluster_shape(const void *kernel, int threads, size_t smem);

// launch `kernel` as nclusters clusters of csize blocks on stream st
template <class... Args>
cudaError_t launch_cluster(const void *kernel, uint32_t nclusters, uint32_t csize, int threads, size_t smem,
                           cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nclusters * csize);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  void *ptrs[] = {(void *)&args...};
  return cudaLaunchKernelExC(&cfg, kernel, ptrs);
}

// A side stream forked from `main` (when on): work issued on st runs
// concurrently with main's, and main waits for it when this goes out of scope.
struct SideLaunch {
  cudaStream_t main = nullptr, st = nullptr;
  cudaEvent_t ev = nullptr;
  SideLaunch(cudaStream_t m, bool on);
  ~SideLaunch();
};

// ------------------------------------------------------------------ graph
// Internal graph in 32-bit CSR form plus the degree-priority labelled
// adjacency used by Alg. 1.  Edge id = position in the U-side CSR.
struct Graph {
  uint32_t nu = 0, nv = 0, m = 0;
  // U-side CSR (edge id = position) and V-side CSR with edge ids
  uint32_t *u_off = nullptr, *u_adj = nullptr;
  uint32_t *v_off = nullptr, *v_adj = nullptr, *v_eid = nullptr;
  // labelled adjacency over W = U u V (label 0 = highest priority, Alg. 1 l.2-4)
  uint32_t n = 0;
  uint32_t *lab_off = nullptr, *lab_adj = nullptr, *lab_eid = nullptr;
  uint32_t *g2lab = nullptr;  // gidx (u, or nu+v) -> label
  uint32_t *lab2g = nullptr;  // label -> gidx
  uint32_t maxdeg = 0;
  uint64_t wedge_bound = 0;  // sum over edges of min(d_u, d_v)
  bool has_labels = false;
};

// Validate a device CSR and build the internal graph.  want_labels: also
// build the labelled adjacency (needed by counting); want_eid: keep the edge
// ids of the labelled adjacency (per-edge counts, BE-Index).
void build_graph(Arena &a, const pbng_bigraph &g, bool want_labels, bool want_eid, Graph &G);

// -------------------------------------------------------------- counting
struct CountOut {
  uint64_t *cnt_lab = nullptr;   // per label (size n), accumulated (caller zeroes)
  uint64_t *cnt_e = nullptr;     // per edge (size m) or null
  const uint8_t *lab_alive = nullptr;  // restrict to alive labels (null = all)
  const uint8_t *lab_isU = nullptr;    // side of each label (needed when want_side >= 0)
  int want_side = -1;            // -1 both; 0 only U labels' counts; 1 only V labels'
  uint64_t *wedges = nullptr;    // optional device counters [3]: wedges, expansions, updates
  uint64_t *be_nb = nullptr;     // optional per-label BE-Index sizes: blooms started at the label
  uint64_t *be_np = nullptr;     // and their twin pairs (caller zeroes both)
  int scratch = PBNG_SCRATCH_AUTO;  // scratch counters of the heavier starts (pbng_opts.count_scratch)
};
// Alg. 1 over the labelled adjacency (all starts).
void count_butterflies(Arena &a, const Graph &G, const CountOut &o);

// side flags of labels: isU[label] = 1 if the label is a U vertex
uint8_t *label_sides(Arena &a, const Graph &G);

// ------------------------------------------------------------ find_range
struct RangeState {  // device-side state of the weighted selection
  unsigned long long kmin, kmax, wsum;  // key range and total work of the remaining entities
  unsigned long long prefix, below, tgt, est, theta_hi;
  unsigned long long hist[256];
  unsigned done;  // blocks finished with the current digit
};
void set_u64(Arena &a, uint64_t *p, uint64_t v);
// theta_hi for the remaining entities alist[0..na) with supports sup[] and
// work wl[j] (aligned with alist): 1 + smallest K with work(sup <= K) >= tgt.
// Leaves theta_hi in rs->theta_hi; *est = work(sup <= K).  Synchronises.
uint64_t range_select(Arena &a, RangeState *rs, const uint32_t *alist, uint32_t na, const uint64_t *sup, const uint64_t *wl,
                      uint64_t kmin, uint64_t kmax, uint64_t tgt, uint64_t *est);

// ------------------------------------------------------------------ tip
struct TipParams {
  uint32_t P;
  int bounds_mode;
  const uint64_t *bounds;
  uint32_t n_bounds;
  int recount, compact, graph_rounds;
  uint32_t bucket_shift;  // 0 = automatic
  uint32_t warp_max_w, group_max_w, item_w;  // coarse-peel schedule, 0 = default
  uint32_t fd_cluster_min;                   // fine phase: smallest partition for a cluster team
  int count_scratch;                         // counting: scratch counters (PBNG_SCRATCH_*)
  double learned_vet;                        // learned bounds: most work of a range, x target (<= 0: unjudged)
  uint64_t timeout_ns;
  const float *mlp_params;  // learned bounds (bounds_mode == PBNG_BOUNDS_LEARNED)
  uint32_t mlp_hidden, mlp_out;
  std::vector<uint64_t> *bounds_used;  // optional record of theta(2..) used
  bool coarse_only = false;            // stop after the coarse phase (no tip numbers written)
};
void tip_decompose(Arena &a, Graph &G, int side, const TipParams &p, uint64_t *theta_out, pbng_stats *st);

// ------------------------------------------------------------ k-tips
// Component of every vertex of `side` in the k-tips (smallest member id), or
// 0xffffffff when theta < k; theta on the device.  Optional counters.
void tip_components(Arena &a, Graph &G, int side, const uint64_t *theta, uint64_t k, uint32_t *out, uint64_t *wedges,
                    uint64_t *joins);
// Component of every edge in the k-wings (smallest member edge id), or
// 0xffffffff when theta_e < k; theta on the device.
void wing_components(Arena &a, Graph &G, const uint64_t *theta, uint64_t k, uint32_t *out, uint64_t *wedges,
                     uint64_t *joins);

// ------------------------------------------------------- learned bounds
uint64_t bound_features(Arena &a, const uint64_t *sup, const uint32_t *p_off, uint32_t nx, float *out128,
                        const uint32_t *deg = nullptr);
// min(d_u, d_v) of every edge (U-CSR order): the degree of an edge in the
// wing proposer's features
void edge_min_degrees(Arena &a, const Graph &G, uint32_t *out);
std::vector<uint64_t> propose_bounds(Arena &a, const float *params, uint32_t hidden, uint32_t out, const float *feat,
                                     uint64_t max_support);

// ------------------------------------------------------------------ wing
// BE-Index (Sec. 2.3): blooms with their numbers k0 and first twin pair boff,
// twin pairs (pe1[q], pe2[q]) of bloom pbloom[q], and every edge's pairs
// elink[eoff[e] .. eoff[e+1]).
struct BEIndex {
  uint32_t nb = 0;
  size_t np = 0;
  uint32_t *k0 = nullptr, *boff = nullptr, *pe1 = nullptr, *pe2 = nullptr, *pbloom = nullptr;
  uint32_t *eoff = nullptr, *elink = nullptr;
};
void be_index_build(Arena &a, const Graph &G, unsigned long long *sup_e, uint64_t *cctr, BEIndex &I, int scratch);
// out_e[e] = sum over the blooms B of e of (k_B - 1); *total = sum over blooms of C(k_B, 2)
void be_index_sums(Arena &a, const Graph &G, uint64_t *out_e, uint64_t *total, pbng_stats *st);
void wing_decompose(Arena &a, Graph &G, const TipParams &p, uint64_t *theta_out, pbng_stats *st);

}  // namespace pbng
