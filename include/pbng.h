/*
 * pbng.h -- C ABI of the GB300 (sm_103a) butterfly counting and two-phase
 * bipartite peeling library (tip and wing decomposition).
 *
 * Method: "Parallel Peeling of Bipartite Networks for Hierarchical Dense
 * Subgraph Discovery" (Lakhotia, Kannan, Prasanna).  Every entry point cites
 * the passage that defines the operation it performs.
 *
 * Conventions shared by every call
 *  - A bipartite graph G(W=(U,V),E) is passed as its U-side CSR: u_off has
 *    nu+1 offsets (u_off[0]=0, u_off[nu]=m, non-decreasing), u_adj has m
 *    neighbour ids in [0,nv), each row strictly increasing (sorted, no
 *    duplicate edges).  The edge id of an edge is its position in u_adj.
 *    Limits: nu+nv < 2^31, m < 2^31.
 *  - Pointers are DEVICE pointers (caller-owned; e.g. torch CUDA tensors)
 *    unless opts->mem == PBNG_MEM_HOST, in which case graph and output
 *    pointers are host pointers and the library copies them to and from
 *    the device inside the call.
 *  - Scratch memory is allocated by the library from a stream-ordered
 *    pool on the current device and released before the call returns;
 *    caller memory is never freed or retained.
 *  - Work is issued on opts->stream (a cudaStream_t; NULL = legacy default
 *    stream).  Calls synchronise that stream before returning, so that
 *    device-side errors are reported by the return value.
 *  - Every call returns PBNG_OK (0) or a negative PBNG_E* status; on error
 *    the contents of output buffers are unspecified.  pbng_strerror() names
 *    a status; pbng_last_error_detail() gives a one-line detail of the last
 *    failure on the calling thread.
 *  - Counts, tip numbers and wing numbers are exact uint64 integers.
 */
#ifndef PBNG_H
#define PBNG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PBNG_OK 0
#define PBNG_EINVAL (-1)    /* invalid argument or malformed CSR */
#define PBNG_ENOMEM (-2)    /* device allocation failed */
#define PBNG_ECUDA (-3)     /* CUDA runtime error */
#define PBNG_ETIMEOUT (-4)  /* a bounded device-side wait gave up */
#define PBNG_EOVERFLOW (-5) /* a count could exceed 2^64-1 */
#define PBNG_EBOUNDS (-6)   /* explicit partition bounds not strictly increasing */

typedef struct pbng_bigraph {
  uint32_t nu, nv;       /* |U|, |V| */
  uint64_t m;            /* |E| */
  const uint64_t *u_off; /* nu+1 offsets */
  const uint32_t *u_adj; /* m neighbour ids in [0,nv), rows strictly increasing */
} pbng_bigraph;

typedef enum { PBNG_SIDE_U = 0, PBNG_SIDE_V = 1 } pbng_side;

enum {
  PBNG_BOUNDS_ESTIMATOR = 0, /* find_range with adaptive targets (Sec. 3.1.3) */
  PBNG_BOUNDS_LEARNED = 1,   /* bounds proposed by the MLP in opts->mlp_params (pbng_mlp_forward) */
  PBNG_BOUNDS_EXPLICIT = 2   /* caller-supplied bounds */
};
enum { PBNG_MEM_DEVICE = 0, PBNG_MEM_HOST = 1 };

typedef struct pbng_opts {
  int bounds_mode;         /* PBNG_BOUNDS_*; default ESTIMATOR */
  const uint64_t *bounds;  /* EXPLICIT: host array of n_bounds strictly increasing upper
                              bounds theta(2..), one per coarse partition; a bound that would
                              peel nothing falls back to the estimator */
  uint32_t n_bounds;
  int recount;             /* 1 (default): batch re-count when cheaper than peeling (Sec. 5.1) */
  int compact;             /* 1 (default): dynamic graph updates (Sec. 5.2) */
  int mem;                 /* PBNG_MEM_DEVICE (default) or PBNG_MEM_HOST */
  int graph_rounds;        /* tip only. 1: the coarse-phase rounds of each range run as one
                              CUDA graph whose conditional WHILE node loops on the device
                              (no host round trip per round); every round peels, so
                              `recount` is not used; results are identical.  Default 0 */
  uint64_t timeout_ns;     /* limit for bounded device waits; 0 = 10 s */
  void *stream;            /* cudaStream_t */
  const float *mlp_params; /* LEARNED: device float32 parameters, layout of pbng_mlp_forward, in =
                              128 features (pbng_bound_features for tip, pbng_wing_bound_features
                              for wing), out = bounds proposed; the estimator judges each bound
                              (learned_vet below) */
  uint32_t mlp_hidden, mlp_out;
  uint64_t *bounds_out;    /* optional host array receiving the upper bounds theta(2), theta(3), ...
                              actually used (the last, unbounded range is not listed) */
  uint32_t n_bounds_out;   /* capacity of bounds_out.  One bound is written per range that was
                              closed by a finite bound: stats->parts_used - 1 when the last range
                              used is the unbounded range P, stats->parts_used when a finite bound
                              already took every remaining entity (at most this many are stored;
                              every bound is >= 1, the rest of the array is left as it was) */
  uint32_t bucket_shift;   /* tip: the coarse peel cuts the peeled side's ids into buckets of
                              2^bucket_shift ids (at most 512 buckets); 0 (default) = automatic
                              (15, raised when needed), else 14..30; results are identical */
  /* tip coarse-peel schedule (0 = default; results are identical for every value):
     an active vertex with W wedges is peeled by one warp when W <= warp_max_w (at most 512,
     default 512), by a 256-thread group when W <= group_max_w (warp_max_w..2048, default 2048),
     else by blocks, one per item of at least item_w wedges (>= 4096, default 32768) */
  uint32_t warp_max_w, group_max_w, item_w;
  uint32_t fd_cluster_min;  /* fine phase: a partition with at least this many entities (wing: edges,
                               tip: vertices) is peeled by a cluster of thread blocks sharing its
                               step state instead of one block; 0 = default (32768), 0xffffffff =
                               never; results are identical */
  uint32_t count_scratch;   /* counting (Alg. 1) scratch counters of a start with more than 256 wedges:
                               PBNG_SCRATCH_AUTO (0, default: dense shared counters for the 16384
                               highest-priority starts, shared hashes up to 4096 wedges, then dense
                               counters over all vertices in global memory), PBNG_SCRATCH_HASH (no
                               dense shared class), PBNG_SCRATCH_DENSE (dense shared counters only:
                               16-bit, over chunks of 32768 labels beyond the first 16384),
                               PBNG_SCRATCH_DENSE32 (the same with 32-bit counters); results are
                               identical */
  float learned_vet;        /* LEARNED: the estimator judges each learned bound by the work of the
                               range it closes; a range holding more than learned_vet times the
                               estimator's target work (remaining work over remaining partitions)
                               takes the estimator's bound instead.  0 = default (2.0); negative =
                               learned bounds are not judged; NaN is rejected.  Results are
                               identical */
} pbng_opts;

enum { PBNG_SCRATCH_AUTO = 0, PBNG_SCRATCH_HASH = 1, PBNG_SCRATCH_DENSE = 2, PBNG_SCRATCH_DENSE32 = 3 };

typedef struct pbng_stats {
  uint64_t wedges_count;   /* wedges traversed by the initial count (Alg. 1) */
  uint64_t wedges_cd;      /* wedges traversed by coarse-phase peeling + re-counts */
  uint64_t wedges_fd;      /* wedges traversed by fine-phase peeling */
  uint64_t updates;        /* support updates applied (atomic decrements) */
  uint64_t links;          /* BE-Index links (wing) */
  uint64_t blooms;         /* BE-Index blooms (wing) */
  uint64_t rounds;         /* coarse-phase peeling iterations (rho) */
  uint64_t recounts;       /* rounds that re-counted instead of peeling */
  uint64_t fd_steps;       /* fine-phase peeling steps summed over partitions */
  uint64_t wedge_bound;    /* wedge bound of counting, sum over edges of min(d_u, d_v) */
  uint64_t ns_setup, ns_count, ns_cd, ns_part, ns_fd, ns_total;
  uint32_t parts_used;     /* non-empty coarse partitions */
  uint32_t reserved;
  /* kernel-level measurements (CUDA events bracketing the launches of each
     kernel group on the call's stream) and the algorithmic bytes those
     launches must move: 4 B per wedge traversed, 12 B per (vertex, middle
     vertex) expansion, 16 B per 64-bit support update, 8 B per frontier
     entity; wing: 8 B per bloom-edge link, 16 B per update, 8 B per bloom */
  uint64_t launches;       /* kernels launched by the call */
  uint64_t ns_k_count, ns_k_peel, ns_k_fd;     /* counting / coarse peel / fine peel kernels */
  uint64_t bytes_count, bytes_peel, bytes_fd;  /* algorithmic bytes of those kernels */
  uint64_t n_k_count, n_k_peel, n_k_fd;        /* launches in each group */
  uint64_t fd_work_max, fd_work_sum;           /* fine-phase work per partition (tip: wedges of
                                                  G_i with both ends in U_i; wing: sum of init
                                                  supports): largest and total, for imbalance */
  uint64_t fd_part_steps_max;                  /* most fine-phase steps taken by one partition */
  uint64_t fd_part_cycles_max;                 /* most SM clock cycles spent on one partition */
} pbng_stats;

/* Fill *o with the defaults listed above. */
void pbng_opts_init(pbng_opts *o);

/* Per-vertex and per-edge butterfly counts (Sec. 2.1, Alg. 1 "pveBcnt"):
 * out_u[u] = butterflies containing u (nu entries), out_v[v] likewise (nv
 * entries), out_e[e] = butterflies containing edge e (m entries, edge-id
 * order).  Any output may be NULL to skip it.  Vertex-priority wedge
 * traversal: vertices relabelled by decreasing degree, each wedge
 * start-mid-last expanded only when last has the highest priority. */
int pbng_count(const pbng_bigraph *g, uint64_t *out_u, uint64_t *out_v, uint64_t *out_e,
               const pbng_opts *opts, pbng_stats *stats);

/* Tip decomposition of one vertex side (Sec. 2.2 Def. 2 and the tip number
 * theta_u; two-phase PBNG of Sec. 3.1 adapted to tips, Sec. 3.2): out_tip[x]
 * = tip number of vertex x of the peeled side (nu entries for PBNG_SIDE_U,
 * nv for PBNG_SIDE_V).  P = number of coarse partitions (P >= 1; the paper
 * uses 150).  The result does not depend on P or on the bounds. */
int pbng_tip_decompose(const pbng_bigraph *g, pbng_side side, uint32_t P, uint64_t *out_tip,
                       const pbng_opts *opts, pbng_stats *stats);

/* Wing decomposition (Sec. 2.2 Def. 1 and the wing number theta_e; PBNG
 * with the BE-Index, Sec. 2.3, 3.3, Alg. 4-6): out_wing[e] = wing number of
 * edge e (m entries, edge-id order).  P >= 1 coarse partitions. */
int pbng_wing_decompose(const pbng_bigraph *g, uint32_t P, uint64_t *out_wing, const pbng_opts *opts,
                        pbng_stats *stats);

/* Tip decomposition of n independent graphs in one pass: the graphs are
 * peeled together as their disjoint union (butterflies never cross graphs,
 * so each graph's tip numbers are those of its own decomposition, Sec. 2.2),
 * sharing every launch, coarse round and fine-phase work queue.  outs[i]
 * receives the tip numbers of graph i's peeled side.  With PBNG_MEM_DEVICE
 * every gs[i] pointer and outs[i] is a device pointer; gs and outs
 * themselves are host arrays.  Every graph's own CSR is checked first (the
 * conventions above, with graph i's own nv and m); a malformed graph fails
 * the call with PBNG_EINVAL and pbng_last_error_detail() names its index.
 * opts->bounds_out receives the bounds used for the union, and
 * stats->ns_setup the time to build the union's internal graph. */
int pbng_tip_decompose_batch(const pbng_bigraph *gs, uint32_t n, pbng_side side, uint32_t P,
                             uint64_t *const *outs, const pbng_opts *opts, pbng_stats *stats);

/* Wing numbers of many independent graphs in one call: the graphs are
 * decomposed as their disjoint union (no butterfly crosses two graphs, so
 * every graph's wing numbers are its own); outs[i] (m_i entries, graph i's
 * U-CSR edge order) receives graph i's numbers (may be NULL when m_i = 0).
 * Pointers, per-graph checks, bounds_out and ns_setup as for
 * pbng_tip_decompose_batch. */
int pbng_wing_decompose_batch(const pbng_bigraph *gs, uint32_t n, uint32_t P, uint64_t *const *outs,
                              const pbng_opts *opts, pbng_stats *stats);

/* k-tips from tip numbers (Def. 2; the k-tip hierarchy indexed by tip numbers,
 * Sec. 2.2).  theta: the tip numbers of `side` (as written by
 * pbng_tip_decompose), one uint64 per vertex.  out_comp[x] receives, for
 * every vertex with theta[x] >= k, the smallest id of its k-tip: the
 * vertices of that side with tip number >= k, joined whenever two of them
 * share at least two neighbours (lie in a common butterfly), split into
 * connected components.  Vertices with theta[x] < k get 0xffffffff.  k = 0
 * takes every vertex (a vertex in no butterfly is its own component).
 * Pointers live where opts->mem says (device by default).  Errors as for
 * pbng_tip_decompose; PBNG_ETIMEOUT if a union-find retry limit is hit. */
int pbng_tip_components(const pbng_bigraph *g, pbng_side side, const uint64_t *theta, uint64_t k,
                        uint32_t *out_comp, const pbng_opts *opts, pbng_stats *stats);

/* k-wings from wing numbers (Def. 1): theta holds the m wing numbers (U-CSR
 * edge order, as written by pbng_wing_decompose).  out_comp[e] receives, for
 * every edge with theta[e] >= k, the smallest edge id of its k-wing: the
 * edges with wing number >= k, two of them joined whenever they lie in a
 * common butterfly all of whose edges have wing number >= k, split into
 * connected components; other edges get 0xffffffff.  Pointers and errors as
 * for pbng_tip_components. */
int pbng_wing_components(const pbng_bigraph *g, const uint64_t *theta, uint64_t k, uint32_t *out_comp,
                         const pbng_opts *opts, pbng_stats *stats);

/* Per-vertex butterfly counts of the U side, computed WITHOUT ANY DEVICE
 * ALLOCATION.  The paper has no counterpart: this is an access path for
 * callers that cannot allocate device memory, such as code that must stay
 * inside a fixed, pre-reserved memory budget or whose device memory is owned
 * by another framework's allocator.  out_u[u] = sum over u' != u of
 * C(|N_u cap N_u'|, 2), the same values pbng_count() writes to out_u.
 * Both CSRs are supplied by the caller: u_off/u_adj as for pbng_bigraph and
 * v_off/v_adj (nv+1 offsets, m ids in [0,nu)) the transpose of it; pass the
 * two swapped to count the V side.  Offsets and ids are range-checked;
 * a v-side CSR that is in range but not the transpose gives unspecified
 * counts.  All pointers are device pointers; the call synchronises `stream`
 * (a cudaStream_t, NULL = legacy default stream).
 * Scratch: one fixed 64 MiB array in device global memory, declared in the
 * library, which every GPU that loads the library holds until the process
 * exits.  It limits nu to 16,777,216; a larger nu is rejected with
 * PBNG_EINVAL before any device work.  Every call on a device shares that
 * array and finds the previous call's contents in it (each call clears the
 * part it uses first), so calls that overlap on the GPU, for example on two
 * streams at once, race and give wrong counts.  The first call on each
 * device looks up the array's device address with cudaGetSymbolAddress
 * while that device is current; make that first call before any stream
 * capture.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  Status codes as for the other calls; pbng_last_error_detail()
 * names the cause of a failure. */
int pbng_vertex_counts_noalloc(uint32_t nu, uint32_t nv, uint64_t m, const uint64_t *u_off,
                               const uint32_t *u_adj, const uint64_t *v_off, const uint32_t *v_adj,
                               uint64_t *out_u, void *stream);

/* Partition bounds of the coarse phase (Sec. 3.1.3, find_range with
 * adaptive targets; Sec. 4.1 Th. 2: any strictly increasing bounds give the
 * same tip numbers, so bounds only change speed).  Runs the counting and
 * coarse phase of pbng_tip_decompose on `side` with the same options
 * (opts->bounds_mode: the estimator, or the learned proposer of
 * opts->mlp_params judged by the estimator as in pbng_tip_decompose, or
 * explicit bounds) and stops before the fine phase.  out_bounds (host array
 * of P+1 entries) receives theta(1) = 0, then the upper bound theta(i+1) of
 * every range used, then UINT64_MAX (theta(P+1) = +infinity, and every range
 * not needed).  Feeding out_bounds[1..] back as explicit bounds reproduces
 * the same ranges. */
int pbng_propose_bounds(const pbng_bigraph *g, pbng_side side, uint32_t P, uint64_t *out_bounds,
                        const pbng_opts *opts);

/* BE-Index sums (Sec. 2.3, Property 1 and Property 2): builds the
 * Bloom-Edge-Index used by pbng_wing_decompose and reports, for every edge
 * e, out_e[e] = sum over the maximal priority blooms B containing e of
 * (k_B - 1) (m entries, edge-id order; equals the butterfly count of e), and
 * *out_total (host) = sum over all blooms of C(k_B, 2) (equals the number of
 * butterflies of the graph).  stats->links and stats->blooms give the
 * index's size.  Pointers as for pbng_wing_decompose. */
int pbng_be_index_sums(const pbng_bigraph *g, uint64_t *out_e, uint64_t *out_total, const pbng_opts *opts,
                       pbng_stats *stats);

/* Features of the learned bound proposer (no counterpart in the paper's
 * method; the bounds it feeds only change speed, Sec. 4.1 Th. 2): out[0..63]
 * = fractions of the peeled side's vertices per half-octave degree bin
 * (bin 0: d = 0, 1: d = 1, else 2L-2 + the second-highest bit of d, L = bit
 * length), out[64..127] = fractions of vertices whose initial butterfly count
 * (Sec. 2.1) has a bit length j bits below that of the largest count (j = 0..63).
 * The proposer's outputs are relative to the largest count K:
 * y_i = log2(1 + b_i) / log2(1 + K).  out: 128 floats of device memory. */
int pbng_bound_features(const pbng_bigraph *g, pbng_side side, float *out, const pbng_opts *opts);

/* Features of the learned wing bound proposer, the same histograms over the
 * edges: out[0..63] by the half-octave bin of min(d_u, d_v) of each edge,
 * out[64..127] by how many bits each edge's initial butterfly count (Sec. 2.1,
 * per edge) lies below the largest one.  out: 128 floats of device memory. */
int pbng_wing_bound_features(const pbng_bigraph *g, float *out, const pbng_opts *opts);

/* MLP of the learned proposer, FP32, on the device.  params packs
 * [W1 (in x hidden), b1, W2 (hidden x hidden), b2, W3 (hidden x out), b3]
 * row-major; y = relu(relu(x W1 + b1) W2 + b2) W3 + b3 for each of the B
 * rows of X (B x in) into Y (B x out).  All pointers are device pointers;
 * each call synchronises `stream`. */
int pbng_mlp_forward(const float *params, uint32_t in, uint32_t hidden, uint32_t out, const float *X, uint32_t B,
                     float *Y, void *stream);
/* Gradient of the mean squared error (1/(B out)) sum (y - t)^2 with respect
 * to params (same layout) into grad, and the loss into *loss (device). */
int pbng_mlp_grad(const float *params, uint32_t in, uint32_t hidden, uint32_t out, const float *X, const float *T,
                  uint32_t B, float *grad, float *loss, void *stream);
/* One Adam step (bias-corrected, step >= 1) over n parameters. */
int pbng_mlp_adam(float *params, const float *grad, float *m, float *v, uint64_t n, float lr, float beta1, float beta2,
                  float eps, uint32_t step, void *stream);

/* Name of a status code. */
const char *pbng_strerror(int status);
/* Detail of the most recent failure on this thread ("" if none). */
const char *pbng_last_error_detail(void);
/* Library version, major*10000 + minor*100 + patch. */
int pbng_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PBNG_H */
