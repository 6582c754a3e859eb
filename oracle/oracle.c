/*
 * CPU oracle for butterfly counting and tip / wing decomposition.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library imports, links or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or table with the GPU
 * path.
 *
 * Everything here is plain, sequential and exact (64-bit unsigned integers):
 *
 *  - Butterfly counts by their definition (Sec. 2, Tab. 1; Sec. 2.1): the
 *    butterflies of u in U are sum over u' != u of C(|N_u cap N_u'|, 2); the
 *    butterflies of edge (u, v) are sum over u' in N_v \ {u} of
 *    (|N_u cap N_u'| - 1).  The 2-hop traversal visits every wedge with u as
 *    an endpoint (the naive O(sum_v d_v^2) method, not the priority-ordered
 *    Alg. 1), so it shares no ordering logic with the counting kernels.
 *  - Bottom-up peeling, BUP (Sec. 2.2, Alg. 2): repeatedly remove the
 *    remaining entity of minimum support (ties: smallest id), record its
 *    support as its tip / wing number, and lower the support of every entity
 *    that shared butterflies with it, clamped from below at the recorded
 *    number.  Tip peels one vertex side only (Sec. 2.2: a k-tip keeps all of
 *    the other side); wing peels edges and finds the butterflies of the
 *    removed edge by the wedge scan of Alg. 2's update function.
 *  - Membership-restricted supports used by the full-size sampled checks:
 *    the butterflies an entity has inside a given entity subset.
 *
 * Vertex ids are uint32, CSR offsets uint64, counts uint64.  Edge id = the
 * edge's position in u_adj.  All arrays are host memory owned by the caller.
 * Return value: 0 on success, -1 on allocation failure.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static uint64_t choose2(uint64_t c) { return c * (c - 1) / 2; }

/* transpose of the U-side CSR: V-side CSR plus, for each V-side slot, the
 * id of the edge it represents */
typedef struct { uint64_t *off; uint32_t *adj; uint64_t *eid; } vcsr_t;

static int make_vcsr(uint32_t nu, uint32_t nv, const uint64_t *u_off, const uint32_t *u_adj, vcsr_t *t) {
  uint64_t m = u_off[nu];
  t->off = (uint64_t *)calloc((size_t)nv + 1, sizeof(uint64_t));
  t->adj = (uint32_t *)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
  t->eid = (uint64_t *)malloc((size_t)(m ? m : 1) * sizeof(uint64_t));
  uint64_t *fill = (uint64_t *)malloc(((size_t)nv + 1) * sizeof(uint64_t));
  if (!t->off || !t->adj || !t->eid || !fill) {
    free(t->off); free(t->adj); free(t->eid); free(fill); return -1;
  }
  for (uint64_t e = 0; e < m; e++) t->off[u_adj[e] + 1]++;
  for (uint32_t v = 0; v < nv; v++) t->off[v + 1] += t->off[v];
  memcpy(fill, t->off, ((size_t)nv + 1) * sizeof(uint64_t));
  for (uint32_t u = 0; u < nu; u++)
    for (uint64_t e = u_off[u]; e < u_off[u + 1]; e++) {
      uint32_t v = u_adj[e];
      t->adj[fill[v]] = u;
      t->eid[fill[v]] = e;
      fill[v]++;
    }
  free(fill);
  return 0;
}
static void free_vcsr(vcsr_t *t) { free(t->off); free(t->adj); free(t->eid); }

/* c[u'] = |N_u cap N_u'| for every u' != u with include[u'] (NULL = all),
 * accumulated into the dense array cnt; touched u' are listed in list.
 * Returns the number of touched entries. */
static uint64_t common_counts(uint32_t u, const uint64_t *u_off, const uint32_t *u_adj, const vcsr_t *t,
                              const uint8_t *include, uint32_t *cnt, uint32_t *list) {
  uint64_t nt = 0;
  for (uint64_t e = u_off[u]; e < u_off[u + 1]; e++) {
    uint32_t v = u_adj[e];
    for (uint64_t q = t->off[v]; q < t->off[v + 1]; q++) {
      uint32_t w = t->adj[q];
      if (w == u || (include && !include[w])) continue;
      if (cnt[w]++ == 0) list[nt++] = w;
    }
  }
  return nt;
}

/* Per-vertex butterfly counts of side U: out[u] = sum_{u'!=u} C(c(u,u'),2). */
int oracle_vertex_counts(uint32_t nu, uint32_t nv, const uint64_t *u_off, const uint32_t *u_adj, uint64_t *out) {
  vcsr_t t;
  if (make_vcsr(nu, nv, u_off, u_adj, &t)) return -1;
  uint32_t *cnt = (uint32_t *)calloc((size_t)nu + 1, sizeof(uint32_t));
  uint32_t *list = (uint32_t *)malloc(((size_t)nu + 1) * sizeof(uint32_t));
  if (!cnt || !list) { free(cnt); free(list); free_vcsr(&t); return -1; }
  for (uint32_t u = 0; u < nu; u++) {
    uint64_t nt = common_counts(u, u_off, u_adj, &t, NULL, cnt, list), s = 0;
    for (uint64_t i = 0; i < nt; i++) { s += choose2(cnt[list[i]]); cnt[list[i]] = 0; }
    out[u] = s;
  }
  free(cnt); free(list); free_vcsr(&t);
  return 0;
}

/* The same per-vertex counts computed by all host threads (OpenMP over the
 * vertices u; each thread has its own counter array).  Used to time the
 * counting step on every host core; returns the threads used, or -1. */
int oracle_vertex_counts_parallel(uint32_t nu, uint32_t nv, const uint64_t *u_off, const uint32_t *u_adj, uint64_t *out) {
  vcsr_t t;
  if (make_vcsr(nu, nv, u_off, u_adj, &t)) return -1;
  int threads = 1, failed = 0;
#ifdef _OPENMP
#pragma omp parallel reduction(| : failed)
#endif
  {
#ifdef _OPENMP
#pragma omp single
    threads = omp_get_num_threads();
#endif
    uint32_t *cnt = (uint32_t *)calloc((size_t)nu + 1, sizeof(uint32_t));
    uint32_t *list = (uint32_t *)malloc(((size_t)nu + 1) * sizeof(uint32_t));
    if (!cnt || !list) {
      failed = 1;
    } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
      for (int64_t ui = 0; ui < (int64_t)nu; ui++) {
        uint32_t u = (uint32_t)ui;
        uint64_t nt = common_counts(u, u_off, u_adj, &t, NULL, cnt, list), s = 0;
        for (uint64_t i = 0; i < nt; i++) { s += choose2(cnt[list[i]]); cnt[list[i]] = 0; }
        out[u] = s;
      }
    }
    free(cnt); free(list);
  }
  free_vcsr(&t);
  return failed ? -1 : threads;
}

/* Per-edge butterfly counts: out[(u,v)] = sum_{u' in N_v, u' != u} (c(u,u') - 1). */
int oracle_edge_counts(uint32_t nu, uint32_t nv, const uint64_t *u_off, const uint32_t *u_adj, uint64_t *out) {
  vcsr_t t;
  if (make_vcsr(nu, nv, u_off, u_adj, &t)) return -1;
  uint32_t *cnt = (uint32_t *)calloc((size_t)nu + 1, sizeof(uint32_t));
  uint32_t *list = (uint32_t *)malloc(((size_t)nu + 1) * sizeof(uint32_t));
  if (!cnt || !list) { free(cnt); free(list); free_vcsr(&t); return -1; }
  for (uint32_t u = 0; u < nu; u++) {
    uint64_t nt = common_counts(u, u_off, u_adj, &t, NULL, cnt, list);
    for (uint64_t e = u_off[u]; e < u_off[u + 1]; e++) {
      uint32_t v = u_adj[e];
      uint64_t s = 0;
      for (uint64_t q = t.off[v]; q < t.off[v + 1]; q++) {
        uint32_t w = t.adj[q];
        if (w != u) s += cnt[w] - 1; /* cnt[w] >= 1 because v is common */
      }
      out[e] = s;
    }
    for (uint64_t i = 0; i < nt; i++) cnt[list[i]] = 0;
  }
  free(cnt); free(list); free_vcsr(&t);
  return 0;
}

/* ------------------------------------------------ indexed min-heap
 * Keyed by (support, id): the minimum support first, ties by smallest id. */
typedef struct { uint64_t *key; uint64_t *heap; uint64_t *pos; uint64_t n; } heap_t;

static int hless(const heap_t *h, uint64_t a, uint64_t b) {
  return h->key[a] < h->key[b] || (h->key[a] == h->key[b] && a < b);
}
static void hswap(heap_t *h, uint64_t i, uint64_t j) {
  uint64_t a = h->heap[i], b = h->heap[j];
  h->heap[i] = b; h->heap[j] = a; h->pos[b] = i; h->pos[a] = j;
}
static void sift_up(heap_t *h, uint64_t i) {
  while (i > 0) {
    uint64_t p = (i - 1) / 2;
    if (!hless(h, h->heap[i], h->heap[p])) break;
    hswap(h, i, p); i = p;
  }
}
static void sift_down(heap_t *h, uint64_t i) {
  for (;;) {
    uint64_t l = 2 * i + 1, r = l + 1, b = i;
    if (l < h->n && hless(h, h->heap[l], h->heap[b])) b = l;
    if (r < h->n && hless(h, h->heap[r], h->heap[b])) b = r;
    if (b == i) break;
    hswap(h, i, b); i = b;
  }
}
static int heap_init(heap_t *h, uint64_t *key, uint64_t n) {
  h->key = key; h->n = n;
  h->heap = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
  h->pos = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
  if (!h->heap || !h->pos) { free(h->heap); free(h->pos); return -1; }
  for (uint64_t i = 0; i < n; i++) { h->heap[i] = i; h->pos[i] = i; }
  for (uint64_t i = n / 2; i-- > 0;) sift_down(h, i);
  return 0;
}
static uint64_t heap_pop(heap_t *h) {
  uint64_t top = h->heap[0];
  h->n--;
  if (h->n) { hswap(h, 0, h->n); sift_down(h, 0); }
  return top;
}
/* lower the key of id to k (k <= current key) */
static void heap_lower(heap_t *h, uint64_t id, uint64_t k) { h->key[id] = k; sift_up(h, h->pos[id]); }
static void heap_free(heap_t *h) { free(h->heap); free(h->pos); }

/* support <- max(level, support - dec) */
static uint64_t clamp_sub(uint64_t s, uint64_t dec, uint64_t level) {
  return (s >= level + dec) ? s - dec : level;
}

/* Tip decomposition of side U by bottom-up peeling (Alg. 2 applied to the
 * vertices of U, Sec. 2.2).  theta[u] receives the tip number of u. */
int oracle_tip_bup(uint32_t nu, uint32_t nv, const uint64_t *u_off, const uint32_t *u_adj, uint64_t *theta) {
  uint64_t *sup = (uint64_t *)malloc(((size_t)nu + 1) * sizeof(uint64_t));
  if (!sup) return -1;
  if (oracle_vertex_counts(nu, nv, u_off, u_adj, sup)) { free(sup); return -1; }
  vcsr_t t;
  if (make_vcsr(nu, nv, u_off, u_adj, &t)) { free(sup); return -1; }
  uint32_t *cnt = (uint32_t *)calloc((size_t)nu + 1, sizeof(uint32_t));
  uint32_t *list = (uint32_t *)malloc(((size_t)nu + 1) * sizeof(uint32_t));
  uint8_t *alive = (uint8_t *)malloc((size_t)nu + 1);
  heap_t h;
  if (!cnt || !list || !alive || heap_init(&h, sup, nu)) {
    free(cnt); free(list); free(alive); free(sup); free_vcsr(&t); return -1;
  }
  memset(alive, 1, nu);
  uint64_t level = 0;
  while (h.n) {
    uint32_t u = (uint32_t)heap_pop(&h);
    theta[u] = sup[u];          /* Alg. 2: the entity number is its support */
    level = sup[u];
    alive[u] = 0;
    uint64_t nt = common_counts(u, u_off, u_adj, &t, alive, cnt, list);
    for (uint64_t i = 0; i < nt; i++) {
      uint32_t w = list[i];
      uint64_t c = cnt[w];
      cnt[w] = 0;
      if (c >= 2) heap_lower(&h, w, clamp_sub(sup[w], choose2(c), level));
    }
  }
  heap_free(&h); free(cnt); free(list); free(alive); free(sup); free_vcsr(&t);
  return 0;
}

/* position of edge (u, v) in u_adj, or -1 */
static int64_t find_edge(const uint64_t *u_off, const uint32_t *u_adj, uint32_t u, uint32_t v) {
  uint64_t lo = u_off[u], hi = u_off[u + 1];
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (u_adj[mid] < v) lo = mid + 1; else hi = mid;
  }
  return (lo < u_off[u + 1] && u_adj[lo] == v) ? (int64_t)lo : -1;
}

/* Wing decomposition by bottom-up peeling (Alg. 2).  theta[e] receives the
 * wing number of edge e (edge id = position in u_adj). */
int oracle_wing_bup(uint32_t nu, uint32_t nv, const uint64_t *u_off, const uint32_t *u_adj, uint64_t *theta) {
  uint64_t m = u_off[nu];
  uint64_t *sup = (uint64_t *)malloc((size_t)(m ? m : 1) * sizeof(uint64_t));
  uint32_t *eu = (uint32_t *)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
  uint8_t *alive = (uint8_t *)malloc((size_t)(m ? m : 1));
  if (!sup || !eu || !alive) { free(sup); free(eu); free(alive); return -1; }
  if (oracle_edge_counts(nu, nv, u_off, u_adj, sup)) { free(sup); free(eu); free(alive); return -1; }
  vcsr_t t;
  if (make_vcsr(nu, nv, u_off, u_adj, &t)) { free(sup); free(eu); free(alive); return -1; }
  for (uint32_t u = 0; u < nu; u++)
    for (uint64_t e = u_off[u]; e < u_off[u + 1]; e++) eu[e] = u;
  memset(alive, 1, (size_t)m);
  heap_t h;
  if (heap_init(&h, sup, m)) { free(sup); free(eu); free(alive); free_vcsr(&t); return -1; }
  uint64_t level = 0;
  while (h.n) {
    uint64_t e = heap_pop(&h);
    theta[e] = sup[e];
    level = sup[e];
    alive[e] = 0;
    uint32_t u = eu[e], v = u_adj[e];
    /* butterflies (u, v, u', v') of the remaining graph: e1 = (u, v'),
     * e2 = (u', v), e3 = (u', v') must all still be present */
    for (uint64_t e1 = u_off[u]; e1 < u_off[u + 1]; e1++) {
      uint32_t v2 = u_adj[e1];
      if (v2 == v || !alive[e1]) continue;
      for (uint64_t q = t.off[v2]; q < t.off[v2 + 1]; q++) {
        uint32_t u2 = t.adj[q];
        uint64_t e3 = t.eid[q];
        if (u2 == u || !alive[e3]) continue;
        int64_t e2 = find_edge(u_off, u_adj, u2, v);
        if (e2 < 0 || !alive[e2]) continue;
        heap_lower(&h, e1, clamp_sub(sup[e1], 1, level));
        heap_lower(&h, (uint64_t)e2, clamp_sub(sup[e2], 1, level));
        heap_lower(&h, e3, clamp_sub(sup[e3], 1, level));
      }
    }
  }
  heap_free(&h); free(sup); free(eu); free(alive); free_vcsr(&t);
  return 0;
}

/* Butterflies that vertex u (side U) has with the members of side U marked
 * in member[] (u itself need not be marked): sum over members u' != u of
 * C(c(u,u'), 2).  Used for sampled checks at sizes where full peeling is
 * too slow.  Returns UINT64_MAX on allocation failure. */
uint64_t oracle_vertex_support_within(uint32_t nu, uint32_t nv, const uint64_t *u_off, const uint32_t *u_adj,
                                      const uint64_t *v_off, const uint32_t *v_adj, const uint8_t *member,
                                      uint32_t u) {
  uint32_t *cnt = (uint32_t *)calloc((size_t)nu + 1, sizeof(uint32_t));
  uint32_t *list = (uint32_t *)malloc(((size_t)nu + 1) * sizeof(uint32_t));
  if (!cnt || !list) { free(cnt); free(list); return UINT64_MAX; }
  (void)nv;
  uint64_t nt = 0, s = 0;
  for (uint64_t e = u_off[u]; e < u_off[u + 1]; e++) {
    uint32_t v = u_adj[e];
    for (uint64_t q = v_off[v]; q < v_off[v + 1]; q++) {
      uint32_t w = v_adj[q];
      if (w == u || !member[w]) continue;
      if (cnt[w]++ == 0) list[nt++] = w;
    }
  }
  for (uint64_t i = 0; i < nt; i++) s += choose2(cnt[list[i]]);
  free(cnt); free(list);
  return s;
}

/* Butterflies of edge e = (u, v) whose other three edges are all marked in
 * member[] (indexed by edge id).  Needs the V-side CSR with edge ids. */
uint64_t oracle_edge_support_within(uint32_t nu, const uint64_t *u_off, const uint32_t *u_adj,
                                    const uint64_t *v_off, const uint32_t *v_adj, const uint64_t *v_eid,
                                    const uint8_t *member, uint64_t e) {
  uint32_t u = 0;
  { /* owner of edge e */
    uint32_t lo = 0, hi = nu;
    while (hi - lo > 1) { uint32_t mid = lo + (hi - lo) / 2; if (u_off[mid] <= e) lo = mid; else hi = mid; }
    u = lo;
  }
  uint32_t v = u_adj[e];
  uint64_t s = 0;
  for (uint64_t e1 = u_off[u]; e1 < u_off[u + 1]; e1++) {
    uint32_t v2 = u_adj[e1];
    if (v2 == v || !member[e1]) continue;
    for (uint64_t q = v_off[v2]; q < v_off[v2 + 1]; q++) {
      uint32_t u2 = v_adj[q];
      uint64_t e3 = v_eid[q];
      if (u2 == u || !member[e3]) continue;
      int64_t e2 = find_edge(u_off, u_adj, u2, v);
      if (e2 >= 0 && member[e2]) s++;
    }
  }
  return s;
}

/* V-side CSR with edge ids, for callers of the *_within checks. */
int oracle_transpose(uint32_t nu, uint32_t nv, const uint64_t *u_off, const uint32_t *u_adj,
                     uint64_t *v_off, uint32_t *v_adj, uint64_t *v_eid) {
  vcsr_t t;
  if (make_vcsr(nu, nv, u_off, u_adj, &t)) return -1;
  uint64_t m = u_off[nu];
  memcpy(v_off, t.off, ((size_t)nv + 1) * sizeof(uint64_t));
  memcpy(v_adj, t.adj, (size_t)m * sizeof(uint32_t));
  memcpy(v_eid, t.eid, (size_t)m * sizeof(uint64_t));
  free_vcsr(&t);
  return 0;
}
