/*
 * Seeded synthetic bipartite graph generators.
 *
 * This module is shared by the CPU oracle and the GPU library's tests and
 * benchmark.  It holds none of the butterfly / peeling arithmetic: it only
 * draws edge sets and writes them as a sorted U-side CSR.
 *
 * Determinism: every random number comes from xoshiro256** seeded through
 * splitmix64 (integer only), and the only floating point used (Chung-Lu
 * weights, log-uniform draws) is computed with +,-,*,/ alone by det_log /
 * det_exp below.  Built with -ffp-contract=off, the same seed yields the
 * same graph on x86-64 and on aarch64.
 *
 * Workload shapes follow the synthetic stand-ins for the paper's KONECT
 * graphs (Sec. 6.1, Tab. 2): uniform random, Chung-Lu power-law with a
 * degree cap, and Chung-Lu with planted dense bicliques.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ RNG */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static void rng_seed(rng_t *r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}
static uint64_t rng_next(rng_t *r) {
  uint64_t *s = r->s;
  uint64_t res = rotl64(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = rotl64(s[3], 45);
  return res;
}
/* uniform integer in [0, n) (n > 0), multiply-shift */
static uint64_t rng_below(rng_t *r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}
/* uniform double in [0, 1) */
static double rng_unit(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* --------------------------------------- deterministic log / exp / pow */
static const double DLN2 = 0.69314718055994530942;

/* natural log for x > 0: x = f * 2^k with f in [0.75, 1.5), then
 * ln f = 2 atanh(z), z = (f-1)/(f+1), by its power series. */
static double det_log(double x) {
  int k = 0;
  while (x >= 1.5) { x *= 0.5; k++; }
  while (x < 0.75) { x *= 2.0; k--; }
  double z = (x - 1.0) / (x + 1.0), z2 = z * z, term = z, sum = 0.0;
  for (int i = 0; i < 24; i++) { sum += term / (double)(2 * i + 1); term *= z2; }
  return 2.0 * sum + (double)k * DLN2;
}
/* e^y: y = k ln2 + r, |r| <= ln2/2, Taylor series for e^r, times 2^k */
static double det_exp(double y) {
  double kf = y / DLN2;
  long k = (long)(kf >= 0 ? kf + 0.5 : kf - 0.5);
  double r = y - (double)k * DLN2, term = 1.0, sum = 1.0;
  for (int i = 1; i < 28; i++) { term *= r / (double)i; sum += term; }
  while (k > 0) { sum *= 2.0; k--; }
  while (k < 0) { sum *= 0.5; k++; }
  return sum;
}
static double det_pow(double x, double a) { return det_exp(a * det_log(x)); }

/* ------------------------------------------------------ edge hash set */
typedef struct {
  uint64_t *slot; uint64_t cap; /* power of two; empty slot = ~0 */
  uint64_t *keys; uint64_t n, kcap; /* insertion-ordered key list */
} eset_t;

static uint64_t mix64(uint64_t k) {
  k ^= k >> 33; k *= 0xff51afd7ed558ccdull; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ull; k ^= k >> 33;
  return k;
}
static int eset_init(eset_t *s, uint64_t max_keys) {
  uint64_t cap = 1024;
  while (cap < 2 * max_keys + 16) cap <<= 1;
  s->slot = (uint64_t *)malloc(cap * sizeof(uint64_t));
  s->keys = (uint64_t *)malloc((max_keys + 1) * sizeof(uint64_t));
  if (!s->slot || !s->keys) { free(s->slot); free(s->keys); return -1; }
  memset(s->slot, 0xff, cap * sizeof(uint64_t));
  s->cap = cap; s->n = 0; s->kcap = max_keys;
  return 0;
}
static void eset_free(eset_t *s) { free(s->slot); free(s->keys); }
/* returns 1 if inserted, 0 if present, -1 if full */
static int eset_insert(eset_t *s, uint64_t key) {
  uint64_t h = mix64(key) & (s->cap - 1);
  while (s->slot[h] != ~0ull) {
    if (s->slot[h] == key) return 0;
    h = (h + 1) & (s->cap - 1);
  }
  if (s->n >= s->kcap) return -1;
  s->slot[h] = key;
  s->keys[s->n++] = key;
  return 1;
}
/* LSD radix sort of 64-bit keys, 16 bits per pass */
static int sort_u64(uint64_t *a, uint64_t n) {
  uint64_t *tmp = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
  uint64_t *cnt = (uint64_t *)malloc(65536 * sizeof(uint64_t));
  if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
  uint64_t *src = a, *dst = tmp;
  for (int pass = 0; pass < 4; pass++) {
    int sh = pass * 16;
    memset(cnt, 0, 65536 * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; i++) cnt[(src[i] >> sh) & 0xffff]++;
    uint64_t acc = 0;
    for (int b = 0; b < 65536; b++) { uint64_t c = cnt[b]; cnt[b] = acc; acc += c; }
    for (uint64_t i = 0; i < n; i++) dst[cnt[(src[i] >> sh) & 0xffff]++] = src[i];
    uint64_t *t = src; src = dst; dst = t;
  }
  /* 4 passes: result is back in a */
  free(tmp); free(cnt);
  return 0;
}

/* write sorted keys (u<<32|v) as a CSR; returns 0 */
static void keys_to_csr(const uint64_t *keys, uint64_t m, uint32_t nu, uint64_t *u_off, uint32_t *u_adj) {
  memset(u_off, 0, (size_t)(nu + 1) * sizeof(uint64_t));
  for (uint64_t i = 0; i < m; i++) u_off[(keys[i] >> 32) + 1]++;
  for (uint32_t u = 0; u < nu; u++) u_off[u + 1] += u_off[u];
  for (uint64_t i = 0; i < m; i++) u_adj[i] = (uint32_t)(keys[i] & 0xffffffffull);
}

/* ------------------------------------------------------------ uniform */
/* m distinct (u, v) pairs drawn uniformly.  u_off has nu+1 entries, u_adj m.
 * Returns the edge count, or a negative value on error. */
int64_t gen_uniform(uint32_t nu, uint32_t nv, uint64_t m, uint64_t seed, uint64_t *u_off, uint32_t *u_adj) {
  if ((double)m > 0.9 * (double)nu * (double)nv) return -1;
  rng_t r; rng_seed(&r, seed);
  eset_t s;
  if (eset_init(&s, m)) return -2;
  while (s.n < m) {
    uint64_t u = rng_below(&r, nu), v = rng_below(&r, nv);
    eset_insert(&s, (u << 32) | v);
  }
  if (sort_u64(s.keys, m)) { eset_free(&s); return -2; }
  keys_to_csr(s.keys, m, nu, u_off, u_adj);
  eset_free(&s);
  return (int64_t)m;
}

/* ------------------------------------------------------------ Chung-Lu */
/* Integer sampling weights for one side: expected degree of vertex i is
 * proportional to (i+1)^(-1/(gamma-1)), scaled to sum m and clipped at cap. */
static uint64_t *cl_cumweights(uint32_t n, uint64_t m, double gamma, uint32_t cap) {
  double beta = 1.0 / (gamma - 1.0);
  double *raw = (double *)malloc((size_t)n * sizeof(double));
  uint64_t *cum = (uint64_t *)malloc((size_t)(n + 1) * sizeof(uint64_t));
  if (!raw || !cum) { free(raw); free(cum); return NULL; }
  double sum = 0.0;
  for (uint32_t i = 0; i < n; i++) { raw[i] = det_pow((double)i + 1.0, -beta); sum += raw[i]; }
  cum[0] = 0;
  for (uint32_t i = 0; i < n; i++) {
    double d = (double)m * raw[i] / sum;
    if (d > (double)cap) d = (double)cap;
    uint64_t w = (uint64_t)(d * 256.0) + 1;
    cum[i + 1] = cum[i] + w;
  }
  free(raw);
  return cum;
}
static uint32_t cl_draw(rng_t *r, const uint64_t *cum, uint32_t n) {
  uint64_t x = rng_below(r, cum[n]);
  uint32_t lo = 0, hi = n; /* find i with cum[i] <= x < cum[i+1] */
  while (hi - lo > 1) {
    uint32_t mid = lo + (hi - lo) / 2;
    if (cum[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

/* Chung-Lu bipartite graph with m distinct edges, exponents gu (U) and gv (V),
 * degree cap dmax (also clipped to the other side's size), plus nplant planted
 * bicliques of size a x b with a, b uniform in [plant_lo, plant_hi] on random
 * vertex subsets (union with the Chung-Lu edges).  cap_edges is the capacity
 * of u_adj.  Returns the final edge count, or a negative value on error. */
int64_t gen_chung_lu(uint32_t nu, uint32_t nv, uint64_t m, double gu, double gv, uint32_t dmax,
                     uint32_t nplant, uint32_t plant_lo, uint32_t plant_hi, uint64_t seed,
                     uint64_t cap_edges, uint64_t *u_off, uint32_t *u_adj) {
  if (nu == 0 || nv == 0 || gu <= 1.0 || gv <= 1.0) return -1;
  uint32_t cap_u = dmax < nv ? dmax : nv, cap_v = dmax < nu ? dmax : nu;
  if ((double)m > 0.5 * (double)nu * (double)nv) return -1;
  uint64_t max_plant = (uint64_t)nplant * plant_hi * plant_hi;
  if (m + max_plant > cap_edges) return -3;
  rng_t r; rng_seed(&r, seed);
  uint64_t *cu = cl_cumweights(nu, m, gu, cap_u), *cv = cl_cumweights(nv, m, gv, cap_v);
  uint32_t *du = (uint32_t *)calloc(nu, sizeof(uint32_t)), *dv = (uint32_t *)calloc(nv, sizeof(uint32_t));
  eset_t s;
  if (!cu || !cv || !du || !dv || eset_init(&s, m + max_plant)) {
    free(cu); free(cv); free(du); free(dv); return -2;
  }
  uint64_t attempts = 0, limit = 200 * m + 1000000;
  int64_t rc = 0;
  while (s.n < m) {
    if (++attempts > limit) { rc = -4; break; }
    uint32_t u = cl_draw(&r, cu, nu), v = cl_draw(&r, cv, nv);
    if (du[u] >= cap_u || dv[v] >= cap_v) continue;
    if (eset_insert(&s, ((uint64_t)u << 32) | v) == 1) { du[u]++; dv[v]++; }
  }
  if (rc == 0 && nplant) {
    uint8_t *mu = (uint8_t *)calloc(nu, 1), *mv = (uint8_t *)calloc(nv, 1);
    uint32_t *pu = (uint32_t *)malloc((size_t)plant_hi * sizeof(uint32_t));
    uint32_t *pv = (uint32_t *)malloc((size_t)plant_hi * sizeof(uint32_t));
    if (!mu || !mv || !pu || !pv) rc = -2;
    for (uint32_t p = 0; rc == 0 && p < nplant; p++) {
      uint32_t a = plant_lo + (uint32_t)rng_below(&r, plant_hi - plant_lo + 1);
      uint32_t b = plant_lo + (uint32_t)rng_below(&r, plant_hi - plant_lo + 1);
      if (a > nu) a = nu;
      if (b > nv) b = nv;
      for (uint32_t i = 0; i < a;) { uint32_t x = (uint32_t)rng_below(&r, nu); if (!mu[x]) { mu[x] = 1; pu[i++] = x; } }
      for (uint32_t j = 0; j < b;) { uint32_t y = (uint32_t)rng_below(&r, nv); if (!mv[y]) { mv[y] = 1; pv[j++] = y; } }
      for (uint32_t i = 0; i < a; i++)
        for (uint32_t j = 0; j < b; j++) eset_insert(&s, ((uint64_t)pu[i] << 32) | pv[j]);
      for (uint32_t i = 0; i < a; i++) mu[pu[i]] = 0;
      for (uint32_t j = 0; j < b; j++) mv[pv[j]] = 0;
    }
    free(mu); free(mv); free(pu); free(pv);
  }
  if (rc == 0) {
    if (sort_u64(s.keys, s.n)) rc = -2;
    else { keys_to_csr(s.keys, s.n, nu, u_off, u_adj); rc = (int64_t)s.n; }
  }
  eset_free(&s); free(cu); free(cv); free(du); free(dv);
  return rc;
}

/* Draw the shape of one graph of a heterogeneous batch: edge count
 * log-uniform in [m_lo, m_hi], |U|:|V| ratio uniform in [r_lo, r_hi],
 * exponent uniform in [g_lo, g_hi], plant count uniform in [0, plant_max].
 * out: [m, nu, nv, nplant, dmax] and gamma in *gamma. */
void gen_batch_shape(uint64_t seed, uint64_t m_lo, uint64_t m_hi, double r_lo, double r_hi,
                     double g_lo, double g_hi, uint32_t plant_max, uint32_t dmax_cap,
                     uint64_t *out, double *gamma) {
  rng_t r; rng_seed(&r, seed ^ 0x5bd1e995ull);
  double lm = det_log((double)m_lo) + rng_unit(&r) * (det_log((double)m_hi) - det_log((double)m_lo));
  uint64_t m = (uint64_t)det_exp(lm);
  if (m < m_lo) m = m_lo;
  if (m > m_hi) m = m_hi;
  double ratio = r_lo + rng_unit(&r) * (r_hi - r_lo);
  double g = g_lo + rng_unit(&r) * (g_hi - g_lo);
  uint32_t nplant = (uint32_t)rng_below(&r, (uint64_t)plant_max + 1);
  uint64_t n = m / 5;
  uint64_t nu = (uint64_t)((double)n * ratio / (1.0 + ratio) + 0.5);
  if (nu < 2) nu = 2;
  uint64_t nv = n > nu + 2 ? n - nu : 2;
  /* keep the edge count samplable */
  while ((double)m > 0.25 * (double)nu * (double)nv) { nu += nu / 4 + 1; nv += nv / 4 + 1; }
  uint64_t other = nu < nv ? nu : nv;
  uint64_t dmax = other / 2 < dmax_cap ? other / 2 : dmax_cap;
  /* the cap must leave room for m edges on both sides */
  uint64_t need_u = (3 * m + nu - 1) / nu, need_v = (3 * m + nv - 1) / nv;
  if (dmax < need_u) dmax = need_u;
  if (dmax < need_v) dmax = need_v;
  if (dmax < 2) dmax = 2;
  out[0] = m; out[1] = nu; out[2] = nv; out[3] = nplant; out[4] = dmax;
  *gamma = g;
}

/* test hook: the deterministic math used for the weights */
double gen_det_pow(double x, double a) { return det_pow(x, a); }
