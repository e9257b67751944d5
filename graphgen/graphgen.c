/*
 * graphgen.c — seeded synthetic graph generators producing symmetric CSR.
 *
 * These graphs stand in for the SuiteSparse inputs of the paper's Table 1
 * (web/social/collaboration graphs with heavy-tailed degrees, and road
 * networks with average degree near 2).  Every generator is deterministic
 * given its seed and gives identical output on any IEEE-754 host: random
 * numbers come from a counter-based splitmix64 stream, and the only floating
 * point used (Bernoulli thresholds, geometric skips) is plain +,-,*,/ compiled
 * with -ffp-contract=off, with our own logarithm (no libm).
 *
 * This module holds none of the community-detection arithmetic; it is shared
 * by the tests, the benchmark and the request generator of the server.
 *
 * Output CSR convention (undirected weighted graph):
 *   - each edge {u,v}, u != v, is stored twice: (u,v) and (v,u), same weight;
 *   - a self-loop {u,u} is stored once;
 *   - rows are sorted by column, duplicate entries removed;
 *   - offsets are int64, columns int32, weights int32 > 0.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct {
  int64_t n, nnz;
  int64_t *off;   /* n + 1 */
  int32_t *col;   /* nnz */
  int32_t *w;     /* nnz */
  int32_t *truth; /* n, planted block per vertex (SBM only), else NULL */
} gg_csr;

/* ------------------------------------------------------------------ RNG */

static inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Counter-based stream: value i of stream s under seed. */
static inline uint64_t rnd(uint64_t key, uint64_t i) { return mix64(key + i * 0xD1B54A32D192ED03ull); }
static inline uint64_t stream_key(uint64_t seed, uint64_t s) { return mix64(mix64(seed) ^ (s * 0xA24BAED4963EE407ull)); }
static inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); } /* [0,1) */

/* Natural log for x in (0, 1], from frexp-free exponent extraction and the
 * atanh series log(m) = 2 * sum_k z^(2k+1)/(2k+1), z = (m-1)/(m+1).  Only
 * IEEE basic operations, so the result is identical on every host. */
static double gg_log(double x) {
  union { double d; uint64_t u; } v = {x};
  int e = (int)((v.u >> 52) & 0x7ff) - 1022;
  v.u = (v.u & 0x800FFFFFFFFFFFFFull) | 0x3FE0000000000000ull; /* m in [0.5,1) */
  double m = v.d;
  if (m < 0.70710678118654752) { m *= 2.0; e -= 1; }
  double z = (m - 1.0) / (m + 1.0), z2 = z * z, term = z, s = 0.0;
  for (int k = 0; k < 24; ++k) { s += term / (double)(2 * k + 1); term *= z2; }
  return 2.0 * s + (double)e * 0.69314718055994530942;
}

/* Number of failures before the next success of a Bernoulli(p) sequence. */
static inline int64_t geom_skip(uint64_t r, double lq /* log(1-p) */) {
  double u = 1.0 - u01(r); /* (0,1] */
  double k = gg_log(u) / lq;
  if (k > 9.0e18) return INT64_MAX / 4;
  return (int64_t)k;
}

static inline int32_t hashed_weight(uint64_t key, int64_t u, int64_t v, int32_t wmin, int32_t wmax) {
  if (u > v) { int64_t t = u; u = v; v = t; }
  uint64_t r = mix64(key ^ mix64(((uint64_t)u << 32) ^ (uint64_t)v));
  uint64_t span = (uint64_t)((int64_t)wmax - (int64_t)wmin + 1);
  return (int32_t)((int64_t)wmin + (int64_t)(r % span));
}


/* ---------------------------------------------------- parallel for-loop */

typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi, int tid);
typedef struct { range_fn fn; void *ctx; int64_t lo, hi; int tid; } range_job;

static void *range_run(void *p) {
  range_job *j = (range_job *)p;
  j->fn(j->ctx, j->lo, j->hi, j->tid);
  return NULL;
}

static int gg_threads(void) {
  const char *e = getenv("GRAPHGEN_THREADS");
  long t = e ? atol(e) : sysconf(_SC_NPROCESSORS_ONLN);
  if (t < 1) t = 1;
  if (t > 64) t = 64;
  return (int)t;
}

/* Set in worker threads of gg_sbm_batch: their builds run serially. */
static __thread int gg_in_worker = 0;

/* Split [0, total) into `nt` contiguous chunks, chunk i to thread i. */
static void parallel_for(int nt, int64_t total, range_fn fn, void *ctx) {
  pthread_t th[64];
  range_job jobs[64];
  int ok[64];
  if (total < 65536 || nt < 1 || gg_in_worker) nt = 1;
  if (nt > 64) nt = 64;
  for (int i = 0; i < nt; ++i) {
    jobs[i].fn = fn; jobs[i].ctx = ctx; jobs[i].tid = i;
    jobs[i].lo = total * i / nt; jobs[i].hi = total * (i + 1) / nt;
  }
  for (int i = 1; i < nt; ++i) {
    ok[i] = pthread_create(&th[i], NULL, range_run, &jobs[i]) == 0;
    if (!ok[i]) range_run(&jobs[i]); /* could not start a thread: run inline */
  }
  range_run(&jobs[0]);
  for (int i = 1; i < nt; ++i)
    if (ok[i]) pthread_join(th[i], NULL);
}

/* --------------------------------------------------------- edge buffers */

typedef struct { int64_t m, cap; int32_t *u, *v; } edgebuf;

static int eb_push(edgebuf *b, int64_t u, int64_t v) {
  if (b->m == b->cap) {
    int64_t nc = b->cap ? b->cap * 2 : 1024;
    int32_t *nu = (int32_t *)realloc(b->u, (size_t)nc * 4), *nv = (int32_t *)realloc(b->v, (size_t)nc * 4);
    if (!nu || !nv) { b->u = nu ? nu : b->u; b->v = nv ? nv : b->v; return -1; }
    b->u = nu; b->v = nv; b->cap = nc;
  }
  b->u[b->m] = (int32_t)u; b->v[b->m] = (int32_t)v; b->m++;
  return 0;
}
static void eb_free(edgebuf *b) { free(b->u); free(b->v); b->u = b->v = NULL; b->m = b->cap = 0; }

/* LSD radix sort of 64-bit keys on their low `bits` bits, 11 bits a pass;
 * each pass is a parallel histogram, a serial bucket scan, and a parallel
 * stable scatter (thread t owns chunk t, so the order is the serial one). */
#define RDX 2048
typedef struct { const uint64_t *src; uint64_t *dst; int sh; int64_t (*hist)[RDX]; } rdx_ctx;

static void rdx_hist(void *c, int64_t lo, int64_t hi, int tid) {
  rdx_ctx *x = (rdx_ctx *)c;
  int64_t *h = x->hist[tid];
  memset(h, 0, RDX * 8);
  for (int64_t i = lo; i < hi; ++i) h[(x->src[i] >> x->sh) & (RDX - 1)]++;
}
static void rdx_scatter(void *c, int64_t lo, int64_t hi, int tid) {
  rdx_ctx *x = (rdx_ctx *)c;
  int64_t *h = x->hist[tid];
  for (int64_t i = lo; i < hi; ++i) x->dst[h[(x->src[i] >> x->sh) & (RDX - 1)]++] = x->src[i];
}

static int radix_sort_u64(uint64_t *a, int64_t E, int bits) {
  int nt = gg_threads();
  if (E < 65536 || gg_in_worker) nt = 1;
  uint64_t *t = (uint64_t *)malloc((size_t)(E ? E : 1) * 8);
  int64_t(*h)[RDX] = (int64_t(*)[RDX])malloc((size_t)nt * RDX * 8);
  if (!t || !h) { free(t); free(h); return -1; }
  int passes = 0;
  for (int sh = 0; sh < bits; sh += 11) {
    rdx_ctx cx = {a, t, sh, h};
    parallel_for(nt, E, rdx_hist, &cx);
    int64_t s = 0;
    for (int d = 0; d < RDX; ++d)
      for (int i = 0; i < nt; ++i) { int64_t c = h[i][d]; h[i][d] = s; s += c; }
    parallel_for(nt, E, rdx_scatter, &cx);
    uint64_t *x = a; a = t; t = x;
    ++passes;
  }
  if (passes & 1) { memcpy(t, a, (size_t)E * 8); free(a); } else free(t);
  free(h);
  return 0;
}

typedef struct { const uint64_t *key; int32_t *col, *w; int vb; uint64_t vmask, wkey; int32_t wmin, wmax; } fill_ctx;
static void fill_rows(void *c, int64_t lo, int64_t hi, int tid) {
  fill_ctx *f = (fill_ctx *)c;
  (void)tid;
  for (int64_t i = lo; i < hi; ++i) {
    int64_t u = (int64_t)(f->key[i] >> f->vb), v = (int64_t)(f->key[i] & f->vmask);
    f->col[i] = (int32_t)v;
    f->w[i] = hashed_weight(f->wkey, u, v, f->wmin, f->wmax);
  }
}

/* Symmetrise an undirected edge list into a canonical CSR: both directions
 * for u != v, one entry for a self-loop (dropped if keep_loops == 0),
 * duplicates removed; weights are a hash of the unordered pair so both
 * directions agree.  Entries are sorted as packed (u << 32 | v) keys. */
static int build_csr(int64_t n, const edgebuf *e, int keep_loops, uint64_t wkey, int32_t wmin, int32_t wmax,
                     gg_csr *out) {
  memset(out, 0, sizeof(*out));
  out->n = n;
  int64_t E = 0;
  for (int64_t i = 0; i < e->m; ++i) E += (e->u[i] == e->v[i]) ? (keep_loops ? 1 : 0) : 2;
  uint64_t *key = (uint64_t *)malloc((size_t)(E ? E : 1) * 8);
  if (!key) return -1;
  int64_t k = 0;
  for (int64_t i = 0; i < e->m; ++i) {
    uint64_t a = (uint32_t)e->u[i], b = (uint32_t)e->v[i];
    if (a == b) { if (keep_loops) key[k++] = (a << 32) | b; continue; }
    key[k++] = (a << 32) | b;
    key[k++] = (b << 32) | a;
  }
  int vb = 1;
  while (((int64_t)1 << vb) < n) ++vb;
  /* sort on v bits then u bits: pack u just above v to cut passes */
  for (int64_t i = 0; i < E; ++i) key[i] = ((key[i] >> 32) << vb) | (key[i] & 0xffffffffull);
  if (radix_sort_u64(key, E, 2 * vb)) { free(key); return -1; }
  uint64_t vmask = ((uint64_t)1 << vb) - 1;
  int64_t nnz = 0;
  for (int64_t i = 0; i < E; ++i) {
    if (nnz > 0 && key[nnz - 1] == key[i]) continue;
    key[nnz++] = key[i];
  }
  out->off = (int64_t *)calloc((size_t)n + 1, 8);
  out->col = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * 4);
  out->w = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * 4);
  if (!out->off || !out->col || !out->w) { free(key); return -1; }
  {
    fill_ctx fc = {key, out->col, out->w, vb, vmask, wkey, wmin, wmax};
    parallel_for(gg_threads(), nnz, fill_rows, &fc);
  }
  for (int64_t i = 0; i < nnz; ++i) out->off[(key[i] >> vb) + 1]++;
  for (int64_t i = 0; i < n; ++i) out->off[i + 1] += out->off[i];
  out->nnz = nnz;
  free(key);
  return 0;
}

/* Seeded Fisher-Yates permutation of 0..n-1. */
static int32_t *make_perm(uint64_t key, int64_t n) {
  int32_t *p = (int32_t *)malloc((size_t)(n ? n : 1) * 4);
  if (!p) return NULL;
  for (int64_t i = 0; i < n; ++i) p[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    int64_t j = (int64_t)(rnd(key, (uint64_t)i) % (uint64_t)(i + 1));
    int32_t t = p[i]; p[i] = p[j]; p[j] = t;
  }
  return p;
}

/* --------------------------------------------------------------- public */

void gg_free(gg_csr *g) {
  if (!g) return;
  free(g->off); free(g->col); free(g->w); free(g->truth);
  memset(g, 0, sizeof(*g));
}

/* Edge list to CSR (for hand-made graphs): m undirected edges. */
int gg_from_edges(int64_t n, int64_t m, const int32_t *u, const int32_t *v, int keep_loops, uint64_t seed,
                  int32_t wmin, int32_t wmax, gg_csr *out) {
  edgebuf e = {0, 0, NULL, NULL};
  for (int64_t i = 0; i < m; ++i) {
    if (u[i] < 0 || u[i] >= n || v[i] < 0 || v[i] >= n) { eb_free(&e); return -2; }
    if (eb_push(&e, u[i], v[i])) { eb_free(&e); return -1; }
  }
  int rc = build_csr(n, &e, keep_loops, stream_key(seed, 99), wmin, wmax, out);
  eb_free(&e);
  return rc;
}

/* Planted-partition stochastic block model.  Vertices are split into k
 * blocks of near-equal size (the first n % k blocks one larger); a pair is an
 * edge with probability p_in inside a block and p_out across blocks.
 * Vertex ids are shuffled with a seeded permutation (so ids carry no block
 * locality); truth[v] is the planted block of vertex v. */
int gg_sbm(uint64_t seed, int64_t n, int64_t k, double p_in, double p_out, int32_t wmin, int32_t wmax,
           gg_csr *out) {
  memset(out, 0, sizeof(*out));
  if (n < 0 || k < 1 || k > (n ? n : 1) || p_in < 0 || p_in > 1 || p_out < 0 || p_out > 1) return -2;
  int64_t *bstart = (int64_t *)malloc((size_t)(k + 1) * 8);
  int32_t *blk = (int32_t *)malloc((size_t)(n ? n : 1) * 4);
  int32_t *perm = make_perm(stream_key(seed, 1), n);
  if (!bstart || !blk || !perm) { free(bstart); free(blk); free(perm); return -1; }
  int64_t base = n / k, rem = n % k, s = 0;
  for (int64_t b = 0; b < k; ++b) { bstart[b] = s; s += base + (b < rem ? 1 : 0); }
  bstart[k] = n;
  for (int64_t b = 0; b < k; ++b)
    for (int64_t x = bstart[b]; x < bstart[b + 1]; ++x) blk[x] = (int32_t)b;
  edgebuf e = {0, 0, NULL, NULL};
  uint64_t key_in = stream_key(seed, 2), key_out = stream_key(seed, 3);
  uint64_t ctr = 0;
  /* Within-block pairs (x, y), x < y, flattened row by row; geometric skips. */
  if (p_in > 0) {
    double lq = (p_in < 1.0) ? gg_log(1.0 - p_in) : 0.0;
    for (int64_t b = 0; b < k; ++b) {
      int64_t lo = bstart[b], hi = bstart[b + 1];
      int64_t x = lo, y = lo; /* current candidate is (x, y+1..) */
      for (;;) {
        int64_t skip = (p_in >= 1.0) ? 0 : geom_skip(rnd(key_in, ctr++), lq);
        int64_t t = y + 1 + skip; /* next y */
        while (x < hi && t >= hi) { t = t - hi + (x + 2); x += 1; }
        if (x >= hi - 1) break;
        y = t;
        if (eb_push(&e, perm[x], perm[y])) goto oom;
      }
    }
  }
  /* Cross-block pairs: for row x, candidates are y in [end of x's block, n). */
  if (p_out > 0 && k > 1) {
    double lq = (p_out < 1.0) ? gg_log(1.0 - p_out) : 0.0;
    int64_t x = 0, y = (n > 0) ? bstart[blk[0] + 1] - 1 : 0;
    for (;;) {
      int64_t skip = (p_out >= 1.0) ? 0 : geom_skip(rnd(key_out, ctr++), lq);
      int64_t t = y + 1 + skip;
      while (x < n && t >= n) { x += 1; if (x >= n) break; t = t - n + bstart[blk[x] + 1]; }
      if (x >= n) break;
      y = t;
      if (eb_push(&e, perm[x], perm[y])) goto oom;
    }
  }
  if (build_csr(n, &e, 1, stream_key(seed, 4), wmin, wmax, out)) goto oom;
  eb_free(&e);
  out->truth = (int32_t *)malloc((size_t)(n ? n : 1) * 4);
  if (!out->truth) { gg_free(out); free(bstart); free(blk); free(perm); return -1; }
  for (int64_t x = 0; x < n; ++x) out->truth[perm[x]] = blk[x];
  free(bstart); free(blk); free(perm);
  return 0;
oom:
  eb_free(&e); free(bstart); free(blk); free(perm); gg_free(out);
  return -1;
}

typedef struct { uint64_t key; int scale; int64_t n, N; uint64_t ta, tb, tc; const int32_t *perm; int32_t *u, *v; } rmat_ctx;
static void rmat_edges(void *c, int64_t lo, int64_t hi, int tid) {
  rmat_ctx *x = (rmat_ctx *)c;
  (void)tid;
  for (int64_t i = lo; i < hi; ++i) {
    int64_t u = 0, v = 0;
    uint64_t r = 0;
    for (int l = 0; l < x->scale; ++l) {
      if ((l & 1) == 0) r = rnd(x->key, (uint64_t)i * 16 + (uint64_t)(l >> 1));
      uint64_t q = (l & 1) ? (r >> 32) : (r & 0xffffffffull);
      /* quadrants in order a (0,0), b (0,1), c (1,0), d (1,1) */
      int64_t bu = (int64_t)(q >= x->tb), bv = (int64_t)((q >= x->ta) & (q < x->tb)) | (int64_t)(q >= x->tc);
      u = (u << 1) | bu; v = (v << 1) | bv;
    }
    if (x->n != x->N) { u %= x->n; v %= x->n; }
    x->u[i] = x->perm[u]; x->v[i] = x->perm[v];
  }
}

/* R-MAT (Chakrabarti et al.): m = edge_factor * 2^scale edges, each drawn by
 * descending `scale` levels of the 2x2 recursive matrix with probabilities
 * (a, b, c, d = 1-a-b-c).  Endpoints are then reduced mod n (n <= 2^scale;
 * n = 0 means 2^scale) and relabelled by a seeded permutation.  Self-loops
 * are removed and duplicate edges merged (one hashed weight per unordered
 * pair), then the list is symmetrised. */
int gg_rmat(uint64_t seed, int scale, int64_t n, double edge_factor, double a, double b, double c, int32_t wmin,
            int32_t wmax, gg_csr *out) {
  memset(out, 0, sizeof(*out));
  if (scale < 1 || scale > 30 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0 || edge_factor < 0) return -2;
  int64_t N = (int64_t)1 << scale;
  if (n <= 0) n = N;
  if (n > N) return -2;
  int64_t m = (int64_t)(edge_factor * (double)N + 0.5);
  uint64_t ta = (uint64_t)(a * 4294967296.0), tb = (uint64_t)((a + b) * 4294967296.0),
           tc = (uint64_t)((a + b + c) * 4294967296.0);
  uint64_t key = stream_key(seed, 5);
  int32_t *perm = make_perm(stream_key(seed, 6), n);
  edgebuf e = {0, 0, NULL, NULL};
  if (!perm) return -1;
  e.cap = m ? m : 1;
  e.u = (int32_t *)malloc((size_t)e.cap * 4); e.v = (int32_t *)malloc((size_t)e.cap * 4);
  if (!e.u || !e.v) { eb_free(&e); free(perm); return -1; }
  {
    rmat_ctx rc = {key, scale, n, N, ta, tb, tc, perm, e.u, e.v};
    parallel_for(gg_threads(), m, rmat_edges, &rc);
    e.m = m;
  }
  free(perm);
  int rc = build_csr(n, &e, 0, stream_key(seed, 7), wmin, wmax, out);
  eb_free(&e);
  return rc;
}

/* Road-like graph: side x side 4-neighbour grid, each grid edge kept with
 * probability 1 - drop, plus round(shortcut_frac * kept) uniform random
 * long-range edges; vertex id = row * side + column (spatial locality kept,
 * as in OpenStreetMap exports). */
int gg_grid_road(uint64_t seed, int64_t side, double drop, double shortcut_frac, int32_t wmin, int32_t wmax,
                 gg_csr *out) {
  memset(out, 0, sizeof(*out));
  if (side < 1 || side > 46340 || drop < 0 || drop > 1 || shortcut_frac < 0) return -2;
  int64_t n = side * side;
  uint64_t key = stream_key(seed, 8), skey = stream_key(seed, 9);
  uint64_t keep_thr = (uint64_t)((1.0 - drop) * 18446744073709551615.0);
  if (drop <= 0.0) keep_thr = UINT64_MAX;
  edgebuf e = {0, 0, NULL, NULL};
  e.cap = 2 * n + 16;
  e.u = (int32_t *)malloc((size_t)e.cap * 4); e.v = (int32_t *)malloc((size_t)e.cap * 4);
  if (!e.u || !e.v) { eb_free(&e); return -1; }
  for (int64_t r = 0; r < side; ++r)
    for (int64_t c = 0; c < side; ++c) {
      int64_t x = r * side + c;
      if (c + 1 < side && (drop <= 0.0 || rnd(key, (uint64_t)x * 2) < keep_thr))
        if (eb_push(&e, x, x + 1)) goto oom;
      if (r + 1 < side && (drop <= 0.0 || rnd(key, (uint64_t)x * 2 + 1) < keep_thr))
        if (eb_push(&e, x, x + side)) goto oom;
    }
  {
    int64_t kept = e.m;
    int64_t ns = (int64_t)(shortcut_frac * (double)kept + 0.5);
    for (int64_t i = 0; i < ns && n > 1; ++i) {
      uint64_t r = rnd(skey, (uint64_t)i);
      int64_t u = (int64_t)((r & 0xffffffffull) % (uint64_t)n), v = (int64_t)((r >> 32) % (uint64_t)n);
      if (u == v) v = (v + 1) % n;
      if (eb_push(&e, u, v)) goto oom;
    }
  }
  {
    int rc = build_csr(n, &e, 0, stream_key(seed, 10), wmin, wmax, out);
    eb_free(&e);
    return rc;
  }
oom:
  eb_free(&e); gg_free(out);
  return -1;
}

/* Counter-based uniform double in [0,1): exported for the host-side request
 * generators (log-uniform sizes, Poisson arrivals) so they share the stream. */
double gg_uniform(uint64_t seed, uint64_t stream, uint64_t i) { return u01(rnd(stream_key(seed, stream), i)); }
double gg_logn(double x) { return gg_log(x); }

/* Many SBM graphs at once, built on a pool of threads (one graph per task),
 * then packed into one block-diagonal CSR: graph g owns vertices
 * [vo[g], vo[g+1]).  Specs per graph: seed, n, k, p_in, p_out. */
typedef struct {
  int64_t count;
  const uint64_t *seed;
  const int64_t *n, *k;
  const double *p_in, *p_out;
  int32_t wmin, wmax;
  gg_csr *parts;
  int64_t next;
  pthread_mutex_t mu;
  int failed;
} batch_job;

static void *batch_worker(void *p) {
  batch_job *b = (batch_job *)p;
  gg_in_worker = 1;
  for (;;) {
    pthread_mutex_lock(&b->mu);
    int64_t g = b->next++;
    pthread_mutex_unlock(&b->mu);
    if (g >= b->count) break;
    if (gg_sbm(b->seed[g], b->n[g], b->k[g], b->p_in[g], b->p_out[g], b->wmin, b->wmax, &b->parts[g])) {
      pthread_mutex_lock(&b->mu);
      b->failed = 1;
      pthread_mutex_unlock(&b->mu);
    }
  }
  return NULL;
}

int gg_sbm_batch(int64_t count, const uint64_t *seed, const int64_t *n, const int64_t *k, const double *p_in,
                 const double *p_out, int32_t wmin, int32_t wmax, gg_csr *out, int64_t *vo) {
  memset(out, 0, sizeof(*out));
  batch_job b;
  memset(&b, 0, sizeof(b));
  b.count = count; b.seed = seed; b.n = n; b.k = k; b.p_in = p_in; b.p_out = p_out;
  b.wmin = wmin; b.wmax = wmax;
  b.parts = (gg_csr *)calloc((size_t)(count ? count : 1), sizeof(gg_csr));
  if (!b.parts) return -1;
  pthread_mutex_init(&b.mu, NULL);
  int nt = gg_threads();
  pthread_t th[64];
  int ok[64];
  for (int i = 0; i < nt; ++i) ok[i] = pthread_create(&th[i], NULL, batch_worker, &b) == 0;
  for (int i = 0; i < nt; ++i)
    if (ok[i]) pthread_join(th[i], NULL);
  batch_worker(&b); /* finishes whatever threads could not be started */
  pthread_mutex_destroy(&b.mu);
  int rc = b.failed ? -1 : 0;
  int64_t N = 0, E = 0;
  vo[0] = 0;
  for (int64_t g = 0; g < count && !rc; ++g) {
    N += b.parts[g].n;
    E += b.parts[g].nnz;
    vo[g + 1] = N;
  }
  if (!rc) {
    out->n = N;
    out->nnz = E;
    out->off = (int64_t *)malloc((size_t)(N + 1) * 8);
    out->col = (int32_t *)malloc((size_t)(E ? E : 1) * 4);
    out->w = (int32_t *)malloc((size_t)(E ? E : 1) * 4);
    out->truth = (int32_t *)malloc((size_t)(N ? N : 1) * 4);
    if (!out->off || !out->col || !out->w || !out->truth) rc = -1;
  }
  if (!rc) {
    int64_t e0 = 0;
    out->off[0] = 0;
    for (int64_t g = 0; g < count; ++g) {
      gg_csr *p = &b.parts[g];
      int64_t v0 = vo[g];
      for (int64_t i = 0; i < p->n; ++i) {
        out->off[v0 + i + 1] = p->off[i + 1] + e0;
        out->truth[v0 + i] = p->truth ? p->truth[i] : 0;
      }
      for (int64_t x = 0; x < p->nnz; ++x) {
        out->col[e0 + x] = p->col[x] + (int32_t)v0;
        out->w[e0 + x] = p->w[x];
      }
      e0 += p->nnz;
    }
  }
  for (int64_t g = 0; g < count; ++g) gg_free(&b.parts[g]);
  free(b.parts);
  if (rc) gg_free(out);
  return rc;
}
