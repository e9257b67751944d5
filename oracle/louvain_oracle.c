/*
 * louvain_oracle.c — plain, single-threaded reference of the Louvain method.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA engine is
 * checked against.  Only the tests, the smoke check and the CPU-baseline /
 * reference arm of the benchmark may load it; the engine never calls it and
 * shares no code, header or table with it.
 *
 * What it follows (Section 3.2 of the paper, "Louvain algorithm"):
 *   - every vertex starts in its own community;
 *   - local-moving phase: each vertex moves to the neighbouring community
 *     with the greatest modularity increase, or stays if none increases it;
 *     the phase repeats while the total modularity change of an iteration is
 *     above `tolerance`;
 *   - aggregation phase: each community becomes a super-vertex; edges between
 *     communities are merged with summed weights, edges inside a community
 *     become a summed self-loop;
 *   - a pass is local-moving + aggregation; passes repeat while the pass's
 *     modularity increase is above `pass_tolerance` (0);
 *   - threshold scaling: tolerance starts at 0.01 and is divided by the
 *     decline factor 10 after every pass;
 *   - asynchronous (Gauss-Seidel) and synchronous (Jacobi) variants;
 *   - the top level of the dendrogram is the result.
 *
 * The paper writes no formula; modularity is Newman-Girvan with resolution
 * 1 in this CSR convention (each undirected edge stored in both directions,
 * a self-loop stored once):
 *   K_i      = sum of row i (self-loop included),  M = sum_i K_i,
 *   L_c      = sum of entries (u,v) with u and v in c,
 *   Sigma_c  = sum of K_i over i in c,
 *   Q        = (M * sum_c L_c - sum_c Sigma_c^2) / M^2.
 * Moving vertex i from d to c != d changes Q by 2 * gain / M^2 with
 *   gain = (M K_{i->c} - K_i Sigma_c) - (M K_{i->d} - K_i (Sigma_d - K_i)),
 * K_{i->x} the weight from i to vertices of x other than i.  All of it is
 * integer arithmetic in 128 bits, so decisions are exact.
 *
 * Readings where the paper is silent (also listed with the design notes):
 *   - ties between equally good communities go to the lowest community id,
 *     a move needs gain > 0, candidates are neighbour communities other than
 *     the vertex's own;
 *   - vertices are visited in ascending id;
 *   - "total change in modularity" of an iteration is the sum of the gains
 *     of the vertices that moved, S; the phase stops when
 *     (2.0 * dbl(S)) / dbl(M^2) <= tolerance, dbl() being the correctly
 *     rounded conversion of the exact integer.  In sequential (asynchronous)
 *     order 2S is exactly the change of the Q numerator N over the iteration;
 *     in synchronous order it is not (decisions taken together overlap), so
 *     stop_rule 1 reads the phrase as that exact change instead: the phase
 *     stops when dbl(N_after_iteration - N_before_iteration) / dbl(M^2) <=
 *     tolerance, N recomputed from the membership;
 *   - at most max_iterations iterations per pass and max_passes passes;
 *   - a pass with no move ends the run; otherwise its level is kept, and the
 *     run ends when dbl(N_after - N_before) / dbl(M^2) <= pass_tolerance
 *     (N = Q numerator) or at max_passes; aggregation is done only when
 *     another pass follows;
 *   - communities are renumbered by ascending old id; coarse rows are sorted
 *     by column;
 *   - optional pruning: in the first iteration of a pass every vertex is
 *     active, later a vertex is active iff it or a neighbour moved in the
 *     previous iteration;
 *   - synchronous means every decision of an iteration sees the memberships,
 *     community totals and community sizes as they were when the iteration
 *     began (Jacobi); with `subrounds` P > 1 the vertices are split into the
 *     classes i mod P, run one class after the other, each class Jacobi on
 *     the state left by the classes before it (the coarse-grained form of
 *     Section 2: a set of vertices processed in parallel);
 *   - singleton guard (synchronous only): a vertex alone in its community
 *     does not move to another single-vertex community with a higher id
 *     (the minimum-label rule of Grappolo, which the paper cites): without
 *     it, Jacobi updates swap pairs of singletons forever;
 *   - colour classes (synchronous, optional): the classes are a greedy
 *     colouring of the pass graph instead of i mod P, so that no two
 *     neighbours decide in the same class (Section 2's coarse-grained form,
 *     a set of vertices processed in parallel, as in the Grappolo heuristics
 *     it cites); see colour_classes().
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

typedef struct {
  int mode; /* 0 synchronous, 1 asynchronous */
  double tolerance, tolerance_decline, pass_tolerance;
  int max_iterations, max_passes, prune;
  int singleton_guard; /* synchronous only: see decide() */
  int subrounds;       /* synchronous only: vertex classes i mod P run in sequence */
  int colour_classes;  /* synchronous only: vertex classes from colour_classes() instead of i mod P */
  int stop_rule;       /* 0: an iteration's change is S, the sum of its movers' gains; 1: the exact
                          change of the Q numerator over the iteration, recomputed from the membership */
} or_options;

/* ------------------------------------------------------------ helpers */

static void split128(i128 x, int64_t *hi, uint64_t *lo) {
  *lo = (uint64_t)x;
  *hi = (int64_t)(x >> 64);
}

/* ---------------------------------------------------- modularity (a9) */

/* Exact Q numerator N = M * sum_c L_c - sum_c Sigma_c^2 for membership memb
 * (values in [0, n)); also returns M.  Direct from the definitions above. */
static i128 q_numerator(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w, const int32_t *memb,
                        int64_t *M_out) {
  i128 *sig = (i128 *)calloc((size_t)(n ? n : 1), sizeof(i128));
  i128 L = 0, M = 0, sq = 0;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      M += w[e];
      sig[memb[u]] += w[e];
      if (memb[col[e]] == memb[u]) L += w[e];
    }
  for (int64_t c = 0; c < n; ++c) sq += sig[c] * sig[c];
  free(sig);
  *M_out = (int64_t)M;
  return M * L - sq;
}

int or_modularity(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w, const int32_t *memb,
                  int64_t *num_hi, uint64_t *num_lo, int64_t *M_out, double *q) {
  for (int64_t u = 0; u < n; ++u)
    if (memb[u] < 0 || memb[u] >= n) return -2;
  int64_t M;
  i128 N = q_numerator(n, off, col, w, memb, &M);
  split128(N, num_hi, num_lo);
  *M_out = M;
  *q = (M == 0) ? 0.0 : (double)N / (double)((i128)M * M);
  return 0;
}

/* ------------------------------------------- one vertex's decision (a2, a3) */

/* score(x) = M K_{i->x} - K_i Sigma'_x, where Sigma'_x is Sigma_x without i;
 * the gain of moving i from d to c is score(c) - score(d). */
static i128 score(int64_t M, int64_t Kix, int64_t Ki, i128 sig_without_i) {
  return (i128)M * Kix - (i128)Ki * sig_without_i;
}

typedef struct {
  int64_t n;
  int64_t *acc;   /* dense accumulator indexed by community, zero between uses */
  int32_t *seen;  /* communities touched for the current vertex */
  int64_t nseen;
} scratch;

/* Best move of vertex i under membership memb and community totals sig.
 * Returns the target community (or -1 to stay) and its gain. */
static int32_t decide(scratch *s, int64_t i, const int64_t *off, const int32_t *col, const int64_t *w,
                      const int32_t *memb, const int64_t *K, const int64_t *sig, const int64_t *size, int guard,
                      int64_t M, i128 *gain_out) {
  s->nseen = 0;
  for (int64_t e = off[i]; e < off[i + 1]; ++e) {
    int64_t j = col[e];
    if (j == i) continue; /* self-loop: not a link to another vertex */
    int32_t c = memb[j];
    if (s->acc[c] == 0) s->seen[s->nseen++] = c;
    s->acc[c] += w[e];
  }
  int32_t d = memb[i];
  i128 score_d = score(M, s->acc[d], K[i], (i128)sig[d] - K[i]);
  i128 best = 0;
  int32_t best_c = -1;
  for (int64_t t = 0; t < s->nseen; ++t) {
    int32_t c = s->seen[t];
    if (c == d) continue;
    i128 g = score(M, s->acc[c], K[i], sig[c]) - score_d;
    if (g > best || (g == best && best_c >= 0 && c < best_c)) { best = g; best_c = c; }
  }
  for (int64_t t = 0; t < s->nseen; ++t) s->acc[s->seen[t]] = 0;
  if (guard && best_c >= 0 && size[d] == 1 && size[best_c] == 1 && best_c > d) best_c = -1;
  *gain_out = best_c >= 0 ? best : 0;
  return best_c;
}

/* Candidate gains of vertex i (for checking the gain formula): all
 * neighbour communities other than memb[i], ascending, with their gains. */
int64_t or_vertex_gains(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w, const int32_t *memb,
                        int64_t i, int32_t *out_c, int64_t *out_hi, uint64_t *out_lo, int64_t cap) {
  int64_t *K = (int64_t *)calloc((size_t)n, 8), *sig = (int64_t *)calloc((size_t)n, 8), M = 0;
  int64_t *acc = (int64_t *)calloc((size_t)n, 8);
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = off[u]; e < off[u + 1]; ++e) { K[u] += w[e]; M += w[e]; }
  for (int64_t u = 0; u < n; ++u) sig[memb[u]] += K[u];
  for (int64_t e = off[i]; e < off[i + 1]; ++e)
    if (col[e] != i) acc[memb[col[e]]] += w[e];
  int32_t d = memb[i];
  i128 score_d = score(M, acc[d], K[i], (i128)sig[d] - K[i]);
  int64_t cnt = 0;
  for (int64_t c = 0; c < n; ++c) {
    if (c == d || acc[c] == 0) continue;
    if (cnt < cap) {
      i128 g = score(M, acc[c], K[i], sig[c]) - score_d;
      out_c[cnt] = (int32_t)c;
      split128(g, &out_hi[cnt], &out_lo[cnt]);
    }
    ++cnt;
  }
  free(K); free(sig); free(acc);
  return cnt;
}

/* ------------------------------------------------------ colour classes */

/* The lowbias32 integer hash (C. Wellons, "Prospecting for hash functions"). */
static uint32_t lowbias32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

typedef struct {
  uint32_t h;
  int32_t v;
} pri_item;

/* descending hash, then ascending id */
static int pri_cmp(const void *a, const void *b) {
  const pri_item *x = (const pri_item *)a, *y = (const pri_item *)b;
  if (x->h != y->h) return x->h > y->h ? -1 : 1;
  return (x->v > y->v) - (x->v < y->v);
}

/* Vertex classes of pass `pass` on an n-vertex graph: a greedy colouring
 * capped at 64 classes.  Vertex v's priority is lowbias32(v XOR s) with
 * s = 0x9E3779B9 * (pass + 1) (mod 2^32); the vertices take their class one
 * at a time in descending priority (ties: lower id first), each the smallest
 * class in 0..62 that none of its already-classed neighbours holds, else 63.
 * Classes below 63 hold no two neighbours.  Returns the number of classes
 * (largest class + 1; 1 for an empty graph). */
static int colour_classes(int64_t n, const int64_t *off, const int32_t *col, int pass, int32_t *cls) {
  const uint32_t salt = 0x9E3779B9u * (uint32_t)(pass + 1);
  pri_item *order = (pri_item *)malloc((size_t)(n ? n : 1) * sizeof(pri_item));
  for (int64_t v = 0; v < n; ++v) {
    order[v].h = lowbias32((uint32_t)v ^ salt);
    order[v].v = (int32_t)v;
    cls[v] = -1;
  }
  qsort(order, (size_t)n, sizeof(pri_item), pri_cmp);
  int top = 0;
  for (int64_t t = 0; t < n; ++t) {
    const int32_t v = order[t].v;
    uint64_t used = 0;
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      const int32_t u = col[e];
      if (u != v && cls[u] >= 0) used |= (uint64_t)1 << cls[u];
    }
    int c = 0;
    while (c < 63 && ((used >> c) & 1)) ++c;
    cls[v] = c;
    if (c > top) top = c;
  }
  free(order);
  return top + 1;
}

int or_colour_classes(int64_t n, const int64_t *off, const int32_t *col, int pass, int32_t *cls) {
  if (n < 0 || !off || !cls) return -1;
  return colour_classes(n, off, col, pass, cls);
}

/* ------------------------------------------------------- result record */

typedef struct {
  int64_t n, nnz;
  int64_t *off;
  int32_t *col;
  int64_t *w;
} graph;

typedef struct {
  int64_t n0;
  int32_t *top;
  int64_t M;
  i128 Qnum;
  double Q;
  int npasses; /* passes whose local-moving ran */
  /* per pass (index p < npasses) */
  int64_t pass_n[64], pass_nnz[64], pass_k[64], pass_moves[64];
  int pass_iters[64], pass_level[64]; /* level recorded? */
  i128 pass_Nbefore[64], pass_Nafter[64];
  int32_t *level[64];   /* renumbered membership of pass p (length pass_n[p]) */
  graph coarse[64];     /* graph after aggregation of pass p (if it ran) */
  int coarse_built[64];
  /* per iteration, all passes in order */
  int64_t niters, cap_iters;
  int64_t *it_moves;
  i128 *it_S;
  int *it_pass;
} or_result;

static void push_iter(or_result *r, int pass, int64_t moves, i128 S) {
  if (r->niters == r->cap_iters) {
    int64_t c = r->cap_iters ? r->cap_iters * 2 : 64;
    r->it_moves = (int64_t *)realloc(r->it_moves, (size_t)c * 8);
    r->it_S = (i128 *)realloc(r->it_S, (size_t)c * sizeof(i128));
    r->it_pass = (int *)realloc(r->it_pass, (size_t)c * sizeof(int));
    r->cap_iters = c;
  }
  r->it_moves[r->niters] = moves;
  r->it_S[r->niters] = S;
  r->it_pass[r->niters] = pass;
  r->niters++;
}

static double dbl_ratio(i128 num, i128 den) { return (double)num / (double)den; }

/* ---------------------------------------------------- aggregation (a7) */

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Coarse graph over k communities: entry (C, D) sums the weights of all
 * fine entries (u, v) with level[u] = C and level[v] = D; rows ascending. */
static graph aggregate(const graph *g, const int32_t *level, int64_t k) {
  graph h;
  h.n = k;
  int64_t *mstart = (int64_t *)calloc((size_t)k + 1, 8);
  int32_t *members = (int32_t *)malloc((size_t)(g->n ? g->n : 1) * 4);
  for (int64_t u = 0; u < g->n; ++u) mstart[level[u] + 1]++;
  for (int64_t c = 0; c < k; ++c) mstart[c + 1] += mstart[c];
  int64_t *fill = (int64_t *)malloc((size_t)(k ? k : 1) * 8);
  memcpy(fill, mstart, (size_t)k * 8);
  for (int64_t u = 0; u < g->n; ++u) members[fill[level[u]]++] = (int32_t)u;
  free(fill);
  int64_t *acc = (int64_t *)calloc((size_t)(k ? k : 1), 8);
  int32_t *seen = (int32_t *)malloc((size_t)(k ? k : 1) * 4);
  h.off = (int64_t *)calloc((size_t)k + 1, 8);
  int64_t cap = g->nnz ? g->nnz : 1;
  h.col = (int32_t *)malloc((size_t)cap * 4);
  h.w = (int64_t *)malloc((size_t)cap * 8);
  int64_t nnz = 0;
  for (int64_t C = 0; C < k; ++C) {
    int64_t ns = 0;
    for (int64_t t = mstart[C]; t < mstart[C + 1]; ++t) {
      int64_t u = members[t];
      for (int64_t e = g->off[u]; e < g->off[u + 1]; ++e) {
        int32_t D = level[g->col[e]];
        if (acc[D] == 0) seen[ns++] = D;
        acc[D] += g->w[e];
      }
    }
    /* ascending columns */
    qsort(seen, (size_t)ns, sizeof(int32_t), cmp_i32);
    for (int64_t t = 0; t < ns; ++t) {
      h.col[nnz] = seen[t];
      h.w[nnz] = acc[seen[t]];
      acc[seen[t]] = 0;
      ++nnz;
    }
    h.off[C + 1] = nnz;
  }
  h.nnz = nnz;
  free(mstart); free(members); free(acc); free(seen);
  return h;
}

/* ------------------------------------------------------- driver (a1-a8) */

static void free_graph(graph *g) { free(g->off); free(g->col); free(g->w); memset(g, 0, sizeof(*g)); }

void or_free(or_result *r) {
  if (!r) return;
  free(r->top);
  for (int p = 0; p < 64; ++p) {
    free(r->level[p]);
    if (r->coarse_built[p]) free_graph(&r->coarse[p]);
  }
  free(r->it_moves); free(r->it_S); free(r->it_pass);
  free(r);
}

/* Louvain from an initial membership of the input (init, values in [0, n);
   NULL = singletons, the method as the paper states it).  With init, pass 0
   starts from init's communities (totals and sizes summed over their members),
   its "before" numerator is init's, and its level is kept even when no vertex
   moves, so the result is never coarser than init's renumbering requires. */
or_result *or_louvain_from(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w,
                           const or_options *opt, int record_levels, const int32_t *init) {
  if (opt->max_passes > 64 || opt->max_passes < 0 || opt->max_iterations < 0) return NULL;
  if (init)
    for (int64_t v = 0; v < n; ++v)
      if (init[v] < 0 || init[v] >= n) return NULL;
  or_result *r = (or_result *)calloc(1, sizeof(or_result));
  r->n0 = n;
  r->top = (int32_t *)malloc((size_t)(n ? n : 1) * 4);
  for (int64_t v = 0; v < n; ++v) r->top[v] = (int32_t)v;

  /* the pass graph: starts as a copy of the input */
  graph g;
  g.n = n;
  g.nnz = off[n];
  g.off = (int64_t *)malloc((size_t)(n + 1) * 8);
  g.col = (int32_t *)malloc((size_t)(g.nnz ? g.nnz : 1) * 4);
  g.w = (int64_t *)malloc((size_t)(g.nnz ? g.nnz : 1) * 8);
  memcpy(g.off, off, (size_t)(n + 1) * 8);
  memcpy(g.col, col, (size_t)g.nnz * 4);
  memcpy(g.w, w, (size_t)g.nnz * 8);

  int64_t M = 0;
  for (int64_t e = 0; e < g.nnz; ++e) M += g.w[e];
  r->M = M;
  i128 M2 = (i128)M * M;
  double tol = opt->tolerance;
  i128 Qnum = 0;
  {
    /* the partition pass 0 starts from: singletons, or init */
    int32_t *id = (int32_t *)malloc((size_t)(n ? n : 1) * 4);
    for (int64_t v = 0; v < n; ++v) id[v] = init ? init[v] : (int32_t)v;
    int64_t Mx;
    Qnum = q_numerator(n, g.off, g.col, g.w, id, &Mx);
    free(id);
  }

  for (int p = 0; p < opt->max_passes && M > 0; ++p) {
    int64_t np = g.n;
    /* a1: pass init */
    int64_t *K = (int64_t *)calloc((size_t)(np ? np : 1), 8);
    int64_t *sig = (int64_t *)calloc((size_t)(np ? np : 1), 8);
    int64_t *size = (int64_t *)calloc((size_t)(np ? np : 1), 8);
    int32_t *memb = (int32_t *)malloc((size_t)(np ? np : 1) * 4);
    int32_t *mv_i = (int32_t *)malloc((size_t)(np ? np : 1) * 4), *mv_c = (int32_t *)malloc((size_t)(np ? np : 1) * 4);
    uint8_t *active = (uint8_t *)malloc((size_t)(np ? np : 1));
    uint8_t *moved = (uint8_t *)calloc((size_t)(np ? np : 1), 1);
    const int warm = p == 0 && init != NULL;
    for (int64_t i = 0; i < np; ++i) {
      for (int64_t e = g.off[i]; e < g.off[i + 1]; ++e) K[i] += g.w[e];
      memb[i] = warm ? init[i] : (int32_t)i;
      active[i] = 1;
    }
    for (int64_t i = 0; i < np; ++i) {
      sig[memb[i]] += K[i];
      size[memb[i]] += 1;
    }
    i128 Nbefore = Qnum;
    i128 Nprev = Nbefore;   /* Q numerator before the current iteration (stop_rule 1) */
    scratch s;
    s.n = np;
    s.acc = (int64_t *)calloc((size_t)(np ? np : 1), 8);
    s.seen = (int32_t *)malloc((size_t)(np ? np : 1) * 4);
    int64_t pass_moves = 0;
    int iters = 0;
    int P = opt->subrounds > 1 ? opt->subrounds : 1;
    int32_t *cls = NULL;   /* colour classes of this pass */
    if (opt->mode == 0 && opt->colour_classes) {
      cls = (int32_t *)malloc((size_t)(np ? np : 1) * 4);
      P = colour_classes(np, g.off, g.col, p, cls);
    }
    /* local-moving phase (a2-a5) */
    for (int it = 0; it < opt->max_iterations; ++it) {
      i128 S = 0;
      int64_t moves = 0;
      memset(moved, 0, (size_t)np);
      if (opt->mode == 0) {
        /* synchronous: the decisions of one class all see the state left by
           the previous classes; the class's moves are applied together */
        for (int ch = 0; ch < P; ++ch) {
          int64_t nm = 0;
          for (int64_t i = cls ? 0 : ch; i < np; i += cls ? 1 : P) {
            if (!active[i] || (cls && cls[i] != ch)) continue;
            i128 gain;
            int32_t c = decide(&s, i, g.off, g.col, g.w, memb, K, sig, size, opt->singleton_guard, M, &gain);
            if (c >= 0) { mv_i[nm] = (int32_t)i; mv_c[nm] = c; ++nm; S += gain; }
          }
          for (int64_t t = 0; t < nm; ++t) {
            int32_t i = mv_i[t], c = mv_c[t];
            sig[memb[i]] -= K[i]; size[memb[i]] -= 1;
            sig[c] += K[i]; size[c] += 1;
            memb[i] = c;
            moved[i] = 1;
          }
          moves += nm;
        }
      } else {
        /* asynchronous: each move is applied before the next vertex */
        for (int64_t i = 0; i < np; ++i) {
          if (!active[i]) continue;
          i128 gain;
          int32_t c = decide(&s, i, g.off, g.col, g.w, memb, K, sig, size, 0, M, &gain);
          if (c >= 0) {
            sig[memb[i]] -= K[i]; size[memb[i]] -= 1;
            sig[c] += K[i]; size[c] += 1;
            memb[i] = c;
            S += gain; ++moves; moved[i] = 1;
          }
        }
      }
      push_iter(r, p, moves, S);
      pass_moves += moves;
      ++iters;
      if (opt->prune) {
        for (int64_t i = 0; i < np; ++i) {
          uint8_t a = moved[i];
          for (int64_t e = g.off[i]; e < g.off[i + 1] && !a; ++e) a = moved[g.col[e]];
          active[i] = a;
        }
      }
      int settled;
      if (opt->stop_rule == 1) {
        int64_t Mx;
        const i128 Nit = q_numerator(np, g.off, g.col, g.w, memb, &Mx);
        settled = dbl_ratio(Nit - Nprev, M2) <= tol;
        Nprev = Nit;
      } else {
        settled = (2.0 * (double)S) / (double)M2 <= tol;
      }
      if (settled) break;
    }
    r->pass_n[p] = np;
    r->pass_nnz[p] = g.nnz;
    r->pass_moves[p] = pass_moves;
    r->pass_iters[p] = iters;
    r->pass_Nbefore[p] = Nbefore;
    r->npasses = p + 1;
    free(s.acc); free(s.seen); free(mv_i); free(mv_c); free(active); free(moved); free(size); free(cls);
    if (pass_moves == 0 && !warm) {
      r->pass_Nafter[p] = Nbefore;
      r->pass_k[p] = np;
      free(K); free(sig); free(memb);
      break;
    }
    /* a6: renumber by ascending old id, compose the dendrogram */
    int32_t *newid = (int32_t *)malloc((size_t)(np ? np : 1) * 4);
    for (int64_t c = 0; c < np; ++c) newid[c] = -1;
    for (int64_t i = 0; i < np; ++i) newid[memb[i]] = 0;
    int64_t k = 0;
    for (int64_t c = 0; c < np; ++c)
      if (newid[c] == 0) newid[c] = (int32_t)k++;
    int32_t *level = (int32_t *)malloc((size_t)(np ? np : 1) * 4);
    for (int64_t i = 0; i < np; ++i) level[i] = newid[memb[i]];
    free(newid);
    for (int64_t v = 0; v < n; ++v) r->top[v] = level[r->top[v]];
    int64_t Mx;
    i128 Nafter = q_numerator(np, g.off, g.col, g.w, memb, &Mx);
    r->pass_Nafter[p] = Nafter;
    r->pass_k[p] = k;
    Qnum = Nafter;
    int stop = dbl_ratio(Nafter - Nbefore, M2) <= opt->pass_tolerance || p + 1 == opt->max_passes;
    if (!stop) {
      graph h = aggregate(&g, level, k);
      free_graph(&g);
      g = h;
      if (record_levels) {
        graph c;
        c.n = h.n; c.nnz = h.nnz;
        c.off = (int64_t *)malloc((size_t)(h.n + 1) * 8);
        c.col = (int32_t *)malloc((size_t)(h.nnz ? h.nnz : 1) * 4);
        c.w = (int64_t *)malloc((size_t)(h.nnz ? h.nnz : 1) * 8);
        memcpy(c.off, h.off, (size_t)(h.n + 1) * 8);
        memcpy(c.col, h.col, (size_t)h.nnz * 4);
        memcpy(c.w, h.w, (size_t)h.nnz * 8);
        r->coarse[p] = c;
        r->coarse_built[p] = 1;
      }
      tol = tol / opt->tolerance_decline;
    }
    if (record_levels) r->level[p] = level; else free(level);
    r->pass_level[p] = 1;
    free(K); free(sig); free(memb);
    if (stop) break;
  }
  free_graph(&g);
  r->Qnum = Qnum;
  r->Q = (M == 0) ? 0.0 : dbl_ratio(Qnum, M2);
  return r;
}

or_result *or_louvain(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w, const or_options *opt,
                      int record_levels) {
  return or_louvain_from(n, off, col, w, opt, record_levels, NULL);
}

/* ------------------------------------------------------------ accessors */

void or_result_summary(const or_result *r, int64_t *out /* 8 */, double *q) {
  out[0] = r->n0;
  out[1] = r->M;
  split128(r->Qnum, &out[2], (uint64_t *)&out[3]);
  out[4] = r->npasses;
  out[5] = r->niters;
  out[6] = 0;
  out[7] = 0;
  *q = r->Q;
}

void or_result_top(const or_result *r, int32_t *out) { memcpy(out, r->top, (size_t)r->n0 * 4); }

/* Per pass p: [n, nnz, k, moves, iters, level_recorded, coarse_built, coarse_nnz,
 *              Nbefore_hi, Nbefore_lo, Nafter_hi, Nafter_lo] */
void or_result_pass(const or_result *r, int p, int64_t *out /* 12 */) {
  out[0] = r->pass_n[p];
  out[1] = r->pass_nnz[p];
  out[2] = r->pass_k[p];
  out[3] = r->pass_moves[p];
  out[4] = r->pass_iters[p];
  out[5] = r->level[p] != NULL;
  out[6] = r->coarse_built[p];
  out[7] = r->coarse_built[p] ? r->coarse[p].nnz : 0;
  split128(r->pass_Nbefore[p], &out[8], (uint64_t *)&out[9]);
  split128(r->pass_Nafter[p], &out[10], (uint64_t *)&out[11]);
}

/* Per iteration t: [pass, moves, S_hi, S_lo] */
void or_result_iter(const or_result *r, int64_t t, int64_t *out /* 4 */) {
  out[0] = r->it_pass[t];
  out[1] = r->it_moves[t];
  split128(r->it_S[t], &out[2], (uint64_t *)&out[3]);
}

void or_result_level(const or_result *r, int p, int32_t *out) {
  memcpy(out, r->level[p], (size_t)r->pass_n[p] * 4);
}

void or_result_coarse(const or_result *r, int p, int64_t *off, int32_t *col, int64_t *w) {
  const graph *c = &r->coarse[p];
  memcpy(off, c->off, (size_t)(c->n + 1) * 8);
  memcpy(col, c->col, (size_t)c->nnz * 4);
  memcpy(w, c->w, (size_t)c->nnz * 8);
}

/* Standalone aggregation (for invariant tests): level in [0, k). */
int or_aggregate(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w, const int32_t *level,
                 int64_t k, int64_t *out_off /* k+1 */, int32_t *out_col /* cap */, int64_t *out_w, int64_t cap,
                 int64_t *out_nnz) {
  for (int64_t u = 0; u < n; ++u)
    if (level[u] < 0 || level[u] >= k) return -2;
  graph g = {n, off[n], (int64_t *)off, (int32_t *)col, (int64_t *)w};
  graph h = aggregate(&g, level, k);
  *out_nnz = h.nnz;
  int rc = 0;
  if (h.nnz > cap) rc = -3;
  else {
    memcpy(out_off, h.off, (size_t)(k + 1) * 8);
    memcpy(out_col, h.col, (size_t)h.nnz * 4);
    memcpy(out_w, h.w, (size_t)h.nnz * 8);
  }
  free_graph(&h);
  return rc;
}

/* ---------------------------------------------- brute-force optimum (O2) */

/* Maximum Q numerator over all set partitions of n <= 12 vertices
 * (restricted growth strings), with the first maximising partition. */
int or_brute_best(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w, int32_t *best_memb,
                  int64_t *num_hi, uint64_t *num_lo, int64_t *count) {
  if (n < 1 || n > 12) return -2;
  int32_t a[12], mx[12];
  i128 best = 0;
  int have = 0;
  int64_t cnt = 0, M;
  for (int64_t i = 0; i < n; ++i) { a[i] = 0; mx[i] = 0; }
  for (;;) {
    i128 N = q_numerator(n, off, col, w, a, &M);
    ++cnt;
    if (!have || N > best) { best = N; have = 1; memcpy(best_memb, a, (size_t)n * 4); }
    /* next restricted growth string: a[0] = 0, a[i] <= 1 + max(a[0..i-1]) */
    int64_t i = n - 1;
    while (i > 0 && a[i] == mx[i - 1] + 1) --i;
    if (i == 0) break;
    a[i]++;
    mx[i] = a[i] > mx[i - 1] ? a[i] : mx[i - 1];
    for (int64_t j = i + 1; j < n; ++j) { a[j] = 0; mx[j] = mx[i]; }
  }
  split128(best, num_hi, num_lo);
  *count = cnt;
  return 0;
}
