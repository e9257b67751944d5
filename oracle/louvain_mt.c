/*
 * louvain_mt.c — multi-threaded CPU Louvain, the paper's own shared-memory
 * design, as a CPU baseline for the benchmark.
 *
 * NOT THE ORACLE.  Only bench.py's CPU-baseline leg and its own CPU tests
 * run it; no parity test compares the GPU engine with it.  It shares no code
 * with the CUDA engine or with louvain_oracle.c.
 *
 * What it follows (Section 3.2 of the paper, the OpenMP experiment): the
 * asynchronous Louvain method (Gauss-Seidel: a vertex's move is visible to
 * the vertices decided after it) with the vertices of each local-moving
 * iteration shared among threads; every thread keeps its own hashtable of
 * neighbouring-community weights (here a dense accumulator indexed by
 * community plus the list of the keys it touched, the usual collision-free
 * form); memberships are read and written in place by all threads and the
 * community totals are updated with atomic adds.  Passes, threshold scaling
 * (tolerance divided by the decline factor after every pass), pass tolerance,
 * iteration and pass limits, and the gain formula and tie rule are those of
 * the oracle's asynchronous mode:
 *   gain(i: d->c) = (M K_{i->c} - K_i Sigma_c) - (M K_{i->d} - K_i (Sigma_d - K_i)),
 *   ties to the lowest community id, a move needs gain > 0, the iteration's
 *   change is S (the sum of its movers' gains): stop when 2S/M^2 <= tolerance.
 * Aggregation is parallel over communities (each thread its own dense
 * accumulator), renumbering by ascending community id.  With one thread the
 * run is the sequential asynchronous method in ascending vertex order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

typedef struct {
  double tolerance, tolerance_decline, pass_tolerance;
  int max_iterations, max_passes, threads;
} mt_options;

typedef struct {
  int64_t n, nnz;
  int64_t *off;
  int32_t *col;
  int64_t *w;
} mt_graph;

int mt_threads_available(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Q numerator M * sum_c L_c - sum_c Sigma_c^2 of membership memb on g. */
static i128 mt_qnum(const mt_graph *g, const int32_t *memb, int64_t M) {
  int64_t n = g->n;
  int64_t *sig = (int64_t *)calloc((size_t)(n ? n : 1), 8);
  i128 L = 0, sq = 0;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = g->off[u]; e < g->off[u + 1]; ++e) {
      sig[memb[u]] += g->w[e];
      if (memb[g->col[e]] == memb[u]) L += g->w[e];
    }
  for (int64_t c = 0; c < n; ++c) sq += (i128)sig[c] * sig[c];
  free(sig);
  return (i128)M * L - sq;
}

/* One asynchronous local-moving phase; returns the iterations run and adds
 * the entries scanned to *scanned. */
static int mt_local_moving(const mt_graph *g, int32_t *memb, int64_t *sig, const int64_t *K, int64_t M,
                           double tol, int max_iter, int threads, int64_t *moves_out, int64_t *scanned) {
  const int64_t n = g->n;
  const i128 M2 = (i128)M * M;
  int64_t moves_total = 0;
  int it = 0;
  for (; it < max_iter; ++it) {
    i128 S = 0;
    int64_t moves = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(threads)
#endif
    {
      int64_t *acc = (int64_t *)calloc((size_t)(n ? n : 1), 8);
      int32_t *seen = (int32_t *)malloc((size_t)(n ? n : 1) * 4);
      i128 S_t = 0;
      int64_t mv_t = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1024) nowait
#endif
      for (int64_t i = 0; i < n; ++i) {
        int64_t ns = 0;
        for (int64_t e = g->off[i]; e < g->off[i + 1]; ++e) {
          const int32_t j = g->col[e];
          if (j == i) continue;
          const int32_t c = __atomic_load_n(&memb[j], __ATOMIC_RELAXED);
          if (acc[c] == 0) seen[ns++] = c;
          acc[c] += g->w[e];
        }
        const int32_t d = memb[i];
        const int64_t sd = __atomic_load_n(&sig[d], __ATOMIC_RELAXED);
        const i128 score_d = (i128)M * acc[d] - (i128)K[i] * (sd - K[i]);
        i128 best = 0;
        int32_t best_c = -1;
        for (int64_t t = 0; t < ns; ++t) {
          const int32_t c = seen[t];
          if (c != d) {
            const i128 g_c = (i128)M * acc[c] - (i128)K[i] * __atomic_load_n(&sig[c], __ATOMIC_RELAXED) - score_d;
            if (g_c > best || (g_c == best && best_c >= 0 && c < best_c)) {
              best = g_c;
              best_c = c;
            }
          }
          acc[c] = 0;
        }
        if (best_c >= 0) {
          __atomic_fetch_sub(&sig[d], K[i], __ATOMIC_RELAXED);
          __atomic_fetch_add(&sig[best_c], K[i], __ATOMIC_RELAXED);
          __atomic_store_n(&memb[i], best_c, __ATOMIC_RELAXED);
          S_t += best;
          ++mv_t;
        }
      }
#ifdef _OPENMP
#pragma omp critical
#endif
      {
        S += S_t;
        moves += mv_t;
      }
      free(acc);
      free(seen);
    }
    *scanned += g->nnz;
    moves_total += moves;
    if ((2.0 * (double)S) / (double)M2 <= tol) {
      ++it;
      break;
    }
  }
  *moves_out = moves_total;
  return it;
}

/* Coarse graph of g under level (values in [0, k)): parallel over
 * communities, each thread with its own dense accumulator; rows ascending. */
static int cmp_i32(const void *a, const void *b) {
  const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

static mt_graph mt_aggregate(const mt_graph *g, const int32_t *level, int64_t k, int threads) {
  mt_graph h;
  h.n = k;
  int64_t *mstart = (int64_t *)calloc((size_t)k + 1, 8);
  int32_t *members = (int32_t *)malloc((size_t)(g->n ? g->n : 1) * 4);
  for (int64_t u = 0; u < g->n; ++u) mstart[level[u] + 1]++;
  for (int64_t c = 0; c < k; ++c) mstart[c + 1] += mstart[c];
  int64_t *fill = (int64_t *)malloc((size_t)(k ? k : 1) * 8);
  memcpy(fill, mstart, (size_t)k * 8);
  for (int64_t u = 0; u < g->n; ++u) members[fill[level[u]]++] = (int32_t)u;
  free(fill);
  int64_t *rlen = (int64_t *)calloc((size_t)k + 1, 8);
  int32_t **rcol = (int32_t **)calloc((size_t)(k ? k : 1), sizeof(int32_t *));
  int64_t **rw = (int64_t **)calloc((size_t)(k ? k : 1), sizeof(int64_t *));
#ifdef _OPENMP
#pragma omp parallel num_threads(threads)
#endif
  {
    int64_t *acc = (int64_t *)calloc((size_t)(k ? k : 1), 8);
    int32_t *seen = (int32_t *)malloc((size_t)(k ? k : 1) * 4);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
    for (int64_t C = 0; C < k; ++C) {
      int64_t ns = 0;
      for (int64_t t = mstart[C]; t < mstart[C + 1]; ++t) {
        const int64_t u = members[t];
        for (int64_t e = g->off[u]; e < g->off[u + 1]; ++e) {
          const int32_t D = level[g->col[e]];
          if (acc[D] == 0) seen[ns++] = D;
          acc[D] += g->w[e];
        }
      }
      qsort(seen, (size_t)ns, 4, cmp_i32);
      rcol[C] = (int32_t *)malloc((size_t)(ns ? ns : 1) * 4);
      rw[C] = (int64_t *)malloc((size_t)(ns ? ns : 1) * 8);
      for (int64_t t = 0; t < ns; ++t) {
        rcol[C][t] = seen[t];
        rw[C][t] = acc[seen[t]];
        acc[seen[t]] = 0;
      }
      rlen[C] = ns;
    }
    free(acc);
    free(seen);
  }
  h.off = (int64_t *)calloc((size_t)k + 1, 8);
  for (int64_t C = 0; C < k; ++C) h.off[C + 1] = h.off[C] + rlen[C];
  h.nnz = h.off[k];
  h.col = (int32_t *)malloc((size_t)(h.nnz ? h.nnz : 1) * 4);
  h.w = (int64_t *)malloc((size_t)(h.nnz ? h.nnz : 1) * 8);
  for (int64_t C = 0; C < k; ++C) {
    memcpy(h.col + h.off[C], rcol[C], (size_t)rlen[C] * 4);
    memcpy(h.w + h.off[C], rw[C], (size_t)rlen[C] * 8);
    free(rcol[C]);
    free(rw[C]);
  }
  free(rcol); free(rw); free(rlen); free(mstart); free(members);
  return h;
}

/* The whole run.  top[n] receives the final membership; out[0] = passes,
 * out[1] = iterations, out[2] = moves, out[3] = entries scanned by local
 * moving, out[4..5] = Q numerator (hi, lo), out[6] = M; *q = Q.  Returns the
 * threads used, or < 0 on bad options. */
int mt_louvain(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w, const mt_options *opt,
               int32_t *top, int64_t *out, double *q) {
  if (n < 0 || opt->max_passes < 0 || opt->max_iterations < 1 || opt->threads < 1) return -1;
  const int threads = opt->threads;
  mt_graph g;
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
  for (int64_t v = 0; v < n; ++v) top[v] = (int32_t)v;
  int32_t *id = (int32_t *)malloc((size_t)(n ? n : 1) * 4);
  for (int64_t v = 0; v < n; ++v) id[v] = (int32_t)v;
  i128 Qnum = mt_qnum(&g, id, M);
  free(id);
  double tol = opt->tolerance;
  int passes = 0, iters = 0;
  int64_t moves_all = 0, scanned = 0;
  const i128 M2 = (i128)M * M;
  for (int p = 0; p < opt->max_passes && M > 0; ++p) {
    const int64_t np = g.n;
    int64_t *K = (int64_t *)calloc((size_t)(np ? np : 1), 8);
    int64_t *sig = (int64_t *)malloc((size_t)(np ? np : 1) * 8);
    int32_t *memb = (int32_t *)malloc((size_t)(np ? np : 1) * 4);
    for (int64_t i = 0; i < np; ++i) {
      for (int64_t e = g.off[i]; e < g.off[i + 1]; ++e) K[i] += g.w[e];
      sig[i] = K[i];
      memb[i] = (int32_t)i;
    }
    int64_t moves = 0;
    iters += mt_local_moving(&g, memb, sig, K, M, tol, opt->max_iterations, threads, &moves, &scanned);
    ++passes;
    moves_all += moves;
    free(K);
    free(sig);
    if (moves == 0) {
      free(memb);
      break;
    }
    int32_t *newid = (int32_t *)malloc((size_t)(np ? np : 1) * 4);
    for (int64_t c = 0; c < np; ++c) newid[c] = -1;
    for (int64_t i = 0; i < np; ++i) newid[memb[i]] = 0;
    int64_t k = 0;
    for (int64_t c = 0; c < np; ++c)
      if (newid[c] == 0) newid[c] = (int32_t)k++;
    for (int64_t i = 0; i < np; ++i) memb[i] = newid[memb[i]];
    free(newid);
    for (int64_t v = 0; v < n; ++v) top[v] = memb[top[v]];
    const i128 Nafter = mt_qnum(&g, memb, M);
    const int stop = (double)(Nafter - Qnum) / (double)M2 <= opt->pass_tolerance || p + 1 == opt->max_passes;
    Qnum = Nafter;
    if (!stop) {
      mt_graph h = mt_aggregate(&g, memb, k, threads);
      free(g.off); free(g.col); free(g.w);
      g = h;
      tol /= opt->tolerance_decline;
    }
    free(memb);
    if (stop) break;
  }
  free(g.off); free(g.col); free(g.w);
  out[0] = passes;
  out[1] = iters;
  out[2] = moves_all;
  out[3] = scanned;
  out[4] = (int64_t)(Qnum >> 64);
  out[5] = (int64_t)(uint64_t)Qnum;
  out[6] = M;
  *q = M == 0 ? 0.0 : (double)Qnum / (double)M2;
  return threads;
}
