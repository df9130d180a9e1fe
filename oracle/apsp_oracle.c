/*
 * apsp_oracle.c -- CPU oracle for all-pairs shortest paths over the (min,+) semiring.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no source, header, table or helper with the
 * CUDA path and must never be called from the product library.
 *
 * Everything here is the plain definition, written out slowly:
 *
 *   - oracle_fw_i64 / oracle_fw_f64: the Floyd-Warshall recurrence of the paper's Eq. 1,
 *       d^{k+1}[i,j] = min{ d^k[i,j], d^k[i,k] + d^k[k,j] },
 *     run as the textbook k-i-j triple loop over all n intermediate vertices (Sec. 2).
 *     Integer inputs are widened to int64 and floating inputs to fp64 by the caller, so no
 *     sum here can overflow or round differently from the exact path length (fp32 weights
 *     widen exactly; an fp64 sum of a few hundred fp32 values is exact to ~1e-13 relative).
 *   - oracle_minplus_i64 / oracle_minplus_f64: the (min,+) product of Eq. 2,
 *       Z[i,j] = min_k ( X[i,k] + Y[k,j] ),
 *     as a triple loop, optionally folded into an existing Z (Z = min(Z, X (x) Y)).
 *   - oracle_minplus_rows_i32 / _f32: selected rows of the same product, reading operands in
 *     their 32-bit storage types and widening each value to int64 / fp64 as it is read (used to
 *     check rows of a product too large for the full triple loop).
 *   - oracle_fw_pred_i64 / _f64: Eq. 1 with the predecessor indices of Sec. 2: pred[i][j]
 *     starts as i where the edge i -> j exists and, whenever the path through k shortens
 *     d[i][j], becomes pred[k][j], the vertex before j on the path from k.
 *   - oracle_last_hop_i64 / _f32: the predecessor matrix by its plain definition from a closed
 *     d and the costs w: pred[i][j] = the smallest k != j minimising d[i][k] + w[k][j] (the
 *     argmin of Sec. 3.1 restricted to the last edge), -1 on the diagonal and where the
 *     minimum is unreachable.  The float32 variant adds in float32 (one rounding per sum),
 *     the precision in which the library takes the same decision.
 *   - oracle_bellman_ford_rows_i64 / _f64: single-source distances by Bellman-Ford (n - 1 rounds
 *     relaxing every edge), valid with negative weights; a further round that still improves
 *     a distance reports a negative cycle reachable from the source.  The independent check for
 *     graphs with negative edges (Sec. 3.1 allows them as long as no cycle is negative).
 *   - oracle_dijkstra_rows_i64 / _f64: single-source shortest paths from selected sources by
 *     textbook O(n^2) array Dijkstra (valid because every weight is >= 0; Sec. 3.1 assumes
 *     no negative cycles and the generator draws costs >= 0, Sec. 3.4).  It is a second,
 *     independent algorithm for the same distances, used to check large matrices by rows.
 *
 * Conventions shared with the tests (not with the CUDA path):
 *   - int64: an entry >= inf means "no edge / unreachable"; such operands are skipped and
 *     every result >= inf is written back as exactly inf.
 *   - fp64: +infinity means "no edge / unreachable"; IEEE arithmetic does the rest.
 *   - the diagonal is forced to 0 (a self-loop costs nothing, Sec. 3.4).
 *   - matrices are dense row-major with leading dimension n.
 *
 * `threads` > 1 splits the i loop (for FW, at each fixed k) or the source list (Dijkstra)
 * over OpenMP threads.  For FW this is race-free because row k itself never changes at step
 * k: d[k][k] = 0 and weights are non-negative, so d[k][k] + d[k][j] is never < d[k][j].
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC apsp_oracle.c -o _oracle.so  (see build.py).
 * Defining ORACLE_PLANT=<n> compiles a deliberately wrong variant; the tests use those
 * variants to show that the pins catch each planted mistake.
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

static void set_threads(int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
}

int oracle_openmp_enabled(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

/* The k-i-j loop of Eq. 1 for intermediate vertices k in [k0, k1), int64 with threshold inf.
 * oracle_fw_i64 runs it for every k; the benchmark's CPU baseline times a prefix of it. */
void oracle_fw_i64_steps(int64_t *d, int64_t n, int64_t inf, int64_t k0, int64_t k1, int threads) {
  set_threads(threads);
#if ORACLE_PLANT == 2 /* plant 2: intermediate vertex innermost (i-j-k): not Floyd-Warshall */
  (void)k0; (void)k1;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      for (int64_t k = 0; k < n; ++k)
        if (d[i * n + k] < inf && d[k * n + j] < inf && d[i * n + k] + d[k * n + j] < d[i * n + j])
          d[i * n + j] = d[i * n + k] + d[k * n + j];
#else
  for (int64_t k = k0; k < k1; ++k) {
    const int64_t *rowk = d + k * n;
#pragma omp parallel for schedule(static) if (threads > 1)
    for (int64_t i = 0; i < n; ++i) {
      int64_t *rowi = d + i * n;
      const int64_t dik = rowi[k];
      if (dik >= inf) continue; /* no path i -> k yet: nothing to relax through k */
      for (int64_t j = 0; j < n; ++j) {
#if ORACLE_PLANT == 3 /* plant 3: swapped index, d[i][k] + d[j][k] */
        const int64_t dkj = d[j * n + k];
#else
        const int64_t dkj = rowk[j];
#endif
        if (dkj >= inf) continue;
        const int64_t s = dik + dkj;
        if (s < rowi[j]) rowi[j] = s;
      }
    }
  }
#endif
}

/* Eq. 1 over int64 with an "unreachable" threshold inf. In place on d (n x n). */
void oracle_fw_i64(int64_t *d, int64_t n, int64_t inf, int threads) {
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < n; ++j)
      if (d[i * n + j] >= inf) d[i * n + j] = inf;
#if ORACLE_PLANT != 1 /* plant 1: forget that a vertex reaches itself at cost 0 */
    d[i * n + i] = 0;
#endif
  }
  oracle_fw_i64_steps(d, n, inf, 0, n, threads);
  for (int64_t i = 0; i < n * n; ++i)
    if (d[i] >= inf) d[i] = inf;
}

/* The k-i-j loop of Eq. 1 over fp64 for k in [k0, k1); +infinity = unreachable. */
void oracle_fw_f64_steps(double *d, int64_t n, int64_t k0, int64_t k1, int threads) {
  set_threads(threads);
  for (int64_t k = k0; k < k1; ++k) {
    const double *rowk = d + k * n;
#pragma omp parallel for schedule(static) if (threads > 1)
    for (int64_t i = 0; i < n; ++i) {
      double *rowi = d + i * n;
      const double dik = rowi[k];
      if (isinf(dik)) continue;
      for (int64_t j = 0; j < n; ++j) {
        const double s = dik + rowk[j];
        if (s < rowi[j]) rowi[j] = s;
      }
    }
  }
}

/* Eq. 1 over fp64 with +infinity as "unreachable". In place on d (n x n). */
void oracle_fw_f64(double *d, int64_t n, int threads) {
  for (int64_t i = 0; i < n; ++i) d[i * n + i] = 0.0;
  oracle_fw_f64_steps(d, n, 0, n, threads);
}

/* Eq. 2: Z = X (x) Y, or Z = min(Z, X (x) Y) when accumulate != 0.
 * X is M x K, Y is K x N, Z is M x N, all dense row-major. int64 with threshold inf. */
void oracle_minplus_i64(int64_t *Z, const int64_t *X, const int64_t *Y, int64_t M, int64_t N,
                        int64_t K, int64_t inf, int accumulate) {
  for (int64_t i = 0; i < M; ++i)
    for (int64_t j = 0; j < N; ++j) {
      int64_t best = accumulate ? Z[i * N + j] : inf;
      if (best > inf) best = inf;
      for (int64_t k = 0; k < K; ++k) {
#if ORACLE_PLANT == 4 /* plant 4: transposed operand, X[k][i] + Y[j][k] (square cases only) */
        const int64_t x = X[k * K + i], y = Y[j * N + k];
#else
        const int64_t x = X[i * K + k], y = Y[k * N + j];
#endif
        if (x >= inf || y >= inf) continue;
        if (x + y < best) best = x + y;
      }
      Z[i * N + j] = best >= inf ? inf : best;
    }
}

void oracle_minplus_f64(double *Z, const double *X, const double *Y, int64_t M, int64_t N,
                        int64_t K, int accumulate) {
  for (int64_t i = 0; i < M; ++i)
    for (int64_t j = 0; j < N; ++j) {
      double best = accumulate ? Z[i * N + j] : INFINITY;
      for (int64_t k = 0; k < K; ++k) {
        const double s = X[i * K + k] + Y[k * N + j];
        if (s < best) best = s;
      }
      Z[i * N + j] = best;
    }
}

/* Selected rows of Eq. 2 on operands in their storage types: for r < nrows,
 *   Z[r][j] = min_k ( X[rows[r]][k] + Y[k][j] )      (folded into Z when accumulate != 0),
 * X is M x K and Y is K x N (int32, leading dimensions K and N), Z is nrows x N int64.  Each value
 * is widened to int64 as it is read, so no sum overflows.  The candidate sums are those of
 * oracle_minplus_i64; they are visited k-outer (a row of Y at a time) because the minimum of a
 * set does not depend on the order it is taken in, and a column walk of a large Y would take
 * hours.  Entries >= inf are missing; a result >= inf is written as inf. */
void oracle_minplus_rows_i32(int64_t *Z, const int32_t *X, const int32_t *Y, int64_t N, int64_t K,
                             const int64_t *rows, int64_t nrows, int64_t inf, int accumulate, int threads) {
  set_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) if (threads > 1)
  for (int64_t r = 0; r < nrows; ++r) {
#if ORACLE_PLANT == 8 /* plant 8: the r-th row of X instead of row rows[r] */
    const int32_t *x = X + r * K;
#else
    const int32_t *x = X + rows[r] * K;
#endif
    int64_t *z = Z + r * N;
    for (int64_t j = 0; j < N; ++j) {
      int64_t v = accumulate ? z[j] : inf;
      z[j] = v > inf ? inf : v;
    }
    for (int64_t k = 0; k < K; ++k) {
      const int64_t xk = x[k];
      if (xk >= inf) continue;
      const int32_t *y = Y + k * N;
      for (int64_t j = 0; j < N; ++j) {
        const int64_t ykj = y[j];
        if (ykj >= inf) continue;
        if (xk + ykj < z[j]) z[j] = xk + ykj;
      }
    }
  }
}

/* The same over float32 operands, each widened to fp64 as it is read (the sum of two fp32
 * values is exact in fp64); +infinity = missing. */
void oracle_minplus_rows_f32(double *Z, const float *X, const float *Y, int64_t N, int64_t K,
                             const int64_t *rows, int64_t nrows, int accumulate, int threads) {
  set_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) if (threads > 1)
  for (int64_t r = 0; r < nrows; ++r) {
    const float *x = X + rows[r] * K;
    double *z = Z + r * N;
    if (!accumulate)
      for (int64_t j = 0; j < N; ++j) z[j] = INFINITY;
    for (int64_t k = 0; k < K; ++k) {
      const double xk = x[k];
      if (isinf(xk)) continue;
      const float *y = Y + k * N;
      for (int64_t j = 0; j < N; ++j) {
        const double s = xk + (double)y[j];
        if (s < z[j]) z[j] = s;
      }
    }
  }
}

/* Array Dijkstra from each source in src[0..nsrc): out is nsrc x n.
 * w is the n x n weight matrix (entry >= inf: no edge); the diagonal is ignored. */
void oracle_dijkstra_rows_i64(const int64_t *w, int64_t n, int64_t inf, const int64_t *src,
                              int64_t nsrc, int64_t *out, int threads) {
  set_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) if (threads > 1)
  for (int64_t s = 0; s < nsrc; ++s) {
    int64_t *dist = out + s * n;
    unsigned char *done = (unsigned char *)calloc((size_t)n, 1);
    for (int64_t v = 0; v < n; ++v) dist[v] = inf;
    dist[src[s]] = 0;
    for (;;) {
      int64_t u = -1, du = inf;
      for (int64_t v = 0; v < n; ++v)
        if (!done[v] && dist[v] < du) { du = dist[v]; u = v; }
      if (u < 0) break; /* every remaining vertex is unreachable */
      done[u] = 1;
      const int64_t *row = w + u * n;
      for (int64_t v = 0; v < n; ++v) {
        if (v == u || done[v] || row[v] >= inf) continue;
        if (du + row[v] < dist[v]) dist[v] = du + row[v];
      }
    }
    for (int64_t v = 0; v < n; ++v)
      if (dist[v] >= inf) dist[v] = inf;
    free(done);
  }
}

void oracle_dijkstra_rows_f64(const double *w, int64_t n, const int64_t *src, int64_t nsrc,
                              double *out, int threads) {
  set_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) if (threads > 1)
  for (int64_t s = 0; s < nsrc; ++s) {
    double *dist = out + s * n;
    unsigned char *done = (unsigned char *)calloc((size_t)n, 1);
    for (int64_t v = 0; v < n; ++v) dist[v] = INFINITY;
    dist[src[s]] = 0.0;
    for (;;) {
      int64_t u = -1;
      double du = INFINITY;
      for (int64_t v = 0; v < n; ++v)
        if (!done[v] && dist[v] < du) { du = dist[v]; u = v; }
      if (u < 0) break;
      done[u] = 1;
      const double *row = w + u * n;
      for (int64_t v = 0; v < n; ++v) {
        if (v == u || done[v] || isinf(row[v])) continue;
        if (du + row[v] < dist[v]) dist[v] = du + row[v];
      }
    }
    free(done);
  }
}

/* Eq. 1 with predecessor indices (Sec. 2), int64 with threshold inf; d is closed in place like
 * oracle_fw_i64 and pred (n x n) receives the predecessor of j on the path found from i. */
void oracle_fw_pred_i64(int64_t *d, int64_t *pred, int64_t n, int64_t inf) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      if (d[i * n + j] >= inf) d[i * n + j] = inf;
      if (i == j) d[i * n + j] = 0;
      pred[i * n + j] = (i != j && d[i * n + j] < inf) ? i : -1;
    }
  for (int64_t k = 0; k < n; ++k)
    for (int64_t i = 0; i < n; ++i) {
      const int64_t dik = d[i * n + k];
      if (dik >= inf) continue;
      for (int64_t j = 0; j < n; ++j) {
        const int64_t dkj = d[k * n + j];
        if (dkj >= inf) continue;
        if (dik + dkj < d[i * n + j]) {
          d[i * n + j] = dik + dkj;
          pred[i * n + j] = pred[k * n + j];
        }
      }
    }
}

void oracle_fw_pred_f64(double *d, int64_t *pred, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      if (i == j) d[i * n + j] = 0.0;
      pred[i * n + j] = (i != j && !isinf(d[i * n + j])) ? i : -1;
    }
  for (int64_t k = 0; k < n; ++k)
    for (int64_t i = 0; i < n; ++i) {
      const double dik = d[i * n + k];
      if (isinf(dik)) continue;
      for (int64_t j = 0; j < n; ++j)
        if (dik + d[k * n + j] < d[i * n + j]) {
          d[i * n + j] = dik + d[k * n + j];
          pred[i * n + j] = pred[k * n + j];
        }
    }
}

/* pred[i][j] = smallest k != j minimising d[i][k] + w[k][j] over int64 (entries >= inf are
 * unreachable / missing); -1 when i == j or no finite sum stays below inf.  Only the source
 * rows rows[0..nrows) are computed: d and pred hold those rows (nrows x n), w is n x n. */
void oracle_last_hop_i64(const int64_t *d, const int64_t *w, int64_t *pred, int64_t n, const int64_t *rows,
                         int64_t nrows, int64_t inf, int threads) {
  set_threads(threads);
#pragma omp parallel for schedule(static) if (threads > 1)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = rows[r];
    for (int64_t j = 0; j < n; ++j) {
      int64_t best = inf, arg = -1;
      if (i != j)
        for (int64_t k = 0; k < n; ++k) {
#if ORACLE_PLANT != 6 /* plant 6: let j be its own last hop */
          if (k == j) continue;
#endif
          const int64_t dik = d[r * n + k];
#if ORACLE_PLANT == 5 /* plant 5: transposed cost, w[j][k] */
          const int64_t wkj = w[j * n + k];
#else
          const int64_t wkj = w[k * n + j];
#endif
          if (dik >= inf || wkj >= inf) continue;
          if (dik + wkj < best) { best = dik + wkj; arg = k; }
        }
      pred[r * n + j] = arg;
    }
  }
}

/* The same over float32 sums (round to nearest); +infinity = unreachable / missing. */
void oracle_last_hop_f32(const float *d, const float *w, int64_t *pred, int64_t n, const int64_t *rows,
                         int64_t nrows, int threads) {
  set_threads(threads);
#pragma omp parallel for schedule(static) if (threads > 1)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = rows[r];
    for (int64_t j = 0; j < n; ++j) {
      float best = INFINITY;
      int64_t arg = -1;
      if (i != j)
        for (int64_t k = 0; k < n; ++k) {
          if (k == j) continue;
          const float s = d[r * n + k] + w[k * n + j];
          if (s < best) { best = s; arg = k; }
        }
      pred[r * n + j] = arg;
    }
  }
}

/* Bellman-Ford from each source in src[0..nsrc): out is nsrc x n, neg[s] = 1 when a negative
 * cycle is reachable from src[s] (its row is then not meaningful).  int64, entries >= inf are
 * missing edges; the diagonal of w is ignored. */
void oracle_bellman_ford_rows_i64(const int64_t *w, int64_t n, int64_t inf, const int64_t *src, int64_t nsrc,
                                  int64_t *out, int *neg, int threads) {
  set_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) if (threads > 1)
  for (int64_t s = 0; s < nsrc; ++s) {
    int64_t *dist = out + s * n;
    for (int64_t v = 0; v < n; ++v) dist[v] = inf;
    dist[src[s]] = 0;
#if ORACLE_PLANT == 7 /* plant 7: one relaxation round too few */
    const int64_t rounds = n - 1 > 0 ? n - 2 : 0;
#else
    const int64_t rounds = n - 1;
#endif
    for (int64_t r = 0; r < rounds; ++r) {
      int changed = 0;
      for (int64_t u = 0; u < n; ++u) {
        if (dist[u] >= inf) continue;
        for (int64_t v = 0; v < n; ++v) {
          const int64_t wuv = w[u * n + v];
          if (v == u || wuv >= inf) continue;
          if (dist[u] + wuv < dist[v]) { dist[v] = dist[u] + wuv; changed = 1; }
        }
      }
      if (!changed) break;
    }
    neg[s] = 0;
    for (int64_t u = 0; u < n && !neg[s]; ++u) {
      if (dist[u] >= inf) continue;
      for (int64_t v = 0; v < n; ++v) {
        const int64_t wuv = w[u * n + v];
        if (v != u && wuv < inf && dist[u] + wuv < dist[v]) { neg[s] = 1; break; }
      }
    }
  }
}

void oracle_bellman_ford_rows_f64(const double *w, int64_t n, const int64_t *src, int64_t nsrc, double *out,
                                  int *neg, int threads) {
  set_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) if (threads > 1)
  for (int64_t s = 0; s < nsrc; ++s) {
    double *dist = out + s * n;
    for (int64_t v = 0; v < n; ++v) dist[v] = INFINITY;
    dist[src[s]] = 0.0;
    for (int64_t r = 0; r < n - 1; ++r) {
      int changed = 0;
      for (int64_t u = 0; u < n; ++u) {
        if (isinf(dist[u])) continue;
        for (int64_t v = 0; v < n; ++v) {
          const double wuv = w[u * n + v];
          if (v == u || isinf(wuv)) continue;
          if (dist[u] + wuv < dist[v]) { dist[v] = dist[u] + wuv; changed = 1; }
        }
      }
      if (!changed) break;
    }
    neg[s] = 0;
    for (int64_t u = 0; u < n && !neg[s]; ++u) {
      if (isinf(dist[u])) continue;
      for (int64_t v = 0; v < n; ++v) {
        const double wuv = w[u * n + v];
        if (v != u && !isinf(wuv) && dist[u] + wuv < dist[v]) { neg[s] = 1; break; }
      }
    }
  }
}
