/*
 * oracle/brandes.c - plain, slow, CPU reference for betweenness centrality.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header or helper with the CUDA path.
 *
 * What it computes: Eq. 1 of the paper, bc[v] = sum over ordered pairs
 * (s, t), s != v != t, s != t, of sigma_st(v) / sigma_st, on the graph as
 * given (no shattering, no compression).  It does so with Algorithm 1
 * (Bc-Org): per source a BFS with a FIFO queue that counts shortest paths
 * (phase 1), then back-propagation in reverse BFS order with Eq. 3
 * (phase 2), and bc[w] += delta[w] for w != s.  The predecessor lists P[w]
 * of Algorithm 1 are taken from their definition (Section 2.1): the
 * neighbours v of w with d[v] = d[w] - 1.
 *
 * Path counts can exceed the double range on large grids, so every sigma is
 * held as a pair (m, e) meaning m * 2^e with m in [0.5, 1) (or m = 0): an
 * extended exponent per vertex.  Integers below 2^53 stay exact.
 *
 * Sources are split over threads statically (source i -> thread i mod T);
 * each thread sums into its own array and the arrays are added in thread
 * order, so a run is deterministic for a given thread count.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EXPORT __attribute__((visibility("default")))

typedef struct {
  double m;  /* 0 or in [0.5, 1) */
  int64_t e; /* value = m * 2^e */
} xnum;

static xnum xn_make(double x, int64_t e) {
  xnum r;
  if (x == 0.0) {
    r.m = 0.0;
    r.e = 0;
    return r;
  }
  int k;
  r.m = frexp(x, &k);
  r.e = e + k;
  return r;
}

static xnum xn_add(xnum a, xnum b) {
  if (a.m == 0.0) return b;
  if (b.m == 0.0) return a;
  if (a.e < b.e) {
    xnum t = a;
    a = b;
    b = t;
  }
  int64_t diff = b.e - a.e; /* <= 0 */
  double bs = diff < -1100 ? 0.0 : ldexp(b.m, (int)diff);
  return xn_make(a.m + bs, a.e);
}

/* a / b as a plain double (0 on underflow); b != 0 */
static double xn_ratio(xnum a, xnum b) {
  int64_t diff = a.e - b.e;
  if (diff < -1100) return 0.0;
  if (diff > 1100) return INFINITY;
  return ldexp(a.m / b.m, (int)diff);
}

/* One source of Algorithm 1.  Fills d, sig, del; order[] receives the BFS
 * queue (which is also the stack S of the algorithm).  Adds delta[w] to
 * bc[w] for w != s when bc is not NULL.  Returns the number of vertices
 * reached. */
static int64_t brandes_source(int64_t n, const int64_t *rp, const int32_t *col, int64_t s, int32_t *d,
                              xnum *sig, double *del, int32_t *order, double *bc) {
  for (int64_t v = 0; v < n; v++) {
    d[v] = -1;
    sig[v].m = 0.0;
    sig[v].e = 0;
    del[v] = 0.0;
  }
  int64_t head = 0, tail = 0;
  order[tail++] = (int32_t)s;
  d[s] = 0;
  sig[s] = xn_make(1.0, 0);
  /* phase 1: BFS from s */
  while (head < tail) {
    int32_t v = order[head++];
    for (int64_t k = rp[v]; k < rp[v + 1]; k++) {
      int32_t w = col[k];
      if (d[w] < 0) {
        order[tail++] = w;
        d[w] = d[v] + 1;
      }
      if (d[w] == d[v] + 1) sig[w] = xn_add(sig[w], sig[v]);
    }
  }
  /* phase 2: back-propagation, popping the stack (reverse queue order) */
  for (int64_t i = tail - 1; i >= 0; i--) {
    int32_t w = order[i];
    for (int64_t k = rp[w]; k < rp[w + 1]; k++) {
      int32_t v = col[k];
      if (d[v] == d[w] - 1) del[v] += xn_ratio(sig[v], sig[w]) * (1.0 + del[w]);
    }
    if (w != s && bc) bc[w] += del[w];
  }
  return tail;
}

/* bc over the given sources (all sources when src == NULL).  Returns 0, or
 * -1 on allocation failure. */
static int bc_run(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *src, int64_t k,
                  int nthreads, double *bc_out) {
  if (nthreads < 1) nthreads = 1;
  double *part = (double *)calloc((size_t)nthreads * (size_t)(n > 0 ? n : 1), sizeof(double));
  if (!part) return -1;
  int failed = 0;
#pragma omp parallel num_threads(nthreads)
  {
    int t = omp_get_thread_num();
    int32_t *d = (int32_t *)malloc((size_t)n * sizeof(int32_t) + 4);
    xnum *sig = (xnum *)malloc((size_t)n * sizeof(xnum) + 16);
    double *del = (double *)malloc((size_t)n * sizeof(double) + 8);
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t) + 4);
    if (!d || !sig || !del || !order) {
#pragma omp atomic write
      failed = 1;
    } else {
      double *mine = part + (size_t)t * (size_t)n;
      for (int64_t i = t; i < k; i += nthreads) {
        int64_t s = src ? src[i] : i;
        brandes_source(n, rp, col, s, d, sig, del, order, mine);
      }
    }
    free(d);
    free(sig);
    free(del);
    free(order);
  }
  if (!failed) {
    for (int64_t v = 0; v < n; v++) {
      double acc = 0.0;
      for (int t = 0; t < nthreads; t++) acc += part[(size_t)t * (size_t)n + (size_t)v];
      bc_out[v] = acc;
    }
  }
  free(part);
  return failed ? -1 : 0;
}

/* Full betweenness (Eq. 1) of every vertex. */
OR_EXPORT int oracle_bc(int64_t n, const int64_t *row_ptr, const int32_t *col, int nthreads,
                        double *bc_out) {
  if (n < 0) return -2;
  if (n == 0) return 0;
  return bc_run(n, row_ptr, col, NULL, n, nthreads, bc_out);
}

/* Partial sum sum_{s in src} delta_s(v) for every v (sources may repeat). */
OR_EXPORT int oracle_bc_sources(int64_t n, const int64_t *row_ptr, const int32_t *col,
                                const int64_t *src, int64_t k, int nthreads, double *bc_out) {
  if (n < 0 || k < 0) return -2;
  for (int64_t i = 0; i < k; i++)
    if (src[i] < 0 || src[i] >= n) return -2;
  if (n == 0) return 0;
  return bc_run(n, row_ptr, col, src, k, nthreads, bc_out);
}

/* Single source: distances (-1 unreachable), sigma as mantissa * 2^exp2 with
 * the mantissa in [0.5, 1) (0 when unreachable), and delta_s(v). */
OR_EXPORT int oracle_sssp(int64_t n, const int64_t *row_ptr, const int32_t *col, int64_t s,
                          int32_t *d, double *sig_m, int64_t *sig_e, double *delta) {
  if (n <= 0 || s < 0 || s >= n) return -2;
  xnum *sig = (xnum *)malloc((size_t)n * sizeof(xnum));
  int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!sig || !order) {
    free(sig);
    free(order);
    return -1;
  }
  brandes_source(n, row_ptr, col, s, d, sig, delta, order, NULL);
  for (int64_t v = 0; v < n; v++) {
    sig_m[v] = sig[v].m;
    sig_e[v] = sig[v].e;
  }
  free(sig);
  free(order);
  return 0;
}

/* Sum over ordered reachable pairs (s, t), s != t, of d(s,t) - 1, and the
 * number of such pairs.  A property of Eq. 1: the pair dependencies of one
 * pair add up to the number of interior vertices of a shortest path. */
OR_EXPORT int oracle_pair_stats(int64_t n, const int64_t *row_ptr, const int32_t *col, int nthreads,
                                double *sum_dm1, int64_t *pairs) {
  if (n < 0) return -2;
  double tot = 0.0;
  int64_t cnt = 0;
  int failed = 0;
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads) reduction(+ : tot, cnt)
  {
    int t = omp_get_thread_num();
    int32_t *d = (int32_t *)malloc((size_t)n * sizeof(int32_t) + 4);
    int32_t *q = (int32_t *)malloc((size_t)n * sizeof(int32_t) + 4);
    if (!d || !q) {
#pragma omp atomic write
      failed = 1;
    } else {
      for (int64_t s = t; s < n; s += nthreads) {
        for (int64_t v = 0; v < n; v++) d[v] = -1;
        int64_t h = 0, tl = 0;
        q[tl++] = (int32_t)s;
        d[s] = 0;
        while (h < tl) {
          int32_t v = q[h++];
          if (v != s) {
            tot += (double)(d[v] - 1);
            cnt += 1;
          }
          for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; k++)
            if (d[col[k]] < 0) {
              d[col[k]] = d[v] + 1;
              q[tl++] = col[k];
            }
        }
      }
    }
    free(d);
    free(q);
  }
  *sum_dm1 = tot;
  *pairs = cnt;
  return failed ? -1 : 0;
}
