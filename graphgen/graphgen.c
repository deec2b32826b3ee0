/*
 * graphgen.c - seeded synthetic graph generators.
 *
 * Input tooling only: this file holds no betweenness arithmetic.  Both the
 * oracle tests and the CUDA path draw their inputs from here; neither side's
 * arithmetic lives here.
 *
 * Every graph is undirected, unweighted, loop-free and stored as a CSR with
 * int64 row offsets and int32 column ids, each row sorted ascending and free
 * of duplicates (the 32-bit CRS of the paper's Section 4).  Every generator
 * ends with a seeded random relabelling, because the paper shows that the
 * natural order of a graph changes the BFS cost (Section 4.1).
 *
 * PRNG: xoshiro256** (Blackman and Vigna) seeded through splitmix64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ PRNG */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_step(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

GG_EXPORT uint64_t gg_splitmix64(uint64_t x) { return splitmix64_step(&x); }

static void rng_seed(rng_t *r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; i++) r->s[i] = splitmix64_step(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_u64(rng_t *r) {
  uint64_t *s = r->s;
  uint64_t out = rotl64(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return out;
}

/* uniform double in [0, 1) with 53 random bits */
static double rng_unif(rng_t *r) { return (double)(rng_u64(r) >> 11) * 0x1.0p-53; }

/* unbiased integer in [0, n), n >= 1 (multiply-high with rejection) */
static uint64_t rng_below(rng_t *r, uint64_t n) {
  uint64_t threshold = (0 - n) % n; /* 2^64 mod n */
  for (;;) {
    __uint128_t m = (__uint128_t)rng_u64(r) * n;
    if ((uint64_t)m >= threshold) return (uint64_t)(m >> 64);
  }
}

/* uniform integer in [lo, hi] */
static int64_t rng_range(rng_t *r, int64_t lo, int64_t hi) {
  return lo + (int64_t)rng_below(r, (uint64_t)(hi - lo + 1));
}

/* ------------------------------------------------------------ edge list */
typedef struct {
  int32_t *u, *v;
  int64_t len, cap;
} elist;

static int el_push(elist *e, int64_t a, int64_t b) {
  if (e->len == e->cap) {
    int64_t nc = e->cap ? e->cap * 2 : 1024;
    int32_t *nu = (int32_t *)realloc(e->u, (size_t)nc * sizeof(int32_t));
    if (!nu) return -1;
    e->u = nu;
    int32_t *nv = (int32_t *)realloc(e->v, (size_t)nc * sizeof(int32_t));
    if (!nv) return -1;
    e->v = nv;
    e->cap = nc;
  }
  e->u[e->len] = (int32_t)a;
  e->v[e->len] = (int32_t)b;
  e->len++;
  return 0;
}

static void el_free(elist *e) {
  free(e->u);
  free(e->v);
  e->u = e->v = NULL;
  e->len = e->cap = 0;
}

/* ------------------------------------------------------------------ CSR */
typedef struct {
  int64_t n;
  int64_t nnz;
  int64_t *row_ptr; /* n+1 */
  int32_t *col;     /* nnz */
} gg_csr;

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Symmetrise, drop self-loops, sort rows and drop duplicates. */
static int build_csr(int64_t n, const elist *e, gg_csr *out) {
  int64_t *rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!rp) return -1;
  for (int64_t i = 0; i < e->len; i++) {
    if (e->u[i] == e->v[i]) continue;
    rp[e->u[i] + 1]++;
    rp[e->v[i] + 1]++;
  }
  for (int64_t i = 0; i < n; i++) rp[i + 1] += rp[i];
  int32_t *col = (int32_t *)malloc((size_t)(rp[n] > 0 ? rp[n] : 1) * sizeof(int32_t));
  int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  if (!col || !fill) {
    free(rp);
    free(col);
    free(fill);
    return -1;
  }
  memcpy(fill, rp, (size_t)n * sizeof(int64_t));
  for (int64_t i = 0; i < e->len; i++) {
    int32_t a = e->u[i], b = e->v[i];
    if (a == b) continue;
    col[fill[a]++] = b;
    col[fill[b]++] = a;
  }
  free(fill);
  /* sort + dedup each row, compacting in place */
  int64_t w = 0;
  int64_t start = rp[0];
  for (int64_t v = 0; v < n; v++) {
    int64_t end = rp[v + 1];
    int64_t len = end - start;
    if (len > 1) qsort(col + start, (size_t)len, sizeof(int32_t), cmp_i32);
    int64_t row_begin = w;
    for (int64_t k = start; k < end; k++) {
      if (k > start && col[k] == col[k - 1]) continue;
      col[w++] = col[k];
    }
    rp[v] = row_begin;
    start = end;
  }
  rp[n] = w;
  out->n = n;
  out->nnz = w;
  out->row_ptr = rp;
  out->col = col;
  return 0;
}

/* Random permutation pi of [0,n) (Fisher-Yates). */
static int32_t *random_perm(rng_t *r, int64_t n) {
  int32_t *p = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!p) return NULL;
  for (int64_t i = 0; i < n; i++) p[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; i--) {
    int64_t j = (int64_t)rng_below(r, (uint64_t)i + 1);
    int32_t t = p[i];
    p[i] = p[j];
    p[j] = t;
  }
  return p;
}

/* Relabel the edge list by a seeded permutation, then build the CSR. */
static int finish(rng_t *r, int64_t n, elist *e, gg_csr *out) {
  int32_t *p = random_perm(r, n);
  if (!p) return -1;
  for (int64_t i = 0; i < e->len; i++) {
    e->u[i] = p[e->u[i]];
    e->v[i] = p[e->v[i]];
  }
  free(p);
  return build_csr(n, e, out);
}

GG_EXPORT void gg_free(void *p) { free(p); }

/* ------------------------------------------------------------ Chung-Lu */
/*
 * Chung-Lu graph by endpoint sampling: expected-degree weights
 * w_i = c * (i+1)^(-1/(gamma-1)), scaled so that their mean is mean_deg and
 * capped at sqrt(sum w); round(n*mean_deg/2) edges are drawn with both
 * endpoints proportional to w.  Self-loops and repeats are dropped by the
 * CSR build.  Vertices are appended to `e` at ids [base, base+n).
 */
static int chung_lu_edges(rng_t *r, int64_t n, double gamma, double mean_deg, int64_t base,
                          elist *e) {
  if (n <= 1) return 0;
  double *cdf = (double *)malloc((size_t)n * sizeof(double));
  if (!cdf) return -1;
  double expo = -1.0 / (gamma - 1.0), sum = 0.0;
  for (int64_t i = 0; i < n; i++) {
    cdf[i] = pow((double)(i + 1), expo);
    sum += cdf[i];
  }
  double scale = mean_deg * (double)n / sum, total = 0.0;
  double cap = sqrt(mean_deg * (double)n);
  for (int64_t i = 0; i < n; i++) {
    double w = cdf[i] * scale;
    if (w > cap) w = cap;
    total += w;
    cdf[i] = total;
  }
  int64_t m = (int64_t)llround((double)n * mean_deg / 2.0);
  for (int64_t k = 0; k < m; k++) {
    int64_t ends[2];
    for (int t = 0; t < 2; t++) {
      double x = rng_unif(r) * total;
      int64_t lo = 0, hi = n - 1;
      while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (cdf[mid] > x) hi = mid;
        else lo = mid + 1;
      }
      ends[t] = lo;
    }
    if (ends[0] == ends[1]) continue;
    if (el_push(e, base + ends[0], base + ends[1])) {
      free(cdf);
      return -1;
    }
  }
  free(cdf);
  return 0;
}

GG_EXPORT int gg_chung_lu(int64_t n, double gamma, double mean_deg, uint64_t seed, gg_csr *out) {
  rng_t r;
  rng_seed(&r, seed);
  elist e = {0};
  int rc = chung_lu_edges(&r, n, gamma, mean_deg, 0, &e);
  if (!rc) rc = finish(&r, n, &e, out);
  el_free(&e);
  return rc;
}

/* ------------------------------------------------------- Erdos-Renyi G(s,p) */
/* All pairs i < j on ids [base, base+s) with probability p, by geometric
 * skipping over the pairs in row-major lower-triangular order. */
static int er_edges(rng_t *r, int64_t s, double p, const int64_t *ids, elist *e) {
  if (s < 2 || p <= 0.0) return 0;
  if (p >= 1.0) {
    for (int64_t i = 1; i < s; i++)
      for (int64_t j = 0; j < i; j++)
        if (el_push(e, ids[i], ids[j])) return -1;
    return 0;
  }
  double lq = log(1.0 - p);
  int64_t i = 1, j = -1;
  for (;;) {
    double u = rng_unif(r);
    int64_t skip = (int64_t)floor(log(1.0 - u) / lq);
    j += 1 + skip;
    while (j >= i && i < s) {
      j -= i;
      i++;
    }
    if (i >= s) break;
    if (el_push(e, ids[i], ids[j])) return -1;
  }
  return 0;
}

/* ------------------------------------------------------- the five configs */

/* 1: Chung-Lu core (n_core, gamma 2.5, mean degree 4) plus n_pend pendant
 * vertices, each attached to a uniformly chosen core vertex. */
static int cfg_small(rng_t *r, int64_t n_core, int64_t n_pend, gg_csr *out) {
  elist e = {0};
  int rc = chung_lu_edges(r, n_core, 2.5, 4.0, 0, &e);
  for (int64_t k = 0; !rc && k < n_pend; k++)
    rc = el_push(&e, n_core + k, (int64_t)rng_below(r, (uint64_t)n_core));
  if (!rc) rc = finish(r, n_core + n_pend, &e, out);
  el_free(&e);
  return rc;
}

/* 2: n_blocks Erdos-Renyi blocks, sizes round(exp(U[ln 4, ln 512])), edge
 * probability min(1, 6/(s-1)); block b >= 1 reuses one vertex of a uniformly
 * chosen earlier block (uniform vertex of it) as its own first vertex.  Then
 * chains of U{1..20} new vertices hang off uniform block vertices until the
 * chain vertices are 20% of all vertices. */
static int cfg_articulation(rng_t *r, int64_t n_blocks, gg_csr *out) {
  elist e = {0};
  int64_t *boff = (int64_t *)malloc((size_t)(n_blocks + 1) * sizeof(int64_t));
  int64_t *ids = (int64_t *)malloc(512 * sizeof(int64_t));
  int rc = (!boff || !ids) ? -1 : 0;
  int64_t nv = 0;
  for (int64_t b = 0; !rc && b < n_blocks; b++) {
    int64_t s = (int64_t)llround(exp(log(4.0) + rng_unif(r) * (log(512.0) - log(4.0))));
    if (s < 4) s = 4;
    if (s > 512) s = 512;
    double p = 6.0 / (double)(s - 1);
    if (p > 1.0) p = 1.0;
    boff[b] = nv;
    if (b == 0) {
      for (int64_t i = 0; i < s; i++) ids[i] = nv + i;
      nv += s;
    } else {
      int64_t pb = (int64_t)rng_below(r, (uint64_t)b);
      int64_t lo = boff[pb], hi = boff[pb + 1];
      ids[0] = lo + (int64_t)rng_below(r, (uint64_t)(hi - lo));
      for (int64_t i = 1; i < s; i++) ids[i] = nv + i - 1;
      nv += s - 1;
    }
    boff[b + 1] = nv;
    rc = er_edges(r, s, p, ids, &e);
  }
  int64_t n_block_vtx = nv;
  int64_t target_chain = (int64_t)ceil(0.25 * (double)n_block_vtx); /* 20% of the total */
  int64_t chain_vtx = 0;
  while (!rc && chain_vtx < target_chain) {
    int64_t len = rng_range(r, 1, 20);
    int64_t prev = (int64_t)rng_below(r, (uint64_t)n_block_vtx);
    for (int64_t k = 0; !rc && k < len; k++) {
      rc = el_push(&e, prev, nv);
      prev = nv++;
    }
    chain_vtx += len;
  }
  if (!rc) rc = finish(r, nv, &e, out);
  free(boff);
  free(ids);
  el_free(&e);
  return rc;
}

/* 3: Chung-Lu core (n_core, gamma 2.1, mean degree 12).  Twin groups: a
 * uniformly chosen core vertex x of degree >= 2 that is not yet in a group
 * gets g-1 copies, g = U{2..8}, until group_vtx vertices (seeds + copies) are
 * in groups.  Every core edge {x,y} becomes the complete bipartite set of
 * edges between x's group and y's group, so each group is a set of vertices
 * with one shared open neighbourhood.  Then n_pend pendant vertices are
 * attached to uniform core vertices that are in no group. */
static int cfg_twins(rng_t *r, int64_t n_core, int64_t group_vtx, int64_t n_pend, gg_csr *out) {
  elist core = {0}, e = {0};
  gg_csr c = {0};
  int rc = chung_lu_edges(r, n_core, 2.1, 12.0, 0, &core);
  if (!rc) rc = build_csr(n_core, &core, &c);
  el_free(&core);
  int64_t *gstart = (int64_t *)malloc((size_t)n_core * sizeof(int64_t)); /* first copy id */
  int32_t *gsize = (int32_t *)malloc((size_t)n_core * sizeof(int32_t));
  if (!rc && (!gstart || !gsize)) rc = -1;
  int64_t nv = n_core, in_groups = 0;
  if (!rc) {
    for (int64_t v = 0; v < n_core; v++) {
      gstart[v] = -1;
      gsize[v] = 1;
    }
    int64_t tries = 0;
    while (in_groups < group_vtx && tries < 100 * n_core) {
      tries++;
      int64_t x = (int64_t)rng_below(r, (uint64_t)n_core);
      if (gsize[x] > 1 || c.row_ptr[x + 1] - c.row_ptr[x] < 2) continue;
      int64_t g = rng_range(r, 2, 8);
      gsize[x] = (int32_t)g;
      gstart[x] = nv;
      nv += g - 1;
      in_groups += g;
    }
    /* blow up every core edge x<y into group(x) x group(y) */
    for (int64_t x = 0; !rc && x < n_core; x++) {
      for (int64_t k = c.row_ptr[x]; !rc && k < c.row_ptr[x + 1]; k++) {
        int64_t y = c.col[k];
        if (y <= x) continue;
        for (int64_t a = 0; !rc && a < gsize[x]; a++) {
          int64_t va = a == 0 ? x : gstart[x] + a - 1;
          for (int64_t b = 0; !rc && b < gsize[y]; b++) {
            int64_t vb = b == 0 ? y : gstart[y] + b - 1;
            rc = el_push(&e, va, vb);
          }
        }
      }
    }
    for (int64_t k = 0; !rc && k < n_pend; k++) {
      int64_t x;
      do x = (int64_t)rng_below(r, (uint64_t)n_core);
      while (gsize[x] > 1);
      rc = el_push(&e, nv + k, x);
    }
    nv += n_pend;
  }
  if (!rc) rc = finish(r, nv, &e, out);
  free(gstart);
  free(gsize);
  free(c.row_ptr);
  free(c.col);
  el_free(&e);
  return rc;
}

/* union-find helpers for the road-like config */
static int64_t uf_find(int64_t *p, int64_t x) {
  while (p[x] != x) {
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

/* 4: side x side grid with 4-neighbour edges; exactly 25% of the edges are
 * deleted (seeded shuffle); the largest connected component is kept.  Then
 * 10% of the outer-perimeter vertices of that component each get a random
 * tree of U{1..64} new vertices, depth <= 8 below the perimeter vertex (each
 * new vertex hangs off a uniform earlier tree vertex of depth < 8). */
static int cfg_road(rng_t *r, int64_t side, gg_csr *out) {
  int64_t n = side * side;
  int64_t ne = 2 * side * (side - 1);
  int64_t *ea = (int64_t *)malloc((size_t)ne * sizeof(int64_t));
  int64_t *par = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *cnt = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  int32_t *newid = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  elist e = {0};
  int rc = (!ea || !par || !cnt || !newid) ? -1 : 0;
  if (!rc) {
    /* edge k < side*(side-1): horizontal (row k/(side-1), col k%(side-1)),
     * else vertical (row j/side, col j%side) with j = k - side*(side-1) */
    int64_t nh = side * (side - 1);
    for (int64_t k = 0; k < ne; k++) ea[k] = k;
    for (int64_t i = ne - 1; i > 0; i--) {
      int64_t j = (int64_t)rng_below(r, (uint64_t)i + 1);
      int64_t t = ea[i];
      ea[i] = ea[j];
      ea[j] = t;
    }
    int64_t ndel = ne / 4;
    for (int64_t v = 0; v < n; v++) par[v] = v;
    for (int64_t t = ndel; t < ne; t++) {
      int64_t k = ea[t], a, b;
      if (k < nh) {
        a = (k / (side - 1)) * side + k % (side - 1);
        b = a + 1;
      } else {
        int64_t j = k - nh;
        a = j;
        b = j + side;
      }
      ea[t] = a * n + b; /* keep the surviving edge as a packed pair */
      int64_t ra = uf_find(par, a), rb = uf_find(par, b);
      if (ra != rb) par[ra < rb ? rb : ra] = ra < rb ? ra : rb;
    }
    int64_t best = 0;
    for (int64_t v = 0; v < n; v++) {
      int64_t rv = uf_find(par, v);
      if (++cnt[rv] > cnt[best]) best = rv;
    }
    int64_t nv = 0;
    for (int64_t v = 0; v < n; v++) newid[v] = uf_find(par, v) == best ? (int32_t)nv++ : -1;
    for (int64_t t = ndel; !rc && t < ne; t++) {
      int64_t a = ea[t] / n, b = ea[t] % n;
      if (newid[a] >= 0 && newid[b] >= 0) rc = el_push(&e, newid[a], newid[b]);
    }
    /* perimeter vertices inside the kept component */
    int64_t *per = (int64_t *)malloc((size_t)(4 * side) * sizeof(int64_t));
    int64_t np = 0;
    if (!per) rc = -1;
    for (int64_t v = 0; !rc && v < n; v++) {
      int64_t i = v / side, j = v % side;
      if ((i == 0 || j == 0 || i == side - 1 || j == side - 1) && newid[v] >= 0) per[np++] = newid[v];
    }
    /* choose 10% of them without repetition (partial Fisher-Yates) */
    int64_t ntrees = np / 10;
    int64_t depth[66], tid[66];
    for (int64_t k = 0; !rc && k < ntrees; k++) {
      int64_t j = k + (int64_t)rng_below(r, (uint64_t)(np - k));
      int64_t t = per[k];
      per[k] = per[j];
      per[j] = t;
      int64_t size = rng_range(r, 1, 64);
      tid[0] = per[k];
      int64_t cnt_t = 1;
      depth[0] = 0;
      for (int64_t q = 0; !rc && q < size; q++) {
        int64_t parent;
        do parent = (int64_t)rng_below(r, (uint64_t)cnt_t);
        while (depth[parent] >= 8);
        tid[cnt_t] = nv;
        depth[cnt_t] = depth[parent] + 1;
        rc = el_push(&e, tid[parent], nv);
        nv++;
        cnt_t++;
      }
    }
    free(per);
    if (!rc) rc = finish(r, nv, &e, out);
  }
  free(ea);
  free(par);
  free(cnt);
  free(newid);
  el_free(&e);
  return rc;
}

/*
 * Configs by id.  scale_pct (1..100) shrinks the sizes for fast tests (100 =
 * full size).  The full sizes:
 *   1: 2,000 core + 600 pendants
 *   2: 5,000 blocks + 20% chains
 *   3: 500,000 core, 150,000 in twin groups, 350,000 pendants
 *   4: 1500 x 1500 grid
 */
GG_EXPORT int gg_config(int id, uint64_t seed, int scale_pct, gg_csr *out) {
  if (scale_pct < 1 || scale_pct > 100) return -2;
  rng_t r;
  rng_seed(&r, seed);
  double f = scale_pct / 100.0;
  switch (id) {
    case 1: return cfg_small(&r, (int64_t)llround(2000 * f), (int64_t)llround(600 * f), out);
    case 2: return cfg_articulation(&r, (int64_t)llround(5000 * f) > 0 ? (int64_t)llround(5000 * f) : 1, out);
    case 3:
      return cfg_twins(&r, (int64_t)llround(500000 * f), (int64_t)llround(150000 * f),
                       (int64_t)llround(350000 * f), out);
    case 4: {
      int64_t side = (int64_t)llround(1500 * sqrt(f));
      return cfg_road(&r, side < 4 ? 4 : side, out);
    }
    default: return -2;
  }
}

/*
 * 5: a batch of `count` independent Chung-Lu graphs (gamma 2.3, mean degree
 * 8), sizes round(exp(U[ln n_min, ln n_max])), graph i seeded with
 * splitmix64(seed + i).  They are packed into one CSR with global ids;
 * vtx_off (count+1, malloc'ed) gives each graph's vertex range.
 */
GG_EXPORT int gg_batch(uint64_t seed, int64_t count, int64_t n_min, int64_t n_max, gg_csr *out,
                       int64_t **vtx_off_out) {
  if (count < 1 || n_min < 2 || n_max < n_min) return -2;
  int64_t *off = (int64_t *)malloc((size_t)(count + 1) * sizeof(int64_t));
  if (!off) return -1;
  elist e = {0};
  int rc = 0;
  int64_t nv = 0;
  rng_t sizes;
  rng_seed(&sizes, seed ^ 0x5A5A5A5A5A5A5A5AULL);
  for (int64_t i = 0; !rc && i < count; i++) {
    int64_t ni = (int64_t)llround(exp(log((double)n_min) + rng_unif(&sizes) * (log((double)n_max) - log((double)n_min))));
    rng_t r;
    rng_seed(&r, gg_splitmix64(seed + (uint64_t)i));
    off[i] = nv;
    int64_t first = e.len;
    rc = chung_lu_edges(&r, ni, 2.3, 8.0, nv, &e);
    /* relabel inside the graph's own id range */
    int32_t *p = rc ? NULL : random_perm(&r, ni);
    if (!rc && !p) rc = -1;
    for (int64_t k = first; !rc && k < e.len; k++) {
      e.u[k] = (int32_t)(nv + p[e.u[k] - nv]);
      e.v[k] = (int32_t)(nv + p[e.v[k] - nv]);
    }
    free(p);
    nv += ni;
  }
  off[count] = nv;
  if (!rc) rc = build_csr(nv, &e, out);
  el_free(&e);
  if (rc) {
    free(off);
    return rc;
  }
  *vtx_off_out = off;
  return 0;
}

/* Build a CSR from an explicit edge list (used for the small test families). */
GG_EXPORT int gg_from_edges(int64_t n, int64_t m, const int32_t *u, const int32_t *v, gg_csr *out) {
  elist e = {0};
  for (int64_t i = 0; i < m; i++) {
    if (u[i] < 0 || v[i] < 0 || u[i] >= n || v[i] >= n) {
      el_free(&e);
      return -2;
    }
    if (el_push(&e, u[i], v[i])) {
      el_free(&e);
      return -1;
    }
  }
  int rc = build_csr(n, &e, out);
  el_free(&e);
  return rc;
}
