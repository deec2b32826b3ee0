/*
 * oracle/shatter.c - plain CPU definitions of the pieces a shattered graph is
 * made of.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header or helper with the CUDA path.
 *
 * Each function states the definition it writes out; none of them uses the
 * linear-time algorithms the paper relies on (Section 3.4), so that they can
 * be read against the definitions in Section 2 by eye:
 *
 *  - 2-core: the largest subgraph of minimum degree 2, found by deleting
 *    vertices of degree < 2 until none is left (what degree-1 removal of
 *    Section 3.3.1, applied until nothing changes, leaves of a graph that is
 *    not a tree);
 *  - biconnected components (Section 2): two edges that share a vertex c lie
 *    in one biconnected component exactly when their other ends are still
 *    connected once c is removed; the components are the classes of the
 *    transitive closure of that relation over adjacent edges;
 *  - reach (Section 3.2): the number of vertices of G that a vertex v of a
 *    piece P stands for, i.e. v itself plus every vertex x of v's connected
 *    component from which no vertex of P other than v can be reached once v
 *    is removed:  reach = N_C - |vertices reachable from P \ {v} in G - v|.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EXPORT __attribute__((visibility("default")))

/* in_core[v] = 1 iff v is in the 2-core of the subgraph induced by mask
 * (mask may be NULL for the whole graph). */
OR_EXPORT int oracle_two_core(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *mask,
                              uint8_t *in_core) {
  int64_t *deg = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  if (!deg) return -1;
  for (int64_t v = 0; v < n; v++) {
    in_core[v] = mask ? mask[v] : 1;
  }
  for (int64_t v = 0; v < n; v++) {
    deg[v] = 0;
    if (!in_core[v]) continue;
    for (int64_t k = rp[v]; k < rp[v + 1]; k++) deg[v] += in_core[col[k]];
  }
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int64_t v = 0; v < n; v++) {
      if (in_core[v] && deg[v] < 2) {
        in_core[v] = 0;
        changed = 1;
        for (int64_t k = rp[v]; k < rp[v + 1]; k++)
          if (in_core[col[k]]) deg[col[k]]--;
      }
    }
  }
  free(deg);
  return 0;
}

/* Connected components of the subgraph induced by mask (NULL = all):
 * label[v] = component id (0..count-1, by smallest member), -1 outside the
 * mask.  Returns the count, or -1 on allocation failure. */
OR_EXPORT int64_t oracle_components(int64_t n, const int64_t *rp, const int32_t *col,
                                    const uint8_t *mask, int32_t *label) {
  int32_t *q = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!q) return -1;
  for (int64_t v = 0; v < n; v++) label[v] = -1;
  int64_t cnt = 0;
  for (int64_t s = 0; s < n; s++) {
    if ((mask && !mask[s]) || label[s] >= 0) continue;
    int64_t h = 0, t = 0;
    q[t++] = (int32_t)s;
    label[s] = (int32_t)cnt;
    while (h < t) {
      int32_t v = q[h++];
      for (int64_t k = rp[v]; k < rp[v + 1]; k++) {
        int32_t w = col[k];
        if ((mask && !mask[w]) || label[w] >= 0) continue;
        label[w] = (int32_t)cnt;
        q[t++] = w;
      }
    }
    cnt++;
  }
  free(q);
  return cnt;
}

static int64_t uf_find(int64_t *p, int64_t x) {
  while (p[x] != x) {
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

static void uf_union(int64_t *p, int64_t a, int64_t b) {
  a = uf_find(p, a);
  b = uf_find(p, b);
  if (a == b) return;
  if (a < b) p[b] = a;
  else p[a] = b;
}

/* Index of entry (v -> u) in v's row, or -1 (rows sorted ascending). */
static int64_t find_entry(const int64_t *rp, const int32_t *col, int64_t v, int32_t u) {
  int64_t lo = rp[v], hi = rp[v + 1];
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (col[mid] < u) lo = mid + 1;
    else hi = mid;
  }
  return (lo < rp[v + 1] && col[lo] == u) ? lo : -1;
}

/*
 * Biconnected components of the subgraph induced by mask (NULL = all).
 * edge_block[k] for every CSR entry k = (u -> v) with both ends in the mask
 * is the block id (0..count-1, numbered by the smallest entry index of an
 * edge in it); -1 otherwise.  Both directions of an edge get the same id.
 * Returns the number of blocks, -1 on allocation failure, -2 if the CSR is
 * not symmetric.  O(n (n + m)).
 */
OR_EXPORT int64_t oracle_blocks(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *mask,
                                int64_t *edge_block) {
  int64_t nnz = rp[n];
  int64_t *uf = (int64_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
  int64_t *canon = (int64_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
  int32_t *lab = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t *q = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int64_t *first = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t rc = 0;
  if (!uf || !canon || !lab || !q || !first) rc = -1;
  /* undirected edge id = entry index of its (min -> max) direction */
  for (int64_t u = 0; !rc && u < n; u++)
    for (int64_t k = rp[u]; k < rp[u + 1]; k++) {
      int32_t v = col[k];
      if (u < v) canon[k] = k;
      else {
        int64_t r = find_entry(rp, col, v, (int32_t)u);
        if (r < 0) {
          rc = -2;
          break;
        }
        canon[k] = r;
      }
    }
  for (int64_t k = 0; k < nnz; k++) uf[k] = k;
  for (int64_t c = 0; !rc && c < n; c++) {
    if (mask && !mask[c]) continue;
    /* components of (masked graph) - c */
    for (int64_t v = 0; v < n; v++) lab[v] = -1;
    int32_t nl = 0;
    for (int64_t k = rp[c]; k < rp[c + 1]; k++) {
      int32_t a = col[k];
      if ((mask && !mask[a]) || lab[a] >= 0) continue;
      int64_t h = 0, t = 0;
      q[t++] = a;
      lab[a] = nl;
      while (h < t) {
        int32_t v = q[h++];
        for (int64_t j = rp[v]; j < rp[v + 1]; j++) {
          int32_t w = col[j];
          if (w == c || (mask && !mask[w]) || lab[w] >= 0) continue;
          lab[w] = nl;
          q[t++] = w;
        }
      }
      nl++;
    }
    /* edges at c whose far ends share a component of G - c share a block */
    for (int32_t i = 0; i < nl; i++) first[i] = -1;
    for (int64_t k = rp[c]; k < rp[c + 1]; k++) {
      int32_t a = col[k];
      if (mask && !mask[a]) continue;
      int32_t l = lab[a];
      if (first[l] < 0) first[l] = canon[k];
      else uf_union(uf, first[l], canon[k]);
    }
  }
  int64_t nb = 0;
  if (!rc) {
    int64_t *bid = (int64_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    if (!bid) rc = -1;
    for (int64_t k = 0; !rc && k < nnz; k++) bid[k] = -1;
    for (int64_t u = 0; !rc && u < n; u++)
      for (int64_t k = rp[u]; k < rp[u + 1]; k++) {
        int32_t v = col[k];
        if (mask && (!mask[u] || !mask[v])) {
          edge_block[k] = -1;
          continue;
        }
        int64_t r = uf_find(uf, canon[k]);
        if (bid[r] < 0) bid[r] = -2; /* mark: numbered in a second pass */
      }
    /* number blocks by smallest canonical entry index */
    for (int64_t k = 0; !rc && k < nnz; k++) {
      if (canon[k] != k) continue;
      int64_t r = uf_find(uf, k);
      if (bid[r] == -2) bid[r] = nb++;
    }
    for (int64_t u = 0; !rc && u < n; u++)
      for (int64_t k = rp[u]; k < rp[u + 1]; k++) {
        int32_t v = col[k];
        if (mask && (!mask[u] || !mask[v])) continue;
        edge_block[k] = bid[uf_find(uf, canon[k])];
      }
    free(bid);
  }
  free(uf);
  free(canon);
  free(lab);
  free(q);
  free(first);
  return rc ? rc : nb;
}

/*
 * reach of every (piece, vertex) slot.  Pieces are given as vertex lists:
 * piece p owns piece_vtx[piece_off[p] .. piece_off[p+1]).  reach_out has one
 * entry per slot:  N_C - |vertices reachable from P \ {v} in G - v|, where
 * N_C is the size of v's connected component in G (the whole graph, mask
 * ignored).  Returns 0, -1 on allocation failure.
 */
OR_EXPORT int oracle_reach(int64_t n, const int64_t *rp, const int32_t *col, int64_t npieces,
                           const int64_t *piece_off, const int32_t *piece_vtx, int64_t *reach_out) {
  int32_t *lab = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t *q = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t *comp = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int64_t *csize = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  if (!lab || !q || !comp || !csize) {
    free(lab);
    free(q);
    free(comp);
    free(csize);
    return -1;
  }
  /* N_C per vertex */
  for (int64_t v = 0; v < n; v++) comp[v] = -1;
  int32_t nc = 0;
  for (int64_t s = 0; s < n; s++) {
    if (comp[s] >= 0) continue;
    int64_t h = 0, t = 0;
    q[t++] = (int32_t)s;
    comp[s] = nc;
    while (h < t) {
      int32_t v = q[h++];
      for (int64_t k = rp[v]; k < rp[v + 1]; k++)
        if (comp[col[k]] < 0) {
          comp[col[k]] = nc;
          q[t++] = col[k];
        }
    }
    csize[nc] = t;
    nc++;
  }
  for (int64_t v = 0; v < n; v++) lab[v] = -1;
  int32_t stamp = 0;
  for (int64_t p = 0; p < npieces; p++) {
    for (int64_t i = piece_off[p]; i < piece_off[p + 1]; i++) {
      int32_t v = piece_vtx[i];
      stamp++;
      /* multi-source BFS in G - v from every other vertex of the piece */
      int64_t h = 0, t = 0;
      lab[v] = stamp; /* v is removed: never entered */
      for (int64_t j = piece_off[p]; j < piece_off[p + 1]; j++) {
        int32_t x = piece_vtx[j];
        if (lab[x] == stamp) continue;
        lab[x] = stamp;
        q[t++] = x;
      }
      while (h < t) {
        int32_t x = q[h++];
        for (int64_t k = rp[x]; k < rp[x + 1]; k++) {
          int32_t w = col[k];
          if (lab[w] == stamp) continue;
          lab[w] = stamp;
          q[t++] = w;
        }
      }
      reach_out[i] = csize[comp[v]] - t;
    }
  }
  free(lab);
  free(q);
  free(comp);
  free(csize);
  return 0;
}
