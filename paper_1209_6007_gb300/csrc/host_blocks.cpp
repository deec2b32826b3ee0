// host_blocks.cpp - pieces of the graph left by degree-1 removal, built on
// the host: biconnected components with the reach of every copy
// (Sections 3.2.1-3.2.2 and the one-pass decomposition of Section 3.4), or
// plain connected components when articulation shattering is off.
#include <algorithm>
#include <utility>

#include "common.h"

namespace bcs {

namespace {

struct Builder {
  HostPieces *out;
  std::vector<int32_t> mark, loc;
  std::vector<int32_t> verts;
  std::vector<int64_t> deg;
  std::vector<int64_t> fill;

  explicit Builder(int64_t n, HostPieces *o) : out(o), mark(n, -1), loc(n, 0) {
    out->piece_off.assign(1, 0);
    out->srow.assign(1, 0);
  }

  // Append one piece given its edges (pairs of original ids) and a function
  // giving the reach of each of its vertices.
  template <class ReachFn>
  void emit(const std::pair<int32_t, int32_t> *edges, size_t ne, int64_t N, ReachFn reach_of) {
    const int32_t pid = (int32_t)out->npieces();
    verts.clear();
    for (size_t i = 0; i < ne; i++) {
      int32_t a = edges[i].first, b = edges[i].second;
      if (mark[a] != pid) {
        mark[a] = pid;
        verts.push_back(a);
      }
      if (mark[b] != pid) {
        mark[b] = pid;
        verts.push_back(b);
      }
    }
    std::sort(verts.begin(), verts.end());
    const int64_t base = out->nslots();
    const int64_t nv = (int64_t)verts.size();
    for (int64_t i = 0; i < nv; i++) {
      loc[verts[i]] = (int32_t)(base + i);
      out->slot_org.push_back(verts[i]);
      out->slot_reach.push_back(reach_of(verts[i]));
      out->slot_piece.push_back(pid);
    }
    deg.assign(nv, 0);
    for (size_t i = 0; i < ne; i++) {
      deg[loc[edges[i].first] - base]++;
      deg[loc[edges[i].second] - base]++;
    }
    const int64_t e0 = out->srow.back();
    fill.assign(nv, 0);
    for (int64_t i = 0; i < nv; i++) {
      fill[i] = out->srow.back();
      out->srow.push_back(out->srow.back() + deg[i]);
    }
    out->scol.resize(out->srow.back());
    for (size_t i = 0; i < ne; i++) {
      int32_t la = loc[edges[i].first], lb = loc[edges[i].second];
      out->scol[fill[la - base]++] = lb;
      out->scol[fill[lb - base]++] = la;
    }
    for (int64_t i = 0; i < nv; i++)
      std::sort(out->scol.begin() + out->srow[base + i], out->scol.begin() + out->srow[base + i + 1]);
    (void)e0;
    out->piece_off.push_back(out->nslots());
    out->piece_N.push_back(N);
  }
};

}  // namespace

int host_build_pieces(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *alive, const int32_t *reach,
                      const int64_t *ccN, const int32_t *cclab, bool articulation, HostPieces *out) {
  *out = HostPieces();
  Builder B(n, out);
  if (articulation) {
    // Iterative Hopcroft-Tarjan over the live vertices.  A block is emitted
    // when the DFS returns from child u to p with low[u] >= disc[p]; p is
    // then the block's top vertex.  With subR[x] the reach summed over x's
    // DFS subtree and childblk[x] the subR of the children of x that start
    // blocks below x:
    //   top p of the block through child u:  reach = N - subR[u]
    //   any other vertex x of the block:     reach = reach[x] + childblk[x]
    // i.e. everything on the far side of the copy (Eq. 4), so the reach of
    // a block sums to N.
    std::vector<int32_t> disc(n, 0), low(n, 0), parent(n, -1);
    std::vector<int64_t> it(n, 0), subR(n, 0), childblk(n, 0);
    std::vector<std::pair<int32_t, int32_t>> estack;
    std::vector<int32_t> dfs;
    int32_t t = 0;
    for (int64_t r = 0; r < n; r++) {
      if (!alive[r] || disc[r]) continue;
      bool has = false;
      for (int64_t k = rp[r]; k < rp[r + 1] && !has; k++) has = alive[col[k]] != 0;
      if (!has) continue;
      disc[r] = low[r] = ++t;
      parent[r] = -1;
      it[r] = rp[r];
      subR[r] = reach[r];
      dfs.push_back((int32_t)r);
      while (!dfs.empty()) {
        const int32_t u = dfs.back();
        if (it[u] < rp[u + 1]) {
          const int32_t w = col[it[u]++];
          if (!alive[w]) continue;
          if (!disc[w]) {
            estack.emplace_back(u, w);
            parent[w] = u;
            disc[w] = low[w] = ++t;
            it[w] = rp[w];
            subR[w] = reach[w];
            dfs.push_back(w);
          } else if (w != parent[u] && disc[w] < disc[u]) {
            estack.emplace_back(u, w);
            low[u] = std::min(low[u], disc[w]);
          }
        } else {
          dfs.pop_back();
          const int32_t p = parent[u];
          if (p < 0) continue;
          low[p] = std::min(low[p], low[u]);
          subR[p] += subR[u];
          if (low[u] >= disc[p]) {
            childblk[p] += subR[u];
            size_t beg = estack.size();
            while (beg > 0) {
              --beg;
              if (estack[beg].first == p && estack[beg].second == u) break;
            }
            const int64_t top_reach = ccN[p] - subR[u];
            B.emit(estack.data() + beg, estack.size() - beg, ccN[p], [&](int32_t x) -> int32_t {
              return (int32_t)(x == p ? top_reach : reach[x] + childblk[x]);
            });
            estack.resize(beg);
          }
        }
      }
    }
  } else {
    // Connected components of the live graph with at least two vertices
    // (degree-1 removal never disconnects a component).
    std::vector<int64_t> cnt(n, 0);
    for (int64_t v = 0; v < n; v++)
      if (alive[v]) cnt[cclab[v]]++;
    std::vector<std::pair<int32_t, int32_t>> edges;
    std::vector<int64_t> start(n, -1);
    // vertices of each label in ascending order
    std::vector<int64_t> off(n + 1, 0);
    for (int64_t v = 0; v < n; v++) off[v + 1] = off[v] + (cnt[v] >= 2 ? cnt[v] : 0);
    std::vector<int32_t> members(off[n]);
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    for (int64_t v = 0; v < n; v++)
      if (alive[v] && cnt[cclab[v]] >= 2) members[pos[cclab[v]]++] = (int32_t)v;
    for (int64_t l = 0; l < n; l++) {
      if (cnt[l] < 2) continue;
      edges.clear();
      for (int64_t i = off[l]; i < off[l + 1]; i++) {
        int32_t v = members[i];
        for (int64_t k = rp[v]; k < rp[v + 1]; k++)
          if (alive[col[k]] && col[k] > v) edges.emplace_back(v, col[k]);
      }
      B.emit(edges.data(), edges.size(), ccN[members[off[l]]], [&](int32_t x) -> int32_t { return reach[x]; });
    }
  }
  return BCS_OK;
}

}  // namespace bcs
