// blocks_device.cu - the pieces of the graph left by degree-1 removal, built
// on the device: biconnected components with the reach of every copy
// (Sections 3.2.1-3.2.2, all articulation vertices at once as in Section 3.4),
// or connected components when articulation shattering is off.
//
// Biconnected components follow Tarjan and Vishkin's characterisation over
// any rooted spanning tree, here a BFS forest (one tree per component, rooted
// at its live vertex of largest degree, the smallest id among those; every
// vertex takes its smallest-id neighbour of
// the previous level as parent, so the forest is deterministic; the preorder
// numbers depend on the order of atomics, the blocks do not):
//   pre[v]  preorder number, nd[v] subtree size,
//   low[v]/high[v]  min/max of pre over v's subtree and the far ends of the
//                   non-tree edges leaving it.
// Tree edges e(w) = (parent[w], w) are joined (union-find) when
//   (1) a non-tree edge {u, w} exists (in a BFS tree u and w are never
//       ancestor and descendant, so every non-tree edge qualifies), or
//   (2) w's subtree reaches outside its parent v's subtree:
//       low[w] < pre[v] or high[w] >= pre[v] + nd[v]   (v not a root).
// Each class of tree edges is one block; a non-tree edge belongs to the block
// of its endpoints' tree edges.
//
// Copies and reach.  Every block has exactly one vertex that enters it from
// outside, its top t (the parent of its topmost tree edges); every other
// vertex of the block is there through its own tree edge (its home block).
// With subR[x] the reach summed over x's subtree:
//   top copy of block b:   reach = N_C - sum of subR[c] over b's tree edges
//                           hanging directly below t
//   home copy of v:        reach = reach[v] + sum of subR[c] over v's children
//                           c that start other blocks
// i.e. everything on the far side of the copy (Eq. 4); each block's reach
// sums to N_C.
//
// Slots (piece, vertex) are numbered per block: the top copy first, then the
// home copies in ascending vertex id (stable radix sort by block).  Each
// copy's row is the matching subsequence of the input row, so rows stay in
// ascending original id.
#include <cuda/atomic>

#include <algorithm>
#include <cstdio>

#include "bc_math.cuh"
#include "common.h"
#include "coop.cuh"
#include "uf.cuh"

namespace bcs {

static inline int gridv(int64_t work, int block, int max_blocks) {
  int64_t b = (work + block - 1) / block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ void push_aggr(int32_t *queue, unsigned long long *count, int32_t v) {
  unsigned mask = __activemask();
  int leader = __ffs(mask) - 1;
  int lane = threadIdx.x & 31;
  int rank = __popc(mask & ((1u << lane) - 1));
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  queue[base + rank] = v;
}

__global__ void k_iota_i32_dev(int64_t n, int32_t *p) {
  GRID_STRIDE(i, n) { p[i] = (int32_t)i; }
}

// live degree of every live vertex (0 for removed ones)
__global__ void k_alive_deg(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const uint8_t *__restrict__ alive, int32_t *adeg) {
  GRID_STRIDE(v, n) {
    int32_t d = 0;
    if (alive[v])
      for (int64_t k = rp[v]; k < rp[v + 1]; k++) d += alive[col[k]];
    adeg[v] = d;
  }
}

// root of each component's tree: its live vertex of largest live degree,
// the smallest id among those (a hub tends to sit near the middle of the
// graph, so the BFS has fewer levels than from an arbitrary vertex; any root
// is correct).  key = degree * 2^32 + (2^31 - 1 - id), maximised; lanes of
// a warp with the same label combine first: a giant component would
// otherwise send one atomic per vertex to a single address.
__global__ void k_roots(int64_t n, const int32_t *__restrict__ adeg, const int32_t *__restrict__ label,
                        unsigned long long *root_key) {
  GRID_STRIDE(v, n) {
    const int32_t dv = adeg[v];
    if (dv > 0) {
      const int32_t l = label[v];
      const unsigned m = __match_any_sync(__activemask(), l);
      const unsigned dmax = __reduce_max_sync(m, (unsigned)dv);
      const unsigned lo = __reduce_min_sync(m, (unsigned)dv == dmax ? (unsigned)v : 0xffffffffu);
      if ((int)(threadIdx.x & 31) == __ffs(m) - 1)
        atomicMax(root_key + l, ((unsigned long long)dmax << 32) | (unsigned long long)(0x7fffffffu - lo));
    }
  }
}

// level: 0 for the roots, LEVEL_NONE for the other live vertices,
// LEVEL_DEAD for removed ones (so the BFS tests liveness and visits with
// one load)
constexpr int32_t LEVEL_NONE = -1, LEVEL_DEAD = -2;

__global__ void k_bfs_init(int64_t n, const uint8_t *__restrict__ alive, const int32_t *__restrict__ adeg,
                           const int32_t *__restrict__ label, const unsigned long long *__restrict__ root_key,
                           int32_t *level, int32_t *parent, int32_t *order, unsigned long long *tail) {
  GRID_STRIDE(v, n) {
    const bool root =
        adeg[v] > 0 && (int64_t)(0x7fffffffu - (unsigned)(root_key[label[v]] & 0xffffffffull)) == v;
    parent[v] = root ? -1 : INT32_MAX;  // the BFS takes the minimum over the level above
    level[v] = root ? 0 : (alive[v] ? LEVEL_NONE : LEVEL_DEAD);
    if (root) push_aggr(order, tail, (int32_t)v);
  }
}

__device__ __forceinline__ bool is_tree_edge(const int32_t *parent, int32_t u, int32_t w) {
  return parent[w] == u || parent[u] == w;
}

constexpr int FOREST_THREADS = 1024;
constexpr int FOREST_SUB = 8;  // lanes per frontier row in the BFS

__device__ __forceinline__ void stamp(long long *stamps, int k) {
  if (stamps && blockIdx.x == 0 && threadIdx.x == 0) {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    stamps[k] = t;
  }
}

__device__ __forceinline__ int64_t vload64(const int64_t *p) { return *(volatile const int64_t *)p; }

// The whole spanning-forest pass in one cooperative launch.
//  1. BFS levels from the queued roots (one grid-wide wait per level), a
//     frontier vertex's row walked by FOREST_SUB lanes; the parent of w is
//     its smallest-id neighbour on the level above (an atomic minimum over
//     the edges that reach w), and each parent counts its children one
//     level later, once the minimum is final.
//  2. Subtree sizes nd, reach sums subR and sibling offsets off, bottom-up
//     without level waits: every leaf starts a walk towards its root and a
//     vertex is passed on by whichever child completes it last (the
//     completion counter is an acquire-release atomic, so the last arriver
//     sees every sibling's sums).  off[c] is c's place among its siblings,
//     taken with one atomic on the parent's cursor once nd[c] is final, and
//     the parent's size is 1 + its cursor.
//  3. Preorder pre[v] = pre[parent] + 1 + off[v]: each vertex walks up until
//     it meets an ancestor whose number is already published, so no vertex
//     ever waits; subtrees are contiguous ranges [pre, pre + nd).
//  4. low/high: own preorder number and those of non-tree neighbours, then
//     min/max over subtrees with the same last-arriver walk as step 2.
// out[0] = number of levels, out[1] = forest size.  `stamps` (optional)
// receives the global timer at each phase boundary.
__global__ void k_forest_coop(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const uint8_t *__restrict__ alive, const int32_t *__restrict__ reach, int32_t *level,
                              int32_t *parent, int32_t *order, unsigned long long *lcount, int32_t *nchild,
                              int32_t *done, int32_t *off, int32_t *nd, int64_t *subR, int32_t *pre, int32_t *low,
                              int32_t *high, int32_t *out, const unsigned long long *nroots, int32_t *cursor,
                              long long *stamps, GridBarrier bar) {
  // lcount[l] counts the vertices discovered on level l (one counter per
  // level, so reading one level's size never races with the next level's
  // discovery and a single barrier per level suffices)
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  stamp(stamps, 0);
  int64_t lo = 0, hi = (int64_t)*nroots;
  int L = 0;
  const int sl = (int)(threadIdx.x % FOREST_SUB);
  const int64_t sub0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / FOREST_SUB;
  const int64_t nsub = (int64_t)gridDim.x * blockDim.x / FOREST_SUB;
  for (;;) {
    for (int64_t i = lo + sub0; i < hi; i += nsub) {  // discover level L+1
      const int32_t v = order[i];
      if (sl == 0 && L > 0) atomicAdd(nchild + uf_vload(parent + v), 1);  // final since the last wait
      for (int64_t k = rp[v] + sl; k < rp[v + 1]; k += FOREST_SUB) {
        const int32_t w = col[k];
        int32_t lw = uf_vload(level + w);
        if (lw == LEVEL_DEAD) continue;
        if (lw < 0) {
          lw = atomicCAS(level + w, LEVEL_NONE, L + 1);
          if (lw < 0) {
            const unsigned mask = __activemask();
            const int leader = __ffs(mask) - 1;
            const int ln = threadIdx.x & 31;
            unsigned long long base = 0;
            if (ln == leader) base = atomicAdd(lcount + L + 1, (unsigned long long)__popc(mask));
            base = __shfl_sync(mask, base, leader);
            order[hi + base + __popc(mask & ((1u << ln) - 1))] = w;
          }
        }
        if (lw < 0 || lw == L + 1) atomicMin(parent + w, v);
      }
    }
    if (!grid_wait(bar)) return;
    const int64_t nhi = hi + (int64_t)*(volatile unsigned long long *)(lcount + L + 1);
    if (nhi == hi) break;
    lo = hi;
    hi = nhi;
    L++;
  }
  const int nlev = L + 1;
  const int64_t cnt = hi;
  stamp(stamps, 1);
  COOP_STRIDE(i, 0, cnt) {
    const int32_t v = order[i];
    nd[v] = 1;
    subR[v] = reach[v];
    pre[v] = level[v] == 0 ? 0 : -1;
    cursor[v] = 0;
    done[v] = 0;
  }
  if (!grid_wait(bar)) return;
  COOP_STRIDE(i, 0, cnt) {  // subtree sizes, reach sums and sibling offsets
    int32_t v = order[i];
    if (nchild[v] != 0) continue;
    int32_t ndv = 1;  // a leaf
    while (level[v] != 0) {
      const int32_t p = parent[v];
      off[v] = atomicAdd(cursor + p, ndv);
      atomicAdd((unsigned long long *)(subR + p), (unsigned long long)vload64(subR + v));
      // release: this child's sums are visible to whichever child completes p;
      // acquire for that last child: it sees every sibling's
      cuda::atomic_ref<int32_t, cuda::thread_scope_device> dp(done[p]);
      if (dp.fetch_add(1, cuda::memory_order_acq_rel) + 1 != nchild[p]) break;
      ndv = 1 + uf_vload(cursor + p);  // p's subtree: itself and its children's
      nd[p] = ndv;
      v = p;
    }
  }
  if (!grid_wait(bar)) return;
  stamp(stamps, 2);
  COOP_STRIDE(i, 0, cnt) {  // preorder numbers
    const int32_t v = order[i];
    if (level[v] == 0) continue;
    int32_t acc = 0, a = v;
    for (;;) {
      acc += 1 + off[a];
      const int32_t p = parent[a];
      const int32_t pp = uf_vload(pre + p);
      if (pp >= 0) {
        acc += pp;
        break;
      }
      a = p;
    }
    *(volatile int32_t *)(pre + v) = acc;
  }
  if (!grid_wait(bar)) return;
  stamp(stamps, 3);
  COOP_STRIDE(i, 0, cnt) {  // own pre and the far ends of non-tree edges
    const int32_t u = order[i];
    int32_t a = pre[u], b = pre[u];
    for (int64_t k = rp[u]; k < rp[u + 1]; k++) {
      const int32_t w = col[k];
      if (!alive[w] || parent[w] == u || parent[u] == w) continue;
      a = min(a, pre[w]);
      b = max(b, pre[w]);
    }
    low[u] = a;
    high[u] = b;
    done[u] = 0;
  }
  if (!grid_wait(bar)) return;
  COOP_STRIDE(i, 0, cnt) {  // low/high over subtrees
    int32_t v = order[i];
    if (nchild[v] != 0) continue;
    while (level[v] != 0) {
      const int32_t p = parent[v];
      atomicMin(low + p, uf_vload(low + v));
      atomicMax(high + p, uf_vload(high + v));
      cuda::atomic_ref<int32_t, cuda::thread_scope_device> dp(done[p]);
      if (dp.fetch_add(1, cuda::memory_order_acq_rel) + 1 != nchild[p]) break;
      v = p;
    }
  }
  if (!grid_wait(bar)) return;
  stamp(stamps, 4);
  if (lead) {
    out[0] = nlev;
    out[1] = (int32_t)cnt;
  }
}

// union-find over tree edges, identified by their child vertex
__global__ void k_tv_unite(int64_t cnt, const int32_t *__restrict__ order, const int64_t *__restrict__ rp,
                           const int32_t *__restrict__ col, const uint8_t *__restrict__ alive,
                           const int32_t *__restrict__ parent, const int32_t *__restrict__ level,
                           const int32_t *__restrict__ pre, const int32_t *__restrict__ nd,
                           const int32_t *__restrict__ low, const int32_t *__restrict__ high, int32_t *uf) {
  GRID_STRIDE(i, cnt) {
    const int32_t u = order[i];
    if (level[u] == 0) continue;  // roots carry no tree edge
    for (int64_t k = rp[u]; k < rp[u + 1]; k++) {
      const int32_t w = col[k];
      if (w > u && alive[w] && !is_tree_edge(parent, u, w)) uf_unite(uf, u, w);  // rule (1)
    }
    const int32_t v = parent[u];
    if (level[v] > 0 && (low[u] < pre[v] || high[u] >= pre[v] + nd[v])) uf_unite(uf, u, v);  // rule (2)
  }
}

// flag[v] = 1 for the representative tree edge of each block
__global__ void k_tv_finish(int64_t cnt, const int32_t *__restrict__ order, const int32_t *__restrict__ level, int32_t *uf,
                            int32_t *blk, int64_t *flag) {
  GRID_STRIDE(i, cnt) {
    const int32_t v = order[i];
    if (level[v] == 0) continue;
    const int32_t r = uf_find(uf, v);
    blk[v] = r;
    flag[v] = (r == v);
  }
}

// block index of each non-root tree vertex; tops, side sums and block sizes
__global__ void k_blocks_top(int64_t cnt, const int32_t *__restrict__ order, const int32_t *__restrict__ level,
                             const int32_t *__restrict__ parent, const int32_t *__restrict__ blk,
                             const int64_t *__restrict__ bidx, const int64_t *__restrict__ subR, int32_t *bid, int32_t *top,
                             int64_t *side, int64_t *childblk, int64_t *bcnt) {
  GRID_STRIDE(i, cnt) {
    const int32_t c = order[i];
    if (level[c] == 0) continue;
    const int32_t b = (int32_t)bidx[blk[c]];
    bid[c] = b;
    atomicAdd((unsigned long long *)(bcnt + b), 1ull);
    const int32_t p = parent[c];
    const int32_t bp = level[p] > 0 ? (int32_t)bidx[blk[p]] : -1;
    if (bp != b) {
      top[b] = p;
      atomicAdd((unsigned long long *)(side + b), (unsigned long long)subR[c]);
      if (bp >= 0) atomicAdd((unsigned long long *)(childblk + p), (unsigned long long)subR[c]);
    }
  }
}

// connected-component pieces: every live vertex with a live edge has one slot
__global__ void k_cc_pieces(int64_t n, const int32_t *__restrict__ adeg, const int32_t *__restrict__ label,
                            const int64_t *__restrict__ pidx, int32_t *bid, int64_t *bcnt) {
  GRID_STRIDE(v, n) {
    if (adeg[v] == 0) continue;
    const int32_t b = (int32_t)pidx[label[v]];
    bid[v] = b;
    atomicAdd((unsigned long long *)(bcnt + b), 1ull);
  }
}

__global__ void k_flag_label_used(int64_t n, const int32_t *__restrict__ adeg, const int32_t *__restrict__ label,
                                  int64_t *flag) {
  GRID_STRIDE(v, n) {
    if (adeg[v] > 0) flag[label[v]] = 1;
  }
}

// list (key = piece, value = vertex) of the vertices holding a home slot, in
// ascending vertex order
__global__ void k_home_list(int64_t n, const int64_t *__restrict__ hpos, const int64_t *__restrict__ hflag,
                            const int32_t *__restrict__ bid, uint32_t *keys, int32_t *vals) {
  GRID_STRIDE(v, n) {
    if (!hflag[v]) continue;
    keys[hpos[v]] = (uint32_t)bid[v];
    vals[hpos[v]] = (int32_t)v;
  }
}

__global__ void k_home_flags(int64_t n, const int32_t *__restrict__ adeg, const int32_t *__restrict__ level, bool art,
                             int64_t *hflag) {
  GRID_STRIDE(v, n) { hflag[v] = art ? (adeg[v] > 0 && level[v] > 0) : (adeg[v] > 0); }
}

__global__ void k_home_slots(int64_t nh, const uint32_t *__restrict__ keys, const int32_t *__restrict__ vals, int tops,
                             const int32_t *__restrict__ reach, const int64_t *__restrict__ childblk, int32_t *home_slot,
                             int32_t *slot_org, int32_t *slot_reach, int32_t *slot_piece) {
  GRID_STRIDE(i, nh) {
    const int32_t v = vals[i];
    const int32_t b = (int32_t)keys[i];
    const int64_t s = i + (tops ? (int64_t)b + 1 : 0);
    home_slot[v] = (int32_t)s;
    slot_org[s] = v;
    slot_reach[s] = reach[v] + (int32_t)(childblk ? childblk[v] : 0);
    slot_piece[s] = b;
  }
}

__global__ void k_top_slots(int64_t nb, const int64_t *__restrict__ boff, const int32_t *__restrict__ top,
                            const int64_t *__restrict__ side, const int64_t *__restrict__ N, int32_t *top_slot,
                            int32_t *slot_org, int32_t *slot_reach, int32_t *slot_piece, int64_t *piece_N) {
  GRID_STRIDE(b, nb) {
    const int64_t s = boff[b];
    const int32_t t = top[b];
    top_slot[b] = (int32_t)s;
    slot_org[s] = t;
    slot_reach[s] = (int32_t)(N[t] - side[b]);
    slot_piece[s] = (int32_t)b;
    piece_N[b] = N[t];
  }
}

__global__ void k_piece_N_cc(int64_t nh, const int32_t *__restrict__ vals, const uint32_t *__restrict__ keys,
                             const int64_t *__restrict__ N, int64_t *piece_N) {
  GRID_STRIDE(i, nh) { piece_N[keys[i]] = N[vals[i]]; }
}

// block of the edge {v, w} and the slots of both ends in it
__device__ __forceinline__ void edge_slots(bool art, int32_t v, int32_t w, const int32_t *parent, const int32_t *level,
                                           const int32_t *bid, const int32_t *home_slot, const int32_t *top_slot,
                                           int32_t &sv, int32_t &sw) {
  if (!art) {
    sv = home_slot[v];
    sw = home_slot[w];
    return;
  }
  const int32_t hv = level[v] > 0 ? bid[v] : -1;
  const int32_t be = parent[w] == v ? bid[w] : hv;  // tree edge to a child, or v's own block
  sv = be == hv ? home_slot[v] : top_slot[be];
  sw = (level[w] > 0 && bid[w] == be) ? home_slot[w] : top_slot[be];
}

__global__ void k_slot_degrees(int64_t cnt, const int32_t *__restrict__ verts, bool art, const int64_t *__restrict__ rp,
                               const int32_t *__restrict__ col, const uint8_t *__restrict__ alive,
                               const int32_t *__restrict__ parent, const int32_t *__restrict__ level,
                               const int32_t *__restrict__ bid, const int32_t *__restrict__ home_slot,
                               const int32_t *__restrict__ top_slot, int64_t *sdeg) {
  GRID_STRIDE(i, cnt) {
    const int32_t v = verts[i];
    const int32_t hs = home_slot[v];  // most of v's entries go to its home slot: counted in a register
    int64_t nh = 0;
    for (int64_t k = rp[v]; k < rp[v + 1]; k++) {
      const int32_t w = col[k];
      if (!alive[w]) continue;
      int32_t sv, sw;
      edge_slots(art, v, w, parent, level, bid, home_slot, top_slot, sv, sw);
      if (sv == hs) nh++;
      else sdeg[sv]++;  // every slot of v is written only by v's thread
    }
    if (nh > 0) sdeg[hs] += nh;  // nh > 0 implies a home slot
  }
}

__global__ void k_slot_fill(int64_t cnt, const int32_t *__restrict__ verts, bool art, const int64_t *__restrict__ rp,
                            const int32_t *__restrict__ col, const uint8_t *__restrict__ alive,
                            const int32_t *__restrict__ parent, const int32_t *__restrict__ level,
                            const int32_t *__restrict__ bid, const int32_t *__restrict__ home_slot,
                            const int32_t *__restrict__ top_slot, int64_t *cursor, int32_t *scol) {
  GRID_STRIDE(i, cnt) {
    const int32_t v = verts[i];
    const int32_t hs = home_slot[v];
    int64_t hpos = hs >= 0 ? cursor[hs] : 0;  // the home slot's cursor stays in a register
    for (int64_t k = rp[v]; k < rp[v + 1]; k++) {
      const int32_t w = col[k];
      if (!alive[w]) continue;
      int32_t sv, sw;
      edge_slots(art, v, w, parent, level, bid, home_slot, top_slot, sv, sw);
      if (sv == hs) scol[hpos++] = sw;
      else scol[cursor[sv]++] = sw;
    }
  }
}

__global__ void k_piece_maxdeg(int64_t nslots, const int64_t *__restrict__ srow, const int32_t *__restrict__ slot_piece,
                               int32_t *maxdeg) {
  GRID_STRIDE(s, nslots) { atomicMax(maxdeg + slot_piece[s], (int32_t)(srow[s + 1] - srow[s])); }
}

static int read_i64(Ctx &ctx, const int64_t *d, int64_t *h, int count) {
  BCS_CUDA(cudaMemcpyAsync(h, d, count * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  return BCS_OK;
}

int device_pieces(Ctx &ctx, const DevGraph &g, const uint8_t *alive, const int32_t *reach, const int64_t *N,
                  const int32_t *label, bool art, DevPieces *out) {
  const int64_t n = g.n;
  const int B = 256;
  const int gv = gridv(n, B, ctx.num_sms * 32);
  Tracer tr("pieces", ctx.stream);
  DBuf<int32_t> adeg, level, parent, order, bid, home_slot, pre, nd, low, high, uf, blk, top, top_slot;
  DBuf<unsigned long long> root_key;
  DBuf<int64_t> subR, side, childblk, flag, fscan, bcnt, boff, tot, hflag, hpos;
  BCS_TRY(adeg.alloc(n, ctx.stream));
  BCS_TRY(level.alloc(n, ctx.stream));
  BCS_TRY(parent.alloc(n, ctx.stream));
  BCS_TRY(bid.alloc(n, ctx.stream));
  BCS_TRY(home_slot.alloc(n, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(home_slot.p, 0xFF, n * sizeof(int32_t), ctx.stream));  // -1: no home copy (roots)
  BCS_TRY(flag.alloc(n, ctx.stream));
  BCS_TRY(fscan.alloc(n, ctx.stream));
  BCS_TRY(tot.alloc(2, ctx.stream));
  BCS_TRY(hflag.alloc(n, ctx.stream));
  BCS_TRY(hpos.alloc(n, ctx.stream));
  k_alive_deg<<<gv, B, 0, ctx.stream>>>(n, g.rp, g.col, alive, adeg.p);
  ctx.launches++;

  int64_t nb = 0;           // pieces
  int64_t tree_cnt = 0;     // vertices in the forest (art) / with a slot
  std::vector<int64_t> lvl_off;
  if (art) {
    BCS_TRY(root_key.alloc(n, ctx.stream));
    BCS_TRY(order.alloc(n, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(root_key.p, 0, n * sizeof(unsigned long long), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(tot.p, 0, 2 * sizeof(int64_t), ctx.stream));
    k_roots<<<gv, B, 0, ctx.stream>>>(n, adeg.p, label, root_key.p);
    k_bfs_init<<<gv, B, 0, ctx.stream>>>(n, alive, adeg.p, label, root_key.p, level.p, parent.p, order.p,
                                         (unsigned long long *)tot.p);
    ctx.launches += 2;
    BCS_CUDA(cudaGetLastError());
  tr.mark("roots");
    // the spanning forest in one cooperative launch
    BCS_TRY(pre.alloc(n, ctx.stream));
    BCS_TRY(nd.alloc(n, ctx.stream));
    BCS_TRY(subR.alloc(n, ctx.stream));
    BCS_TRY(low.alloc(n, ctx.stream));
    BCS_TRY(high.alloc(n, ctx.stream));
    BCS_TRY(uf.alloc(n, ctx.stream));
    BCS_TRY(blk.alloc(n, ctx.stream));
    DBuf<int32_t> nchild, done, off, fout, ferr;
    DBuf<unsigned int> barw;
    DBuf<unsigned long long> lcount;
    DBuf<long long> stamps;
    BCS_TRY(nchild.alloc(n, ctx.stream));
    BCS_TRY(done.alloc(n, ctx.stream));
    BCS_TRY(off.alloc(n, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(nchild.p, 0, n * sizeof(int32_t), ctx.stream));
    BCS_TRY(lcount.alloc(n + 2, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(lcount.p, 0, (n + 2) * sizeof(unsigned long long), ctx.stream));
    BCS_TRY(fout.alloc(2, ctx.stream));
    BCS_TRY(ferr.alloc(1, ctx.stream));
    BCS_TRY(barw.alloc(2, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(barw.p, 0, 2 * sizeof(unsigned int), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(ferr.p, 0, sizeof(int32_t), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(fout.p, 0, 2 * sizeof(int32_t), ctx.stream));
    if (tr.on) {
      BCS_TRY(stamps.alloc(5, ctx.stream));
      BCS_CUDA(cudaMemsetAsync(stamps.p, 0, 5 * sizeof(long long), ctx.stream));
    }
    // one CTA of FOREST_THREADS per SM: few arrivals per grid-wide wait
    int per_sm = 0;
    BCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forest_coop, FOREST_THREADS, 0));
    if (per_sm < 1) {
      set_error("the spanning-forest kernel cannot be resident");
      return BCS_ECUDA;
    }
    const int coop_grid = ctx.num_sms;
    GridBarrier gb{barw.p, barw.p + 1, ferr.p, (long long)ctx.max_wait};
    unsigned long long *lcountp = lcount.p;
    const unsigned long long *nrootsp = (const unsigned long long *)tot.p;
    DBuf<int32_t> cursor;
    BCS_TRY(cursor.alloc(n, ctx.stream));
    int32_t *cursorp = cursor.p, *nchildp = nchild.p, *donep = done.p, *offp = off.p;
    int32_t *ndp = nd.p, *prep = pre.p, *lowp = low.p, *highp = high.p, *foutp = fout.p;
    int64_t *subRp = subR.p;
    int32_t *levelp = level.p, *parentp = parent.p, *orderp = order.p;
    long long *stampsp = stamps.p;
    const int64_t *rpp = g.rp;
    const int32_t *colp = g.col;
    const uint8_t *alivep = alive;
    const int32_t *reachp = reach;
    void *args[] = {(void *)&rpp,     (void *)&colp,   (void *)&alivep, (void *)&reachp,  (void *)&levelp,
                    (void *)&parentp, (void *)&orderp, (void *)&lcountp, (void *)&nchildp, (void *)&donep,
                    (void *)&offp,    (void *)&ndp,    (void *)&subRp,  (void *)&prep,    (void *)&lowp,
                    (void *)&highp,   (void *)&foutp,  (void *)&nrootsp, (void *)&cursorp, (void *)&stampsp,
                    (void *)&gb};
    BCS_CUDA(cudaLaunchCooperativeKernel((const void *)k_forest_coop, dim3(coop_grid), dim3(FOREST_THREADS), args, 0,
                                         ctx.stream));
    ctx.launches++;
    int32_t hres[3] = {0, 0, 0};
    BCS_CUDA(cudaMemcpyAsync(hres, fout.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx.stream));
    BCS_CUDA(cudaMemcpyAsync(hres + 2, ferr.p, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx.stream));
    BCS_CUDA(cudaStreamSynchronize(ctx.stream));
    if (hres[2] & ERR_TIMEOUT) {
      set_error("a grid-wide wait of the spanning-forest kernel ran out (opts->max_wait)");
      return BCS_ETIMEOUT;
    }
    if (tr.on) {
      long long ts[5];
      BCS_CUDA(cudaMemcpy(ts, stamps.p, sizeof(ts), cudaMemcpyDeviceToHost));
      std::fprintf(stderr, "[bcs trace] forest phases: bfs %.3f sizes %.3f preorder %.3f lowhigh %.3f ms\n",
                   (ts[1] - ts[0]) * 1e-6, (ts[2] - ts[1]) * 1e-6, (ts[3] - ts[2]) * 1e-6, (ts[4] - ts[3]) * 1e-6);
    }
    const int nlev_h = hres[0];
    tree_cnt = hres[1];
    lvl_off.assign(1, (int64_t)nlev_h);  // only the level count is kept on the host
    const int gt = gridv(tree_cnt, B, ctx.num_sms * 32);
  tr.mark("forest");
    // union-find over tree edges
    k_iota_i32_dev<<<gv, B, 0, ctx.stream>>>(n, uf.p);
    BCS_CUDA(cudaMemsetAsync(flag.p, 0, n * sizeof(int64_t), ctx.stream));
    k_tv_unite<<<gt, B, 0, ctx.stream>>>(tree_cnt, order.p, g.rp, g.col, alive, parent.p, level.p, pre.p, nd.p, low.p,
                                        high.p, uf.p);
    k_tv_finish<<<gt, B, 0, ctx.stream>>>(tree_cnt, order.p, level.p, uf.p, blk.p, flag.p);
    ctx.launches += 3;
    BCS_CUDA(cudaGetLastError());
  tr.mark("unite");
    BCS_TRY(launch_exclusive_scan(ctx, flag.p, fscan.p, n, tot.p));
    BCS_TRY(read_i64(ctx, tot.p, &nb, 1));
    BCS_TRY(top.alloc(nb, ctx.stream));
    BCS_TRY(side.alloc(nb, ctx.stream));
    BCS_TRY(bcnt.alloc(nb, ctx.stream));
    BCS_TRY(childblk.alloc(n, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(side.p, 0, nb * sizeof(int64_t), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(childblk.p, 0, n * sizeof(int64_t), ctx.stream));
    BCS_TRY(launch_fill_i64(ctx, bcnt.p, nb, 1));  // the top copy
    k_blocks_top<<<gt, B, 0, ctx.stream>>>(tree_cnt, order.p, level.p, parent.p, blk.p, fscan.p, subR.p, bid.p, top.p,
                                          side.p, childblk.p, bcnt.p);
    ctx.launches++;
    BCS_CUDA(cudaGetLastError());
  } else {
    // pieces = connected components (of the live graph) with a live edge
    BCS_CUDA(cudaMemsetAsync(flag.p, 0, n * sizeof(int64_t), ctx.stream));
    k_flag_label_used<<<gv, B, 0, ctx.stream>>>(n, adeg.p, label, flag.p);
    ctx.launches++;
    BCS_TRY(launch_exclusive_scan(ctx, flag.p, fscan.p, n, tot.p));
    BCS_TRY(read_i64(ctx, tot.p, &nb, 1));
    BCS_TRY(bcnt.alloc(nb, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(bcnt.p, 0, nb * sizeof(int64_t), ctx.stream));
    k_cc_pieces<<<gv, B, 0, ctx.stream>>>(n, adeg.p, label, fscan.p, bid.p, bcnt.p);
    ctx.launches++;
    BCS_CUDA(cudaGetLastError());
  }
  tr.mark("blocks");
  // slots: offsets per piece, then the home copies sorted by (piece, vertex)
  BCS_TRY(out->piece_off.alloc(nb + 1, ctx.stream));
  BCS_TRY(launch_exclusive_scan(ctx, bcnt.p, out->piece_off.p, nb, tot.p));
  BCS_CUDA(cudaMemcpyAsync(out->piece_off.p + nb, tot.p, sizeof(int64_t), cudaMemcpyDeviceToDevice, ctx.stream));
  k_home_flags<<<gv, B, 0, ctx.stream>>>(n, adeg.p, level.p, art, hflag.p);
  ctx.launches++;
  BCS_TRY(launch_exclusive_scan(ctx, hflag.p, hpos.p, n, tot.p + 1));
  int64_t h2[2];
  BCS_TRY(read_i64(ctx, tot.p, h2, 2));
  const int64_t S = h2[0], H = h2[1];
  out->npieces = nb;
  out->nslots = S;
  DBuf<uint32_t> keys, tkeys;
  DBuf<int32_t> vals, tvals;
  BCS_TRY(keys.alloc(H, ctx.stream));
  BCS_TRY(vals.alloc(H, ctx.stream));
  BCS_TRY(tkeys.alloc(H, ctx.stream));
  BCS_TRY(tvals.alloc(H, ctx.stream));
  k_home_list<<<gv, B, 0, ctx.stream>>>(n, hpos.p, hflag.p, bid.p, keys.p, vals.p);
  ctx.launches++;
  int bits = 1;
  while (bits < 32 && ((int64_t)1 << bits) < nb) bits++;
  tr.mark("list");
  BCS_TRY(radix_sort_pairs(ctx, keys.p, vals.p, tkeys.p, tvals.p, H, bits));
  tr.mark("sort");
  BCS_TRY(out->slot_org.alloc(S, ctx.stream));
  BCS_TRY(out->slot_reach.alloc(S, ctx.stream));
  BCS_TRY(out->slot_piece.alloc(S, ctx.stream));
  BCS_TRY(out->piece_N.alloc(nb, ctx.stream));
  k_home_slots<<<gridv(H, B, ctx.num_sms * 32), B, 0, ctx.stream>>>(H, keys.p, vals.p, art ? 1 : 0, reach,
                                                                    art ? childblk.p : nullptr, home_slot.p,
                                                                    out->slot_org.p, out->slot_reach.p,
                                                                    out->slot_piece.p);
  ctx.launches++;
  if (art) {
    BCS_TRY(top_slot.alloc(nb, ctx.stream));
    k_top_slots<<<gridv(nb, B, ctx.num_sms * 32), B, 0, ctx.stream>>>(nb, out->piece_off.p, top.p, side.p, N,
                                                                      top_slot.p, out->slot_org.p, out->slot_reach.p,
                                                                      out->slot_piece.p, out->piece_N.p);
  } else {
    k_piece_N_cc<<<gridv(H, B, ctx.num_sms * 32), B, 0, ctx.stream>>>(H, vals.p, keys.p, N, out->piece_N.p);
  }
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  tr.mark("slots");
  // rows: each vertex's thread walks its input row once per pass
  const int32_t *verts = art ? order.p : vals.p;
  const int64_t nverts = art ? tree_cnt : H;
  const int gw = gridv(nverts, B, ctx.num_sms * 32);
  DBuf<int64_t> sdeg, cursor;
  BCS_TRY(sdeg.alloc(S + 1, ctx.stream));
  BCS_TRY(cursor.alloc(S + 1, ctx.stream));
  BCS_TRY(out->srow.alloc(S + 1, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(sdeg.p, 0, (S + 1) * sizeof(int64_t), ctx.stream));
  k_slot_degrees<<<gw, B, 0, ctx.stream>>>(nverts, verts, art, g.rp, g.col, alive, parent.p, level.p, bid.p,
                                           home_slot.p, art ? top_slot.p : nullptr, sdeg.p);
  ctx.launches++;
  BCS_TRY(launch_exclusive_scan(ctx, sdeg.p, out->srow.p, S + 1, tot.p));
  BCS_CUDA(cudaMemcpyAsync(cursor.p, out->srow.p, (S + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, ctx.stream));
  int64_t E = 0;
  BCS_TRY(read_i64(ctx, tot.p, &E, 1));
  out->nentries = E;
  BCS_TRY(out->scol.alloc(E, ctx.stream));
  k_slot_fill<<<gw, B, 0, ctx.stream>>>(nverts, verts, art, g.rp, g.col, alive, parent.p, level.p, bid.p, home_slot.p,
                                        art ? top_slot.p : nullptr, cursor.p, out->scol.p);
  ctx.launches++;
  tr.mark("rows");
  BCS_TRY(out->piece_maxdeg.alloc(nb, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(out->piece_maxdeg.p, 0, nb * sizeof(int32_t), ctx.stream));
  k_piece_maxdeg<<<gridv(S, B, ctx.num_sms * 32), B, 0, ctx.stream>>>(S, out->srow.p, out->slot_piece.p,
                                                                      out->piece_maxdeg.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  tr.mark("maxdeg");
  ctx.stats.bfs_levels = art ? lvl_off[0] : 0;
  ctx.stats.n_slots = S;
  return BCS_OK;
}

}  // namespace bcs
