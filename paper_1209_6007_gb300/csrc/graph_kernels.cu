// graph_kernels.cu - whole-graph kernels: CSR check, connected components,
// degree-1 removal rounds, prefix sums, bc initialisation and map-back.
#include <algorithm>
#include <mutex>

#include "common.h"
#include "coop.cuh"
#include "uf.cuh"

namespace bcs {

static inline int grid_for(int64_t work, int block, int max_blocks) {
  int64_t b = (work + block - 1) / block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

// Pinned 8-byte scratch per host thread for small device->host reads.
// ---------------------------------------------------------------- validate
// Warp per row: bounds, self-loops, strictly ascending rows (no duplicates)
// and symmetry (binary search of u in the row of each neighbour).
// flags: 1 range/offsets, 2 self-loop, 4 unsorted/duplicate, 8 asymmetric.
__global__ void k_validate(int64_t n, int64_t nnz, const int64_t *__restrict__ rp,
                           const int32_t *__restrict__ col, int *flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int f = 0;
  for (int64_t u = warp; u < n; u += nwarps) {
    const int64_t b = rp[u], e = rp[u + 1];
    if (b < 0 || b > e || e > nnz || (u == 0 && b != 0) || (u == n - 1 && e != nnz)) {
      f |= 1;
      continue;
    }
    for (int64_t k = b + lane; k < e; k += 32) {
      const int32_t v = col[k];
      if (v < 0 || v >= n) {
        f |= 1;
        continue;
      }
      if (v == u) f |= 2;
      if (k > b && col[k - 1] >= v) f |= 4;
      int64_t lo = rp[v], hi = rp[v + 1];
      if (lo < 0 || hi > nnz || lo > hi) {
        f |= 1;
        continue;
      }
      const int64_t end = hi;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < (int32_t)u) lo = mid + 1;
        else hi = mid;
      }
      if (lo >= end || col[lo] != (int32_t)u) f |= 8;
    }
  }
  f = __reduce_or_sync(0xffffffffu, f);
  if (lane == 0 && f) atomicOr(flags, f);
}

// flag 16: an edge joins two graphs of a batch (vertex ranges vtx_off)
__global__ void k_validate_batch(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                 const int64_t *__restrict__ vtx_off, int64_t count, int *flags) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = count;  // graph g with vtx_off[g] <= u < vtx_off[g+1]
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (vtx_off[mid] <= u) lo = mid;
      else hi = mid;
    }
    const int64_t a = vtx_off[lo], b = vtx_off[lo + 1];
    for (int64_t k = rp[u]; k < rp[u + 1]; k++)
      if (col[k] < a || col[k] >= b) {
        atomicOr(flags, 16);
        break;
      }
  }
}

int launch_validate_batch(Ctx &ctx, const DevGraph &g, const int64_t *d_vtx_off, int64_t count, int *d_flags) {
  if (g.n == 0) return BCS_OK;
  k_validate_batch<<<grid_for(g.n, 256, ctx.num_sms * 32), 256, 0, ctx.stream>>>(g.n, g.rp, g.col, d_vtx_off, count,
                                                                                  d_flags);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

int launch_validate(Ctx &ctx, const DevGraph &g, int *d_flags) {
  BCS_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(int), ctx.stream));
  if (g.n == 0) return BCS_OK;
  int block = 256;
  int grid = grid_for(g.n * 32, block, ctx.num_sms * 16);
  k_validate<<<grid, block, 0, ctx.stream>>>(g.n, g.nnz, g.rp, g.col, d_flags);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

// ---------------------------------------------------- connected components
__global__ void k_iota(int64_t n, int32_t *p) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    p[v] = (int32_t)v;
}

// Connected components follow Afforest (Sutton, Ben-Nun and Barak, 2018):
// link every vertex to its first R neighbours, compress, find the component
// that holds most of a fixed sample of vertices, then process the remaining
// edges only of vertices outside it (an edge into that component is handled
// from its other end, and edges inside it change nothing).
constexpr int CC_FIRST = 2;
constexpr int CC_SAMPLE = 1024;

__global__ void k_cc_link_first(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                int32_t *parent) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = rp[v], e = min(rp[v + 1], b + CC_FIRST);
    for (int64_t k = b; k < e; k++) uf_unite(parent, (int32_t)v, col[k]);
  }
}

// after the first links: every vertex points at its root, and lab keeps a
// read-only copy (the first-phase component) for the last pass
__global__ void k_cc_compress(int64_t n, int32_t *parent, int32_t *lab) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = uf_find(parent, (int32_t)v);
    parent[v] = r;
    lab[v] = r;
  }
}

// one CTA of CC_SAMPLE threads: the most frequent root of a fixed sample
// (ties to the smallest root)
__global__ void k_cc_sample(int64_t n, const int32_t *__restrict__ parent, int32_t *dominant) {
  __shared__ int32_t roots[CC_SAMPLE];
  __shared__ unsigned long long best;
  const int t = threadIdx.x;
  const int64_t v = (int64_t)(((unsigned long long)t * 2654435761ull) % (unsigned long long)n);
  roots[t] = parent[v];
  if (t == 0) best = ~0ull;
  __syncthreads();
  int c = 0;
  for (int j = 0; j < CC_SAMPLE; j++) c += roots[j] == roots[t];
  // larger count first, then the smaller root
  atomicMin(&best, ((unsigned long long)(CC_SAMPLE - c) << 32) | (unsigned long long)(uint32_t)roots[t]);
  __syncthreads();
  if (t == 0) *dominant = (int32_t)(best & 0xffffffffull);
}

// One vertex per thread; the remaining edges of a vertex with more than 32
// of them are walked by its whole warp instead.  An edge inside one
// first-phase component (same lab) changes nothing and is skipped on two
// independent read-only loads; only edges between components run the
// union-find.
__global__ void k_cc_link_rest(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                               int32_t *parent, const int32_t *__restrict__ lab, const int32_t *__restrict__ dominant) {
  const int lane = threadIdx.x & 31;
  const int32_t c = *dominant;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t u = base + lane;  // warp-uniform trip count: `base` is the same across the warp
    int64_t b = 0, e = 0;
    int32_t lu = c;
    if (u < n) {
      lu = lab[u];
      if (lu != c) {
        b = rp[u] + CC_FIRST;
        e = rp[u + 1];
      }
    }
    const bool wide = e - b > 32;
    if (!wide)
      for (int64_t k = b; k < e; k++) {
        const int32_t v = col[k];
        if (lab[v] != lu) uf_unite(parent, (int32_t)u, v);
      }
    for (unsigned m = __ballot_sync(0xffffffffu, wide); m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      const int64_t wu = __shfl_sync(0xffffffffu, u, src);
      const int32_t wl = __shfl_sync(0xffffffffu, lu, src);
      const int64_t wb = __shfl_sync(0xffffffffu, b, src), we = __shfl_sync(0xffffffffu, e, src);
      for (int64_t k = wb + lane; k < we; k += 32) {
        const int32_t v = col[k];
        if (lab[v] != wl) uf_unite(parent, (int32_t)wu, v);
      }
    }
  }
}

// Roots go to a separate array: the path-halving writes of concurrent finds
// only ever touch `parent`, so a written label is never overwritten.  Lanes
// with the same root add their count once (a giant component would otherwise
// take one atomic per vertex on a single address).
__global__ void k_cc_finish(int64_t n, int32_t *parent, int32_t *label, unsigned long long *cnt) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = uf_find(parent, (int32_t)v);
    label[v] = r;
    const unsigned act = __activemask();
    const unsigned m = __match_any_sync(act, r);
    if ((threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(cnt + r, (unsigned long long)__popc(m));
  }
}

__global__ void k_cc_size(int64_t n, const int32_t *__restrict__ label, const int64_t *__restrict__ cnt,
                          int64_t *N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    N[v] = cnt[label[v]];
}

int launch_cc(Ctx &ctx, const DevGraph &g, int32_t *d_label, int64_t *d_N) {
  if (g.n == 0) return BCS_OK;
  DBuf<int64_t> cnt;
  DBuf<int32_t> parent, lab, dom;
  BCS_TRY(cnt.alloc(g.n, ctx.stream));
  BCS_TRY(parent.alloc(g.n, ctx.stream));
  BCS_TRY(lab.alloc(g.n, ctx.stream));
  BCS_TRY(dom.alloc(1, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(cnt.p, 0, g.n * sizeof(int64_t), ctx.stream));
  int block = 256;
  int gv = grid_for(g.n, block, ctx.num_sms * 32);
  k_iota<<<gv, block, 0, ctx.stream>>>(g.n, parent.p);
  k_cc_link_first<<<gv, block, 0, ctx.stream>>>(g.n, g.rp, g.col, parent.p);
  k_cc_compress<<<gv, block, 0, ctx.stream>>>(g.n, parent.p, lab.p);
  k_cc_sample<<<1, CC_SAMPLE, 0, ctx.stream>>>(g.n, lab.p, dom.p);
  k_cc_link_rest<<<gv, block, 0, ctx.stream>>>(g.n, g.rp, g.col, parent.p, lab.p, dom.p);
  k_cc_finish<<<gv, block, 0, ctx.stream>>>(g.n, parent.p, d_label, (unsigned long long *)cnt.p);
  k_cc_size<<<gv, block, 0, ctx.stream>>>(g.n, d_label, cnt.p, d_N);
  ctx.launches += 7;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

// ------------------------------------------------------ degree-1 removal
// Section 3.3.1.  Leaves are removed in rounds: every vertex of live degree
// 1 at the start of a round is removed in that round, except that of two
// adjacent leaves (a component reduced to one edge) only the larger id is
// removed, into the smaller.  For a removed leaf u with neighbour v,
// r = reach[u] and N = |C| (the sum of reach over C never changes):
//   bc[u] += (r - 1)(N - r),  bc[v] += r (N - r - 1),  reach[v] += r.
// These terms depend only on u's own reach, which no other removal of the
// same round touches, so the leaves of a round are independent.
__device__ __forceinline__ void push_warp_aggregated(int32_t *queue, unsigned long long *count, int32_t v) {
  unsigned mask = __activemask();
  int leader = __ffs(mask) - 1;
  int lane = threadIdx.x & 31;
  int rank = __popc(mask & ((1u << lane) - 1));
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  queue[base + rank] = v;
}

constexpr int PEEL_THREADS = 1024;

// All rounds in one cooperative launch, one grid-wide wait per round.
// cnt[r] is the size of round r's frontier (one counter per round, so no
// counter is reset while another CTA may still read it).  The arrays the
// rounds change (deg, reach, alive, bcpre) are plain pointers: no read of
// them may go through the non-coherent read-only path.  out[0] = rounds run.
__global__ void k_peel_coop(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const int64_t *__restrict__ N, int32_t *deg, int32_t *reach, uint8_t *alive,
                            int64_t *bcpre, int32_t *fa, int32_t *fb, int32_t *stamp, unsigned long long *cnt,
                            int64_t *out, GridBarrier bar) {
  COOP_STRIDE(v, 0, n) {
    const int32_t d = (int32_t)(rp[v + 1] - rp[v]);
    deg[v] = d;
    reach[v] = 1;
    alive[v] = 1;
    bcpre[v] = 0;
    stamp[v] = d == 1 ? 0 : -1;
    if (d == 1) push_warp_aggregated(fa, cnt, (int32_t)v);
  }
  if (!grid_wait(bar)) return;
  int32_t *cur = fa, *nxt = fb;
  int64_t r = 0;
  for (;; r++) {
    const int64_t fcount = (int64_t)*(volatile unsigned long long *)(cnt + r);
    if (fcount == 0) break;
    // Decide and apply in one pass, with the outcome of deciding every
    // removal against the degrees at the start of the round.  A neighbour is
    // live iff its degree word is positive (a lone vertex has no
    // neighbours); stamp[v] is the round whose frontier holds v (each vertex
    // enters a frontier once, when its degree reaches 1), so a live v with
    // stamp r was a leaf when the round began.  A leaf u of this round has
    // one live neighbour v, and only v can change that during the round: if
    // v is a leaf of this round too, the larger id is removed into the
    // smaller, and the smaller sees either v's stamp or no live neighbour
    // left, and stays.  u's reach is final: every other neighbour was
    // removed into it in earlier rounds.
    COOP_STRIDE(i, 0, fcount) {
      const int32_t u = cur[i];
      if (uf_vload(deg + u) != 1) continue;
      int32_t v = -1;
      for (int64_t k = rp[u]; k < rp[u + 1]; k++) {
        if (uf_vload(deg + col[k]) > 0) {
          v = col[k];
          break;
        }
      }
      if (v < 0 || (uf_vload(stamp + v) == (int32_t)r && u < v)) continue;
      const int64_t ru = reach[u];
      const int64_t nc = N[u];
      atomicAdd((unsigned long long *)(bcpre + u), (unsigned long long)((ru - 1) * (nc - ru)));
      atomicAdd((unsigned long long *)(bcpre + v), (unsigned long long)(ru * (nc - ru - 1)));
      atomicAdd(reach + v, (int32_t)ru);
      alive[u] = 0;
      deg[u] = 0;
      if (atomicSub(deg + v, 1) == 2) {
        stamp[v] = (int32_t)(r + 1);
        push_warp_aggregated(nxt, cnt + r + 1, v);
      }
    }
    if (!grid_wait(bar)) return;
    int32_t *t = cur;
    cur = nxt;
    nxt = t;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = r;
}

int run_peel(Ctx &ctx, const DevGraph &g, const int64_t *d_N, uint8_t *d_alive, int32_t *d_reach,
             int64_t *d_bcpre) {
  if (g.n == 0) return BCS_OK;
  DBuf<int32_t> deg, fa, fb, stamp, err;
  DBuf<unsigned long long> cnt;
  DBuf<unsigned int> barw;
  DBuf<int64_t> out;
  BCS_TRY(deg.alloc(g.n, ctx.stream));
  BCS_TRY(fa.alloc(g.n, ctx.stream));
  BCS_TRY(fb.alloc(g.n, ctx.stream));
  BCS_TRY(stamp.alloc(g.n, ctx.stream));
  BCS_TRY(cnt.alloc(g.n + 2, ctx.stream));  // a round removes at least one vertex: at most n rounds
  BCS_TRY(barw.alloc(2, ctx.stream));
  BCS_TRY(err.alloc(1, ctx.stream));
  BCS_TRY(out.alloc(1, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(cnt.p, 0, (g.n + 2) * sizeof(unsigned long long), ctx.stream));
  BCS_CUDA(cudaMemsetAsync(barw.p, 0, 2 * sizeof(unsigned int), ctx.stream));
  BCS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int32_t), ctx.stream));
  BCS_CUDA(cudaMemsetAsync(out.p, 0, sizeof(int64_t), ctx.stream));
  int per_sm = 0;
  BCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel_coop, PEEL_THREADS, 0));
  if (per_sm < 1) {
    set_error("the degree-1 removal kernel cannot be resident");
    return BCS_ECUDA;
  }
  GridBarrier gb{barw.p, barw.p + 1, err.p, (long long)ctx.max_wait};
  int64_t n = g.n;
  const int64_t *rpp = g.rp, *Np = d_N;
  const int32_t *colp = g.col;
  int32_t *degp = deg.p, *reachp = d_reach, *fap = fa.p, *fbp = fb.p, *stp = stamp.p;
  uint8_t *alivep = d_alive;
  int64_t *bcp = d_bcpre, *outp = out.p;
  unsigned long long *cntp = cnt.p;
  void *args[] = {(void *)&n,     (void *)&rpp,   (void *)&colp, (void *)&Np,   (void *)&degp,
                  (void *)&reachp, (void *)&alivep, (void *)&bcp,  (void *)&fap,  (void *)&fbp,
                  (void *)&stp,   (void *)&cntp,  (void *)&outp, (void *)&gb};
  BCS_CUDA(cudaLaunchCooperativeKernel((const void *)k_peel_coop, dim3(ctx.num_sms), dim3(PEEL_THREADS), args, 0,
                                       ctx.stream));
  ctx.launches++;
  int64_t res[2] = {0, 0};
  BCS_CUDA(cudaMemcpyAsync(res, out.p, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx.stream));
  int32_t e = 0;
  BCS_CUDA(cudaMemcpyAsync(&e, err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  if (e & ERR_TIMEOUT) {
    set_error("a grid-wide wait of the degree-1 removal kernel ran out (opts->max_wait)");
    return BCS_ETIMEOUT;
  }
  ctx.stats.peel_rounds = res[0];
  return BCS_OK;
}

// ------------------------------------------------------------ bc helpers
__global__ void k_bc_init(int64_t n, const int64_t *__restrict__ bcpre, double *bc) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    bc[v] = bcpre ? (double)bcpre[v] : 0.0;
}

int launch_bc_init(Ctx &ctx, int64_t n, const int64_t *d_bcpre, double *d_bc) {
  if (n == 0) return BCS_OK;
  k_bc_init<<<grid_for(n, 256, ctx.num_sms * 32), 256, 0, ctx.stream>>>(n, d_bcpre, d_bc);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

// Eq. 5: bc[v] += bc'[v'] for every copy v' of v (a merged vertex stands for
// each of its members, so every pre-merge slot reads its merged vertex).
__global__ void k_mapback(int64_t nslots, const int32_t *__restrict__ slot_org, const int32_t *__restrict__ slot_to_m,
                          const double *__restrict__ bcp, const double *__restrict__ slot_corr, double *bc) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nslots; p += (int64_t)gridDim.x * blockDim.x) {
    double x = bcp[slot_to_m[p]];
    if (slot_corr) x += slot_corr[p];
    if (x != 0.0) atomicAdd(bc + slot_org[p], x);
  }
}

int launch_mapback(Ctx &ctx, int64_t nslots, const int32_t *slot_org, const int32_t *slot_to_m, const double *bcp,
                   double *d_bc, const double *slot_corr) {
  if (nslots == 0) return BCS_OK;
  k_mapback<<<grid_for(nslots, 256, ctx.num_sms * 32), 256, 0, ctx.stream>>>(nslots, slot_org, slot_to_m, bcp,
                                                                             slot_corr, d_bc);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

int launch_fill_i32(Ctx &ctx, int32_t *p, int64_t n, int32_t v) {
  if (n == 0) return BCS_OK;
  k_fill_i32<<<grid_for(n, 256, ctx.num_sms * 32), 256, 0, ctx.stream>>>(p, n, v);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

__global__ void k_fill_i64(int64_t *p, int64_t n, int64_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

int launch_fill_i64(Ctx &ctx, int64_t *p, int64_t n, int64_t v) {
  if (n == 0) return BCS_OK;
  k_fill_i64<<<grid_for(n, 256, ctx.num_sms * 32), 256, 0, ctx.stream>>>(p, n, v);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

__global__ void k_add_f64(double *dst, const double *__restrict__ src, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] += src[i];
}

int launch_add_f64(Ctx &ctx, double *dst, const double *src, int64_t n) {
  if (n == 0) return BCS_OK;
  k_add_f64<<<grid_for(n, 256, ctx.num_sms * 32), 256, 0, ctx.stream>>>(dst, src, n);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

// ------------------------------------------------------------ prefix sum
// Exclusive scan of int64: each block scans SCAN_TILE elements and writes
// its total; the totals are scanned recursively and added back.
constexpr int SCAN_BLOCK = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t x, int64_t *warp_sums, int64_t *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < (SCAN_BLOCK / 32) ? warp_sums[lane] : 0;
    int64_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < (SCAN_BLOCK / 32)) warp_sums[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  int64_t r = inc - x + warp_sums[wid];
  __syncthreads();
  return r;
}

__global__ void k_scan_tiles(const int64_t *__restrict__ in, int64_t *out, int64_t n, int64_t *tile_sums) {
  __shared__ int64_t warp_sums[SCAN_BLOCK / 32];
  __shared__ int64_t total;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; i++) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    s += v[i];
  }
  int64_t off = block_exclusive_scan(s, warp_sums, &total);
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; i++) {
    if (base + i < n) out[base + i] = off;
    off += v[i];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *__restrict__ tile_off) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const int64_t add = tile_off[blockIdx.x];
  for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x)
    if (base + i < n) out[base + i] += add;
}

int launch_exclusive_scan(Ctx &ctx, const int64_t *in, int64_t *out, int64_t n, int64_t *d_total) {
  if (n == 0) {
    BCS_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int64_t), ctx.stream));
    return BCS_OK;
  }
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles > INT32_MAX) {
    set_error("scan too large");
    return BCS_EINVAL;
  }
  DBuf<int64_t> sums, sums_off;
  BCS_TRY(sums.alloc(tiles, ctx.stream));
  BCS_TRY(sums_off.alloc(tiles, ctx.stream));
  k_scan_tiles<<<(unsigned)tiles, SCAN_BLOCK, 0, ctx.stream>>>(in, out, n, sums.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  if (tiles == 1) {
    BCS_CUDA(cudaMemcpyAsync(d_total, sums.p, sizeof(int64_t), cudaMemcpyDeviceToDevice, ctx.stream));
    return BCS_OK;
  }
  BCS_TRY(launch_exclusive_scan(ctx, sums.p, sums_off.p, tiles, d_total));
  k_scan_add<<<(unsigned)tiles, SCAN_BLOCK, 0, ctx.stream>>>(out, n, sums_off.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

}  // namespace bcs
