// order.cu - BFS ordering of the input graph (Section 4.1): vertices close
// in the graph get close ids, so a traversal touches nearby memory.
//
// Every connected component is searched at once, from its smallest vertex
// (the component labels are the smallest ids), level by level in one
// cooperative launch; the queue order, made contiguous per component by a
// stable sort on the label, numbers the vertices: new id i is the old vertex
// perm[i], and inv[perm[i]] = i.  The renumbered CSR keeps every row in
// ascending order (two stable radix sorts: by column, then by row).
#include <algorithm>

#include "common.h"
#include "coop.cuh"
#include "uf.cuh"

namespace bcs {

constexpr int ORDER_THREADS = 1024;
constexpr int ORDER_SUB = 8;  // lanes per frontier row

__device__ __forceinline__ void push_one(int32_t *queue, unsigned long long *count, int64_t base_off, int32_t v) {
  const unsigned mask = __activemask();
  const int leader = __ffs(mask) - 1;
  const int ln = threadIdx.x & 31;
  unsigned long long base = 0;
  if (ln == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  queue[base_off + base + __popc(mask & ((1u << ln) - 1u))] = v;
}

// level 0: the smallest vertex of every component
__global__ void k_order_roots(int64_t n, const int32_t *__restrict__ label, int32_t *level, int32_t *queue,
                              unsigned long long *cnt0) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const bool root = label[v] == (int32_t)v;
    level[v] = root ? 0 : -1;
    if (root) push_one(queue, cnt0, 0, (int32_t)v);
  }
}

// The level-synchronous search; lcount[l] counts level l (one counter per
// level, so one grid-wide wait per level suffices).  out[0] = vertices queued.
__global__ void k_order_bfs(const int64_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t *level,
                            int32_t *queue, unsigned long long *lcount, int64_t *out, GridBarrier bar) {
  const int sl = (int)(threadIdx.x % ORDER_SUB);
  const int64_t sub0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / ORDER_SUB;
  const int64_t nsub = (int64_t)gridDim.x * blockDim.x / ORDER_SUB;
  int64_t lo = 0, hi = (int64_t)*(volatile unsigned long long *)lcount;
  for (int L = 0;; L++) {
    for (int64_t i = lo + sub0; i < hi; i += nsub) {
      const int32_t v = queue[i];
      for (int64_t k = rp[v] + sl; k < rp[v + 1]; k += ORDER_SUB) {
        const int32_t w = col[k];
        if (uf_vload(level + w) < 0 && atomicCAS(level + w, -1, L + 1) < 0) push_one(queue, lcount + L + 1, hi, w);
      }
    }
    if (!grid_wait(bar)) return;
    const int64_t nhi = hi + (int64_t)*(volatile unsigned long long *)(lcount + L + 1);
    if (nhi == hi) break;
    lo = hi;
    hi = nhi;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = hi;
}

__global__ void k_order_keys(int64_t n, const int32_t *__restrict__ queue, const int32_t *__restrict__ label,
                             uint32_t *keys) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = (uint32_t)label[queue[i]];
}

__global__ void k_order_inv(int64_t n, const int32_t *__restrict__ perm, int32_t *inv, int64_t *deg2,
                            const int64_t *__restrict__ rp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = perm[i];
    inv[v] = (int32_t)i;
    deg2[i] = rp[v + 1] - rp[v];
  }
}

// renumbered rows (not yet sorted): keys = new column ids, vals = entry
// positions; rowid[e] = the new row of entry e
__global__ void k_order_fill(int64_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ inv,
                             const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const int64_t *__restrict__ rp2, uint32_t *keys, int32_t *vals, int32_t *rowid) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const int32_t v = perm[i];
    const int64_t b = rp[v], d = rp[v + 1] - b, o = rp2[i];
    for (int64_t k = lane; k < d; k += 32) {
      keys[o + k] = (uint32_t)inv[col[b + k]];
      vals[o + k] = (int32_t)(o + k);
      rowid[o + k] = (int32_t)i;
    }
  }
}

// second pass keys: the row of each entry in column order
__global__ void k_order_rowkeys(int64_t nnz, const int32_t *__restrict__ pos, const int32_t *__restrict__ rowid,
                                uint32_t *keys) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x)
    keys[j] = (uint32_t)rowid[pos[j]];
}

__global__ void k_order_gather_col(int64_t nnz, const int32_t *__restrict__ pos, const uint32_t *__restrict__ colkey,
                                   int32_t *col2) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x)
    col2[j] = (int32_t)colkey[pos[j]];
}

__global__ void k_order_map_back(int64_t n, const int32_t *__restrict__ inv, const double *__restrict__ bc2,
                                 double *bc) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    bc[v] = bc2[inv[v]];
}

static inline int grid_of(int64_t work, int block, int cap) {
  int64_t b = (work + block - 1) / block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

static int bits_for(int64_t n) {
  int b = 1;
  while (b < 32 && ((int64_t)1 << b) < n) b++;
  return b;
}

int bfs_order_graph(Ctx &ctx, const DevGraph &g, DBuf<int64_t> *rp2, DBuf<int32_t> *col2, DBuf<int32_t> *inv) {
  const int64_t n = g.n, nnz = g.nnz;
  const int B = 256;
  const int gv = grid_of(n, B, ctx.num_sms * 32);
  DBuf<int32_t> label, level, queue, perm;
  DBuf<int64_t> N;
  BCS_TRY(label.alloc(n, ctx.stream));
  BCS_TRY(N.alloc(n, ctx.stream));
  BCS_TRY(launch_cc(ctx, g, label.p, N.p));
  BCS_TRY(level.alloc(n, ctx.stream));
  BCS_TRY(queue.alloc(n, ctx.stream));
  DBuf<unsigned long long> lcount;
  BCS_TRY(lcount.alloc(n + 2, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(lcount.p, 0, (n + 2) * sizeof(unsigned long long), ctx.stream));
  k_order_roots<<<gv, B, 0, ctx.stream>>>(n, label.p, level.p, queue.p, lcount.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  {  // the search, one cooperative launch with a bounded wait per level
    int per_sm = 0;
    BCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_order_bfs, ORDER_THREADS, 0));
    if (per_sm < 1) {
      set_error("the ordering kernel cannot be resident");
      return BCS_ECUDA;
    }
    DBuf<int> err;
    DBuf<unsigned int> barw;
    DBuf<int64_t> out;
    BCS_TRY(err.alloc(1, ctx.stream));
    BCS_TRY(barw.alloc(2, ctx.stream));
    BCS_TRY(out.alloc(1, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(barw.p, 0, 2 * sizeof(unsigned int), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(out.p, 0, sizeof(int64_t), ctx.stream));
    GridBarrier gb{barw.p, barw.p + 1, err.p, (long long)ctx.max_wait};
    const int64_t *rpp = g.rp;
    const int32_t *colp = g.col;
    int32_t *levelp = level.p, *queuep = queue.p;
    unsigned long long *lcp = lcount.p;
    int64_t *outp = out.p;
    void *args[] = {(void *)&rpp, (void *)&colp, (void *)&levelp, (void *)&queuep, (void *)&lcp, (void *)&outp,
                    (void *)&gb};
    BCS_CUDA(cudaLaunchCooperativeKernel((const void *)k_order_bfs, dim3(ctx.num_sms), dim3(ORDER_THREADS), args, 0,
                                         ctx.stream));
    ctx.launches++;
    int h_err = 0;
    int64_t queued = 0;
    BCS_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
    BCS_CUDA(cudaMemcpyAsync(&queued, out.p, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx.stream));
    BCS_CUDA(cudaStreamSynchronize(ctx.stream));
    if (h_err & ERR_TIMEOUT) {
      set_error("a grid-wide wait of the ordering kernel ran out (opts->max_wait)");
      return BCS_ETIMEOUT;
    }
    if (queued != n) {
      set_error("BFS ordering reached " + std::to_string(queued) + " of " + std::to_string(n) + " vertices");
      return BCS_ECUDA;
    }
  }
  // contiguous per component, BFS order inside: stable sort by label
  {
    DBuf<uint32_t> keys, tk;
    DBuf<int32_t> tv;
    BCS_TRY(keys.alloc(n, ctx.stream));
    BCS_TRY(tk.alloc(n, ctx.stream));
    BCS_TRY(tv.alloc(n, ctx.stream));
    k_order_keys<<<gv, B, 0, ctx.stream>>>(n, queue.p, label.p, keys.p);
    ctx.launches++;
    BCS_TRY(radix_sort_pairs(ctx, keys.p, queue.p, tk.p, tv.p, n, bits_for(n)));
  }
  perm.swap(queue);
  // the renumbered CSR
  DBuf<int64_t> deg2, tot;
  BCS_TRY(inv->alloc(n, ctx.stream));
  BCS_TRY(deg2.alloc(n + 1, ctx.stream));
  BCS_TRY(tot.alloc(1, ctx.stream));
  BCS_TRY(rp2->alloc(n + 1, ctx.stream));
  k_order_inv<<<gv, B, 0, ctx.stream>>>(n, perm.p, inv->p, deg2.p, g.rp);
  ctx.launches++;
  BCS_CUDA(cudaMemsetAsync(deg2.p + n, 0, sizeof(int64_t), ctx.stream));
  BCS_TRY(launch_exclusive_scan(ctx, deg2.p, rp2->p, n + 1, tot.p));
  BCS_TRY(col2->alloc(nnz, ctx.stream));
  if (nnz > 0) {
    DBuf<uint32_t> keys, tk;
    DBuf<int32_t> pos, tv, rowid;
    BCS_TRY(keys.alloc(nnz, ctx.stream));
    BCS_TRY(tk.alloc(nnz, ctx.stream));
    BCS_TRY(pos.alloc(nnz, ctx.stream));
    BCS_TRY(tv.alloc(nnz, ctx.stream));
    BCS_TRY(rowid.alloc(nnz, ctx.stream));
    k_order_fill<<<grid_of(n * 32, B, ctx.num_sms * 32), B, 0, ctx.stream>>>(n, perm.p, inv->p, g.rp, g.col, rp2->p,
                                                                             keys.p, pos.p, rowid.p);
    ctx.launches++;
    BCS_CUDA(cudaGetLastError());
    DBuf<uint32_t> colkey;  // the unsorted new column ids, by entry position
    BCS_TRY(colkey.alloc(nnz, ctx.stream));
    BCS_CUDA(cudaMemcpyAsync(colkey.p, keys.p, nnz * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx.stream));
    BCS_TRY(radix_sort_pairs(ctx, keys.p, pos.p, tk.p, tv.p, nnz, bits_for(n)));  // by column
    const int ge = grid_of(nnz, B, ctx.num_sms * 32);
    k_order_rowkeys<<<ge, B, 0, ctx.stream>>>(nnz, pos.p, rowid.p, keys.p);
    ctx.launches++;
    BCS_TRY(radix_sort_pairs(ctx, keys.p, pos.p, tk.p, tv.p, nnz, bits_for(n)));  // then by row, stably
    k_order_gather_col<<<ge, B, 0, ctx.stream>>>(nnz, pos.p, colkey.p, col2->p);
    ctx.launches++;
    BCS_CUDA(cudaGetLastError());
  }
  return BCS_OK;
}

// level 0 of a search from one root
__global__ void k_bfs_root(int64_t n, int32_t root, int32_t *level, int32_t *queue, unsigned long long *lcount) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    level[v] = v == root ? 0 : -1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    queue[0] = root;
    lcount[0] = 1ull;
  }
}

int bfs_queue(Ctx &ctx, const int64_t *rp, const int32_t *col, int64_t n, int32_t root, int32_t *queue_out,
              int *depth, int64_t *reached) {
  *depth = 0;
  *reached = n;
  if (n <= 1) {
    if (n == 1) BCS_CUDA(cudaMemcpyAsync(queue_out, &root, sizeof(int32_t), cudaMemcpyHostToDevice, ctx.stream));
    return BCS_OK;
  }
  DBuf<int32_t> level;
  DBuf<unsigned long long> lcount;
  BCS_TRY(level.alloc(n, ctx.stream));
  BCS_TRY(lcount.alloc(n + 2, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(lcount.p, 0, (n + 2) * sizeof(unsigned long long), ctx.stream));
  k_bfs_root<<<grid_of(n, 256, ctx.num_sms * 8), 256, 0, ctx.stream>>>(n, root, level.p, queue_out, lcount.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  int per_sm = 0;
  BCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_order_bfs, ORDER_THREADS, 0));
  if (per_sm < 1) {
    set_error("the ordering kernel cannot be resident");
    return BCS_ECUDA;
  }
  DBuf<int> err;
  DBuf<unsigned int> barw;
  DBuf<int64_t> out;
  BCS_TRY(err.alloc(1, ctx.stream));
  BCS_TRY(barw.alloc(2, ctx.stream));
  BCS_TRY(out.alloc(1, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), ctx.stream));
  BCS_CUDA(cudaMemsetAsync(barw.p, 0, 2 * sizeof(unsigned int), ctx.stream));
  GridBarrier gb{barw.p, barw.p + 1, err.p, (long long)ctx.max_wait};
  int32_t *levelp = level.p, *queuep = queue_out;
  unsigned long long *lcp = lcount.p;
  int64_t *outp = out.p;
  void *args[] = {(void *)&rp, (void *)&col, (void *)&levelp, (void *)&queuep, (void *)&lcp, (void *)&outp,
                  (void *)&gb};
  BCS_CUDA(cudaLaunchCooperativeKernel((const void *)k_order_bfs, dim3(ctx.num_sms), dim3(ORDER_THREADS), args, 0,
                                       ctx.stream));
  ctx.launches++;
  // the deepest level: the last non-empty level counter (the first 4,096 are enough to tell a
  // shallow graph from a deep one)
  const int64_t nl = std::min<int64_t>(n + 2, 4096);
  std::vector<unsigned long long> lc(nl);
  int h_err = 0;
  int64_t queued = 0;
  BCS_CUDA(cudaMemcpyAsync(lc.data(), lcount.p, nl * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(&queued, out.p, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  if (h_err & ERR_TIMEOUT) {
    set_error("a grid-wide wait of the BFS kernel ran out (opts->max_wait)");
    return BCS_ETIMEOUT;
  }
  *reached = queued;
  int d = 0;
  for (int64_t l = 0; l < nl; l++)
    if (lc[l]) d = (int)l;
  *depth = lc[nl - 1] ? (int)n : d;  // past the counters read: deep
  return BCS_OK;
}

// BFS order of every connected component at once (each from its smallest
// vertex), the components kept contiguous: queue_out[0..n), *depth the
// deepest level over all components.
int bfs_queue_components(Ctx &ctx, const DevGraph &g, int32_t *queue_out, int *depth) {
  const int64_t n = g.n;
  *depth = 0;
  if (n == 0) return BCS_OK;
  DBuf<int32_t> label, level;
  DBuf<int64_t> N;
  DBuf<unsigned long long> lcount;
  BCS_TRY(label.alloc(n, ctx.stream));
  BCS_TRY(N.alloc(n, ctx.stream));
  BCS_TRY(launch_cc(ctx, g, label.p, N.p));
  BCS_TRY(level.alloc(n, ctx.stream));
  BCS_TRY(lcount.alloc(n + 2, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(lcount.p, 0, (n + 2) * sizeof(unsigned long long), ctx.stream));
  k_order_roots<<<grid_of(n, 256, ctx.num_sms * 32), 256, 0, ctx.stream>>>(n, label.p, level.p, queue_out, lcount.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  DBuf<int> err;
  DBuf<unsigned int> barw;
  DBuf<int64_t> out;
  BCS_TRY(err.alloc(1, ctx.stream));
  BCS_TRY(barw.alloc(2, ctx.stream));
  BCS_TRY(out.alloc(1, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), ctx.stream));
  BCS_CUDA(cudaMemsetAsync(barw.p, 0, 2 * sizeof(unsigned int), ctx.stream));
  GridBarrier gb{barw.p, barw.p + 1, err.p, (long long)ctx.max_wait};
  const int64_t *rpp = g.rp;
  const int32_t *colp = g.col;
  int32_t *levelp = level.p, *queuep = queue_out;
  unsigned long long *lcp = lcount.p;
  int64_t *outp = out.p;
  void *args[] = {(void *)&rpp, (void *)&colp, (void *)&levelp, (void *)&queuep, (void *)&lcp, (void *)&outp,
                  (void *)&gb};
  BCS_CUDA(cudaLaunchCooperativeKernel((const void *)k_order_bfs, dim3(ctx.num_sms), dim3(ORDER_THREADS), args, 0,
                                       ctx.stream));
  ctx.launches++;
  const int64_t nl = std::min<int64_t>(n + 2, 4096);
  std::vector<unsigned long long> lc(nl);
  int h_err = 0;
  int64_t queued = 0;
  BCS_CUDA(cudaMemcpyAsync(lc.data(), lcount.p, nl * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(&queued, out.p, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  if (h_err & ERR_TIMEOUT) {
    set_error("a grid-wide wait of the BFS kernel ran out (opts->max_wait)");
    return BCS_ETIMEOUT;
  }
  if (queued != n) {
    set_error("BFS ordering reached " + std::to_string(queued) + " of " + std::to_string(n) + " vertices");
    return BCS_ECUDA;
  }
  int d = 0;
  for (int64_t l = 0; l < nl; l++)
    if (lc[l]) d = (int)l;
  *depth = lc[nl - 1] ? (int)n : d;
  // contiguous per component, BFS order inside: stable sort by label
  DBuf<uint32_t> keys, tk;
  DBuf<int32_t> tv;
  BCS_TRY(keys.alloc(n, ctx.stream));
  BCS_TRY(tk.alloc(n, ctx.stream));
  BCS_TRY(tv.alloc(n, ctx.stream));
  k_order_keys<<<grid_of(n, 256, ctx.num_sms * 32), 256, 0, ctx.stream>>>(n, queue_out, label.p, keys.p);
  ctx.launches++;
  BCS_TRY(radix_sort_pairs(ctx, keys.p, queue_out, tk.p, tv.p, n, bits_for(n)));
  return BCS_OK;
}

__global__ void k_order_map_sources(int64_t k, const int64_t *__restrict__ src, const int32_t *__restrict__ inv,
                                    int64_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = inv[src[i]];
}

int map_sources_to_order(Ctx &ctx, const int64_t *src, int64_t k, const int32_t *inv, std::vector<int64_t> *out) {
  out->resize(k);
  if (k == 0) return BCS_OK;
  DBuf<int64_t> d_src, d_out;
  BCS_TRY(d_src.alloc(k, ctx.stream));
  BCS_TRY(d_out.alloc(k, ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(d_src.p, src, k * sizeof(int64_t), cudaMemcpyHostToDevice, ctx.stream));
  k_order_map_sources<<<grid_of(k, 256, ctx.num_sms * 8), 256, 0, ctx.stream>>>(k, d_src.p, inv, d_out.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  BCS_CUDA(cudaMemcpyAsync(out->data(), d_out.p, k * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  return BCS_OK;
}

int launch_order_map_back(Ctx &ctx, int64_t n, const int32_t *inv, const double *bc2, double *bc) {
  if (n == 0) return BCS_OK;
  k_order_map_back<<<grid_of(n, 256, ctx.num_sms * 32), 256, 0, ctx.stream>>>(n, inv, bc2, bc);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

}  // namespace bcs
