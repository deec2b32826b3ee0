// side.cu - compression with side vertices (Section 3.3.2, Algorithm 3)
// over the merged pieces.
//
// A side vertex u has a clique for a neighbourhood, so no shortest path
// passes through it: it is only ever an end point.  The paper removes side
// vertices one at a time; each first runs a Bc-Reach search of its own in
// which every other vertex w receives reach[u] * (2 delta(w) - (reach[w] - 1))
// (the pairs that end at u counted once more, by symmetry), and u itself
// receives (reach[u] - 1) times the total reach left in the piece.
//
// Here a whole set S of side vertices of a piece leaves at once, which gives
// the same sums without an order:
//
// * the side pass: every u in S is a source on the full piece, with every
//   vertex outside S weighted 2 reach as a target (S members count once,
//   the pair being seen from both of its ends) - that is Bc-Reach with
//   reach2[w] = 2 reach[w] for w outside S;
// * the reduced pass: every other vertex is a source on the piece without S
//   (distances and path counts between them do not change: no shortest path
//   passes through S);
// * closed forms: reach2 also raised the delta initialisation of every
//   vertex v outside S by reach[v] in each side search, so v loses
//   reach[v] * SW (SW = sum of reach * ident over S); a side vertex u is a
//   target-side end point of the pairs from every source outside S, each
//   giving reach[u] - 1, so u gains (reach[u] - 1) * NW (NW = sum of
//   reach * ident outside S).
//
// With identical-vertex classes (ident > 1) the test runs on the merged
// graph: the Bc-Reach search of the merged piece never sees pairs inside a
// class (their terms are closed forms of the merge), so a vertex whose
// merged neighbours are pairwise adjacent is never inside a merged shortest
// path.  Side detection tests vertices of degree <= SIDE_MAXDEG only; any
// subset of side vertices gives the same bc.
#include <algorithm>

#include "common.h"

namespace bcs {

namespace {

constexpr int SIDE_MAXDEG = 64;
constexpr int SIDE_BLOCK = 256;

inline int grid_of(int64_t work, int max_blocks) {
  int64_t b = (work + SIDE_BLOCK - 1) / SIDE_BLOCK;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, max_blocks));
}

// the piece holding merged vertex v: the last p with piece_off[p] <= v
__device__ __forceinline__ int64_t piece_of(const int64_t *__restrict__ piece_off, int64_t P, int64_t v) {
  int64_t lo = 0, hi = P - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (piece_off[mid] <= v)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// whether the row col[a..b) of a piece holds the vertex of original id x:
// rows are in ascending original id (local ids put a block's top vertex
// first, so they are not), org[base + local id] = original id.  A row out
// of that order could only hide a side vertex, never invent one.
__device__ __forceinline__ bool row_has(const int32_t *__restrict__ col, const int32_t *__restrict__ org,
                                        int64_t base, int64_t a, int64_t b, int32_t x) {
  while (a < b) {
    const int64_t mid = (a + b) >> 1;
    const int32_t c = org[base + col[mid]];
    if (c == x) return true;
    if (c < x)
      a = mid + 1;
    else
      b = mid;
  }
  return false;
}

// side[v] = 1 if v's merged neighbours are pairwise adjacent (binary
// searches by original id); nside[p]
// counts them per piece; vpiece[v] = v's piece
__global__ void k_side_mark(int64_t M, const int64_t *__restrict__ piece_off, int64_t P,
                            const int64_t *__restrict__ mrow, const int32_t *__restrict__ mcol,
                            const int32_t *__restrict__ morg, int32_t *vpiece, uint8_t *side, int32_t *nside) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = piece_of(piece_off, P, v);
    const int64_t base = piece_off[p];
    const int64_t r0 = mrow[v], r1 = mrow[v + 1];
    bool s = r1 > r0 && r1 - r0 <= SIDE_MAXDEG;
    for (int64_t i = r0; s && i < r1; i++) {
      const int64_t a = base + mcol[i];
      const int64_t a0 = mrow[a], a1 = mrow[a + 1];
      for (int64_t j = i + 1; j < r1; j++)
        if (!row_has(mcol, morg, base, a0, a1, morg[base + mcol[j]])) {
          s = false;
          break;
        }
    }
    vpiece[v] = (int32_t)p;
    side[v] = s;
    if (s) atomicAdd(nside + p, 1);
  }
}

// reach2 (targets outside S doubled in pieces that have side vertices), the
// scan input side[v] + 2^32 red[v] (red: v belongs to a reduced piece), and
// the per-piece sums SW / NW of reach * ident over S and outside it
__global__ void k_side_prep(int64_t M, const int32_t *__restrict__ vpiece, const uint8_t *__restrict__ side,
                            const int32_t *__restrict__ nside, const int32_t *__restrict__ reach,
                            const int32_t *__restrict__ ident, int32_t *reach2, int64_t *flags,
                            unsigned long long *sw, unsigned long long *nw) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = vpiece[v];
    const bool has = nside[p] > 0, sv = side[v] != 0;
    const int32_t r = reach ? reach[v] : 1;
    const int32_t k = ident ? ident[v] : 1;
    reach2[v] = (has && !sv) ? 2 * r : r;
    flags[v] = (int64_t)sv | ((int64_t)(has && !sv) << 32);
    if (has) atomicAdd(sv ? sw + p : nw + p, (unsigned long long)((int64_t)r * k));
  }
}

// low and high halves of the packed scan: side vertices / reduced vertices
// before v
__device__ __forceinline__ int64_t side_before(int64_t x) { return x & 0xffffffffll; }
__device__ __forceinline__ int64_t red_before(int64_t x) { return x >> 32; }

// The side-source map, the reduced pieces' degrees, weights and ids, and
// the closed-form terms.
__global__ void k_side_lists(int64_t M, const int32_t *__restrict__ vpiece, const int64_t *__restrict__ piece_off,
                             const int64_t *__restrict__ mrow, const int32_t *__restrict__ mcol,
                             const uint8_t *__restrict__ side, const int64_t *__restrict__ scan,
                             const int32_t *__restrict__ nside, const int32_t *__restrict__ reach,
                             const int32_t *__restrict__ ident, const unsigned long long *__restrict__ sw,
                             const unsigned long long *__restrict__ nw, int64_t *srcmap, int64_t *rdeg,
                             int32_t *rreach, int32_t *rident, int32_t *rmap, unsigned long long *rnnz, double *bcp) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = vpiece[v];
    if (nside[p] == 0) continue;
    const int64_t base = piece_off[p];
    const int64_t r = reach ? reach[v] : 1;
    if (side[v]) {
      srcmap[base + (side_before(scan[v]) - side_before(scan[base]))] = v - base;
      bcp[v] += (double)((r - 1) * (int64_t)nw[p]);
      continue;
    }
    bcp[v] -= (double)(r * (int64_t)sw[p]);
    const int64_t x = red_before(scan[v]);
    int64_t d = 0;
    for (int64_t i = mrow[v]; i < mrow[v + 1]; i++) d += side[base + mcol[i]] == 0;
    rdeg[x] = d;
    rreach[x] = (int32_t)r;
    if (rident) rident[x] = ident ? ident[v] : 1;
    rmap[x] = (int32_t)v;
    atomicAdd(rnnz + p, (unsigned long long)d);
  }
}

// the reduced CSR: each row keeps its neighbours outside S, renumbered
// inside the reduced piece (ascending order is kept)
__global__ void k_side_fill(int64_t M, const int32_t *__restrict__ vpiece, const int64_t *__restrict__ piece_off,
                            const int64_t *__restrict__ mrow, const int32_t *__restrict__ mcol,
                            const uint8_t *__restrict__ side, const int64_t *__restrict__ flags,
                            const int64_t *__restrict__ scan, const int64_t *__restrict__ rrow, int32_t *rcol) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (int64_t)gridDim.x * blockDim.x) {
    if (red_before(flags[v]) == 0) continue;
    const int64_t base = piece_off[vpiece[v]];
    const int64_t rbase = red_before(scan[base]);
    int64_t pos = rrow[red_before(scan[v])];
    for (int64_t i = mrow[v]; i < mrow[v + 1]; i++) {
      const int64_t w = base + mcol[i];
      if (!side[w]) rcol[pos++] = (int32_t)(red_before(scan[w]) - rbase);
    }
  }
}

__global__ void k_side_scatter(int64_t nred, const int32_t *__restrict__ rmap, const double *__restrict__ bred,
                               double *bcp) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nred; x += (int64_t)gridDim.x * blockDim.x)
    bcp[rmap[x]] += bred[x];
}

}  // namespace

int run_bcreach_side(Ctx &ctx, const DevMerged &m, const std::vector<CompDesc> &comps, const BcInput &in,
                     const BcPlanOpts &po, int64_t n_graph) {
  const int64_t M = m.nmerged, P = m.npieces, E = m.nentries;
  // reach <= n_graph, and the doubled target weights must stay in int32
  if (M == 0 || P == 0 || n_graph >= ((int64_t)1 << 30)) return run_bcreach(ctx, comps, in, po);
  Tracer tr("side", ctx.stream);
  StageTimer tm(ctx.stream);
  tm.start();
  const int maxb = ctx.num_sms * 16;
  const int gm = grid_of(M, maxb);
  // every array sized for the worst case (no piece loses a vertex), so the
  // step needs one host synchronisation, for the descriptors
  DBuf<uint8_t> side;
  DBuf<int32_t> vpiece, nside, reach2, rreach, rident, rmap, rcol;
  DBuf<int64_t> flags, scan, srcmap, rdeg, rrow, totals;
  DBuf<unsigned long long> sums;  // sw[P], nw[P], rnnz[P]
  BCS_TRY(side.alloc(M, ctx.stream));
  BCS_TRY(vpiece.alloc(M, ctx.stream));
  BCS_TRY(nside.alloc(P, ctx.stream));
  BCS_TRY(reach2.alloc(M, ctx.stream));
  BCS_TRY(flags.alloc(M, ctx.stream));
  BCS_TRY(scan.alloc(M, ctx.stream));
  BCS_TRY(srcmap.alloc(M, ctx.stream));
  BCS_TRY(rdeg.alloc(M, ctx.stream));
  BCS_TRY(rrow.alloc(M + 1, ctx.stream));
  BCS_TRY(rreach.alloc(M, ctx.stream));
  if (in.ident) BCS_TRY(rident.alloc(M, ctx.stream));
  BCS_TRY(rmap.alloc(M, ctx.stream));
  BCS_TRY(rcol.alloc(std::max<int64_t>(E, 1), ctx.stream));
  BCS_TRY(totals.alloc(1, ctx.stream));
  BCS_TRY(sums.alloc(3 * P, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(nside.p, 0, P * sizeof(int32_t), ctx.stream));
  BCS_CUDA(cudaMemsetAsync(sums.p, 0, 3 * P * sizeof(unsigned long long), ctx.stream));
  BCS_CUDA(cudaMemsetAsync(rdeg.p, 0, M * sizeof(int64_t), ctx.stream));
  unsigned long long *sw = sums.p, *nw = sums.p + P, *rnnz = sums.p + 2 * P;
  k_side_mark<<<gm, SIDE_BLOCK, 0, ctx.stream>>>(M, m.piece_off.p, P, m.mrow.p, m.mcol.p, m.morg.p, vpiece.p,
                                                 side.p, nside.p);
  k_side_prep<<<gm, SIDE_BLOCK, 0, ctx.stream>>>(M, vpiece.p, side.p, nside.p, in.reach, in.ident, reach2.p,
                                                 flags.p, sw, nw);
  ctx.launches += 2;
  BCS_CUDA(cudaGetLastError());
  BCS_TRY(launch_exclusive_scan(ctx, flags.p, scan.p, M, totals.p));
  k_side_lists<<<gm, SIDE_BLOCK, 0, ctx.stream>>>(M, vpiece.p, m.piece_off.p, m.mrow.p, m.mcol.p, side.p, scan.p,
                                                  nside.p, in.reach, in.ident, sw, nw, srcmap.p, rdeg.p, rreach.p,
                                                  in.ident ? rident.p : nullptr, rmap.p, rnnz, in.bcp);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  BCS_TRY(launch_exclusive_scan(ctx, rdeg.p, rrow.p, M, rrow.p + M));
  k_side_fill<<<gm, SIDE_BLOCK, 0, ctx.stream>>>(M, vpiece.p, m.piece_off.p, m.mrow.p, m.mcol.p, side.p, flags.p,
                                                 scan.p, rrow.p, rcol.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  std::vector<int32_t> h_nside(P);
  std::vector<unsigned long long> h_rnnz(P);
  int64_t h_tot = 0;
  BCS_CUDA(cudaMemcpyAsync(h_nside.data(), nside.p, P * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(h_rnnz.data(), rnnz, P * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(&h_tot, totals.p, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  const int64_t nside_total = h_tot & 0xffffffffll, nred = h_tot >> 32;
  ctx.stats.n_side = nside_total;
  tr.mark("mark+reduce");
  if (nside_total == 0) {
    tm.stop_into(ctx, &ctx.stats.ms_side);
    return run_bcreach(ctx, comps, in, po);
  }
  DBuf<double> bred;
  BCS_TRY(bred.alloc(std::max<int64_t>(nred, 1), ctx.stream));
  BCS_CUDA(cudaMemsetAsync(bred.p, 0, std::max<int64_t>(nred, 1) * sizeof(double), ctx.stream));
  // descriptors: the side pass over every piece (its side vertices as the
  // sources where it has some, else all of its vertices), the reduced pass
  // over the pieces with side vertices
  std::vector<CompDesc> cside(comps), cred;
  int64_t roff = 0;
  for (int64_t p = 0; p < P; p++) {
    const int32_t ns = h_nside[p];
    if (ns == 0) continue;
    cside[p].src_off = comps[p].vtx_off;
    cside[p].nsrc = ns;
    const int32_t nr = comps[p].n - ns;
    if (nr > 0) {
      CompDesc c = comps[p];
      c.vtx_off = roff;
      c.row_off = roff;
      c.n = nr;
      c.nnz = (int64_t)h_rnnz[p];
      c.src_off = -1;
      c.nsrc = -1;
      cred.push_back(c);
    }
    roff += nr;
  }
  tm.stop_into(ctx, &ctx.stats.ms_side);
  BcInput a = in;
  a.reach = reach2.p;
  BcPlanOpts pa = po;
  pa.srcmap = srcmap.p;
  BCS_TRY(run_bcreach(ctx, cside, a, pa));
  const int64_t items = ctx.stats.n_small_items, nlarge = ctx.stats.n_large_sources;
  const double wse = ctx.stats.work_sources_entries, wsv = ctx.stats.work_sources_vertices;
  tr.mark("side pass");
  if (!cred.empty()) {
    BcInput b;
    b.row = rrow.p;
    b.col = rcol.p;
    b.reach = rreach.p;
    b.ident = in.ident ? rident.p : nullptr;
    b.bcp = bred.p;
    BCS_TRY(run_bcreach(ctx, cred, b, po));
    k_side_scatter<<<grid_of(nred, maxb), SIDE_BLOCK, 0, ctx.stream>>>(nred, rmap.p, bred.p, in.bcp);
    ctx.launches++;
    BCS_CUDA(cudaGetLastError());
    ctx.stats.n_small_items += items;
    ctx.stats.n_large_sources += nlarge;
    ctx.stats.work_sources_entries += wse;
    ctx.stats.work_sources_vertices += wsv;
  }
  tr.mark("reduced pass");
  return BCS_OK;
}

}  // namespace bcs
