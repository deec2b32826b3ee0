// resplit.cu - one more articulation split after identical-vertex merging
// (the preprocessing of Section 3.4 repeated once: merging can leave a
// merged vertex as a cut vertex, Fig. 3).
//
// The merged pieces are taken as a graph of their own (merged vertices,
// global ids) whose vertex v weighs T[v] = reach[v] * ident[v] (a merged
// vertex stands for ident[v] members of reach[v] each; with classes of
// unequal reach, T is the class's reach sum), and split into biconnected
// blocks by the same device code as the input graph.  A copy of v in a
// block then weighs T[v] plus everything beyond v away from that block, as
// for any cut vertex (Eq. 4 with weights).  When v stands for k identical
// members, every path across v goes through exactly one of them, so in the
// block each member carries 1/k of the weight beyond it: the copy keeps
// ident k and its dependency starts at T_copy / k - 1, a fractional start
// the Bc-Reach kernels already take (so does its source weight, T_copy).
// A merged leaf is the two-vertex block case of the same rule.  The blocks'
// bc' are added to the merged vertices, whose own map-back then runs as
// before.
#include <algorithm>
#include <cmath>

#include "common.h"

namespace bcs {

namespace {

constexpr int RS_BLOCK = 256;

inline int rs_grid(int64_t work, int max_blocks) {
  int64_t b = (work + RS_BLOCK - 1) / RS_BLOCK;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, max_blocks));
}

// the piece holding merged vertex v: the last p with piece_off[p] <= v
__device__ __forceinline__ int64_t rs_piece_of(const int64_t *__restrict__ piece_off, int64_t P, int64_t v) {
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

// the merged pieces as one graph: global column ids, per-vertex weight T,
// component size N (the piece's), component label (its first vertex) and
// liveness
__global__ void k_rs_graph(int64_t M, const int64_t *__restrict__ piece_off, int64_t P,
                           const int64_t *__restrict__ piece_N, const int64_t *__restrict__ mrow,
                           const int32_t *__restrict__ mcol, const int32_t *__restrict__ mreach,
                           const int32_t *__restrict__ mident, const double *__restrict__ minit, int32_t *gcol,
                           int32_t *T, int64_t *N, int32_t *label, uint8_t *alive) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = rs_piece_of(piece_off, P, v);
    const int64_t base = piece_off[p];
    for (int64_t e = mrow[v]; e < mrow[v + 1]; e++) gcol[e] = (int32_t)(base + mcol[e]);
    const int32_t k = mident ? mident[v] : 1;
    T[v] = minit ? (int32_t)llrint((minit[v] + 1.0) * (double)k) : mreach[v] * k;
    N[v] = piece_N[p];
    label[v] = (int32_t)base;
    alive[v] = 1;
  }
}

// ident of each new piece vertex (its merged vertex's) and its dependency
// start T_copy / ident - 1
__global__ void k_rs_weights(int64_t M2, const int32_t *__restrict__ morg2, const int32_t *__restrict__ treach,
                             const int32_t *__restrict__ mident, int32_t *ident2, double *init2) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M2; x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = mident ? mident[morg2[x]] : 1;
    ident2[x] = k;
    init2[x] = (double)treach[x] / (double)k - 1.0;
  }
}

}  // namespace

int run_bcreach_resplit(Ctx &ctx, DevMerged &m, const BcInput &in, const BcPlanOpts &po) {
  const int64_t M = m.nmerged, P = m.npieces, E = m.nentries;
  if (M == 0 || P == 0) return BCS_OK;
  Tracer tr("resplit", ctx.stream);
  const int maxb = ctx.num_sms * 16;
  DBuf<int32_t> gcol, T, label;
  DBuf<int64_t> N;
  DBuf<uint8_t> alive;
  BCS_TRY(gcol.alloc(std::max<int64_t>(E, 1), ctx.stream));
  BCS_TRY(T.alloc(M, ctx.stream));
  BCS_TRY(label.alloc(M, ctx.stream));
  BCS_TRY(N.alloc(M, ctx.stream));
  BCS_TRY(alive.alloc(M, ctx.stream));
  k_rs_graph<<<rs_grid(M, maxb), RS_BLOCK, 0, ctx.stream>>>(M, m.piece_off.p, P, m.piece_N.p, m.mrow.p, m.mcol.p,
                                                           m.mreach.p, in.ident ? m.mident.p : nullptr, m.minit.p,
                                                           gcol.p, T.p, N.p, label.p, alive.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  DevGraph g2;
  g2.n = M;
  g2.nnz = E;
  g2.rp = m.mrow.p;
  g2.col = gcol.p;
  DevPieces pc2;
  BCS_TRY(device_pieces(ctx, g2, alive.p, T.p, N.p, label.p, true, &pc2));
  tr.mark("blocks");
  DevMerged m2;
  BCS_TRY(device_merge(ctx, pc2, false, false, &m2));
  tr.mark("compact");
  const int64_t M2 = m2.nmerged, P2 = m2.npieces;
  ctx.stats.n_pieces = P2;
  if (M2 == 0 || P2 == 0) return BCS_OK;
  DBuf<int32_t> ident2;
  DBuf<double> init2;
  BCS_TRY(ident2.alloc(M2, ctx.stream));
  BCS_TRY(init2.alloc(M2, ctx.stream));
  k_rs_weights<<<rs_grid(M2, maxb), RS_BLOCK, 0, ctx.stream>>>(M2, m2.morg.p, m2.mreach.p,
                                                               in.ident ? m.mident.p : nullptr, ident2.p, init2.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  // a new piece lies inside one merged piece: the sum of ident over a
  // vertex's neighbours is bounded as it was there
  int32_t fan = 1;
  for (int32_t d : m.h_piece_maxdeg) fan = std::max(fan, d);
  std::vector<CompDesc> comps2(P2);
  for (int64_t p = 0; p < P2; p++) {
    CompDesc c;
    c.vtx_off = m2.h_piece_off[p];
    c.row_off = m2.h_piece_off[p];
    c.n = (int32_t)(m2.h_piece_off[p + 1] - m2.h_piece_off[p]);
    c.maxdeg = std::max<int32_t>(1, m2.h_piece_maxdeg[p]);
    c.nnz = m2.h_piece_ent[p];
    c.fan = (double)fan;
    comps2[p] = c;
  }
  BcInput b;
  b.row = m2.mrow.p;
  b.col = m2.mcol.p;
  b.reach = m2.mreach.p;
  b.ident = in.ident ? ident2.p : nullptr;
  b.init = init2.p;
  b.bcp = m2.mcorr.p;  // zero: nothing merged in this pass
  BCS_TRY(run_bcreach(ctx, comps2, b, po));
  tr.mark("bcreach");
  // each new piece vertex's bc' onto its merged vertex
  BCS_TRY(launch_mapback(ctx, m2.nslots, m2.slot_org.p, m2.slot_to_m.p, m2.mcorr.p, in.bcp));
  return BCS_OK;
}

}  // namespace bcs
