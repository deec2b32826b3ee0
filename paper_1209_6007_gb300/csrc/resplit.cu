// resplit.cu - the preprocessing of Section 3.4 repeated to a fixpoint:
// merging identical vertices can leave a merged vertex as a cut vertex
// (Fig. 3), and splitting there can make copies identical to other
// vertices of their block, so split and merge alternate until a round
// merges nothing.
//
// A round takes the current pieces as a graph of their own (their
// vertices, global ids) whose vertex v weighs T[v] = reach[v] * ident[v] (a
// merged vertex stands for ident[v] members of reach[v] each; with classes
// of unequal reach, T is the class's reach sum), and splits it into
// biconnected blocks by the same device code as the input graph.  A copy of
// v in a block then weighs T[v] plus everything beyond v away from that
// block, as for any cut vertex (Eq. 4 with weights).  When v stands for k
// identical members, every path across v goes through exactly one of them,
// so in the block each member carries 1/k of the weight beyond it.  The
// blocks' identical vertices are then merged with classes keyed on the
// neighbourhood alone, each copy being a sub-unit of k members of total
// weight T_copy: the class of K members and weight T keeps ident K, its
// dependency starts at T / K - 1 (a fractional start the Bc-Reach kernels
// already take) and its source weight is T; the per-member and neighbour
// terms of a class of sub-units are added in closed form (ident_kernels.cu).
// A merged leaf is the two-vertex block case of the same rule.  Bc-Reach
// runs on the last round's pieces; bc' then goes back one round at a time
// (a copy's value onto the vertex it copies, with its own terms) until it
// reaches the first merge's vertices, whose own map-back runs as before.
// Every round's pieces are a valid Bc-Reach input, so the loop may stop
// early (FIX_MAX_ROUNDS) without changing the result.
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

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

// the members each slot of a round's pieces stands for: its vertex's ident
__global__ void k_rs_subk(int64_t S, const int32_t *__restrict__ slot_org, const int32_t *__restrict__ mident,
                          int32_t *sub_k) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < S; x += (int64_t)gridDim.x * blockDim.x)
    sub_k[x] = mident ? mident[slot_org[x]] : 1;
}

}  // namespace

constexpr int FIX_MAX_ROUNDS = 64;

// One round: split the pieces of `cur` at their cut vertices (weights T)
// and, with `merge`, merge the identical vertices of the blocks.
static int split_and_merge(Ctx &ctx, DevMerged &cur, bool ident, bool merge, DevMerged *next) {
  const int64_t M = cur.nmerged, P = cur.npieces, E = cur.nentries;
  const int maxb = ctx.num_sms * 16;
  DBuf<int32_t> gcol, T, label, sub_k;
  DBuf<int64_t> N;
  DBuf<uint8_t> alive;
  BCS_TRY(gcol.alloc(std::max<int64_t>(E, 1), ctx.stream));
  BCS_TRY(T.alloc(M, ctx.stream));
  BCS_TRY(label.alloc(M, ctx.stream));
  BCS_TRY(N.alloc(M, ctx.stream));
  BCS_TRY(alive.alloc(M, ctx.stream));
  k_rs_graph<<<rs_grid(M, maxb), RS_BLOCK, 0, ctx.stream>>>(M, cur.piece_off.p, P, cur.piece_N.p, cur.mrow.p,
                                                           cur.mcol.p, cur.mreach.p, ident ? cur.mident.p : nullptr,
                                                           cur.minit.p, gcol.p, T.p, N.p, label.p, alive.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  DevGraph g2;
  g2.n = M;
  g2.nnz = E;
  g2.rp = cur.mrow.p;
  g2.col = gcol.p;
  DevPieces pc2;
  BCS_TRY(device_pieces(ctx, g2, alive.p, T.p, N.p, label.p, true, &pc2));
  if (!merge) return device_merge(ctx, pc2, false, false, next);  // every copy keeps reach T_copy
  // classes keyed on the neighbourhood alone; a class of one slot keeps its
  // copy's ident k and dependency start T_copy / k - 1
  const int64_t S2 = pc2.nslots;
  BCS_TRY(sub_k.alloc(std::max<int64_t>(S2, 1), ctx.stream));
  if (S2 > 0) {
    k_rs_subk<<<rs_grid(S2, maxb), RS_BLOCK, 0, ctx.stream>>>(S2, pc2.slot_org.p, ident ? cur.mident.p : nullptr,
                                                             sub_k.p);
    ctx.launches++;
    BCS_CUDA(cudaGetLastError());
  }
  return device_merge(ctx, pc2, true, true, next, sub_k.p);
}

int run_bcreach_resplit(Ctx &ctx, DevMerged &m, const BcInput &in, const BcPlanOpts &po) {
  if (m.nmerged == 0 || m.npieces == 0) return BCS_OK;
  Tracer tr("resplit", ctx.stream);
  const bool ident = in.ident != nullptr;
  // rounds[r]: the pieces after round r + 1 (its slots are copies of the
  // vertices of the round before, or of m)
  std::vector<std::unique_ptr<DevMerged>> rounds;
  DevMerged *cur = &m;
  for (int r = 0; r < FIX_MAX_ROUNDS; r++) {
    rounds.emplace_back(new DevMerged());
    DevMerged *next = rounds.back().get();
    BCS_TRY(split_and_merge(ctx, *cur, ident, ident, next));
    tr.mark("round");
    cur = next;
    // nothing merged: splitting again would give the same blocks
    if (!ident || next->nmerged == next->nslots || next->nmerged == 0) break;
  }
  ctx.stats.n_rounds = (int64_t)rounds.size();
  DevMerged &last = *cur;
  const int64_t P2 = last.npieces;
  ctx.stats.n_pieces = P2;
  if (last.nmerged > 0 && P2 > 0) {
    // a piece lies inside one piece of the first merge: the sum of ident over
    // a vertex's neighbours is bounded by the original degrees, as it was there
    int32_t fan = 1;
    for (int32_t d : m.h_piece_maxdeg) fan = std::max(fan, d);
    std::vector<CompDesc> comps2(P2);
    for (int64_t p = 0; p < P2; p++) {
      CompDesc c;
      c.vtx_off = last.h_piece_off[p];
      c.row_off = last.h_piece_off[p];
      c.n = (int32_t)(last.h_piece_off[p + 1] - last.h_piece_off[p]);
      c.maxdeg = std::max<int32_t>(1, last.h_piece_maxdeg[p]);
      c.nnz = last.h_piece_ent[p];
      c.fan = (double)fan;
      comps2[p] = c;
    }
    BcInput b;
    b.row = last.mrow.p;
    b.col = last.mcol.p;
    b.reach = last.mreach.p;
    b.ident = ident ? last.mident.p : nullptr;
    b.init = last.minit.p;
    b.bcp = last.mcorr.p;  // starts with the last round's neighbour terms
    BCS_TRY(run_bcreach(ctx, comps2, b, po));
    tr.mark("bcreach");
  }
  // bc' back one round at a time: each copy's value (and its own terms) onto
  // the vertex it copies
  for (int64_t r = (int64_t)rounds.size() - 1; r >= 0; r--) {
    DevMerged &x = *rounds[r];
    double *prev = r > 0 ? rounds[r - 1]->mcorr.p : in.bcp;
    if (x.nslots > 0)
      BCS_TRY(launch_mapback(ctx, x.nslots, x.slot_org.p, x.slot_to_m.p, x.mcorr.p, prev, x.slot_corr.p));
  }
  return BCS_OK;
}

}  // namespace bcs
