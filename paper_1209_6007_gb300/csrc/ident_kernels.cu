// ident_kernels.cu - identical-vertex compression (Section 3.3.3) on the
// device, and the compaction that turns pieces into the Bc-Reach input.
//
// Within a piece, vertices u and v are type-I identical when their open
// neighbourhoods are equal and type-II identical when their closed
// neighbourhoods are equal.  By default only vertices of equal reach are
// merged (the paper leaves reach and ident together unspecified; with equal
// reach every member keeps the same dependency initialisation reach - 1 and
// the same source weight, so one representative stands for all of them);
// the `unequal` option keys classes on the neighbourhood alone (below).
//
// Detection (Section 3.4 uses a neighbourhood hash and explicit comparison
// on collision): every slot gets an order-free 64-bit hash of its open
// neighbourhood (sum of a 64-bit mix of the neighbours' original ids) and of
// its closed one; (piece, hash, degree, reach) goes into an open-addressing
// table whose value is the member with the smallest original id; every slot
// then compares its row (ascending original ids) with that candidate's row
// exactly.  A
// fingerprint collision can only make a merge fail, never a wrong merge.
//
// Terms added when a class of K members of reach r is merged into one
// vertex (derived from Eq. 1 with reach; the paper gives the r = 1 case):
//   every member:               (K - 1) r (r - 1)
//   type I, every neighbour:    K (K - 1) r^2 / K_N,  K_N = the degree of a
//                               member (all ordered pairs of members' sides
//                               go through one common neighbour, each one
//                               taking an equal share, as Section 3.3.3
//                               spreads the r = 1 pairs)
//
// With `unequal`, classes are keyed on the neighbourhood alone and members
// may differ in reach r_i (R = sum r_i, Q = sum r_i^2 over the class).  In
// Bc-Reach a member i as a target contributes r_i + X (X the part from
// beyond it, the same for all members), so the merged vertex carries the
// target weight R + K X: that is Bc-Reach with the fractional dependency
// start R / K - 1 (and source weight R).  What differs per member becomes a
// closed form on each copy:
//   member i:                   (r_i - 1)(R - r_i)  [pairs from the other
//                               members' sides into i's own side]
//                               + (r_i - R/K)(N_C - R)  [its own start
//                               against the sources outside the class]
//   type I, every neighbour:    (R^2 - Q) / K_N
// (both reduce to the equal-reach terms when every r_i = r).
#include "common.h"

namespace bcs {

static inline int grid_for(int64_t work, int block, int max_blocks) {
  int64_t b = (work + block - 1) / block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

// MurmurHash3 64-bit finalizer.
__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdULL;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ULL;
  k ^= k >> 33;
  return k;
}

__global__ void k_ident_hash(int64_t nslots, const int64_t *__restrict__ srow, const int32_t *__restrict__ scol,
                             const int32_t *__restrict__ org, const int32_t *__restrict__ reach,
                             const int32_t *__restrict__ piece, uint64_t *fp_open, uint64_t *fp_closed) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nslots; x += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h = 0;
    const int64_t b = srow[x], e = srow[x + 1];
    for (int64_t k = b; k < e; k++) h += fmix64((uint64_t)org[scol[k]] + 1);
    const uint64_t hc = h + fmix64((uint64_t)org[x] + 1);
    const uint64_t tag = fmix64(((uint64_t)(uint32_t)piece[x] << 32) ^ (uint64_t)(e - b)) ^
                         fmix64((uint64_t)(uint32_t)(reach ? reach[x] : 0) * 0x9E3779B97F4A7C15ULL + 7);
    uint64_t fo = fmix64(h ^ tag), fc = fmix64(hc ^ tag ^ 0xD6E8FEB86659FD93ULL);
    fp_open[x] = fo ? fo : 1;
    fp_closed[x] = fc ? fc : 1;
  }
}

// Insert both fingerprints; slot_of[2x+t] = table index of slot x's key.
// The table value keeps the smallest (original id, slot) of its key, so the
// class representative is the member with the smallest original id.
__global__ void k_ident_insert(int64_t nslots, const uint64_t *__restrict__ fp_open,
                               const uint64_t *__restrict__ fp_closed, const int32_t *__restrict__ org,
                               unsigned long long *keys, unsigned long long *vals, uint64_t mask, int64_t *slot_of) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nslots; x += (int64_t)gridDim.x * blockDim.x) {
    for (int t = 0; t < 2; t++) {
      const uint64_t f = t ? fp_closed[x] : fp_open[x];
      uint64_t i = f & mask;
      for (uint64_t probe = 0; probe <= mask; probe++) {
        unsigned long long old = atomicCAS(keys + i, 0ull, (unsigned long long)f);
        if (old == 0ull || old == f) {
          atomicMin(vals + i, ((unsigned long long)(uint32_t)org[x] << 32) | (unsigned long long)(uint32_t)x);
          slot_of[2 * x + t] = (int64_t)i;
          break;
        }
        i = (i + 1) & mask;
      }
    }
  }
}

__device__ bool rows_equal_open(const int64_t *srow, const int32_t *scol, int64_t x, int64_t c) {
  const int64_t bx = srow[x], ex = srow[x + 1], bc = srow[c], ec = srow[c + 1];
  if (ex - bx != ec - bc) return false;
  for (int64_t i = 0; i < ex - bx; i++)
    if (scol[bx + i] != scol[bc + i]) return false;
  return true;
}

// closed rows equal: row(x) + {x} == row(c) + {c}
__device__ bool rows_equal_closed(const int64_t *srow, const int32_t *scol, int64_t x, int64_t c) {
  const int64_t bx = srow[x], ex = srow[x + 1], bc = srow[c], ec = srow[c + 1];
  if (ex - bx != ec - bc) return false;
  int64_t i = bx, j = bc;
  bool x_in_c = false, c_in_x = false;
  while (i < ex || j < ec) {
    int64_t a = i < ex ? scol[i] : INT64_MAX;
    int64_t b = j < ec ? scol[j] : INT64_MAX;
    if (a == c) {
      c_in_x = true;
      i++;
      continue;
    }
    if (b == x) {
      x_in_c = true;
      j++;
      continue;
    }
    if (a != b) return false;
    i++;
    j++;
  }
  return x_in_c && c_in_x;
}

__global__ void k_ident_verify(int64_t nslots, const int64_t *__restrict__ srow, const int32_t *__restrict__ scol,
                               const int32_t *__restrict__ reach, const int32_t *__restrict__ piece,
                               const unsigned long long *__restrict__ vals, const int64_t *__restrict__ slot_of,
                               int32_t *cls, int8_t *typ) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nslots; x += (int64_t)gridDim.x * blockDim.x) {
    int32_t rep = (int32_t)x;
    for (int t = 0; t < 2 && rep == x; t++) {
      const int32_t c = (int32_t)(vals[slot_of[2 * x + t]] & 0xffffffffull);
      if (c == x) continue;
      if (piece[c] != piece[x] || (reach && reach[c] != reach[x])) continue;
      bool ok = t ? rows_equal_closed(srow, scol, x, c) : rows_equal_open(srow, scol, x, c);
      if (ok) {
        rep = c;
        typ[c] = (int8_t)(t + 1);
      }
    }
    cls[x] = rep;
  }
}

__global__ void k_ident_count(int64_t nslots, const int32_t *__restrict__ cls, int32_t *cnt) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nslots; x += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + cls[x], 1);
}

__global__ void k_ident_corr(int64_t nslots, const int64_t *__restrict__ srow, const int32_t *__restrict__ scol,
                             const int32_t *__restrict__ reach, const int32_t *__restrict__ cls,
                             const int32_t *__restrict__ cnt, const int8_t *__restrict__ typ, double *corr) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nslots; c += (int64_t)gridDim.x * blockDim.x) {
    if (cls[c] != c) continue;
    const double K = (double)cnt[c];
    if (K < 2.0) continue;
    const double r = (double)reach[c];
    atomicAdd(corr + c, (K - 1.0) * r * (r - 1.0));
    if (typ[c] == 1) {
      const int64_t b = srow[c], e = srow[c + 1];
      const double amt = K * (K - 1.0) * r * r / (double)(e - b);
      for (int64_t k = b; k < e; k++) {
        const int32_t y = scol[k];
        if (cls[y] == y) atomicAdd(corr + y, amt);
      }
    }
  }
}

// unequal reach: R, Q and K of every class, on its representative.  With
// sub_k (the preprocessing loop's later rounds) a slot is a sub-unit of
// sub_k[x] members of total weight reach[x]; else one member.
__global__ void k_ident_sums(int64_t nslots, const int32_t *__restrict__ cls, const int32_t *__restrict__ reach,
                             const int32_t *__restrict__ sub_k, unsigned long long *rsum, unsigned long long *qsum,
                             unsigned long long *ksum) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nslots; x += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long r = (unsigned long long)reach[x];
    atomicAdd(rsum + cls[x], r);
    atomicAdd(qsum + cls[x], r * r);
    atomicAdd(ksum + cls[x], (unsigned long long)(sub_k ? sub_k[x] : 1));
  }
}

// unequal reach: the neighbour terms (on representatives, as corr) and each
// copy's own terms (slot_corr); N[p] = size of piece p's connected component.
// A slot x of weight T_x standing for k_x members of weight t_x = T_x / k_x
// each, in a class of K members and weight T:
//   each member of x:            (t_x - T/K)(N_C - T) + (t_x - 1)(T - T_x)
//   type I, each member of a neighbour:  (T^2 - sum T_x^2) / K_N,
//                                K_N = the members of the class's neighbours
// (pairs inside a sub-unit were counted when it formed; with one member per
// slot these are the terms above).
__global__ void k_ident_corr_unequal(int64_t nslots, const int64_t *__restrict__ srow,
                                     const int32_t *__restrict__ scol, const int32_t *__restrict__ reach,
                                     const int32_t *__restrict__ sub_k, const int32_t *__restrict__ piece,
                                     const int64_t *__restrict__ N, const int32_t *__restrict__ cls,
                                     const int32_t *__restrict__ cnt, const int8_t *__restrict__ typ,
                                     const unsigned long long *__restrict__ rsum,
                                     const unsigned long long *__restrict__ qsum,
                                     const unsigned long long *__restrict__ ksum, double *corr, double *slot_corr) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nslots; x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cls[x];
    if (cnt[c] < 2) {
      slot_corr[x] = 0.0;
      continue;
    }
    const int64_t R = (int64_t)rsum[c], NC = N[piece[x]];
    const double K = (double)ksum[c], T = (double)R, Tx = (double)reach[x];
    const double tx = Tx / (double)(sub_k ? sub_k[x] : 1);
    slot_corr[x] = (tx - T / K) * (double)(NC - R) + (tx - 1.0) * (T - Tx);
    if (c == x && typ[c] == 1) {
      const int64_t b = srow[c], e = srow[c + 1];
      int64_t KN = e - b;
      if (sub_k) {
        KN = 0;
        for (int64_t k = b; k < e; k++) KN += sub_k[scol[k]];
      }
      const double amt = (double)(R * R - (int64_t)qsum[c]) / (double)KN;
      for (int64_t k = b; k < e; k++) {
        const int32_t y = scol[k];
        if (cls[y] == y) atomicAdd(corr + y, amt);
      }
    }
  }
}

// keep[x] = 1 for class representatives; ndeg[x] = their degree after merging
__global__ void k_merge_degrees(int64_t nslots, const int64_t *__restrict__ srow, const int32_t *__restrict__ scol,
                                const int32_t *__restrict__ cls, int64_t *keep, int64_t *ndeg) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nslots; x += (int64_t)gridDim.x * blockDim.x) {
    const bool k = cls[x] == x;
    int64_t d = 0;
    if (k)
      for (int64_t i = srow[x]; i < srow[x + 1]; i++) {
        const int32_t y = scol[i];
        d += (cls[y] == y && y != x);
      }
    keep[x] = k;
    ndeg[x] = d;
  }
}

__global__ void k_merge_emit(int64_t nslots, const int64_t *__restrict__ srow, const int32_t *__restrict__ scol,
                             const int32_t *__restrict__ cls, const int32_t *__restrict__ piece,
                             const int64_t *__restrict__ piece_off, const int64_t *__restrict__ mslot,
                             const int64_t *__restrict__ mrow_scan, const int32_t *__restrict__ org,
                             const int32_t *__restrict__ reach, const int32_t *__restrict__ cnt,
                             const double *__restrict__ corr, const unsigned long long *__restrict__ rsum,
                             const unsigned long long *__restrict__ ksum, int64_t *mrow, int32_t *mcol,
                             int32_t *morg, int32_t *mreach, int32_t *mident, double *mcorr, double *minit,
                             int32_t *slot_to_m) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nslots; x += (int64_t)gridDim.x * blockDim.x) {
    slot_to_m[x] = (int32_t)mslot[cls[x]];
    if (cls[x] != x) continue;
    const int64_t m = mslot[x];
    const int64_t base = mslot[piece_off[piece[x]]];
    int64_t pos = mrow_scan[x];
    mrow[m] = pos;
    for (int64_t i = srow[x]; i < srow[x + 1]; i++) {
      const int32_t y = scol[i];
      if (cls[y] == y && y != x) mcol[pos++] = (int32_t)(mslot[y] - base);
    }
    morg[m] = org[x];
    mreach[m] = reach[x];
    const int64_t K = ksum ? (int64_t)ksum[x] : (cnt ? cnt[x] : 1);  // members
    mident[m] = (int32_t)K;
    mcorr[m] = corr ? corr[x] : 0.0;
    if (minit) minit[m] = (double)rsum[x] / (double)K - 1.0;
  }
}

__global__ void k_piece_bounds(int64_t npieces, const int64_t *__restrict__ piece_off, const int64_t *__restrict__ mslot,
                               int64_t nmerged, const int64_t *__restrict__ mrow, int64_t *mpiece_off,
                               int64_t *mpiece_row) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= npieces; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = p < npieces ? mslot[piece_off[p]] : nmerged;
    mpiece_off[p] = m;
    mpiece_row[p] = mrow[m];
  }
}

__global__ void k_iota32(int64_t n, int32_t *p) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

int device_merge(Ctx &ctx, DevPieces &pc, bool identical, bool unequal, DevMerged *out, const int32_t *sub_k) {
  unequal = unequal && identical;
  const int64_t P = pc.npieces, S = pc.nslots;
  out->npieces = P;
  out->nslots = S;
  const int64_t *piece_off = pc.piece_off.p, *srow = pc.srow.p;
  const int32_t *scol = pc.scol.p, *spiece = pc.slot_piece.p, *sreach = pc.slot_reach.p;
  out->slot_org.swap(pc.slot_org);
  out->piece_N.swap(pc.piece_N);
  const int block = 256;
  const int gs = grid_for(S, block, ctx.num_sms * 32);
  Tracer tr("merge", ctx.stream);

  DBuf<int32_t> cls, cnt;
  DBuf<int8_t> typ;
  DBuf<double> corr;
  DBuf<unsigned long long> rsum, qsum, ksum;
  BCS_TRY(cls.alloc(S, ctx.stream));
  if (identical && S > 0) {
    DBuf<uint64_t> fo, fc;
    DBuf<unsigned long long> keys, vals;
    DBuf<int64_t> slot_of;
    uint64_t tsize = 1;
    while (tsize < (uint64_t)(4 * S)) tsize <<= 1;
    BCS_TRY(fo.alloc(S, ctx.stream));
    BCS_TRY(fc.alloc(S, ctx.stream));
    BCS_TRY(keys.alloc(tsize, ctx.stream));
    BCS_TRY(vals.alloc(tsize, ctx.stream));
    BCS_TRY(slot_of.alloc(2 * S, ctx.stream));
    BCS_TRY(cnt.alloc(S, ctx.stream));
    BCS_TRY(typ.alloc(S, ctx.stream));
    BCS_TRY(corr.alloc(S, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(keys.p, 0, tsize * sizeof(unsigned long long), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(vals.p, 0xFF, tsize * sizeof(unsigned long long), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(cnt.p, 0, S * sizeof(int32_t), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(typ.p, 0, S * sizeof(int8_t), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(corr.p, 0, S * sizeof(double), ctx.stream));
    const int32_t *key_reach = unequal ? nullptr : sreach;  // reach is part of the class key unless unequal
    k_ident_hash<<<gs, block, 0, ctx.stream>>>(S, srow, scol, out->slot_org.p, key_reach, spiece, fo.p, fc.p);
    k_ident_insert<<<gs, block, 0, ctx.stream>>>(S, fo.p, fc.p, out->slot_org.p, keys.p, vals.p, tsize - 1, slot_of.p);
    k_ident_verify<<<gs, block, 0, ctx.stream>>>(S, srow, scol, key_reach, spiece, vals.p, slot_of.p, cls.p, typ.p);
    k_ident_count<<<gs, block, 0, ctx.stream>>>(S, cls.p, cnt.p);
    ctx.launches += 4;
    if (unequal) {
      BCS_TRY(rsum.alloc(S, ctx.stream));
      BCS_TRY(qsum.alloc(S, ctx.stream));
      BCS_TRY(ksum.alloc(S, ctx.stream));
      BCS_TRY(out->slot_corr.alloc(S, ctx.stream));
      BCS_CUDA(cudaMemsetAsync(rsum.p, 0, S * sizeof(unsigned long long), ctx.stream));
      BCS_CUDA(cudaMemsetAsync(qsum.p, 0, S * sizeof(unsigned long long), ctx.stream));
      BCS_CUDA(cudaMemsetAsync(ksum.p, 0, S * sizeof(unsigned long long), ctx.stream));
      k_ident_sums<<<gs, block, 0, ctx.stream>>>(S, cls.p, sreach, sub_k, rsum.p, qsum.p, ksum.p);
      k_ident_corr_unequal<<<gs, block, 0, ctx.stream>>>(S, srow, scol, sreach, sub_k, spiece, out->piece_N.p, cls.p,
                                                         cnt.p, typ.p, rsum.p, qsum.p, ksum.p, corr.p,
                                                         out->slot_corr.p);
      ctx.launches += 2;
    } else {
      k_ident_corr<<<gs, block, 0, ctx.stream>>>(S, srow, scol, sreach, cls.p, cnt.p, typ.p, corr.p);
      ctx.launches++;
    }
    BCS_CUDA(cudaGetLastError());
  } else if (S > 0) {
    k_iota32<<<gs, block, 0, ctx.stream>>>(S, cls.p);
    ctx.launches++;
  }
  tr.mark("classes");
  // compaction
  DBuf<int64_t> keep, ndeg, mslot, mrow_scan, totals;
  BCS_TRY(keep.alloc(S, ctx.stream));
  BCS_TRY(ndeg.alloc(S, ctx.stream));
  BCS_TRY(mslot.alloc(S + 1, ctx.stream));
  BCS_TRY(mrow_scan.alloc(S + 1, ctx.stream));
  BCS_TRY(totals.alloc(2, ctx.stream));
  if (S > 0) {
    k_merge_degrees<<<gs, block, 0, ctx.stream>>>(S, srow, scol, cls.p, keep.p, ndeg.p);
    ctx.launches++;
  }
  BCS_TRY(launch_exclusive_scan(ctx, keep.p, mslot.p, S, totals.p));
  BCS_TRY(launch_exclusive_scan(ctx, ndeg.p, mrow_scan.p, S, totals.p + 1));
  int64_t h_tot[2] = {0, 0};
  BCS_CUDA(cudaMemcpyAsync(h_tot, totals.p, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  const int64_t M = h_tot[0], ME = h_tot[1];
  tr.mark("sizes");
  out->nmerged = M;
  out->nentries = ME;
  BCS_TRY(out->mrow.alloc(M + 1, ctx.stream));
  BCS_TRY(out->mcol.alloc(ME, ctx.stream));
  BCS_TRY(out->morg.alloc(M, ctx.stream));
  BCS_TRY(out->mreach.alloc(M, ctx.stream));
  BCS_TRY(out->mident.alloc(M, ctx.stream));
  BCS_TRY(out->mcorr.alloc(M, ctx.stream));
  if (unequal) BCS_TRY(out->minit.alloc(M, ctx.stream));
  BCS_TRY(out->slot_to_m.alloc(S, ctx.stream));
  BCS_TRY(out->piece_off.alloc(P + 1, ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(out->mrow.p + M, totals.p + 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, ctx.stream));
  if (S > 0) {
    k_merge_emit<<<gs, block, 0, ctx.stream>>>(S, srow, scol, cls.p, spiece, piece_off, mslot.p, mrow_scan.p,
                                               out->slot_org.p, sreach, identical ? cnt.p : nullptr,
                                               identical ? corr.p : nullptr, unequal ? rsum.p : nullptr,
                                               unequal ? ksum.p : nullptr, out->mrow.p,
                                               out->mcol.p, out->morg.p, out->mreach.p, out->mident.p, out->mcorr.p,
                                               unequal ? out->minit.p : nullptr, out->slot_to_m.p);
    ctx.launches++;
  }
  tr.mark("emit");
  DBuf<int64_t> prow;
  BCS_TRY(prow.alloc(P + 1, ctx.stream));
  k_piece_bounds<<<grid_for(P + 1, block, ctx.num_sms * 8), block, 0, ctx.stream>>>(P, piece_off, mslot.p, M,
                                                                                    out->mrow.p, out->piece_off.p,
                                                                                    prow.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  out->h_piece_off.resize(P + 1);
  std::vector<int64_t> hrow(P + 1);
  BCS_CUDA(cudaMemcpyAsync(out->h_piece_off.data(), out->piece_off.p, (P + 1) * sizeof(int64_t),
                           cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(hrow.data(), prow.p, (P + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx.stream));
  out->h_piece_maxdeg.resize(P);
  if (P)
    BCS_CUDA(cudaMemcpyAsync(out->h_piece_maxdeg.data(), pc.piece_maxdeg.p, P * sizeof(int32_t),
                             cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  tr.mark("tables");
  out->h_piece_ent.resize(P);
  for (int64_t p = 0; p < P; p++) out->h_piece_ent[p] = hrow[p + 1] - hrow[p];
  return BCS_OK;
}

}  // namespace bcs
