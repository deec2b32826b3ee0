// wide.cu - Bc-Reach (Algorithm 2 with the identical-vertex terms of
// Section 3.3.3) on one large piece of small BFS depth, with every SM of the
// GPU working on one batch of 32 sources at a time.
//
// Why the whole GPU on one batch: on a small-world piece (hundreds of
// thousands of vertices, a handful of BFS levels) the per-vertex records of a
// batch stay in L2 only while few batches are in flight; one batch per GPU
// keeps them there, and the BFS levels are few enough that one grid-wide
// wait per level costs little.
//
// Sources: 32 per batch, lane i of every warp stands for the batch's source
// i.  Consecutive vertices of a BFS order of the piece form a batch: they sit
// close together, so a vertex is reached by most of the batch's sources at
// the same level or one apart, and each visit of its row serves many lanes.
//
// Per vertex v, for the batch:
//   lv[v]      2 bits per source: 0 = not reached, else (BFS level mod 3) + 1.
//              Neighbours are at most one level apart, so levels L-1, L, L+1
//              of a neighbour are told apart by the level mod 3;
//   nxt[k][v]  sources that reach v at a level L with L mod 3 = k (built by
//              atomicOr during the previous level's pass);
//   sig[v][s]  path count of source s (exact int64 while the level's counts
//              times the piece's fan-out stay below 2^62, else FP64 scaled
//              by a power of two per (level, source)); in phase 2 it is
//              overwritten by the coefficient c = ident (1 + delta) / sigma
//              (FP64, or FP32 mantissa and exponent in the FP32-delta mode).
// A vertex has one queue entry per level at which some source reaches it;
// the entry's mask holds those sources.  An entry is split into work items of
// at most WIDE_CH row entries (a warp each); the items of a split (hub) entry
// add their partial sums into a per-entry accumulator and the last of them
// finishes the entry.
//
// Phase 1, level L (one pass, one grid-wide wait): each item of an entry
// (w, f) walks its part of w's row, 32 entries per step (one per lane):
//   * path counts (Algorithm 1): sigma[w][s] = sum over neighbours u on level
//     L-1 for s (s in f) of sigma[u][s] * (u the source ? 1 : ident[u]);
//   * discovery: sources in f that have not reached u mark u at level L+1;
//     the first to mark it queues u (warp-aggregated, ballot + scan).
// Phase 2, levels deepest first (one pass each): delta of Eq. 3 in the
// coefficient form, delta[v] = reach[v] - 1 + sigma[v] * sum over successors
// w of c[w]; bc'[v] += reach[s] * ident[s] * delta[v] for v != s, summed over
// the entry's sources in the warp and added once per entry.
#include <algorithm>
#include <cfloat>
#include <cstring>

#include "bc_math.cuh"
#include "common.h"
#include "coop.cuh"

namespace bcs {

constexpr int WIDE_THREADS = 256;
constexpr int WIDE_CH = 256;      // row entries per work item (longer rows are split)
constexpr int WIDE_LCAP = 1024;   // BFS levels one batch may index
constexpr int ERR_CAP = 8;        // a queue, item or accumulator array ran out (never with the sizes below)

struct WideScratch {
  uint64_t *lv;              // [n]
  uint32_t *nxt;             // [3][n]
  double *sig;               // [n][32]
  int32_t *queue;            // [qcap] vertex of each entry
  uint32_t *qmask;           // [qcap] sources of each entry
  int32_t *qhub;             // [qcap] accumulator slot of a split entry, else -1
  int32_t *qdone;            // [qcap] finished items of a split entry
  unsigned long long *items; // [icap] entry index << 32 | first row entry of the item
  double *hacc;              // [hcap][32] accumulators of split entries
  unsigned long long *cnt;   // [WIDE_LCAP + 2] entries per level
  unsigned long long *icnt;  // [WIDE_LCAP + 2] items per level
  unsigned long long *hubs;  // [1] accumulator slots handed out in the batch
  int64_t *qoff, *ioff;      // [WIDE_LCAP + 2] first entry / item of each level
  unsigned long long *lmax;  // [WIDE_LCAP][32] largest stored count per (level, source), as bits
  int32_t *lexp;             // [WIDE_LCAP][32] power-of-two exponent of each level's stored counts
  int32_t *lkind;            // [WIDE_LCAP] 1: the level's counts are int64
  int64_t n, qcap, icap, hcap;
};

// sources whose 2-bit field equals c (c in 1..3)
__device__ __forceinline__ uint32_t lanes_with_code(uint64_t w, uint32_t c) {
  const uint64_t x = w ^ (0x5555555555555555ull * (uint64_t)c);
  return compact2(~(x | (x >> 1)));
}

// sources that have reached the vertex (non-zero field)
__device__ __forceinline__ uint32_t lanes_reached(uint64_t w) { return compact2(w | (w >> 1)); }

__device__ __forceinline__ uint32_t level_code(int L) { return (uint32_t)(L % 3) + 1u; }

__device__ __forceinline__ int warp_max_i(int x) {
  for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  return x;
}

// float -> double from the bit pattern (integer instructions only; the
// hardware conversion issues on the FP64 pipe).  Finite inputs.
__device__ __forceinline__ double f32_to_f64_bits(float x) {
  const unsigned int b = __float_as_uint(x);
  const unsigned int e = (b >> 23) & 0xffu;
  if (e == 0u) return (double)x;  // zero or subnormal: rare, take the conversion
  const unsigned long long s = (unsigned long long)(b >> 31) << 63;
  return __longlong_as_double((long long)(s | ((unsigned long long)(e - 127u + 1023u) << 52) |
                                          ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// Queue the vertices this warp's lanes discovered for level Lnext
// (warp-collective): entries and their items are appended with one atomic
// per warp each (ballot, then a scan of the item counts).
__device__ __forceinline__ void wide_enqueue(bool enq, int32_t u, const int64_t *__restrict__ row, const WideScratch &S,
                                             int Lnext, int64_t qbase, int64_t ibase, int lane, int *err) {
  const unsigned bm = __ballot_sync(0xffffffffu, enq);
  if (!bm) return;
  int nch = 0;
  if (enq) {
    const int64_t d = __ldg(row + u + 1) - __ldg(row + u);
    nch = (int)((d + WIDE_CH - 1) / WIDE_CH);
    if (nch < 1) nch = 1;
  }
  int inc = nch;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  const int tot = __shfl_sync(0xffffffffu, inc, 31);
  const int ld = __ffs(bm) - 1;
  unsigned long long qb = 0, ib = 0;
  if (lane == ld) {
    qb = atomicAdd(S.cnt + Lnext, (unsigned long long)__popc(bm));
    ib = atomicAdd(S.icnt + Lnext, (unsigned long long)tot);
  }
  qb = __shfl_sync(0xffffffffu, qb, ld);
  ib = __shfl_sync(0xffffffffu, ib, ld);
  if (enq) {
    const int64_t q = qbase + (int64_t)qb + __popc(bm & ((1u << lane) - 1u));
    const int64_t i0 = ibase + (int64_t)ib + (inc - nch);
    if (q >= S.qcap || i0 + nch > S.icap) {
      atomicOr(err, ERR_CAP);
      return;
    }
    S.queue[q] = u;
    S.qdone[q] = 0;
    int32_t h = -1;
    if (nch > 1) {
      const unsigned long long hh = atomicAdd(S.hubs, 1ull);
      if ((int64_t)hh >= S.hcap) atomicOr(err, ERR_CAP);
      else h = (int32_t)hh;
    }
    S.qhub[q] = h;
    for (int c = 0; c < nch; c++) S.items[i0 + c] = ((unsigned long long)q << 32) | (unsigned long long)(c * WIDE_CH);
  }
}

template <bool REACH, bool IDENT, bool FP32>
__global__ void __launch_bounds__(WIDE_THREADS) k_bcreach_wide(
    const int64_t *__restrict__ row, const int32_t *__restrict__ col, int32_t n, double fan,
    const int32_t *__restrict__ reach, const double *__restrict__ init_f, const int32_t *__restrict__ ident,
    const int32_t *__restrict__ order, int32_t nsrc, double *bcp, WideScratch S, GridBarrier bar, int *err,
    unsigned long long *dag_total, int sig_cap) {
  const int lane = threadIdx.x & 31;
  const int64_t gtid = (int64_t)blockIdx.x * WIDE_THREADS + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * WIDE_THREADS;
  const int64_t gwarp = gtid >> 5, nwarps = nthreads >> 5;
  const bool leader = blockIdx.x == 0 && threadIdx.x < 32;  // writes the per-level records
  long long *const sigi = (long long *)S.sig;
  const int flg = ceil_log2_pos(fan);
  // stored FP64 counts of a level stay at or below 2^t_hi, so the next level's
  // sums (at most fan times larger) stay finite; a rescale brings them to 2^t_lo
  const int t_hi = 1000 - flg, t_lo = t_hi - 400;
  unsigned long long dag = 0;
  const int nbatch = (nsrc + 31) / 32;
  for (int b = 0; b < nbatch; b++) {
    const int32_t my_src = 32 * b + lane < nsrc ? __ldg(order + 32 * b + lane) : -1;
    double ws = 0.0;  // the source's weight reach[s] * ident[s]
    if (my_src >= 0)
      ws = (REACH ? (init_f ? __ldg(init_f + my_src) + 1.0 : (double)__ldg(reach + my_src)) : 1.0) *
           (IDENT ? (double)__ldg(ident + my_src) : 1.0);
    // ------------------------------------------------ level 0: the sources
    if (leader) {
      // one entry per distinct source vertex (a source list may repeat one):
      // the lowest lane of each group of equal sources makes it
      const bool act = my_src >= 0;
      const unsigned grp = __match_any_sync(0xffffffffu, my_src);
      const bool head = act && (__ffs(grp) - 1) == lane;
      const unsigned hm = __ballot_sync(0xffffffffu, head);
      int nch = 0;
      if (head) {
        const int64_t d = row[my_src + 1] - row[my_src];
        nch = (int)((d + WIDE_CH - 1) / WIDE_CH);
        if (nch < 1) nch = 1;
      }
      int inc = nch;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      const int tot = __shfl_sync(0xffffffffu, inc, 31);
      if (lane == 0) *S.hubs = 0ull;
      __syncwarp();
      if (act) sigi[(size_t)my_src * 32 + lane] = 1;
      if (head) {
        const int q = __popc(hm & ((1u << lane) - 1u));  // entry index among the heads
        S.queue[q] = my_src;
        S.qdone[q] = 0;
        S.qhub[q] = nch > 1 ? (int32_t)atomicAdd(S.hubs, 1ull) : -1;
        S.lv[my_src] = spread2(grp);  // level 0 (code 1) for every lane of the group
        S.nxt[my_src] = grp;          // nxt[0]
        for (int c = 0; c < nch; c++)
          S.items[inc - nch + c] = ((unsigned long long)q << 32) | (unsigned long long)(c * WIDE_CH);
      }
      S.lmax[lane] = act ? 1ull : 0ull;
      if (lane == 0) {
        S.cnt[0] = (unsigned long long)__popc(hm);
        S.icnt[0] = (unsigned long long)tot;
      }
    }
    if (!grid_wait(bar)) return;
    // ------------------------------------------------ phase 1
    int64_t qlo = 0, ilo = 0, qprev = 0;
    int L = 0, kind_prev = 1;
    for (;;) {
      const int64_t nq = (int64_t)__ldcg(S.cnt + L), ni = (int64_t)__ldcg(S.icnt + L);
      // (the capacities hold every batch; the clamps only keep reads in bounds)
      const int64_t qhi = min(qlo + nq, S.qcap), ihi = min(ilo + ni, S.icap);
      // representation of level L's counts and the scale of level L-1's
      int kind = 1, kprev = 0, X = 0;
      if (L > 0) {
        const unsigned long long mp = __ldcg(S.lmax + (size_t)(L - 1) * 32 + lane);
        const int Xp = __ldcg(S.lexp + (size_t)(L - 1) * 32 + lane);
        int top;  // binary exponent of the lane's largest count of level L-1
        if (kind_prev) {
          const unsigned long long mall = warp_max_u64(mp);
          const int lg = mall ? 64 - __clzll((long long)mall) : 0;
          kind = lg + flg <= 62 ? 1 : 0;
          top = mp ? 63 - __clzll((long long)mp) : 0;
        } else {
          kind = 0;
          const int ex = (int)((mp >> 52) & 0x7ff) - 1023;  // binary exponent of the level's largest count
          kprev = ex > t_hi ? ex - t_lo : 0;
          top = ex;
        }
        if (mp && top + Xp > sig_cap && gtid < 32) atomicOr(err, ERR_OVERFLOW);
        X = Xp + kprev;
      }
      if (leader) {
        S.lexp[(size_t)L * 32 + lane] = X;
        if (lane == 0) {
          S.lkind[L] = kind;
          S.qoff[L] = qlo;
          S.ioff[L] = ilo;
        }
      }
      // the previous level's nxt plane is read: clear it for level L+2
      if (L > 0) {
        uint32_t *np = S.nxt + (size_t)((L - 1) % 3) * S.n;
        for (int64_t i = qprev + gtid; i < qlo; i += nthreads) np[__ldcg(S.queue + i)] = 0u;
      }
      if (nq == 0) break;  // every thread sees the same counts
      if (L + 2 >= WIDE_LCAP) {
        if (gtid == 0) atomicOr(err, ERR_DEPTH);
        return;
      }
      const uint32_t code_prev = level_code(L + 2), code_next = level_code(L + 1);  // (L-1) mod 3 = (L+2) mod 3
      const uint32_t *nxt_cur = S.nxt + (size_t)(L % 3) * S.n;
      uint32_t *nxt_next = S.nxt + (size_t)((L + 1) % 3) * S.n;
      const double kscale = pow2_int(-kprev);
      unsigned long long wmax = 0ull;  // this lane's largest stored count of level L in this warp's items
      for (int64_t it = ilo + gwarp; it < ihi; it += nwarps) {
        const unsigned long long itv = __ldcg(S.items + it);
        const int64_t i = (int64_t)(itv >> 32);
        const int64_t c0 = (int64_t)(itv & 0xffffffffull);
        const int32_t w = __ldcg(S.queue + i);
        const uint32_t f = __ldcg(nxt_cur + w);
        const int64_t rb = __ldg(row + w), re = __ldg(row + w + 1);
        const int64_t e0 = rb + c0, e1 = min(re, e0 + WIDE_CH);
        const bool split = re - rb > WIDE_CH;
        if (c0 == 0 && lane == 0) S.qmask[i] = f;
        const bool mine = (f >> lane) & 1u;
        long long ai = 0;
        double ad = 0.0;
        for (int64_t e = e0; e < e1; e += 32) {
          const bool has = e + lane < e1;
          const int32_t u = has ? __ldg(col + e + lane) : 0;
          const uint64_t lu = has ? __ldcg(S.lv + u) : 0ull;
          uint32_t pm = 0u, dm = 0u;
          if (has) {
            if (L > 0) pm = lanes_with_code(lu, code_prev) & f;
            dm = f & ~lanes_reached(lu);
          }
          bool enq = false;
          if (dm) {
            const unsigned long long old = atomicOr((unsigned long long *)(S.lv + u), spread2(dm) * code_next);
            const uint32_t nm = dm & ~lanes_reached(old);
            if (nm) enq = atomicOr(nxt_next + u, nm) == 0u;
          }
          wide_enqueue(enq, u, row, S, L + 1, qhi, ihi, lane, err);
          // path counts from the predecessors among these entries, four
          // loads in flight at a time
          unsigned bal = __ballot_sync(0xffffffffu, pm != 0u);
          while (bal) {
            int32_t vv[4];
            bool on[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
              const int j = bal ? __ffs(bal) - 1 : 0;
              const uint32_t m = bal ? __shfl_sync(0xffffffffu, pm, j) : 0u;
              vv[k] = __shfl_sync(0xffffffffu, u, j);
              on[k] = (m >> lane) & 1u;
              bal &= bal - 1u;
            }
            if (kind) {
              long long x[4];
#pragma unroll
              for (int k = 0; k < 4; k++) x[k] = on[k] ? __ldcg(sigi + (size_t)vv[k] * 32 + lane) : 0ll;
#pragma unroll
              for (int k = 0; k < 4; k++) {
                if (IDENT && L > 1 && on[k]) x[k] *= (long long)__ldg(ident + vv[k]);
                ai += x[k];
              }
            } else {
              double x[4];
              if (kind_prev) {
#pragma unroll
                for (int k = 0; k < 4; k++)
                  x[k] = on[k] ? i64_to_f64_pos(__ldcg(sigi + (size_t)vv[k] * 32 + lane) | 0ll) : 0.0;
              } else {
#pragma unroll
                for (int k = 0; k < 4; k++) x[k] = on[k] ? __ldcg(S.sig + (size_t)vv[k] * 32 + lane) : 0.0;
              }
#pragma unroll
              for (int k = 0; k < 4; k++) {
                if (!on[k]) continue;
                if (IDENT && L > 1) x[k] *= (double)__ldg(ident + vv[k]);
                ad += x[k];
              }
            }
          }
        }
        if (L == 0) continue;  // the sources' counts are set
        if (!kind && kprev) ad *= kscale;
        if (!split) {
          if (mine) {
            if (kind) {
              sigi[(size_t)w * 32 + lane] = ai;
              wmax = (unsigned long long)ai > wmax ? (unsigned long long)ai : wmax;
            } else {
              S.sig[(size_t)w * 32 + lane] = ad;
              const unsigned long long bits = (unsigned long long)__double_as_longlong(ad);
              wmax = bits > wmax ? bits : wmax;
            }
          }
        } else {
          const int32_t h = __ldcg(S.qhub + i);
          if (h >= 0 && mine) {
            if (kind) atomicAdd((unsigned long long *)(S.hacc + (size_t)h * 32 + lane), (unsigned long long)ai);
            else atomicAdd(S.hacc + (size_t)h * 32 + lane, ad);
          }
          __threadfence();
          const int nch = (int)((re - rb + WIDE_CH - 1) / WIDE_CH);
          int last = 0;
          if (lane == 0) last = atomicAdd(S.qdone + i, 1) == nch - 1;
          last = __shfl_sync(0xffffffffu, last, 0);
          if (last && h >= 0) {
            __threadfence();
            if (mine) {
              double *slot = S.hacc + (size_t)h * 32 + lane;
              if (kind) {
                const long long t = __ldcg((const long long *)slot);
                sigi[(size_t)w * 32 + lane] = t;
                wmax = (unsigned long long)t > wmax ? (unsigned long long)t : wmax;
              } else {
                const double t = __ldcg(slot);
                S.sig[(size_t)w * 32 + lane] = t;
                const unsigned long long bits = (unsigned long long)__double_as_longlong(t);
                wmax = bits > wmax ? bits : wmax;
              }
              *slot = 0.0;  // the accumulator serves phase 2 next
            }
          }
        }
      }
      if (wmax) atomicMax(S.lmax + (size_t)L * 32 + lane, wmax);
      if (!grid_wait(bar)) return;
      kind_prev = kind;
      qprev = qlo;
      qlo = qhi;
      ilo = ihi;
      L++;
    }
    const int Lmax = L - 1;
    const int64_t qtotal = qlo, itotal = ilo;  // held by every thread (the last level's end is not in ioff yet)
    // ------------------------------------------------ phase 2
    // level 0 holds only the sources themselves: nothing to add there
    for (int l = Lmax; l >= 1; l--) {
      const int64_t ia = __ldcg(S.ioff + l), ib = min(l == Lmax ? itotal : __ldcg(S.ioff + l + 1), S.icap);
      const int kind_l = __ldcg(S.lkind + l);
      const int Xl = __ldcg(S.lexp + (size_t)l * 32 + lane);
      const int Xn = l < Lmax ? __ldcg(S.lexp + (size_t)(l + 1) * 32 + lane) : Xl;
      const double scl = pow2_int(Xl - Xn);  // sigma[v] / sigma[w] in stored units: times 2^(X_l - X_{l+1})
      const uint32_t code_succ = level_code(l + 1);
      for (int64_t it = ia + gwarp; it < ib; it += nwarps) {
        const unsigned long long itv = __ldcg(S.items + it);
        const int64_t i = (int64_t)(itv >> 32);
        const int64_t c0 = (int64_t)(itv & 0xffffffffull);
        const int32_t v = __ldcg(S.queue + i);
        const uint32_t f = __ldcg(S.qmask + i);
        const int64_t rb = __ldg(row + v), re = __ldg(row + v + 1);
        const int64_t e0 = rb + c0, e1 = min(re, e0 + WIDE_CH);
        const bool split = re - rb > WIDE_CH;
        const bool mine = (f >> lane) & 1u;
        // own path count: FP64 value, or FP32 mantissa and binary exponent
        double sv = 1.0;
        int ev = 0;
        float mv = 1.0f;
        if (mine) {
          if (kind_l) {
            const long long si = __ldcg(sigi + (size_t)v * 32 + lane);
            if (FP32) split_pow2_i64(si, ev, mv);
            else sv = i64_to_f64_pos(si);
          } else {
            sv = __ldcg(S.sig + (size_t)v * 32 + lane);
            if (FP32) split_pow2(sv, ev, mv);
          }
          ev += Xl;
        }
        double s64 = 0.0;
        float s32 = 0.0f;
        if (l < Lmax) {
          for (int64_t e = e0; e < e1; e += 32) {
            const bool has = e + lane < e1;
            const int32_t u = has ? __ldg(col + e + lane) : 0;
            const uint64_t lu = has ? __ldcg(S.lv + u) : 0ull;
            const uint32_t sm = has ? lanes_with_code(lu, code_succ) & f : 0u;
            unsigned bal = __ballot_sync(0xffffffffu, sm != 0u);
            while (bal) {
              int32_t ww[4];
              bool on[4];
#pragma unroll
              for (int k = 0; k < 4; k++) {
                const int j = bal ? __ffs(bal) - 1 : 0;
                const uint32_t m = bal ? __shfl_sync(0xffffffffu, sm, j) : 0u;
                ww[k] = __shfl_sync(0xffffffffu, u, j);
                on[k] = (m >> lane) & 1u;
                bal &= bal - 1u;
              }
              if (!FP32) {
                double x[4];
#pragma unroll
                for (int k = 0; k < 4; k++) x[k] = on[k] ? __ldcg(S.sig + (size_t)ww[k] * 32 + lane) : 0.0;
#pragma unroll
                for (int k = 0; k < 4; k++)
                  if (on[k]) {
                    s64 += x[k];
                    dag++;
                  }
              } else {
                unsigned long long x[4];
#pragma unroll
                for (int k = 0; k < 4; k++)
                  x[k] = on[k] ? __ldcg((const unsigned long long *)S.sig + (size_t)ww[k] * 32 + lane) : 0ull;
#pragma unroll
                for (int k = 0; k < 4; k++)
                  if (on[k]) {
                    const float cc = __uint_as_float((unsigned int)(x[k] & 0xffffffffull));
                    const int xe = ev - (int)(x[k] >> 32);  // <= 0: sigma[v] <= sigma[w]
                    if (xe >= -126) s32 = fmaf(cc, __int_as_float((127 + xe) << 23), s32);
                    dag++;
                  }
              }
            }
          }
        }
        bool fin = !split;
        if (split) {  // partial sums of a split entry meet in its accumulator
          const int32_t h = __ldcg(S.qhub + i);
          if (h >= 0 && mine) {
            if (!FP32) atomicAdd(S.hacc + (size_t)h * 32 + lane, s64);
            else atomicAdd((float *)(S.hacc + (size_t)h * 32 + lane), s32);
          }
          __threadfence();
          const int nch = (int)((re - rb + WIDE_CH - 1) / WIDE_CH);
          int last = 0;
          if (lane == 0) last = atomicAdd(S.qdone + i, 1) == 2 * nch - 1;
          fin = __shfl_sync(0xffffffffu, last, 0) && h >= 0;
          if (fin) {
            __threadfence();
            if (mine) {
              double *slot = S.hacc + (size_t)h * 32 + lane;
              if (!FP32) s64 = __ldcg(slot);
              else s32 = __ldcg((const float *)slot);
              *slot = 0.0;
            }
          }
        }
        if (!fin) continue;
        double dv = 0.0;
        float contrib32 = 0.0f;
        double contrib64 = 0.0;
        if (mine) {
          const double init = REACH ? (init_f ? __ldg(init_f + v) : (double)(__ldg(reach + v) - 1)) : 0.0;
          if (!FP32) {
            dv = fma(sv, s64 * scl, init);
            const double kv = IDENT ? (double)__ldg(ident + v) : 1.0;
            S.sig[(size_t)v * 32 + lane] = fma(kv, dv, kv) * recip_pos(sv);
            if (v != my_src) contrib64 = ws * dv;
          } else {
            const float df = fmaf(mv, s32, (float)init);
            const float kv = IDENT ? (float)__ldg(ident + v) : 1.0f;
            const float cc = fmaf(kv, df, kv) / mv;
            ((unsigned long long *)S.sig)[(size_t)v * 32 + lane] =
                ((unsigned long long)(unsigned int)ev << 32) | (unsigned long long)__float_as_uint(cc);
            if (v != my_src) contrib32 = (float)ws * df;
          }
        }
        // bc'[v] gains the entry's sources' terms, summed in the warp
        if (!FP32) {
          for (int o = 16; o > 0; o >>= 1) contrib64 += __shfl_down_sync(0xffffffffu, contrib64, o);
          if (lane == 0 && contrib64 != 0.0) atomicAdd(bcp + v, contrib64);
        } else {
          for (int o = 16; o > 0; o >>= 1) contrib32 += __shfl_down_sync(0xffffffffu, contrib32, o);
          if (lane == 0 && contrib32 != 0.0f) atomicAdd(bcp + v, f32_to_f64_bits(contrib32));
        }
      }
      if (!grid_wait(bar)) return;
    }
    // ------------------------------------------------ clear for the next batch
    for (int64_t i = gtid; i < qtotal; i += nthreads) {
      const int32_t v = __ldcg(S.queue + i);
      S.lv[v] = 0ull;
      S.nxt[v] = 0u;
      S.nxt[S.n + v] = 0u;
      S.nxt[2 * S.n + v] = 0u;
    }
    for (int64_t k = gtid; k < (int64_t)(Lmax + 2) * 32; k += nthreads) {
      S.lmax[k] = 0ull;
      if (k < Lmax + 2) {
        S.cnt[k] = 0ull;
        S.icnt[k] = 0ull;
      }
    }
    {
      const int64_t nh = (int64_t)__ldcg(S.hubs) * 32;
      for (int64_t k = gtid; k < nh; k += nthreads) S.hacc[k] = 0.0;
    }
    if (!grid_wait(bar)) return;
  }
  if (dag) atomicAdd(dag_total, dag);
}

// ---------------------------------------------------------- host side
template <bool R, bool I, bool F>
static int wide_launch_t(Ctx &ctx, int per_sm_cap, void **args) {
  int per_sm = 0;
  BCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bcreach_wide<R, I, F>, WIDE_THREADS, 0));
  if (per_sm < 1) {
    set_error("the wide Bc-Reach kernel cannot be resident");
    return BCS_ECUDA;
  }
  per_sm = std::min(per_sm, per_sm_cap);
  BCS_CUDA(cudaLaunchCooperativeKernel((const void *)k_bcreach_wide<R, I, F>, dim3(ctx.num_sms * per_sm),
                                       dim3(WIDE_THREADS), args, 0, ctx.stream));
  ctx.launches++;
  return BCS_OK;
}

int wide_depth_limit() { return (WIDE_LCAP - 4) / 2; }

int run_wide(Ctx &ctx, const CompDesc &c, const BcInput &in, bool fp32, const int32_t *d_order, int32_t nsrc,
             int *d_err, unsigned long long *d_dag) {
  if (nsrc <= 0 || c.n < 2) return BCS_OK;
  const int64_t n = c.n;
  const int64_t qcap = 32 * n + 64;
  // every entry has one item per WIDE_CH row entries; over a batch a vertex
  // has at most 32 entries
  const int64_t icap = qcap + 32 * (c.nnz / WIDE_CH + 1);
  // accumulator slots: at most one per entry of a vertex with a split row
  const int64_t hcap = std::min<int64_t>(qcap, 32 * (c.nnz / WIDE_CH + 1));
  DBuf<uint64_t> lv;
  DBuf<uint32_t> nxt, qmask;
  DBuf<double> sig, hacc;
  DBuf<int32_t> queue, qhub, qdone, lexp, lkind;
  DBuf<unsigned long long> items, cnt, icnt, hubs, lmax, barw;
  DBuf<int64_t> qoff, ioff;
  const cudaStream_t s = ctx.stream;
  BCS_TRY(lv.alloc(n, s));
  BCS_TRY(nxt.alloc(3 * n, s));
  BCS_TRY(sig.alloc(32 * n, s));
  BCS_TRY(queue.alloc(qcap, s));
  BCS_TRY(qmask.alloc(qcap, s));
  BCS_TRY(qhub.alloc(qcap, s));
  BCS_TRY(qdone.alloc(qcap, s));
  BCS_TRY(items.alloc(icap, s));
  BCS_TRY(hacc.alloc(hcap * 32, s));
  BCS_TRY(cnt.alloc(WIDE_LCAP + 2, s));
  BCS_TRY(icnt.alloc(WIDE_LCAP + 2, s));
  BCS_TRY(hubs.alloc(1, s));
  BCS_TRY(qoff.alloc(WIDE_LCAP + 2, s));
  BCS_TRY(ioff.alloc(WIDE_LCAP + 2, s));
  BCS_TRY(lmax.alloc((size_t)WIDE_LCAP * 32, s));
  BCS_TRY(lexp.alloc((size_t)WIDE_LCAP * 32, s));
  BCS_TRY(lkind.alloc(WIDE_LCAP, s));
  BCS_TRY(barw.alloc(1, s));
  BCS_CUDA(cudaMemsetAsync(lv.p, 0, n * 8, s));
  BCS_CUDA(cudaMemsetAsync(nxt.p, 0, 3 * n * 4, s));
  BCS_CUDA(cudaMemsetAsync(hacc.p, 0, hcap * 32 * 8, s));
  BCS_CUDA(cudaMemsetAsync(cnt.p, 0, (WIDE_LCAP + 2) * 8, s));
  BCS_CUDA(cudaMemsetAsync(icnt.p, 0, (WIDE_LCAP + 2) * 8, s));
  BCS_CUDA(cudaMemsetAsync(lmax.p, 0, (size_t)WIDE_LCAP * 32 * 8, s));
  BCS_CUDA(cudaMemsetAsync(barw.p, 0, 8, s));
  WideScratch S{lv.p,    nxt.p,  sig.p,  queue.p, qmask.p, qhub.p, qdone.p, items.p, hacc.p, cnt.p,
                icnt.p,  hubs.p, qoff.p, ioff.p,  lmax.p,  lexp.p, lkind.p, n,       qcap,   icap,
                hcap};
  GridBarrier gb{(unsigned int *)barw.p, (unsigned int *)barw.p + 1, d_err, (long long)ctx.max_wait};
  const int64_t *row = in.row + c.row_off;
  const int32_t *colp = in.col;
  int32_t nn = c.n;
  double fan = c.fan;
  const bool R = in.reach != nullptr || in.init != nullptr, I = in.ident != nullptr;
  const int32_t *reach = in.reach && !in.init ? in.reach + c.vtx_off : nullptr;
  const double *init_f = in.init ? in.init + c.vtx_off : nullptr;
  const int32_t *ident = in.ident ? in.ident + c.vtx_off : nullptr;
  double *bcp = in.bcp + c.vtx_off;
  int cap_lg2 = ctx.sigma_cap_lg2;
  void *args[] = {(void *)&row,   (void *)&colp, (void *)&nn,     (void *)&fan, (void *)&reach,
                  (void *)&init_f, (void *)&ident, (void *)&d_order, (void *)&nsrc, (void *)&bcp,
                  (void *)&S,      (void *)&gb,    (void *)&d_err,   (void *)&d_dag, (void *)&cap_lg2};
  int cap = 8;
  if (const char *e = std::getenv("BCS_WIDE_CTAS_PER_SM")) cap = std::max(1, std::atoi(e));
  return BCS_DISPATCH3(wide_launch_t, R, I, fp32, ctx, cap, args);
}

}  // namespace bcs
