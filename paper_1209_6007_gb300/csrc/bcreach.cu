// bcreach.cu - Bc-Reach (Algorithm 2 with the identical-vertex terms of
// Section 3.3.3) over many components in persistent launches.
//
// Per source s of a component (local ids, reach r[], ident k[]):
//   phase 1 (BFS, Algorithm 1):  d[s] = 0, sigma[s] = 1,
//     sigma[w] += sigma[v] * (v == s ? 1 : k[v])  for every DAG edge v -> w
//   phase 2 (Eq. 3 with reach and ident):
//     delta[v] = r[v] - 1 + sum_{w: d[w] = d[v]+1} sigma[v]/sigma[w] * k[w] * (1 + delta[w])
//     bc'[v]  += r[s] * k[s] * delta[v]   for v != s
// Phase 2 is evaluated in the equivalent "coefficient" form
//     c[w] = k[w] (1 + delta[w]) / sigma[w],   delta[v] = r[v] - 1 + sigma[v] * sum_w c[w]
// so that each shortest-path-DAG edge costs one addition and each vertex one
// reciprocal (from a table for small integer counts).
//
// A group of threads (one warp up to a whole CTA) runs one source at a time,
// level-synchronously: the BFS queue doubles as the stack of Algorithm 1 and
// its level boundaries are kept, so phase 2 walks the levels deepest first
// and pulls from the successors (no atomics in phase 2).
//
// Path counts are exact 64-bit integers while a level's growth bound stays
// below 2^62; past it they are FP64 and each level carries a power-of-two
// exponent: when a level's largest count passes 2^960 the whole level is
// scaled by an exact power of two, and phase 2 multiplies by 2^(e[L] - e[L+1]).
//
// FP32 mode keeps delta and the per-edge sums in FP32: c is stored as an FP32
// value relative to the binary exponent of sigma[w] (held next to it), so
// sigma's full range is kept without FP64 arithmetic in phase 2.
#include <algorithm>
#include <cfloat>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <set>

#include "bc_math.cuh"
#include "common.h"

namespace bcs {

constexpr int SMALL_THREADS = 256;
// Shared memory one small-path CTA may use: a piece whose state for a single
// source does not fit goes to the global-memory path.
constexpr size_t SMALL_SMEM = 100 * 1024;
constexpr int SMALL_MAX_GROUPS = 8;
constexpr int DISC_CH = 4;  // row entries per step of the shared-memory discovery pass (divides 32)
constexpr int LARGE_THREADS = 512;
// BFS depth above which large pieces run one source per CTA rather than 32
constexpr int MS_DEPTH_LIMIT = 64;
// Large pieces with at least this many vertices and a BFS eccentricity (from
// their first vertex) of at most WIDE_MAX_ECC run on the whole-GPU path
constexpr int WIDE_MIN_N = 32768;
constexpr int WIDE_MAX_ECC = 40;
// Pieces of at most MID_MAX_N vertices that do not fit shared memory can run
// one 64-source batch per CTA (BCS_LARGE_PATH=mid), by default only if
// MID_BY_DEFAULT and they give at least MID_MIN_UNITS_PER_SM batches per SM.
// Off: on the uneven batch of pieces up to 4,096 vertices it measured 3 %
// slower than 32 sources per CTA (4.14 s against 4.04 s per call).
constexpr int MID_MAX_N = 65536;
constexpr int64_t MID_MIN_UNITS_PER_SM = 8;
constexpr bool MID_BY_DEFAULT = false;

struct SmallItem {
  int32_t comp;
  int32_t s_begin;  // index range into the source list (or local ids)
  int32_t s_end;
  int32_t ngroups;  // groups (concurrent sources) per CTA, 1..8
};

// ------------------------------------------------------------------ group
struct Group {
  int rank, size, bar;
  __device__ __forceinline__ void sync() const {
    if (size == 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(size) : "memory");
  }
};

__device__ __forceinline__ double group_max(const Group &g, double x, volatile double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  if (g.size == 32) return x;
  if ((g.rank & 31) == 0) red[g.rank >> 5] = x;
  g.sync();
  double r = red[0];
  for (int i = 1; i < (g.size >> 5); i++) r = fmax(r, red[i]);
  g.sync();
  return r;
}

__device__ __forceinline__ int vld(const int32_t *p) { return *(volatile const int32_t *)p; }

template <bool FP32>
struct CoefT;
template <>
struct CoefT<false> {
  using type = double;
};
template <>
struct CoefT<true> {
  using type = Coef32;
};

// Reciprocals 1/k of the integers k < RECIP_TABLE (entry 0 unused), filled
// once per device by IEEE division (correctly rounded).
constexpr int RECIP_TABLE = 1024;
static __device__ double g_recip_table[RECIP_TABLE];

__global__ void k_fill_recip_table() {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < RECIP_TABLE; k += gridDim.x * blockDim.x)
    g_recip_table[k] = k == 0 ? 0.0 : 1.0 / (double)k;
}

// State of one source, in shared (small path) or global (large path) memory.
template <bool FP32, typename QT = int32_t>
struct SrcState {
  int32_t *d;
  double *sig;
  typename CoefT<FP32>::type *coef;  // global path: sigma * ident in phase 1; shared path: == sig
  QT *queue;                         // 16-bit local ids on the shared-memory path
  uint32_t *dmask;     // shared-memory path: DAG successors among the first 32 row entries
  int32_t *lvl_start;  // levels + 2
  int32_t *lvl_exp;    // levels + 1
  int *qtail;          // shared counter
  double *red;         // shared, 16 doubles: group maxima, and the source weight
};
constexpr int RED_WS = 15;  // slot of the source weight in SrcState::red

struct Weights {  // global-memory path: the int32 arrays; shared path: only the FP64 copies
  const int32_t *reach;   // local, nullable
  const int32_t *ident;   // local, nullable
  const double *init_d;   // reach - 1 as FP64, nullable (converted on the fly)
  const double *ident_d;  // ident as FP64, nullable
  bool frac;              // init_d may be fractional: never read reach as an integer
};

struct Debug {
  int32_t *d;
  double *sig;
  int32_t *exp;
  double *delta;
};


// One source of Bc-Reach over a component held as (row, col) with local ids.
// RESET_BY_QUEUE: the distances start at -1 and are put back that way
// through the queue at the end (global-memory path); else they are
// initialised here (shared-memory path).  acc is private to the group (plain
// adds).  dag counts the shortest-path DAG edges seen in phase 2.
//
// Path counts are integers.  While the growth bound fan^L of a level stays
// below 2^62 they are summed as exact 64-bit integers (the FP64 pipe is the
// scarce one on GB300, and below 2^53 the values are the same bits as an
// FP64 sum); the first level whose bound could pass 2^62 converts the level
// before it to FP64 once, and from there on counts are FP64 with a
// power-of-two exponent per level.  sig holds int64 on the integer levels.
//
// Shared-memory path (!RESET_BY_QUEUE): one pass over a level's rows both
// discovers the next level and, on the integer levels, pushes the path
// counts along the DAG edges it finds (shared-memory atomics); each vertex
// also keeps the DAG edges among its first 32 row entries as a bit mask, so
// phase 2 visits only the successors; its phase-2 coefficients overwrite the
// path counts in place.  The global-memory path pulls the counts in a second
// pass and finds successors by their level (pushing through L2 atomics
// measured slower on deep graphs, where that path is used).
template <bool REACH, bool IDENT, bool FP32, bool RESET_BY_QUEUE, typename RowT, typename ColT, typename QT>
__device__ void bcreach_source(const Group &g, const int32_t s, const int32_t n, const RowT *__restrict__ row,
                               const ColT *__restrict__ col, const Weights wt, const SrcState<FP32, QT> st,
                               double *acc, const double fan, int *err, const Debug *dbg,
                               unsigned long long &dag, int *lmax_out = nullptr) {
  // reach and ident as integers: from the int32 arrays on the global-memory
  // path, from the FP64 copies (integer instructions) on the shared path
  auto ident_i = [&](int32_t v) -> long long {
    return wt.ident ? (long long)wt.ident[v] : f64_to_i64_exact(wt.ident_d[v]);
  };
  auto reach_i = [&](int32_t v) -> long long {
    return wt.reach ? (long long)wt.reach[v] : f64_to_i64_exact(wt.init_d[v]) + 1;
  };
  int32_t *const d = st.d;
  double *const sig = st.sig;
  long long *const sigi = (long long *)st.sig;
  double *const sk = (double *)st.coef;  // global path: sigma[v] * (v == s ? 1 : ident[v]) in phase 1
  long long *const ski = (long long *)st.coef;
  constexpr bool PUSH = !RESET_BY_QUEUE;
  // Shared-memory path: the coefficient of phase 2 overwrites the path count
  // of the same vertex (st.coef == st.sig); phase 1 keeps sigma alone and
  // multiplies by ident where it reads it.
  constexpr bool ALIAS = PUSH;
  long long *const pull_src = IDENT ? ski : sigi;  // sigma * ident (the source counts once)
  if (!RESET_BY_QUEUE) {
    for (int v = g.rank; v < n; v += g.size) {
      d[v] = -1;
      sigi[v] = 0;
    }
    g.sync();
  }
  if (g.rank == 0) {
    d[s] = 0;
    sigi[s] = 1;
    ski[s] = 1;
    st.queue[0] = s;
    *st.qtail = 1;
    st.lvl_start[0] = 0;
    st.lvl_start[1] = 1;
    st.lvl_exp[0] = 0;
  }
  g.sync();
  // ---------------------------------------------------------- phase 1
  int lo = 0, hi = 1, L = 0, ecur = 0;
  int lint = 1 << 30;  // first FP64 level
  // growth bound of the current level's counts as a power of two, kept in
  // integers: level-uniform FP64 tests would be evaluated by every lane
  const int flg = ceil_log2_pos(fan);
  int blg = 0;
  for (;;) {
    // level L+1 keeps integer counts while its growth bound stays below 2^62
    const bool push = PUSH && lint > L + 1 && blg + flg < 62;
    // below 2^31 every partial sum fits the low word: 32-bit atomics
    const bool push32 = push && blg + flg < 31;
    // discover level L+1 (integer work only)
    for (int i = lo + g.rank; i < hi; i += g.size) {
      const int32_t v = st.queue[i];
      const RowT eb = row[v], ee = row[v + 1];
      if (PUSH) {
        // sigma[v] * ident[v], formed by v's own lane (sigma[v] is final)
        const long long pv = !push ? 0 : (IDENT && v != s ? sigi[v] * ident_i(v) : sigi[v]);
        uint32_t m = 0u;
        // DISC_CH row entries at a time, so that their shared-memory round
        // trips overlap instead of forming one chain per entry
        for (RowT e0 = eb; e0 < ee; e0 += DISC_CH) {
          int32_t w[DISC_CH];
          int dw[DISC_CH];
#pragma unroll
          for (int j = 0; j < DISC_CH; j++) w[j] = e0 + j < ee ? (int32_t)col[e0 + j] : -1;
#pragma unroll
          for (int j = 0; j < DISC_CH; j++) dw[j] = w[j] >= 0 ? vld(d + w[j]) : L;  // L: no DAG edge
          unsigned won = 0u, dagb = 0u;
#pragma unroll
          for (int j = 0; j < DISC_CH; j++) {
            const int r = dw[j] < 0 ? atomicCAS(d + w[j], -1, L + 1) : dw[j];
            won |= (unsigned)(r < 0) << j;
            dagb |= (unsigned)(r < 0 || r == L + 1) << j;
          }
          if (won) {  // one counter update for the vertices this lane claimed
            int pos = atomicAdd(st.qtail, __popc(won));
#pragma unroll
            for (int j = 0; j < DISC_CH; j++)
              if (won >> j & 1u) st.queue[pos++] = w[j];
          }
#pragma unroll
          for (int j = 0; j < DISC_CH; j++) {
            if (dagb >> j & 1u) {
              if (push32) atomicAdd((unsigned int *)(sigi + w[j]), (unsigned int)pv);
              else if (push) atomicAdd((unsigned long long *)(sigi + w[j]), (unsigned long long)pv);
            }
          }
          if (e0 - eb < 32) m |= dagb << (int)(e0 - eb);
        }
        st.dmask[v] = m;
      } else {
        for (RowT e = eb; e < ee; e++) {
          const int32_t w = (int32_t)col[e];
          if (vld(d + w) < 0 && atomicCAS(d + w, -1, L + 1) == -1) st.queue[atomicAdd(st.qtail, 1)] = w;
        }
      }
    }
    g.sync();
    const int nhi = vld(st.qtail);
    g.sync();
    if (nhi == hi) break;
    blg += flg;
    if (lint > L + 1 && blg >= 62) {
      // level L+1 may not fit 63 bits: it is pulled in FP64 from level L
      // (shared-memory path: level L's counts turn FP64 in place, so level L
      // is the first FP64 level)
      lint = ALIAS ? L : L + 1;
      for (int i = lo + g.rank; i < hi; i += g.size) {
        const int32_t v = st.queue[i];
        if (ALIAS) sig[v] = (double)sigi[v];
        else sk[v] = (double)pull_src[v];
      }
      g.sync();
    }
    if (push) {
      // the counts of level L+1 are complete
    } else if (L + 1 < lint) {  // path counts of level L+1, pulled from level L (one add per DAG edge)
      for (int i = hi + g.rank; i < nhi; i += g.size) {
        const int32_t w = st.queue[i];
        long long a = 0;
        const RowT eb = row[w], ee = row[w + 1];
        for (RowT e = eb; e < ee; e++) {
          const int32_t u = (int32_t)col[e];
          if (d[u] == L) a += pull_src[u];
        }
        sigi[w] = a;
        if (IDENT) ski[w] = a * (long long)wt.ident[w];
      }
    } else {
      for (int i = hi + g.rank; i < nhi; i += g.size) {
        const int32_t w = st.queue[i];
        double a = 0.0;
        const RowT eb = row[w], ee = row[w + 1];
        for (RowT e = eb; e < ee; e++) {
          const int32_t u = (int32_t)col[e];
          if (d[u] == L) a += ALIAS ? (IDENT && u != s ? sig[u] * wt.ident_d[u] : sig[u]) : sk[u];
        }
        sig[w] = a;
        if (!ALIAS) sk[w] = IDENT ? a * (wt.ident_d ? wt.ident_d[w] : (double)wt.ident[w]) : a;
      }
      if (blg > 900) {
        g.sync();
        double m = 0.0;
        for (int i = hi + g.rank; i < nhi; i += g.size) m = fmax(m, sig[st.queue[i]]);
        m = group_max(g, m, st.red);
        if (!(m <= DBL_MAX)) {
          if (g.rank == 0) atomicOr(err, ERR_OVERFLOW);
        } else if (m > 0x1p960) {
          const int k = ilogb(m) - 959;
          for (int i = hi + g.rank; i < nhi; i += g.size) {
            const int32_t w = st.queue[i];
            sig[w] = scalbn(sig[w], -k);
            if (!ALIAS) sk[w] = scalbn(sk[w], -k);
          }
          m = scalbn(m, -k);
          ecur += k;
        }
        blg = m >= 1.0 ? ceil_log2_pos(m) : 0;
        g.sync();
      }
    }
    lo = hi;
    hi = nhi;
    L++;
    if (g.rank == 0) {
      st.lvl_start[L + 1] = hi;
      st.lvl_exp[L] = ecur;
    }
  }
  const int Lmax = L;
  if (lmax_out && g.rank == 0) atomicMax(lmax_out, Lmax);
  // the source's weight reach[s] * ident[s] waits in shared memory: read
  // per vertex, it is never recomputed (FP64) inside the divergent loop
  if (g.rank == 0)
    st.red[RED_WS] = (REACH && wt.frac) ? (wt.init_d[s] + 1.0) * (double)(IDENT ? ident_i(s) : 1ll)
                                        : (double)((REACH ? reach_i(s) : 1ll) * (IDENT ? ident_i(s) : 1ll));
  g.sync();
  // ---------------------------------------------------------- phase 2
  unsigned long long ndag = 0;
  for (int l = Lmax; l >= 0; l--) {
    const int a = st.lvl_start[l], b = st.lvl_start[l + 1];
    const int de = (l < Lmax) ? st.lvl_exp[l] - st.lvl_exp[l + 1] : 0;
    const double scl = pow2_int(de);
    const bool is_int = l < lint;
    for (int i = a + g.rank; i < b; i += g.size) {
      const int32_t v = st.queue[i];
      double dv;
      if (!FP32) {
        const long long si = is_int ? sigi[v] : 0;
        const double sv = is_int ? i64_to_f64_pos(si) : sig[v];
        double sum = 0.0;
        if (l < Lmax) {
          // successors first as a bit mask (integer work), then FP64 adds
          // only for them: an FP64 warp instruction costs the pipe the same
          // whatever its active lanes, so the FP64 loop should run as few
          // iterations as possible (the DAG out-degree, not the degree)
          const RowT eb = row[v], ee = row[v + 1];
          for (RowT e0 = eb; e0 < ee; e0 += 32) {
            uint32_t mask = 0u;
            if (PUSH && e0 == eb) {
              mask = st.dmask[v];
            } else {
              const int cnt = (int)((ee - e0) < 32 ? (ee - e0) : 32);
              for (int j = 0; j < cnt; j++) mask |= (uint32_t)(d[(int32_t)col[e0 + j]] == l + 1) << j;
            }
            ndag += __popc(mask);
            while (mask) {  // one FP64 add per successor (pairing them measured slower)
              const int j = __ffs(mask) - 1;
              mask &= mask - 1u;
              sum += ((const double *)st.coef)[(int32_t)col[e0 + j]];
            }
          }
          if (de != 0) sum *= scl;
        }
        const double init = REACH ? (wt.init_d ? wt.init_d[v] : (double)(wt.reach[v] - 1)) : 0.0;
        dv = fma(sv, sum, init);
        if (l > 0) {  // the source's coefficient is never read
          const double kv = IDENT ? (wt.ident_d ? wt.ident_d[v] : (double)wt.ident[v]) : 1.0;
          // 1/sigma: small integer counts (the usual case) from a table of
          // correctly rounded reciprocals, so a warp whose lanes all have one
          // issues no FP64 work for it
          double r;
          if (PUSH && is_int && si < RECIP_TABLE) r = g_recip_table[si];
          else r = recip_pos(sv);
          ((double *)st.coef)[v] = fma(kv, dv, kv) * r;
        }
      } else {
        int ev;
        float mv;
        if (is_int) split_pow2_i64(sigi[v], ev, mv);
        else split_pow2(sig[v], ev, mv);
        ev += st.lvl_exp[l];
        float sum = 0.0f;
        if (l < Lmax) {
          const RowT eb = row[v], ee = row[v + 1];
          for (RowT e0 = eb; e0 < ee; e0 += 32) {
            uint32_t mask = 0u;
            if (PUSH && e0 == eb) {
              mask = st.dmask[v];
            } else {
              const int cnt = (int)((ee - e0) < 32 ? (ee - e0) : 32);
              for (int j = 0; j < cnt; j++) mask |= (uint32_t)(d[(int32_t)col[e0 + j]] == l + 1) << j;
            }
            ndag += __popc(mask);
            while (mask) {  // two successors per step: their loads overlap
              const int j0 = __ffs(mask) - 1;
              mask &= mask - 1u;
              const int j1 = mask ? __ffs(mask) - 1 : -1;
              mask &= mask - 1u;
              const Coef32 c0 = ((const Coef32 *)st.coef)[(int32_t)col[e0 + j0]];
              const Coef32 c1 = j1 >= 0 ? ((const Coef32 *)st.coef)[(int32_t)col[e0 + j1]] : Coef32{0.0f, ev};
              const int x0 = ev - c0.e, x1 = ev - c1.e;  // <= 0: sigma[v] <= sigma[w]
              if (x0 >= -126) sum = fmaf(c0.c, __int_as_float((127 + x0) << 23), sum);
              if (x1 >= -126) sum = fmaf(c1.c, __int_as_float((127 + x1) << 23), sum);
            }
          }
        }
        const float df =
            fmaf(mv, sum, REACH ? (wt.frac ? (float)wt.init_d[v] : (float)(reach_i(v) - 1)) : 0.0f);
        dv = (double)df;
        if (l > 0) {
          const float kv = IDENT ? (float)ident_i(v) : 1.0f;
          Coef32 cv;
          cv.c = fmaf(kv, df, kv) / mv;
          cv.e = ev;
          ((Coef32 *)st.coef)[v] = cv;
        }
      }
      if (v != s) acc[v] = fma(st.red[RED_WS], dv, acc[v]);
      if (dbg) dbg->delta[v] = dv;
    }
    g.sync();
  }
  dag += ndag;
  if (dbg) {
    for (int i = g.rank; i < hi; i += g.size) {
      const int32_t v = st.queue[i];
      const int lv = d[v];
      dbg->d[v] = lv;
      dbg->sig[v] = lv < lint ? (double)sigi[v] : sig[v];
      dbg->exp[v] = st.lvl_exp[lv];
    }
    g.sync();
  }
  if (RESET_BY_QUEUE) {
    for (int i = g.rank; i < hi; i += g.size) d[st.queue[i]] = -1;
    g.sync();
  }
}

// ---------------------------------------------------------- small path
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// per group: distances and DAG masks (4 bytes each), the queue (2 bytes),
// path counts (later the coefficients, in place) and the group's bc
// accumulator (8 bytes each); the accumulator comes last
__host__ __device__ inline size_t small_acc_offset(int64_t n) {
  return align16((size_t)n * 4) * 2 + align16((size_t)n * 2) + align16((size_t)n * 8);
}
__host__ __device__ inline size_t small_group_bytes(int64_t n) { return small_acc_offset(n) + align16((size_t)n * 8); }

// bytes of shared memory a component needs with `ng` concurrent sources:
// the component (rows, 16-bit columns, reach and ident with their FP64 copies) once,
// and per group the distances, queue, DAG masks, path counts / coefficients
// and its own bc accumulator
__host__ __device__ inline size_t small_smem_bytes(int64_t n, int64_t nnz, int ng, bool reach, bool ident) {
  size_t b = align16((size_t)(n + 1) * 4) + align16((size_t)nnz * 2);
  if (reach) b += align16((size_t)n * 8);
  if (ident) b += align16((size_t)n * 8);
  return b + small_group_bytes(n) * (size_t)ng;
}

template <bool REACH, bool IDENT, bool FP32>
__global__ void __launch_bounds__(SMALL_THREADS) k_bcreach_small(
    const SmallItem *__restrict__ items, int nitems, int *item_counter, const CompDesc *__restrict__ comps,
    const int64_t *__restrict__ g_row, const int32_t *__restrict__ g_col, const int32_t *__restrict__ g_reach,
    const int32_t *__restrict__ g_ident, const double *__restrict__ g_init, const int64_t *__restrict__ srcs,
    double *bcp, int32_t *lvl_scratch, int lvl_stride, int *err, unsigned long long *dag_total) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ int s_next;                     // the item's next unclaimed source
  __shared__ int s_claim[SMALL_MAX_GROUPS];  // the source each group claimed last
  __shared__ int s_qtail[SMALL_MAX_GROUPS];
  __shared__ double s_red[SMALL_MAX_GROUPS][16];
  const int tid = threadIdx.x;
  unsigned long long dag = 0;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(item_counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const SmallItem item = items[it];
    const CompDesc c = comps[item.comp];
    const int n = c.n;
    const int nnz = (int)c.nnz;
    const int ng = item.ngroups;
    unsigned char *p = smem;
    int32_t *row = (int32_t *)p;
    p += align16((size_t)(n + 1) * 4);
    uint16_t *col = (uint16_t *)p;  // local ids of a shared-memory piece fit 16 bits
    p += align16((size_t)nnz * 2);
    // reach - 1 and ident as FP64 only (integers are read back from them)
    double *init_d = nullptr, *ident_d = nullptr;
    if (REACH) {
      init_d = (double *)p;
      p += align16((size_t)n * 8);
    }
    if (IDENT) {
      ident_d = (double *)p;
      p += align16((size_t)n * 8);
    }
    const size_t per = small_group_bytes(n);
    const int64_t r0 = g_row[c.row_off];
    for (int v = tid; v <= n; v += SMALL_THREADS) row[v] = (int32_t)(g_row[c.row_off + v] - r0);
    for (int e = tid; e < nnz; e += SMALL_THREADS) col[e] = (uint16_t)g_col[r0 + e];
    for (int v = tid; v < n; v += SMALL_THREADS) {
      if (REACH) init_d[v] = g_init ? g_init[c.vtx_off + v] : (double)(g_reach[c.vtx_off + v] - 1);
      if (IDENT) ident_d[v] = (double)g_ident[c.vtx_off + v];
    }
    if (tid == 0) s_next = item.s_begin;
    // zero every group's accumulator
    for (int x = tid; x < ng * n; x += SMALL_THREADS) {
      const int gi = x / n, v = x - gi * n;
      double *a = (double *)(p + per * gi + small_acc_offset(n));
      a[v] = 0.0;
    }
    __syncthreads();
    // whole warps per group, every warp in one: group k takes warps
    // [k W / ng, (k + 1) W / ng), so sizes differ by at most one warp, and
    // each group claims its next source from the item (a larger group
    // finishes its sources sooner and takes more of them)
    constexpr int W = SMALL_THREADS / 32;
    const int warp = tid >> 5;
    const int gid = ((warp + 1) * ng - 1) / W;
    const int w0 = (gid * W) / ng, w1 = ((gid + 1) * W) / ng;
    Group g{tid - w0 * 32, (w1 - w0) * 32, 1 + gid};
    unsigned char *q = p + per * gid;
    SrcState<FP32, uint16_t> st;
    st.d = (int32_t *)q;
    q += align16((size_t)n * 4);
    st.queue = (uint16_t *)q;
    q += align16((size_t)n * 2);
    st.dmask = (uint32_t *)q;
    q += align16((size_t)n * 4);
    st.sig = (double *)q;
    st.coef = (typename CoefT<FP32>::type *)q;  // same storage (see bcreach_source)
    q += align16((size_t)n * 8);
    double *acc = (double *)q;
    int32_t *lv = lvl_scratch + ((size_t)blockIdx.x * SMALL_MAX_GROUPS + gid) * (size_t)lvl_stride * 2;
    st.lvl_start = lv;
    st.lvl_exp = lv + lvl_stride;
    st.qtail = &s_qtail[gid];
    st.red = s_red[gid];
    Weights wt{nullptr, nullptr, init_d, ident_d, g_init != nullptr};
    for (;;) {
      // every member reads the claim before the source's first group wait,
      // so the next claim cannot overwrite it early
      if (g.rank == 0) s_claim[gid] = atomicAdd(&s_next, 1);
      g.sync();
      const int i = s_claim[gid];
      if (i >= item.s_end) break;
      const int32_t s = (srcs && c.src_off >= 0) ? (int32_t)srcs[c.src_off + i] : i;
      bcreach_source<REACH, IDENT, FP32, false>(g, s, n, row, col, wt, st, acc, c.fan, err, nullptr, dag);
    }
    __syncthreads();
    // add the groups' accumulators in group order and flush once
    for (int v = tid; v < n; v += SMALL_THREADS) {
      double t = 0.0;
      for (int gi = 0; gi < ng; gi++)
        t += ((const double *)(p + per * gi + small_acc_offset(n)))[v];
      if (t != 0.0) atomicAdd(bcp + c.vtx_off + v, t);
    }
    __syncthreads();
  }
  if (dag_total && dag) atomicAdd(dag_total, dag);
}

// ---------------------------------------------------------- large path
struct LargeSrc {
  int32_t comp;
  int32_t s;
};

// Per-CTA global scratch of the large path: each array holds grid * nmax
// entries, CTA b owning [b * nmax, (b+1) * nmax) (lvl arrays: nmax + 2).
struct LargeScratch {
  int32_t *d;      // -1 between sources
  int32_t *queue;
  double *sig;     // 0 between sources
  double *coef;    // 8 bytes per vertex in both precisions
  double *acc;     // 0 between components
  int32_t *lvl_start;
  int32_t *lvl_exp;
  int64_t nmax;
};

template <bool REACH, bool IDENT, bool FP32>
__global__ void __launch_bounds__(LARGE_THREADS) k_bcreach_large(
    const LargeSrc *__restrict__ work, int64_t nwork, unsigned long long *counter, const CompDesc *__restrict__ comps,
    const int64_t *__restrict__ g_row, const int32_t *__restrict__ g_col, const int32_t *__restrict__ g_reach,
    const int32_t *__restrict__ g_ident, const double *__restrict__ g_init, double *bcp, LargeScratch sc, int *err,
    Debug dbg_in, int use_dbg, unsigned long long *dag_total, int *lmax) {
  __shared__ unsigned long long s_idx;
  __shared__ int s_qtail;
  __shared__ double s_red[16];
  const size_t b = blockIdx.x;
  SrcState<FP32> st;
  st.d = sc.d + b * sc.nmax;
  st.queue = sc.queue + b * sc.nmax;
  st.dmask = nullptr;
  st.sig = sc.sig + b * sc.nmax;
  st.coef = (typename CoefT<FP32>::type *)(sc.coef + b * sc.nmax);
  double *acc = sc.acc + b * sc.nmax;
  st.lvl_start = sc.lvl_start + b * (sc.nmax + 2);
  st.lvl_exp = sc.lvl_exp + b * (sc.nmax + 2);
  st.qtail = &s_qtail;
  st.red = s_red;
  Group g{(int)threadIdx.x, (int)blockDim.x, 0};
  unsigned long long dag = 0;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(counter, 1ull);
    __syncthreads();
    const unsigned long long idx = s_idx;
    __syncthreads();
    const int next = idx < (unsigned long long)nwork ? work[idx].comp : -1;
    if (next != cur && cur >= 0) {  // flush the accumulator of the previous component
      const CompDesc c = comps[cur];
      for (int v = threadIdx.x; v < c.n; v += blockDim.x) {
        if (acc[v] != 0.0) atomicAdd(bcp + c.vtx_off + v, acc[v]);
        acc[v] = 0.0;
      }
      __syncthreads();
    }
    cur = next;
    if (next < 0) break;
    const CompDesc c = comps[cur];
    Weights wt{REACH && !g_init ? g_reach + c.vtx_off : nullptr, IDENT ? g_ident + c.vtx_off : nullptr,
               REACH && g_init ? g_init + c.vtx_off : nullptr, nullptr, g_init != nullptr};
    bcreach_source<REACH, IDENT, FP32, true>(g, work[idx].s, c.n, g_row + c.row_off, g_col, wt, st, acc, c.fan, err,
                                             use_dbg ? &dbg_in : nullptr, dag, lmax);
  }
  if (dag_total && dag) atomicAdd(dag_total, dag);
}

// bytes of global scratch per large-path CTA
static size_t large_scratch_bytes(int64_t nmax) { return (size_t)nmax * (4 + 4 + 8 + 8 + 8) + (size_t)(nmax + 2) * 8; }

// ---------------------------------------------------------- host side
// The shared-memory kernel's attribute (opt-in shared memory) and its
// occupancy per shared-memory size are queried once per device and cached:
// each query is a driver call on the host's critical path.
static std::mutex g_small_mu;
static std::map<long long, int> g_small_occ;  // (variant, device, smem) -> CTAs per SM

template <bool R, bool I, bool F>
static int small_prepare(int device) {
  static std::mutex mu;
  static std::set<int> done;
  std::lock_guard<std::mutex> lk(mu);
  if (!done.count(device)) {
    BCS_CUDA(cudaFuncSetAttribute(k_bcreach_small<R, I, F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SMALL_SMEM));
    done.insert(device);
  }
  return BCS_OK;
}

// The reciprocal table, filled once per device (on the legacy stream, which
// orders it before any later work of every blocking stream).
static int recip_table_ready(int device) {
  static std::mutex mu;
  static std::set<int> done;
  std::lock_guard<std::mutex> lk(mu);
  if (!done.count(device)) {
    k_fill_recip_table<<<4, 256>>>();
    BCS_CUDA(cudaGetLastError());
    BCS_CUDA(cudaDeviceSynchronize());
    done.insert(device);
  }
  return BCS_OK;
}

// CTAs of the shared-memory kernel that fit on one SM with `smem` bytes each
template <bool R, bool I, bool F>
static int small_ctas_per_sm(int device, size_t smem, int *out) {
  const long long key = ((long long)(R * 4 + I * 2 + F) << 48) | ((long long)device << 32) | (long long)smem;
  {
    std::lock_guard<std::mutex> lk(g_small_mu);
    auto it = g_small_occ.find(key);
    if (it != g_small_occ.end()) {
      *out = it->second;
      return BCS_OK;
    }
  }
  BCS_TRY((small_prepare<R, I, F>(device)));
  BCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_bcreach_small<R, I, F>, SMALL_THREADS, smem));
  if (*out < 1) *out = 1;
  std::lock_guard<std::mutex> lk(g_small_mu);
  g_small_occ[key] = *out;
  return BCS_OK;
}

template <bool R, bool I, bool F>
static int launch_small_t(Ctx &ctx, int grid, size_t smem, const SmallItem *items, int nitems, int *counter,
                          const CompDesc *comps, const BcInput &in, const int64_t *srcs, int32_t *lvl, int lvl_stride,
                          int *err, unsigned long long *dag) {
  BCS_TRY((small_prepare<R, I, F>(ctx.device)));
  BCS_TRY(recip_table_ready(ctx.device));
  auto kern = k_bcreach_small<R, I, F>;
  kern<<<grid, SMALL_THREADS, smem, ctx.stream>>>(items, nitems, counter, comps, in.row, in.col, in.reach, in.ident,
                                                 in.init, srcs, in.bcp, lvl, lvl_stride, err, dag);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

template <bool R, bool I, bool F>
static int launch_large_t(Ctx &ctx, int grid, const LargeSrc *work, int64_t nwork, unsigned long long *counter,
                          const CompDesc *comps, const BcInput &in, const LargeScratch &sc, int *err,
                          const Debug &dbg, int use_dbg, unsigned long long *dag, int *lmax = nullptr) {
  k_bcreach_large<R, I, F><<<grid, LARGE_THREADS, 0, ctx.stream>>>(work, nwork, counter, comps, in.row, in.col,
                                                                  in.reach, in.ident, in.init, in.bcp, sc, err, dbg,
                                                                  use_dbg, dag, lmax);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

// The small-path work splits the autotuner tries: most sources a CTA runs
// at once, and the shared-memory budget per CTA (100 KB: 2 CTAs per SM,
// 72 KB: 3, 54 KB: 4).  The default is the first.
struct Split {
  int ng_cap;
  size_t budget;
};
static const Split TUNE_SPLITS[] = {{8, SMALL_SMEM}, {8, 72 * 1024}, {8, 54 * 1024}, {4, SMALL_SMEM}};

// Process-wide cache of the autotuner's choice (index + 1 into TUNE_SPLITS)
// per shape bucket.
static std::mutex g_tune_mu;
static std::map<long long, int> g_tune;

static int tuned_split(long long key) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  return it == g_tune.end() ? 0 : it->second;
}

static void remember_split(long long key, int choice) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = choice;
}

// Besides the small-path work split, the autotuner picks, by timing each
// candidate once per shape bucket and caching the fastest:
//  * the small/large threshold: the shared memory a piece may need for one
//    source to take the small path (SMALL_LIMITS); pieces above it take the
//    large-piece path.  Timed over the pieces that fit the largest limit.
//  * the kernel of each large piece: the whole-GPU kernel (where the
//    piece's depth allows it), 32-source batches (where its depth is below
//    4 x MS_DEPTH_LIMIT: their cost grows with the levels of a batch), or
//    one source per CTA, each timed on a sample of the piece's sources that
//    fills the GPU for that kernel.
// Every candidate runs into a scratch accumulator; the call then runs with
// the choice.  Without the autotuner the fixed limits above decide.
static const size_t SMALL_LIMITS[] = {SMALL_SMEM, 64 * 1024, 40 * 1024};
static std::map<long long, int> g_tune_limit, g_tune_large;

static int tuned_in(std::map<long long, int> &m, long long key) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = m.find(key);
  return it == m.end() ? 0 : it->second;
}

static void remember_in(std::map<long long, int> &m, long long key, int v) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  m[key] = v;
}

static long long bits_of(double x) { return x < 1.0 ? 0 : (long long)std::log2(x) + 1; }

// One Bc-Reach run over `comps` into a scratch accumulator, timed; the
// call's statistics are left as they were.
static int time_candidate(Ctx &ctx, const std::vector<CompDesc> &comps, const BcInput &in, const BcPlanOpts &po,
                          double *ms) {
  int64_t ntot = 1;
  for (const CompDesc &c : comps) ntot = std::max<int64_t>(ntot, c.vtx_off + c.n);
  DBuf<double> scratch;
  BCS_TRY(scratch.alloc(ntot, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(scratch.p, 0, ntot * sizeof(double), ctx.stream));
  BcInput in2 = in;
  in2.bcp = scratch.p;
  const bool at = ctx.autotune;
  const bcs_stats saved = ctx.stats;
  const size_t npend = ctx.pending.size();
  ctx.autotune = false;
  StageTimer t(ctx.stream);
  t.start();
  const int rc = run_bcreach(ctx, comps, in2, po);
  *ms = t.stop_ms();
  ctx.autotune = at;
  ctx.stats = saved;
  for (size_t i = npend; i < ctx.pending.size(); i++) {  // the candidate's stage times are not the call's
    cudaEventSynchronize(ctx.pending[i].b);
    cudaEventDestroy(ctx.pending[i].a);
    cudaEventDestroy(ctx.pending[i].b);
  }
  ctx.pending.resize(npend);
  return rc;
}

// Times the large-piece kernels on samples of one piece's sources (every
// vertex a source) and sets *choice to the fastest per source.  The samples
// are what each kernel sees in a full run: consecutive vertices of the BFS
// order from the piece's first vertex (d_ord) for the whole-GPU kernel,
// consecutive ids for the others.
static int tune_large_piece(Ctx &ctx, const CompDesc &c, const BcInput &in, const BcPlanOpts &po, bool wide_ok,
                            int depth, const int32_t *d_ord, int *choice) {
  struct Cand {
    int path;
    int64_t m;
  };
  const int64_t ns = nsrc_of(c), sms = ctx.num_sms;
  std::vector<Cand> cands;
  if (wide_ok) cands.push_back({LARGE_PATH_WIDE, 512});
  if (depth <= 4 * MS_DEPTH_LIMIT) cands.push_back({LARGE_PATH_BATCHED, 32 * sms});
  cands.push_back({LARGE_PATH_PER_SOURCE, 6 * sms});
  *choice = cands[0].path;
  if (cands.size() == 1) return BCS_OK;
  double best = 0.0;
  for (const Cand &cd : cands) {
    const int64_t m = std::min(cd.m, std::max<int64_t>(1, ns / 4));
    const int64_t at = (ns - m) / 2;
    std::vector<int64_t> src(m);
    if (cd.path == LARGE_PATH_WIDE) {
      std::vector<int32_t> h(m);
      BCS_CUDA(cudaMemcpyAsync(h.data(), d_ord + at, m * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx.stream));
      BCS_CUDA(cudaStreamSynchronize(ctx.stream));
      for (int64_t i = 0; i < m; i++) src[i] = h[i];
    } else {
      for (int64_t i = 0; i < m; i++) src[i] = at + i;
    }
    BcPlanOpts p2 = po;
    p2.sources = src.data();
    p2.nsources = m;
    p2.large_path = cd.path;
    p2.force_large = true;
    double ms = 0.0;
    BCS_TRY(time_candidate(ctx, std::vector<CompDesc>{c}, in, p2, &ms));
    const double rate = (double)m / std::max(ms, 1e-3);
    if (std::getenv("BCS_TRACE"))
      std::fprintf(stderr, "[bcs] tune large piece n=%d kernel %d: %lld sources in %.3f ms\n", c.n, cd.path,
                   (long long)m, ms);
    if (rate > best) {
      best = rate;
      *choice = cd.path;
    }
  }
  return BCS_OK;
}

int run_bcreach(Ctx &ctx, const std::vector<CompDesc> &comps_in, const BcInput &in, const BcPlanOpts &po) {
  Tracer tr("bcreach", ctx.stream);
  const bool R = in.reach != nullptr || in.init != nullptr, I = in.ident != nullptr, F = po.fp32_delta;
  const bool dbg = po.dbg_d || po.dbg_sig || po.dbg_exp || po.dbg_delta;
  const int64_t C = (int64_t)comps_in.size();
  if (po.sources && (C != 1 || po.srcmap)) {
    set_error("a source list needs exactly one component and no source map");
    return BCS_EINVAL;
  }
  // a host source list is the one component's source map (uploaded below)
  std::vector<CompDesc> comps_src;
  if (po.sources) {
    comps_src = comps_in;
    comps_src[0].src_off = 0;
    comps_src[0].nsrc = (int32_t)po.nsources;
  }
  const std::vector<CompDesc> &comps = po.sources ? comps_src : comps_in;
  // the large-piece kernel, if fixed: by the caller, or by BCS_LARGE_PATH
  // (wide|batched|per_source; wide_all, for tests: every piece runs on the
  // large-piece path, and on the whole-GPU kernel wherever that can take it)
  int lp_mode = po.large_path;
  bool all_large = false;
  if (const char *e = std::getenv("BCS_LARGE_PATH")) {
    if (!std::strcmp(e, "wide_all") || !std::strcmp(e, "mid_all")) all_large = true;
    if (!std::strcmp(e, "mid_all")) lp_mode = LARGE_PATH_MID;
    if (!std::strcmp(e, "wide") || !std::strcmp(e, "wide_all")) lp_mode = LARGE_PATH_WIDE;
    if (!std::strcmp(e, "batched")) lp_mode = LARGE_PATH_BATCHED;
    if (!std::strcmp(e, "per_source")) lp_mode = LARGE_PATH_PER_SOURCE;
    if (!std::strcmp(e, "mid")) lp_mode = LARGE_PATH_MID;
  }
  const bool tune = ctx.autotune && lp_mode == LARGE_PATH_AUTO && !dbg && !po.sources && !po.srcmap &&
                    !po.force_large && !po.per_source_large;
  // the small/large threshold
  size_t small_limit = po.small_limit ? po.small_limit : SMALL_SMEM;
  if (tune && !po.small_limit) {
    std::vector<CompDesc> elig;  // pieces that fit the largest limit
    double cost = 0.0, band = 0.0;
    const size_t lowest = SMALL_LIMITS[sizeof(SMALL_LIMITS) / sizeof(SMALL_LIMITS[0]) - 1];
    for (const CompDesc &c : comps) {
      const int64_t ns = nsrc_of(c);
      if (c.n < 2 || ns == 0 || c.n > 65535) continue;
      const size_t s1 = small_smem_bytes(c.n, c.nnz, 1, R, I);
      if (s1 > SMALL_SMEM) continue;
      elig.push_back(c);
      cost += (double)ns * (double)(c.nnz + c.n);
      if (s1 > lowest) band += (double)ns * (double)(c.nnz + c.n);
    }
    if (band > 0.0) {
      const long long key = ((long long)(R * 2 + I) << 40) | (bits_of(cost) << 20) | bits_of(band);
      int ch = tuned_in(g_tune_limit, key);
      if (!ch) {
        double best = 1e300;
        for (int k = 0; k < (int)(sizeof(SMALL_LIMITS) / sizeof(SMALL_LIMITS[0])); k++) {
          BcPlanOpts p2 = po;
          p2.small_limit = SMALL_LIMITS[k];
          double ms = 0.0;
          BCS_TRY(time_candidate(ctx, elig, in, p2, &ms));
          if (std::getenv("BCS_TRACE"))
            std::fprintf(stderr, "[bcs] tune small/large threshold %zu B: %.3f ms\n", SMALL_LIMITS[k], ms);
          if (ms < best) {
            best = ms;
            ch = k + 1;
          }
        }
        remember_in(g_tune_limit, key, ch);
      }
      small_limit = SMALL_LIMITS[ch - 1];
      ctx.stats.tuned |= 1;
    }
  }
  ctx.stats.small_limit = (int64_t)small_limit;
  std::vector<SmallItem> items;
  std::vector<LargeSrc> work;
  std::vector<int32_t> large, small;
  int64_t nmax_large = 0, nmax_small = 0;
  double work_se = 0.0, work_sv = 0.0, total_small_cost = 0.0;
  for (int64_t ci = 0; ci < C; ci++) {
    const CompDesc &c = comps[ci];
    if (c.n < 2) continue;
    const int64_t ns = nsrc_of(c);
    if (ns == 0) continue;
    work_se += (double)ns * (double)c.nnz;
    work_sv += (double)ns * (double)c.n;
    const bool fits = !po.force_large && !all_large && !dbg && c.n <= 65535 &&
                      small_smem_bytes(c.n, c.nnz, 1, R, I) <= small_limit;
    if (fits) {
      small.push_back((int32_t)ci);
      total_small_cost += (double)ns * (double)(c.nnz + c.n);
      nmax_small = std::max<int64_t>(nmax_small, c.n);
    } else {
      large.push_back((int32_t)ci);
      nmax_large = std::max<int64_t>(nmax_large, c.n);
    }
  }
  // The small-path work split: a piece runs up to `ng_cap` sources at once
  // per CTA (the most that fit in SMALL_SMEM); the launch takes exactly the
  // shared memory its largest item needs, so occupancy follows the plan.
  // Items of similar cost go first-largest into a persistent queue.
  // pieces by cost class (the power of two of n + nnz), largest first, in
  // piece order within a class: the persistent queue hands out the longest
  // items first.  A counting sort: one pass, no comparisons.
  {
    int64_t cnt[65] = {0};
    std::vector<int32_t> cls(small.size());
    for (size_t k = 0; k < small.size(); k++) {
      const CompDesc &c = comps[small[k]];
      cls[k] = 63 - __builtin_clzll((unsigned long long)(c.nnz + c.n) | 1ull);
      cnt[cls[k]]++;
    }
    int64_t off[65], o = 0;
    for (int b = 64; b >= 0; b--) {
      off[b] = o;
      o += cnt[b];
    }
    std::vector<int32_t> sorted(small.size());
    for (size_t k = 0; k < small.size(); k++) sorted[off[cls[k]]++] = small[k];
    small.swap(sorted);
  }
  auto plan_small = [&](int ng_cap, size_t budget, std::vector<SmallItem> &out, size_t &smem, int &grid) -> int {
    out.clear();
    smem = 0;
    std::vector<int> ngs(small.size());
    for (size_t k = 0; k < small.size(); k++) {
      const CompDesc &c = comps[small[k]];
      int ng = 1;  // a piece that does not fit the budget even alone still runs (up to SMALL_SMEM)
      for (int cand = ng_cap; cand >= 1; cand--)
        if (small_smem_bytes(c.n, c.nnz, cand, R, I) <= budget) {
          ng = cand;
          break;
        }
      ngs[k] = ng;
      smem = std::max(smem, small_smem_bytes(c.n, c.nnz, ng, R, I));
    }
    int per_sm = 1;
    BCS_TRY(BCS_DISPATCH3(small_ctas_per_sm, R, I, F, ctx.device, smem, &per_sm));
    grid = ctx.num_sms * per_sm;
    const double target = total_small_cost / (double)((int64_t)grid * SMALL_MAX_GROUPS) + 1.0;
    for (size_t k = 0; k < small.size(); k++) {
      const CompDesc &c = comps[small[k]];
      const int ng = ngs[k];
      const int64_t ns = nsrc_of(c);
      int64_t chunk = (int64_t)std::max(1.0, target / (double)(c.nnz + c.n));
      chunk = ((chunk + ng - 1) / ng) * ng;
      for (int64_t b = 0; b < ns; b += chunk)
        out.push_back(SmallItem{small[k], (int32_t)b, (int32_t)std::min<int64_t>(ns, b + chunk), ng});
    }
    grid = (int)std::min<int64_t>(grid, (int64_t)out.size());
    return BCS_OK;
  };
  // Large pieces of small BFS depth: the whole GPU on one 32-source batch at
  // a time (wide.cu), the sources taken in the BFS order of the piece from
  // its first vertex (neighbouring sources share most of their levels).  The
  // BFS from that vertex also bounds the depth: no source reaches deeper than
  // twice its eccentricity.  BCS_LARGE_PATH=wide takes every large piece
  // whose depth allows it; batched|per_source take none.
  struct WidePiece {
    int32_t ci;
    std::shared_ptr<DBuf<int32_t>> order;
    int32_t nsrc;
    int depth_bound;
  };
  std::vector<WidePiece> wide;
  // large pieces the autotuner gave to 32-source batches, or to one source per CTA
  std::vector<int32_t> ms_tuned, ps_tuned;
  // Mid-size pieces (at most MID_MAX_N vertices, every vertex a source or
  // one piece with a source list): one 64-source batch per CTA (wide.cu),
  // when forced, or when they are many enough to keep every CTA busy.
  std::vector<int32_t> mid;
  if (!dbg && !po.per_source_large && !po.srcmap &&
      (lp_mode == LARGE_PATH_MID || (lp_mode == LARGE_PATH_AUTO && MID_BY_DEFAULT))) {
    std::vector<int32_t> rest;
    int64_t units = 0;
    for (int32_t ci : large) {
      const CompDesc &c = comps[ci];
      if (c.n <= MID_MAX_N && (c.src_off < 0 || po.sources)) {
        mid.push_back(ci);
        units += (nsrc_of(c) + 63) / 64;
      } else {
        rest.push_back(ci);
      }
    }
    if (lp_mode == LARGE_PATH_MID || units >= MID_MIN_UNITS_PER_SM * (int64_t)ctx.num_sms) {
      large.swap(rest);
    } else {
      mid.clear();
    }
  }
  {
    const bool force_wide = lp_mode == LARGE_PATH_WIDE;
    const bool no_wide = lp_mode == LARGE_PATH_BATCHED || lp_mode == LARGE_PATH_PER_SOURCE;
    std::vector<int32_t> rest;
    for (int32_t ci : large) {
      const CompDesc &c = comps[ci];
      // tuning pays only over many sources
      const bool tune_this = tune && c.src_off < 0 && nsrc_of(c) >= 24LL * ctx.num_sms;
      const bool cand = !no_wide && !dbg && !po.per_source_large && (c.src_off < 0 || po.sources) &&
                        (force_wide || tune_this || c.n >= WIDE_MIN_N);
      if (!cand) {
        rest.push_back(ci);
        continue;
      }
      auto ord = std::make_shared<DBuf<int32_t>>();
      BCS_TRY(ord->alloc(c.n, ctx.stream));
      int depth = 0;
      int64_t reached = 0;
      BCS_TRY(bfs_queue(ctx, in.row + c.row_off, in.col, c.n, 0, ord->p, &depth, &reached));
      if (reached != c.n && c.row_off == 0) {
        // a whole graph of several components (the plain calls; pieces are
        // connected): every component searched from its smallest vertex
        DevGraph g{c.n, c.nnz, in.row, in.col};
        BCS_TRY(bfs_queue_components(ctx, g, ord->p, &depth));
        reached = c.n;
      }
      // every source's BFS depth is at most twice its component's root's
      const int bound = 2 * depth + 2;
      const bool wide_ok = bound <= wide_depth_limit() && reached == c.n;
      int choice = LARGE_PATH_AUTO;
      if (tune_this) {
        const long long key = ((long long)(R * 2 + I) << 40) | (bits_of(c.n) << 24) |
                              (bits_of((double)c.nnz / c.n) << 16) | bits_of(depth);
        choice = tuned_in(g_tune_large, key);
        if (!choice) {
          BCS_TRY(tune_large_piece(ctx, c, in, po, wide_ok, depth, ord->p, &choice));
          remember_in(g_tune_large, key, choice);
        }
        ctx.stats.tuned |= 1ll << choice;
        if (choice == LARGE_PATH_BATCHED) ms_tuned.push_back(ci);
        if (choice == LARGE_PATH_PER_SOURCE) ps_tuned.push_back(ci);
        if (choice != LARGE_PATH_WIDE) continue;
      }
      const bool heuristic = !force_wide && choice == LARGE_PATH_AUTO;
      if (!wide_ok || (heuristic && (depth > WIDE_MAX_ECC || c.n < WIDE_MIN_N))) {
        rest.push_back(ci);
        continue;
      }
      int32_t ns = (int32_t)nsrc_of(c);
      if (po.sources) {  // the caller's sources, in the caller's order
        std::vector<int32_t> h(po.nsources);
        for (int64_t i = 0; i < po.nsources; i++) h[i] = (int32_t)po.sources[i];
        BCS_TRY(ord->alloc(std::max<int64_t>(po.nsources, 1), ctx.stream));
        BCS_CUDA(cudaMemcpyAsync(ord->p, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx.stream));
        BCS_CUDA(cudaStreamSynchronize(ctx.stream));
        ns = (int32_t)po.nsources;
      }
      wide.push_back(WidePiece{ci, ord, ns, bound});
    }
    large.swap(rest);
  }
  // Large pieces: 32 sources per CTA when there are enough batches to give
  // every SM two of them and their scratch fits at least one CTA per SM,
  // else one source per CTA (more CTAs in flight).
  // BCS_LARGE_PATH=batched|per_source overrides the choice.
  int64_t nbatches = 0;
  for (int32_t ci : large) nbatches += (nsrc_of(comps[ci]) + 31) / 32;
  bool use_ms = !large.empty() && !dbg && !po.per_source_large && !po.srcmap && nbatches >= 2 * (int64_t)ctx.num_sms;
  if (use_ms) {
    // its per-CTA scratch grows with the piece: with fewer CTAs than SMs the
    // batches serialise (high-diameter graphs of millions of vertices)
    int64_t fit = 0;
    BCS_TRY(ms_ctas_that_fit(nmax_large, &fit));
    if (fit < ctx.num_sms) use_ms = false;
  }
  bool forced = false;  // a fixed large path (BCS_LARGE_PATH, or the caller's) overrides the choice
  if (!large.empty() && !dbg && !po.per_source_large && !po.srcmap) {
    if (lp_mode == LARGE_PATH_BATCHED) use_ms = forced = true;
    if (lp_mode == LARGE_PATH_PER_SOURCE) {
      use_ms = false;
      forced = true;
    }
  }
  // the one-source-per-CTA list for large pieces, from the `skip`-th source
  // of each piece on (debug output, the depth probe's remainder, or the
  // fallback when a graph is too deep for the 32-source kernel)
  // the sources of large pieces with a device source map, on the host
  std::vector<std::vector<int64_t>> large_map(po.srcmap ? large.size() : 0);
  if (po.srcmap) {
    for (size_t k = 0; k < large.size(); k++) {
      const CompDesc &c = comps[large[k]];
      if (c.src_off < 0) continue;
      large_map[k].resize(nsrc_of(c));
      if (!large_map[k].empty())
        BCS_CUDA(cudaMemcpyAsync(large_map[k].data(), po.srcmap + c.src_off, large_map[k].size() * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, ctx.stream));
    }
    BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  }
  auto large_src = [&](size_t k, int64_t i) -> int32_t {
    if (po.sources) return (int32_t)po.sources[i];
    if (po.srcmap && comps[large[k]].src_off >= 0) return (int32_t)large_map[k][i];
    return (int32_t)i;
  };
  auto build_work = [&](int64_t skip) {
    work.clear();
    for (size_t k = 0; k < large.size(); k++) {
      const int64_t ns = nsrc_of(comps[large[k]]);
      for (int64_t i = skip; i < ns; i++) work.push_back(LargeSrc{large[k], large_src(k, i)});
    }
  };
  if (!use_ms) build_work(0);
  tr.mark("classify");
  int ng_cap = SMALL_MAX_GROUPS;
  size_t budget = SMALL_SMEM;
  size_t smem_small = 0;
  int grid_small = 0;
  // the autotuner's choice for this shape bucket, if it has one already
  long long tune_key = 0;
  int tuned = 0;
  if (ctx.autotune && !small.empty()) {
    const int kb = 64 - __builtin_clzll((unsigned long long)std::max<int64_t>(nmax_small, 1));
    const int wb = (int)std::log2(std::max(total_small_cost, 1.0));
    tune_key = ((long long)(R * 4 + I * 2 + F) << 40) | ((long long)kb << 20) | (long long)wb;
    tuned = tuned_split(tune_key);
    if (tuned) {
      ng_cap = TUNE_SPLITS[tuned - 1].ng_cap;
      budget = TUNE_SPLITS[tuned - 1].budget;
    }
  }
  if (!small.empty()) BCS_TRY(plan_small(ng_cap, budget, items, smem_small, grid_small));
  tr.mark("plan0");
  ctx.stats.n_small_items = (int64_t)items.size();
  ctx.stats.n_large_sources = 0;
  for (int32_t ci : large) ctx.stats.n_large_sources += nsrc_of(comps[ci]);
  for (int32_t ci : ms_tuned) ctx.stats.n_large_sources += nsrc_of(comps[ci]);
  for (int32_t ci : ps_tuned) ctx.stats.n_large_sources += nsrc_of(comps[ci]);
  for (int32_t ci : mid) ctx.stats.n_large_sources += nsrc_of(comps[ci]);
  for (const WidePiece &wp : wide) ctx.stats.n_large_sources += wp.nsrc;
  ctx.stats.work_sources_entries = work_se;
  ctx.stats.work_sources_vertices = work_sv;
  if (small.empty() && large.empty() && wide.empty() && ms_tuned.empty() && ps_tuned.empty() && mid.empty())
    return BCS_OK;

  DBuf<CompDesc> d_comps;
  DBuf<int> d_err;
  DBuf<unsigned long long> d_dag;
  BCS_TRY(d_comps.alloc(C, ctx.stream));
  BCS_TRY(d_err.alloc(4, ctx.stream));
  BCS_TRY(d_dag.alloc(1, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(d_dag.p, 0, sizeof(unsigned long long), ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(d_comps.p, comps.data(), C * sizeof(CompDesc), cudaMemcpyHostToDevice, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(d_err.p, 0, 4 * sizeof(int), ctx.stream));
  DBuf<int64_t> d_srcs;
  if (po.sources && !items.empty()) {
    BCS_TRY(d_srcs.alloc(po.nsources, ctx.stream));
    BCS_CUDA(cudaMemcpyAsync(d_srcs.p, po.sources, po.nsources * sizeof(int64_t), cudaMemcpyHostToDevice, ctx.stream));
  }
  tr.mark("upload");
  if (!items.empty()) {
    StageTimer tm(ctx.stream);
    tm.start();
    const int lvl_stride = (int)nmax_small + 2;
    const size_t grid_cap = (size_t)ctx.num_sms * (2048 / SMALL_THREADS);  // resident CTAs per SM at most
    DBuf<int32_t> lvl;
    BCS_TRY(lvl.alloc(grid_cap * SMALL_MAX_GROUPS * lvl_stride * 2, ctx.stream));
    DBuf<SmallItem> d_items;
    BCS_TRY(d_items.alloc(std::max<size_t>(items.size() * 2, 1), ctx.stream));
    auto run_small = [&](const std::vector<SmallItem> &its, size_t smem, int grid, double *target) -> int {
      if (its.size() > d_items.n) BCS_TRY(d_items.alloc(its.size(), ctx.stream));
      BCS_CUDA(cudaMemcpyAsync(d_items.p, its.data(), its.size() * sizeof(SmallItem), cudaMemcpyHostToDevice,
                               ctx.stream));
      BCS_CUDA(cudaMemsetAsync(d_err.p + 1, 0, sizeof(int), ctx.stream));
      BcInput tin = in;
      tin.bcp = target;
      return BCS_DISPATCH3(launch_small_t, R, I, F, ctx, grid, smem, d_items.p, (int)its.size(), d_err.p + 1,
                           d_comps.p, tin, po.sources ? d_srcs.p : po.srcmap, lvl.p, lvl_stride, d_err.p, d_dag.p);
    };
    tr.mark("alloc");
    if (ctx.autotune && tuned == 0) {
      // tune once per shape bucket: time each split into a scratch
      // accumulator and keep the fastest
      int best = 0;
      {
        int64_t ntot = 0;
        for (const CompDesc &c : comps) ntot = std::max<int64_t>(ntot, c.vtx_off + c.n);
        DBuf<double> scratch;
        BCS_TRY(scratch.alloc(ntot, ctx.stream));
        double best_ms = 1e30;
        for (int cand = 0; cand < (int)(sizeof(TUNE_SPLITS) / sizeof(TUNE_SPLITS[0])); cand++) {
          std::vector<SmallItem> its;
          size_t sm = 0;
          int gr = 0;
          BCS_TRY(plan_small(TUNE_SPLITS[cand].ng_cap, TUNE_SPLITS[cand].budget, its, sm, gr));
          BCS_CUDA(cudaMemsetAsync(scratch.p, 0, ntot * 8, ctx.stream));
          StageTimer tt(ctx.stream);
          tt.start();
          BCS_TRY(run_small(its, sm, gr, scratch.p));
          const double ms = tt.stop_ms();
          if (std::getenv("BCS_TRACE"))
            std::fprintf(stderr, "[bcs] tune small split ng_cap=%d budget=%zu: %zu items, %d CTAs, %zu B smem, %.3f ms\n",
                         TUNE_SPLITS[cand].ng_cap, TUNE_SPLITS[cand].budget, its.size(), gr, sm, ms);
          if (ms < best_ms) {
            best_ms = ms;
            best = cand + 1;
          }
        }
        BCS_CUDA(cudaMemsetAsync(d_dag.p, 0, sizeof(unsigned long long), ctx.stream));
        remember_split(tune_key, best);
      }
      ng_cap = TUNE_SPLITS[best - 1].ng_cap;
      budget = TUNE_SPLITS[best - 1].budget;
      BCS_TRY(plan_small(ng_cap, budget, items, smem_small, grid_small));
      ctx.stats.n_small_items = (int64_t)items.size();
      tm.start();
    }
    tr.mark("plan");
    ctx.stats.small_ng_cap = ng_cap;
    ctx.stats.small_smem_budget = (int64_t)budget;
    BCS_TRY(run_small(items, smem_small, grid_small, in.bcp));
    tm.stop_into(ctx, &ctx.stats.ms_bcreach_small);
    tr.mark("small");
  }
  for (const WidePiece &wp : wide) {
    StageTimer tm(ctx.stream);
    tm.start();
    BCS_TRY(run_wide(ctx, comps[wp.ci], in, F, wp.order->p, wp.nsrc, wp.depth_bound, d_err.p, d_dag.p));
    tm.stop_into(ctx, &ctx.stats.ms_bcreach_large);
    tr.mark("wide");
  }
  if (!mid.empty()) {
    StageTimer tm(ctx.stream);
    tm.start();
    DBuf<int32_t> d_ord;
    if (po.sources) {  // one piece: its sources, as local ids
      std::vector<int32_t> h(po.nsources);
      for (int64_t i = 0; i < po.nsources; i++) h[i] = (int32_t)po.sources[i];
      BCS_TRY(d_ord.alloc(std::max<int64_t>(po.nsources, 1), ctx.stream));
      BCS_CUDA(cudaMemcpyAsync(d_ord.p, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx.stream));
      BCS_CUDA(cudaStreamSynchronize(ctx.stream));
    }
    std::vector<int32_t> too_deep;
    BCS_TRY(run_mid(ctx, comps, mid, in, F, po.sources ? d_ord.p : nullptr, d_comps.p, d_err.p, d_dag.p, &too_deep));
    // pieces too deep for its levels (or not connected): one source per CTA
    ps_tuned.insert(ps_tuned.end(), too_deep.begin(), too_deep.end());
    tm.stop_into(ctx, &ctx.stats.ms_bcreach_large);
    tr.mark("mid");
  }
  // one source per CTA over the given list; *d_lmax (optional) receives the
  // deepest BFS level any of them reached
  auto run_per_source = [&](const std::vector<LargeSrc> &w, int *d_lmax) -> int {
    StageTimer tm(ctx.stream);
    tm.start();
    DBuf<LargeSrc> d_work;
    DBuf<unsigned long long> counter;
    BCS_TRY(d_work.alloc(w.size(), ctx.stream));
    BCS_CUDA(cudaMemcpyAsync(d_work.p, w.data(), w.size() * sizeof(LargeSrc), cudaMemcpyHostToDevice, ctx.stream));
    BCS_TRY(counter.alloc(1, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned long long), ctx.stream));
    // CTAs: up to 3 per SM, fewer when the scratch would take more than half
    // of the free device memory
    size_t free_b = 0, total_b = 0;
    BCS_CUDA(cudaMemGetInfo(&free_b, &total_b));
    int64_t grid = (int64_t)ctx.num_sms * 3;
    grid = std::min<int64_t>(grid, (int64_t)w.size());
    const size_t per = large_scratch_bytes(nmax_large);
    if ((size_t)grid * per > free_b / 2) grid = std::max<int64_t>(1, (int64_t)(free_b / 2 / per));
    const size_t G = (size_t)grid, NM = (size_t)nmax_large;
    DBuf<int32_t> sd, sq, sls, sle;
    DBuf<double> ssig, scoef, sacc;
    BCS_TRY(sd.alloc(G * NM, ctx.stream));
    BCS_TRY(sq.alloc(G * NM, ctx.stream));
    BCS_TRY(ssig.alloc(G * NM, ctx.stream));
    BCS_TRY(scoef.alloc(G * NM, ctx.stream));
    BCS_TRY(sacc.alloc(G * NM, ctx.stream));
    BCS_TRY(sls.alloc(G * (NM + 2), ctx.stream));
    BCS_TRY(sle.alloc(G * (NM + 2), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(sd.p, 0xFF, G * NM * sizeof(int32_t), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(ssig.p, 0, G * NM * sizeof(double), ctx.stream));
    BCS_CUDA(cudaMemsetAsync(sacc.p, 0, G * NM * sizeof(double), ctx.stream));
    LargeScratch sc{sd.p, sq.p, ssig.p, scoef.p, sacc.p, sls.p, sle.p, (int64_t)NM};
    Debug dbgs{po.dbg_d, po.dbg_sig, po.dbg_exp, po.dbg_delta};
    BCS_TRY(BCS_DISPATCH3(launch_large_t, R, I, F, ctx, (int)grid, d_work.p, (int64_t)w.size(), counter.p, d_comps.p,
                          in, sc, d_err.p, dbgs, dbg ? 1 : 0, d_dag.p, d_lmax));
    tm.stop_into(ctx, &ctx.stats.ms_bcreach_large);
    return BCS_OK;
  };
  int64_t skip = 0;  // leading sources of each large piece already done
  if (use_ms && !forced) {
    // Depth probe: the first wave runs one source per CTA (useful work
    // either way) and reports how deep its BFS went.  The 32-source kernel
    // pays per BFS level and queues a vertex once per distinct level its
    // sources reach it at, so on deep graphs (roads, grids) the remaining
    // sources also run one per CTA.
    const int64_t wave = (int64_t)ctx.num_sms * 3;
    skip = std::max<int64_t>(1, wave / (int64_t)large.size());
    std::vector<LargeSrc> probe;
    for (size_t k = 0; k < large.size(); k++) {
      const int64_t ns = nsrc_of(comps[large[k]]);
      for (int64_t i = 0; i < std::min(ns, skip); i++) probe.push_back(LargeSrc{large[k], large_src(k, i)});
    }
    DBuf<int> d_lmax;
    BCS_TRY(d_lmax.alloc(1, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(d_lmax.p, 0, sizeof(int), ctx.stream));
    BCS_TRY(run_per_source(probe, d_lmax.p));
    int lmax = 0;
    BCS_CUDA(cudaMemcpyAsync(&lmax, d_lmax.p, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
    BCS_CUDA(cudaStreamSynchronize(ctx.stream));
    if (lmax > MS_DEPTH_LIMIT) {
      use_ms = false;
      build_work(skip);
    }
  }
  if (use_ms) {
    StageTimer tm(ctx.stream);
    tm.start();
    bool depth_failed = false;
    BCS_TRY(run_ms(ctx, comps, large, in, F, po.sources, po.nsources, skip, d_comps.p, d_err.p, d_dag.p,
                   &depth_failed));
    if (depth_failed) build_work(skip);
    tm.stop_into(ctx, &ctx.stats.ms_bcreach_large);
  }
  // the pieces the autotuner placed (every vertex a source)
  if (!ms_tuned.empty()) {
    StageTimer tm(ctx.stream);
    tm.start();
    bool depth_failed = false;
    BCS_TRY(run_ms(ctx, comps, ms_tuned, in, F, nullptr, 0, 0, d_comps.p, d_err.p, d_dag.p, &depth_failed));
    if (depth_failed) ps_tuned.insert(ps_tuned.end(), ms_tuned.begin(), ms_tuned.end());
    tm.stop_into(ctx, &ctx.stats.ms_bcreach_large);
  }
  for (int32_t ci : ps_tuned) {
    if (po.sources)
      for (int64_t i = 0; i < po.nsources; i++) work.push_back(LargeSrc{ci, (int32_t)po.sources[i]});
    else
      for (int32_t i = 0; i < comps[ci].n; i++) work.push_back(LargeSrc{ci, i});
  }
  if (!work.empty()) BCS_TRY(run_per_source(work, nullptr));
  int h_err = 0;
  unsigned long long h_dag = 0;
  BCS_CUDA(cudaMemcpyAsync(&h_err, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(&h_dag, d_dag.p, sizeof(h_dag), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  ctx.stats.dag_edges += (int64_t)h_dag;
  if (h_err & ERR_OVERFLOW) {
    set_error("shortest-path counts overflowed the FP64 range within one BFS level");
    return BCS_EOVERFLOW;
  }
  if (h_err & ERR_DEPTH) {
    set_error("a Bc-Reach batch needed more BFS levels than its bound");
    return BCS_ECUDA;
  }
  if (h_err & ERR_TIMEOUT) {
    set_error("a grid-wide wait of the Bc-Reach kernel ran out (opts->max_wait)");
    return BCS_ETIMEOUT;
  }
  return BCS_OK;
}

// ------------------------------------------- fixed-scratch plain Brandes
// Plain Brandes (reach = ident = 1) over one component of n vertices on the
// global-memory path, with every piece of device state carved out of a
// caller-given scratch region instead of allocated.  Used by the
// allocation-free entry point.

__global__ void k_fixed_setup(LargeSrc *work, int32_t n, CompDesc *comp, CompDesc desc,
                              unsigned long long *counter, int *err) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) work[i] = LargeSrc{0, i};
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *comp = desc;
    *counter = 0ull;
    *err = 0;
  }
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
static_assert(sizeof(LargeSrc) == FIXED_WORK_ITEM_BYTES, "work item size");
static_assert(sizeof(CompDesc) <= 256, "component descriptor size");

int launch_plain_fixed_scratch(Ctx &ctx, const int64_t *row, const int32_t *col, int32_t n, double *bc,
                               unsigned char *scratch, int64_t nmax, int ctas, bool fp32) {
  const size_t G = (size_t)ctas, N = (size_t)nmax;
  unsigned char *p = scratch;
  LargeSrc *work = (LargeSrc *)p;
  p += up256(N * sizeof(LargeSrc));
  CompDesc *comp = (CompDesc *)p;
  p += up256(sizeof(CompDesc));
  unsigned long long *counter = (unsigned long long *)p;
  p += 256;
  int *err = (int *)p;
  p += 256;
  if (p != scratch + fixed_scratch_arrays_offset(N)) {
    set_error("fixed scratch layout mismatch");
    return BCS_ECUDA;
  }
  LargeScratch sc;
  sc.nmax = (int64_t)N;
  sc.d = (int32_t *)p;
  p += up256(G * N * 4);
  sc.queue = (int32_t *)p;
  p += up256(G * N * 4);
  sc.sig = (double *)p;
  p += up256(G * N * 8);
  sc.coef = (double *)p;
  p += up256(G * N * 8);
  sc.acc = (double *)p;
  p += up256(G * N * 8);
  sc.lvl_start = (int32_t *)p;
  p += up256(G * (N + 2) * 4);
  sc.lvl_exp = (int32_t *)p;
  // the region keeps whatever the previous call left: put back the states
  // the kernel expects at its start (d = -1, sigma = 0, accumulators 0)
  BCS_CUDA(cudaMemsetAsync(sc.d, 0xFF, G * N * 4, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(sc.sig, 0, G * N * 8, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(sc.acc, 0, G * N * 8, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(bc, 0, (size_t)n * sizeof(double), ctx.stream));
  // n bounds the degree, hence the growth of path counts per level
  CompDesc desc{0, 0, n, n, 0, (double)(n > 1 ? n : 1)};
  k_fixed_setup<<<(n + 255) / 256, 256, 0, ctx.stream>>>(work, n, comp, desc, counter, err);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  Debug none{nullptr, nullptr, nullptr, nullptr};
  BcInput in;
  in.row = row;
  in.col = col;
  in.bcp = bc;
  const int grid = (int)std::min<int64_t>(ctas, n);
  if (fp32)
    BCS_TRY((launch_large_t<false, false, true>(ctx, grid, work, n, counter, comp, in, sc, err, none, 0, nullptr)));
  else
    BCS_TRY((launch_large_t<false, false, false>(ctx, grid, work, n, counter, comp, in, sc, err, none, 0, nullptr)));
  int h_err = 0;
  BCS_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  if (h_err & ERR_OVERFLOW) {
    set_error("shortest-path counts overflowed the FP64 range within one BFS level");
    return BCS_EOVERFLOW;
  }
  return BCS_OK;
}

}  // namespace bcs
