// wide.cu - Bc-Reach (Algorithm 2 with the identical-vertex terms of
// Section 3.3.3) on one large piece of small BFS depth, with every SM of the
// GPU working on one batch of 64 (or 32) sources at a time; and the same
// batch on one CTA at a time for many mid-size pieces (k_bcreach_mid, at the
// end of the file).
//
// Why the whole GPU on one batch: on a small-world piece (hundreds of
// thousands of vertices, a handful of BFS levels) the per-vertex records of a
// batch stay in L2 only while few batches are in flight; one batch per GPU
// keeps them there, and the BFS levels are few enough that one grid-wide
// wait per level costs little.
//
// Sources: 64 per batch (32 with BCS_WIDE_SOURCES=32); lane l of every warp
// stands for the batch's sources l and l + 32.  Consecutive vertices of a
// BFS order of the piece form a batch: they sit close together, so most of
// the batch reaches a vertex at the same level, and one visit of its row
// serves many lanes.
//
// Per (vertex v, source s) of the batch:
//   lvl[v][s]   BFS level (one byte, 0xFF = not reached): the sources of a
//               vertex share one or two 32-byte sectors;
//   sig[v][s]   path count sigma_s(v), accumulated by the pushes of the
//               level above (exact int64 while the level's bound allows,
//               else FP64 scaled by a power of two per (level, source));
//   dsum[v][s]  phase 2: sum over the successors w of c[w] = ident[w] (1 +
//               delta_s(w)) / sigma_s(w), accumulated by their pushes.
// Per level, a bitmap of the vertices some source reaches on it.
//
// Phase 1, level L (one pass, one grid-wide wait): every vertex v of the
// level, for the lanes s with lvl[v][s] = L, walks its row (32 entries at a
// time, their level bytes moved through shared memory so each lane reads its
// own source's byte), and for every neighbour u that is not reached, or is
// reached on level L+1, adds sigma_s(v) * ident[v] (1 for the source itself)
// to sig[u][s] (Algorithm 1's path counting, pushed), marking u on level L+1
// (a plain byte store: every writer writes the same value) and in the next
// level's bitmap.  Nothing waits on an atomic's result.
// Phase 2, levels deepest first: delta_s(v) = reach[v] - 1 + sigma_s(v) *
// dsum[v][s] (Eq. 3 in the coefficient form), bc'[v] += reach[s] ident[s]
// delta_s(v) for v != s (summed over the lanes, added once per vertex), and
// c[v] is pushed into dsum of the predecessors (neighbours on level L-1).
// A slot is set back to zero once its vertex is finished, so the next batch
// finds sig and dsum cleared without a sweep.
// Rows longer than WIDE_CH entries are cut into items of WIDE_CH entries,
// spread over all warps; pushing needs no partial sums, so the items of one
// row are independent.
#include <algorithm>
#include <cfloat>
#include <cstdlib>
#include <cstring>

#include "bc_math.cuh"
#include "common.h"
#include "coop.cuh"

namespace bcs {

constexpr int WIDE_THREADS = 256;
constexpr int WIDE_WARPS = WIDE_THREADS / 32;
constexpr int WIDE_CH = 64;  // row entries per item of a long row
// The light rows of a pass are handed out in units of WIDE_UNIT vertices (a
// part of a bitmap word) when the level holds many vertices, so that the
// last warps of the pass finish soon after the others, else whole words
// (fewer grabs of empty units); WIDE_GRAB units (or long-row items) at a time.
constexpr int WIDE_UNIT = 8;
constexpr int WIDE_UPW = 32 / WIDE_UNIT;  // units per bitmap word
constexpr int WIDE_GRAB = 2;
// The work of a pass is handed out from WIDE_SHARDS counters on separate
// cache lines (one address would serialise every warp's grab).
constexpr int WIDE_SHARDS = 8;

struct WideScratch {
  uint8_t *lvl;              // [n][32]
  double *sig;               // [n][32]
  double *dsum;              // [n][32]
  uint32_t *bits;            // [lcap][nwords]
  int32_t *flag;             // [lcap + 1] some vertex on the level
  int32_t *wctr;             // [2 lcap][WIDE_SHARDS][32] work handed out in each pass (phase 1, phase 2)
  int32_t *lcount;           // [lcap + 1][WIDE_SHARDS][32] first reaches per level, summed over the
                             // tiles that made them (a vertex counts once per such tile): its size, roughly
  unsigned long long *lmax;  // [lcap][32] largest stored count of (level, source), as bits
  int32_t *kshift;           // [lcap][32] power of two taken off the level's counts when pushed
  int32_t *lkind;            // [lcap + 1] 1: the level's counts are int64
  const uint32_t *heavy;     // [nwords] vertices whose rows are cut into items
  const int32_t *hv;         // [*nh] vertex of each item of a long row
  const int32_t *hc;         // [*nh] first row entry of the item
  const int32_t *hlist;      // [*nhv] the vertices with long rows
  const int32_t *counts;     // [2]: nh, nhv
  unsigned long long *trace; // nullable: (tag, time) pairs of the first batches' passes (BCS_TRACE)
  int64_t n, nwords;
  int lcap;
};

constexpr int WIDE_TRACE_BATCHES = 4;
constexpr int WIDE_TRACE_CAP = 1024;  // pairs

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

// 2^e as a float for e <= 127, 0 below -126
__device__ __forceinline__ float pow2f_int(int e) { return e < -126 ? 0.0f : __int_as_float((127 + e) << 23); }

__device__ __forceinline__ int warp_max_int(int x) {
  for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// The level bytes of up to 32 neighbours (S per neighbour, one neighbour per
// lane), moved through shared memory so that lane s can read the bytes of
// its own sources in every row.
// A row of the tile is padded by 16 bytes so that the 16-byte stores of
// eight consecutive lanes fall on distinct banks.
template <int SPL>
struct NbrTile {
  uint4 lv[32][2 * SPL + 1];
  uint32_t off[32];  // u * S: the neighbour's first slot
};

// Row entries [e, e + cnt) of col and their level bytes into the tile
// (warp-collective); returns lane j's neighbour (-1 past the end).
template <int SPL>
__device__ __forceinline__ int32_t load_tile(NbrTile<SPL> &t, const int32_t *__restrict__ col, int64_t e, int cnt,
                                             const uint8_t *lvl, int lane) {
  int32_t u = -1;
  if (lane < cnt) {
    u = __ldg(col + e + lane);
    const uint4 *p = (const uint4 *)(lvl + (size_t)u * (32 * SPL));
#pragma unroll
    for (int q = 0; q < 2 * SPL; q++) t.lv[lane][q] = __ldcg(p + q);
    t.off[lane] = (uint32_t)u * (uint32_t)(32 * SPL);
  }
  __syncwarp();
  return u;
}

// The work of a pass (long-row items, then bitmap words) is handed out
// WIDE_GRAB units at a time from WIDE_SHARDS counters, shard h owning the
// grabs starting at h * WIDE_GRAB, (h + WIDE_SHARDS) * WIDE_GRAB, ...  Returns
// the first unit of the warp's next grab, or -1 once every shard is used up
// (warp-collective).  A warp stays on its shard until it is used up, then
// reads all the counters at once and moves to the next shard with work left;
// every failed claim follows another warp's successful one, so the loop ends.
__device__ __forceinline__ int shard_grabs(int64_t total, int h) {
  return (int)((total - (int64_t)h * WIDE_GRAB + (int64_t)WIDE_SHARDS * WIDE_GRAB - 1) /
               ((int64_t)WIDE_SHARDS * WIDE_GRAB));
}

__device__ __forceinline__ int64_t wide_grab(int32_t *ctrs, int64_t total, int &shard, int lane) {
  for (;;) {
    int g = 0;
    if (lane == 0) {  // claim the shard's next grab, unless it is already used up
      int32_t *ctr = ctrs + shard * 32;
      const int lim = shard_grabs(total, shard);
      g = *(volatile int32_t *)ctr < lim ? atomicAdd(ctr, 1) : lim;
    }
    g = __shfl_sync(0xffffffffu, g, 0);
    const int64_t w0 = (int64_t)g * WIDE_SHARDS * WIDE_GRAB + (int64_t)shard * WIDE_GRAB;
    if (w0 < total) return w0;
    bool left = false;
    if (lane < WIDE_SHARDS) left = *(volatile int32_t *)(ctrs + lane * 32) < shard_grabs(total, lane);
    const unsigned bm = __ballot_sync(0xffffffffu, left);
    if (!bm) return -1;
    // bit i of rot: shard (shard + 1 + i) mod WIDE_SHARDS has work left
    const unsigned rot = (bm | (bm << WIDE_SHARDS)) >> (shard + 1);
    shard = (shard + __ffs(rot)) % WIDE_SHARDS;
  }
}

// the light vertices of unit ku of a level's bitmap (upw units per word),
// as the bits of its word
__device__ __forceinline__ uint32_t unit_bits(const uint32_t *bits, const uint32_t *heavy, int64_t ku, int upw,
                                              int64_t &wd) {
  wd = ku / upw;
  const int ub = 32 / upw;
  const uint32_t sel = ub == 32 ? 0xffffffffu : (((1u << ub) - 1u) << ((int)(ku % upw) * ub));
  return __ldcg(bits + wd) & ~__ldg(heavy + wd) & sel;
}

// units per bitmap word for a pass over level L: fine units when the level
// holds an eighth of the vertices or more (every thread decides alike)
__device__ __forceinline__ int level_upw(const int32_t *lcount, int L, int64_t n) {
  int64_t c = 0;
#pragma unroll
  for (int h = 0; h < WIDE_SHARDS; h++) c += __ldcg(lcount + ((size_t)L * WIDE_SHARDS + h) * 32);
  return 8 * c >= n ? WIDE_UPW : 1;
}

template <int SPL>
__device__ __forceinline__ uint32_t tile_byte(const NbrTile<SPL> &t, int j, int s) {
  return ((const uint8_t *)&t.lv[j][0])[s];
}

// Where a batch runs: the whole grid, one grid-wide wait per pass
// (k_bcreach_wide), or one CTA, one CTA-wide wait per pass (k_bcreach_mid).
struct GridScope {
  GridBarrier bar;
  __device__ __forceinline__ int64_t rank() const { return (int64_t)blockIdx.x * WIDE_THREADS + threadIdx.x; }
  __device__ __forceinline__ int64_t size() const { return (int64_t)gridDim.x * WIDE_THREADS; }
  __device__ __forceinline__ bool leader() const { return blockIdx.x == 0 && threadIdx.x < 32; }
  __device__ __forceinline__ bool sync() const { return grid_wait(bar); }
};
struct CtaScope {
  __device__ __forceinline__ int64_t rank() const { return threadIdx.x; }
  __device__ __forceinline__ int64_t size() const { return WIDE_THREADS; }
  __device__ __forceinline__ bool leader() const { return threadIdx.x < 32; }
  __device__ __forceinline__ bool sync() const {
    __syncthreads();
    return true;
  }
};

// One piece's inputs (row offsets, local neighbour ids, weights and the bc'
// target, all indexed by the piece's local vertex ids)
struct WideIn {
  const int64_t *row;
  const int32_t *col;
  double fan;  // bound on sigma growth per level
  const int32_t *reach;
  const double *init_f;
  const int32_t *ident;
  double *bcp;
};

// a CTA's shared memory for batches
template <int SPL>
struct WideSmem {
  NbrTile<SPL> tile[WIDE_WARPS];
  int32_t src[32 * SPL];  // the batch's sources (-1 past the end of the list)
  double ws[32 * SPL];    // their weights reach[s] * ident[s]
};

// One batch of SB = 32 SPL sources: order[base .. base + SB) below nsrc (no
// order: the ids base ..).  Lane l of every warp stands for sources l,
// l + 32, ... of the batch.  Returns false when a wait ran out or the batch
// needed more levels than the scratch holds (err says which).
template <bool REACH, bool IDENT, bool FP32, int SPL, class Scope>
__device__ __forceinline__ bool wide_batch(const Scope &sc, const WideIn &P, const WideScratch &S, WideSmem<SPL> &sm,
                                           const int32_t *__restrict__ order, int64_t base, int64_t nsrc, int *err,
                                           unsigned long long &dag, int sig_cap, int b, int &tpos) {
  constexpr int SB = 32 * SPL;  // sources per batch
  const int64_t *__restrict__ row = P.row;
  const int32_t *__restrict__ col = P.col;
  const int32_t *__restrict__ reach = P.reach;
  const double *__restrict__ init_f = P.init_f;
  const int32_t *__restrict__ ident = P.ident;
  double *const bcp = P.bcp;
  int32_t *const s_src = sm.src;
  double *const s_ws = sm.ws;
  const int lane = threadIdx.x & 31;
  NbrTile<SPL> &tile = sm.tile[threadIdx.x >> 5];
  const int64_t gtid = sc.rank();
  const int64_t nthreads = sc.size();
  const bool leader = sc.leader();  // writes the per-level records
  long long *const sigi = (long long *)S.sig;
  // the slot of (vertex u, source s) is u * SB + s
  uint8_t *const lvl_l = S.lvl + lane;
  unsigned long long *const sigu_l = (unsigned long long *)S.sig + lane;
  double *const sigd_l = S.sig + lane;
  double *const dsum_l = S.dsum + lane;
  const int nh = S.counts[0], nhv = S.counts[1];
  const int flg = ceil_log2_pos(P.fan);
  // stored FP64 counts of a level stay at or below 2^t_hi when pushed, so the
  // next level's sums (at most fan times larger) stay finite; a rescale
  // brings them to 2^t_lo
  const int t_hi = 1000 - flg, t_lo = t_hi - 400;
  // trace: thread 0 of the scope stamps the end of each pass of the first batches
  auto mark = [&](unsigned tag) {
    if (S.trace && b >= 0 && b < WIDE_TRACE_BATCHES && gtid == 0 && tpos < WIDE_TRACE_CAP) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      S.trace[2 * tpos] = ((unsigned long long)b << 32) | tag;
      S.trace[2 * tpos + 1] = t;
      tpos++;
    }
  };
  // every CTA keeps the batch's sources and weights in shared memory (the
  // previous batch's last use of them ended at a grid-wide wait)
  if (threadIdx.x < SB) {
    const int64_t i = base + threadIdx.x;
    const int32_t sv = i < nsrc ? (order ? __ldg(order + i) : (int32_t)i) : -1;
    s_src[threadIdx.x] = sv;
    s_ws[threadIdx.x] =
        sv < 0 ? 0.0
               : (REACH ? (init_f ? __ldg(init_f + sv) + 1.0 : (double)__ldg(reach + sv)) : 1.0) *
                     (IDENT ? (double)__ldg(ident + sv) : 1.0);
  }
  // ------------------------------------------------ level 0: the sources
  if (leader) {
#pragma unroll
    for (int q = 0; q < SPL; q++) {
      const int64_t i = base + 32 * q + lane;
      const int32_t sv = i < nsrc ? (order ? __ldg(order + i) : (int32_t)i) : -1;
      if (sv >= 0) {  // a repeated source is simply two slots of one vertex
        S.lvl[(size_t)sv * SB + 32 * q + lane] = 0;
        sigi[(size_t)sv * SB + 32 * q + lane] = 1;
        atomicOr(S.bits + (sv >> 5), 1u << (sv & 31));
      }
    }
    if (lane == 0) {
      S.flag[0] = 1;
      S.lkind[0] = 1;
      S.lcount[0] = SB;
    }
  }
  if (!sc.sync()) return false;
  mark(0xF000u);
  // ------------------------------------------------ phase 1
  int L = 0;
  int Y[SPL];  // exponent of level L's stored counts, per source
#pragma unroll
  for (int q = 0; q < SPL; q++) Y[q] = 0;
  for (;;) {
    if (!__ldcg(S.flag + L)) break;  // every thread sees the same flags
    if (L + 2 >= S.lcap) {
      if (gtid == 0) atomicOr(err, ERR_DEPTH);
      return false;
    }
    // the representation of the counts: level L's (decided one pass ago),
    // the power of two its pushes drop, and level L+1's
    const int kind = __ldcg(S.lkind + L);
    int k[SPL], bexp_max = 0;
#pragma unroll
    for (int q = 0; q < SPL; q++) {
      int bexp = 0;  // level L's stored counts are below 2^bexp
      if (L > 0) {
        const size_t x = (size_t)(L - 1) * SB + 32 * q + lane;
        const unsigned long long mp = __ldcg(S.lmax + x);
        const int kp = __ldcg(S.kshift + x);
        const int ep = __ldcg(S.lkind + L - 1) ? (mp ? 63 - __clzll((long long)mp) : 0)
                                               : (int)((mp >> 52) & 0x7ff) - 1023;
        bexp = ep + 1 - kp + flg;
      }
      k[q] = (!kind && bexp > t_hi) ? bexp - t_lo : 0;
      bexp_max = max(bexp_max, bexp);
      if (bexp - k[q] + Y[q] > sig_cap && gtid < 32) atomicOr(err, ERR_OVERFLOW);
      if (leader) S.kshift[(size_t)L * SB + 32 * q + lane] = k[q];
    }
    const int kind_next = kind && warp_max_int(bexp_max) + flg < 62;
    if (leader && lane == 0) S.lkind[L + 1] = kind_next;
    const uint32_t *bits_cur = S.bits + (size_t)L * S.nwords;
    uint32_t *bits_next = S.bits + (size_t)(L + 1) * S.nwords;
    unsigned long long wmax[SPL];
#pragma unroll
    for (int q = 0; q < SPL; q++) wmax[q] = 0ull;
    bool found = false;
    int nfirst = 0;  // first reaches this warp made (lane 0's count)
    // one vertex (its whole row, or one item of a long row)
    auto visit = [&](int32_t v, int64_t e0, int64_t e1) {
      bool on[SPL];
      // the value pushed for each source: int64 bits when level L+1's
      // counts are integers, else the bits of a double
      unsigned long long pv[SPL];
      const long long idv = (IDENT && L > 0) ? (long long)__ldg(ident + v) : 1ll;
      bool any = false;
#pragma unroll
      for (int q = 0; q < SPL; q++) {
        const size_t x = (size_t)v * SB + 32 * q + lane;
        on[q] = __ldcg(S.lvl + x) == (uint8_t)L;
        pv[q] = 0ull;
        if (on[q]) {
          if (kind) {
            const long long r = __ldcg(sigi + x);
            wmax[q] = (unsigned long long)r > wmax[q] ? (unsigned long long)r : wmax[q];
            pv[q] = kind_next ? (unsigned long long)(r * idv)
                              : (unsigned long long)__double_as_longlong(i64_to_f64_pos(r) * (double)idv);
          } else {
            const double r = __ldcg(S.sig + x);
            const unsigned long long rb = (unsigned long long)__double_as_longlong(r);
            wmax[q] = rb > wmax[q] ? rb : wmax[q];
            double p = r * pow2_int(-k[q]);
            if (IDENT && L > 0) p *= (double)idv;
            pv[q] = (unsigned long long)__double_as_longlong(p);
          }
        }
        any |= on[q];
      }
      if (!__any_sync(0xffffffffu, any)) return;
      const uint32_t nextl = (uint32_t)(L + 1);
      for (int64_t e = e0; e < e1; e += 32) {
        const int cnt = (int)min((int64_t)32, e1 - e);
        const int32_t uj = load_tile(tile, col, e, cnt, S.lvl, lane);
        unsigned fr = 0u;  // entries one of this lane's sources reaches first (bit j: entry j)
#pragma unroll
        for (int q = 0; q < SPL; q++) {
          if (!on[q]) continue;
          for (int j = 0; j < cnt; j++) {
            const uint32_t bu = tile_byte(tile, j, 32 * q + lane);
            if (bu == 0xFFu || bu == nextl) {  // DAG edge v -> u for this source
              const uint32_t off = tile.off[j] + 32 * q;
              if (bu == 0xFFu) {
                lvl_l[off] = (uint8_t)nextl;
                fr |= 1u << j;
              }
              if (kind_next) atomicAdd(sigu_l + off, pv[q]);
              else atomicAdd(sigd_l + off, __longlong_as_double((long long)pv[q]));
            }
          }
        }
        // entry j marks its vertex in the next level's bitmap if any source reached it first
        const unsigned frw = __reduce_or_sync(0xffffffffu, fr);
        if ((frw >> lane) & 1u) atomicOr(bits_next + (uj >> 5), 1u << (uj & 31));
        found |= frw != 0u;
        nfirst += __popc(frw);
        __syncwarp();
      }
    };
    // work: the items of long rows (the longest work) first, then the
    // bitmap's words (light rows), handed out WIDE_GRAB at a time
    int shard = (int)((gtid >> 5) % WIDE_SHARDS);
    const int upw = level_upw(S.lcount, L, S.n);
    const int64_t total = S.nwords * upw + nh;
    for (;;) {
      const int64_t w0 = wide_grab(S.wctr + (size_t)2 * L * WIDE_SHARDS * 32, total, shard, lane);
      if (w0 < 0) break;
      for (int64_t wi = w0; wi < min((int64_t)w0 + WIDE_GRAB, total); wi++) {
        if (wi >= nh) {
          int64_t wd;
          uint32_t m = unit_bits(bits_cur, S.heavy, wi - nh, upw, wd);
          while (m) {
            const int32_t v = (int32_t)(wd * 32 + __ffs(m) - 1);
            m &= m - 1u;
            visit(v, __ldg(row + v), __ldg(row + v + 1));
          }
        } else {
          const int32_t v = __ldg(S.hv + wi);
          if ((__ldcg(bits_cur + (v >> 5)) >> (v & 31)) & 1u) {
            const int64_t rb = __ldg(row + v), re = __ldg(row + v + 1);
            const int64_t e0 = rb + __ldg(S.hc + wi);
            visit(v, e0, min(re, e0 + WIDE_CH));
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < SPL; q++)
      if (wmax[q]) atomicMax(S.lmax + (size_t)L * SB + 32 * q + lane, wmax[q]);
    if (__any_sync(0xffffffffu, found) && lane == 0) S.flag[L + 1] = 1;
    if (lane == 0 && nfirst)
      atomicAdd(S.lcount + ((size_t)(L + 1) * WIDE_SHARDS + (gtid >> 5) % WIDE_SHARDS) * 32, nfirst);
    if (!sc.sync()) return false;
    mark(0x1000u | (unsigned)L);
#pragma unroll
    for (int q = 0; q < SPL; q++) Y[q] += k[q];
    L++;
  }
  const int Lmax = L - 1;
  // ------------------------------------------------ phase 2
  // level 0 holds only the sources themselves: nothing to add there
  for (int l = Lmax; l >= 1; l--) {
    const int kind_l = __ldcg(S.lkind + l);
    int kl[SPL];
#pragma unroll
    for (int q = 0; q < SPL; q++) kl[q] = __ldcg(S.kshift + (size_t)l * SB + 32 * q + lane);
    const uint32_t *bits_l = S.bits + (size_t)l * S.nwords;
    // one vertex: its dependencies, its bc' terms (first item only) and the
    // pushes of its coefficients to the predecessors
    auto visit = [&](int32_t v, int64_t e0, int64_t e1, bool first, bool light) {
      bool on[SPL];
      double cpush[SPL];
      double contrib64 = 0.0;
      float contrib32 = 0.0f;
      bool any = false;
      const double init = REACH ? (init_f ? __ldg(init_f + v) : (double)(__ldg(reach + v) - 1)) : 0.0;
#pragma unroll
      for (int q = 0; q < SPL; q++) {
        const size_t x = (size_t)v * SB + 32 * q + lane;
        on[q] = __ldcg(S.lvl + x) == (uint8_t)l;
        cpush[q] = 0.0;
        if (on[q]) {
          const double ds = __ldcg(S.dsum + x);
          if (!FP32) {
            const double sv = kind_l ? i64_to_f64_pos(__ldcg(sigi + x)) : __ldcg(S.sig + x);
            const double dv = fma(sv, ds * pow2_int(-kl[q]), init);
            const double kv = IDENT ? (double)__ldg(ident + v) : 1.0;
            cpush[q] = fma(kv, dv, kv) * recip_pos(sv);
            if (v != s_src[32 * q + lane]) contrib64 = fma(s_ws[32 * q + lane], dv, contrib64);
          } else {
            int ev, ed = 0;
            float mv, md = 0.0f;
            if (kind_l) split_pow2_i64(__ldcg(sigi + x), ev, mv);
            else split_pow2(__ldcg(S.sig + x), ev, mv);
            if (ds > 0.0) split_pow2(ds, ed, md);
            const float df = fmaf(mv * md, pow2f_int(ev + ed - kl[q]), (float)init);
            const float kv = IDENT ? (float)__ldg(ident + v) : 1.0f;
            const float cm = fmaf(kv, df, kv) / mv;  // c[v] = cm * 2^-ev in stored units
            cpush[q] = __longlong_as_double(__double_as_longlong(f32_to_f64_bits(cm)) - ((long long)ev << 52));
            if (v != s_src[32 * q + lane]) contrib32 = fmaf((float)s_ws[32 * q + lane], df, contrib32);
          }
          if (light) {  // the slots are finished: clear them for the next batch
            S.sig[x] = 0.0;
            S.dsum[x] = 0.0;
          }
        }
        any |= on[q];
      }
      if (first) {  // bc'[v] gains the vertex's sources' terms, summed in the warp
        if (!FP32) {
          for (int o = 16; o > 0; o >>= 1) contrib64 += __shfl_down_sync(0xffffffffu, contrib64, o);
          if (lane == 0 && contrib64 != 0.0) atomicAdd(bcp + v, contrib64);
        } else {
          for (int o = 16; o > 0; o >>= 1) contrib32 += __shfl_down_sync(0xffffffffu, contrib32, o);
          if (lane == 0 && contrib32 != 0.0f) atomicAdd(bcp + v, f32_to_f64_bits(contrib32));
        }
      }
      if (l == 1 || !__any_sync(0xffffffffu, any)) return;  // the sources' own dependencies are not needed
      const uint32_t prevl = (uint32_t)(l - 1);
      for (int64_t e = e0; e < e1; e += 32) {
        const int cnt = (int)min((int64_t)32, e1 - e);
        load_tile(tile, col, e, cnt, S.lvl, lane);
#pragma unroll
        for (int q = 0; q < SPL; q++) {
          if (!on[q]) continue;
          for (int j = 0; j < cnt; j++) {
            if (tile_byte(tile, j, 32 * q + lane) == prevl) {  // a predecessor of v for this source
              atomicAdd(dsum_l + tile.off[j] + 32 * q, cpush[q]);
              dag++;
            }
          }
        }
        __syncwarp();
      }
    };
    int shard = (int)((gtid >> 5) % WIDE_SHARDS);
    const int upw = level_upw(S.lcount, l, S.n);
    const int64_t total = S.nwords * upw + nh;
    for (;;) {
      const int64_t w0 = wide_grab(S.wctr + (size_t)(2 * l + 1) * WIDE_SHARDS * 32, total, shard, lane);
      if (w0 < 0) break;
      for (int64_t wi = w0; wi < min((int64_t)w0 + WIDE_GRAB, total); wi++) {
        if (wi >= nh) {
          int64_t wd;
          uint32_t m = unit_bits(bits_l, S.heavy, wi - nh, upw, wd);
          while (m) {
            const int32_t v = (int32_t)(wd * 32 + __ffs(m) - 1);
            m &= m - 1u;
            visit(v, __ldg(row + v), __ldg(row + v + 1), true, true);
          }
        } else {
          const int32_t v = __ldg(S.hv + wi);
          if ((__ldcg(bits_l + (v >> 5)) >> (v & 31)) & 1u) {
            const int64_t rb = __ldg(row + v), re = __ldg(row + v + 1);
            const int32_t c0 = __ldg(S.hc + wi);
            visit(v, rb + c0, min(re, rb + c0 + WIDE_CH), c0 == 0, false);
          }
        }
      }
    }
    if (!sc.sync()) return false;
    mark(0x2000u | (unsigned)l);
  }
  // ------------------------------------------------ clear for the next batch
  {
    uint4 *p = (uint4 *)S.lvl;
    const uint4 ff = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
    for (int64_t i = gtid; i < S.n * (SB / 16); i += nthreads) p[i] = ff;
    for (int64_t i = gtid; i < (int64_t)(Lmax + 2) * S.nwords; i += nthreads) S.bits[i] = 0u;
    for (int64_t i = gtid; i < (int64_t)(Lmax + 3) * max(SB, 2 * WIDE_SHARDS); i += nthreads) {
      if (i < (int64_t)(Lmax + 2) * SB) S.lmax[i] = 0ull;
      if (i < Lmax + 3) S.flag[i] = 0;
      if (i < 2 * (Lmax + 2) * WIDE_SHARDS) S.wctr[i * 32] = 0;
      if (i < (Lmax + 2) * WIDE_SHARDS) S.lcount[i * 32] = 0;
    }
    for (int64_t i = gtid; i < (int64_t)nhv * SB; i += nthreads) {  // long rows' slots (items shared them)
      const size_t x = (size_t)__ldg(S.hlist + (i / SB)) * SB + (i % SB);
      S.sig[x] = 0.0;
      S.dsum[x] = 0.0;
    }
    if (leader) {  // level 0
#pragma unroll
      for (int q = 0; q < SPL; q++)
        if (s_src[32 * q + lane] >= 0) sigi[(size_t)s_src[32 * q + lane] * SB + 32 * q + lane] = 0;
    }
  }
  if (!sc.sync()) return false;
  mark(0xE000u);
  return true;
}

// The whole grid on one batch at a time, over every batch of one piece.
template <bool REACH, bool IDENT, bool FP32, int MINB, int SPL>
__global__ void __launch_bounds__(WIDE_THREADS, MINB) k_bcreach_wide(
    const int64_t *__restrict__ row, const int32_t *__restrict__ col, double fan, const int32_t *__restrict__ reach,
    const double *__restrict__ init_f, const int32_t *__restrict__ ident, const int32_t *__restrict__ order,
    int32_t nsrc, double *bcp, WideScratch S, GridBarrier bar, int *err, unsigned long long *dag_total, int sig_cap) {
  constexpr int SB = 32 * SPL;
  __shared__ WideSmem<SPL> sm;
  const GridScope sc{bar};
  const WideIn P{row, col, fan, reach, init_f, ident, bcp};
  unsigned long long dag = 0;
  int tpos = 0;
  const int nbatch = (nsrc + SB - 1) / SB;
  for (int b = 0; b < nbatch; b++)
    if (!wide_batch<REACH, IDENT, FP32, SPL>(sc, P, S, sm, order, (int64_t)SB * b, nsrc, err, dag, sig_cap, b, tpos))
      return;
  if (dag) atomicAdd(dag_total, dag);
}


// ------------------------------------------------------ mid-size pieces
// Pieces too large for shared memory but small enough that many of their
// batches run at once: the batch above on one CTA, its waits CTA-wide, the
// per-(vertex, source) state in the CTA's own region of global memory.
// Batches of all the listed pieces are handed out from one queue (largest
// pieces first).  No long-row items: a warp walks a whole row.  A piece's
// BFS depth from its first vertex is found once, by the first CTA that
// takes one of its batches; a piece too deep for MID_LCAP levels, or not
// connected, is marked and left to the caller.
constexpr int MID_LCAP = 64;

struct MidUnit {
  int32_t comp;  // index into the component descriptors
  int32_t base;  // the batch's first source
};

// per-CTA regions (strides: nmax vertices, nwmax bitmap words)
struct MidScratch {
  uint8_t *lvl;
  double *sig, *dsum;
  uint32_t *bits;
  const uint32_t *heavy;  // all zero (no long-row items), shared
  int32_t *flag, *wctr, *lcount, *kshift, *lkind;
  unsigned long long *lmax;
  const int32_t *counts;  // {0, 0}, shared
  int64_t nmax, nwmax;
};

template <int SPL>
__device__ __forceinline__ WideScratch mid_slice(const MidScratch &M, int cta) {
  constexpr int SB = 32 * SPL;
  const size_t c = (size_t)cta;
  WideScratch S;
  S.lvl = M.lvl + c * M.nmax * SB;
  S.sig = M.sig + c * M.nmax * SB;
  S.dsum = M.dsum + c * M.nmax * SB;
  S.bits = M.bits + c * MID_LCAP * M.nwmax;
  S.flag = M.flag + c * (MID_LCAP + 1);
  S.wctr = M.wctr + c * 2 * MID_LCAP * WIDE_SHARDS * 32;
  S.lcount = M.lcount + c * (MID_LCAP + 1) * WIDE_SHARDS * 32;
  S.lmax = M.lmax + c * MID_LCAP * SB;
  S.kshift = M.kshift + c * MID_LCAP * SB;
  S.lkind = M.lkind + c * (MID_LCAP + 1);
  S.heavy = M.heavy;
  S.hv = S.hc = S.hlist = nullptr;
  S.counts = M.counts;
  S.trace = nullptr;
  S.n = 0;
  S.nwords = 0;
  S.lcap = MID_LCAP;
  return S;
}

// Does every source of the piece stay within the level cap?  BFS from
// vertex 0 (levels in the level bytes of slot 0, frontiers in the level
// bitmaps, both left cleared): the piece must be connected and 2 ecc + 4
// levels must fit (no source reaches deeper than twice vertex 0's
// eccentricity).  CTA-collective.
template <int SPL>
__device__ bool mid_depth_fits(const int64_t *__restrict__ row, const int32_t *__restrict__ col, int32_t n,
                               const WideScratch &S) {
  constexpr int SB = 32 * SPL;
  __shared__ int s_found;
  const int nw = (n + 31) / 32;
  if (threadIdx.x == 0) {
    S.lvl[0] = 0;
    S.bits[0] = 1u;
  }
  int L = 0, reached = 1;
  bool fits = true;
  for (;;) {
    if (threadIdx.x == 0) s_found = 0;
    __syncthreads();
    const uint32_t *cur = S.bits + (size_t)L * nw;
    uint32_t *nxt = S.bits + (size_t)(L + 1) * nw;
    int found = 0;
    for (int v = threadIdx.x; v < n; v += WIDE_THREADS) {
      if (!((__ldcg(cur + (v >> 5)) >> (v & 31)) & 1u)) continue;
      for (int64_t e = __ldg(row + v); e < __ldg(row + v + 1); e++) {
        const int32_t u = __ldg(col + e);
        if (__ldcg(S.lvl + (size_t)u * SB) != 0xFFu) continue;
        const uint32_t bit = 1u << (u & 31);
        if (!(atomicOr(nxt + (u >> 5), bit) & bit)) {  // the first to reach u
          S.lvl[(size_t)u * SB] = (uint8_t)(L + 1);
          found++;
        }
      }
    }
    if (found) atomicAdd(&s_found, found);
    __syncthreads();
    const int more = s_found;  // vertices first reached on level L + 1
    __syncthreads();           // read by every thread before the next pass resets it
    if (!more) break;
    reached += more;
    L++;
    if (2 * L + 4 > MID_LCAP) {  // deeper than the levels hold
      fits = false;
      break;
    }
  }
  if (reached != n) fits = false;
  for (int v = threadIdx.x; v < n; v += WIDE_THREADS) S.lvl[(size_t)v * SB] = 0xFF;
  for (int64_t i = threadIdx.x; i < (int64_t)(L + 2) * nw; i += WIDE_THREADS) S.bits[i] = 0u;
  __syncthreads();
  return fits;
}

// Batches of the mid-size pieces, one per CTA at a time.  depth_state per
// component: 0 unknown, 1 fits, 2 too deep (its batches are skipped).
// order (nullable, one piece only): the sources, else every vertex.
template <bool REACH, bool IDENT, bool FP32, int SPL>
__global__ void __launch_bounds__(WIDE_THREADS, 4) k_bcreach_mid(
    const CompDesc *__restrict__ comps, const MidUnit *__restrict__ units, int nunits, int *unit_ctr,
    const int64_t *__restrict__ g_row, const int32_t *__restrict__ g_col, const int32_t *__restrict__ g_reach,
    const double *__restrict__ g_init, const int32_t *__restrict__ g_ident, double *g_bcp,
    const int32_t *__restrict__ order, MidScratch M, int32_t *depth_state, int *err,
    unsigned long long *dag_total, int sig_cap) {
  __shared__ WideSmem<SPL> sm;
  __shared__ int s_unit, s_state;
  const CtaScope sc;
  WideScratch S = mid_slice<SPL>(M, blockIdx.x);
  unsigned long long dag = 0;
  int tpos = 0;
  for (;;) {
    if (threadIdx.x == 0) s_unit = atomicAdd(unit_ctr, 1);
    __syncthreads();
    const int u = s_unit;
    if (u >= nunits) break;
    const MidUnit un = units[u];
    const CompDesc c = comps[un.comp];
    const int64_t *row = g_row + c.row_off;
    S.n = c.n;
    S.nwords = (c.n + 31) / 32;
    if (threadIdx.x == 0) s_state = *(volatile int32_t *)(depth_state + un.comp);
    __syncthreads();
    int st = s_state;
    if (st == 0) {
      st = mid_depth_fits<SPL>(row, g_col, c.n, S) ? 1 : 2;
      if (threadIdx.x == 0) depth_state[un.comp] = st;
    }
    if (st != 1) {
      __syncthreads();  // s_unit and s_state are read before the next claim
      continue;
    }
    const WideIn P{row,
                   g_col,
                   c.fan,
                   (REACH && g_reach && !g_init) ? g_reach + c.vtx_off : nullptr,
                   g_init ? g_init + c.vtx_off : nullptr,
                   IDENT ? g_ident + c.vtx_off : nullptr,
                   g_bcp + c.vtx_off};
    if (!wide_batch<REACH, IDENT, FP32, SPL>(sc, P, S, sm, order, un.base, nsrc_of(c), err, dag, sig_cap, -1, tpos))
      break;
  }
  if (dag) atomicAdd(dag_total, dag);
}

// The vertices whose rows are cut into items (more than WIDE_CH entries),
// as a bitmap, a list, and the list of items.
__global__ void k_wide_heavy(int64_t n, const int64_t *__restrict__ row, uint32_t *heavy, int32_t *hlist,
                             int32_t *hv, int32_t *hc, int32_t *counts) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = row[v + 1] - row[v];
    if (d <= WIDE_CH) continue;
    atomicOr(heavy + (v >> 5), 1u << (v & 31));
    hlist[atomicAdd(counts + 1, 1)] = (int32_t)v;
    const int nch = (int)((d + WIDE_CH - 1) / WIDE_CH);
    const int at = atomicAdd(counts, nch);
    for (int c = 0; c < nch; c++) {
      hv[at + c] = (int32_t)v;
      hc[at + c] = c * WIDE_CH;
    }
  }
}

// ---------------------------------------------------------- host side
template <bool R, bool I, bool F, int MINB, int SPL>
static int wide_launch_mb(Ctx &ctx, int per_sm_cap, void **args) {
  int per_sm = 0;
  BCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bcreach_wide<R, I, F, MINB, SPL>, WIDE_THREADS,
                                                         0));
  if (per_sm < 1) {
    set_error("the wide Bc-Reach kernel cannot be resident");
    return BCS_ECUDA;
  }
  per_sm = std::min(per_sm, per_sm_cap);
  BCS_CUDA(cudaLaunchCooperativeKernel((const void *)k_bcreach_wide<R, I, F, MINB, SPL>,
                                       dim3(ctx.num_sms * per_sm), dim3(WIDE_THREADS), args, 0, ctx.stream));
  ctx.launches++;
  return BCS_OK;
}

// 32 or 64 sources per batch; register budgets of 5 or 6 CTAs per SM
template <bool R, bool I, bool F>
static int wide_launch_t(Ctx &ctx, int spl, int per_sm_cap, void **args) {
  if (spl == 2)
    return per_sm_cap <= 5 ? wide_launch_mb<R, I, F, 5, 2>(ctx, per_sm_cap, args)
                           : wide_launch_mb<R, I, F, 6, 2>(ctx, per_sm_cap, args);
  return per_sm_cap <= 5 ? wide_launch_mb<R, I, F, 5, 1>(ctx, per_sm_cap, args)
                         : wide_launch_mb<R, I, F, 6, 1>(ctx, per_sm_cap, args);
}

int wide_depth_limit() { return 250; }

int run_wide(Ctx &ctx, const CompDesc &c, const BcInput &in, bool fp32, const int32_t *d_order, int32_t nsrc,
             int depth_bound, int *d_err, unsigned long long *d_dag) {
  if (nsrc <= 0 || c.n < 2) return BCS_OK;
  int spl = 2;  // sources per lane: 64 per batch
  if (const char *e = std::getenv("BCS_WIDE_SOURCES")) spl = std::atoi(e) <= 32 ? 1 : 2;
  const int SB = 32 * spl;
  const int64_t n = c.n, nwords = (n + 31) / 32;
  // no source of the piece reaches deeper than depth_bound
  const int lcap = std::min(depth_bound, wide_depth_limit()) + 3;
  const int64_t hmax = c.nnz / WIDE_CH + 1;  // vertices with long rows, at most
  const cudaStream_t s = ctx.stream;
  DBuf<uint8_t> lvl;
  DBuf<double> sig, dsum;
  DBuf<uint32_t> bits, heavy;
  DBuf<int32_t> flag, wctr, lcount, kshift, lkind, hlist, hv, hc, counts;
  DBuf<unsigned long long> lmax, barw, trace;
  const bool tracing = std::getenv("BCS_TRACE") != nullptr;
  if (tracing) {
    BCS_TRY(trace.alloc(2 * WIDE_TRACE_CAP, s));
    BCS_CUDA(cudaMemsetAsync(trace.p, 0, 2 * WIDE_TRACE_CAP * 8, s));
  }
  BCS_TRY(lvl.alloc(SB * n, s));
  BCS_TRY(sig.alloc(SB * n, s));
  BCS_TRY(dsum.alloc(SB * n, s));
  BCS_TRY(bits.alloc((size_t)lcap * nwords, s));
  BCS_TRY(heavy.alloc(nwords, s));
  BCS_TRY(flag.alloc(lcap + 1, s));
  BCS_TRY(wctr.alloc((size_t)2 * lcap * WIDE_SHARDS * 32, s));
  BCS_TRY(lcount.alloc((size_t)(lcap + 1) * WIDE_SHARDS * 32, s));
  BCS_TRY(kshift.alloc((size_t)lcap * SB, s));
  BCS_TRY(lkind.alloc(lcap + 1, s));
  BCS_TRY(lmax.alloc((size_t)lcap * SB, s));
  BCS_TRY(hlist.alloc(hmax, s));
  BCS_TRY(hv.alloc(2 * hmax, s));
  BCS_TRY(hc.alloc(2 * hmax, s));
  BCS_TRY(counts.alloc(2, s));
  BCS_TRY(barw.alloc(1, s));
  BCS_CUDA(cudaMemsetAsync(lvl.p, 0xFF, SB * n, s));
  BCS_CUDA(cudaMemsetAsync(sig.p, 0, SB * n * 8, s));
  BCS_CUDA(cudaMemsetAsync(dsum.p, 0, SB * n * 8, s));
  BCS_CUDA(cudaMemsetAsync(bits.p, 0, (size_t)lcap * nwords * 4, s));
  BCS_CUDA(cudaMemsetAsync(heavy.p, 0, nwords * 4, s));
  BCS_CUDA(cudaMemsetAsync(flag.p, 0, (lcap + 1) * 4, s));
  BCS_CUDA(cudaMemsetAsync(wctr.p, 0, (size_t)2 * lcap * WIDE_SHARDS * 32 * 4, s));
  BCS_CUDA(cudaMemsetAsync(lcount.p, 0, (size_t)(lcap + 1) * WIDE_SHARDS * 32 * 4, s));
  BCS_CUDA(cudaMemsetAsync(lmax.p, 0, (size_t)lcap * SB * 8, s));
  BCS_CUDA(cudaMemsetAsync(counts.p, 0, 8, s));
  BCS_CUDA(cudaMemsetAsync(barw.p, 0, 8, s));
  const int64_t *row = in.row + c.row_off;
  k_wide_heavy<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx.num_sms * 8), 256, 0, s>>>(
      n, row, heavy.p, hlist.p, hv.p, hc.p, counts.p);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  WideScratch S{lvl.p,   sig.p,   dsum.p,   bits.p,  flag.p,  wctr.p,    lcount.p, lmax.p, kshift.p, lkind.p, heavy.p,
                hv.p,    hc.p,    hlist.p,  counts.p, tracing ? trace.p : nullptr, n, nwords, lcap};
  GridBarrier gb{(unsigned int *)barw.p, (unsigned int *)barw.p + 1, d_err, (long long)ctx.max_wait};
  const int32_t *colp = in.col;
  double fan = c.fan;
  const bool R = in.reach != nullptr || in.init != nullptr, I = in.ident != nullptr;
  const int32_t *reach = in.reach && !in.init ? in.reach + c.vtx_off : nullptr;
  const double *init_f = in.init ? in.init + c.vtx_off : nullptr;
  const int32_t *ident = in.ident ? in.ident + c.vtx_off : nullptr;
  double *bcp = in.bcp + c.vtx_off;
  int cap_lg2 = ctx.sigma_cap_lg2;
  void *args[] = {(void *)&row,     (void *)&colp, (void *)&fan, (void *)&reach, (void *)&init_f,
                  (void *)&ident,   (void *)&d_order, (void *)&nsrc, (void *)&bcp, (void *)&S,
                  (void *)&gb,      (void *)&d_err, (void *)&d_dag, (void *)&cap_lg2};
  int cap = 6;
  if (const char *e = std::getenv("BCS_WIDE_CTAS_PER_SM")) cap = std::max(1, std::atoi(e));
  ctx.stats.n_wide_batches += (nsrc + SB - 1) / SB;
  BCS_TRY(BCS_DISPATCH3(wide_launch_t, R, I, fp32, ctx, spl, cap, args));
  if (tracing) {  // the first batches' pass times (us) to stderr
    std::vector<unsigned long long> tr(2 * WIDE_TRACE_CAP);
    BCS_CUDA(cudaMemcpyAsync(tr.data(), trace.p, tr.size() * 8, cudaMemcpyDeviceToHost, s));
    BCS_CUDA(cudaStreamSynchronize(s));
    std::string line;
    for (int i = 1; i < WIDE_TRACE_CAP && tr[2 * i + 1]; i++) {
      const unsigned tag = (unsigned)(tr[2 * i] & 0xffffffffu);
      char buf[64];
      const char *kind = (tag >> 12) == 1 ? "p1L" : (tag >> 12) == 2 ? "p2L" : (tag >> 12) == 0xE ? "clear" : "setup";
      std::snprintf(buf, sizeof(buf), " %s%u:%.1f", kind, tag & 0xfffu, (tr[2 * i + 1] - tr[2 * i - 1]) * 1e-3);
      line += buf;
      if ((tag >> 12) == 0xE) {
        std::fprintf(stderr, "[bcs trace] wide batch %llu us:%s\n", tr[2 * i] >> 32, line.c_str());
        line.clear();
      }
    }
  }
  return BCS_OK;
}

// ---------------------------------------------------------- mid-size launcher
template <bool R, bool I, bool F>
static int mid_launch_t(Ctx &ctx, int grid, void **args) {
  BCS_CUDA(cudaLaunchKernel((const void *)k_bcreach_mid<R, I, F, 2>, dim3(grid), dim3(WIDE_THREADS), args, 0,
                            ctx.stream));
  ctx.launches++;
  return BCS_OK;
}

template <bool R, bool I, bool F>
static int mid_ctas_per_sm(int *out) {
  BCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_bcreach_mid<R, I, F, 2>, WIDE_THREADS, 0));
  return BCS_OK;
}

int run_mid(Ctx &ctx, const std::vector<CompDesc> &comps, const std::vector<int32_t> &pieces, const BcInput &in,
            bool fp32, const int32_t *d_order, const CompDesc *d_comps, int *d_err, unsigned long long *d_dag,
            std::vector<int32_t> *too_deep) {
  too_deep->clear();
  if (pieces.empty()) return BCS_OK;
  constexpr int SB = 64;
  const cudaStream_t s = ctx.stream;
  const bool R = in.reach != nullptr || in.init != nullptr, I = in.ident != nullptr;
  // the batches, largest pieces first
  std::vector<int32_t> order(pieces);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return comps[a].n > comps[b].n; });
  std::vector<MidUnit> units;
  int64_t nmax = 1;
  for (int32_t ci : order) {
    const CompDesc &c = comps[ci];
    nmax = std::max<int64_t>(nmax, c.n);
    for (int64_t b = 0; b < nsrc_of(c); b += SB) units.push_back(MidUnit{ci, (int32_t)b});
  }
  if (units.empty()) return BCS_OK;
  const int64_t nwmax = (nmax + 31) / 32;
  const size_t per_cta = (size_t)nmax * SB * 17 + (size_t)MID_LCAP * nwmax * 4 +
                         (size_t)MID_LCAP * SB * 12 + (size_t)(3 * MID_LCAP + 1) * WIDE_SHARDS * 32 * 4 + 1024;
  int per_sm = 1;
  BCS_TRY(BCS_DISPATCH3(mid_ctas_per_sm, R, I, fp32, &per_sm));
  int64_t grid = (int64_t)ctx.num_sms * std::max(1, std::min(per_sm, 4));
  size_t free_b = 0, total_b = 0;
  BCS_CUDA(cudaMemGetInfo(&free_b, &total_b));
  grid = std::min<int64_t>(grid, (int64_t)(free_b / 2 / per_cta));
  grid = std::min<int64_t>(grid, (int64_t)units.size());
  if (grid < 1) {
    set_error("not enough device memory for one mid-size Bc-Reach CTA");
    return BCS_ENOMEM;
  }
  const size_t G = (size_t)grid;
  DBuf<uint8_t> lvl;
  DBuf<double> sig, dsum;
  DBuf<uint32_t> bits, heavy;
  DBuf<int32_t> flag, wctr, lcount, kshift, lkind, counts, state, ctr;
  DBuf<unsigned long long> lmax;
  DBuf<MidUnit> d_units;
  BCS_TRY(lvl.alloc(G * nmax * SB, s));
  BCS_TRY(sig.alloc(G * nmax * SB, s));
  BCS_TRY(dsum.alloc(G * nmax * SB, s));
  BCS_TRY(bits.alloc(G * MID_LCAP * nwmax, s));
  BCS_TRY(heavy.alloc(nwmax, s));
  BCS_TRY(flag.alloc(G * (MID_LCAP + 1), s));
  BCS_TRY(wctr.alloc(G * 2 * MID_LCAP * WIDE_SHARDS * 32, s));
  BCS_TRY(lcount.alloc(G * (MID_LCAP + 1) * WIDE_SHARDS * 32, s));
  BCS_TRY(kshift.alloc(G * MID_LCAP * SB, s));
  BCS_TRY(lkind.alloc(G * (MID_LCAP + 1), s));
  BCS_TRY(lmax.alloc(G * MID_LCAP * SB, s));
  BCS_TRY(counts.alloc(2, s));
  BCS_TRY(state.alloc(comps.size(), s));
  BCS_TRY(ctr.alloc(1, s));
  BCS_TRY(d_units.alloc(units.size(), s));
  BCS_CUDA(cudaMemsetAsync(lvl.p, 0xFF, G * nmax * SB, s));
  BCS_CUDA(cudaMemsetAsync(sig.p, 0, G * nmax * SB * 8, s));
  BCS_CUDA(cudaMemsetAsync(dsum.p, 0, G * nmax * SB * 8, s));
  BCS_CUDA(cudaMemsetAsync(bits.p, 0, G * MID_LCAP * nwmax * 4, s));
  BCS_CUDA(cudaMemsetAsync(heavy.p, 0, nwmax * 4, s));
  BCS_CUDA(cudaMemsetAsync(flag.p, 0, G * (MID_LCAP + 1) * 4, s));
  BCS_CUDA(cudaMemsetAsync(wctr.p, 0, G * 2 * MID_LCAP * WIDE_SHARDS * 32 * 4, s));
  BCS_CUDA(cudaMemsetAsync(lcount.p, 0, G * (MID_LCAP + 1) * WIDE_SHARDS * 32 * 4, s));
  BCS_CUDA(cudaMemsetAsync(kshift.p, 0, G * MID_LCAP * SB * 4, s));
  BCS_CUDA(cudaMemsetAsync(lkind.p, 0, G * (MID_LCAP + 1) * 4, s));
  BCS_CUDA(cudaMemsetAsync(lmax.p, 0, G * MID_LCAP * SB * 8, s));
  BCS_CUDA(cudaMemsetAsync(counts.p, 0, 8, s));
  BCS_CUDA(cudaMemsetAsync(state.p, 0, comps.size() * 4, s));
  BCS_CUDA(cudaMemsetAsync(ctr.p, 0, 4, s));
  BCS_CUDA(cudaMemcpyAsync(d_units.p, units.data(), units.size() * sizeof(MidUnit), cudaMemcpyHostToDevice, s));
  MidScratch M{lvl.p,    sig.p,   dsum.p,   bits.p, heavy.p, flag.p, wctr.p,
               lcount.p, kshift.p, lkind.p, lmax.p, counts.p, nmax,   nwmax};
  const int nunits = (int)units.size();
  const int64_t *row = in.row;
  const int32_t *col = in.col, *reach = in.reach, *ident = in.ident;
  const double *init = in.init;
  double *bcp = in.bcp;
  int cap_lg2 = ctx.sigma_cap_lg2;
  void *args[] = {(void *)&d_comps, (void *)&d_units.p, (void *)&nunits, (void *)&ctr.p,  (void *)&row,
                  (void *)&col,     (void *)&reach,     (void *)&init,   (void *)&ident,  (void *)&bcp,
                  (void *)&d_order, (void *)&M,         (void *)&state.p, (void *)&d_err, (void *)&d_dag,
                  (void *)&cap_lg2};
  BCS_TRY(BCS_DISPATCH3(mid_launch_t, R, I, fp32, ctx, (int)grid, args));
  BCS_CUDA(cudaGetLastError());
  std::vector<int32_t> h_state(comps.size());
  BCS_CUDA(cudaMemcpyAsync(h_state.data(), state.p, comps.size() * 4, cudaMemcpyDeviceToHost, s));
  BCS_CUDA(cudaStreamSynchronize(s));
  for (int32_t ci : pieces) {
    if (h_state[ci] == 2) too_deep->push_back(ci);
    else ctx.stats.n_wide_batches += (nsrc_of(comps[ci]) + SB - 1) / SB;
  }
  return BCS_OK;
}

}  // namespace bcs
