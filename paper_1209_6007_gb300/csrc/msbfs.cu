// msbfs.cu - Bc-Reach on large pieces, 32 sources at a time per CTA.
//
// The sources of a batch share every adjacency read: a CTA runs the
// level-synchronous BFS of all 32 of them together, one bit (or one lane) per
// source.  Per vertex it keeps
//   vis   32-bit mask of the sources that have reached it,
//   nxt   bits discovered for the next level (built with atomicOr),
//   lv    the BFS level of each source modulo 4, two bits per source in one
//         64-bit word.  Adjacent vertices are at most one level apart, so
//         "w is on level L+1 for source b" is decided by the level mod 4
//         (together with vis for sources that have not reached w),
//   sc    32 values, lane b's path count (phase 1: exact int64 while the
//         level's growth bound stays below 2^62, FP64 after), then its FP64
//         phase-2 coefficient (the path count is not needed any more by then),
// and the vertices of each level in a queue (a vertex is queued once per
// level in which it gains sources, so at most 32 times).
//
// Phase 1, per level: (a) discovery, warp per frontier vertex with the lanes
// over its neighbours: bits = sources of v on level L minus those that
// already reached w; (b) per newly reached vertex w, warp per vertex with the
// lanes over the sources: sigma[w][b] = sum over neighbours v on level L for
// b of sigma[v][b] * ident[v] (ident of the source itself counts 1).
// Phase 2 (Eq. 3 with reach and ident, coefficient form as in bcreach.cu),
// per level deepest first, warp per queued vertex with lanes over sources.
// Path counts carry a power-of-two exponent per (level, source), as in the
// single-source kernels.
#include <algorithm>
#include <cfloat>

#include "bc_math.cuh"
#include "common.h"

namespace bcs {

constexpr int MS_THREADS = 512;
constexpr int MS_WARPS = MS_THREADS / 32;
constexpr int MS_LCAP = 65536;  // BFS levels one batch may index

struct MsBatch {
  int32_t comp;
  int32_t first;  // sources are src[first .. first + count), or those ids when there is no list
  int32_t count;  // 1..32
  int32_t pad;
};

struct MsScratch {
  uint32_t *vis, *nxt;  // [G][nmax]
  uint64_t *lv;         // [G][nmax]
  double *sc;           // [G][nmax][32]
  double *acc;          // [G][nmax]
  int32_t *queue;       // [G][qcap]
  uint32_t *qmask;      // [G][qcap] the sources for which the entry's vertex is on the entry's level
  int32_t *qoff;        // [G][MS_LCAP + 2]
  int32_t *lexp;        // [G][MS_LCAP][32]
  int64_t nmax, qcap;
};

// sources whose 2-bit level field equals L mod 4 (reachedness not checked)
__device__ __forceinline__ uint32_t at_level(uint64_t lv, int L) {
  const uint64_t x = lv ^ (0x5555555555555555ull * (uint64_t)(L & 3));
  return compact2(~(x | (x >> 1)));
}

__device__ __forceinline__ uint64_t set_level(uint64_t lv, uint32_t bits, int L) {
  const uint64_t s = spread2(bits);
  return (lv & ~(s * 3ull)) | (s * (uint64_t)(L & 3));
}

template <bool REACH, bool IDENT, bool FP32>
__global__ void __launch_bounds__(MS_THREADS) k_bcreach_ms(
    const MsBatch *__restrict__ batches, int nbatch, int *counter, const CompDesc *__restrict__ comps,
    const int64_t *__restrict__ g_row, const int32_t *__restrict__ g_col, const int32_t *__restrict__ g_reach,
    const int32_t *__restrict__ g_ident, const double *__restrict__ g_init, const int32_t *__restrict__ srcs,
    double *bcp, MsScratch S, int *err, unsigned long long *dag_total) {
  __shared__ int s_batch, s_qtail;
  __shared__ int32_t s_src[32];
  __shared__ double s_ws[32];
  __shared__ double s_red[MS_WARPS][32];
  __shared__ int s_k[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t B = blockIdx.x;
  uint32_t *const vis = S.vis + B * S.nmax;
  uint32_t *const nxt = S.nxt + B * S.nmax;
  uint64_t *const lv = S.lv + B * S.nmax;
  double *const sc = S.sc + B * S.nmax * 32;
  long long *const sci = (long long *)sc;  // the same slots while a level's counts are integers
  double *const acc = S.acc + B * S.nmax;
  int32_t *const queue = S.queue + B * S.qcap;
  uint32_t *const qmask = S.qmask + B * S.qcap;
  int32_t *const qoff = S.qoff + B * (MS_LCAP + 2);
  int32_t *const lexp = S.lexp + B * (size_t)MS_LCAP * 32;
  unsigned long long dag = 0;
  int cur = -1;
  for (;;) {
    if (tid == 0) s_batch = atomicAdd(counter, 1);
    __syncthreads();
    const int bi = s_batch;
    __syncthreads();
    const int next = bi < nbatch ? batches[bi].comp : -1;
    if (next != cur && cur >= 0) {
      const CompDesc c = comps[cur];
      for (int v = tid; v < c.n; v += MS_THREADS) {
        if (acc[v] != 0.0) atomicAdd(bcp + c.vtx_off + v, acc[v]);
        acc[v] = 0.0;
      }
      __syncthreads();
    }
    cur = next;
    if (next < 0) break;
    const MsBatch bt = batches[bi];
    const CompDesc c = comps[bt.comp];
    const int64_t *row = g_row + c.row_off;
    const int32_t *reach = REACH && !g_init ? g_reach + c.vtx_off : nullptr;
    const double *init_f = REACH && g_init ? g_init + c.vtx_off : nullptr;  // fractional reach - 1
    const int32_t *ident = IDENT ? g_ident + c.vtx_off : nullptr;
    if (tid < 32) {
      const int32_t s = tid < bt.count ? (srcs ? srcs[bt.first + tid] : bt.first + tid) : -1;
      s_src[tid] = s;
      s_ws[tid] = s < 0 ? 0.0
                        : (REACH ? (init_f ? init_f[s] + 1.0 : (double)reach[s]) : 1.0) *
                              (IDENT ? (double)ident[s] : 1.0);
      if (s >= 0) atomicOr(nxt + s, 1u << tid);
    }
    if (tid == 0) s_qtail = 0;
    __syncthreads();
    if (tid < bt.count) {  // the lowest bit of a source vertex queues it once
      const int32_t s = s_src[tid];
      if ((nxt[s] & ((1u << tid) - 1u)) == 0) queue[atomicAdd(&s_qtail, 1)] = s;
    }
    __syncthreads();
    int hi = s_qtail;
    // level 0: sigma = 1 for each source
    for (int i = warp; i < hi; i += MS_WARPS) {
      const int32_t v = queue[i];
      const uint32_t N = nxt[v];
      if ((N >> lane) & 1u) sci[(size_t)v * 32 + lane] = 1;
      __syncwarp();
      if (lane == 0) {
        qmask[i] = N;
        vis[v] = N;
        lv[v] = set_level(0ull, N, 0);
        nxt[v] = 0;
      }
    }
    if (tid == 0) {
      qoff[0] = 0;
      qoff[1] = hi;
    }
    if (tid < 32) lexp[tid] = 0;
    __syncthreads();
    int lo = 0, L = 0;
    double bound = 1.0;
    bool depth_fail = false;
    // Path counts are exact 64-bit integers while the level's growth bound
    // (an integer power of two) stays below 2^62; the first level past it is
    // pulled in FP64, widening the integers of the level before as it reads
    // them (lint = first FP64 level).
    int lint = MS_LCAP + 2;
    const int flg = ceil_log2_pos(c.fan);
    int blg = 0;
    // ------------------------------------------------------------ phase 1
    for (;;) {
      for (int i = lo + warp; i < hi; i += MS_WARPS) {
        const int32_t v = queue[i];
        const uint32_t f = qmask[i];  // a vertex's own sources may sit on levels 4 apart: use the entry's mask
        for (int64_t e = row[v] + lane; e < row[v + 1]; e += 32) {
          const int32_t w = g_col[e];
          const uint32_t nb = f & ~*(volatile uint32_t *)(vis + w);
          if (nb && atomicOr(nxt + w, nb) == 0u) queue[atomicAdd(&s_qtail, 1)] = w;
        }
      }
      __syncthreads();
      const int nhi = *(volatile int *)&s_qtail;
      __syncthreads();
      if (nhi == hi) break;
      if (L + 2 >= MS_LCAP) {
        depth_fail = true;
        break;
      }
      const bool int_next = lint > L + 1 && blg + flg < 62;  // level L+1 keeps integer counts
      if (!int_next && lint > L + 1) lint = L + 1;          // the first FP64 level
      const bool from_int = L < lint;                         // level L still holds integers
      // path counts of the newly reached (vertex, source) pairs; vis and lv
      // of the new level are written only after every pull has read them.
      // Neighbours are fetched 32 at a time (id, level word, reached mask in
      // one round trip) and walked through shuffles, so the per-source loads
      // of a chunk are independent of each other.
      for (int i = hi + warp; i < nhi; i += MS_WARPS) {
        const int32_t w = queue[i];
        const uint32_t N = nxt[w];
        double a = 0.0;
        long long ai = 0;
        const int64_t eb = row[w], ee = row[w + 1];
        for (int64_t e0 = eb; e0 < ee; e0 += 32) {
          const int cnt = (int)min((int64_t)32, ee - e0);
          int32_t vj = 0;
          uint32_t mj = 0u;
          if (lane < cnt) {
            vj = g_col[e0 + lane];
            mj = at_level(lv[vj], L) & vis[vj] & N;  // neighbours' levels differ by <= 1: mod 4 is exact
          }
          if (__any_sync(0xffffffffu, mj != 0u)) {
            for (int j = 0; j < cnt; j++) {
              const uint32_t m = __shfl_sync(0xffffffffu, mj, j);
              const int32_t v = __shfl_sync(0xffffffffu, vj, j);
              if ((m >> lane) & 1u) {
                if (int_next) {
                  ai += sci[(size_t)v * 32 + lane] * (IDENT && L > 0 ? (long long)ident[v] : 1ll);
                } else {
                  double x = from_int ? i64_to_f64_pos(sci[(size_t)v * 32 + lane]) : sc[(size_t)v * 32 + lane];
                  if (IDENT && L > 0) x *= (double)ident[v];
                  a += x;
                }
              }
            }
          }
        }
        if ((N >> lane) & 1u) {
          if (int_next) sci[(size_t)w * 32 + lane] = ai;
          else sc[(size_t)w * 32 + lane] = a;
        }
      }
      __syncthreads();
      for (int i = hi + tid; i < nhi; i += MS_THREADS) {
        const int32_t w = queue[i];
        const uint32_t N = nxt[w];
        qmask[i] = N;
        vis[w] |= N;
        lv[w] = set_level(lv[w], N, L + 1);
        nxt[w] = 0;
      }
      __syncthreads();
      bound *= c.fan;
      blg += flg;
      int kadd = 0;  // exponent added to this level for source `lane`
      if (bound > 0x1p900) {  // per-source maximum of the new level
        double m = 0.0;
        for (int i = hi + warp; i < nhi; i += MS_WARPS) {
          const int32_t w = queue[i];
          if ((qmask[i] >> lane) & 1u) m = fmax(m, sc[(size_t)w * 32 + lane]);
        }
        s_red[warp][lane] = m;
        __syncthreads();
        if (tid < 32) {
          double mm = 0.0;
          for (int j = 0; j < MS_WARPS; j++) mm = fmax(mm, s_red[j][tid]);
          int kk = 0;
          if (!(mm <= DBL_MAX)) atomicOr(err, ERR_OVERFLOW);
          else if (mm > 0x1p960) kk = ilogb(mm) - 959;
          s_k[tid] = kk;
          s_red[0][tid] = kk ? scalbn(mm, -kk) : mm;
        }
        __syncthreads();
        double newb = 0.0;
        for (int j = 0; j < 32; j++) newb = fmax(newb, s_red[0][j]);
        kadd = s_k[lane];
        if (__any_sync(0xffffffffu, kadd != 0)) {
          for (int i = hi + warp; i < nhi; i += MS_WARPS) {
            const int32_t w = queue[i];
            if (kadd && ((qmask[i] >> lane) & 1u))
              sc[(size_t)w * 32 + lane] = scalbn(sc[(size_t)w * 32 + lane], -kadd);
          }
        }
        bound = newb;
        __syncthreads();
      }
      if (tid < 32) lexp[(size_t)(L + 1) * 32 + tid] = lexp[(size_t)L * 32 + tid] + kadd;
      lo = hi;
      hi = nhi;
      L++;
      if (tid == 0) qoff[L + 1] = hi;
      __syncthreads();
    }
    if (depth_fail) {
      if (tid == 0) atomicOr(err, ERR_DEPTH);
      return;  // every result of this launch is discarded by the host
    }
    const int Lmax = L;
    // ------------------------------------------------------------ phase 2
    const int32_t my_src = s_src[lane];
    const double ws = s_ws[lane];
    for (int l = Lmax; l >= 0; l--) {
      const int a = qoff[l], b = qoff[l + 1];
      const int de = l < Lmax ? lexp[(size_t)l * 32 + lane] - lexp[(size_t)(l + 1) * 32 + lane] : 0;
      const double scl = de == 0 ? 1.0 : (de < -1070 ? 0.0 : scalbn(1.0, de));
      const int my_e = lexp[(size_t)l * 32 + lane];
      for (int i = a + warp; i < b; i += MS_WARPS) {
        const int32_t v = queue[i];
        const uint32_t act = qmask[i];
        const bool on = (act >> lane) & 1u;
        double contrib = 0.0;
        // successors' coefficients: neighbours fetched 32 at a time
        double sum64 = 0.0;
        float sum32 = 0.0f;
        int ev = 0;
        float mv = 1.0f;
        double sv = 1.0;
        if (on) {
          if (l < lint) {  // an integer level
            const long long si = sci[(size_t)v * 32 + lane];
            sv = i64_to_f64_pos(si);
            if (FP32) split_pow2_i64(si, ev, mv);
          } else {
            sv = sc[(size_t)v * 32 + lane];
            if (FP32) split_pow2(sv, ev, mv);
          }
          if (FP32) ev += my_e;
        }
        if (l < Lmax) {
          const int64_t eb = row[v], ee = row[v + 1];
          for (int64_t e0 = eb; e0 < ee; e0 += 32) {
            const int cnt = (int)min((int64_t)32, ee - e0);
            int32_t wj = 0;
            uint32_t mj = 0u;
            if (lane < cnt) {
              wj = g_col[e0 + lane];
              mj = at_level(lv[wj], l + 1) & vis[wj] & act;
            }
            if (__any_sync(0xffffffffu, mj != 0u)) {
              for (int j = 0; j < cnt; j++) {
                const uint32_t m = __shfl_sync(0xffffffffu, mj, j);
                const int32_t w = __shfl_sync(0xffffffffu, wj, j);
                if ((m >> lane) & 1u) {
                  if (!FP32) {
                    sum64 += sc[(size_t)w * 32 + lane];
                  } else {
                    const Coef32 cw = ((const Coef32 *)sc)[(size_t)w * 32 + lane];
                    const int x = ev - cw.e;
                    if (x >= -126) sum32 = fmaf(cw.c, __int_as_float((127 + x) << 23), sum32);
                  }
                  dag++;
                }
              }
            }
          }
        }
        if (on) {
          const double init = REACH ? (init_f ? init_f[v] : (double)(reach[v] - 1)) : 0.0;
          double dv;
          if (!FP32) {
            if (de != 0) sum64 *= scl;
            dv = fma(sv, sum64, init);
            if (l > 0) {
              const double kv = IDENT ? (double)ident[v] : 1.0;
              sc[(size_t)v * 32 + lane] = fma(kv, dv, kv) * recip_pos(sv);
            }
          } else {
            const float df = fmaf(mv, sum32, (float)init);
            dv = (double)df;
            if (l > 0) {
              const float kv = IDENT ? (float)ident[v] : 1.0f;
              Coef32 cv;
              cv.c = fmaf(kv, df, kv) / mv;
              cv.e = ev;
              ((Coef32 *)sc)[(size_t)v * 32 + lane] = cv;
            }
          }
          if (v != my_src) contrib = ws * dv;
        }
        // bc'[v] += sum over the batch's sources, added in lane order
        for (int o = 16; o > 0; o >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, o);
        if (lane == 0 && contrib != 0.0) acc[v] += contrib;
      }
      __syncthreads();
    }
    // clear the per-vertex masks for the next batch (nxt is already 0)
    for (int i = tid; i < hi; i += MS_THREADS) vis[queue[i]] = 0u;
    __syncthreads();
  }
  if (dag_total && dag) atomicAdd(dag_total, dag);
}

// ------------------------------------------------------------ host side
template <bool R, bool I, bool F>
static int launch_ms_t(Ctx &ctx, int grid, const MsBatch *batches, int nbatch, int *counter, const CompDesc *comps,
                       const BcInput &in, const int32_t *srcs, const MsScratch &sc, int *err,
                       unsigned long long *dag) {
  k_bcreach_ms<R, I, F><<<grid, MS_THREADS, 0, ctx.stream>>>(batches, nbatch, counter, comps, in.row, in.col, in.reach,
                                                             in.ident, in.init, srcs, in.bcp, sc, err, dag);
  ctx.launches++;
  BCS_CUDA(cudaGetLastError());
  return BCS_OK;
}

#define MS_DISPATCH(R, I, F, ...)                                                                   \
  ((R) ? ((I) ? ((F) ? launch_ms_t<true, true, true>(__VA_ARGS__) : launch_ms_t<true, true, false>(__VA_ARGS__))    \
              : ((F) ? launch_ms_t<true, false, true>(__VA_ARGS__) : launch_ms_t<true, false, false>(__VA_ARGS__))) \
       : ((I) ? ((F) ? launch_ms_t<false, true, true>(__VA_ARGS__) : launch_ms_t<false, true, false>(__VA_ARGS__)) \
              : ((F) ? launch_ms_t<false, false, true>(__VA_ARGS__) : launch_ms_t<false, false, false>(__VA_ARGS__))))

// global scratch of one 32-source CTA over pieces of at most nmax vertices
static size_t ms_bytes_per_cta(int64_t nmax) {
  const int64_t qcap = 32 * nmax + 32;
  return (size_t)nmax * (4 + 4 + 8 + 8 + 256) + (size_t)qcap * 8 + (size_t)(MS_LCAP + 2) * 4 +
         (size_t)MS_LCAP * 32 * 4;
}

int ms_ctas_that_fit(int64_t nmax, int64_t *out) {
  size_t free_b = 0, total_b = 0;
  BCS_CUDA(cudaMemGetInfo(&free_b, &total_b));
  *out = (int64_t)(free_b / 2 / ms_bytes_per_cta(nmax));
  return BCS_OK;
}

int run_ms(Ctx &ctx, const std::vector<CompDesc> &comps, const std::vector<int32_t> &large, const BcInput &in,
           bool fp32, const int64_t *sources, int64_t nsources, int64_t skip, const CompDesc *d_comps, int *d_err,
           unsigned long long *d_dag, bool *depth_failed) {
  *depth_failed = false;
  std::vector<MsBatch> batches;
  std::vector<int32_t> hsrc;
  int64_t nmax = 0;
  for (int32_t ci : large) {
    const CompDesc &c = comps[ci];
    nmax = std::max<int64_t>(nmax, c.n);
    const int64_t ns = sources ? nsources : c.n;
    for (int64_t b = skip; b < ns; b += 32) {
      const int cnt = (int)std::min<int64_t>(32, ns - b);
      batches.push_back(MsBatch{ci, (int32_t)(sources ? b : b), cnt, 0});
    }
  }
  if (batches.empty()) return BCS_OK;
  if (sources) {
    hsrc.resize(nsources);
    for (int64_t i = 0; i < nsources; i++) hsrc[i] = (int32_t)sources[i];
  }
  const int64_t qcap = 32 * nmax + 32;
  const size_t per = ms_bytes_per_cta(nmax);
  size_t free_b = 0, total_b = 0;
  BCS_CUDA(cudaMemGetInfo(&free_b, &total_b));
  int64_t grid = std::min<int64_t>((int64_t)ctx.num_sms * 2, (int64_t)batches.size());
  if ((size_t)grid * per > free_b / 2) grid = std::max<int64_t>(1, (int64_t)(free_b / 2 / per));
  const size_t G = (size_t)grid, NM = (size_t)nmax;
  DBuf<MsBatch> d_batches;
  DBuf<int32_t> d_src, qq, qo, le;
  DBuf<uint32_t> qm;
  DBuf<int> counter;
  DBuf<uint32_t> vis, nxt;
  DBuf<uint64_t> lvb;
  DBuf<double> scb, accb;
  BCS_TRY(d_batches.alloc(batches.size(), ctx.stream));
  BCS_CUDA(cudaMemcpyAsync(d_batches.p, batches.data(), batches.size() * sizeof(MsBatch), cudaMemcpyHostToDevice,
                           ctx.stream));
  if (sources) {
    BCS_TRY(d_src.alloc(hsrc.size(), ctx.stream));
    BCS_CUDA(cudaMemcpyAsync(d_src.p, hsrc.data(), hsrc.size() * 4, cudaMemcpyHostToDevice, ctx.stream));
  }
  BCS_TRY(counter.alloc(1, ctx.stream));
  BCS_TRY(vis.alloc(G * NM, ctx.stream));
  BCS_TRY(nxt.alloc(G * NM, ctx.stream));
  BCS_TRY(lvb.alloc(G * NM, ctx.stream));
  BCS_TRY(scb.alloc(G * NM * 32, ctx.stream));
  BCS_TRY(accb.alloc(G * NM, ctx.stream));
  BCS_TRY(qq.alloc(G * (size_t)qcap, ctx.stream));
  BCS_TRY(qm.alloc(G * (size_t)qcap, ctx.stream));
  BCS_TRY(qo.alloc(G * (MS_LCAP + 2), ctx.stream));
  BCS_TRY(le.alloc(G * (size_t)MS_LCAP * 32, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(int), ctx.stream));
  BCS_CUDA(cudaMemsetAsync(vis.p, 0, G * NM * 4, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(nxt.p, 0, G * NM * 4, ctx.stream));
  BCS_CUDA(cudaMemsetAsync(accb.p, 0, G * NM * 8, ctx.stream));
  MsScratch sc{vis.p, nxt.p, lvb.p, scb.p, accb.p, qq.p, qm.p, qo.p, le.p, (int64_t)NM, qcap};
  // with fewer vertices than indexable levels the depth can never run out;
  // otherwise accumulate into a separate array so a failed launch leaves no trace
  const bool may_fail = nmax + 2 >= MS_LCAP;
  DBuf<double> tmp;
  BcInput tin = in;
  if (may_fail) {
    int64_t ntot = 0;
    for (const CompDesc &c : comps) ntot = std::max<int64_t>(ntot, c.vtx_off + c.n);
    BCS_TRY(tmp.alloc(ntot, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(tmp.p, 0, ntot * 8, ctx.stream));
    tin.bcp = tmp.p;
  }
  BCS_TRY(MS_DISPATCH(in.reach != nullptr || in.init != nullptr, in.ident != nullptr, fp32, ctx, (int)grid, d_batches.p,
                      (int)batches.size(), counter.p, d_comps, tin, sources ? d_src.p : nullptr, sc, d_err, d_dag));
  if (may_fail) {
    int h_err = 0;
    BCS_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
    BCS_CUDA(cudaStreamSynchronize(ctx.stream));
    if (h_err & ERR_DEPTH) {
      BCS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), ctx.stream));
      *depth_failed = true;
      return BCS_OK;
    }
    int64_t ntot = (int64_t)tmp.n;
    BCS_TRY(launch_add_f64(ctx, in.bcp, tmp.p, ntot));
  }
  ctx.stats.n_ms_batches += (int64_t)batches.size();
  ctx.stats.batch_ctas = grid;
  return BCS_OK;
}

}  // namespace bcs
