// abi.cpp - the extern "C" entry points declared in include/bcshatter.h.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <cstdio>
#include <cstdlib>

#include "common.h"

namespace bcs {

static thread_local std::string t_err;
static thread_local bcs_stats t_stats{};
static thread_local bool t_stats_valid = false;

void set_error(const std::string &msg) { t_err = msg; }

int64_t &alloc_budget() {
  static thread_local int64_t budget = -1;
  return budget;
}
const std::string &get_error() { return t_err; }

StageTimer::StageTimer(cudaStream_t stream) : s(stream) {
  cudaEventCreate(&a);
  cudaEventCreate(&b);
}
StageTimer::~StageTimer() {
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
}
void StageTimer::start() {
  if (!a) {  // handed to the call by stop_into
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  cudaEventRecord(a, s);
}
double StageTimer::stop_ms() {
  float ms = 0.f;
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  cudaEventElapsedTime(&ms, a, b);
  return (double)ms;
}
void StageTimer::stop_into(Ctx &ctx, double *dst) {
  cudaEventRecord(b, s);
  ctx.pending.push_back(Ctx::Pending{a, b, dst});
  a = b = nullptr;  // the call owns the events now; a later start() makes new ones
}
void resolve_stage_times(Ctx &ctx) {
  for (const Ctx::Pending &p : ctx.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
      *p.dst += (double)ms;
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  ctx.pending.clear();
}

static double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

Tracer::Tracer(const char *scope_name, cudaStream_t stream)
    : scope(scope_name), s(stream), on(std::getenv("BCS_TRACE") != nullptr) {
  mark("start");
}

void Tracer::mark(const char *name) {
  if (!on) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, s);
  marks.emplace_back(name, e);
  host_ms.push_back(now_ms());
}

Tracer::~Tracer() {
  if (!on || marks.empty()) return;
  cudaEventSynchronize(marks.back().second);
  std::string line = std::string("[bcs trace] ") + scope + ":";
  for (size_t i = 1; i < marks.size(); i++) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, marks[i - 1].second, marks[i].second);
    char buf[128];
    std::snprintf(buf, sizeof(buf), " %s %.3f/%.3f", marks[i].first, ms, host_ms[i] - host_ms[i - 1]);
    line += buf;
  }
  std::fprintf(stderr, "%s ms (gpu/host)\n", line.c_str());
  for (auto &m : marks) cudaEventDestroy(m.second);
}

static std::mutex g_pool_mu;
static std::set<int> g_pool_ready;

int make_ctx(const bcs_opts *opts, Ctx *ctx) {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    cudaGetLastError();
    set_error(std::string("no CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "count is 0"));
    return BCS_ENODEV;
  }
  int dev = 0;
  BCS_CUDA(cudaGetDevice(&dev));
  if (opts && opts->device >= 0) {
    if (opts->device >= count) {
      set_error("opts->device out of range");
      return BCS_EINVAL;
    }
    dev = opts->device;
  }
  BCS_CUDA(cudaSetDevice(dev));
  ctx->device = dev;
  BCS_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev));
  int optin = 0;
  BCS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  ctx->smem_optin = (size_t)optin;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_ready.count(dev)) {
      cudaMemPool_t pool;
      BCS_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
      uint64_t thr = UINT64_MAX;
      BCS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
      g_pool_ready.insert(dev);
    }
  }
  ctx->stream = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
  const int64_t mw = opts ? opts->max_wait : 0;
  ctx->max_wait = mw == 0 ? DEFAULT_MAX_WAIT : (mw < 0 ? 0 : mw);
  ctx->autotune = opts && opts->autotune;
  const char *fa = std::getenv("BCS_TEST_FAIL_ALLOC");
  alloc_budget() = fa ? std::max<int64_t>(0, std::atoll(fa)) : -1;
  if (const char *sc = std::getenv("BCS_TEST_SIGMA_CAP")) ctx->sigma_cap_lg2 = std::max(1, std::atoi(sc));
  return BCS_OK;
}

// Restores the caller's current device when a call ends.
struct DeviceGuard {
  int prev = -1;
  DeviceGuard() {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      prev = -1;
      cudaGetLastError();
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};


// ------------------------------------------------------------ input
static int check_csr(const bcs_csr *g) {
  if (!g) {
    set_error("csr is NULL");
    return BCS_EINVAL;
  }
  if (g->n < 0 || g->nnz < 0) {
    set_error("negative n or nnz");
    return BCS_EINVAL;
  }
  if (g->n >= (int64_t)INT32_MAX - 2) {
    set_error("n does not fit 32-bit vertex ids");
    return BCS_EINVAL;
  }
  if (g->n > 0 && (!g->row_ptr || (g->nnz > 0 && !g->col))) {
    set_error("row_ptr or col is NULL");
    return BCS_EINVAL;
  }
  if (g->n > 0 && !g->on_device) {
    if (g->row_ptr[0] != 0 || g->row_ptr[g->n] != g->nnz) {
      set_error("row_ptr[0] must be 0 and row_ptr[n] must equal nnz");
      return BCS_EINVAL;
    }
  }
  return BCS_OK;
}

struct Input {
  DevGraph g;
  DBuf<int64_t> rp;
  DBuf<int32_t> col;
};

static int upload_and_validate(Ctx &ctx, const bcs_csr *h, Input *in, const int64_t *batch_off = nullptr,
                               int64_t batch_count = 0) {
  in->g.n = h->n;
  in->g.nnz = h->nnz;
  if (h->on_device) {
    in->g.rp = h->row_ptr;
    in->g.col = h->col;
  } else {
    StageTimer tm(ctx.stream);
    tm.start();
    BCS_TRY(in->rp.alloc(h->n + 1, ctx.stream));
    BCS_TRY(in->col.alloc(h->nnz, ctx.stream));
    BCS_CUDA(cudaMemcpyAsync(in->rp.p, h->row_ptr, (h->n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, ctx.stream));
    if (h->nnz)
      BCS_CUDA(cudaMemcpyAsync(in->col.p, h->col, h->nnz * sizeof(int32_t), cudaMemcpyHostToDevice, ctx.stream));
    in->g.rp = in->rp.p;
    in->g.col = in->col.p;
    tm.stop_into(ctx, &ctx.stats.ms_upload);
  }
  StageTimer tm(ctx.stream);
  tm.start();
  DBuf<int> flags;
  BCS_TRY(flags.alloc(1, ctx.stream));
  BCS_TRY(launch_validate(ctx, in->g, flags.p));
  DBuf<int64_t> d_off;
  if (batch_off) {
    BCS_TRY(d_off.alloc(batch_count + 1, ctx.stream));
    BCS_CUDA(cudaMemcpyAsync(d_off.p, batch_off, (batch_count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                             ctx.stream));
    BCS_TRY(launch_validate_batch(ctx, in->g, d_off.p, batch_count, flags.p));
  }
  int f = 0;
  BCS_CUDA(cudaMemcpyAsync(&f, flags.p, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  tm.stop_into(ctx, &ctx.stats.ms_validate);
  if (f) {
    std::string m = "malformed CSR:";
    if (f & 1) m += " offsets or ids out of range;";
    if (f & 2) m += " self-loop;";
    if (f & 4) m += " row not strictly ascending (unsorted or duplicate entry);";
    if (f & 8) m += " not symmetric;";
    if (f & 16) m += " an edge joins two graphs of the batch;";
    set_error(m);
    return BCS_EINVAL;
  }
  return BCS_OK;
}

static int output_bc(Ctx &ctx, const bcs_csr *h, const double *d_bc, double *bc_out) {
  if (h->on_device) {
    if (d_bc != bc_out)
      BCS_CUDA(cudaMemcpyAsync(bc_out, d_bc, h->n * sizeof(double), cudaMemcpyDeviceToDevice, ctx.stream));
    BCS_CUDA(cudaStreamSynchronize(ctx.stream));
  } else {
    StageTimer tm(ctx.stream);
    tm.start();
    BCS_CUDA(cudaMemcpyAsync(bc_out, d_bc, h->n * sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
    tm.stop_into(ctx, &ctx.stats.ms_download);
  }
  return BCS_OK;
}

// max degree of the input (bound on path-count growth per BFS level)
static int max_degree(Ctx &ctx, const bcs_csr *h, const DevGraph &g, int64_t *out) {
  int64_t mx = 0;
  if (!h->on_device) {
    for (int64_t v = 0; v < h->n; v++) mx = std::max(mx, h->row_ptr[v + 1] - h->row_ptr[v]);
  } else {
    std::vector<int64_t> rp(h->n + 1);
    BCS_CUDA(cudaMemcpyAsync(rp.data(), g.rp, (h->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx.stream));
    BCS_CUDA(cudaStreamSynchronize(ctx.stream));
    for (int64_t v = 0; v < h->n; v++) mx = std::max(mx, rp[v + 1] - rp[v]);
  }
  *out = mx;
  return BCS_OK;
}

// ------------------------------------------------------------ plain
static int plain_impl(Ctx &ctx, const bcs_csr *h, const int64_t *src, int64_t k, double *bc_out, BcPlanOpts po) {
  Input in;
  BCS_TRY(upload_and_validate(ctx, h, &in));
  DBuf<double> bc;
  double *d_bc = bc_out;
  if (!h->on_device) {
    BCS_TRY(bc.alloc(h->n, ctx.stream));
    d_bc = bc.p;
  }
  BCS_CUDA(cudaMemsetAsync(d_bc, 0, h->n * sizeof(double), ctx.stream));
  int64_t mxd = 0;
  BCS_TRY(max_degree(ctx, h, in.g, &mxd));
  std::vector<CompDesc> comps(1);
  comps[0] = CompDesc{0, 0, (int32_t)h->n, (int32_t)mxd, h->nnz, (double)std::max<int64_t>(mxd, 1)};
  BcInput bi;
  bi.row = in.g.rp;
  bi.col = in.g.col;
  bi.bcp = d_bc;
  po.sources = src;
  po.nsources = k;
  BCS_TRY(run_bcreach(ctx, comps, bi, po));
  ctx.stats.n_pieces = 1;
  ctx.stats.n_slots = ctx.stats.n_merged = h->n;
  ctx.stats.n_entries = h->nnz;
  ctx.stats.work_nm = (double)h->n * (double)(h->nnz / 2);
  return output_bc(ctx, h, d_bc, bc_out);
}

// ------------------------------------------------------------ shattered
struct Shattered {
  DBuf<int64_t> bcpre;
  DevPieces pc;
  DevMerged merged;
  std::vector<CompDesc> comps;
};

static int shatter_impl(Ctx &ctx, const bcs_csr *h, const Input &in, uint32_t steps, Shattered *S) {
  const int64_t n = h->n;
  const bool D = steps & BCS_STEP_D, A = steps & BCS_STEP_A, I = steps & BCS_STEP_I;
  DBuf<int32_t> label, reach;
  DBuf<int64_t> N;
  DBuf<uint8_t> alive;
  BCS_TRY(label.alloc(n, ctx.stream));
  BCS_TRY(N.alloc(n, ctx.stream));
  BCS_TRY(reach.alloc(n, ctx.stream));
  BCS_TRY(alive.alloc(n, ctx.stream));
  BCS_TRY(S->bcpre.alloc(n, ctx.stream));
  Tracer tr("shatter", ctx.stream);
  {
    StageTimer tm(ctx.stream);
    tm.start();
    BCS_TRY(launch_cc(ctx, in.g, label.p, N.p));
    tm.stop_into(ctx, &ctx.stats.ms_cc);
  }
  {
    StageTimer tm(ctx.stream);
    tm.start();
    if (D) {
      BCS_TRY(run_peel(ctx, in.g, N.p, alive.p, reach.p, S->bcpre.p));
    } else {
      BCS_CUDA(cudaMemsetAsync(alive.p, 1, n, ctx.stream));
      BCS_TRY(launch_fill_i32(ctx, reach.p, n, 1));
      BCS_CUDA(cudaMemsetAsync(S->bcpre.p, 0, n * sizeof(int64_t), ctx.stream));
    }
    tm.stop_into(ctx, &ctx.stats.ms_peel);
  }
  tr.mark("cc+peel");
  {
    StageTimer tm(ctx.stream);
    tm.start();
    BCS_TRY(device_pieces(ctx, in.g, alive.p, reach.p, N.p, label.p, A, &S->pc));
    tm.stop_into(ctx, &ctx.stats.ms_blocks);
  }
  tr.mark("pieces");
  {
    StageTimer tm(ctx.stream);
    tm.start();
    BCS_TRY(device_merge(ctx, S->pc, I, (steps & BCS_STEP_U) != 0, &S->merged));
    tm.stop_into(ctx, &ctx.stats.ms_ident);
  }
  tr.mark("merge");
  // component descriptors
  const DevMerged &m = S->merged;
  const int64_t P = m.npieces;
  S->comps.resize(P);
  double work_nm = 0.0;
  for (int64_t p = 0; p < P; p++) {
    CompDesc c;
    c.vtx_off = m.h_piece_off[p];
    c.row_off = m.h_piece_off[p];
    c.n = (int32_t)(m.h_piece_off[p + 1] - m.h_piece_off[p]);
    c.maxdeg = std::max<int32_t>(1, m.h_piece_maxdeg[p]);
    c.nnz = m.h_piece_ent[p];
    // sum of ident over a merged vertex's neighbours <= its degree before merging
    c.fan = (double)c.maxdeg;
    S->comps[p] = c;
    work_nm += (double)c.n * (double)(c.nnz / 2);
  }
  ctx.stats.n_pieces = P;
  ctx.stats.n_slots = m.nslots;
  ctx.stats.n_merged = m.nmerged;
  ctx.stats.n_entries = m.nentries;
  ctx.stats.work_nm = work_nm;
  return BCS_OK;
}

static int shattered_impl(Ctx &ctx, const bcs_csr *h, const bcs_opts *o, double *bc_out,
                          const int64_t *batch_off = nullptr, int64_t batch_count = 0) {
  Tracer tr("shattered", ctx.stream);
  Input in;
  BCS_TRY(upload_and_validate(ctx, h, &in, batch_off, batch_count));
  tr.mark("validate");
  const uint32_t steps = o ? o->steps : BCS_STEPS_ALL;
  Shattered S;
  BCS_TRY(shatter_impl(ctx, h, in, steps, &S));
  tr.mark("shatter");
  DevMerged &m = S.merged;
  BcInput bi;
  bi.row = m.mrow.p;
  bi.col = m.mcol.p;
  bi.reach = (steps & (BCS_STEP_D | BCS_STEP_A)) ? m.mreach.p : nullptr;
  bi.ident = (steps & BCS_STEP_I) ? m.mident.p : nullptr;
  bi.init = m.minit.p;  // classes of unequal reach only
  bi.bcp = m.mcorr.p;  // starts with the identical-vertex terms
  BcPlanOpts po;
  po.fp32_delta = o && o->delta_fp32;
  if (steps & BCS_STEP_L)
    BCS_TRY(run_bcreach_resplit(ctx, m, bi, po));
  else if (steps & BCS_STEP_S)
    BCS_TRY(run_bcreach_side(ctx, m, S.comps, bi, po, h->n));
  else
    BCS_TRY(run_bcreach(ctx, S.comps, bi, po));
  tr.mark("bcreach");
  DBuf<double> bc;
  double *d_bc = bc_out;
  if (!h->on_device) {
    BCS_TRY(bc.alloc(h->n, ctx.stream));
    d_bc = bc.p;
  }
  {
    StageTimer tm(ctx.stream);
    tm.start();
    BCS_TRY(launch_bc_init(ctx, h->n, S.bcpre.p, d_bc));
    BCS_TRY(launch_mapback(ctx, m.nslots, m.slot_org.p, m.slot_to_m.p, m.mcorr.p, d_bc, m.slot_corr.p));
    tm.stop_into(ctx, &ctx.stats.ms_mapback);
  }
  tr.mark("mapback");
  return output_bc(ctx, h, d_bc, bc_out);
}

// BCS_STEP_O: run `run(renumbered csr, device bc of it, inv)` on the graph
// renumbered in BFS order, then map bc back to the caller's ids.
template <class F>
static int with_bfs_order(Ctx &ctx, const bcs_csr *h, double *bc_out, F &&run) {
  Input in;
  BCS_TRY(upload_and_validate(ctx, h, &in));
  DBuf<int64_t> rp2;
  DBuf<int32_t> col2, inv;
  BCS_TRY(bfs_order_graph(ctx, in.g, &rp2, &col2, &inv));
  bcs_csr h2{h->n, h->nnz, rp2.p, col2.p, 1};
  DBuf<double> bc2, bcd;
  BCS_TRY(bc2.alloc(h->n, ctx.stream));
  BCS_TRY(run(&h2, bc2.p, inv.p));
  double *d_bc = bc_out;
  if (!h->on_device) {
    BCS_TRY(bcd.alloc(h->n, ctx.stream));
    d_bc = bcd.p;
  }
  BCS_TRY(launch_order_map_back(ctx, h->n, inv.p, bc2.p, d_bc));
  return output_bc(ctx, h, d_bc, bc_out);
}

}  // namespace bcs

// step S (side vertices) takes integer target weights: not with U or L,
// whose weights are fractional; U and L go together (the loop's merges are
// of unequal weight anyway)
static bool optional_steps_compatible(uint32_t steps) {
  return !((steps & BCS_STEP_S) && (steps & (BCS_STEP_U | BCS_STEP_L)));
}

// ================================================================ C ABI
using namespace bcs;

struct bcs_components {
  int64_t n = 0;
  std::vector<int64_t> piece_vtx_off, piece_N, row_ptr, member_off, bc_pre;
  std::vector<int32_t> col, org, reach, ident, member;
  std::vector<double> bc_corr;
};

template <class F>
static int guarded(const bcs_opts *opts, F &&body) {
  DeviceGuard dg;
  try {
    double t0 = now_ms();
    Ctx ctx;
    int rc = make_ctx(opts, &ctx);
    if (rc != BCS_OK) return rc;
    rc = body(ctx);
    resolve_stage_times(ctx);
    if (rc == BCS_OK) {
      ctx.stats.ms_total = now_ms() - t0;
      ctx.stats.kernel_launches = ctx.launches;
      t_stats = ctx.stats;
      t_stats_valid = true;
    }
    return rc;
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    return BCS_ENOMEM;
  } catch (const std::exception &e) {
    set_error(std::string("internal error: ") + e.what());
    return BCS_ECUDA;
  }
}

extern "C" {

__attribute__((visibility("default"))) int bcs_bc_plain(const bcs_csr *csr, const bcs_opts *opts, double *bc_out) {
  int rc = check_csr(csr);
  if (rc != BCS_OK) return rc;
  if (csr->n == 0) return BCS_OK;
  if (!bc_out) {
    set_error("bc_out is NULL");
    return BCS_EINVAL;
  }
  return guarded(opts, [&](Ctx &ctx) {
    BcPlanOpts po;
    po.fp32_delta = opts && opts->delta_fp32;
    if (opts && (opts->steps & BCS_STEP_O))
      return with_bfs_order(ctx, csr, bc_out, [&](const bcs_csr *h2, double *bc2, const int32_t *) {
        return plain_impl(ctx, h2, nullptr, 0, bc2, po);
      });
    return plain_impl(ctx, csr, nullptr, 0, bc_out, po);
  });
}

__attribute__((visibility("default"))) int bcs_bc_shattered(const bcs_csr *csr, const bcs_opts *opts,
                                                            double *bc_out) {
  int rc = check_csr(csr);
  if (rc != BCS_OK) return rc;
  if (csr->n == 0) return BCS_OK;
  if (!bc_out) {
    set_error("bc_out is NULL");
    return BCS_EINVAL;
  }
  if (opts && (opts->steps & ~(BCS_STEPS_ALL | BCS_STEP_O | BCS_STEP_S | BCS_STEP_U | BCS_STEP_L))) {
    set_error("unknown bits in opts->steps");
    return BCS_EINVAL;
  }
  if (opts && !optional_steps_compatible(opts->steps)) {
    set_error("BCS_STEP_S does not combine with BCS_STEP_U or BCS_STEP_L");
    return BCS_EINVAL;
  }
  return guarded(opts, [&](Ctx &ctx) {
    if (opts && (opts->steps & BCS_STEP_O)) {
      bcs_opts o2 = *opts;
      o2.steps &= BCS_STEPS_ALL | BCS_STEP_S | BCS_STEP_U | BCS_STEP_L;
      return with_bfs_order(ctx, csr, bc_out, [&](const bcs_csr *h2, double *bc2, const int32_t *) {
        return shattered_impl(ctx, h2, &o2, bc2);
      });
    }
    return shattered_impl(ctx, csr, opts, bc_out);
  });
}

__attribute__((visibility("default"))) int bcs_bc_shattered_batch(const int64_t *graph_vtx_off, int64_t count,
                                                                  const bcs_csr *packed, const bcs_opts *opts,
                                                                  double *bc_out) {
  int rc = check_csr(packed);
  if (rc != BCS_OK) return rc;
  if (count < 1 || !graph_vtx_off) {
    set_error("a batch needs count >= 1 graphs and their vertex offsets");
    return BCS_EINVAL;
  }
  if (graph_vtx_off[0] != 0 || graph_vtx_off[count] != packed->n) {
    set_error("graph_vtx_off must start at 0 and end at n");
    return BCS_EINVAL;
  }
  for (int64_t g = 0; g < count; g++)
    if (graph_vtx_off[g + 1] < graph_vtx_off[g]) {
      set_error("graph_vtx_off must be ascending");
      return BCS_EINVAL;
    }
  if (opts && ((opts->steps & ~(BCS_STEPS_ALL | BCS_STEP_S | BCS_STEP_U | BCS_STEP_L)) ||
                !optional_steps_compatible(opts->steps))) {
    set_error("unknown bits in opts->steps");
    return BCS_EINVAL;
  }
  if (packed->n == 0) return BCS_OK;
  if (!bc_out) {
    set_error("bc_out is NULL");
    return BCS_EINVAL;
  }
  return guarded(opts, [&](Ctx &ctx) { return shattered_impl(ctx, packed, opts, bc_out, graph_vtx_off, count); });
}

__attribute__((visibility("default"))) int bcs_bc_sources(const bcs_csr *csr, const int64_t *src, int64_t k,
                                                          const bcs_opts *opts, double *bc_out) {
  int rc = check_csr(csr);
  if (rc != BCS_OK) return rc;
  if (k < 0 || (k > 0 && !src)) {
    set_error("bad source list");
    return BCS_EINVAL;
  }
  for (int64_t i = 0; i < k; i++)
    if (src[i] < 0 || src[i] >= csr->n) {
      set_error("source id out of range");
      return BCS_EINVAL;
    }
  if (csr->n == 0) return BCS_OK;
  if (!bc_out) {
    set_error("bc_out is NULL");
    return BCS_EINVAL;
  }
  return guarded(opts, [&](Ctx &ctx) {
    BcPlanOpts po;
    po.fp32_delta = opts && opts->delta_fp32;
    if (k == 0) {
      Input in;
      BCS_TRY(upload_and_validate(ctx, csr, &in));
      if (csr->on_device) {
        BCS_CUDA(cudaMemsetAsync(bc_out, 0, csr->n * sizeof(double), ctx.stream));
        BCS_CUDA(cudaStreamSynchronize(ctx.stream));
      } else {
        std::memset(bc_out, 0, csr->n * sizeof(double));
      }
      return BCS_OK;
    }
    if (opts && (opts->steps & BCS_STEP_O))
      return with_bfs_order(ctx, csr, bc_out, [&](const bcs_csr *h2, double *bc2, const int32_t *inv) {
        std::vector<int64_t> src2;
        BCS_TRY(map_sources_to_order(ctx, src, k, inv, &src2));
        return plain_impl(ctx, h2, src2.data(), k, bc2, po);
      });
    return plain_impl(ctx, csr, src, k, bc_out, po);
  });
}

__attribute__((visibility("default"))) int bcs_debug_sssp(const bcs_csr *csr, int64_t s, const bcs_opts *opts,
                                                          int32_t *d, double *sigma_mant, int32_t *sigma_exp2,
                                                          double *delta) {
  int rc = check_csr(csr);
  if (rc != BCS_OK) return rc;
  if (s < 0 || s >= csr->n) {
    set_error("source out of range");
    return BCS_EINVAL;
  }
  return guarded(opts, [&](Ctx &ctx) {
    const int64_t n = csr->n;
    DBuf<int32_t> dd, de;
    DBuf<double> ds, ddl, bc;
    BCS_TRY(dd.alloc(n, ctx.stream));
    BCS_TRY(de.alloc(n, ctx.stream));
    BCS_TRY(ds.alloc(n, ctx.stream));
    BCS_TRY(ddl.alloc(n, ctx.stream));
    BCS_TRY(bc.alloc(n, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(dd.p, 0xFF, n * 4, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(de.p, 0, n * 4, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(ds.p, 0, n * 8, ctx.stream));
    BCS_CUDA(cudaMemsetAsync(ddl.p, 0, n * 8, ctx.stream));
    BcPlanOpts po;
    po.fp32_delta = opts && opts->delta_fp32;
    po.dbg_d = dd.p;
    po.dbg_sig = ds.p;
    po.dbg_exp = de.p;
    po.dbg_delta = ddl.p;
    bcs_csr hcsr = *csr;
    // outputs of this call are host arrays; the bc sum goes to a scratch array
    const bool dev_in = csr->on_device != 0;
    int64_t src = s;
    Input in;
    BCS_TRY(upload_and_validate(ctx, csr, &in));
    int64_t mxd = 0;
    BCS_TRY(max_degree(ctx, csr, in.g, &mxd));
    std::vector<CompDesc> comps(1);
    comps[0] = CompDesc{0, 0, (int32_t)n, (int32_t)mxd, csr->nnz, (double)std::max<int64_t>(mxd, 1)};
    BcInput bi;
    bi.row = in.g.rp;
    bi.col = in.g.col;
    bi.bcp = bc.p;
    BCS_CUDA(cudaMemsetAsync(bc.p, 0, n * 8, ctx.stream));
    po.sources = &src;
    po.nsources = 1;
    (void)hcsr;
    (void)dev_in;
    BCS_TRY(run_bcreach(ctx, comps, bi, po));
    if (d) BCS_CUDA(cudaMemcpyAsync(d, dd.p, n * 4, cudaMemcpyDeviceToHost, ctx.stream));
    if (sigma_mant) BCS_CUDA(cudaMemcpyAsync(sigma_mant, ds.p, n * 8, cudaMemcpyDeviceToHost, ctx.stream));
    if (sigma_exp2) BCS_CUDA(cudaMemcpyAsync(sigma_exp2, de.p, n * 4, cudaMemcpyDeviceToHost, ctx.stream));
    if (delta) BCS_CUDA(cudaMemcpyAsync(delta, ddl.p, n * 8, cudaMemcpyDeviceToHost, ctx.stream));
    BCS_CUDA(cudaStreamSynchronize(ctx.stream));
    return BCS_OK;
  });
}

__attribute__((visibility("default"))) int bcs_shatter(const bcs_csr *csr, const bcs_opts *opts,
                                                       bcs_components **out) {
  int rc = check_csr(csr);
  if (rc != BCS_OK) return rc;
  if (!out) {
    set_error("out is NULL");
    return BCS_EINVAL;
  }
  if (opts && (opts->steps & ~BCS_STEPS_ALL)) {
    set_error("unknown bits in opts->steps");
    return BCS_EINVAL;
  }
  *out = nullptr;
  auto *c = new (std::nothrow) bcs_components();
  if (!c) {
    set_error("host allocation failed");
    return BCS_ENOMEM;
  }
  c->n = csr->n;
  if (csr->n == 0) {
    c->piece_vtx_off.assign(1, 0);
    c->row_ptr.assign(1, 0);
    c->member_off.assign(1, 0);
    *out = c;
    return BCS_OK;
  }
  rc = guarded(opts, [&](Ctx &ctx) {
    Input in;
    BCS_TRY(upload_and_validate(ctx, csr, &in));
    Shattered S;
    BCS_TRY(shatter_impl(ctx, csr, in, opts ? opts->steps : BCS_STEPS_ALL, &S));
    const DevMerged &m = S.merged;
    const int64_t M = m.nmerged, E = m.nentries, SL = m.nslots, n = csr->n;
    c->piece_vtx_off = m.h_piece_off;
    c->piece_N.resize(m.npieces);
    if (m.npieces)
      BCS_CUDA(cudaMemcpyAsync(c->piece_N.data(), m.piece_N.p, m.npieces * 8, cudaMemcpyDeviceToHost, ctx.stream));
    c->row_ptr.resize(M + 1);
    c->col.resize(E);
    c->org.resize(M);
    c->reach.resize(M);
    c->ident.resize(M);
    c->bc_corr.resize(M);
    c->bc_pre.resize(n);
    std::vector<int32_t> s2m(SL), sorg(SL);
    BCS_CUDA(cudaMemcpyAsync(c->row_ptr.data(), m.mrow.p, (M + 1) * 8, cudaMemcpyDeviceToHost, ctx.stream));
    if (E) BCS_CUDA(cudaMemcpyAsync(c->col.data(), m.mcol.p, E * 4, cudaMemcpyDeviceToHost, ctx.stream));
    if (M) {
      BCS_CUDA(cudaMemcpyAsync(c->org.data(), m.morg.p, M * 4, cudaMemcpyDeviceToHost, ctx.stream));
      BCS_CUDA(cudaMemcpyAsync(c->reach.data(), m.mreach.p, M * 4, cudaMemcpyDeviceToHost, ctx.stream));
      BCS_CUDA(cudaMemcpyAsync(c->ident.data(), m.mident.p, M * 4, cudaMemcpyDeviceToHost, ctx.stream));
      BCS_CUDA(cudaMemcpyAsync(c->bc_corr.data(), m.mcorr.p, M * 8, cudaMemcpyDeviceToHost, ctx.stream));
    }
    if (SL) {
      BCS_CUDA(cudaMemcpyAsync(s2m.data(), m.slot_to_m.p, SL * 4, cudaMemcpyDeviceToHost, ctx.stream));
      BCS_CUDA(cudaMemcpyAsync(sorg.data(), m.slot_org.p, SL * 4, cudaMemcpyDeviceToHost, ctx.stream));
    }
    BCS_CUDA(cudaMemcpyAsync(c->bc_pre.data(), S.bcpre.p, n * 8, cudaMemcpyDeviceToHost, ctx.stream));
    BCS_CUDA(cudaStreamSynchronize(ctx.stream));
    // members: pre-merge slots grouped by merged vertex, each list ascending
    c->member_off.assign(M + 1, 0);
    for (int64_t x = 0; x < SL; x++) c->member_off[s2m[x] + 1]++;
    for (int64_t i = 0; i < M; i++) c->member_off[i + 1] += c->member_off[i];
    c->member.resize(SL);
    std::vector<int64_t> pos(c->member_off.begin(), c->member_off.end() - 1);
    for (int64_t x = 0; x < SL; x++) c->member[pos[s2m[x]]++] = sorg[x];
    for (int64_t i = 0; i < M; i++)
      std::sort(c->member.begin() + c->member_off[i], c->member.begin() + c->member_off[i + 1]);
    return BCS_OK;
  });
  if (rc != BCS_OK) {
    delete c;
    return rc;
  }
  *out = c;
  return BCS_OK;
}

__attribute__((visibility("default"))) int bcs_components_get(const bcs_components *c, bcs_components_view *v) {
  if (!c || !v) {
    set_error("NULL argument");
    return BCS_EINVAL;
  }
  v->n = c->n;
  v->n_pieces = (int64_t)c->piece_vtx_off.size() - 1;
  v->n_merged = (int64_t)c->org.size();
  v->n_entries = (int64_t)c->col.size();
  v->n_members = (int64_t)c->member.size();
  v->piece_vtx_off = c->piece_vtx_off.data();
  v->piece_N = c->piece_N.data();
  v->row_ptr = c->row_ptr.data();
  v->col = c->col.data();
  v->org = c->org.data();
  v->reach = c->reach.data();
  v->ident = c->ident.data();
  v->member_off = c->member_off.data();
  v->member = c->member.data();
  v->bc_pre = c->bc_pre.data();
  v->bc_corr = c->bc_corr.data();
  return BCS_OK;
}

__attribute__((visibility("default"))) void bcs_components_free(bcs_components *c) { delete c; }

__attribute__((visibility("default"))) int bcs_last_stats(bcs_stats *out) {
  if (!out) {
    set_error("NULL argument");
    return BCS_EINVAL;
  }
  if (!t_stats_valid) {
    set_error("no successful call yet on this thread");
    return BCS_EINVAL;
  }
  *out = t_stats;
  return BCS_OK;
}

__attribute__((visibility("default"))) const char *bcs_last_error(void) { return t_err.c_str(); }

__attribute__((visibility("default"))) int bcs_version(void) { return 100; }

}  // extern "C"
