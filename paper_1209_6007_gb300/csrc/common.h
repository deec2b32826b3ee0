// common.h - internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/bcshatter.h"

namespace bcs {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
const std::string &get_error();

struct Status {
  int code = BCS_OK;
  bool ok() const { return code == BCS_OK; }
};

#define BCS_CUDA(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      ::bcs::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));              \
      return (e_ == cudaErrorMemoryAllocation) ? BCS_ENOMEM : BCS_ECUDA;                 \
    }                                                                                    \
  } while (0)

// call FN<R, I, F>(...) for runtime flags R, I, F
#define BCS_DISPATCH3(FN, R, I, F, ...)                             \
  ((R) ? ((I) ? ((F) ? FN<true, true, true>(__VA_ARGS__)            \
                     : FN<true, true, false>(__VA_ARGS__))          \
              : ((F) ? FN<true, false, true>(__VA_ARGS__)           \
                     : FN<true, false, false>(__VA_ARGS__)))        \
       : ((I) ? ((F) ? FN<false, true, true>(__VA_ARGS__)           \
                     : FN<false, true, false>(__VA_ARGS__))         \
              : ((F) ? FN<false, false, true>(__VA_ARGS__)          \
                     : FN<false, false, false>(__VA_ARGS__))))

#define BCS_TRY(expr)        \
  do {                       \
    int rc_ = (expr);        \
    if (rc_ != BCS_OK) return rc_; \
  } while (0)

// Test hooks set per call from the environment (host side only; nothing
// reaches the GPU through them):
//   BCS_TEST_FAIL_ALLOC=k  the call's device allocations after the first k
//                          fail as if the device were out of memory;
//   BCS_TEST_SIGMA_CAP=k   path counts above 2^k count as out of range (the
//                          whole-GPU Bc-Reach kernel reports BCS_EOVERFLOW).
// alloc_budget() < 0: no limit.
int64_t &alloc_budget();

// ------------------------------------------------------- device buffers
// Stream-ordered device allocation from the device's default memory pool
// (its release threshold is raised once per device so freed blocks stay
// cached between calls).
template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  cudaStream_t s = 0;
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  void swap(DBuf &o) {
    std::swap(p, o.p);
    std::swap(n, o.n);
    std::swap(s, o.s);
  }
  int alloc(size_t count, cudaStream_t stream) {
    release();
    int64_t &budget = alloc_budget();
    if (budget == 0) {
      set_error("device allocation refused by BCS_TEST_FAIL_ALLOC");
      return BCS_ENOMEM;
    }
    if (budget > 0) budget--;
    s = stream;
    n = count;
    size_t bytes = (count > 0 ? count : 1) * sizeof(T);
    cudaError_t e = cudaMallocAsync((void **)&p, bytes, stream);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error(std::string("cudaMallocAsync(") + std::to_string(bytes) + " B): " + cudaGetErrorString(e));
      return BCS_ENOMEM;
    }
    return BCS_OK;
  }
};

// ------------------------------------------------------- call context
struct Ctx {
  // stage times resolved when the call ends: (start, stop, stat to add to)
  struct Pending {
    cudaEvent_t a, b;
    double *dst;
  };
  std::vector<Pending> pending;
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  cudaStream_t stream = 0;
  bcs_stats stats{};
  bool timing = true;
  int64_t launches = 0;
  // spin limit of device-side waits (grid barriers); < 0: give up at once
  int64_t max_wait = 0;
  bool autotune = false;
  // binary exponent above which a path count counts as out of range
  // (BCS_TEST_SIGMA_CAP; else effectively unlimited)
  int sigma_cap_lg2 = 1 << 30;
};

// Default number of polls (each followed by a short sleep) a device-side
// wait makes before it gives up and reports BCS_ETIMEOUT (about a second).
constexpr int64_t DEFAULT_MAX_WAIT = 1 << 24;

int make_ctx(const bcs_opts *opts, Ctx *ctx);

// CUDA-event stopwatch on the call's stream.
struct StageTimer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s = 0;
  StageTimer(cudaStream_t stream);
  ~StageTimer();
  void start();
  double stop_ms();  // synchronises on the stop event (for a choice taken now)
  // records the stop without waiting; *dst gains the time when the call
  // ends (resolve_stage_times), so the host runs ahead of the device
  void stop_into(Ctx &ctx, double *dst);
};
// add every pending stage time to its stat and release the events
void resolve_stage_times(Ctx &ctx);

// Optional per-stage trace: with the environment variable BCS_TRACE set,
// marks are CUDA events on the call's stream and the gaps between them are
// printed to stderr when the tracer goes out of scope, each with the host
// time that passed between the same marks (a host step shows up as GPU time
// well below host time).
struct Tracer {
  const char *scope;
  cudaStream_t s;
  bool on;
  std::vector<std::pair<const char *, cudaEvent_t>> marks;
  std::vector<double> host_ms;  // host clock at each mark
  Tracer(const char *scope_name, cudaStream_t stream);
  ~Tracer();
  void mark(const char *name);
};

// ------------------------------------------------------- graph on device
struct DevGraph {
  int64_t n = 0, nnz = 0;
  const int64_t *rp = nullptr;
  const int32_t *col = nullptr;
};

// Pieces (components of the shattered graph) before identical merging, on
// the device: slots are (piece, original vertex) pairs, contiguous per piece;
// scol holds global slot ids; each row is in ascending original id.
struct DevPieces {
  int64_t npieces = 0, nslots = 0, nentries = 0;
  DBuf<int64_t> piece_off;     // npieces+1 (slot offsets)
  DBuf<int64_t> piece_N;       // npieces
  DBuf<int64_t> srow;          // nslots+1
  DBuf<int32_t> slot_org;      // nslots
  DBuf<int32_t> slot_reach;    // nslots
  DBuf<int32_t> slot_piece;    // nslots
  DBuf<int32_t> scol;          // nentries
  DBuf<int32_t> piece_maxdeg;  // npieces
};

// Build the pieces from the graph left by degree-1 removal: alive[v] vertex
// still present, reach[v] its reach, N[v] size of its connected component in
// the input, label[v] that component's id.  art: biconnected components
// (else connected components).
int device_pieces(Ctx &ctx, const DevGraph &g, const uint8_t *alive, const int32_t *reach, const int64_t *N,
                  const int32_t *label, bool art, DevPieces *out);

// Stable LSD radix sort of (key, value) pairs; keys < 2^key_bits.
int radix_sort_pairs(Ctx &ctx, uint32_t *keys, int32_t *vals, uint32_t *tk, int32_t *tv, int64_t n, int key_bits);

// Pieces after identical merging, on the device.
struct DevMerged {
  int64_t npieces = 0, nmerged = 0, nentries = 0, nslots = 0;
  DBuf<int64_t> piece_off;   // npieces+1 (merged vertex offsets)
  DBuf<int64_t> piece_N;     // npieces
  DBuf<int64_t> mrow;        // nmerged+1
  DBuf<int32_t> mcol;        // nentries (local ids)
  DBuf<int32_t> morg;        // nmerged
  DBuf<int32_t> mreach;      // nmerged
  DBuf<int32_t> mident;      // nmerged
  DBuf<double> mcorr;        // nmerged
  DBuf<int32_t> slot_org;    // nslots (pre-merge)
  DBuf<int32_t> slot_to_m;   // nslots -> merged vertex
  // classes of unequal reach only: the merged vertex's dependency start
  // (sum of its members' reach) / ident - 1, and each copy's own terms
  DBuf<double> minit;        // nmerged
  DBuf<double> slot_corr;    // nslots
  std::vector<int64_t> h_piece_off;  // host copies for planning
  std::vector<int64_t> h_piece_ent;  // entries per piece
  std::vector<int32_t> h_piece_maxdeg;  // largest degree per piece before merging
};

// identical: merge identical vertices; unequal: key classes on the
// neighbourhood alone (members may differ in reach); sub_k (nullable, with
// unequal): slot x stands for sub_k[x] members whose weights sum to its reach
int device_merge(Ctx &ctx, DevPieces &pc, bool identical, bool unequal, DevMerged *out,
                 const int32_t *sub_k = nullptr);

// ------------------------------------------------------- graph kernels
int launch_validate(Ctx &ctx, const DevGraph &g, int *d_flags);
int launch_validate_batch(Ctx &ctx, const DevGraph &g, const int64_t *d_vtx_off, int64_t count, int *d_flags);
int launch_cc(Ctx &ctx, const DevGraph &g, int32_t *d_label, int64_t *d_N);
int run_peel(Ctx &ctx, const DevGraph &g, const int64_t *d_N, uint8_t *d_alive, int32_t *d_reach,
             int64_t *d_bcpre);
int launch_bc_init(Ctx &ctx, int64_t n, const int64_t *d_bcpre, double *d_bc);
// bc[org of slot] += bcp[merged vertex of slot] (+ slot_corr[slot], nullable)
int launch_mapback(Ctx &ctx, int64_t nslots, const int32_t *slot_org, const int32_t *slot_to_m,
                   const double *bcp, double *d_bc, const double *slot_corr = nullptr);
int launch_fill_i32(Ctx &ctx, int32_t *p, int64_t n, int32_t v);
int launch_fill_i64(Ctx &ctx, int64_t *p, int64_t n, int64_t v);
int launch_add_f64(Ctx &ctx, double *dst, const double *src, int64_t n);
int launch_exclusive_scan(Ctx &ctx, const int64_t *in, int64_t *out, int64_t n, int64_t *d_total);

// ------------------------------------------------------- BFS ordering
// Renumber g in BFS order (order.cu): rp2/col2 the renumbered CSR (rows
// ascending), inv[old id] = new id.
int bfs_order_graph(Ctx &ctx, const DevGraph &g, DBuf<int64_t> *rp2, DBuf<int32_t> *col2, DBuf<int32_t> *inv);
// bc[v] = bc2[inv[v]]
int launch_order_map_back(Ctx &ctx, int64_t n, const int32_t *inv, const double *bc2, double *bc);
// the new ids of a host list of source ids (host result)
int map_sources_to_order(Ctx &ctx, const int64_t *src, int64_t k, const int32_t *inv, std::vector<int64_t> *out);

// ------------------------------------------------------- Bc-Reach
// One component handed to the Bc-Reach kernels.
struct CompDesc {
  int64_t vtx_off;  // first vertex (global index into reach/ident/bcp arrays)
  int64_t row_off;  // pointer to row offsets: row[vtx_off .. vtx_off+n]
  int32_t n;        // vertices
  int32_t maxdeg;   // largest degree
  int64_t nnz;      // CSR entries
  double fan;       // bound on sigma growth per level (max over v of sum of
                    // ident over its neighbours)
  // sources: with a source map, the piece's sources are the local ids
  // map[src_off .. src_off + nsrc); src_off < 0: every vertex 0..n-1
  int64_t src_off = -1;
  int32_t nsrc = -1;  // < 0: n
};
__host__ __device__ inline int64_t nsrc_of(const CompDesc &c) { return c.nsrc >= 0 ? c.nsrc : c.n; }

struct BcInput {
  const int64_t *row = nullptr;   // global row offsets (indexed by vertex)
  const int32_t *col = nullptr;   // local neighbour ids
  const int32_t *reach = nullptr; // nullable (all 1)
  const int32_t *ident = nullptr; // nullable (all 1)
  // nullable: the dependency start reach - 1 as FP64, possibly fractional
  // (a class of unequal reaches merged into one vertex); when given it
  // replaces reach, and the source weight is (init + 1) * ident
  const double *init = nullptr;
  double *bcp = nullptr;          // accumulation target, indexed by vertex
};

enum { LARGE_PATH_AUTO = 0, LARGE_PATH_WIDE = 1, LARGE_PATH_BATCHED = 2, LARGE_PATH_PER_SOURCE = 3, LARGE_PATH_MID = 4 };

struct BcPlanOpts {
  bool fp32_delta = false;
  const int64_t *sources = nullptr;  // host; nullable = every vertex
  int64_t nsources = 0;
  // device source map of the pieces whose src_off >= 0 (local ids, int64);
  // large pieces then run one source per CTA
  const int64_t *srcmap = nullptr;
  bool force_large = false;           // route every piece through the global path
  bool per_source_large = false;      // large pieces one source per CTA (no 32-source batches)
  // large-piece kernel: 0 chosen by the plan (or the autotuner), else one of
  // the LARGE_PATH_* values (the BCS_LARGE_PATH variable overrides it)
  int large_path = 0;
  // shared memory a piece may need for one source to take the small path
  // (0: the default limit); set by the autotuner's threshold candidates
  size_t small_limit = 0;
  // debug output for a single source (large path only)
  int32_t *dbg_d = nullptr;
  double *dbg_sig = nullptr;
  int32_t *dbg_exp = nullptr;
  double *dbg_delta = nullptr;
};

// Bc-Reach with 32 sources per CTA over the listed (large) components;
// *depth_failed reports a graph too deep for its level index (nothing is
// then added to in.bcp).
// CTAs of the 32-source kernel whose global scratch fits in half of the free
// device memory, for pieces of at most nmax vertices
int ms_ctas_that_fit(int64_t nmax, int64_t *out);
// skip: leading sources of every large piece that were already processed
int run_ms(Ctx &ctx, const std::vector<CompDesc> &comps, const std::vector<int32_t> &large, const BcInput &in,
           bool fp32, const int64_t *sources, int64_t nsources, int64_t skip, const CompDesc *d_comps, int *d_err,
           unsigned long long *d_dag, bool *depth_failed);

// Plan and run Bc-Reach over the given components.  comps are host
// descriptors; their vertex ranges index BcInput's arrays.
int run_bcreach(Ctx &ctx, const std::vector<CompDesc> &comps, const BcInput &in, const BcPlanOpts &po);

// Bc-Reach over one large piece of small BFS depth with the whole GPU on one
// 32-source batch at a time (wide.cu).  d_order: the piece's sources (local
// ids, device), taken 32 at a time in this order.
// depth_bound: no source of the piece reaches deeper (at most
// wide_depth_limit()).
int run_wide(Ctx &ctx, const CompDesc &c, const BcInput &in, bool fp32, const int32_t *d_order, int32_t nsrc,
             int depth_bound, int *d_err, unsigned long long *d_dag);
// deepest BFS level run_wide can index
int wide_depth_limit();
// Bc-Reach over the listed mid-size pieces (every vertex a source, or with
// d_order the one piece's sources), one 64-source batch per CTA at a time
// (wide.cu).  d_comps: the device copy of comps.  Pieces found too deep for
// its level cap, or not connected, are left undone and listed in too_deep.
int run_mid(Ctx &ctx, const std::vector<CompDesc> &comps, const std::vector<int32_t> &pieces, const BcInput &in,
            bool fp32, const int32_t *d_order, const CompDesc *d_comps, int *d_err, unsigned long long *d_dag,
            std::vector<int32_t> *too_deep);
// BFS of a connected graph from `root` (rows at rp[v]..rp[v+1] of col):
// queue_out[0..*reached) the vertices in the order the search reaches them,
// *depth the deepest level (order.cu)
int bfs_queue(Ctx &ctx, const int64_t *rp, const int32_t *col, int64_t n, int32_t root, int32_t *queue_out,
              int *depth, int64_t *reached);
// BFS order of every connected component of g (rows start at 0), each from
// its smallest vertex, components contiguous; *depth the deepest level
int bfs_queue_components(Ctx &ctx, const DevGraph &g, int32_t *queue_out, int *depth);

// Bc-Reach after one more articulation split of the merged pieces
// (resplit.cu): in.bcp (the merged vertices' bc') gains the new pieces' bc'.
int run_bcreach_resplit(Ctx &ctx, DevMerged &m, const BcInput &in, const BcPlanOpts &po);

// Bc-Reach over the merged pieces with side vertices taken out (side.cu):
// the same bc' as run_bcreach(comps, in, po), with in.bcp accumulated.
// n_graph: vertices of the input graph (a bound on reach).
int run_bcreach_side(Ctx &ctx, const DevMerged &m, const std::vector<CompDesc> &comps, const BcInput &in,
                     const BcPlanOpts &po, int64_t n_graph);

}  // namespace bcs

namespace bcs {
// Plain Brandes over one component with all device state carved out of
// `scratch` (fixed_scratch_bytes(nmax, ctas) bytes); allocates nothing.
constexpr size_t FIXED_WORK_ITEM_BYTES = 8;
constexpr size_t fixed_up256(size_t x) { return (x + 255) & ~(size_t)255; }
// Layout of the region, in order: work items (nmax), the component
// descriptor, the work counter and the error word (256 bytes each), then the
// per-CTA arrays.  fixed_scratch_arrays_offset(nmax) is where the per-CTA
// arrays start; the first of them (distances, reset by the launcher) may
// serve as a one-word flag before the launch.
constexpr size_t fixed_scratch_arrays_offset(size_t nmax) { return fixed_up256(nmax * FIXED_WORK_ITEM_BYTES) + 3 * 256; }
constexpr size_t fixed_scratch_bytes(size_t nmax, size_t ctas) {
  return fixed_scratch_arrays_offset(nmax) + fixed_up256(ctas * nmax * 4) * 2 + fixed_up256(ctas * nmax * 8) * 3 +
         fixed_up256(ctas * (nmax + 2) * 4) * 2;
}
int launch_plain_fixed_scratch(Ctx &ctx, const int64_t *row, const int32_t *col, int32_t n, double *bc,
                               unsigned char *scratch, int64_t nmax, int ctas, bool fp32);
}  // namespace bcs
