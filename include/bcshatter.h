/*
 * bcshatter.h - C ABI of the GB300 shattered betweenness-centrality library.
 *
 * The library computes vertex betweenness centrality (BC) of an undirected,
 * unweighted, loop-free graph, as defined by Eq. 1 of Sariyuce, Saule, Kaya
 * and Catalyurek, "Shattering and Compressing Networks for Centrality
 * Analysis" (Section 2.1):
 *
 *     bc[v] = sum over ordered pairs (s, t), s != v != t, s != t, of
 *             sigma_st(v) / sigma_st
 *
 * (ordered pairs, no normalisation; unreachable pairs add nothing; a vertex
 * alone in its connected component gets 0).
 *
 * Graph input (Section 2 and Section 4: "compressed row storage using 32-bit
 * data types"): a symmetric CSR.  row_ptr has n+1 int64 entries with
 * row_ptr[0] = 0 and row_ptr[n] = nnz; col has nnz int32 vertex ids.  Every
 * undirected edge {u,v} appears as both u->v and v->u, rows are sorted in
 * strictly ascending order (no duplicate entries) and there are no
 * self-loops.  The library checks all of this and returns BCS_EINVAL when it
 * does not hold.  n may be 0 (nothing is computed, BCS_OK).
 *
 * Memory: every pointer argument is caller-owned and is never freed or kept
 * by the library after the call returns.  When csr->on_device is 1, row_ptr,
 * col and the bc_out array of the call are device pointers on the selected
 * device; otherwise all of them are host pointers and the library copies
 * through device memory it allocates itself.  Outputs are written only when
 * the call returns BCS_OK.
 *
 * Streams: all device work of a call is issued on opts->stream (a
 * cudaStream_t, NULL = the legacy default stream).  The calls are
 * synchronous: when they return, every output has been written.
 *
 * Errors: every call returns BCS_OK (0) or a negative BCS_E* code;
 * bcs_last_error() gives a message for the calling thread's last failure.
 * Calls from several host threads are allowed; they share no mutable state
 * apart from the per-device memory pool and a few process-wide caches, each
 * behind a lock: the autotuner's choices, kernel occupancies, and a table of
 * reciprocals that the first Bc-Reach call on a device fills (one kernel
 * launch and a device-wide synchronisation).
 *
 * Environment: BCS_TRACE (any value) prints per-stage timings to stderr;
 * BCS_LARGE_PATH=wide|batched|per_source|mid forces the kernel used for
 * pieces too large for shared memory (the whole GPU on one batch of 64
 * sources, 32 sources per CTA, one source per CTA, or one 64-source batch
 * per CTA for pieces of at most 65,536 vertices), which is otherwise chosen
 * from the pieces' sizes and count, their BFS depth, the number of sources
 * and the memory each kernel needs (or by the autotuner);
 * BCS_LARGE_PATH=wide_all|mid_all (for tests) sends every piece through the
 * whole-GPU kernel, or the one-batch-per-CTA kernel, where its depth allows.
 */
#ifndef BCSHATTER_H
#define BCSHATTER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BCS_OK 0
#define BCS_EINVAL (-1)    /* malformed CSR or argument */
#define BCS_ENOMEM (-2)    /* device or host allocation failed */
#define BCS_ECUDA (-3)     /* a CUDA runtime call failed */
#define BCS_ETIMEOUT (-4)  /* a bounded device-side wait ran out */
#define BCS_EOVERFLOW (-5) /* path counts left the range the kernels can scale */
#define BCS_ENODEV (-6)    /* no usable CUDA device */

/* Shattering / compression steps (the combination letters of Section 4.2). */
#define BCS_STEP_D 1u /* degree-1 vertices, Section 3.3.1 */
#define BCS_STEP_A 2u /* articulation vertices and bridges, Sections 3.2.1-3.2.2 */
#define BCS_STEP_I 4u /* identical vertices (type I and II), Section 3.3.3 */
#define BCS_STEPS_ALL 7u
/* BFS ordering (Section 4.1), opt-in and not part of BCS_STEPS_ALL: the
 * graph is renumbered in BFS order (one search per connected component, from
 * its smallest vertex; components kept contiguous), the call runs on the
 * renumbered graph and bc is mapped back to the caller's ids.  Taken by
 * bcs_bc_plain, bcs_bc_shattered and bcs_bc_sources. */
#define BCS_STEP_O 8u
/* Side vertices (Section 3.3.2, Algorithm 3), opt-in and not part of
 * BCS_STEPS_ALL: in every merged piece, the vertices whose neighbours are
 * pairwise adjacent (degree <= 64) leave the piece; each runs one Bc-Reach
 * search on the full piece with the other vertices counted twice as targets,
 * the rest run on the piece without them, and two closed-form terms complete
 * bc'.  The result is the same bc.  Taken by bcs_bc_shattered and
 * bcs_bc_shattered_batch. */
#define BCS_STEP_S 16u
/* Identical vertices of unequal reach (the reading of Section 3.3.3 where
 * reach and ident meet), opt-in and not part of BCS_STEPS_ALL: with
 * BCS_STEP_I, classes are keyed on the neighbourhood alone; a class of K
 * members with reaches r_i becomes one vertex whose dependency starts at
 * (sum r_i) / K - 1 and whose source weight is sum r_i, and each member's own
 * terms are added to its copy in closed form.  The result is the same bc.
 * Taken by bcs_bc_shattered and bcs_bc_shattered_batch; not combinable with
 * BCS_STEP_S (BCS_EINVAL). */
#define BCS_STEP_U 32u
/* The preprocessing of Section 3.4 repeated to a fixpoint (merging can leave
 * a merged vertex as a cut vertex, Fig. 3, and splitting there can make
 * copies identical to other vertices), opt-in and not part of BCS_STEPS_ALL:
 * the merged pieces are split into biconnected blocks again, each merged
 * vertex weighing reach * ident and a cut copy of a vertex standing for k
 * members carrying 1/k of the weight beyond it per member; with BCS_STEP_I
 * the blocks' identical vertices are merged again (classes keyed on the
 * neighbourhood alone, each copy a sub-unit of k members), and split and
 * merge repeat until a round merges nothing (at most 64 rounds; every
 * round's pieces give the same bc).  The result is the same bc.  Taken by
 * bcs_bc_shattered and bcs_bc_shattered_batch; combinable with BCS_STEP_U,
 * not with BCS_STEP_S (BCS_EINVAL). */
#define BCS_STEP_L 64u

typedef struct bcs_csr {
  int64_t n;              /* number of vertices */
  int64_t nnz;            /* number of CSR entries (2 x undirected edges) */
  const int64_t *row_ptr; /* n+1 row offsets */
  const int32_t *col;     /* nnz neighbour ids */
  int32_t on_device;      /* 1: row_ptr, col and bc_out are device pointers */
} bcs_csr;

typedef struct bcs_opts {
  uint32_t steps;     /* BCS_STEP_* mask for bcs_bc_shattered / bcs_shatter */
  int32_t delta_fp32; /* 1: dependency recurrence (Eq. 3) in FP32; path counts
                         and the bc sums stay FP64 */
  int32_t autotune;   /* 1: pick by timing the candidates once per shape
                         bucket, then reuse the choice: the shared-memory
                         Bc-Reach work split (how many sources a CTA runs at
                         once), the small/large threshold (the shared memory
                         a piece may need to take the small path), and the
                         kernel of each large piece with many sources
                         (whole-GPU, 32-source batches or one source per
                         CTA, each timed on a sample of its sources) */
  int32_t device;     /* CUDA device ordinal; -1 = the current device */
  void *stream;       /* cudaStream_t for all device work; NULL = default */
  int64_t max_wait;   /* polls a device-side wait (grid barrier) makes before
                         the call gives up with BCS_ETIMEOUT; 0 = default
                         (about a second); < 0 = give up at once (tests) */
} bcs_opts;

/* Per-call statistics of the calling thread's last successful call. */
typedef struct bcs_stats {
  int64_t n_pieces;        /* components handed to Bc-Reach */
  int64_t n_slots;         /* vertex copies over all pieces before merging */
  int64_t n_merged;        /* vertices over all pieces after identical merging */
  int64_t n_entries;       /* CSR entries over all pieces after merging */
  int64_t peel_rounds;     /* degree-1 removal rounds */
  int64_t n_small_items;   /* shared-memory work items */
  int64_t n_large_sources; /* sources run on the global-memory path */
  int64_t kernel_launches; /* kernels this call launched */
  int64_t bfs_levels;      /* levels of the BFS forest of the biconnected split */
  int64_t dag_edges;       /* shortest-path DAG edges visited by Bc-Reach
                              (summed over sources), when counted */
  int64_t n_ms_batches;    /* 32-source batches on the large-piece path */
  int64_t batch_ctas;      /* CTAs of the 32-source launch */
  int64_t small_ng_cap;    /* most sources one small-path CTA ran at once */
  int64_t small_smem_budget; /* shared-memory budget per small-path CTA (bytes) */
  int64_t n_side;          /* side vertices taken out of the pieces (BCS_STEP_S) */
  int64_t n_wide_batches;  /* source batches (64, or 32) run with the whole GPU on
                              one batch (large pieces of small BFS depth), or one
                              per CTA on mid-size pieces (BCS_LARGE_PATH=mid) */
  int64_t n_rounds;        /* split-and-merge rounds of the preprocessing loop
                              (BCS_STEP_L) */
  int64_t small_limit;     /* shared memory (bytes) a piece may need for one source
                              to take the small path: fixed, or the autotuner's */
  int64_t tuned;           /* the autotuner's choices this call, as bits: 1 the
                              small/large threshold; 1 << k a large piece on
                              kernel k (1 whole-GPU, 2 32-source batches, 3 one
                              source per CTA) */
  double work_nm;          /* sum over pieces of n_c * m_c (m_c undirected) */
  double work_sources_entries; /* sum over processed sources of the piece's CSR entries */
  double work_sources_vertices; /* sum over processed sources of the piece's vertices */
  double ms_total;         /* wall time of the call, host clock */
  double ms_upload;        /* host -> device copies of the input */
  double ms_validate;      /* CSR check */
  double ms_cc;            /* connected components */
  double ms_peel;          /* degree-1 removal */
  double ms_blocks;        /* biconnected split (device kernels and the host
                              steps between them) */
  double ms_ident;         /* identical-vertex merging */
  double ms_plan;          /* work list */
  double ms_bcreach_small; /* Bc-Reach, shared-memory kernel */
  double ms_bcreach_large; /* Bc-Reach, global-memory kernel */
  double ms_mapback;       /* bc accumulation and map back */
  double ms_download;      /* device -> host copy of bc */
  double ms_side;          /* side-vertex marking and the reduced pieces */
} bcs_stats;

/*
 * Plain Brandes (Algorithm 1, Bc-Org) on the whole graph, nothing shattered:
 * bc_out[v] for all n vertices (FP64, n entries).
 */
int bcs_bc_plain(const bcs_csr *csr, const bcs_opts *opts, double *bc_out);

/*
 * Shattered and compressed BC (Section 3): the steps in opts->steps are
 * applied once in the order D, A, I (then S or L, if set, on the merged pieces);
 * Bc-Reach (Algorithm 2, with the identical-vertex terms of Section 3.3.3,
 * and Algorithm 3's searches for side vertices) runs on every piece; the piece
 * scores are mapped back with Eq. 5 (bc[v] = sum over copies v' of v of
 * bc'[v']) plus the closed-form terms of the removed vertices.  The result
 * equals Eq. 1 on the input graph (Theorem 1 and its corollaries).
 */
int bcs_bc_shattered(const bcs_csr *csr, const bcs_opts *opts, double *bc_out);

/*
 * Betweenness of many independent graphs at once (the paper's Eq. 1 applied
 * to each graph): `packed` holds count graphs in one CSR, graph g owning the
 * vertex ids [graph_vtx_off[g], graph_vtx_off[g+1]) (host array of count+1
 * ascending offsets, graph_vtx_off[0] = 0, graph_vtx_off[count] = n).  No
 * edge may join two graphs (BCS_EINVAL otherwise).  Because no shortest path
 * crosses graphs, the pieces of all graphs are shattered together and share
 * one persistent Bc-Reach launch; bc_out[v] is v's betweenness within its
 * own graph.
 */
int bcs_bc_shattered_batch(const int64_t *graph_vtx_off, int64_t count, const bcs_csr *packed,
                           const bcs_opts *opts, double *bc_out);

/*
 * Partial Brandes sum over a list of k sources (Eq. 2):
 * bc_out[v] = sum_{i<k} delta_{src[i]}(v), with delta_s(s) taken as 0.
 * src is a host array of k ids in [0, n) (repeats allowed).
 */
int bcs_bc_sources(const bcs_csr *csr, const int64_t *src, int64_t k, const bcs_opts *opts,
                   double *bc_out);

/*
 * Single-source Brandes for tests (Algorithm 1, one source s): host arrays
 * of n entries each: d (BFS distance, -1 unreachable), sigma as
 * sigma_mant * 2^sigma_exp2 (sigma_mant 0 when unreachable) and delta_s(v)
 * (Eq. 3; delta_s(s) as computed by the recursion).  Any output may be NULL.
 */
int bcs_debug_sssp(const bcs_csr *csr, int64_t s, const bcs_opts *opts, int32_t *d,
                   double *sigma_mant, int32_t *sigma_exp2, double *delta);

/* Largest graph bcs_bc_plain_noalloc accepts (vertices). */
#define BCS_NOALLOC_MAX_N 16384

/*
 * Plain Brandes, as bcs_bc_plain, without allocating any device memory.
 * The paper has no counterpart: this variant exists for callers that cannot
 * let a library allocate on the GPU, such as a serving process that gives
 * nearly all device memory to its own pool at start-up, or a latency-critical
 * loop that must never enter the CUDA allocator.
 *
 * Arguments: csr->on_device must be 1 (row_ptr, col and bc_out are device
 * pointers on the selected device); csr->n <= BCS_NOALLOC_MAX_N, otherwise
 * BCS_EINVAL with a message.  bc_out receives n FP64 values.
 *
 * Memory: the kernels' state lives in one static device array of about
 * 42 MB (64 CTAs x 16,384 vertices), which every GPU that loads this library
 * holds until the process exits.  The first call on a device looks up that
 * array's address (cudaGetSymbolAddress) and may load the library's device
 * code; make that first call before any stream capture.  The address is kept
 * for the life of the process, so resetting the device (cudaDeviceReset)
 * between calls is not supported.  Every call shares
 * the array and resets the parts that must start cleared, so calls that
 * overlap on the GPU (two streams, two threads) race and must not be issued.
 */
int bcs_bc_plain_noalloc(const bcs_csr *csr, const bcs_opts *opts, double *bc_out);

/* The pieces bcs_shatter returns (library-owned, host memory). */
typedef struct bcs_components bcs_components;

typedef struct bcs_components_view {
  int64_t n;         /* vertices of the input graph */
  int64_t n_pieces;  /* pieces (components of the shattered graph) */
  int64_t n_merged;  /* vertices over all pieces after identical merging */
  int64_t n_entries; /* local CSR entries over all pieces */
  int64_t n_members; /* (piece, original vertex) slots before merging */
  const int64_t *piece_vtx_off;   /* n_pieces+1: piece p owns merged vertices
                                     [piece_vtx_off[p], piece_vtx_off[p+1]) */
  const int64_t *piece_N;         /* n_pieces: size of the connected
                                     component of the input the piece came from */
  const int64_t *row_ptr;         /* n_merged+1: global offsets into col */
  const int32_t *col;             /* n_entries: neighbour ids local to the piece */
  const int32_t *org;             /* n_merged: original id of the kept vertex */
  const int32_t *reach;           /* n_merged: reach (Section 3.2) */
  const int32_t *ident;           /* n_merged: ident (Section 3.3.3) */
  const int64_t *member_off;      /* n_merged+1 into member */
  const int32_t *member;          /* n_members: original ids each merged vertex
                                     stands for (itself included), ascending */
  const int64_t *bc_pre;          /* n: exact integer terms of the vertices
                                     removed by degree-1 compression */
  const double *bc_corr;          /* n_merged: identical-vertex terms of
                                     Section 3.3.3 added to every member */
} bcs_components_view;

/* Run the steps of opts->steps and return the pieces (D, A, I applied once,
 * in that order).  *out must be freed with bcs_components_free. */
int bcs_shatter(const bcs_csr *csr, const bcs_opts *opts, bcs_components **out);

/* Fill *view with pointers into c (valid until bcs_components_free). */
int bcs_components_get(const bcs_components *c, bcs_components_view *view);

void bcs_components_free(bcs_components *c);

/* Statistics of the calling thread's last successful BC call. */
int bcs_last_stats(bcs_stats *out);

/* Message for the calling thread's last error ("" if none). */
const char *bcs_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int bcs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BCSHATTER_H */
