// noalloc.cu - plain Brandes without any device allocation.
//
// Some callers cannot let a library allocate device memory: a serving
// process that hands nearly all of the GPU's memory to its own pool at
// start-up, or a latency-critical loop that must never enter the CUDA
// allocator.  bcs_bc_plain_noalloc serves them: the global-memory state the
// Bc-Reach kernel needs lives in one file-scope static device array of fixed
// size, which every GPU that loads this library holds until the process
// exits.  The caller still provides the graph and the output on the device.
#include <mutex>

#include "common.h"

namespace bcs {

constexpr int64_t NOALLOC_MAX_N = BCS_NOALLOC_MAX_N;  // vertices
constexpr int NOALLOC_CTAS = 64;                      // CTAs sharing the scratch
constexpr size_t NOALLOC_BYTES = fixed_scratch_bytes(NOALLOC_MAX_N, NOALLOC_CTAS);

// The scratch.  In host code this name is only a host-side stand-in for the
// array; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {
std::mutex g_mu;
constexpr int MAX_DEVICES = 64;
unsigned char *g_addr[MAX_DEVICES] = {};
}  // namespace

// Device address of the scratch on the current device (looked up once per
// device, with that device current, and kept for the life of the process: a
// device reset, which would move the array, is not supported).
static int noalloc_scratch(int device, unsigned char **out) {
  if (device < 0 || device >= MAX_DEVICES) {
    set_error("device ordinal out of range for the static scratch table");
    return BCS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      set_error(std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
      return BCS_ECUDA;
    }
    g_addr[device] = (unsigned char *)ptr;
  }
  *out = g_addr[device];
  return BCS_OK;
}

}  // namespace bcs

using namespace bcs;

extern "C" __attribute__((visibility("default"))) int bcs_bc_plain_noalloc(const bcs_csr *csr,
                                                                           const bcs_opts *opts,
                                                                           double *bc_out) {
  if (!csr) {
    set_error("csr is NULL");
    return BCS_EINVAL;
  }
  if (csr->n < 0 || csr->nnz < 0) {
    set_error("negative n or nnz");
    return BCS_EINVAL;
  }
  if (csr->n == 0) return BCS_OK;
  if (!csr->on_device) {
    set_error("bcs_bc_plain_noalloc needs the graph and bc_out in device memory (csr->on_device = 1)");
    return BCS_EINVAL;
  }
  if (csr->n > NOALLOC_MAX_N) {
    set_error("bcs_bc_plain_noalloc handles at most " + std::to_string(NOALLOC_MAX_N) + " vertices, got " +
              std::to_string(csr->n));
    return BCS_EINVAL;
  }
  if (!csr->row_ptr || (csr->nnz > 0 && !csr->col) || !bc_out) {
    set_error("NULL pointer argument");
    return BCS_EINVAL;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    prev = -1;
  }
  Ctx ctx;
  int rc = make_ctx(opts, &ctx);
  if (rc == BCS_OK) {
    unsigned char *scratch = nullptr;
    rc = noalloc_scratch(ctx.device, &scratch);
    if (rc == BCS_OK) {
      // The CSR check needs one int of device memory: it borrows the first
      // word of the per-CTA distance arrays, which the launcher
      // re-initialises right after.
      int *flags = (int *)(scratch + fixed_scratch_arrays_offset(NOALLOC_MAX_N));
      DevGraph g;
      g.n = csr->n;
      g.nnz = csr->nnz;
      g.rp = csr->row_ptr;
      g.col = csr->col;
      rc = launch_validate(ctx, g, flags);
      int f = 0;
      if (rc == BCS_OK) {
        if (cudaMemcpyAsync(&f, flags, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx.stream) != cudaSuccess) {
          set_error("reading the CSR check flags failed");
          rc = BCS_ECUDA;
        } else if (f) {
          set_error("malformed CSR (offsets/ids out of range, self-loop, unsorted/duplicate or asymmetric)");
          rc = BCS_EINVAL;
        }
      }
      if (rc == BCS_OK)
        rc = launch_plain_fixed_scratch(ctx, csr->row_ptr, csr->col, (int32_t)csr->n, bc_out, scratch,
                                        NOALLOC_MAX_N, NOALLOC_CTAS, opts && opts->delta_fp32);
    }
  }
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}
