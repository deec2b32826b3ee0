// sort.cu - stable LSD radix sort of (uint32 key, int32 value) pairs.
//
// 8-bit digits.  A tile of 1024 pairs is handled by one CTA of 8 warps; each
// warp owns 128 consecutive pairs, taken as 4 chunks of 32.  Inside a chunk,
// __match_any_sync groups the lanes holding the same digit, so a pair's rank
// among equal digits before it is a popcount: tiles, warps, chunks and lanes
// are all visited in input order, which makes every pass stable.
#include "common.h"

namespace bcs {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_CHUNKS = 4;
constexpr int RS_TILE = RS_THREADS * RS_CHUNKS;  // 1024
constexpr int RS_DIGITS = 256;

// per-warp digit histogram of this tile, in shared memory
__device__ void rs_warp_hist(const uint32_t *__restrict__ keys, int64_t n, int shift, int (*h)[RS_DIGITS]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = lane; d < RS_DIGITS; d += 32) h[w][d] = 0;
  __syncwarp();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (32 * RS_CHUNKS);
  for (int c = 0; c < RS_CHUNKS; c++) {
    const int64_t i = base + c * 32 + lane;
    const int digit = i < n ? (int)((keys[i] >> shift) & 255u) : RS_DIGITS;
    const unsigned m = __match_any_sync(0xffffffffu, digit);
    if (digit < RS_DIGITS && lane == __ffs(m) - 1) h[w][digit] += __popc(m);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_count(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                         int64_t ntiles, int64_t *cnt) {
  __shared__ int h[RS_WARPS][RS_DIGITS];
  rs_warp_hist(keys, n, shift, h);
  __syncthreads();
  for (int d = threadIdx.x; d < RS_DIGITS; d += RS_THREADS) {
    int s = 0;
    for (int w = 0; w < RS_WARPS; w++) s += h[w][d];
    cnt[(int64_t)d * ntiles + blockIdx.x] = s;  // digit-major: the scan gives global positions
  }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t *__restrict__ kin,
                                                           const int32_t *__restrict__ vin, uint32_t *kout,
                                                           int32_t *vout, int64_t n, int shift, int64_t ntiles,
                                                           const int64_t *__restrict__ off) {
  __shared__ int h[RS_WARPS][RS_DIGITS];
  __shared__ int64_t run[RS_WARPS][RS_DIGITS];
  rs_warp_hist(kin, n, shift, h);
  __syncthreads();
  for (int d = threadIdx.x; d < RS_DIGITS; d += RS_THREADS) {
    int64_t p = off[(int64_t)d * ntiles + blockIdx.x];
    for (int w = 0; w < RS_WARPS; w++) {
      run[w][d] = p;
      p += h[w][d];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (32 * RS_CHUNKS);
  for (int c = 0; c < RS_CHUNKS; c++) {
    const int64_t i = base + c * 32 + lane;
    const bool ok = i < n;
    const uint32_t k = ok ? kin[i] : 0u;
    const int digit = ok ? (int)((k >> shift) & 255u) : RS_DIGITS;
    const unsigned m = __match_any_sync(0xffffffffu, digit);
    if (ok) {
      const int64_t pos = run[w][digit] + __popc(m & ((1u << lane) - 1u));
      kout[pos] = k;
      vout[pos] = vin[i];
    }
    __syncwarp();
    if (ok && lane == __ffs(m) - 1) run[w][digit] += __popc(m);
    __syncwarp();
  }
}

// Sort n pairs by key (ascending, stable).  Keys must be < 2^key_bits.
// Results end up in (keys, vals); (tk, tv) are scratch of the same size.
int radix_sort_pairs(Ctx &ctx, uint32_t *keys, int32_t *vals, uint32_t *tk, int32_t *tv, int64_t n, int key_bits) {
  if (n <= 1) return BCS_OK;
  const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  if (ntiles > INT32_MAX) {
    set_error("radix sort input too large");
    return BCS_EINVAL;
  }
  DBuf<int64_t> cnt, off, tot;
  BCS_TRY(cnt.alloc((size_t)RS_DIGITS * ntiles, ctx.stream));
  BCS_TRY(off.alloc((size_t)RS_DIGITS * ntiles, ctx.stream));
  BCS_TRY(tot.alloc(1, ctx.stream));
  uint32_t *ka = keys, *kb = tk;
  int32_t *va = vals, *vb = tv;
  int passes = 0;
  for (int shift = 0; shift < key_bits; shift += 8) {
    k_rs_count<<<(unsigned)ntiles, RS_THREADS, 0, ctx.stream>>>(ka, n, shift, ntiles, cnt.p);
    ctx.launches++;
    BCS_CUDA(cudaGetLastError());
    BCS_TRY(launch_exclusive_scan(ctx, cnt.p, off.p, RS_DIGITS * ntiles, tot.p));
    k_rs_scatter<<<(unsigned)ntiles, RS_THREADS, 0, ctx.stream>>>(ka, va, kb, vb, n, shift, ntiles, off.p);
    ctx.launches++;
    BCS_CUDA(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
    passes++;
  }
  if (passes & 1) {
    BCS_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx.stream));
    BCS_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx.stream));
  }
  return BCS_OK;
}

}  // namespace bcs
