// Grid-wide waits for cooperative launches (all CTAs co-resident).
#pragma once
#include <cstdint>

#include "bc_math.cuh"

namespace bcs {

// ------------------------------------------------ grid barrier (bounded)
// Sense-reversing barrier over all CTAs of a cooperative launch (which
// guarantees they are co-resident).  Each wait polls at most `limit` times;
// a CTA that runs out, or that sees another CTA's error, sets ERR_TIMEOUT
// and the kernel returns, so no wait is unbounded.
struct GridBarrier {
  unsigned int *count;
  unsigned int *gen;
  int *err;
  long long limit;
};

static __device__ bool grid_wait(const GridBarrier &b) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = *(volatile unsigned int *)b.gen;
    __threadfence();
    if (atomicAdd(b.count, 1u) == gridDim.x - 1) {
      *(volatile unsigned int *)b.count = 0u;
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      long long polls = 0;
      unsigned ns = 32;  // back off between polls so the arriving CTAs' atomics are not crowded out
      while (*(volatile unsigned int *)b.gen == g) {
        if (polls++ >= b.limit || *(volatile int *)b.err) {
          ok = 0;
          break;
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
      }
    }
    __threadfence();
    if (!ok) atomicOr(b.err, ERR_TIMEOUT);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// grid-stride loop over [lo, hi) for a cooperative kernel
#define COOP_STRIDE(i, lo, hi) \
  for (int64_t i = (lo) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (hi); i += (int64_t)gridDim.x * blockDim.x)

}  // namespace bcs
