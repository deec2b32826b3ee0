// uf.cuh - lock-free union-find used by the component and block kernels.
// Hooking always puts the larger root under the smaller one, so parent
// pointers only decrease and a root is the smallest id of its set; path
// halving writes only ever touch non-root entries.
#pragma once
#include <stdint.h>

namespace bcs {

__device__ __forceinline__ int32_t uf_vload(const int32_t *p) { return *(volatile const int32_t *)p; }

__device__ __forceinline__ int32_t uf_find(int32_t *p, int32_t x) {
  for (;;) {
    int32_t px = uf_vload(p + x);
    if (px == x) return x;
    int32_t gpx = uf_vload(p + px);
    if (gpx == px) return px;
    *(volatile int32_t *)(p + x) = gpx;
    x = gpx;
  }
}

__device__ __forceinline__ void uf_unite(int32_t *p, int32_t a, int32_t b) {
  for (;;) {
    a = uf_find(p, a);
    b = uf_find(p, b);
    if (a == b) return;
    if (a < b) {
      int32_t t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(p + a, a, b) == a) return;
  }
}

}  // namespace bcs
