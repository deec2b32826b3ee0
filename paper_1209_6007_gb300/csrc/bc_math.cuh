// bc_math.cuh - device arithmetic shared by the Bc-Reach kernels.
#pragma once
#include <stdint.h>

namespace bcs {

struct Coef32 {
  float c;
  int32_t e;
};

// error flags written by the kernels
constexpr int ERR_OVERFLOW = 1;  // path counts left the range one BFS level can scale
constexpr int ERR_DEPTH = 2;     // a multi-source batch needed more BFS levels than it can index
constexpr int ERR_TIMEOUT = 4;   // a bounded device-side wait ran out

// Binary exponent of a positive double and its [1,2) mantissa as FP32,
// straight from the bit pattern (no FP64 instruction).  Only the rare
// subnormal input takes the library route.
__device__ __forceinline__ void split_pow2(double x, int &e, float &m) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex != 0) {
    e = ex - 1023;
    m = __int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff));
  } else {
    e = ilogb(x);
    m = (float)scalbn(x, -e);
  }
}

// (double)x for 0 < x < 2^63, rounded to nearest even, built from integer
// instructions only (the hardware conversion issues on GB300's FP64 pipe).
__device__ __forceinline__ double i64_to_f64_pos(long long x) {
  const unsigned long long u = (unsigned long long)x;
  const int e = 63 - __clzll(x);  // floor(log2 x)
  unsigned long long m;           // 53-bit significand with the leading one
  if (e <= 52) {
    m = u << (52 - e);
  } else {
    const int sh = e - 52;
    m = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    m += (rem > half || (rem == half && (m & 1ull))) ? 1ull : 0ull;  // a carry to 2^53 bumps the exponent
  }
  return __longlong_as_double((long long)(((unsigned long long)(e + 1023) << 52) + (m - (1ull << 52))));
}

// A double holding a non-negative integer below 2^53, as an integer, from
// the bit pattern (integer instructions only).
__device__ __forceinline__ long long f64_to_i64_exact(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < 0) return 0;  // 0.0
  const unsigned long long m = (unsigned long long)(b & 0x000fffffffffffffLL) | (1ull << 52);
  return (long long)(e >= 52 ? m << (e - 52) : m >> (52 - e));
}

// ceil(log2 x) for x >= 1 from the bit pattern (integer instructions only)
__device__ __forceinline__ int ceil_log2_pos(double x) {
  const long long b = __double_as_longlong(x);
  return (int)((b >> 52) & 0x7ff) - 1023 + ((b & 0x000fffffffffffffLL) != 0);
}

// 2^k as a double for k <= 1023, built from the bits (0 below the normal range)
__device__ __forceinline__ double pow2_int(int k) {
  return k < -1022 ? 0.0 : __longlong_as_double((long long)(k + 1023) << 52);
}

// Integer part of a 64-bit path count: binary exponent and [1,2) mantissa
// as FP32 (integer instructions only); x >= 1.
__device__ __forceinline__ void split_pow2_i64(long long x, int &e, float &m) {
  e = 63 - __clzll(x);
  const unsigned long long u = (unsigned long long)x;
  const unsigned long long mant = e >= 23 ? (u >> (e - 23)) : (u << (23 - e));
  m = __int_as_float(0x3f800000 | (int)(mant & 0x7fffffull));
}

// 1/x for a positive double.  The mantissa m in [1,2) gets an FP32 hardware
// reciprocal approximation r (relative error e = 1 - m r of about 2^-22),
// refined by one third-order step of the series 1/m = r (1 + e + e^2 + ...):
// r <- r + r (e + e^2), leaving an error near e^3 ~ 2^-66, below FP64
// rounding, in three FMAs.  The exponent is put back by integer arithmetic
// on the bit pattern.
// Inputs here are path counts scaled into [2^-900, 2^960], far from the
// subnormal and overflow ends; anything else takes the IEEE division.
__device__ __forceinline__ double recip_pos(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex < 64 || ex > 2000) return 1.0 / x;
  const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff))));
  const int fb = __float_as_int(rf);  // rf in (0.5, 1]: widen to FP64 through the bits
  double r = __longlong_as_double(((long long)(((fb >> 23) & 0xff) - 127 + 1023) << 52) |
                                  ((long long)(fb & 0x7fffff) << 29));
  const double e = fma(-m, r, 1.0);
  r = fma(r, fma(e, e, e), r);
  return __longlong_as_double(__double_as_longlong(r) - ((long long)(ex - 1023) << 52));
}

// Per-source 2-bit fields packed in one 64-bit word (32 sources, source i in
// bits 2i and 2i+1).
// bit i of x -> bit 2i
__device__ __forceinline__ uint64_t spread2(uint32_t x) {
  uint64_t v = x;
  v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
  v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
  v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
  v = (v | (v << 2)) & 0x3333333333333333ull;
  v = (v | (v << 1)) & 0x5555555555555555ull;
  return v;
}

// bit 2i of v -> bit i
__device__ __forceinline__ uint32_t compact2(uint64_t v) {
  v &= 0x5555555555555555ull;
  v = (v | (v >> 1)) & 0x3333333333333333ull;
  v = (v | (v >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  v = (v | (v >> 4)) & 0x00FF00FF00FF00FFull;
  v = (v | (v >> 8)) & 0x0000FFFF0000FFFFull;
  v = (v | (v >> 16)) & 0x00000000FFFFFFFFull;
  return (uint32_t)v;
}

}  // namespace bcs
