// Integer-pipe helpers for 64-bit fixed-point values: FP64 -> fixed point,
// fixed point -> FP64, and Q62 products.  FP64 arithmetic issues at a small
// fraction of the integer rate on this part, so the emulation kernels move
// values between FP64 and fixed point by bit manipulation of the IEEE-754
// encoding.
#pragma once

#include <cstdint>

namespace flapw {
namespace fx {

__device__ __forceinline__ uint64_t absbits(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// round(x 2^shift0) as a signed integer (half away from zero); zero and
// subnormal x give 0.  The caller keeps |x| 2^shift0 below 2^62.
__device__ __forceinline__ long long fixed_point(double x, int shift0) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;
  const uint64_t mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = ex - 1075 + shift0;
  long long X;
  if (sh >= 0) {
    X = (long long)(mant << sh);
  } else {
    const int r = -sh;
    X = (r > 62) ? 0 : (long long)((mant + (1ull << (r - 1))) >> r);
  }
  return (b >> 63) ? -X : X;
}

// x 2^ex rounded to the nearest double (ties to even), built from the bits.
// Results below the normal range flush to a signed zero and above it become
// a signed infinity (the emulation's scaled values stay far from both).
__device__ __forceinline__ double to_double(long long x, int ex) {
  if (x == 0) return 0.0;
  const uint64_t sgn = x < 0 ? (1ull << 63) : 0ull;
  uint64_t m = x < 0 ? 0ull - (uint64_t)x : (uint64_t)x;
  const int lz = __clzll((long long)m);
  m <<= lz;  // leading one at bit 63
  uint64_t mant = m >> 11;
  const uint64_t rem = m & 0x7FFull;
  int e2 = 63 - lz + ex;  // |value| in [2^e2, 2^(e2 + 1))
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++e2;
    }
  }
  const int be = e2 + 1023;
  if (be <= 0) return __longlong_as_double((long long)sgn);
  if (be >= 2047) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sgn | ((uint64_t)be << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// floor(a b / 2^62) for a Q62 factor b (|b| <= 2^62) and |a b| < 2^125.
__device__ __forceinline__ long long mul_q62(long long a, long long b) {
  const long long hi = __mul64hi(a, b);
  const uint64_t lo = (uint64_t)a * (uint64_t)b;
  return (long long)(((uint64_t)hi << 2) | (lo >> 62));
}

// An integer |d| < 2^22 as an exact float, by the 1.5 x 2^23 magic number.
__device__ __forceinline__ float small_int_to_float(int d) {
  return __fsub_rn(__int_as_float(0x4B400000 + d), 12582912.0f);
}

}  // namespace fx
}  // namespace flapw
