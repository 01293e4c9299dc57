// Split-precision slicing of the FP64 operand for the emulated contraction.
//
// Every operand row (one plane wave G of one problem) gets a power-of-two
// scale 2^e with max_k max(|Re Z_kG|, |Im Z_kG|) < 2^e.  Each entry x is then
// rounded to the fixed-point integer X = round(x 2^{7s - e}) (|X| <= 2^{7s})
// and written as s balanced base-128 digits
//     X = sum_{i=0}^{s-1} d_i 128^{s-1-i},  |d_0| <= 128,  |d_i| <= 64 (i > 0),
// each carried exactly by an fp16 value.  A product of two leading digits is
// at most 2^14, of a leading and a later digit 2^13, of two later digits
// 2^12, so 1024, 2048 and 4096 of them respectively sum exactly in FP32.  Everything here is integer bit
// manipulation of the IEEE-754 encoding: FP64 arithmetic is scarce on this
// part.  The rounding of X is the only approximation (|x - X 2^{e-7s}| <=
// 2^{e-7s-1}).
//
// Output layout: SL[slice][plane][row][k], k contiguous, fp16; plane 0 = Re,
// 1 = Im.  Columns outside the problem's valid K ranges are written as 0.
// Without a problem table every row's valid range is [0, k_valid).
#include <cstdint>

#include "fixed64.cuh"
#include "flapw_internal.h"

namespace flapw {
namespace {

using fx::absbits;
using fx::fixed_point;

// Writes the NS balanced base-128 digits of the fixed-point values X0, X1 (two
// adjacent columns) as fp16 pairs d2[i] = (digit i of X0, digit i of X1).  The
// digits are small integers: each goes to FP32 exactly by the magic-number
// addition and the pair to fp16 by one packed conversion, so no FP64 or
// 64-bit-integer conversion instruction is involved.
template <int NS>
__device__ __forceinline__ void digits2(long long X0, long long X1, __half2 (&d2)[NS]) {
#pragma unroll
  for (int i = NS - 1; i >= 1; --i) {
    const long long a = ((X0 + 64) & 127) - 64, b = ((X1 + 64) & 127) - 64;
    d2[i] = __floats2half2_rn(fx::small_int_to_float((int)a), fx::small_int_to_float((int)b));
    X0 = (X0 - a) >> kSliceBits;
    X1 = (X1 - b) >> kSliceBits;
  }
  d2[0] = __floats2half2_rn(fx::small_int_to_float((int)X0), fx::small_int_to_float((int)X1));
}

// 4 CTAs per SM (64 registers): the kernel is bound by integer issue, and the
// extra resident warps hide its memory latency better than the registers
// they cost (config 2: 0.35 -> 0.28 ms for both halves).
template <int NS>
__global__ void __launch_bounds__(256, 4) slicer_kernel(const double2* __restrict__ Z, int64_t k_alloc,
                                                     const Prob* __restrict__ probs,
                                                     const int* __restrict__ row_prob, int64_t k_valid,
                                                     int64_t rows, int64_t row0,
                                                     __half* __restrict__ SL, int* __restrict__ rexp) {
  __shared__ unsigned long long red[8];
  const int64_t row = row0 + blockIdx.x;
  int64_t kp = k_valid, kn = 0;
  if (probs) {
    const Prob P = probs[row_prob[row]];
    kp = P.kp;
    kn = P.kn;
  }
  const int64_t kp_pad = neg_base((int)kp);
  const double2* zr = Z + row * k_alloc;
  auto valid = [&](int64_t c) { return c < kp || (c >= kp_pad && c < kp_pad + kn); };
  unsigned long long m = 0;
  for (int64_t c = threadIdx.x; c < k_alloc; c += blockDim.x) {
    if (valid(c)) {
      const double2 z = zr[c];
      const unsigned long long a = absbits(z.x), b = absbits(z.y);
      m = a > m ? a : m;
      m = b > m ? b : m;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_down_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_down_sync(0xffffffffu, m, o);
      m = v > m ? v : m;
    }
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  const unsigned long long M = red[0];
  const int e = (M == 0) ? 0 : (int)((M >> 52) & 0x7FF) - 1022;  // M < 2^e
  if (threadIdx.x == 0) rexp[row] = e;
  const int shift0 = kSliceBits * NS - e;
  const int64_t plane_stride = rows * k_alloc;
  for (int64_t c0 = (int64_t)threadIdx.x * 8; c0 < k_alloc; c0 += (int64_t)blockDim.x * 8) {
    double2 z[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) z[q] = valid(c0 + q) ? zr[c0 + q] : make_double2(0.0, 0.0);
#pragma unroll
    for (int plane = 0; plane < 2; ++plane) {
      __align__(16) __half2 d[NS][4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        __half2 d2[NS];
        digits2<NS>(fixed_point(plane ? z[q].y : z[q].x, shift0),
                    fixed_point(plane ? z[q + 1].y : z[q + 1].x, shift0), d2);
#pragma unroll
        for (int i = 0; i < NS; ++i) d[i][q / 2] = d2[i];
      }
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        __half* dst = SL + ((int64_t)(2 * i + plane)) * plane_stride + row * k_alloc + c0;
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(d[i]);
      }
    }
  }
}

// One warp per row of at most 512 columns (all valid); 8 rows per CTA.
template <int NS>
__global__ void __launch_bounds__(256) slicer_rows_kernel(const double2* __restrict__ Z,
                                                          int64_t k_alloc, int64_t rows,
                                                          __half* __restrict__ SL,
                                                          int* __restrict__ rexp) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= rows) return;
  const double2* zr = Z + row * k_alloc;
  unsigned long long m = 0;
  for (int64_t c = lane; c < k_alloc; c += 32) {
    const double2 z = zr[c];
    const unsigned long long a = absbits(z.x), b = absbits(z.y);
    m = a > m ? a : m;
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  const int e = (m == 0) ? 0 : (int)((m >> 52) & 0x7FF) - 1022;  // max < 2^e
  if (lane == 0) rexp[row] = e;
  const int shift0 = kSliceBits * NS - e;
  const int64_t plane_stride = rows * k_alloc;
  for (int64_t c0 = (int64_t)lane * 8; c0 < k_alloc; c0 += 256) {
    double2 z[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) z[q] = zr[c0 + q];
#pragma unroll
    for (int plane = 0; plane < 2; ++plane) {
      __align__(16) __half2 d[NS][4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        __half2 d2[NS];
        digits2<NS>(fixed_point(plane ? z[q].y : z[q].x, shift0),
                    fixed_point(plane ? z[q + 1].y : z[q + 1].x, shift0), d2);
#pragma unroll
        for (int i = 0; i < NS; ++i) d[i][q / 2] = d2[i];
      }
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        __half* dst = SL + ((int64_t)(2 * i + plane)) * plane_stride + row * k_alloc + c0;
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(d[i]);
      }
    }
  }
}

}  // namespace

cudaError_t launch_slicer(const double2* Z, int64_t k_alloc, const Prob* probs,
                          const int* row_prob, int64_t k_valid, int64_t rows, int64_t row0,
                          int64_t nrows, int n_slices, __half* SL, int* rexp, cudaStream_t st) {
  if (nrows == 0) return cudaSuccess;
  const unsigned grid = (unsigned)nrows;
  switch (n_slices) {
#define FLAPW_SLICER_CASE(NS)                                                                    \
  case NS:                                                                                       \
    slicer_kernel<NS><<<grid, 256, 0, st>>>(Z, k_alloc, probs, row_prob, k_valid, rows, row0, SL, \
                                            rexp);                                                \
    break;
    FLAPW_SLICER_CASE(4)
    FLAPW_SLICER_CASE(5)
    FLAPW_SLICER_CASE(6)
    FLAPW_SLICER_CASE(7)
    FLAPW_SLICER_CASE(8)
#undef FLAPW_SLICER_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace flapw

namespace flapw {

cudaError_t launch_slicer_rows(const double2* Z, int64_t k_alloc, int64_t rows, int n_slices,
                               __half* SL, int* rexp, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  if (k_alloc % 8 != 0 || k_alloc > 512) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)((rows + 7) / 8);
  if (n_slices == kOpSlices)
    slicer_rows_kernel<kOpSlices><<<grid, 256, 0, st>>>(Z, k_alloc, rows, SL, rexp);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace flapw
