// Double-float arithmetic: a value as an unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi) / 2, about 48 significant bits), on the FP32
// pipes.  The error-free transformations are Knuth's TwoSum, Dekker's
// Fast2Sum and the FMA-based TwoProduct; every operation is written with an
// _rn intrinsic, since contracting any of them into an FMA would break the
// transformations.  Relative error of one operation: a few 2^-48.
#pragma once

namespace flapw {
namespace dfl {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df make(float2 v) { return df{v.x, v.y}; }

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly, given |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df add(df x, df y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df mul(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);  // exact: x.hi y.hi = p + e
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  df r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// x y + z
__device__ __forceinline__ df fma(df x, df y, df z) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  float s, e2;
  two_sum(p, z.hi, s, e2);
  e2 = __fadd_rn(e2, __fadd_rn(e, z.lo));
  df r;
  fast_two_sum(s, e2, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df neg(df x) { return df{-x.hi, -x.lo}; }

__device__ __forceinline__ double to_double(df x) { return (double)x.hi + (double)x.lo; }

// x ~ hi + lo with hi = fl(x), lo = fl(x - hi): within 2^-48 |x| for |x| in
// the FP32 normal range.
__device__ __forceinline__ float2 split(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}

}  // namespace dfl
}  // namespace flapw
