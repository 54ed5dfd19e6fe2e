// Double-float arithmetic for the FP32-storage form: a value is the unevaluated
// pair of floats hi + lo (|lo| <= ulp(hi) / 2), built from the error-free
// transformations of Knuth (TwoSum) and Dekker (the exact product error, here
// through fmaf), with the single-rounding-pair ("sloppy") addition of Dekker's
// double-length arithmetic (Numer. Math. 18, 1971): about 44 bits per
// operation, 2^20 times finer than FP32 storage, on the FP32 pipe, which GB300
// runs about 60 times faster than FP64.  The exponent range is float's.
#pragma once

#include <cuda_runtime.h>

namespace bcgs {

struct df {
  float hi, lo;
};
__device__ __forceinline__ double df_dbl(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_from(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {  // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }  // a b + c
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }


}  // namespace bcgs
