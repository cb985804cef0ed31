// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers, giving about 48 significant bits on the FP32 pipes.  GB300 runs FP64 at 1/61 of
// its FP32 rate, so the FP64-class accumulations of the rangefinder (Gram matrices and the
// products Y*D whose factors are ill-conditioned) use this type in the FP32/BF16 modes.
//
// Building blocks (published error-free transformations):
//   TwoSum (Knuth): s = a + b, e = exact rounding error of the sum, no ordering condition.
//   FastTwoSum (Dekker): same when |a| >= |b|.
//   TwoProd with FMA: p = a*b, e = fma(a, b, -p) is the exact rounding error of the product.
// fma() below is the compensated dot-product step of Ogita, Rump and Oishi (Dot2): the
// running sum keeps hi through TwoSum and collects every rounding error in lo, so a dot
// product is as accurate as if computed with twice the FP32 precision.  The _rn intrinsics
// keep the compiler from contracting the error-free transformations into FMAs.
#pragma once

#include <cuda_runtime.h>

namespace qs {

using ::fma;   // keep the FP32/FP64 overloads visible next to the df64 one

struct df64 {
  float hi, lo;
  __host__ __device__ df64() : hi(0.f), lo(0.f) {}
  __host__ __device__ df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit df64(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ explicit df64(float f) : hi(f), lo(0.f) {}
  __host__ __device__ explicit df64(double d) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
  }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df64(s, e);
}

// Renormalised copy (|lo| <= ulp(hi) / 2) by TwoSum: the compensated fma() below leaves lo
// unnormalised, so hi alone may even have the wrong sign; anything that starts from an FP32
// estimate of hi (reciprocal, square root) renormalises first.
__device__ __forceinline__ df64 df_norm(df64 a) {
  const float s = __fadd_rn(a.hi, a.lo);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(a.lo, bb));
  return df64(s, e);
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return df_fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// c + a*b, compensated (Dot2 step); lo collects all rounding errors.
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(c.hi, p);
  const float bb = __fsub_rn(s, c.hi);
  const float err = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  return df64(s, __fadd_rn(c.lo, __fadd_rn(err, e)));
}

// c + a*b for an FP32 a (a double-float whose low part is zero): the a.lo * b.hi term of the
// general step is dropped, one FMA fewer, same result.
__device__ __forceinline__ df64 fma(float a, df64 b, df64 c) {
  const float p = __fmul_rn(a, b.hi);
  float e = __fmaf_rn(a, b.hi, -p);
  e = __fmaf_rn(a, b.lo, e);
  const float s = __fadd_rn(c.hi, p);
  const float bb = __fsub_rn(s, c.hi);
  const float err = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  return df64(s, __fadd_rn(c.lo, __fadd_rn(err, e)));
}

__device__ __forceinline__ df64 fma(df64 a, float b, df64 c) { return fma(b, a, c); }

// c + a*b for FP32 a and b: their product is exactly p + e (TwoProd), two FMAs fewer than the
// general step.
__device__ __forceinline__ df64 fma(float a, float b, df64 c) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(c.hi, p);
  const float bb = __fsub_rn(s, c.hi);
  const float err = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  return df64(s, __fadd_rn(c.lo, __fadd_rn(err, e)));
}

}  // namespace qs
