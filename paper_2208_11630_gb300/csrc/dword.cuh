// dword.cuh -- double-word arithmetic on the FP32 pipe.
//
// A double-word number is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi) / 2, i.e. 48 significant bits: relative precision near
// 2^-47, against 2^-53 for FP64.  On this GPU an FP32 FMA issues at 64x the
// FP64 rate, so a few FP32 operations per FP64 one still run the update well
// ahead of the FP64 pipe.  The exponent range is FP32's (normal down to
// 1.2e-38); smaller magnitudes lose relative precision gradually.
//
// Building blocks (error-free transformations): Knuth's TwoSum, Dekker's
// Fast2Sum (|a| >= |b|), and the FMA-based TwoProd.  On top of them, the
// double-word sum, product and quotient follow Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic" (ACM TOMS 44, 2017): the sum of two double-words (the fast
// variant, whose error is bounded relative to |x| + |y|), the product with
// two FMA cross terms, and the quotient by one FP32 reciprocal with a
// double-word residual correction.  The square root and reciprocal square
// root take one Newton correction of the FP32 hardware approximation,
// evaluated in double-word arithmetic.
#pragma once

#include <cuda_runtime.h>

namespace fx {
// The type and its operations live in a namespace of their own: calls with
// double-word arguments find them by argument-dependent lookup, while
// unqualified fabs/sqrt/fma on float or double keep finding the CUDA ones.
namespace dword {

struct __align__(8) dw {
  float hi, lo;
  dw() = default;
  __host__ __device__ constexpr dw(float h, float l) : hi(h), lo(l) {}
  // nearest double-word of an FP64 value (exact split: d - hi is exact in FP64)
  __device__ __forceinline__ dw(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

namespace dwops {

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ dw two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dw(s, e);
}
// s + e = a + b exactly, for |a| >= |b| or a = 0 (Dekker)
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return dw(s, e);
}
// p + e = a * b exactly (FMA)
__device__ __forceinline__ dw two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  return dw(p, e);
}

}  // namespace dwops

__device__ __forceinline__ dw operator-(dw x) { return dw(-x.hi, -x.lo); }

__device__ __forceinline__ dw operator+(dw x, dw y) {
  const dw s = dwops::two_sum(x.hi, y.hi);
  const float v = __fadd_rn(x.lo, y.lo);
  const float w = __fadd_rn(s.lo, v);
  return dwops::fast_two_sum(s.hi, w);
}
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }
__device__ __forceinline__ dw &operator+=(dw &x, dw y) { return x = x + y; }

__device__ __forceinline__ dw operator*(dw x, dw y) {
  // the lo * lo term is below 2^-48 of the product and is left out
  const dw p = dwops::two_prod(x.hi, y.hi);
  float t = __fmul_rn(x.hi, y.lo);
  t = __fmaf_rn(x.lo, y.hi, t);
  return dwops::fast_two_sum(p.hi, __fadd_rn(p.lo, t));
}

// x / y: quotient estimate q from an FP32 reciprocal of y.hi, the residual
// x - q y (its leading product exact through TwoProd), one correction term
__device__ __forceinline__ dw operator/(dw x, dw y) {
  const float r = __fdividef(1.0f, y.hi);
  const float q = __fmul_rn(x.hi, r);
  const dw qy = dwops::two_prod(q, y.hi);
  // residual (x - q y) to FP32 accuracy: the leading terms cancel exactly
  float res = __fsub_rn(x.hi, qy.hi);
  res = __fsub_rn(res, qy.lo);
  res = __fadd_rn(res, x.lo);
  res = __fmaf_rn(-q, y.lo, res);
  return dwops::fast_two_sum(q, __fmul_rn(res, r));
}

__device__ __forceinline__ dw fma(dw a, dw b, dw c) { return a * b + c; }

__device__ __forceinline__ bool operator<(dw x, dw y) {
  return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo);
}
__device__ __forceinline__ bool operator>(dw x, dw y) { return y < x; }
__device__ __forceinline__ bool operator<=(dw x, dw y) { return !(y < x); }
__device__ __forceinline__ bool operator>=(dw x, dw y) { return !(x < y); }

__device__ __forceinline__ dw fabs(dw x) { return x.hi < 0.0f ? -x : x; }
__device__ __forceinline__ dw fmin(dw x, dw y) { return y < x ? y : x; }
__device__ __forceinline__ dw fmax(dw x, dw y) { return x < y ? y : x; }

// 1 / sqrt(x), x > 0: y0 = FP32 approximation, e = 1 - x y0^2 in double-word
// arithmetic, y = y0 (1 - e)^(-1/2) to second order: y0 + y0 e (1/2 + 3e/8)
__device__ __forceinline__ dw rsqrt(dw x) {
  const float y0 = rsqrtf(x.hi);
  const dw y2 = dwops::two_prod(y0, y0);
  const dw e = dw(1.0f, 0.0f) - x * y2;
  const float c = __fmul_rn(__fmul_rn(y0, e.hi), __fmaf_rn(0.375f, e.hi, 0.5f));
  return dwops::fast_two_sum(y0, c);
}

// sqrt(x), x >= 0: s0 = FP32 root, s = s0 + (x - s0^2) / (2 s0)
__device__ __forceinline__ dw sqrt(dw x) {
  if (!(x.hi > 0.0f)) return dw(0.0f, 0.0f);
  const float s0 = __fsqrt_rn(x.hi);
  const dw r = x - dwops::two_prod(s0, s0);
  return dwops::fast_two_sum(s0, __fdividef(r.hi, 2.0f * s0));
}

}  // namespace dword
using dword::dw;
}  // namespace fx
