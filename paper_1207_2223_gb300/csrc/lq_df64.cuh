// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  Built
// from the error-free transformations of Knuth (TwoSum: the rounding error of
// a + b is itself a float, recovered with six additions) and Dekker (TwoProd:
// with a fused multiply-add the rounding error of a * b is fma(a, b, -a*b)),
// renormalised with Dekker's FastTwoSum.  It runs on the FP32 pipe, which on
// this part is ~60x faster than the FP64 pipe; the solver uses it for the
// intermediate true residuals of mixed-precision CG, where ~1e-14 relative
// accuracy is far below the residuals being corrected (the final residual is
// still certified in FP64).
//
// Every operation uses the _rn intrinsics so the compiler cannot contract or
// reorder the compensated sums.
#pragma once
#include <cuda_runtime.h>

namespace lq {

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // (host and device: kernel arguments such as kappa are converted on the host)
  __host__ __device__ __forceinline__ explicit df64(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ __forceinline__ explicit df64(float v) : hi(v), lo(0.f) {}
  // split of a double into the nearest float and the float nearest the remainder
  __host__ __device__ __forceinline__ explicit df64(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df64 r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);                // TwoProd error term
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df64 r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
// The kernels call fma() unqualified inside this namespace, which hides the
// global overloads: forward the built-in types to them.
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }

// a * b + c with one renormalisation
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, f;
  two_sum(p, c.hi, s, f);
  f = __fadd_rn(f, __fadd_rn(e, c.lo));
  df64 r;
  fast_two_sum(s, f, r.hi, r.lo);
  return r;
}

}  // namespace lq
