// df64.cuh -- double-float arithmetic: a real as the unevaluated sum hi + lo
// of two floats (|lo| <= ulp(hi)/2), ~48 significant bits, computed on the
// FP32 pipe.
//
// GB300 executes FP32 at ~58x its FP64 rate, so a product or sum carried as
// two floats with error-free transformations (Dekker's product via FMA,
// Knuth's two-sum) is far faster than the FP64 instruction it replaces while
// keeping ~1e-14 relative accuracy.  Used for the link algebra of the DF64
// form (links stored as hi/lo float pairs); the exponentials, the noise, the
// determinant re-projection and every reduction stay in FP64.
//
// Error-free building blocks (exact for finite inputs without overflow):
//   two_sum(a, b):      s + e = a + b exactly, s = fl(a + b)        (Knuth)
//   fast_two_sum(a, b): the same when |a| >= |b|                     (Dekker)
//   a * b = p + e with p = fl(a b), e = fma(a, b, -p)               (FMA split)
#pragma once
#include <cuda_runtime.h>

namespace clgc {

// Keep the library overloads (float, double) visible next to the df64 ones.
using ::fma;
using ::isfinite;

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // explicit: a double never turns into a df64 (or back) without a visible cast
  __device__ __forceinline__ explicit df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __device__ __forceinline__ explicit df64(int i) : hi((float)i), lo(0.0f) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df64(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return df64(s, b - (s - a));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// a * b + c with one renormalisation
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const df64 s = df_two_sum(p, c.hi);
  return df_fast_two_sum(s.hi, s.lo + (e + c.lo));
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

__device__ __forceinline__ bool isfinite(df64 x) { return ::isfinite(x.hi) && ::isfinite(x.lo); }

// Storage of a complex df64 number: (re.hi, re.lo, im.hi, im.lo).
__device__ __forceinline__ float4 df_pack(df64 re, df64 im) { return make_float4(re.hi, re.lo, im.hi, im.lo); }

}  // namespace clgc
