// df64.cuh -- double-float arithmetic: a real as the unevaluated sum hi + lo
// of two floats (|lo| <= ulp(hi)/2), ~48 significant bits, computed on the
// FP32 pipe.
//
// GB300 executes FP32 at ~58x its FP64 rate, so a product or sum carried as
// two floats with error-free transformations (Dekker's product via FMA,
// Knuth's two-sum) is far faster than the FP64 instruction it replaces while
// keeping ~1e-14 relative accuracy.  Used by the DF64 form (links stored as
// hi/lo float pairs) for the link algebra, the noise (ln, sqrt, sincospi
// below), the exponentials and the determinant re-projection; only the
// reductions' final sums are FP64.
//
// Error-free building blocks (exact for finite inputs without overflow):
//   two_sum(a, b):      s + e = a + b exactly, s = fl(a + b)        (Knuth)
//   fast_two_sum(a, b): the same when |a| >= |b|                     (Dekker)
//   a * b = p + e with p = fl(a b), e = fma(a, b, -p)               (FMA split)
// A rounded product p that is later added to something is formed with
// __fmul_rn, which the compiler never contracts into an FMA: a contracted
// p + c would no longer be the fl(p + c) the error terms assume.
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
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// a * b + c with one renormalisation
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
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

// A double constant split into hi + lo at compile time.
__host__ __device__ constexpr df64 df_const(double d) {
  return df64((float)d, (float)(d - (double)(float)d));
}

// x 2^k (exact while hi and lo stay normal).
__device__ __forceinline__ df64 df_ldexp(df64 x, int k) { return df64(ldexpf(x.hi, k), ldexpf(x.lo, k)); }

// a / b by long division with float quotient digits (Dekker 1971): q1 from
// the float quotient, q2 and q3 from the remainders a - b q1 and
// a - b (q1 + q2), each remainder formed in double-float.
__device__ __forceinline__ df64 df_div(df64 a, df64 b) {
  const float inv = 1.0f / b.hi;
  const float q1 = a.hi * inv;
  df64 r = a - b * df64(q1, 0.0f);
  const float q2 = r.hi * inv;
  r = r - b * df64(q2, 0.0f);
  const float q3 = r.hi * inv;
  const df64 q = df_fast_two_sum(q1, q2);
  return q + df64(q3, 0.0f);
}

// sqrt(v), v > 0: the float root s corrected by (v - s^2) / (2 s) with s^2
// split exactly (Dekker 1971's sqrt2).
__device__ __forceinline__ df64 df_sqrt(df64 v) {
  const float s = sqrtf(v.hi);
  const float p = __fmul_rn(s, s);
  const float e = fmaf(s, s, -p);
  const float d = ((v.hi - p) - e) + v.lo;
  return df_fast_two_sum(s, d * (0.5f / s));
}

// ln of M 2^e given num = M - 1 and den = M + 1 (M in [1/sqrt2, sqrt2)):
// ln M = 2 atanh(z) = 2 z sum_k z^(2k) / (2k + 1), z = num / den, |z| <=
// 0.1716.  Terms k = 0..4 in double-float, k = 5..9 (below 2^-25 of the
// sum, so float suffices for them) in float; k = 10 and up are below 2^-50.
__device__ __forceinline__ df64 df_log_core(df64 num, df64 den, int e) {
  const df64 z = df_div(num, den);
  const df64 w = z * z;
  float t = 1.0f / 19.0f;
  t = fmaf(t, w.hi, 1.0f / 17.0f);
  t = fmaf(t, w.hi, 1.0f / 15.0f);
  t = fmaf(t, w.hi, 1.0f / 13.0f);
  t = fmaf(t, w.hi, 1.0f / 11.0f);
  df64 P = df64(t, 0.0f);
  P = fma(P, w, df_const(1.0 / 9.0));
  P = fma(P, w, df_const(1.0 / 7.0));
  P = fma(P, w, df_const(1.0 / 5.0));
  P = fma(P, w, df_const(1.0 / 3.0));
  P = fma(P, w, df64(1.0f, 0.0f));
  const df64 lnM = df_ldexp(z * P, 1);
  return fma(df64((float)e, 0.0f), df_const(0.69314718055994530942), lnM);
}

// ln x for a normal x > 0: x = M 2^e with M in [1/sqrt2, sqrt2).
__device__ __forceinline__ df64 df_log(df64 x) {
  int e;
  const float m = frexpf(x.hi, &e);  // x.hi = m 2^e, m in [1/2, 1)
  if (m < 0.70710678f) e -= 1;
  const df64 M = df_ldexp(x, -e);
  const df64 num = df_two_sum(M.hi - 1.0f, M.lo);  // M.hi - 1 is exact (Sterbenz)
  return df_log_core(num, M + df64(1.0f, 0.0f), e);
}

// ln u for u in (0, 1) given also v = 1 - u exactly: for u > 3/4 the series
// takes M - 1 = -v, so ln u keeps its relative accuracy however close u is
// to 1 (there u itself, rounded to ~48 bits, would not).
__device__ __forceinline__ df64 df_log_unit(df64 u, df64 v) {
  if (v.hi < 0.25f) return df_log_core(-v, df64(2.0f, 0.0f) - v, 0);
  return df_log(u);
}

// sin(pi t) and cos(pi t) for 0 <= t <= 2: t = q/2 + r with q = rint(2t),
// |r| <= 1/4, x = pi r (|x| <= pi/4), and the Taylor series in y = x^2 of
// sin x / x = 1 - y S(y) and cos x = C(y).  The terms below 2^-25 of the sum
// (y^4 and up in S, y^6 and up in C) run in float, the rest in double-float;
// the first terms left out (y^7/17!, y^9/18!) are below 2^-50.
__device__ __forceinline__ void df_sincospi(df64 t, df64* sn, df64* cs) {
  const float q = rintf(2.0f * t.hi);
  const df64 r = df_two_sum(t.hi - 0.5f * q, t.lo);  // t.hi - q/2 is exact (Sterbenz)
  const df64 x = r * df_const(3.14159265358979323846);
  const df64 y = x * x;
  float a = 1.0f / 1307674368000.0f;              // 1/15!
  a = fmaf(a, y.hi, -1.0f / 6227020800.0f);       // -1/13!
  a = fmaf(a, y.hi, 1.0f / 39916800.0f);          // 1/11!
  float b = 1.0f / 20922789888000.0f;             // 1/16!
  b = fmaf(b, y.hi, -1.0f / 87178291200.0f);      // -1/14!
  b = fmaf(b, y.hi, 1.0f / 479001600.0f);         // 1/12!
  df64 S = df64(a, 0.0f), C = df64(b, 0.0f);
  S = fma(S, y, df_const(-1.0 / 362880.0));
  C = fma(C, y, df_const(-1.0 / 3628800.0));
  S = fma(S, y, df_const(1.0 / 5040.0));
  C = fma(C, y, df_const(1.0 / 40320.0));
  S = fma(S, y, df_const(-1.0 / 120.0));
  C = fma(C, y, df_const(-1.0 / 720.0));
  S = fma(S, y, df_const(1.0 / 6.0));
  C = fma(C, y, df_const(1.0 / 24.0));
  C = fma(C, y, df64(-0.5f, 0.0f));
  S = fma(S, -y, df64(1.0f, 0.0f));  // sin x / x
  C = fma(C, y, df64(1.0f, 0.0f));   // cos x
  S = S * x;
  // pi t = q pi/2 + x: rotate by the quadrant
  const int qi = ((int)q) & 3;
  const df64 s0 = (qi & 1) ? C : S, c0 = (qi & 1) ? S : C;
  *sn = (qi & 2) ? -s0 : s0;
  *cs = ((qi + 1) & 2) ? -c0 : c0;
}

// Storage of a complex df64 number: (re.hi, re.lo, im.hi, im.lo).
__device__ __forceinline__ float4 df_pack(df64 re, df64 im) { return make_float4(re.hi, re.lo, im.hi, im.lo); }

}  // namespace clgc
