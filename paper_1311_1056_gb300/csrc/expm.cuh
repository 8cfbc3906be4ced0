// expm.cuh -- matrix exponentials of traceless 3x3 matrices and the det = 1
// re-projection: FP64 (the FP64 and FP32-storage forms) and double-float
// (the *_df variants of the DF64 form, same steps).
//
// Method (Cayley-Hamilton reduction): a traceless 3x3 A satisfies
//   A^3 = c1 A + c0 1,  c1 = Tr(A^2)/2,  c0 = det A = Tr(A^3)/3,
// so every power series in A collapses to a 1 + b A + c A^2.  The truncated
// Taylor series of exp is evaluated by Horner's rule directly on the three
// coefficients: multiplying a 1 + b A + c A^2 by A gives
//   (c c0) 1 + (a + c c1) A + b A^2,
// i.e. 8 FP64 operations per term instead of a 3x3 product.  The number of
// terms follows from the Frobenius norm r (remainder r^(N+1)/(N+1)! < 2^-54);
// for r > 1 the argument is scaled by 2^-s and the coefficients are squared
// s times in the same three-term representation.
//
// The Hermitian variant (cooling transformation Omega = exp(H), H = -eps
// alpha f_a lambda_a, Sec. 2, eq. "eq:24") has real c0, c1 and real
// coefficients, and produces exp(-H) = Omega^{-1} from the same H^2.
#pragma once
#include "su3.cuh"

namespace clgc {

__constant__ double c_invfact[28] = {
    1.0, 1.0, 0.5, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320,
    1.0 / 362880, 1.0 / 3628800, 1.0 / 39916800, 1.0 / 479001600, 1.0 / 6227020800.0,
    1.0 / 87178291200.0, 1.0 / 1307674368000.0, 1.0 / 20922789888000.0,
    1.0 / 355687428096000.0, 1.0 / 6402373705728000.0, 1.0 / 121645100408832000.0,
    1.0 / 2432902008176640000.0, 1.0 / 51090942171709440000.0,
    1.0 / 1124000727777607680000.0, 1.0 / 25852016738884976640000.0,
    1.0 / 620448401733239439360000.0, 1.0 / 15511210043330985984000000.0,
    1.0 / 403291461126605635584000000.0, 1.0 / 10888869450418352160768000000.0};

// The same table split into double-float constants.
__constant__ df64 c_invfact_df[28] = {
    df_const(1.0), df_const(1.0), df_const(0.5), df_const(1.0 / 6), df_const(1.0 / 24),
    df_const(1.0 / 120), df_const(1.0 / 720), df_const(1.0 / 5040), df_const(1.0 / 40320),
    df_const(1.0 / 362880), df_const(1.0 / 3628800), df_const(1.0 / 39916800),
    df_const(1.0 / 479001600), df_const(1.0 / 6227020800.0), df_const(1.0 / 87178291200.0),
    df_const(1.0 / 1307674368000.0), df_const(1.0 / 20922789888000.0),
    df_const(1.0 / 355687428096000.0), df_const(1.0 / 6402373705728000.0),
    df_const(1.0 / 121645100408832000.0), df_const(1.0 / 2432902008176640000.0),
    df_const(1.0 / 51090942171709440000.0), df_const(1.0 / 1124000727777607680000.0),
    df_const(1.0 / 25852016738884976640000.0), df_const(1.0 / 620448401733239439360000.0),
    df_const(1.0 / 15511210043330985984000000.0), df_const(1.0 / 403291461126605635584000000.0),
    df_const(1.0 / 10888869450418352160768000000.0)};

// Truncation tolerance of the Taylor series (last term r^N / N! below it).
// FP64 results: 1.4e-17, under the FP64 rounding of the result (2^-53 =
// 1.1e-16).  The FP32-storage form rounds the exponential to FP32 (2^-24 =
// 6e-8) as soon as it is formed, so its series, still evaluated in FP64,
// stops at 1e-11: a truncation error 6,000 times below that rounding, and
// about a third fewer terms for the CL update's argument.
const float TAYLOR_TOL_FP64 = 1.4e-17f;
const float TAYLOR_TOL_FP32_STORAGE = 1.0e-11f;
template <typename T>
__host__ __device__ constexpr float taylor_tol() {
  return sizeof(T) == 4 ? TAYLOR_TOL_FP32_STORAGE : TAYLOR_TOL_FP64;
}

// Number of Taylor terms for ||B||_F <= r <= 1 (float arithmetic: an estimate
// on the cheap pipe; the bound has a factor > 2 of slack at the cut).
__device__ __forceinline__ int taylor_terms(float r, float tol = TAYLOR_TOL_FP64) {
  float t = 1.0f;
  int n = 0;
  do {
    ++n;
    t *= r / (float)n;
  } while (t >= tol && n < 26);
  return n;
}

// Squarings for a norm r > 1: ceil(log2 r), at most 100.  A runaway field
// can give r = +inf (or a norm beyond float range); the cap keeps the
// squaring loop bounded, and the result then overflows to inf/NaN, which the
// observables report as non-finite links.
__device__ __forceinline__ int scaling_steps(float r) {
  return (int)ceilf(log2f(fminf(r, 1.0e30f)));
}

// exp(A) for traceless complex A.  The matrix work (A^2, the final
// a + b A + c A^2) is done in the link type T (FP64 or FP32); the scalar
// Cayley-Hamilton recurrences run in FP64.
// r_hint >= 0 is the Frobenius norm of A when the caller has it (e.g. from an
// FP32 copy); < 0 computes it.  tol: the series' truncation tolerance.
template <typename T>
__device__ __forceinline__ void expm_traceless(mat<T>& E, const mat<T>& A, float r_hint = -1.f,
                                               float tol = TAYLOR_TOL_FP64) {
  mat<T> A2;
  mul(A2, A, A);
  const cx<T> t1 = trace(A2), t0 = trace_mul(A2, A);
  cx<double> c1 = {(double)t1.re, (double)t1.im};
  c1.re *= 0.5;
  c1.im *= 0.5;
  cx<double> c0 = {(double)t0.re, (double)t0.im};
  c0.re *= (1.0 / 3.0);
  c0.im *= (1.0 / 3.0);
  float r = r_hint >= 0.f ? r_hint : sqrtf((float)norm2(A));
  int s = 0;
  double sc = 1.0;  // scaling 2^-s
  cx<double> b0 = c0, b1 = c1;  // det and Tr(B^2)/2 of B = A 2^-s
  if (r > 1.0f) {
    s = scaling_steps(r);
    sc = ldexp(1.0, -s);
    r = (float)(r * sc);
    const double sc2 = sc * sc;
    b0 = cx<double>{c0.re * sc2 * sc, c0.im * sc2 * sc};
    b1 = cx<double>{c1.re * sc2, c1.im * sc2};
  }
  int N = taylor_terms(r, tol);
  cx<double> a = {c_invfact[N], 0.0}, b = {0.0, 0.0}, c = {0.0, 0.0};
  for (int k = N - 1; k >= 0; --k) {
    cx<double> na = cfma(c, b0, cx<double>{c_invfact[k], 0.0});
    cx<double> nb = cfma(c, b1, a);
    c = b;
    b = nb;
    a = na;
  }
  for (int i = 0; i < s; ++i) {  // (a + bB + cB^2)^2 with B^3 = b1 B + b0
    cx<double> bc = cmul(b, c);
    cx<double> cc = cmul(c, c);
    cx<double> na = cmul(a, a);
    na = cfma(cx<double>{2.0 * bc.re, 2.0 * bc.im}, b0, na);
    cx<double> nb = cmul(cx<double>{2.0 * a.re, 2.0 * a.im}, b);
    nb = cfma(cx<double>{2.0 * bc.re, 2.0 * bc.im}, b1, nb);
    nb = cfma(cc, b0, nb);
    cx<double> nc = cmul(b, b);
    nc = cfma(cx<double>{2.0 * a.re, 2.0 * a.im}, c, nc);
    nc = cfma(cc, b1, nc);
    a = na;
    b = nb;
    c = nc;
  }
  if (s > 0) {  // back to powers of A: b B = (b sc) A, c B^2 = (c sc^2) A^2
    b.re *= sc;
    b.im *= sc;
    c.re *= sc * sc;
    c.im *= sc * sc;
  }
  const cx<T> aT = {(T)a.re, (T)a.im}, bT = {(T)b.re, (T)b.im}, cT = {(T)c.re, (T)c.im};
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    cx<T> v = cmul(bT, A.e[k]);
    v = cfma(cT, A2.e[k], v);
    if (k % 4 == 0) v = cadd(v, aT);
    E.e[k] = v;
  }
}

// The same exponential entirely in double-float (the DF64 form): the scalar
// recurrences too, with the coefficients of c_invfact_df.  A2 is the
// caller's workspace for A^2; E may be A itself (E is formed entry by entry
// from the same entries of A and A^2).
__device__ __forceinline__ void expm_traceless_df(mat<df64>& E, const mat<df64>& A, mat<df64>& A2) {
  mul_df_compact(A2, A, A);
  const cx<df64> t1 = trace(A2), t0 = trace_mul(A2, A);
  const df64 third = df_const(1.0 / 3.0);
  const cx<df64> c1 = {df_ldexp(t1.re, -1), df_ldexp(t1.im, -1)};
  const cx<df64> c0 = {t0.re * third, t0.im * third};
  float r = sqrtf((float)norm2(A));
  int s = 0;
  cx<df64> b0 = c0, b1 = c1;  // det and Tr(B^2)/2 of B = A 2^-s
  if (r > 1.0f) {
    s = scaling_steps(r);
    r = ldexpf(r, -s);
    b0 = cx<df64>{df_ldexp(c0.re, -3 * s), df_ldexp(c0.im, -3 * s)};
    b1 = cx<df64>{df_ldexp(c1.re, -2 * s), df_ldexp(c1.im, -2 * s)};
  }
  const int N = taylor_terms(r);
  const df64 zero(0.0f, 0.0f);
  cx<df64> a = {c_invfact_df[N], zero}, b = {zero, zero}, c = {zero, zero};
  for (int k = N - 1; k >= 0; --k) {
    const cx<df64> na = cfma(c, b0, cx<df64>{c_invfact_df[k], zero});
    const cx<df64> nb = cfma(c, b1, a);
    c = b;
    b = nb;
    a = na;
  }
  for (int i = 0; i < s; ++i) {  // (a + bB + cB^2)^2 with B^3 = b1 B + b0
    const cx<df64> bc = cmul(b, c), cc = cmul(c, c);
    const cx<df64> bc2 = {df_ldexp(bc.re, 1), df_ldexp(bc.im, 1)};
    const cx<df64> a2 = {df_ldexp(a.re, 1), df_ldexp(a.im, 1)};
    cx<df64> na = cmul(a, a);
    na = cfma(bc2, b0, na);
    cx<df64> nb = cmul(a2, b);
    nb = cfma(bc2, b1, nb);
    nb = cfma(cc, b0, nb);
    cx<df64> nc = cmul(b, b);
    nc = cfma(a2, c, nc);
    nc = cfma(cc, b1, nc);
    a = na;
    b = nb;
    c = nc;
  }
  if (s > 0) {  // back to powers of A
    b = cx<df64>{df_ldexp(b.re, -s), df_ldexp(b.im, -s)};
    c = cx<df64>{df_ldexp(c.re, -2 * s), df_ldexp(c.im, -2 * s)};
  }
#pragma unroll 1
  for (int k = 0; k < 9; ++k) {  // rolled: the matrices are in memory (the DF64 workspace)
    cx<df64> v = cmul(b, A.e[k]);
    v = cfma(c, A2.e[k], v);
    if (k % 4 == 0) v = cadd(v, a);
    E.e[k] = v;
  }
}

// Packed Hermitian 3x3: d0, d1, d2 real diagonal, o01, o02, o12 upper entries.
struct herm {
  double d0, d1, d2;
  cx<double> o01, o02, o12;
};

__device__ __forceinline__ void herm_square(herm& q, const herm& h) {
  double n01 = fma(h.o01.re, h.o01.re, h.o01.im * h.o01.im);
  double n02 = fma(h.o02.re, h.o02.re, h.o02.im * h.o02.im);
  double n12 = fma(h.o12.re, h.o12.re, h.o12.im * h.o12.im);
  q.d0 = fma(h.d0, h.d0, n01 + n02);
  q.d1 = fma(h.d1, h.d1, n01 + n12);
  q.d2 = fma(h.d2, h.d2, n02 + n12);
  // (H^2)_01 = (d0 + d1) o01 + o02 conj(o12)
  double s01 = h.d0 + h.d1, s02 = h.d0 + h.d2, s12 = h.d1 + h.d2;
  q.o01.re = fma(s01, h.o01.re, fma(h.o02.re, h.o12.re, h.o02.im * h.o12.im));
  q.o01.im = fma(s01, h.o01.im, fma(h.o02.im, h.o12.re, -h.o02.re * h.o12.im));
  // (H^2)_02 = (d0 + d2) o02 + o01 o12
  q.o02.re = fma(s02, h.o02.re, fma(h.o01.re, h.o12.re, -h.o01.im * h.o12.im));
  q.o02.im = fma(s02, h.o02.im, fma(h.o01.re, h.o12.im, h.o01.im * h.o12.re));
  // (H^2)_12 = (d1 + d2) o12 + conj(o01) o02
  q.o12.re = fma(s12, h.o12.re, fma(h.o01.re, h.o02.re, h.o01.im * h.o02.im));
  q.o12.im = fma(s12, h.o12.im, fma(h.o01.re, h.o02.im, -h.o01.im * h.o02.re));
}

// Omega = exp(H) and Omega^{-1} = exp(-H) for traceless Hermitian H.
__device__ __forceinline__ void expm_hermitian_pair(herm& om, herm& omi, const herm& h,
                                                    float tol = TAYLOR_TOL_FP64) {
  herm h2;
  herm_square(h2, h);
  double c1 = 0.5 * (h2.d0 + h2.d1 + h2.d2);  // Tr H^2 / 2 = ||H||_F^2 / 2
  // det H = d0 d1 d2 + 2 Re(o01 o12 conj(o02)) - d0|o12|^2 - d1|o02|^2 - d2|o01|^2
  double t_re = fma(h.o01.re, h.o12.re, -h.o01.im * h.o12.im);
  double t_im = fma(h.o01.re, h.o12.im, h.o01.im * h.o12.re);
  double c0 = h.d0 * h.d1 * h.d2;
  c0 = fma(2.0, fma(t_re, h.o02.re, t_im * h.o02.im), c0);
  c0 = fma(-h.d0, fma(h.o12.re, h.o12.re, h.o12.im * h.o12.im), c0);
  c0 = fma(-h.d1, fma(h.o02.re, h.o02.re, h.o02.im * h.o02.im), c0);
  c0 = fma(-h.d2, fma(h.o01.re, h.o01.re, h.o01.im * h.o01.im), c0);
  float r = sqrtf((float)(2.0 * c1));
  int s = 0;
  double sc = 1.0;
  double b1 = c1, b0 = c0;
  if (r > 1.0f) {
    s = scaling_steps(r);
    sc = ldexp(1.0, -s);
    r = (float)(r * sc);
    b1 = c1 * sc * sc;
    b0 = c0 * sc * sc * sc;
  }
  int N = taylor_terms(r, tol);
  // exp(B) = a + bB + cB^2 and exp(-B) = ap - bp B + cp B^2 (det(-B) = -det B)
  double a = c_invfact[N], b = 0.0, c = 0.0;
  double ap = a, bp = 0.0, cp = 0.0;
  for (int k = N - 1; k >= 0; --k) {
    double na = fma(c, b0, c_invfact[k]);
    double nb = fma(c, b1, a);
    c = b;
    b = nb;
    a = na;
    double nap = fma(-cp, b0, c_invfact[k]);
    double nbp = fma(cp, b1, ap);
    cp = bp;
    bp = nbp;
    ap = nap;
  }
  for (int i = 0; i < s; ++i) {
    double na = fma(2.0 * b * c, b0, a * a);
    double nb = fma(c * c, b0, fma(2.0 * b * c, b1, 2.0 * a * b));
    double nc = fma(c * c, b1, fma(2.0 * a, c, b * b));
    a = na; b = nb; c = nc;
    na = fma(-2.0 * bp * cp, b0, ap * ap);
    nb = fma(-cp * cp, b0, fma(2.0 * bp * cp, b1, 2.0 * ap * bp));
    nc = fma(cp * cp, b1, fma(2.0 * ap, cp, bp * bp));
    ap = na; bp = nb; cp = nc;
  }
  if (s > 0) {
    b *= sc;
    c *= sc * sc;
    bp *= sc;
    cp *= sc * sc;
  }
  bp = -bp;  // exp(-H) = ap - bp H + cp H^2
  om.d0 = fma(c, h2.d0, fma(b, h.d0, a));
  om.d1 = fma(c, h2.d1, fma(b, h.d1, a));
  om.d2 = fma(c, h2.d2, fma(b, h.d2, a));
  om.o01 = cx<double>{fma(c, h2.o01.re, b * h.o01.re), fma(c, h2.o01.im, b * h.o01.im)};
  om.o02 = cx<double>{fma(c, h2.o02.re, b * h.o02.re), fma(c, h2.o02.im, b * h.o02.im)};
  om.o12 = cx<double>{fma(c, h2.o12.re, b * h.o12.re), fma(c, h2.o12.im, b * h.o12.im)};
  omi.d0 = fma(cp, h2.d0, fma(bp, h.d0, ap));
  omi.d1 = fma(cp, h2.d1, fma(bp, h.d1, ap));
  omi.d2 = fma(cp, h2.d2, fma(bp, h.d2, ap));
  omi.o01 = cx<double>{fma(cp, h2.o01.re, bp * h.o01.re), fma(cp, h2.o01.im, bp * h.o01.im)};
  omi.o02 = cx<double>{fma(cp, h2.o02.re, bp * h.o02.re), fma(cp, h2.o02.im, bp * h.o02.im)};
  omi.o12 = cx<double>{fma(cp, h2.o12.re, bp * h.o12.re), fma(cp, h2.o12.im, bp * h.o12.im)};
}

// det(U)^(-1/3) on the principal branch.  Near det = 1 (|det - 1| < 1e-4, the
// normal case after an update that preserves det up to rounding) the binomial
// series (1 + d)^(-1/3) = 1 - d/3 + 2d^2/9 - 14d^3/81 + 35d^4/243 - ... is
// exact to 1e-17; below |d| = 3e-6 (rounding drift of FP64 or FP32 links) its
// first three terms already are (the next is 14/81 |d|^3 < 5e-18);
// otherwise |det|^(-1/3) exp(-i arg(det)/3).
__device__ __forceinline__ cx<double> det_inv_cuberoot(cx<double> d) {
  cx<double> e = {d.re - 1.0, d.im};
  const double e2 = fma(e.re, e.re, e.im * e.im);
  if (e2 < 1e-11) {
    cx<double> p = {2.0 / 9.0, 0.0};
    p = cfma(p, e, cx<double>{-1.0 / 3.0, 0.0});
    p = cfma(p, e, cx<double>{1.0, 0.0});
    return p;
  }
  if (e2 < 1e-8) {
    cx<double> p = {35.0 / 243.0, 0.0};
    p = cfma(p, e, cx<double>{-14.0 / 81.0, 0.0});
    p = cfma(p, e, cx<double>{2.0 / 9.0, 0.0});
    p = cfma(p, e, cx<double>{-1.0 / 3.0, 0.0});
    p = cfma(p, e, cx<double>{1.0, 0.0});
    return p;
  }
  double mag = exp(-log(hypot(d.re, d.im)) / 3.0);
  double ang = -atan2(d.im, d.re) / 3.0;
  double sn, cs;
  sincos(ang, &sn, &cs);
  return cx<double>{mag * cs, mag * sn};
}

// Double-float Hermitian 3x3 and its exponential pair (the DF64 form's
// cooling transformation), the same steps as above in double-float.
struct herm_df {
  df64 d0, d1, d2;
  cx<df64> o01, o02, o12;
};

__device__ __forceinline__ df64 df_abs2(cx<df64> z) { return fma(z.re, z.re, z.im * z.im); }

__device__ __forceinline__ void herm_square_df(herm_df& q, const herm_df& h) {
  const df64 n01 = df_abs2(h.o01), n02 = df_abs2(h.o02), n12 = df_abs2(h.o12);
  q.d0 = fma(h.d0, h.d0, n01 + n02);
  q.d1 = fma(h.d1, h.d1, n01 + n12);
  q.d2 = fma(h.d2, h.d2, n02 + n12);
  const df64 s01 = h.d0 + h.d1, s02 = h.d0 + h.d2, s12 = h.d1 + h.d2;
  // (H^2)_01 = (d0 + d1) o01 + o02 conj(o12)
  q.o01.re = fma(s01, h.o01.re, fma(h.o02.re, h.o12.re, h.o02.im * h.o12.im));
  q.o01.im = fma(s01, h.o01.im, fma(h.o02.im, h.o12.re, -(h.o02.re * h.o12.im)));
  // (H^2)_02 = (d0 + d2) o02 + o01 o12
  q.o02.re = fma(s02, h.o02.re, fma(h.o01.re, h.o12.re, -(h.o01.im * h.o12.im)));
  q.o02.im = fma(s02, h.o02.im, fma(h.o01.re, h.o12.im, h.o01.im * h.o12.re));
  // (H^2)_12 = (d1 + d2) o12 + conj(o01) o02
  q.o12.re = fma(s12, h.o12.re, fma(h.o01.re, h.o02.re, h.o01.im * h.o02.im));
  q.o12.im = fma(s12, h.o12.im, fma(h.o01.re, h.o02.im, -(h.o01.im * h.o02.re)));
}

// c 1 + b H + c2 H^2 for real coefficients
__device__ __forceinline__ void herm_combine_df(herm_df& o, df64 a, df64 b, df64 c, const herm_df& h,
                                                const herm_df& h2) {
  o.d0 = fma(c, h2.d0, fma(b, h.d0, a));
  o.d1 = fma(c, h2.d1, fma(b, h.d1, a));
  o.d2 = fma(c, h2.d2, fma(b, h.d2, a));
  o.o01 = cx<df64>{fma(c, h2.o01.re, b * h.o01.re), fma(c, h2.o01.im, b * h.o01.im)};
  o.o02 = cx<df64>{fma(c, h2.o02.re, b * h.o02.re), fma(c, h2.o02.im, b * h.o02.im)};
  o.o12 = cx<df64>{fma(c, h2.o12.re, b * h.o12.re), fma(c, h2.o12.im, b * h.o12.im)};
}

// Omega = exp(H) and Omega^{-1} = exp(-H) for traceless Hermitian H.
__device__ __forceinline__ void expm_hermitian_pair_df(herm_df& om, herm_df& omi, const herm_df& h) {
  herm_df h2;
  herm_square_df(h2, h);
  const df64 c1 = df_ldexp(h2.d0 + h2.d1 + h2.d2, -1);
  // det H = d0 d1 d2 + 2 Re(o01 o12 conj(o02)) - d0|o12|^2 - d1|o02|^2 - d2|o01|^2
  const df64 t_re = fma(h.o01.re, h.o12.re, -(h.o01.im * h.o12.im));
  const df64 t_im = fma(h.o01.re, h.o12.im, h.o01.im * h.o12.re);
  df64 c0 = h.d0 * h.d1 * h.d2;
  c0 = c0 + df_ldexp(fma(t_re, h.o02.re, t_im * h.o02.im), 1);
  c0 = fma(-h.d0, df_abs2(h.o12), c0);
  c0 = fma(-h.d1, df_abs2(h.o02), c0);
  c0 = fma(-h.d2, df_abs2(h.o01), c0);
  float r = sqrtf(2.0f * c1.hi);
  int s = 0;
  df64 b1 = c1, b0 = c0;
  if (r > 1.0f) {
    s = scaling_steps(r);
    r = ldexpf(r, -s);
    b1 = df_ldexp(c1, -2 * s);
    b0 = df_ldexp(c0, -3 * s);
  }
  const int N = taylor_terms(r);
  // exp(B) = a + bB + cB^2 and exp(-B) = ap - bp B + cp B^2 (det(-B) = -det B)
  const df64 zero(0.0f, 0.0f);
  df64 a = c_invfact_df[N], b = zero, c = zero;
  df64 ap = a, bp = zero, cp = zero;
  for (int k = N - 1; k >= 0; --k) {
    const df64 na = fma(c, b0, c_invfact_df[k]);
    const df64 nb = fma(c, b1, a);
    c = b;
    b = nb;
    a = na;
    const df64 nap = fma(-cp, b0, c_invfact_df[k]);
    const df64 nbp = fma(cp, b1, ap);
    cp = bp;
    bp = nbp;
    ap = nap;
  }
  for (int i = 0; i < s; ++i) {
    df64 bc2 = df_ldexp(b * c, 1), cc = c * c, a2 = df_ldexp(a, 1);
    df64 na = fma(bc2, b0, a * a);
    df64 nb = fma(cc, b0, fma(bc2, b1, a2 * b));
    df64 nc = fma(cc, b1, fma(a2, c, b * b));
    a = na; b = nb; c = nc;
    bc2 = df_ldexp(bp * cp, 1), cc = cp * cp, a2 = df_ldexp(ap, 1);
    na = fma(-bc2, b0, ap * ap);
    nb = fma(-cc, b0, fma(bc2, b1, a2 * bp));
    nc = fma(cc, b1, fma(a2, cp, bp * bp));
    ap = na; bp = nb; cp = nc;
  }
  if (s > 0) {
    b = df_ldexp(b, -s);
    c = df_ldexp(c, -2 * s);
    bp = df_ldexp(bp, -s);
    cp = df_ldexp(cp, -2 * s);
  }
  herm_combine_df(om, a, b, c, h, h2);
  herm_combine_df(omi, ap, -bp, cp, h, h2);  // exp(-H) = ap - bp H + cp H^2
}

// det(U)^(-1/3) in double-float: the binomial series near det = 1 (the
// normal case), else the FP64 branch above.
__device__ __forceinline__ cx<df64> det_inv_cuberoot_df(cx<df64> d) {
  const cx<df64> e = {d.re - df64(1.0f, 0.0f), d.im};
  if (e.re.hi * e.re.hi + e.im.hi * e.im.hi < 1e-8f) {
    const df64 zero(0.0f, 0.0f);
    cx<df64> p = {df_const(35.0 / 243.0), zero};
    p = cfma(p, e, cx<df64>{df_const(-14.0 / 81.0), zero});
    p = cfma(p, e, cx<df64>{df_const(2.0 / 9.0), zero});
    p = cfma(p, e, cx<df64>{df_const(-1.0 / 3.0), zero});
    p = cfma(p, e, cx<df64>{df64(1.0f, 0.0f), zero});
    return p;
  }
  const cx<double> z = det_inv_cuberoot(cx<double>{(double)d.re, (double)d.im});
  return cx<df64>{df64(z.re), df64(z.im)};
}

}  // namespace clgc
