// su3.cuh -- 3x3 complex matrix algebra for the CL / gauge-cooling kernels.
//
// Templated on the real type T (double for the FP64 form, float for the
// FP32-storage form, df64 for the double-float form).  Every product is written as explicit fused
// multiply-adds so the FP64 instruction count of a kernel can be read off the
// code: a complex multiply-accumulate is 4 FMA, a 3x3 matrix product 108.
//
// Matrices are row-major, element k = 3*row + col.  Inverses of SL(3,C)
// matrices are taken as adjugates (det = 1 is kept by the re-projection after
// every CL update, Sec. 2: det U = 1 on SL(N,C)).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cvt.cuh"
#include "df64.cuh"

namespace clgc {

template <typename T>
struct cx {
  T re, im;
};

// A double-float complex entry is one 16-byte vector (re.hi, re.lo, im.hi,
// im.lo): aligned so that it moves with one 128-bit load or store.
template <>
struct alignas(16) cx<df64> {
  df64 re, im;
};

template <typename T>
struct mat {
  cx<T> e[9];
};

// The 3x3 matrices a kernel works on.  FP64 and FP32: plain locals, which the
// compiler keeps in registers.  Double-float: the out-of-line products take
// their operands by address, which would place every matrix of the kernel in
// the per-thread stack (local memory); with hundreds of threads per SM that
// stack outgrows L1 and its dirty lines reach DRAM.  The slots live in
// dynamic shared memory instead, 144 bytes per slot and thread: slot i of
// thread t at mat index (first + i) * blockDim.x + t.  144 bytes is an odd
// multiple of 16, so the 16-byte accesses of a quarter warp to the same
// entry of consecutive threads' slots hit distinct banks.
template <typename T, int N>
struct Work {
  mat<T> m[N];
  __device__ __forceinline__ explicit Work(int) {}
  __device__ __forceinline__ mat<T>& operator[](int i) { return m[i]; }
};
template <int N>
struct Work<df64, N> {
  mat<df64>* base;
  __device__ __forceinline__ explicit Work(int first) {
    extern __shared__ mat<df64> df_work_slots[];
    base = df_work_slots + first * blockDim.x + threadIdx.x;
  }
  __device__ __forceinline__ mat<df64>& operator[](int i) { return base[i * blockDim.x]; }
};

template <typename T> struct vec2_of;
template <> struct vec2_of<double> { typedef double2 type; };
template <> struct vec2_of<float> { typedef float2 type; };
template <> struct vec2_of<df64> { typedef float4 type; };  // (re.hi, re.lo, im.hi, im.lo)

// One complex entry to / from its storage vector.
__device__ __forceinline__ cx<double> unpack(double2 v) { return cx<double>{v.x, v.y}; }
__device__ __forceinline__ cx<float> unpack(float2 v) { return cx<float>{v.x, v.y}; }
__device__ __forceinline__ cx<df64> unpack(float4 v) { return cx<df64>{df64(v.x, v.y), df64(v.z, v.w)}; }
__device__ __forceinline__ double2 pack(cx<double> c) { return make_double2(c.re, c.im); }
__device__ __forceinline__ float2 pack(cx<float> c) { return make_float2(c.re, c.im); }
__device__ __forceinline__ float4 pack(cx<df64> c) { return df_pack(c.re, c.im); }

template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  cx<T> r;
  r.re = a.re * b.re;
  r.re = fma(-a.im, b.im, r.re);
  r.im = a.re * b.im;
  r.im = fma(a.im, b.re, r.im);
  return r;
}
// acc + a*b
template <typename T>
__device__ __forceinline__ cx<T> cfma(cx<T> a, cx<T> b, cx<T> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc - a*b
template <typename T>
__device__ __forceinline__ cx<T> cfms(cx<T> a, cx<T> b, cx<T> acc) {
  acc.re = fma(-a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) {
  return cx<T>{a.re + b.re, a.im + b.im};
}
template <typename T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) {
  return cx<T>{a.re - b.re, a.im - b.im};
}

template <typename T>
__device__ __forceinline__ void set_zero(mat<T>& a) {
#pragma unroll
  for (int k = 0; k < 9; ++k) a.e[k] = cx<T>{T(0), T(0)};
}
template <typename T>
__device__ __forceinline__ void set_ident(mat<T>& a) {
#pragma unroll
  for (int k = 0; k < 9; ++k) a.e[k] = cx<T>{(k % 4 == 0) ? T(1) : T(0), T(0)};
}

// c = a * b
template <typename T>
__device__ __forceinline__ void mul(mat<T>& c, const mat<T>& a, const mat<T>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> s = cmul(a.e[3 * i], b.e[j]);
      s = cfma(a.e[3 * i + 1], b.e[3 + j], s);
      s = cfma(a.e[3 * i + 2], b.e[6 + j], s);
      c.e[3 * i + j] = s;
    }
}
// c += a * b  (SIGN = +1) or c -= a * b (SIGN = -1)
template <int SIGN, typename T>
__device__ __forceinline__ void mul_acc(mat<T>& c, const mat<T>& a, const mat<T>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> s = c.e[3 * i + j];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        s = (SIGN > 0) ? cfma(a.e[3 * i + k], b.e[3 * k + j], s)
                       : cfms(a.e[3 * i + k], b.e[3 * k + j], s);
      c.e[3 * i + j] = s;
    }
}
// c += s * a  (SIGN = +1) or c -= s * a, s real
template <int SIGN, typename T>
__device__ __forceinline__ void axpy(mat<T>& c, T s, const mat<T>& a) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    c.e[k].re = fma(SIGN > 0 ? s : -s, a.e[k].re, c.e[k].re);
    c.e[k].im = fma(SIGN > 0 ? s : -s, a.e[k].im, c.e[k].im);
  }
}

// c = h u with h Hermitian (real diagonal): 10 instead of 12 operations per entry.
template <typename T>
__device__ __forceinline__ void mul_herm_left(mat<T>& c, const mat<T>& h, const mat<T>& u) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T d = h.e[4 * i].re;
      cx<T> s = {d * u.e[3 * i + j].re, d * u.e[3 * i + j].im};
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k != i) s = cfma(h.e[3 * i + k], u.e[3 * k + j], s);
      c.e[3 * i + j] = s;
    }
}
// c = u h with h Hermitian (real diagonal).
template <typename T>
__device__ __forceinline__ void mul_herm_right(mat<T>& c, const mat<T>& u, const mat<T>& h) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T d = h.e[4 * j].re;
      cx<T> s = {d * u.e[3 * i + j].re, d * u.e[3 * i + j].im};
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k != j) s = cfma(u.e[3 * i + k], h.e[3 * k + j], s);
      c.e[3 * i + j] = s;
    }
}

// Double-float products as out-of-line functions.  Inlined, one double-float
// 3x3 product is ~1,400 instructions and the force kernels no longer fit the
// instruction cache (the warps then wait on instruction fetch); called, every
// product site shares one body and takes its operands by address (in the
// kernels' shared-memory workspace, Work above).  The FP64 and FP32 forms
// keep their inlined products.
static __device__ __noinline__ void mul_df(mat<df64>& c, const mat<df64>& a, const mat<df64>& b);
static __device__ __noinline__ void mul_acc_df(mat<df64>& c, const mat<df64>& a, const mat<df64>& b, int sign);
template <>
__device__ __forceinline__ void mul<df64>(mat<df64>& c, const mat<df64>& a, const mat<df64>& b) {
  mul_df(c, a, b);
}
template <>
__device__ __forceinline__ void mul_acc<+1, df64>(mat<df64>& c, const mat<df64>& a, const mat<df64>& b) {
  mul_acc_df(c, a, b, +1);
}
template <>
__device__ __forceinline__ void mul_acc<-1, df64>(mat<df64>& c, const mat<df64>& a, const mat<df64>& b) {
  mul_acc_df(c, a, b, -1);
}
// One entry of a double-float product, sum_k x_k y_k over its six real terms
// (three complex products), accumulated as in the Dot2 algorithm of Ogita,
// Rump and Oishi (SIAM J. Sci. Comput. 26, 2005): each term split exactly
// into p + e (FMA), the p's summed by Knuth's two-sum into s, every rounding
// error and every e gathered in one float lo, and s + lo renormalised once at
// the end.  The dependency chain through s is one add per term, so the terms
// of the real and the imaginary part overlap instead of waiting on a
// renormalised accumulator (~9 dependent operations per double-float FMA);
// the result carries ~2^-48 of sum |term|, as the chained form does.
struct dacc {
  float s, lo;
};
__device__ __forceinline__ void dacc_prod_terms(float& p, float& e, df64 x, df64 y) {
  p = __fmul_rn(x.hi, y.hi);
  e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
}
__device__ __forceinline__ dacc dacc_first(df64 x, df64 y) {
  dacc a;
  dacc_prod_terms(a.s, a.lo, x, y);
  return a;
}
__device__ __forceinline__ void dacc_add(dacc& a, df64 x, df64 y) {
  float p, e;
  dacc_prod_terms(p, e, x, y);
  const float t = a.s + p;
  const float bb = t - a.s;
  const float err = (a.s - (t - bb)) + (p - bb);
  a.s = t;
  a.lo += err + e;
}
__device__ __forceinline__ df64 dacc_get(const dacc& a) { return df_two_sum(a.s, a.lo); }
// Folds lo back into s; over long sums (the cooling gradient's 48 terms per
// entry) this every few terms keeps lo, and so its own rounding, small.
__device__ __forceinline__ void dacc_norm(dacc& a) {
  const df64 t = df_two_sum(a.s, a.lo);
  a.s = t.hi;
  a.lo = t.lo;
}

// The products run row by row: row i of a in registers, the row's three
// entries accumulated side by side (six independent chains per row, and a's
// row read once), the row written at the end.  So c may be a itself
// (mul_left_inplace_df), and each entry adds its terms in the same order as
// an entry-by-entry product would.
static __device__ __noinline__ void mul_df(mat<df64>& c, const mat<df64>& a, const mat<df64>& b) {
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {  // rolled: one row's code in the instruction cache
    const cx<df64> x0 = a.e[3 * i], x1 = a.e[3 * i + 1], x2 = a.e[3 * i + 2];
    dacc re[3], im[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const cx<df64> y = b.e[j];
      re[j] = dacc_first(x0.re, y.re);
      im[j] = dacc_first(x0.re, y.im);
      dacc_add(re[j], -x0.im, y.im);
      dacc_add(im[j], x0.im, y.re);
    }
#pragma unroll
    for (int k = 1; k < 3; ++k) {
      const cx<df64> x = k == 1 ? x1 : x2;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const cx<df64> y = b.e[3 * k + j];
        dacc_add(re[j], x.re, y.re);
        dacc_add(re[j], -x.im, y.im);
        dacc_add(im[j], x.re, y.im);
        dacc_add(im[j], x.im, y.re);
      }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) c.e[3 * i + j] = cx<df64>{dacc_get(re[j]), dacc_get(im[j])};
  }
}
// The same product one entry at a time (both loops rolled): a third of the
// code, for kernels that already wait on instruction fetch (the update).
static __device__ __noinline__ void mul_df_compact(mat<df64>& c, const mat<df64>& a, const mat<df64>& b) {
#pragma unroll 1
  for (int i = 0; i < 3; ++i)
#pragma unroll 1
    for (int j = 0; j < 3; ++j) {
      const cx<df64> x0 = a.e[3 * i], y0 = b.e[j];
      dacc re = dacc_first(x0.re, y0.re), im = dacc_first(x0.re, y0.im);
      dacc_add(re, -x0.im, y0.im);
      dacc_add(im, x0.im, y0.re);
#pragma unroll
      for (int k = 1; k < 3; ++k) {
        const cx<df64> x = a.e[3 * i + k], y = b.e[3 * k + j];
        dacc_add(re, x.re, y.re);
        dacc_add(re, -x.im, y.im);
        dacc_add(im, x.re, y.im);
        dacc_add(im, x.im, y.re);
      }
      c.e[3 * i + j] = cx<df64>{dacc_get(re), dacc_get(im)};
    }
}
// a <- a b in place (row i of a is in registers before it is overwritten):
// one workspace slot fewer.
static __device__ __forceinline__ void mul_left_inplace_df(mat<df64>& a, const mat<df64>& b) { mul_df(a, a, b); }
static __device__ __noinline__ void mul_acc_df(mat<df64>& c, const mat<df64>& a, const mat<df64>& b, int sign) {
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {
    cx<df64> x[3] = {a.e[3 * i], a.e[3 * i + 1], a.e[3 * i + 2]};
    if (sign < 0)
#pragma unroll
      for (int k = 0; k < 3; ++k) x[k] = cx<df64>{-x[k].re, -x[k].im};
    dacc re[3], im[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const cx<df64> c0 = c.e[3 * i + j];
      re[j] = dacc{c0.re.hi, c0.re.lo};
      im[j] = dacc{c0.im.hi, c0.im.lo};
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const cx<df64> y = b.e[3 * k + j];
        dacc_add(re[j], x[k].re, y.re);
        dacc_add(re[j], -x[k].im, y.im);
        dacc_add(im[j], x[k].re, y.im);
        dacc_add(im[j], x[k].im, y.re);
      }
#pragma unroll
    for (int j = 0; j < 3; ++j) c.e[3 * i + j] = cx<df64>{dacc_get(re[j]), dacc_get(im[j])};
  }
}

// Adjugate: adj(a) a = det(a) 1; for det a = 1 it is the inverse.
template <typename T>
__device__ __forceinline__ void adj(mat<T>& r, const mat<T>& a) {
  const cx<T>* m = a.e;
  r.e[0] = cfms(m[5], m[7], cmul(m[4], m[8]));
  r.e[1] = cfms(m[1], m[8], cmul(m[2], m[7]));
  r.e[2] = cfms(m[2], m[4], cmul(m[1], m[5]));
  r.e[3] = cfms(m[3], m[8], cmul(m[5], m[6]));
  r.e[4] = cfms(m[2], m[6], cmul(m[0], m[8]));
  r.e[5] = cfms(m[0], m[5], cmul(m[2], m[3]));
  r.e[6] = cfms(m[4], m[6], cmul(m[3], m[7]));
  r.e[7] = cfms(m[0], m[7], cmul(m[1], m[6]));
  r.e[8] = cfms(m[1], m[3], cmul(m[0], m[4]));
}

template <typename T>
__device__ __forceinline__ cx<T> det(const mat<T>& a) {
  const cx<T>* m = a.e;
  cx<T> c0 = cfms(m[5], m[7], cmul(m[4], m[8]));
  cx<T> c1 = cfms(m[3], m[8], cmul(m[5], m[6]));
  cx<T> c2 = cfms(m[4], m[6], cmul(m[3], m[7]));
  return cfma(m[2], c2, cfma(m[1], c1, cmul(m[0], c0)));
}

template <typename T>
__device__ __forceinline__ cx<T> trace(const mat<T>& a) {
  return cx<T>{a.e[0].re + a.e[4].re + a.e[8].re, a.e[0].im + a.e[4].im + a.e[8].im};
}

// Re Tr(a b) and Im Tr(a b) without forming the product.
template <typename T>
__device__ __forceinline__ cx<T> trace_mul(const mat<T>& a, const mat<T>& b) {
  cx<T> s = cmul(a.e[0], b.e[0]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (i + k > 0) s = cfma(a.e[3 * i + k], b.e[3 * k + i], s);
  return s;
}

// sum_ij |a_ij|^2 = Tr a a^+
template <typename T>
__device__ __forceinline__ T norm2(const mat<T>& a) {
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) s = fma(a.e[k].re, a.e[k].re, fma(a.e[k].im, a.e[k].im, s));
  return s;
}

// One real from type S to type D; float <-> double on the integer pipe (cvt.cuh).
template <typename D, typename S>
__device__ __forceinline__ D cvt(S x) {
  return (D)x;
}
template <>
__device__ __forceinline__ double cvt<double, float>(float x) {
  return f2d(x);
}
template <>
__device__ __forceinline__ float cvt<float, double>(double x) {
  return d2f(x);
}

template <typename D, typename S>
__device__ __forceinline__ void convert(mat<D>& d, const mat<S>& s) {
#pragma unroll
  for (int k = 0; k < 9; ++k) d.e[k] = cx<D>{cvt<D>(s.e[k].re), cvt<D>(s.e[k].im)};
}

// SoA field access: element k of matrix (plane, site) at ((plane*9 + k)*V + site).
template <typename T>
__device__ __forceinline__ void load(mat<T>& a, const typename vec2_of<T>::type* __restrict__ f,
                                     int plane, int site, int V) {
  const typename vec2_of<T>::type* p = f + (size_t)plane * 9 * V + site;
#pragma unroll
  for (int k = 0; k < 9; ++k) a.e[k] = unpack(__ldg(p + (size_t)k * V));
}
template <typename T>
__device__ __forceinline__ void store(typename vec2_of<T>::type* __restrict__ f, int plane,
                                      int site, int V, const mat<T>& a) {
  typename vec2_of<T>::type* p = f + (size_t)plane * 9 * V + site;
#pragma unroll
  for (int k = 0; k < 9; ++k) p[(size_t)k * V] = pack(a.e[k]);
}

}  // namespace clgc
