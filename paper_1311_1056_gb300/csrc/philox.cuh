// philox.cuh -- counter-based noise for the CL update and the random starts.
//
// Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw, "Parallel
// random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64
// multiplies with the Weyl key schedule.  Keys and counters:
//   key     = (seed & 0xffffffff, seed >> 32)
//   counter = (site, step, slot | stream << 8, j)
// stream 0 = CL noise (slot = mu), 1 = random gauge transformation (slot 0),
// 2 = hot start (slot = mu).  Counter j gives one Box-Muller pair from the
// uniforms u = (k + 1/2) 2^-52, k = (w0 >> 6) 2^26 + (w1 >> 6), which lie in (0,1).
// The noise of a link is a function of (seed, step, site, mu) only, so a
// replay, a CUDA graph or a different launch shape draws the same numbers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bm_tables.cuh"
#include "df64.cuh"

namespace clgc {

enum { STREAM_CL = 0, STREAM_GAUGE = 1, STREAM_HOT = 2 };

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 philox_words(uint64_t seed, uint32_t step, uint32_t site,
                                              uint32_t slot, uint32_t stream, uint32_t j) {
  return philox4x32_10(make_uint4(site, step, slot | (stream << 8), j),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// ------------------------------------------------------ FP64 Box-Muller
// GB300 issues FP64 at 1/64 of its FP32 rate, and CUDA's general log and
// sincospi took ~60 of the ~80 FP64 issue slots of a Box-Muller pair.  The
// arguments here are narrow -- uniforms (k + 1/2) 2^-52 with 0 <= k < 2^52 --
// so the pair uses table-driven versions (Tang's method: a tabulated value at
// the nearest grid point combined with a short polynomial in the remainder;
// tables and coefficients from bm_tables.py), ~13 + ~15 slots, within 2-3
// ulp of the correctly rounded values (cl_selftest_box_muller compares them
// with CUDA's functions).

// u = (k + 1/2) 2^-52 from its bits: n = 2k + 1 with top bit p is u = n 2^-53.
__device__ __forceinline__ double u52_bits(uint64_t k) {
  const uint64_t n = 2 * k + 1;
  const int p = 63 - __clzll((long long)n);  // 0 .. 52
  const uint64_t mant = (n << (52 - p)) & 0xFFFFFFFFFFFFFull;
  return __longlong_as_double((long long)(((uint64_t)(p - 53 + 1023) << 52) | mant));
}

// ln u for normal u in (0, 1): u = 2^e m with m in [sqrt(1/2), sqrt(2)), c the
// nearest multiple of 1/128, ln u = e ln 2 + ln c + ln(1 + t), t = (m - c)/c,
// |t| <= 1/180, ln(1 + t) to t^7 (the next term is below 2^-56 relative).
__device__ __forceinline__ double ln_unit(double u) {
  const uint64_t b = (uint64_t)__double_as_longlong(u);
  const uint64_t mant = b & 0xFFFFFFFFFFFFFull;
  const bool high = mant >= 0x6A09E667F3BCDull;  // m >= sqrt(2): take m / 2, e + 1
  const int e = (int)(b >> 52) - 1023 + (high ? 1 : 0);
  const int j = high ? 64 + (int)((mant + (1ull << 45)) >> 46) : 128 + (int)((mant + (1ull << 44)) >> 45);
  const double m = __longlong_as_double((long long)(((high ? 1022ull : 1023ull) << 52) | mant));
  // c = j / 128 from its bits (90 <= j <= 181)
  const double c = j >= 128 ? __longlong_as_double((long long)((1023ull << 52) | ((uint64_t)(j - 128) << 45)))
                            : __longlong_as_double((long long)((1022ull << 52) | ((uint64_t)(j - 64) << 46)));
  const double2 rl = __ldg(&BM_LN_TAB[j - 90]);  // (1 / c, ln c)
  const double t = (m - c) * rl.x;                // m - c is exact
  double q = fma(t, 1.0 / 7.0, -1.0 / 6.0);
  q = fma(t, q, 1.0 / 5.0);
  q = fma(t, q, -0.25);
  q = fma(t, q, 1.0 / 3.0);
  q = fma(t, q, -0.5);
  const double lp = fma(t * t, q, t);             // ln(1 + t)
  // e as a double without a conversion instruction (|e| <= 53)
  const double ed = __longlong_as_double(0x4338000000000000ll + e) - 6755399441055744.0;
  const double hi = fma(ed, BM_LN2_HI, rl.y);     // e LN2_HI is exact
  const double lo = fma(ed, BM_LN2_LO, lp);
  return hi + lo;
}

// sin(pi x), cos(pi x) for x = 2u = (2k + 1) 2^-52: x = j / 64 + y with j the
// nearest multiple (0 .. 128) and |y| <= 1/128 exact, then the angle-sum
// formulas with the tabulated sin, cos(pi j / 64) and Taylor polynomials in y.
__device__ __forceinline__ void sincospi_2u52(uint64_t k, double* sn, double* cs) {
  const uint64_t n = 2 * k + 1;
  const int j = (int)((n + (1ull << 45)) >> 46);
  const long long r = (long long)n - ((long long)j << 46);  // |r| <= 2^45
  const double y = (__longlong_as_double(0x4338000000000000ll + r) - 6755399441055744.0) * 0x1p-52;
  const double y2 = y * y;
  const double sp = y * fma(y2, fma(y2, fma(y2, BM_S7, BM_S5), BM_S3), BM_S1);
  const double cp = fma(y2, fma(y2, fma(y2, fma(y2, BM_C8, BM_C6), BM_C4), BM_C2), 1.0);
  const double2 t = __ldg(&BM_SC_TAB[j]);  // (sin, cos)(pi j / 64)
  *sn = fma(t.x, cp, t.y * sp);
  *cs = fma(t.y, cp, -(t.x * sp));
}

// 2*NP standard normal numbers, Box-Muller in FP64.
template <int NP>
__device__ __forceinline__ void normals_f64(double* g, uint64_t seed, uint32_t step, uint32_t site,
                                            uint32_t slot, uint32_t stream) {
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    uint4 w = philox_words(seed, step, site, slot, stream, (uint32_t)j);
    const uint64_t k1 = ((uint64_t)(w.x >> 6) << 26) | (w.y >> 6), k2 = ((uint64_t)(w.z >> 6) << 26) | (w.w >> 6);
    double rad = sqrt(-2.0 * ln_unit(u52_bits(k1)));
    double s, c;
    sincospi_2u52(k2, &s, &c);
    g[2 * j] = rad * c;
    g[2 * j + 1] = rad * s;
  }
}

// The 52-bit uniform (k + 1/2) 2^-52 in double-float from three exact float
// pieces: bits 51..28 of k, bits 27..4, and bits 3..0 plus the half.
__device__ __forceinline__ df64 uniform52_df(uint32_t hi, uint32_t lo) {
  const uint32_t h = hi >> 6, l = lo >> 6;  // k = h 2^26 + l
  const float A = (float)(h >> 2) * 5.9604644775390625e-8f;                                // 2^-24
  const float B = (float)(((h & 3u) << 22) | (l >> 4)) * 3.5527136788005009e-15f;         // 2^-48
  const float C = ((float)(l & 15u) + 0.5f) * 2.220446049250313080847e-16f;              // 2^-52
  return df_two_sum(A, B) + df64(C, 0.0f);
}

// The same numbers in double-float (~2^-46 relative), with no FP64
// instruction: ln, sqrt and sincospi of df64.cuh.  Used by the DF64 form.
template <int NP>
__device__ __forceinline__ void normals_df64(df64* g, uint64_t seed, uint32_t step, uint32_t site,
                                             uint32_t slot, uint32_t stream) {
#pragma unroll 1
  for (int j = 0; j < NP; ++j) {  // rolled: one pair's ~450 instructions, not NP copies, in the instruction cache
    uint4 w = philox_words(seed, step, site, slot, stream, (uint32_t)j);
    // 1 - u1 = (k' + 1/2) 2^-52 with k' the 52-bit complement of k: exact
    const df64 u1 = uniform52_df(w.x, w.y), v1 = uniform52_df(~w.x, ~w.y);
    const df64 u2 = uniform52_df(w.z, w.w);
    const df64 rad = df_sqrt(df_ldexp(-df_log_unit(u1, v1), 1));
    df64 s, c;
    df_sincospi(df_ldexp(u2, 1), &s, &c);
    g[2 * j] = rad * c;
    g[2 * j + 1] = rad * s;
  }
}

// The same numbers to float precision, with no FP64 instruction.  The radius
// uniform is the 52-bit one, (k_hi 2^26 + k_lo + 1/2) 2^-52, summed in float:
// it keeps float's relative precision down to the smallest u1, where the
// logarithm is steep (a 24-bit grid u = (k + 1/2) 2^-24 would be off by a
// relative 2^-24 / u1 there, ~1 % for the rare u1 ~ 1e-5 of the tail).  The
// angle uniform needs absolute precision only: u2 = (k + 1/2) 2^-24 from the
// top 24 bits of its first word.  Used by the FP32-storage form, whose links
// carry FP32 precision anyway.
template <int NP>
__device__ __forceinline__ void normals_f32(float* g, uint64_t seed, uint32_t step, uint32_t site,
                                            uint32_t slot, uint32_t stream) {
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    uint4 w = philox_words(seed, step, site, slot, stream, (uint32_t)j);
    float u1 = fmaf((float)(w.x >> 6), 1.490116119384765625e-8f,            // 2^-26
                    ((float)(w.y >> 6) + 0.5f) * 2.220446049250313080847e-16f);  // 2^-52
    float u2 = ((float)(w.z >> 8) + 0.5f) * 5.9604644775390625e-8f;
    float rad = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    g[2 * j] = rad * c;
    g[2 * j + 1] = rad * s;
  }
}

}  // namespace clgc
