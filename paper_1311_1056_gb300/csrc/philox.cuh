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

__device__ __forceinline__ double uniform52(uint32_t hi, uint32_t lo) {
  double k = fma((double)(hi >> 6), 67108864.0, (double)(lo >> 6));
  return (k + 0.5) * (1.0 / 4503599627370496.0);
}

__device__ __forceinline__ uint4 philox_words(uint64_t seed, uint32_t step, uint32_t site,
                                              uint32_t slot, uint32_t stream, uint32_t j) {
  return philox4x32_10(make_uint4(site, step, slot | (stream << 8), j),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// 2*NP standard normal numbers, Box-Muller in FP64.
template <int NP>
__device__ __forceinline__ void normals_f64(double* g, uint64_t seed, uint32_t step, uint32_t site,
                                            uint32_t slot, uint32_t stream) {
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    uint4 w = philox_words(seed, step, site, slot, stream, (uint32_t)j);
    double u1 = uniform52(w.x, w.y), u2 = uniform52(w.z, w.w);
    double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
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
