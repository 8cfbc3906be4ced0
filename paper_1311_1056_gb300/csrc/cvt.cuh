// cvt.cuh -- float <-> double conversions on the integer pipe.
//
// On this GPU a conversion between float and double issues on the FP64 pipe
// at that pipe's rate (two per SM per clock, the rate of a DFMA).  In the
// FP32-storage form the FP64 pipe carries the exponentials, the det
// re-projection and the reductions, and the conversions into and out of
// them (the exponent into FP64, the exponential and the det factor back to
// float, the product back to FP64 for its det) took about a fifth of that
// pipe's issue slots.
//
// IEEE-754 binary32 and binary64 differ only in field widths (8/23 vs 11/52
// exponent/mantissa bits) and exponent bias (127 vs 1023).  So a normal
// float widens exactly by moving its fields and adding 1023 - 127 = 896 to
// the exponent, and a double whose value lies in the normal float range
// narrows by keeping the top 23 mantissa bits and rounding on the 29 dropped
// ones, to nearest with ties to even (a carry out of the mantissa correctly
// bumps the exponent, up to +inf above FLT_MAX).  Both are a few integer
// operations.  Zeros are handled in place; subnormal, infinite and NaN
// values, which the hot path does not produce, take the hardware
// conversion.  cl_selftest_convert checks both against the hardware
// conversions bit for bit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace clgc {

// Exact float -> double.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned mag = u & 0x7fffffffu;
  const unsigned ef = mag >> 23;
  if (ef - 1u < 254u) {  // normal: exponent field 1..254
    const unsigned hi = (u & 0x80000000u) | ((mag >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(u << 29));
  }
  if (mag == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  return (double)f;
}

// double -> float, round to nearest, ties to even.
__device__ __forceinline__ float d2f(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned mag = hi & 0x7fffffffu;
  const unsigned ed = mag >> 20;
  if (ed - 897u < 254u) {  // the float exponent field ed - 896 is 1..254
    unsigned r = (hi & 0x80000000u) | ((mag - (896u << 20)) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;
    r += (unsigned)(rest > 0x10000000u) | ((unsigned)(rest == 0x10000000u) & r);
    return __uint_as_float(r);
  }
  if ((mag | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
  return __double2float_rn(d);
}

}  // namespace clgc
