// Split of a double d into the float-float pair (RN(d), RN(d - RN(d))) --
// the two roundings to nearest even that converting d to float, and the exact
// remainder d - RN(d) to float, give -- with 32-bit integer and FP32
// operations only.
//
// GB300 issues FP64 arithmetic, and conversions from and to FP64, at 2 per SM
// per clock against 128 for FP32; a kernel that only turns FP64 state into
// float-float pairs is bound by that pipe when it converts with FP64
// operations (four per value). Here the significand is cut at bit 24 with
// integer operations, rounded to nearest even, and the remainder (at most 29
// bits) is rounded to float by one FMA of two exactly representable halves.
//
// The fast path covers 2^-60 <= |d| < 2^100 and d = +-0, where both parts are
// normal floats (or zero); ff_split_fast returns false elsewhere (subnormal,
// tiny, huge, infinite or NaN d), and the caller converts with FP64
// operations. The header also compiles as plain C++ so that the host tests
// can check it bit for bit against the FP64 conversion.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define LP_FFS_FN __host__ __device__ __forceinline__
#else
#include <math.h>
#include <string.h>
#define LP_FFS_FN static inline
#endif

LP_FFS_FN uint64_t ffs_bits_of(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  memcpy(&b, &d, sizeof b);
  return b;
#endif
}

LP_FFS_FN float ffs_float_of(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
#endif
}

// x (< 2^23) as a float, exactly: 2^23 + x has the bit pattern 0x4b000000 | x
LP_FFS_FN float ffs_small(uint32_t x) {
  return ffs_float_of(0x4b000000u | x) - 8388608.0f;
}

LP_FFS_FN float ffs_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}

LP_FFS_FN bool ff_split_fast(double d, float* h, float* l) {
  const uint64_t b = ffs_bits_of(d);
  const uint32_t hi32 = (uint32_t)(b >> 32), lo32 = (uint32_t)b;
  const uint32_t sign = hi32 & 0x80000000u;
  if (((hi32 & 0x7fffffffu) | lo32) == 0u) {  // +-0: RN(d) = d, remainder +0
    *h = ffs_float_of(sign);
    *l = 0.0f;
    return true;
  }
  const int e = (int)((hi32 >> 20) & 0x7ffu) - 1023;  // unbiased exponent
  if (e < -60 || e >= 100) return false;
  // 53-bit significand m = 1.f (as an integer): its top 24 bits q, low 29 bits r
  uint32_t q = (((hi32 & 0x000fffffu) | 0x00100000u) << 3) | (lo32 >> 29);
  const uint32_t r = lo32 & 0x1fffffffu;
  const bool up = r > 0x10000000u || (r == 0x10000000u && (q & 1u));
  q += up ? 1u : 0u;
  // RN(d) = q 2^(e-23); q = 2^24 carries into the exponent field
  *h = ffs_float_of(sign | ((((uint32_t)(e + 127)) << 23) + (q - 0x00800000u)));
  // d - RN(d) = +-a 2^(e-52) with a <= 2^28; RN(a) from its two 15-bit halves
  // (exact in FP32) with one rounding
  const uint32_t a = up ? 0x20000000u - r : r;
  const float fa = ffs_fma(ffs_small(a >> 15), 32768.0f, ffs_small(a & 0x7fffu));
  // the remainder's sign: d's, flipped when RN(d) rounded away from zero; +0 when exact
  const uint32_t ls = a == 0u ? 0u : (sign ^ (up ? 0x80000000u : 0u));
  *l = fa * ffs_float_of(ls | (((uint32_t)(e - 52 + 127)) << 23));  // exact: 2^(e-52) >= 2^-112
  return true;
}

// float -> double, exactly, with integer operations (the conversion
// instruction runs on the FP64 pipe): a normal float's exponent is re-biased
// and its significand shifted into place; zeros keep their sign; subnormal,
// infinite and NaN floats take the conversion instruction.
LP_FFS_FN double ffs_double_of_bits(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
#endif
}
LP_FFS_FN double ffs_to_double(float f) {
  uint32_t b;
#ifdef __CUDA_ARCH__
  b = __float_as_uint(f);
#else
  memcpy(&b, &f, sizeof b);
#endif
  const uint32_t e = (b >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  if ((b & 0x7fffffffu) == 0u) return ffs_double_of_bits(sign);
  if (e == 0u || e == 0xffu) return (double)f;
  return ffs_double_of_bits(sign | ((uint64_t)(e + 896u) << 52) |
                            ((uint64_t)(b & 0x007fffffu) << 29));
}
