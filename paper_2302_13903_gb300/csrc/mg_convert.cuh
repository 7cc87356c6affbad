// mg_convert.cuh -- conversions between IEEE 754 binary64 / binary32 and
// 64-bit integers, rounding to nearest with ties to even, in integer
// arithmetic.
//
// The hardware conversions between 64-bit integers and floating point, and
// from binary64 to binary32, issue on the FP64 pipe, which on this GPU runs at
// about 1/60 of the FP32 rate.  The whole-array passes of the fixed-point
// outer loop convert every cell, so with them they would be bound by that pipe
// instead of by memory.  The functions below compute the same values from the
// definitions of the encodings (sign bit, biased exponent, significand with its
// implicit leading 1) with shifts, adds and compares; every result is the
// correctly rounded one, i.e. the same bits the hardware conversion returns.
// Inputs outside a function's stated range saturate as the hardware does.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace mg {
namespace cvt {

// round(m / 2^n), ties to even, for n >= 1 and m < 2^63 (the result is 0 for
// n >= 64).
__device__ __forceinline__ uint64_t shr_rne(uint64_t m, int n) {
  if (n >= 64) return 0;
  const uint64_t q = m >> n;
  const uint64_t rem = m & ((1ULL << n) - 1);
  const uint64_t half = 1ULL << (n - 1);
  return q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
}

// binary64 -> int64; |x| >= 2^63 saturates, NaN gives 0.
__device__ __forceinline__ long long d2ll_rn(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ff);
  const uint64_t frac = u & 0xFFFFFFFFFFFFFULL;
  const bool neg = (u >> 63) != 0;
  if (e == 0x7ff && frac) return 0;
  if (e >= 1086) return neg ? (long long)0x8000000000000000ULL : 0x7fffffffffffffffLL;
  const uint64_t m = frac | (e ? (1ULL << 52) : 0);  // x = m 2^(e - 1075) (e >= 1)
  const int k = e - 1075;
  const uint64_t a = k >= 0 ? (m << k) : shr_rne(m, -k);
  return neg ? (long long)(0 - a) : (long long)a;
}

// int64 -> binary64.
__device__ __forceinline__ double ll2d_rn(long long v) {
  if (v == 0) return 0.0;
  const uint64_t s = (uint64_t)v >> 63;
  const uint64_t a = s ? 0 - (uint64_t)v : (uint64_t)v;
  const int p = 63 - __clzll((long long)a);  // 2^p <= a < 2^(p+1)
  const uint64_t q = p <= 52 ? (a << (52 - p)) : shr_rne(a, p - 52);  // in [2^52, 2^53]
  // q's leading bit adds one to the biased exponent p + 1022; q = 2^53 (a
  // rounding carry) adds two, which is 2^(p+1) with a zero significand
  return __longlong_as_double((long long)((s << 63) + ((uint64_t)(p + 1022) << 52) + q));
}

// int64 v times 2^-S -> binary64: the exponent of ll2d_rn(v) lowered by S,
// which is exact while the result stays a normal number (|S| well inside the
// exponent range); otherwise a rounded scale in FP64.
__device__ __forceinline__ double ll2d_pow2_rn(long long v, int S) {
  if (v == 0) return 0.0;
  const uint64_t s = (uint64_t)v >> 63;
  const uint64_t a = s ? 0 - (uint64_t)v : (uint64_t)v;
  const int p = 63 - __clzll((long long)a);
  const int E = p + 1023 - S;  // biased exponent of the result
  if (E < 1 || E > 2046) return ldexp(ll2d_rn(v), -S);
  const uint64_t q = p <= 52 ? (a << (52 - p)) : shr_rne(a, p - 52);
  return __longlong_as_double((long long)((s << 63) + ((uint64_t)(E - 1) << 52) + q));
}

// binary64 -> binary32, subnormal results included.
__device__ __forceinline__ float d2f_rn(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint32_t s = (uint32_t)(u >> 63) << 31;
  const int e = (int)((u >> 52) & 0x7ff);
  const uint64_t frac = u & 0xFFFFFFFFFFFFFULL;
  if (e == 0x7ff) return __uint_as_float(s | 0x7f800000u | (frac ? 0x400000u : 0u));
  const int E = e - 896;  // binary32 biased exponent of the same power of two
  uint32_t bits;
  if (E >= 255) {
    bits = 0x7f800000u;  // beyond the binary32 range
  } else if (E >= 1) {
    const uint64_t q = shr_rne(frac | (1ULL << 52), 29);  // in [2^23, 2^24]
    bits = ((uint32_t)(E - 1) << 23) + (uint32_t)q;
    if (bits > 0x7f800000u) bits = 0x7f800000u;
  } else if (e == 0) {
    bits = 0;  // |x| < 2^-1022
  } else {
    // a multiple of the binary32 subnormal unit 2^-149: x / 2^-149 = m 2^(e - 926)
    bits = (uint32_t)shr_rne(frac | (1ULL << 52), 926 - e);
  }
  return __uint_as_float(s | bits);
}

// binary32 -> int64; |x| >= 2^63 saturates, NaN gives 0.
__device__ __forceinline__ long long f2ll_rn(float x) {
  const uint32_t u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xff);
  const bool neg = (u >> 31) != 0;
  if (e == 0xff && (u & 0x7fffff)) return 0;
  if (e >= 190) return neg ? (long long)0x8000000000000000ULL : 0x7fffffffffffffffLL;
  const uint64_t m = (uint64_t)((u & 0x7fffffu) | (e ? 0x800000u : 0u));  // x = m 2^(e - 150)
  const int k = e - 150;
  const uint64_t a = k >= 0 ? (m << k) : shr_rne(m, -k);
  return neg ? (long long)(0 - a) : (long long)a;
}

// int64 -> binary32.
__device__ __forceinline__ float ll2f_rn(long long v) {
  if (v == 0) return 0.f;
  const uint32_t s = (uint32_t)((uint64_t)v >> 63);
  const uint64_t a = s ? 0 - (uint64_t)v : (uint64_t)v;
  const int p = 63 - __clzll((long long)a);
  const uint64_t q = p <= 23 ? (a << (23 - p)) : shr_rne(a, p - 23);  // in [2^23, 2^24]
  return __uint_as_float((s << 31) + ((uint32_t)(p + 126) << 23) + (uint32_t)q);
}

}  // namespace cvt
}  // namespace mg
