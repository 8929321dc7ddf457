// dg_convert.cuh -- float <-> double conversions written on the integer pipes, from the IEEE-754
// binary32/binary64 encodings.
#pragma once
#include <cuda_runtime.h>

// IEEE-754 conversions on the integer pipes (GB300 issues FP64 instructions, conversions included,
// at 1/64 of the FP32 rate). Normal numbers take a short branch-free path (exponent rebias by an
// integer add; round to nearest even as rest + lsb > half); the rest take the general path below.
// float -> double is exact; float subnormals (|f| < 2^-126) become zero, infinities and NaNs are kept.
static __device__ __forceinline__ double f2d_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7FFFFFFFu;
  if (a - 0x00800000u < 0x7F000000u) {  // normal float: rebias the exponent by 1023 - 127 = 896
    const unsigned hi = ((a >> 3) + (896u << 20)) | (u & 0x80000000u);
    return __hiloint2double((int)hi, (int)(a << 29));
  }
  const unsigned ex = (u >> 23) & 0xFFu;
  const unsigned long long man = (unsigned long long)(u & 0x7FFFFFu) << 29;
  const unsigned long long e64 = ex == 0u ? 0ull : ex == 0xFFu ? 0x7FFull : (unsigned long long)(ex + 896u);
  const unsigned long long mag = ex == 0u ? 0ull : (e64 << 52) | man;
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) | mag));
}
// double -> float, round to nearest even; results below the normal float range become zero,
// overflow gives infinity, NaN stays NaN
static __device__ __forceinline__ float d2f_int(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ahi = hi & 0x7FFFFFFFu;
  if (ahi - (897u << 20) < (254u << 20)) {  // float exponent 1..254: rebias, keep 23 mantissa bits, round
    unsigned q = ((ahi - (896u << 20)) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;
    q += (rest + (q & 1u)) > 0x10000000u ? 1u : 0u;  // nearest even; a carry moves to the next binade
    return __uint_as_float(q | (hi & 0x80000000u));   // (or to infinity above the largest float)
  }
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7FFull);
  const unsigned long long man = b & 0xFFFFFFFFFFFFFull;
  const int fe = ex - 896;
  if (ex == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (man ? 0x400000u : 0u));
  if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
  if (fe <= 0) return __uint_as_float(sign);
  const unsigned m = (unsigned)(man >> 29);
  const unsigned rest = (unsigned)(man & 0x1FFFFFFFull), half = 0x10000000u;
  unsigned r = ((unsigned)fe << 23) | m;
  r += (rest > half || (rest == half && (m & 1u))) ? 1u : 0u;  // a carry moves to the next binade
  return __uint_as_float(sign | r);
}
