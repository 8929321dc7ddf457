// dg_convert.cuh -- float <-> double conversions written on the integer pipes, from the IEEE-754
// binary32/binary64 encodings.
#pragma once
#include <cuda_runtime.h>

// IEEE-754 conversions on the integer pipes (GB300 issues FP64 instructions, conversions included,
// at 1/64 of the FP32 rate). float -> double is exact; float subnormals (|f| < 2^-126) become
// zero, infinities and NaNs are kept.
static __device__ __forceinline__ double f2d_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFFu;
  const unsigned long long man = (unsigned long long)(u & 0x7FFFFFu) << 29;
  const unsigned long long e64 = ex == 0u ? 0ull : ex == 0xFFu ? 0x7FFull : (unsigned long long)(ex + 896u);
  const unsigned long long mag = ex == 0u ? 0ull : (e64 << 52) | man;
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) | mag));
}
// double -> float, round to nearest even; results below the normal float range become zero,
// overflow gives infinity, NaN stays NaN
static __device__ __forceinline__ float d2f_int(double x) {
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
