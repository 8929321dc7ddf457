// dg_dual.cuh -- forward-mode dual numbers with K derivative components, used to differentiate the
// pointwise Riemann fluxes for the adjoint (vector-Jacobian product) of the surface term: seeding
// the ten inputs (U_L, U_R) gives the full 5 x 10 Jacobian in one evaluation of the flux code.
#pragma once
#include <cuda_runtime.h>

template <int K>
struct Dual {
  double v;
  double d[K];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(double x) : v(x) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = 0.0;
  }
};

template <int K>
__device__ __forceinline__ Dual<K> operator+(const Dual<K> &a, const Dual<K> &b) {
  Dual<K> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K> &a, const Dual<K> &b) {
  Dual<K> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K> &a) {
  Dual<K> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator*(const Dual<K> &a, const Dual<K> &b) {
  Dual<K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator/(const Dual<K> &a, const Dual<K> &b) {
  Dual<K> r;
  const double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> &operator+=(Dual<K> &a, const Dual<K> &b) { return a = a + b; }
template <int K>
__device__ __forceinline__ Dual<K> &operator*=(Dual<K> &a, const Dual<K> &b) { return a = a * b; }
template <int K>
__device__ __forceinline__ bool operator<(const Dual<K> &a, const Dual<K> &b) { return a.v < b.v; }
template <int K>
__device__ __forceinline__ bool operator<=(const Dual<K> &a, const Dual<K> &b) { return a.v <= b.v; }
template <int K>
__device__ __forceinline__ bool operator>(const Dual<K> &a, const Dual<K> &b) { return a.v > b.v; }

template <int K>
__device__ __forceinline__ Dual<K> sqrt(const Dual<K> &a) {
  Dual<K> r;
  r.v = ::sqrt(a.v);
  const double h = 0.5 / r.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * h;
  return r;
}
// 1/sqrt(a); d/da a^(-1/2) = -a^(-3/2) / 2
template <int K>
__device__ __forceinline__ Dual<K> rsq(const Dual<K> &a) {
  Dual<K> r;
  r.v = ::rsqrt(a.v);
  const double h = -0.5 * r.v * r.v * r.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * h;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> log(const Dual<K> &a) {
  Dual<K> r;
  r.v = ::log(a.v);
  const double ia = 1.0 / a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * ia;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> fabs(const Dual<K> &a) { return a.v < 0.0 ? -a : a; }
// the derivative follows the larger argument (the left one on ties)
template <int K>
__device__ __forceinline__ Dual<K> fmax(const Dual<K> &a, const Dual<K> &b) { return b.v > a.v ? b : a; }
