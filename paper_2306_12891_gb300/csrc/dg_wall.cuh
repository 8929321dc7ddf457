// dg_wall.cuh -- the wall model of Sec. 3: Spalding's law of the wall (Eq. (2)) solved for the
// friction velocity by Newton's method, with the van Driest transform (Eq. (5)) of the input
// velocity. Templated on the arithmetic type; shared by the face kernel and dg_wall_model.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

// y+ of u+: u+ + 0.1108 [exp(0.4 u+) - 1 - 0.4u+ - (0.4u+)^2/2! - (0.4u+)^3/3! - (0.4u+)^4/4!]
template <typename R>
static __device__ __forceinline__ R spalding_y(R up) {
  const R k = R(0.4) * up;
  return up + R(0.1108) * (exp(k) - R(1) - k - k * k / R(2) - k * k * k / R(6) - k * k * k * k / R(24));
}
template <typename R>
static __device__ __forceinline__ R spalding_dy(R up) {
  const R k = R(0.4) * up;
  return R(1) + R(0.1108) * R(0.4) * (exp(k) - R(1) - k - k * k / R(2) - k * k * k / R(6));
}

// u+ with u+ y+(u+) = Re_h = h U / nu. The left side is increasing and convex for u+ > 0 and
// y+ >= u+, so the root is at most sqrt(Re_h): Newton from min(sqrt(Re_h), 60) decreases
// monotonically to it (one overshoot from below when the root exceeds 60). At most 100 steps.
template <typename R>
static __device__ __forceinline__ R wall_uplus(R Re, int &iters) {
  iters = 0;
  if (!(Re > R(0))) return R(0);
  R up = sqrt(Re);
  if (up > R(60)) up = R(60);
  const R tol = std::is_same<R, float>::value ? R(1e-6) : R(1e-15);
  for (int it = 0; it < 100; ++it) {
    const R y = spalding_y(up), dy = spalding_dy(up);
    const R step = (up * y - Re) / (y + up * dy);
    up -= step;
    iters = it + 1;
    if (fabs(step) <= tol * fabs(up)) break;
  }
  return up;
}

// b of the van Driest transform: b = sqrt(r m) / sqrt(1 + r m), m = (gamma-1)/2 Ma^2, r = Pr^(1/3)
static inline double van_driest_b(double mainf, double gamma, double Pr) {
  const double m = 0.5 * (gamma - 1.0) * mainf * mainf * cbrt(Pr);
  return sqrt(m) / sqrt(1.0 + m);
}

// friction velocity for tangential speed U at wall distance h, kinematic viscosity nu; with the van
// Driest transform u_eq = (u_inf / b) asin(b U / u_inf) when vd != 0 and b > 0
template <typename R>
static __device__ __forceinline__ R wall_utau(R U, R h, R nu, R uinf, R b, int vd, int &iters) {
  R ueq = U;
  if (vd && b > R(0) && uinf > R(0)) ueq = uinf / b * asin(b * U / uinf);
  iters = 0;
  if (!(ueq > R(0))) return R(0);
  const R up = wall_uplus(h * ueq / nu, iters);
  return ueq / up;
}
