// dg_invariants_node.cuh -- the per-node integrand of the integral diagnostics, shared by the
// context reduction (k_invariants) and the allocation-free one (dg_invariants_noalloc), so the two
// cannot drift apart.
//
// With the quadrature weight wq = w_i w_j w_k J of a node, its state Uv and right-hand side Tv, it
// adds to acc[8]:
//   acc[0..4] += wq Ut_v                          (conservation: the weighted sums of the RHS)
//   acc[5]    += wq v(U) . Ut                     (entropy production, v = entropy variables
//                                                  ((gamma - s)/(gamma - 1) - rho|u|^2/(2p), rho u/p, -rho/p),
//                                                  s = ln(p rho^-gamma))
//   acc[6]    += wq rho|u|^2 / 2                  (kinetic energy)
//   acc[7]    += wq (u . (rho u)_t - |u|^2 rho_t / 2)   (its rate)
#pragma once

__device__ __forceinline__ void invariants_node(double gam, double wq, const double Uv[5], const double Tv[5],
                                                double acc[8]) {
  const double r = Uv[0], ir = 1.0 / r;
  const double u = Uv[1] * ir, v = Uv[2] * ir, w = Uv[3] * ir;
  const double q2 = u * u + v * v + w * w;
  const double p = (gam - 1.0) * (Uv[4] - 0.5 * r * q2);
  const double s = log(p) - gam * log(r);
  const double ip = 1.0 / p;
  const double ev[5] = {(gam - s) / (gam - 1.0) - 0.5 * r * q2 * ip, r * u * ip, r * v * ip, r * w * ip, -r * ip};
#pragma unroll
  for (int m = 0; m < 5; ++m) acc[m] += wq * Tv[m];
  acc[5] += wq * (ev[0] * Tv[0] + ev[1] * Tv[1] + ev[2] * Tv[2] + ev[3] * Tv[3] + ev[4] * Tv[4]);
  acc[6] += wq * 0.5 * r * q2;
  acc[7] += wq * (u * Tv[1] + v * Tv[2] + w * Tv[3] - 0.5 * q2 * Tv[0]);
}
