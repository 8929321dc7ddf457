// dg_adjoint.cuh -- discrete adjoint (vector-Jacobian product) of the FP64 split-form DGSEM
// right-hand side L(U) for ONE polynomial degree; included after dg_kernels.cuh in the same
// translation unit (same anonymous namespace, same constant tables).
//
// Given a cotangent lambda of Ut = L(U), the kernels form Ubar = (dL/dU)^T lambda, the transpose
// of exactly the operator the forward kernels apply (zero-diagonal flux differencing with the
// SBP surface identity, Riemann flux once per face point, BR1 lifting with central face values,
// -(1/(2 w_b)) phi_nb for the neighbour's viscous flux, -1/J). With l = -lambda/J per node:
//
//   adj_face    per face point: c = s/w_0 (l_L - l_R) is the cotangent of F*(U_L, U_R, n); its
//               transposed Jacobian goes to both sides' face slots. Roe and LLF: hand-written
//               reverse mode of the forward statements; EC: forward-mode dual numbers (5 seeds per
//               pass, 2 passes) through the same templated code the forward kernel runs.
//   adj_visc    (Navier-Stokes) per element: transpose the viscous divergence (D^T sweeps of l,
//               neighbour term through the face), the contravariant projection and the
//               Navier-Stokes-Fourier flux (pointwise, at the viscous stress the forward lifting
//               recorded for this state), then the lifting (D^T sweeps, central face value):
//               cotangents of (u, v, w, T) per node plus face slots for the neighbour's share.
//   adj_volume  per element: the two-point flux differencing transposed pair by pair. With
//               sums S = x_i + x_m the Kennedy-Gruber / Pirozzoli fluxes are polynomials in
//               (S_rho, S_u, S_p, S_X), so each pair adds the same cotangent vector to both of its
//               nodes' primitive accumulators; then per node the primitive cotangents (plus the
//               viscous ones) are chained to the conservative variables, the face slots are added,
//               and either Ubar is written or the LSERK(5,4) reverse stage is applied in place.
#pragma once
#include "dg_dual.cuh"

namespace {

// ---------------------------------------------------------------------------------------------
// reverse-mode derivatives of the Riemann fluxes (the statements of riemann<double>, transposed)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double sgn_of(double x) { return x < 0.0 ? -1.0 : 1.0; }  // d|x|/dx, +1 at 0

// primitives of one side: ir = 1/rho (given: (1/sqrt(rho))^2, as the forward solver forms it),
// u = m ir, p = (gamma-1)(E - |m|^2 ir / 2)
struct Side {
  double ir, u[3], p, un;
};

__device__ __forceinline__ Side side_of(const double U[5], const double nv[3], double gm1, double ir) {
  Side s;
  s.ir = ir;
  s.u[0] = U[1] * s.ir;
  s.u[1] = U[2] * s.ir;
  s.u[2] = U[3] * s.ir;
  s.p = gm1 * (U[4] - 0.5 * (U[1] * s.u[0] + U[2] * s.u[1] + U[3] * s.u[2]));
  s.un = s.u[0] * nv[0] + s.u[1] * nv[1] + s.u[2] * nv[2];
  return s;
}

// cotangents of (u, p, un, ir) of one side -> cotangent of U (added to g)
__device__ __forceinline__ void side_back(const double U[5], const Side &s, const double nv[3], double gm1,
                                          double cu[3], double cp, double cun, double cir, double g[5]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) cu[k] += cun * nv[k];
  // p = gm1 (E - |m|^2 ir / 2): dp/dE = gm1, dp/dm_k = -gm1 u_k, dp/dir = -gm1 |m|^2 / 2
  g[4] += gm1 * cp;
  const double m2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
  cir -= 0.5 * gm1 * m2 * cp;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    g[1 + k] += cu[k] * s.ir - gm1 * s.u[k] * cp;
    cir += cu[k] * U[1 + k];
  }
  g[0] -= cir * s.ir * s.ir;
}

// Euler flux F = (rho un, m un + p n, (E + p) un) of one side, reversed: adds dF^T cF to the side's
// cotangents (cu, cp, cun) and to g directly
__device__ __forceinline__ void flux_back(const double U[5], const Side &s, const double nv[3], const double cF[5],
                                          double &cp, double &cun, double g[5]) {
  cun += cF[0] * U[0] + cF[1] * U[1] + cF[2] * U[2] + cF[3] * U[3] + cF[4] * (U[4] + s.p);
  cp += cF[1] * nv[0] + cF[2] * nv[1] + cF[3] * nv[2] + cF[4] * s.un;
#pragma unroll
  for (int v = 0; v < 5; ++v) g[v] += cF[v] * s.un;
}

// gL = (dF*/dU_L)^T cF, gR = (dF*/dU_R)^T cF for the LLF flux
__device__ void llf_vjp(const double UL[5], const double UR[5], const double nv[3], double gam, const double cF[5],
                        double gL[5], double gR[5]) {
  const double gm1 = gam - 1.0;
  const double rsL = rsq(UL[0]), rsR = rsq(UR[0]);
  const Side L = side_of(UL, nv, gm1, rsL * rsL), R = side_of(UR, nv, gm1, rsR * rsR);
  const double cL = sqrt(gam * L.p * L.ir), cR = sqrt(gam * R.p * R.ir);
  const double aL = fabs(L.un) + cL, aR = fabs(R.un) + cR;
  const bool rwins = aR > aL;  // the forward's max picks the right argument only when strictly larger
  const double lam = rwins ? aR : aL;
  double clam = 0.0, hF[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    hF[v] = 0.5 * cF[v];
    gL[v] = 0.5 * lam * cF[v];
    gR[v] = -0.5 * lam * cF[v];
    clam -= 0.5 * cF[v] * (UR[v] - UL[v]);
  }
  double cuL[3] = {0, 0, 0}, cuR[3] = {0, 0, 0}, cpL = 0, cpR = 0, cunL = 0, cunR = 0, cirL = 0, cirR = 0;
  flux_back(UL, L, nv, hF, cpL, cunL, gL);
  flux_back(UR, R, nv, hF, cpR, cunR, gR);
  // lam = |un_X| + sqrt(gamma p_X / rho_X) of the winning side X
  if (rwins) {
    cunR += clam * sgn_of(R.un);
    cpR += clam * 0.5 * cR / R.p;
    gR[0] -= clam * 0.5 * cR * R.ir;
  } else {
    cunL += clam * sgn_of(L.un);
    cpL += clam * 0.5 * cL / L.p;
    gL[0] -= clam * 0.5 * cL * L.ir;
  }
  side_back(UL, L, nv, gm1, cuL, cpL, cunL, cirL, gL);
  side_back(UR, R, nv, gm1, cuR, cpR, cunR, cirR, gR);
}

// the same for Roe's flux (no entropy fix), statement by statement in reverse; as in the forward
// solver, one reciprocal square root per side (1/rho = rs^2, sqrt(rho) = rho rs, 1/(2 sqrt(rho)) = rs/2)
// and one for the sound speed (c = c^2 rc, 1/c^2 = rc^2, 1/(2c) = rc/2)
__device__ void roe_vjp(const double UL[5], const double UR[5], const double nv[3], double gam, const double cF[5],
                        double gL[5], double gR[5]) {
  const double gm1 = gam - 1.0;
  const double rsL = rsq(UL[0]), rsR = rsq(UR[0]);
  const Side L = side_of(UL, nv, gm1, rsL * rsL), R = side_of(UR, nv, gm1, rsR * rsR);
  // forward
  const double sL = UL[0] * rsL, sR = UR[0] * rsR;
  const double iw = 1.0 / (sL + sR);
  double ut[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) ut[k] = (sL * L.u[k] + sR * R.u[k]) * iw;
  const double EpL = UL[4] + L.p, EpR = UR[4] + R.p;
  const double hL = EpL * L.ir, hR = EpR * R.ir;
  const double Ht = (sL * hL + sR * hR) * iw;
  const double q2 = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
  const double c2 = gm1 * (Ht - 0.5 * q2);
  const double rc = rsq(c2);
  const double ct = c2 * rc, ic2 = rc * rc;
  const double rt = sL * sR;
  const double unt = ut[0] * nv[0] + ut[1] * nv[1] + ut[2] * nv[2];
  const double dr = UR[0] - UL[0], dp = R.p - L.p;
  const double du[3] = {R.u[0] - L.u[0], R.u[1] - L.u[1], R.u[2] - L.u[2]};
  const double dun = du[0] * nv[0] + du[1] * nv[1] + du[2] * nv[2];
  const double A1 = dp - rt * ct * dun, A5 = dp + rt * ct * dun;
  const double a1 = 0.5 * A1 * ic2, a5 = 0.5 * A5 * ic2, a2 = dr - dp * ic2;
  double dt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) dt[k] = du[k] - dun * nv[k];
  const double s1 = fabs(unt - ct), s5 = fabs(unt + ct), l2 = fabs(unt);
  const double l1a1 = s1 * a1, l5a5 = s5 * a5, l2a2 = l2 * a2, l2r = l2 * rt;
  const double utdt = ut[0] * dt[0] + ut[1] * dt[1] + ut[2] * dt[2];
  // reverse: F = (FL + FR - D) / 2
  double cD[5], hF[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) { hF[v] = 0.5 * cF[v]; cD[v] = -hF[v]; }
  double cnt = cD[1] * nv[0] + cD[2] * nv[1] + cD[3] * nv[2];  // sum_k cD_k n_k
  double cut_dot = cD[1] * ut[0] + cD[2] * ut[1] + cD[3] * ut[2];
  const double c_l1a1 = cD[0] + cut_dot - ct * cnt + cD[4] * (Ht - unt * ct);
  const double c_l5a5 = cD[0] + cut_dot + ct * cnt + cD[4] * (Ht + unt * ct);
  const double c_l2a2 = cD[0] + cut_dot + cD[4] * 0.5 * q2;
  const double c_l2r = cD[1] * dt[0] + cD[2] * dt[1] + cD[3] * dt[2] + cD[4] * utdt;
  const double sum15 = l1a1 + l5a5 + l2a2;
  double c_ut[3], c_dt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c_ut[k] = cD[1 + k] * sum15 + cD[4] * l2r * dt[k];
    c_dt[k] = (cD[1 + k] + cD[4] * ut[k]) * l2r;
  }
  double c_ct = (l5a5 - l1a1) * (cnt + cD[4] * unt);
  double c_unt = cD[4] * ct * (l5a5 - l1a1);
  double c_Ht = cD[4] * (l1a1 + l5a5);
  double c_q2 = cD[4] * 0.5 * l2a2;
  // products with the wave speeds
  const double c_a1 = c_l1a1 * s1, c_a5 = c_l5a5 * s5, c_a2 = c_l2a2 * l2;
  const double c_s1 = c_l1a1 * a1, c_s5 = c_l5a5 * a5;
  const double c_l2 = c_l2a2 * a2 + c_l2r * rt;
  double c_rt = c_l2r * l2;
  const double g1 = sgn_of(unt - ct), g5 = sgn_of(unt + ct), g2 = sgn_of(unt);
  c_unt += g1 * c_s1 + g5 * c_s5 + g2 * c_l2;
  c_ct += -g1 * c_s1 + g5 * c_s5;
  // tangential jump dt = du - dun n
  double c_du[3];
  double c_dun = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) { c_du[k] = c_dt[k]; c_dun -= c_dt[k] * nv[k]; }
  // wave strengths
  double c_dr = c_a2, c_dp = -c_a2 * ic2, c_ic2 = -c_a2 * dp;
  c_dp += 0.5 * (c_a1 + c_a5) * ic2;
  const double cdiff = 0.5 * (c_a5 - c_a1) * ic2;  // cotangent of rt ct dun
  c_rt += cdiff * ct * dun;
  c_ct += cdiff * rt * dun;
  c_dun += cdiff * rt * ct;
  c_ic2 += 0.5 * (c_a1 * A1 + c_a5 * A5);
#pragma unroll
  for (int k = 0; k < 3; ++k) { c_du[k] += c_dun * nv[k]; c_ut[k] += c_unt * nv[k]; }
  // Roe averages
  double c_c2 = -c_ic2 * ic2 * ic2 + c_ct * 0.5 * rc;
  c_Ht += gm1 * c_c2;
  c_q2 -= 0.5 * gm1 * c_c2;
#pragma unroll
  for (int k = 0; k < 3; ++k) c_ut[k] += 2.0 * ut[k] * c_q2;
  // the weights: d ut/d sL = iw (uL - ut), d Ht/d sL = iw (hL - Ht) (the same for R), d ut/d uL = sL iw
  double xL = c_Ht * (hL - Ht), xR = c_Ht * (hR - Ht);
  const double wL = sL * iw, wR = sR * iw;
  const double c_hL = c_Ht * wL, c_hR = c_Ht * wR;
  double cuL[3], cuR[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    xL += c_ut[k] * (L.u[k] - ut[k]);
    xR += c_ut[k] * (R.u[k] - ut[k]);
    cuL[k] = c_ut[k] * wL - c_du[k];
    cuR[k] = c_ut[k] * wR + c_du[k];
  }
  const double c_sL = c_rt * sR + iw * xL, c_sR = c_rt * sL + iw * xR;
  // enthalpies h = (E + p) ir
  double cpL = -c_dp + c_hL * L.ir, cpR = c_dp + c_hR * R.ir;
  double cirL = c_hL * EpL, cirR = c_hR * EpR;
#pragma unroll
  for (int v = 0; v < 5; ++v) { gL[v] = 0.0; gR[v] = 0.0; }
  gL[4] += c_hL * L.ir;
  gR[4] += c_hR * R.ir;
  gL[0] += -c_dr + c_sL * 0.5 * rsL;
  gR[0] += c_dr + c_sR * 0.5 * rsR;
  double cunL = 0.0, cunR = 0.0;
  flux_back(UL, L, nv, hF, cpL, cunL, gL);
  flux_back(UR, R, nv, hF, cpR, cunR, gR);
  side_back(UL, L, nv, gm1, cuL, cpL, cunL, cirL, gL);
  side_back(UR, R, nv, gm1, cuR, cpR, cunR, cirR, gR);
}

// ---------------------------------------------------------------------------------------------
// adjoint of the face kernel
// ---------------------------------------------------------------------------------------------
template <int SF>
__global__ void __launch_bounds__(128) k_adj_face(const DgDevice d, const double *__restrict__ U,
                                                  const double *__restrict__ lam, double *__restrict__ slots) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)d.nF * nn) return;
  const int f = (int)(t / nn), pq = (int)(t % nn), p = pq % n, q = pq / n;
  const int *F5 = d.face + 5 * f;
  const int eL = F5[0], fL = F5[1], eR = F5[2], fR = F5[3], o = F5[4];
  int p2, q2;
  orient_map(o, p, q, p2, q2);
  const int nodeL = face_node(fL, p, q), nodeR = face_node(fR, p2, q2);
  const int pqR = p2 + n * q2;
  const double *nr = d.nrm + (size_t)f * 4 * nn + pq;
  double UL[5], UR[5], cF[5];
  load_state<double>(d, U, eL, nodeL, UL);
  load_state<double>(d, U, eR, nodeR, UR);
  const double iJL = d.invJ[(size_t)eL * nnn + nodeL], iJR = d.invJ[(size_t)eR * nnn + nodeR];
  const double sw = nr[3 * nn] * c_invw[0];  // w_0 = w_N
#pragma unroll
  for (int v = 0; v < 5; ++v)
    cF[v] = sw * (iJR * lam[((size_t)eR * 5 + v) * nnn + nodeR] - iJL * lam[((size_t)eL * 5 + v) * nnn + nodeL]);
  if (SF != SF_EC) {  // hand-written reverse mode
    const double nv[3] = {nr[0], nr[nn], nr[2 * nn]};
    double gL[5], gR[5];
    if (SF == SF_ROE) roe_vjp(UL, UR, nv, d.gamma, cF, gL, gR);
    else llf_vjp(UL, UR, nv, d.gamma, cF, gL, gR);
    double *oL = slots + ((size_t)eL * 6 + fL) * 5 * nn + pq;
    double *oR = slots + ((size_t)eR * 6 + fR) * 5 * nn + pqR;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      oL[k * nn] = gL[k];
      oR[k * nn] = gR[k];
    }
    return;
  }
  // entropy-conservative flux: forward-mode dual numbers through riemann<>
  using D5 = Dual<5>;
  const D5 nv[3] = {D5(nr[0]), D5(nr[nn]), D5(nr[2 * nn])};
  const D5 gam(d.gamma), zero(0.0);
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    D5 A[5], B[5], Fd[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      A[v] = D5(UL[v]);
      B[v] = D5(UR[v]);
      if (side == 0) A[v].d[v] = 1.0;
      else B[v].d[v] = 1.0;
    }
    riemann<D5>(SF, A, B, nv, gam, zero, zero, Fd);
    double *out = slots + ((size_t)(side ? eR : eL) * 6 + (side ? fR : fL)) * 5 * nn + (side ? pqR : pq);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      double gk = 0.0;
#pragma unroll
      for (int v = 0; v < 5; ++v) gk += cF[v] * Fd[v].d[k];
      out[k * nn] = gk;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// adjoint of the lifting + viscous flux + viscous divergence (Navier-Stokes)
// The flux is linear in the lifted gradients except for the work term u.tau, whose derivative
// needs the viscous stress tau at the state: the forward lifting records it per node (the record
// the reverse sweep keeps with each stage state), so no gradient is formed here.
// shared memory per element: W[3][nnn] (u, v, w), L[4][nnn] (l of momentum and energy),
// H[12][nnn] (cotangent of the direction-d reference derivative of w_q), Om[3][nnn]
// ---------------------------------------------------------------------------------------------
constexpr int ADJV_SLOTS = 22;

// the neighbour's volume node facing face point (pp, qq) of element e's face f
__device__ __forceinline__ void neighbour_node(const DgDevice &d, size_t e, int f, int pp, int qq, int &nb, int &fnb,
                                               int &nbnode, int &nbpq) {
  const int *ef = d.ef + (e * 6 + f) * 4;
  nb = ef[0];
  fnb = ef[1];
  int p2, q2;
  orient_map(ef[2], pp, qq, p2, q2);
  nbnode = face_node(fnb, p2, q2);
  nbpq = p2 + n * q2;
}

__global__ void __launch_bounds__(LIFT_THREADS) k_adj_visc(const DgDevice d, const double *__restrict__ U,
                                                           const double *__restrict__ lam,
                                                           const double *__restrict__ tau, double *__restrict__ cotW,
                                                           double *__restrict__ sigma) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  double *Ws = reinterpret_cast<double *>(sm_raw);  // [EPB][3][nnn]
  double *Ls = Ws + LIFT_EPB * 3 * nnn;              // [EPB][4][nnn]
  double *Hs = Ls + LIFT_EPB * 4 * nnn;              // [EPB][12][nnn]
  double *Os = Hs + LIFT_EPB * 12 * nnn;             // [EPB][3][nnn]
  // D in shared memory, rows padded: the sweeps index it by the thread's own node, which would
  // serialise a constant-memory load
  __shared__ double sD[n][n + 1];
  for (int t = threadIdx.x; t < nn; t += blockDim.x) sD[t / n][t % n] = c_D[t];
  const int e0 = blockIdx.x * LIFT_EPB;
  for (int t = threadIdx.x; t < LIFT_EPB * nnn; t += blockDim.x) {
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    const size_t gi = (size_t)e * 5 * nnn + node;
    const double ir = 1.0 / U[gi];  // u as the lifting forms it
    double *W = Ws + le * 3 * nnn + node;
    W[0] = U[gi + nnn] * ir;
    W[nnn] = U[gi + 2 * nnn] * ir;
    W[2 * nnn] = U[gi + 3 * nnn] * ir;
    const double miJ = -d.invJ[(size_t)e * nnn + node];
#pragma unroll
    for (int q = 0; q < 4; ++q) Ls[(le * 4 + q) * nnn + node] = miJ * lam[gi + (1 + q) * nnn];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < LIFT_EPB * nnn; t += blockDim.x) {
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    const int ijk[3] = {node % n, (node / n) % n, node / nn};
    const double *W = Ws + le * 3 * nnn;
    const double *L = Ls + le * 4 * nnn;
    // reverse seed: zeta[dd][q] = cotangent of the contravariant viscous flux Fv^dd_q at this node
    double zeta[3][4];
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      const int id = ijk[dd];
      const int st = dd == 0 ? 1 : dd == 1 ? n : nn;
      const int base = node - id * st;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double z = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m)
          if (m != id) z -= sD[m][id] * L[q * nnn + base + m * st];
        zeta[dd][q] = z;
      }
      if (id == 0 || id == N) {  // the neighbour's viscous divergence reads this node's flux
        const int f = 2 * dd + (id == N ? 1 : 0);
        const int pp = dd == 0 ? ijk[1] : ijk[0], qq = dd == 2 ? ijk[1] : ijk[2];
        int nb, fnb, nbnode, nbpq;
        neighbour_node(d, e, f, pp, qq, nb, fnb, nbnode, nbpq);
        const double sgf = (f & 1) ? 0.5 : -0.5;
        const double kn = c_invw[id] * sgf * -d.invJ[(size_t)nb * nnn + nbnode];  // (1/w_b)(+-1/2) l = -lam/J
#pragma unroll
        for (int q = 0; q < 4; ++q) zeta[dd][q] += kn * lam[((size_t)nb * 5 + 1 + q) * nnn + nbnode];
      }
    }
    double Ja[3][3];
#pragma unroll
    for (int dd = 0; dd < 3; ++dd)
#pragma unroll
      for (int c = 0; c < 3; ++c) Ja[dd][c] = d.Ja[(((size_t)e * 3 + dd) * 3 + c) * nnn + node];
    // the lifting forms tau and the heat flux from J grad w with 1/J in mu and kappa; their
    // transposes carry the same factors, and with them the 1/J of H below
    const double iJ = d.invJ[(size_t)e * nnn + node];
    const double mu = d.mu * iJ, kappa = d.kappa * iJ;
    const double u[3] = {W[node], W[nnn + node], W[2 * nnn + node]};
    const double *tr = tau + (size_t)e * 6 * nnn + node;
    const double txx = tr[0], tyy = tr[nnn], tzz = tr[2 * nnn], txy = tr[3 * nnn], txz = tr[4 * nnn],
                 tyz = tr[5 * nnn];
    const double ta[3][3] = {{txx, txy, txz}, {txy, tyy, tyz}, {txz, tyz, tzz}};
    // Z[c][q]: cotangent of the Cartesian viscous flux F_c,q (F_c,k = tau_kc; F_c,3 = u.tau_c + kappa dT/dx_c)
    double Z[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) Z[c][q] = Ja[0][c] * zeta[0][q] + Ja[1][c] * zeta[1][q] + Ja[2][c] * zeta[2][q];
    double Y[3][3], om[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      om[k] = Z[0][3] * ta[k][0] + Z[1][3] * ta[k][1] + Z[2][3] * ta[k][2];
#pragma unroll
      for (int c = 0; c < 3; ++c) Y[k][c] = Z[c][k] + Z[c][3] * u[k];
    }
    const double trY = Y[0][0] + Y[1][1] + Y[2][2];
    double Gm[4][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) Gm[k][c] = mu * (Y[k][c] + Y[c][k]) - (k == c ? 2.0 / 3.0 * mu * trY : 0.0);
#pragma unroll
    for (int c = 0; c < 3; ++c) Gm[3][c] = kappa * Z[c][3];
    double *H = Hs + le * 12 * nnn + node;
#pragma unroll
    for (int dd = 0; dd < 3; ++dd)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        H[(dd * 4 + q) * nnn] = Ja[dd][0] * Gm[q][0] + Ja[dd][1] * Gm[q][1] + Ja[dd][2] * Gm[q][2];
#pragma unroll
    for (int k = 0; k < 3; ++k) Os[(le * 3 + k) * nnn + node] = om[k];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < LIFT_EPB * nnn; t += blockDim.x) {
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    const int ijk[3] = {node % n, (node / n) % n, node / nn};
    const double *H = Hs + le * 12 * nnn;
    double cw[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      const int id = ijk[dd];
      const int st = dd == 0 ? 1 : dd == 1 ? n : nn;
      const int base = node - id * st;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m) s += sD[m][id] * H[(dd * 4 + q) * nnn + base + m * st];
        cw[q] += s;
      }
      if (id == 0 || id == N) {
        const int f = 2 * dd + (id == N ? 1 : 0);
        const int pq = (dd == 0 ? ijk[1] : ijk[0]) + n * (dd == 2 ? ijk[1] : ijk[2]);
        const double hs = (id == N ? 0.5 : -0.5) * c_invw[id];
        double *sg = sigma + ((size_t)e * 6 + f) * 4 * nn + pq;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const double h = hs * H[(dd * 4 + q) * nnn + node];
          cw[q] -= h;
          sg[q * nn] = h;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) cw[k] += Os[(le * 3 + k) * nnn + node];
#pragma unroll
    for (int q = 0; q < 4; ++q) cotW[((size_t)e * 4 + q) * nnn + node] = cw[q];
  }
}

// ---------------------------------------------------------------------------------------------
// adjoint of the volume kernel
// staged per element: P[6][PS] = (rho, u, v, w, 4p, X) with X = h (Pirozzoli) or e = E/rho (KG),
// Lm[5][PS] = l, and per direction Acc[3][6][PS] = cotangents of (rho, u, v, w, 4p, X)
// ---------------------------------------------------------------------------------------------
constexpr int ADJ_NP = 6;
constexpr int ADJ_SLOTS = ADJ_NP + 5 + 18;
// elements per CTA and CTAs per SM of the adjoint volume kernel: its shared memory (29 staged slots
// per element) is 1.4x the forward's, so at N = 5 one element per CTA lets three CTAs share an SM
// (12 warps) where two elements per CTA fitted only one (7 warps)
__host__ __device__ constexpr int adj_epb() { return N == 1 ? 8 : N == 2 ? 4 : N == 3 ? 2 : N == 4 ? 3 : 1; }
constexpr int ADJ_EPB = adj_epb();
constexpr int ADJ_THREADS = round32(3 * nn * ADJ_EPB);
constexpr int ADJ_MINB = N == 5 ? 3 : N == 6 ? 2 : 1;

// Transposed flux differencing along one line. The forward pair term (scaled by the folded
// 1/2 factors) is c.F with F0 = S_rho V, F_k = F0 S_u,k + S_p S_j,k, F4 = F0 S_X (+ S_p V / 2 for KG),
// V = S_u . S_j and c_v = D'_im l_i,v + D'_mi l_m,v (D' = D/4 for mass, D/8 otherwise).
// one node's staged values for the transposed pair terms
struct AdjNode {
  double r, u, v, w, p, x, l[5], jx, jy, jz;
};

__device__ __forceinline__ AdjNode adj_node(const double *__restrict__ P, const double *__restrict__ Lm, int a,
                                            const double *__restrict__ Jd, int g) {
  AdjNode q;
  q.r = P[a]; q.u = P[PS + a]; q.v = P[2 * PS + a]; q.w = P[3 * PS + a]; q.p = P[4 * PS + a]; q.x = P[5 * PS + a];
#pragma unroll
  for (int k = 0; k < 5; ++k) q.l[k] = Lm[k * PS + a];
  q.jx = __ldg(Jd + g); q.jy = __ldg(Jd + nnn + g); q.jz = __ldg(Jd + 2 * nnn + g);
  return q;
}

// the six primitive cotangents of the pair (i, m), shared by both nodes. The pair cotangents
// c_v = D'_im l_i,v + D'_mi l_m,v are D'_im t_v with t_v = l_i,v + (D_mi/D_im) l_m,v (the mass part's
// factor 2, D/4 against D/8, is in the staged l_0); D'_im = D_im/8 then scales phi, the pressure
// cotangent and F0 once instead of every c_v.
template <int VF>
__device__ __forceinline__ void adj_pair(const AdjNode &a, const AdjNode &b, double de, double dr, double g[6]) {
  const double Sr = a.r + b.r, Su = a.u + b.u, Sv = a.v + b.v, Sw = a.w + b.w;
  const double Sp = a.p + b.p, Sx = a.x + b.x;
  const double Sjx = a.jx + b.jx, Sjy = a.jy + b.jy, Sjz = a.jz + b.jz;
  const double t0 = a.l[0] + dr * b.l[0];
  const double t1 = a.l[1] + dr * b.l[1];
  const double t2 = a.l[2] + dr * b.l[2];
  const double t3 = a.l[3] + dr * b.l[3];
  const double t4 = a.l[4] + dr * b.l[4];
  const double Vp = Su * Sjx + Sv * Sjy + Sw * Sjz;
  const double F0 = de * (Sr * Vp);                                   // D'_im F0
  const double phi = de * (t0 + t1 * Su + t2 * Sv + t3 * Sw + t4 * Sx);  // d(c.F)/dF0
  double gV = phi * Sr, gP = de * (t1 * Sjx + t2 * Sjy + t3 * Sjz);
  if (VF == VF_KG) {
    const double c4 = de * t4;
    gV += 0.5 * c4 * Sp;
    gP += 0.5 * c4 * Vp;
  }
  g[0] = phi * Vp;
  g[1] = t1 * F0 + gV * Sjx;
  g[2] = t2 * F0 + gV * Sjy;
  g[3] = t3 * F0 + gV * Sjz;
  g[4] = gP;
  g[5] = t4 * F0;
}

// Transposed flux differencing along one line, two rows at a time (as the forward line_fluxdiff2):
// the cotangent sums of nodes i and i+1 stay in registers while partner m runs over i+2..N, so each
// partner's staged values and partial sums are read (and written back) once for two pairs.
template <int VF>
__device__ __forceinline__ void adj_line(const double *__restrict__ P, const double *__restrict__ Lm, int pb, int ps,
                                         const double *__restrict__ Jd, int gb, int gs, double *__restrict__ Ac) {
#pragma unroll 1
  for (int i = 0; i < n - 1; i += 2) {
    const int a0 = pb + i * ps, a1 = a0 + ps;
    const AdjNode n0 = adj_node(P, Lm, a0, Jd, gb + i * gs), n1 = adj_node(P, Lm, a1, Jd, gb + (i + 1) * gs);
    double ac0[6], ac1[6];
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      ac0[v] = (i == 0) ? 0.0 : Ac[v * PS + a0];
      ac1[v] = (i == 0) ? 0.0 : Ac[v * PS + a1];
    }
    {
      double g[6];
      adj_pair<VF>(n0, n1, c_De[i * n + i + 1], c_Dr[i * n + i + 1], g);
#pragma unroll
      for (int v = 0; v < 6; ++v) { ac0[v] += g[v]; ac1[v] += g[v]; }
    }
#pragma unroll
    for (int m = i + 2; m < n; ++m) {
      const int am = pb + m * ps;
      const AdjNode nm = adj_node(P, Lm, am, Jd, gb + m * gs);
      double g0[6], g1[6];
      adj_pair<VF>(n0, nm, c_De[i * n + m], c_Dr[i * n + m], g0);
      adj_pair<VF>(n1, nm, c_De[(i + 1) * n + m], c_Dr[(i + 1) * n + m], g1);
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        ac0[v] += g0[v];
        ac1[v] += g1[v];
        const double gm = g0[v] + g1[v];
        if (i == 0) Ac[v * PS + am] = gm;
        else Ac[v * PS + am] += gm;
      }
    }
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      Ac[v * PS + a0] = ac0[v];
      Ac[v * PS + a1] = ac1[v];
    }
  }
}

template <int VF>
__global__ void __launch_bounds__(ADJ_THREADS, ADJ_MINB) k_adj_volume(const DgDevice d, const double *__restrict__ U,
                                                              const double *lam, const double *__restrict__ fslots,
                                                              const double *__restrict__ cotW,
                                                              const double *__restrict__ sigma, double *out,
                                                              double *gbar, int mode, double dt, double A, double B,
                                                              int update_g) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  double *P = reinterpret_cast<double *>(sm_raw);  // [EPB][6][PS]
  double *Lm = P + ADJ_EPB * ADJ_NP * PS;          // [EPB][5][PS]
  double *Acc = Lm + ADJ_EPB * 5 * PS;             // [EPB][3][6][PS]
  const int e0 = blockIdx.x * ADJ_EPB;
  const double gam = d.gamma, gm1 = gam - 1.0;
  // the thread's nodes (the same in staging and in the per-node part): their 1/rho stays in registers
  constexpr int RN = (ADJ_EPB * nnn + ADJ_THREADS - 1) / ADJ_THREADS;
  double irr[RN];
#pragma unroll
  for (int rr = 0; rr < RN; ++rr) {
    const int t = threadIdx.x + rr * ADJ_THREADS;
    if (t >= ADJ_EPB * nnn) continue;
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    double Uv[5];
    load_state<double>(d, U, e, node, Uv);
    const double r = Uv[0], ir = 1.0 / r;
    irr[rr] = ir;
    const double u = Uv[1] * ir, v = Uv[2] * ir, w = Uv[3] * ir;
    const double p = gm1 * (Uv[4] - 0.5 * (Uv[1] * u + Uv[2] * v + Uv[3] * w));
    if (!(r > 0.0) || !(p > 0.0) || !isfinite(Uv[4])) flag_set(d.flag, 1);
    const int pn = pidx(node);
    double *Pe = P + le * ADJ_NP * PS + pn;
    Pe[0] = r; Pe[PS] = u; Pe[2 * PS] = v; Pe[3 * PS] = w; Pe[4 * PS] = 4.0 * p;
    Pe[5 * PS] = VF == VF_PIR ? (Uv[4] + p) * ir : Uv[4] * ir;
    const double miJ = -d.invJ[(size_t)e * nnn + node];
    // l = -lambda/J; the mass component doubled (its split-form factor is D/4, the others' D/8)
#pragma unroll
    for (int k = 0; k < 5; ++k)
      Lm[(le * 5 + k) * PS + pn] = (k == 0 ? 2.0 * miJ : miJ) * lam[((size_t)e * 5 + k) * nnn + node];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ADJ_EPB * 3 * nn; t += blockDim.x) {
    const int le = t / (3 * nn), r = t % (3 * nn), dir = r / nn, line = r % nn, e = e0 + le;
    if (e >= d.nE) continue;
    int pb, ps, gb, gs, a, b;
    line_geom(dir, line, pb, ps, gb, gs, a, b);
    adj_line<VF>(P + le * ADJ_NP * PS, Lm + le * 5 * PS, pb, ps, d.Ja + ((size_t)e * 3 + dir) * 3 * nnn, gb, gs,
                 Acc + (le * 3 + dir) * ADJ_NP * PS);
  }
  __syncthreads();
  const bool ns = d.equations == 1;
  const double iR = 1.0 / d.R;
#pragma unroll
  for (int rr = 0; rr < RN; ++rr) {
    const int t = threadIdx.x + rr * ADJ_THREADS;
    if (t >= ADJ_EPB * nnn) continue;
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    const int ijk[3] = {node % n, (node / n) % n, node / nn};
    const int pn = pidx(node);
    const double *Pe = P + le * ADJ_NP * PS + pn;
    const double u[3] = {Pe[PS], Pe[2 * PS], Pe[3 * PS]}, p = 0.25 * Pe[4 * PS], X = Pe[5 * PS];
    double gp[6];
#pragma unroll
    for (int v = 0; v < 6; ++v)
      gp[v] = Acc[(le * 3 + 0) * ADJ_NP * PS + v * PS + pn] + Acc[(le * 3 + 1) * ADJ_NP * PS + v * PS + pn] +
              Acc[(le * 3 + 2) * ADJ_NP * PS + v * PS + pn];
    const double ir = irr[rr];
    double g_r = gp[0], g_u[3] = {gp[1], gp[2], gp[3]}, g_p = 4.0 * gp[4];
    const double g_x = gp[5];
    if (ns) {  // cotangents of (u, v, w, T) from the viscous adjoint, own part + the neighbours' face shares
      double cw[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) cw[q] = cotW[((size_t)e * 4 + q) * nnn + node];
#pragma unroll
      for (int dd = 0; dd < 3; ++dd) {
        const int id = ijk[dd];
        if (id != 0 && id != N) continue;
        const int f = 2 * dd + (id == N ? 1 : 0);
        const int pp = dd == 0 ? ijk[1] : ijk[0], qq = dd == 2 ? ijk[1] : ijk[2];
        int nb, fnb, nbnode, nbpq;
        neighbour_node(d, e, f, pp, qq, nb, fnb, nbnode, nbpq);
        const double *sg = sigma + ((size_t)nb * 6 + fnb) * 4 * nn + nbpq;
#pragma unroll
        for (int q = 0; q < 4; ++q) cw[q] += sg[q * nn];
      }
      g_u[0] += cw[0];
      g_u[1] += cw[1];
      g_u[2] += cw[2];
      g_p += cw[3] * ir * iR;         // T = p / (rho R)
      g_r -= cw[3] * p * ir * ir * iR;
    }
    // chain to U = (rho, m, E): u = m / rho, p = (gamma-1)(E - |m|^2 / (2 rho)), X = h = (E + p)/rho
    // (Pirozzoli) or e = E/rho (KG). With gx = g_X/rho, p reaches U with weight a = (gamma-1) g_p, and
    // for h also through E + p: a = (gamma-1)(g_p + gx), and dh/dE = gamma/rho = (gamma-1)/rho + 1/rho
    const double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double gx = g_x * ir;
    const double a = VF == VF_PIR ? gm1 * (g_p + gx) : gm1 * g_p;
    double gU[5];
    gU[0] = g_r - ir * (g_u[0] * u[0] + g_u[1] * u[1] + g_u[2] * u[2]) + (0.5 * a) * q2 - gx * X;
#pragma unroll
    for (int k = 0; k < 3; ++k) gU[1 + k] = ir * g_u[k] - a * u[k];
    gU[4] = a + gx;
    // advective surface terms: transposed Riemann-flux Jacobians in this element's face slots
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      const int id = ijk[dd];
      if (id != 0 && id != N) continue;
      const int f = 2 * dd + (id == N ? 1 : 0);
      const int pq = (dd == 0 ? ijk[1] : ijk[0]) + n * (dd == 2 ? ijk[1] : ijk[2]);
      const double *fs = fslots + ((size_t)e * 6 + f) * 5 * nn + pq;
#pragma unroll
      for (int v = 0; v < 5; ++v) gU[v] += fs[v * nn];
    }
    const size_t gi = (size_t)e * 5 * nnn + node;
    if (mode == 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) out[gi + v * nnn] = gU[v];
    } else {  // reverse LSERK stage: Ubar += dt * VJP; gbar = A gbar + B Ubar (gbar is lam, read above)
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double ub = out[gi + v * nnn] + dt * gU[v];
        out[gi + v * nnn] = ub;
        if (update_g) gbar[gi + v * nnn] = A * gbar[gi + v * nnn] + B * ub;
      }
    }
  }
}

// gradient of the kinetic-energy integral sum_e sum_ijk w_i w_j w_k J rho |u|^2 / 2
__global__ void __launch_bounds__(256) k_ke_grad(const DgDevice d, const double *__restrict__ U,
                                                 double *__restrict__ grad) {
  const long long total = (long long)d.nE * nnn;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const size_t e = (size_t)(t / nnn);
    const int node = (int)(t % nnn);
    const double wq = c_w[node % n] * c_w[(node / n) % n] * c_w[node / nn] * d.J[t];
    const double *Ue = U + e * 5 * nnn + node;
    const double ir = 1.0 / Ue[0];
    const double u = Ue[nnn] * ir, v = Ue[2 * nnn] * ir, w = Ue[3 * nnn] * ir;
    double *G = grad + e * 5 * nnn + node;
    G[0] = -0.5 * wq * (u * u + v * v + w * w);
    G[nnn] = wq * u;
    G[2 * nnn] = wq * v;
    G[3 * nnn] = wq * w;
    G[4 * nnn] = 0.0;
  }
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
void launch_adj_face(const DgDevice &d, const double *U, const double *lam, double *slots, cudaStream_t s) {
  const long long pts = (long long)d.nF * nn;
  const unsigned grid = (unsigned)((pts + 127) / 128);
  switch (d.sflux) {
    case SF_LLF: k_adj_face<SF_LLF><<<grid, 128, 0, s>>>(d, U, lam, slots); break;
    case SF_ROE: k_adj_face<SF_ROE><<<grid, 128, 0, s>>>(d, U, lam, slots); break;
    default: k_adj_face<SF_EC><<<grid, 128, 0, s>>>(d, U, lam, slots); break;
  }
}

void launch_adj_visc(const DgDevice &d, const double *U, const double *lam, const double *tau, double *cotW,
                     double *sigma, cudaStream_t s) {
  const size_t smem = sizeof(double) * LIFT_EPB * ADJV_SLOTS * nnn;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_adj_visc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  k_adj_visc<<<(d.nE + LIFT_EPB - 1) / LIFT_EPB, LIFT_THREADS, smem, s>>>(d, U, lam, tau, cotW, sigma);
}

template <int VF>
void launch_adj_volume_t(const DgDevice &d, const double *U, const double *lam, const double *fslots,
                         const double *cotW, const double *sigma, double *out, double *gbar, int mode, double dt,
                         double A, double B, int update_g, cudaStream_t s) {
  const size_t smem = sizeof(double) * ADJ_EPB * ADJ_SLOTS * PS;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_adj_volume<VF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  k_adj_volume<VF><<<(d.nE + ADJ_EPB - 1) / ADJ_EPB, ADJ_THREADS, smem, s>>>(d, U, lam, fslots, cotW, sigma, out,
                                                                            gbar, mode, dt, A, B, update_g);
}

void launch_adj_volume(const DgDevice &d, const double *U, const double *lam, const double *fslots,
                       const double *cotW, const double *sigma, double *out, double *gbar, int mode, double dt,
                       double A, double B, int update_g, cudaStream_t s) {
  if (d.vflux == VF_KG)
    launch_adj_volume_t<VF_KG>(d, U, lam, fslots, cotW, sigma, out, gbar, mode, dt, A, B, update_g, s);
  else
    launch_adj_volume_t<VF_PIR>(d, U, lam, fslots, cotW, sigma, out, gbar, mode, dt, A, B, update_g, s);
}

void launch_ke_grad(const DgDevice &d, const double *U, double *grad, cudaStream_t s) {
  k_ke_grad<<<8 * 152, 256, 0, s>>>(d, U, grad);
}

}  // namespace
