// dg_kernels.cuh -- sm_103a kernels of the split-form DGSEM right-hand side for ONE polynomial
// degree. Included by dg_kernels_nN.cu with DG_N defined; everything lives in an anonymous
// namespace so each translation unit has its own constant-memory tables.
//
// Per RK stage (Sec. 2; Sec. 4.1):
//   [indicator -> spread]   modified Persson indicator on rho*p (Sec. 4.1, Eq. (7)), alpha per element
//   face                    Riemann flux s F*(U_L, U_R, n) once per face point (Roe / LLF / EC),
//                           BR1 face jumps w* - w for the lifting (Navier-Stokes)
//   [lift]                  BR1 gradients of (u, v, w, T) and the contravariant viscous flux
//   volume                  split-form flux differencing along the three line families, viscous
//                           divergence, surface terms, FV subcell operator + blend (Sec. 4.1,
//                           Eq. (6)), Jacobian, and the fused LSERK(5,4) stage update
//
// Algebra used by the volume kernel (exact identities of the LGL/SBP operator): with
// D_00 = -1/(2 w_0), D_NN = 1/(2 w_N) and zero interior diagonal, the diagonal volume term
// 2 D_ii F(U_i) cancels the -F(U_i)/w_b part of the strong-form surface term, so the kernel
// sums off-diagonal pairs only and adds (1/w_b) F*_out at boundary nodes; for the viscous
// (BR1 central) flux the same cancellation leaves -(1/(2 w_b)) phi_nb, the neighbour's outward
// normal viscous flux. Pair symmetry F#(U_i,U_m) = F#(U_m,U_i) halves the two-point fluxes.
//
// Arithmetic type R: double for the FP64 path; float for the FP32-bulk path, where the flux,
// lifting and accumulation arithmetic is FP32 while U is read as FP64, metrics and Jacobian are
// computed in FP64 (the kernels read an FP32 rounding of Ja), and the LSERK register and state
// accumulate in FP64 (the FP32 kernels of dg_fp32.cuh form the stage increment as an FP32 product). In FP32 the state is carried with E' = E - p_ref/(gamma-1) so that the
// pressure p' = p - p_ref is formed from O(1) numbers; the momentum flux uses p' throughout
// (volume, surface and subcell fluxes). The constant p_ref part of that flux contributes
// p_ref times the discrete metric identity sum_d D_d Ja^d, which is zero, so the shift is exact.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "dg_convert.cuh"
#include "dg_internal.h"
#include "dg_invariants_node.cuh"
#include "dg_wall.cuh"

#ifndef DG_N
#error "define DG_N before including dg_kernels.cuh"
#endif

namespace {

constexpr int N = DG_N;
constexpr int n = N + 1;
constexpr int nn = n * n;
constexpr int nnn = nn * n;
constexpr int PS = n * (n + 1) * n;  // padded stride of one staged node quantity

__constant__ double c_D[nn];      // D_im
__constant__ double c_D2[nn];     // 2 D_im, zero diagonal
__constant__ double c_Dq[nn];     // D_im / 4 (scaled mass flux), zero diagonal
__constant__ double c_De[nn];     // D_im / 8 (scaled momentum / energy flux), zero diagonal
__constant__ double c_Dr[nn];     // D_mi / D_im (i != m; the LGL D has no zero off the diagonal), zero diagonal
__constant__ double c_w[n], c_invw[n], c_xi[n], c_xh[n + 1];
__constant__ double c_ihx[n];  // 1 / (xi_i - xi_{i-1}), i = 1..N (minmod slopes)
// even-odd halves of the zero-diagonal D (n even, h = n/2): the LGL D is centro-antisymmetric,
// D_{N-i,N-m} = -D_im, so y = D' f splits into VP (f_m + f_{N-m}) and VM (f_m - f_{N-m}), m < h:
// VP_im = (D'_im + D'_{i,N-m}) / 2, VM_im = (D'_im - D'_{i,N-m}) / 2, y_i = A_i + B_i, y_{N-i} = B_i - A_i
constexpr int EO_H = (n % 2 == 0) ? n / 2 : 1;
__constant__ double c_VP[EO_H * EO_H], c_VM[EO_H * EO_H];
__constant__ float f_VP[EO_H * EO_H], f_VM[EO_H * EO_H];
// the same halves of the full D (diagonal included; D_NN = -D_00 keeps the symmetry), for the lifting
__constant__ double c_FP[EO_H * EO_H], c_FM[EO_H * EO_H];
__constant__ double c_Vinv[nn];
__constant__ float f_D[nn], f_D2[nn], f_Dq[nn], f_De[nn];
__constant__ float f_w[n], f_invw[n], f_xi[n], f_xh[n + 1], f_ihx[n];

// basis tables in the arithmetic type
template <typename R> struct Tab;
template <> struct Tab<double> {
  static __device__ __forceinline__ double D(int k) { return c_D[k]; }
  static __device__ __forceinline__ double D2(int k) { return c_D2[k]; }
  static __device__ __forceinline__ double Dq(int k) { return c_Dq[k]; }
  static __device__ __forceinline__ double De(int k) { return c_De[k]; }
  static __device__ __forceinline__ double w(int k) { return c_w[k]; }
  static __device__ __forceinline__ double invw(int k) { return c_invw[k]; }
  static __device__ __forceinline__ double xi(int k) { return c_xi[k]; }
  static __device__ __forceinline__ double xh(int k) { return c_xh[k]; }
  static __device__ __forceinline__ double ihx(int k) { return c_ihx[k]; }
  static __device__ __forceinline__ double VP(int k) { return c_VP[k]; }
  static __device__ __forceinline__ double VM(int k) { return c_VM[k]; }
};
template <> struct Tab<float> {
  static __device__ __forceinline__ float D(int k) { return f_D[k]; }
  static __device__ __forceinline__ float D2(int k) { return f_D2[k]; }
  static __device__ __forceinline__ float Dq(int k) { return f_Dq[k]; }
  static __device__ __forceinline__ float De(int k) { return f_De[k]; }
  static __device__ __forceinline__ float w(int k) { return f_w[k]; }
  static __device__ __forceinline__ float invw(int k) { return f_invw[k]; }
  static __device__ __forceinline__ float xi(int k) { return f_xi[k]; }
  static __device__ __forceinline__ float xh(int k) { return f_xh[k]; }
  static __device__ __forceinline__ float ihx(int k) { return f_ihx[k]; }
  static __device__ __forceinline__ float VP(int k) { return f_VP[k]; }
  static __device__ __forceinline__ float VM(int k) { return f_VM[k]; }
};

// per-context constants in the arithmetic type (precomputed on the host)
template <typename R> struct Cst;
template <> struct Cst<double> {
  static __device__ __forceinline__ double gam(const DgDevice &d) { return d.gamma; }
  static __device__ __forceinline__ double gm1(const DgDevice &d) { return d.gm1; }
  static __device__ __forceinline__ double igm1(const DgDevice &d) { return d.igm1; }
  static __device__ __forceinline__ double iR(const DgDevice &d) { return d.iR; }
  static __device__ __forceinline__ double pref(const DgDevice &d) { return d.p_ref; }
  static __device__ __forceinline__ double href(const DgDevice &d) { return d.href; }
  static __device__ __forceinline__ double mu(const DgDevice &d) { return d.mu; }
  static __device__ __forceinline__ double kappa(const DgDevice &d) { return d.kappa; }
};
template <> struct Cst<float> {
  static __device__ __forceinline__ float gam(const DgDevice &d) { return d.gamma_f; }
  static __device__ __forceinline__ float gm1(const DgDevice &d) { return d.gm1_f; }
  static __device__ __forceinline__ float igm1(const DgDevice &d) { return d.igm1_f; }
  static __device__ __forceinline__ float iR(const DgDevice &d) { return d.iR_f; }
  static __device__ __forceinline__ float pref(const DgDevice &d) { return d.p_ref_f; }
  static __device__ __forceinline__ float href(const DgDevice &d) { return d.href_f; }
  static __device__ __forceinline__ float mu(const DgDevice &d) { return d.mu_f; }
  static __device__ __forceinline__ float kappa(const DgDevice &d) { return d.kappa_f; }
};

// per-stage buffers and metric copies in the arithmetic type
template <typename R> struct Buf;
template <> struct Buf<double> {
  static __device__ __forceinline__ double *Fsurf(const DgDevice &d) { return d.Fsurf; }
  static __device__ __forceinline__ double *Wsurf(const DgDevice &d) { return d.Wsurf; }
  static __device__ __forceinline__ double *Fv(const DgDevice &d) { return d.Fv; }
  static __device__ __forceinline__ double *Fwall(const DgDevice &d) { return d.Fwall; }
  static __device__ __forceinline__ const double *Ja(const DgDevice &d) { return d.Ja; }
  static __device__ __forceinline__ const double *nrm(const DgDevice &d) { return d.nrm; }
};
template <> struct Buf<float> {
  static __device__ __forceinline__ float *Fsurf(const DgDevice &d) { return d.Fsurf_f; }
  static __device__ __forceinline__ float *Wsurf(const DgDevice &d) { return d.Wsurf_f; }
  static __device__ __forceinline__ float *Fv(const DgDevice &d) { return d.Fv_f; }
  static __device__ __forceinline__ float *Fwall(const DgDevice &d) { return d.Fwall_f; }
  static __device__ __forceinline__ const float *Ja(const DgDevice &d) { return d.Jaf; }
  static __device__ __forceinline__ const float *nrm(const DgDevice &d) { return d.nrm_f; }
};

// whether the state is carried shifted by the reference pressure (FP32 only)
template <typename R> constexpr bool kShift = std::is_same<R, float>::value;

enum { VF_KG = 0, VF_PIR = 1, VF_EC = 2, VF_CEN = 3 };
enum { SF_LLF = 0, SF_ROE = 1, SF_EC = 2 };

__host__ __device__ constexpr int round32(int x) { return (x + 31) / 32 * 32; }
// elements per CTA of the volume kernel: make 3 n^2 line threads x EPB fill whole warps
__host__ __device__ constexpr int vol_epb() {
  return N == 1 ? 8 : N == 2 ? 4 : N == 3 ? 2 : N == 4 ? 3 : N == 5 ? 2 : 1;
}
constexpr int VOL_EPB = vol_epb();
constexpr int VOL_THREADS = round32(3 * nn * VOL_EPB);
template <typename R, bool SC> __host__ __device__ constexpr int vol_threads() { return VOL_THREADS; }
// minimum resident CTAs per SM the register budget must allow (FP32 uses half the shared memory)
template <typename R, bool SC> __host__ __device__ constexpr int vol_min_blocks() {
  return std::is_same<R, float>::value && !SC ? 3 : 2;
}
// staged quantities per node: rho, u, v, w, 4 p_m, X, Y (+ p' for the FV operator)
template <bool SC> __host__ __device__ constexpr int vol_np() { return SC ? 8 : 7; }
// lifting kernel: whole elements per CTA, a thread per node (looped above 256 threads)
__host__ __device__ constexpr int lift_epb() { return nnn >= 128 ? 1 : (128 + nnn - 1) / nnn; }
constexpr int LIFT_EPB = lift_epb();
constexpr int LIFT_THREADS = round32(LIFT_EPB * nnn) > 256 ? 256 : round32(LIFT_EPB * nnn);

__device__ __forceinline__ int pidx(int node) {  // padded staging index of node (i,j,k)
  const int i = node % n, j = (node / n) % n, k = node / nn;
  return i + (n + 1) * (j + n * k);
}

__device__ __forceinline__ int face_node(int f, int p, int q) {
  const int b = (f & 1) ? N : 0;
  switch (f >> 1) {
    case 0: return b + n * (p + n * q);
    case 1: return p + n * (b + n * q);
    default: return p + n * (q + n * b);
  }
}

// the wall-model exchange node: `k` nodes from face f along the element's line through face point (p, q)
__device__ __forceinline__ int exchange_node(int f, int p, int q, int k) {
  const int b = (f & 1) ? N - k : k;
  switch (f >> 1) {
    case 0: return b + n * (p + n * q);
    case 1: return p + n * (b + n * q);
    default: return p + n * (q + n * b);
  }
}

__device__ __forceinline__ void orient_map(int o, int p, int q, int &p2, int &q2) {
  int a = p, b = q;
  if (o & 4) { a = q; b = p; }
  if (o & 1) a = N - a;
  if (o & 2) b = N - b;
  p2 = a;
  q2 = b;
}

__device__ __forceinline__ void flag_set(int *flag, int bit) { atomicOr(flag, bit); }

__device__ __forceinline__ double to_double(float f) { return (double)f; }
__device__ __forceinline__ double to_double(double x) { return x; }

// five conservative values of node `node` of element e, in the arithmetic type: the FP64 state,
// or in FP32 its shadow copy (E' = E - p_ref/(gamma-1) already applied, rounded once)
template <typename R>
__device__ __forceinline__ void load_state(const DgDevice &d, const double *__restrict__ U, size_t e, int node,
                                           R out[5]) {
  if (kShift<R>) {
    const float *Ue = d.Uf + e * 5 * nnn + node;
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v] = (R)Ue[v * nnn];
  } else {
    const double *Ue = U + e * 5 * nnn + node;
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v] = (R)Ue[v * nnn];
  }
}

// FP32 shadow of the state: Uf = float(U), with E' = E - p_ref/(gamma-1) formed in FP64 first
__global__ void __launch_bounds__(256) k_shadow(const DgDevice d, const double *__restrict__ U) {
  const long long total = (long long)d.nE * 5 * nnn;
  const double eref = d.eref;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int v = (int)((t / nnn) % 5);
    d.Uf[t] = (float)(v == 4 ? U[t] - eref : U[t]);
  }
}

// ---------------------------------------------------------------------------------------------
// pointwise physics (pressure p' = p - p_ref enters the momentum flux; p_ref = 0 in FP64)
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }

// Euler flux through the (unit or metric) vector a, given ir = 1/rho; returns u.a and the true
// pressure p
template <typename R>
__device__ __forceinline__ void euler_flux_ir(const R U[5], R ir, R gam, R pref, R href, const R a[3], R F[5], R &un,
                                              R &p) {
  const R u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
  const R pm = (gam - R(1)) * (U[4] - R(0.5) * (U[1] * u + U[2] * v + U[3] * w));  // p'
  un = u * a[0] + v * a[1] + w * a[2];
  F[0] = U[0] * un;
  F[1] = U[1] * un + pm * a[0];
  F[2] = U[2] * un + pm * a[1];
  F[3] = U[3] * un + pm * a[2];
  if (kShift<R>) {
    p = pm + pref;
    F[4] = (U[4] + pm + href) * un;  // E + p = E' + p' + gamma p_ref/(gamma-1)
  } else {
    p = pm;
    F[4] = (U[4] + pm) * un;
  }
}

template <typename R>
__device__ __forceinline__ R logmean(R a, R b) {
  // (a - b) / ln(a/b); Ismail-Roe series where the ratio is close to 1
  const R z = a / b;
  const R f = (z - R(1)) / (z + R(1));
  const R u = f * f;
  const R cut = kShift<R> ? R(1e-2) : R(1e-4);
  if (u < cut) return (a + b) / (R(2) * (R(1) + u * (R(1.0 / 3.0) + u * (R(0.2) + u * R(1.0 / 7.0)))));
  return (a - b) / log(z);
}

// Chandrashekar's entropy-conservative two-point flux through the vector a (true pressures)
template <typename R>
__device__ __forceinline__ void ec_flux(R rL, R uL, R vL, R wL, R pL, R rR, R uR, R vR, R wR, R pR, const R a[3], R gam,
                                        R pref, R F[5]) {
  const R bL = R(0.5) * rL / pL, bR = R(0.5) * rR / pR;
  const R rln = logmean(rL, rR), bln = logmean(bL, bR);
  const R um = R(0.5) * (uL + uR), vm = R(0.5) * (vL + vR), wm = R(0.5) * (wL + wR);
  const R phat = R(0.5) * (rL + rR) / (bL + bR) - pref;
  const R q2 = R(0.5) * (uL * uL + vL * vL + wL * wL + uR * uR + vR * vR + wR * wR);
  const R V = um * a[0] + vm * a[1] + wm * a[2];
  F[0] = rln * V;
  F[1] = F[0] * um + phat * a[0];
  F[2] = F[0] * vm + phat * a[1];
  F[3] = F[0] * wm + phat * a[2];
  // energy: uses the true p-hat
  F[4] = F[0] * (R(0.5) / ((gam - R(1)) * bln) - R(0.5) * q2) + um * F[1] + vm * F[2] + wm * F[3] +
         pref * (um * a[0] + vm * a[1] + wm * a[2]);
}

// Riemann flux F*(UL, UR, nv) for a unit normal nv; also returns each side's 1/rho and true pressure
// (the face kernel's BR1 face values reuse them)
template <typename R>
__device__ __forceinline__ void riemann(int sf, const R UL[5], const R UR[5], const R nv[3], R gam, R pref, R href,
                                        R F[5], R &irL, R &irR, R &pL, R &pR) {
  const R gm1 = gam - R(1);
  // one reciprocal square root per side: 1/sqrt(rho); 1/rho is its square and sqrt(rho) = rho/sqrt(rho)
  const R rsL = rsq(UL[0]), rsR = rsq(UR[0]);
  irL = rsL * rsL;
  irR = rsR * rsR;
  if (sf == SF_EC) {
    const R uL = UL[1] * irL, vL = UL[2] * irL, wL = UL[3] * irL;
    const R uR = UR[1] * irR, vR = UR[2] * irR, wR = UR[3] * irR;
    pL = gm1 * (UL[4] - R(0.5) * (UL[1] * uL + UL[2] * vL + UL[3] * wL)) + (kShift<R> ? pref : R(0));
    pR = gm1 * (UR[4] - R(0.5) * (UR[1] * uR + UR[2] * vR + UR[3] * wR)) + (kShift<R> ? pref : R(0));
    ec_flux<R>(UL[0], uL, vL, wL, pL, UR[0], uR, vR, wR, pR, nv, gam, kShift<R> ? pref : R(0), F);
    return;
  }
  R FL[5], FR[5], unL, unR;
  euler_flux_ir<R>(UL, irL, gam, pref, href, nv, FL, unL, pL);
  euler_flux_ir<R>(UR, irR, gam, pref, href, nv, FR, unR, pR);
  if (sf == SF_LLF) {
    const R cL = sqrt(gam * pL * irL), cR = sqrt(gam * pR * irR);
    const R lam = fmax(fabs(unL) + cL, fabs(unR) + cR);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = R(0.5) * (FL[v] + FR[v] - lam * (UR[v] - UL[v]));
    return;
  }
  // Roe: sqrt(rho)-weighted average state, three wave families, no entropy fix. With
  // s = sqrt(rho), the weight of side k is s_k / (s_L + s_R), so the averages of u and H are
  // sum_k (m_k / s_k) / (s_L + s_R) = sum_k a_k m_k with a_k = (1/sqrt(rho_k)) / (s_L + s_R).
  const R sL = UL[0] * rsL, sR = UR[0] * rsR;
  const R iw = R(1) / (sL + sR);
  const R aL = rsL * iw, aR = rsR * iw;
  const R uL = UL[1] * irL, vL = UL[2] * irL, wL = UL[3] * irL;
  const R uR = UR[1] * irR, vR = UR[2] * irR, wR = UR[3] * irR;
  const R ut = aL * UL[1] + aR * UR[1], vt = aL * UL[2] + aR * UR[2], wt = aL * UL[3] + aR * UR[3];
  const R EpL = kShift<R> ? UL[4] + pL - pref + href : UL[4] + pL;  // E + p
  const R EpR = kShift<R> ? UR[4] + pR - pref + href : UR[4] + pR;
  const R Ht = aL * EpL + aR * EpR;
  const R q2 = ut * ut + vt * vt + wt * wt;
  const R c2 = gm1 * (Ht - R(0.5) * q2);
  const R rc = rsq(c2);  // 1/c; c = c^2/c and 1/c^2 = (1/c)^2
  const R ct = c2 * rc, ic2 = rc * rc;
  const R rt = sL * sR;
  const R unt = ut * nv[0] + vt * nv[1] + wt * nv[2];
  const R dr = UR[0] - UL[0], dp = pR - pL;
  const R du = uR - uL, dv = vR - vL, dw = wR - wL;
  const R dun = du * nv[0] + dv * nv[1] + dw * nv[2];
  const R a1 = R(0.5) * (dp - rt * ct * dun) * ic2;
  const R a5 = R(0.5) * (dp + rt * ct * dun) * ic2;
  const R a2 = dr - dp * ic2;
  const R dut = du - dun * nv[0], dvt = dv - dun * nv[1], dwt = dw - dun * nv[2];
  const R l1a1 = fabs(unt - ct) * a1, l5a5 = fabs(unt + ct) * a5, l2 = fabs(unt);
  const R l2a2 = l2 * a2, l2r = l2 * rt;
  // dissipation sum_k |lambda_k| alpha_k r_k, collected: with s15 = l1a1 + l5a5 and c15 = c (l5a5 - l1a1),
  // the two acoustic waves give s15 (u~, H~) + c15 (n, u~_n)
  const R s15 = l1a1 + l5a5, c15 = ct * (l5a5 - l1a1);
  R D[5];
  D[0] = s15 + l2a2;
  D[1] = D[0] * ut + c15 * nv[0] + l2r * dut;
  D[2] = D[0] * vt + c15 * nv[1] + l2r * dvt;
  D[3] = D[0] * wt + c15 * nv[2] + l2r * dwt;
  D[4] = s15 * Ht + c15 * unt + l2a2 * R(0.5) * q2 + l2r * (ut * dut + vt * dvt + wt * dwt);
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = R(0.5) * (FL[v] + FR[v] - D[v]);
}

template <typename R>
__device__ __forceinline__ void riemann(int sf, const R UL[5], const R UR[5], const R nv[3], R gam, R pref, R href,
                                        R F[5]) {
  R irL, irR, pL, pR;
  riemann<R>(sf, UL, UR, nv, gam, pref, href, F, irL, irR, pL, pR);
}

// ---------------------------------------------------------------------------------------------
// init: curl-form metrics, Jacobian, face normals (FP64), FP32 copies
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ double dsweep(const double *f, int node, int d) {
  const int i = node % n, j = (node / n) % n, k = node / nn;
  const int id = d == 0 ? i : d == 1 ? j : k;
  const int st = d == 0 ? 1 : d == 1 ? n : nn;
  const int base = node - id * st;
  double s = 0.0;
#pragma unroll
  for (int m = 0; m < n; ++m) s += c_D[id * n + m] * f[base + m * st];
  return s;
}

// One CTA per element. Ja^d_c = D_k(X_l D_j X_m) - D_j(X_l D_k X_m), (d,j,k), (c,m,l) cyclic;
// J = det(D-derivatives of X). X is taken relative to the element's first node: the metric
// terms are translation invariant, and absolute coordinates (|x| >> h) would make the
// products X_l D_j X_m cancel to O(|x|/h) of rounding.
__global__ void __launch_bounds__(256) k_metrics(const DgDevice d) {
  extern __shared__ double sm[];
  double *X = sm;              // [3][nnn]
  double *dX = X + 3 * nnn;    // [c][dd][nnn]
  double *T1 = dX + 9 * nnn;   // [nnn]
  double *T2 = T1 + nnn;       // [nnn]
  const int e = blockIdx.x;
  const double *xe = d.xyz + (size_t)e * 3 * nnn;
  for (int t = threadIdx.x; t < 3 * nnn; t += blockDim.x) X[t] = xe[t] - xe[(t / nnn) * nnn];
  __syncthreads();
  for (int t = threadIdx.x; t < 9 * nnn; t += blockDim.x) {
    const int node = t % nnn, cd = t / nnn, c = cd / 3, dd = cd % 3;
    dX[cd * nnn + node] = dsweep(X + c * nnn, node, dd);
  }
  __syncthreads();
  for (int dir = 0; dir < 3; ++dir) {
    const int j = (dir + 1) % 3, k = (dir + 2) % 3;
    for (int c = 0; c < 3; ++c) {
      const int m = (c + 1) % 3, l = (c + 2) % 3;
      for (int node = threadIdx.x; node < nnn; node += blockDim.x) {
        T1[node] = X[l * nnn + node] * dX[(m * 3 + j) * nnn + node];
        T2[node] = X[l * nnn + node] * dX[(m * 3 + k) * nnn + node];
      }
      __syncthreads();
      for (int node = threadIdx.x; node < nnn; node += blockDim.x)
        d.Ja[(((size_t)e * 3 + dir) * 3 + c) * nnn + node] = dsweep(T1, node, k) - dsweep(T2, node, j);
      __syncthreads();
    }
  }
  for (int node = threadIdx.x; node < nnn; node += blockDim.x) {
    double a[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int dd = 0; dd < 3; ++dd) a[c][dd] = dX[(c * 3 + dd) * nnn + node];
    const double J = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                     a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    d.J[(size_t)e * nnn + node] = J;
    d.invJ[(size_t)e * nnn + node] = 1.0 / J;
    if (!(J > 0.0) || !isfinite(J)) flag_set(d.flag, 2);
  }
}

// One thread per face point: unit normal and area factor from the L element's metric.
__global__ void __launch_bounds__(256) k_face_normals(const DgDevice d) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)d.nF * nn) return;
  const int f = (int)(t / nn), pq = (int)(t % nn), p = pq % n, q = pq / n;
  const int eL = d.face[5 * f + 0], fL = d.face[5 * f + 1];
  const int dL = fL >> 1;
  const double sg = (fL & 1) ? 1.0 : -1.0;
  const int node = face_node(fL, p, q);
  double a[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) a[c] = sg * d.Ja[(((size_t)eL * 3 + dL) * 3 + c) * nnn + node];
  const double s = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  const double is = 1.0 / s;
  double *o = d.nrm + (size_t)f * 4 * nn + pq;
  o[0] = a[0] * is;
  o[nn] = a[1] * is;
  o[2 * nn] = a[2] * is;
  o[3 * nn] = s;
  if (d.face[5 * f + 2] < 0 && d.hwm) {  // wall face: distance of the wall-model exchange node
    const int xnode = exchange_node(fL, p, q, d.wm_index);
    double h2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double dx = d.xyz[((size_t)eL * 3 + c) * nnn + xnode] - d.xyz[((size_t)eL * 3 + c) * nnn + node];
      h2 += dx * dx;
    }
    d.hwm[(size_t)f * nn + pq] = sqrt(h2);
  }
}

// FP32 roundings of the FP64 metric terms and face normals (FP32-bulk path)
__global__ void __launch_bounds__(256) k_round_geometry(const DgDevice d) {
  const long long nja = (long long)d.nE * 9 * nnn, nnr = (long long)d.nF * 4 * nn, nij = (long long)d.nE * nnn;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nja + nnr + nij;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < nja) d.Jaf[t] = (float)d.Ja[t];
    else if (t < nja + nnr) d.nrm_f[t - nja] = (float)d.nrm[t - nja];
    else d.invJf[t - nja - nnr] = (float)d.invJ[t - nja - nnr];
  }
}

// ---------------------------------------------------------------------------------------------
// wall-modelled wall face point (Sec. 3): advective flux against the mirror state, BR1 jump to the
// mirror state's face value, and the wall shear stress of the wall model as the viscous flux
// ---------------------------------------------------------------------------------------------
template <typename R, int SF>
__device__ __forceinline__ void wall_face(const DgDevice &d, const double *__restrict__ U, int f, int pq, int eL,
                                          int fL, R pref, R href, R gam) {
  const int p = pq % n, q = pq / n;
  const int node = face_node(fL, p, q);
  R UL[5], UG[5], nv[3], Fs[5];
  load_state<R>(d, U, eL, node, UL);
  const R *nr = Buf<R>::nrm(d) + (size_t)f * 4 * nn + pq;
  nv[0] = nr[0];
  nv[1] = nr[nn];
  nv[2] = nr[2 * nn];
  const R s = nr[3 * nn];
  const R mn = UL[1] * nv[0] + UL[2] * nv[1] + UL[3] * nv[2];
  UG[0] = UL[0];
  UG[4] = UL[4];
#pragma unroll
  for (int c = 0; c < 3; ++c) UG[1 + c] = UL[1 + c] - R(2) * mn * nv[c];
  riemann<R>(SF, UL, UG, nv, gam, pref, href, Fs);
  R *oL = Buf<R>::Fsurf(d) + ((size_t)eL * 6 + fL) * 5 * nn + pq;
#pragma unroll
  for (int v = 0; v < 5; ++v) oL[v * nn] = s * Fs[v];
  if (d.equations != 1) return;
  // BR1: w* - w = (w_ghost - w) / 2 = (-(u.n) n, 0)
  const R un = mn / UL[0];
  R *jL = Buf<R>::Wsurf(d) + ((size_t)eL * 6 + fL) * 4 * nn + pq;
#pragma unroll
  for (int c = 0; c < 3; ++c) jL[c * nn] = -un * nv[c];
  jL[3 * nn] = R(0);
  // wall model at the exchange node
  R Ux[5];
  load_state<R>(d, U, eL, exchange_node(fL, p, q, d.wm_index), Ux);
  const R irx = R(1) / Ux[0];
  const R ux[3] = {Ux[1] * irx, Ux[2] * irx, Ux[3] * irx};
  const R uxn = ux[0] * nv[0] + ux[1] * nv[1] + ux[2] * nv[2];
  const R ut[3] = {ux[0] - uxn * nv[0], ux[1] - uxn * nv[1], ux[2] - uxn * nv[2]};
  const R Ut = sqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
  R *fw = Buf<R>::Fwall(d) + (size_t)f * 4 * nn + pq;
  R tw[3] = {R(0), R(0), R(0)};
  if (Ut > R(0)) {
    int it;
    const R utau = wall_utau<R>(Ut, (R)d.hwm[(size_t)f * nn + pq], Cst<R>::mu(d) * irx, (R)d.wm_uinf, (R)d.wm_b,
                                d.wm_vd, it);
    const R tau = Ux[0] * utau * utau;
#pragma unroll
    for (int c = 0; c < 3; ++c) tw[c] = -tau * ut[c] / Ut;  // outward viscous flux: the wall's drag
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) fw[c * nn] = s * tw[c];
  fw[3 * nn] = R(0);  // adiabatic wall at rest
}

// ---------------------------------------------------------------------------------------------
// face kernel: Riemann flux once per face point, stored outward for both sides
// ---------------------------------------------------------------------------------------------
template <typename R, int SF>
__global__ void __launch_bounds__(256) k_face(const DgDevice d, const double *__restrict__ U) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)d.nF * nn) return;
  const int f = (int)(t / nn), pq = (int)(t % nn), p = pq % n, q = pq / n;
  const int *F5 = d.face + 5 * f;
  const int eL = F5[0], fL = F5[1], eR = F5[2], fR = F5[3], o = F5[4];
  const R pref = Cst<R>::pref(d), href = Cst<R>::href(d), gam = Cst<R>::gam(d);
  if (eR < 0) {  // wall-modelled wall
    wall_face<R, SF>(d, U, f, pq, eL, fL, pref, href, gam);
    return;
  }
  int p2, q2;
  orient_map(o, p, q, p2, q2);
  const int nodeL = face_node(fL, p, q), nodeR = face_node(fR, p2, q2);
  const int pqR = p2 + n * q2;
  R UL[5], UR[5], nv[3];
  load_state<R>(d, U, eL, nodeL, UL);
  load_state<R>(d, U, eR, nodeR, UR);
  const R *nr = Buf<R>::nrm(d) + (size_t)f * 4 * nn + pq;
  nv[0] = nr[0];
  nv[1] = nr[nn];
  nv[2] = nr[2 * nn];
  const R s = nr[3 * nn];
  R Fs[5], irL, irR, pL, pR;
  riemann<R>(SF, UL, UR, nv, gam, pref, href, Fs, irL, irR, pL, pR);
  R *oL = Buf<R>::Fsurf(d) + ((size_t)eL * 6 + fL) * 5 * nn;
  R *oR = Buf<R>::Fsurf(d) + ((size_t)eR * 6 + fR) * 5 * nn;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    oL[v * nn + pq] = s * Fs[v];
    oR[v * nn + pqR] = -s * Fs[v];
  }
  if (d.equations == 1) {  // BR1 face values of (u, v, w, T), from the Riemann solver's 1/rho and p
    const R wL[3] = {UL[1] * irL, UL[2] * irL, UL[3] * irL};
    const R wR[3] = {UR[1] * irR, UR[2] * irR, UR[3] * irR};
    const R iR = Cst<R>::iR(d);
    const R jump[4] = {R(0.5) * (wR[0] - wL[0]), R(0.5) * (wR[1] - wL[1]), R(0.5) * (wR[2] - wL[2]),
                       R(0.5) * (pR * irR - pL * irL) * iR};
    R *jL = Buf<R>::Wsurf(d) + ((size_t)eL * 6 + fL) * 4 * nn;
    R *jR = Buf<R>::Wsurf(d) + ((size_t)eR * 6 + fR) * 4 * nn;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      jL[c * nn + pq] = jump[c];
      jR[c * nn + pqR] = -jump[c];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// BR1 lifting + viscous flux: grad w = (1/J)[sum_d Ja^d D_d w + sum_faces (1/w_b) s n_out (w* - w)],
// then Fv^d = sum_c Ja^d_c Fv_c(U, grad w) stored per node (4 components: momentum, energy).
// ---------------------------------------------------------------------------------------------
// resident 256-thread CTAs per SM the register budget must allow: FP32 five (48 registers), FP64 three
template <typename R> __host__ __device__ constexpr int lift_min_blocks() { return std::is_same<R, float>::value ? 5 : 3; }

// (u, v, w, T) of one node from its state values (lifted quantities of BR1)
template <typename R>
__device__ __forceinline__ void lift_prim(const R Uv[5], R gm1, R iR, R pref, R Wn[4]) {
  const R r = Uv[0], ir = R(1) / r;
  const R u = Uv[1] * ir, v = Uv[2] * ir, w = Uv[3] * ir;
  R p = gm1 * (Uv[4] - R(0.5) * r * (u * u + v * v + w * w));
  if (kShift<R>) p += pref;
  Wn[0] = u;
  Wn[1] = v;
  Wn[2] = w;
  Wn[3] = p * ir * iR;
}

// one node's BR1 gradients and contravariant viscous flux: W = the element's lifted quantities
// [4][nnn] (shared memory), Jae its metric terms [3 d][3 c][nnn], Wse its BR1 face jumps [6][4][nn],
// iJ this node's 1/J; writes the element's Fv [3 d][4][nnn] at `node` (out = the element's Fv).
// tau (FP64 only, optional): the element's viscous stress record [6][nnn] (xx, yy, zz, xy, xz, yz),
// which the adjoint's viscous kernel reads instead of forming the gradients again
template <typename R, bool PRE = false>
__device__ __forceinline__ void lift_node(const DgDevice &d, int node, const R *__restrict__ W,
                                          const R (*__restrict__ sD)[n + 1], const R *__restrict__ Jae,
                                          const R *__restrict__ Wse, R iJ, R mu, R kappa, R *__restrict__ out,
                                          const R *__restrict__ S = nullptr, double *__restrict__ tau = nullptr) {
  // PRE: the reference derivatives D_dd w_q of this element come precomputed in S [3 dd][4 q][nnn]
  const int ijk[3] = {node % n, (node / n) % n, node / nn};
  R Ja[3][3];
#pragma unroll
  for (int dd = 0; dd < 3; ++dd)
#pragma unroll
    for (int c = 0; c < 3; ++c) Ja[dd][c] = Jae[(dd * 3 + c) * nnn + node];
  R g[4][3];
#pragma unroll
  for (int q = 0; q < 4; ++q) g[q][0] = g[q][1] = g[q][2] = R(0);
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    const int id = ijk[dd];
    const int st = dd == 0 ? 1 : dd == 1 ? n : nn;
    const int base = node - id * st;
    // the reference derivative along dd, plus the surface term (1/w_b)(+-)(w* - w) on the face of
    // direction dd through this node, before the one contraction with Ja^dd
    R s[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      s[q] = R(0);
      if constexpr (PRE) {
        s[q] = S[(dd * 4 + q) * nnn + node];
      } else {
#pragma unroll
        for (int m = 0; m < n; ++m) s[q] += sD[id][m] * W[q * nnn + base + m * st];
      }
    }
    if (id == 0 || id == N) {
      const int f = 2 * dd + (id == N ? 1 : 0);
      const R sc = (id == N ? R(1) : R(-1)) * Tab<R>::invw(id);
      const int pp = dd == 0 ? ijk[1] : ijk[0];
      const int qq = dd == 2 ? ijk[1] : ijk[2];
      const R *js = Wse + f * 4 * nn + pp + n * qq;
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] += sc * js[q * nn];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      g[q][0] += Ja[dd][0] * s[q];
      g[q][1] += Ja[dd][1] * s[q];
      g[q][2] += Ja[dd][2] * s[q];
    }
  }
  // g holds J grad w; the flux below is linear in grad w, so 1/J goes into mu and kappa (two
  // multiplies per node instead of twelve)
  mu *= iJ;
  kappa *= iJ;
  // Navier-Stokes-Fourier flux in Cartesian direction c: (tau_xc, tau_yc, tau_zc, u.tau_c + kappa dT/dx_c)
  const R u = W[node], v = W[nnn + node], w = W[2 * nnn + node];
  const R div = g[0][0] + g[1][1] + g[2][2];
  const R t23 = R(2.0 / 3.0) * mu * div;
  const R txx = R(2) * mu * g[0][0] - t23, tyy = R(2) * mu * g[1][1] - t23, tzz = R(2) * mu * g[2][2] - t23;
  const R txy = mu * (g[0][1] + g[1][0]), txz = mu * (g[0][2] + g[2][0]), tyz = mu * (g[1][2] + g[2][1]);
  if constexpr (std::is_same<R, double>::value) {
    if (tau) {
      tau[node] = txx; tau[nnn + node] = tyy; tau[2 * nnn + node] = tzz;
      tau[3 * nnn + node] = txy; tau[4 * nnn + node] = txz; tau[5 * nnn + node] = tyz;
    }
  }
  R Fc[3][4];
  Fc[0][0] = txx; Fc[0][1] = txy; Fc[0][2] = txz; Fc[0][3] = u * txx + v * txy + w * txz + kappa * g[3][0];
  Fc[1][0] = txy; Fc[1][1] = tyy; Fc[1][2] = tyz; Fc[1][3] = u * txy + v * tyy + w * tyz + kappa * g[3][1];
  Fc[2][0] = txz; Fc[2][1] = tyz; Fc[2][2] = tzz; Fc[2][3] = u * txz + v * tyz + w * tzz + kappa * g[3][2];
#pragma unroll
  for (int dd = 0; dd < 3; ++dd)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      out[(dd * 4 + q) * nnn + node] = Ja[dd][0] * Fc[0][q] + Ja[dd][1] * Fc[1][q] + Ja[dd][2] * Fc[2][q];
}

template <typename R>
__global__ void __launch_bounds__(LIFT_THREADS, lift_min_blocks<R>()) k_lift(const DgDevice d, const double *__restrict__ U,
                                                                             double *__restrict__ tau) {
  __shared__ R W[LIFT_EPB][4][nnn];
  __shared__ R sD[n][n + 1];  // D, rows padded: lanes read different rows without bank conflicts
  for (int t = threadIdx.x; t < nn; t += blockDim.x) sD[t / n][t % n] = Tab<R>::D(t);
  const int e0 = blockIdx.x * LIFT_EPB;
  const R gm1 = Cst<R>::gm1(d), iR = Cst<R>::iR(d);
  const R pref = Cst<R>::pref(d);
  for (int t = threadIdx.x; t < LIFT_EPB * nnn; t += blockDim.x) {
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    R Uv[5], Wn[4];
    load_state<R>(d, U, e, node, Uv);
    lift_prim<R>(Uv, gm1, iR, pref, Wn);
#pragma unroll
    for (int q = 0; q < 4; ++q) W[le][q][node] = Wn[q];
  }
  __syncthreads();
  const R mu = Cst<R>::mu(d), kappa = Cst<R>::kappa(d);
  // the thread's nodes unrolled, so that their metric loads are in flight together
#pragma unroll
  for (int rr = 0; rr < (LIFT_EPB * nnn + LIFT_THREADS - 1) / LIFT_THREADS; ++rr) {
    const int t = threadIdx.x + rr * LIFT_THREADS;
    if (t >= LIFT_EPB * nnn) continue;
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    const R iJ = kShift<R> ? (R)d.invJf[(size_t)e * nnn + node] : (R)d.invJ[(size_t)e * nnn + node];
    lift_node<R>(d, node, &W[le][0][0], sD, Buf<R>::Ja(d) + (size_t)e * 9 * nnn,
                 Buf<R>::Wsurf(d) + (size_t)e * 6 * 4 * nn, iJ, mu, kappa, Buf<R>::Fv(d) + (size_t)e * 12 * nnn,
                 nullptr, tau ? tau + (size_t)e * 6 * nnn : nullptr);
  }
}

// FP64 lifting with the reference derivatives formed along lines (used at N = 7): one thread per line of the
// element(s) applies D to all four lifted quantities with the even-odd halves of D (the LGL D is
// centro-antisymmetric), n^2/2 + 2n operations per line and quantity instead of the n^2 of n node-wise
// sweeps; the derivatives go to shared memory, and the node-wise part (metric contraction, surface
// terms, viscous flux, contravariant projection) is lift_node's. Dynamic shared memory:
// W [EPB][4][nnn] and S [EPB][3][4][nnn] doubles.
constexpr size_t LIFT_LINES_SMEM = sizeof(double) * LIFT_EPB * 16 * nnn;
__global__ void __launch_bounds__(LIFT_THREADS, lift_min_blocks<double>()) k_lift_lines(const DgDevice d,
                                                                                      const double *__restrict__ U,
                                                                                      double *__restrict__ tau) {
  if constexpr (n % 2 == 0) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    double *W = reinterpret_cast<double *>(sm_raw);  // [EPB][4][nnn]
    double *S = W + LIFT_EPB * 4 * nnn;              // [EPB][12][nnn]
    __shared__ double sD[n][n + 1];
    for (int t = threadIdx.x; t < nn; t += blockDim.x) sD[t / n][t % n] = c_D[t];
    const int e0 = blockIdx.x * LIFT_EPB;
    const double gm1 = d.gm1, iR = d.iR;
    for (int t = threadIdx.x; t < LIFT_EPB * nnn; t += blockDim.x) {
      const int le = t / nnn, node = t % nnn, e = e0 + le;
      if (e >= d.nE) continue;
      double Uv[5], Wn[4];
      load_state<double>(d, U, e, node, Uv);
      lift_prim<double>(Uv, gm1, iR, 0.0, Wn);
#pragma unroll
      for (int q = 0; q < 4; ++q) W[(le * 4 + q) * nnn + node] = Wn[q];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < LIFT_EPB * 3 * nn; t += blockDim.x) {
      const int le = t / (3 * nn), r = t % (3 * nn), dir = r / nn, line = r % nn;
      if (e0 + le >= d.nE) continue;
      const int a = line % n, b = line / n;
      const int base = dir == 0 ? n * (a + n * b) : dir == 1 ? a + nn * b : a + n * b;
      const int st = dir == 0 ? 1 : dir == 1 ? n : nn;
      const double *We = W + le * 4 * nnn;
      double *Se = S + (le * 12 + dir * 4) * nnn;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double ev[EO_H], od[EO_H];
#pragma unroll
        for (int m = 0; m < EO_H; ++m) {
          const double f0 = We[q * nnn + base + m * st], f1 = We[q * nnn + base + (N - m) * st];
          ev[m] = f0 + f1;
          od[m] = f0 - f1;
        }
#pragma unroll
        for (int i = 0; i < EO_H; ++i) {
          double pa = 0.0, pb = 0.0;
#pragma unroll
          for (int m = 0; m < EO_H; ++m) {
            pa += c_FP[i * EO_H + m] * ev[m];
            pb += c_FM[i * EO_H + m] * od[m];
          }
          Se[q * nnn + base + i * st] = pa + pb;
          Se[q * nnn + base + (N - i) * st] = pb - pa;
        }
      }
    }
    __syncthreads();
    const double mu = d.mu, kappa = d.kappa;
#pragma unroll
    for (int rr = 0; rr < (LIFT_EPB * nnn + LIFT_THREADS - 1) / LIFT_THREADS; ++rr) {
      const int t = threadIdx.x + rr * LIFT_THREADS;
      if (t >= LIFT_EPB * nnn) continue;
      const int le = t / nnn, node = t % nnn, e = e0 + le;
      if (e >= d.nE) continue;
      lift_node<double, true>(d, node, W + le * 4 * nnn, sD, d.Ja + (size_t)e * 9 * nnn,
                              d.Wsurf + (size_t)e * 6 * 4 * nn, d.invJ[(size_t)e * nnn + node], mu, kappa,
                              d.Fv + (size_t)e * 12 * nnn, S + le * 12 * nnn,
                              tau ? tau + (size_t)e * 6 * nnn : nullptr);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// volume kernel
// ---------------------------------------------------------------------------------------------

// Flux differencing along one line of n nodes: acc_i = sum_{m != i} 2 D_im F#(U_i, U_m) with
// the metric average {Ja}. For Kennedy-Gruber and Pirozzoli the flux is formed from plain sums
// S = x_i + x_m and the 1/2 factors are folded into the coefficients (D/4 for mass, D/8 otherwise).
// Node i's sums stay in registers while m runs over i+1..N; node m's share of each pair goes
// straight to the line's accumulator in shared memory (the line belongs to this thread alone).
// Ac points at the direction's accumulator [5][PS] of this element, indexed like P.
// Staged slots: 0 rho, 1 u, 2 v, 3 w, 4 4 p' (momentum pressure), 5 X, 6 Y with
// PIR: X = h; KG: X = e = E/rho, Y = 2p; EC: Y = p; central: X = E + p.
template <typename R, int VF>
__device__ __forceinline__ void line_fluxdiff(const R *__restrict__ P, int pb, int ps, const R *__restrict__ Jd,
                                              int gb, int gs, R gam, R pref, R *__restrict__ Ac) {
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    const int ai = pb + i * ps, gi = gb + i * gs;
    const R ri = P[ai], ui = P[PS + ai], vi = P[2 * PS + ai], wi = P[3 * PS + ai];
    const R p4i = P[4 * PS + ai], xi_ = P[5 * PS + ai], yi = P[6 * PS + ai];
    const R jxi = __ldg(Jd + gi), jyi = __ldg(Jd + nnn + gi), jzi = __ldg(Jd + 2 * nnn + gi);
    R ac[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) ac[v] = (i == 0) ? R(0) : Ac[v * PS + ai];
#pragma unroll
    for (int m = i + 1; m < n; ++m) {
      const int am = pb + m * ps, gm = gb + m * gs;
      const R rm = P[am], um = P[PS + am], vm = P[2 * PS + am], wm = P[3 * PS + am];
      const R p4m = P[4 * PS + am], xm = P[5 * PS + am], ym = P[6 * PS + am];
      const R jxm = __ldg(Jd + gm), jym = __ldg(Jd + nnn + gm), jzm = __ldg(Jd + 2 * nnn + gm);
      R F[5], ci[5], cm[5];
      if (VF == VF_PIR || VF == VF_KG) {
        const R Sjx = jxi + jxm, Sjy = jyi + jym, Sjz = jzi + jzm;
        const R Su = ui + um, Sv = vi + vm, Sw = wi + wm;
        const R Vp = Su * Sjx + Sv * Sjy + Sw * Sjz;  // 4 {u}.{Ja}
        F[0] = (ri + rm) * Vp;                        // 8 F_rho
        const R Sp = p4i + p4m;                       // 4 (p'_i + p'_m)
        F[1] = F[0] * Su + Sp * Sjx;                  // 16 F_rho u
        F[2] = F[0] * Sv + Sp * Sjy;
        F[3] = F[0] * Sw + Sp * Sjz;
        if (VF == VF_PIR) F[4] = F[0] * (xi_ + xm);            // 16 {rho}V{h}
        else F[4] = F[0] * (xi_ + xm) + (yi + ym) * Vp;        // 16 ({rho}V{e} + {p}V)
        ci[0] = Tab<R>::Dq(i * n + m); cm[0] = Tab<R>::Dq(m * n + i);
#pragma unroll
        for (int v = 1; v < 5; ++v) { ci[v] = Tab<R>::De(i * n + m); cm[v] = Tab<R>::De(m * n + i); }
      } else {
        const R a[3] = {R(0.5) * (jxi + jxm), R(0.5) * (jyi + jym), R(0.5) * (jzi + jzm)};
        if (VF == VF_EC) {
          ec_flux<R>(ri, ui, vi, wi, yi, rm, um, vm, wm, ym, a, gam, kShift<R> ? pref : R(0), F);
        } else {  // central: mean of the two Euler fluxes through {Ja}; slot 5 = E + p
          const R Vi = ui * a[0] + vi * a[1] + wi * a[2], Vm = um * a[0] + vm * a[1] + wm * a[2];
          const R pm2 = R(0.125) * (p4i + p4m);
          F[0] = R(0.5) * (ri * Vi + rm * Vm);
          F[1] = R(0.5) * (ri * ui * Vi + rm * um * Vm) + pm2 * a[0];
          F[2] = R(0.5) * (ri * vi * Vi + rm * vm * Vm) + pm2 * a[1];
          F[3] = R(0.5) * (ri * wi * Vi + rm * wm * Vm) + pm2 * a[2];
          F[4] = R(0.5) * (xi_ * Vi + xm * Vm);
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) { ci[v] = Tab<R>::D2(i * n + m); cm[v] = Tab<R>::D2(m * n + i); }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        ac[v] += ci[v] * F[v];
        if (i == 0) Ac[v * PS + am] = cm[v] * F[v];
        else Ac[v * PS + am] += cm[v] * F[v];
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) Ac[v * PS + ai] = ac[v];
  }
}

// Viscous divergence along one line: Ac[1+q]_i -= sum_{m != i} D_im Fv^d_q(m) for the line's n
// nodes (the diagonal cancels against the surface term, see the file header). Fvd points at the
// element's contravariant viscous flux of this direction [4][nnn].
template <typename R>
__device__ __forceinline__ void line_viscous(const R *__restrict__ Fvd, int gb, int gs, int pb, int ps,
                                             R *__restrict__ Ac) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    R f[n];
#pragma unroll
    for (int m = 0; m < n; ++m) f[m] = __ldg(Fvd + q * nnn + gb + m * gs);
    if constexpr (n % 2 == 0) {  // even-odd: n^2/2 + 2n operations per line instead of n^2
      R ev[EO_H], od[EO_H];
#pragma unroll
      for (int m = 0; m < EO_H; ++m) { ev[m] = f[m] + f[N - m]; od[m] = f[m] - f[N - m]; }
#pragma unroll
      for (int i = 0; i < EO_H; ++i) {
        R a = R(0), b = R(0);
#pragma unroll
        for (int m = 0; m < EO_H; ++m) {
          a += Tab<R>::VP(i * EO_H + m) * ev[m];
          b += Tab<R>::VM(i * EO_H + m) * od[m];
        }
        Ac[(1 + q) * PS + pb + i * ps] -= a + b;
        Ac[(1 + q) * PS + pb + (N - i) * ps] -= b - a;
      }
    } else {
#pragma unroll
      for (int i = 0; i < n; ++i) {
        R s = R(0);
#pragma unroll
        for (int m = 0; m < n; ++m)
          if (m != i) s += Tab<R>::D(i * n + m) * f[m];
        Ac[(1 + q) * PS + pb + i * ps] -= s;
      }
    }
  }
}

// (rho, u, v, w, p') of staged node a for the FV operator (slot 7 holds p')
template <typename R>
__device__ __forceinline__ void staged_prim(const R *__restrict__ P, int a, R q[5]) {
  q[0] = P[a]; q[1] = P[PS + a]; q[2] = P[2 * PS + a]; q[3] = P[3 * PS + a]; q[4] = P[7 * PS + a];
}

// reconstructed left/right interface states of subcell i (minmod slopes in primitive variables;
// first order in the outer subcells and wherever the reconstruction loses positivity)
template <typename R>
__device__ __forceinline__ void subcell_states(const R *__restrict__ P, int pb, int ps, int i, R pref, R qL[5],
                                               R qR[5]) {
  R q[5];
  staged_prim<R>(P, pb + i * ps, q);
  R sg[5] = {R(0), R(0), R(0), R(0), R(0)};
  if (i > 0 && i < N) {
    R qb[5], qf[5];
    staged_prim<R>(P, pb + (i - 1) * ps, qb);
    staged_prim<R>(P, pb + (i + 1) * ps, qf);
    const R hb = Tab<R>::ihx(i), hf = Tab<R>::ihx(i + 1);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const R sb = (q[v] - qb[v]) * hb, sf_ = (qf[v] - q[v]) * hf;
      sg[v] = (sb * sf_ <= R(0)) ? R(0) : (fabs(sb) < fabs(sf_) ? sb : sf_);
    }
  }
  const R dl = Tab<R>::xh(i) - Tab<R>::xi(i), dr = Tab<R>::xh(i + 1) - Tab<R>::xi(i);
#pragma unroll
  for (int v = 0; v < 5; ++v) { qL[v] = q[v] + sg[v] * dl; qR[v] = q[v] + sg[v] * dr; }
  const R pad = kShift<R> ? pref : R(0);
  if (qL[0] <= R(0) || qL[4] + pad <= R(0) || qR[0] <= R(0) || qR[4] + pad <= R(0)) {
#pragma unroll
    for (int v = 0; v < 5; ++v) { qL[v] = q[v]; qR[v] = q[v]; }
  }
}

// conservative state from (rho, u, v, w, p') in the kernel's representation (E' in FP32)
template <typename R>
__device__ __forceinline__ void cons_of(const R q[5], R igm1, R U[5]) {
  U[0] = q[0]; U[1] = q[0] * q[1]; U[2] = q[0] * q[2]; U[3] = q[0] * q[3];
  U[4] = q[4] * igm1 + R(0.5) * q[0] * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
}

// FV subcell operator along one line (Sec. 4.1): Riemann fluxes at the N interior subcell
// interfaces with telescoped interface metrics a_{i+1/2} = a_{i-1/2} + w_i (D Ja)_i, the DG surface
// fluxes at the element faces, and Ac_i = (f_{i+1/2} - f_{i-1/2}) / w_i written to shared memory.
template <typename R>
__device__ __forceinline__ void line_fv(const R *__restrict__ P, int pb, int ps, const R *__restrict__ Jd, int gb,
                                        int gs, const R *Fm, const R *Fp, int sf, R gam, R igm1, R pref, R href,
                                        R *__restrict__ Ac) {
  R fl[5];  // flux at the left interface of the current subcell, +xi direction
#pragma unroll
  for (int v = 0; v < 5; ++v) fl[v] = -Fm[v * nn];
  R a[3] = {__ldg(Jd + gb), __ldg(Jd + nnn + gb), __ldg(Jd + 2 * nnn + gb)};
  R qLn[5], qRn[5];
  subcell_states<R>(P, pb, ps, 0, pref, qLn, qRn);
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    R fr[5];
    const R qRi[5] = {qRn[0], qRn[1], qRn[2], qRn[3], qRn[4]};
    if (i < N) {
      subcell_states<R>(P, pb, ps, i + 1, pref, qLn, qRn);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        R dj = R(0);
#pragma unroll
        for (int m = 0; m < n; ++m) dj += Tab<R>::D(i * n + m) * __ldg(Jd + c * nnn + gb + m * gs);
        a[c] += Tab<R>::w(i) * dj;
      }
      const R a2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
      const R is = rsq(a2);  // 1/|a|; |a| = |a|^2 / |a|
      const R s = a2 * is;
      const R nv[3] = {a[0] * is, a[1] * is, a[2] * is};
      R UL[5], UR[5], Fs[5];
      cons_of<R>(qRi, igm1, UL);
      cons_of<R>(qLn, igm1, UR);
      riemann<R>(sf, UL, UR, nv, gam, pref, href, Fs);
#pragma unroll
      for (int v = 0; v < 5; ++v) fr[v] = s * Fs[v];
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) fr[v] = Fp[v * nn];
    }
    const R iw = Tab<R>::invw(i);
#pragma unroll
    for (int v = 0; v < 5; ++v) { Ac[v * PS + pb + i * ps] = (fr[v] - fl[v]) * iw; fl[v] = fr[v]; }
  }
}

// line geometry of line `line` of direction `dir`: staging base/stride (padded) and global base/stride
__device__ __forceinline__ void line_geom(int dir, int line, int &pb, int &ps, int &gb, int &gs, int &a, int &b) {
  a = line % n;
  b = line / n;
  if (dir == 0) { pb = (n + 1) * (a + n * b); ps = 1; gb = n * (a + n * b); gs = 1; }
  else if (dir == 1) { pb = a + (n + 1) * n * b; ps = n + 1; gb = a + nn * b; gs = n; }
  else { pb = a + (n + 1) * b; ps = (n + 1) * n; gb = a + n * b; gs = nn; }
}

template <typename R, int VF, bool SC>
__global__ void __launch_bounds__(vol_threads<R, SC>(), vol_min_blocks<R, SC>()) k_volume(const DgDevice d, const double *U, double *out,
                                                        double *__restrict__ g, int mode, int first, double dt,
                                                        double A, double B) {
  constexpr int NP = vol_np<SC>();
  extern __shared__ __align__(16) unsigned char sm_raw[];
  R *P = reinterpret_cast<R *>(sm_raw);  // [EPB][NP][PS]
  R *Acc = P + VOL_EPB * NP * PS;         // [EPB][3][5][PS]
  R *AccT = Acc + VOL_EPB * 15 * PS;      // [EPB][5][nnn] (SC only)
  const int e0 = blockIdx.x * VOL_EPB;
  const R gam = Cst<R>::gam(d), gm1 = Cst<R>::gm1(d);
  const R pref = Cst<R>::pref(d), href = Cst<R>::href(d);
  const double eref = d.eref;
  const R *Jab = Buf<R>::Ja(d);
  const int vf = VF;
  // phase A: stage primitive quantities
  for (int t = threadIdx.x; t < VOL_EPB * nnn; t += blockDim.x) {
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    R Uv[5];
    load_state<R>(d, U, e, node, Uv);
    const R r = Uv[0], m1 = Uv[1], m2 = Uv[2], m3 = Uv[3], E = Uv[4];
    const R ir = R(1) / r;
    const R u = m1 * ir, v = m2 * ir, w = m3 * ir;
    const R pm = gm1 * (E - R(0.5) * (m1 * u + m2 * v + m3 * w));  // p' (= p in FP64)
    const R p = kShift<R> ? pm + pref : pm;
    const R Et = kShift<R> ? E + (R)eref : E;
    if (!(r > R(0)) || !(p > R(0)) || !isfinite(E)) flag_set(d.flag, 1);
    R *Pe = P + le * NP * PS + pidx(node);
    Pe[0] = r; Pe[PS] = u; Pe[2 * PS] = v; Pe[3 * PS] = w; Pe[4 * PS] = R(4) * pm;
    if (vf == VF_PIR) Pe[5 * PS] = (Et + p) * ir;
    else if (vf == VF_KG) { Pe[5 * PS] = Et * ir; Pe[6 * PS] = R(2) * p; }
    else if (vf == VF_EC) Pe[6 * PS] = p;
    else Pe[5 * PS] = Et + p;
    if (SC) Pe[7 * PS] = pm;
  }
  __syncthreads();
  // phase B: flux differencing, one thread per line, the three line families at once
  for (int t = threadIdx.x; t < VOL_EPB * 3 * nn; t += blockDim.x) {
    const int le = t / (3 * nn), r = t % (3 * nn), dir = r / nn, line = r % nn, e = e0 + le;
    if (e >= d.nE) continue;
    int pb, ps, gb, gs, a, b;
    line_geom(dir, line, pb, ps, gb, gs, a, b);
    // viscous divergence joins the line sums, except under the blend (which must not weight it)
    const bool visc = !SC && d.equations == 1;
    line_fluxdiff<R, VF>(P + le * NP * PS, pb, ps, Jab + ((size_t)e * 3 + dir) * 3 * nnn, gb, gs, gam, pref,
                         Acc + (le * 3 + dir) * 5 * PS);
    if (visc)
      line_viscous<R>(Buf<R>::Fv(d) + ((size_t)e * 12 + dir * 4) * nnn, gb, gs, pb, ps, Acc + (le * 3 + dir) * 5 * PS);
  }
  __syncthreads();
  const R *Fsb = Buf<R>::Fsurf(d);
  if (SC) {
    // DG total (volume + surface) per node into AccT, then the FV operator into Acc
    for (int t = threadIdx.x; t < VOL_EPB * nnn; t += blockDim.x) {
      const int le = t / nnn, node = t % nnn, e = e0 + le;
      if (e >= d.nE) continue;
      const int ijk[3] = {node % n, (node / n) % n, node / nn};
      const int pn = pidx(node);
      R s[5];
#pragma unroll
      for (int v = 0; v < 5; ++v)
        s[v] = Acc[(le * 3 + 0) * 5 * PS + v * PS + pn] + Acc[(le * 3 + 1) * 5 * PS + v * PS + pn] +
               Acc[(le * 3 + 2) * 5 * PS + v * PS + pn];
#pragma unroll
      for (int dd = 0; dd < 3; ++dd) {
        const int id = ijk[dd];
        if (id != 0 && id != N) continue;
        const int f = 2 * dd + (id == N ? 1 : 0);
        const int pp = dd == 0 ? ijk[1] : ijk[0], qq = dd == 2 ? ijk[1] : ijk[2];
        const R *fs = Fsb + ((size_t)e * 6 + f) * 5 * nn + pp + n * qq;
#pragma unroll
        for (int v = 0; v < 5; ++v) s[v] += Tab<R>::invw(id) * fs[v * nn];
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) AccT[(le * 5 + v) * nnn + node] = s[v];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < VOL_EPB * 3 * nn; t += blockDim.x) {
      const int le = t / (3 * nn), r = t % (3 * nn), dir = r / nn, line = r % nn, e = e0 + le;
      if (e >= d.nE) continue;
      if (!(d.alpha[e] > 0.0)) continue;
      int pb, ps, gb, gs, a, b;
      line_geom(dir, line, pb, ps, gb, gs, a, b);
      const R *Fm = Fsb + ((size_t)e * 6 + 2 * dir) * 5 * nn + a + n * b;
      const R *Fp = Fsb + ((size_t)e * 6 + 2 * dir + 1) * 5 * nn + a + n * b;
      line_fv<R>(P + le * NP * PS, pb, ps, Jab + ((size_t)e * 3 + dir) * 3 * nnn, gb, gs, Fm, Fp, d.sflux, gam,
                 Cst<R>::igm1(d), pref, href, Acc + (le * 3 + dir) * 5 * PS);
    }
    __syncthreads();
  }
  // phase C: per node -- surface terms, viscous divergence, blend, Jacobian, output / LSERK
  const bool ns = d.equations == 1;
  const R *Fvb = Buf<R>::Fv(d);
  for (int t = threadIdx.x; t < VOL_EPB * nnn; t += blockDim.x) {
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    const int ijk[3] = {node % n, (node / n) % n, node / nn};
    const int pn = pidx(node);
    R s[5];
    if (SC) {
      const R al = (R)d.alpha[e];
#pragma unroll
      for (int v = 0; v < 5; ++v) s[v] = AccT[(le * 5 + v) * nnn + node];
      if (al > R(0)) {
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const R fv = Acc[(le * 3 + 0) * 5 * PS + v * PS + pn] + Acc[(le * 3 + 1) * 5 * PS + v * PS + pn] +
                       Acc[(le * 3 + 2) * 5 * PS + v * PS + pn];
          s[v] = al * fv + (R(1) - al) * s[v];
        }
      }
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v)
        s[v] = Acc[(le * 3 + 0) * 5 * PS + v * PS + pn] + Acc[(le * 3 + 1) * 5 * PS + v * PS + pn] +
               Acc[(le * 3 + 2) * 5 * PS + v * PS + pn];
#pragma unroll
      for (int dd = 0; dd < 3; ++dd) {
        const int id = ijk[dd];
        if (id != 0 && id != N) continue;
        const int f = 2 * dd + (id == N ? 1 : 0);
        const int pp = dd == 0 ? ijk[1] : ijk[0], qq = dd == 2 ? ijk[1] : ijk[2];
        const R *fs = Fsb + ((size_t)e * 6 + f) * 5 * nn + pp + n * qq;
#pragma unroll
        for (int v = 0; v < 5; ++v) s[v] += Tab<R>::invw(id) * fs[v * nn];
      }
    }
    if (ns) {
      const R *Fve = Fvb + (size_t)e * 12 * nnn;
      R vis[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
      for (int dd = 0; dd < 3; ++dd) {
        const int id = ijk[dd];
        if (SC) {  // (without the blend the line threads of phase B already added this part)
          const int st = dd == 0 ? 1 : dd == 1 ? n : nn;
          const int base = node - id * st;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            R acc = R(0);
#pragma unroll
            for (int m = 0; m < n; ++m)
              if (m != id) acc += Tab<R>::D(id * n + m) * Fve[(dd * 4 + q) * nnn + base + m * st];
            vis[q] += acc;
          }
        }
        if (id == 0 || id == N) {  // -(1/(2 w_b)) phi_nb, phi_nb = neighbour's outward normal viscous flux
          const int f = 2 * dd + (id == N ? 1 : 0);
          const int pp = dd == 0 ? ijk[1] : ijk[0], qq = dd == 2 ? ijk[1] : ijk[2];
          const int *ef = d.ef + ((size_t)e * 6 + f) * 4;
          const int nb = ef[0], fnb = ef[1], o = ef[2];
          if (nb < 0) {  // wall: (1/w_b) (F*_wall - (+-) Fv_own / 2), the wall-model flux F*_wall outward
            const R *fw = Buf<R>::Fwall(d) + (size_t)ef[3] * 4 * nn + pp + n * qq;
            const R hs = (id == N) ? R(0.5) : R(-0.5);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              vis[q] += Tab<R>::invw(id) * (fw[q * nn] - hs * Fve[(dd * 4 + q) * nnn + node]);
            continue;
          }
          int p2, q2;
          orient_map(o, pp, qq, p2, q2);
          const int nbnode = face_node(fnb, p2, q2);
          const R sg = (fnb & 1) ? R(0.5) : R(-0.5);
          const R *Fvn = Fvb + ((size_t)nb * 12 + (fnb >> 1) * 4) * nnn + nbnode;
#pragma unroll
          for (int q = 0; q < 4; ++q) vis[q] -= Tab<R>::invw(id) * sg * Fvn[q * nnn];
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) s[1 + q] -= vis[q];
    }
    const double miJ = -d.invJ[(size_t)e * nnn + node];
    const size_t gi = (size_t)e * 5 * nnn + node;
    if (mode == 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) out[gi + v * nnn] = miJ * to_double(s[v]);
    } else {
      const double fac = dt * miJ;  // the stage increment dt Ut = (dt (-1/J)) s: one multiply per node
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double du = fac * to_double(s[v]);
        const double gv = first ? du : A * g[gi + v * nnn] + du;
        g[gi + v * nnn] = gv;
        const double un = U[gi + v * nnn] + B * gv;
        out[gi + v * nnn] = un;
        if (kShift<R>) d.Uf[gi + v * nnn] = (float)(v == 4 ? un - eref : un);
      }
    }
  }
}

}  // namespace

#include "dg_fp32.cuh"  // the FP32-bulk volume and lifting kernels without the blend

namespace {

// ---------------------------------------------------------------------------------------------
// modified Persson indicator (Sec. 4.1, Eq. (7)) and the neighbour extension (FP64)
// ---------------------------------------------------------------------------------------------
// One warp per element (IND_WARPS elements per CTA): q = rho p staged in shared memory, its modal
// coefficients by three tensor-product passes with the inverse Vandermonde (a padded shared-memory
// copy, so lanes reading different rows do not serialise on constant memory), the shell energies
// reduced with warp shuffles; no block-wide barrier after the table load. The kernel is bound by the
// FP64 pipe, so it saves FP64 instructions:
//  - q = rho p = (gamma - 1)(rho E - |m|^2 / 2), with no division;
//  - each pass uses the parity of the Legendre modes on the symmetric LGL nodes,
//    Vinv[a][N-i] = (-1)^a Vinv[a][i]: with q+-_i = q_i +- q_(N-i), output a needs the first half of
//    row a against q+ (a even) or q- (a odd), n(n+1)/2 multiplies per line instead of n^2;
//  - the threshold T of Eq. (7) and -s/T are per-context constants from the host.
constexpr int IND_WARPS = 4;
constexpr int IND_H = (n + 1) / 2;  // first half of a line, the middle node included when n is odd

// one pass along a line of stride st starting at `base`: out[base + a st] = sum_i Vinv[a][i] in[base + i st]
__device__ __forceinline__ void ind_pass(const double (*__restrict__ sV)[n + 1], const double *__restrict__ in,
                                         double *__restrict__ out, int base, int st, int a) {
  double s = 0.0;
  const double sg = (a & 1) ? -1.0 : 1.0;
#pragma unroll
  for (int i = 0; i < n / 2; ++i) s += sV[a][i] * (in[base + i * st] + sg * in[base + (N - i) * st]);
  if (n & 1) s += sV[a][N / 2] * in[base + (N / 2) * st];  // the middle node (odd n; zero for odd a)
  out[base + a * st] = s;
}

__global__ void __launch_bounds__(32 * IND_WARPS) k_indicator(const DgDevice d, const double *__restrict__ U) {
  __shared__ double sV[n][n + 1];
  __shared__ double q[IND_WARPS][nnn], t1[IND_WARPS][nnn];
  for (int t = threadIdx.x; t < nn; t += blockDim.x) sV[t / n][t % n] = c_Vinv[t];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * IND_WARPS + w;
  if (e >= d.nE) return;
  const double gm1 = d.gm1;
  double *qw = q[w], *tw = t1[w];
  for (int node = lane; node < nnn; node += 32) {
    const double *Ue = U + (size_t)e * 5 * nnn + node;
    const double r = Ue[0], m1 = Ue[nnn], m2 = Ue[2 * nnn], m3 = Ue[3 * nnn];
    qw[node] = gm1 * (r * Ue[4 * nnn] - 0.5 * (m1 * m1 + m2 * m2 + m3 * m3));
  }
  __syncwarp();
  for (int node = lane; node < nnn; node += 32) {  // xi: (i,j,k) -> (a,j,k)
    const int a = node % n;
    ind_pass(sV, qw, tw, node - a, 1, a);
  }
  __syncwarp();
  for (int node = lane; node < nnn; node += 32) {  // eta
    const int b = (node / n) % n;
    ind_pass(sV, tw, qw, node - b * n, n, b);
  }
  __syncwarp();
  for (int node = lane; node < nnn; node += 32) {  // zeta into t1
    const int c = node / nn;
    ind_pass(sV, qw, tw, node - c * nn, nn, c);
  }
  __syncwarp();
  double all = 0.0, shN = 0.0, shN1 = 0.0;
  for (int node = lane; node < nnn; node += 32) {  // the shell energies
    const int a = node % n, b = (node / n) % n, c = node / nn;
    const int M = max(a, max(b, c));
    const double m2 = tw[node] * tw[node];
    all += m2;
    if (M == N) shN += m2;
    if (M == N - 1) shN1 += m2;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    all += __shfl_down_sync(0xffffffffu, all, o);
    shN += __shfl_down_sync(0xffffffffu, shN, o);
    shN1 += __shfl_down_sync(0xffffffffu, shN1, o);
  }
  if (lane == 0) {
    const double tot = all, sN = shN, sN1 = shN1;
    double E = tot > 1e-300 ? sN / tot : 0.0;
    if (N >= 2) {
      const double tot1 = tot - sN;
      const double E1 = tot1 > 1e-300 ? sN1 / tot1 : 0.0;
      E = fmax(E, E1);
    }
    double al = 1.0 / (1.0 + exp(d.ind_k * (E - d.ind_T)));
    if (al < d.alpha_min) al = 0.0;
    if (al > d.alpha_max) al = d.alpha_max;
    d.alpha_raw[e] = al;
  }
}

__global__ void __launch_bounds__(256) k_spread(const DgDevice d, double *alpha_out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.nE) return;
  double a = d.alpha_raw[e];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int nb = d.ef[(e * 6 + f) * 4];
    if (nb >= 0) a = fmax(a, 0.5 * d.alpha_raw[nb]);
  }
  alpha_out[e] = a;
}

// ---------------------------------------------------------------------------------------------
// reductions: integral invariants and the time-step estimate (deterministic two-pass, FP64)
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_invariants(const DgDevice d, const double *__restrict__ U,
                                                    const double *__restrict__ Ut) {
  __shared__ double red[8][256];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long total = (long long)d.nE * nnn;
  const double gam = d.gamma;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(t / nnn), node = (int)(t % nnn);
    const int i = node % n, j = (node / n) % n, k = node / nn;
    const double wq = c_w[i] * c_w[j] * c_w[k] * d.J[t];
    const size_t b = (size_t)e * 5 * nnn + node;
    double Uv[5], Tv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) { Uv[v] = U[b + v * nnn]; Tv[v] = Ut[b + v * nnn]; }
    invariants_node(gam, wq, Uv, Tv, acc);
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) red[m][threadIdx.x] = acc[m];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int m = 0; m < 8; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 8) d.red[blockIdx.x * 8 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_reduce_partials(const double *__restrict__ part, int nblocks, int width, int op_min, double *out) {
  // one thread per output column, fixed summation order (deterministic)
  const int c = threadIdx.x;
  if (c >= width) return;
  double s = op_min ? part[c] : 0.0;
  for (int b = op_min ? 1 : 0; b < nblocks; ++b) {
    const double x = part[b * width + c];
    s = op_min ? fmin(s, x) : s + x;
  }
  out[c] = s;
}

__global__ void __launch_bounds__(256) k_max_dt(const DgDevice d, const double *__restrict__ U) {
  __shared__ double red[256];
  double best = 1e300;
  const long long total = (long long)d.nE * nnn;
  const double gam = d.gamma;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(t / nnn), node = (int)(t % nnn);
    const size_t b = (size_t)e * 5 * nnn + node;
    const double r = U[b], ir = 1.0 / r;
    const double u = U[b + nnn] * ir, v = U[b + 2 * nnn] * ir, w = U[b + 3 * nnn] * ir;
    const double p = (gam - 1.0) * (U[b + 4 * nnn] - 0.5 * r * (u * u + v * v + w * w));
    const double c = sqrt(gam * p * ir);
    double lam = 0.0;
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      const double *Jd = d.Ja + ((size_t)e * 3 + dd) * 3 * nnn + node;
      const double ax = Jd[0], ay = Jd[nnn], az = Jd[2 * nnn];
      lam += fabs(u * ax + v * ay + w * az) + c * sqrt(ax * ax + ay * ay + az * az);
    }
    best = fmin(best, 2.0 * d.J[t] / ((2.0 * N + 1.0) * lam));
  }
  red[threadIdx.x] = best;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) d.red[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------------
cudaError_t upload(const DgTables &t) {
  if (t.N != N) return cudaErrorInvalidValue;
  double D2[nn], Dq[nn], De[nn], Dr[nn];
  float fD[nn], fD2[nn], fDq[nn], fDe[nn], fw[n], finvw[n], fxi[n], fxh[n + 1];
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < n; ++m) {
      const double v = (i == m) ? 0.0 : t.D[i * n + m];
      D2[i * n + m] = 2.0 * v;
      Dq[i * n + m] = 0.25 * v;
      De[i * n + m] = 0.125 * v;
      Dr[i * n + m] = (i == m) ? 0.0 : t.D[m * n + i] / t.D[i * n + m];
      fD[i * n + m] = (float)t.D[i * n + m];
      fD2[i * n + m] = (float)D2[i * n + m];
      fDq[i * n + m] = (float)Dq[i * n + m];
      fDe[i * n + m] = (float)De[i * n + m];
    }
  for (int i = 0; i < n; ++i) { fw[i] = (float)t.w[i]; finvw[i] = (float)t.invw[i]; fxi[i] = (float)t.xi[i]; }
  for (int i = 0; i <= n; ++i) fxh[i] = (float)t.xh[i];
  double vp[EO_H * EO_H] = {0.0}, vm[EO_H * EO_H] = {0.0}, fp_[EO_H * EO_H] = {0.0}, fm_[EO_H * EO_H] = {0.0};
  float fvp[EO_H * EO_H] = {0.0f}, fvm[EO_H * EO_H] = {0.0f};
  if (n % 2 == 0)
    for (int i = 0; i < EO_H; ++i)
      for (int m = 0; m < EO_H; ++m) {
        const double a = (i == m) ? 0.0 : t.D[i * n + m], b = (i == N - m) ? 0.0 : t.D[i * n + (N - m)];
        vp[i * EO_H + m] = 0.5 * (a + b);
        vm[i * EO_H + m] = 0.5 * (a - b);
        fvp[i * EO_H + m] = (float)vp[i * EO_H + m];
        fvm[i * EO_H + m] = (float)vm[i * EO_H + m];
        fp_[i * EO_H + m] = 0.5 * (t.D[i * n + m] + t.D[i * n + (N - m)]);
        fm_[i * EO_H + m] = 0.5 * (t.D[i * n + m] - t.D[i * n + (N - m)]);
      }
  double ihx[n];
  float fihx[n];
  ihx[0] = 0.0;
  for (int i = 1; i < n; ++i) ihx[i] = 1.0 / (t.xi[i] - t.xi[i - 1]);
  for (int i = 0; i < n; ++i) fihx[i] = (float)ihx[i];
  cudaError_t err = cudaSuccess;
  err = err ? err : cudaMemcpyToSymbol(c_ihx, ihx, sizeof(double) * n);
  err = err ? err : cudaMemcpyToSymbol(c_VP, vp, sizeof(vp));
  err = err ? err : cudaMemcpyToSymbol(c_VM, vm, sizeof(vm));
  err = err ? err : cudaMemcpyToSymbol(f_VP, fvp, sizeof(fvp));
  err = err ? err : cudaMemcpyToSymbol(f_VM, fvm, sizeof(fvm));
  err = err ? err : cudaMemcpyToSymbol(c_FP, fp_, sizeof(fp_));
  err = err ? err : cudaMemcpyToSymbol(c_FM, fm_, sizeof(fm_));
  err = err ? err : cudaMemcpyToSymbol(f_ihx, fihx, sizeof(float) * n);
  err = err ? err : cudaMemcpyToSymbol(c_D, t.D, sizeof(double) * nn);
  err = err ? err : cudaMemcpyToSymbol(c_D2, D2, sizeof(double) * nn);
  err = err ? err : cudaMemcpyToSymbol(c_Dq, Dq, sizeof(double) * nn);
  err = err ? err : cudaMemcpyToSymbol(c_De, De, sizeof(double) * nn);
  err = err ? err : cudaMemcpyToSymbol(c_Dr, Dr, sizeof(double) * nn);
  err = err ? err : cudaMemcpyToSymbol(c_w, t.w, sizeof(double) * n);
  err = err ? err : cudaMemcpyToSymbol(c_invw, t.invw, sizeof(double) * n);
  err = err ? err : cudaMemcpyToSymbol(c_xi, t.xi, sizeof(double) * n);
  err = err ? err : cudaMemcpyToSymbol(c_xh, t.xh, sizeof(double) * (n + 1));
  err = err ? err : cudaMemcpyToSymbol(c_Vinv, t.Vinv, sizeof(double) * nn);
  err = err ? err : cudaMemcpyToSymbol(f_D, fD, sizeof(float) * nn);
  err = err ? err : cudaMemcpyToSymbol(f_D2, fD2, sizeof(float) * nn);
  err = err ? err : cudaMemcpyToSymbol(f_Dq, fDq, sizeof(float) * nn);
  err = err ? err : cudaMemcpyToSymbol(f_De, fDe, sizeof(float) * nn);
  err = err ? err : cudaMemcpyToSymbol(f_w, fw, sizeof(float) * n);
  err = err ? err : cudaMemcpyToSymbol(f_invw, finvw, sizeof(float) * n);
  err = err ? err : cudaMemcpyToSymbol(f_xi, fxi, sizeof(float) * n);
  err = err ? err : cudaMemcpyToSymbol(f_xh, fxh, sizeof(float) * (n + 1));
  return err;
}

void launch_metrics(const DgDevice &d, cudaStream_t s) {
  const size_t smem = sizeof(double) * 14 * nnn;
  cudaFuncSetAttribute(k_metrics, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_metrics<<<d.nE, 256, smem, s>>>(d);
}

void launch_face_normals(const DgDevice &d, cudaStream_t s) {
  const long long pts = (long long)d.nF * nn;
  k_face_normals<<<(unsigned)((pts + 255) / 256), 256, 0, s>>>(d);
  if (d.precision == 1) k_round_geometry<<<4 * 152, 256, 0, s>>>(d);
}

template <typename R>
void launch_face_t(const DgDevice &d, const double *U, cudaStream_t s) {
  const long long pts = (long long)d.nF * nn;
  const unsigned grid = (unsigned)((pts + 255) / 256);
  switch (d.sflux) {
    case SF_LLF: k_face<R, SF_LLF><<<grid, 256, 0, s>>>(d, U); break;
    case SF_ROE: k_face<R, SF_ROE><<<grid, 256, 0, s>>>(d, U); break;
    default: k_face<R, SF_EC><<<grid, 256, 0, s>>>(d, U); break;
  }
}

void launch_face(const DgDevice &d, const double *U, cudaStream_t s) {
  if (d.precision == 1) launch_face_t<float>(d, U, s);
  else launch_face_t<double>(d, U, s);
}

void launch_lift(const DgDevice &d, const double *U, double *tau, cudaStream_t s) {
  if (TMA_OK && d.precision == 1 && d.use_tma) {  // FP32-bulk: the TMA-fed persistent form
    static int grid_lt = 0;
    if (!grid_lt) {
      cudaFuncSetAttribute(k_lift_f32_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LT_SMEM);
      int dev = 0, sms = 0, per_sm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lift_f32_tma, LT_THREADS, LT_SMEM);
      grid_lt = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int blocks = d.nE < grid_lt ? d.nE : grid_lt;
    k_lift_f32_tma<<<blocks, LT_THREADS, LT_SMEM, s>>>(d);
    return;
  }
  const unsigned grid = (d.nE + LIFT_EPB - 1) / LIFT_EPB;
  if (d.precision == 1) {
    k_lift<float><<<grid, LIFT_THREADS, 0, s>>>(d, U, nullptr);
  } else if (n == 8) {  // measured faster at N = 7 (7.32 -> 7.00 ms at 32^3); slower at N = 5 (+3 %)
    static bool attr_set = false;
    if (!attr_set) {
      cudaFuncSetAttribute(k_lift_lines, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LIFT_LINES_SMEM);
      attr_set = true;
    }
    k_lift_lines<<<grid, LIFT_THREADS, LIFT_LINES_SMEM, s>>>(d, U, tau);
  } else {
    k_lift<double><<<grid, LIFT_THREADS, 0, s>>>(d, U, tau);
  }
}

template <typename R, int VF, bool SC>
void launch_volume_t(const DgDevice &d, const double *U, double *out, double *g, int mode, int first, double dt,
                     double A, double B, cudaStream_t s) {
  const size_t smem =
      sizeof(R) * (VOL_EPB * vol_np<SC>() * PS + VOL_EPB * 15 * PS + (SC ? VOL_EPB * 5 * nnn : 0));
  static bool attr_set = false;  // per instantiation; setting it twice is harmless
  if (!attr_set) {
    cudaFuncSetAttribute(k_volume<R, VF, SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  k_volume<R, VF, SC><<<(d.nE + VOL_EPB - 1) / VOL_EPB, vol_threads<R, SC>(), smem, s>>>(d, U, out, g, mode, first, dt, A,
                                                                                    B);
}

template <int VF>
void launch_volume_f32(const DgDevice &d, const double *U, double *out, double *g, int mode, int first, double dt,
                       double A, double B, cudaStream_t s) {
  const bool aligned = !(((uintptr_t)U | (uintptr_t)out | (uintptr_t)g) & 15u);
  // pair-symmetric line kernel, warp-specialised. Its warp groups trade registers (setmaxnreg), which
  // is only safe if the block is launched with exactly the registers the split assumes; any other
  // compiled count takes the warp-specialised node kernel instead.
  static int grid_ln = 0;  // > 0: usable, < 0: not usable
  if (LN_OK && d.use_tma == 3 && aligned && grid_ln == 0) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k_volume_f32_line<VF>) == cudaSuccess && fa.numRegs == LN_REG_LAUNCH) {
      cudaFuncSetAttribute(k_volume_f32_line<VF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LN_SMEM);
      int dev = 0, sms = 0, per_sm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_volume_f32_line<VF>, LN_THREADS, LN_SMEM);
      grid_ln = per_sm == 1 ? sms : -1;  // one block per SM: the register split needs the whole file
    } else {
      grid_ln = -1;
    }
  }
  if (LN_OK && d.use_tma == 3 && aligned && grid_ln > 0) {
    const int blocks = d.nE < grid_ln ? d.nE : grid_ln;
    k_volume_f32_line<VF><<<blocks, LN_THREADS, LN_SMEM, s>>>(d, U, out, g, mode, first, dt, A, B);
    return;
  }
  if (TMA_OK && d.use_tma >= 2 && aligned) {  // warp-specialised persistent kernel
    static int grid_ws = 0;
    if (!grid_ws) {
      cudaFuncSetAttribute(k_volume_f32_ws<VF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WS_SMEM);
      int dev = 0, sms = 0, per_sm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_volume_f32_ws<VF>, WS_THREADS, WS_SMEM);
      grid_ws = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int blocks = d.nE < grid_ws ? d.nE : grid_ws;
    k_volume_f32_ws<VF><<<blocks, WS_THREADS, WS_SMEM, s>>>(d, U, out, g, mode, first, dt, A, B);
    return;
  }
  if (TMA_OK && d.use_tma && aligned) {
    static int grid = 0;  // persistent: CTAs resident on all SMs at once
    if (!grid) {
      cudaFuncSetAttribute(k_volume_f32_tma<VF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TB_SMEM);
      int dev = 0, sms = 0, per_sm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_volume_f32_tma<VF>, TMA_THREADS, TB_SMEM);
      grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int blocks = d.nE < grid ? d.nE : grid;
    k_volume_f32_tma<VF><<<blocks, TMA_THREADS, TB_SMEM, s>>>(d, U, out, g, mode, first, dt, A, B);
    return;
  }
  const size_t smem = sizeof(float) * NODE_EPB * NODE_SLOTS * nnn;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_volume_f32<VF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  k_volume_f32<VF><<<(d.nE + NODE_EPB - 1) / NODE_EPB, NODE_THREADS, smem, s>>>(d, U, out, g, mode, first, dt, A, B);
}

template <typename R>
void launch_volume_r(const DgDevice &d, const double *U, double *out, double *g, int mode, int first, double dt,
                     double A, double B, cudaStream_t s) {
  const bool sc = d.shock_capturing != 0;
  if (std::is_same<R, float>::value && !sc) {  // FP32-bulk without the blend: node-per-thread kernel
    switch (d.vflux) {
      case VF_KG: launch_volume_f32<VF_KG>(d, U, out, g, mode, first, dt, A, B, s); return;
      case VF_PIR: launch_volume_f32<VF_PIR>(d, U, out, g, mode, first, dt, A, B, s); return;
      case VF_EC: launch_volume_f32<VF_EC>(d, U, out, g, mode, first, dt, A, B, s); return;
      default: launch_volume_f32<VF_CEN>(d, U, out, g, mode, first, dt, A, B, s); return;
    }
  }
  switch (d.vflux) {
    case VF_KG:
      if (sc) launch_volume_t<R, VF_KG, true>(d, U, out, g, mode, first, dt, A, B, s);
      else launch_volume_t<R, VF_KG, false>(d, U, out, g, mode, first, dt, A, B, s);
      break;
    case VF_PIR:
      if (sc) launch_volume_t<R, VF_PIR, true>(d, U, out, g, mode, first, dt, A, B, s);
      else launch_volume_t<R, VF_PIR, false>(d, U, out, g, mode, first, dt, A, B, s);
      break;
    case VF_EC:
      if (sc) launch_volume_t<R, VF_EC, true>(d, U, out, g, mode, first, dt, A, B, s);
      else launch_volume_t<R, VF_EC, false>(d, U, out, g, mode, first, dt, A, B, s);
      break;
    default:
      if (sc) launch_volume_t<R, VF_CEN, true>(d, U, out, g, mode, first, dt, A, B, s);
      else launch_volume_t<R, VF_CEN, false>(d, U, out, g, mode, first, dt, A, B, s);
      break;
  }
}

void launch_volume(const DgDevice &d, const double *U, double *out, double *g, int mode, int first, double dt,
                   double A, double B, cudaStream_t s) {
  if (d.precision == 1) launch_volume_r<float>(d, U, out, g, mode, first, dt, A, B, s);
  else launch_volume_r<double>(d, U, out, g, mode, first, dt, A, B, s);
}

void launch_indicator(const DgDevice &d, const double *U, cudaStream_t s) {
  k_indicator<<<(d.nE + IND_WARPS - 1) / IND_WARPS, 32 * IND_WARPS, 0, s>>>(d, U);
}

void launch_shadow(const DgDevice &d, const double *U, cudaStream_t s) { k_shadow<<<8 * 152, 256, 0, s>>>(d, U); }

void launch_spread(const DgDevice &d, double *alpha_out, cudaStream_t s) {
  k_spread<<<(d.nE + 255) / 256, 256, 0, s>>>(d, alpha_out);
}

void launch_invariants(const DgDevice &d, const double *U, const double *Ut, double *out8, cudaStream_t s) {
  const long long total = (long long)d.nE * nnn;
  int blocks = (int)((total + 255) / 256);
  if (blocks > DG_RED_BLOCKS) blocks = DG_RED_BLOCKS;
  k_invariants<<<blocks, 256, 0, s>>>(d, U, Ut);
  k_reduce_partials<<<1, 32, 0, s>>>(d.red, blocks, 8, 0, out8);
}

void launch_max_dt(const DgDevice &d, const double *U, double *out, cudaStream_t s) {
  const long long total = (long long)d.nE * nnn;
  int blocks = (int)((total + 255) / 256);
  if (blocks > DG_RED_BLOCKS) blocks = DG_RED_BLOCKS;
  k_max_dt<<<blocks, 256, 0, s>>>(d, U);
  k_reduce_partials<<<1, 32, 0, s>>>(d.red, blocks, 1, 1, out);
}

}  // namespace
