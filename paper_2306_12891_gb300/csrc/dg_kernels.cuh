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
// computed in FP64 (the kernels read an FP32 rounding of Ja), and the 1/J scaling and the LSERK
// update stay FP64. In FP32 the state is carried with E' = E - p_ref/(gamma-1) so that the
// pressure p' = p - p_ref is formed from O(1) numbers; the momentum flux uses p' throughout
// (volume, surface and subcell fluxes). The constant p_ref part of that flux contributes
// p_ref times the discrete metric identity sum_d D_d Ja^d, which is zero, so the shift is exact.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "dg_convert.cuh"
#include "dg_internal.h"
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
__constant__ double c_w[n], c_invw[n], c_xi[n], c_xh[n + 1];
__constant__ double c_Vinv[nn];
__constant__ float f_D[nn], f_D2[nn], f_Dq[nn], f_De[nn];
__constant__ float f_w[n], f_invw[n], f_xi[n], f_xh[n + 1];

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
};

// per-context constants in the arithmetic type (precomputed on the host)
template <typename R> struct Cst;
template <> struct Cst<double> {
  static __device__ __forceinline__ double gam(const DgDevice &d) { return d.gamma; }
  static __device__ __forceinline__ double gm1(const DgDevice &d) { return d.gm1; }
  static __device__ __forceinline__ double iR(const DgDevice &d) { return d.iR; }
  static __device__ __forceinline__ double pref(const DgDevice &d) { return d.p_ref; }
  static __device__ __forceinline__ double href(const DgDevice &d) { return d.href; }
  static __device__ __forceinline__ double mu(const DgDevice &d) { return d.mu; }
  static __device__ __forceinline__ double kappa(const DgDevice &d) { return d.kappa; }
};
template <> struct Cst<float> {
  static __device__ __forceinline__ float gam(const DgDevice &d) { return d.gamma_f; }
  static __device__ __forceinline__ float gm1(const DgDevice &d) { return d.gm1_f; }
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

// Euler flux through the (unit or metric) vector a; returns u.a and the true pressure p
template <typename R>
__device__ __forceinline__ void euler_flux_n(const R U[5], R gam, R pref, R href, const R a[3], R F[5], R &un, R &p) {
  const R ir = R(1) / U[0];
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

// Riemann flux F*(UL, UR, nv) for a unit normal nv
template <typename R>
__device__ __forceinline__ void riemann(int sf, const R UL[5], const R UR[5], const R nv[3], R gam, R pref, R href,
                                        R F[5]) {
  const R gm1 = gam - R(1);
  if (sf == SF_EC) {
    const R irL = R(1) / UL[0], irR = R(1) / UR[0];
    const R uL = UL[1] * irL, vL = UL[2] * irL, wL = UL[3] * irL;
    const R uR = UR[1] * irR, vR = UR[2] * irR, wR = UR[3] * irR;
    const R pL = gm1 * (UL[4] - R(0.5) * (UL[1] * uL + UL[2] * vL + UL[3] * wL)) + (kShift<R> ? pref : R(0));
    const R pR = gm1 * (UR[4] - R(0.5) * (UR[1] * uR + UR[2] * vR + UR[3] * wR)) + (kShift<R> ? pref : R(0));
    ec_flux<R>(UL[0], uL, vL, wL, pL, UR[0], uR, vR, wR, pR, nv, gam, kShift<R> ? pref : R(0), F);
    return;
  }
  R FL[5], FR[5], unL, unR, pL, pR;
  euler_flux_n<R>(UL, gam, pref, href, nv, FL, unL, pL);
  euler_flux_n<R>(UR, gam, pref, href, nv, FR, unR, pR);
  if (sf == SF_LLF) {
    const R cL = sqrt(gam * pL / UL[0]), cR = sqrt(gam * pR / UR[0]);
    const R lam = fmax(fabs(unL) + cL, fabs(unR) + cR);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = R(0.5) * (FL[v] + FR[v] - lam * (UR[v] - UL[v]));
    return;
  }
  // Roe: sqrt(rho)-weighted average state, three wave families, no entropy fix
  const R sL = sqrt(UL[0]), sR = sqrt(UR[0]);
  const R iw = R(1) / (sL + sR);
  const R irL = R(1) / UL[0], irR = R(1) / UR[0];
  const R uL = UL[1] * irL, vL = UL[2] * irL, wL = UL[3] * irL;
  const R uR = UR[1] * irR, vR = UR[2] * irR, wR = UR[3] * irR;
  const R ut = (sL * uL + sR * uR) * iw, vt = (sL * vL + sR * vR) * iw, wt = (sL * wL + sR * wR) * iw;
  const R EpL = kShift<R> ? UL[4] + pL - pref + href : UL[4] + pL;  // E + p
  const R EpR = kShift<R> ? UR[4] + pR - pref + href : UR[4] + pR;
  const R Ht = (sL * EpL * irL + sR * EpR * irR) * iw;
  const R q2 = ut * ut + vt * vt + wt * wt;
  const R c2 = gm1 * (Ht - R(0.5) * q2);
  const R ct = sqrt(c2), ic2 = R(1) / c2;
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
  R D[5];
  D[0] = l1a1 + l5a5 + l2a2;
  D[1] = l1a1 * (ut - ct * nv[0]) + l5a5 * (ut + ct * nv[0]) + l2a2 * ut + l2r * dut;
  D[2] = l1a1 * (vt - ct * nv[1]) + l5a5 * (vt + ct * nv[1]) + l2a2 * vt + l2r * dvt;
  D[3] = l1a1 * (wt - ct * nv[2]) + l5a5 * (wt + ct * nv[2]) + l2a2 * wt + l2r * dwt;
  D[4] = l1a1 * (Ht - unt * ct) + l5a5 * (Ht + unt * ct) + l2a2 * R(0.5) * q2 + l2r * (ut * dut + vt * dvt + wt * dwt);
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = R(0.5) * (FL[v] + FR[v] - D[v]);
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
  R Fs[5];
  riemann<R>(SF, UL, UR, nv, gam, pref, href, Fs);
  R *oL = Buf<R>::Fsurf(d) + ((size_t)eL * 6 + fL) * 5 * nn;
  R *oR = Buf<R>::Fsurf(d) + ((size_t)eR * 6 + fR) * 5 * nn;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    oL[v * nn + pq] = s * Fs[v];
    oR[v * nn + pqR] = -s * Fs[v];
  }
  if (d.equations == 1) {
    const R irL = R(1) / UL[0], irR = R(1) / UR[0];
    const R wL[3] = {UL[1] * irL, UL[2] * irL, UL[3] * irL};
    const R wR[3] = {UR[1] * irR, UR[2] * irR, UR[3] * irR};
    const R gm1 = gam - R(1);
    R pL = gm1 * (UL[4] - R(0.5) * (UL[1] * wL[0] + UL[2] * wL[1] + UL[3] * wL[2]));
    R pR = gm1 * (UR[4] - R(0.5) * (UR[1] * wR[0] + UR[2] * wR[1] + UR[3] * wR[2]));
    if (kShift<R>) { pL += pref; pR += pref; }
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
// iJ this node's 1/J; writes the element's Fv [3 d][4][nnn] at `node` (out = the element's Fv)
template <typename R>
__device__ __forceinline__ void lift_node(const DgDevice &d, int node, const R *__restrict__ W,
                                          const R (*__restrict__ sD)[n + 1], const R *__restrict__ Jae,
                                          const R *__restrict__ Wse, R iJ, R mu, R kappa, R *__restrict__ out) {
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
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      R s = R(0);
#pragma unroll
      for (int m = 0; m < n; ++m) s += sD[id][m] * W[q * nnn + base + m * st];
      g[q][0] += Ja[dd][0] * s;
      g[q][1] += Ja[dd][1] * s;
      g[q][2] += Ja[dd][2] * s;
    }
    // surface terms on the faces of direction dd through this node
    if (id == 0 || id == N) {
      const int f = 2 * dd + (id == N ? 1 : 0);
      const R sc = (id == N ? R(1) : R(-1)) * Tab<R>::invw(id);
      const int pp = dd == 0 ? ijk[1] : ijk[0];
      const int qq = dd == 2 ? ijk[1] : ijk[2];
      const R *js = Wse + f * 4 * nn + pp + n * qq;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const R jq = sc * js[q * nn];
        g[q][0] += Ja[dd][0] * jq;
        g[q][1] += Ja[dd][1] * jq;
        g[q][2] += Ja[dd][2] * jq;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) { g[q][0] *= iJ; g[q][1] *= iJ; g[q][2] *= iJ; }
  // Navier-Stokes-Fourier flux in Cartesian direction c: (tau_xc, tau_yc, tau_zc, u.tau_c + kappa dT/dx_c)
  const R u = W[node], v = W[nnn + node], w = W[2 * nnn + node];
  const R div = g[0][0] + g[1][1] + g[2][2];
  const R t23 = R(2.0 / 3.0) * mu * div;
  const R txx = R(2) * mu * g[0][0] - t23, tyy = R(2) * mu * g[1][1] - t23, tzz = R(2) * mu * g[2][2] - t23;
  const R txy = mu * (g[0][1] + g[1][0]), txz = mu * (g[0][2] + g[2][0]), tyz = mu * (g[1][2] + g[2][1]);
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
__global__ void __launch_bounds__(LIFT_THREADS, lift_min_blocks<R>()) k_lift(const DgDevice d, const double *__restrict__ U) {
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
                 Buf<R>::Wsurf(d) + (size_t)e * 6 * 4 * nn, iJ, mu, kappa, Buf<R>::Fv(d) + (size_t)e * 12 * nnn);
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
    const R hb = R(1) / (Tab<R>::xi(i) - Tab<R>::xi(i - 1)), hf = R(1) / (Tab<R>::xi(i + 1) - Tab<R>::xi(i));
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
__device__ __forceinline__ void cons_of(const R q[5], R gm1, R U[5]) {
  U[0] = q[0]; U[1] = q[0] * q[1]; U[2] = q[0] * q[2]; U[3] = q[0] * q[3];
  U[4] = q[4] / gm1 + R(0.5) * q[0] * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
}

// FV subcell operator along one line (Sec. 4.1): Riemann fluxes at the N interior subcell
// interfaces with telescoped interface metrics a_{i+1/2} = a_{i-1/2} + w_i (D Ja)_i, the DG surface
// fluxes at the element faces, and Ac_i = (f_{i+1/2} - f_{i-1/2}) / w_i written to shared memory.
template <typename R>
__device__ __forceinline__ void line_fv(const R *__restrict__ P, int pb, int ps, const R *__restrict__ Jd, int gb,
                                        int gs, const R *Fm, const R *Fp, int sf, R gam, R pref, R href,
                                        R *__restrict__ Ac) {
  const R gm1 = gam - R(1);
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
      const R s = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      const R is = R(1) / s;
      const R nv[3] = {a[0] * is, a[1] * is, a[2] * is};
      R UL[5], UR[5], Fs[5];
      cons_of<R>(qRi, gm1, UL);
      cons_of<R>(qLn, gm1, UR);
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
    line_fluxdiff<R, VF>(P + le * NP * PS, pb, ps, Jab + ((size_t)e * 3 + dir) * 3 * nnn, gb, gs, gam, pref,
                         Acc + (le * 3 + dir) * 5 * PS);
    // viscous divergence joins the line sums, except under the blend (which must not weight it)
    if (!SC && d.equations == 1)
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
      line_fv<R>(P + le * NP * PS, pb, ps, Jab + ((size_t)e * 3 + dir) * 3 * nnn, gb, gs, Fm, Fp, d.sflux, gam, pref,
                 href, Acc + (le * 3 + dir) * 5 * PS);
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
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double ut = miJ * to_double(s[v]);
        const double gv = first ? dt * ut : A * g[gi + v * nnn] + dt * ut;
        g[gi + v * nnn] = gv;
        const double un = U[gi + v * nnn] + B * gv;
        out[gi + v * nnn] = un;
        if (kShift<R>) d.Uf[gi + v * nnn] = (float)(v == 4 ? un - eref : un);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// FP32-bulk volume kernel without the blend: one thread per node. FP32 flux arithmetic is cheap on
// this GPU, so the pair symmetry that halves the FP64 work is given up here: each thread forms
// all 3(n-1) two-point fluxes of its node's lines and keeps its sums in registers, which removes
// the partner accumulators and two block barriers of the line-per-thread layout, and the metric
// terms are staged in shared memory with the primitives (one coalesced load per element).
// ---------------------------------------------------------------------------------------------
constexpr int NODE_EPB = nnn >= 256 ? 1 : 256 / nnn;
constexpr int NODE_THREADS = round32(NODE_EPB * nnn);
constexpr int NODE_SLOTS = 7 + 9 + 12;  // staged primitives, metric terms, contravariant viscous flux


// scaled two-point flux of the staged nodes a and b through the metric sums Sj (see line_fluxdiff);
// P holds the staged quantities [7][nnn] (node index, no padding)
template <int VF>
__device__ __forceinline__ void pair_flux_f(const float *__restrict__ P, int a, int b, float Sjx, float Sjy,
                                            float Sjz, float gam, float pref, float F[5]) {
  const float ri = P[a], ui = P[nnn + a], vi = P[2 * nnn + a], wi = P[3 * nnn + a];
  const float rm = P[b], um = P[nnn + b], vm = P[2 * nnn + b], wm = P[3 * nnn + b];
  if (VF == VF_PIR || VF == VF_KG) {
    const float Su = ui + um, Sv = vi + vm, Sw = wi + wm;
    const float Vp = Su * Sjx + Sv * Sjy + Sw * Sjz;
    F[0] = (ri + rm) * Vp;
    const float Sp = P[4 * nnn + a] + P[4 * nnn + b];
    F[1] = F[0] * Su + Sp * Sjx;
    F[2] = F[0] * Sv + Sp * Sjy;
    F[3] = F[0] * Sw + Sp * Sjz;
    if (VF == VF_PIR) F[4] = F[0] * (P[5 * nnn + a] + P[5 * nnn + b]);
    else F[4] = F[0] * (P[5 * nnn + a] + P[5 * nnn + b]) + (P[6 * nnn + a] + P[6 * nnn + b]) * Vp;
  } else {
    const float av[3] = {0.5f * Sjx, 0.5f * Sjy, 0.5f * Sjz};
    if (VF == VF_EC) {
      ec_flux<float>(ri, ui, vi, wi, P[6 * nnn + a], rm, um, vm, wm, P[6 * nnn + b], av, gam, pref, F);
    } else {
      const float Vi = ui * av[0] + vi * av[1] + wi * av[2], Vm = um * av[0] + vm * av[1] + wm * av[2];
      const float pm2 = 0.125f * (P[4 * nnn + a] + P[4 * nnn + b]);
      F[0] = 0.5f * (ri * Vi + rm * Vm);
      F[1] = 0.5f * (ri * ui * Vi + rm * um * Vm) + pm2 * av[0];
      F[2] = 0.5f * (ri * vi * Vi + rm * vm * Vm) + pm2 * av[1];
      F[3] = 0.5f * (ri * wi * Vi + rm * wm * Vm) + pm2 * av[2];
      F[4] = 0.5f * (P[5 * nnn + a] * Vi + P[5 * nnn + b] * Vm);
    }
  }
}

// staged quantities of one node (rho, u, v, w, 4p', X, Y; see k_volume) from its FP32 shadow state;
// Pn points at the node's entry of P [7][nnn]
template <int VF>
__device__ __forceinline__ void f32_stage(const DgDevice &d, const float Uv[5], float *Pn) {
  const float gm1 = d.gm1_f, pref = d.p_ref_f;
  const float r = Uv[0], ir = 1.0f / r;
  const float u = Uv[1] * ir, v = Uv[2] * ir, w = Uv[3] * ir;
  const float pm = gm1 * (Uv[4] - 0.5f * (Uv[1] * u + Uv[2] * v + Uv[3] * w));
  const float p = pm + pref;
  const float Et = Uv[4] + (float)d.eref;
  if (!(r > 0.0f) || !(p > 0.0f) || !isfinite(Uv[4])) flag_set(d.flag, 1);
  Pn[0] = r; Pn[nnn] = u; Pn[2 * nnn] = v; Pn[3 * nnn] = w; Pn[4 * nnn] = 4.0f * pm;
  if (VF == VF_PIR) Pn[5 * nnn] = (Et + p) * ir;
  else if (VF == VF_KG) { Pn[5 * nnn] = Et * ir; Pn[6 * nnn] = 2.0f * p; }
  else if (VF == VF_EC) Pn[6 * nnn] = p;
  else Pn[5 * nnn] = Et + p;
}

// D_im with a zero diagonal, rows padded to n + 1 floats, in shared memory: the node-per-thread
// kernels index it by the thread's own node, which would serialise a constant-memory load
constexpr int DZ_STRIDE = n + 1;
__device__ __forceinline__ void fill_dz(float *Dz, int tid, int nthreads) {
  for (int t = tid; t < nn; t += nthreads) Dz[(t / n) * DZ_STRIDE + t % n] = 0.5f * f_D2[t];  // exact
}

// the node's flux differencing, surface terms and (Navier-Stokes) viscous divergence with the
// neighbour's or the wall's viscous trace, summed into s. P [7][nnn], J [9][nnn] (slot 3d + c),
// F [12][nnn] (contravariant viscous flux of this element) staged; Fs = this element's face slots
// [6][5][nn] (shared or global memory); Dz from fill_dz.
// The line sums skip the zero diagonal (partner m = mm or mm + 1) and take D itself; the split-form
// scalings D/4 (mass), D/8 (momentum, energy) or 2D (EC, central) are powers of two, applied once at
// the end, so the flux-differencing sums are those of the scaled tables bit for bit.
template <int VF>
__device__ __forceinline__ void f32_node_terms(const DgDevice &d, const float *__restrict__ P,
                                               const float *__restrict__ J, const float *__restrict__ F,
                                               const float *__restrict__ Fs, const float *__restrict__ Dz,
                                               int e, int node, float s[5]) {
  const float gam = d.gamma_f, pref = d.p_ref_f;
  const bool ns = d.equations == 1;
  const int ijk[3] = {node % n, (node / n) % n, node / nn};
  float a[5];  // flux differencing with D
#pragma unroll
  for (int v = 0; v < 5; ++v) a[v] = s[v] = 0.0f;
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    const int id = ijk[dd];
    const int st = dd == 0 ? 1 : dd == 1 ? n : nn;
    const int base = node - id * st;
    const float *Dr = Dz + id * DZ_STRIDE;
    const float *Fvd = F + (dd * 4) * nnn;
    const float jx = J[(3 * dd) * nnn + node], jy = J[(3 * dd + 1) * nnn + node], jz = J[(3 * dd + 2) * nnn + node];
    float vq[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int mm = 0; mm < N; ++mm) {
      const int m = mm + (mm >= id ? 1 : 0);
      const int am = base + m * st;
      const float c = Dr[m];
      float Fp[5];
      pair_flux_f<VF>(P, node, am, jx + J[(3 * dd) * nnn + am], jy + J[(3 * dd + 1) * nnn + am],
                      jz + J[(3 * dd + 2) * nnn + am], gam, pref, Fp);
#pragma unroll
      for (int v = 0; v < 5; ++v) a[v] += c * Fp[v];
      if (ns) {  // viscous divergence along the line
#pragma unroll
        for (int q = 0; q < 4; ++q) vq[q] += c * Fvd[q * nnn + am];
      }
    }
    const bool face = id == 0 || id == N;
    const int f = 2 * dd + (id == N ? 1 : 0);
    const int pp = dd == 0 ? ijk[1] : ijk[0], qq = dd == 2 ? ijk[1] : ijk[2];
    const float iw = id == 0 ? f_invw[0] : f_invw[N];  // two uniform constant loads
    if (face) {  // surface term: (1/w_b) times the outward face flux
      const float *fs = Fs + f * 5 * nn + pp + n * qq;
#pragma unroll
      for (int v = 0; v < 5; ++v) s[v] += iw * fs[v * nn];
    }
    if (ns) {
#pragma unroll
      for (int q = 0; q < 4; ++q) s[1 + q] -= vq[q];
      // the neighbour's outward normal viscous flux -(1/(2 w_b)) phi_nb at the element faces
      if (face) {
        const int *ef = d.ef + ((size_t)e * 6 + f) * 4;
        const int nb = ef[0], fnb = ef[1], o = ef[2];
        if (nb < 0) {  // wall-model flux: (1/w_b) (F*_wall - (+-) Fv_own / 2), see k_volume
          const float *fw = d.Fwall_f + (size_t)ef[3] * 4 * nn + pp + n * qq;
          const float hs = (id == N) ? 0.5f : -0.5f;
#pragma unroll
          for (int q = 0; q < 4; ++q) s[1 + q] -= iw * (fw[q * nn] - hs * F[(dd * 4 + q) * nnn + node]);
        } else {
          int p2, q2;
          orient_map(o, pp, qq, p2, q2);
          const int nbnode = face_node(fnb, p2, q2);
          const float sg = (fnb & 1) ? 0.5f : -0.5f;
          const float *Fvn = d.Fv_f + ((size_t)nb * 12 + (fnb >> 1) * 4) * nnn + nbnode;
#pragma unroll
          for (int q = 0; q < 4; ++q) s[1 + q] += iw * sg * Fvn[q * nnn];
        }
      }
    }
  }
  if (VF == VF_PIR || VF == VF_KG) {
    s[0] += 0.25f * a[0];
#pragma unroll
    for (int v = 1; v < 5; ++v) s[v] += 0.125f * a[v];
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) s[v] += 2.0f * a[v];
  }
}

// -1/J and the output / LSERK(5,4) stage in FP64 for one node; Ue, ge point at this element's state
// and register slices [5][nnn] to read (shared or global memory), out and g are global
__device__ __forceinline__ void f32_finish_reg(const DgDevice &d, const double Uv[5], const double gv0[5],
                                               double iJ, double *out, double *__restrict__ g, int e, int node,
                                               const float s[5], int mode, int first, double dt, double A,
                                               double B) {
  // Uv, gv0, iJ: this node's U, g and 1/J.
  // The right-hand side -s/J, or the stage increment dt (-1/J) s, is one FP32 product of the FP32 sum
  // s with the factor -1/J or dt (-1/J), formed in FP64 and rounded once (GB300 issues FP64 at 1/64
  // of the FP32 rate, and this epilogue bounds the kernel); the LSERK register and the state
  // accumulate in FP64. Explicit roundings (no compiler contraction) keep every kernel variant's bits.
  const double miJ = -iJ;
  const size_t gi = (size_t)e * 5 * nnn + node;
  if (mode == 0) {
    const float c = d2f_int(miJ);
#pragma unroll
    for (int v = 0; v < 5; ++v) out[gi + v * nnn] = f2d_int(__fmul_rn(s[v], c));
    return;
  }
  const float c = d2f_int(__dmul_rn(dt, miJ));
  const double eref = d.eref;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double du = f2d_int(__fmul_rn(s[v], c));
    const double gv = first ? du : __fma_rn(A, gv0[v], du);
    g[gi + v * nnn] = gv;
    const double un = __fma_rn(B, gv, Uv[v]);
    out[gi + v * nnn] = un;
    d.Uf[gi + v * nnn] = d2f_int(v == 4 ? __dsub_rn(un, eref) : un);
  }
}

// the same with this element's U, g and 1/J read from global memory or a shared-memory copy
__device__ __forceinline__ void f32_finish(const DgDevice &d, const double *Ue, const double *ge,
                                           const double *iJe, double *out, double *__restrict__ g, int e,
                                           int node, const float s[5], int mode, int first, double dt,
                                           double A, double B) {
  double Uv[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, gv0[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (mode == 1) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      Uv[v] = Ue[node + v * nnn];
      if (!first) gv0[v] = ge[node + v * nnn];
    }
  }
  f32_finish_reg(d, Uv, gv0, iJe[node], out, g, e, node, s, mode, first, dt, A, B);
}

template <int VF>
__global__ void __launch_bounds__(NODE_THREADS, 2) k_volume_f32(const DgDevice d, const double *U, double *out,
                                                                 double *__restrict__ g, int mode, int first,
                                                                 double dt, double A, double B) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float *P = reinterpret_cast<float *>(sm_raw);  // [EPB][7][nnn] staged primitives
  float *JS = P + NODE_EPB * 7 * nnn;            // [EPB][9][nnn] metric terms Ja^d_c, slot 3d + c
  float *FS = JS + NODE_EPB * 9 * nnn;           // [EPB][12][nnn] contravariant viscous flux (NS)
  __shared__ float s_Dz[n * DZ_STRIDE];
  fill_dz(s_Dz, threadIdx.x, blockDim.x);
  const int e0 = blockIdx.x * NODE_EPB;
  for (int t = threadIdx.x; t < NODE_EPB * nnn; t += blockDim.x) {
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    float Uv[5];
    load_state<float>(d, U, e, node, Uv);
    f32_stage<VF>(d, Uv, P + le * 7 * nnn + node);
    const float *Jn = d.Jaf + (size_t)e * 9 * nnn + node;
    float *Je = JS + le * 9 * nnn + node;
#pragma unroll
    for (int k = 0; k < 9; ++k) Je[k * nnn] = Jn[k * nnn];
    if (d.equations == 1) {
      const float *Fn = d.Fv_f + (size_t)e * 12 * nnn + node;
      float *Fe = FS + le * 12 * nnn + node;
#pragma unroll
      for (int k = 0; k < 12; ++k) Fe[k * nnn] = Fn[k * nnn];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NODE_EPB * nnn; t += blockDim.x) {
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    float s[5];
    f32_node_terms<VF>(d, P + le * 7 * nnn, JS + le * 9 * nnn, FS + le * 12 * nnn,
                       d.Fsurf_f + (size_t)e * 6 * 5 * nn, s_Dz, e, node, s);
    const size_t ge0 = (size_t)e * 5 * nnn;
    f32_finish(d, U + ge0, g + ge0, d.invJ + (size_t)e * nnn, out, g, e, node, s, mode, first, dt, A, B);
  }
}

// ---------------------------------------------------------------------------------------------
// The same FP32-bulk volume operator as a persistent kernel fed by TMA bulk copies: one CTA per SM
// (or two) walks its elements; each element's contiguous slices -- FP32 state, metric terms,
// viscous flux, face slots and the FP64 state and LSERK register -- are copied into shared memory
// with cp.async.bulk one element ahead (double buffer, one mbarrier per buffer), so the next
// element's loads overlap this element's arithmetic. Needs element slices that are multiples of
// 16 bytes (N = 3, 5, 7) and 16-byte aligned U, g and output.
// ---------------------------------------------------------------------------------------------
constexpr bool TMA_OK = (N == 3 || N == 5 || N == 7);
constexpr int TMA_THREADS = round32(nnn);
constexpr unsigned TB_UF = 5u * nnn * 4u, TB_JA = 9u * nnn * 4u, TB_FV = 12u * nnn * 4u, TB_FS = 30u * nn * 4u;
constexpr unsigned TB_U = 5u * nnn * 8u, TB_G = 5u * nnn * 8u, TB_IJ = nnn * 8u;
constexpr unsigned TB_BUF = TB_UF + TB_JA + TB_FV + TB_FS + TB_U + TB_G + TB_IJ;
constexpr unsigned TB_P = 7u * nnn * 4u;
constexpr unsigned TB_SMEM = 2u * TB_BUF + TB_P + 16u;
static_assert(!TMA_OK || (TB_UF % 16 == 0 && TB_JA % 16 == 0 && TB_FV % 16 == 0 && TB_FS % 16 == 0 &&
                          TB_U % 16 == 0 && TB_IJ % 16 == 0 && TB_P % 16 == 0), "TMA slices must be multiples of 16 bytes");
static_assert(!TMA_OK || TB_SMEM <= 232448, "TMA kernel exceeds the shared memory of one CTA");

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// wait for the phase with the given parity, giving up after ~2^31 clock cycles (about a second)
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  while (true) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

template <int VF>
__global__ void __launch_bounds__(TMA_THREADS, 1) k_volume_f32_tma(const DgDevice d, const double *U, double *out,
                                                                    double *g, int mode, int first, double dt,
                                                                    double A, double B) {
  extern __shared__ __align__(128) unsigned char sm_tma[];
  float *P = reinterpret_cast<float *>(sm_tma + 2 * TB_BUF);
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(sm_tma + 2 * TB_BUF + TB_P);
  __shared__ int s_ok;
  __shared__ float s_Dz[n * DZ_STRIDE];
  const bool ns = d.equations == 1;
  const bool needU = mode == 1, needG = mode == 1 && !first;
  const unsigned bytes =
      TB_UF + TB_JA + TB_FS + TB_IJ + (ns ? TB_FV : 0u) + (needU ? TB_U : 0u) + (needG ? TB_G : 0u);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(smem_addr(&bar[0]));
    mbar_init(smem_addr(&bar[1]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fill_dz(s_Dz, tid, blockDim.x);
  __syncthreads();
  // copies of element group k into buffer k & 1 (thread 0)
  auto issue = [&](int k) {
    const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
    if (e >= d.nE) return;
    unsigned char *b = sm_tma + (k & 1) * TB_BUF;
    const unsigned mb = smem_addr(&bar[k & 1]);
    mbar_expect_tx(mb, bytes);
    bulk_g2s(smem_addr(b), d.Uf + e * 5 * nnn, TB_UF, mb);
    bulk_g2s(smem_addr(b + TB_UF), d.Jaf + e * 9 * nnn, TB_JA, mb);
    if (ns) bulk_g2s(smem_addr(b + TB_UF + TB_JA), d.Fv_f + e * 12 * nnn, TB_FV, mb);
    bulk_g2s(smem_addr(b + TB_UF + TB_JA + TB_FV), d.Fsurf_f + e * 30 * nn, TB_FS, mb);
    if (needU) bulk_g2s(smem_addr(b + TB_UF + TB_JA + TB_FV + TB_FS), U + e * 5 * nnn, TB_U, mb);
    if (needG) bulk_g2s(smem_addr(b + TB_UF + TB_JA + TB_FV + TB_FS + TB_U), g + e * 5 * nnn, TB_G, mb);
    bulk_g2s(smem_addr(b + TB_UF + TB_JA + TB_FV + TB_FS + TB_U + TB_G), d.invJ + e * nnn, TB_IJ, mb);
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }
  for (int k = 0;; ++k) {
    const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
    if (e >= d.nE) break;
    const unsigned mb = smem_addr(&bar[k & 1]), parity = (unsigned)((k >> 1) & 1);
    if (tid == 0) s_ok = mbar_wait(mb, parity) ? 1 : 0;
    __syncthreads();
    if (!s_ok) {  // a copy never completed: report, wait (bounded) for the other buffer's copy, stop
      if (tid == 0) {
        flag_set(d.flag, 4);
        if (e + gridDim.x < d.nE) mbar_wait(smem_addr(&bar[(k + 1) & 1]), (unsigned)(((k + 1) >> 1) & 1));
      }
      return;
    }
    mbar_wait(mb, parity);  // completed: returns at once and orders this thread's reads after the copy
    const unsigned char *b = sm_tma + (k & 1) * TB_BUF;
    const float *Uf = reinterpret_cast<const float *>(b);
    const float *Jb = reinterpret_cast<const float *>(b + TB_UF);
    const float *Fb = reinterpret_cast<const float *>(b + TB_UF + TB_JA);
    const float *Sb = reinterpret_cast<const float *>(b + TB_UF + TB_JA + TB_FV);
    const double *Ub = reinterpret_cast<const double *>(b + TB_UF + TB_JA + TB_FV + TB_FS);
    const double *Gb = reinterpret_cast<const double *>(b + TB_UF + TB_JA + TB_FV + TB_FS + TB_U);
    const double *Ib = reinterpret_cast<const double *>(b + TB_UF + TB_JA + TB_FV + TB_FS + TB_U + TB_G);
    if (tid < nnn) {
      const float Uv[5] = {Uf[tid], Uf[nnn + tid], Uf[2 * nnn + tid], Uf[3 * nnn + tid], Uf[4 * nnn + tid]};
      f32_stage<VF>(d, Uv, P + tid);
    }
    __syncthreads();
    if (tid < nnn) {
      float s[5];
      f32_node_terms<VF>(d, P, Jb, Fb, Sb, s_Dz, (int)e, tid, s);
      f32_finish(d, Ub, Gb, Ib, out, g, (int)e, tid, s, mode, first, dt, A, B);
    }
    __syncthreads();  // buffer k & 1 and P are free again
    if (tid == 0) issue(k + 2);
  }
}

// ---------------------------------------------------------------------------------------------
// Warp-specialised form of the TMA kernel: 16 compute warps stage the primitives and form the
// per-node sums of element k while 4 epilogue warps apply -1/J and the FP64 LSERK update to element
// k-1, so the FP64 epilogue overlaps the FP32 flux arithmetic instead of following it. The sums
// pass through shared memory (two buffers); hand-offs use mbarriers: full[b] (the compute threads
// arrive when sums are written) and empty[b] (the epilogue threads arrive when they are consumed).
// Every wait is bounded; the compute warps leave their loop together after a block-level barrier
// among themselves.
// ---------------------------------------------------------------------------------------------
constexpr int WS_COMPUTE = TMA_THREADS;
constexpr int WS_EPI = 128;
constexpr int WS_THREADS = WS_COMPUTE + WS_EPI;
constexpr unsigned WS_CBUF = TB_UF + TB_JA + TB_FV + TB_FS;  // per-element TMA slices (no U, g)
constexpr unsigned WS_S = 5u * nnn * 4u;                      // per-node sums of one element
constexpr unsigned WS_UG = TB_U + TB_G + TB_IJ;              // FP64 state, register and 1/J of one element
constexpr unsigned WS_SMEM = 2u * WS_CBUF + TB_P + 2u * WS_S + WS_UG + 64u;
static_assert(!TMA_OK || WS_SMEM <= 232448, "warp-specialised kernel exceeds the shared memory of one CTA");

__device__ __forceinline__ void mbar_init_n(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int VF>
__global__ void __launch_bounds__(WS_THREADS, 1) k_volume_f32_ws(const DgDevice d, const double *U, double *out,
                                                                  double *g, int mode, int first, double dt,
                                                                  double A, double B) {
  extern __shared__ __align__(128) unsigned char sm_tma[];
  float *P = reinterpret_cast<float *>(sm_tma + 2 * WS_CBUF);
  float *S = reinterpret_cast<float *>(sm_tma + 2 * WS_CBUF + TB_P);  // [2][5][nnn]
  unsigned char *UG = sm_tma + 2 * WS_CBUF + TB_P + 2 * WS_S;  // U [5][nnn], g [5][nnn], 1/J [nnn] (FP64)
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(UG + WS_UG);
  // bar[0..1]: TMA arrival per buffer; bar[2..3]: sums full; bar[4..5]: sums empty; bar[6]: U, g arrival
  __shared__ int s_abort, s_abort_e;
  __shared__ float s_Dz[n * DZ_STRIDE];
  const bool ns = d.equations == 1;
  const unsigned bytes = TB_UF + TB_JA + TB_FS + (ns ? TB_FV : 0u);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(smem_addr(&bar[0]));
    mbar_init(smem_addr(&bar[1]));
    mbar_init_n(smem_addr(&bar[2]), WS_COMPUTE);
    mbar_init_n(smem_addr(&bar[3]), WS_COMPUTE);
    mbar_init_n(smem_addr(&bar[4]), WS_EPI);
    mbar_init_n(smem_addr(&bar[5]), WS_EPI);
    mbar_init(smem_addr(&bar[6]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    s_abort_e = 0;
  }
  fill_dz(s_Dz, tid, blockDim.x);
  __syncthreads();
  auto issue = [&](int k) {
    const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
    if (e >= d.nE) return;
    unsigned char *b = sm_tma + (k & 1) * WS_CBUF;
    const unsigned mb = smem_addr(&bar[k & 1]);
    mbar_expect_tx(mb, bytes);
    bulk_g2s(smem_addr(b), d.Uf + e * 5 * nnn, TB_UF, mb);
    bulk_g2s(smem_addr(b + TB_UF), d.Jaf + e * 9 * nnn, TB_JA, mb);
    if (ns) bulk_g2s(smem_addr(b + TB_UF + TB_JA), d.Fv_f + e * 12 * nnn, TB_FV, mb);
    bulk_g2s(smem_addr(b + TB_UF + TB_JA + TB_FV), d.Fsurf_f + e * 30 * nn, TB_FS, mb);
  };
  if (tid < WS_COMPUTE) {
    if (tid == 0) {
      issue(0);
      issue(1);
    }
    int k = 0;
    for (;; ++k) {
      const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
      if (e >= d.nE) break;
      const int b = k & 1;
      const unsigned parity = (unsigned)((k >> 1) & 1);
      if (!mbar_wait(smem_addr(&bar[b]), parity)) s_abort = 1;
      const unsigned char *buf = sm_tma + b * WS_CBUF;
      const float *Uf = reinterpret_cast<const float *>(buf);
      if (tid < nnn && !s_abort) {
        const float Uv[5] = {Uf[tid], Uf[nnn + tid], Uf[2 * nnn + tid], Uf[3 * nnn + tid], Uf[4 * nnn + tid]};
        f32_stage<VF>(d, Uv, P + tid);
      }
      named_sync(1, WS_COMPUTE);
      if (s_abort) break;
      float sv[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      if (tid < nnn)
        f32_node_terms<VF>(d, P, reinterpret_cast<const float *>(buf + TB_UF),
                           reinterpret_cast<const float *>(buf + TB_UF + TB_JA),
                           reinterpret_cast<const float *>(buf + TB_UF + TB_JA + TB_FV), s_Dz, (int)e, tid, sv);
      // the sums buffer b is free once the epilogue has consumed element k - 2
      if (k >= 2 && !mbar_wait(smem_addr(&bar[4 + b]), (unsigned)(((k >> 1) - 1) & 1))) s_abort = 1;
      if (tid < nnn) {
        float *Sb = S + b * 5 * nnn + tid;
#pragma unroll
        for (int v = 0; v < 5; ++v) Sb[v * nnn] = sv[v];
      }
      mbar_arrive(smem_addr(&bar[2 + b]));
      named_sync(1, WS_COMPUTE);  // buffer b and P are free again
      if (s_abort) break;
      if (tid == 0) issue(k + 2);
    }
    if (s_abort && tid == 0) {  // report; wait (bounded) for the next element's copy still in flight
      flag_set(d.flag, 4);
      if ((long long)blockIdx.x + (long long)(k + 1) * gridDim.x < d.nE)
        mbar_wait(smem_addr(&bar[(k + 1) & 1]), (unsigned)(((k + 1) >> 1) & 1));
    }
  } else {
    // epilogue warps: the FP64 state, register and 1/J of each element arrive by TMA one element
    // ahead (issued by the group's first thread once the whole group has finished with the buffer)
    const int et = tid - WS_COMPUTE;
    const bool needU = mode == 1, needG = mode == 1 && !first;
    const unsigned ug_bytes = TB_IJ + (needU ? TB_U : 0u) + (needG ? TB_G : 0u);
    auto issue_ug = [&](int k) {
      const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
      if (e >= d.nE) return;
      const unsigned mb = smem_addr(&bar[6]);
      mbar_expect_tx(mb, ug_bytes);
      if (needU) bulk_g2s(smem_addr(UG), U + e * 5 * nnn, TB_U, mb);
      if (needG) bulk_g2s(smem_addr(UG + TB_U), g + e * 5 * nnn, TB_G, mb);
      bulk_g2s(smem_addr(UG + TB_U + TB_G), d.invJ + e * nnn, TB_IJ, mb);
    };
    if (et == 0) issue_ug(0);
    int k = 0;
    for (;; ++k) {
      const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
      if (e >= d.nE) break;
      const int b = k & 1;
      if (!mbar_wait(smem_addr(&bar[2 + b]), (unsigned)((k >> 1) & 1))) s_abort_e = 1;
      if (!mbar_wait(smem_addr(&bar[6]), (unsigned)(k & 1))) s_abort_e = 1;
      if (!s_abort_e) {
        const float *Sb = S + b * 5 * nnn;
        const double *Ue = reinterpret_cast<const double *>(UG), *ge = reinterpret_cast<const double *>(UG + TB_U),
                     *iJe = reinterpret_cast<const double *>(UG + TB_U + TB_G);
        // all of the thread's nodes at once (unrolled): their conversion and FP64 chains overlap
#pragma unroll
        for (int r = 0; r < (nnn + WS_EPI - 1) / WS_EPI; ++r) {
          const int node = et + r * WS_EPI;
          if (node < nnn) {
            const float sv[5] = {Sb[node], Sb[nnn + node], Sb[2 * nnn + node], Sb[3 * nnn + node],
                                 Sb[4 * nnn + node]};
            f32_finish(d, Ue, ge, iJe, out, g, (int)e, node, sv, mode, first, dt, A, B);
          }
        }
      }
      mbar_arrive(smem_addr(&bar[4 + b]));
      named_sync(2, WS_EPI);  // the group is done with the U, g buffer
      if (s_abort_e) break;
      if (et == 0) issue_ug(k + 1);
    }
    if (s_abort_e && et == 0) {  // report; wait (bounded) for this element's copy, the one in flight
      flag_set(d.flag, 4);
      mbar_wait(smem_addr(&bar[6]), (unsigned)(k & 1));
    }
  }
}

// ---------------------------------------------------------------------------------------------
// FP32-bulk volume operator with pair symmetry (N = 7). 192 line threads (one per x, y or z line of
// the element) form each two-point flux once, for both of its nodes, and keep the sums of their
// line's eight nodes in registers. The per-direction sums go to shared memory, where 8 epilogue
// warps add the three directions and apply -1/J and the FP64 LSERK update to element k-1 while the
// line threads work on element k. The FP32 state, metric terms and viscous flux arrive by TMA bulk
// copies one element ahead (as in k_volume_f32_ws); the face slots and the neighbours' viscous
// traces at a line's two end nodes come from global memory at the start of its line phase. Staged
// primitives and the sums use an XOR-swizzled node order (ln_sw), so that x, y and z lines and
// node-consecutive warps all access them without shared-memory bank conflicts.
// The sums are kept unscaled: the split-form factors (1/4 mass, 1/8 momentum and energy for KG and
// Pirozzoli; 2 for EC and central) are powers of two, applied once by the epilogue, and the surface
// and viscous terms enter divided by them (exact).
// ---------------------------------------------------------------------------------------------
constexpr bool LN_OK = (N == 7);
// four warp groups: two of epilogue warps (threads 0-255), two of line warps (256-511: 192 line
// threads, 64 that only help staging); setmaxnreg moves registers from the epilogue groups to the
// line groups, whose eight nodes' values and sums need ~168 per thread
constexpr int LN_EPI = 256;
constexpr int LN_GROUP = 256;       // threads of the line warp groups
constexpr int LN_COMPUTE = 3 * nn;  // line threads
constexpr int LN_THREADS = LN_EPI + LN_GROUP;
constexpr int LN_REG_LAUNCH = 65536 / LN_THREADS, LN_REG_LINE = 168, LN_REG_EPI = 88;
static_assert(LN_EPI * LN_REG_EPI + LN_GROUP * LN_REG_LINE <= LN_THREADS * LN_REG_LAUNCH,
              "the register split must fit the registers the block is launched with");
constexpr unsigned LN_CBUF = TB_UF + TB_JA + TB_FV;  // per-element TMA slices of the line phase
constexpr unsigned LN_ACC = 15u * nnn * 4u;          // [3 d][5][nnn] per-direction sums
constexpr unsigned LN_SMEM = 2u * LN_CBUF + TB_P + 2u * LN_ACC + WS_UG + 64u;
static_assert(!LN_OK || LN_SMEM <= 232448 - 256, "line kernel exceeds the shared memory of one CTA");
static_assert(!LN_OK || (LN_CBUF % 16 == 0 && LN_ACC % 16 == 0), "shared-memory regions must stay 16-byte aligned");
static_assert(!LN_OK || (nnn % LN_EPI == 0 && nnn % LN_GROUP == 0 && LN_COMPUTE <= LN_GROUP),
              "the epilogue and staging threads take whole nodes");

// bijective swizzle of node (i, j, k) = i + 8 j + 64 k for N = 7 (identity otherwise): the five
// low bits (the bank) are (i ^ j, (j ^ k) mod 4), which differ across the 32 lanes of an x, y or z
// line warp and of a warp of consecutive nodes
__device__ __forceinline__ int ln_sw(int node) {
  if (N != 7) return node;
  const int i = node & 7, j = (node >> 3) & 7, k = node >> 6;
  return ((i ^ j) & 7) | (((j ^ k) & 3) << 3) | ((j >> 2) << 5) | (k << 6);
}

// two-point flux of staged values held in registers (slots as in f32_stage); Sj = Ja_i + Ja_m
template <int VF>
__device__ __forceinline__ void pair_flux_reg(float ri, float ui, float vi, float wi, float p4i, float xi, float yi,
                                              float rm, float um, float vm, float wm, float p4m, float xm, float ym,
                                              float Sjx, float Sjy, float Sjz, float gam, float pref, float F[5]) {
  if (VF == VF_PIR || VF == VF_KG) {
    const float Su = ui + um, Sv = vi + vm, Sw = wi + wm;
    const float Vp = Su * Sjx + Sv * Sjy + Sw * Sjz;
    F[0] = (ri + rm) * Vp;
    const float Sp = p4i + p4m;
    F[1] = F[0] * Su + Sp * Sjx;
    F[2] = F[0] * Sv + Sp * Sjy;
    F[3] = F[0] * Sw + Sp * Sjz;
    if (VF == VF_PIR) F[4] = F[0] * (xi + xm);
    else F[4] = F[0] * (xi + xm) + (yi + ym) * Vp;
  } else {
    const float av[3] = {0.5f * Sjx, 0.5f * Sjy, 0.5f * Sjz};
    if (VF == VF_EC) {
      ec_flux<float>(ri, ui, vi, wi, yi, rm, um, vm, wm, ym, av, gam, pref, F);
    } else {
      const float Vi = ui * av[0] + vi * av[1] + wi * av[2], Vm = um * av[0] + vm * av[1] + wm * av[2];
      const float pm2 = 0.125f * (p4i + p4m);
      F[0] = 0.5f * (ri * Vi + rm * Vm);
      F[1] = 0.5f * (ri * ui * Vi + rm * um * Vm) + pm2 * av[0];
      F[2] = 0.5f * (ri * vi * Vi + rm * vm * Vm) + pm2 * av[1];
      F[3] = 0.5f * (ri * wi * Vi + rm * wm * Vm) + pm2 * av[2];
      F[4] = 0.5f * (xi * Vi + xm * Vm);
    }
  }
}

// the line's values and sums (registers); pairs (I, M), I < M, visited by template recursion so
// that every array index is a compile-time constant
struct LineRegs {
  float r[n], u[n], v[n], w[n], p4[n], x[n], y[n], jx[n], jy[n], jz[n];
  float acc[n][5];
};
template <int VF, int I, int M>
__device__ __forceinline__ void line_pairs(LineRegs &R, float gam, float pref) {
  if constexpr (I < n - 1) {
    float F[5];
    pair_flux_reg<VF>(R.r[I], R.u[I], R.v[I], R.w[I], R.p4[I], R.x[I], R.y[I], R.r[M], R.u[M], R.v[M], R.w[M],
                      R.p4[M], R.x[M], R.y[M], R.jx[I] + R.jx[M], R.jy[I] + R.jy[M], R.jz[I] + R.jz[M], gam, pref, F);
    const float ci = f_D[I * n + M], cm = f_D[M * n + I];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R.acc[I][v] += ci * F[v];
      R.acc[M][v] += cm * F[v];
    }
    if constexpr (M + 1 < n) line_pairs<VF, I, M + 1>(R, gam, pref);
    else line_pairs<VF, I + 1, I + 2>(R, gam, pref);
  }
}

__device__ __forceinline__ void regs_inc_line() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(LN_REG_LINE));
}
__device__ __forceinline__ void regs_dec_epi() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(LN_REG_EPI));
}

template <int VF>
__global__ void __launch_bounds__(LN_THREADS, 1) k_volume_f32_line(const DgDevice d, const double *U, double *out,
                                                                    double *g, int mode, int first, double dt,
                                                                    double A, double B) {
  if constexpr (LN_OK) {
    extern __shared__ __align__(128) unsigned char sm_tma[];
    float *P = reinterpret_cast<float *>(sm_tma + 2 * LN_CBUF);            // [7][nnn], swizzled
    float *ACC = reinterpret_cast<float *>(sm_tma + 2 * LN_CBUF + TB_P);  // [2][3][5][nnn], swizzled
    unsigned char *UG = sm_tma + 2 * LN_CBUF + TB_P + 2 * LN_ACC;          // U, g, 1/J (FP64)
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(UG + WS_UG);
    // bar[0..1]: TMA arrival per buffer; bar[2..3]: sums full; bar[4..5]: sums empty; bar[6]: U, g, 1/J
    __shared__ int s_abort, s_abort_e;
    constexpr bool SPLIT = (VF == VF_PIR || VF == VF_KG);
    // 1 / (split-form factor) per variable: the sums are unscaled (see above)
    constexpr float ISC0 = SPLIT ? 4.0f : 0.5f, ISC1 = SPLIT ? 8.0f : 0.5f;
    const bool ns = d.equations == 1;
    const unsigned bytes = TB_UF + TB_JA + (ns ? TB_FV : 0u);
    const int tid = threadIdx.x;
    if (tid == 0) {
      mbar_init(smem_addr(&bar[0]));
      mbar_init(smem_addr(&bar[1]));
      mbar_init_n(smem_addr(&bar[2]), LN_GROUP);
      mbar_init_n(smem_addr(&bar[3]), LN_GROUP);
      mbar_init_n(smem_addr(&bar[4]), LN_EPI);
      mbar_init_n(smem_addr(&bar[5]), LN_EPI);
      mbar_init(smem_addr(&bar[6]));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      s_abort = 0;
      s_abort_e = 0;
    }
    __syncthreads();
    auto issue = [&](int k) {
      const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
      if (e >= d.nE) return;
      unsigned char *b = sm_tma + (k & 1) * LN_CBUF;
      const unsigned mb = smem_addr(&bar[k & 1]);
      mbar_expect_tx(mb, bytes);
      bulk_g2s(smem_addr(b), d.Uf + e * 5 * nnn, TB_UF, mb);
      bulk_g2s(smem_addr(b + TB_UF), d.Jaf + e * 9 * nnn, TB_JA, mb);
      if (ns) bulk_g2s(smem_addr(b + TB_UF + TB_JA), d.Fv_f + e * 12 * nnn, TB_FV, mb);
    };
    if (tid >= LN_EPI) {
      regs_inc_line();
      const int ct = tid - LN_EPI;  // thread of the line warp groups
      const bool line = ct < LN_COMPUTE;
      if (ct == 0) {
        issue(0);
        issue(1);
      }
      // this thread's line: direction dd (warp-uniform), position (la, lb) on the faces 2dd, 2dd+1
      const int dd = line ? ct / nn : 0, L = ct % nn, la = L % n, lb = L / n;
      const int st = dd == 0 ? 1 : dd == 1 ? n : nn;
      const int base = dd == 0 ? n * la + nn * lb : dd == 1 ? la + nn * lb : la + n * lb;
      const float gam = d.gamma_f, pref = d.p_ref_f;
      const float iw0 = f_invw[0], iwN = f_invw[N];
      // face records of the line's two faces, loaded one element ahead (a warp issues in order: an
      // address computed from a just-loaded record would stall it for a full memory latency)
      int4 rec_next[2] = {make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0)};
      if (ns && line && blockIdx.x < d.nE) {
        rec_next[0] = *reinterpret_cast<const int4 *>(d.ef + ((size_t)blockIdx.x * 6 + 2 * dd) * 4);
        rec_next[1] = *reinterpret_cast<const int4 *>(d.ef + ((size_t)blockIdx.x * 6 + 2 * dd + 1) * 4);
      }
      int k = 0;
      for (;; ++k) {
        const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
        if (e >= d.nE) break;
        const int b = k & 1;
        const int4 rec[2] = {rec_next[0], rec_next[1]};
        if (ns && line && e + gridDim.x < d.nE) {
          rec_next[0] = *reinterpret_cast<const int4 *>(d.ef + ((size_t)(e + gridDim.x) * 6 + 2 * dd) * 4);
          rec_next[1] = *reinterpret_cast<const int4 *>(d.ef + ((size_t)(e + gridDim.x) * 6 + 2 * dd + 1) * 4);
        }
        if (!mbar_wait(smem_addr(&bar[b]), (unsigned)((k >> 1) & 1))) s_abort = 1;
        const unsigned char *buf = sm_tma + b * LN_CBUF;
        const float *Uf = reinterpret_cast<const float *>(buf);
        const float *Jb = reinterpret_cast<const float *>(buf + TB_UF);
        const float *Fb = reinterpret_cast<const float *>(buf + TB_UF + TB_JA);
        if (!s_abort)
          for (int t = ct; t < nnn; t += LN_GROUP) {
            const float Uv[5] = {Uf[t], Uf[nnn + t], Uf[2 * nnn + t], Uf[3 * nnn + t], Uf[4 * nnn + t]};
            f32_stage<VF>(d, Uv, P + ln_sw(t));
          }
        named_sync(1, LN_GROUP);
        if (s_abort) break;
        if (line) {
        // end-node data from global memory, loaded before the pair sums so that its latency overlaps them
        float fs[2][5], fnb[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        int wall[2] = {0, 0};
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int f = 2 * dd + side;
          const float *Fs = d.Fsurf_f + ((size_t)e * 6 + f) * 5 * nn + L;
#pragma unroll
          for (int v = 0; v < 5; ++v) fs[side][v] = Fs[v * nn];
          if (ns) {
            const int4 r4 = rec[side];
            if (r4.x >= 0) {
              int p2, q2;
              orient_map(r4.z, la, lb, p2, q2);
              const float *Fvn = d.Fv_f + ((size_t)r4.x * 12 + (r4.y >> 1) * 4) * nnn + face_node(r4.y, p2, q2);
#pragma unroll
              for (int q = 0; q < 4; ++q) fnb[side][q] = Fvn[q * nnn];
            } else {  // wall: the wall-model flux, combined with the own trace below
              const float *fw = d.Fwall_f + (size_t)r4.w * 4 * nn + L;
#pragma unroll
              for (int q = 0; q < 4; ++q) fnb[side][q] = fw[q * nn];
              wall[side] = 1;
            }
          }
        }
        // the line's staged values and metric terms Ja^dd
        LineRegs R;
#pragma unroll
        for (int i = 0; i < n; ++i) {
          const int nd = base + i * st, sw = ln_sw(nd);
          R.r[i] = P[sw]; R.u[i] = P[nnn + sw]; R.v[i] = P[2 * nnn + sw]; R.w[i] = P[3 * nnn + sw];
          R.p4[i] = P[4 * nnn + sw];
          R.x[i] = (VF == VF_EC) ? 0.0f : P[5 * nnn + sw];
          R.y[i] = (VF == VF_KG || VF == VF_EC) ? P[6 * nnn + sw] : 0.0f;
          R.jx[i] = Jb[(3 * dd) * nnn + nd];
          R.jy[i] = Jb[(3 * dd + 1) * nnn + nd];
          R.jz[i] = Jb[(3 * dd + 2) * nnn + nd];
#pragma unroll
          for (int v = 0; v < 5; ++v) R.acc[i][v] = 0.0f;
        }
        // each pair (i, m), i < m, once: node i takes D_im F, node m takes D_mi F (F is symmetric)
        line_pairs<VF, 0, 1>(R, gam, pref);
        float (&acc)[n][5] = R.acc;
        // surface terms: (1/w_b) times the outward face flux at the end nodes
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const float isc = v == 0 ? ISC0 : ISC1;
          acc[0][v] += (isc * iw0) * fs[0][v];
          acc[N][v] += (isc * iwN) * fs[1][v];
        }
        if (ns) {
          // viscous divergence along the line, then the neighbour's normal viscous flux or the wall
          // term at the end nodes (see k_volume)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float fv[n];
#pragma unroll
            for (int m = 0; m < n; ++m) fv[m] = Fb[(dd * 4 + q) * nnn + base + m * st];
#pragma unroll
            for (int i = 0; i < n; ++i) {
              float t = 0.0f;
#pragma unroll
              for (int m = 0; m < n; ++m)
                if (m != i) t += f_D[i * n + m] * fv[m];
              acc[i][1 + q] -= ISC1 * t;
            }
            const float sg0 = (rec[0].y & 1) ? 0.5f : -0.5f, sg1 = (rec[1].y & 1) ? 0.5f : -0.5f;
            acc[0][1 + q] += wall[0] ? -(ISC1 * iw0) * (fnb[0][q] + 0.5f * fv[0]) : (ISC1 * iw0 * sg0) * fnb[0][q];
            acc[N][1 + q] += wall[1] ? -(ISC1 * iwN) * (fnb[1][q] - 0.5f * fv[N]) : (ISC1 * iwN * sg1) * fnb[1][q];
          }
        }
        // the sums buffer b is free once the epilogue has consumed element k - 2
        if (k >= 2 && !mbar_wait(smem_addr(&bar[4 + b]), (unsigned)(((k >> 1) - 1) & 1))) s_abort = 1;
        float *Ab = ACC + (b * 3 + dd) * 5 * nnn;
#pragma unroll
        for (int i = 0; i < n; ++i) {
          const int sw = ln_sw(base + i * st);
#pragma unroll
          for (int v = 0; v < 5; ++v) Ab[v * nnn + sw] = acc[i][v];
        }
        }  // line
        mbar_arrive(smem_addr(&bar[2 + b]));
        named_sync(1, LN_GROUP);  // buffer b and P are free again
        if (s_abort) break;
        if (ct == 0) issue(k + 2);
      }
      if (s_abort && ct == 0) {  // report; wait (bounded) for the next element's copy still in flight
        flag_set(d.flag, 4);
        if ((long long)blockIdx.x + (long long)(k + 1) * gridDim.x < d.nE)
          mbar_wait(smem_addr(&bar[(k + 1) & 1]), (unsigned)(((k + 1) >> 1) & 1));
      }
    } else {
      // epilogue warps: sum the three directions, scale, -1/J and the FP64 LSERK stage; the FP64
      // state, register and 1/J arrive by TMA one element ahead (issued once the group is done)
      regs_dec_epi();
      const int et = tid;
      const bool needU = mode == 1, needG = mode == 1 && !first;
      const unsigned ug_bytes = TB_IJ + (needU ? TB_U : 0u) + (needG ? TB_G : 0u);
      auto issue_ug = [&](int k) {
        const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
        if (e >= d.nE) return;
        const unsigned mb = smem_addr(&bar[6]);
        mbar_expect_tx(mb, ug_bytes);
        if (needU) bulk_g2s(smem_addr(UG), U + e * 5 * nnn, TB_U, mb);
        if (needG) bulk_g2s(smem_addr(UG + TB_U), g + e * 5 * nnn, TB_G, mb);
        bulk_g2s(smem_addr(UG + TB_U + TB_G), d.invJ + e * nnn, TB_IJ, mb);
      };
      if (et == 0) issue_ug(0);
      constexpr float SC0 = SPLIT ? 0.25f : 2.0f, SC1 = SPLIT ? 0.125f : 2.0f;
      int k = 0;
      for (;; ++k) {
        const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
        if (e >= d.nE) break;
        const int b = k & 1;
        if (!mbar_wait(smem_addr(&bar[2 + b]), (unsigned)((k >> 1) & 1))) s_abort_e = 1;
        if (!mbar_wait(smem_addr(&bar[6]), (unsigned)(k & 1))) s_abort_e = 1;
        // the thread's nodes' sums, U, g and 1/J into registers first; then the sums buffer and the
        // U, g, 1/J buffer are released (the next element's copy overlaps this element's FP64 stage)
        constexpr int R = nnn / LN_EPI;
        float sv[R][5];
        double Uv[R][5], gv0[R][5], iJ[R];
        if (!s_abort_e) {
          const float *A0 = ACC + (b * 3) * 5 * nnn, *A1 = A0 + 5 * nnn, *A2 = A1 + 5 * nnn;
          const double *Ue = reinterpret_cast<const double *>(UG), *ge = reinterpret_cast<const double *>(UG + TB_U),
                       *iJe = reinterpret_cast<const double *>(UG + TB_U + TB_G);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int node = et + r * LN_EPI, sw = ln_sw(node);
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              sv[r][v] = (v == 0 ? SC0 : SC1) * ((A0[v * nnn + sw] + A1[v * nnn + sw]) + A2[v * nnn + sw]);
              Uv[r][v] = needU ? Ue[node + v * nnn] : 0.0;
              gv0[r][v] = needG ? ge[node + v * nnn] : 0.0;
            }
            iJ[r] = iJe[node];
          }
        }
        mbar_arrive(smem_addr(&bar[4 + b]));
        named_sync(2, LN_EPI);  // the group is done with the U, g, 1/J buffer
        if (s_abort_e) break;
        if (et == 0) issue_ug(k + 1);
#pragma unroll
        for (int r = 0; r < R; ++r)
          f32_finish_reg(d, Uv[r], gv0[r], iJ[r], out, g, (int)e, et + r * LN_EPI, sv[r], mode, first, dt, A, B);
      }
      if (s_abort_e && et == 0) {  // report; wait (bounded) for this element's copy, the one in flight
        flag_set(d.flag, 4);
        mbar_wait(smem_addr(&bar[6]), (unsigned)(k & 1));
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// FP32-bulk BR1 lifting as a persistent kernel fed by TMA (N = 3, 5, 7): one thread per node, two
// CTAs per SM; each element's FP32 state, metric terms, 1/J and BR1 face jumps arrive by
// cp.async.bulk one element ahead into a double buffer, so the loads of the next element overlap
// this element's arithmetic. The per-node arithmetic is lift_prim / lift_node, as in k_lift.
// ---------------------------------------------------------------------------------------------
constexpr int LT_THREADS = TMA_THREADS;
constexpr unsigned LT_IJ = nnn * 4u, LT_WS = 24u * nn * 4u;
constexpr unsigned LT_BUF = TB_UF + TB_JA + LT_IJ + LT_WS;
constexpr unsigned LT_SMEM = 2u * LT_BUF + 4u * nnn * 4u + 16u;
static_assert(!TMA_OK || (LT_IJ % 16 == 0 && LT_WS % 16 == 0 && LT_BUF % 16 == 0),
              "TMA slices must be multiples of 16 bytes");

__global__ void __launch_bounds__(LT_THREADS, 2) k_lift_f32_tma(const DgDevice d) {
  extern __shared__ __align__(128) unsigned char sm_tma[];
  float *W = reinterpret_cast<float *>(sm_tma + 2 * LT_BUF);  // [4][nnn]
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(sm_tma + 2 * LT_BUF + 4 * nnn * 4);
  __shared__ float sD[n][n + 1];
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  for (int t = tid; t < nn; t += blockDim.x) sD[t / n][t % n] = f_D[t];
  if (tid == 0) {
    mbar_init(smem_addr(&bar[0]));
    mbar_init(smem_addr(&bar[1]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int k) {
    const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
    if (e >= d.nE) return;
    unsigned char *b = sm_tma + (k & 1) * LT_BUF;
    const unsigned mb = smem_addr(&bar[k & 1]);
    mbar_expect_tx(mb, LT_BUF);
    bulk_g2s(smem_addr(b), d.Uf + e * 5 * nnn, TB_UF, mb);
    bulk_g2s(smem_addr(b + TB_UF), d.Jaf + e * 9 * nnn, TB_JA, mb);
    bulk_g2s(smem_addr(b + TB_UF + TB_JA), d.invJf + e * nnn, LT_IJ, mb);
    bulk_g2s(smem_addr(b + TB_UF + TB_JA + LT_IJ), d.Wsurf_f + e * 24 * nn, LT_WS, mb);
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }
  const float gm1 = d.gm1_f, iR = d.iR_f, pref = d.p_ref_f, mu = d.mu_f, kappa = d.kappa_f;
  for (int k = 0;; ++k) {
    const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
    if (e >= d.nE) break;
    const unsigned mb = smem_addr(&bar[k & 1]), parity = (unsigned)((k >> 1) & 1);
    if (tid == 0) s_ok = mbar_wait(mb, parity) ? 1 : 0;
    __syncthreads();
    if (!s_ok) {  // a copy never completed: report, wait (bounded) for the other buffer's copy, stop
      if (tid == 0) {
        flag_set(d.flag, 4);
        if (e + gridDim.x < d.nE) mbar_wait(smem_addr(&bar[(k + 1) & 1]), (unsigned)(((k + 1) >> 1) & 1));
      }
      return;
    }
    mbar_wait(mb, parity);  // completed: returns at once and orders this thread's reads after the copy
    const unsigned char *b = sm_tma + (k & 1) * LT_BUF;
    const float *Uf = reinterpret_cast<const float *>(b);
    const float *Jb = reinterpret_cast<const float *>(b + TB_UF);
    const float *Ib = reinterpret_cast<const float *>(b + TB_UF + TB_JA);
    const float *Sb = reinterpret_cast<const float *>(b + TB_UF + TB_JA + LT_IJ);
    if (tid < nnn) {
      const float Uv[5] = {Uf[tid], Uf[nnn + tid], Uf[2 * nnn + tid], Uf[3 * nnn + tid], Uf[4 * nnn + tid]};
      float Wn[4];
      lift_prim<float>(Uv, gm1, iR, pref, Wn);
#pragma unroll
      for (int q = 0; q < 4; ++q) W[q * nnn + tid] = Wn[q];
    }
    __syncthreads();
    if (tid < nnn) lift_node<float>(d, tid, W, sD, Jb, Sb, Ib[tid], mu, kappa, d.Fv_f + (size_t)e * 12 * nnn);
    __syncthreads();  // buffer k & 1 and W are free again
    if (tid == 0) issue(k + 2);
  }
}

// ---------------------------------------------------------------------------------------------
// modified Persson indicator (Sec. 4.1, Eq. (7)) and the neighbour extension (FP64)
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_indicator(const DgDevice d, const double *__restrict__ U) {
  __shared__ double q[nnn], t1[nnn];
  __shared__ double red[3][128];
  const int e = blockIdx.x;
  const double gm1 = d.gamma - 1.0;
  for (int node = threadIdx.x; node < nnn; node += blockDim.x) {
    const double *Ue = U + (size_t)e * 5 * nnn + node;
    const double r = Ue[0];
    const double p = gm1 * (Ue[4 * nnn] - 0.5 * (Ue[nnn] * Ue[nnn] + Ue[2 * nnn] * Ue[2 * nnn] + Ue[3 * nnn] * Ue[3 * nnn]) / r);
    q[node] = r * p;
  }
  __syncthreads();
  // modal coefficients: three tensor-product passes with the inverse Vandermonde
  for (int node = threadIdx.x; node < nnn; node += blockDim.x) {  // xi: (i,j,k) -> (a,j,k)
    const int a = node % n, base = node - a;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) s += c_Vinv[a * n + i] * q[base + i];
    t1[node] = s;
  }
  __syncthreads();
  for (int node = threadIdx.x; node < nnn; node += blockDim.x) {  // eta
    const int b = (node / n) % n, base = node - b * n;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < n; ++j) s += c_Vinv[b * n + j] * t1[base + j * n];
    q[node] = s;
  }
  __syncthreads();
  double all = 0.0, shN = 0.0, shN1 = 0.0;
  for (int node = threadIdx.x; node < nnn; node += blockDim.x) {  // zeta, then the shell energies
    const int a = node % n, b = (node / n) % n, c = node / nn, base = node - c * nn;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < n; ++k) s += c_Vinv[c * n + k] * q[base + k * nn];
    const int M = max(a, max(b, c));
    const double m2 = s * s;
    all += m2;
    if (M == N) shN += m2;
    if (M == N - 1) shN1 += m2;
  }
  red[0][threadIdx.x] = all;
  red[1][threadIdx.x] = shN;
  red[2][threadIdx.x] = shN1;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tot = red[0][0], sN = red[1][0], sN1 = red[2][0];
    double E = tot > 1e-300 ? sN / tot : 0.0;
    if (N >= 2) {
      const double tot1 = tot - sN;
      const double E1 = tot1 > 1e-300 ? sN1 / tot1 : 0.0;
      E = fmax(E, E1);
    }
    const double T = 0.5 * pow(10.0, -1.8 * pow((double)(N + 1), 0.25));
    double al = 1.0 / (1.0 + exp(-d.sharpness / T * (E - T)));
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
  double D2[nn], Dq[nn], De[nn];
  float fD[nn], fD2[nn], fDq[nn], fDe[nn], fw[n], finvw[n], fxi[n], fxh[n + 1];
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < n; ++m) {
      const double v = (i == m) ? 0.0 : t.D[i * n + m];
      D2[i * n + m] = 2.0 * v;
      Dq[i * n + m] = 0.25 * v;
      De[i * n + m] = 0.125 * v;
      fD[i * n + m] = (float)t.D[i * n + m];
      fD2[i * n + m] = (float)D2[i * n + m];
      fDq[i * n + m] = (float)Dq[i * n + m];
      fDe[i * n + m] = (float)De[i * n + m];
    }
  for (int i = 0; i < n; ++i) { fw[i] = (float)t.w[i]; finvw[i] = (float)t.invw[i]; fxi[i] = (float)t.xi[i]; }
  for (int i = 0; i <= n; ++i) fxh[i] = (float)t.xh[i];
  cudaError_t err = cudaSuccess;
  err = err ? err : cudaMemcpyToSymbol(c_D, t.D, sizeof(double) * nn);
  err = err ? err : cudaMemcpyToSymbol(c_D2, D2, sizeof(double) * nn);
  err = err ? err : cudaMemcpyToSymbol(c_Dq, Dq, sizeof(double) * nn);
  err = err ? err : cudaMemcpyToSymbol(c_De, De, sizeof(double) * nn);
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

void launch_lift(const DgDevice &d, const double *U, cudaStream_t s) {
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
  if (d.precision == 1) k_lift<float><<<grid, LIFT_THREADS, 0, s>>>(d, U);
  else k_lift<double><<<grid, LIFT_THREADS, 0, s>>>(d, U);
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

void launch_indicator(const DgDevice &d, const double *U, cudaStream_t s) { k_indicator<<<d.nE, 128, 0, s>>>(d, U); }

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
