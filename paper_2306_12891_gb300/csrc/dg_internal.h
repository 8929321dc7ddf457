// dg_internal.h -- shared between the C-ABI layer (dg_api.cu) and the per-degree kernel
// translation units (dg_kernels_nN.cu). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#define DG_NMAX 7           // highest polynomial degree with compiled kernels
#define DG_NVAR 5

// Basis tables for one N, built on the host (dg_basis.cpp) and copied into each kernel
// translation unit's constant memory.
struct DgTables {
  int N;
  double xi[DG_NMAX + 1], w[DG_NMAX + 1], invw[DG_NMAX + 1];
  double D[(DG_NMAX + 1) * (DG_NMAX + 1)];     // D[i*n+m] = l_m'(xi_i)
  double Vinv[(DG_NMAX + 1) * (DG_NMAX + 1)];  // inverse orthonormal-Legendre Vandermonde
  double xh[DG_NMAX + 2];                      // FV subcell interfaces -1 + cumulative weights
};

// Plain view of a context's device state, passed by value to every kernel.
struct DgDevice {
  int N, nE, nF;
  int equations, vflux, sflux, precision, shock_capturing;
  double gamma, R, mu, kappa, alpha_min, alpha_max, sharpness, alpha_fixed;
  double ind_T, ind_k;  // indicator threshold T = 0.5 10^(-1.8 (N+1)^(1/4)) (Eq. (7)) and -sharpness / T
  double p_ref;        // reference pressure removed from the momentum flux (FP32-bulk only; 0 in FP64)
  // per-context constants computed once on the host (the FP32 kernels would otherwise form them
  // per thread on the FP64 pipe): gamma-1, 1/R, p_ref gamma/(gamma-1), p_ref/(gamma-1), and their
  // FP32 roundings
  double gm1, iR, href, eref, igm1;
  float gamma_f, gm1_f, iR_f, p_ref_f, href_f, mu_f, kappa_f, igm1_f;
  // wall-modelled walls (faces with elemR = -1; Sec. 3): exchange node index, van Driest on/off
  // with b = sqrt(r m)/sqrt(1 + r m), m = (gamma-1)/2 Ma_inf^2, r = Pr^(1/3), and freestream speed
  int use_tma;         // FP32-bulk volume operator through the TMA-fed persistent kernel (N = 3, 5, 7)
  int n_walls;         // number of wall faces (0: fully periodic)
  int wm_index, wm_vd;
  double wm_uinf, wm_b;
  double *hwm;         // [nF][n^2] wall distance of the exchange node (wall faces only)
  double *Fwall;       // [nF][4][n^2] outward wall-model viscous flux s F_v.n (momentum, energy), wall faces
  float *Fwall_f;      // FP32-bulk version
  // geometry (built at init)
  const double *xyz;   // [nE][3][n^3]  (init only)
  double *Ja;          // [nE][3 d][3 c][n^3]
  double *J;           // [nE][n^3]
  double *invJ;        // [nE][n^3]
  float *Jaf;          // FP32 copy of Ja for the FP32-bulk path (or null)
  double *nrm;         // [nF][4][n^2]: unit normal (x,y,z) outward from L, area factor s
  float *nrm_f;        // FP32 copy of nrm for the FP32-bulk path (or null)
  const int *face;     // [nF][5]
  int *ef;             // [nE][6][4]: neighbour element, neighbour local face, orientation own->nb, face id
  // per-stage work buffers
  double *Fsurf;       // [nE][6][5][n^2] outward advective surface flux, own face-point order
  double *Wsurf;       // [nE][6][4][n^2] BR1 lifting jump (w* - w_own), own order
  double *Fv;          // [nE][3 d][4][n^3] contravariant viscous flux (momentum x,y,z, energy)
  float *Fsurf_f, *Wsurf_f, *Fv_f;  // FP32-bulk versions
  float *Uf;           // FP32-bulk: FP32 shadow of the state [nE][5][n^3], E shifted by p_ref/(gamma-1)
  float *invJf;        // FP32-bulk: FP32 copy of 1/J for the lifting
  float *facf;         // FP32-bulk: float(dt (-1/J)) for the step size of the current LSERK call
  double *alpha_raw;   // [nE]
  double *alpha;       // [nE]
  double *red;         // reduction partials
  int *flag;           // bit 0: non-physical state met; bit 1: J <= 0 at init
};

// Kernel entry points compiled for one polynomial degree (one translation unit per N).
struct DgKernelTable {
  int N;
  cudaError_t (*upload)(const DgTables &t);
  void (*metrics)(const DgDevice &d, cudaStream_t s);
  void (*face_normals)(const DgDevice &d, cudaStream_t s);
  void (*face)(const DgDevice &d, const double *U, cudaStream_t s);
  // tau: null, or (FP64) the viscous stress record [nE][6][n^3] the lifting also writes for the adjoint
  void (*lift)(const DgDevice &d, const double *U, double *tau, cudaStream_t s);
  // mode 0: out = Ut. mode 1: LSERK stage in place on out (== U): g = first ? dt*Ut : A g + dt*Ut;
  // U += B g.
  void (*volume)(const DgDevice &d, const double *U, double *out, double *g, int mode, int first, double dt,
                 double A, double B, cudaStream_t s);
  void (*indicator)(const DgDevice &d, const double *U, cudaStream_t s);
  void (*spread)(const DgDevice &d, double *alpha_out, cudaStream_t s);
  void (*invariants)(const DgDevice &d, const double *U, const double *Ut, double *out8_dev, cudaStream_t s);
  void (*max_dt)(const DgDevice &d, const double *U, double *out_dev, cudaStream_t s);
  void (*shadow)(const DgDevice &d, const double *U, cudaStream_t s);  // FP32 shadow of U (FP32-bulk)
  // adjoint (FP64, no shock capturing): transposed Riemann-flux Jacobians into face slots
  // [nE][6][5][n^2]; viscous adjoint into cotW [nE][4][n^3] (u, v, w, T) and sigma [nE][6][4][n^2];
  // volume adjoint. mode 0: out = (dL/dU)^T lam. mode 1: reverse LSERK stage, out (= Ubar) += dt *
  // VJP, then, if update_g, gbar (== lam) = A gbar + B Ubar.
  void (*adj_face)(const DgDevice &d, const double *U, const double *lam, double *slots, cudaStream_t s);
  // tau: the lifting's viscous stress record of the same state U
  void (*adj_visc)(const DgDevice &d, const double *U, const double *lam, const double *tau, double *cotW,
                   double *sigma, cudaStream_t s);
  void (*adj_volume)(const DgDevice &d, const double *U, const double *lam, const double *fslots, const double *cotW,
                     const double *sigma, double *out, double *gbar, int mode, double dt, double A, double B,
                     int update_g, cudaStream_t s);
  void (*ke_grad)(const DgDevice &d, const double *U, double *grad, cudaStream_t s);  // d(kinetic energy)/dU
};

extern const DgKernelTable dg_kernels_n1, dg_kernels_n2, dg_kernels_n3, dg_kernels_n4, dg_kernels_n5,
    dg_kernels_n6, dg_kernels_n7;

// Host-side basis construction (dg_basis.cpp): returns 0 on success.
int dg_build_tables(int N, DgTables *t);

// Reduction buffer size (doubles) the kernels may use in DgDevice::red.
#define DG_RED_BLOCKS 1024
#define DG_RED_DOUBLES (DG_RED_BLOCKS * 8 + 8)
