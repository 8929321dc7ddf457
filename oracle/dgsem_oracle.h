/*
 * dgsem_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the explicit split-form DGSEM method of
 * "Towards Exascale CFD Simulations Using the Discontinuous Galerkin Solver FLEXI"
 * (arXiv 2306.12891): the right-hand side of the compressible Euler / Navier-Stokes
 * equations on curved hexahedra (split-form flux differencing on Legendre-Gauss-Lobatto
 * nodes, Sec. 2 "Performance" and Sec. 4.1 "Hybrid DGSE/FV subcell scheme"), its
 * explicit Runge-Kutta time step (Sec. 2, Eq. (1) counts its stages), the modified
 * Persson indicator (Sec. 4.1, Eq. (7)) and the DG/FV convex blend (Sec. 4.1, Eq. (6)).
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark may load
 * this library. It shares no code with the CUDA path. Every routine uses plain loops
 * in the order the method states them; no blocking, fusion or reordering.
 *
 * Array layouts (all row-major, element-major):
 *   n = N+1 nodes per direction, node index = i + n*(j + n*k), i along xi.
 *   U, Ut   [n_elems][5][n][n][n]   conservative (rho, rho u, rho v, rho w, E)
 *   xyz     [n_elems][3][n][n][n]   physical coordinates of the LGL nodes
 *   Ja      [n_elems][3 (d)][3 (c)][n][n][n]  contravariant metric J a^d, component c
 *   J       [n_elems][n][n][n]
 *   faces   [n_faces][5] = (elemL, faceL, elemR, faceR, orient)
 *           local faces 0:xi-,1:xi+,2:eta-,3:eta+,4:zeta-,5:zeta+;
 *           face point (p,q) = tangential indices in increasing dimension order;
 *           orient maps L's (p,q) to R's: (a,b) = bit2 ? (q,p) : (p,q),
 *           then a -> N-a if bit0, b -> N-b if bit1.
 */
#ifndef DGSEM_ORACLE_H
#define DGSEM_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

/* orc_real is the type of every quantity that depends on the state U. The default build
 * uses double. The complex-step build (-DORC_COMPLEX_STEP, a second library) runs the same
 * source on double _Complex: for a real state U, direction V and h = 1e-30, Im L(U + i h V) / h
 * is the directional derivative of the right-hand side L (and of the LSERK step) with no
 * cancellation error, which makes it the reference for the discrete adjoint. Metrics, basis
 * and coefficients stay double in both builds. */
#ifdef ORC_COMPLEX_STEP
#include <complex.h>
typedef double _Complex orc_real;
#else
typedef double orc_real;
#endif

enum { ORC_EULER = 0, ORC_NAVIER_STOKES = 1 };
enum { ORC_VF_KG = 0, ORC_VF_PIROZZOLI = 1, ORC_VF_EC = 2, ORC_VF_CENTRAL = 3 };
enum { ORC_SF_LLF = 0, ORC_SF_ROE = 1, ORC_SF_EC = 2 };
enum { ORC_BC_WALL_MODEL = 0 };

typedef struct {
  int N;
  int n_elems;
  const double *xyz;
  int n_faces;
  const int *faces;
  int equations;       /* ORC_EULER | ORC_NAVIER_STOKES */
  int vflux;           /* ORC_VF_* */
  int sflux;           /* ORC_SF_* */
  double gamma, R, mu, Pr;
  int shock_capturing; /* 0/1: DG/FV blend with the modal indicator */
  double alpha_min, alpha_max, sharpness;
  double alpha_fixed;  /* >= 0: blend with this coefficient on every element instead */
  /* wall-modelled walls (faces with elemR = -1, faceR = ORC_BC_WALL_MODEL; Sec. 3): the wall shear
   * stress comes from Spalding's law at the exchange node wm_index nodes away from the wall, with
   * the input velocity mapped by the van Driest transform when wm_van_driest != 0 */
  int wm_index;
  double wm_uinf, wm_mainf;
  int wm_van_driest;
} orc_problem;

/* Opaque precomputed state (basis, metrics, connectivity). */
typedef struct orc_state orc_state;

/* ---- basis (Sec. 2: LGL nodes) ---- */
int orc_lgl(int N, double *xi, double *w);
int orc_dmatrix(int N, const double *xi, double *D);             /* D[i*n+j] = l_j'(xi_i) */
int orc_legendre_vandermonde(int N, const double *xi, double *V);/* V[j*n+k] = phi_k(xi_j), orthonormal */
int orc_invert(int n, const double *A, double *Ainv);            /* Gauss-Jordan, partial pivoting */

/* ---- geometry ---- */
int orc_metrics(int N, int n_elems, const double *xyz, double *Ja, double *J);

/* ---- pointwise fluxes (exposed for unit pins) ---- */
orc_real orc_logmean(orc_real a, orc_real b);
void orc_flux_contra(const orc_real U[5], const double a[3], double gamma, orc_real F[5]);
void orc_twopoint(int kind, const orc_real UL[5], const orc_real UR[5], const double aL[3],
                  const double aR[3], double gamma, orc_real F[5]);
void orc_riemann(int kind, const orc_real UL[5], const orc_real UR[5], const double nhat[3],
                 double gamma, orc_real F[5]);
/* gradU[r][c] = d u_r / d x_c, gradT[c]; Fv[c][v] = viscous flux in Cartesian direction c */
void orc_viscous_flux(const orc_real U[5], const orc_real gradU[9], const orc_real gradT[3],
                      double mu, double kappa, double gamma, orc_real Fv[15]);

/* ---- wall model (Sec. 3, Eq. (2) Spalding's law of the wall, Eq. (5) van Driest transform) ---- */
double orc_spalding_yplus(double uplus);                 /* y+ of u+ */
/* u+ solving u+ * y+(u+) = Re_h = h U / nu (Newton, monotone from above); *iters = iterations used */
orc_real orc_wall_uplus(orc_real Re_h, int *iters);
/* equivalent incompressible velocity of u (Eq. (5)); u itself when mainf == 0 */
orc_real orc_van_driest(orc_real u, double uinf, double mainf, double gamma, double Pr);
/* friction velocity at wall distance h for tangential speed U and kinematic viscosity nu */
orc_real orc_wall_utau(orc_real U, double h, orc_real nu, double uinf, double mainf, double gamma, double Pr,
                       int van_driest);

/* ---- solver ---- */
orc_state *orc_create(const orc_problem *pb, int *status);
void orc_destroy(orc_state *s);
const double *orc_state_Ja(const orc_state *s);
const double *orc_state_J(const orc_state *s);
/* out_mask (n_elems bytes, nullable): compute Ut only where mask != 0 (others set to 0).
 * alpha (n_elems, nullable): receives the blending coefficient used (0 without shock capturing). */
int orc_rhs(orc_state *s, const orc_real *U, orc_real *Ut, const unsigned char *out_mask, orc_real *alpha);
int orc_indicator(orc_state *s, const orc_real *U, orc_real *alpha_raw, orc_real *alpha);
int orc_lserk_step(orc_state *s, orc_real *U, double dt, double t);
int orc_invariants(orc_state *s, const orc_real *U, const orc_real *Ut, orc_real out[8]);
int orc_max_dt(orc_state *s, const orc_real *U, double cfl, double *dt);

/* LSERK(5,4) on a generic system u' = f(u, t) (used to pin the scheme on scalar ODEs). */
typedef void (*orc_rhs_fn)(const orc_real *u, orc_real *ut, double t, void *ctx);
int orc_lserk_generic(int n, orc_real *u, double dt, double t, orc_rhs_fn f, void *ctx);
void orc_lserk_coefficients(double A[5], double B[5], double c[5]);

#ifdef __cplusplus
}
#endif
#endif
