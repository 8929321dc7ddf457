/*
 * dgsem_oracle.c -- TEST INFRASTRUCTURE ONLY (see dgsem_oracle.h).
 *
 * Plain FP64 CPU restatement of the split-form DGSEM of arXiv 2306.12891 and the
 * published methods it builds on:
 *   - DGSEM strong form on Legendre-Gauss-Lobatto (LGL) nodes, whose summation-by-parts
 *     property lets the volume operator be written in flux-differencing form (Sec. 4.1);
 *   - split-form two-point volume fluxes: Kennedy-Gruber, Pirozzoli, Chandrashekar's
 *     entropy-conservative flux (Ismail-Roe logarithmic mean), central;
 *   - Roe and local Lax-Friedrichs (LLF) surface Riemann fluxes;
 *   - BR1 lifting of the primitive gradients (u, v, w, T) for the Navier-Stokes-Fourier
 *     viscous fluxes (Sec. 4: "Navier--Stokes--Fourier equations");
 *   - curvilinear metric terms in Kopriva's discrete curl form;
 *   - the hybrid DG/FV convex blend U_t = a U_t^FV + (1-a) U_t^DG (Sec. 4.1, Eq. (6)) with a
 *     second-order minmod FV scheme in the interior subcells and first order in the outer
 *     subcells (Sec. 4.1), blending coefficient from the modified Persson indicator
 *     (Sec. 4.1, Eq. (7)), clipped to [alpha_min, alpha_max] (Sec. 4.2) and extended to face
 *     neighbours by a factor 1/2 (Sec. 4.1);
 *   - the explicit low-storage Runge-Kutta scheme LSERK(5,4) of Carpenter and Kennedy
 *     (the "explicit Runge--Kutta scheme" of Sec. 2).
 * Readings of points the paper leaves open are listed in the repository's design notes.
 */
#include "dgsem_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Arithmetic on state-dependent quantities. The default build is plain double. The
 * complex-step build (-DORC_COMPLEX_STEP, see dgsem_oracle.h) runs the same statements on
 * double _Complex: branches and clips decide on the real part, and |x|, max(a, b) follow the
 * real part's sign and order, so the imaginary part carries the exact one-sided derivative. */
#ifdef ORC_COMPLEX_STEP
#define RE(x) creal(x)
#define R_SQRT csqrt
#define R_LOG clog
#define R_EXP cexp
#define R_ASIN casin
static orc_real R_ABS(orc_real x) { return creal(x) < 0.0 ? -x : x; }
static orc_real R_MAX(orc_real a, orc_real b) { return creal(b) > creal(a) ? b : a; }
#else
#define RE(x) (x)
#define R_SQRT sqrt
#define R_LOG log
#define R_EXP exp
#define R_ASIN asin
#define R_ABS fabs
#define R_MAX fmax
#endif

#define NVAR 5
#define NMAX 15

/* ======================================================================= */
/* 1. Basis                                                                 */
/* ======================================================================= */

/* Legendre polynomial P_N(x) and its derivative by the three-term recurrence. */
static void legendre_ld(int N, long double x, long double *P, long double *dP) {
  if (N == 0) { *P = 1.0L; *dP = 0.0L; return; }
  long double p0 = 1.0L, p1 = x, d0 = 0.0L, d1 = 1.0L;
  for (int k = 2; k <= N; ++k) {
    long double p2 = ((2.0L * k - 1.0L) * x * p1 - (k - 1.0L) * p0) / k;
    long double d2 = d0 + (2.0L * k - 1.0L) * p1; /* P'_k = P'_{k-2} + (2k-1) P_{k-1} */
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

/* LGL nodes: the end points and the roots of P_N'(x); weights 2/(N(N+1) P_N(x_j)^2). */
int orc_lgl(int N, double *xi, double *w) {
  if (N < 1 || N > NMAX) return -1;
  long double x[NMAX + 1];
  x[0] = -1.0L; x[N] = 1.0L;
  for (int j = 1; j < N; ++j) {
    long double t = -cosl(3.14159265358979323846264338327950288L * j / N); /* Chebyshev-Lobatto guess */
    for (int it = 0; it < 100; ++it) {
      long double P, dP;
      legendre_ld(N, t, &P, &dP);
      /* Legendre ODE: (1-x^2) P'' = 2x P' - N(N+1) P */
      long double d2P = (2.0L * t * dP - N * (N + 1.0L) * P) / (1.0L - t * t);
      long double dt = dP / d2P;
      t -= dt;
      if (fabsl(dt) < 1e-22L) break;
    }
    x[j] = t;
  }
  /* the node set is symmetric about 0 */
  for (int j = 0; j <= N / 2; ++j) {
    long double s = 0.5L * (x[N - j] - x[j]);
    x[j] = -s; x[N - j] = s;
  }
  if (N % 2 == 0) x[N / 2] = 0.0L;
  for (int j = 0; j <= N; ++j) {
    long double P, dP;
    legendre_ld(N, x[j], &P, &dP);
    xi[j] = (double)x[j];
    w[j] = (double)(2.0L / (N * (N + 1.0L) * P * P));
  }
  return 0;
}

/* Lagrange derivative matrix D_ij = l_j'(xi_i) from barycentric weights,
 * diagonal by the negative-sum rule. */
int orc_dmatrix(int N, const double *xi, double *D) {
  int n = N + 1;
  long double lam[NMAX + 1];
  for (int j = 0; j < n; ++j) {
    long double p = 1.0L;
    for (int k = 0; k < n; ++k)
      if (k != j) p *= ((long double)xi[j] - (long double)xi[k]);
    lam[j] = 1.0L / p;
  }
  for (int i = 0; i < n; ++i) {
    long double diag = 0.0L;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      long double v = (lam[j] / lam[i]) / ((long double)xi[i] - (long double)xi[j]);
      D[i * n + j] = (double)v;
      diag -= v;
    }
    D[i * n + i] = (double)diag;
  }
  return 0;
}

/* Orthonormal Legendre basis phi_k = sqrt((2k+1)/2) P_k evaluated at the nodes. */
int orc_legendre_vandermonde(int N, const double *xi, double *V) {
  int n = N + 1;
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) {
      long double P, dP;
      legendre_ld(k, xi[j], &P, &dP);
      V[j * n + k] = (double)(sqrtl((2.0L * k + 1.0L) / 2.0L) * P);
    }
  return 0;
}

int orc_invert(int n, const double *A, double *Ainv) {
  double M[NMAX + 1][2 * (NMAX + 1)];
  if (n > NMAX + 1) return -1;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i][j] = (j < n) ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (M[piv][c] == 0.0) return -2;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) { double t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t; }
    double inv = 1.0 / M[c][c];
    for (int j = 0; j < 2 * n; ++j) M[c][j] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = M[r][c];
      for (int j = 0; j < 2 * n; ++j) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i][n + j];
  return 0;
}

/* ======================================================================= */
/* 2. Indexing helpers                                                      */
/* ======================================================================= */

static inline int nidx(int n, int i, int j, int k) { return i + n * (j + n * k); }

/* 3D index of node (i,j,k) and its index along direction d */
static inline void nsplit(int n, int node, int ijk[3]) {
  ijk[0] = node % n; ijk[1] = (node / n) % n; ijk[2] = node / (n * n);
}
static inline int njoin(int n, const int ijk[3]) { return nidx(n, ijk[0], ijk[1], ijk[2]); }

/* volume node of face point (p,q) on local face f */
static int face_node(int N, int f, int p, int q) {
  int n = N + 1, b = (f % 2) ? N : 0;
  switch (f / 2) {
    case 0: return nidx(n, b, p, q);
    case 1: return nidx(n, p, b, q);
    default: return nidx(n, p, q, b);
  }
}

static void orient_map(int N, int orient, int p, int q, int *p2, int *q2) {
  int a = p, b = q;
  if (orient & 4) { a = q; b = p; }
  if (orient & 1) a = N - a;
  if (orient & 2) b = N - b;
  *p2 = a; *q2 = b;
}

/* ======================================================================= */
/* 3. Geometry: curl-form metrics and Jacobian                             */
/* ======================================================================= */

/* derivative along reference direction d of a nodal field f (one element) */
static void dderiv(int N, const double *D, const double *f, int d, double *out) {
  int n = N + 1, nnn = n * n * n;
  for (int node = 0; node < nnn; ++node) {
    int ijk[3];
    nsplit(n, node, ijk);
    int i = ijk[d];
    double s = 0.0;
    for (int m = 0; m < n; ++m) {
      int t[3] = {ijk[0], ijk[1], ijk[2]};
      t[d] = m;
      s += D[i * n + m] * f[njoin(n, t)];
    }
    out[node] = s;
  }
}

/* Ja^i_n = d_k (X_l d_j X_m) - d_j (X_l d_k X_m), (i,j,k) and (n,m,l) cyclic;
 * J = det(dX_c/dxi_j) with derivatives by D.
 * The metric terms do not depend on the coordinate origin (a constant added to X_l cancels
 * since d_j d_k = d_k d_j), so X is taken relative to the element's first node: with absolute
 * coordinates the products X_l d_j X_m are O(|x|/h) larger than the result and round badly. */
int orc_metrics(int N, int n_elems, const double *xyz, double *Ja, double *J) {
  if (N < 1 || N > NMAX) return -1;
  int n = N + 1, nnn = n * n * n;
  double xi[NMAX + 1], w[NMAX + 1], D[(NMAX + 1) * (NMAX + 1)];
  orc_lgl(N, xi, w);
  orc_dmatrix(N, xi, D);
  double *dX = (double *)malloc(sizeof(double) * 9 * nnn);
  double *A = (double *)malloc(sizeof(double) * nnn);
  double *B = (double *)malloc(sizeof(double) * nnn);
  double *dA = (double *)malloc(sizeof(double) * nnn);
  double *dB = (double *)malloc(sizeof(double) * nnn);
  double *X = (double *)malloc(sizeof(double) * 3 * nnn);
  for (int e = 0; e < n_elems; ++e) {
    const double *Xabs = xyz + (size_t)e * 3 * nnn;
    for (int c = 0; c < 3; ++c)
      for (int node = 0; node < nnn; ++node) X[c * nnn + node] = Xabs[c * nnn + node] - Xabs[c * nnn];
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) dderiv(N, D, X + c * nnn, d, dX + (c * 3 + d) * nnn);
    for (int i = 0; i < 3; ++i) {
      int j = (i + 1) % 3, k = (i + 2) % 3;
      for (int c = 0; c < 3; ++c) {
        int m = (c + 1) % 3, l = (c + 2) % 3;
        for (int node = 0; node < nnn; ++node) {
          A[node] = X[l * nnn + node] * dX[(m * 3 + j) * nnn + node];
          B[node] = X[l * nnn + node] * dX[(m * 3 + k) * nnn + node];
        }
        dderiv(N, D, A, k, dA);
        dderiv(N, D, B, j, dB);
        double *out = Ja + (((size_t)e * 3 + i) * 3 + c) * nnn;
        for (int node = 0; node < nnn; ++node) out[node] = dA[node] - dB[node];
      }
    }
    for (int node = 0; node < nnn; ++node) {
      double a[3][3];
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) a[c][d] = dX[(c * 3 + d) * nnn + node];
      J[(size_t)e * nnn + node] = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                                  a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                                  a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    }
  }
  free(X); free(dX); free(A); free(B); free(dA); free(dB);
  return 0;
}

/* ======================================================================= */
/* 4. Pointwise physics                                                     */
/* ======================================================================= */

static void primitive(const orc_real U[5], double gamma, orc_real *rho, orc_real u[3], orc_real *p) {
  *rho = U[0];
  u[0] = U[1] / U[0]; u[1] = U[2] / U[0]; u[2] = U[3] / U[0];
  *p = (gamma - 1.0) * (U[4] - 0.5 * U[0] * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
}

/* Euler flux in Cartesian direction c */
static void flux_cart(const orc_real U[5], int c, double gamma, orc_real F[5]) {
  orc_real rho, u[3], p;
  primitive(U, gamma, &rho, u, &p);
  F[0] = rho * u[c];
  F[1] = U[1] * u[c] + (c == 0 ? p : 0.0);
  F[2] = U[2] * u[c] + (c == 1 ? p : 0.0);
  F[3] = U[3] * u[c] + (c == 2 ? p : 0.0);
  F[4] = (U[4] + p) * u[c];
}

/* contravariant flux F.a = sum_c a_c F_c(U) */
void orc_flux_contra(const orc_real U[5], const double a[3], double gamma, orc_real F[5]) {
  for (int v = 0; v < NVAR; ++v) F[v] = 0.0;
  for (int c = 0; c < 3; ++c) {
    orc_real Fc[5];
    flux_cart(U, c, gamma, Fc);
    for (int v = 0; v < NVAR; ++v) F[v] += a[c] * Fc[v];
  }
}

/* logarithmic mean (a-b)/(ln a - ln b), Ismail-Roe series near a = b */
orc_real orc_logmean(orc_real a, orc_real b) {
  orc_real zeta = a / b;
  orc_real f = (zeta - 1.0) / (zeta + 1.0);
  orc_real u = f * f;
  if (RE(u) < 1e-4) {
    orc_real F = 1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0;
    return (a + b) / (2.0 * F);
  }
  return (a - b) / R_LOG(zeta);
}

/* two-point volume flux with metric average {Ja} (a_avg) */
void orc_twopoint(int kind, const orc_real UL[5], const orc_real UR[5], const double aL[3],
                  const double aR[3], double gamma, orc_real F[5]) {
  double a[3] = {0.5 * (aL[0] + aR[0]), 0.5 * (aL[1] + aR[1]), 0.5 * (aL[2] + aR[2])};
  orc_real rL, uL[3], pL, rR, uR[3], pR;
  primitive(UL, gamma, &rL, uL, &pL);
  primitive(UR, gamma, &rR, uR, &pR);
  orc_real rho_m = 0.5 * (rL + rR), p_m = 0.5 * (pL + pR);
  orc_real u_m[3] = {0.5 * (uL[0] + uR[0]), 0.5 * (uL[1] + uR[1]), 0.5 * (uL[2] + uR[2])};
  orc_real V = u_m[0] * a[0] + u_m[1] * a[1] + u_m[2] * a[2];
  if (kind == ORC_VF_CENTRAL) {
    orc_real FL[5], FR[5];
    orc_flux_contra(UL, a, gamma, FL);
    orc_flux_contra(UR, a, gamma, FR);
    for (int v = 0; v < NVAR; ++v) F[v] = 0.5 * (FL[v] + FR[v]);
    return;
  }
  if (kind == ORC_VF_KG || kind == ORC_VF_PIROZZOLI) {
    F[0] = rho_m * V;
    for (int c = 0; c < 3; ++c) F[1 + c] = rho_m * V * u_m[c] + p_m * a[c];
    if (kind == ORC_VF_KG) {
      orc_real e_m = 0.5 * (UL[4] / rL + UR[4] / rR);           /* total specific energy */
      F[4] = rho_m * V * e_m + p_m * V;
    } else {
      orc_real h_m = 0.5 * ((UL[4] + pL) / rL + (UR[4] + pR) / rR); /* total specific enthalpy */
      F[4] = rho_m * V * h_m;
    }
    return;
  }
  /* Chandrashekar entropy-conservative flux */
  orc_real bL = rL / (2.0 * pL), bR = rR / (2.0 * pR);
  orc_real rho_ln = orc_logmean(rL, rR), beta_ln = orc_logmean(bL, bR);
  orc_real beta_m = 0.5 * (bL + bR);
  orc_real phat = rho_m / (2.0 * beta_m);
  orc_real q2_m = 0.5 * ((uL[0] * uL[0] + uL[1] * uL[1] + uL[2] * uL[2]) +
                       (uR[0] * uR[0] + uR[1] * uR[1] + uR[2] * uR[2]));
  F[0] = rho_ln * V;
  for (int c = 0; c < 3; ++c) F[1 + c] = F[0] * u_m[c] + phat * a[c];
  F[4] = F[0] * (1.0 / (2.0 * (gamma - 1.0) * beta_ln) - 0.5 * q2_m) +
         u_m[0] * F[1] + u_m[1] * F[2] + u_m[2] * F[3];
}

/* Riemann flux F*(UL, UR, n) for a unit normal n */
void orc_riemann(int kind, const orc_real UL[5], const orc_real UR[5], const double n[3],
                 double gamma, orc_real F[5]) {
  if (kind == ORC_SF_EC) {
    orc_twopoint(ORC_VF_EC, UL, UR, n, n, gamma, F);
    return;
  }
  orc_real FL[5], FR[5];
  orc_flux_contra(UL, n, gamma, FL);
  orc_flux_contra(UR, n, gamma, FR);
  orc_real rL, uL[3], pL, rR, uR[3], pR;
  primitive(UL, gamma, &rL, uL, &pL);
  primitive(UR, gamma, &rR, uR, &pR);
  orc_real unL = uL[0] * n[0] + uL[1] * n[1] + uL[2] * n[2];
  orc_real unR = uR[0] * n[0] + uR[1] * n[1] + uR[2] * n[2];
  if (kind == ORC_SF_LLF) {
    orc_real cL = R_SQRT(gamma * pL / rL), cR = R_SQRT(gamma * pR / rR);
    orc_real lam = R_MAX(R_ABS(unL) + cL, R_ABS(unR) + cR);
    for (int v = 0; v < NVAR; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (UR[v] - UL[v]);
    return;
  }
  /* Roe: Roe-averaged state, wave strengths and eigenvectors; no entropy fix */
  orc_real sL = R_SQRT(rL), sR = R_SQRT(rR);
  orc_real ut[3];
  for (int c = 0; c < 3; ++c) ut[c] = (sL * uL[c] + sR * uR[c]) / (sL + sR);
  orc_real HL = (UL[4] + pL) / rL, HR = (UR[4] + pR) / rR;
  orc_real Ht = (sL * HL + sR * HR) / (sL + sR);
  orc_real q2t = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
  orc_real ct = R_SQRT((gamma - 1.0) * (Ht - 0.5 * q2t));
  orc_real rt = sL * sR;
  orc_real unt = ut[0] * n[0] + ut[1] * n[1] + ut[2] * n[2];
  orc_real drho = rR - rL, dp = pR - pL;
  orc_real du[3] = {uR[0] - uL[0], uR[1] - uL[1], uR[2] - uL[2]};
  orc_real dun = du[0] * n[0] + du[1] * n[1] + du[2] * n[2];
  orc_real a1 = (dp - rt * ct * dun) / (2.0 * ct * ct);
  orc_real a5 = (dp + rt * ct * dun) / (2.0 * ct * ct);
  orc_real a2 = drho - dp / (ct * ct);
  orc_real dut[3] = {du[0] - dun * n[0], du[1] - dun * n[1], du[2] - dun * n[2]};
  orc_real l1 = R_ABS(unt - ct), l5 = R_ABS(unt + ct), l2 = R_ABS(unt);
  orc_real diss[5];
  diss[0] = l1 * a1 + l5 * a5 + l2 * a2;
  for (int c = 0; c < 3; ++c)
    diss[1 + c] = l1 * a1 * (ut[c] - ct * n[c]) + l5 * a5 * (ut[c] + ct * n[c]) +
                  l2 * (a2 * ut[c] + rt * dut[c]);
  diss[4] = l1 * a1 * (Ht - unt * ct) + l5 * a5 * (Ht + unt * ct) +
            l2 * (a2 * 0.5 * q2t + rt * (ut[0] * dut[0] + ut[1] * dut[1] + ut[2] * dut[2]));
  for (int v = 0; v < NVAR; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * diss[v];
}

/* Navier-Stokes-Fourier viscous flux, constant mu, Stokes hypothesis */
void orc_viscous_flux(const orc_real U[5], const orc_real gradU[9], const orc_real gradT[3], double mu,
                      double kappa, double gamma, orc_real Fv[15]) {
  orc_real rho, u[3], p;
  primitive(U, gamma, &rho, u, &p);
  orc_real div = gradU[0] + gradU[4] + gradU[8];
  orc_real tau[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      tau[r][c] = mu * (gradU[r * 3 + c] + gradU[c * 3 + r] - (r == c ? 2.0 / 3.0 * div : 0.0));
  for (int c = 0; c < 3; ++c) {
    Fv[c * 5 + 0] = 0.0;
    for (int r = 0; r < 3; ++r) Fv[c * 5 + 1 + r] = tau[r][c];
    Fv[c * 5 + 4] = u[0] * tau[0][c] + u[1] * tau[1][c] + u[2] * tau[2][c] + kappa * gradT[c];
  }
}

/* ======================================================================= */
/* 4b. Wall model (Sec. 3)                                                  */
/* ======================================================================= */

/* Spalding's law of the wall (Eq. (2)): y+ = u+ + 0.1108 [exp(0.4 u+) - 1 - 0.4u+ - (0.4u+)^2/2!
 * - (0.4u+)^3/3! - (0.4u+)^4/4!] */
static orc_real spalding(orc_real up) {
  orc_real k = 0.4 * up;
  return up + 0.1108 * (R_EXP(k) - 1.0 - k - k * k / 2.0 - k * k * k / 6.0 - k * k * k * k / 24.0);
}
/* dy+/du+ */
static orc_real spalding_d(orc_real up) {
  orc_real k = 0.4 * up;
  return 1.0 + 0.1108 * 0.4 * (R_EXP(k) - 1.0 - k - k * k / 2.0 - k * k * k / 6.0);
}

double orc_spalding_yplus(double uplus) {
#ifdef ORC_COMPLEX_STEP
  return creal(spalding(uplus));
#else
  return spalding(uplus);
#endif
}

/* With y+ = h u_tau / nu and u+ = U / u_tau, Spalding's law becomes g(u+) = u+ y+(u+) - Re_h = 0
 * with Re_h = h U / nu. g is increasing and convex for u+ > 0 and y+(u+) >= u+, so the root lies
 * at or below sqrt(Re_h); Newton started at min(sqrt(Re_h), 60) decreases monotonically to it
 * (or overshoots once from below when the root exceeds 60, Re_h > 1.7e11). */
orc_real orc_wall_uplus(orc_real Re_h, int *iters) {
  if (!(RE(Re_h) > 0.0)) { if (iters) *iters = 0; return 0.0; }
  orc_real up = R_SQRT(Re_h);
  if (RE(up) > 60.0) up = 60.0;
  int it = 0;
  for (; it < 100; ++it) {
    orc_real g = up * spalding(up) - Re_h;
    orc_real dg = spalding(up) + up * spalding_d(up);
    orc_real step = g / dg;
    up = up - step;
    if (fabs(RE(step)) <= 1e-15 * fabs(RE(up))) { ++it; break; }
  }
  if (iters) *iters = it;
  return up;
}

/* van Driest transform with freestream edge values (Eq. (5)):
 * u_eq = (u_inf / b) asin(b u / u_inf), b = sqrt(r m) / sqrt(1 + r m), m = (gamma-1)/2 Ma_inf^2,
 * recovery factor r = Pr^(1/3) */
orc_real orc_van_driest(orc_real u, double uinf, double mainf, double gamma, double Pr) {
  double m = 0.5 * (gamma - 1.0) * mainf * mainf * cbrt(Pr);
  double b = sqrt(m) / sqrt(1.0 + m);
  if (!(b > 0.0) || !(uinf > 0.0)) return u;
  return uinf / b * R_ASIN(b * u / uinf);
}

orc_real orc_wall_utau(orc_real U, double h, orc_real nu, double uinf, double mainf, double gamma, double Pr,
                       int van_driest) {
  orc_real ueq = van_driest ? orc_van_driest(U, uinf, mainf, gamma, Pr) : U;
  if (!(RE(ueq) > 0.0)) return 0.0;
  orc_real up = orc_wall_uplus(h * ueq / nu, NULL);
  return ueq / up;
}

/* ======================================================================= */
/* 5. Solver state                                                          */
/* ======================================================================= */

struct orc_state {
  orc_problem pb;
  int N, n, nn, nnn, nE, nF;
  double xi[NMAX + 1], w[NMAX + 1], D[(NMAX + 1) * (NMAX + 1)], Vinv[(NMAX + 1) * (NMAX + 1)];
  double *Ja, *J;
  int *slot_face;   /* [nE][6] global face id */
  int *slot_side;   /* [nE][6] 0 = this element is L, 1 = R */
  int *slot_nbelem; /* [nE][6] neighbour element */
  int *slot_nbnode; /* [nE][6][nn] neighbour volume node facing own face point (p,q) */
  orc_real *grad;     /* [nE][4][3][nnn] lifted gradients of (u,v,w,T) */
  orc_real *Gadv;     /* [nE][6][5][nn] outward advective surface flux, own point order */
  orc_real *Gvis;     /* [nE][6][5][nn] outward viscous surface flux */
  orc_real *alpha_raw;
  unsigned char *mark;
};

static double kappa_of(const orc_problem *pb) {
  return pb->mu * pb->gamma * pb->R / ((pb->gamma - 1.0) * pb->Pr);
}

orc_state *orc_create(const orc_problem *pb, int *status) {
  *status = -1;
  if (pb->N < 1 || pb->N > NMAX || pb->n_elems <= 0 || pb->n_faces <= 0) return NULL;
  orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
  s->pb = *pb;
  s->N = pb->N; s->n = pb->N + 1; s->nn = s->n * s->n; s->nnn = s->nn * s->n;
  s->nE = pb->n_elems; s->nF = pb->n_faces;
  int n = s->n, nn = s->nn, nnn = s->nnn, nE = s->nE;
  orc_lgl(s->N, s->xi, s->w);
  orc_dmatrix(s->N, s->xi, s->D);
  double V[(NMAX + 1) * (NMAX + 1)];
  orc_legendre_vandermonde(s->N, s->xi, V);
  orc_invert(n, V, s->Vinv);
  s->Ja = (double *)malloc(sizeof(double) * 9 * (size_t)nE * nnn);
  s->J = (double *)malloc(sizeof(double) * (size_t)nE * nnn);
  orc_metrics(s->N, nE, pb->xyz, s->Ja, s->J);
  s->slot_face = (int *)malloc(sizeof(int) * 6 * nE);
  s->slot_side = (int *)malloc(sizeof(int) * 6 * nE);
  s->slot_nbelem = (int *)malloc(sizeof(int) * 6 * nE);
  s->slot_nbnode = (int *)malloc(sizeof(int) * 6 * (size_t)nE * nn);
  for (int i = 0; i < 6 * nE; ++i) s->slot_face[i] = -1;
  for (int f = 0; f < s->nF; ++f) {
    const int *F = pb->faces + 5 * f;
    int eL = F[0], fL = F[1], eR = F[2], fR = F[3], o = F[4];
    if (eR == -1) { /* wall face: one slot, the wall model imposes the boundary condition */
      if (eL < 0 || eL >= nE || fL < 0 || fL > 5 || fR != ORC_BC_WALL_MODEL || s->slot_face[eL * 6 + fL] >= 0 ||
          pb->wm_index < 1 || pb->wm_index > pb->N) {
        orc_destroy(s); *status = -2; return NULL;
      }
      s->slot_face[eL * 6 + fL] = f; s->slot_side[eL * 6 + fL] = 0; s->slot_nbelem[eL * 6 + fL] = -1;
      continue;
    }
    if (eL < 0 || eL >= nE || eR < 0 || eR >= nE || fL < 0 || fL > 5 || fR < 0 || fR > 5 || o < 0 || o > 7 ||
        s->slot_face[eL * 6 + fL] >= 0 || s->slot_face[eR * 6 + fR] >= 0) {
      orc_destroy(s); *status = -2; return NULL;
    }
    s->slot_face[eL * 6 + fL] = f; s->slot_side[eL * 6 + fL] = 0; s->slot_nbelem[eL * 6 + fL] = eR;
    s->slot_face[eR * 6 + fR] = f; s->slot_side[eR * 6 + fR] = 1; s->slot_nbelem[eR * 6 + fR] = eL;
    for (int q = 0; q < n; ++q)
      for (int p = 0; p < n; ++p) {
        int p2, q2;
        orient_map(s->N, o, p, q, &p2, &q2);
        s->slot_nbnode[((size_t)eL * 6 + fL) * nn + p + n * q] = face_node(s->N, fR, p2, q2);
        s->slot_nbnode[((size_t)eR * 6 + fR) * nn + p2 + n * q2] = face_node(s->N, fL, p, q);
      }
  }
  for (int i = 0; i < 6 * nE; ++i)
    if (s->slot_face[i] < 0) { orc_destroy(s); *status = -2; return NULL; }
  for (size_t i = 0; i < (size_t)nE * nnn; ++i)
    if (!(s->J[i] > 0.0)) { orc_destroy(s); *status = -3; return NULL; }
  if (pb->equations == ORC_NAVIER_STOKES) { /* viscous buffers only where they are used */
    s->grad = (orc_real *)calloc((size_t)nE * 12 * nnn, sizeof(orc_real));
    s->Gvis = (orc_real *)calloc((size_t)nE * 6 * NVAR * nn, sizeof(orc_real));
  }
  s->Gadv = (orc_real *)calloc((size_t)nE * 6 * NVAR * nn, sizeof(orc_real));
  s->alpha_raw = (orc_real *)calloc(nE, sizeof(orc_real));
  s->mark = (unsigned char *)calloc(nE, 1);
  *status = 0;
  return s;
}

void orc_destroy(orc_state *s) {
  if (!s) return;
  free(s->Ja); free(s->J); free(s->slot_face); free(s->slot_side); free(s->slot_nbelem);
  free(s->slot_nbnode); free(s->grad); free(s->Gadv); free(s->Gvis); free(s->alpha_raw);
  free(s->mark);
  free(s);
}

const double *orc_state_Ja(const orc_state *s) { return s->Ja; }
const double *orc_state_J(const orc_state *s) { return s->J; }

static void load_state(const orc_state *s, const orc_real *U, int e, int node, orc_real out[5]) {
  for (int v = 0; v < NVAR; ++v) out[v] = U[((size_t)e * NVAR + v) * s->nnn + node];
}
static void load_metric(const orc_state *s, int e, int d, int node, double a[3]) {
  for (int c = 0; c < 3; ++c) a[c] = s->Ja[(((size_t)e * 3 + d) * 3 + c) * s->nnn + node];
}
static void load_grad(const orc_state *s, int e, int node, orc_real gU[9], orc_real gT[3]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) gU[r * 3 + c] = s->grad[(((size_t)e * 4 + r) * 3 + c) * s->nnn + node];
  for (int c = 0; c < 3; ++c) gT[c] = s->grad[(((size_t)e * 4 + 3) * 3 + c) * s->nnn + node];
}

/* mirror image of U about the plane with normal direction a (any length): the momentum's normal
 * component changes sign, density and energy stay */
static void wall_ghost(const orc_real U[5], const double a[3], orc_real G[5]) {
  double s = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  double nh[3] = {a[0] / s, a[1] / s, a[2] / s};
  orc_real mn = U[1] * nh[0] + U[2] * nh[1] + U[3] * nh[2];
  G[0] = U[0];
  for (int c = 0; c < 3; ++c) G[1 + c] = U[1 + c] - 2.0 * mn * nh[c];
  G[4] = U[4];
}

/* lifted variables w = (u, v, w, T), T = p/(rho R) */
static void lifted_vars(const orc_state *s, const orc_real U[5], orc_real wv[4]) {
  orc_real rho, u[3], p;
  primitive(U, s->pb.gamma, &rho, u, &p);
  wv[0] = u[0]; wv[1] = u[1]; wv[2] = u[2]; wv[3] = p / (rho * s->pb.R);
}

/* ======================================================================= */
/* 6. BR1 lifting: J grad w = sum_d Ja^d (D_d w) + surface terms (w* - w) s n_out / w_b  */
/* ======================================================================= */

static void lift_element(orc_state *s, const orc_real *U, int e) {
  int N = s->N, n = s->n, nnn = s->nnn;
  orc_real *wv = (orc_real *)malloc(sizeof(orc_real) * 4 * nnn);
  orc_real *Jg = (orc_real *)calloc(12 * (size_t)nnn, sizeof(orc_real));
  for (int node = 0; node < nnn; ++node) {
    orc_real Un[5], t[4];
    load_state(s, U, e, node, Un);
    lifted_vars(s, Un, t);
    for (int q = 0; q < 4; ++q) wv[q * nnn + node] = t[q];
  }
  /* volume part */
  for (int node = 0; node < nnn; ++node) {
    int ijk[3];
    nsplit(n, node, ijk);
    for (int d = 0; d < 3; ++d) {
      double a[3];
      load_metric(s, e, d, node, a);
      for (int q = 0; q < 4; ++q) {
        orc_real dw = 0.0;
        for (int m = 0; m < n; ++m) {
          int t[3] = {ijk[0], ijk[1], ijk[2]};
          t[d] = m;
          dw += s->D[ijk[d] * n + m] * wv[q * nnn + njoin(n, t)];
        }
        for (int c = 0; c < 3; ++c) Jg[(q * 3 + c) * nnn + node] += a[c] * dw;
      }
    }
  }
  /* surface part */
  for (int f = 0; f < 6; ++f) {
    int d = f / 2, sgn = (f % 2) ? 1 : -1;
    double wb = s->w[(f % 2) ? N : 0];
    int nb = s->slot_nbelem[e * 6 + f];
    for (int q = 0; q < n; ++q)
      for (int p = 0; p < n; ++p) {
        int node = face_node(N, f, p, q);
        orc_real Unb[5], wnb[4];
        double a[3];
        load_metric(s, e, d, node, a);
        if (nb < 0) { /* wall: ghost state mirrored about the wall, same temperature */
          orc_real Ui[5];
          load_state(s, U, e, node, Ui);
          wall_ghost(Ui, a, Unb);
        } else {
          load_state(s, U, nb, s->slot_nbnode[((size_t)e * 6 + f) * s->nn + p + n * q], Unb);
        }
        lifted_vars(s, Unb, wnb);
        for (int qv = 0; qv < 4; ++qv) {
          orc_real wown = wv[qv * nnn + node];
          orc_real wstar = 0.5 * (wown + wnb[qv]);
          for (int c = 0; c < 3; ++c) Jg[(qv * 3 + c) * nnn + node] += (wstar - wown) * sgn * a[c] / wb;
        }
      }
  }
  for (int k = 0; k < 12; ++k)
    for (int node = 0; node < nnn; ++node)
      s->grad[((size_t)e * 12 + k) * nnn + node] = Jg[k * nnn + node] / s->J[(size_t)e * nnn + node];
  free(wv); free(Jg);
}

/* ======================================================================= */
/* 7. Modified Persson indicator (Sec. 4.1, Eq. (7))                         */
/* ======================================================================= */

static orc_real indicator_element(const orc_state *s, const orc_real *U, int e) {
  int N = s->N, n = s->n, nnn = s->nnn;
  orc_real *qv = (orc_real *)malloc(sizeof(orc_real) * nnn);
  orc_real *m = (orc_real *)malloc(sizeof(orc_real) * nnn);
  for (int node = 0; node < nnn; ++node) {
    orc_real Un[5], rho, u[3], p;
    load_state(s, U, e, node, Un);
    primitive(Un, s->pb.gamma, &rho, u, &p);
    qv[node] = rho * p;
  }
  /* modal coefficients in the orthonormal Legendre basis: m = (Vinv x Vinv x Vinv) q */
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        orc_real sum = 0.0;
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
              sum += s->Vinv[a * n + i] * s->Vinv[b * n + j] * s->Vinv[c * n + k] * qv[nidx(n, i, j, k)];
        m[nidx(n, a, b, c)] = sum;
      }
  orc_real shell[NMAX + 1] = {0}, tot[NMAX + 1] = {0};
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        int M = a > b ? a : b;
        M = M > c ? M : c;
        shell[M] += m[nidx(n, a, b, c)] * m[nidx(n, a, b, c)];
      }
  for (int M = 0; M <= N; ++M) tot[M] = (M ? tot[M - 1] : 0.0) + shell[M];
  orc_real EN = RE(tot[N]) > 1e-300 ? shell[N] / tot[N] : 0.0;
  orc_real E = EN;
  if (N >= 2) {
    orc_real EN1 = RE(tot[N - 1]) > 1e-300 ? shell[N - 1] / tot[N - 1] : 0.0;
    E = RE(EN1) > RE(EN) ? EN1 : EN;
  }
  double T = 0.5 * pow(10.0, -1.8 * pow(N + 1.0, 0.25));
  orc_real alpha = 1.0 / (1.0 + R_EXP(-s->pb.sharpness / T * (E - T)));
  if (RE(alpha) < s->pb.alpha_min) alpha = 0.0;
  if (RE(alpha) > s->pb.alpha_max) alpha = s->pb.alpha_max;
  free(qv); free(m);
  return alpha;
}

int orc_indicator(orc_state *s, const orc_real *U, orc_real *alpha_raw, orc_real *alpha) {
  for (int e = 0; e < s->nE; ++e) alpha_raw[e] = indicator_element(s, U, e);
  for (int e = 0; e < s->nE; ++e) {
    orc_real a = alpha_raw[e];
    for (int f = 0; f < 6; ++f) {
      if (s->slot_nbelem[e * 6 + f] < 0) continue;
      orc_real b = 0.5 * alpha_raw[s->slot_nbelem[e * 6 + f]];
      if (RE(b) > RE(a)) a = b;
    }
    alpha[e] = a;
  }
  return 0;
}

/* ======================================================================= */
/* 8. FV subcell operator on one element (Sec. 4.1; Hennemann et al. 2021)  */
/* ======================================================================= */

static orc_real minmod(orc_real a, orc_real b) {
  if (RE(a) * RE(b) <= 0.0) return 0.0;
  return (fabs(RE(a)) < fabs(RE(b))) ? a : b;
}

/* Test hook, 0 in every use but one: the reconstruction pins set it to plant a deliberate mistake
 * and check that they then fail. 1: no slopes anywhere (first order everywhere); 2: one-sided slopes
 * in the outer subcells too; 3: states evaluated at the midpoints between nodes instead of at the
 * subcell interfaces; 4: the larger slope where minmod takes the smaller (maxmod); 5: interface
 * metrics averaged from the two neighbouring nodes instead of telescoped from Ja_0. */
int orc_fv_plant = 0;

static orc_real maxmod(orc_real a, orc_real b) {
  if (RE(a) * RE(b) <= 0.0) return 0.0;
  return (fabs(RE(a)) < fabs(RE(b))) ? b : a;
}

static void cons_from_prim(const orc_real q[5], double gamma, orc_real U[5]) {
  U[0] = q[0];
  U[1] = q[0] * q[1]; U[2] = q[0] * q[2]; U[3] = q[0] * q[3];
  U[4] = q[4] / (gamma - 1.0) + 0.5 * q[0] * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
}

/* accFV[5][nnn] (reference-space divergence, before -1/J) */
static void fv_element(const orc_state *s, const orc_real *U, int e, orc_real *accFV) {
  int N = s->N, n = s->n, nnn = s->nnn;
  double gamma = s->pb.gamma;
  double xh[NMAX + 2]; /* subcell interfaces xi_{i+1/2}, i = -1..N */
  xh[0] = -1.0;
  for (int i = 0; i <= N; ++i) xh[i + 1] = xh[i] + s->w[i];
  double xr[NMAX + 2]; /* where the reconstructed states are evaluated: the interfaces */
  for (int i = 0; i <= n; ++i)
    xr[i] = (orc_fv_plant == 3 && i > 0 && i < n) ? 0.5 * (s->xi[i - 1] + s->xi[i]) : xh[i];
  for (size_t i = 0; i < (size_t)NVAR * nnn; ++i) accFV[i] = 0.0;
  for (int d = 0; d < 3; ++d) {
    int fm = 2 * d, fp = 2 * d + 1;
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        /* the line: nodes with (tangential) indices (a,b), running along d */
        int nodes[NMAX + 1];
        for (int i = 0; i < n; ++i) {
          int t[3];
          if (d == 0) { t[0] = i; t[1] = a; t[2] = b; }
          else if (d == 1) { t[0] = a; t[1] = i; t[2] = b; }
          else { t[0] = a; t[1] = b; t[2] = i; }
          nodes[i] = njoin(n, t);
        }
        orc_real q[NMAX + 1][5];
        for (int i = 0; i < n; ++i) {
          orc_real Un[5], rho, u[3], p;
          load_state(s, U, e, nodes[i], Un);
          primitive(Un, gamma, &rho, u, &p);
          q[i][0] = rho; q[i][1] = u[0]; q[i][2] = u[1]; q[i][3] = u[2]; q[i][4] = p;
        }
        /* minmod slopes, interior subcells only; outer subcells first order */
        orc_real qL[NMAX + 1][5], qR[NMAX + 1][5];
        for (int i = 0; i < n; ++i) {
          orc_real sig[5] = {0, 0, 0, 0, 0};
          if (i > 0 && i < N && orc_fv_plant != 1) {
            for (int v = 0; v < 5; ++v) {
              orc_real a = (q[i][v] - q[i - 1][v]) / (s->xi[i] - s->xi[i - 1]);
              orc_real b = (q[i + 1][v] - q[i][v]) / (s->xi[i + 1] - s->xi[i]);
              sig[v] = orc_fv_plant == 4 ? maxmod(a, b) : minmod(a, b);
            }
          } else if (orc_fv_plant == 2) {
            int i0 = i == 0 ? 0 : N - 1;
            for (int v = 0; v < 5; ++v) sig[v] = (q[i0 + 1][v] - q[i0][v]) / (s->xi[i0 + 1] - s->xi[i0]);
          }
          for (int v = 0; v < 5; ++v) {
            qL[i][v] = q[i][v] + sig[v] * (xr[i] - s->xi[i]);
            qR[i][v] = q[i][v] + sig[v] * (xr[i + 1] - s->xi[i]);
          }
          if (RE(qL[i][0]) <= 0.0 || RE(qL[i][4]) <= 0.0 || RE(qR[i][0]) <= 0.0 || RE(qR[i][4]) <= 0.0)
            for (int v = 0; v < 5; ++v) { qL[i][v] = q[i][v]; qR[i][v] = q[i][v]; }
        }
        /* subcell interface metrics: a_{-1/2} = Ja_0, a_{i+1/2} = a_{i-1/2} + w_i (D Ja)_i */
        double ah[NMAX + 2][3], Jl[NMAX + 1][3];
        for (int i = 0; i < n; ++i) load_metric(s, e, d, nodes[i], Jl[i]);
        for (int c = 0; c < 3; ++c) ah[0][c] = Jl[0][c];
        for (int i = 0; i <= N; ++i)
          for (int c = 0; c < 3; ++c) {
            double dj = 0.0;
            for (int m = 0; m < n; ++m) dj += s->D[i * n + m] * Jl[m][c];
            ah[i + 1][c] = ah[i][c] + s->w[i] * dj;
            if (orc_fv_plant == 5 && i < N) ah[i + 1][c] = 0.5 * (Jl[i][c] + Jl[i + 1][c]);
          }
        /* fluxes at the N+2 subcell interfaces, in +xi_d direction */
        orc_real fh[NMAX + 2][5];
        /* element boundaries: the DG surface flux (outward at +, inward at -); the line's
         * tangential indices (a,b) are the face point (p,q) of both end faces */
        for (int v = 0; v < NVAR; ++v) {
          fh[0][v] = -s->Gadv[(((size_t)e * 6 + fm) * NVAR + v) * s->nn + a + n * b];
          fh[n][v] = s->Gadv[(((size_t)e * 6 + fp) * NVAR + v) * s->nn + a + n * b];
        }
        for (int i = 0; i < N; ++i) {
          orc_real UL[5], UR[5];
          double nh[3];
          cons_from_prim(qR[i], gamma, UL);
          cons_from_prim(qL[i + 1], gamma, UR);
          double sa = sqrt(ah[i + 1][0] * ah[i + 1][0] + ah[i + 1][1] * ah[i + 1][1] + ah[i + 1][2] * ah[i + 1][2]);
          for (int c = 0; c < 3; ++c) nh[c] = ah[i + 1][c] / sa;
          orc_real Fs[5];
          orc_riemann(s->pb.sflux, UL, UR, nh, gamma, Fs);
          for (int v = 0; v < NVAR; ++v) fh[i + 1][v] = sa * Fs[v];
        }
        for (int i = 0; i < n; ++i)
          for (int v = 0; v < NVAR; ++v)
            accFV[v * nnn + nodes[i]] += (fh[i + 1][v] - fh[i][v]) / s->w[i];
      }
  }
}

/* ======================================================================= */
/* 9. Right-hand side                                                       */
/* ======================================================================= */

/* Surface fluxes of a wall-modelled wall face (Sec. 3) into the slot of element e, face f:
 *  - advective: the Riemann flux against the mirror state (no penetration);
 *  - viscous (Navier-Stokes): the wall shear stress of the wall model, tau_w = rho u_tau^2,
 *    against the tangential velocity at the exchange node (wm_index nodes from the wall along the
 *    element's wall-normal line, distance h = |x_exchange - x_wall|, nu = mu / rho there), with an
 *    adiabatic wall at rest (no energy flux). */
static void wall_face(orc_state *s, const orc_real *U, int e, int f) {
  const orc_problem *pb = &s->pb;
  int N = s->N, n = s->n, nn = s->nn, nnn = s->nnn;
  int d = f / 2, side = f % 2, sgn = side ? 1 : -1;
  int ns = pb->equations == ORC_NAVIER_STOKES;
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < n; ++p) {
      int node = face_node(N, f, p, q);
      int ijk[3];
      nsplit(n, node, ijk);
      orc_real Ui[5], Ug[5], Fa[5];
      double a[3], nh[3];
      load_state(s, U, e, node, Ui);
      load_metric(s, e, d, node, a);
      double sa = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      for (int c = 0; c < 3; ++c) nh[c] = sgn * a[c] / sa;
      wall_ghost(Ui, a, Ug);
      orc_riemann(pb->sflux, Ui, Ug, nh, pb->gamma, Fa);
      for (int v = 0; v < NVAR; ++v) s->Gadv[(((size_t)e * 6 + f) * NVAR + v) * nn + p + n * q] = sa * Fa[v];
      if (!ns) continue;
      int t[3] = {ijk[0], ijk[1], ijk[2]};
      t[d] = side ? N - pb->wm_index : pb->wm_index;
      int xnode = njoin(n, t);
      orc_real Ux[5], rho, u[3], pr;
      load_state(s, U, e, xnode, Ux);
      primitive(Ux, pb->gamma, &rho, u, &pr);
      double h = 0.0;
      for (int c = 0; c < 3; ++c) {
        double dx = pb->xyz[((size_t)e * 3 + c) * nnn + xnode] - pb->xyz[((size_t)e * 3 + c) * nnn + node];
        h += dx * dx;
      }
      h = sqrt(h);
      orc_real un = u[0] * nh[0] + u[1] * nh[1] + u[2] * nh[2];
      orc_real ut[3] = {u[0] - un * nh[0], u[1] - un * nh[1], u[2] - un * nh[2]};
      orc_real Ut = R_SQRT(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
      orc_real Fv[5] = {0, 0, 0, 0, 0};
      if (RE(Ut) > 0.0) {
        orc_real utau = orc_wall_utau(Ut, h, pb->mu / rho, pb->wm_uinf, pb->wm_mainf, pb->gamma, pb->Pr,
                                      pb->wm_van_driest);
        orc_real tau = rho * utau * utau;
        for (int c = 0; c < 3; ++c) Fv[1 + c] = -tau * ut[c] / Ut; /* outward viscous flux: drag */
      }
      for (int v = 0; v < NVAR; ++v) s->Gvis[(((size_t)e * 6 + f) * NVAR + v) * nn + p + n * q] = sa * Fv[v];
    }
}

int orc_rhs(orc_state *s, const orc_real *U, orc_real *Ut, const unsigned char *out_mask, orc_real *alpha_out) {
  const orc_problem *pb = &s->pb;
  int N = s->N, n = s->n, nn = s->nn, nnn = s->nnn, nE = s->nE;
  int ns = (pb->equations == ORC_NAVIER_STOKES);
  double gamma = pb->gamma, kappa = kappa_of(pb);
  unsigned char *need = s->mark;
  unsigned char *near = (unsigned char *)calloc(nE, 1);
  for (int e = 0; e < nE; ++e) need[e] = out_mask ? (out_mask[e] != 0) : 1;
  for (int e = 0; e < nE; ++e) {
    if (!need[e]) continue;
    near[e] = 1;
    for (int f = 0; f < 6; ++f)
      if (s->slot_nbelem[e * 6 + f] >= 0) near[s->slot_nbelem[e * 6 + f]] = 1;
  }

  /* 1. blending coefficient (indicator on the element and its neighbours) */
  orc_real *alpha = (orc_real *)calloc(nE, sizeof(orc_real));
  if (pb->shock_capturing && pb->alpha_fixed >= 0.0) {
    for (int e = 0; e < nE; ++e) alpha[e] = pb->alpha_fixed;
  } else if (pb->shock_capturing) {
    for (int e = 0; e < nE; ++e)
      if (near[e]) s->alpha_raw[e] = indicator_element(s, U, e);
    for (int e = 0; e < nE; ++e) {
      if (!need[e]) continue;
      orc_real a = s->alpha_raw[e];
      for (int f = 0; f < 6; ++f) {
        if (s->slot_nbelem[e * 6 + f] < 0) continue;
        orc_real b = 0.5 * s->alpha_raw[s->slot_nbelem[e * 6 + f]];
        if (RE(b) > RE(a)) a = b;
      }
      alpha[e] = a;
    }
  }

  /* 2. BR1 lifting on every element whose gradient a needed face or volume uses */
  if (ns)
    for (int e = 0; e < nE; ++e)
      if (near[e]) lift_element(s, U, e);

  /* 3. surface fluxes, once per face, stored outward for both sides */
  for (int f = 0; f < s->nF; ++f) {
    const int *F = pb->faces + 5 * f;
    int eL = F[0], fL = F[1], eR = F[2], fR = F[3], o = F[4];
    if (eR < 0) {
      if (need[eL]) wall_face(s, U, eL, fL);
      continue;
    }
    if (!need[eL] && !need[eR]) continue;
    int dL = fL / 2, sgnL = (fL % 2) ? 1 : -1;
    for (int q = 0; q < n; ++q)
      for (int p = 0; p < n; ++p) {
        int p2, q2;
        orient_map(N, o, p, q, &p2, &q2);
        int nodeL = face_node(N, fL, p, q), nodeR = face_node(N, fR, p2, q2);
        orc_real UL[5], UR[5], Fa[5], Fv[5] = {0, 0, 0, 0, 0};
        double a[3], nh[3];
        load_state(s, U, eL, nodeL, UL);
        load_state(s, U, eR, nodeR, UR);
        load_metric(s, eL, dL, nodeL, a);
        double sa = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        for (int c = 0; c < 3; ++c) nh[c] = sgnL * a[c] / sa;
        orc_riemann(pb->sflux, UL, UR, nh, gamma, Fa);
        if (ns) {
          orc_real gUL[9], gTL[3], gUR[9], gTR[3], FvL[15], FvR[15];
          load_grad(s, eL, nodeL, gUL, gTL);
          load_grad(s, eR, nodeR, gUR, gTR);
          orc_viscous_flux(UL, gUL, gTL, pb->mu, kappa, gamma, FvL);
          orc_viscous_flux(UR, gUR, gTR, pb->mu, kappa, gamma, FvR);
          for (int v = 0; v < NVAR; ++v) {
            Fv[v] = 0.0;
            for (int c = 0; c < 3; ++c) Fv[v] += 0.5 * (FvL[c * 5 + v] + FvR[c * 5 + v]) * nh[c];
          }
        }
        for (int v = 0; v < NVAR; ++v) {
          s->Gadv[(((size_t)eL * 6 + fL) * NVAR + v) * nn + p + n * q] = sa * Fa[v];
          s->Gadv[(((size_t)eR * 6 + fR) * NVAR + v) * nn + p2 + n * q2] = -sa * Fa[v];
          if (ns) {
            s->Gvis[(((size_t)eL * 6 + fL) * NVAR + v) * nn + p + n * q] = sa * Fv[v];
            s->Gvis[(((size_t)eR * 6 + fR) * NVAR + v) * nn + p2 + n * q2] = -sa * Fv[v];
          }
        }
      }
  }

  /* 4. volume integral, surface terms, Jacobian; optional FV blend */
  orc_real *acc_a = (orc_real *)malloc(sizeof(orc_real) * NVAR * nnn);
  orc_real *acc_v = (orc_real *)malloc(sizeof(orc_real) * NVAR * nnn);
  orc_real *accFV = (orc_real *)malloc(sizeof(orc_real) * NVAR * nnn);
  orc_real *Fvc = (orc_real *)malloc(sizeof(orc_real) * 3 * NVAR * nnn); /* contravariant viscous flux */
  for (int e = 0; e < nE; ++e) {
    if (!need[e]) {
      for (int v = 0; v < NVAR; ++v)
        for (int node = 0; node < nnn; ++node) Ut[((size_t)e * NVAR + v) * nnn + node] = 0.0;
      continue;
    }
    if (ns)
      for (int node = 0; node < nnn; ++node) {
        orc_real Un[5], gU[9], gT[3], Fv[15];
        load_state(s, U, e, node, Un);
        load_grad(s, e, node, gU, gT);
        orc_viscous_flux(Un, gU, gT, pb->mu, kappa, gamma, Fv);
        for (int d = 0; d < 3; ++d) {
          double a[3];
          load_metric(s, e, d, node, a);
          for (int v = 0; v < NVAR; ++v)
            Fvc[(d * NVAR + v) * nnn + node] = a[0] * Fv[0 * 5 + v] + a[1] * Fv[1 * 5 + v] + a[2] * Fv[2 * 5 + v];
        }
      }
    for (int node = 0; node < nnn; ++node) {
      int ijk[3];
      nsplit(n, node, ijk);
      orc_real Ui[5], sa[5] = {0, 0, 0, 0, 0}, sv[5] = {0, 0, 0, 0, 0};
      load_state(s, U, e, node, Ui);
      for (int d = 0; d < 3; ++d) {
        double ai[3];
        load_metric(s, e, d, node, ai);
        for (int m = 0; m < n; ++m) {
          int t[3] = {ijk[0], ijk[1], ijk[2]};
          t[d] = m;
          int nm = njoin(n, t);
          orc_real Um[5], Fs[5];
          double am[3];
          load_state(s, U, e, nm, Um);
          load_metric(s, e, d, nm, am);
          orc_twopoint(pb->vflux, Ui, Um, ai, am, gamma, Fs);
          double Dim = s->D[ijk[d] * n + m];
          for (int v = 0; v < NVAR; ++v) sa[v] += 2.0 * Dim * Fs[v];
          if (ns)
            for (int v = 0; v < NVAR; ++v) sv[v] += Dim * Fvc[(d * NVAR + v) * nnn + nm];
        }
        /* surface terms at the faces this node lies on */
        for (int side = 0; side < 2; ++side) {
          int b = side ? N : 0;
          if (ijk[d] != b) continue;
          int f = 2 * d + side, sgn = side ? 1 : -1;
          int p = (d == 0) ? ijk[1] : ijk[0];
          int q = (d == 2) ? ijk[1] : ijk[2];
          orc_real Fi[5];
          orc_flux_contra(Ui, ai, gamma, Fi);
          for (int v = 0; v < NVAR; ++v) {
            sa[v] += (s->Gadv[(((size_t)e * 6 + f) * NVAR + v) * nn + p + n * q] - sgn * Fi[v]) / s->w[b];
            if (ns)
              sv[v] += (s->Gvis[(((size_t)e * 6 + f) * NVAR + v) * nn + p + n * q] -
                        sgn * Fvc[(d * NVAR + v) * nnn + node]) / s->w[b];
          }
        }
      }
      for (int v = 0; v < NVAR; ++v) { acc_a[v * nnn + node] = sa[v]; acc_v[v * nnn + node] = sv[v]; }
    }
    orc_real al = alpha[e];
    if (pb->shock_capturing && RE(al) > 0.0) fv_element(s, U, e, accFV);
    for (int v = 0; v < NVAR; ++v)
      for (int node = 0; node < nnn; ++node) {
        double Jn = s->J[(size_t)e * nnn + node];
        orc_real adv_dg = -acc_a[v * nnn + node] / Jn;
        orc_real adv = adv_dg;
        if (pb->shock_capturing && RE(al) > 0.0) {
          orc_real adv_fv = -accFV[v * nnn + node] / Jn;
          adv = al * adv_fv + (1.0 - al) * adv_dg;
        }
        Ut[((size_t)e * NVAR + v) * nnn + node] = adv + (ns ? acc_v[v * nnn + node] / Jn : 0.0);
      }
  }
  if (alpha_out)
    for (int e = 0; e < nE; ++e) alpha_out[e] = alpha[e];
  free(acc_a); free(acc_v); free(accFV); free(Fvc); free(alpha); free(near);
  return 0;
}

/* ======================================================================= */
/* 10. LSERK(5,4), Carpenter-Kennedy 2N-storage                             */
/* ======================================================================= */

void orc_lserk_coefficients(double A[5], double B[5], double c[5]) {
  A[0] = 0.0;
  A[1] = -567301805773.0 / 1357537059087.0;
  A[2] = -2404267990393.0 / 2016746695238.0;
  A[3] = -3550918686646.0 / 2091501179385.0;
  A[4] = -1275806237668.0 / 842570457699.0;
  B[0] = 1432997174477.0 / 9575080441755.0;
  B[1] = 5161836677717.0 / 13612068292357.0;
  B[2] = 1720146321549.0 / 2090206949498.0;
  B[3] = 3134564353537.0 / 4481467310338.0;
  B[4] = 2277821191437.0 / 14882151754819.0;
  c[0] = 0.0;
  c[1] = 1432997174477.0 / 9575080441755.0;
  c[2] = 2526269341429.0 / 6820363962896.0;
  c[3] = 2006345519317.0 / 3224310063776.0;
  c[4] = 2802321613138.0 / 2924317926251.0;
}

/* g := 0; for each stage s: g = A_s g + dt f(u, t + c_s dt); u = u + B_s g */
int orc_lserk_generic(int n, orc_real *u, double dt, double t, orc_rhs_fn f, void *ctx) {
  double A[5], B[5], c[5];
  orc_lserk_coefficients(A, B, c);
  orc_real *g = (orc_real *)calloc(n, sizeof(orc_real));
  orc_real *ut = (orc_real *)malloc(sizeof(orc_real) * n);
  for (int st = 0; st < 5; ++st) {
    f(u, ut, t + c[st] * dt, ctx);
    for (int i = 0; i < n; ++i) {
      g[i] = A[st] * g[i] + dt * ut[i];
      u[i] = u[i] + B[st] * g[i];
    }
  }
  free(g); free(ut);
  return 0;
}

static void dg_rhs_cb(const orc_real *u, orc_real *ut, double t, void *ctx) {
  (void)t;
  orc_rhs((orc_state *)ctx, u, ut, NULL, NULL);
}

int orc_lserk_step(orc_state *s, orc_real *U, double dt, double t) {
  return orc_lserk_generic(s->nE * NVAR * s->nnn, U, dt, t, dg_rhs_cb, s);
}

/* ======================================================================= */
/* 11. Integral invariants and time-step estimate                           */
/* ======================================================================= */

/* out[0..4] = sum J w Ut_v; out[5] = sum J w (v . Ut), v = entropy variables;
 * out[6] = sum J w (rho |u|^2 / 2); out[7] = sum J w d/dt(rho |u|^2 / 2) */
int orc_invariants(orc_state *s, const orc_real *U, const orc_real *Ut, orc_real out[8]) {
  int n = s->n, nnn = s->nnn;
  double gamma = s->pb.gamma;
  for (int k = 0; k < 8; ++k) out[k] = 0.0;
  for (int e = 0; e < s->nE; ++e)
    for (int node = 0; node < nnn; ++node) {
      int ijk[3];
      nsplit(n, node, ijk);
      double wq = s->w[ijk[0]] * s->w[ijk[1]] * s->w[ijk[2]] * s->J[(size_t)e * nnn + node];
      orc_real Un[5], Utn[5], rho, u[3], p;
      load_state(s, U, e, node, Un);
      load_state(s, Ut, e, node, Utn);
      primitive(Un, gamma, &rho, u, &p);
      orc_real q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
      orc_real sent = R_LOG(p) - gamma * R_LOG(rho);
      orc_real v[5] = {(gamma - sent) / (gamma - 1.0) - rho * q2 / (2.0 * p), rho * u[0] / p, rho * u[1] / p,
                     rho * u[2] / p, -rho / p};
      for (int k = 0; k < 5; ++k) out[k] += wq * Utn[k];
      out[5] += wq * (v[0] * Utn[0] + v[1] * Utn[1] + v[2] * Utn[2] + v[3] * Utn[3] + v[4] * Utn[4]);
      out[6] += wq * 0.5 * rho * q2;
      out[7] += wq * (u[0] * Utn[1] + u[1] * Utn[2] + u[2] * Utn[3] - 0.5 * q2 * Utn[0]);
    }
  return 0;
}

/* dt = cfl * min over nodes of 2 J / ((2N+1) sum_d (|u . Ja^d| + c |Ja^d|)) */
int orc_max_dt(orc_state *s, const orc_real *U, double cfl, double *dt) {
  int nnn = s->nnn;
  double best = INFINITY;
  for (int e = 0; e < s->nE; ++e)
    for (int node = 0; node < nnn; ++node) {
      orc_real Un[5], rho, u[3], p;
      load_state(s, U, e, node, Un);
      primitive(Un, s->pb.gamma, &rho, u, &p);
      double c = sqrt(s->pb.gamma * RE(p) / RE(rho)), lam = 0.0;
      for (int d = 0; d < 3; ++d) {
        double a[3];
        load_metric(s, e, d, node, a);
        lam += fabs(RE(u[0]) * a[0] + RE(u[1]) * a[1] + RE(u[2]) * a[2]) + c * sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      }
      double v = 2.0 * s->J[(size_t)e * nnn + node] / ((2.0 * s->N + 1.0) * lam);
      if (v < best) best = v;
    }
  *dt = cfl * best;
  return 0;
}
