// dg_basis.cpp -- host construction of the Legendre-Gauss-Lobatto tables (Sec. 2: split-form DG
// on LGL nodes) that the kernels read from constant memory.
//
//  - nodes: roots of q(x) = L_{N+1}(x) - L_{N-1}(x) (= c (x^2-1) L_N'(x)), Newton with q' = (2N+1) L_N;
//  - weights: w_j = 2 / (N(N+1) L_N(x_j)^2);
//  - derivative matrix, closed form for LGL nodes: D_ij = L_N(x_i) / (L_N(x_j) (x_i - x_j)) for i != j,
//    D_00 = -N(N+1)/4, D_NN = N(N+1)/4, zero diagonal otherwise;
//  - inverse of the orthonormal Legendre Vandermonde V_jk = sqrt((2k+1)/2) L_k(x_j) from the
//    discrete orthogonality of LGL quadrature: V^-1 = diag(1/g_k) V^T W, g_k = 1 (k < N),
//    g_N = (2N+1)/N (the quadrature is inexact for L_N^2).
#include <cmath>

#include "dg_internal.h"

namespace {

typedef long double ld;

// L_0..L_K at x by the Bonnet recurrence
void legendre_all(int K, ld x, ld *L) {
  L[0] = 1.0L;
  if (K >= 1) L[1] = x;
  for (int k = 1; k < K; ++k) L[k + 1] = ((2 * k + 1) * x * L[k] - k * L[k - 1]) / (k + 1);
}

}  // namespace

int dg_build_tables(int N, DgTables *t) {
  if (N < 1 || N > DG_NMAX || !t) return -1;
  const int n = N + 1;
  t->N = N;
  ld x[DG_NMAX + 1], LN[DG_NMAX + 1];
  ld L[DG_NMAX + 3];
  x[0] = -1.0L;
  x[N] = 1.0L;
  for (int j = 1; j < N; ++j) {
    // start from the Chebyshev-Gauss-Lobatto point, refine by Newton on q
    ld z = -std::cos((ld)M_PI * (ld)j / (ld)N);
    for (int it = 0; it < 60; ++it) {
      legendre_all(N + 1, z, L);
      ld q = L[N + 1] - L[N - 1];
      ld dq = (2 * N + 1) * L[N];
      ld step = q / dq;
      z -= step;
      if (std::fabs((double)step) < 1e-19) break;
    }
    x[j] = z;
  }
  for (int j = 1; j < (N + 1) / 2; ++j) {  // enforce the symmetry of the node set
    ld s = 0.5L * (x[N - j] - x[j]);
    x[j] = -s;
    x[N - j] = s;
  }
  if (N % 2 == 0) x[N / 2] = 0.0L;
  for (int j = 0; j < n; ++j) {
    legendre_all(N, x[j], L);
    LN[j] = L[N];
    t->xi[j] = (double)x[j];
    t->w[j] = (double)(2.0L / ((ld)N * (N + 1) * L[N] * L[N]));
    t->invw[j] = (double)(((ld)N * (N + 1) * L[N] * L[N]) / 2.0L);
  }
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < n; ++m) {
      ld v;
      if (i != m) v = LN[i] / (LN[m] * (x[i] - x[m]));
      else if (i == 0) v = -(ld)N * (N + 1) / 4.0L;
      else if (i == N) v = (ld)N * (N + 1) / 4.0L;
      else v = 0.0L;
      t->D[i * n + m] = (double)v;
    }
  for (int k = 0; k < n; ++k) {
    ld g = (k < N) ? 1.0L : (ld)(2 * N + 1) / (ld)N;
    ld nk = std::sqrt((ld)(2 * k + 1) / 2.0L);
    for (int j = 0; j < n; ++j) {
      legendre_all(N, x[j], L);
      ld wj = 2.0L / ((ld)N * (N + 1) * LN[j] * LN[j]);
      t->Vinv[k * n + j] = (double)(nk * L[k] * wj / g);
    }
  }
  t->xh[0] = -1.0;
  ld acc = -1.0L;
  for (int i = 0; i < n; ++i) {
    acc += 2.0L / ((ld)N * (N + 1) * LN[i] * LN[i]);
    t->xh[i + 1] = (double)acc;
  }
  t->xh[n] = 1.0;
  return 0;
}
