"""Pins of the oracle's LGL basis (nodes, weights, derivative matrix, Legendre Vandermonde)
against closed forms, quadrature exactness, the summation-by-parts identity the split form
relies on (Sec. 4.1) and numpy's own Legendre root finder."""
import math

import numpy as np
import pytest

from paper_2306_12891_gb300 import workloads as W

S5 = 1.0 / math.sqrt(5.0)
S37 = math.sqrt(3.0 / 7.0)
CLOSED = {
    1: ([-1.0, 1.0], [1.0, 1.0]),
    2: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1.0, -S5, S5, 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1.0, -S37, 0.0, S37, 1.0], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("N", sorted(CLOSED))
def test_lgl_closed_forms(oracle_mod, N):
    xi, w = oracle_mod.lgl(N)
    np.testing.assert_allclose(xi, CLOSED[N][0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, CLOSED[N][1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", range(1, 16))
def test_lgl_matches_numpy_and_quadrature(oracle_mod, N):
    xi, w = oracle_mod.lgl(N)
    np.testing.assert_allclose(xi, W.lgl_points(N), rtol=0, atol=4e-15)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * N):  # exact to degree 2N-1
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, xi ** k) - exact) < 2e-14
    # and not exact at degree 2N (so the pin above can fail)
    assert abs(np.dot(w, xi ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-11


@pytest.mark.parametrize("N", range(1, 12))
def test_dmatrix_polynomial_exactness_and_sbp(oracle_mod, N):
    xi, w = oracle_mod.lgl(N)
    D = oracle_mod.dmatrix(N, xi)
    for k in range(0, N + 1):
        dk = k * xi ** (k - 1) if k > 0 else np.zeros_like(xi)
        assert np.abs(D @ xi ** k - dk).max() <= 1e-13 * N * N
    # summation by parts: W D + (W D)^T = B = diag(-1, 0, ..., 0, 1)
    Q = np.diag(w) @ D
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    assert np.abs(Q + Q.T - B).max() < 1e-13 * N
    assert abs(D[0, 0] + N * (N + 1) / 4.0) < 1e-12 * N * N
    assert abs(D[N, N] - N * (N + 1) / 4.0) < 1e-12 * N * N
    # interior diagonal vanishes (nodes symmetric about 0)
    if N >= 2:
        assert np.abs(np.diag(D)[1:-1]).max() < 1e-12 * N


@pytest.mark.parametrize("N", range(1, 10))
def test_legendre_vandermonde_orthonormal(oracle_mod, N):
    xi, w = oracle_mod.lgl(N)
    V = oracle_mod.legendre_vandermonde(N, xi)
    M = V.T @ np.diag(w) @ V
    for k in range(N + 1):
        for l in range(N + 1):
            if k + l <= 2 * N - 1:  # products LGL quadrature integrates exactly
                assert abs(M[k, l] - (1.0 if k == l else 0.0)) < 1e-13
    # the modes are the Legendre polynomials scaled to unit L2 norm: phi_1 = sqrt(3/2) x
    np.testing.assert_allclose(V[:, 1], math.sqrt(1.5) * xi, rtol=0, atol=1e-15)
    np.testing.assert_allclose(V[:, 0], math.sqrt(0.5), rtol=0, atol=1e-15)
