"""Pins of the oracle's curl-form metrics and Jacobian: affine closed forms, the discrete
metric identities that give freestream preservation on curved meshes, and convergence to
the analytic cofactor matrix of the sine map x' = x + 0.05 sin x sin y sin z."""
import math

import numpy as np
import pytest

from paper_2306_12891_gb300 import workloads as W


def test_affine_metrics(oracle_mod):
    N = 4
    xyz, _ = W.box_mesh(N, (2, 3, 5), lo=(0, -1, 2), hi=(3, 2, 7))
    Ja, J = oracle_mod.metrics(N, xyz)
    hx, hy, hz = 3 / 2, 3 / 3, 5 / 5
    np.testing.assert_allclose(J, hx * hy * hz / 8, rtol=1e-13)
    expect = np.diag([hy * hz / 4, hx * hz / 4, hx * hy / 4])
    for d in range(3):
        for c in range(3):
            np.testing.assert_allclose(Ja[:, d, c], expect[d, c], rtol=0, atol=1e-13)


def test_affine_metrics_far_from_the_origin(oracle_mod):
    """Fine elements at coordinates ~2*pi: the metric terms must not lose accuracy to the
    coordinate offset (they are translation invariant)."""
    N = 7
    for K in (4, 32):
        xyz, _ = W.box_mesh(N, (K, K, K))
        last = xyz[-1:]  # the element farthest from the origin
        Ja, J = oracle_mod.metrics(N, last)
        h2 = np.pi / K
        # the node coordinates themselves carry ~1e-16 * 2 pi of rounding, which |D| ~ N^2/4
        # amplifies to a few 1e-13 relative; absolute coordinates in the products cost 3e-12
        # (K = 4) and 1e-10 (K = 32)
        np.testing.assert_allclose(J, h2 ** 3, rtol=5e-13)
        np.testing.assert_allclose(Ja[:, 0, 0], h2 ** 2, rtol=5e-13)
        assert np.abs(Ja[:, 0, 1:]).max() < 5e-13 * h2 ** 2


def _divergence(D, F):
    """sum_d D_d F^d over one element's nodal arrays F[d][k][j][i]."""
    out = np.einsum("im,kjm->kji", D, F[0])
    out += np.einsum("jm,kmi->kji", D, F[1])
    out += np.einsum("km,mji->kji", D, F[2])
    return out


def _generic_map(x, y, z):
    return (x + 0.1 * np.sin(y) * np.cos(z), y + 0.1 * np.sin(z) * np.sin(x) + 0.05 * np.sin(2 * x),
            z + 0.1 * np.sin(x) * np.cos(y))


@pytest.mark.parametrize("mapping", ["sine_0.05", "generic"])
@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_discrete_metric_identities_on_curved_mesh(oracle_mod, N, mapping):
    xyz, _ = W.box_mesh(N, (3, 2, 2), mapping=_generic_map if mapping == "generic" else mapping)
    Ja, J = oracle_mod.metrics(N, xyz)
    D = oracle_mod.dmatrix(N)
    worst = 0.0
    for e in range(xyz.shape[0]):
        for c in range(3):
            worst = max(worst, np.abs(_divergence(D, Ja[e, :, c])).max())
    assert worst < 1e-13 * N * N
    assert (J > 0).all()
    # the nodal cross-product form x_eta x x_zeta (same geometry) violates the identity,
    # so this pin can fail
    if N >= 3 and mapping == "generic":
        X = xyz[0]
        dX = np.stack([np.einsum("im,ckjm->ckji", D, X), np.einsum("jm,ckmi->ckji", D, X),
                       np.einsum("km,cmji->ckji", D, X)], 0)  # [d][c]
        cross = np.stack([np.cross(dX[1], dX[2], axis=0), np.cross(dX[2], dX[0], axis=0),
                          np.cross(dX[0], dX[1], axis=0)], 0)  # [d][c]
        assert max(np.abs(_divergence(D, cross[:, c])).max() for c in range(3)) > 1e-8


def _analytic_sine_map(x, y, z):
    s = 0.05
    g = np.stack([s * np.cos(x) * np.sin(y) * np.sin(z), s * np.sin(x) * np.cos(y) * np.sin(z),
                  s * np.sin(x) * np.sin(y) * np.cos(z)])  # grad of the perturbation
    detA = 1.0 + g.sum(0)
    return g, detA


def test_metrics_converge_to_analytic_cofactors(oracle_mod):
    """x = X(xi) = sine map of an affine cell of width h: J = (h/2)^3 det A,
    Ja^d_c = (h/2)^2 [(1 + sum g) delta_dc - g_c] with A = I + 1 g^T."""
    errs = []
    for N in (3, 5, 7):
        nel = 3
        h = 2 * math.pi / nel
        xyz, _ = W.box_mesh(N, (nel, nel, nel))
        Ja, J = oracle_mod.metrics(N, W.box_mesh(N, (nel, nel, nel), mapping="sine_0.05")[0])
        x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
        g, detA = _analytic_sine_map(x, y, z)
        eJ = np.abs(J - (h / 2) ** 3 * detA).max()
        eJa = 0.0
        for d in range(3):
            for c in range(3):
                exact = (h / 2) ** 2 * ((1 + g.sum(0)) * (d == c) - g[c])
                eJa = max(eJa, np.abs(Ja[:, d, c] - exact).max())
        errs.append((eJ, eJa))
    assert errs[-1][0] < 1e-5 and errs[-1][1] < 1e-5
    assert errs[0][0] > 10 * errs[-1][0] and errs[0][1] > 10 * errs[-1][1]
