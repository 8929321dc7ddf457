"""Pins of the oracle's pointwise fluxes: consistency and symmetry of the split-form two-point
fluxes, Tadmor's entropy-conservation condition for the EC flux, Riemann-flux consistency,
conservation and upwinding, the stationary contact for Roe, the logarithmic mean against
high-precision arithmetic, and the Navier-Stokes-Fourier viscous flux in closed-form cases."""
import math

import numpy as np
import pytest

GAMMA = 1.4


def rand_state(rng, vel=1.0):
    rho = rng.uniform(0.5, 2.0)
    u = rng.uniform(-vel, vel, 3)
    p = rng.uniform(0.5, 2.0)
    E = p / (GAMMA - 1) + 0.5 * rho * u @ u
    return np.array([rho, rho * u[0], rho * u[1], rho * u[2], E])


def prim(U):
    rho = U[0]
    u = U[1:4] / rho
    p = (GAMMA - 1) * (U[4] - 0.5 * rho * u @ u)
    return rho, u, p


def entropy_vars_and_potential(U, n):
    rho, u, p = prim(U)
    s = math.log(p) - GAMMA * math.log(rho)
    v = np.array([(GAMMA - s) / (GAMMA - 1) - rho * (u @ u) / (2 * p), rho * u[0] / p, rho * u[1] / p,
                  rho * u[2] / p, -rho / p])
    psi = rho * (u @ n)  # flux potential of the entropy -rho s/(gamma-1)
    return v, psi


@pytest.mark.parametrize("kind", ["kg", "pirozzoli", "ec", "central"])
def test_twopoint_consistent_and_symmetric(oracle_mod, kind):
    rng = np.random.default_rng(1)
    for _ in range(50):
        UL, UR = rand_state(rng), rand_state(rng)
        aL, aR = rng.normal(size=3), rng.normal(size=3)
        F = oracle_mod.twopoint(kind, UL, UL, aL, aL)
        np.testing.assert_allclose(F, oracle_mod.flux_contra(UL, aL), rtol=1e-13, atol=1e-13)
        F1 = oracle_mod.twopoint(kind, UL, UR, aL, aR)
        F2 = oracle_mod.twopoint(kind, UR, UL, aR, aL)
        np.testing.assert_allclose(F1, F2, rtol=1e-14, atol=1e-14)


def test_euler_flux_of_rest_state_is_pressure(oracle_mod):
    U = np.array([1.3, 0.0, 0.0, 0.0, 2.0 / (GAMMA - 1)])
    a = np.array([0.3, -1.2, 0.7])
    np.testing.assert_allclose(oracle_mod.flux_contra(U, a), [0, 2 * 0.3, -2 * 1.2, 2 * 0.7, 0], atol=1e-15)


def test_kg_and_pirozzoli_share_mass_and_momentum(oracle_mod):
    rng = np.random.default_rng(2)
    UL, UR = rand_state(rng), rand_state(rng)
    a = rng.normal(size=3)
    Fk = oracle_mod.twopoint("kg", UL, UR, a, a)
    Fp = oracle_mod.twopoint("pirozzoli", UL, UR, a, a)
    np.testing.assert_allclose(Fk[:4], Fp[:4], rtol=1e-15)
    assert abs(Fk[4] - Fp[4]) > 1e-6


def test_ec_flux_satisfies_tadmor_condition(oracle_mod):
    """(v_R - v_L) . F = psi_R - psi_L for Chandrashekar's flux, unit normal or metric vector."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        UL, UR = rand_state(rng), rand_state(rng)
        n = rng.normal(size=3)
        if rng.uniform() < 0.5:
            n /= np.linalg.norm(n)
        F = oracle_mod.twopoint("ec", UL, UR, n, n)
        vL, psiL = entropy_vars_and_potential(UL, n)
        vR, psiR = entropy_vars_and_potential(UR, n)
        lhs, rhs = (vR - vL) @ F, psiR - psiL
        assert abs(lhs - rhs) <= 1e-12 * (1 + np.abs(vR - vL) @ np.abs(F))
    # nearly equal states exercise the series branch of the log mean
    UL = rand_state(rng)
    UR = UL * (1 + 1e-7)
    n = np.array([0.0, 1.0, 0.0])
    F = oracle_mod.twopoint("ec", UL, UR, n, n)
    vL, psiL = entropy_vars_and_potential(UL, n)
    vR, psiR = entropy_vars_and_potential(UR, n)
    assert abs((vR - vL) @ F - (psiR - psiL)) < 1e-14


def test_ec_flux_is_not_kg(oracle_mod):
    rng = np.random.default_rng(4)
    UL, UR = rand_state(rng), rand_state(rng)
    n = np.array([1.0, 0, 0])
    vL, psiL = entropy_vars_and_potential(UL, n)
    vR, psiR = entropy_vars_and_potential(UR, n)
    F = oracle_mod.twopoint("kg", UL, UR, n, n)
    assert abs((vR - vL) @ F - (psiR - psiL)) > 1e-6  # the Tadmor pin above can fail


def test_logmean_against_mpmath(oracle_mod):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for a, b in [(1.0, 1.0 + 1e-9), (2.0, 2.0 * (1 + 1e-5)), (1.0, 1.02), (1.0, 1.1), (3.0, 1.5), (0.1, 10.0)]:
        exact = (mp.mpf(a) - mp.mpf(b)) / (mp.log(mp.mpf(a)) - mp.log(mp.mpf(b)))
        got = oracle_mod.logmean(a, b)
        assert abs(got - float(exact)) <= 1e-15 * float(exact)  # a few ulp
        assert oracle_mod.logmean(b, a) == pytest.approx(got, rel=1e-15)
    assert oracle_mod.logmean(1.7, 1.7) == pytest.approx(1.7, rel=1e-16)


@pytest.mark.parametrize("kind", ["llf", "roe", "ec"])
def test_riemann_consistent_and_conservative(oracle_mod, kind):
    rng = np.random.default_rng(5)
    for _ in range(50):
        UL, UR = rand_state(rng), rand_state(rng)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        np.testing.assert_allclose(oracle_mod.riemann(kind, UL, UL, n), oracle_mod.flux_contra(UL, n),
                                   rtol=1e-13, atol=1e-13)
        # the flux leaving L through n enters R through -n
        np.testing.assert_allclose(oracle_mod.riemann(kind, UL, UR, n), -oracle_mod.riemann(kind, UR, UL, -n),
                                   rtol=1e-13, atol=1e-13)


def test_roe_stationary_contact_is_exact(oracle_mod):
    n = np.array([0.6, 0.0, 0.8])
    t = np.array([0.8, 0.0, -0.6])
    for rhoL, rhoR in [(1.0, 3.0), (0.2, 0.9)]:
        p = 1.7
        UL = np.array([rhoL, 0.4 * rhoL * t[0], 0.0, 0.4 * rhoL * t[2], p / (GAMMA - 1) + 0.5 * rhoL * 0.16])
        UR = np.array([rhoR, -0.3 * rhoR * t[0], 0.0, -0.3 * rhoR * t[2], p / (GAMMA - 1) + 0.5 * rhoR * 0.09])
        F = oracle_mod.riemann("roe", UL, UR, n)
        np.testing.assert_allclose(F, [0.0, p * n[0], 0.0, p * n[2], 0.0], atol=1e-14)
        # LLF smears the same contact (so this pin distinguishes the two)
        assert np.abs(oracle_mod.riemann("llf", UL, UR, n) - F).max() > 1e-3


def test_roe_upwinds_supersonic_flow(oracle_mod):
    """Roe's linearisation reproduces F_R - F_L exactly, so with all wave speeds of one sign the
    flux is the upwind physical flux."""
    rng = np.random.default_rng(6)
    n = np.array([1.0, 0.0, 0.0])
    for sgn in (1.0, -1.0):
        for _ in range(20):
            rho = rng.uniform(0.8, 1.2, 2)
            p = rng.uniform(0.8, 1.2, 2)
            U = []
            for r, pp in zip(rho, p):
                u = np.array([sgn * rng.uniform(3.0, 4.0), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5)])
                U.append(np.array([r, r * u[0], r * u[1], r * u[2], pp / (GAMMA - 1) + 0.5 * r * u @ u]))
            F = oracle_mod.riemann("roe", U[0], U[1], n)
            up = U[0] if sgn > 0 else U[1]
            np.testing.assert_allclose(F, oracle_mod.flux_contra(up, n), rtol=1e-12, atol=1e-12)


def test_viscous_flux_closed_forms(oracle_mod):
    mu, kappa = 0.3, 0.7
    U = np.array([1.2, 1.2 * 0.5, 1.2 * -0.2, 1.2 * 0.1, 3.0])
    u = U[1:4] / U[0]
    zeroT = np.zeros(3)
    # isotropic dilatation: the Stokes hypothesis gives a trace-free stress, so no stress at all
    Fv = oracle_mod.viscous_flux(U, np.eye(3).ravel() * 2.5, zeroT, mu, kappa)
    assert np.abs(Fv).max() < 1e-15
    # rigid rotation: antisymmetric velocity gradient, no stress
    Om = np.array([[0, -1.0, 2.0], [1.0, 0, -3.0], [-2.0, 3.0, 0]])
    assert np.abs(oracle_mod.viscous_flux(U, Om.ravel(), zeroT, mu, kappa)).max() < 1e-15
    # simple shear du/dy = g
    g = 1.7
    G = np.zeros((3, 3))
    G[0, 1] = g
    Fv = oracle_mod.viscous_flux(U, G.ravel(), zeroT, mu, kappa)
    expect = np.zeros((3, 5))
    expect[1, 1] = mu * g          # tau_xy in the y-flux of x-momentum
    expect[0, 2] = mu * g          # tau_yx in the x-flux of y-momentum
    expect[0, 4] = u[1] * mu * g   # work of the stress
    expect[1, 4] = u[0] * mu * g
    np.testing.assert_allclose(Fv, expect, atol=1e-15)
    # pure temperature gradient: Fourier heat flux only
    gT = np.array([0.1, -0.4, 2.0])
    Fv = oracle_mod.viscous_flux(U, np.zeros(9), gT, mu, kappa)
    np.testing.assert_allclose(Fv[:, 4], kappa * gT, atol=1e-15)
    assert np.abs(Fv[:, :4]).max() == 0.0
    # uniaxial strain du/dx = a: tau_xx = 4/3 mu a, tau_yy = tau_zz = -2/3 mu a
    a = 0.9
    G = np.zeros((3, 3))
    G[0, 0] = a
    Fv = oracle_mod.viscous_flux(U, G.ravel(), zeroT, mu, kappa)
    np.testing.assert_allclose([Fv[0, 1], Fv[1, 2], Fv[2, 3]], [4 / 3 * mu * a, -2 / 3 * mu * a, -2 / 3 * mu * a],
                               rtol=1e-15)
