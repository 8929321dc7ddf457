"""Pins of the oracle's wall model (Sec. 3) and of its wall boundary condition.

Spalding's law (Sec. 3, Eq. (2)) is pinned by its expansions, not by retyping it: near the wall
y+ - u+ = 0.1108 (0.4 u+)^5 / 5! + O(u+^6) (the subtracted polynomial is the Taylor series of the
exponential to fourth order), and far from it u+ -> ln(y+)/0.4 + B with B = -ln(0.1108)/0.4 = 5.50
(the classical log law). The Newton inversion is pinned by round trips and by the viscous-sublayer
closed form u_tau = sqrt(nu U / h). The van Driest transform (Eq. (5)) is pinned by its Ma -> 0
limit, its arcsin series, and by the relation b^2 = 1 - T_e / T_aw with the recovery temperature
T_aw / T_e = 1 + Pr^(1/3) (gamma-1)/2 Ma^2 (the reading used for the garbled temperature ratio).
The wall boundary condition is pinned by discrete conservation of mass and energy (no
penetration, adiabatic wall at rest), by a fluid at rest staying at rest, and by uniform flow
along the walls, whose only force is the wall shear: d/dt of the total x-momentum equals
-tau_w times the wall area, with tau_w from an independent root finder (scipy brentq).
"""
import numpy as np
import pytest

from helpers import flux_scale
from paper_2306_12891_gb300 import workloads as W

KAPPA, C = 0.4, 0.1108


def test_spalding_near_wall_expansion(oracle_mod):
    # leading term of y+ - u+ is C (kappa u+)^5 / 120: a dropped or wrong polynomial term changes it
    for up in (1e-2, 2e-2, 4e-2):
        lead = C * (KAPPA * up) ** 5 / 120.0
        got = oracle_mod.spalding_yplus(up) - up
        assert abs(got / lead - 1.0) < 0.05 * (up / 1e-2), (up, got, lead)


def test_spalding_log_law_limit(oracle_mod):
    B = -np.log(C) / KAPPA
    assert abs(B - 5.5) < 0.01  # the law's constants are the classical log-law kappa = 0.4, B = 5.5
    for up in (30.0, 40.0, 50.0):
        yp = oracle_mod.spalding_yplus(up)
        loglaw = np.log(yp) / KAPPA + B
        assert abs(up - loglaw) < 0.05 if up == 30.0 else abs(up - loglaw) < 2e-3, (up, loglaw)


@pytest.mark.parametrize("up", [1e-3, 0.3, 2.0, 8.0, 11.0, 17.0, 25.0, 40.0, 62.0, 70.0])
def test_newton_round_trip(oracle_mod, up):
    Re = up * oracle_mod.spalding_yplus(up)
    got, iters = oracle_mod.wall_uplus(Re)
    assert abs(got - up) <= 2e-15 * up, (got, up)
    assert 1 <= iters <= 100


def test_viscous_sublayer_closed_form(oracle_mod):
    # y+ < ~1: u+ = y+, so U / u_tau = h u_tau / nu, u_tau = sqrt(nu U / h)
    U, h, nu = 1e-3, 1e-3, 1e-3
    utau = oracle_mod.wall_utau(U, h, nu)
    assert abs(utau / np.sqrt(nu * U / h) - 1.0) < 1e-6


def test_newton_against_independent_root_finder(oracle_mod):
    from scipy.optimize import brentq

    rng = np.random.default_rng(5)
    for _ in range(20):
        U, h, nu = rng.uniform(0.1, 2.0), 10 ** rng.uniform(-4, -1), 10 ** rng.uniform(-7, -4)
        Re = h * U / nu
        f = lambda up: up * (up + C * (np.exp(KAPPA * up) - 1 - KAPPA * up - (KAPPA * up) ** 2 / 2
                                       - (KAPPA * up) ** 3 / 6 - (KAPPA * up) ** 4 / 24)) - Re
        up = brentq(f, 1e-12, 200.0, xtol=1e-15, rtol=1e-15)
        assert abs(oracle_mod.wall_utau(U, h, nu) - U / up) <= 1e-13 * U / up


def test_van_driest(oracle_mod):
    gamma, Pr, uinf = 1.4, 0.72, 1.3
    assert oracle_mod.van_driest(0.7, uinf, 0.0, gamma, Pr) == 0.7  # Ma -> 0: no transform
    for Ma in (0.3, 0.8, 2.0):
        Taw_Te = 1.0 + Pr ** (1.0 / 3.0) * 0.5 * (gamma - 1.0) * Ma ** 2
        b = np.sqrt(1.0 - 1.0 / Taw_Te)  # b^2 = 1 - T_e / T_aw
        for u in (0.1, 0.6, 1.3):
            x = b * u / uinf
            series = uinf / b * (x + x ** 3 / 6 + 3 * x ** 5 / 40 + 15 * x ** 7 / 336 + 105 * x ** 9 / 3456)
            got = oracle_mod.van_driest(u, uinf, Ma, gamma, Pr)
            tol = 10 * abs(uinf / b) * x ** 11 + 1e-15
            assert abs(got - series) <= tol, (Ma, u, got, series)
            assert got >= u  # the equivalent incompressible velocity exceeds the compressible one


def _channel(N=3, nel=(3, 2, 3), hz=2.0):
    return W.box_mesh(N, nel, lo=(0.0, 0.0, 0.0), hi=(2.0 * np.pi, np.pi, hz), z_walls=True)


def _state(xyz, seed=1):
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    rng = np.random.default_rng(seed)
    r = lambda: rng.uniform(-1, 1)
    rho = 1.0 + 0.05 * np.sin(x + r()) * np.cos(z)
    u = 0.8 + 0.1 * np.sin(y + r()) * np.sin(np.pi * z / 2)
    v = 0.05 * np.cos(x + r())
    w = 0.05 * np.sin(x) * np.sin(np.pi * z / 2) + 0.03 * np.cos(y + r())
    p = 1.0 / 1.4 + 0.02 * np.cos(x + y + r())
    return W.cons_from_prim(rho, u, v, w, p)


@pytest.mark.parametrize("kw", [dict(equations="euler", vflux="pirozzoli", sflux="roe"),
                                dict(equations="euler", vflux="kg", sflux="llf"),
                                dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=1e-3),
                                dict(equations="ns", vflux="kg", sflux="llf", mu=1e-2, wm_index=2,
                                     wm_van_driest=True, wm_mainf=0.8)])
def test_wall_channel_conserves_mass_and_energy(oracle_mod, kw):
    xyz, faces = _channel()
    U = _state(xyz)
    o = oracle_mod.Oracle(3, xyz, faces, **kw)
    Ut = o.rhs(U)
    w = oracle_mod.lgl(3)[1]
    wq = np.einsum("k,j,i->kji", w, w, w)[None] * o.J
    tot = np.einsum("ekji,evkji->v", wq, Ut)
    mag = np.einsum("ekji,evkji->v", wq, np.abs(Ut))
    assert abs(tot[0]) <= 1e-13 * mag[0] and abs(tot[4]) <= 1e-13 * mag[4], tot / mag
    # the walls do exert forces: x-momentum is not conserved with viscosity
    if kw["equations"] == "ns":
        assert abs(tot[1]) > 1e-6 * mag[1]


def test_fluid_at_rest_stays_at_rest(oracle_mod):
    xyz, faces = _channel()
    U = W.cons_from_prim(*(np.ones_like(xyz[:, 0]) * c for c in (1.2, 0.0, 0.0, 0.0, 0.9)))
    Ut = oracle_mod.Oracle(3, xyz, faces, equations="ns", vflux="pirozzoli", sflux="roe", mu=1e-3).rhs(U)
    assert np.abs(Ut).max() < 1e-13


@pytest.mark.parametrize("wm_index,vd", [(1, False), (2, False), (1, True)])
def test_uniform_flow_wall_shear(oracle_mod, wm_index, vd):
    """Uniform flow U along x between the walls z = 0 and z = Hz: no interior gradients, so the total
    x-momentum changes only by the wall shear, -2 tau_w Lx Ly, with tau_w = rho u_tau^2 and u_tau the
    root of Spalding's law at the exchange distance (brentq, independent of the oracle's Newton)."""
    from scipy.optimize import brentq

    N, nz, Hz, Ub, mu, rho, Ma = 3, 3, 2.0, 0.9, 2e-4, 1.1, 0.8
    xyz, faces = _channel(N, (2, 2, nz), Hz)
    one = np.ones_like(xyz[:, 0])
    U = W.cons_from_prim(rho * one, Ub * one, 0 * one, 0 * one, 0.8 * one)
    o = oracle_mod.Oracle(N, xyz, faces, equations="ns", vflux="pirozzoli", sflux="roe", mu=mu, wm_index=wm_index,
                          wm_van_driest=vd, wm_uinf=1.0, wm_mainf=Ma)
    Ut = o.rhs(U)
    w = oracle_mod.lgl(N)[1]
    xi = oracle_mod.lgl(N)[0]
    wq = np.einsum("k,j,i->kji", w, w, w)[None] * o.J
    dmom = np.einsum("ekji,ekji->", wq, Ut[:, 1])
    h = (xi[wm_index] - xi[0]) / 2.0 * (Hz / nz)
    ueq = Ub
    if vd:
        m = 0.5 * 0.4 * Ma ** 2 * 0.72 ** (1.0 / 3.0)
        b = np.sqrt(m) / np.sqrt(1 + m)
        ueq = 1.0 / b * np.arcsin(b * Ub / 1.0)
    Re = h * ueq * rho / mu
    f = lambda up: up * (up + C * (np.exp(KAPPA * up) - 1 - KAPPA * up - (KAPPA * up) ** 2 / 2
                                   - (KAPPA * up) ** 3 / 6 - (KAPPA * up) ** 4 / 24)) - Re
    utau = ueq / brentq(f, 1e-12, 200.0, xtol=1e-15, rtol=1e-15)
    want = -2.0 * rho * utau ** 2 * (2 * np.pi) * np.pi
    assert abs(dmom / want - 1.0) < 1e-12, (dmom, want)
    # everything else is at rest: mass, y/z-momentum and energy rates vanish node by node (to the
    # rounding of the flux terms they difference)
    scale = flux_scale(U, o.Ja, o.J, oracle_mod.dmatrix(N))
    for v in (0, 2, 3, 4):
        assert np.abs(Ut[:, v]).max() < 1e-12 * scale[v], (v, np.abs(Ut[:, v]).max(), scale[v])
