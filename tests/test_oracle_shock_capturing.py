"""Pins of the oracle's shock-capturing pieces: the modified Persson indicator (Sec. 4.1, Eq. (7))
on states of known modal content, the clipping to [0.01, 0.7] (Sec. 4.2), the factor-1/2
extension to neighbours (Sec. 4.1), and the FV subcell operator (freestream, conservation,
no new extrema at a discontinuity, consistency) and the DG/FV blend (Sec. 4.1, Eq. (6))."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as L

from paper_2306_12891_gb300 import workloads as W

S = math.log((1 - 1e-4) / 1e-4)


def threshold(N):
    return 0.5 * 10.0 ** (-1.8 * (N + 1) ** 0.25)


def single_element_state(N, rho_of_xi):
    xyz, faces = W.box_mesh(N, (1, 1, 1), lo=(-1, -1, -1), hi=(1, 1, 1))
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    rho = rho_of_xi(x, y, z)
    zero = np.zeros_like(x)
    U = W.cons_from_prim(rho, zero, zero, zero, np.ones_like(x))  # p = 1, so q = rho p = rho
    return xyz, faces, U


def phi(N, x):
    c = np.zeros(N + 1)
    c[N] = 1.0
    return math.sqrt((2 * N + 1) / 2) * L.legval(x, c)


@pytest.mark.parametrize("N", [3, 5, 7])
def test_indicator_on_known_modal_content(oracle_mod, N):
    """q = 1 + beta * phi_N(xi) phi_0 phi_0 has modes m_000 = 2 sqrt 2, m_N00 = beta, so
    E = beta^2 / (8 + beta^2); pick beta for E = T/4, T, 2T."""
    T = threshold(N)
    for ratio, expect in [(0.25, 0.0), (1.0, 0.5), (2.0, 0.7)]:
        E = ratio * T
        beta = math.sqrt(8 * E / (1 - E))
        xyz, faces, U = single_element_state(N, lambda x, y, z: 1.0 + beta * phi(N, x) / 2.0)
        o = oracle_mod.Oracle(N, xyz, faces, shock_capturing=True)
        raw, a = o.indicator(U)
        alpha = 1.0 / (1.0 + math.exp(-S / T * (E - T)))
        if ratio == 0.25:
            assert alpha < 0.01
        assert raw[0] == pytest.approx(expect, abs=1e-9), (ratio, raw, alpha)
        assert a[0] == pytest.approx(expect, abs=1e-9)


def test_indicator_zero_for_low_degree_content(oracle_mod):
    N = 5
    xyz, faces, U = single_element_state(N, lambda x, y, z: 1.0 + 0.3 * x + 0.2 * y * y - 0.1 * x * z ** 3)
    o = oracle_mod.Oracle(N, xyz, faces, shock_capturing=True)
    raw, a = o.indicator(U)
    assert raw[0] == 0.0 and a[0] == 0.0


def test_alpha_extends_to_neighbours_by_half(oracle_mod):
    N = 4
    xyz, faces = W.box_mesh(N, (4, 1, 1), lo=(0, 0, 0), hi=(4, 1, 1))
    x = xyz[:, 0]
    zero = np.zeros_like(x)
    rho = np.ones_like(x)
    rho[1] += 0.5 * np.sign(np.sin(7 * x[1]))  # rough data in element 1 only
    U = W.cons_from_prim(rho, zero, zero, zero, np.ones_like(x))
    o = oracle_mod.Oracle(N, xyz, faces, shock_capturing=True)
    raw, a = o.indicator(U)
    assert raw[1] == pytest.approx(0.7) and raw[0] == raw[2] == raw[3] == 0.0
    np.testing.assert_allclose(a, [0.35, 0.7, 0.35, 0.0])
    _, alpha_used = o.rhs(U, return_alpha=True)
    np.testing.assert_allclose(alpha_used, a)


FV_ONLY = dict(shock_capturing=True, alpha_fixed=1.0)  # pure FV subcell operator on every element


def _generic_map(x, y, z):
    return (x + 0.1 * np.sin(y) * np.cos(z), y + 0.1 * np.sin(z) * np.sin(x) + 0.05 * np.sin(2 * x),
            z + 0.1 * np.sin(x) * np.cos(y))


@pytest.mark.parametrize("sf", ["llf", "roe"])
def test_fv_freestream_and_conservation(oracle_mod, sf):
    N = 4
    xyz, faces = W.box_mesh(N, (3, 2, 2), mapping=_generic_map)
    o = oracle_mod.Oracle(N, xyz, faces, vflux="pirozzoli", sflux=sf, **FV_ONLY)
    U = W.freestream(xyz)
    Ut, alpha = o.rhs(U, return_alpha=True)
    assert (alpha == 1.0).all()
    assert np.abs(Ut).max() < 1e-12
    try:  # interface metrics averaged from the nodes instead of telescoped from Ja_0: no freestream
        _plant(oracle_mod, 5)
        assert np.abs(o.rhs(U)).max() > 1e-6
    finally:
        _plant(oracle_mod, 0)
    U = W.random_smooth_state(xyz, seed=5, amp=0.1)
    U = U * (1.0 + 0.01 * np.random.default_rng(6).uniform(-1, 1, U.shape))
    Ut = o.rhs(U)
    inv = o.invariants(U, Ut)
    w = oracle_mod.lgl(N)[1]
    wq = np.einsum("k,j,i->kji", w, w, w)[None] * o.J
    mag = np.einsum("ekji,evkji->v", wq, np.abs(Ut))
    assert (np.abs(inv[:5]) <= 1e-13 * mag).all()


def test_fv_creates_no_new_extrema_at_a_contact(oracle_mod):
    """A density jump moving with u = (1, 0, 0), p = 1, advanced by forward-Euler steps (the
    monotone setting of a minmod/LLF scheme; LSERK(5,4) itself is not strong-stability
    preserving): the FV subcell scheme keeps rho inside its initial range; pure DG does not
    (so the pin can fail)."""
    N = 5
    xyz, faces = W.box_mesh(N, (4, 1, 1), lo=(0, 0, 0), hi=(1, 0.25, 0.25))
    x = xyz[:, 0]
    rho = np.where((x > 0.3) & (x < 0.62), 2.0, 1.0)
    zero = np.zeros_like(x)
    U = W.cons_from_prim(rho, np.ones_like(x), zero, zero, np.ones_like(x))
    res = {}
    for name, kw in [("fv", FV_ONLY), ("dg", {})]:
        o = oracle_mod.Oracle(N, xyz, faces, vflux="pirozzoli", sflux="llf", **kw)
        dt = o.max_dt(U, 0.2)
        V = U.copy()
        for _ in range(10):
            V = V + dt * o.rhs(V)
        res[name] = (V[:, 0].min(), V[:, 0].max())
    assert res["fv"][0] >= 1.0 - 1e-12 and res["fv"][1] <= 2.0 + 1e-12, res
    assert res["dg"][0] < 1.0 - 1e-3 or res["dg"][1] > 2.0 + 1e-3, res


@pytest.mark.parametrize("eq", ["euler", "ns"])
def test_fv_and_dg_agree_elementwise_in_the_mean(oracle_mod, eq):
    """Both operators are conservative and share the element-boundary fluxes, so on every
    element sum_i J_i w_i Ut_i is the same for DG and FV (and hence for any blend): this is
    what lets the blend act element by element without a surface-integral correction."""
    N = 4
    xyz, faces = W.box_mesh(N, (3, 2, 2), mapping=_generic_map)
    U = W.random_smooth_state(xyz, seed=21, amp=0.1)
    U = U * (1.0 + 0.02 * np.random.default_rng(22).uniform(-1, 1, U.shape))
    kw = dict(equations=eq, vflux="pirozzoli", sflux="llf", mu=0.02)
    fv = oracle_mod.Oracle(N, xyz, faces, **kw, **FV_ONLY)
    dg = oracle_mod.Oracle(N, xyz, faces, **kw)
    w = oracle_mod.lgl(N)[1]
    wq = np.einsum("k,j,i->kji", w, w, w)[None] * fv.J
    Ufv, Udg = fv.rhs(U), dg.rhs(U)
    mfv = np.einsum("ekji,evkji->ev", wq, Ufv)
    mdg = np.einsum("ekji,evkji->ev", wq, Udg)
    scale = np.einsum("ekji,evkji->v", wq, np.abs(Udg))
    assert np.abs(mfv - mdg).max() < 1e-13 * scale.max()
    assert np.abs(Ufv - Udg).max() > 1e-3  # pointwise they differ


def test_blend_acts_on_the_advective_part_only(oracle_mod):
    N = 3
    xyz, faces = W.box_mesh(N, (3, 2, 2), mapping=_generic_map)
    U = W.random_smooth_state(xyz, seed=9, amp=0.1)
    kw = dict(vflux="pirozzoli", sflux="roe", mu=0.05)
    ns_sc = oracle_mod.Oracle(N, xyz, faces, equations="ns", **kw, **FV_ONLY).rhs(U)
    eu_sc = oracle_mod.Oracle(N, xyz, faces, equations="euler", **kw, **FV_ONLY).rhs(U)
    ns = oracle_mod.Oracle(N, xyz, faces, equations="ns", **kw).rhs(U)
    eu = oracle_mod.Oracle(N, xyz, faces, equations="euler", **kw).rhs(U)
    np.testing.assert_allclose(ns_sc - eu_sc, ns - eu, rtol=0, atol=1e-12 * np.abs(ns).max())
    assert np.abs(eu_sc - eu).max() > 1e-4  # FV differs from DG on these data


# ------------------------------------------------------------------ the subcell reconstruction itself
#
# Sec. 4.1: the FV subcells are second order inside the element and first order in the two outer
# subcells; Hennemann et al.: minmod slopes of the primitive variables, states evaluated at the
# subcell interfaces (the cumulative LGL weights). The pins use a contact -- u = (U, 0, 0), p
# constant, rho piecewise linear in x -- on a Cartesian element, where a second-order reconstruction
# is exact: where both interfaces of a subcell see one line from both sides, the Riemann flux is the
# exact flux of that line and the subcell's rho_t is exactly -U b (b = the line's slope), so which
# subcells are exact tells what was reconstructed where.

U_ADV = 0.6


def _plant(oracle_mod, k):
    import ctypes

    ctypes.c_int.in_dll(oracle_mod.lib(), "orc_fv_plant").value = k


def _contact(N, rho_of_x):
    """Two Cartesian elements on [0,2]x[0,1]x[0,1]; returns (xyz, faces, U, x nodes of element 0)."""
    xyz, faces = W.box_mesh(N, (2, 1, 1), lo=(0, 0, 0), hi=(2, 1, 1))
    x = xyz[:, 0]
    zero = np.zeros_like(x)
    U = W.cons_from_prim(rho_of_x(x), U_ADV + zero, zero, zero, 1.0 + zero)
    return xyz, faces, U, xyz[0, 0, 0, 0, :]


def _subcell_rates(oracle_mod, N, xyz, faces, U):
    """rho_t of element 0 per subcell along x (after checking it is the same on every y-z line)."""
    o = oracle_mod.Oracle(N, xyz, faces, vflux="pirozzoli", sflux="llf", **FV_ONLY)
    r = o.rhs(U)[0, 0]  # [k][j][i]
    assert np.abs(r - r[:1, :1, :]).max() <= 1e-13 * np.abs(r).max()
    return r[0, 0, :]


def _exact_set(rates, slopes):
    """Subcells whose rho_t equals -U b for the slope b of the line they sit on."""
    return {i for i in range(len(rates)) if abs(rates[i] + U_ADV * slopes[i]) <= 1e-10 * abs(U_ADV * slopes[i])}


@pytest.mark.parametrize("N", [5, 7])
def test_fv_reconstruction_exact_for_linear_data_in_interior_subcells(oracle_mod, N):
    b = 0.2
    xyz, faces, U, _ = _contact(N, lambda x: 1.5 + b * x)
    rates = _subcell_rates(oracle_mod, N, xyz, faces, U)
    exact = _exact_set(rates, [b] * (N + 1))
    assert exact == set(range(2, N - 1)), exact  # second order inside
    for i in (1, N - 1):  # next to a first-order outer subcell: the interface jump adds dissipation
        assert abs(rates[i] + U_ADV * b) > 1e-3 * U_ADV * b
    try:
        for plant in (1, 2, 3):  # no slopes; slopes in the outer subcells; states off the interfaces
            _plant(oracle_mod, plant)
            got = _exact_set(_subcell_rates(oracle_mod, N, xyz, faces, U), [b] * (N + 1))
            assert got != set(range(2, N - 1)), (plant, got)
    finally:
        _plant(oracle_mod, 0)


@pytest.mark.parametrize("b1,b2", [(0.1, 0.3), (0.3, 0.1), (0.2, -0.3)])
def test_fv_minmod_takes_the_smaller_slope_at_a_kink(oracle_mod, b1, b2):
    """rho has a kink at node k = 3 of element 0 (N = 7): slopes b1 left of it, b2 right of it.
    Minmod gives node k the smaller slope of the same sign, or none at an extremum. The exact
    subcells are then those whose two interfaces each see one line from both sides (subcells 1 and
    6 border the first-order outer subcells and are never exact):
      |b1| < |b2|: node k carries the left line, interface k+1/2 jumps -> {2, 5} exact;
      |b1| > |b2|: node k carries the right line, interface k-1/2 jumps -> {4, 5} exact;
      opposite signs: node k is flat, both interfaces jump -> {5} exact;
    and the larger slope (maxmod) gives {4, 5} instead of {2, 5} when |b1| < |b2|."""
    N, k = 7, 3
    xk = None

    def rho(x):
        return 1.5 + np.where(x < xk, b1 * (x - xk), b2 * (x - xk))

    _, _, _, xs = _contact(N, lambda x: x)
    xk = xs[k]
    xyz, faces, U, _ = _contact(N, rho)
    slopes = [b1 if i < k else b2 for i in range(N + 1)]
    rates = _subcell_rates(oracle_mod, N, xyz, faces, U)
    exact = _exact_set(rates, slopes)
    want = {2, 5} if abs(b1) < abs(b2) and b1 * b2 > 0 else ({4, 5} if b1 * b2 > 0 else {5})
    assert exact == want, exact
    assert abs(rates[k] + U_ADV * slopes[k]) > 1e-3 * abs(U_ADV * slopes[k])
    if abs(b1) < abs(b2) and b1 * b2 > 0:
        try:
            _plant(oracle_mod, 4)
            got = _exact_set(_subcell_rates(oracle_mod, N, xyz, faces, U), slopes)
            assert got == {4, 5}, got
        finally:
            _plant(oracle_mod, 0)
