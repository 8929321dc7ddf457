"""Pins of the oracle's LSERK(5,4) time step (Carpenter-Kennedy 2N-storage): exact integration
of polynomials in t up to degree 3 (which fixes the stage times c), the stability polynomial
1 + z + z^2/2 + z^3/6 + z^4/24 + O(z^5) on y' = lambda y, and fourth-order convergence on a
nonlinear ODE; plus the DG step itself conserving the weighted integrals."""
import math

import numpy as np

from paper_2306_12891_gb300 import workloads as W


def test_polynomials_in_time_are_integrated_exactly(oracle_mod):
    for k in range(1, 5):  # y' = k t^(k-1), degree <= 3
        for t0, dt in [(0.0, 0.7), (1.3, 0.25)]:
            y = oracle_mod.lserk_generic(np.array([0.0]), dt, t0, lambda u, t, k=k: np.array([k * t ** (k - 1)]))
            assert abs(y[0] - ((t0 + dt) ** k - t0 ** k)) < 1e-14
    # degree 4 is not integrated exactly (so the pin can fail)
    y = oracle_mod.lserk_generic(np.array([0.0]), 0.7, 0.0, lambda u, t: np.array([5 * t ** 4]))
    assert abs(y[0] - 0.7 ** 5) > 1e-6


def test_stability_polynomial(oracle_mod):
    zs = np.linspace(-2.5, 0.5, 9)
    R = np.array([oracle_mod.lserk_generic(np.array([1.0]), 1.0, 0.0, lambda u, t, z=z: z * u)[0] for z in zs])
    coef = np.linalg.lstsq(np.vander(zs, 6, increasing=True), R, rcond=None)[0]
    np.testing.assert_allclose(coef[:5], [1, 1, 1 / 2, 1 / 6, 1 / 24], rtol=0, atol=1e-11)
    assert abs(coef[5] - 1 / 120) > 1e-4  # five stages, fourth order: the z^5 term is not 1/120
    resid = R - np.vander(zs, 6, increasing=True) @ coef
    assert np.abs(resid).max() < 1e-13     # exactly a quintic


def test_fourth_order_on_nonlinear_ode(oracle_mod):
    # y' = y^2 - t, solved from y(0) = 0.5 to T = 1 against a fine-step reference, and
    # y' = y^2 with exact solution 1/(1/y0 - t)
    def solve(f, y0, T, n):
        y = np.array([y0])
        for s in range(n):
            y = oracle_mod.lserk_generic(y, T / n, s * T / n, f)
        return y[0]
    f = lambda u, t: u * u
    exact = 1.0 / (1.0 / 0.5 - 1.0)
    errs = [abs(solve(f, 0.5, 1.0, n) - exact) for n in (10, 20, 40)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 3.8, (errs, rates)


def test_dg_step_conserves_integrals(oracle_mod):
    N = 3
    xyz, faces = W.box_mesh(N, (3, 3, 3), mapping="sine_0.05")
    o = oracle_mod.Oracle(N, xyz, faces, equations="ns", vflux="pirozzoli", sflux="roe", mu=0.01)
    U0 = W.taylor_green(xyz)
    dt = o.max_dt(U0, 0.5)
    U1 = o.lserk_step(U0, dt)
    w = oracle_mod.lgl(N)[1]
    wq = np.einsum("k,j,i->kji", w, w, w)[None] * o.J
    I0 = np.einsum("ekji,evkji->v", wq, U0)
    I1 = np.einsum("ekji,evkji->v", wq, U1)
    assert np.abs(I1 - I0).max() < 1e-13 * np.abs(I0).max()
    assert np.abs(U1 - U0).max() > 1e-6
