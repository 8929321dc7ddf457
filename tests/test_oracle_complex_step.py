"""Pins of the oracle's complex-step build, the reference for the discrete adjoint.

Oracle(..., complex_step=True) runs the same C source in complex arithmetic, so Im L(U + ihV)/h is
the directional derivative of the oracle's own right-hand side L. What pins it to something other
than itself:
  - its real part is the real build's result;
  - it agrees with central finite differences of the real build (to the FD truncation error);
  - two exact scaling laws of the discrete operator. With constant mu, every flux used here (KG,
    Pirozzoli, EC, central; LLF, Roe, EC; the BR1 viscous flux) satisfies
      L_adv(a U) = a L_adv(U), L_visc(a U) = L_visc(U)                      (density scaling)
      L(S_b U) = b S_b L_adv(U) + S_b L_visc(U),  S_b = diag(1, b, b, b, b^2)   (velocity scaling)
    so that, differentiating at a = b = 1, (dL/dU) U = L_adv(U) and
    (dL/dU) (S' U) = L_adv(U) + S' L(U) with S' = diag(0, 1, 1, 1, 2). The second law involves the
    viscous part, so a dropped derivative anywhere in the advective or viscous path breaks one of them;
  - discrete conservation: sum_i J_i w_i (dL/dU V)_i = 0 on periodic meshes, for every V;
  - for the LSERK step of the Euler equations, the step map inherits degree-1 homogeneity.
"""
import numpy as np
import pytest

from paper_2306_12891_gb300 import workloads as W

COMBOS = [
    dict(equations="euler", vflux="kg", sflux="llf"),
    dict(equations="euler", vflux="pirozzoli", sflux="roe"),
    dict(equations="euler", vflux="ec", sflux="ec"),
    dict(equations="euler", vflux="central", sflux="llf"),
    dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=0.02),
    dict(equations="ns", vflux="kg", sflux="llf", mu=0.05),
]
S_PRIME = np.array([0.0, 1.0, 1.0, 1.0, 2.0])[None, :, None, None, None]


def _case(N=3, nel=(2, 2, 3), seed=1, rotated=False):
    gen = lambda x, y, z: (x + 0.1 * np.sin(y) * np.cos(z), y + 0.1 * np.sin(z) * np.sin(x) + 0.05 * np.sin(2 * x),
                           z + 0.1 * np.sin(x) * np.cos(y))
    if rotated:
        xyz, faces, _ = W.rotated_box_mesh(N, nel, seed=seed, mapping=gen)
    else:
        xyz, faces = W.box_mesh(N, nel, mapping=gen)
    U = W.random_smooth_state(xyz, seed=seed, amp=0.1)
    U = U * (1.0 + 0.05 * np.random.default_rng(seed + 1).uniform(-1, 1, U.shape))
    scale = np.abs(U).reshape(U.shape[0], 5, -1).max(axis=(0, 2))[None, :, None, None, None]
    V = np.random.default_rng(seed + 2).standard_normal(U.shape) * scale
    return xyz, faces, U, V


def _pair(orc, N, xyz, faces, **kw):
    return orc.Oracle(N, xyz, faces, **kw), orc.Oracle(N, xyz, faces, complex_step=True, **kw)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("kw", COMBOS)
def test_real_part_is_the_real_build(oracle_mod, kw):
    xyz, faces, U, V = _case()
    o, oc = _pair(oracle_mod, 3, xyz, faces, **kw)
    r = o.rhs(U)
    z = oc.rhs(U.astype(np.complex128))
    assert np.abs(z.imag).max() == 0.0
    assert _rel(z.real, r) <= 4e-15


@pytest.mark.parametrize("kw", COMBOS)
def test_jvp_matches_central_differences(oracle_mod, kw):
    xyz, faces, U, V = _case(rotated=True)
    o, oc = _pair(oracle_mod, 3, xyz, faces, **kw)
    jv = oc.jvp(U, V)
    errs = []
    for eps in (1e-4, 1e-5):
        fd = (o.rhs(U + eps * V) - o.rhs(U - eps * V)) / (2 * eps)
        errs.append(_rel(fd, jv))
    # second-order truncation error: shrinks ~100x with eps (until round-off), and is small
    assert errs[1] < 1e-6, errs
    assert errs[1] < 0.05 * errs[0] or errs[1] < 1e-9, errs


def test_jvp_fv_blend_away_from_minmod_kinks(oracle_mod):
    """The FV subcell operator is piecewise smooth (minmod, first-order fallback): complex step gives
    the one-sided derivative, which central differences reproduce except at the few nodes whose
    slope choice flips within +-eps."""
    kw = dict(equations="euler", vflux="pirozzoli", sflux="llf", shock_capturing=True, alpha_fixed=0.4)
    xyz, faces, U, V = _case(rotated=True)
    o, oc = _pair(oracle_mod, 3, xyz, faces, **kw)
    jv = oc.jvp(U, V)
    eps = 1e-6
    fd = (o.rhs(U + eps * V) - o.rhs(U - eps * V)) / (2 * eps)
    bad = np.abs(fd - jv) > 1e-6 * np.abs(jv).max()
    assert bad.mean() < 0.01, bad.mean()


@pytest.mark.parametrize("kw", COMBOS)
def test_density_scaling_law(oracle_mod, kw):
    """(dL/dU) U = L_adv(U): the advective operator is homogeneous of degree 1, the viscous of degree 0."""
    xyz, faces, U, V = _case(N=2, nel=(3, 2, 2), seed=4)
    o, oc = _pair(oracle_mod, 2, xyz, faces, **kw)
    adv = oracle_mod.Oracle(2, xyz, faces, **{**kw, "equations": "euler", "mu": 0.0}).rhs(U)
    assert _rel(oc.jvp(U, U), adv) <= 5e-14


@pytest.mark.parametrize("kw", COMBOS)
def test_velocity_scaling_law(oracle_mod, kw):
    """(dL/dU)(S'U) = L_adv(U) + S' L(U): exercises the viscous derivative (energy flux u.tau, heat flux)."""
    xyz, faces, U, V = _case(N=3, nel=(2, 3, 2), seed=6)
    o, oc = _pair(oracle_mod, 3, xyz, faces, **kw)
    L = o.rhs(U)
    adv = oracle_mod.Oracle(3, xyz, faces, **{**kw, "equations": "euler", "mu": 0.0}).rhs(U)
    want = adv + S_PRIME * L
    assert _rel(oc.jvp(U, S_PRIME * U), want) <= 5e-14
    if kw["equations"] == "ns":  # the law fails if the viscous part is treated as degree 1 like the rest
        assert _rel(adv + S_PRIME * adv + (L - adv), want) > 1e-6


def test_velocity_scaling_detects_a_planted_mistake(oracle_mod):
    """Dropping the viscous derivative (a JVP of the advective part only) violates the law."""
    kw = COMBOS[4]
    xyz, faces, U, V = _case(N=3, nel=(2, 2, 2), seed=8)
    o = oracle_mod.Oracle(3, xyz, faces, **kw)
    oce = oracle_mod.Oracle(3, xyz, faces, complex_step=True, **{**kw, "equations": "euler", "mu": 0.0})
    L = o.rhs(U)
    adv = oracle_mod.Oracle(3, xyz, faces, **{**kw, "equations": "euler", "mu": 0.0}).rhs(U)
    assert _rel(oce.jvp(U, S_PRIME * U), adv + S_PRIME * L) > 1e-4


@pytest.mark.parametrize("kw", [COMBOS[1], COMBOS[4]])
def test_jvp_conserves(oracle_mod, kw):
    xyz, faces, U, V = _case(seed=9)
    o, oc = _pair(oracle_mod, 3, xyz, faces, **kw)
    jv = oc.jvp(U, V)
    w = oracle_mod.lgl(3)[1]
    wq = np.einsum("k,j,i->kji", w, w, w)[None] * o.J
    tot = np.einsum("ekji,evkji->v", wq, jv)
    mag = np.einsum("ekji,evkji->v", wq, np.abs(jv))
    assert (np.abs(tot) <= 1e-13 * mag).all(), tot / mag


def test_lserk_tangent(oracle_mod):
    kw = COMBOS[4]
    xyz, faces, U, V = _case(N=2, nel=(2, 2, 2), seed=10)
    o, oc = _pair(oracle_mod, 2, xyz, faces, **kw)
    dt = o.max_dt(U, 0.5)
    UK, tan = oc.lserk_jvp(U, V, dt, steps=2)
    ref = o.lserk_step(o.lserk_step(U, dt), dt)
    assert _rel(UK, ref) <= 1e-15
    eps = 1e-6
    fp = o.lserk_step(o.lserk_step(U + eps * V, dt), dt)
    fm = o.lserk_step(o.lserk_step(U - eps * V, dt), dt)
    assert _rel((fp - fm) / (2 * eps), tan) < 1e-6
    # Euler: the step map is homogeneous of degree 1, so its tangent along U is the step itself
    oe = oracle_mod.Oracle(2, xyz, faces, complex_step=True, equations="euler", vflux="pirozzoli", sflux="roe")
    UK, tan = oe.lserk_jvp(U, U, dt, steps=1)
    assert _rel(tan, UK) <= 5e-14


def test_dense_jacobian_columns(oracle_mod):
    kw = COMBOS[4]
    xyz, faces, U, V = _case(N=1, nel=(2, 2, 2), seed=12)
    o, oc = _pair(oracle_mod, 1, xyz, faces, **kw)
    Jm = oc.jacobian(U)
    assert Jm.shape == (U.size, U.size)
    assert _rel((Jm @ V.reshape(-1)).reshape(U.shape), oc.jvp(U, V)) <= 1e-13
