"""Pins of the oracle's full right-hand side against what the method and the mathematics fix:
freestream preservation on curved meshes, discrete conservation, entropy conservation of the
EC split form (and dissipation of LLF/Roe), convergence to the exact Euler and Navier-Stokes
operators (computed symbolically), the Taylor-Green kinetic energy, and the consistency of the
element-subset evaluation used for sampled full-size parity."""
import numpy as np
import pytest

from helpers import flux_scale
from paper_2306_12891_gb300 import workloads as W

COMBOS = [("kg", "llf", "euler"), ("pirozzoli", "roe", "euler"), ("ec", "ec", "euler"),
          ("central", "llf", "euler"), ("pirozzoli", "roe", "ns"), ("kg", "llf", "ns")]


def _generic_map(x, y, z):
    return (x + 0.1 * np.sin(y) * np.cos(z), y + 0.1 * np.sin(z) * np.sin(x) + 0.05 * np.sin(2 * x),
            z + 0.1 * np.sin(x) * np.cos(y))


def _quad_weights(o):
    import oracle

    w = oracle.lgl(o.N)[1]
    return np.einsum("k,j,i->kji", w, w, w)


@pytest.mark.parametrize("vf,sf,eq", COMBOS)
@pytest.mark.parametrize("mapping", ["sine_0.05", "generic"])
def test_freestream_preserved_on_curved_mesh(oracle_mod, vf, sf, eq, mapping):
    N = 4
    xyz, faces = W.box_mesh(N, (3, 2, 2), mapping=_generic_map if mapping == "generic" else mapping)
    o = oracle_mod.Oracle(N, xyz, faces, equations=eq, vflux=vf, sflux=sf, mu=0.05)
    U = W.freestream(xyz)
    Ut = o.rhs(U)
    scale = flux_scale(U, o.Ja, o.J, oracle_mod.dmatrix(N))
    err = np.abs(Ut).reshape(Ut.shape[0], 5, -1).max(axis=(0, 2))
    assert (err <= 1e-13 * scale.max()).all(), (err, scale)


@pytest.mark.parametrize("vf,sf,eq", COMBOS)
def test_discrete_conservation(oracle_mod, vf, sf, eq):
    N = 3
    xyz, faces = W.box_mesh(N, (3, 3, 2), mapping=_generic_map)
    o = oracle_mod.Oracle(N, xyz, faces, equations=eq, vflux=vf, sflux=sf, mu=0.05)
    U = W.random_smooth_state(xyz, seed=7, amp=0.1)
    Ut = o.rhs(U)
    inv = o.invariants(U, Ut)
    wq = _quad_weights(o)[None] * o.J
    mag = np.einsum("ekji,evkji->v", wq, np.abs(Ut))
    assert (np.abs(inv[:5]) <= 1e-13 * mag).all(), (inv[:5], mag)


def test_entropy_conservation_and_dissipation(oracle_mod):
    N = 4
    xyz, faces = W.box_mesh(N, (3, 2, 2), mapping=_generic_map)
    U = W.random_smooth_state(xyz, seed=11, amp=0.1)
    U = U * (1.0 + 0.01 * np.random.default_rng(12).uniform(-1, 1, U.shape))  # jumps at faces
    rates = {}
    for vf, sf in [("ec", "ec"), ("ec", "llf"), ("ec", "roe"), ("kg", "ec")]:
        o = oracle_mod.Oracle(N, xyz, faces, vflux=vf, sflux=sf)
        Ut = o.rhs(U)
        rates[(vf, sf)] = o.invariants(U, Ut)[5]
    assert abs(rates[("ec", "ec")]) < 1e-12
    assert rates[("ec", "llf")] < -1e-6 and rates[("ec", "roe")] < -1e-6
    assert abs(rates[("kg", "ec")]) > 1e-8  # KG is not entropy conservative: the pin can fail


def _ev(f, xyz):
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    return np.stack([np.broadcast_to(np.asarray(a, dtype=float), x.shape) for a in f(x, y, z)], 1)


@pytest.mark.parametrize("vf,sf", [("kg", "llf"), ("pirozzoli", "roe"), ("ec", "ec")])
def test_euler_rhs_converges_on_density_wave(oracle_mod, vf, sf):
    """rho = 1 + 0.2 sin(pi(x+y+z)), u = (1,1,1), p = 1: U_t = rho_t (1, 1, 1, 1, 3/2) with
    rho_t = -0.6 pi cos(pi(x+y+z)). The RHS error must fall at order about N."""
    N = 3
    errs = []
    for K in (2, 4, 8):
        xyz, faces = W.box_mesh(N, (K, K, K), lo=(-1, -1, -1), hi=(1, 1, 1))
        o = oracle_mod.Oracle(N, xyz, faces, vflux=vf, sflux=sf)
        U = W.density_wave(xyz)
        s = xyz.sum(1)
        rt = -0.6 * np.pi * np.cos(np.pi * s)
        exact = np.stack([rt, rt, rt, rt, 1.5 * rt], 1)
        errs.append(np.abs(o.rhs(U) - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > N - 0.6, (errs, rates)
    assert errs[-1] < 0.03  # about 1.5% of max|rho_t| at 8^3 elements, N = 3


def _ns_exact(mu, gamma=1.4, R=1.0, Pr=0.72):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    X = [x, y, z]
    rho = 1 + sp.Rational(1, 10) * sp.sin(x) * sp.cos(y) + sp.Rational(1, 20) * sp.cos(z)
    vel = [sp.Rational(1, 2) * sp.sin(y) * sp.cos(z) + sp.Rational(1, 5), sp.Rational(2, 5) * sp.cos(x) * sp.sin(z),
           sp.Rational(3, 10) * sp.sin(x + y)]
    p = 1 + sp.Rational(1, 10) * sp.cos(x) * sp.cos(y) * sp.sin(z)
    E = p / (gamma - 1) + rho * sum(v * v for v in vel) / 2
    U = [rho] + [rho * v for v in vel] + [E]
    T = p / (rho * R)
    div = sum(sp.diff(vel[c], X[c]) for c in range(3))
    kap = mu * gamma * R / ((gamma - 1) * Pr)
    adv, vis = [0] * 5, [0] * 5
    for c in range(3):
        Fa = [rho * vel[c]] + [rho * vel[r] * vel[c] + (p if r == c else 0) for r in range(3)] + [(E + p) * vel[c]]
        tau = [mu * (sp.diff(vel[r], X[c]) + sp.diff(vel[c], X[r]) - (sp.Rational(2, 3) * div if r == c else 0))
               for r in range(3)]
        Fv = [0] + tau + [sum(vel[r] * tau[r] for r in range(3)) + kap * sp.diff(T, X[c])]
        for v in range(5):
            adv[v] += -sp.diff(Fa[v], X[c])
            vis[v] += sp.diff(Fv[v], X[c])
    return sp.lambdify(X, U, "numpy"), sp.lambdify(X, adv, "numpy"), sp.lambdify(X, vis, "numpy")


def test_navier_stokes_rhs_converges_to_symbolic_operator(oracle_mod):
    """Curved periodic mesh, BR1 + Pirozzoli + Roe: the oracle's RHS tends to
    -div F_adv + div F_visc of a smooth manufactured state; the viscous part (RHS(mu) - RHS(0))
    tends to div F_visc on its own."""
    mu = 0.1
    fU, fadv, fvis = _ns_exact(mu)
    N = 4
    e_tot, e_vis = [], []
    for K in (2, 4, 8):
        xyz, faces = W.box_mesh(N, (K, K, K), mapping="sine_0.05")
        U = _ev(fU, xyz)
        adv, vis = _ev(fadv, xyz), _ev(fvis, xyz)
        o1 = oracle_mod.Oracle(N, xyz, faces, equations="ns", vflux="pirozzoli", sflux="roe", mu=mu)
        o0 = oracle_mod.Oracle(N, xyz, faces, equations="ns", vflux="pirozzoli", sflux="roe", mu=0.0)
        r1, r0 = o1.rhs(U), o0.rhs(U)
        e_tot.append(np.sqrt(((r1 - adv - vis) ** 2).mean()))
        e_vis.append(np.sqrt((((r1 - r0) - vis)[:, 1:] ** 2).mean()))
    # RMS error; BR1's second-derivative terms converge at about order N-1 (measured 2.5-2.9 at N=4)
    assert e_tot[-1] < 5e-4 and e_vis[-1] < 5e-4, (e_tot, e_vis)
    assert np.log2(e_tot[-2] / e_tot[-1]) > 2.2 and np.log2(e_vis[-2] / e_vis[-1]) > 2.2, (e_tot, e_vis)
    # a 10% error in the heat conductivity would not pass
    o_bad = oracle_mod.Oracle(N, xyz, faces, equations="ns", vflux="pirozzoli", sflux="roe", mu=mu, Pr=0.72 * 1.1)
    assert np.sqrt(((o_bad.rhs(U) - r0 - vis)[:, 4] ** 2).mean()) > 3 * e_vis[-1]


def test_taylor_green_initial_kinetic_energy(oracle_mod):
    for N, tol in ((3, 2e-3), (7, 1e-9)):
        xyz, faces = W.box_mesh(N, (4, 4, 4))
        o = oracle_mod.Oracle(N, xyz, faces)
        U = W.taylor_green(xyz)
        inv = o.invariants(U, np.zeros_like(U))
        vol = (2 * np.pi) ** 3
        assert abs(inv[6] / vol - 0.125) < tol


def test_element_subset_matches_full_rhs(oracle_mod):
    N = 3
    xyz, faces = W.box_mesh(N, (4, 3, 3), mapping=_generic_map)
    U = W.random_smooth_state(xyz, seed=3, amp=0.1)
    for eq, sc in [("ns", False), ("euler", True)]:
        o = oracle_mod.Oracle(N, xyz, faces, equations=eq, vflux="pirozzoli", sflux="roe", mu=0.05,
                              shock_capturing=sc, alpha_fixed=0.6)
        full = o.rhs(U)
        mask = [0, 5, 17, 35]
        part = o.rhs(U, mask=mask)
        np.testing.assert_array_equal(part[mask], full[mask])
        others = np.setdiff1d(np.arange(o.nE), mask)
        assert not part[others].any()


@pytest.mark.parametrize("eq,sc", [("euler", False), ("ns", False), ("euler", True)])
def test_rhs_invariant_under_element_rotation(oracle_mod, eq, sc):
    """Re-indexing elements by rotations of the reference cube (face table rebuilt from the
    coordinates, so faces of most of the eight orientations occur) changes nothing but the node
    labels: the right-hand side of a rotated element is the rotated right-hand side."""
    N = 3
    xyz, faces = W.box_mesh(N, (3, 2, 2), mapping=_generic_map)
    xr, fr, rots = W.rotated_box_mesh(N, (3, 2, 2), seed=3, mapping=_generic_map)
    assert len(set(fr[:, 4])) >= 5
    kw = dict(equations=eq, vflux="pirozzoli", sflux="roe", mu=0.05)
    if sc:
        kw.update(shock_capturing=True, alpha_fixed=0.4)
    field = lambda x: W.random_smooth_state(x, seed=5, amp=0.1)
    R1 = oracle_mod.Oracle(N, xyz, faces, **kw).rhs(field(xyz))
    R2 = oracle_mod.Oracle(N, xr, fr, **kw).rhs(field(xr))
    err = max(np.abs((W.relabel_element(N, R1[e], r) if r else R1[e]) - R2[e]).max() for e, r in enumerate(rots))
    assert err < 1e-12 * np.abs(R1).max()
    # a wrong orientation code is detected (the pin can fail)
    bad = fr.copy()
    i = int(np.nonzero(bad[:, 4] != 0)[0][0])
    bad[i, 4] = 0
    R3 = oracle_mod.Oracle(N, xr, bad, **kw).rhs(field(xr))
    assert np.abs(R3 - R2).max() > 1e-3 * np.abs(R1).max()


def test_paper_freestream_workload_is_a_steady_state(oracle_mod):
    """The paper's performance case (N = 7, periodic Cartesian box, Navier-Stokes, Pirozzoli + Roe +
    BR1, free stream), reduced to 2^3 elements: a uniform flow is an exact steady state of the
    discretisation, so the right-hand side vanishes to rounding (relative to the flux scale)."""
    w = W.WORKLOADS["freestream_ns_n7_32x32x32"].with_(nel=(2, 2, 2))
    xyz, faces = w.mesh()
    U = w.initial_state(xyz)
    assert np.ptp(U[:, 0]) == 0.0 and np.ptp(U[:, 4]) == 0.0  # uniform density and energy
    o = oracle_mod.Oracle(w.N, xyz, faces, **w.physics())
    Ut = o.rhs(U)
    scale = flux_scale(U, o.Ja, o.J, oracle_mod.dmatrix(w.N))
    err = np.abs(Ut).reshape(Ut.shape[0], 5, -1).max(axis=(0, 2))
    assert (err <= 1e-13 * scale.max()).all(), (err, scale)


# ------------------------------------------------------------------ split forms as product-rule derivatives
#
# Flux differencing with a two-point flux that is a product of arithmetic means equals a product-rule
# split of the derivative (Fisher & Carpenter 2013; Gassner, Winters & Kopriva 2016, for SBP
# operators with D 1 = 0):
#   sum_m 2 D_im {a}{b}     = (a D b + b D a + D(ab))_i / 2
#   sum_m 2 D_im {a}{b}{c}  = (ab Dc + ac Db + bc Da + a D(bc) + b D(ac) + c D(ab) + D(abc))_i / 4
#   sum_m 2 D_im {p}        = (D p)_i
# So on a Cartesian mesh, for a continuous state (no surface terms), the Euler right-hand side of each
# volume flux is a known combination of plain D-derivatives of products: Pirozzoli's energy flux
# {rho}{u}{h} is the cubic split of rho u h, Kennedy-Gruber's {rho}{u}{e} + {p}{u} the cubic split of
# rho u e plus the quadratic split of p u, the central flux the plain derivative of F. An energy
# average formed another way ({rho h} for {rho}{h}, say) changes the result, and KG's and
# Pirozzoli's expectations tell the two apart, so each pins the other's energy flux too.

def _split_rhs(kind, U, D, h, gamma=1.4):
    """-sum_d (2/h_d) split_d for a Cartesian element of sides h; U [nE][5][k][j][i]."""
    rho = U[:, 0]
    u = [U[:, 1 + c] / rho for c in range(3)]
    p = (gamma - 1.0) * (U[:, 4] - 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2))
    e, hh = U[:, 4] / rho, (U[:, 4] + p) / rho
    out = np.zeros(U.shape)
    for d in range(3):
        ax = 3 - d  # node index i + n(j + n k), array [e][k][j][i]: direction 0 is the last axis

        def Dd(f):
            return np.moveaxis(np.tensordot(D, np.moveaxis(f, ax, 0), axes=(1, 0)), 0, ax)

        def q2(a, b):
            return 0.5 * (a * Dd(b) + b * Dd(a) + Dd(a * b))

        def q3(a, b, c):
            return 0.25 * (a * b * Dd(c) + a * c * Dd(b) + b * c * Dd(a) + a * Dd(b * c) + b * Dd(a * c)
                           + c * Dd(a * b) + Dd(a * b * c))

        ud = u[d]
        if kind == "central":
            F = [rho * ud] + [rho * u[c] * ud + (p if c == d else 0.0) for c in range(3)] + [(U[:, 4] + p) * ud]
            vol = [Dd(f) for f in F]
        else:
            vol = [q2(rho, ud)] + [q3(rho, ud, u[c]) + (Dd(p) if c == d else 0.0) for c in range(3)]
            vol.append(q3(rho, ud, hh) if kind == "pirozzoli" else q3(rho, ud, e) + q2(p, ud))
        for v in range(5):
            out[:, v] -= (2.0 / h[d]) * vol[v]
    return out


@pytest.mark.parametrize("kind", ["pirozzoli", "kg", "central"])
def test_split_form_volume_flux_equals_product_rule_split(oracle_mod, kind):
    N = 5
    lo, hi, nel = (0.0, 0.0, 0.0), (2 * np.pi, 2 * np.pi, 2 * np.pi), (2, 3, 2)
    xyz, faces = W.box_mesh(N, nel, lo=lo, hi=hi)
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    # high wavenumbers on a coarse mesh: the splits are equivalent at any resolution, and under-resolved
    # data make the discretisation difference between the two energy averages large
    rho = 1.0 + 0.3 * np.sin(5 * x + 4 * y) * np.cos(3 * z)
    U = W.cons_from_prim(rho, 0.4 + 0.3 * np.cos(4 * y) * np.sin(5 * z), 0.2 * np.sin(3 * x + 4 * z),
                         -0.3 * np.cos(5 * x) * np.sin(4 * y), 1.0 + 0.2 * np.cos(4 * x - 3 * z) * np.sin(5 * y))
    D = oracle_mod.dmatrix(N)
    h = [(hi[d] - lo[d]) / nel[d] for d in range(3)]
    got = oracle_mod.Oracle(N, xyz, faces, vflux=kind, sflux="llf").rhs(U)
    want = _split_rhs(kind, U, D, h)
    mag = np.abs(want).max()
    print(f"SPLIT {kind}: max|oracle - split| / max|split| = {np.abs(got - want).max() / mag:.2e}")
    assert np.abs(got - want).max() <= 1e-11 * mag, np.abs(got - want).max() / mag
    if kind != "central":  # the other energy average is far off: the pin sees the energy flux
        other = _split_rhs("kg" if kind == "pirozzoli" else "pirozzoli", U, D, h)
        assert np.abs(got[:, 4] - other[:, 4]).max() > 1e-2 * np.abs(want[:, 4]).max()
        np.testing.assert_allclose(got[:, :4], other[:, :4], rtol=0, atol=1e-12 * mag)
