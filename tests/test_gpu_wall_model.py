"""Wall-modelled walls (Sec. 3) on the GPU against the oracle, through the C ABI.

- dg_wall_model (the per-wall-point Newton solve of Spalding's law, with and without the van Driest
  transform) against the oracle's wall_utau, point by point;
- the right-hand side of wall-bounded channels (walls at z = 0 and z = Hz, periodic in x and y):
  FP64 element by element within ULP_FACTOR times the oracle's one-ulp spread and 1e-12 of the
  flux scale (tests/helpers.py), FP32-bulk within 64 * 2^-24 of the flux scale, for several degrees, flux pairs, exchange indices and the DG/FV blend;
- at full size (N = 5, 48 x 24 x 24 channel): sampled wall and interior elements against the oracle,
  discrete conservation of mass and energy, and the exact wall-shear drain of x-momentum for uniform
  flow along the walls.
"""
import numpy as np
import pytest

from helpers import (check_fp64, face_jump_magnitude, flux_scale, normwise, parity, subcell_range_magnitude,
                     ulp_spread)
from paper_2306_12891_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
TOL32 = 64 * 2.0 ** -24
KAPPA, C = 0.4, 0.1108


@pytest.fixture(scope="module")
def env(oracle_mod):
    import torch

    from paper_2306_12891_gb300 import build, dg

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    dg.lib()
    return dg, oracle_mod, torch


def _curved(x, y, z):
    # curves the channel interior; the walls z = 0 and z = Hz stay planes
    return (x + 0.05 * np.sin(y) * np.sin(np.pi * z), y + 0.05 * np.sin(x) * np.sin(np.pi * z),
            z + 0.05 * np.sin(x) * np.sin(y) * np.sin(np.pi * z))


def _channel(N, nel, mapping=None, Hz=2.0):
    return W.box_mesh(N, nel, lo=(0.0, 0.0, 0.0), hi=(2.0 * np.pi, np.pi, Hz), mapping=mapping, z_walls=True)


def _state(xyz, seed=1):
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    rng = np.random.default_rng(seed)
    r = lambda: rng.uniform(-1, 1)
    rho = 1.0 + 0.05 * np.sin(x + r()) * np.cos(z)
    u = 0.8 + 0.1 * np.sin(y + r()) * np.sin(np.pi * z / 2)
    v = 0.05 * np.cos(x + r())
    w = 0.05 * np.sin(x) * np.sin(np.pi * z / 2) + 0.03 * np.cos(y + r())
    p = 1.0 / 1.4 + 0.02 * np.cos(x + y + r())
    U = W.cons_from_prim(rho, u, v, w, p)
    return U * (1.0 + 0.01 * rng.uniform(-1, 1, U.shape))


def test_wall_model_points_match_oracle(env):
    dg, orc, torch = env
    rng = np.random.default_rng(3)
    n = 2000
    U = rng.uniform(0.0, 2.0, n)
    U[:5] = 0.0
    h = 10 ** rng.uniform(-5, -0.5, n)
    nu = 10 ** rng.uniform(-7, -3, n)
    for vd, Ma in ((False, 0.0), (True, 0.8), (True, 2.0)):
        ut, it = dg.wall_model(*(torch.from_numpy(a).cuda() for a in (U, h, nu)), uinf=2.5, mainf=Ma,
                               van_driest=vd)
        ut, it = ut.cpu().numpy(), it.cpu().numpy()
        ref = np.array([orc.wall_utau(U[i], h[i], nu[i], 2.5, Ma, 1.4, 0.72, vd) for i in range(n)])
        err = np.abs(ut - ref) / np.maximum(np.abs(ref), 1e-300)
        print(f"WALL-MODEL vd={vd} Ma={Ma}: max rel err {err.max():.2e}, Newton iterations {it.min()}..{it.max()}")
        assert err.max() <= 1e-14
        assert (ut[:5] == 0).all() and it.max() <= 100


def _check(env, N, xyz, faces, U0, tol, precision="fp64", **phys):
    dg, orc, torch = env
    extra = dict(precision="fp32_bulk", p_ref=1.0 / 1.4) if precision == "fp32_bulk" else {}
    gpu = dg.DG(N, xyz, faces, **extra, **phys)
    ref = orc.Oracle(N, xyz, faces, **phys)
    Ut = gpu.rhs(torch.from_numpy(U0).cuda()).cpu().numpy()
    gpu.check()
    if precision == "fp64":
        spread, Ur = ulp_spread(lambda X, V: orc.Oracle(N, X, faces, **phys).rhs(V), xyz, U0,
                                period=(2 * np.pi, np.pi, 2.0), base=ref.rhs(U0))
        sub = subcell_range_magnitude(U0, ref.Ja) if phys.get("shock_capturing") else None
        check_fp64(f"wall N={N} {phys}", Ut, Ur, spread,
                   flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(N), faces=faces, N=N, jump=sub), tol=tol)
        return
    Ur = ref.rhs(U0)
    err = parity(Ut, Ur, flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(N), state_dissipation=True))
    print(f"PARITY32-WALL N={N} {phys}: flux-scale {err} normwise {normwise(Ut, Ur)}")
    assert (err <= tol).all(), (err, normwise(Ut, Ur))


@pytest.mark.parametrize("phys", [
    dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=1e-3),
    dict(equations="ns", vflux="kg", sflux="llf", mu=1e-2, wm_index=2),
    dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=2e-4, wm_van_driest=True, wm_mainf=0.8, wm_uinf=1.0),
    dict(equations="euler", vflux="pirozzoli", sflux="roe"),
])
@pytest.mark.parametrize("N,nel", [(3, (3, 2, 3)), (5, (2, 2, 2)), (7, (2, 1, 2))])
def test_channel_rhs_fp64(env, phys, N, nel):
    xyz, faces = _channel(N, nel, mapping=_curved)
    _check(env, N, xyz, faces, _state(xyz, seed=N), TOL, **phys)


@pytest.mark.parametrize("phys", [dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=1e-3),
                                  dict(equations="ns", vflux="kg", sflux="llf", mu=1e-2, wm_index=3,
                                       wm_van_driest=True, wm_mainf=0.5, wm_uinf=1.0)])
def test_channel_rhs_fp32_bulk(env, phys):
    xyz, faces = _channel(5, (3, 2, 2), mapping=_curved)
    _check(env, 5, xyz, faces, _state(xyz, seed=9), TOL32, precision="fp32_bulk", **phys)


def test_channel_with_fv_blend(env):
    xyz, faces = _channel(5, (2, 2, 3))
    _check(env, 5, xyz, faces, _state(xyz, seed=10), TOL, equations="ns", vflux="pirozzoli", sflux="llf", mu=1e-3,
           shock_capturing=True, alpha_fixed=0.4)


def test_full_size_channel_conservation_and_wall_shear(env):
    """N = 5 on a 48 x 24 x 24 channel (3.0M DOF): mass and energy are conserved to round-off with
    walls (no penetration, adiabatic wall at rest); uniform flow along the walls loses x-momentum at
    exactly 2 tau_w Lx Ly, tau_w from an independent root of Spalding's law at the exchange distance."""
    from scipy.optimize import brentq

    dg, orc, torch = env
    N, nel, Hz = 5, (48, 24, 24), 2.0
    xyz, faces = _channel(N, nel, Hz=Hz)
    phys = dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=2e-4, wm_index=1)
    gpu = dg.DG(N, xyz, faces, **phys)
    _, J = gpu.metrics()
    xi, w, _ = dg.basis(N)
    wq = torch.from_numpy(np.einsum("k,j,i->kji", w, w, w)).cuda()[None] * J
    U0 = _state(xyz, seed=12)
    U = torch.from_numpy(U0).cuda()
    Ut = gpu.rhs(U)
    # element by element against the oracle on sampled elements: both walls and the interior
    nx, ny, nz = nel
    rng = np.random.default_rng(20230626)
    bottom, top = rng.choice(nx * ny, 5, replace=False), (nz - 1) * nx * ny + rng.choice(nx * ny, 5, replace=False)
    sample = sorted(set(bottom) | set(top) | set(rng.choice(nx * ny * nz, 6, replace=False)))
    period = (2 * np.pi, np.pi, Hz)
    ref = orc.Oracle(N, xyz, faces, **phys)
    Ut_ref = ref.rhs(U0, mask=sample)[sample]
    spread, _ = ulp_spread(lambda X, V: orc.Oracle(N, X, faces, **phys).rhs(V, mask=sample)[sample], xyz, U0,
                           period=period, base=Ut_ref)
    scale = flux_scale(U0[sample], ref.Ja[sample], ref.J[sample], orc.dmatrix(N),
                       jump=face_jump_magnitude(U0, faces, N, ref.Ja, elements=sample)[sample])
    check_fp64("wall channel 48x24x24 sampled elements", Ut.cpu().numpy()[sample], Ut_ref, spread, scale)
    tot = torch.einsum("ekji,evkji->v", wq, Ut).cpu().numpy()
    mag = torch.einsum("ekji,evkji->v", wq, Ut.abs()).cpu().numpy()
    print(f"WALL full size: sum J w Ut / sum J w |Ut| = {tot / mag}")
    assert abs(tot[0]) <= 1e-13 * mag[0] and abs(tot[4]) <= 1e-13 * mag[4]
    rho, Ub = 1.1, 0.9
    one = np.ones_like(xyz[:, 0])
    Uu = torch.from_numpy(W.cons_from_prim(rho * one, Ub * one, 0 * one, 0 * one, 0.8 * one)).cuda()
    dmom = float(torch.einsum("ekji,ekji->", wq, gpu.rhs(Uu)[:, 1]))
    h = (xi[1] - xi[0]) / 2.0 * (Hz / nel[2])
    Re = h * Ub * rho / phys["mu"]
    f = lambda up: up * (up + C * (np.exp(KAPPA * up) - 1 - KAPPA * up - (KAPPA * up) ** 2 / 2
                                   - (KAPPA * up) ** 3 / 6 - (KAPPA * up) ** 4 / 24)) - Re
    utau = Ub / brentq(f, 1e-12, 200.0, xtol=1e-15, rtol=1e-15)
    want = -2.0 * rho * utau ** 2 * (2 * np.pi) * np.pi
    print(f"WALL full size uniform flow: d(x-momentum)/dt {dmom:.15e}, -2 tau_w A {want:.15e}")
    assert abs(dmom / want - 1.0) < 1e-11
    gpu.check()


def test_wall_faces_refused_by_the_adjoint(env):
    dg, orc, torch = env
    xyz, faces = _channel(3, (2, 2, 2))
    gpu = dg.DG(3, xyz, faces, equations="ns", vflux="pirozzoli", sflux="roe", mu=1e-3)
    U = torch.from_numpy(_state(xyz)).cuda()
    with pytest.raises(dg.DGError) as ei:
        gpu.rhs_vjp(U, U.clone())
    assert ei.value.status == -6


def test_bad_wall_parameters(env):
    dg, orc, torch = env
    xyz, faces = _channel(3, (2, 2, 2))
    with pytest.raises(dg.DGError) as ei:
        dg.DG(3, xyz, faces, equations="ns", mu=1e-3, wm_index=0)
    assert ei.value.status == -1
    bad = faces.copy()
    bad[bad[:, 2] == -1, 3] = 7  # unknown boundary kind
    with pytest.raises(dg.DGError) as ei:
        dg.DG(3, xyz, bad, equations="ns", mu=1e-3)
    assert ei.value.status == -2
