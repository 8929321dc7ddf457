"""FP32-bulk precision form against the FP64 oracle.

Volume, surface and lifting arithmetic run in FP32 with FP32 accumulation; U is read as FP64,
metrics and Jacobian are computed in FP64, and the LSERK register/state accumulation and the
reductions stay FP64 (the stage increment is the FP32 sum times the factor dt (-1/J), formed in FP64
and rounded once). The error of each result against the FP64 oracle is stated (printed as
PARITY32 lines) and bounded: relative to the flux scale of tests/helpers.py the right-hand side
must agree to TOL32 = 64 * 2^-24 (~3.8e-6) -- FP32 rounding of the O(3(N+1)) flux-difference terms
-- and time-stepped states relative to dt * scale per stage.
"""
import numpy as np
import pytest

from helpers import flux_scale as _flux_scale, normwise, parity
from paper_2306_12891_gb300 import workloads as W

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -24
TOL32 = 64 * EPS32
P0_TGV = 1.0 / (1.4 * 0.1 ** 2)  # Taylor-Green background pressure at Ma 0.1


def flux_scale(U, Ja, J, D):
    """The flux scale with the FP32 state-rounding term c |Ja| |U| of the Riemann dissipation: in this
    form the dissipation differences states rounded to FP32 (tests/helpers.py)."""
    return _flux_scale(U, Ja, J, D, state_dissipation=True)


@pytest.fixture(scope="module")
def env(oracle_mod):
    import torch

    from paper_2306_12891_gb300 import build, dg

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    dg.lib()
    return dg, oracle_mod, torch


def _generic_map(x, y, z):
    return (x + 0.1 * np.sin(y) * np.cos(z), y + 0.1 * np.sin(z) * np.sin(x) + 0.05 * np.sin(2 * x),
            z + 0.1 * np.sin(x) * np.cos(y))


def rhs_pair(env, N, xyz, faces, U0, p_ref=0.0, **phys):
    dg, orc, torch = env
    gpu = dg.DG(N, xyz, faces, precision="fp32_bulk", p_ref=p_ref, **phys)
    ref = orc.Oracle(N, xyz, faces, **phys)
    Ut = gpu.rhs(torch.from_numpy(U0).cuda()).cpu().numpy()
    gpu.check()
    return gpu, ref, Ut, ref.rhs(U0)


def test_fp32_rhs_tgv_ns_n7_curved(env):
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n7_48x48x48_curved_fp32"].with_(nel=(4, 4, 4))
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    scale = None
    errs = {}
    for pr in (0.0, P0_TGV):
        gpu, ref, Ut, Ur = rhs_pair(env, w.N, xyz, faces, U0, p_ref=pr, **w.physics())
        if scale is None:
            scale = flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(w.N))
        errs[pr] = parity(Ut, Ur, scale)
        print(f"PARITY32 tgv N=7 4^3 p_ref={pr:.3f}: flux-scale {errs[pr]} normwise {normwise(Ut, Ur)}")
    assert (errs[P0_TGV] <= TOL32).all(), errs
    # removing the background pressure is exact and helps the momentum equations
    assert errs[P0_TGV][1:4].max() < errs[0.0][1:4].max()


@pytest.mark.parametrize("vf,sf,eq", [("kg", "llf", "euler"), ("pirozzoli", "roe", "euler"), ("pirozzoli", "roe", "ns"),
                                      ("ec", "ec", "euler"), ("central", "llf", "ns")])
@pytest.mark.parametrize("N,nel", [(3, (5, 3, 1)), (5, (3, 3, 3)), (7, (2, 1, 3))])
def test_fp32_rhs_combinations(env, vf, sf, eq, N, nel):
    dg, orc, torch = env
    xyz, faces = W.box_mesh(N, nel, mapping=_generic_map)
    U0 = W.random_smooth_state(xyz, seed=N + 3, amp=0.1)
    U0 = U0 * (1.0 + 0.01 * np.random.default_rng(4).uniform(-1, 1, U0.shape))
    gpu, ref, Ut, Ur = rhs_pair(env, N, xyz, faces, U0, p_ref=1.0 / 1.4, equations=eq, vflux=vf, sflux=sf, mu=0.02)
    err = parity(Ut, Ur, flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(N)))
    print(f"PARITY32 N={N} {vf}/{sf}/{eq}: {err}")
    assert (err <= TOL32).all(), (err, normwise(Ut, Ur))


def test_fp32_rotated_elements(env):
    dg, orc, torch = env
    N = 5
    xyz, faces, _ = W.rotated_box_mesh(N, (3, 2, 3), seed=7, mapping=_generic_map)
    U0 = W.random_smooth_state(xyz, seed=2, amp=0.1)
    gpu, ref, Ut, Ur = rhs_pair(env, N, xyz, faces, U0, p_ref=1.0 / 1.4, equations="ns", vflux="pirozzoli",
                                sflux="roe", mu=0.02)
    err = parity(Ut, Ur, flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(N)))
    print(f"PARITY32 rotated N={N}: {err}")
    assert (err <= TOL32).all(), (err, normwise(Ut, Ur))


@pytest.mark.parametrize("alpha", [1.0, 0.37])
def test_fp32_fv_blend(env, alpha):
    dg, orc, torch = env
    N = 5
    xyz, faces = W.box_mesh(N, (3, 2, 3), mapping=_generic_map)
    U0 = W.random_smooth_state(xyz, seed=11, amp=0.1)
    U0 = U0 * (1.0 + 0.05 * np.random.default_rng(12).uniform(-1, 1, U0.shape))
    gpu, ref, Ut, Ur = rhs_pair(env, N, xyz, faces, U0, p_ref=1.0 / 1.4, equations="euler", vflux="pirozzoli",
                                sflux="llf", shock_capturing=True, alpha_fixed=alpha)
    err = parity(Ut, Ur, flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(N)))
    print(f"PARITY32 FV alpha={alpha}: {err}")
    assert (err <= TOL32).all(), (err, normwise(Ut, Ur))


def test_fp32_freestream_and_conservation(env):
    dg, orc, torch = env
    N = 7
    xyz, faces = W.box_mesh(N, (3, 2, 2), mapping=_generic_map)
    U0 = W.freestream(xyz)
    gpu, ref, Ut, _ = rhs_pair(env, N, xyz, faces, U0, p_ref=1.0 / 1.4, equations="ns", vflux="pirozzoli", sflux="roe",
                               mu=0.01)
    scale = flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(N))
    assert np.abs(Ut).max() <= TOL32 * scale.max()
    U0 = W.random_smooth_state(xyz, seed=8, amp=0.1)
    U = torch.from_numpy(U0).cuda()
    Ut = gpu.rhs(U)
    inv = gpu.invariants(U, Ut)  # FP64 reduction of the FP32-computed right-hand side
    w = orc.lgl(N)[1]
    wq = np.einsum("k,j,i->kji", w, w, w)[None] * ref.J
    mag = np.einsum("ekji,evkji->v", wq, np.abs(Ut.cpu().numpy()))
    print(f"PARITY32 conservation: {np.abs(inv[:5]) / mag}")
    assert (np.abs(inv[:5]) <= 1e3 * EPS32 * mag).all()


def test_fp32_ten_steps_tgv(env):
    """Ten LSERK(5,4) steps of the FP32-bulk form against the FP64 oracle; L2 and Linf per variable."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n7_48x48x48_curved_fp32"].with_(nel=(3, 3, 3))
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    gpu = dg.DG(w.N, xyz, faces, precision="fp32_bulk", p_ref=P0_TGV, **w.physics())
    ref = orc.Oracle(w.N, xyz, faces, **w.physics())
    dt = ref.max_dt(U0, w.cfl)
    U = torch.from_numpy(U0).cuda()
    Ur = U0.copy()
    K = 10
    for _ in range(K):
        gpu.lserk_step(U, dt)
        Ur = ref.lserk_step(Ur, dt)
    U32 = U.cpu().numpy()
    d = (U32 - Ur).reshape(Ur.shape[0], 5, -1)
    linf = np.abs(d).max(axis=(0, 2))
    l2 = np.sqrt((d ** 2).mean(axis=(0, 2)))
    change = np.abs(Ur - U0).reshape(Ur.shape[0], 5, -1).max(axis=(0, 2))
    scale = flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(w.N))
    print(f"PARITY32 tgv N=7 3^3 after {K} steps: Linf {linf} L2 {l2}; Linf/change {linf / change}")
    assert (linf <= 5 * K * TOL32 * dt * scale).all(), (linf, dt * scale)


def test_integer_pipe_conversions(env):
    """The FP32-bulk epilogue converts float <-> double on the integer pipes; it must agree bit for
    bit with the GPU's own conversions (round to nearest even) outside the documented flush range."""
    dg, orc, torch = env
    bad = dg.check_conversions(1 << 24)
    print(f"conversion mismatches (f2d, d2f) over 2^24 patterns each: {bad}")
    assert bad == (0, 0)


@pytest.mark.parametrize("N,phys", [(3, dict(equations="euler", vflux="kg", sflux="llf")),
                                    (5, dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=0.02)),
                                    (7, dict(equations="ns", vflux="ec", sflux="ec", mu=0.02)),
                                    (4, dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=0.02))])
def test_tma_kernel_matches_plain_kernel(env, N, phys):
    """The TMA-fed persistent FP32 volume kernel runs the same per-node arithmetic as the plain one:
    identical bits for the right-hand side and for LSERK steps (N = 4 has no TMA form: same path)."""
    dg, orc, torch = env
    xyz, faces = W.box_mesh(N, (3, 2, 3), mapping=_generic_map)
    U0 = torch.from_numpy(W.random_smooth_state(xyz, seed=N, amp=0.1)).cuda()
    res = []
    for mode in (0, 1, 2):
        s = dg.DG(N, xyz, faces, precision="fp32_bulk", p_ref=1.0 / 1.4, **phys)
        s.use_tma(mode)
        Ut = s.rhs(U0)
        U = U0.clone()
        s.lserk_steps(U, 1e-3, 3)
        s.check()
        res.append((Ut, U))
    for r in res[1:]:
        assert torch.equal(res[0][0], r[0]) and torch.equal(res[0][1], r[1])


def test_tma_kernel_with_walls(env):
    dg, orc, torch = env
    xyz, faces = W.box_mesh(5, (3, 2, 3), lo=(0, 0, 0), hi=(2 * np.pi, np.pi, 2.0), z_walls=True)
    U0 = torch.from_numpy(W.random_smooth_state(xyz, seed=3, amp=0.1)).cuda()
    res = []
    for mode in (0, 1, 2):
        s = dg.DG(5, xyz, faces, precision="fp32_bulk", p_ref=1.0 / 1.4, equations="ns", vflux="pirozzoli",
                  sflux="roe", mu=1e-3)
        s.use_tma(mode)
        res.append(s.rhs(U0))
        s.check()
    assert torch.equal(res[0], res[1]) and torch.equal(res[0], res[2])


def test_full_size_fp32_rhs_sampled(env):
    """The FP32-bulk form at its full size (N = 7, 48^3 curved, 56.6M DOF, the launch configuration
    bench.py times) against the FP64 oracle on a sample of elements (box corners and random ones)."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n7_48x48x48_curved_fp32"]
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    gpu = dg.DG(w.N, xyz, faces, precision="fp32_bulk", p_ref=P0_TGV, **w.physics())
    Ut = gpu.rhs(torch.from_numpy(U0).cuda()).cpu().numpy()
    gpu.check()
    nx, ny, nz = w.nel
    corners = [0, nx - 1, nx * ny - 1, nx * ny * nz - 1]
    sample = sorted(set(corners + list(np.random.default_rng(48).choice(w.n_elems, 8, replace=False))))
    ref = orc.Oracle(w.N, xyz, faces, **w.physics())
    Ur = ref.rhs(U0, mask=sample)
    scale = flux_scale(U0[sample], ref.Ja[sample], ref.J[sample], orc.dmatrix(w.N))
    err = parity(Ut[sample], Ur[sample], scale)
    print(f"PARITY32 full size 48^3: {err}")
    assert (err <= TOL32).all(), err


def _line_pair(env, xyz, faces, U0, mode, p_ref=1.0 / 1.4, **phys):
    dg, orc, torch = env
    gpu = dg.DG(7, xyz, faces, precision="fp32_bulk", p_ref=p_ref, **phys)
    gpu.use_tma(mode)
    Ut = gpu.rhs(torch.from_numpy(U0).cuda()).cpu().numpy()
    gpu.check()
    return gpu, Ut


@pytest.mark.parametrize("vf,sf,eq", [("kg", "llf", "euler"), ("pirozzoli", "roe", "ns"), ("kg", "roe", "ns"),
                                      ("ec", "ec", "euler"), ("central", "llf", "ns")])
def test_line_kernel_rhs(env, vf, sf, eq):
    """The pair-symmetric FP32 line kernel (dg_use_tma(3), N = 7) against the FP64 oracle on a curved
    mesh. Its sums run in another order than the node kernels', so it is held to the FP32 tolerance,
    not to their bits."""
    dg, orc, torch = env
    xyz, faces = W.box_mesh(7, (2, 3, 2), mapping=_generic_map)
    U0 = W.random_smooth_state(xyz, seed=21, amp=0.1)
    U0 = U0 * (1.0 + 0.01 * np.random.default_rng(22).uniform(-1, 1, U0.shape))
    phys = dict(equations=eq, vflux=vf, sflux=sf, mu=0.02)
    _, Ut = _line_pair(env, xyz, faces, U0, 3, **phys)
    ref = orc.Oracle(7, xyz, faces, **phys)
    Ur = ref.rhs(U0)
    scale = flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(7))
    err = parity(Ut, Ur, scale)
    _, Ut0 = _line_pair(env, xyz, faces, U0, 0, **phys)
    err0 = parity(Ut0, Ur, scale)
    print(f"PARITY32 line kernel {vf}/{sf}/{eq}: {err} (node kernel {err0})")
    assert (err <= TOL32).all(), (err, normwise(Ut, Ur))


def test_line_kernel_rotated_elements_and_walls(env):
    dg, orc, torch = env
    phys = dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=0.02)
    xyz, faces, _ = W.rotated_box_mesh(7, (3, 2, 2), seed=9, mapping=_generic_map)
    U0 = W.random_smooth_state(xyz, seed=23, amp=0.1)
    _, Ut = _line_pair(env, xyz, faces, U0, 3, **phys)
    ref = orc.Oracle(7, xyz, faces, **phys)
    err = parity(Ut, ref.rhs(U0), flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(7)))
    print(f"PARITY32 line kernel rotated elements: {err}")
    assert (err <= TOL32).all(), err
    xyz, faces = W.box_mesh(7, (2, 2, 3), lo=(0, 0, 0), hi=(2 * np.pi, np.pi, 2.0), z_walls=True)
    U0 = W.random_smooth_state(xyz, seed=24, amp=0.1)
    phys = dict(phys, mu=1e-3, wm_index=2)
    _, Ut = _line_pair(env, xyz, faces, U0, 3, **phys)
    ref = orc.Oracle(7, xyz, faces, **phys)
    err = parity(Ut, ref.rhs(U0), flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(7)))
    print(f"PARITY32 line kernel wall-modelled channel: {err}")
    assert (err <= TOL32).all(), err


def test_line_kernel_steps(env):
    """Ten LSERK steps through the line kernel's fused FP64 epilogue against the FP64 oracle, and the
    graph-replayed steps bit for bit against directly launched ones."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n7_48x48x48_curved_fp32"].with_(nel=(3, 3, 3))
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    ref = orc.Oracle(w.N, xyz, faces, **w.physics())
    dt = ref.max_dt(U0, w.cfl)
    K = 10
    outs = []
    for graphs in (True, False):
        gpu = dg.DG(w.N, xyz, faces, precision="fp32_bulk", p_ref=P0_TGV, **w.physics())
        gpu.use_tma(3)
        gpu.use_graphs(graphs)
        U = torch.from_numpy(U0).cuda()
        gpu.lserk_steps(U, dt, K)
        gpu.check()
        outs.append(U)
    assert torch.equal(outs[0], outs[1])
    Ur = U0.copy()
    for _ in range(K):
        Ur = ref.lserk_step(Ur, dt)
    d = (outs[0].cpu().numpy() - Ur).reshape(Ur.shape[0], 5, -1)
    linf = np.abs(d).max(axis=(0, 2))
    scale = flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(w.N))
    print(f"PARITY32 line kernel after {K} steps: Linf {linf}")
    assert (linf <= 5 * K * TOL32 * dt * scale).all(), (linf, dt * scale)
