"""GPU parity: libdg's CUDA kernels (through the C ABI) against the FP64 CPU oracle on the
same seeded inputs, element by element.

Every FP64 comparison asserts and prints two figures per conservative variable (tests/helpers.py):
- normwise: max |Ut_GPU - Ut_oracle| may not exceed ULP_FACTOR times the oracle's own spread under
  seeded one-ulp perturbations of its inputs (state values and mesh points), i.e. the GPU must agree
  with the oracle as closely as the problem's conditioning lets any two correct FP64 evaluations
  agree (the printed "normwise" and "bound" are relative to max |Ut_oracle|);
- flux scale: max |Ut_GPU - Ut_oracle| <= 1e-12 scale_v, scale_v = ||2D||_inf max_nodes
  sum_d |F^d_v(U)| / J, the largest flux-difference term the right-hand side sums.
Time-stepped states use the spread of the oracle's own time-stepped states, and dt * scale_v per
stage.
"""
import numpy as np
import pytest

from helpers import (TOL, check_fp64, face_jump_magnitude, flux_scale, full_size_ulp_spread, parity,
                     saved_state_ulp_spread, subcell_range_magnitude, ulp_spread)
from paper_2306_12891_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def pair(env, N, xyz, faces, **phys):
    dg, orc, torch = env
    return dg.DG(N, xyz, faces, **phys), orc.Oracle(N, xyz, faces, **phys)


def check_rhs(env, N, xyz, faces, U0, period=2 * np.pi, **phys):
    dg, orc, torch = env
    gpu, ref = pair(env, N, xyz, faces, **phys)
    U = torch.from_numpy(U0).cuda()
    Ut = gpu.rhs(U).cpu().numpy()
    spread, Ut_ref = ulp_spread(lambda X, V: orc.Oracle(N, X, faces, **phys).rhs(V), xyz, U0, period=period,
                                base=ref.rhs(U0))
    sub = subcell_range_magnitude(U0, ref.Ja) if phys.get("shock_capturing") else None
    scale = flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(N), faces=faces, N=N, jump=sub)
    err, _ = check_fp64(f"N={N} nE={xyz.shape[0]} {phys}", Ut, Ut_ref, spread, scale)
    gpu.check()
    return gpu, ref, err


def jumpy(U, seed, amp=0.01):
    return U * (1.0 + amp * np.random.default_rng(seed).uniform(-1, 1, U.shape))


# ------------------------------------------------------------------ the small Euler workload in full

def test_tgv_euler_n3_rhs_and_ten_steps(env):
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_euler_n3_4x4x4"]
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    gpu, ref, _ = check_rhs(env, w.N, xyz, faces, U0, **w.physics())
    dt = ref.max_dt(U0, w.cfl)
    assert gpu.max_dt(torch.from_numpy(U0).cuda(), w.cfl) == pytest.approx(dt, rel=1e-13)
    U = torch.from_numpy(U0).cuda()
    for _ in range(w.steps):
        gpu.lserk_step(U, dt)

    def evolve(X, V):
        o = orc.Oracle(w.N, X, faces, **w.physics())
        for _ in range(w.steps):
            V = o.lserk_step(V, dt)
        return V

    spread, Uref = ulp_spread(evolve, xyz, U0)
    scale = flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(w.N))
    check_fp64("tgv_euler_n3_4x4x4 ten steps", U.cpu().numpy(), Uref, spread, dt * scale, tol=5 * w.steps * TOL)
    assert np.abs(Uref - U0).max() > 1e-3  # the state moved


# ------------------------------------------------------------------ flux / physics combinations, ragged meshes

COMBOS = [("kg", "llf", "euler"), ("pirozzoli", "roe", "euler"), ("ec", "ec", "euler"), ("central", "llf", "euler"),
          ("pirozzoli", "roe", "ns"), ("kg", "llf", "ns"), ("ec", "ec", "ns")]


@pytest.mark.parametrize("vf,sf,eq", COMBOS)
@pytest.mark.parametrize("N,nel", [(2, (3, 5, 3)), (3, (5, 3, 1)), (5, (3, 3, 3)), (7, (2, 1, 3))])
def test_rhs_combinations_on_ragged_curved_meshes(env, vf, sf, eq, N, nel):
    xyz, faces = W.box_mesh(N, nel, mapping=_generic_map)
    U0 = jumpy(W.random_smooth_state(xyz, seed=N * 7 + len(vf), amp=0.1), seed=3)
    check_rhs(env, N, xyz, faces, U0, equations=eq, vflux=vf, sflux=sf, mu=0.02)


@pytest.mark.parametrize("N", range(1, 8))
def test_rhs_every_degree(env, N):
    xyz, faces = W.box_mesh(N, (2, 3, 2), mapping="sine_0.05")
    U0 = jumpy(W.taylor_green(xyz), seed=N)
    check_rhs(env, N, xyz, faces, U0, equations="ns", vflux="pirozzoli", sflux="roe", mu=1.0 / 1600)


@pytest.mark.parametrize("N,eq,sc", [(3, "ns", False), (5, "euler", True), (7, "ns", False), (2, "euler", False)])
def test_rhs_on_mesh_with_rotated_elements(env, N, eq, sc):
    """Unstructured connectivity: half the elements re-indexed by cube rotations, faces of most of
    the eight orientation codes, face table rebuilt from the node coordinates."""
    xyz, faces, _ = W.rotated_box_mesh(N, (3, 2, 3), seed=N, mapping=_generic_map)
    assert len(set(faces[:, 4])) >= 4
    U0 = jumpy(W.random_smooth_state(xyz, seed=N, amp=0.1), seed=N + 1)
    extra = dict(shock_capturing=True, alpha_fixed=0.4) if sc else {}
    check_rhs(env, N, xyz, faces, U0, equations=eq, vflux="pirozzoli", sflux="roe", mu=0.02, **extra)


def test_single_element_periodic_mesh(env):
    N = 4
    xyz, faces = W.box_mesh(N, (1, 1, 1), mapping=_generic_map)
    U0 = jumpy(W.random_smooth_state(xyz, seed=5, amp=0.1), seed=6)
    check_rhs(env, N, xyz, faces, U0, equations="ns", vflux="kg", sflux="roe", mu=0.05)


def test_freestream_on_curved_mesh(env):
    dg, orc, torch = env
    N = 7
    xyz, faces = W.box_mesh(N, (3, 2, 2), mapping=_generic_map)
    U0 = W.freestream(xyz)
    gpu, ref = pair(env, N, xyz, faces, equations="ns", vflux="pirozzoli", sflux="roe", mu=0.01)
    Ut = gpu.rhs(torch.from_numpy(U0).cuda()).cpu().numpy()
    scale = flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(N))
    print(f"FREESTREAM N={N}: GPU max|Ut| {np.abs(Ut).max():.2e}, oracle {np.abs(ref.rhs(U0)).max():.2e}, "
          f"flux scale {scale.max():.2e}")
    assert np.abs(Ut).max() <= TOL * scale.max()


# ------------------------------------------------------------------ the N=7 Navier-Stokes physics, reduced mesh

def test_tgv_ns_n7_curved_reduced_rhs_and_step(env):
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n7_32x32x32_curved"].with_(nel=(4, 4, 4))
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    gpu, ref, _ = check_rhs(env, w.N, xyz, faces, U0, **w.physics())
    dt = ref.max_dt(U0, w.cfl)
    U = torch.from_numpy(U0).cuda()
    gpu.lserk_step(U, dt)
    spread, U1 = ulp_spread(lambda X, V: orc.Oracle(w.N, X, faces, **w.physics()).lserk_step(V, dt), xyz, U0)
    scale = flux_scale(U0, ref.Ja, ref.J, orc.dmatrix(w.N))
    check_fp64("tgv_ns_n7_4x4x4 one step", U.cpu().numpy(), U1, spread, dt * scale, tol=5 * TOL)


# ------------------------------------------------------------------ shock capturing

def test_indicator_and_blended_rhs_on_blast(env):
    dg, orc, torch = env
    w = W.WORKLOADS["blast_euler_fv_n5_64x64x64"].with_(nel=(6, 6, 6))
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    gpu, ref = pair(env, w.N, xyz, faces, **w.physics())
    U = torch.from_numpy(U0).cuda()
    alpha = gpu.indicator(U).cpu().numpy()
    raw_ref, alpha_ref = ref.indicator(U0)
    assert (alpha_ref > 0).sum() >= 10 and (alpha_ref == 0).sum() >= 10  # both regimes present
    np.testing.assert_allclose(alpha, alpha_ref, rtol=0, atol=1e-12)
    check_rhs(env, w.N, xyz, faces, U0, period=1.0, **w.physics())


@pytest.mark.parametrize("alpha", [1.0, 0.37])
@pytest.mark.parametrize("sf,eq", [("llf", "euler"), ("roe", "euler"), ("roe", "ns")])
def test_fv_blend_with_fixed_alpha(env, alpha, sf, eq):
    N = 5
    xyz, faces = W.box_mesh(N, (3, 2, 3), mapping=_generic_map)
    U0 = jumpy(W.random_smooth_state(xyz, seed=11, amp=0.1), seed=12, amp=0.05)
    check_rhs(env, N, xyz, faces, U0, equations=eq, vflux="pirozzoli", sflux=sf, mu=0.02, shock_capturing=True,
              alpha_fixed=alpha)


# ------------------------------------------------------------------ reductions and host entry point

def test_invariants_match_oracle(env):
    dg, orc, torch = env
    N = 5
    xyz, faces = W.box_mesh(N, (3, 3, 2), mapping="sine_0.05")
    U0 = jumpy(W.taylor_green(xyz), seed=2)
    gpu, ref = pair(env, N, xyz, faces, equations="ns", vflux="pirozzoli", sflux="roe", mu=0.01)
    U = torch.from_numpy(U0).cuda()
    Ut = gpu.rhs(U)
    inv = gpu.invariants(U, Ut)
    inv_ref = ref.invariants(U0, Ut.cpu().numpy())
    np.testing.assert_allclose(inv, inv_ref, rtol=1e-12, atol=1e-12 * np.abs(inv_ref).max())
    assert np.abs(inv[:5]).max() < 1e-10  # conservation on the GPU


def test_host_buffer_step_equals_device_step(env):
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_euler_n3_4x4x4"]
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    gpu = dg.DG(w.N, xyz, faces, **w.physics())
    U = torch.from_numpy(U0).cuda()
    gpu.lserk_step(U, 1e-3)
    Uh = torch.from_numpy(U0.copy()).pin_memory()  # page-locked: copied by the SMs over the host link
    gpu.lserk_step_host(Uh, 1e-3)
    assert torch.equal(Uh, U.cpu())
    Up = torch.from_numpy(U0.copy())  # pageable: copied by the copy engines, four streams
    gpu.lserk_step_host(Up, 1e-3)
    assert torch.equal(Up, U.cpu())
    # page-locked but not 16-byte aligned (a view one double in): the copy engines again
    big = torch.zeros(U0.size + 1, dtype=torch.float64).pin_memory()
    Uo = big[1:].view(U0.shape)
    Uo.copy_(torch.from_numpy(U0))
    gpu.lserk_step_host(Uo, 1e-3)
    assert torch.equal(Uo, U.cpu())
    # a non-finite step size is refused before anything is copied
    with pytest.raises(dg.DGError) as ei:
        gpu.lserk_step_host(Uo, float("nan"))
    assert ei.value.status == -1
    assert torch.equal(Uo, U.cpu())


def test_host_buffer_step_with_a_size_not_a_multiple_of_16_bytes(env):
    """N = 2 on three elements: 405 doubles, so the state is not a whole number of 16-byte words."""
    dg, orc, torch = env
    N = 2
    xyz, faces = W.box_mesh(N, (3, 1, 1), mapping=_generic_map)
    U0 = jumpy(W.random_smooth_state(xyz, seed=4, amp=0.1), seed=5)
    assert (U0.size * 8) % 16 != 0
    gpu = dg.DG(N, xyz, faces, equations="ns", vflux="pirozzoli", sflux="roe", mu=0.02)
    U = torch.from_numpy(U0).cuda()
    gpu.lserk_step(U, 1e-4)
    Uh = torch.from_numpy(U0.copy()).pin_memory()
    gpu.lserk_step_host(Uh, 1e-4)
    assert torch.equal(Uh, U.cpu())


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_host_buffer_step_navier_stokes_n7(env, precision):
    """With a page-locked host state the last stage's volume kernel writes the new state straight into
    host memory: the same bits as the device step, for the FP64 and the FP32-bulk kernels at N = 7,
    over consecutive calls (each call uploads its own input)."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n7_32x32x32_curved"].with_(nel=(3, 3, 3))
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    gpu = dg.DG(w.N, xyz, faces, precision=precision, **w.physics())
    U = torch.from_numpy(U0).cuda()
    dt = gpu.max_dt(U, w.cfl)
    Uh = torch.from_numpy(U0.copy()).pin_memory()
    for _ in range(3):
        gpu.lserk_step(U, dt)
        gpu.lserk_step_host(Uh, dt)
        assert torch.equal(Uh, U.cpu())
    gpu.check()


# ------------------------------------------------------------------ full-size workloads, sampled outputs

@pytest.mark.parametrize("name,extra", [("tgv_ns_n7_32x32x32_curved", {}), ("blast_euler_fv_n5_64x64x64", {}),
                                        ("blast_euler_fv_n5_64x64x64", {"alpha_fixed": 0.5})])
def test_full_size_rhs_sampled(env, name, extra):
    """The full-size workload on the GPU; the oracle evaluates a sample of elements (corners
    of the box and random ones) one by one. At 64^3 the blast front (tanh width 0.01 = 0.64 h)
    is resolved, so the indicator flags no element at t = 0 (the blend is then pure DG, and the
    sampled alphas must agree); the fixed-alpha case runs the FV subcell path everywhere."""
    dg, orc, torch = env
    w = W.WORKLOADS[name]
    phys = dict(w.physics(), **extra)
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    gpu = dg.DG(w.N, xyz, faces, **phys)
    U = torch.from_numpy(U0).cuda()
    Ut = gpu.rhs(U).cpu().numpy()
    gpu.check()
    nx, ny, nz = w.nel
    corners = [0, nx - 1, nx * ny - 1, nx * ny * nz - 1]
    rng = np.random.default_rng(20230622)
    sample = sorted(set(corners + list(rng.choice(w.n_elems, 12, replace=False))))
    ref = orc.Oracle(w.N, xyz, faces, **phys)
    Ut_ref, alpha_ref = ref.rhs(U0, mask=sample, return_alpha=True)
    if w.shock_capturing and "alpha_fixed" not in extra:
        alpha = gpu.indicator(U).cpu().numpy()
        np.testing.assert_allclose(alpha[sample], alpha_ref[sample], rtol=0, atol=1e-12)
    spread = full_size_ulp_spread(name, extra, sample, Ut_ref[sample])
    jump = face_jump_magnitude(U0, faces, w.N, ref.Ja, elements=sample)[sample]
    if phys.get("shock_capturing"):
        jump = jump + subcell_range_magnitude(U0[sample], ref.Ja[sample])
    scale = flux_scale(U0[sample], ref.Ja[sample], ref.J[sample], orc.dmatrix(w.N), jump=jump)
    check_fp64(f"full-size {name} {extra}", Ut[sample], Ut_ref[sample], spread, scale)


def test_full_size_shocked_blast_indicator_and_fv_rhs(env, tmp_path):
    """The shock-capturing workload where it does FV work: the blast at 64^3 advanced on the GPU for
    its 200 LSERK steps (dt from the CFL condition every 20 steps), when the indicator flags a shell of
    elements around the shock. At that state: alpha of every element against the oracle's indicator,
    and the right-hand side of sampled troubled and untroubled elements against the oracle (the FV
    subcell operator on real troubled elements, not a fixed alpha)."""
    dg, orc, torch = env
    name = "blast_euler_fv_n5_64x64x64"
    w = W.WORKLOADS[name]
    xyz, faces = w.mesh()
    gpu = dg.DG(w.N, xyz, faces, **w.physics())
    U = torch.from_numpy(w.initial_state(xyz)).cuda()
    for _ in range(w.steps // 20):
        gpu.lserk_steps(U, gpu.max_dt(U, w.cfl), 20)
    gpu.check()
    alpha = gpu.indicator(U).cpu().numpy()
    Ut = gpu.rhs(U).cpu().numpy()
    Uh = U.cpu().numpy()
    ref = orc.Oracle(w.N, xyz, faces, **w.physics())
    _, alpha_ref = ref.indicator(Uh)
    troubled = np.flatnonzero(alpha_ref > 0)
    print(f"SHOCKED blast: troubled fraction {troubled.size / w.n_elems:.4f}, "
          f"max |alpha - alpha_oracle| {np.abs(alpha - alpha_ref).max():.2e}")
    assert 0.02 < troubled.size / w.n_elems < 0.3
    np.testing.assert_allclose(alpha, alpha_ref, rtol=0, atol=1e-12)
    rng = np.random.default_rng(20230625)
    calm = np.flatnonzero(alpha_ref == 0)
    sample = sorted(set(rng.choice(troubled, 12, replace=False)) | set(rng.choice(calm, 4, replace=False)))
    Ut_ref = ref.rhs(Uh, mask=sample)[sample]
    path = str(tmp_path / "U.npy")
    np.save(path, Uh)
    spread = saved_state_ulp_spread(name, path, sample, Ut_ref)
    jump = face_jump_magnitude(Uh, faces, w.N, ref.Ja, elements=sample)[sample]
    jump = jump + subcell_range_magnitude(Uh[sample], ref.Ja[sample])
    scale = flux_scale(Uh[sample], ref.Ja[sample], ref.J[sample], orc.dmatrix(w.N), jump=jump)
    check_fp64("shocked blast 64^3 after 200 steps, sampled elements", Ut[sample], Ut_ref, spread, scale)
    # the FP32-bulk form's right-hand side at the same state (FV subcells in FP32), within its tolerance
    g32 = dg.DG(w.N, xyz, faces, precision="fp32_bulk", **w.physics())
    Ut32 = g32.rhs(U).cpu().numpy()[sample]
    g32.check()
    scale32 = flux_scale(Uh[sample], ref.Ja[sample], ref.J[sample], orc.dmatrix(w.N), state_dissipation=True,
                         jump=jump)
    err32 = parity(Ut32, Ut_ref, scale32)
    print(f"PARITY32 shocked blast 64^3 sampled elements: flux-scale {err32}")
    assert (err32 <= 64 * 2.0 ** -24).all(), err32


def test_full_size_lserk_step_matches_stagewise_definition(env):
    """The fused LSERK(5,4) update of the volume kernel equals the 2N-storage definition
    g = A_s g + dt L(U); U = U + B_s g applied with separate right-hand sides."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n7_32x32x32_curved"]
    xyz, faces = w.mesh()
    U0 = torch.from_numpy(w.initial_state(xyz)).cuda()
    gpu = dg.DG(w.N, xyz, faces, **w.physics())
    dt = gpu.max_dt(U0, w.cfl)
    A, B, _ = orc.lserk_coefficients()
    U = U0.clone()
    g = torch.zeros_like(U)
    for s in range(5):
        g = A[s] * g + dt * gpu.rhs(U)
        U = U + B[s] * g
    V = U0.clone()
    gpu.lserk_step(V, dt)
    U0h = U0.cpu().numpy()
    Ja_s, J_s = gpu.metrics()
    scale = flux_scale(U0h, Ja_s.cpu().numpy(), J_s.cpu().numpy(), orc.dmatrix(w.N))
    err = parity(V.cpu().numpy(), U.cpu().numpy(), dt * scale)
    assert (err <= 5 * TOL).all(), err
    gpu.check()


# ------------------------------------------------------------------ errors and edge cases

def test_init_rejects_bad_input(env):
    dg, orc, torch = env
    N = 3
    xyz, faces = W.box_mesh(N, (2, 2, 2))
    phys = dict(equations="euler", vflux="kg", sflux="llf")
    bad = faces.copy()
    bad[1, 1] = bad[0, 1]  # a face slot used twice
    with pytest.raises(dg.DGError) as ei:
        dg.DG(N, xyz, bad, **phys)
    assert ei.value.status == -2
    with pytest.raises(dg.DGError) as ei:
        dg.DG(N, xyz, faces[:-1], **phys)  # an unconnected face slot
    assert ei.value.status == -2
    with pytest.raises(dg.DGError) as ei:
        dg.DG(8, np.zeros((8, 3, 9, 9, 9)), faces, **phys)
    assert ei.value.status == -1
    with pytest.raises(dg.DGError) as ei:
        dg.DG(N, xyz[:0], faces[:0], **phys)  # empty mesh
    assert ei.value.status == -1
    flipped = xyz.copy()
    flipped[3] = flipped[3][:, :, :, ::-1]  # mirror one element: J < 0
    with pytest.raises(dg.DGError) as ei:
        dg.DG(N, flipped, faces, **phys)
    assert ei.value.status == -3


def test_nonphysical_state_is_reported(env):
    dg, orc, torch = env
    N = 3
    xyz, faces = W.box_mesh(N, (2, 2, 2))
    gpu = dg.DG(N, xyz, faces, equations="euler", vflux="kg", sflux="llf")
    U0 = W.freestream(xyz)
    U0[1, 0, 1, 1, 1] = -1.0  # negative density at one interior node
    U = torch.from_numpy(U0).cuda()
    gpu.rhs(U)
    with pytest.raises(dg.DGError) as ei:
        gpu.check()
    assert ei.value.status == -5
    gpu.check()  # the flag was cleared


def test_timing_and_launch_counts(env):
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n7_32x32x32_curved"].with_(nel=(2, 2, 2))
    xyz, faces = w.mesh()
    gpu = dg.DG(w.N, xyz, faces, **w.physics())
    U = torch.from_numpy(w.initial_state(xyz)).cuda()
    c0 = gpu.launch_count()
    gpu.timing_enable(True)
    gpu.lserk_steps(U, 1e-4, 2)
    t = gpu.timing_get()
    assert gpu.launch_count() - c0 == 2 * 5 * 3  # face, lift, volume per stage
    assert t["volume"][1] == 10 and t["face"][1] == 10 and t["lift"][1] == 10
    assert t["volume"][0] > 0
