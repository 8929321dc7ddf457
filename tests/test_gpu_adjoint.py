"""Discrete adjoint (vector-Jacobian products) of the CUDA path against the oracle's complex-step
derivatives, through the C ABI.

Reference: Oracle(..., complex_step=True) evaluates the oracle's own right-hand side L (and LSERK
step) at U + i h e_j, giving column j of dL/dU exactly (no cancellation error). So
(dL/dU^T lambda)_j = sum_i (dL/dU)_ij lambda_i is known element by element, for every j on small
meshes (dense Jacobian) and for sampled j on larger ones.

Tolerance: the adjoint is a sum of products of Jacobian entries and cotangents; two FP64
evaluations differ by rounding of those terms. The error of each conservative variable is taken
relative to scale_v = max over the checked j of variable v of sum_i |(dL/dU)_ij| |lambda_i| (computed
from the same complex-step columns) and must be <= 1e-12 (the FP64 parity bound). Identities that
hold at any size (discrete conservation, the scaling laws of the operator) are checked at the
benchmark sizes with the GPU forward and adjoint alone.
"""
import numpy as np
import pytest

from helpers import flux_scale
from paper_2306_12891_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ADJ_TOL = 1e-12
CS_H = 1e-30
S_PRIME = np.array([0.0, 1.0, 1.0, 1.0, 2.0])[None, :, None, None, None]


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


def _case(N, nel, seed=1, rotated=False):
    if rotated:
        xyz, faces, _ = W.rotated_box_mesh(N, nel, seed=seed, mapping=_generic_map)
    else:
        xyz, faces = W.box_mesh(N, nel, mapping=_generic_map)
    U = W.random_smooth_state(xyz, seed=seed, amp=0.1)
    U = U * (1.0 + 0.02 * np.random.default_rng(seed + 1).uniform(-1, 1, U.shape))
    lam = np.random.default_rng(seed + 2).standard_normal(U.shape)
    return xyz, faces, U, lam


def _columns(oc, U, lam, cols, step=None):
    """Complex-step columns j of dL/dU (or of the LSERK step map if step = dt): returns
    (J^T lam)_j and sum_i |J_ij| |lam_i| for each j in cols."""
    Uf = U.reshape(-1)
    Z = Uf.astype(np.complex128)
    ref, scl = np.zeros(len(cols)), np.zeros(len(cols))
    for k, j in enumerate(cols):
        Z[j] += 1j * CS_H
        out = oc.lserk_step(Z.reshape(U.shape), step) if step is not None else oc.rhs(Z.reshape(U.shape))
        col = out.imag.reshape(-1) / CS_H
        ref[k] = col @ lam.reshape(-1)
        scl[k] = np.abs(col) @ np.abs(lam.reshape(-1))
        Z[j] = Uf[j]
    return ref, scl


def _compare(got, U, cols, ref, scl, label):
    nnn = U[0, 0].size
    var = (np.asarray(cols) // nnn) % 5
    err = np.zeros(5)
    for v in range(5):
        m = var == v
        if m.any():
            err[v] = np.abs(got[m] - ref[m]).max() / scl[m].max()
    print(f"PARITY-ADJ {label}: {err}")
    assert (err <= ADJ_TOL).all(), err
    return err


def _gpu(env, N, xyz, faces, **phys):
    dg, orc, torch = env
    return dg.DG(N, xyz, faces, **phys)


def _vjp(env, gpu, U, lam):
    dg, orc, torch = env
    out = gpu.rhs_vjp(torch.from_numpy(U).cuda(), torch.from_numpy(lam).cuda()).cpu().numpy()
    gpu.check()
    return out


COMBOS = [
    dict(equations="euler", vflux="kg", sflux="llf"),
    dict(equations="euler", vflux="pirozzoli", sflux="roe"),
    dict(equations="euler", vflux="kg", sflux="ec"),
    dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=0.02),
    dict(equations="ns", vflux="kg", sflux="llf", mu=0.05),
]


@pytest.mark.parametrize("phys", COMBOS)
@pytest.mark.parametrize("N,nel", [(1, (3, 2, 2)), (2, (2, 2, 2))])
def test_rhs_vjp_every_column(env, phys, N, nel):
    """Every entry of (dL/dU)^T lambda on small curved meshes."""
    dg, orc, torch = env
    xyz, faces, U, lam = _case(N, nel, seed=N + 5)
    oc = orc.Oracle(N, xyz, faces, complex_step=True, **phys)
    cols = np.arange(U.size)
    ref, scl = _columns(oc, U, lam, cols)
    got = _vjp(env, _gpu(env, N, xyz, faces, **phys), U, lam).reshape(-1)
    _compare(got, U, cols, ref, scl, f"dense N={N} {phys}")


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_rhs_vjp_every_degree_rotated(env, N):
    """Sampled entries for every compiled degree on a mesh with re-oriented elements (Navier-Stokes,
    Pirozzoli + Roe)."""
    dg, orc, torch = env
    phys = dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=0.02)
    xyz, faces, U, lam = _case(N, (2, 2, 2) if N > 3 else (3, 2, 2), seed=11 + N, rotated=True)
    oc = orc.Oracle(N, xyz, faces, complex_step=True, **phys)
    cols = np.sort(np.random.default_rng(N).choice(U.size, size=min(U.size, 150), replace=False))
    ref, scl = _columns(oc, U, lam, cols)
    got = _vjp(env, _gpu(env, N, xyz, faces, **phys), U, lam).reshape(-1)[cols]
    _compare(got, U, cols, ref, scl, f"sampled N={N} rotated")


def test_rhs_vjp_tgv_state(env):
    """The adjoint workload's own state (perturbed Taylor-Green vortex at Ma 0.1) at N = 5."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n5_24x24x24_adjoint"].with_(nel=(2, 2, 2))
    xyz, faces = w.mesh()
    U = w.initial_state(xyz)
    lam = np.random.default_rng(3).standard_normal(U.shape)
    oc = orc.Oracle(w.N, xyz, faces, complex_step=True, **w.physics())
    cols = np.sort(np.random.default_rng(4).choice(U.size, size=200, replace=False))
    ref, scl = _columns(oc, U, lam, cols)
    got = _vjp(env, _gpu(env, w.N, xyz, faces, **w.physics()), U, lam).reshape(-1)[cols]
    _compare(got, U, cols, ref, scl, "perturbed TGV N=5")


def test_lserk_step_vjp(env):
    """Reverse of one LSERK(5,4) step against complex-step columns of the oracle's step map."""
    dg, orc, torch = env
    phys = dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=0.02)
    N = 3
    xyz, faces, U, lam = _case(N, (2, 2, 2), seed=21)
    ref_solver = orc.Oracle(N, xyz, faces, **phys)
    oc = orc.Oracle(N, xyz, faces, complex_step=True, **phys)
    dt = ref_solver.max_dt(U, 0.5)
    cols = np.sort(np.random.default_rng(5).choice(U.size, size=80, replace=False))
    ref, scl = _columns(oc, U, lam, cols, step=dt)
    gpu = _gpu(env, N, xyz, faces, **phys)
    Ubar = torch.from_numpy(lam).cuda()
    gpu.lserk_step_vjp(torch.from_numpy(U).cuda(), Ubar, dt)
    got = Ubar.cpu().numpy().reshape(-1)[cols]
    gpu.check()
    _compare(got, U, cols, ref, scl, "LSERK step N=3")


def test_checkpoint_schedules_agree(env):
    """Every checkpoint interval recomputes the same states with the same kernels: identical bits."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n5_24x24x24_adjoint"].with_(nel=(3, 3, 3))
    xyz, faces = w.mesh()
    gpu = _gpu(env, w.N, xyz, faces, **w.physics())
    U0 = torch.from_numpy(w.initial_state(xyz)).cuda()
    dt = gpu.max_dt(U0, w.cfl)
    K = 7
    UK = gpu.lserk_steps(U0.clone(), dt, K)
    seed = gpu.kinetic_energy_grad(UK)
    outs = []
    for interval in (1, 3, 7, 20):
        Ub = seed.clone()
        gpu.lserk_steps_vjp(U0, Ub, dt, K, interval)
        outs.append(Ub)
    # a small memory budget: segment stage states are not kept, each step's stages are recomputed
    gpu.adjoint_memory_limit(1.0)
    for interval in (3, 7):
        Ub = seed.clone()
        gpu.lserk_steps_vjp(U0, Ub, dt, K, interval)
        outs.append(Ub)
    gpu.adjoint_memory_limit(0.0)
    # by hand: store every state, reverse step by step
    states = [U0.clone()]
    for _ in range(K):
        states.append(gpu.lserk_step(states[-1].clone(), dt))
    Ub = seed.clone()
    for k in range(K - 1, -1, -1):
        gpu.lserk_step_vjp(states[k], Ub, dt)
    outs.append(Ub)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    gpu.check()


def test_recorded_run_reverses_to_the_same_bits(env):
    """dg_lserk_steps_record + dg_lserk_steps_vjp_recorded (every stage state kept, or checkpoints
    under a small memory budget) give the same final state as dg_lserk_steps and the same cotangent
    as dg_lserk_steps_vjp; a new recording invalidates the old tape."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n5_24x24x24_adjoint"].with_(nel=(3, 3, 3))
    xyz, faces = w.mesh()
    gpu = _gpu(env, w.N, xyz, faces, **w.physics())
    U0 = torch.from_numpy(w.initial_state(xyz)).cuda()
    dt = gpu.max_dt(U0, w.cfl)
    K = 7
    UK = gpu.lserk_steps(U0.clone(), dt, K)
    seed = gpu.kinetic_energy_grad(UK)
    want = seed.clone()
    gpu.lserk_steps_vjp(U0, want, dt, K, 3)
    for limit in (0.0, 1.0):  # default budget: all stage states; 1 byte: checkpoints every 3 steps
        gpu.adjoint_memory_limit(limit)
        V = U0.clone()
        tape = gpu.lserk_steps_record(V, dt, K, 3)
        assert torch.equal(V, UK)
        Ub = seed.clone()
        gpu.lserk_steps_vjp_recorded(tape, Ub)
        assert torch.equal(Ub, want)
    gpu.adjoint_memory_limit(0.0)
    t1 = gpu.lserk_steps_record(U0.clone(), dt, 2, 2)
    assert gpu.tape_current() == t1
    t2 = gpu.lserk_steps_record(U0.clone(), dt, 2, 2)
    assert gpu.tape_current() == t2 != t1
    with pytest.raises(dg.DGError) as ei:
        gpu.lserk_steps_vjp_recorded(t1, seed.clone())
    assert ei.value.status == -1
    gpu.check()


def test_recording_budget_counts_the_stress_records(env):
    """A Navier-Stokes recording keeps each stage state with the lifting's viscous stress record (6/5 of a
    state): under a budget that holds the states but not their records it keeps checkpoints instead,
    and both recordings reverse to the same bits as the checkpointed sweep from U0."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n5_24x24x24_adjoint"].with_(nel=(4, 4, 4))
    xyz, faces = w.mesh()
    U0 = torch.from_numpy(w.initial_state(xyz)).cuda()
    S = U0.numel() * 8
    T = S // 5 * 6
    K = 4
    full = 5 * K
    ref = _gpu(env, w.N, xyz, faces, **w.physics())
    dt = ref.max_dt(U0, w.cfl)
    seed = ref.kinetic_energy_grad(ref.lserk_steps(U0.clone(), dt, K))
    want = seed.clone()
    ref.lserk_steps_vjp(U0, want, dt, K, 2)
    grown = []
    for limit in ((full + 5) * S + full * T - 1, (full + 5) * S + full * T):
        gpu = _gpu(env, w.N, xyz, faces, **w.physics())
        gpu.adjoint_memory_limit(float(limit))
        U = U0.clone()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        tape = gpu.lserk_steps_record(U, dt, K, 2)
        torch.cuda.synchronize()
        grown.append(free0 - torch.cuda.mem_get_info()[0])
        Ub = seed.clone()
        gpu.lserk_steps_vjp_recorded(tape, Ub)
        assert torch.equal(Ub, want)
        gpu.check()
        gpu.close()
    # one byte short: two checkpoints only (1.1 MB; allocation granularity may round it up to a few
    # MB); at the limit: every stage state and its record (24 MB)
    assert grown[0] < 0.25 * full * (S + T), grown
    assert grown[1] >= 0.9 * full * (S + T), grown


def _ke_complex(U, J, w):
    """Kinetic-energy integral of a complex state (analytic continuation, no conjugation)."""
    wq = np.einsum("k,j,i->kji", w, w, w)[None] * J
    m2 = U[:, 1] * U[:, 1] + U[:, 2] * U[:, 2] + U[:, 3] * U[:, 3]
    return (wq * 0.5 * m2 / U[:, 0]).sum()


def test_kinetic_energy_gradient_through_steps_vs_oracle(env):
    """d KE(U_K) / d U_0 . v: checkpointed GPU adjoint against the oracle's complex-step tangent,
    on the adjoint workload reduced to 3^3 elements and K = 6 steps (checkpoints every 4)."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n5_24x24x24_adjoint"].with_(nel=(3, 3, 3))
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    gpu = _gpu(env, w.N, xyz, faces, **w.physics())
    oc = orc.Oracle(w.N, xyz, faces, complex_step=True, **w.physics())
    ref_solver = orc.Oracle(w.N, xyz, faces, **w.physics())
    dt = ref_solver.max_dt(U0, w.cfl)
    K = 6
    Ud = torch.from_numpy(U0).cuda()
    UK = gpu.lserk_steps(Ud.clone(), dt, K)
    g = gpu.kinetic_energy_grad(UK)
    gpu.lserk_steps_vjp(Ud, g, dt, K, 4)
    g = g.cpu().numpy()
    gpu.check()
    _, wts = orc.lgl(w.N)
    rng = np.random.default_rng(31)
    for r in range(3):
        v = W.tgv_perturbed(xyz, seed=1000 + r, amp=1.0) - W.taylor_green(xyz)
        Z = U0 + 1j * CS_H * v
        for _ in range(K):
            Z = oc.lserk_step(Z, dt)
        want = _ke_complex(Z, ref_solver.J, wts).imag / CS_H
        got = float((g * v).sum())
        rel = abs(got - want) / abs(want)
        print(f"PARITY-ADJ KE gradient . v ({r}): gpu {got:.15e} oracle {want:.15e} rel {rel:.2e}")
        assert rel <= 1e-11, (got, want)
    del rng


def test_kinetic_energy_gradient_full_size_finite_differences(env):
    """The differentiation workload at full size (N = 5, 24^3, K = 50, checkpoints every 10):
    d KE(U_K)/dU_0 . v against central differences of the GPU forward (eps = 1e-6) on seeded
    smooth directions. FD truncation ~ eps^2 and round-off ~ 1e-16 KE / eps bound the agreement."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n5_24x24x24_adjoint"]
    xyz, faces = w.mesh()
    U0n = w.initial_state(xyz)
    gpu = _gpu(env, w.N, xyz, faces, **w.physics())
    U0 = torch.from_numpy(U0n).cuda()
    dt = gpu.max_dt(U0, w.cfl)
    K, interval = w.steps, 10

    def ke_after(U):
        UK = gpu.lserk_steps(U.clone(), dt, K)
        return gpu.invariants(UK, UK)[6]

    UK = gpu.lserk_steps(U0.clone(), dt, K)
    g = gpu.kinetic_energy_grad(UK)
    gpu.lserk_steps_vjp(U0, g, dt, K, interval)
    eps = 1e-6
    for r in range(4):
        v = torch.from_numpy(W.tgv_perturbed(xyz, seed=2000 + r, amp=1.0) - W.taylor_green(xyz)).cuda()
        fd = (ke_after(U0 + eps * v) - ke_after(U0 - eps * v)) / (2 * eps)
        got = float((g * v).sum())
        rel = abs(got - fd) / abs(fd)
        print(f"ADJ-FD full size direction {r}: adjoint {got:.12e} FD {fd:.12e} rel {rel:.2e}")
        assert rel < 1e-6, (got, fd)
    gpu.check()


def test_full_size_vjp_sampled_columns(env):
    """The adjoint at the differentiation workload's full size (N = 5, 24^3, 3.0M DOF): sampled entries
    of (dL/dU)^T lambda against complex-step columns of the oracle. Column j of dL/dU is nonzero only
    on the element of node j and its first and second face neighbours (BR1 reaches across two faces),
    so the oracle evaluates the right-hand side on those elements alone."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n5_24x24x24_adjoint"]
    xyz, faces = w.mesh()
    U = w.initial_state(xyz)
    lam = np.random.default_rng(24).standard_normal(U.shape)
    gpu = _gpu(env, w.N, xyz, faces, **w.physics())
    got = gpu.rhs_vjp(torch.from_numpy(U).cuda(), torch.from_numpy(lam).cuda()).cpu().numpy().reshape(-1)
    gpu.check()
    oc = orc.Oracle(w.N, xyz, faces, complex_step=True, **w.physics())
    nbr = {}
    for eL, fL, eR, fR, o in faces:
        nbr.setdefault(int(eL), set()).add(int(eR))
        nbr.setdefault(int(eR), set()).add(int(eL))
    nnn = (w.N + 1) ** 3
    cols = np.sort(np.random.default_rng(25).choice(U.size, size=12, replace=False))
    ref, scl = np.zeros(len(cols)), np.zeros(len(cols))
    Z = U.astype(np.complex128)
    for k, j in enumerate(cols):
        e = int(j // (5 * nnn))
        mask = {e} | nbr[e]
        for m in list(mask):
            mask |= nbr[m]
        mask = sorted(mask)
        flat = Z.reshape(-1)
        flat[j] += 1j * CS_H
        col = oc.rhs(Z, mask=mask).imag[mask] / CS_H
        flat[j] = U.reshape(-1)[j]
        ref[k] = (col * lam[mask]).sum()
        scl[k] = (np.abs(col) * np.abs(lam[mask])).sum()
    _compare(got[cols], U, cols, ref, scl, "full size 24^3 sampled columns")


def test_conservation_of_the_adjoint_full_size(env):
    """Periodic meshes conserve sum_i J_i w_i Ut_i for every U, so lambda = J w e_v is in the left
    null space of dL/dU: its VJP vanishes (benchmark workload, N = 7, 32^3, curved)."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n7_32x32x32_curved"]
    xyz, faces = w.mesh()
    gpu = _gpu(env, w.N, xyz, faces, **w.physics())
    U = torch.from_numpy(w.initial_state(xyz)).cuda()
    _, J = gpu.metrics()
    xi, wq, _ = dg.basis(w.N)
    wt = torch.from_numpy(np.einsum("k,j,i->kji", wq, wq, wq)).cuda()[None] * J
    sign = torch.from_numpy(np.random.default_rng(7).choice([-1.0, 1.0], size=J.shape)).cuda()
    for v in range(5):
        lam = torch.zeros_like(U)
        lam[:, v] = wt
        ref = torch.zeros_like(U)
        ref[:, v] = wt * sign  # same magnitudes, no cancellation: the size of the terms summed
        z = gpu.rhs_vjp(U, lam).abs().amax().item()
        s = gpu.rhs_vjp(U, ref).abs().amax().item()
        print(f"ADJ conservation v={v}: max|VJP(Jw e_v)| = {z:.3e} (scale {s:.3e}, ratio {z / s:.2e})")
        assert z <= 1e-12 * s
    gpu.check()


def test_scaling_laws_full_size(env):
    """<(dL/dU)^T lam, U> = <lam, L_adv(U)> and <(dL/dU)^T lam, S'U> = <lam, L_adv(U) + S' L(U)> on
    the benchmark workload (exact laws of the discrete operator, see the oracle's complex-step pins);
    measured relative to sum |lam| flux scale."""
    dg, orc, torch = env
    w = W.WORKLOADS["tgv_ns_n7_32x32x32_curved"]
    xyz, faces = w.mesh()
    Un = w.initial_state(xyz)
    gpu = _gpu(env, w.N, xyz, faces, **w.physics())
    adv = _gpu(env, w.N, xyz, faces, **{**w.physics(), "equations": "euler", "mu": 0.0})
    U = torch.from_numpy(Un).cuda()
    lam = torch.from_numpy(np.random.default_rng(8).standard_normal(Un.shape)).cuda()
    mu = gpu.rhs_vjp(U, lam)
    L, La = gpu.rhs(U), adv.rhs(U)
    Sp = torch.from_numpy(S_PRIME).cuda()
    Ja, J = gpu.metrics()
    scale = torch.from_numpy(flux_scale(Un, Ja.cpu().numpy(), J.cpu().numpy(), dg.basis(w.N)[2])).cuda()
    ref_mag = float((lam.abs() * scale[None, :, None, None, None]).sum())
    e1 = abs(float((mu * U).sum() - (lam * La).sum())) / ref_mag
    e2 = abs(float((mu * Sp * U).sum() - (lam * (La + Sp * L)).sum())) / ref_mag
    print(f"ADJ scaling laws full size: density {e1:.2e}, velocity {e2:.2e}")
    assert e1 <= ADJ_TOL and e2 <= ADJ_TOL


def test_autograd_functions(env):
    dg, orc, torch = env
    from paper_2306_12891_gb300 import autograd as AG

    w = W.WORKLOADS["tgv_ns_n5_24x24x24_adjoint"].with_(nel=(2, 2, 2))
    xyz, faces = w.mesh()
    gpu = _gpu(env, w.N, xyz, faces, **w.physics())
    U0 = torch.from_numpy(w.initial_state(xyz)).cuda()
    lam = torch.from_numpy(np.random.default_rng(9).standard_normal(U0.shape)).cuda()
    X = U0.clone().requires_grad_(True)
    (AG.rhs(gpu, X) * lam).sum().backward()
    assert torch.equal(X.grad, gpu.rhs_vjp(U0, lam))
    dt = gpu.max_dt(U0, w.cfl)
    X = U0.clone().requires_grad_(True)
    ke = AG.kinetic_energy(gpu, AG.lserk_steps(gpu, X, dt, 5, 2))
    ke.backward()
    g = gpu.kinetic_energy_grad(gpu.lserk_steps(U0.clone(), dt, 5))
    gpu.lserk_steps_vjp(U0, g, dt, 5, 2)
    assert torch.equal(X.grad, g)
    UK = gpu.lserk_steps(U0.clone(), dt, 5)
    assert abs(ke.item() - gpu.invariants(UK, UK)[6]) == 0.0
    # two recorded forwards before either backward: the first one's tape is gone, so its backward
    # recomputes from U0 (the same bits); the second reverses its own tape
    X1, X2 = U0.clone().requires_grad_(True), U0.clone().requires_grad_(True)
    ke1 = AG.kinetic_energy(gpu, AG.lserk_steps(gpu, X1, dt, 5, 2))
    ke2 = AG.kinetic_energy(gpu, AG.lserk_steps(gpu, X2, dt, 5, 2))
    ke1.backward()
    ke2.backward()
    assert torch.equal(X1.grad, g) and torch.equal(X2.grad, g)


def test_kinetic_energy_gradient_closed_form(env):
    dg, orc, torch = env
    N = 4
    xyz, faces, U, lam = _case(N, (2, 2, 3), seed=40)
    gpu = _gpu(env, N, xyz, faces)
    g = gpu.kinetic_energy_grad(torch.from_numpy(U).cuda()).cpu().numpy()
    _, J = gpu.metrics()
    _, wts = orc.lgl(N)
    Z = U.astype(np.complex128)
    want = np.zeros(U.shape)
    for v in range(5):  # complex step of the numpy KE, one variable at a time (all nodes at once: KE is a sum)
        Zv = Z.copy()
        Zv[:, v] += 1j * CS_H
        wq = np.einsum("k,j,i->kji", wts, wts, wts)[None] * J.cpu().numpy()
        m2 = Zv[:, 1] ** 2 + Zv[:, 2] ** 2 + Zv[:, 3] ** 2
        want[:, v] = (wq * 0.5 * m2 / Zv[:, 0]).imag / CS_H
    assert np.abs(g - want).max() <= 1e-14 * np.abs(want).max()


@pytest.mark.parametrize("kw", [dict(precision="fp32_bulk", equations="ns", vflux="pirozzoli", sflux="roe", mu=0.01),
                                dict(shock_capturing=True, vflux="pirozzoli", sflux="llf"),
                                dict(vflux="ec", sflux="ec"), dict(vflux="central", sflux="llf")])
def test_adjoint_unsupported_forms_are_refused(env, kw):
    dg, orc, torch = env
    xyz, faces, U, lam = _case(2, (2, 2, 2), seed=50)
    gpu = _gpu(env, 2, xyz, faces, **kw)
    Ud, ld = torch.from_numpy(U).cuda(), torch.from_numpy(lam).cuda()
    with pytest.raises(dg.DGError) as ei:
        gpu.rhs_vjp(Ud, ld)
    assert ei.value.status == -6
    with pytest.raises(dg.DGError) as ei:
        gpu.lserk_steps_vjp(Ud, ld.clone(), 1e-4, 3, 2)
    assert ei.value.status == -6
