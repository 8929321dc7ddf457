"""Long-run accuracy against the FP64 oracle (the precision form's error after K steps).

The N = 7 curved Taylor-Green workload of the precision study (Navier-Stokes, Pirozzoli, Roe, BR1,
Re 1600, Ma 0.1), reduced to 4^3 elements so that the oracle can follow it: 500 LSERK(5,4) steps
(t = 1.5) with the GPU in FP64 and in the FP32-bulk form, against the oracle. Two oracle runs go in
spawned host processes while the GPU works: from the initial state, and from the initial state and
mesh points moved by one ulp (seeded), whose distance from the first is the conditioning of the
500-step map.

Stated and asserted, every 100 steps, per conservative variable (momentum components relative to
the largest momentum component, so that rho w, zero at t = 0, is not divided by ~0):
- FP64: Linf <= ULP_FACTOR times the oracle's one-ulp spread of the same step;
- FP32-bulk: Linf <= 1e-5 and L2 <= 2e-6 relative; the kinetic-energy dissipation rate
  -d/dt sum J w rho|u|^2/2 within 1e-4 relative of the oracle's.
The printed LONGRUN lines are the figures of the precision summary.
"""
import multiprocessing

import numpy as np
import pytest

from helpers import ULP_FACTOR, oracle_trajectory

pytestmark = pytest.mark.gpu
NAME = "tgv_ns_n7_48x48x48_curved_fp32"
NEL = (4, 4, 4)
STEPS, EVERY = 500, 100
P0_TGV = 1.0 / (1.4 * 0.1 ** 2)


def _rel_errors(U, Uref, wq):
    """Linf and L2 (quadrature-weighted) of U - Uref per variable, relative to max |Uref_v| (momentum:
    to the largest momentum component)."""
    d = (U - Uref).reshape(Uref.shape[0], 5, -1)
    ref = np.abs(Uref).reshape(Uref.shape[0], 5, -1).max(axis=(0, 2))
    ref[1:4] = ref[1:4].max()
    w = wq.reshape(wq.shape[0], -1)
    linf = np.abs(d).max(axis=(0, 2)) / ref
    l2 = np.sqrt((w[:, None, :] * d * d).sum(axis=(0, 2)) / w.sum()) / ref
    return linf, l2


def test_long_run_fp64_and_fp32_bulk_against_oracle(oracle_mod):
    import torch

    from paper_2306_12891_gb300 import build, dg
    from paper_2306_12891_gb300 import workloads as W

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    w = W.WORKLOADS[NAME].with_(nel=NEL)
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    dt = oracle_mod.Oracle(w.N, xyz, faces, **w.physics()).max_dt(U0, w.cfl)
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(2) as pool:
        runs = pool.map_async(oracle_trajectory, [(NAME, NEL, STEPS, EVERY, dt, None),
                                                  (NAME, NEL, STEPS, EVERY, dt, 20230624)])
        gpu = {}
        for form, extra in (("fp64", {}), ("fp32_bulk", dict(precision="fp32_bulk", p_ref=P0_TGV))):
            s = dg.DG(w.N, xyz, faces, **extra, **w.physics())
            U = torch.from_numpy(U0).cuda()
            states, invs = [U0.copy()], [s.invariants(U, s.rhs(U))]
            for _ in range(STEPS // EVERY):
                s.lserk_steps(U, dt, EVERY)
                states.append(U.cpu().numpy())
                invs.append(s.invariants(U, s.rhs(U)))
            s.check()
            gpu[form] = (states, invs)
        (ref_states, ref_invs), (pert_states, _) = runs.get(timeout=1800)
    _, wts = oracle_mod.lgl(w.N)
    _, J = dg.DG(w.N, xyz, faces, **w.physics()).metrics()
    wq = np.einsum("k,j,i->kji", wts, wts, wts)[None] * J.cpu().numpy()
    for j in range(1, len(ref_states)):
        k = j * EVERY
        Ur = ref_states[j]
        spread, _ = _rel_errors(pert_states[j], Ur, wq)
        e64, l64 = _rel_errors(gpu["fp64"][0][j], Ur, wq)
        e32, l32 = _rel_errors(gpu["fp32_bulk"][0][j], Ur, wq)
        eps_ref = -ref_invs[j][7]
        d_eps = abs(-gpu["fp32_bulk"][1][j][7] - eps_ref) / abs(eps_ref)
        d_eps64 = abs(-gpu["fp64"][1][j][7] - eps_ref) / abs(eps_ref)
        print(f"LONGRUN step {k} t={k * dt:.3f}: oracle 1-ulp spread Linf {spread}")
        print(f"LONGRUN step {k} FP64: Linf {e64} L2 {l64}; KE-dissipation rate rel diff {d_eps64:.2e}")
        print(f"LONGRUN step {k} FP32-bulk: Linf {e32} L2 {l32}; KE-dissipation rate {eps_ref:.6e}, "
              f"rel diff {d_eps:.2e}")
        assert (e64 <= ULP_FACTOR * spread).all(), (k, e64, spread)
        assert (e32 <= 1e-5).all() and (l32 <= 2e-6).all(), (k, e32, l32)
        assert d_eps <= 1e-4, (k, d_eps)
    assert np.abs(ref_states[-1] - U0).max() > 1e-2  # the flow has moved
