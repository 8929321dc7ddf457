"""Gradient of the kinetic energy after K LSERK steps through the discrete adjoint, checked
against central finite differences of the forward solver, with timings.

    python -m paper_2306_12891_gb300.adjoint_study [--directions 20] [--eps 1e-6] [--nel 24]
        [--steps 50] [--interval 10] [--out adjoint.json]

Workload: Navier-Stokes (Pirozzoli split form, Roe, BR1) at N = 5 on the curved 24^3 mesh, a
Taylor-Green base state with a seeded perturbation from its lowest four Fourier modes (amplitude
1e-2); objective J(U0) = sum J w rho|u|^2/2 at step K. The gradient comes from a recorded forward
run (dg_lserk_steps_record), dg_kinetic_energy_grad at U_K and dg_lserk_steps_vjp_recorded; the
same gradient from U0 alone (checkpoints every `interval` steps, dg_lserk_steps_vjp) is timed too
and must agree bit for bit.
Each of the seeded smooth directions v is checked against (J(U0 + eps v) - J(U0 - eps v)) / (2 eps)
computed with dg_lserk_steps.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from .workloads import WORKLOADS, taylor_green, tgv_perturbed


def run(steps: int = 50, interval: int = 10, directions: int = 20, eps: float = 1e-6, nel: int | None = None,
        workload: str = "tgv_ns_n5_24x24x24_adjoint") -> dict:
    import torch

    from . import build, dg

    build.build()
    w = WORKLOADS[workload]
    if nel:
        w = w.with_(nel=(nel,) * 3)
    xyz, faces = w.mesh()
    U0 = torch.from_numpy(w.initial_state(xyz)).cuda()
    free0 = torch.cuda.mem_get_info()[0]
    s = dg.DG(w.N, xyz, faces, **w.physics())
    dt = s.max_dt(U0, w.cfl)

    def objective(U):
        UK = s.lserk_steps(U.clone(), dt, steps)
        return s.invariants(UK, UK)[6]

    def gradient():  # recorded forward run, then the reverse sweep (no recomputation when HBM holds the tape)
        UK = U0.clone()
        tape = s.lserk_steps_record(UK, dt, steps, interval)
        g = s.kinetic_energy_grad(UK)
        s.lserk_steps_vjp_recorded(tape, g)
        return g

    def gradient_from_u0():  # checkpoints every `interval` steps, each segment recomputed once
        UK = s.lserk_steps(U0.clone(), dt, steps)
        g = s.kinetic_energy_grad(UK)
        s.lserk_steps_vjp(U0, g, dt, steps, interval)
        return g

    gradient()  # warm-up (allocates the tape and work buffers)
    gradient_from_u0()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record()
    g_ckpt = gradient_from_u0()
    c1.record()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    J0 = objective(U0)
    e[1].record()
    s.timing_enable(True)
    s.timing_get()
    e[2].record()
    g = gradient()
    e[3].record()
    torch.cuda.synchronize()
    kt = s.timing_get()
    s.timing_enable(False)
    fwd_ms, grad_ms = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    ckpt_ms = c0.elapsed_time(c1)
    assert torch.equal(g, g_ckpt), "recorded and checkpointed gradients differ"
    # one plain VJP of the right-hand side (kernel throughput)
    lam = torch.randn_like(U0)
    s.rhs_vjp(U0, lam)
    reps = 5
    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    v0.record()
    for _ in range(reps):
        s.rhs_vjp(U0, lam)
    v1.record()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Ut = torch.empty_like(U0)
    r0.record()
    for _ in range(reps):
        s.rhs(U0, Ut)
    r1.record()
    torch.cuda.synchronize()
    vjp_ms, rhs_ms = v0.elapsed_time(v1) / reps, r0.elapsed_time(r1) / reps
    rows = []
    base = taylor_green(xyz)
    for r in range(directions):
        v = torch.from_numpy(tgv_perturbed(xyz, seed=5000 + r, amp=1.0) - base).cuda()
        fd = (objective(U0 + eps * v) - objective(U0 - eps * v)) / (2 * eps)
        ad = float((g * v).sum())
        rows.append({"direction": r, "adjoint": ad, "fd": fd, "rel": abs(ad - fd) / abs(fd)})
    s.check()
    rels = [x["rel"] for x in rows]
    return {"workload": workload if not nel else f"{workload} reduced to {nel}^3", "N": w.N,
            "elements": w.n_elems, "dofs": w.dofs, "steps": steps, "interval": interval, "dt": dt,
            "objective": J0, "eps": eps, "forward_ms": fwd_ms, "gradient_ms": grad_ms,
            "gradient_over_forward": grad_ms / fwd_ms, "gradient_from_u0_checkpointed_ms": ckpt_ms,
            "rhs_ms": rhs_ms, "rhs_vjp_ms": vjp_ms,
            "vjp_over_rhs": vjp_ms / rhs_ms,
            "library_memory_gb": (free0 - free1) / 1e9,
            "gradient_kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in kt.items() if v[1]},
            "fd_rel_max": max(rels), "fd_rel_median": float(np.median(rels)), "directions": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--interval", type=int, default=10)
    ap.add_argument("--directions", type=int, default=20)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--nel", type=int, default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    t0 = time.perf_counter()
    res = run(a.steps, a.interval, a.directions, a.eps, a.nel)
    res["wall_s"] = time.perf_counter() - t0
    text = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    print(json.dumps({k: v for k, v in res.items() if k != "directions"}))


if __name__ == "__main__":
    main()
