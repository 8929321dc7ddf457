"""Long-run accuracy of the FP32-bulk form against the FP64 form.

Both forms advance the same workload from the same initial state with the same time step; every
`every` steps the FP32-bulk state is compared with the FP64 state (L2 and Linf per conservative
variable, relative to the FP64 state's magnitude) and the volume-averaged kinetic energy and its
dissipation rate -dKE/dt (from the right-hand side through dg_invariants) are recorded for both.

    python -m paper_2306_12891_gb300.precision_study [--steps 1000] [--every 100] [--nel 48]
        [--out precision.json]

The FP64 path stands in for the FP64 oracle at this size: it matches the oracle to rounding on
the same physics, right-hand side by right-hand side (tests/test_gpu_parity.py) and over 500 steps of
the same workload on 4^3 elements (tests/test_gpu_long_run.py, within the oracle's own one-ulp
spread), while the oracle cannot run 1000 steps of 56.6M DOF.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from .workloads import WORKLOADS


def run(workload: str = "tgv_ns_n7_48x48x48_curved_fp32", steps: int = 1000, every: int = 100,
        nel: int | None = None, p_ref: float | None = None) -> dict:
    import torch

    from . import build, dg

    build.build()
    w = WORKLOADS[workload]
    if nel:
        w = w.with_(nel=(nel,) * 3)
    if p_ref is None:
        p_ref = 1.0 / (w.gamma * 0.1 ** 2) if w.initial == "tgv" else 0.0
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    phys = w.physics()
    s64 = dg.DG(w.N, xyz, faces, precision="fp64", **phys)
    s32 = dg.DG(w.N, xyz, faces, precision="fp32_bulk", p_ref=p_ref, **phys)
    U64 = torch.from_numpy(U0).cuda()
    U32 = U64.clone()
    dt = s64.max_dt(U64, w.cfl)
    _, J = s64.metrics()
    xi, wq, _ = dg.basis(w.N)
    vol = float(torch.einsum("ekji,k,j,i->", J, *(torch.from_numpy(wq).cuda(),) * 3))
    rows = []
    t64 = t32 = 0.0

    def record(k):
        d = (U32 - U64).reshape(U64.shape[0], 5, -1)
        ref = U64.reshape(U64.shape[0], 5, -1)
        scale = ref.abs().amax(dim=(0, 2))
        linf = (d.abs().amax(dim=(0, 2)) / scale).tolist()
        l2 = (torch.sqrt((d ** 2).mean(dim=(0, 2))) / scale).tolist()
        inv64 = s64.invariants(U64, s64.rhs(U64))
        inv32 = s32.invariants(U32, s32.rhs(U32))
        ke64, ke32 = inv64[6] / vol, inv32[6] / vol
        eps64, eps32 = -inv64[7] / vol, -inv32[7] / vol
        rows.append({"step": k, "t": k * dt, "linf_rel": linf, "l2_rel": l2, "ke_fp64": ke64, "ke_fp32": ke32,
                     "dissipation_fp64": eps64, "dissipation_fp32": eps32,
                     "dissipation_drift_rel": (eps32 - eps64) / abs(eps64) if eps64 else None})

    record(0)
    k = 0
    while k < steps:
        m = min(every, steps - k)
        torch.cuda.synchronize()
        a = time.perf_counter()
        s64.lserk_steps(U64, dt, m, t=k * dt)
        torch.cuda.synchronize()
        b = time.perf_counter()
        s32.lserk_steps(U32, dt, m, t=k * dt)
        torch.cuda.synchronize()
        t64 += b - a
        t32 += time.perf_counter() - b
        k += m
        record(k)
    s64.check()
    s32.check()
    dof_stages = w.dofs * 5 * steps
    return {"workload": workload if not nel else f"{workload} reduced to {nel}^3", "steps": steps, "dt": dt,
            "p_ref": p_ref, "fp64_dof_stage_per_s": dof_stages / t64, "fp32_dof_stage_per_s": dof_stages / t32,
            "speedup": t64 / t32, "records": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="tgv_ns_n7_48x48x48_curved_fp32", choices=sorted(WORKLOADS))
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--nel", type=int, default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = run(a.workload, a.steps, a.every, a.nel)
    text = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    last = res["records"][-1]
    print(json.dumps({"steps": res["steps"], "speedup": res["speedup"], "linf_rel": last["linf_rel"],
                      "l2_rel": last["l2_rel"], "dissipation_drift_rel": last["dissipation_drift_rel"]}))


if __name__ == "__main__":
    main()
