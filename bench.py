"""Benchmark of the DGSEM hot path on GB300: LSERK(5,4) steps of the N=7 curved Taylor-Green
Navier-Stokes workload (Pirozzoli split form, Roe, BR1; 32^3 elements, 16.8M DOF), FP64.

One step = one LSERK(5,4) time step = five right-hand-side evaluations plus the stage updates
over the whole mesh. Reported metric: DOF-stage updates per second (= 1/PID per GPU, the
paper's performance index, Sec. 2 Eq. (1), with #cores := #GPUs), plus the PID itself.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 (launched by torch.distributed.run) every rank runs an independent replica of the
workload (the solver keeps each mesh on one GPU); value = total DOF-stage updates / max time.
`--impl reference` times the FP64 CPU oracle instead, one process per host core, each on a bounded
sub-box of the same workload. The default line also carries the FP32-bulk form, the adjoint, the
wall model, the shock-capturing workload's 200 steps, the other named workloads and the oracle's
host rate (each block can be switched off for profiling runs).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2306_12891_gb300.workloads import WORKLOADS  # noqa: E402

WORKLOAD = "tgv_ns_n7_32x32x32_curved"
METRIC = "DOF-stage updates/s (1/PID), N=7 split-form Navier-Stokes, FP64"
UNIT = "DOF-stage/s"
STAGES = 5
P0_TGV = 1.0 / (1.4 * 0.1 ** 2)  # background pressure of the Ma 0.1 Taylor-Green vortex
# DRAM bytes per element of one volume-kernel launch (dram__bytes_read.sum + dram__bytes_write.sum),
# from an ncu capture of the current kernel on the 24^3 case (a later LSERK stage: 2060.27 MB read,
# 545.17 MB written for 13824 elements), scaled to a launch by the element count (the kernel's
# traffic is per element). None once the kernel has changed since that capture.
VOLUME_DRAM_BYTES_PER_ELEMENT = (2060.267008e6 + 545.168640e6) / 24 ** 3
# DRAM bytes (read + write) of one FP32-bulk volume launch (pair-symmetric line kernel, stage factor) per
# element, from one ncu capture at the full 32^3 size of the second stage of a step (3492.2 MB read,
# 1625.3 MB written for 32768 elements)
VOLUME_F32_DRAM_BYTES_PER_ELEMENT = (3492.2e6 + 1625.3e6) / 32 ** 3


# how the FP64 flop counts below are made: from the statements of each kernel as built (an FMA two
# flops, a division or reciprocal square root one; the even-odd line sweeps count what they execute),
# which ncu's executed DFMA/DADD/DMUL counts match to a few per cent
FLOPS_BASIS = "kernel statements as built (FMA = 2, div/rsqrt = 1, even-odd sweeps as executed)"


def scaled_traffic(bytes_per_element, n_elems: int, applies: bool = True):
    """A captured per-element DRAM count scaled to a launch by the element count; None when there is no
    capture of the current kernel (or it does not apply to this configuration)."""
    return bytes_per_element * n_elems if (bytes_per_element is not None and applies) else None


def viscous_sweep_flops_per_node(N: int) -> float:
    """Flops per node, direction and quantity of a line sweep with the zero-diagonal D (the viscous
    divergence): with the even-odd halves of the centro-antisymmetric LGL D (even n = N + 1) a line
    of n nodes takes n sums and differences, n^2 / 2 FMA and 2n combinations: n^2 + 3n flops with the
    accumulation; otherwise N FMA and the accumulation: 2N + 1 per node."""
    n = N + 1
    return (n + 3.0) if n % 2 == 0 else (2.0 * N + 1.0)


def volume_kernel_flops_per_element(N: int, navier_stokes: bool) -> float:
    """Algorithmic FP64 flops of one volume-kernel launch (a later LSERK stage) per element (FMA = 2
    flops, a division or reciprocal square root 1), counted from the formulas the kernel evaluates:
      pair flux (Pirozzoli, plain sums, 1/2 factors folded into D):
        6 sums + V (mul + 2 FMA = 5) + F_rho (add + mul = 2) + p-sum 1 + momentum 3 x (mul + FMA) = 9
        + energy (add + mul = 2) + accumulation into both nodes 10 FMA = 20        -> 45 per pair,
        3 n^2 n(n-1)/2 pairs per element;
      per node: primitives 15; direction sum 10; stage factor dt (-1/J) 1 and per variable the
        increment, the register and the state (mul + 2 FMA) 25; Navier-Stokes: the viscous
        divergence 12 viscous_sweep_flops_per_node(N) and 4 subtractions;
      per face point (6 n^2 per element): surface terms 10; Navier-Stokes: the neighbour's viscous
        trace 8."""
    n = N + 1
    pairs = 3 * n * n * n * (n - 1) // 2
    per_node = 15 + 10 + 26 + ((12 * viscous_sweep_flops_per_node(N) + 4) if navier_stokes else 0)
    per_face_pt = 10 + (8 if navier_stokes else 0)
    return 45.0 * pairs + per_node * n ** 3 + per_face_pt * 6 * n * n


def lift_uses_lines(N: int) -> bool:
    """Whether the FP64 lifting forms the reference derivatives along lines (k_lift_lines)."""
    return N == 7


def lift_kernel_flops_per_element(N: int) -> float:
    """Algorithmic FP64 flops of one BR1 lifting launch per element (FMA = 2, a division 1), from the
    kernel's statements: primitives and T 15 per node; per direction and lifted variable the
    reference derivative -- along lines with the even-odd halves of D (N = 7: n^2 + 2n per line and
    quantity, n + 2 per node) or node-wise (n FMA, 2n) -- and the metric contraction 3 FMA; 1/J into
    mu and kappa 2; the viscous flux 40; the contravariant flux 12 x (mul + 2 FMA) = 60; the surface
    terms, added to the reference derivative before its contraction, 4 FMA = 8 per (node, face) pair,
    6 n^2 pairs per element."""
    n = N + 1
    sweep = (n + 2.0) if lift_uses_lines(N) else 2.0 * n
    return (15 + 12 * (sweep + 6) + 2 + 40 + 60) * n ** 3 + 8 * 6 * n * n


def face_kernel_flops_per_point() -> float:
    """Algorithmic FP64 flops per face point of the face kernel for Roe + Navier-Stokes (FMA = 2, a
    division or reciprocal square root 1), from its statements: two Euler fluxes 2 x 28; Roe's
    averages from one reciprocal square root per side, the sound speed, wave strengths and the
    dissipation with the two acoustic waves collected 115; the two outward slot values 10; the BR1
    jumps of (u, v, w, T) 11."""
    return 56.0 + 115.0 + 10.0 + 11.0


def adjoint_volume_flops_per_element(N: int, navier_stokes: bool) -> float:
    """Algorithmic FP64 flops of one adjoint-volume launch per element (FMA = 2 flops), counted from
    the statements of the kernel:
      pair (KG/Pirozzoli transposed): 9 sums, 5 pair cotangents t_v = l_i + (D_mi/D_im) l_m (FMA,
        10), V 5, F0 scaled by D_im/8 2, d(c.F)/dF0 9, gV 1, gP 6, the six primitive cotangents 12,
        accumulation into both nodes 12 -> 65 per pair, 3 n^2 n(n-1)/2 pairs per element;
      per node: primitives and l = -lambda/J 20, direction sum 12, chain to U 25, reverse LSERK 20,
        Navier-Stokes: T chain 6 and the neighbours' face shares 4 per face point;
      per face point: 5 additions of the face slots."""
    n = N + 1
    pairs = 3 * n * n * n * (n - 1) // 2
    per_node = 20 + 12 + 25 + 20 + (6 if navier_stokes else 0)
    per_face_pt = 5 + (4 if navier_stokes else 0)
    return 65.0 * pairs + per_node * n ** 3 + per_face_pt * 6 * n * n


def adjoint_visc_flops_per_element(N: int) -> float:
    """Algorithmic FP64 flops of one adjoint-viscous launch per element (FMA = 2 flops, a division 1),
    counted from the statements of the kernel (BR1 lifting, viscous flux and viscous divergence
    transposed, at the viscous stress the forward lifting recorded):
      per node: (u, v, w) and l = -lambda/J 9; per direction and lifted variable the transposed
        sweep of l, N FMA: 24 N; mu/J, kappa/J 2; Z = Ja^T zeta 60; omega and Y 33; trace 2;
        Gamma 26; H = Ja Gamma 60; the transposed D sweeps of H and their sums 12 (2n + 1); omega
        added 3 -> 48 n + 183 per node;
      per (node, face) pair on the element surface (6 n^2 per element): the neighbour's share of the
        transposed divergence 14, the face slot 9 -> 23."""
    n = N + 1
    return (48.0 * n + 183.0) * n ** 3 + 23.0 * 6 * n * n


def fv_subcell_flops_per_element(N: int, riemann_flops: float) -> float:
    """Algorithmic FP64 flops of the FV subcell operator of one element (the blend's extra work on a
    troubled element), from the statements of the kernel, per line of n subcells: the reconstructed
    interface states (minmod slopes of 5 primitives in the n - 2 interior subcells 51, first-order
    outer subcells 22), and at each of the N interior interfaces the telescoped metric 3 (2n + 2),
    the unit normal 10, two conservative states 20, the Riemann flux `riemann_flops`, the area factor
    5 and the subcell update 10 (plus 10 for the last subcell); 3 n^2 lines per element. The blend
    itself adds 15 per node."""
    n = N + 1
    per_line = 51.0 * (n - 2) + 22.0 * 2 + N * (3 * (2 * n + 2) + 10 + 20 + riemann_flops + 5 + 10) + 10
    return 3 * n * n * per_line + 15.0 * n ** 3


LLF_FLOPS = 82.0  # two Euler fluxes 2 x 26, two sound speeds 6, the wave-speed bound 4, the flux 20


def fp32_kernel_bytes_per_launch(N: int, n_elems: int) -> dict:
    """Algorithmic DRAM bytes of one launch of each FP32-bulk kernel of the Navier-Stokes step:
      volume: volume_kernel_bytes_per_element(N, True, 4) per element;
      (the once-per-call stage-factor and shadow refreshes are counted under "other" as the shadow's)
      lift: the FP32 shadow state 20, metric terms 36 and 1/J 4 per node in, the BR1 face jumps
        (6 faces x 4 x n^2 floats per element) in, the contravariant viscous flux 48 per node out;
      face: per face point (3 n^2 per element) both elements' shadow states 40 and the normal and area
        16 in, both outward flux slots 40 and BR1 jumps 32 out, the face record 20 per face;
      other (the shadow refresh k_shadow): U 40 in, the FP32 shadow 20 out per node."""
    n = N + 1
    nodes = n ** 3 * n_elems
    return {"volume": volume_kernel_bytes_per_element(N, True, 4) * n_elems,
            "lift": nodes * (20 + 36 + 4 + 48) + 6 * 4 * n * n * 4 * n_elems,
            "face": 3 * n * n * n_elems * (40 + 16 + 40 + 32) + 3 * n_elems * 20,
            "other": nodes * 60.0}


def fp32_step_roofline(N: int, n_elems: int, kt: dict, region_ms: float) -> dict:
    """Whole-step HBM roofline of the FP32-bulk form: every kernel's algorithmic bytes (times its
    launches in the timed region) against the timed region, and per kernel against its own time."""
    per = fp32_kernel_bytes_per_launch(N, n_elems)
    total, kernels = 0.0, {}
    for k, (ms, cnt) in kt.items():
        if not cnt or k not in per:
            continue
        b = per[k] * cnt
        total += b
        gbs = b / (ms * 1e-3) / 1e9
        kernels[k] = {"bytes_per_launch": per[k], "ms_per_launch": ms / cnt, "achieved": gbs, "frac": gbs / HBM_GBS}
    gbs = total / (region_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": HBM_GBS, "unit": "GB/s", "frac": gbs / HBM_GBS,
            "bytes_per_step": total / max(1, kt.get("volume", (0, 1))[1] // STAGES), "kernels": kernels,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}


def volume_kernel_bytes_per_element(N: int, navier_stokes: bool, real_bytes: int) -> float:
    """Algorithmic DRAM bytes of one volume-kernel launch per element in an LSERK stage after the
    first: U and the LSERK register g read and written (FP64), the metric terms Ja (real type), the
    per-node factor of the Jacobian (FP64 1/J; in FP32-bulk the float stage factor dt (-1/J)), the
    element's six face slots of outward flux (real type) and, for Navier-Stokes, the contravariant
    viscous flux (12 per node) and the neighbours' normal viscous flux at the faces (4 per face point).
    The FP32-bulk kernel also reads and writes the FP32 shadow of U (5 floats per node each way)."""
    n = N + 1
    nodes, fpts = n ** 3, 6 * n * n
    b = nodes * (4 * 5 * 8 + (8 if real_bytes == 8 else 4)) + nodes * 9 * real_bytes + fpts * 5 * real_bytes
    if navier_stokes:
        b += nodes * 12 * real_bytes + fpts * 4 * real_bytes
    if real_bytes == 4:
        b += nodes * 5 * 4 * 2
    return float(b)


def _measured_hbm_gbs() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # the profiling recipe's fallback


HBM_GBS = _measured_hbm_gbs()


def dist_setup(n_gpus: int):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as td

        torch.cuda.set_device(local)
        td.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as td

        td.barrier()


def max_over_ranks(world, x: float) -> float:
    """Largest x over the ranks (the timed region ends when the slowest replica ends)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as td

    dev = "cuda" if td.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def aggregate(world: int, units_per_rank: float, seconds_per_rank: float) -> float:
    """Whole-job throughput of `world` independent replicas: all ranks' units / the slowest rank's time."""
    return world * units_per_rank / max_over_ranks(world, seconds_per_rank)


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(device_index), "-lms", "200"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


THROTTLE_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def throttled(clk: dict) -> bool:
    """Clock record of a timed region that must not be reported: a hardware or thermal slowdown, or
    SM clocks held well below their maximum with no reason given (a leftover clock lock)."""
    if any(r in THROTTLE_REASONS for r in clk.get("reasons", [])):
        return True
    sm, smax = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    return bool(sm and smax and sm < 0.8 * smax and not clk.get("reasons"))


def _oracle_worker(kind: str, nel: int, seconds: float, warmup: int, steps: int, barrier, queue) -> None:
    """One host process of the oracle timing: the same physics on an nel^3-element sub-box of the
    workload; after a common start (barrier), right-hand sides for `seconds` (kind "rhs") or `steps`
    LSERK(5,4) steps after `warmup` untimed ones (kind "steps"). Puts (DOF-stages, seconds)."""
    import oracle

    w = WORKLOADS[WORKLOAD].with_(nel=(nel,) * 3)
    xyz, faces = w.mesh()
    U = w.initial_state(xyz)
    ref = oracle.Oracle(w.N, xyz, faces, **w.physics())
    dt = ref.max_dt(U, w.cfl)
    if kind == "rhs":
        ref.rhs(U)
    for _ in range(warmup if kind == "steps" else 0):
        U = ref.lserk_step(U, dt)
    barrier.wait()
    t0 = time.perf_counter()
    stages = 0
    if kind == "rhs":
        while time.perf_counter() - t0 < seconds:
            ref.rhs(U)
            stages += 1
    else:
        for _ in range(steps):
            U = ref.lserk_step(U, dt)
            stages += STAGES
    queue.put((w.dofs * stages, time.perf_counter() - t0))


def oracle_parallel(kind: str, nel: int, procs: int, seconds: float = 0.0, warmup: int = 0, steps: int = 0):
    """The oracle, as it stands, in `procs` host processes at once (spawned, so no GPU context is
    inherited), each on its own sub-box; returns the total DOF-stages per second over the slowest
    process's time and the per-process results."""
    import multiprocessing

    import oracle

    oracle.build()
    ctx = multiprocessing.get_context("spawn")
    barrier, queue = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(kind, nel, seconds, warmup, steps, barrier, queue))
          for _ in range(procs)]
    for p in ps:
        p.start()
    res = [queue.get(timeout=600) for _ in ps]
    for p in ps:
        p.join()
    return sum(r[0] for r in res) / max(max(r[1] for r in res), 1e-9), res


def host_cpu() -> dict:
    """Host core count and CPU model name (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model}


def cpu_baseline(seconds: float = 12.0) -> dict:
    """The FP64 oracle, as it stands, on the host cores: right-hand sides of the same physics on a
    6^3-element sub-box of the workload (110,592 DOF) per process, for ~`seconds`; one process per
    host core at once, and the single-process rate beside it."""
    cpu = host_cpu()
    procs = cpu["nproc"] or 1
    value, res = oracle_parallel("rhs", 6, procs, seconds=seconds)
    single, _ = oracle_parallel("rhs", 6, 1, seconds=seconds / 2)
    stages = sum(r[0] for r in res) // WORKLOADS[WORKLOAD].with_(nel=(6, 6, 6)).dofs
    return {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{stages} right-hand sides of the same physics on 6x6x6-element sub-boxes (110592 DOF each), "
                      f"FP64 C oracle in {procs} processes at once, {max(r[1] for r in res):.1f} s",
            "single_core_value": single, "host": cpu}


def run_reference(args):
    """Reference arm: the oracle timed on the host cores, on bounded samples of the workload."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOADS[WORKLOAD].with_(nel=(3, 3, 3))
    cpu = host_cpu()
    procs = cpu["nproc"] or 1
    value, res = oracle_parallel("steps", 3, procs, warmup=args.warmup, steps=args.steps)
    el = max(r[1] for r in res)
    sample = (f"each step: one LSERK(5,4) step of the same physics on a 3x3x3-element sub-box ({w.dofs} DOF) "
              f"in each of {procs} processes at once (FP64 C oracle, one process per host core)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_elements": w.n_elems, "N": w.N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample,
                             "host": cpu},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def step_roofline(N: int, dof_stage_per_s: float, peak_fp64: float) -> dict:
    """Whole-step FP64 roofline of the Navier-Stokes step (Pirozzoli, Roe, BR1, periodic box): the
    algorithmic flops of the volume, lifting and face kernels per DOF and stage against the measured
    FP64 peak; PID_roof = flops / peak and frac = PID_roof / PID_measured."""
    n = N + 1
    nodes = n ** 3
    flops = (volume_kernel_flops_per_element(N, True) + lift_kernel_flops_per_element(N) +
             face_kernel_flops_per_point() * 3 * n * n) / nodes
    pid = 1.0 / dof_stage_per_s
    return {"bound": "alu", "flops_per_dof_stage": flops, "pid_roof_s": flops / peak_fp64, "pid_s": pid,
            "frac": flops / peak_fp64 / pid, "peak": peak_fp64 / 1e12, "unit": "TFLOP/s",
            "peak_source": "measured FP64 FMA probe (dg_probe_fma), live", "flops_basis": FLOPS_BASIS}


ADJOINT_WORKLOAD = "tgv_ns_n5_24x24x24_adjoint"


def run_adjoint(stream, peak_fp64: float, interval: int = 10) -> dict:
    """The differentiation form: gradient of the kinetic energy after K = 50 LSERK steps with
    respect to the initial state (N = 5, 24^3, Navier-Stokes): a recorded forward run
    (dg_lserk_steps_record keeps every stage state when HBM allows), dg_kinetic_energy_grad and the
    reverse sweep; also the same gradient from U0 alone with checkpoints every `interval` steps
    (dg_lserk_steps_vjp). Timed with CUDA events against the plain forward run."""
    import torch

    from paper_2306_12891_gb300 import dg

    w = WORKLOADS[ADJOINT_WORKLOAD]
    xyz, faces = w.mesh()
    s = dg.DG(w.N, xyz, faces, stream=stream, **w.physics())
    U0 = torch.from_numpy(w.initial_state(xyz)).cuda()
    dt = s.max_dt(U0, w.cfl)
    K = w.steps

    def gradient():  # recorded forward run (every stage state kept in HBM), then the reverse sweep
        UK = U0.clone()
        tape = s.lserk_steps_record(UK, dt, K, interval)
        g = s.kinetic_energy_grad(UK)
        s.lserk_steps_vjp_recorded(tape, g)
        return g

    def gradient_from_u0():  # the same gradient from U0 alone: checkpoints, each segment recomputed once
        UK = s.lserk_steps(U0.clone(), dt, K)
        g = s.kinetic_energy_grad(UK)
        s.lserk_steps_vjp(U0, g, dt, K, interval)
        return g

    gradient()  # warm-up: allocates the tape and work buffers
    gradient_from_u0()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    s.lserk_steps(U0.clone(), dt, K)
    ev[1].record(stream)
    s.timing_enable(True)
    s.timing_get()
    ev[2].record(stream)
    gradient()
    ev[3].record(stream)
    torch.cuda.synchronize()
    kt = s.timing_get()
    s.timing_enable(False)
    ev[4].record(stream)
    gradient_from_u0()
    ev[5].record(stream)
    torch.cuda.synchronize()
    s.check()
    fwd_ms, grad_ms = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    grad_ckpt_ms = ev[4].elapsed_time(ev[5])
    adj_ms, adj_n = kt.get("adj_volume", (0.0, 0))
    flops = adjoint_volume_flops_per_element(w.N, True) * w.n_elems
    achieved = flops / (adj_ms / adj_n * 1e-3) if adj_n else 0.0
    vis_ms, vis_n = kt.get("adj_visc", (0.0, 0))
    vflops = adjoint_visc_flops_per_element(w.N) * w.n_elems
    vachieved = vflops / (vis_ms / vis_n * 1e-3) if vis_n else 0.0
    total = sum(v[0] for v in kt.values())
    return {"workload": ADJOINT_WORKLOAD, "N": w.N, "elements": w.n_elems, "dofs": w.dofs, "steps": K,
            "checkpoint_interval": interval, "objective": "kinetic energy at step K (sum J w rho|u|^2/2)",
            "forward_ms": fwd_ms, "gradient_ms": grad_ms, "gradient_over_forward": grad_ms / fwd_ms,
            "gradient_from_u0_checkpointed_ms": grad_ckpt_ms,
            "value": w.dofs * STAGES * K / (grad_ms * 1e-3), "unit": "DOF-stage/s (reverse sweep incl. recomputation)",
            "roofline": {"bound": "alu", "kernel": "adj_volume (transposed flux differencing, FP64 pipe)",
                         "achieved": achieved / 1e12, "peak": peak_fp64 / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / peak_fp64, "traffic": None, "flops_per_launch": flops},
            "visc_roofline": {"bound": "alu", "kernel": "adj_visc (transposed BR1 lifting and viscous flux, FP64 pipe)",
                              "achieved": vachieved / 1e12, "peak": peak_fp64 / 1e12, "unit": "TFLOP/s",
                              "frac": vachieved / peak_fp64, "traffic": None, "flops_per_launch": vflops},
            "kernels": {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / max(total, 1e-9), 4)}
                        for k, v in kt.items() if v[1]}}


def run_other_workloads(stream) -> dict:
    """Throughput of the other named workloads (the benchmark table's remaining rows): the small N=3
    Euler case (launch bound; CUDA-graph replay on), the paper's free-stream benchmark case (N=7, 32^3
    Cartesian, Navier-Stokes), the blast with DG/FV blending at 64^3 (as named)
    and 40^3 (the size the quoted DOF count implies), and the FP32-bulk 48^3 form."""
    import torch

    from paper_2306_12891_gb300 import dg

    cases = [("tgv_euler_n3_4x4x4", None, 200, {}), ("freestream_ns_n7_32x32x32", None, 5, {}),
             ("blast_euler_fv_n5_64x64x64", None, 5, {}),
             ("blast_euler_fv_n5_64x64x64", 40, 5, {}),
             ("tgv_ns_n7_48x48x48_curved_fp32", None, 5, dict(precision="fp32_bulk", p_ref=P0_TGV))]
    out = {}
    for name, nel, steps, extra in cases:
        w = WORKLOADS[name] if nel is None else WORKLOADS[name].with_(nel=(nel,) * 3)
        xyz, faces = w.mesh()
        s = dg.DG(w.N, xyz, faces, stream=stream, **extra, **w.physics())
        U = torch.from_numpy(w.initial_state(xyz)).cuda()
        dt = s.max_dt(U, w.cfl)
        s.lserk_steps(U, dt, 3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.lserk_steps(U, dt, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        s.check()
        ms = e0.elapsed_time(e1) / steps
        key = name if nel is None else f"{name} at {nel}^3"
        row = {"N": w.N, "elements": w.n_elems, "dofs": w.dofs, "steps": steps, "ms_per_step": ms,
               "value": w.dofs * STAGES / (ms * 1e-3), "unit": UNIT, "precision": extra.get("precision", "fp64")}
        if w.shock_capturing:
            alpha = s.indicator(U)
            row["troubled_fraction"] = float((alpha > 0).double().mean())
        out[key] = row
        del s
    return out


SC_WORKLOAD = "blast_euler_fv_n5_64x64x64"


def run_shock_capturing(stream, peak_fp64: float, steps: int = 200, chunk: int = 20, timed: int = 5) -> dict:
    """The shock-capturing workload where it does FV work (Sec. 4.1-4.2): the blast at 64^3 as named,
    run for its 200 LSERK(5,4) steps (dt from the CFL condition at the start of every chunk of
    `chunk` steps, since the blast's wave speeds change), with the troubled fraction (alpha > 0) after
    each chunk. Kernel timings over `timed` steps at three points: the initial state (the smooth
    front: no element troubled, the volume kernel's DG path only), the state after the 200 steps
    (the shock formed: a shell of troubled elements), and that state with alpha = 1 on every element
    (the FV subcell operator everywhere). The blended volume kernel's roofline comes from the last
    (every element does the DG and the FV work), and the load balance of skipping FV work per element
    from the middle one against the line between the other two."""
    import torch

    from paper_2306_12891_gb300 import dg

    w = WORKLOADS[SC_WORKLOAD]
    xyz, faces = w.mesh()
    s = dg.DG(w.N, xyz, faces, stream=stream, **w.physics())
    U = torch.from_numpy(w.initial_state(xyz)).cuda()

    def timed_steps(solver, V):
        dt_ = solver.max_dt(V, w.cfl)
        V2 = V.clone()
        solver.lserk_steps(V2, dt_, 3)
        solver.timing_enable(True)
        solver.timing_get()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        solver.lserk_steps(V2, dt_, timed)
        e1.record(stream)
        torch.cuda.synchronize()
        kt = solver.timing_get()
        solver.timing_enable(False)
        solver.check()
        vol_ms, vol_n = kt["volume"]
        return {"ms_per_step": e0.elapsed_time(e1) / timed, "volume_ms_per_launch": vol_ms / vol_n,
                "troubled_fraction": float((solver.indicator(V2) > 0).double().mean()),
                "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in kt.items() if v[1]}}

    out = {"workload": SC_WORKLOAD, "N": w.N, "elements": w.n_elems, "dofs": w.dofs}
    out["initial"] = timed_steps(s, U)
    fractions, t_run = [], 0.0
    torch.cuda.synchronize()
    for k in range(steps // chunk):
        dt = s.max_dt(U, w.cfl)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.lserk_steps(U, dt, chunk)
        e1.record(stream)
        torch.cuda.synchronize()
        t_run += e0.elapsed_time(e1)
        s.check()
        fractions.append(round(float((s.indicator(U) > 0).double().mean()), 5))
    out["run"] = {"steps": steps, "ms_per_step": t_run / steps, "value": w.dofs * STAGES * steps / (t_run * 1e-3),
                  "unit": UNIT, "troubled_fraction_every_%d_steps" % chunk: fractions}
    out["shocked"] = timed_steps(s, U)
    del s
    s1 = dg.DG(w.N, xyz, faces, stream=stream, **{**w.physics(), "alpha_fixed": 1.0})
    out["fv_everywhere"] = timed_steps(s1, U)
    del s1
    t0, t1 = out["initial"]["volume_ms_per_launch"], out["fv_everywhere"]["volume_ms_per_launch"]
    f = out["shocked"]["troubled_fraction"]
    lin = t0 + f * (t1 - t0)
    out["load_balance"] = {"troubled_fraction": f, "volume_ms_linear_model": lin,
                           "volume_ms_measured": out["shocked"]["volume_ms_per_launch"],
                           "measured_over_model": out["shocked"]["volume_ms_per_launch"] / lin}
    flops = (volume_kernel_flops_per_element(w.N, False) + fv_subcell_flops_per_element(w.N, LLF_FLOPS)) * w.n_elems
    achieved = flops / (t1 * 1e-3)
    out["roofline"] = {"bound": "alu", "kernel": "volume with the DG/FV blend, alpha = 1 on every element (FP64 pipe)",
                       "achieved": achieved / 1e12, "peak": peak_fp64 / 1e12, "unit": "TFLOP/s",
                       "frac": achieved / peak_fp64, "traffic": None, "flops_per_launch": flops}
    return out


WALL_WORKLOAD = "channel_wm_ns_n5_48x24x24"


def run_wall_model(stream, steps: int = 5, warmup: int = 3) -> dict:
    """Cost of the wall model (Sec. 3): LSERK steps of the wall-modelled channel against the same
    mesh, state and physics with the walls replaced by periodic faces, FP64."""
    import torch

    from paper_2306_12891_gb300 import dg

    out = {"workload": WALL_WORKLOAD}
    for label, walls in (("walls", True), ("periodic", False)):
        w = WORKLOADS[WALL_WORKLOAD].with_(z_walls=walls)
        xyz, faces = w.mesh()
        s = dg.DG(w.N, xyz, faces, stream=stream, **w.physics())
        U = torch.from_numpy(WORKLOADS[WALL_WORKLOAD].initial_state(xyz)).cuda()
        dt = s.max_dt(U, w.cfl)
        s.lserk_steps(U, dt, warmup)
        s.timing_enable(True)
        s.timing_get()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.lserk_steps(U, dt, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        kt = s.timing_get()
        s.check()
        ms = e0.elapsed_time(e1) / steps
        out[label] = {"ms_per_step": ms, "value": w.dofs * STAGES / (ms * 1e-3), "unit": UNIT,
                      "face_ms_per_launch": kt["face"][0] / kt["face"][1]}
        if walls:
            out["wall_faces"] = int((faces[:, 2] < 0).sum())
        del s
    out["overhead"] = out["walls"]["ms_per_step"] / out["periodic"]["ms_per_step"] - 1.0
    return out


def run_gpu(args):
    import torch

    from paper_2306_12891_gb300 import build, dg

    world, rank, local = dist_setup(args.gpus)
    if rank == 0 or not os.path.exists(dg.LIB_PATH):
        build.build()
    barrier(world)
    w = WORKLOADS[args.workload]
    if args.nel:  # a smaller mesh of the same workload (profiling runs)
        w = w.with_(nel=(args.nel,) * 3)
    fp32_main = args.precision == "fp32_bulk"
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    stream = torch.cuda.current_stream()
    p_ref = P0_TGV if w.initial == "tgv" else 0.0
    prec = dict(precision="fp32_bulk", p_ref=p_ref) if fp32_main else {}
    if args.alpha_fixed is not None:  # profiling runs of the blended volume kernel: alpha fixed on every element
        prec["alpha_fixed"] = args.alpha_fixed
    solver = dg.DG(w.N, xyz, faces, stream=stream, **prec, **w.physics())
    solver.use_tma(args.tma_mode)
    U = torch.from_numpy(U0).cuda()
    dt = solver.max_dt(U, w.cfl)
    peak_fp64 = dg.probe_fma("fp64", stream)

    # device-resident timed region
    solver.lserk_steps(U, dt, args.warmup)
    solver.check()

    def timed_region():
        torch.cuda.synchronize()
        barrier(world)
        clocks = ClockSampler(local)
        solver.timing_enable(True)
        solver.timing_get()  # reset
        l0 = solver.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        solver.lserk_steps(U, dt, args.steps, t=args.warmup * dt)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms_ = e0.elapsed_time(e1)
        clk_ = clocks.stop()
        launches_ = solver.launch_count() - l0
        ktimes_ = solver.timing_get()
        solver.timing_enable(False)
        solver.check()
        return max_over_ranks(world, ms_), clk_, launches_, ktimes_

    ms, clk, launches, ktimes = timed_region()
    if throttled(clk) and world == 1:  # a throttled region is measured once more (same step count)
        ms, clk, launches, ktimes = timed_region()
        clk["remeasured"] = True

    # end to end through the host-buffer entry point: copies in and out every step
    Uh = torch.from_numpy(U.cpu().numpy()).pin_memory()
    solver.lserk_step_host(Uh, dt)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 5))
    for k in range(e2e_steps):
        solver.lserk_step_host(Uh, dt)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)

    # the FP32-bulk form on the same workload: throughput and its error against the FP64 state
    fp32 = None
    if args.fp32 and not fp32_main:
        U64 = U.clone()  # FP64 state after warmup + steps (the e2e steps ran on a host copy)
        n_done = args.warmup + args.steps
        del solver
        s32 = dg.DG(w.N, xyz, faces, stream=stream, precision="fp32_bulk", p_ref=p_ref, **w.physics())
        s32.use_tma(args.tma_mode)
        V = torch.from_numpy(U0).cuda()
        s32.lserk_steps(V, dt, args.warmup)
        torch.cuda.synchronize()
        barrier(world)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s32.timing_enable(True)
        s32.timing_get()
        f0.record(stream)
        s32.lserk_steps(V, dt, args.steps)
        f1.record(stream)
        torch.cuda.synchronize()
        ms32 = max_over_ranks(world, f0.elapsed_time(f1))
        kt32 = s32.timing_get()
        s32.timing_enable(False)
        step32 = fp32_step_roofline(w.N, w.n_elems, kt32, ms32)
        s32.lserk_steps(V, dt, n_done - args.warmup - args.steps)
        s32.check()
        d = (V - U64).abs().amax(dim=(0, 2, 3, 4))
        change = (U64 - torch.from_numpy(U0).cuda()).abs().amax(dim=(0, 2, 3, 4))
        scale = U64.abs().amax(dim=(0, 2, 3, 4))
        value32 = world * w.dofs * STAGES * args.steps / (ms32 * 1e-3)
        fp32 = {"value": value32, "unit": UNIT, "ms_per_step": ms32 / args.steps,
                "speedup_vs_fp64": value32 / (world * w.dofs * STAGES * args.steps / (ms * 1e-3)),
                "steps_compared": n_done,
                "linf_err_rel_to_state": (d / scale).tolist(),
                "linf_err_rel_to_change": (d / change).tolist(),
                "p_ref": p_ref, "step_roofline": step32,
                "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in kt32.items() if v[1]}}
        v32_ms, v32_n = kt32.get("volume", (0.0, 0))
        if v32_n:  # the FP32 volume kernel against the copy bandwidth (algorithmic bytes per launch)
            b32 = volume_kernel_bytes_per_element(w.N, True, 4) * w.n_elems
            gbs = b32 / (v32_ms / v32_n * 1e-3) / 1e9
            fp32["roofline"] = {"bound": "hbm", "kernel": "volume (FP32-bulk)", "achieved": gbs, "peak": HBM_GBS,
                                "unit": "GB/s", "frac": gbs / HBM_GBS, "bytes_per_launch": b32,
                                "traffic": scaled_traffic(VOLUME_F32_DRAM_BYTES_PER_ELEMENT, w.n_elems, w.N == 7),
                                "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}
        del s32

    dofs = w.dofs
    total_updates = world * dofs * STAGES * args.steps
    value = total_updates / (ms * 1e-3)
    vol_ms, vol_n = ktimes.get("volume", (0.0, 0))
    vol_s = vol_ms / vol_n * 1e-3 if vol_n else None
    if fp32_main:  # HBM-bound: algorithmic bytes of the volume kernel against the measured copy bandwidth
        bytes_launch = volume_kernel_bytes_per_element(w.N, True, 4) * w.n_elems
        roofline = {"bound": "hbm", "kernel": "volume (FP32-bulk)", "achieved": bytes_launch / vol_s / 1e9,
                    "peak": HBM_GBS, "unit": "GB/s", "frac": bytes_launch / vol_s / 1e9 / HBM_GBS,
                    "traffic": scaled_traffic(VOLUME_F32_DRAM_BYTES_PER_ELEMENT, w.n_elems, w.N == 7),
                    "bytes_per_launch": bytes_launch,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}
    else:
        flops_launch = volume_kernel_flops_per_element(w.N, True) * w.n_elems
        achieved = flops_launch / vol_s
        roofline = {"bound": "alu", "kernel": "volume (split-form flux differencing, FP64 pipe)",
                    "achieved": achieved / 1e12, "peak": peak_fp64 / 1e12, "unit": "TFLOP/s",
                    "frac": achieved / peak_fp64,
                    "traffic": scaled_traffic(VOLUME_DRAM_BYTES_PER_ELEMENT, w.n_elems),
                    "flops_per_launch": flops_launch, "peak_source": "measured FP64 FMA probe (dg_probe_fma), live",
                    "flops_basis": FLOPS_BASIS}
    state_bytes = U.numel() * 8
    if rank != 0:
        return
    breakdown = {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / max(1e-9, sum(x[0] for x in ktimes.values())), 4)}
                 for k, v in ktimes.items() if v[1]}
    line = {
        "metric": METRIC if not fp32_main else METRIC.replace("FP64", "FP32-bulk"), "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if fp32_main else "f64", "data": "synthetic",
        "config": {"workload": (args.workload if not args.nel else f"{args.workload} reduced to {args.nel}^3")
                   + (f", alpha fixed at {args.alpha_fixed}" if args.alpha_fixed is not None else ""),
                   "N": w.N, "elements": w.n_elems, "dofs": dofs,
                   "physics": "Navier-Stokes, Pirozzoli split form, Roe, BR1, curved mesh, TGV Re 1600 Ma 0.1",
                   "precision": args.precision, "dt": dt, "cfl": w.cfl,
                   **({"fp32_kernel_form": args.tma_mode} if fp32_main else {}),
                   "l2": f"inputs larger than L2 (state {state_bytes / 1e6:.0f} MB, working set > 5 GB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "pid_s_per_dof_stage": 1.0 / (value / world),
        "step_roofline": (step_roofline(w.N, value / world, peak_fp64) if not fp32_main
                          else fp32_step_roofline(w.N, w.n_elems, ktimes, ms)),
        "roofline": roofline,
        "kernels": breakdown,
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": {"value": world * dofs * STAGES * e2e_steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes},
    }
    if fp32:
        line["fp32_bulk"] = fp32
    if args.adjoint and not args.nel and world == 1:
        line["adjoint"] = run_adjoint(stream, peak_fp64)
    if args.wall and not args.nel and world == 1:
        line["wall_model"] = run_wall_model(stream)
    if args.others and not args.nel and world == 1:
        line["other_workloads"] = run_other_workloads(stream)
    if args.shock and not args.nel and world == 1:
        try:
            line["shock_capturing"] = run_shock_capturing(stream, peak_fp64)
        except dg.DGError as ex:  # a non-physical state in the blast run is reported, not fatal to the line
            line["shock_capturing"] = {"workload": SC_WORKLOAD, "error": str(ex)}
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-fp32", dest="fp32", action="store_false", help="skip the FP32-bulk comparison")
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false", help="skip the adjoint (gradient) block")
    ap.add_argument("--no-wall", dest="wall", action="store_false", help="skip the wall-model cost block")
    ap.add_argument("--no-others", dest="others", action="store_false", help="skip the other workloads' throughput")
    ap.add_argument("--no-shock", dest="shock", action="store_false",
                    help="skip the shock-capturing block (the blast's 200 steps with FV work)")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_bulk"])
    ap.add_argument("--nel", type=int, default=None, help="elements per direction (default: the workload's 32)")
    ap.add_argument("--alpha-fixed", type=float, default=None,
                    help="shock-capturing workloads: a fixed blending coefficient on every element (profiling)")
    ap.add_argument("--tma-mode", type=int, default=3, choices=[0, 1, 2, 3],
                    help="FP32-bulk kernel form (dg_use_tma): 3 pair-symmetric line kernel (default), "
                         "2 warp-specialised node kernel, 1 TMA node kernel, 0 plain kernels")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
