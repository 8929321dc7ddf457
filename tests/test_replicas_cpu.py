"""The multi-GPU path of bench.py is replicas only (the solver keeps each mesh on one GPU): every
rank runs the whole workload, the ranks meet at barriers around the timed region, and the reported
value is all ranks' units divided by the slowest rank's time. This exercises that host logic with
world_size 2 on the gloo backend (CPU processes, no GPU)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as td

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    bench.barrier(world)
    seconds = 1.0 + rank  # rank 1 is the slower replica
    m = bench.max_over_ranks(world, seconds)
    value = bench.aggregate(world, 1000.0, seconds)
    bench.barrier(world)
    out.put((rank, m, value))
    td.destroy_process_group()


def test_two_replicas_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]            # both ranks see the slowest rank's time
    assert [r[2] for r in res] == [1000.0, 1000.0]      # 2 x 1000 units / 2 s


def test_throttle_rule():
    """Timed regions whose clock record shows a hardware/thermal slowdown, or SM clocks held well
    below their maximum with no reason (a leftover lock), are measured again; a power cap is kept."""
    import bench

    assert bench.throttled({"reasons": ["hw_thermal_slowdown"], "sm_mhz": 2070, "sm_max_mhz": 2070})
    assert bench.throttled({"reasons": [], "sm_mhz": 1100.0, "sm_max_mhz": 2070.0})
    assert not bench.throttled({"reasons": ["sw_power_cap"], "sm_mhz": 1500.0, "sm_max_mhz": 2070.0})
    assert not bench.throttled({"reasons": [], "sm_mhz": 2070.0, "sm_max_mhz": 2070.0})
    assert not bench.throttled({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]})


def test_oracle_timing_in_parallel_processes():
    """The CPU baseline's parallel oracle timing: spawned processes, each on its own sub-box, start
    together and report their DOF-stages and time; the total rate is the sum over the slowest time."""
    import bench

    value, res = bench.oracle_parallel("steps", 2, 2, warmup=0, steps=1)
    assert len(res) == 2
    dofs = bench.WORKLOADS[bench.WORKLOAD].with_(nel=(2, 2, 2)).dofs
    assert all(r[0] == dofs * bench.STAGES for r in res)
    assert value == pytest.approx(2 * dofs * bench.STAGES / max(r[1] for r in res))
    cpu = bench.host_cpu()
    assert cpu["nproc"] and cpu["nproc"] >= 1
