"""CUDA-graph replay of the LSERK step sequence: identical bits to launching every kernel, for the
FP64 and FP32-bulk forms, with shock capturing, across changes of U and dt (recapture), and
interleaved with single steps; plus the time per step of the launch-bound N = 3, 4^3 workload."""
import time

import numpy as np
import pytest

from paper_2306_12891_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2306_12891_gb300 import build, dg

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    dg.lib()
    return dg, torch


@pytest.mark.parametrize("name,extra", [("tgv_euler_n3_4x4x4", {}),
                                        ("tgv_ns_n7_32x32x32_curved", dict(precision="fp32_bulk", p_ref=1 / 1.4e-2)),
                                        ("tgv_euler_n3_4x4x4", dict(shock_capturing=True))])
def test_graph_replay_is_bit_identical(env, name, extra):
    """(the third case runs the indicator and the DG/FV blend inside the graph)"""
    dg, torch = env
    w = W.WORKLOADS[name]
    if "shock_capturing" in extra:
        w = w.with_(shock_capturing=True)
        extra = {}
    if w.n_elems > 64:
        w = w.with_(nel=(4, 4, 4))
    xyz, faces = w.mesh()
    U0 = torch.from_numpy(w.initial_state(xyz)).cuda()
    out = []
    for graphs in (False, True):
        s = dg.DG(w.N, xyz, faces, **extra, **w.physics())
        s.use_graphs(graphs)
        dt = s.max_dt(U0, w.cfl)
        U = U0.clone()
        l0 = s.launch_count()
        s.lserk_steps(U, dt, 7)
        s.lserk_step(U, dt)              # a single step between replays
        s.lserk_steps(U, 0.5 * dt, 4)     # new dt: recapture
        V = U.clone()
        s.lserk_steps(V, dt, 3)           # new U: recapture
        s.check()
        out.append((U.clone(), V.clone(), s.launch_count() - l0))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_small_case_time_per_step(env):
    dg, torch = env
    w = W.WORKLOADS["tgv_euler_n3_4x4x4"]
    xyz, faces = w.mesh()
    U = torch.from_numpy(w.initial_state(xyz)).cuda()
    res = {}
    for graphs in (False, True):
        s = dg.DG(w.N, xyz, faces, **w.physics())
        s.use_graphs(graphs)
        dt = s.max_dt(U, w.cfl)
        s.lserk_steps(U.clone(), dt, 10)
        V = U.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.lserk_steps(V, dt, 1000)
        torch.cuda.synchronize()
        res[graphs] = (time.perf_counter() - t0) / 1000 * 1e6
    print(f"GRAPHS N=3 4^3 Euler: {res[False]:.1f} us/step launched, {res[True]:.1f} us/step replayed "
          f"(x{res[False] / res[True]:.2f})")
    assert res[True] < res[False]
