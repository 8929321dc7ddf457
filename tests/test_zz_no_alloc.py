"""The allocation-free diagnostics entry point, dg_invariants_noalloc.

It is for callers that cannot allocate device memory where they need the integrals (a host
framework whose caching allocator holds nearly all of the device memory, or real-time and embedded
code that forbids allocation after start-up): its partial sums live in a fixed array inside the
library instead of context memory. This file is
collected last so that a run stopping at the first failure has already run every other test.
"""
import ctypes

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


def _noalloc(dg, torch, N, nE, gamma, U, Ut, J, out):
    return dg.lib().dg_invariants_noalloc(N, nE, gamma, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(Ut.data_ptr()),
                                          ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("name,nel", [("tgv_euler_n3_4x4x4", None), ("tgv_ns_n7_32x32x32_curved", (3, 2, 4))])
def test_noalloc_invariants_match_dg_invariants_twice(env, name, nel):
    dg, torch = env
    w = W.WORKLOADS[name]
    if nel:
        w = w.with_(nel=nel)
    xyz, faces = w.mesh()
    solver = dg.DG(w.N, xyz, faces, **w.physics())
    U = torch.from_numpy(w.initial_state(xyz)).cuda()
    _, J = solver.metrics()
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):  # two calls in a row on different states
        if call == 1:
            solver.lserk_step(U, 1e-3)
        Ut = solver.rhs(U)
        ref = solver.invariants(U, Ut)  # the existing entry point (context scratch, synchronising)
        st = _noalloc(dg, torch, w.N, solver.nE, 1.4, U, Ut, J, out)
        assert st == 0, dg.STATUS.get(st, st)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_noalloc_several_rows_then_fewer(env):
    """Several chunk rows with a partial last one (N = 7 on 5x5x5 elements: 64,000 nodes, 4 rows of
    16,384), then a smaller call on 2x2x3 elements (6,144 nodes, 1 row): the second call must read
    only the rows it wrote, not the first call's leftovers. Each result against dg_invariants."""
    dg, torch = env
    w = W.WORKLOADS["tgv_ns_n7_32x32x32_curved"]
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    for nel in [(5, 5, 5), (2, 2, 3)]:
        ww = w.with_(nel=nel)
        xyz, faces = ww.mesh()
        solver = dg.DG(ww.N, xyz, faces, **ww.physics())
        U = torch.from_numpy(ww.initial_state(xyz)).cuda()
        _, J = solver.metrics()
        Ut = solver.rhs(U)
        ref = solver.invariants(U, Ut)
        assert _noalloc(dg, torch, ww.N, solver.nE, 1.4, U, Ut, J, out) == 0
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_noalloc_rejects_sizes_beyond_its_array(env):
    dg, torch = env
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    # 262,144 elements of degree 5 = 56.6M nodes > 33,554,432: refused before any launch
    st = _noalloc(dg, torch, 5, 262144, 1.4, dummy, dummy, dummy, dummy)
    assert st == -6  # DG_ERR_UNSUPPORTED
    st = _noalloc(dg, torch, 9, 8, 1.4, dummy, dummy, dummy, dummy)
    assert st == -1  # DG_ERR_ARG: degree out of range
