"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every function
include/dg.h declares, and its host-side basis tables agree with the oracle's."""
import ctypes
import subprocess

import numpy as np
import pytest


@pytest.fixture(scope="module")
def dg_mod():
    from paper_2306_12891_gb300 import build, dg

    build.build()
    return dg


def test_every_declared_function_is_exported(dg_mod):
    names = dg_mod.header_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(dg_mod.LIB_PATH)
    missing = [nm for nm in names if not hasattr(L, nm)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", dg_mod.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported


def test_library_targets_sm103a(dg_mod):
    """Every translation unit is compiled for sm_103a alone (the build's -gencode flags), and the
    library those flags produced exists and loads."""
    from paper_2306_12891_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert all(f in build.CU_FLAGS for f in build.ARCH)
    ctypes.CDLL(dg_mod.LIB_PATH)


def test_host_basis_matches_oracle(dg_mod, oracle_mod):
    for N in range(1, 8):
        xi, w, D = dg_mod.basis(N)
        xo, wo = oracle_mod.lgl(N)
        np.testing.assert_allclose(xi, xo, rtol=0, atol=1e-15)
        np.testing.assert_allclose(w, wo, rtol=0, atol=1e-15)
        np.testing.assert_allclose(D, oracle_mod.dmatrix(N), rtol=0, atol=1e-15 * N * N * N)


def test_basis_rejects_unsupported_degree(dg_mod):
    with pytest.raises(dg_mod.DGError):
        dg_mod.basis(8)
    assert dg_mod.lib().dg_status_string(-3) == b"non-positive Jacobian"
