"""Calibration of the FP64 parity bound that the GPU tests assert (tests/helpers.py): the GPU's
right-hand side may differ from the oracle's by at most ULP_FACTOR times the oracle's own spread
under seeded one-ulp perturbations of its inputs (state values and mesh points).

Two facts make that a bound on rounding and nothing else:
- a second correct FP64 evaluation -- the oracle compiled with FMA contraction, which rounds the
  fluxes and every sum differently -- lies within one spread of the oracle;
- a small planted mistake (gamma wrong in its ninth digit; in its seventh on the Ma 0.1 N = 7
  Taylor-Green case, whose curved-mesh metric rounding against p0 ~ 71 makes it the worst
  conditioned) exceeds the bound.
The spread of the state alone is printed beside it: it is what a bound would be if the metric
terms were exact, and on the Taylor-Green case it is ~500 times smaller.
"""
import numpy as np
import pytest

from helpers import ULP_FACTOR, flux_scale, per_var_max, ulp_spread
from paper_2306_12891_gb300 import workloads as W


def _generic_map(x, y, z):
    return (x + 0.1 * np.sin(y) * np.cos(z), y + 0.1 * np.sin(z) * np.sin(x) + 0.05 * np.sin(2 * x),
            z + 0.1 * np.sin(x) * np.cos(y))


def _cases():
    out = []
    w = W.WORKLOADS["tgv_ns_n7_32x32x32_curved"].with_(nel=(4, 4, 4))
    out.append(("tgv_ns_n7_4x4x4_curved", w.N, w, None, w.physics()))
    w = W.WORKLOADS["tgv_euler_n3_4x4x4"]
    out.append(("tgv_euler_n3_4x4x4", w.N, w, None, w.physics()))
    out.append(("random_ns_n5_curved", 5, None, 5, dict(equations="ns", vflux="pirozzoli", sflux="roe", mu=0.02)))
    out.append(("random_euler_n5_fv_blend", 5, None, 6, dict(equations="euler", vflux="pirozzoli", sflux="llf",
                                                               shock_capturing=True, alpha_fixed=0.5)))
    return out


CASES = _cases()


def _mesh_state(N, w, seed):
    if w is not None:
        xyz, faces = w.mesh()
        return xyz, faces, w.initial_state(xyz)
    xyz, faces = W.box_mesh(N, (3, 2, 3), mapping=_generic_map)
    U = W.random_smooth_state(xyz, seed=seed, amp=0.1)
    return xyz, faces, U * (1.0 + 0.01 * np.random.default_rng(seed + 1).uniform(-1, 1, U.shape))


@pytest.mark.parametrize("tag,N,w,seed,phys", CASES, ids=[c[0] for c in CASES])
def test_parity_bound_is_a_rounding_bound(oracle_mod, tag, N, w, seed, phys):
    xyz, faces, U0 = _mesh_state(N, w, seed)
    ref = oracle_mod.Oracle(N, xyz, faces, **phys)
    spread, base = ulp_spread(lambda X, V: oracle_mod.Oracle(N, X, faces, **phys).rhs(V), xyz, U0,
                              base=ref.rhs(U0))
    state_only, _ = ulp_spread(lambda X, V: ref.rhs(V), xyz, U0, base=base)
    assert (state_only <= spread).all()
    bound = ULP_FACTOR * spread
    mag = per_var_max(base)
    scale = flux_scale(U0, ref.Ja, ref.J, oracle_mod.dmatrix(N))
    # a second correct FP64 evaluation: inside one spread (so ULP_FACTOR leaves a margin of 10)
    other = oracle_mod.Oracle(N, xyz, faces, contracted=True, **phys).rhs(U0)
    e_fma = per_var_max(other - base)
    assert (e_fma > 0).any()  # it really rounds differently
    assert (e_fma <= spread).all(), (tag, e_fma / spread)
    # planted mistakes: gamma wrong in the seventh digit everywhere; in the ninth off the Ma 0.1 case
    rel = 1e-7 if tag.startswith("tgv_ns_n7") else 1e-9
    bad = oracle_mod.Oracle(N, xyz, faces, **{**phys, "gamma": 1.4 * (1.0 + rel)}).rhs(U0)
    e_bad = per_var_max(bad - base)
    print(f"BOUND {tag}: bound/|Ut| {bound / mag} (state alone {ULP_FACTOR * state_only / mag}) "
          f"fma/spread {e_fma / spread} planted({rel:g})/bound {e_bad / bound} planted flux-scale {e_bad / scale}")
    assert (e_bad > 2.0 * bound).any(), (tag, e_bad / bound)


def test_mesh_perturbation_keeps_the_mesh_closed():
    """The mesh points move as a set: copies of one physical point in neighbouring elements, and its
    periodic images, get the same one-ulp move, so every face still matches its neighbour's."""
    from helpers import mesh_ulp_perturb

    xyz, faces = W.box_mesh(3, (3, 2, 2), mapping="sine_0.05")
    X = mesh_ulp_perturb(xyz, 7)
    assert 0.3 < (X != xyz).mean() < 0.9  # about two thirds of the coordinates move
    assert np.abs(X - xyz).max() <= 1e-14 * np.abs(xyz).max() + 1e-300
    # element 0's +x face against element 1's -x face (shared nodes), and the y and z faces
    np.testing.assert_array_equal(X[0][:, :, :, -1], X[1][:, :, :, 0])
    np.testing.assert_array_equal(X[0][:, :, -1, :], X[3][:, :, 0, :])
    np.testing.assert_array_equal(X[0][:, -1, :, :], X[6][:, 0, :, :])
    # the periodic image across x: tangential coordinates identical, x one period apart to an ulp
    np.testing.assert_array_equal(X[2][1:, :, :, -1], X[0][1:, :, :, 0])
    assert np.abs(X[2][0, :, :, -1] - X[0][0, :, :, 0] - 2 * np.pi).max() <= 4 * np.spacing(2 * np.pi)
