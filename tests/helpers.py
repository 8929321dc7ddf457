"""Shared test helpers: the parity metrics and magnitude scales (no method arithmetic).

FP64 parity is asserted two ways, and both figures are printed by every FP64 parity test:

1. normwise, against the conditioning of the problem: per conservative variable v,
   err_v = max |Ut_GPU - Ut_oracle|_v must not exceed ULP_FACTOR times the oracle's own spread
   under seeded one-ulp perturbations of its inputs: every state value, and every mesh point,
   moved up, down or not at all by one ulp. Two correct FP64 evaluations of the same operator
   differ by the rounding of what they compute, and a one-ulp change of the inputs moves the oracle
   by that same amount; a dropped term or a wrong index moves it by far more. The bound is printed
   relative to max |Ut_oracle|_v (the normwise error).
   The mesh is perturbed as a set of points: copies of one physical point (a node on a face, edge
   or corner shared by several elements, or its periodic image) move together, so the mesh stays
   closed. This term dominates on curved meshes with a large background pressure: the curl-form
   metric terms of any FP64 evaluation carry rounding of order eps * sum |D| * |X| |dX|, and their
   discrete metric identity -- which cancels p0 * sum_d D_d Ja^d -- holds only to that rounding
   (on the Ma 0.1 N = 7 Taylor-Green case the mesh points move the momentum RHS 500 times further
   than the state does). A second correct evaluation with other rounding in every flux and sum (the
   oracle compiled with FMA contraction) stays inside one spread (tests/test_parity_bound.py);
2. relative to the flux scale (flux_scale below): err_v / scale_v <= 1e-12, where scale_v is the
   size of the largest flux-difference term the right-hand side sums.
"""

import numpy as np

ULP_FACTOR = 4.0
TOL = 1e-12


def per_var_max(X):
    """max |X| per conservative variable of a state-shaped array [nE][5][...]."""
    X = np.abs(np.asarray(X))
    return X.reshape(X.shape[0], 5, -1).max(axis=(0, 2))


def euler_flux_magnitude(U, Ja, gamma=1.4, state_dissipation=False):
    """Per node and variable: sum_d |F^d_v(U)| with F^d the contravariant Euler flux -- the size of
    the advective flux terms the right-hand side differences (numpy, vectorised).

    state_dissipation adds c |Ja^d| |U_v| (c = sound speed). That term belongs only to the FP32-bulk
    form: there the Riemann dissipation lambda (U_R - U_L) differences states already rounded to
    FP32, whose rounding error is eps32 |U|, not eps32 |U_R - U_L|. In FP64 both sides read the same
    FP64 states, so the dissipation term carries rounding of its jump only, which the advective
    magnitude already bounds."""
    rho = U[:, 0]
    u = U[:, 1:4] / rho[:, None]
    p = (gamma - 1.0) * (U[:, 4] - 0.5 * rho * (u * u).sum(1))
    c = np.sqrt(gamma * np.abs(p) / np.abs(rho))
    out = np.zeros(U.shape)
    for d in range(3):
        V = (u * Ja[:, d]).sum(1)  # u . Ja^d
        s = np.sqrt((Ja[:, d] ** 2).sum(1))
        F = [rho * V] + [U[:, 1 + c_] * V + p * Ja[:, d, c_] for c_ in range(3)] + [(U[:, 4] + p) * V]
        for v in range(5):
            out[:, v] += np.abs(F[v])
            if state_dissipation:
                out[:, v] += c * s * np.abs(U[:, v])
    return out


def _face_nodes(N, f):
    """(k, j, i) index arrays [q][p] of the nodes of local face f, face point (p, q)."""
    n = N + 1
    p, q = np.meshgrid(np.arange(n), np.arange(n))  # [q][p]
    b = np.full_like(p, N if f % 2 else 0)
    if f // 2 == 0:
        return q, p, b
    if f // 2 == 1:
        return q, b, p
    return b, q, p


def face_jump_magnitude(U, faces, N, Ja, gamma=1.4, elements=None):
    """Per node and variable: the size of the Riemann dissipation at the element faces,
    lambda s |U_R - U_L|_v with lambda = max over both sides of |u| + c and s = |Ja^d| (zero away from
    faces; interior faces of the face table only). It is the part of the surface flux that the
    advective magnitude misses where the velocity vanishes but the state jumps."""
    n = N + 1
    rho = U[:, 0]
    u2 = (U[:, 1] ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2) / rho ** 2
    p = (gamma - 1.0) * (U[:, 4] - 0.5 * rho * u2)
    lam = np.sqrt(u2) + np.sqrt(gamma * np.abs(p) / np.abs(rho))
    out = np.zeros(U.shape)
    faces = np.asarray(faces)
    faces = faces[faces[:, 2] >= 0]
    if elements is not None:  # only the faces of these elements (the rest of `out` stays zero)
        keep = np.zeros(U.shape[0], bool)
        keep[np.asarray(elements)] = True
        faces = faces[keep[faces[:, 0]] | keep[faces[:, 2]]]
    for fL, fR, o in {tuple(r) for r in faces[:, [1, 3, 4]]}:
        sel = faces[(faces[:, 1] == fL) & (faces[:, 3] == fR) & (faces[:, 4] == o)]
        eL, eR = sel[:, 0], sel[:, 2]
        kL, jL, iL = _face_nodes(N, fL)
        pp, qq = np.meshgrid(np.arange(n), np.arange(n))
        a, b = (qq, pp) if o & 4 else (pp, qq)
        a = N - a if o & 1 else a
        b = N - b if o & 2 else b
        kR, jR, iR = (x[b, a] for x in _face_nodes(N, fR))
        d = fL // 2
        s = np.sqrt((Ja[eL][:, d][:, :, kL, jL, iL] ** 2).sum(1))
        lm = np.maximum(lam[eL][:, kL, jL, iL], lam[eR][:, kR, jR, iR])
        jump = np.abs(U[eL][:, :, kL, jL, iL] - U[eR][:, :, kR, jR, iR]) * (lm * s)[:, None]
        for e_, k_, j_, i_ in ((eL, kL, jL, iL), (eR, kR, jR, iR)):
            cur = out[e_][:, :, k_, j_, i_]
            out[e_[:, None, None, None], np.arange(5)[None, :, None, None], k_[None, None], j_[None, None],
                i_[None, None]] = np.maximum(cur, jump)
    return out


def subcell_range_magnitude(U, Ja, gamma=1.4):
    """Per node and variable, for the FV subcell operator: lambda_e s_e (max_e U_v - min_e U_v), with
    lambda_e the element's largest |u| + c and s_e its largest |Ja^d|. Minmod reconstruction keeps
    every subcell interface state inside the range of the element's nodal values, so this bounds the
    Riemann dissipation of the interior subcell interfaces, which no nodal flux magnitude shows."""
    rho = U[:, 0]
    u2 = (U[:, 1] ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2) / rho ** 2
    p = (gamma - 1.0) * (U[:, 4] - 0.5 * rho * u2)
    lam = (np.sqrt(u2) + np.sqrt(gamma * np.abs(p) / np.abs(rho))).reshape(U.shape[0], -1).max(1)
    s = np.sqrt((Ja ** 2).sum(2)).reshape(U.shape[0], -1).max(1)
    Ue = U.reshape(U.shape[0], 5, -1)
    rng = Ue.max(2) - Ue.min(2)
    return np.broadcast_to((lam * s)[:, None, None] * rng[:, :, None], Ue.shape).reshape(U.shape)


def flux_scale(U, Ja, J, D, gamma=1.4, state_dissipation=False, faces=None, N=None, jump=None):
    """scale_v = max over nodes of ||2D||_inf * (sum_d |F^d_v(U)| (+ the face dissipation
    face_jump_magnitude when the face table, or that magnitude itself, is given)) / J: the size of
    the largest flux-difference sum in the right-hand side, on which rounding acts."""
    mag = euler_flux_magnitude(U, Ja, gamma, state_dissipation)
    if faces is not None:
        mag = mag + face_jump_magnitude(U, faces, N, Ja, gamma)
    if jump is not None:
        mag = mag + jump
    mag = mag / J[:, None]
    d2 = 2.0 * np.abs(D).sum(1).max()
    return d2 * mag.reshape(mag.shape[0], 5, -1).max(axis=(0, 2))


def parity(Ut, Ut_ref, scale):
    """max |Ut - Ut_ref| per variable divided by the flux scale."""
    return per_var_max(np.asarray(Ut) - np.asarray(Ut_ref)) / scale


def normwise(Ut, Ut_ref):
    """max |Ut - Ut_ref| / max |Ut_ref| per variable."""
    return per_var_max(np.asarray(Ut) - np.asarray(Ut_ref)) / np.maximum(per_var_max(Ut_ref), 1e-300)


def ulp_perturb(a, rng):
    """Every entry moved by one ulp up, one ulp down, or left alone (seeded, equal odds)."""
    a = np.asarray(a, dtype=np.float64)
    r = rng.integers(-1, 2, a.shape)
    return np.where(r > 0, np.nextafter(a, np.inf), np.where(r < 0, np.nextafter(a, -np.inf), a))


def _splitmix64(x):
    """The splitmix64 finaliser (Steele, Lea and Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        x = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        x = ((x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)).astype(np.uint64)
        x = ((x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)).astype(np.uint64)
        return x ^ (x >> np.uint64(31))


def mesh_ulp_perturb(xyz, seed, period=2.0 * np.pi):
    """xyz [nE][3][n][n][n] with every mesh point moved by one ulp up, one ulp down, or left alone per
    coordinate (seeded). The draw is a hash of the point's position modulo the box period, so all
    copies of one physical point, periodic images included, move the same way."""
    P = np.moveaxis(np.asarray(xyz, dtype=np.float64), 1, -1)
    per = np.broadcast_to(np.asarray(period, dtype=np.float64), (3,))
    q = (np.round(np.mod(P, per) / per * 2.0 ** 20).astype(np.int64) % (1 << 20)).astype(np.uint64)
    key = (q[..., 0] << np.uint64(40)) | (q[..., 1] << np.uint64(20)) | q[..., 2]
    out = np.empty_like(P)
    for c in range(3):
        r = (_splitmix64(key ^ np.uint64((seed * 3 + c) & 0xFFFFFFFF)) % np.uint64(3)).astype(np.int64) - 1
        x = P[..., c]
        out[..., c] = np.where(r > 0, np.nextafter(x, np.inf), np.where(r < 0, np.nextafter(x, -np.inf), x))
    return np.ascontiguousarray(np.moveaxis(out, -1, 1))


def ulp_spread(evaluate, xyz, U0, count=3, seed=20230622, period=2.0 * np.pi, base=None):
    """Per variable: max over `count` seeded one-ulp perturbations (mesh points and state together) of
    max |evaluate(xyz', U0') - evaluate(xyz, U0)|, where evaluate(xyz, U) runs the oracle. Returns
    (spread, evaluate(xyz, U0))."""
    if base is None:
        base = evaluate(xyz, U0)
    spread = np.zeros(5)
    for k in range(count):
        Xk = mesh_ulp_perturb(xyz, seed + k, period)
        Uk = ulp_perturb(U0, np.random.default_rng(seed + k))
        spread = np.maximum(spread, per_var_max(evaluate(Xk, Uk) - base))
    return spread, base


def check_fp64(tag, Ut, Ut_ref, spread, scale, tol=TOL, factor=ULP_FACTOR):
    """Assert and print both FP64 parity figures (module docstring). Returns (flux-scale, normwise)."""
    err = per_var_max(np.asarray(Ut) - np.asarray(Ut_ref))
    # a variable whose right-hand side is exactly zero (the energy of a fluid at rest) has no normwise
    # figure; it is printed relative to 1 (absolute)
    mag = per_var_max(Ut_ref)
    mag = np.where(mag > 0, mag, 1.0)
    # 0/0 (a variable with no flux terms and no error, e.g. the energy of a fluid at rest) counts as 0
    fs = np.divide(err, scale, out=np.where(err > 0, np.inf, 0.0), where=scale > 0)
    nw, bound = err / mag, factor * spread / mag
    print(f"PARITY {tag}: flux-scale {np.array2string(fs, precision=2)} normwise "
          f"{np.array2string(nw, precision=2)} bound {np.array2string(bound, precision=2)} "
          f"(x{factor:g} oracle 1-ulp spread)")
    assert (fs <= tol).all(), ("flux-scale", fs)
    assert (err <= factor * spread).all(), ("normwise", nw, "bound", bound)
    return fs, nw


def oracle_trajectory(args):
    """Spawned worker: the oracle advancing a named workload (reduced to `nel` elements) by `steps`
    LSERK(5,4) steps of size dt from its initial state, optionally moved by one ulp (seed). Returns
    the states and the oracle's integral diagnostics (dg_invariants' eight numbers) at every
    `every`-th step, the start included. With a seed, the mesh points and the initial state are
    moved by one ulp first (mesh_ulp_perturb, ulp_perturb)."""
    name, nel, steps, every, dt, seed = args
    import oracle
    from paper_2306_12891_gb300 import workloads as W

    w = W.WORKLOADS[name].with_(nel=nel)
    xyz, faces = w.mesh()
    U = w.initial_state(xyz)
    if seed is not None:
        xyz = mesh_ulp_perturb(xyz, seed, np.asarray(w.hi) - np.asarray(w.lo))
        U = ulp_perturb(U, np.random.default_rng(seed))
    ref = oracle.Oracle(w.N, xyz, faces, **w.physics())
    states, invs = [U.copy()], [ref.invariants(U, ref.rhs(U))]
    for k in range(1, steps + 1):
        U = ref.lserk_step(U, dt)
        if k % every == 0:
            states.append(U.copy())
            invs.append(ref.invariants(U, ref.rhs(U)))
    return states, invs


def _full_size_oracle_rhs(args):
    """Spawned worker: the oracle's right-hand side of a named full-size workload on a sample of
    elements, with every input moved by one ulp (mesh_ulp_perturb, ulp_perturb; seed)."""
    name, extra, sample, seed = args
    import oracle
    from paper_2306_12891_gb300 import workloads as W

    w = W.WORKLOADS[name]
    xyz, faces = w.mesh()
    U0 = w.initial_state(xyz)
    period = np.asarray(w.hi) - np.asarray(w.lo)
    xyz, U0 = mesh_ulp_perturb(xyz, seed, period), ulp_perturb(U0, np.random.default_rng(seed))
    ref = oracle.Oracle(w.N, xyz, faces, **dict(w.physics(), **extra))
    return ref.rhs(U0, mask=sample)[sample]


def full_size_ulp_spread(name, extra, sample, base, count=3, seed=20230622):
    """ulp_spread of a full-size workload's sampled right-hand side; the perturbed oracles run at once
    in spawned host processes (each builds the mesh and its oracle again)."""
    import multiprocessing

    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(count) as pool:
        outs = pool.map(_full_size_oracle_rhs, [(name, extra, list(sample), seed + k) for k in range(count)])
    spread = np.zeros(5)
    for o in outs:
        spread = np.maximum(spread, per_var_max(o - base))
    return spread


def _saved_state_oracle_rhs(args):
    """Spawned worker: the oracle's right-hand side of a named full-size workload at a state saved in
    a .npy file, on a sample of elements, with the mesh points and the state moved by one ulp (seed)."""
    name, path, sample, seed = args
    import oracle
    from paper_2306_12891_gb300 import workloads as W

    w = W.WORKLOADS[name]
    xyz, faces = w.mesh()
    U = np.load(path)
    period = np.asarray(w.hi) - np.asarray(w.lo)
    xyz, U = mesh_ulp_perturb(xyz, seed, period), ulp_perturb(U, np.random.default_rng(seed))
    return oracle.Oracle(w.N, xyz, faces, **w.physics()).rhs(U, mask=sample)[sample]


def saved_state_ulp_spread(name, path, sample, base, count=3, seed=20230622):
    """ulp_spread of a full-size workload's sampled right-hand side at a saved state (spawned processes)."""
    import multiprocessing

    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(count) as pool:
        outs = pool.map(_saved_state_oracle_rhs, [(name, path, list(sample), seed + k) for k in range(count)])
    spread = np.zeros(5)
    for o in outs:
        spread = np.maximum(spread, per_var_max(o - base))
    return spread
