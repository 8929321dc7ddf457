"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

Periodic hexahedral box meshes (optionally curved by an analytic map), initial states
and the named workloads. Nothing here is DGSEM arithmetic: LGL node positions come from
numpy's Legendre routines and every field is a closed-form expression evaluated at the
node coordinates. The same arrays feed both the CUDA path and the CPU oracle.

Layouts: xyz [n_elems][3][n][n][n], U [n_elems][5][n][n][n] with node index
i + n*(j + n*k) (i along xi); faces [n_faces][5] = (elemL, faceL, elemR, faceR, orient),
local faces 0:xi-, 1:xi+, 2:eta-, 3:eta+, 4:zeta-, 5:zeta+.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from numpy.polynomial import legendre as _leg

TWO_PI = 2.0 * math.pi
BLAST_SEED = 20230622
ADJOINT_SEED = 20230623
CHANNEL_SEED = 20230624  # perturbation of the Taylor-Green base state for the adjoint workload


def lgl_points(N: int) -> np.ndarray:
    """Legendre-Gauss-Lobatto points on [-1, 1] (ends plus roots of P_N'), via numpy."""
    if N < 1:
        raise ValueError("N >= 1")
    c = np.zeros(N + 1)
    c[N] = 1.0
    dc = _leg.legder(c)
    x = np.sort(np.real(_leg.legroots(dc))) if N >= 2 else np.zeros(0)
    ddc = _leg.legder(dc)
    for _ in range(3):  # polish the companion-matrix roots
        x = x - _leg.legval(x, dc) / _leg.legval(x, ddc)
    x = np.concatenate([[-1.0], x, [1.0]])
    return 0.5 * (x - x[::-1])


def _curved_tgv(x, y, z):
    s = 0.05 * np.sin(x) * np.sin(y) * np.sin(z)
    return x + s, y + s, z + s


MAPPINGS = {None: None, "none": None, "sine_0.05": _curved_tgv}


WALL = -1  # elemR of a wall-modelled boundary face (faceR = 0, the wall-model kind)


def box_mesh(N: int, nel, lo=(0.0, 0.0, 0.0), hi=(TWO_PI, TWO_PI, TWO_PI), mapping=None, z_walls=False):
    """Periodic box of nel = (nx, ny, nz) hexahedra with degree-N LGL nodes.

    Returns (xyz, faces). Node coordinates along each axis are lo + (e + s_i) h with
    s = (1 + xi)/2, so the two elements sharing a face hold bit-identical face nodes.
    `mapping` (a name in MAPPINGS or a callable (x, y, z) -> (x', y', z')) curves the mesh.
    z_walls: the planes z = lo and z = hi are wall-modelled walls (a channel) instead of periodic:
    their faces are (elem, local face, -1, 0, 0).
    """
    nx, ny, nz = (int(v) for v in nel)
    if min(nx, ny, nz) < 1:
        raise ValueError("at least one element per direction")
    n = N + 1
    s = 0.5 * (1.0 + lgl_points(N))
    s[0], s[-1] = 0.0, 1.0
    axes = []
    for d, m in enumerate((nx, ny, nz)):
        h = (hi[d] - lo[d]) / m
        axes.append(lo[d] + (np.arange(m)[:, None] + s[None, :]) * h)  # [m][n]
    ax, ay, az = axes
    # element (ex,ey,ez), node (i,j,k) -> arrays [nz][ny][nx][k][j][i]
    X = np.broadcast_to(ax[None, None, :, None, None, :], (nz, ny, nx, n, n, n))
    Y = np.broadcast_to(ay[None, :, None, None, :, None], (nz, ny, nx, n, n, n))
    Z = np.broadcast_to(az[:, None, None, :, None, None], (nz, ny, nx, n, n, n))
    fmap = MAPPINGS[mapping] if (mapping is None or isinstance(mapping, str)) else mapping
    if fmap is not None:
        X, Y, Z = fmap(X, Y, Z)
    nE = nx * ny * nz
    xyz = np.empty((nE, 3, n, n, n))
    xyz[:, 0] = np.reshape(X, (nE, n, n, n))
    xyz[:, 1] = np.reshape(Y, (nE, n, n, n))
    xyz[:, 2] = np.reshape(Z, (nE, n, n, n))
    e = np.arange(nE)
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    def eid(a, b, c):
        return (a % nx) + nx * ((b % ny) + ny * (c % nz))
    faces = np.empty((3 * nE, 5), dtype=np.int32)
    faces[0::3] = np.stack([e, np.full(nE, 1), eid(ex + 1, ey, ez), np.full(nE, 0), np.zeros(nE, int)], 1)
    faces[1::3] = np.stack([e, np.full(nE, 3), eid(ex, ey + 1, ez), np.full(nE, 2), np.zeros(nE, int)], 1)
    faces[2::3] = np.stack([e, np.full(nE, 5), eid(ex, ey, ez + 1), np.full(nE, 4), np.zeros(nE, int)], 1)
    if z_walls:
        top = faces[2::3][:, 0] // (nx * ny) == nz - 1  # z-faces that would wrap around
        zf = faces[2::3].copy()
        zf[top, 2:] = (WALL, 0, 0)
        bottom = np.stack([e[ez == 0], np.full(int((ez == 0).sum()), 4), np.full(int((ez == 0).sum()), WALL),
                           np.zeros(int((ez == 0).sum()), int), np.zeros(int((ez == 0).sum()), int)], 1)
        faces = np.concatenate([faces[0::3], faces[1::3], zf, bottom]).astype(np.int32)
    return xyz, faces


# ------------------------------------------------------------------ unstructured relabelling

def _proper_rotations():
    """The 24 rotations of the reference cube as (perm, signs): new axis a reads old axis perm[a],
    reversed where signs[a] < 0 (signed permutation matrices with determinant +1)."""
    import itertools

    out = []
    for perm in itertools.permutations(range(3)):
        inv = sum(1 for i in range(3) for j in range(i + 1, 3) if perm[i] > perm[j])
        for signs in itertools.product((1, -1), repeat=3):
            if (-1) ** inv * signs[0] * signs[1] * signs[2] == 1:
                out.append((perm, signs))
    return out


ROTATIONS = _proper_rotations()


def relabel_element(N: int, arr: np.ndarray, rot) -> np.ndarray:
    """Node array [..., n, n, n] (k, j, i) of one element re-indexed by a cube rotation: the new
    node (i'_0, i'_1, i'_2) is the old node with i_{perm[a]} = i'_a (or N - i'_a where signs[a] < 0)."""
    perm, signs = rot
    n = N + 1
    new = np.empty_like(arr)
    idx = np.arange(n)
    for kp in idx:
        for jp in idx:
            for ip in idx:
                new_ijk = (ip, jp, kp)
                old = [0, 0, 0]
                for a in range(3):
                    old[perm[a]] = new_ijk[a] if signs[a] > 0 else N - new_ijk[a]
                new[..., kp, jp, ip] = arr[..., old[2], old[1], old[0]]
    return new


def _face_points(N, X, f):
    """Coordinates [n][n][3] of local face f of one element (X [3][n][n][n]), indexed (q, p)."""
    b = N if f % 2 else 0
    if f // 2 == 0:
        pts = X[:, :, :, b]          # [c][k][j] -> (q=k, p=j)
    elif f // 2 == 1:
        pts = X[:, :, b, :]          # [c][k][i] -> (q=k, p=i)
    else:
        pts = X[:, b, :, :]          # [c][j][i] -> (q=j, p=i)
    return np.moveaxis(pts, 0, -1)   # [q][p][3]


def build_faces(N: int, xyz: np.ndarray, period, tol: float = 1e-9) -> np.ndarray:
    """Face table of a conforming hexahedral mesh from its node coordinates: faces whose node sets
    coincide (modulo the periodic lengths `period`) are paired, and the orientation code mapping
    the first element's face point (p, q) to the second's is found by trying all eight."""
    from scipy.spatial import cKDTree

    L = np.asarray(period, dtype=float)
    n = N + 1

    def wrap(P):
        return np.mod(P, L)

    nE = xyz.shape[0]
    pts = [_face_points(N, xyz[e], f) for e in range(nE) for f in range(6)]
    cent = np.array([wrap(P.reshape(-1, 3).mean(0)) for P in pts])
    cent = np.where(cent >= L * (1 - 1e-12), 0.0, cent)
    pairs = cKDTree(cent, boxsize=L).query_pairs(r=1e-6 * max(1.0, L.max()), output_type="ndarray")
    if 2 * len(pairs) != len(pts) or len(np.unique(pairs)) != len(pts):
        raise ValueError("face centroids do not pair up one to one")
    table = []
    for s1, s2 in pairs:
        P1, P2 = pts[s1], pts[s2]
        for o in range(8):
            ok = True
            for q in range(n):
                for p in range(n):
                    a, b = (q, p) if o & 4 else (p, q)
                    if o & 1:
                        a = N - a
                    if o & 2:
                        b = N - b
                    d = wrap(P1[q, p] - P2[b, a] + 0.5 * L) - 0.5 * L
                    if np.abs(d).max() > tol * max(1.0, L.max()):
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                table.append((s1 // 6, s1 % 6, s2 // 6, s2 % 6, o))
                break
        else:
            raise ValueError(f"faces {divmod(s1, 6)} and {divmod(s2, 6)} meet but their nodes do not")
    return np.asarray(sorted(table), dtype=np.int32)


def rotated_box_mesh(N: int, nel, seed: int, lo=(0.0, 0.0, 0.0), hi=(TWO_PI, TWO_PI, TWO_PI), mapping=None,
                     fraction=0.5):
    """box_mesh with a seeded random subset of elements re-indexed by random cube rotations and the
    face table rebuilt from the coordinates (so faces of all eight orientations appear)."""
    xyz, _ = box_mesh(N, nel, lo, hi, mapping)
    rng = np.random.default_rng(seed)
    rots = [None] * xyz.shape[0]
    for e in range(xyz.shape[0]):
        if rng.uniform() < fraction:
            rots[e] = ROTATIONS[rng.integers(1, len(ROTATIONS))]
            xyz[e] = relabel_element(N, xyz[e], rots[e])
    faces = build_faces(N, xyz, np.asarray(hi) - np.asarray(lo))
    return xyz, faces, rots


# ------------------------------------------------------------------ initial states

def cons_from_prim(rho, u, v, w, p, gamma=1.4) -> np.ndarray:
    """Stack primitive fields into U[nE][5][n][n][n] (E = p/(gamma-1) + rho|u|^2/2)."""
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, rho * w, E], axis=1))


def taylor_green(xyz, mach=0.1, gamma=1.4, rho0=1.0, U0=1.0):
    """Taylor-Green vortex: p0 = rho0 U0^2/(gamma Ma^2), constant density."""
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    p0 = rho0 * U0 * U0 / (gamma * mach * mach)
    u = U0 * np.sin(x) * np.cos(y) * np.cos(z)
    v = -U0 * np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(x)
    p = p0 + rho0 * U0 * U0 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    rho = np.full_like(x, rho0)
    return cons_from_prim(rho, u, v, w, p, gamma)


def blast(xyz, gamma=1.4, seed=BLAST_SEED, noise=0.01):
    """Spherical blast at (1/2,1/2,1/2): p = 100 inside r = 0.3, 1 outside, tanh width 0.01;
    rho = 1 + noise * U(-1, 1) per node (element-major node order), u = 0."""
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
    p = 1.0 + 99.0 * 0.5 * (1.0 - np.tanh((r - 0.3) / 0.01))
    rng = np.random.default_rng(seed)
    rho = 1.0 + noise * rng.uniform(-1.0, 1.0, size=x.size).reshape(x.shape)
    zero = np.zeros_like(x)
    return cons_from_prim(rho, zero, zero, zero, p, gamma)


def freestream(xyz, gamma=1.4, velocity=(0.3, 0.2, 0.1)):
    """Constant state rho = 1, p = 1/gamma (sound speed 1), u = velocity."""
    one = np.ones_like(xyz[:, 0])
    return cons_from_prim(one, velocity[0] * one, velocity[1] * one, velocity[2] * one, one / gamma, gamma)


def density_wave(xyz, t=0.0, gamma=1.4, amp=0.2):
    """rho = 1 + amp sin(pi (x+y+z - 3t)), u = (1,1,1), p = 1: an exact Euler solution on [-1,1]^3."""
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    rho = 1.0 + amp * np.sin(np.pi * (x + y + z - 3.0 * t))
    one = np.ones_like(x)
    return cons_from_prim(rho, one, one, one, one, gamma)


def smooth_field(xyz, rng, modes=4, terms=8):
    """Seeded smooth periodic field on [0,2pi]^3: a sum of `terms` Fourier modes with integer
    wavenumbers |k_i| <= modes (not all zero), random phases and amplitudes in [-1, 1], scaled to
    max |f| = 1 over the nodes."""
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    f = np.zeros_like(x)
    for _ in range(terms):
        k = np.zeros(3, dtype=int)
        while not k.any():
            k = rng.integers(-modes, modes + 1, size=3)
        f += rng.uniform(-1, 1) * np.sin(k[0] * x + k[1] * y + k[2] * z + rng.uniform(0, TWO_PI))
    return f / max(np.abs(f).max(), 1e-300)


def tgv_perturbed(xyz, seed=ADJOINT_SEED, amp=1e-2, modes=4, gamma=1.4, mach=0.1):
    """Taylor-Green vortex plus a seeded smooth perturbation of (rho, u, v, w, p) from the lowest
    `modes` Fourier modes: amplitude amp relative to rho0 = 1, U0 = 1 and rho0 U0^2."""
    base = taylor_green(xyz, mach=mach, gamma=gamma)
    rho = base[:, 0]
    u, v, w = base[:, 1] / rho, base[:, 2] / rho, base[:, 3] / rho
    p = (gamma - 1.0) * (base[:, 4] - 0.5 * rho * (u * u + v * v + w * w))
    rng = np.random.default_rng(seed)
    d = [amp * smooth_field(xyz, rng, modes) for _ in range(5)]
    return cons_from_prim(rho + d[0], u + d[1], v + d[2], w + d[3], p + d[4], gamma)


def channel_flow(xyz, hz=2.0, ub=1.0, mach=0.3, gamma=1.4, seed=CHANNEL_SEED, amp=0.05):
    """Channel between walls z = 0 and z = hz: a turbulent-like mean profile u = ub (2z'(2 - z'))^(1/7)
    (z' = 2z/hz folded to [0, 1]) with a seeded smooth perturbation of all velocity components
    (relative amplitude amp), rho = 1, p = 1/(gamma Ma^2)."""
    zr = np.minimum(xyz[:, 2], hz - xyz[:, 2]) / (0.5 * hz)
    base = ub * np.clip(zr * (2.0 - zr), 0.0, 1.0) ** (1.0 / 7.0)
    rng = np.random.default_rng(seed)
    du = [amp * ub * smooth_field(xyz, rng, modes=2) for _ in range(3)]
    wall = np.sin(np.pi * xyz[:, 2] / hz)  # perturbations vanish at the walls
    one = np.ones_like(xyz[:, 0])
    return cons_from_prim(one, base + du[0] * wall, du[1] * wall, du[2] * wall, one / (gamma * mach ** 2), gamma)


def random_smooth_state(xyz, seed, amp=0.05, gamma=1.4, modes=2):
    """Seeded smooth periodic perturbation of a rest state (for parity tests of generic fields)."""
    rng = np.random.default_rng(seed)
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    fields = []
    for _ in range(5):
        f = np.zeros_like(x)
        for _ in range(3):
            k = rng.integers(-modes, modes + 1, size=3)
            ph = rng.uniform(0, TWO_PI)
            f += rng.uniform(-1, 1) * np.sin(k[0] * x + k[1] * y + k[2] * z + ph)
        fields.append(f)
    rho = 1.0 + amp * fields[0]
    u, v, w = (0.3 + amp * 4 * fields[1]), (-0.2 + amp * 4 * fields[2]), (0.1 + amp * 4 * fields[3])
    p = 1.0 / gamma + amp * fields[4]
    return cons_from_prim(rho, u, v, w, p, gamma)


# ------------------------------------------------------------------ named workloads

@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    N: int
    nel: tuple
    equations: str          # "euler" | "ns"
    vflux: str              # "kg" | "pirozzoli" | "ec" | "central"
    sflux: str              # "llf" | "roe" | "ec"
    initial: str            # "tgv" | "blast" | "freestream" | "density_wave"
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (TWO_PI, TWO_PI, TWO_PI)
    mapping: str | None = None
    mu: float = 0.0
    Pr: float = 0.72
    gamma: float = 1.4
    R: float = 1.0
    shock_capturing: bool = False
    precision: str = "fp64"  # "fp64" | "fp32_bulk"
    steps: int = 10
    cfl: float = 0.9
    z_walls: bool = False   # z = lo and z = hi are wall-modelled walls (a channel)
    wm_index: int = 1

    @property
    def n_elems(self) -> int:
        return int(np.prod(self.nel))

    @property
    def dofs(self) -> int:
        return self.n_elems * (self.N + 1) ** 3

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)

    def mesh(self):
        return box_mesh(self.N, self.nel, self.lo, self.hi, self.mapping, z_walls=self.z_walls)

    def initial_state(self, xyz):
        if self.initial == "tgv":
            return taylor_green(xyz, gamma=self.gamma)
        if self.initial == "blast":
            return blast(xyz, gamma=self.gamma)
        if self.initial == "freestream":
            return freestream(xyz, gamma=self.gamma)
        if self.initial == "density_wave":
            return density_wave(xyz, gamma=self.gamma)
        if self.initial == "tgv_perturbed":
            return tgv_perturbed(xyz, gamma=self.gamma)
        if self.initial == "channel":
            return channel_flow(xyz, hz=self.hi[2] - self.lo[2], gamma=self.gamma)
        raise ValueError(self.initial)

    def physics(self) -> dict:
        out = dict(equations=self.equations, vflux=self.vflux, sflux=self.sflux, gamma=self.gamma,
                   R=self.R, mu=self.mu, Pr=self.Pr, shock_capturing=self.shock_capturing)
        if self.z_walls:
            out.update(wm_index=self.wm_index, wm_uinf=1.0, wm_mainf=0.3, wm_van_driest=True)
        return out


RE_TGV = 1600.0

WORKLOADS = {
    # Euler, N=3, 4^3 periodic Cartesian on [0,2pi]^3, Kennedy-Gruber + LLF, TGV Ma 0.1
    "tgv_euler_n3_4x4x4": Workload("tgv_euler_n3_4x4x4", 3, (4, 4, 4), "euler", "kg", "llf", "tgv",
                                    steps=10, cfl=0.9),
    # Navier-Stokes, N=7, 32^3 curved, Pirozzoli + Roe + BR1, TGV Re 1600 Ma 0.1 Pr 0.72
    "tgv_ns_n7_32x32x32_curved": Workload("tgv_ns_n7_32x32x32_curved", 7, (32, 32, 32), "ns", "pirozzoli",
                                          "roe", "tgv", mapping="sine_0.05", mu=1.0 / RE_TGV,
                                          steps=100, cfl=0.9),
    # the paper's performance benchmark case (Sec. 2): Navier-Stokes, N=7, 32^3 periodic Cartesian
    # [0,2pi]^3, Pirozzoli + Roe + BR1, free stream
    "freestream_ns_n7_32x32x32": Workload("freestream_ns_n7_32x32x32", 7, (32, 32, 32), "ns", "pirozzoli", "roe",
                                          "freestream", mu=1.0 / RE_TGV, steps=100, cfl=0.9),
    # Euler + FV subcell blending, N=5, 64^3 on the unit cube, Pirozzoli + LLF, blast + 1% noise
    "blast_euler_fv_n5_64x64x64": Workload("blast_euler_fv_n5_64x64x64", 5, (64, 64, 64), "euler",
                                           "pirozzoli", "llf", "blast", lo=(0.0, 0.0, 0.0),
                                           hi=(1.0, 1.0, 1.0), shock_capturing=True, steps=200, cfl=0.5),
    # the same physics as the N=7 curved TGV in the FP32-bulk precision form, 48^3 elements
    "tgv_ns_n7_48x48x48_curved_fp32": Workload("tgv_ns_n7_48x48x48_curved_fp32", 7, (48, 48, 48), "ns",
                                               "pirozzoli", "roe", "tgv", mapping="sine_0.05",
                                               mu=1.0 / RE_TGV, precision="fp32_bulk", steps=1000, cfl=0.9),
    # differentiation form: Navier-Stokes (Pirozzoli + Roe + BR1, curved), N=5, 24^3, perturbed TGV;
    # gradient of the kinetic energy after 50 LSERK steps (checkpoints every 10 steps)
    "tgv_ns_n5_24x24x24_adjoint": Workload("tgv_ns_n5_24x24x24_adjoint", 5, (24, 24, 24), "ns", "pirozzoli",
                                           "roe", "tgv_perturbed", mapping="sine_0.05", mu=1.0 / RE_TGV,
                                           steps=50, cfl=0.9),
    # wall-modelled channel (Sec. 3): walls z = 0, 2; periodic 2pi x pi; N = 5, 48 x 24 x 24 elements;
    # Navier-Stokes, Pirozzoli + Roe + BR1, Re_b = 1e5 (mu = 1e-5 at U_b = 1, half height 1), Ma 0.3,
    # Spalding wall shear with the van Driest transform at the first interior node
    "channel_wm_ns_n5_48x24x24": Workload("channel_wm_ns_n5_48x24x24", 5, (48, 24, 24), "ns", "pirozzoli", "roe",
                                          "channel", lo=(0.0, 0.0, 0.0), hi=(TWO_PI, np.pi, 2.0), mu=1e-5,
                                          steps=10, cfl=0.9, z_walls=True, wm_index=1),
}
