"""FP64 CPU oracle of the split-form DGSEM hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement (``dgsem_oracle.c``) of what arXiv 2306.12891's solver
computes: the split-form DGSEM right-hand side on curved hexahedra (Sec. 2, Sec. 4.1),
its explicit Runge-Kutta step (Sec. 2, Eq. (1)), the modified Persson indicator
(Sec. 4.1, Eq. (7)) and the DG/FV blend (Sec. 4.1, Eq. (6)).

A second build of the same source (``ORC_COMPLEX_STEP``, ``Oracle(..., complex_step=True)``)
runs every state-dependent statement in complex arithmetic: ``jvp`` and ``lserk_jvp`` return
Im L(U + i h V) / h, the exact directional derivative of the oracle's own arithmetic (complex
step; no subtractive cancellation), which is the reference for the discrete adjoint.

A third build, compiled with FMA contraction (``Oracle(..., contracted=True)``), is a second
correct FP64 evaluation with other rounding; the tests use it only to calibrate their parity bound.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package. The CUDA path never does, and this package never imports the
CUDA path: the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dgsem_oracle.c")
HDR = os.path.join(HERE, "dgsem_oracle.h")
LIB_PATH = os.path.join(HERE, "_build", "liboracle.so")
LIB_CS_PATH = os.path.join(HERE, "_build", "liboracle_cs.so")
LIB_FMA_PATH = os.path.join(HERE, "_build", "liboracle_fma.so")
CS_STEP = 1e-30  # complex-step size: h^2 is far below one ulp of any value the oracle forms

EQUATIONS = {"euler": 0, "ns": 1, "navier_stokes": 1}
VFLUX = {"kg": 0, "pirozzoli": 1, "ec": 2, "central": 3}
SFLUX = {"llf": 0, "roe": 1, "ec": 2}
# s = ln((1 - 1e-4) / 1e-4): the sigmoid sharpness of Hennemann et al. (not printed in the paper)
DEFAULT_SHARPNESS = float(np.log((1.0 - 1e-4) / 1e-4))

_libs = {}


def build(force: bool = False) -> str:
    """Compile the oracle (and its complex-step build) with plain -O2 and no FMA contraction
    (same results on x86 and Arm)."""
    os.makedirs(os.path.dirname(LIB_PATH), exist_ok=True)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    for path, defs in ((LIB_PATH, []), (LIB_CS_PATH, ["-DORC_COMPLEX_STEP"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < newest:
            tmp = path + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                                   "-fno-fast-math", *defs, "-o", tmp, SRC, "-lm"])
            os.replace(tmp, path)
    return LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("n_elems", ctypes.c_int), ("xyz", ctypes.POINTER(ctypes.c_double)),
                ("n_faces", ctypes.c_int), ("faces", ctypes.POINTER(ctypes.c_int)),
                ("equations", ctypes.c_int), ("vflux", ctypes.c_int), ("sflux", ctypes.c_int),
                ("gamma", ctypes.c_double), ("R", ctypes.c_double), ("mu", ctypes.c_double),
                ("Pr", ctypes.c_double), ("shock_capturing", ctypes.c_int), ("alpha_min", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("sharpness", ctypes.c_double),
                ("alpha_fixed", ctypes.c_double), ("wm_index", ctypes.c_int), ("wm_uinf", ctypes.c_double),
                ("wm_mainf", ctypes.c_double), ("wm_van_driest", ctypes.c_int)]


_DP = ctypes.POINTER(ctypes.c_double)
RHS_FN = ctypes.CFUNCTYPE(None, _DP, _DP, ctypes.c_double, ctypes.c_void_p)


def build_contracted(force: bool = False) -> str:
    """The same source compiled with FMA contraction (-ffp-contract=fast, -O3): a second correct FP64
    evaluation with other rounding, used only to calibrate the parity bound of the tests. Built on
    request, never by build()."""
    os.makedirs(os.path.dirname(LIB_FMA_PATH), exist_ok=True)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if force or not os.path.exists(LIB_FMA_PATH) or os.path.getmtime(LIB_FMA_PATH) < newest:
        tmp = LIB_FMA_PATH + f".tmp{os.getpid()}"
        isa = ["-mfma"] if platform.machine() in ("x86_64", "AMD64") else []  # FMA is baseline on aarch64
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-ffp-contract=fast", *isa,
                               "-fno-fast-math", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB_FMA_PATH)
    return LIB_FMA_PATH


def lib(complex_step: bool = False, contracted: bool = False):
    key = "fma" if contracted else complex_step
    if key not in _libs:
        build()
        if contracted:
            build_contracted()
        L = ctypes.CDLL(LIB_FMA_PATH if contracted else (LIB_CS_PATH if complex_step else LIB_PATH))
        vp = ctypes.c_void_p
        L.orc_create.restype = vp
        L.orc_create.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(ctypes.c_int)]
        L.orc_destroy.argtypes = [vp]
        L.orc_state_Ja.restype = vp
        L.orc_state_Ja.argtypes = [vp]
        L.orc_state_J.restype = vp
        L.orc_state_J.argtypes = [vp]
        L.orc_rhs.argtypes = [vp, vp, vp, vp, vp]
        L.orc_indicator.argtypes = [vp, vp, vp, vp]
        L.orc_lserk_step.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double]
        L.orc_invariants.argtypes = [vp, vp, vp, vp]
        L.orc_max_dt.argtypes = [vp, vp, ctypes.c_double, vp]
        L.orc_lgl.argtypes = [ctypes.c_int, vp, vp]
        L.orc_dmatrix.argtypes = [ctypes.c_int, vp, vp]
        L.orc_legendre_vandermonde.argtypes = [ctypes.c_int, vp, vp]
        L.orc_invert.argtypes = [ctypes.c_int, vp, vp]
        L.orc_metrics.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp]
        L.orc_logmean.restype = ctypes.c_double
        L.orc_logmean.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_flux_contra.argtypes = [vp, vp, ctypes.c_double, vp]
        L.orc_twopoint.argtypes = [ctypes.c_int, vp, vp, vp, vp, ctypes.c_double, vp]
        L.orc_riemann.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.c_double, vp]
        L.orc_viscous_flux.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, vp]
        L.orc_lserk_generic.argtypes = [ctypes.c_int, vp, ctypes.c_double, ctypes.c_double, RHS_FN, vp]
        L.orc_lserk_coefficients.argtypes = [vp, vp, vp]
        if not complex_step:
            L.orc_spalding_yplus.restype = ctypes.c_double
            L.orc_spalding_yplus.argtypes = [ctypes.c_double]
            L.orc_wall_uplus.restype = ctypes.c_double
            L.orc_wall_uplus.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
            L.orc_van_driest.restype = ctypes.c_double
            L.orc_van_driest.argtypes = [ctypes.c_double] * 5
            L.orc_wall_utau.restype = ctypes.c_double
            L.orc_wall_utau.argtypes = [ctypes.c_double] * 7 + [ctypes.c_int]
        _libs[key] = L
    return _libs[key]


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- basis and geometry

def lgl(N: int):
    xi, w = np.zeros(N + 1), np.zeros(N + 1)
    if lib().orc_lgl(N, _p(xi), _p(w)) != 0:
        raise ValueError("N out of range")
    return xi, w


def dmatrix(N: int, xi=None) -> np.ndarray:
    if xi is None:
        xi = lgl(N)[0]
    D = np.zeros((N + 1, N + 1))
    lib().orc_dmatrix(N, _p(_f64(xi)), _p(D))
    return D


def legendre_vandermonde(N: int, xi=None) -> np.ndarray:
    if xi is None:
        xi = lgl(N)[0]
    V = np.zeros((N + 1, N + 1))
    lib().orc_legendre_vandermonde(N, _p(_f64(xi)), _p(V))
    return V


def metrics(N: int, xyz: np.ndarray):
    xyz = _f64(xyz)
    nE = xyz.shape[0]
    n = N + 1
    Ja = np.zeros((nE, 3, 3, n, n, n))
    J = np.zeros((nE, n, n, n))
    lib().orc_metrics(N, nE, _p(xyz), _p(Ja), _p(J))
    return Ja, J


# ---------------------------------------------------------------- pointwise fluxes

def logmean(a: float, b: float) -> float:
    return lib().orc_logmean(a, b)


def flux_contra(U, a, gamma=1.4):
    F = np.zeros(5)
    lib().orc_flux_contra(_p(_f64(U)), _p(_f64(a)), gamma, _p(F))
    return F


def twopoint(kind: str, UL, UR, aL, aR, gamma=1.4):
    F = np.zeros(5)
    lib().orc_twopoint(VFLUX[kind], _p(_f64(UL)), _p(_f64(UR)), _p(_f64(aL)), _p(_f64(aR)), gamma, _p(F))
    return F


def riemann(kind: str, UL, UR, n, gamma=1.4):
    F = np.zeros(5)
    lib().orc_riemann(SFLUX[kind], _p(_f64(UL)), _p(_f64(UR)), _p(_f64(n)), gamma, _p(F))
    return F


def viscous_flux(U, gradU, gradT, mu, kappa, gamma=1.4):
    Fv = np.zeros(15)
    lib().orc_viscous_flux(_p(_f64(U)), _p(_f64(gradU)), _p(_f64(gradT)), mu, kappa, gamma, _p(Fv))
    return Fv.reshape(3, 5)


# ---------------------------------------------------------------- wall model (Sec. 3)

def spalding_yplus(uplus: float) -> float:
    return lib().orc_spalding_yplus(float(uplus))


def wall_uplus(Re_h: float):
    """(u+, Newton iterations) solving u+ y+(u+) = Re_h."""
    it = ctypes.c_int(0)
    return lib().orc_wall_uplus(float(Re_h), ctypes.byref(it)), it.value


def van_driest(u, uinf, mainf, gamma=1.4, Pr=0.72) -> float:
    return lib().orc_van_driest(float(u), float(uinf), float(mainf), float(gamma), float(Pr))


def wall_utau(U, h, nu, uinf=1.0, mainf=0.0, gamma=1.4, Pr=0.72, van_driest_on=False) -> float:
    return lib().orc_wall_utau(float(U), float(h), float(nu), float(uinf), float(mainf), float(gamma), float(Pr),
                               int(bool(van_driest_on)))


def lserk_coefficients():
    A, B, c = np.zeros(5), np.zeros(5), np.zeros(5)
    lib().orc_lserk_coefficients(_p(A), _p(B), _p(c))
    return A, B, c


def lserk_generic(u0, dt: float, t: float, f):
    """One LSERK(5,4) step of u' = f(u, t) for a Python callable f(u, t) -> ndarray."""
    u = _f64(u0).copy()
    n = u.size

    def cb(up, utp, tt, ctx):
        uu = np.ctypeslib.as_array(up, shape=(n,)).copy()
        out = np.ctypeslib.as_array(utp, shape=(n,))
        out[:] = f(uu, tt)

    fn = RHS_FN(cb)
    lib().orc_lserk_generic(n, _p(u), dt, t, fn, None)
    return u


# ---------------------------------------------------------------- solver

class Oracle:
    """The oracle solver for one mesh and one set of physics parameters."""

    def __init__(self, N, xyz, faces, equations="euler", vflux="kg", sflux="llf", gamma=1.4, R=1.0,
                 mu=0.0, Pr=0.72, shock_capturing=False, alpha_min=0.01, alpha_max=0.7,
                 sharpness=DEFAULT_SHARPNESS, alpha_fixed=-1.0, wm_index=1, wm_uinf=1.0, wm_mainf=0.0,
                 wm_van_driest=False, complex_step=False, contracted=False):
        self.cs = bool(complex_step)
        self._L = lib(self.cs, contracted=bool(contracted) and not self.cs)
        self._dtype = np.complex128 if self.cs else np.float64
        self.N = int(N)
        self.n = self.N + 1
        self.xyz = _f64(xyz)
        self.faces = np.ascontiguousarray(faces, dtype=np.int32)
        self.nE = self.xyz.shape[0]
        pb = _Problem()
        pb.N = self.N
        pb.n_elems = self.nE
        pb.xyz = self.xyz.ctypes.data_as(_DP)
        pb.n_faces = self.faces.shape[0]
        pb.faces = self.faces.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        pb.equations = EQUATIONS[equations]
        pb.vflux = VFLUX[vflux]
        pb.sflux = SFLUX[sflux]
        pb.gamma, pb.R, pb.mu, pb.Pr = gamma, R, mu, Pr
        pb.shock_capturing = int(bool(shock_capturing))
        pb.alpha_min, pb.alpha_max, pb.sharpness = alpha_min, alpha_max, sharpness
        pb.alpha_fixed = float(alpha_fixed)
        pb.wm_index, pb.wm_uinf, pb.wm_mainf = int(wm_index), float(wm_uinf), float(wm_mainf)
        pb.wm_van_driest = int(bool(wm_van_driest))
        self._pb = pb
        st = ctypes.c_int(0)
        self._s = self._L.orc_create(ctypes.byref(pb), ctypes.byref(st))
        if not self._s:
            raise ValueError(f"oracle rejected the problem (status {st.value})")
        self.shape = (self.nE, 5, self.n, self.n, self.n)

    def __del__(self):
        if getattr(self, "_s", None):
            self._L.orc_destroy(self._s)
            self._s = None

    @property
    def Ja(self) -> np.ndarray:
        n = self.n
        ptr = ctypes.cast(self._L.orc_state_Ja(self._s), _DP)
        return np.ctypeslib.as_array(ptr, shape=(self.nE, 3, 3, n, n, n)).copy()

    @property
    def J(self) -> np.ndarray:
        n = self.n
        ptr = ctypes.cast(self._L.orc_state_J(self._s), _DP)
        return np.ctypeslib.as_array(ptr, shape=(self.nE, n, n, n)).copy()

    def _U(self, U):
        U = np.ascontiguousarray(U, dtype=self._dtype)
        if U.size != int(np.prod(self.shape)):
            raise ValueError("U has the wrong size")
        return U

    def rhs(self, U, mask=None, return_alpha=False):
        U = self._U(U)
        Ut = np.zeros(self.shape, dtype=self._dtype)
        alpha = np.zeros(self.nE, dtype=self._dtype)
        m = None
        if mask is not None:
            m = np.zeros(self.nE, dtype=np.uint8)
            m[np.asarray(mask)] = 1
        self._L.orc_rhs(self._s, _p(U), _p(Ut), _p(m) if m is not None else None, _p(alpha))
        return (Ut, alpha) if return_alpha else Ut

    def indicator(self, U):
        U = self._U(U)
        raw, a = np.zeros(self.nE, dtype=self._dtype), np.zeros(self.nE, dtype=self._dtype)
        self._L.orc_indicator(self._s, _p(U), _p(raw), _p(a))
        return raw, a

    def lserk_step(self, U, dt, t=0.0):
        U = self._U(U).copy()
        self._L.orc_lserk_step(self._s, _p(U), float(dt), float(t))
        return U

    def invariants(self, U, Ut):
        out = np.zeros(8, dtype=self._dtype)
        self._L.orc_invariants(self._s, _p(self._U(U)), _p(self._U(Ut)), _p(out))
        return out

    def max_dt(self, U, cfl):
        dt = np.zeros(1)
        self._L.orc_max_dt(self._s, _p(self._U(U)), float(cfl), _p(dt))
        return float(dt[0])

    # ------------------------------------------------------------ complex-step derivatives

    def _need_cs(self):
        if not self.cs:
            raise ValueError("derivatives need Oracle(..., complex_step=True)")

    def jvp(self, U, V):
        """(dL/dU)(U) V for the right-hand side L, by complex step."""
        self._need_cs()
        Z = np.asarray(U, dtype=np.float64) + 1j * CS_STEP * np.asarray(V, dtype=np.float64)
        return self.rhs(Z).imag / CS_STEP

    def lserk_jvp(self, U, V, dt, steps=1):
        """Tangent of `steps` LSERK(5,4) steps: returns (U_K, dU_K/dU_0 V), by complex step."""
        self._need_cs()
        Z = np.asarray(U, dtype=np.float64) + 1j * CS_STEP * np.asarray(V, dtype=np.float64)
        for _ in range(steps):
            Z = self.lserk_step(Z, dt)
        return Z.real.copy(), Z.imag / CS_STEP

    def jacobian(self, U):
        """Dense Jacobian dL/dU [M][M], M = n_elems * 5 * n^3, one complex-step column per unknown
        (small meshes only)."""
        self._need_cs()
        U = np.asarray(U, dtype=np.float64).reshape(-1)
        M = U.size
        Jm = np.zeros((M, M))
        Z = U.astype(np.complex128)
        for k in range(M):
            Z[k] += 1j * CS_STEP
            Jm[:, k] = self.rhs(Z).imag.reshape(-1) / CS_STEP
            Z[k] = U[k]
        return Jm
