"""Thin Python binding of libdg (include/dg.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; PyTorch provides device memory
and the stream. There is no CPU fallback: if libdg.so cannot be loaded, or a call fails, an
exception is raised.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "dg.h")

DG_OK = 0
STATUS = {0: "DG_OK", -1: "DG_ERR_ARG", -2: "DG_ERR_MESH", -3: "DG_ERR_JACOBIAN", -4: "DG_ERR_CUDA",
          -5: "DG_ERR_NONPHYSICAL", -6: "DG_ERR_UNSUPPORTED", -7: "DG_ERR_OOM"}
EQUATIONS = {"euler": 0, "ns": 1, "navier_stokes": 1}
VFLUX = {"kg": 0, "pirozzoli": 1, "ec": 2, "central": 3}
SFLUX = {"llf": 0, "roe": 1, "ec": 2}
PRECISION = {"fp64": 0, "fp32_bulk": 1}
DEFAULT_SHARPNESS = float(np.log((1.0 - 1e-4) / 1e-4))


class DGError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Mesh(ctypes.Structure):
    _fields_ = [("n_elems", ctypes.c_int), ("n_geo", ctypes.c_int), ("xyz", ctypes.c_void_p),
                ("n_faces", ctypes.c_int), ("face", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("equations", ctypes.c_int), ("volume_flux", ctypes.c_int), ("surface_flux", ctypes.c_int),
                ("precision", ctypes.c_int), ("gamma", ctypes.c_double), ("R", ctypes.c_double),
                ("mu", ctypes.c_double), ("Pr", ctypes.c_double), ("shock_capturing", ctypes.c_int),
                ("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double), ("sharpness", ctypes.c_double),
                ("alpha_fixed", ctypes.c_double), ("p_ref", ctypes.c_double), ("wm_index", ctypes.c_int),
                ("wm_uinf", ctypes.c_double), ("wm_mainf", ctypes.c_double), ("wm_van_driest", ctypes.c_int)]


_lib = None


def header_functions() -> list[str]:
    """Names of the functions include/dg.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", text)))


def lib() -> ctypes.CDLL:
    """Load libdg.so (built by paper_2306_12891_gb300.build). Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdg.so not built ({LIB_PATH}); run paper_2306_12891_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sig = {
            "dg_init": (i, [ctypes.POINTER(_Mesh), i, i, ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)]),
            "dg_rhs": (i, [vp, vp, vp, d]),
            "dg_lserk_step": (i, [vp, vp, d, d]),
            "dg_lserk_steps": (i, [vp, vp, d, d, i]),
            "dg_lserk_step_host": (i, [vp, vp, d, d]),
            "dg_indicator": (i, [vp, vp, vp]),
            "dg_invariants": (i, [vp, vp, vp, vp]),
            "dg_max_dt": (i, [vp, vp, d, vp]),
            "dg_check": (i, [vp]),
            "dg_get_metrics": (i, [vp, vp, vp]),
            "dg_timing_enable": (i, [vp, i]),
            "dg_timing_get": (i, [vp, vp, vp, vp, i]),
            "dg_launch_count": (ctypes.c_longlong, [vp]),
            "dg_free": (None, [vp]),
            "dg_last_error": (ctypes.c_char_p, [vp]),
            "dg_status_string": (ctypes.c_char_p, [i]),
            "dg_basis": (i, [i, vp, vp, vp]),
            "dg_probe_fma": (i, [i, vp, vp]),
            "dg_invariants_noalloc": (i, [i, i, d, vp, vp, vp, vp, vp]),
            "dg_rhs_vjp": (i, [vp, vp, vp, vp, d]),
            "dg_lserk_step_vjp": (i, [vp, vp, vp, d, d]),
            "dg_lserk_steps_vjp": (i, [vp, vp, vp, d, d, i, i]),
            "dg_kinetic_energy_grad": (i, [vp, vp, vp]),
            "dg_adjoint_memory_limit": (i, [vp, d]),
            "dg_check_conversions": (i, [vp, ctypes.c_longlong, vp]),
            "dg_wall_model": (i, [i, vp, vp, vp, d, d, d, d, i, vp, vp, vp]),
            "dg_use_graphs": (i, [vp, i]),
            "dg_lserk_steps_record": (i, [vp, vp, d, d, i, i, ctypes.POINTER(ctypes.c_longlong)]),
            "dg_lserk_steps_vjp_recorded": (i, [vp, ctypes.c_longlong, vp]),
            "dg_tape_current": (i, [vp, ctypes.POINTER(ctypes.c_longlong)]),
            "dg_use_tma": (i, [vp, i]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def basis(N: int):
    """(xi, w, D) tables the kernels use (host computation, no GPU)."""
    n = N + 1
    xi, w, D = np.zeros(n), np.zeros(n), np.zeros((n, n))
    st = lib().dg_basis(N, xi.ctypes.data, w.ctypes.data, D.ctypes.data)
    if st != DG_OK:
        raise DGError(st, "dg_basis")
    return xi, w, D


def _stream_ptr(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def probe_fma(kind: str = "fp64", stream=None) -> float:
    """Measured FMA throughput in FLOP/s (kind 'fp64' or 'fp32')."""
    out = ctypes.c_double(0.0)
    st = lib().dg_probe_fma(0 if kind == "fp64" else 1, _stream_ptr(stream), ctypes.byref(out))
    if st != DG_OK:
        raise DGError(st, "dg_probe_fma")
    return out.value


def wall_model(U, h, nu, uinf=1.0, mainf=0.0, gamma=1.4, Pr=0.72, van_driest=False, stream=None):
    """(u_tau, Newton iterations) of the wall model for float64 CUDA tensors U, h, nu of one length."""
    import torch

    for t in (U, h, nu):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != U.numel():
            raise ValueError("U, h, nu must be contiguous float64 CUDA tensors of one length")
    utau = torch.empty_like(U)
    iters = torch.empty(U.numel(), dtype=torch.int32, device=U.device)
    st = lib().dg_wall_model(U.numel(), ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(h.data_ptr()),
                             ctypes.c_void_p(nu.data_ptr()), float(uinf), float(mainf), float(gamma), float(Pr),
                             int(bool(van_driest)), ctypes.c_void_p(utau.data_ptr()),
                             ctypes.c_void_p(iters.data_ptr()), _stream_ptr(stream))
    if st != DG_OK:
        raise DGError(st, "dg_wall_model")
    return utau, iters


def check_conversions(count: int = 1 << 24, stream=None):
    """(float->double, double->float) mismatches of the library's integer-pipe conversions against
    the GPU's own, on `count` generated bit patterns each."""
    out = (ctypes.c_longlong * 2)()
    st = lib().dg_check_conversions(_stream_ptr(stream), int(count), out)
    if st != DG_OK:
        raise DGError(st, "dg_check_conversions")
    return int(out[0]), int(out[1])


class DG:
    """A solver context: mesh, degree N, physics and the CUDA stream its calls are queued on."""

    def __init__(self, N, xyz, faces, equations="euler", vflux="kg", sflux="llf", precision="fp64", gamma=1.4,
                 R=1.0, mu=0.0, Pr=0.72, shock_capturing=False, alpha_min=0.01, alpha_max=0.7,
                 sharpness=DEFAULT_SHARPNESS, alpha_fixed=-1.0, p_ref=0.0, wm_index=1, wm_uinf=1.0, wm_mainf=0.0,
                 wm_van_driest=False, stream=None):
        import torch

        self.torch = torch
        self.N, self.n = int(N), int(N) + 1
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        faces = np.ascontiguousarray(faces, dtype=np.int32)
        self.nE = xyz.shape[0]
        self.shape = (self.nE, 5, self.n, self.n, self.n)
        self.numel = int(np.prod(self.shape))
        mesh = _Mesh(self.nE, self.N, xyz.ctypes.data, faces.shape[0], faces.ctypes.data)
        prm = _Params(EQUATIONS[equations], VFLUX[vflux], SFLUX[sflux], PRECISION[precision], gamma, R, mu, Pr,
                      int(bool(shock_capturing)), alpha_min, alpha_max, sharpness, float(alpha_fixed), float(p_ref),
                      int(wm_index), float(wm_uinf), float(wm_mainf), int(bool(wm_van_driest)))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = ctypes.c_void_p(None)
        st = lib().dg_init(ctypes.byref(mesh), self.N, 0, ctypes.byref(prm), ctypes.c_void_p(self.stream.cuda_stream),
                           ctypes.byref(ctx))
        if st != DG_OK:
            raise DGError(st, "dg_init")
        self._ctx = ctx

    # ------------------------------------------------------------------ helpers
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().dg_free(self._ctx)
            self._ctx = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != DG_OK:
            msg = lib().dg_last_error(self._ctx)
            raise DGError(st, f"{what}: {msg.decode() if msg else ''}")

    def _state(self, U, name="U"):
        t = self.torch
        if not isinstance(U, t.Tensor) or U.dtype != t.float64 or not U.is_cuda or not U.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
        if U.numel() != self.numel:
            raise ValueError(f"{name} must have {self.numel} elements")
        return ctypes.c_void_p(U.data_ptr())

    # ------------------------------------------------------------------ solver calls
    def rhs(self, U, Ut=None, t=0.0):
        if Ut is None:
            Ut = self.torch.empty_like(U)
        self._check(lib().dg_rhs(self._ctx, self._state(U), self._state(Ut, "Ut"), float(t)), "dg_rhs")
        return Ut

    def lserk_step(self, U, dt, t=0.0):
        self._check(lib().dg_lserk_step(self._ctx, self._state(U), float(dt), float(t)), "dg_lserk_step")
        return U

    def lserk_steps(self, U, dt, n_steps, t=0.0):
        self._check(lib().dg_lserk_steps(self._ctx, self._state(U), float(dt), float(t), int(n_steps)),
                    "dg_lserk_steps")
        return U

    def lserk_step_host(self, U_host, dt, t=0.0):
        """One step on a host array (numpy float64 or a CPU torch tensor, ideally pinned)."""
        if isinstance(U_host, np.ndarray):
            if U_host.dtype != np.float64 or not U_host.flags.c_contiguous or U_host.size != self.numel:
                raise ValueError("U_host must be a contiguous float64 array of the state's size")
            ptr = U_host.ctypes.data
        else:
            if U_host.dtype != self.torch.float64 or U_host.is_cuda or not U_host.is_contiguous() or \
                    U_host.numel() != self.numel:
                raise ValueError("U_host must be a contiguous float64 CPU tensor of the state's size")
            ptr = U_host.data_ptr()
        self._check(lib().dg_lserk_step_host(self._ctx, ctypes.c_void_p(ptr), float(dt), float(t)),
                    "dg_lserk_step_host")
        return U_host

    # ------------------------------------------------------------------ adjoint
    def rhs_vjp(self, U, lam, Ubar=None, t=0.0):
        """Ubar = (dL/dU)(U)^T lam."""
        if Ubar is None:
            Ubar = self.torch.empty_like(U)
        self._check(lib().dg_rhs_vjp(self._ctx, self._state(U), self._state(lam, "lambda"), self._state(Ubar, "Ubar"),
                                     float(t)), "dg_rhs_vjp")
        return Ubar

    def lserk_step_vjp(self, U, Ubar, dt, t=0.0):
        """In place: Ubar (cotangent after one step from U) -> cotangent of U."""
        self._check(lib().dg_lserk_step_vjp(self._ctx, self._state(U), self._state(Ubar, "Ubar"), float(dt), float(t)),
                    "dg_lserk_step_vjp")
        return Ubar

    def lserk_steps_vjp(self, U0, Ubar, dt, n_steps, interval=10, t=0.0):
        """In place: Ubar (cotangent of U after n_steps from U0) -> cotangent of U0, with checkpoints
        every `interval` steps."""
        self._check(lib().dg_lserk_steps_vjp(self._ctx, self._state(U0), self._state(Ubar, "Ubar"), float(dt),
                                             float(t), int(n_steps), int(interval)), "dg_lserk_steps_vjp")
        return Ubar

    def adjoint_memory_limit(self, nbytes: float = 0.0):
        """Budget for the checkpointed adjoint's state buffers (0: default)."""
        self._check(lib().dg_adjoint_memory_limit(self._ctx, float(nbytes)), "dg_adjoint_memory_limit")

    def lserk_steps_record(self, U, dt, n_steps, interval=10, t=0.0) -> int:
        """Advance U in place by n_steps and record the run for lserk_steps_vjp_recorded; returns
        the tape id."""
        tape = ctypes.c_longlong(0)
        self._check(lib().dg_lserk_steps_record(self._ctx, self._state(U), float(dt), float(t), int(n_steps),
                                                int(interval), ctypes.byref(tape)), "dg_lserk_steps_record")
        return tape.value

    def lserk_steps_vjp_recorded(self, tape: int, Ubar):
        """In place: Ubar (cotangent of the recorded run's final state) -> cotangent of its initial state."""
        self._check(lib().dg_lserk_steps_vjp_recorded(self._ctx, int(tape), self._state(Ubar, "Ubar")),
                    "dg_lserk_steps_vjp_recorded")
        return Ubar

    def tape_current(self) -> int:
        """Id of the recording that lserk_steps_vjp_recorded accepts now (0: none)."""
        tape = ctypes.c_longlong(0)
        self._check(lib().dg_tape_current(self._ctx, ctypes.byref(tape)), "dg_tape_current")
        return tape.value

    def kinetic_energy_grad(self, U, grad=None):
        if grad is None:
            grad = self.torch.empty_like(U)
        self._check(lib().dg_kinetic_energy_grad(self._ctx, self._state(U), self._state(grad, "grad")),
                    "dg_kinetic_energy_grad")
        return grad

    def indicator(self, U, alpha=None):
        if alpha is None:
            alpha = self.torch.empty(self.nE, dtype=self.torch.float64, device=U.device)
        if alpha.dtype != self.torch.float64 or not alpha.is_cuda or alpha.numel() != self.nE:
            raise ValueError("alpha must be a float64 CUDA tensor of n_elems entries")
        self._check(lib().dg_indicator(self._ctx, self._state(U), ctypes.c_void_p(alpha.data_ptr())), "dg_indicator")
        return alpha

    def invariants(self, U, Ut):
        out = np.zeros(8)
        self._check(lib().dg_invariants(self._ctx, self._state(U), self._state(Ut, "Ut"), out.ctypes.data),
                    "dg_invariants")
        return out

    def max_dt(self, U, cfl):
        out = ctypes.c_double(0.0)
        self._check(lib().dg_max_dt(self._ctx, self._state(U), float(cfl), ctypes.byref(out)), "dg_max_dt")
        return out.value

    def check(self):
        self._check(lib().dg_check(self._ctx), "dg_check")

    def metrics(self):
        t = self.torch
        n = self.n
        Ja = t.empty((self.nE, 3, 3, n, n, n), dtype=t.float64, device="cuda")
        J = t.empty((self.nE, n, n, n), dtype=t.float64, device="cuda")
        self._check(lib().dg_get_metrics(self._ctx, ctypes.c_void_p(Ja.data_ptr()), ctypes.c_void_p(J.data_ptr())),
                    "dg_get_metrics")
        return Ja, J

    def use_tma(self, mode=3):
        """FP32-bulk volume kernel: 3 pair-symmetric line kernel (default; N = 7, else mode 2),
        2 warp-specialised node kernel, 1 TMA node kernel, 0 plain node kernel."""
        self._check(lib().dg_use_tma(self._ctx, int(mode)), "dg_use_tma")

    def use_graphs(self, on=True):
        self._check(lib().dg_use_graphs(self._ctx, int(bool(on))), "dg_use_graphs")

    def timing_enable(self, on=True):
        self._check(lib().dg_timing_enable(self._ctx, int(bool(on))), "dg_timing_enable")

    def timing_get(self) -> dict:
        cap = 16
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        cnt = (ctypes.c_longlong * cap)()
        k = lib().dg_timing_get(self._ctx, names, ms, cnt, cap)
        if k < 0:
            raise DGError(-1, "dg_timing_get")
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(k)}

    def launch_count(self) -> int:
        return int(lib().dg_launch_count(self._ctx))
