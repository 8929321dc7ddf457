"""Shared test helpers: the parity metric and magnitude scales (no method arithmetic)."""
import numpy as np


def euler_flux_magnitude(U, Ja, gamma=1.4):
    """Per node and variable: sum_d (|F^d_v(U)| + c |Ja^d| |U_v|) with F^d the contravariant Euler
    flux and c the sound speed -- the size of the advective and dissipative flux terms the
    right-hand side differences (numpy, vectorised)."""
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
            out[:, v] += np.abs(F[v]) + c * s * np.abs(U[:, v])
    return out


def flux_scale(U, Ja, J, D, gamma=1.4):
    """scale_v = max over nodes of ||2D||_inf * sum_d |F^d_v(U)| / J: the size of the largest
    flux-difference sum in the right-hand side, on which FP64 rounding acts."""
    mag = euler_flux_magnitude(U, Ja, gamma) / J[:, None]
    d2 = 2.0 * np.abs(D).sum(1).max()
    return d2 * mag.reshape(mag.shape[0], 5, -1).max(axis=(0, 2))


def parity(Ut, Ut_ref, scale):
    """max |Ut - Ut_ref| per variable divided by the flux scale."""
    diff = np.abs(np.asarray(Ut) - np.asarray(Ut_ref)).reshape(Ut.shape[0], 5, -1).max(axis=(0, 2))
    return diff / scale


def normwise(Ut, Ut_ref):
    """max |Ut - Ut_ref| / max |Ut_ref| per variable (informational)."""
    d = np.abs(np.asarray(Ut) - np.asarray(Ut_ref)).reshape(Ut.shape[0], 5, -1).max(axis=(0, 2))
    r = np.abs(np.asarray(Ut_ref)).reshape(Ut.shape[0], 5, -1).max(axis=(0, 2))
    return d / np.maximum(r, 1e-300)
