"""Closed-form and independent reference solutions used to pin the oracle.

Nothing here calls the oracle or the CUDA path: these are textbook solutions
of the macroscopic equations the method recovers (Eqs. 2-3, 28, 41, 10)."""
from __future__ import annotations

import math

import numpy as np


def stefan_kappa(St: float) -> float:
    """Root of kappa exp(kappa^2) erf(kappa) = St / sqrt(pi): one-phase Neumann
    melting problem (liquid heated at x = 0, solid held at the melting point)."""
    lo, hi = 1e-12, 5.0
    target = St / math.sqrt(math.pi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid * math.exp(mid * mid) * math.erf(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def neumann_two_phase(St_l: float, St_s: float, nu: float) -> float:
    """Root lambda of the two-phase Neumann melting problem: liquid heated at
    x = 0 (Stefan number St_l = c_l (T_w - T_m)/L), subcooled solid far away
    (St_s = c_s (T_m - T_i)/L), nu = sqrt(alpha_l/alpha_s); the front is at
    s = 2 lambda sqrt(alpha_l t).  The interface balance reads
    lambda sqrt(pi) = St_l exp(-lambda^2)/erf(lambda)
                      - St_s exp(-nu^2 lambda^2)/(nu erfc(nu lambda))."""
    def resid(lam):
        return (St_l * math.exp(-lam * lam) / math.erf(lam)
                - St_s * math.exp(-nu * nu * lam * lam) / (nu * math.erfc(nu * lam)) - lam * math.sqrt(math.pi))
    lo, hi = 1e-9, 5.0          # resid(lo) > 0 > resid(hi); resid decreases
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if resid(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def brinkman_channel(x, H, G, K, nu_f, nu_e, phi):
    """Steady unidirectional flow between no-slip walls at x = 0 and x = H under a
    uniform body acceleration G, Forchheimer term off:
    nu_e u'' - phi nu_f u / K + phi G = 0."""
    r = math.sqrt(phi * nu_f / (nu_e * K))
    return G * K / nu_f * (1.0 - np.cosh(r * (x - H / 2.0)) / np.cosh(r * H / 2.0))


def forchheimer_channel_fd(H, G, K, nu_f, nu_e, phi, F_phi, refine=32):
    """Same channel with the Forchheimer term, solved by second-order finite
    differences on a grid ``refine`` times finer and Newton iteration:
    nu_e u'' - phi nu_f u/K - phi F_phi |u| u / sqrt(K) + phi G = 0.
    Returns u at the integer abscissae 0..H."""
    M = int(round(H)) * refine + 1
    xs = np.linspace(0.0, H, M)
    h = xs[1] - xs[0]
    u = np.zeros(M)
    a = phi * nu_f / K
    b = phi * F_phi / math.sqrt(K)
    for _ in range(60):
        R = np.zeros(M)
        R[1:-1] = nu_e * (u[2:] - 2 * u[1:-1] + u[:-2]) / h ** 2 - a * u[1:-1] - b * np.abs(u[1:-1]) * u[1:-1] + phi * G
        J = np.zeros((M, M))
        i = np.arange(1, M - 1)
        J[i, i - 1] = nu_e / h ** 2
        J[i, i + 1] = nu_e / h ** 2
        J[i, i] = -2 * nu_e / h ** 2 - a - 2 * b * np.abs(u[1:-1])
        J[0, 0] = J[-1, -1] = 1.0
        R[0], R[-1] = u[0], u[-1]
        du = np.linalg.solve(J, -R)
        u += du
        if np.abs(du).max() < 1e-18:
            break
    return u[::refine]


def mode_amplitude(v: np.ndarray, k: float) -> float:
    """Amplitude of the Fourier mode of wavenumber k in a periodic 1-D signal."""
    n = v.size
    x = np.arange(n)
    w = v - v.mean()
    return 2.0 / n * math.hypot(float((w * np.sin(k * x)).sum()), float((w * np.cos(k * x)).sum()))
