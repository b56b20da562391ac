"""Kernel polynomial method in plain FP64 (CPU).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline import this module.  It shares no code with the CUDA library.

Paper references (arXiv 2506.07430):

* Eq. 1 -- absorption spectrum I(w) = sum_n |<n|mu|0>|^2 delta(w_n - w).
* Eq. (kpm) and Eq. (moments) -- Im C(w~) from the Jackson-damped Chebyshev
  series with moments Omega_n = <0| mu T_n(H~) mu |0>.
* Methods, "KPM for absorption spectra": Jackson kernel g_n (Eq. jackson), the
  moments written as <alpha|T_n(H~)|alpha> with |alpha> = mu|0>, the vector
  recursion alpha_0 = alpha, alpha_1 = H~ alpha_0,
  alpha_{n+1} = 2 H~ alpha_n - alpha_{n-1}, and the doubling identities
  Omega_2n = 2<alpha_n|alpha_n> - <alpha_0|alpha_0>,
  Omega_2n+1 = 2<alpha_n+1|alpha_n> - <alpha_1|alpha_0>.

Readings taken where the text is silent or garbled:

* Rescaling (Results, "Resolution of absorption spectra", eigenvalue range
  [a,b] rescaled to [-1,1]): H~ = (H - b)/a with a = half-width and b = centre
  of the (padded) spectral interval.
* Jackson kernel: the printed factor (N-n-1) gives g_0 = (N-1)/(N+1) != 1 and
  breaks the sum rule; the kernel of the cited KPM review has (N-n+1), used here,
  with N the number of moments and n = 0 .. N-1.
* Sign and prefactor of Eq. (kpm): reported as the positive density
  I(x) = (g_0 Omega_0 + 2 sum_{n>=1} g_n Omega_n T_n(x)) / (pi sqrt(1-x^2)),
  i.e. -Im C / pi, whose integral over x is Omega_0; in energy units it is
  I(x)/a at w = a x + b.
* N moments come from N/2 vector steps (alpha_1 .. alpha_{N/2}).
"""
from __future__ import annotations

import numpy as np

__all__ = ["jackson", "lorentz", "moments_recursion", "moments_recursion_block",
           "moments_direct", "moments_cross", "moments_cross_eigen", "moments_eigen",
           "chebyshev_nodes", "spectrum", "spectrum_eigen", "scale_from_bounds"]


def jackson(N: int) -> np.ndarray:
    """Jackson damping factors g_0 .. g_{N-1} (Methods, Eq. jackson, with (N-n+1))."""
    n = np.arange(N, dtype=np.float64)
    q = np.pi / (N + 1)
    return ((N - n + 1) * np.cos(q * n) + np.sin(q * n) / np.tan(q)) / (N + 1)


def lorentz(N: int, lam: float = 4.0) -> np.ndarray:
    """Lorentz damping factors g_n = sinh(lam (1 - n/N)) / sinh(lam), n = 0 .. N-1
    (the KPM review cited in Methods; the paper names modified kernels "like the
    Jackson kernel")."""
    n = np.arange(N, dtype=np.float64)
    return np.sinh(lam * (1.0 - n / N)) / np.sinh(lam)


def scale_from_bounds(emin: float, emax: float, eps: float = 0.01):
    """a, b mapping [emin, emax] into [-1 + eps/2, 1 - eps/2]."""
    a = (emax - emin) / (2.0 - eps)
    b = 0.5 * (emax + emin)
    return a, b


def moments_recursion(apply_h, alpha0: np.ndarray, a: float, b: float, nmoments: int,
                      return_direct: bool = False):
    """Omega_0 .. Omega_{N-1} by the Methods recursion and doubling identities.

    ``apply_h(v)`` returns H v.  With ``return_direct`` also returns the direct
    moments <alpha_0|alpha_n> for n <= N/2 (available without extra H products).
    """
    if nmoments < 2 or nmoments % 2:
        raise ValueError("nmoments must be even and >= 2")
    a0 = np.asarray(alpha0, np.float64)
    a1 = (apply_h(a0) - b * a0) / a                 # alpha_1 = H~ alpha_0
    mu = np.empty(nmoments)
    mu[0] = a0 @ a0
    mu[1] = a1 @ a0
    direct = [mu[0], mu[1]]
    prev, cur = a0, a1
    for n in range(1, nmoments // 2):
        nxt = 2.0 * (apply_h(cur) - b * cur) / a - prev   # alpha_{n+1}
        mu[2 * n] = 2.0 * (cur @ cur) - mu[0]
        mu[2 * n + 1] = 2.0 * (nxt @ cur) - mu[1]
        direct.append(a0 @ nxt)
        prev, cur = cur, nxt
    if return_direct:
        return mu, np.array(direct)
    return mu


def moments_recursion_block(apply_h_block, alpha0, a: float, b: float, nmoments: int):
    """``moments_recursion`` for several start vectors at once (rows of ``alpha0``,
    shape (ncol, dim)); ``apply_h_block(V)`` returns H V row by row.  Every column
    runs the same recursion and doubling identities; returns (ncol, nmoments)."""
    if nmoments < 2 or nmoments % 2:
        raise ValueError("nmoments must be even and >= 2")
    a0 = np.array(alpha0, np.float64, ndmin=2)
    a1 = (apply_h_block(a0) - b * a0) / a
    mu = np.empty((a0.shape[0], nmoments))
    mu[:, 0] = np.einsum("ij,ij->i", a0, a0)
    mu[:, 1] = np.einsum("ij,ij->i", a1, a0)
    prev, cur = a0, a1
    for n in range(1, nmoments // 2):
        nxt = 2.0 * (apply_h_block(cur) - b * cur) / a - prev
        mu[:, 2 * n] = 2.0 * np.einsum("ij,ij->i", cur, cur) - mu[:, 0]
        mu[:, 2 * n + 1] = 2.0 * np.einsum("ij,ij->i", nxt, cur) - mu[:, 1]
        prev, cur = cur, nxt
    return mu


def moments_direct(apply_h, alpha0, a, b, nmoments):
    """Omega_n = <alpha_0|T_n(H~)|alpha_0> with one H product per moment."""
    a0 = np.asarray(alpha0, np.float64)
    out = np.empty(nmoments)
    prev = a0
    out[0] = a0 @ a0
    if nmoments == 1:
        return out
    cur = (apply_h(a0) - b * a0) / a
    out[1] = a0 @ cur
    for n in range(2, nmoments):
        nxt = 2.0 * (apply_h(cur) - b * cur) / a - prev
        out[n] = a0 @ nxt
        prev, cur = cur, nxt
    return out


def moments_cross(apply_h, left: np.ndarray, right: np.ndarray, a: float, b: float,
                  nmoments: int):
    """Omega_n = <left|T_n(H~)|right> (Methods: C_AB moments <0|A T_n(H~) B|0> with
    left = A^dagger|0>, right = B|0>), one H product per moment, no doubling."""
    l = np.asarray(left, np.float64)
    prev = np.asarray(right, np.float64)
    out = np.empty(nmoments)
    out[0] = l @ prev
    if nmoments == 1:
        return out
    cur = (apply_h(prev) - b * prev) / a
    out[1] = l @ cur
    for n in range(2, nmoments):
        nxt = 2.0 * (apply_h(cur) - b * cur) / a - prev
        out[n] = l @ nxt
        prev, cur = cur, nxt
    return out


def moments_cross_eigen(evals, U, left, right, a, b, nmoments):
    """Omega_n = sum_k <left|k><k|right> T_n(E~_k) from eigenpairs (columns of U)."""
    x = (np.asarray(evals) - b) / a
    w = (U.T @ np.asarray(left)) * (U.T @ np.asarray(right))
    n = np.arange(nmoments)
    return (np.cos(np.outer(n, np.arccos(x))) * w[None, :]).sum(axis=1)


def moments_eigen(evals: np.ndarray, weights: np.ndarray, a: float, b: float, nmoments: int):
    """Omega_n = sum_k w_k T_n(E~_k), T_n(x) = cos(n arccos x) (Eq. moments in the eigenbasis)."""
    x = (np.asarray(evals) - b) / a
    if np.any(np.abs(x) > 1.0):
        raise ValueError("spectrum outside [-1, 1] after rescaling")
    th = np.arccos(x)
    n = np.arange(nmoments)
    return (np.cos(np.outer(n, th)) * np.asarray(weights)[None, :]).sum(axis=1)


def chebyshev_nodes(M: int) -> np.ndarray:
    """x_k = cos(pi (k + 1/2) / M), k = 0 .. M-1 (descending)."""
    k = np.arange(M, dtype=np.float64)
    return np.cos(np.pi * (k + 0.5) / M)


def spectrum(moments: np.ndarray, a: float, b: float, npoints: int, kernel: str = "jackson",
             lam: float = 4.0):
    """(omega ascending, density in energy units) by a direct cosine sum; kernel
    "jackson", "lorentz" (parameter lam) or "none".

    I(x_k) = (g_0 Omega_0 + 2 sum_{n>=1} g_n Omega_n cos(n theta_k)) / (pi sin theta_k),
    theta_k = pi (k + 1/2) / M, omega_k = a x_k + b, density = I / a.
    """
    mu = np.asarray(moments, np.float64)
    N = len(mu)
    if kernel == "jackson":
        g = jackson(N)
    elif kernel == "lorentz":
        g = lorentz(N, lam)
    else:
        g = np.ones(N)
    mt = g * mu
    k = np.arange(npoints, dtype=np.float64)
    th = np.pi * (k + 0.5) / npoints
    n = np.arange(N, dtype=np.float64)
    cos = np.cos(np.outer(th, n))
    series = mt[0] + 2.0 * (cos[:, 1:] @ mt[1:])
    dens = series / (np.pi * np.sin(th)) / a
    omega = a * np.cos(th) + b
    order = np.argsort(omega)
    return omega[order], dens[order]


def spectrum_eigen(evals, weights, a, b, nmoments, npoints, kernel="jackson"):
    """Eq. 1 evaluated from exact eigenpairs and broadened by the same kernel:
    sum_k w_k [g_0 + 2 sum_n g_n T_n(E~_k) T_n(x)] / (pi sqrt(1-x^2)) / a."""
    x = chebyshev_nodes(npoints)
    g = jackson(nmoments) if kernel == "jackson" else np.ones(nmoments)
    ek = np.arccos((np.asarray(evals) - b) / a)
    tx = np.arccos(x)
    n = np.arange(nmoments)
    Tk = np.cos(np.outer(n, ek))            # (N, K)
    Tx = np.cos(np.outer(n, tx))            # (N, M)
    coef = g.copy()
    coef[1:] *= 2.0
    series = (Tx * coef[:, None]).T @ (Tk @ np.asarray(weights))
    dens = series / (np.pi * np.sqrt(1.0 - x * x)) / a
    omega = a * x + b
    order = np.argsort(omega)
    return omega[order], dens[order]
