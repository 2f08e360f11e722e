"""FP64 oracle of the anti-aliasing windows (test infrastructure only).

Plain numpy restatements of Sect. 4.1 (the PSWF and its side-lobe energy), Sect. 4.2
(the effective window of image domain gridding, Eq. effective_window) and Sect. 4.3
with the appendix (the optimal window, the smallest eigenvector of Rbar).  They use
methods other than the library's, so that the two check each other:

- lambda_0 of the PSWF comes from a Nystrom discretisation of the time-frequency
  limiting operator (sin c(x - t)) / (pi (x - t)) on [-1, 1] with Gauss-Legendre nodes,
  not from a Legendre expansion.  This holds for beta <= 12: beyond it the operator's
  top eigenvalues are all 1 to FP64 precision, the eigenvector is no longer psi_0, and
  the PSWF functions here refuse such beta;
- Qbar comes from the orthonormality of shifted sincs (the integral of
  sinc(x - k) sinc(x - l) over the whole line is delta_kl), as delta_kl minus the
  main-lobe integral over [0, L) by Gauss-Legendre quadrature, not from the cosine
  integral;
- ``aliasing_from_definition`` evaluates the cost of Eq. error directly: the effective
  window f(x, s) = sum_k a_k exp(i 2 pi k s / L) sinc(x - k) squared, integrated over the
  side lobes (x < 0, x > L, truncated far out) and averaged over the allowed shifts, both
  by quadrature.

Readings (the paper is garbled or silent here): sample k sits at x = k and the main lobe
is [0, L); the allowed shifts are |s| <= (L - beta + 1) / 2; the cost is the continuous
mean over s; a window is scored relative to its total energy sum_k a_k^2, so that eps^2
is the smallest eigenvalue of Rbar for a unit vector.  Only the tests use this module.
"""
from __future__ import annotations

import numpy as np


def _gauss_pieces(lo: float, hi: float, n_per_unit: int = 24):
    """Gauss-Legendre nodes and weights on [lo, hi] with n_per_unit nodes per unit interval."""
    x, w = np.polynomial.legendre.leggauss(n_per_unit)
    edges = np.arange(np.floor(lo), np.ceil(hi) + 1.0)
    xs, ws = [], []
    for a in edges[:-1]:
        a0, b0 = max(a, lo), min(a + 1.0, hi)
        if b0 <= a0:
            continue
        xs.append((x + 1.0) / 2.0 * (b0 - a0) + a0)
        ws.append(w / 2.0 * (b0 - a0))
    return np.concatenate(xs), np.concatenate(ws)


# ---------------------------------------------------------------------------
# Sect. 4.1: the PSWF

_PSWF_BETA_MAX = 12.0


def _check_beta(beta: float):
    if not beta <= _PSWF_BETA_MAX:
        raise ValueError(f"the Nystrom PSWF is reliable for beta <= {_PSWF_BETA_MAX}, got {beta}")


def pswf_lambda0(beta: float, n: int = 200) -> float:
    """First eigenvalue lambda_0(c), c = pi beta / 2, of the operator
    (K psi)(x) = int_{-1}^{1} sin(c (x - t)) / (pi (x - t)) psi(t) dt (Nystrom)."""
    _check_beta(beta)
    c = np.pi * beta / 2.0
    x, w = np.polynomial.legendre.leggauss(n)
    d = x[:, None] - x[None, :]
    with np.errstate(invalid="ignore", divide="ignore"):
        K = np.where(d == 0.0, c / np.pi, np.sin(c * d) / (np.pi * d))
    sw = np.sqrt(w)
    return float(np.linalg.eigvalsh(sw[:, None] * K * sw[None, :])[-1])


def pswf_eps(beta: float) -> float:
    """Side-lobe level of the PSWF as a classical-gridding window: sqrt(1 - lambda_0)."""
    return float(np.sqrt(max(1.0 - pswf_lambda0(beta), 0.0)))


def pswf_window(L: int, beta: float, n: int = 200) -> np.ndarray:
    """psi_0(c, eta) at eta = 2 (x - L/2) / L, x = 0 .. L-1, normalised at x = L/2: the
    Nystrom eigenvector, interpolated with the integral equation itself."""
    _check_beta(beta)
    c = np.pi * beta / 2.0
    t, w = np.polynomial.legendre.leggauss(n)
    d = t[:, None] - t[None, :]
    with np.errstate(invalid="ignore", divide="ignore"):
        K = np.where(d == 0.0, c / np.pi, np.sin(c * d) / (np.pi * d))
    sw = np.sqrt(w)
    lam, U = np.linalg.eigh(sw[:, None] * K * sw[None, :])
    psi_nodes = U[:, -1] / sw                         # eigenfunction at the nodes
    eta = 2.0 * (np.arange(L) - L / 2) / L
    de = eta[:, None] - t[None, :]
    with np.errstate(invalid="ignore", divide="ignore"):
        Ke = np.where(de == 0.0, c / np.pi, np.sin(c * de) / (np.pi * de))
    psi = (Ke * w[None, :]) @ psi_nodes / lam[-1]
    return psi / psi[L // 2]


def pswf_eval(beta: float, eta, n: int = 200) -> np.ndarray:
    """psi_0(c = pi beta / 2, eta) at arbitrary eta in [-1, 1], normalised psi_0(0) = 1
    (the Nystrom eigenvector, interpolated with the integral equation)."""
    _check_beta(beta)
    c = np.pi * beta / 2.0
    t, w = np.polynomial.legendre.leggauss(n)
    d = t[:, None] - t[None, :]
    with np.errstate(invalid="ignore", divide="ignore"):
        K = np.where(d == 0.0, c / np.pi, np.sin(c * d) / (np.pi * d))
    sw = np.sqrt(w)
    lam, U = np.linalg.eigh(sw[:, None] * K * sw[None, :])
    psi_nodes = U[:, -1] / sw
    def interp(e):
        e = np.atleast_1d(np.asarray(e, dtype=np.float64))
        de = e[:, None] - t[None, :]
        with np.errstate(invalid="ignore", divide="ignore"):
            Ke = np.where(de == 0.0, c / np.pi, np.sin(c * de) / (np.pi * de))
        return (Ke * w[None, :]) @ psi_nodes / lam[-1]
    return interp(eta) / interp(0.0)[0]


# ---------------------------------------------------------------------------
# Sect. 4.2-4.3 and the appendix: the optimal window of image domain gridding


def qbar(L: int) -> np.ndarray:
    """Qbar_kl = integral over x outside [0, L) of sinc(x - k) sinc(x - l)."""
    xs, ws = _gauss_pieces(0.0, float(L))
    Phi = np.sinc(xs[:, None] - np.arange(L)[None, :])
    return np.eye(L) - Phi.T @ (ws[:, None] * Phi)


def sbar(L: int, beta: float) -> np.ndarray:
    """Sbar_kl = mean of exp(i 2 pi (k - l) s / L) over |s| <= (L - beta + 1) / 2."""
    W = L - beta + 1.0
    k = np.arange(L)
    return np.sinc((k[:, None] - k[None, :]) * W / L)


def rbar(L: int, beta: float) -> np.ndarray:
    return qbar(L) * sbar(L, beta)


def optimal_window(L: int, beta: float):
    """The window minimising a^T Rbar a / a^T a, normalised a[L/2] = 1, and sqrt of the
    minimum (Eq. a_opt)."""
    lam, U = np.linalg.eigh(rbar(L, beta))
    a = U[:, 0] / U[L // 2, 0]
    return a, float(np.sqrt(max(lam[0], 0.0)))


def aliasing(L: int, beta: float, a) -> float:
    a = np.asarray(a, dtype=np.float64)
    return float(np.sqrt(max(a @ rbar(L, beta) @ a / (a @ a), 0.0)))


def aliasing_from_definition(L: int, beta: float, a, x_far: float = 4000.0, n_s: int = 96,
                             n_per_unit: int = 8) -> float:
    """sqrt of Eq. error for window a, evaluated from the effective window directly:
    mean over s in [-(L - beta + 1)/2, (L - beta + 1)/2] of the energy of
    f(x, s) = sum_k a_k exp(i 2 pi k s / L) sinc(x - k) over x in [-x_far, 0) and
    [L, L + x_far], divided by sum_k a_k^2.  The far side lobes fall off as 1/x^2, so the
    truncation leaves out about |sum_k (-1)^k a_k z_k|^2 / (pi^2 x_far) per side."""
    a = np.asarray(a, dtype=np.float64)
    W = L - beta + 1.0
    sg, swt = np.polynomial.legendre.leggauss(n_s)
    s = sg * W / 2.0
    s_w = swt / 2.0                                    # mean over s: weights sum to 1
    k = np.arange(L)
    total = 0.0
    for lo, hi in ((-x_far, 0.0), (float(L), L + x_far)):
        xs, ws = _gauss_pieces(lo, hi, n_per_unit)
        for c0 in range(0, xs.size, 20000):
            xc, wc = xs[c0:c0 + 20000], ws[c0:c0 + 20000]
            Phi = np.sinc(xc[:, None] - k[None, :]) * a[None, :]          # [x][k]
            Z = np.exp(2j * np.pi * np.outer(k, s) / L)                  # [k][s]
            F = Phi @ Z                                                  # [x][s]
            total += float(np.sum(wc[:, None] * (np.abs(F) ** 2) * s_w[None, :]))
    return float(np.sqrt(total / (a @ a)))
