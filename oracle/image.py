"""FP64 oracle of the image-side steps (test infrastructure only).

Alg. 1 last line and Alg. 2 first lines, with the W-layers of Sect. 3.5 and the
effective window of Sect. 4.2:
  image(x, y) = sum_k exp(+2 pi i w0_k n'(x, y)) centred_idft(G_k)(x, y) / (cbar(x) cbar(y)),
  G_k = centred_dft(image exp(-2 pi i w0_k n') / (conj cbar(x) conj cbar(y))),
both un-normalised, with pixel (x, y) at l = (x - N/2) S / N, m = (y - N/2) S / N and
w0_k = (k + k_min) w_step.  cbar is the effective window at zero shift of the 1D window
a: cbar(x) = L^-1 sum_j a_j sum_{m=-L/2}^{L/2-1} exp(2 pi i m (xi_x - xi_j)), xi_x = (x - N/2)/N,
xi_j = (j - L/2)/L, written out as the double sum.  The transforms use numpy's FFT as a
step, with the centring shifts of the definition.  Only the tests use this module.
"""
from __future__ import annotations

import numpy as np


def effective_window(a, L: int, N: int) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    xi = (np.arange(N) - N / 2) / N
    xj = (np.arange(L) - L / 2) / L
    m = np.arange(-L // 2, L // 2)
    ph = np.exp(2j * np.pi * m[None, None, :] * (xi[:, None, None] - xj[None, :, None]))   # [x][j][m]
    return (ph.sum(axis=2) @ a) / L


def centred_idft2(G: np.ndarray) -> np.ndarray:
    """sum_{q,r} G[r][q] exp(+2 pi i ((q - N/2)(x - N/2) + (r - N/2)(y - N/2)) / N), per pol."""
    N = G.shape[0]
    return np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(G, axes=(0, 1)), axes=(0, 1)), axes=(0, 1)) * N * N


def centred_dft2(I: np.ndarray) -> np.ndarray:
    """sum_{x,y} I[y][x] exp(-2 pi i ((q - N/2)(x - N/2) + (r - N/2)(y - N/2)) / N), per pol."""
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(I, axes=(0, 1)), axes=(0, 1)), axes=(0, 1))


def nprime(N: int, S: float) -> np.ndarray:
    l = (np.arange(N) - N / 2) * S / N
    r2 = l[None, :] ** 2 + l[:, None] ** 2
    return np.sqrt(1.0 - r2) - 1.0


def image_from_grid(grid: np.ndarray, S: float, w0s, window, L: int) -> np.ndarray:
    """grid [n_w][N][N][4] -> image [N][N][4] (complex128)."""
    N = grid.shape[1]
    npr = nprime(N, S)
    out = np.zeros(grid.shape[1:], dtype=np.complex128)
    for k, w0 in enumerate(w0s):
        out += centred_idft2(grid[k].astype(np.complex128)) * np.exp(2j * np.pi * w0 * npr)[:, :, None]
    if window is not None:
        cb = effective_window(window, L, N)
        out /= (cb[None, :] * cb[:, None])[:, :, None]
    return out


def grid_from_image(image: np.ndarray, S: float, w0s, window, L: int) -> np.ndarray:
    """image [N][N][4] -> grid [n_w][N][N][4] (complex128), the adjoint of image_from_grid."""
    N = image.shape[0]
    npr = nprime(N, S)
    img = image.astype(np.complex128)
    if window is not None:
        cb = np.conj(effective_window(window, L, N))
        img = img / (cb[None, :] * cb[:, None])[:, :, None]
    return np.stack([centred_dft2(img * np.exp(-2j * np.pi * w0 * npr)[:, :, None]) for w0 in w0s])
