"""FP64 oracle of classical gridding with oversampled A/W-projection kernels.

Test infrastructure only (tests, smoke check, CPU-baseline leg of the bench);
the GPU library never imports it.  This is the gridding the paper compares
image domain gridding against (Sect. 2: gridding with a convolution kernel,
oversampled kernels, W-projection and A-projection), on the same plan,
visibilities and grid layout as the library:

* Window of a kernel (Sect. 2, A-projection): per image pixel of an M x M
  lattice over the image, l_x = (x - M/2) S / M (the pixel positions of
  reading 1 with M in place of L), the 2 x 2 operator of the gridding
  direction X -> b(l, m) exp(2 pi i w n'(l, m)) A_p(l, m)^H X A_q(l, m) as a
  4 x 4 matrix on the polarisations (Mueller form):
      c[(i, j), (a, b)] = b exp(2 pi i w n') conj(A_p[a][i]) A_q[b][j].
* Kernel: the window zero-padded to MO x MO and Fourier transformed (Sect. 2,
  C = F(Z(c))), i.e. for a uv offset delta (pixels)
      C(delta_v, delta_u) = M^-2 sum_{y,x} c[y][x] exp(-2 pi i (delta_u (x - M/2) + delta_v (y - M/2)) / M)
  sampled at delta = integer + multiple of 1/O.
* Gridding: for visibility k at grid position pu = (u f/c) S + N/2 (and pv),
  the support is the M grid pixels q = floor(pu) - M/2 + 1 .. floor(pu) + M/2,
  each with the kernel at the offset q - pu rounded to the nearest 1/O (the
  oversampled table lookup): o = floor(frac(pu) O + 1/2), offset
  d - M/2 + 1 - o / O for support index d (o = O moves to the next pixel).
  grid[layer][r][q] += C . y_k (the 4 x 4 kernel on the 4 polarisations);
  support pixels outside the grid are dropped.
* W-projection: with a plane spacing dw > 0 the window of visibility k uses
  w = j dw, j = floor((w_k - w0) / dw + 1/2), w0 the plan's layer offset of
  its subgrid (so the plan's W-layers act as W-stacking); dw = 0 puts no w-term
  in the kernels (A-projection only).
Kernels belong to (subgrid, j): recomputed for every subgrid, i.e. for every
A-term slot, which is the cost the paper's method avoids.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

C_LIGHT = 299792458.0


def lattice(M: int, S: float):
    """l[y][x], m[y][x], n'[y][x] of the M x M lattice over an image of width S."""
    c = (np.arange(M, dtype=np.float64) - 0.5 * M) * S / M
    l = np.broadcast_to(c[None, :], (M, M))
    m = np.broadcast_to(c[:, None], (M, M))
    return l, m, np.sqrt(1.0 - l * l - m * m) - 1.0


def mueller_window(M: int, S: float, taper, Ap=None, Aq=None, w: float = 0.0) -> np.ndarray:
    """c[y][x][4][4]: the gridding-direction operator b e^{2 pi i w n'} A_p^H X A_q
    as a matrix on vec(X) = (XX, XY, YX, YY).  Ap, Aq: [M][M][4] or None (identity)."""
    _, _, n1 = lattice(M, S)
    s = np.asarray(taper, dtype=np.float64) * np.exp(2j * np.pi * w * n1)
    eye = np.broadcast_to(np.eye(2, dtype=np.complex128), (M, M, 2, 2))
    P = eye if Ap is None else np.asarray(Ap, dtype=np.complex128).reshape(M, M, 2, 2)
    Q = eye if Aq is None else np.asarray(Aq, dtype=np.complex128).reshape(M, M, 2, 2)
    out = np.zeros((M, M, 4, 4), dtype=np.complex128)
    for i in range(2):
        for j in range(2):
            for a in range(2):
                for b in range(2):
                    out[:, :, 2 * i + j, 2 * a + b] = s * np.conj(P[:, :, a, i]) * Q[:, :, b, j]
    return out


def kernel_table(win: np.ndarray, O_: int) -> np.ndarray:
    """[O][O][M][M][...]: the window zero-padded to MO x MO and transformed; entry
    (oy, ox, dy, dx) is the kernel at offset (dy - M/2 + 1 - oy/O, dx - M/2 + 1 - ox/O)."""
    M = win.shape[0]
    MO = M * O_
    Z = np.zeros((MO, MO) + win.shape[2:], dtype=np.complex128)
    idx = (np.arange(M) - M // 2) % MO
    Z[np.ix_(idx, idx)] = win
    F = np.fft.fft2(Z, axes=(0, 1)) / (M * M)
    o = np.arange(O_)
    d = np.arange(M)
    n = (O_ * (d[None, :] - M // 2 + 1) - o[:, None]) % MO          # [o][d]
    return F[n[:, None, :, None], n[None, :, None, :]]


def kernel_at(win: np.ndarray, dv: float, du: float) -> np.ndarray:
    """The kernel of window win at an arbitrary offset (direct sum of its definition)."""
    M = win.shape[0]
    x = np.arange(M) - 0.5 * M
    ex = np.exp(-2j * np.pi * du * x / M)
    ey = np.exp(-2j * np.pi * dv * x / M)
    return np.einsum("y,x,yx...->...", ey, ex, win) / (M * M)


def _position(u_m: float, s: float, S: float, N: int, O_: int):
    """Support start and oversampled phase of one coordinate (FP64, no fused ops)."""
    pu = (u_m * s) * S + 0.5 * N
    iq = float(np.floor(pu))
    o = int(np.floor((pu - iq) * O_ + 0.5))
    if o == O_:
        iq += 1.0
        o = 0
    return pu, int(iq), o


def w_plane(w_m: float, s: float, w0: float, dw: float) -> int:
    """W-projection plane of a visibility: floor((w f/c - w0) / dw + 1/2)."""
    if dw <= 0.0:
        return 0
    return int(np.floor(((w_m * s) - w0) / dw + 0.5))


def grid(wl, p: O.OraclePlan, M: int, O_: int, dw: float = 0.0, aterms=None, taper=None, vis=None, flags=None,
         ids=None, exact: bool = False) -> np.ndarray:
    """Classical gridding of the plan's visibilities (subgrids `ids`, default all)
    into [n_w][N][N][4] (complex128).  aterms [n_slots][n_st][M][M][4] or None
    (identity); taper [M][M] (window b on the kernel lattice).  exact=True
    evaluates each kernel at the visibility's exact offsets from the same support
    pixels and (with dw > 0) at its exact w instead of its plane's: the
    continuous-kernel reference of the oversampled lookup."""
    N, S = wl.grid_size, wl.grid_size * wl.cell_size
    V = wl.vis if vis is None else vis
    F = wl.flags if flags is None else flags
    b = np.ones((M, M)) if taper is None else np.asarray(taper, dtype=np.float64)
    out = np.zeros((p.n_w, N, N, 4), dtype=np.complex128)
    sel = range(p.n_sub) if ids is None else ids
    for sid in sel:
        d = p.desc[sid]
        bl, slot, t0, nt, c0, nc, layer = (int(d[k]) for k in (O.D_BL, O.D_SLOT, O.D_T0, O.D_NT, O.D_C0, O.D_NC,
                                                                 O.D_LAYER))
        w0 = (layer + p.k_min) * wl.w_step if wl.w_step > 0 else 0.0
        pst, qst = (int(x) for x in wl.baselines[bl])
        Ap = None if aterms is None else aterms[slot, pst]
        Aq = None if aterms is None else aterms[slot, qst]
        tables = {}
        for t in range(t0, t0 + nt):
            u, v, w = (float(x) for x in wl.uvw_m[bl, t])
            for c in range(c0, c0 + nc):
                if F is not None and F[bl, t, c]:
                    continue
                s = float(wl.freqs_hz[c]) / C_LIGHT
                y = np.asarray(V[bl, t, c], dtype=np.complex128)
                pu, iq, ox = _position(u, s, S, N, O_)
                pv, ir, oy = _position(v, s, S, N, O_)
                if exact:
                    win = mueller_window(M, S, b, Ap, Aq, ((w * s) - w0) if dw > 0.0 else 0.0)
                    dd = np.arange(M) - M // 2 + 1
                    blk = np.array([[kernel_at(win, float(ir + dy) - pv, float(iq + dx) - pu) for dx in dd]
                                    for dy in dd])
                else:
                    j = w_plane(w, s, w0, dw)
                    if j not in tables:
                        tables[j] = kernel_table(mueller_window(M, S, b, Ap, Aq, j * dw), O_)
                    blk = tables[j][oy, ox]
                contrib = blk @ y                                           # [M][M][4]
                rows = ir - M // 2 + 1 + np.arange(M)
                cols = iq - M // 2 + 1 + np.arange(M)
                rm = (rows >= 0) & (rows < N)
                cm = (cols >= 0) & (cols < N)
                out[layer, rows[rm][:, None], cols[cm][None, :]] += contrib[rm][:, cm]
    return out
