"""FP64 oracle of the residuals and A-term derivatives used for calibration.

Test infrastructure only: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it; the GPU library never imports it.

The paper names calibration as an application of image domain gridding
(Sect. 6, conclusions): a model is fitted to the data, which needs residuals
and derivatives, and with image domain gridding the free parameters can be the
A-terms themselves, with a full image as the model.  The quantities, in the
notation of Sect. 2 (cost function and its derivative) and Sect. 3.4 (A-terms
as 2 x 2 Jones matrices applied in the image domain):

  model visibilities  y_k(A) = degrid of the model grid with A-terms A
                               (Alg. 2: y_k = sum_pix e_k(pix) A_p B A_q^H,
                               e_k = exp(-2 pi i phi_k), B = taper . P, P the
                               subgrid image from split + inverse transform)
  residuals           r_k = yhat_k - y_k(A) for planned, unflagged k (else 0)
  cost                J(A) = sum_k sum_pol |r_k|^2   (unit weights, Eq. cost
                               function with Sigma = I)
  gradient            G = dJ/dRe(A) + i dJ/dIm(A) for every A-term entry
                               [slot][station][y][x][2 x 2]; for a complex
                               direction E, dJ(A + h E)/dh at 0 = Re sum conj(G) E.

Writing R(pix) = sum_k conj(e_k(pix)) r_k -- the gridder's direct sum of the
residuals with neither taper nor A-terms (Alg. 1 inner loops) -- the chain rule
gives, per subgrid of baseline (p, q) in slot a and per pixel,
  G[a][p] += -2 R A_q B^H        G[a][q] += -2 R^H A_p B
(2 x 2 products).  This module composes the pinned oracle steps (oracle.py) in
that order; tests/test_calibration_cpu.py pins the result to finite
differences of J computed by the oracle's degridder alone.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def _mat(a):
    """[..., 4] polarisations -> [..., 2, 2] matrices [[XX, XY], [YX, YY]]."""
    return a.reshape(a.shape[:-1] + (2, 2))


def planned_unflagged(wl, p: O.OraclePlan, flags=None) -> np.ndarray:
    """bool [n_bl][n_t][n_chan]: visibilities that belong to a subgrid and are not flagged."""
    m = np.zeros((wl.n_bl, wl.n_t, wl.n_chan), dtype=bool)
    for d in p.desc:
        m[d[O.D_BL], d[O.D_T0]:d[O.D_T0] + d[O.D_NT], d[O.D_C0]:d[O.D_C0] + d[O.D_NC]] = True
    f = wl.flags if flags is None else flags
    if f is not None:
        m &= np.asarray(f) == 0
    return m


def residual(wl, p: O.OraclePlan, model_grid, vis, flags=None, aterms="wl", taper=None):
    """Residual visibilities r (complex128, vis-shaped; 0 where not planned or
    flagged) and the cost J = sum |r|^2."""
    y = O.degrid(wl, p, model_grid, flags=flags, aterms=aterms, taper=taper)
    mask = planned_unflagged(wl, p, flags)
    r = np.where(mask[..., None], np.asarray(vis, dtype=np.complex128) - y, 0.0)
    return r, float(np.sum(np.abs(r) ** 2))


def gradient(wl, p: O.OraclePlan, model_grid, vis, flags=None, aterms="wl", taper=None):
    """(r, J, G): residuals, cost and the A-term gradient G [n_slots][n_st][L][L][4]
    (complex128)."""
    A = wl.aterms if isinstance(aterms, str) else aterms
    T = wl.taper if taper is None else taper
    L = wl.subgrid_size
    r, J = residual(wl, p, model_grid, vis, flags, A, T)
    # R: the residuals' direct sum, without taper and A-terms (identity, unit taper)
    R = O.subgrid_images(wl, p, vis=r.astype(np.complex64), flags=flags, aterms=None,
                         taper=np.ones((L, L), dtype=np.float32))
    # B = taper . P, P the model's subgrid images (split, inverse transform)
    P = O.dft2(O.split(wl, p, model_grid), +1)
    B = _mat(P) * np.asarray(T, dtype=np.float64)[None, :, :, None, None]
    Rm = _mat(R)
    G = np.zeros((wl.n_slots, wl.n_stations, L, L, 2, 2), dtype=np.complex128)
    eye = np.broadcast_to(np.eye(2, dtype=np.complex128), (L, L, 2, 2))
    for s, d in enumerate(p.desc):
        a = int(d[O.D_SLOT])
        st_p, st_q = (int(x) for x in wl.baselines[int(d[O.D_BL])])
        Ap = eye if A is None else _mat(np.asarray(A[a, st_p], dtype=np.complex128))
        Aq = eye if A is None else _mat(np.asarray(A[a, st_q], dtype=np.complex128))
        BH = np.conj(np.swapaxes(B[s], -1, -2))
        RH = np.conj(np.swapaxes(Rm[s], -1, -2))
        G[a, st_p] += -2.0 * (Rm[s] @ Aq @ BH)
        G[a, st_q] += -2.0 * (RH @ Ap @ B[s])
    return r, J, G.reshape(wl.n_slots, wl.n_stations, L, L, 4)
