"""Anti-aliasing windows (Sect. 4.1-4.3, appendix): oracle pins and library parity, no GPU.

Pins of the oracle (``oracle/taper.py``):
- the PSWF column of Table 1 (tests/golden/table1_aliasing.txt), to its three
  printed figures, for beta <= 9 (beyond that 1 - lambda_0 is below FP64 resolution);
- the cost of Eq. error evaluated from its definition (the effective window of
  Eq. effective_window, integrated over the side lobes and averaged over the
  allowed shifts by quadrature) equals the quadratic form of Rbar, for the optimal,
  the PSWF and a random window;
- the image-domain columns of Table 1 within 15 %: the reading used here (continuous
  mean over |s| <= (L - beta + 1) / 2, main lobe [0, L)) comes out 0.5-14 % below the
  printed values, a gap no other reading closes (recorded as an open reading);
- where the table's image-domain level differs from the PSWF level by more than 15 %,
  the same side of the PSWF level (the bold marks of Table 1).
Parity: the library's host functions (closed forms with the sine and cosine integrals,
Jacobi eigensolver, Legendre-expansion PSWF) against the oracle (quadrature, numpy
eigensolver, Nystrom PSWF).
"""
import os

import numpy as np
import pytest

from oracle import taper as OT

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_aliasing.txt")
LS = [8, 16, 24, 32, 48, 64]


def _table1():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows[float(f[0])] = [None if v == "-" else float(v) for v in f[1:]]
    return rows


def _three_figures(x):
    return float(f"{x:.2e}")


@pytest.mark.parametrize("beta", [3.0, 5.0, 7.0, 9.0])
def test_oracle_pswf_matches_table1(beta):
    assert _three_figures(OT.pswf_eps(beta)) == _table1()[beta][0]


def test_oracle_pswf_window_solves_its_integral_equation():
    # psi_0 is an eigenfunction of F psi = int_{-1}^{1} exp(i c x t) psi(t) dt: the ratio
    # (F psi)(x) / psi(x) is the same at every sample point
    L, beta = 32, 7.0
    c = np.pi * beta / 2
    a = OT.pswf_window(L, beta)
    eta = 2.0 * (np.arange(L) - L / 2) / L
    # F psi at the samples from a fine resampling of psi (Riemann sum, error ~ 1 / Lf)
    Lf = 4096
    af = OT.pswf_window(Lf, beta)
    ef = 2.0 * (np.arange(Lf) - Lf / 2) / Lf
    Fpsi = (np.exp(1j * c * np.outer(eta, ef)) * (2.0 / Lf)) @ af
    ratio = Fpsi / a
    mid = np.abs(eta) < 0.8
    assert np.max(np.abs(ratio[mid] - ratio[L // 2])) < 2e-3 * abs(ratio[L // 2])


@pytest.mark.parametrize("L,beta", [(8, 3.0), (16, 5.0), (16, 3.0)])
def test_oracle_rbar_equals_the_definition(L, beta):
    a_opt, _ = OT.optimal_window(L, beta)
    a_psw = OT.pswf_window(L, beta)
    a_rnd = np.random.default_rng(int(L + 10 * beta)).standard_normal(L)
    for a in (a_opt, a_psw, a_rnd):
        e_r = OT.aliasing(L, beta, a)
        e_d = OT.aliasing_from_definition(L, beta, a)
        # the definition leaves out the side lobes beyond 4000 samples (always low)
        assert -2e-3 < e_d / e_r - 1 < 0.0, (e_d, e_r)


@pytest.mark.parametrize("beta", [3.0, 5.0, 7.0, 9.0])
def test_oracle_idg_columns_near_table1(beta):
    row = _table1()[beta]
    pswf = row[0]
    for L, ref in zip(LS, row[1:]):
        if ref is None or L < beta:
            continue
        _, eps = OT.optimal_window(L, beta)
        assert 0.85 * ref < eps <= 1.001 * ref, (L, beta, eps, ref)
        if ref < 0.85 * pswf:
            assert eps < pswf
        if ref > 1.15 * pswf:
            assert eps > pswf


def test_oracle_optimal_window_is_optimal():
    for L, beta in [(16, 5.0), (32, 7.0)]:
        a, eps = OT.optimal_window(L, beta)
        assert abs(OT.aliasing(L, beta, a) / eps - 1) < 1e-9
        rng = np.random.default_rng(3)
        for _ in range(20):
            b = a + 1e-2 * rng.standard_normal(L)
            assert OT.aliasing(L, beta, b) >= eps
        assert OT.aliasing(L, beta, OT.pswf_window(L, beta)) > eps


# ---------------------------------------------------------------------------
# parity: the library's host functions (no GPU needed)

idg = pytest.importorskip("paper_1909_07226_gb300.idg")


@pytest.fixture(scope="module")
def lib():
    try:
        return idg.load()
    except RuntimeError as e:
        pytest.skip(str(e))


@pytest.mark.parametrize("L,beta", [(8, 3.0), (16, 5.0), (24, 7.0), (32, 7.0), (48, 9.0), (64, 9.0)])
def test_library_windows_match_the_oracle(lib, L, beta):
    a, eps = idg.taper_window(L, beta, idg.TAPER_IDG_OPTIMAL)
    oa, oeps = OT.optimal_window(L, beta)
    tol = 1e-7 if beta < 9 else 1e-4
    assert abs(eps / oeps - 1) < tol
    assert np.max(np.abs(a - oa)) < 1e-6
    assert a[L // 2] == 1.0
    assert abs(idg.taper_aliasing(L, beta, a) / eps - 1) < tol
    assert abs(idg.taper_aliasing(L, beta, 3.0 * oa) / OT.aliasing(L, beta, oa) - 1) < tol
    p, peps = idg.taper_window(L, beta, idg.TAPER_PSWF)
    assert np.max(np.abs(p - OT.pswf_window(L, beta))) < 1e-7
    assert abs(peps / OT.pswf_eps(beta) - 1) < (1e-5 if beta < 9 else 1e-3)


@pytest.mark.parametrize("beta", [3.0, 5.0, 7.0, 9.0])
def test_library_pswf_matches_table1(lib, beta):
    _, eps = idg.taper_window(32, beta, idg.TAPER_PSWF)
    assert _three_figures(eps) == _table1()[beta][0]


def test_library_rejects_bad_arguments(lib):
    for L, beta, kind in [(7, 3.0, 1), (0, 3.0, 1), (1024, 3.0, 1), (16, 0.0, 1), (16, 17.5, 1), (16, 5.0, 9),
                          (16, float("nan"), 0)]:
        with pytest.raises(idg.IDGError):
            idg.taper_window(L, beta, kind)
    with pytest.raises(idg.IDGError):
        idg.taper_aliasing(16, 5.0, np.zeros(16))
    # beyond FP64 resolution the optimal window is refused, not returned arbitrary
    with pytest.raises(idg.IDGError):
        idg.taper_window(128, 15.0, idg.TAPER_IDG_OPTIMAL)
    for L in (16, 24, 32, 48, 64):          # beta = 11 (Table 1's last FP64 row) is still served
        idg.taper_window(L, 11.0, idg.TAPER_IDG_OPTIMAL)


def test_library_pswf_beyond_the_oracle_range(lib):
    # beyond beta ~ 12 the Nystrom oracle cannot separate psi_0 (it refuses); the library's
    # Legendre expansion stays consistent: the window decays monotonically from the centre
    # and its classical level 1 - lambda_0 is below FP64 resolution
    with pytest.raises(ValueError):
        OT.pswf_window(64, 15.0)
    a, eps = idg.taper_window(64, 15.0, idg.TAPER_PSWF)
    assert a[32] == 1.0 and np.all(np.diff(a[:33]) > 0) and np.all(np.diff(a[32:]) < 0)
    assert 0.0 <= eps < 1e-7
