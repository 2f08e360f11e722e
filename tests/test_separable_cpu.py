"""Host-side pins of the separable form (no GPU).

The separable kernels write the phasor of Eq. (ShiftedDirectImaging) as
exp(i (a X + c s(x))) exp(i (b Y + c t(y))) (1 + i c r(x, y)) with
n'(x, y) = s(x) + t(y) + r(x, y).  These tests check, in FP64 numpy and
independently of the library's code, (1) that the factorisation is exact up to
the dropped remainder and that the dropped part obeys the theta^2 / 2 bound the
plan relies on, and (2) that the plan's reported theta equals its definition:
max over planned visibilities of |2 pi (w - w_s)| times max |r|, with the split
through the reference row and column j0 that makes max |r| smallest.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07226_gb300 import synthetic as syn


def _nprime(L, S):
    X = np.arange(L) - L / 2
    l = X * S / L
    m = X * S / L
    ll, mm = np.meshgrid(l, m)            # [y][x]
    return np.sqrt(1.0 - ll * ll - mm * mm) - 1.0


def _split(L, S, j0=None):
    # n' = s(x) + t(y) + r(x, y) through reference row and column j0 (default: the centre)
    j0 = L // 2 if j0 is None else j0
    n1 = _nprime(L, S)
    s = n1[j0, :]                          # row j0: n'(x, j0)
    t = n1[:, j0] - n1[j0, j0]             # column j0, less the shared corner
    r = n1 - s[None, :] - t[:, None]
    return n1, s, t, r


def _best_j0(L, S):
    return min(range(L), key=lambda j: np.abs(_split(L, S, j)[3]).max())


def test_split_reference_off_centre_shrinks_the_remainder():
    # r is about -(l^2 - l0^2)(m^2 - m0^2) / 4: a reference where l0^2 is half the largest
    # l^2 takes max |r| 3 to 4 times below the split through the centre, and the split
    # stays exact
    for L, S in ((32, 0.2), (24, 0.2), (32, 0.5)):
        j0 = _best_j0(L, S)
        n1, s, t, r = _split(L, S, j0)
        np.testing.assert_allclose(s[None, :] + t[:, None] + r, n1, rtol=0, atol=1e-15)
        ratio = np.abs(_split(L, S)[3]).max() / np.abs(r).max()
        assert 3.0 < ratio < 4.5, (L, S, ratio)
        l0 = (j0 - L / 2) * S / L
        assert abs(l0 * l0 - 0.5 * (0.5 * S) ** 2) < 0.25 * (0.5 * S) ** 2


@pytest.mark.parametrize("S,c_max", [(0.04096, 2080.0), (0.128, 700.0), (0.5, 20.0)])
def test_first_order_separable_phasor_error_bound(S, c_max):
    L = 32
    n1, s, t, r = _split(L, S)
    rng = np.random.default_rng(5)
    X = np.arange(L) - L / 2
    for _ in range(20):
        a, b = rng.uniform(-np.pi, np.pi, 2)
        c = rng.uniform(-c_max, c_max)
        exact = np.exp(1j * (a * X[None, :] + b * X[:, None] + c * n1))
        ex = np.exp(1j * (a * X + c * s))
        ey = np.exp(1j * (b * X + c * t))
        sep0 = ey[:, None] * ex[None, :]
        # the zeroth-order factorisation leaves exactly exp(i c r)
        np.testing.assert_allclose(exact, sep0 * np.exp(1j * c * r), rtol=0, atol=1e-12)
        first = sep0 * (1.0 + 1j * c * r)
        theta = abs(c) * np.abs(r).max()
        err = np.abs(first - exact).max()
        assert err <= 0.5 * theta ** 2 * (1 + 1e-9) + 1e-14


def test_remainder_is_fourth_order_in_the_direction_cosines():
    # r = -l^2 m^2 / 4 + O(6th order): halving the field shrinks it 16x
    L = 32
    r1 = np.abs(_split(L, 0.04)[3]).max()
    r2 = np.abs(_split(L, 0.02)[3]).max()
    assert 15.5 < r1 / r2 < 16.5


def _theta_definition(wl):
    # per subgrid: |2 pi (w - w_s)| max |r| with w_s = the subgrid's w offset w0 when
    # that gives a phase within the bound, else the middle of the subgrid's own w range;
    # the plan's phase is the largest, and the subgrids within the bound (with their
    # K_p) are the ones the separable kernels take
    op = O.plan(wl)
    L, S = wl.subgrid_size, wl.grid_size * wl.cell_size
    r_max = np.abs(_split(L, S, _best_j0(L, S))[3]).max()
    c = 299792458.0
    theta, n_sep, kp_sep = 0.0, 0, 0
    for row in op.desc:
        bl, t0, nt, c0, nc = row[O.D_BL], row[O.D_T0], row[O.D_NT], row[O.D_C0], row[O.D_NC]
        w0 = (row[O.D_LAYER] + op.k_min) * wl.w_step if wl.w_step > 0 else 0.0
        w = wl.uvw_m[bl, t0:t0 + nt, 2][:, None] * wl.freqs_hz[None, c0:c0 + nc] / c
        th = 2 * np.pi * np.abs(w - w0).max() * r_max
        if th > 1.38e-3:
            th = 2 * np.pi * 0.5 * (w.max() - w.min()) * r_max
        theta = max(theta, th)
        if th <= 1.38e-3:
            n_sep += 1
            kp_sep += int(row[O.D_KP])
    return theta, n_sep, kp_sep


@pytest.mark.parametrize("kw", [dict(), dict(w_step=20.0, diameter_m=20000.0, n_t=24, max_t=12),
                                dict(N=256, cell=5e-4, diameter_m=800.0), dict(N=256, cell=1e-3, diameter_m=300.0),
                                dict(N=512, cell=1e-3, diameter_m=800.0), dict(N=512, cell=8e-4, diameter_m=800.0)])
def test_plan_reports_the_remainder_phase(kw):
    from paper_1909_07226_gb300 import idg
    args = dict(seed=1032, n_st=5, n_t=48, n_chan=5, L=32, N=128, max_t=48, n_slots=1, flag_p=0.1,
                diameter_m=3000.0)
    args.update(kw)
    wl = syn.make_small(**args)
    p = idg.plan_from_workload(wl)
    want, n_sep, kp_sep = _theta_definition(wl)
    assert p.stats.sep_phase == pytest.approx(want, rel=1e-9, abs=1e-15)
    assert p.stats.separable == (1 if want <= 1.38e-3 else 0)
    assert (p.stats.n_sep_subgrids, p.stats.n_vis_sep) == (n_sep, kp_sep)
    assert p.stats.separable == (1 if n_sep == p.n_subgrids else 0)


def _pieces_definition(wl):
    # subgrids outside the bound: the smallest kt x kc grid of equal blocks of their
    # timesteps and channels (floor cuts) whose blocks each meet the bound with the
    # block's own middle w, if it has at most (rho_L - 1) K_p / F_L blocks
    op = O.plan(wl)
    L, S = wl.subgrid_size, wl.grid_size * wl.cell_size
    r_max = np.abs(_split(L, S, _best_j0(L, S))[3]).max()
    rho = {32: 3.8, 24: 2.7, 16: 1.0}[L]
    F = 200.0 * (L / 32.0) ** 2
    c = 299792458.0
    n_split = n_pieces = kp_split = 0
    for row in op.desc:
        bl, t0, nt, c0, nc, kp = (int(row[i]) for i in (O.D_BL, O.D_T0, O.D_NT, O.D_C0, O.D_NC, O.D_KP))
        w0 = (row[O.D_LAYER] + op.k_min) * wl.w_step if wl.w_step > 0 else 0.0
        w = wl.uvw_m[bl, t0:t0 + nt, 2][:, None] * wl.freqs_hz[None, c0:c0 + nc] / c
        th = 2 * np.pi * np.abs(w - w0).max() * r_max
        if th > 1.38e-3:
            th = 2 * np.pi * 0.5 * (w.max() - w.min()) * r_max
        if th <= 1.38e-3:
            continue
        max_pieces = min(int((rho - 1.0) * kp / F), nt * nc)
        found = 0
        for prod in range(2, max_pieces + 1):
            for kt in range(1, min(nt, prod) + 1):
                kc = prod // kt
                if prod % kt or kc > nc:
                    continue
                blocks = [w[i * nt // kt:(i + 1) * nt // kt, j * nc // kc:(j + 1) * nc // kc]
                          for i in range(kt) for j in range(kc)]
                if all(2 * np.pi * 0.5 * (b.max() - b.min()) * r_max <= 1.38e-3 for b in blocks):
                    found = prod
                    break
            if found:
                break
        if found:
            n_split += 1
            n_pieces += found
            kp_split += kp
    return n_split, n_pieces, kp_split


@pytest.mark.parametrize("kw", [dict(N=512, cell=8e-4, diameter_m=800.0), dict(N=512, cell=8e-4, diameter_m=300.0),
                                dict(L=24, N=384, cell=8e-4, diameter_m=800.0, n_t=96, max_t=96, n_chan=12),
                                dict(L=16, N=256, cell=1.2e-3, diameter_m=800.0, n_t=96, max_t=96, n_chan=12),
                                dict(w_step=5.0, N=512, cell=8e-4, diameter_m=800.0)])
def test_plan_splits_subgrids_outside_the_bound_into_pieces(kw):
    from paper_1909_07226_gb300 import idg
    args = dict(seed=1032, n_st=5, n_t=48, n_chan=5, L=32, N=128, max_t=48, n_slots=1, flag_p=0.1,
                diameter_m=3000.0, df=0.25e6)
    args.update(kw)
    wl = syn.make_small(**args)
    p = idg.plan_from_workload(wl)
    s = p.stats
    assert (s.n_split_subgrids, s.n_pieces, s.n_vis_split) == _pieces_definition(wl)
    assert s.n_sep_subgrids + s.n_split_subgrids <= p.n_subgrids
    assert s.n_vis_sep + s.n_vis_split <= s.n_vis_planned


def test_mixed_plan_splits_its_subgrids():
    # a wide field where only the subgrids of small w spread meet the bound: some, not
    # all, go to the separable kernels
    from paper_1909_07226_gb300 import idg
    wl = syn.make_small(seed=1032, n_st=5, n_t=48, n_chan=5, L=32, N=512, max_t=48, n_slots=1, flag_p=0.1,
                        diameter_m=800.0, cell=8e-4)
    p = idg.plan_from_workload(wl)
    _, n_sep, kp_sep = _theta_definition(wl)
    assert 0 < n_sep < p.n_subgrids
    assert p.stats.separable == 0 and p.stats.n_sep_subgrids == n_sep and 0 < p.stats.n_vis_sep < p.stats.n_vis_planned


def _fma32(a, b, c):
    # fused multiply-add rounded once to FP32: a b of two FP32 values is exact in FP64,
    # and here the sum with c is too (the operands lie within 2^29 of each other)
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _pair(x):
    hi = np.float32(x)
    return hi, np.float32(x - np.float64(hi))


def _pair_coef(xh, xl, sh, sl, oh, ol):
    # restatement of the kernels' float-pair coefficient: two-product by fma, then
    # Knuth's two-sum of p and -oh, the small terms added, one final rounding
    f = np.float32
    p = f(xh * sh)
    e = _fma32(xh, sh, -p)
    e = _fma32(xh, sl, e)
    e = _fma32(xl, sh, e)
    s = f(p - oh)
    bb = f(s - p)
    err = f(f(p - f(s - bb)) + f(-oh - bb))
    return f(s + f(err + f(e - ol)))


def test_float_pair_coefficients_match_fp64_rounded_once():
    """The kernels form a = u (f/c) k_uv - u0 k_uv without FP64 instructions, from
    float pairs.  Over LOFAR-scale magnitudes (|u (f/c) k_uv| up to ~300 rad on a
    4096-pixel grid with 32-pixel subgrids, |a| <= pi) the result is the FP64 value
    correctly rounded to FP32 (within half an ulp, up to the ~2^-48 terms left out),
    where a single FP32 product and difference would be off by up to ~1e-4 rad."""
    rng = np.random.default_rng(7)
    k_uv = 2 * np.pi * 0.05 / 32
    worst_ulps, worst_naive = 0.0, 0.0
    for _ in range(4000):
        u = rng.uniform(-1.0e5, 1.0e5)                     # metres
        fc = rng.uniform(120e6, 190e6) / 299792458.0       # f / c
        u_lambda = u * fc
        u0 = np.round(u_lambda * k_uv / 0.1) * 0.1 / k_uv + rng.uniform(-1, 1) / k_uv
        exact = u_lambda * k_uv - u0 * k_uv
        uh, ul = _pair(u)
        sh, sl = _pair(fc * k_uv)
        oh, ol = _pair(u0 * k_uv)
        got = _pair_coef(uh, ul, sh, sl, oh, ol)
        ulp = np.spacing(np.float32(abs(exact))) if exact != 0 else np.float32(1e-45)
        worst_ulps = max(worst_ulps, abs(np.float64(got) - exact) / np.float64(ulp))
        naive = np.float32(np.float32(np.float32(u) * np.float32(fc * k_uv)) - np.float32(u0 * k_uv))
        worst_naive = max(worst_naive, abs(np.float64(naive) - exact))
    assert worst_ulps <= 0.51, worst_ulps
    assert worst_naive > 1e-5          # the plain FP32 route would not do
