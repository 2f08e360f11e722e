"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formulas: each check computes its
expected value by a different route (a closed form, an exact identity of the
algorithm, a library routine, or an invariant), chosen so that a dropped term,
a wrong sign, an index slip or a transposed operand in the oracle fails at
least one of them.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07226_gb300 import synthetic as syn

C = syn.C_LIGHT


def rel_err(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def vis_pixels(wl):
    """Grid pixel coordinates of every visibility: pu = u/lambda * S + N/2 (Eq. 2, Sect. 2)."""
    S = wl.grid_size * wl.cell_size
    sc = wl.freqs_hz / C
    pu = (wl.uvw_m[:, :, None, 0] * sc[None, None, :]) * S + wl.grid_size / 2
    pv = (wl.uvw_m[:, :, None, 1] * sc[None, None, :]) * S + wl.grid_size / 2
    ww = wl.uvw_m[:, :, None, 2] * sc[None, None, :]
    return pu, pv, ww


# --------------------------------------------------------------------------
# plan (Sect. 3.2)


def test_tiny_config_has_112_subgrids():
    # The tiny workload (28 baselines x 64 timesteps, 16 timesteps per subgrid)
    # partitions into 28 * 4 = 112 subgrids of 16 timesteps x 8 channels.
    wl = syn.make_tiny(with_vis=False)
    p = O.plan(wl)
    assert p.n_sub == 112
    assert p.n_dropped == 0
    assert np.all(p.desc[:, O.D_NT] == 16) and np.all(p.desc[:, O.D_NC] == 8)
    assert np.all(p.desc[:, O.D_KP] == 128)


@pytest.mark.parametrize("kw", [
    dict(seed=1, n_st=7, n_t=40, n_chan=6, L=16, N=64, diameter_m=20000.0, max_t=12),
    dict(seed=2, n_st=5, n_t=30, n_chan=9, L=24, N=96, diameter_m=60000.0, max_t=30, n_slots=3),
    dict(seed=3, n_st=6, n_t=20, n_chan=5, L=16, N=128, w_step=40.0, max_t=20),
    # cell chosen so that long baselines fall off the grid and are dropped
    dict(seed=4, n_st=6, n_t=20, n_chan=4, L=16, N=64, cell=6e-4, diameter_m=8000.0),
])
def test_plan_invariants(kw):
    wl = syn.make_small(with_vis=False, aterms="identity", **kw)
    p = O.plan(wl)
    L, N = wl.subgrid_size, wl.grid_size
    smax = (L - wl.kernel_size + 1) / 2
    pu, pv, ww = vis_pixels(wl)
    owner = -np.ones((wl.n_bl, wl.n_t, wl.n_chan), dtype=np.int64)
    prev = None
    for i, d in enumerate(p.desc):
        b, a, t0, nt, c0, nc, q0, r0, layer, kp = (int(x) for x in d)
        assert kp == nt * nc and 1 <= nt <= wl.max_timesteps
        # one A-term slot per subgrid (Sect. 3.4: a single c_p per block)
        assert wl.aterm_offsets[a] <= t0 and t0 + nt <= wl.aterm_offsets[a + 1]
        assert 0 <= q0 and q0 + L <= N and 0 <= r0 and r0 + L <= N
        sl = (b, slice(t0, t0 + nt), slice(c0, c0 + nc))
        assert np.all(owner[sl] == -1), "visibility assigned twice"
        owner[sl] = i
        # every sample within the allowed shift of the subgrid centre (Sect. 4.3)
        cu, cv = q0 + L // 2, r0 + L // 2
        assert np.max(np.abs(pu[sl] - cu)) <= smax
        assert np.max(np.abs(pv[sl] - cv)) <= smax
        # the centre pixel is the midpoint of the block's extent rounded half up
        assert cu == math.floor(0.5 * (pu[sl].min() + pu[sl].max()) + 0.5)
        assert cv == math.floor(0.5 * (pv[sl].min() + pv[sl].max()) + 0.5)
        if wl.w_step > 0:
            w0 = (layer + p.k_min) * wl.w_step
            assert np.max(ww[sl]) - np.min(ww[sl]) <= wl.w_step
            assert np.max(np.abs(ww[sl] - w0)) <= wl.w_step
        key = (b, a)
        if prev is not None:
            assert key >= prev
        prev = key
    # everything not assigned was counted as dropped, and a dropped sample really
    # cannot be centred in an in-grid subgrid
    assert int(np.sum(owner < 0)) == p.n_dropped
    if p.n_dropped:
        off = owner < 0
        cu = np.floor(pu[off] + 0.5)
        cv = np.floor(pv[off] + 0.5)
        inside = (cu - L / 2 >= 0) & (cu + L / 2 <= N) & (cv - L / 2 >= 0) & (cv + L / 2 <= N)
        # a dropped single sample may only be inside if its channel group was off-grid
        assert np.sum(~inside) > 0
    assert int(np.sum(p.desc[:, O.D_KP])) + p.n_dropped == wl.n_vis


def _block_fit(wl, pu, pv, ww, b, t0, t1, c0, nc):
    """Does the block (b, [t0, t1), [c0, c0+nc)) fit a subgrid: every sample within
    (L - beta + 1)/2 of the rounded-midpoint centre, inside the grid, one w-step."""
    L, N = wl.subgrid_size, wl.grid_size
    smax = (L - wl.kernel_size + 1) / 2
    u, v, w = pu[b, t0:t1, c0:c0 + nc], pv[b, t0:t1, c0:c0 + nc], ww[b, t0:t1, c0:c0 + nc]
    cu = math.floor(0.5 * (u.min() + u.max()) + 0.5)
    cv = math.floor(0.5 * (v.min() + v.max()) + 0.5)
    ok = max(cu - u.min(), u.max() - cu, cv - v.min(), v.max() - cv) <= smax
    ok = ok and cu - L / 2 >= 0 and cu + L / 2 <= N and cv - L / 2 >= 0 and cv + L / 2 <= N
    if wl.w_step > 0:
        ok = ok and (w.max() - w.min()) <= wl.w_step
    return ok


@pytest.mark.parametrize("seed,kw", [
    (6, dict(n_st=5, n_t=48, n_chan=4, L=16, N=256, diameter_m=30000.0, max_t=40, dt=120.0)),
    (7, dict(n_st=4, n_t=40, n_chan=8, L=24, N=128, diameter_m=50000.0, max_t=16, dt=60.0, w_step=30.0)),
])
def test_plan_blocks_are_maximal(seed, kw):
    # Greedy time grouping: a block ends only at the slot end, at T_max, or because
    # adding the next timestep would break the fit.  With the no-larger-than bound
    # of the invariants test this pins the allowed shift (L - beta + 1)/2 exactly.
    wl = syn.make_small(seed=seed, with_vis=False, aterms="identity", **kw)
    p = O.plan(wl)
    pu, pv, ww = vis_pixels(wl)
    n_break = 0
    for d in p.desc:
        b, a, t0, nt, c0, nc = (int(x) for x in d[:6])
        assert _block_fit(wl, pu, pv, ww, b, t0, t0 + nt, c0, nc)
        t_end = int(wl.aterm_offsets[a + 1])
        if t0 + nt < t_end and nt < wl.max_timesteps:
            assert not _block_fit(wl, pu, pv, ww, b, t0, t0 + nt + 1, c0, nc)
            n_break += 1
    assert n_break > 0
    # the channel grouping is the smallest that lets every single timestep fit by size
    for (b, a) in {(int(d[0]), int(d[1])) for d in p.desc}:
        groups = {(int(d[O.D_C0]), int(d[O.D_NC])) for d in p.desc if d[0] == b and d[1] == a}
        G = len(groups)
        if G > 1:
            Gm = G - 1
            sizes = [wl.n_chan // Gm + (g < wl.n_chan % Gm) for g in range(Gm)]
            starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
            L = wl.subgrid_size
            smax = (L - wl.kernel_size + 1) / 2
            some_fail = False
            for t in range(wl.aterm_offsets[a], wl.aterm_offsets[a + 1]):
                for c0, nc in zip(starts, sizes):
                    u = pu[b, t, c0:c0 + nc]
                    v = pv[b, t, c0:c0 + nc]
                    w = ww[b, t, c0:c0 + nc]
                    cu = math.floor(0.5 * (u.min() + u.max()) + 0.5)
                    cv = math.floor(0.5 * (v.min() + v.max()) + 0.5)
                    worst = max(cu - u.min(), u.max() - cu, cv - v.min(), v.max() - cv)
                    if worst > smax or (wl.w_step > 0 and w.max() - w.min() > wl.w_step):
                        some_fail = True
            assert some_fail


def test_plan_centre_rounds_half_up():
    # A block whose extent midpoint is exactly half-way between two pixels is
    # centred on the upper one (reading of "central pixel", Sect. 3.2).  With
    # f = c the wavelength is 1 m and S = 2^-4, so every number below is exact.
    N, L = 64, 16
    cell = 2.0 ** -10
    S = N * cell
    freqs = np.array([C])
    uvw = np.zeros((1, 2, 3))
    uvw[0, 0, 0] = 7.0 / S                 # pu = N/2 + 7
    uvw[0, 1, 0] = 8.0 / S                 # pu = N/2 + 8  -> midpoint N/2 + 7.5
    uvw[0, :, 1] = -3.5 / S                # pv = N/2 - 3.5 exactly
    wl = syn.Workload("half", uvw, freqs, np.array([[0, 1]], dtype=np.int32), np.array([0, 2], dtype=np.int32),
                      2, L, N, cell, 0.0, 7.0, 4, np.ones((L, L), dtype=np.float32))
    p = O.plan(wl)
    assert p.n_sub == 1
    assert p.desc[0, O.D_Q0] + L // 2 == N // 2 + 8
    assert p.desc[0, O.D_R0] + L // 2 == N // 2 - 3


def test_plan_channel_groups_split_long_baselines():
    # long baselines and a wide band: a single subgrid cannot hold all channels,
    # so groups of contiguous channels appear (Fig. 2; channel partitioning)
    wl = syn.make_small(seed=5, n_st=5, n_t=16, n_chan=16, L=16, N=256, diameter_m=60000.0,
                        df=8e6, with_vis=False, aterms="identity")
    p = O.plan(wl)
    assert np.any(p.desc[:, O.D_NC] < wl.n_chan)
    # groups of one (b, slot) tile the band, sizes differ by at most one
    for (b, a) in {(int(d[0]), int(d[1])) for d in p.desc}:
        ds = p.desc[(p.desc[:, 0] == b) & (p.desc[:, 1] == a)]
        groups = sorted({(int(d[O.D_C0]), int(d[O.D_NC])) for d in ds})
        c = 0
        for c0, nc in groups:
            assert c0 == c
            c += nc
        assert c == wl.n_chan
        sizes = [g[1] for g in groups]
        assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


# --------------------------------------------------------------------------
# subgrid transform (Alg. 1/2 "FFT"/"IFFT")


@pytest.mark.parametrize("L", [8, 16, 24, 32])
@pytest.mark.parametrize("sign", [-1, 1])
def test_dft2_is_the_centred_fft(L, sign):
    rng = np.random.default_rng(L)
    x = rng.normal(size=(3, L, L, 4)) + 1j * rng.normal(size=(3, L, L, 4))
    got = O.dft2(x, sign)
    ax = (1, 2)
    xs = np.fft.ifftshift(x, axes=ax)
    ref = np.fft.fft2(xs, axes=ax) if sign < 0 else np.fft.ifft2(xs, axes=ax) * L * L
    ref = np.fft.fftshift(ref, axes=ax) / (L * L)
    assert rel_err(got, ref) < 1e-13


# --------------------------------------------------------------------------
# exact identities of Algorithms 1 and 2


def test_flat_grid_degrids_to_identity():
    # A grid equal to the 2x2 identity everywhere is the transform of a unit point
    # source at the phase centre: every visibility must come out as I_2 exactly
    # (taper centre 1, n'(0,0) = 0, the IFFT of a constant is a centred delta).
    wl = syn.make_small(seed=11, n_st=6, n_t=24, n_chan=4, L=16, N=128, aterms="identity", w_step=0.0)
    p = O.plan(wl)
    g = np.zeros((p.n_w, wl.grid_size, wl.grid_size, 4), dtype=np.complex128)
    g[..., 0] = 1.0
    g[..., 3] = 1.0
    v = O.degrid(wl, p, g)
    mask = np.zeros(v.shape[:3], dtype=bool)
    for d in p.desc:
        mask[d[0], d[2]:d[2] + d[3], d[4]:d[4] + d[5]] = True
    ref = np.zeros(4, dtype=np.complex128)
    ref[0] = ref[3] = 1.0
    assert np.max(np.abs(v[mask] - ref)) < 1e-12
    assert np.all(v[~mask] == 0)


def test_grid_sum_counts_unflagged_visibilities():
    # Summing the grid of V = I_2 gives, per subgrid, the centre pixel of its image,
    # i.e. the number of unflagged samples (identity A-terms, taper centre 1).
    wl = syn.make_small(seed=12, n_st=6, n_t=24, n_chan=4, L=16, N=128, aterms="identity", flag_p=0.2)
    p = O.plan(wl)
    v = np.zeros((wl.n_bl, wl.n_t, wl.n_chan, 4), dtype=np.complex64)
    v[..., 0] = 1.0
    v[..., 3] = 1.0
    g = O.grid(wl, p, vis=v)
    k_unflagged = sum(int(np.sum(wl.flags[d[0], d[2]:d[2] + d[3], d[4]:d[4] + d[5]] == 0)) for d in p.desc)
    s = g.sum(axis=(0, 1, 2))
    assert abs(s[0] - k_unflagged) < 1e-9 and abs(s[3] - k_unflagged) < 1e-9
    assert abs(s[1]) < 1e-9 and abs(s[2]) < 1e-9


@pytest.mark.parametrize("w_step", [0.0, 25.0])
def test_adjointness(w_step):
    # Algorithm 2 is the adjoint of Algorithm 1: <degrid(G), V> = <G, grid(V)>,
    # with random A-terms, flags and (optionally) W-layers.
    wl = syn.make_small(seed=13, n_st=6, n_t=24, n_chan=5, L=16, N=96, w_step=w_step, flag_p=0.1,
                        diameter_m=20000.0)
    p = O.plan(wl)
    rng = np.random.default_rng(0)
    V = (rng.normal(size=wl.vis.shape) + 1j * rng.normal(size=wl.vis.shape)).astype(np.complex64)
    G = rng.normal(size=(p.n_w, wl.grid_size, wl.grid_size, 4)) + 1j * rng.normal(size=(p.n_w, wl.grid_size, wl.grid_size, 4))
    gV = O.grid(wl, p, vis=V)
    dG = O.degrid(wl, p, G)
    lhs = np.vdot(dG, V.astype(np.complex128))
    rhs = np.vdot(G, gV)
    assert abs(lhs - rhs) / abs(rhs) < 1e-12


def _lattice_lm(wl):
    S = wl.grid_size * wl.cell_size
    L = wl.subgrid_size
    c = (np.arange(L) - L / 2) * S / L
    return c, S


def _full_grid_image_on_lattice(g, N, L):
    """Unnormalised centred inverse DFT of an N x N grid, evaluated only on the
    image pixels a = N/2 + (N/L)(x - L/2): I = E G E^T with explicit phasors."""
    R = N // L
    a = N // 2 + R * (np.arange(L) - L // 2)
    u = np.arange(N) - N // 2
    E = np.exp(2j * np.pi * np.outer(a - N // 2, u) / N)      # [L][N]
    return np.einsum("yv,wvup,xu->wyxp", E, g, E)


def _die_on_lattice(wl, V, flags, aterms, w0=0.0, select=None):
    """Direct imaging equation (Eq. DIE, with the 2x2 A-terms of Sect. 3.4) at the
    subgrid lattice points l_x, m_y, brute force over all visibilities."""
    L = wl.subgrid_size
    lx, S = _lattice_lm(wl)
    l = lx[None, :]
    m = lx[:, None]
    n1 = np.sqrt(1 - l * l - m * m) - 1
    out = np.zeros((L, L, 4), dtype=np.complex128)
    sc = wl.freqs_hz / C
    slot_of_t = np.searchsorted(wl.aterm_offsets, np.arange(wl.n_t), side="right") - 1
    for b in range(wl.n_bl):
        p_, q_ = wl.baselines[b]
        for t in range(wl.n_t):
            for c in range(wl.n_chan):
                if flags is not None and flags[b, t, c]:
                    continue
                if select is not None and not select[b, t, c]:
                    continue
                u, v, w = wl.uvw_m[b, t] * sc[c]
                ph = np.exp(2j * np.pi * (u * l + v * m + (w - w0) * n1))
                Vk = V[b, t, c].astype(np.complex128).reshape(2, 2)
                Ap = aterms[slot_of_t[t], p_].astype(np.complex128).reshape(L, L, 2, 2)
                Aq = aterms[slot_of_t[t], q_].astype(np.complex128).reshape(L, L, 2, 2)
                M = np.conj(np.swapaxes(Ap, -1, -2)) @ Vk @ Aq           # A_p^H V A_q
                out += (M.reshape(L, L, 4) * ph[:, :, None])
    return out


def test_grid_matches_direct_imaging_on_the_subgrid_lattice():
    # At image pixels that coincide with subgrid pixel positions, the image of the
    # IDG grid is *exactly* taper x DIE: the Dirichlet interpolation of the subgrid
    # image is exact at its own samples (Sect. 4.2: the gradients cancel at the
    # sample points).  This pins placement (q0, r0, u0, v0), the phasor sign, the
    # transform and the A-term order at once.
    wl = syn.make_small(seed=21, n_st=5, n_t=12, n_chan=3, L=16, N=128, flag_p=0.1, max_t=6, n_slots=2)
    # any taper works for this identity; a non-symmetric one catches a transposed index
    wl.taper = np.random.default_rng(3).uniform(0.5, 1.5, size=(16, 16)).astype(np.float32)
    p = O.plan(wl)
    g = O.grid(wl, p)
    img = _full_grid_image_on_lattice(g, wl.grid_size, wl.subgrid_size)[0]
    assigned = np.zeros((wl.n_bl, wl.n_t, wl.n_chan), dtype=bool)
    for d in p.desc:
        assigned[d[0], d[2]:d[2] + d[3], d[4]:d[4] + d[5]] = True
    die = _die_on_lattice(wl, wl.vis, wl.flags, wl.aterms, select=assigned)
    ref = die * wl.taper.astype(np.float64)[:, :, None]
    assert rel_err(img, ref) < 1e-11


def test_w_layers_match_direct_imaging_per_layer():
    # With W-layers each layer's image on the lattice is the DIE of its own
    # visibilities with w replaced by w - w0 (w0 = k * w_step).
    wl = syn.make_small(seed=22, n_st=5, n_t=12, n_chan=3, L=16, N=128, w_step=15.0, max_t=6,
                        aterms="identity", diameter_m=15000.0)
    p = O.plan(wl)
    assert p.n_w > 1
    g = O.grid(wl, p)
    imgs = _full_grid_image_on_lattice(g, wl.grid_size, wl.subgrid_size)
    for layer in range(p.n_w):
        sel = np.zeros((wl.n_bl, wl.n_t, wl.n_chan), dtype=bool)
        for d in p.desc[p.desc[:, O.D_LAYER] == layer]:
            sel[d[0], d[2]:d[2] + d[3], d[4]:d[4] + d[5]] = True
        w0 = (layer + p.k_min) * wl.w_step
        die = _die_on_lattice(wl, wl.vis, None, wl.aterms, w0=w0, select=sel)
        ref = die * wl.taper.astype(np.float64)[:, :, None]
        assert rel_err(imgs[layer], ref) < 1e-11


def test_degrid_matches_direct_prediction_on_the_subgrid_lattice():
    # A model image whose sources sit on subgrid lattice points is predicted
    # exactly (DME, Eq. DME with the polarised A-terms A_p B A_q^H) by degridding
    # its transform.
    wl = syn.make_small(seed=23, n_st=5, n_t=10, n_chan=3, L=16, N=128, max_t=5, n_slots=2, flag_p=0.1)
    wl.taper = np.random.default_rng(4).uniform(0.5, 1.5, size=(16, 16)).astype(np.float32)
    p = O.plan(wl)
    N, L = wl.grid_size, wl.subgrid_size
    R = N // L
    rng = np.random.default_rng(5)
    pts = [(int(rng.integers(3, L - 3)), int(rng.integers(3, L - 3))) for _ in range(3)]
    B = [rng.normal(size=4) + 1j * rng.normal(size=4) for _ in pts]
    # grid = centred forward DFT of the N x N image (sign -, unnormalised)
    a = np.arange(N) - N // 2
    g = np.zeros((1, N, N, 4), dtype=np.complex128)
    for (y, x), Bk in zip(pts, B):
        ax, ay = R * (x - L // 2), R * (y - L // 2)
        ph = np.exp(-2j * np.pi * (np.outer(a, np.ones(N)) * ay + np.outer(np.ones(N), a) * ax) / N)
        g[0] += ph[:, :, None] * Bk[None, None, :]
    v = O.degrid(wl, p, g)
    lx, S = _lattice_lm(wl)
    sc = wl.freqs_hz / C
    slot_of_t = np.searchsorted(wl.aterm_offsets, np.arange(wl.n_t), side="right") - 1
    ref = np.zeros_like(v)
    for d in p.desc:
        b = d[0]
        p_, q_ = wl.baselines[b]
        for t in range(d[2], d[2] + d[3]):
            for c in range(d[4], d[4] + d[5]):
                if wl.flags[b, t, c]:
                    continue
                u, vv, w = wl.uvw_m[b, t] * sc[c]
                acc = np.zeros((2, 2), dtype=np.complex128)
                for (y, x), Bk in zip(pts, B):
                    l, m = lx[x], lx[y]
                    n1 = math.sqrt(1 - l * l - m * m) - 1
                    Ap = wl.aterms[slot_of_t[t], p_, y, x].astype(np.complex128).reshape(2, 2)
                    Aq = wl.aterms[slot_of_t[t], q_, y, x].astype(np.complex128).reshape(2, 2)
                    acc += wl.taper[y, x] * (Ap @ Bk.reshape(2, 2) @ np.conj(Aq.T)) * np.exp(-2j * np.pi * (u * l + vv * m + w * n1))
                ref[b, t, c] = acc.reshape(4)
    assert rel_err(v, ref) < 1e-11


def _dirichlet(theta, L):
    """sum_{J=-L/2}^{L/2-1} exp(2 pi i J theta) in closed form (geometric series)."""
    theta = np.asarray(theta, dtype=np.float64)
    out = np.empty(theta.shape, dtype=np.complex128)
    near = np.abs(np.sin(np.pi * theta)) < 1e-12
    out[near] = L
    t = theta[~near]
    out[~near] = np.exp(-1j * np.pi * t) * np.sin(np.pi * L * t) / np.sin(np.pi * t)
    return out


def _point_source_grid(wl, l0, m0, B):
    """Exact model grid of a point source: the visibility function sampled at the
    grid points, V(u_q, v_r) = B exp(-2 pi i (u_q l0 + v_r m0)), u_q = (q - N/2)/S."""
    N = wl.grid_size
    S = N * wl.cell_size
    uq = (np.arange(N) - N / 2) / S
    ph = np.exp(-2j * np.pi * (uq[None, :] * l0 + uq[:, None] * m0))
    return (ph[:, :, None] * np.asarray(B)[None, None, :])[None]


def test_point_source_degrid_kernel_form():
    # Degridding a plane-wave grid equals the kernel form: the subgrid image is a
    # product of two Dirichlet kernels (closed form) centred on the source, times
    # the taper and the phasor (Sect. 4.2, Eq. effective_window in discrete form).
    wl = syn.make_small(seed=31, n_st=5, n_t=12, n_chan=3, L=24, N=192, aterms="identity", max_t=6)
    p = O.plan(wl)
    L, N = wl.subgrid_size, wl.grid_size
    S = N * wl.cell_size
    l0, m0 = 0.137 * S, -0.081 * S
    B = np.array([1.0, 0.2 + 0.1j, -0.3j, 0.7])
    v = O.degrid(wl, p, _point_source_grid(wl, l0, m0, B))
    lx = (np.arange(L) - L / 2) * S / L
    Dx = _dirichlet((lx - l0) / S, L)
    Dy = _dirichlet((lx - m0) / S, L)
    img = (Dy[:, None] * Dx[None, :]) / (L * L) * wl.taper.astype(np.float64)
    n1 = np.sqrt(1 - lx[None, :] ** 2 - lx[:, None] ** 2) - 1
    sc = wl.freqs_hz / C
    ref = np.zeros_like(v)
    for d in p.desc:
        b = d[0]
        u0 = (d[O.D_Q0] + L / 2 - N / 2) / S
        v0 = (d[O.D_R0] + L / 2 - N / 2) / S
        for t in range(d[2], d[2] + d[3]):
            for c in range(d[4], d[4] + d[5]):
                u, vv, w = wl.uvw_m[b, t] * sc[c]
                ph = np.exp(-2j * np.pi * ((u - u0) * lx[None, :] + (vv - v0) * lx[:, None] + w * n1))
                ref[b, t, c] = np.exp(-2j * np.pi * (u0 * l0 + v0 * m0)) * np.sum(img * ph) * B
    assert rel_err(v, ref) < 1e-11


def test_point_source_degrid_close_to_measurement_equation():
    # Physics: degridding the model grid of an off-lattice point source reproduces
    # the measurement equation (Eq. 2) up to the effective window at the source,
    # f0 = L^-2 sum c[y][x] D(x) D(y), with an error at the aliasing level of the
    # taper (Sect. 4, Table 1; Fig. 6 reports 1e-5 .. 7e-4 for a 1 Jy source).
    wl = syn.make_small(seed=32, n_st=6, n_t=16, n_chan=3, L=24, N=256, aterms="identity", max_t=8,
                        diameter_m=4000.0)
    p = O.plan(wl)
    L, N = wl.subgrid_size, wl.grid_size
    S = N * wl.cell_size
    l0, m0 = 0.113 * S, 0.072 * S
    v = O.degrid(wl, p, _point_source_grid(wl, l0, m0, [1.0, 0, 0, 1.0]))
    lx = (np.arange(L) - L / 2) * S / L
    f0 = np.sum(wl.taper * (_dirichlet((lx - m0) / S, L)[:, None] * _dirichlet((lx - l0) / S, L)[None, :])) / L ** 2
    n0 = math.sqrt(1 - l0 * l0 - m0 * m0) - 1
    sc = wl.freqs_hz / C
    errs = []
    for d in p.desc:
        b = d[0]
        for t in range(d[2], d[2] + d[3]):
            for c in range(d[4], d[4] + d[5]):
                u, vv, w = wl.uvw_m[b, t] * sc[c]
                me = np.exp(-2j * np.pi * (u * l0 + vv * m0 + w * n0))
                errs.append(abs(v[b, t, c, 0] / f0 - me))
                assert abs(v[b, t, c, 1]) < 1e-12
    errs = np.array(errs)
    # the PSWF taper of beta=7 has side-lobe level ~1e-4 (Table 1, beta=7);
    # position-dependent effective windows stay within a few 1e-3
    assert np.sqrt(np.mean(errs ** 2)) < 3e-3
    assert np.max(errs) < 2e-2


def test_single_visibility_on_a_pixel_grids_to_a_delta():
    # With a flat taper, identity A-terms and w = 0, a visibility exactly on grid
    # pixel (pu, pv) is gridded to that pixel and nowhere else, with unit gain.
    N, L = 64, 16
    cell = 1.0e-3                       # S = 0.064: pixel pitch 1/S = 15.6 wavelengths
    S = N * cell
    freqs = np.array([150e6])
    lam = C / freqs[0]
    pix = [(7, -3), (-11, 5)]
    uvw = np.zeros((2, 1, 3))
    for i, (du, dv) in enumerate(pix):
        uvw[i, 0, 0] = du / S * lam
        uvw[i, 0, 1] = dv / S * lam
    wl = syn.Workload("delta", uvw, freqs, np.array([[0, 1], [0, 2]], dtype=np.int32),
                      np.array([0, 1], dtype=np.int32), 3, L, N, cell, 0.0, 7.0, 4,
                      np.ones((L, L), dtype=np.float32))
    wl.vis = np.array([[[[1 + 2j, 3j, -1, 0.5]]], [[[2, 1j, 0, -1j]]]], dtype=np.complex64)
    p = O.plan(wl)
    g = O.grid(wl, p, aterms=None)
    ref = np.zeros_like(g)
    for i, (du, dv) in enumerate(pix):
        ref[0, N // 2 + dv, N // 2 + du] += wl.vis[i, 0, 0]
    assert np.max(np.abs(g - ref)) < 1e-12


def test_constant_aterms_act_on_the_visibilities():
    # A-terms that are constant over the field can be moved out of the direct sum
    # (Sect. 3.4): gridding with (A_p, A_q) = gridding M_p^H V M_q with identity
    # A-terms, and degridding with them = M_p y M_q^H.  Fails on a transposed or
    # un-conjugated Jones matrix, or on swapped stations.
    wl = syn.make_small(seed=41, n_st=5, n_t=10, n_chan=3, L=16, N=96, aterms="identity", n_slots=2, max_t=5)
    rng = np.random.default_rng(9)
    M = (rng.normal(size=(2, 5, 4)) + 1j * rng.normal(size=(2, 5, 4))).astype(np.complex64)
    A = np.ascontiguousarray(np.broadcast_to(M[:, :, None, None, :], (2, 5, 16, 16, 4)))
    p = O.plan(wl)
    slot_of_t = np.searchsorted(wl.aterm_offsets, np.arange(wl.n_t), side="right") - 1
    Vm = np.zeros_like(wl.vis, dtype=np.complex128)
    for b in range(wl.n_bl):
        p_, q_ = wl.baselines[b]
        for t in range(wl.n_t):
            Mp = M[slot_of_t[t], p_].astype(np.complex128).reshape(2, 2)
            Mq = M[slot_of_t[t], q_].astype(np.complex128).reshape(2, 2)
            for c in range(wl.n_chan):
                Vm[b, t, c] = (np.conj(Mp.T) @ wl.vis[b, t, c].astype(np.complex128).reshape(2, 2) @ Mq).reshape(4)
    # the oracle reads visibilities as complex64: compare the linear maps on
    # complex64-exact inputs by gridding Vm through the identity path in FP64 terms
    g_a = O.grid(wl, p, aterms=A)
    g_i = O.grid(wl, p, vis=Vm.astype(np.complex64), aterms=None)
    assert rel_err(g_a, g_i) < 1e-6          # complex64 rounding of Vm only
    G = rng.normal(size=g_a.shape) + 1j * rng.normal(size=g_a.shape)
    v_a = O.degrid(wl, p, G, aterms=A)
    v_i = O.degrid(wl, p, G, aterms=None)
    ref = np.zeros_like(v_i)
    for b in range(wl.n_bl):
        p_, q_ = wl.baselines[b]
        for t in range(wl.n_t):
            Mp = M[slot_of_t[t], p_].astype(np.complex128).reshape(2, 2)
            Mq = M[slot_of_t[t], q_].astype(np.complex128).reshape(2, 2)
            for c in range(wl.n_chan):
                ref[b, t, c] = (Mp @ v_i[b, t, c].reshape(2, 2) @ np.conj(Mq.T)).reshape(4)
    assert rel_err(v_a, ref) < 1e-12


def test_flags_zero_weight():
    wl = syn.make_small(seed=42, n_st=5, n_t=10, n_chan=3, L=16, N=96, flag_p=0.3)
    p = O.plan(wl)
    v0 = wl.vis.copy()
    v0[wl.flags.astype(bool)] = 0
    g1 = O.grid(wl, p)
    g2 = O.grid(wl, p, vis=v0, flags=np.zeros_like(wl.flags))
    assert np.array_equal(g1, g2)
    G = np.ones_like(g1)
    y = O.degrid(wl, p, G)
    assert np.all(y[wl.flags.astype(bool)] == 0)
