"""Pins of the classical-gridding oracle (oversampled A/W-projection kernels,
Sect. 2), each against something other than the oracle's own formula:

* the kernel table (zero padding + FFT, Sect. 2: C = F(Z(c))) equals the
  direct sum of the kernel's definition at the same fractional offsets;
* with the kernel evaluated exactly, support M = L and the support box on the
  subgrid box, classical gridding of one visibility with random A-terms and a
  w-term equals image domain gridding of it by the (separately pinned) IDG
  oracle, Alg. 1 -- image domain gridding is convolution with the exactly
  evaluated kernel of the same window restricted to the subgrid;
* the oversampled lookup converges to the exact kernel as 1/O (nearest-sample
  error of a smooth kernel), which pins the phase selection;
* W-projection planes reduce to the exact w as the plane spacing shrinks;
* flags are zero weight.
"""
import numpy as np
import pytest

from oracle import classical as CL
from oracle import oracle as O
from paper_1909_07226_gb300 import synthetic as syn


def _single_vis_workload(L=16, N=64, frac_u=0.7, frac_v=0.6, w_m=900.0, seed=5):
    # one baseline, one timestep, one channel, placed so that floor(pu) = Cu - 1:
    # then the classical support [floor(pu) - L/2 + 1, floor(pu) + L/2] is the
    # subgrid box [Cu - L/2, Cu + L/2) of the plan
    rng = np.random.default_rng(seed)
    f = np.array([150e6])
    s = f[0] / CL.C_LIGHT
    cell = 0.9 / N * 0.05
    S = N * cell
    pu, pv = N / 2 + 5 + frac_u, N / 2 - 7 + frac_v
    uvw = np.array([[[(pu - N / 2) / (s * S), (pv - N / 2) / (s * S), w_m]]])
    a = syn.pswf_1d(L, 7.0)
    wl = syn.Workload("single", uvw, f, np.array([[0, 1]], dtype=np.int32), np.array([0, 1], dtype=np.int32), 2, L,
                      N, cell, 0.0, 7.0, 1, syn.separable_taper(a))
    wl.screens = syn.random_jones_screens(rng, 1, 2, S / 2)
    wl.aterms = syn.aterms_on_subgrid(wl.screens, L, S)
    wl.vis = (rng.normal(size=(1, 1, 1, 4)) + 1j * rng.normal(size=(1, 1, 1, 4))).astype(np.complex64)
    return wl


def test_table_equals_direct_kernel_evaluation():
    rng = np.random.default_rng(1)
    M, O_, S = 8, 5, 0.05
    A = rng.normal(size=(M, M, 4)) + 1j * rng.normal(size=(M, M, 4))
    B = rng.normal(size=(M, M, 4)) + 1j * rng.normal(size=(M, M, 4))
    win = CL.mueller_window(M, S, rng.uniform(0.2, 1.0, size=(M, M)), A, B, w=37.5)
    tab = CL.kernel_table(win, O_)
    for _ in range(40):
        oy, ox = rng.integers(0, O_, size=2)
        dy, dx = rng.integers(0, M, size=2)
        ref = CL.kernel_at(win, dy - M // 2 + 1 - oy / O_, dx - M // 2 + 1 - ox / O_)
        assert np.max(np.abs(tab[oy, ox, dy, dx] - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("frac", [(0.7, 0.6), (0.5, 0.95)])
def test_exact_classical_equals_image_domain_gridding(frac):
    wl = _single_vis_workload(frac_u=frac[0], frac_v=frac[1])
    op = O.plan(wl)
    assert op.n_sub == 1
    L = wl.subgrid_size
    cu = op.desc[0, O.D_Q0] + L // 2
    S = wl.grid_size * wl.cell_size
    pu = (wl.uvw_m[0, 0, 0] * (wl.freqs_hz[0] / CL.C_LIGHT)) * S + wl.grid_size / 2
    assert int(np.floor(pu)) == cu - 1
    ref = O.grid(wl, op)
    # (a fine oversampling keeps the support where floor(pu) puts it)
    got = CL.grid(wl, op, M=L, O_=1024, dw=1.0, aterms=wl.aterms, taper=wl.taper, exact=True)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # a wrong role of the stations (A_q^H X A_p) is not the same operator
    bad = CL.grid(wl, op, M=L, O_=1024, dw=1.0, aterms=wl.aterms[:, ::-1], taper=wl.taper, exact=True)
    assert np.max(np.abs(bad - ref)) > 1e-3 * np.max(np.abs(ref))


def test_oversampled_lookup_converges_as_one_over_o():
    wl = syn.make_small(seed=9, n_st=4, n_t=6, n_chan=3, L=16, N=128, max_t=6, n_slots=1, aterms="identity")
    op = O.plan(wl)
    M = 8
    a = syn.pswf_1d(M, 7.0)
    tap = np.outer(a, a)
    errs = []
    for O_ in (8, 32, 128):
        exact = CL.grid(wl, op, M=M, O_=O_, taper=tap, exact=True)     # same support pixels
        g = CL.grid(wl, op, M=M, O_=O_, taper=tap)
        errs.append(np.linalg.norm(g - exact) / np.linalg.norm(exact))
    print("oversampling errors", errs)
    assert errs[0] < 0.1
    for e0, e1 in zip(errs, errs[1:]):
        assert 2.5 < e0 / e1 < 10.0         # first order in 1/O: about x4 per step of 4


def test_w_plane_selection_and_plane_kernel():
    # one visibility with w f/c = 900 lambda: a plane spacing that divides its w exactly
    # reproduces the exact-w kernel up to the oversampling error; a spacing that puts it
    # 20 % off its plane (2.5 planes, rounded to 3) does not
    wl = _single_vis_workload(L=16, frac_u=0.3, frac_v=0.8, w_m=1800.0)
    op = O.plan(wl)
    s = wl.freqs_hz[0] / CL.C_LIGHT
    w_l = wl.uvw_m[0, 0, 2] * s
    M, O_ = 16, 64
    exact = CL.grid(wl, op, M=M, O_=O_, dw=1.0, aterms=wl.aterms, taper=wl.taper, exact=True)
    on = CL.grid(wl, op, M=M, O_=O_, dw=w_l / 3, aterms=wl.aterms, taper=wl.taper)
    off = CL.grid(wl, op, M=M, O_=O_, dw=w_l / 2.5, aterms=wl.aterms, taper=wl.taper)
    assert CL.w_plane(wl.uvw_m[0, 0, 2], s, 0.0, w_l / 2.5) == 3
    no_w = CL.grid(wl, op, M=M, O_=O_, dw=0.0, aterms=wl.aterms, taper=wl.taper)
    e = [np.linalg.norm(g - exact) / np.linalg.norm(exact) for g in (on, off, no_w)]
    print("w-plane errors (on plane, off plane, no w-term)", e)
    assert e[0] < 0.02
    assert e[1] > 5 * e[0] and e[2] > 5 * e[0]


def test_flags_are_zero_weight():
    wl = syn.make_small(seed=11, n_st=4, n_t=6, n_chan=3, L=16, N=64, max_t=6, n_slots=2, flag_p=0.3)
    op = O.plan(wl)
    M = 8
    g = CL.grid(wl, op, M=M, O_=4)
    vis = wl.vis.copy()
    vis[wl.flags.astype(bool)] = 1e6
    assert np.array_equal(CL.grid(wl, op, M=M, O_=4, vis=vis), g)
    unflagged = CL.grid(wl, op, M=M, O_=4, flags=np.zeros_like(wl.flags))
    assert not np.allclose(unflagged, g)


@pytest.mark.parametrize("frac", [(5.7 / 16, 10.2 / 16), (15.6 / 16, 0.3 / 16)])
def test_lookup_takes_the_nearest_oversampled_offset(frac):
    # the table lookup of one visibility equals the exact kernel of the same
    # visibility moved to the nearest multiple of 1/O (round half up; a phase that
    # rounds up to O moves the support one pixel on)
    O_ = 16
    wl = _single_vis_workload(L=16, frac_u=frac[0], frac_v=frac[1])
    op = O.plan(wl)
    moved = _single_vis_workload(L=16, frac_u=np.floor(frac[0] * O_ + 0.5) / O_,
                                 frac_v=np.floor(frac[1] * O_ + 0.5) / O_)
    moved.vis, moved.aterms = wl.vis, wl.aterms
    got = CL.grid(wl, op, M=8, O_=O_, aterms=None, taper=None)
    ref = CL.grid(moved, op, M=8, O_=O_, aterms=None, taper=None, exact=True)
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
