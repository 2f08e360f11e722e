"""Pins of the calibration oracle (residuals, cost and A-term gradient; Sect. 6
application, Sect. 2 cost function, Sect. 3.4 A-terms).

The gradient is pinned to finite differences of the cost, and the cost comes
from the oracle's degridder alone (Alg. 2), an independent route.  Along a
direction E that perturbs the A-terms of ONE station (no baseline pairs a
station with itself), every model visibility is affine in the step h -- the
station enters either as A_p or as A_q^H -- so J(A + h E) is exactly quadratic
in h and the central difference (J(h) - J(-h)) / 2h equals the directional
derivative Re sum conj(G) E exactly, up to rounding.  A mistake in a sign, a
conjugate, a transpose, a factor or a missing term of either station role
changes that derivative.
"""
import numpy as np
import pytest

from oracle import calibration as C
from oracle import oracle as O
from paper_1909_07226_gb300 import synthetic as syn


@pytest.fixture(scope="module")
def case():
    wl = syn.make_small(seed=606, n_st=5, n_t=24, n_chan=4, L=16, N=64, max_t=8, n_slots=2, flag_p=0.15,
                        diameter_m=3000.0)
    op = O.plan(wl)
    model = syn.random_grid(np.random.default_rng(17), op.n_w, wl.grid_size)
    r, J, G = C.gradient(wl, op, model, wl.vis)
    return dict(wl=wl, op=op, model=model, r=r, J=J, G=G)


def _cost(wl, op, model, A):
    return C.residual(wl, op, model, wl.vis, aterms=A.astype(np.complex64))[1]


@pytest.mark.parametrize("slot,station", [(0, 0), (0, 3), (1, 1), (1, 4)])
def test_gradient_equals_central_difference_of_the_cost(case, slot, station):
    wl, op, model, G = case["wl"], case["op"], case["model"], case["G"]
    assert all(p != q for p, q in wl.baselines)
    rng = np.random.default_rng(100 * slot + station)
    E = np.zeros(wl.aterms.shape, dtype=np.complex128)
    E[slot, station] = rng.normal(size=E[slot, station].shape) + 1j * rng.normal(size=E[slot, station].shape)
    A = wl.aterms.astype(np.complex128)
    h = 0.25
    fd = (_cost(wl, op, model, A + h * E) - _cost(wl, op, model, A - h * E)) / (2 * h)
    an = float(np.real(np.sum(np.conj(G) * E)))
    print(f"slot {slot} station {station}: fd={fd:.9e} analytic={an:.9e}")
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-300) + 1e-9 * case["J"]
    assert abs(an) > 1e-3 * case["J"]               # the direction is not degenerate


def test_cost_is_the_residual_norm_and_excludes_flagged_and_dropped(case):
    wl, op, model, r, J = case["wl"], case["op"], case["model"], case["r"], case["J"]
    assert J == pytest.approx(float(np.sum(np.abs(r) ** 2)), rel=1e-14)
    mask = C.planned_unflagged(wl, op)
    assert not mask.all() and mask.any()
    assert np.all(r[~mask] == 0)
    # garbage in the flagged visibilities changes neither the cost nor the gradient
    vis = wl.vis.copy()
    vis[~mask] = 1e6
    r2, J2, G2 = C.gradient(wl, op, model, vis)
    assert J2 == pytest.approx(J, rel=1e-12)
    assert np.max(np.abs(G2 - case["G"])) <= 1e-9 * np.max(np.abs(case["G"]))


def test_gradient_vanishes_where_the_model_fits():
    # observed = the model's own visibilities: r = 0 up to the complex64 rounding of
    # the observed values, so G is rounding-level against a misfit's gradient
    wl = syn.make_small(seed=607, n_st=4, n_t=16, n_chan=3, L=16, N=64, max_t=8, n_slots=1)
    op = O.plan(wl)
    model = syn.random_grid(np.random.default_rng(18), op.n_w, wl.grid_size)
    y = O.degrid(wl, op, model).astype(np.complex64)
    _, J0, G0 = C.gradient(wl, op, model, y)
    _, J1, G1 = C.gradient(wl, op, model, 2 * y)
    assert J0 <= 1e-12 * J1
    assert np.max(np.abs(G0)) <= 1e-6 * np.max(np.abs(G1))


def test_minus_gradient_is_a_descent_direction(case):
    wl, op, model, G, J = case["wl"], case["op"], case["model"], case["G"], case["J"]
    A = wl.aterms.astype(np.complex128)
    eps = 1e-3 * np.linalg.norm(A) / np.linalg.norm(G)
    J_step = _cost(wl, op, model, A - eps * G)
    # first order: J - eps |G|^2 (the direction's derivative is -|G|^2)
    assert J_step < J
    assert (J - J_step) == pytest.approx(eps * np.sum(np.abs(G) ** 2), rel=0.05)
