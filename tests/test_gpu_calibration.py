"""GPU parity of the calibration call (idg_aterm_gradient: residuals, cost and
A-term gradient; Sect. 6 application) against the FP64 calibration oracle,
which is itself pinned to exact finite differences of the cost
(tests/test_calibration_cpu.py).

Tolerance: relative RMS <= 1e-5 on residuals and gradient, 1e-5 relative on the
cost.  The observed visibilities and the model differ by O(1), so the residuals
are not a small difference of large numbers."""
import numpy as np
import pytest

from oracle import calibration as C
from oracle import oracle as O
from paper_1909_07226_gb300 import idg
from paper_1909_07226_gb300 import synthetic as syn
from tests.gpu_util import dev, parity, workload_to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_07226_gb300 import build
    build.build()
    idg.load()


CASES = {
    "L16_wlayers": (dict(seed=81, n_st=6, n_t=40, n_chan=5, L=16, N=128, max_t=20, n_slots=2, flag_p=0.1,
                         w_step=25.0, diameter_m=5000.0), {}),
    "L24": (dict(seed=82, n_st=7, n_t=48, n_chan=6, L=24, N=128, max_t=48, n_slots=3, flag_p=0.1), {}),
    "L32_separable": (dict(seed=83, n_st=6, n_t=96, n_chan=8, L=32, N=128, max_t=96, n_slots=2, flag_p=0.1,
                           diameter_m=2500.0, df=0.25e6), {}),
    "L32_recurrence_tc_transform": (dict(seed=84, n_st=6, n_t=64, n_chan=16, L=32, N=256, max_t=32, n_slots=2,
                                         flag_p=0.05, diameter_m=8000.0),
                                    dict(precision_mode=idg.PHASOR_RECURRENCE, fft_mode=idg.FFT_TC_SPLIT)),
}


def _run(p, wl, G, aterms=True, taper=True):
    import torch
    d = workload_to_device(wl)
    res = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")
    grad = torch.zeros(wl.aterms.shape, dtype=torch.complex64, device="cuda")
    cost = torch.zeros(1, dtype=torch.float64, device="cuda")
    idg.aterm_gradient(p, dev(G), d["vis"], d["flags"], d["aterms"] if aterms else None,
                       d["taper"] if taper else None, res, grad, cost)
    idg.device_errors()
    return res, grad, cost


@pytest.mark.parametrize("case", sorted(CASES))
def test_residual_cost_and_gradient_match_the_oracle(case):
    kw, opt = CASES[case]
    wl = syn.make_small(**kw)
    p = idg.plan_from_workload(wl, **opt)
    op = O.plan(wl)
    G = syn.random_grid(np.random.default_rng(31), p.n_w_layers, wl.grid_size)
    res, grad, cost = _run(p, wl, G)
    r, J, Gr = C.gradient(wl, op, G, wl.vis)
    parity(res.cpu().numpy(), r, f"{case} residuals")
    parity(grad.cpu().numpy(), Gr, f"{case} A-term gradient")
    assert float(cost.item()) == pytest.approx(J, rel=1e-5)


def test_gradient_and_cost_accumulate_and_identity_default():
    import torch
    kw, _ = CASES["L24"]
    wl = syn.make_small(**kw)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    G = syn.random_grid(np.random.default_rng(32), p.n_w_layers, wl.grid_size)
    d = workload_to_device(wl)
    res = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")
    grad = torch.zeros(wl.aterms.shape, dtype=torch.complex64, device="cuda")
    cost = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        idg.aterm_gradient(p, dev(G), d["vis"], d["flags"], d["aterms"], d["taper"], res, grad, cost)
    r, J, Gr = C.gradient(wl, op, G, wl.vis)
    parity(grad.cpu().numpy(), 2 * Gr, "gradient added twice")
    assert float(cost.item()) == pytest.approx(2 * J, rel=1e-5)
    # NULL A-terms: the gradient at identity A-terms; NULL cost: not computed
    grad.zero_()
    idg.aterm_gradient(p, dev(G), d["vis"], d["flags"], None, d["taper"], res, grad, None)
    r0, J0, G0 = C.gradient(wl, op, G, wl.vis, aterms=None)
    parity(res.cpu().numpy(), r0, "residuals at identity A-terms")
    parity(grad.cpu().numpy(), G0, "gradient at identity A-terms")


def test_lofar_slice_gradient():
    # the LOFAR-like workload's first 128 timesteps (1601 subgrids of 32 x 32, one
    # A-term slot, separable plan), the launch configuration the benchmark times
    wl = syn.make_lofar(n_t=128)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    assert p.stats.separable == 1
    G = syn.random_grid(np.random.default_rng(33), p.n_w_layers, wl.grid_size)
    res, grad, cost = _run(p, wl, G)
    r, J, Gr = C.gradient(wl, op, G, wl.vis)
    parity(res.cpu().numpy(), r, "LOFAR slice residuals")
    parity(grad.cpu().numpy(), Gr, "LOFAR slice A-term gradient")
    assert float(cost.item()) == pytest.approx(J, rel=1e-5)
