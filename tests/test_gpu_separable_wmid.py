"""GPU parity of the separable kernels on plans that meet the remainder bound only
with each subgrid's own w offset: the sums use w_s, the middle of the subgrid's
w range, and the kernels apply exp(+-2 pi i (w_s - w0) n'(x, y)) to the subgrid
image (gridder epilogue, degridder prologue).  Against the FP64 oracle, relative
RMS <= 1e-5 (tests.gpu_util.parity)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07226_gb300 import idg
from paper_1909_07226_gb300 import synthetic as syn
from tests.gpu_util import dev, parity, workload_to_device

pytestmark = pytest.mark.gpu

C = 299792458.0
SEP_THETA_MAX = 1.38e-3        # the plan's bound on the remainder phase

CASES = {
    "L24": dict(seed=84, n_st=6, n_t=96, n_chan=8, L=24, N=384, max_t=96, n_slots=3, flag_p=0.1,
                diameter_m=1500.0, df=0.5e6),
    "L24_long": dict(seed=84, n_st=6, n_t=256, n_chan=8, L=24, N=384, max_t=128, n_slots=3, flag_p=0.1,
                     diameter_m=1500.0, df=0.25e6, dt=5.0),
    "L32": dict(seed=88, n_st=6, n_t=256, n_chan=8, L=32, N=320, max_t=128, n_slots=3, flag_p=0.1,
                diameter_m=1500.0, df=0.25e6, dt=5.0),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_07226_gb300 import build
    build.build()
    idg.load()


def theta_with_w0(wl, p):
    # max |2 pi (w - w0)| max |r| with the layer offset w0 (= 0 here, no W-layers)
    L = wl.subgrid_size
    S = wl.grid_size * wl.cell_size

    def n1(x, y):
        l, m = (x - 0.5 * L) * S / L, (y - 0.5 * L) * S / L
        return np.sqrt(1.0 - l * l - m * m) - 1.0

    # the split through the reference row and column j0 that makes max |r| smallest
    r = min(max(abs(n1(x, y) - n1(x, j) - n1(j, y) + n1(j, j)) for y in range(L) for x in range(L))
            for j in range(L))
    dw = 0.0
    for d in p.export():
        w = wl.uvw_m[d[O.D_BL], d[O.D_T0]:d[O.D_T0] + d[O.D_NT], 2]
        f = np.array([wl.freqs_hz[d[O.D_C0]], wl.freqs_hz[d[O.D_C0] + d[O.D_NC] - 1]])
        dw = max(dw, float(np.abs(np.outer(w, f / C)).max()))
    return 2.0 * np.pi * dw * r


@pytest.mark.parametrize("case", sorted(CASES))
def test_separable_with_subgrid_w_offset(case):
    import torch
    wl = syn.make_small(**CASES[case])
    p = idg.plan_from_workload(wl)
    assert wl.w_step == 0.0
    assert p.stats.separable == 1
    assert theta_with_w0(wl, p) > SEP_THETA_MAX >= p.stats.sep_phase    # separable only with w_s
    op = O.plan(wl)
    d = workload_to_device(wl)
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    idg.profile_enable(True)
    try:
        idg.profile_read(reset=True)
        idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
        launches = {k: v["launches"] for k, v in idg.profile_read(reset=True).items() if v["launches"]}
    finally:
        idg.profile_enable(False)
    assert launches == {"gridder": 1}
    G = syn.random_grid(np.random.default_rng(19), p.n_w_layers, wl.grid_size)
    v = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")
    idg.degrid(p, dev(G), d["flags"], d["aterms"], d["taper"], v)
    idg.device_errors()
    parity(g.cpu().numpy(), O.grid(wl, op), f"separable with w_s, grid {case}")
    parity(v.cpu().numpy(), O.degrid(wl, op, G), f"separable with w_s, degrid {case}")
