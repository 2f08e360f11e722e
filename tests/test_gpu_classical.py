"""GPU parity of classical gridding with oversampled A/W-projection kernels
(idg_classical_grid; Sect. 2) against the FP64 classical oracle, which is
itself pinned to direct kernel evaluation, to image domain gridding with the
exact kernel and to the 1/O convergence of the lookup
(tests/test_classical_cpu.py).

The library and the oracle take the same discrete decisions (support start,
table phase, W-projection plane: FP64 with each operation rounded), so the
comparison is at FP32 rounding level: relative RMS <= 1e-5."""
import numpy as np
import pytest

from oracle import classical as CL
from oracle import oracle as O
from paper_1909_07226_gb300 import idg
from paper_1909_07226_gb300 import synthetic as syn
from tests.gpu_util import dev, parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_07226_gb300 import build
    build.build()
    idg.load()


CASES = {
    # name: (workload, support M, oversampling O, plane spacing dw, A-terms on the kernel lattice)
    "L16_M8_O16_identity": (dict(seed=91, n_st=5, n_t=24, n_chan=4, L=16, N=128, max_t=24, n_slots=1,
                                 aterms="identity"), 8, 16, 0.0, False),
    "L24_M8_O8_aterms_wplanes_flags": (dict(seed=92, n_st=6, n_t=20, n_chan=4, L=24, N=128, max_t=10, n_slots=2,
                                            flag_p=0.15, diameter_m=15000.0), 8, 8, 4.0, True),
    "L16_M6_O32_wlayers": (dict(seed=93, n_st=5, n_t=16, n_chan=3, L=16, N=64, max_t=8, n_slots=2, w_step=20.0,
                                diameter_m=20000.0), 6, 32, 2.0, True),
    # the widest support (the builder takes the Mueller entries 4 at a time) and an
    # oversampling that 4 does not divide
    "L32_M32_O6": (dict(seed=95, n_st=4, n_t=8, n_chan=2, L=32, N=128, max_t=8, n_slots=1, diameter_m=3000.0),
                   32, 6, 0.0, True),
    # subgrids on the first grid row: supports reach past the grid and are clipped
    "L32_M16_O4_grid_edge": (dict(seed=94, n_st=5, n_t=12, n_chan=3, L=32, N=96, max_t=12, n_slots=1,
                                  diameter_m=4000.0, cell=3.4529525903487945e-4), 16, 4, 0.0, True),
}


def _case(name):
    kw, M, O_, dw, with_a = CASES[name]
    wl = syn.make_small(**kw)
    S = wl.grid_size * wl.cell_size
    am = syn.aterms_on_subgrid(wl.screens, M, S).astype(np.complex64) if with_a else None
    a = syn.pswf_1d(M, float(M))
    tap = np.outer(a, a).astype(np.float32)
    return wl, M, O_, dw, am, tap


@pytest.mark.parametrize("name", sorted(CASES))
def test_classical_grid_matches_the_oracle(name):
    import torch
    wl, M, O_, dw, am, tap = _case(name)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    idg.classical_grid(p, M, O_, dw, dev(wl.vis), dev(wl.flags), dev(am), dev(tap), g)
    idg.device_errors()
    ref = CL.grid(wl, op, M, O_, dw=dw, aterms=am, taper=tap)
    parity(g.cpu().numpy(), ref, f"classical {name}")


def test_classical_default_window_and_accumulation():
    import torch
    wl, M, O_, dw, am, tap = _case("L16_M8_O16_identity")
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    a, _ = idg.taper_window(M, float(M), idg.TAPER_PSWF)
    ref = CL.grid(wl, op, M, O_, dw=dw, taper=np.outer(a, a).astype(np.float32))
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    for _ in range(2):
        idg.classical_grid(p, M, O_, dw, dev(wl.vis), None, None, None, g)
    idg.device_errors()
    parity(g.cpu().numpy(), 2 * ref, "classical, default window, added twice")
    with pytest.raises(idg.IDGError):
        idg.classical_grid(p, 7, O_, dw, dev(wl.vis), None, None, None, g)      # odd support
    with pytest.raises(idg.IDGError):
        idg.classical_grid(p, M, 0, dw, dev(wl.vis), None, None, None, g)       # no oversampling
