"""GPU tests of the sorted (deterministic) adder, IDG_ADDER_SORTED: one CTA per 32 x 32
grid tile sums the subgrids that overlap it in plan order and adds the sum with plain
stores; a tile that more than 64 subgrids overlap takes a cluster of 8 CTAs, each summing
a fixed segment of the tile's list, the partial sums added in rank order.  The grid
matches the FP64 oracle (relative RMS <= 1e-5, tests.gpu_util.parity) and is the same bit
for bit on repeated calls, through the device-buffer composite call (mixed plan:
separable and direct parts), plan-order ranges, W-layers, the host-buffer call and the
stage add; idg_grid_no_alloc gives the same bits as idg_grid."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07226_gb300 import idg
from paper_1909_07226_gb300 import synthetic as syn
from tests.gpu_util import parity, workload_to_device

pytestmark = pytest.mark.gpu

CASES = {
    # a mixed plan (separable subgrids, pieces are not used with this adder, direct rest)
    "L32_mixed": dict(seed=91, n_st=5, n_t=128, n_chan=16, L=32, N=512, max_t=128, n_slots=2, flag_p=0.1,
                      diameter_m=300.0, cell=8e-4, df=0.25e6),
    "L24_w_layers": dict(seed=94, n_st=5, n_t=64, n_chan=8, L=24, N=256, max_t=32, n_slots=2, flag_p=0.1,
                         diameter_m=20000.0, w_step=20.0),
    # a grid size that is not a multiple of the tile (partial tiles at the edges)
    "L16_ragged_tiles": dict(seed=95, n_st=6, n_t=48, n_chan=4, L=16, N=200, max_t=16, n_slots=1, flag_p=0.0,
                             diameter_m=1500.0),
    # short baselines, short subgrids: 896 subgrids on a few central tiles, 12 (L = 16) and 17
    # (L = 24, ragged edge) of them overlapped by more than 64 subgrids (up to 145 and 205),
    # beside tiles with short lists
    "L16_heavy_tiles": dict(seed=96, n_st=8, n_t=256, n_chan=4, L=16, N=256, max_t=8, n_slots=2, flag_p=0.05,
                            diameter_m=300.0),
    "L24_heavy_tiles_ragged": dict(seed=96, n_st=8, n_t=256, n_chan=4, L=24, N=200, max_t=8, n_slots=2,
                                   flag_p=0.05, diameter_m=300.0),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_07226_gb300 import build
    build.build()
    idg.load()


@pytest.mark.parametrize("case", sorted(CASES))
def test_sorted_adder_matches_the_oracle_bit_for_bit_on_repeats(case):
    import torch
    wl = syn.make_small(**CASES[case])
    p = idg.plan_from_workload(wl, adder_mode=idg.ADDER_SORTED)
    op = O.plan(wl)
    d = workload_to_device(wl)
    shape = (p.n_w_layers, wl.grid_size, wl.grid_size, 4)
    outs = []
    for _ in range(3):
        g = torch.zeros(shape, dtype=torch.complex64, device="cuda")
        idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
        idg.device_errors()
        outs.append(g.cpu().numpy())
    assert all(np.array_equal(outs[0].view(np.uint32), o.view(np.uint32)) for o in outs[1:])
    parity(outs[0], O.grid(wl, op), f"sorted adder {case}")


@pytest.mark.parametrize("case", ["L32_mixed", "L24_heavy_tiles_ragged"])
def test_sorted_adder_ranges_and_host_buffers(case):
    # (in the heavy-tile case the range boundary cuts the long lists: each range's part of
    # a list is split over the cluster on its own)
    import torch
    wl = syn.make_small(**CASES[case])
    p = idg.plan_from_workload(wl, adder_mode=idg.ADDER_SORTED)
    op = O.plan(wl)
    d = workload_to_device(wl)
    n = p.n_subgrids
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    idg.grid_range(p, 0, n // 2, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    idg.grid_range(p, n // 2, n - n // 2, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    idg.device_errors()
    parity(g.cpu().numpy(), O.grid(wl, op), f"sorted adder, two ranges {case}")
    gh = np.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=np.complex64)
    idg.grid_host(p, wl.vis.astype(np.complex64), wl.flags, wl.aterms.astype(np.complex64),
                  wl.taper.astype(np.float32), gh)
    parity(gh, O.grid(wl, op), f"sorted adder, host buffers {case}")


@pytest.mark.parametrize("case", ["L16_ragged_tiles", "L16_heavy_tiles"])
def test_no_alloc_with_the_sorted_adder(case):
    # the static scratch holds the whole plan in plan order: the same bits as idg_grid
    import torch
    wl = syn.make_small(**CASES[case])
    p = idg.plan_from_workload(wl, adder_mode=idg.ADDER_SORTED)
    d = workload_to_device(wl)
    shape = (p.n_w_layers, wl.grid_size, wl.grid_size, 4)
    g0 = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    idg.grid_no_alloc(p, d["vis"], d["flags"], d["aterms"], d["taper"], g0)
    g1 = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g1)
    idg.device_errors()
    a, b = g0.cpu().numpy(), g1.cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    parity(a, O.grid(wl, O.plan(wl)), f"sorted adder, no allocation {case}")


def test_stage_add_of_a_sorted_plan():
    # idg_add_subgrids of a sorted plan takes the tile adder: the same bits on every call,
    # and the oracle's grid after the stage gridder and transform
    import torch
    wl = syn.make_small(**CASES["L24_heavy_tiles_ragged"])
    p = idg.plan_from_workload(wl, adder_mode=idg.ADDER_SORTED)
    d = workload_to_device(wl)
    n, L = p.n_subgrids, wl.subgrid_size
    sub = torch.zeros((n, L, L, 4), dtype=torch.complex64, device="cuda")
    idg.grid_subgrids(p, 0, n, d["vis"], d["flags"], d["aterms"], d["taper"], sub)
    idg.fft_subgrids(p, n, -1, sub)
    outs = []
    for _ in range(2):
        g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
        idg.add_subgrids(p, 0, n, sub, g)
        outs.append(g.cpu().numpy())
    idg.device_errors()
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))
    parity(outs[0], O.grid(wl, O.plan(wl)), "sorted plan, stage calls")
