"""idg_grid_no_alloc: gridding for callers that cannot allocate device memory.

Such callers (a pipeline that reserves its whole device-memory budget up
front, or a host framework whose allocator already holds all free device
memory) use this entry point, whose subgrid scratch is a fixed 64 MiB array
inside the library.  The test calls it through the C ABI twice in a row, on
two different plans, and compares each result with idg_grid's on the same
inputs within the parity tolerance of the other GPU tests, and with the FP64
oracle (the default and the recurrence + split tensor-core forms).  It also checks
that an over-size plan is refused before any work is done and that a call
leaves the free device memory unchanged.  This file is collected last, so a
run that stops at the first failure has run every other test already.
"""
import ctypes

import numpy as np
import pytest

from paper_1909_07226_gb300 import idg
from paper_1909_07226_gb300 import synthetic as syn
from tests.gpu_util import parity, workload_to_device

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 64 << 20


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_07226_gb300 import build
    build.build()
    idg.load()


def _reference_and_no_alloc(wl, **opt):
    import torch
    p = idg.plan_from_workload(wl, **opt)
    assert p.n_subgrids * wl.subgrid_size ** 2 * 32 <= SCRATCH_BYTES
    d = workload_to_device(wl)
    shape = (p.n_w_layers, wl.grid_size, wl.grid_size, 4)
    ref = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], ref)
    out = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    lib = idg.load()
    st = lib.idg_grid_no_alloc(p.handle, ctypes.c_void_p(d["vis"].data_ptr()),
                               ctypes.c_void_p(d["flags"].data_ptr()) if d["flags"] is not None else None,
                               ctypes.c_void_p(d["aterms"].data_ptr()) if d["aterms"] is not None else None,
                               ctypes.c_void_p(d["taper"].data_ptr()), ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.idg_last_error()
    torch.cuda.synchronize()
    return p, ref.cpu().numpy(), out.cpu().numpy()


def _w_layer_workload():
    return syn.make_small(seed=515, n_st=7, n_t=40, n_chan=6, L=32, N=256, max_t=10, n_slots=2, flag_p=0.1,
                          w_step=20.0, diameter_m=15000.0)


@pytest.mark.parametrize("form", ["default", "recurrence_tc_split"])
@pytest.mark.parametrize("case", ["tiny", "L32_w_layers"])
def test_no_alloc_matches_the_oracle(case, form):
    # against the FP64 oracle itself (Alg. 1 end to end), not only against idg_grid
    from oracle import oracle as O
    wl = syn.make_tiny() if case == "tiny" else _w_layer_workload()
    if form == "recurrence_tc_split" and wl.subgrid_size != 32:
        pytest.skip("the split tensor-core transform is built for L = 32")
    opt = {} if form == "default" else dict(precision_mode=idg.PHASOR_RECURRENCE, fft_mode=idg.FFT_TC_SPLIT)
    _, _, out = _reference_and_no_alloc(wl, **opt)
    parity(out, O.grid(wl, O.plan(wl)), f"no-alloc {case} {form} vs oracle")


def test_no_alloc_matches_idg_grid_on_two_calls_in_a_row():
    # first call: the tiny workload (112 subgrids of 24 x 24)
    p1, ref1, out1 = _reference_and_no_alloc(syn.make_tiny())
    parity(out1, ref1, "no-alloc call 1 vs idg_grid")
    # second call: another plan with more subgrids, A-terms, flags, W-layers;
    # the scratch still holds call 1's subgrids and must not leak into it
    wl2 = _w_layer_workload()
    p2, ref2, out2 = _reference_and_no_alloc(wl2)
    assert p2.n_subgrids > p1.n_subgrids and p2.n_w_layers > 1
    parity(out2, ref2, "no-alloc call 2 vs idg_grid")


def test_no_alloc_allocates_nothing():
    import torch
    wl = syn.make_tiny()
    p = idg.plan_from_workload(wl)
    d = workload_to_device(wl)
    g = torch.zeros((1, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    idg.grid_no_alloc(p, d["vis"], None, d["aterms"], d["taper"], g)      # loads the module
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        idg.grid_no_alloc(p, d["vis"], None, d["aterms"], d["taper"], g)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_no_alloc_rejects_plans_beyond_the_scratch():
    import torch
    # 51 325 subgrids of 32 x 32 need 1.6 GB, far beyond the 64 MiB scratch
    wl = syn.make_lofar(with_vis=False, n_t=512)
    p = idg.plan_from_workload(wl)
    assert p.n_subgrids * 32 * 32 * 32 > SCRATCH_BYTES
    g = torch.zeros((1, 8, 8, 4), dtype=torch.complex64, device="cuda")   # never touched
    lib = idg.load()
    st = lib.idg_grid_no_alloc(p.handle, ctypes.c_void_p(g.data_ptr()), None, None,
                               ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(g.data_ptr()), None)
    assert st == 1
    msg = lib.idg_last_error().decode()
    assert "scratch" in msg and str(SCRATCH_BYTES) in msg and "2048 subgrids" in msg


def test_no_alloc_precision_forms_near_the_limit():
    # the channel-recurrence gridder and the split tensor-core transform on the
    # static array, with a plan that fills most of it (the LOFAR-like workload's
    # first 128 timesteps: 1601 subgrids of 32 x 32, 78 % of the 64 MiB)
    wl = syn.make_lofar(n_t=128)
    p, ref, out = _reference_and_no_alloc(wl, precision_mode=idg.PHASOR_RECURRENCE, fft_mode=idg.FFT_TC_SPLIT)
    assert p.n_subgrids * 32 * 32 * 32 > SCRATCH_BYTES // 2
    parity(out, ref, "no-alloc recurrence + tensor-core transform vs idg_grid")


def test_no_alloc_warm_up_call_and_compensated_plans():
    import torch
    lib = idg.load()
    # a plan without subgrids (every visibility off the grid) only resolves the
    # array's address: the warm-up call
    wl = syn.make_small(seed=1, n_st=4, n_t=4, n_chan=2, L=16, N=64, cell=0.02, diameter_m=20000.0)
    p = idg.plan_from_workload(wl)
    assert p.n_subgrids == 0
    d = workload_to_device(wl)
    g = torch.zeros((1, 64, 64, 4), dtype=torch.complex64, device="cuda")
    idg.grid_no_alloc(p, d["vis"], None, None, None, g)
    torch.cuda.synchronize()
    assert float(g.abs().max()) == 0.0
    # the compensated adder would need a grid-sized buffer: refused, grid untouched
    wl = syn.make_tiny()
    p = idg.plan_from_workload(wl, adder_mode=idg.ADDER_COMPENSATED)
    d = workload_to_device(wl)
    g = torch.zeros((1, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(idg.IDGError) as ei:
        idg.grid_no_alloc(p, d["vis"], None, d["aterms"], d["taper"], g)
    assert ei.value.status == 6 and "compensated" in str(ei.value)
    torch.cuda.synchronize()
    assert float(g.abs().max()) == 0.0
