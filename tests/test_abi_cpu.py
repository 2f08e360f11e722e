"""CPU checks of the C ABI: the library loads and exports every declared
symbol, the host planner is bit-exact with the oracle's, and invalid input is
rejected with status codes (no device calls are made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07226_gb300 import build as B
from paper_1909_07226_gb300 import idg
from paper_1909_07226_gb300 import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return idg.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "idg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(idg_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(idg.EXPORTED) == names


def test_status_strings(lib):
    for s in range(7):
        assert lib.idg_status_string(s)


@pytest.mark.parametrize("maker,kw", [
    ("tiny", {}),
    ("small", dict(seed=1, n_st=7, n_t=40, n_chan=6, L=16, N=64, diameter_m=20000.0, max_t=12)),
    ("small", dict(seed=2, n_st=5, n_t=30, n_chan=9, L=24, N=96, diameter_m=60000.0, max_t=30, n_slots=3)),
    ("small", dict(seed=3, n_st=6, n_t=20, n_chan=5, L=16, N=128, w_step=40.0, max_t=20)),
    ("small", dict(seed=4, n_st=6, n_t=20, n_chan=4, L=16, N=64, cell=6e-4, diameter_m=8000.0)),
    ("small", dict(seed=5, n_st=5, n_t=16, n_chan=16, L=16, N=256, diameter_m=60000.0, df=8e6)),
])
def test_plan_bit_exact_with_oracle(lib, maker, kw):
    wl = syn.make_tiny(with_vis=False) if maker == "tiny" else syn.make_small(with_vis=False, aterms="identity", **kw)
    p = idg.plan_from_workload(wl, n_host_threads=3)
    o = O.plan(wl)
    assert p.n_subgrids == o.n_sub
    assert np.array_equal(p.export(), o.desc)
    assert p.stats.n_vis_dropped == o.n_dropped
    assert p.stats.n_w_layers == o.n_w and p.stats.w_layer_min == o.k_min
    assert p.stats.n_vis_planned == int(o.desc[:, O.D_KP].sum())


def test_plan_bit_exact_lofar_config(lib):
    # full-size LOFAR-like workload: 1128 baselines x 4096 timesteps x 16 channels
    wl = syn.make_lofar(with_vis=False)
    p = idg.plan_from_workload(wl)
    o = O.plan(wl)
    assert np.array_equal(p.export(), o.desc)
    assert p.stats.n_vis_dropped == o.n_dropped == 0


def test_plan_independent_of_thread_count(lib):
    wl = syn.make_small(seed=9, n_st=9, n_t=30, n_chan=8, L=16, N=128, diameter_m=40000.0, with_vis=False,
                        aterms="identity")
    d1 = idg.plan_from_workload(wl, n_host_threads=1).export()
    d7 = idg.plan_from_workload(wl, n_host_threads=7).export()
    assert np.array_equal(d1, d7)


def _create(**over):
    wl = syn.make_small(seed=1, n_st=4, n_t=8, n_chan=2, L=16, N=64, with_vis=False, aterms="identity")
    args = dict(uvw_m=wl.uvw_m, freqs_hz=wl.freqs_hz, baselines=wl.baselines, aterm_offsets=wl.aterm_offsets,
                n_stations=wl.n_stations, subgrid_size=wl.subgrid_size, grid_size=wl.grid_size,
                cell_size=wl.cell_size, w_step=0.0)
    opts = {k: over.pop(k) for k in list(over) if k in ("kernel_size", "max_timesteps_per_subgrid",
                                                        "precision_mode", "fft_mode", "adder_mode")}
    args.update(over)
    return idg.plan_create(**args, **opts)


@pytest.mark.parametrize("over,needle", [
    (dict(subgrid_size=15), "even"),
    (dict(subgrid_size=6), "kernel_size"),
    (dict(grid_size=8), "grid_size"),
    (dict(cell_size=-1.0), "cell"),
    (dict(cell_size=1.0), "direction cosines"),
    (dict(w_step=-2.0), "w_step"),
    (dict(max_timesteps_per_subgrid=0), "max_timesteps"),
    (dict(kernel_size=float("nan")), "kernel_size"),
    (dict(precision_mode=7), "precision_mode"),
    (dict(adder_mode=3), "adder_mode"),
    (dict(aterm_offsets=np.array([0, 5, 5, 8], dtype=np.int32)), "increasing"),
    (dict(aterm_offsets=np.array([1, 8], dtype=np.int32)), "start at 0"),
    (dict(baselines=np.array([[0, 9]] * 6, dtype=np.int32)), "station"),
    (dict(n_stations=2), "station"),
    (dict(freqs_hz=np.array([140e6, -1.0])), "frequencies"),
])
def test_plan_rejects_invalid_input(lib, over, needle):
    with pytest.raises(idg.IDGError) as ei:
        _create(**over)
    assert ei.value.status == 1
    assert needle in str(ei.value)


def test_plan_rejects_nonfinite_uvw(lib):
    wl = syn.make_small(seed=1, n_st=4, n_t=8, n_chan=2, L=16, N=64, with_vis=False, aterms="identity")
    uvw = wl.uvw_m.copy()
    uvw[2, 3, 1] = np.nan
    with pytest.raises(idg.IDGError) as ei:
        _create(uvw_m=uvw)
    assert "finite" in str(ei.value)


def test_host_only_plan_rejects_device_calls(lib):
    # without a CUDA device the plan is host-only; device entry points refuse it
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    p = _create()
    assert p.stats.device == -1
    st = lib.idg_grid(p.handle, ctypes.c_void_p(16), None, None, ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert st == 1
    assert b"without a CUDA device" in lib.idg_last_error()


def test_recurrence_needs_uniform_channels(lib):
    wl = syn.make_small(seed=1, n_st=4, n_t=8, n_chan=4, L=16, N=64, with_vis=False, aterms="identity")
    f = wl.freqs_hz.copy()
    f[2] += 3e5
    with pytest.raises(idg.IDGError) as ei:
        _create(freqs_hz=f, precision_mode=idg.PHASOR_RECURRENCE)
    assert "uniformly spaced" in str(ei.value)
    _create(freqs_hz=f)                                   # the direct form accepts any channels
    _create(precision_mode=idg.PHASOR_RECURRENCE)         # uniform channels are accepted


def test_tensor_core_transform_only_for_subgrid_size_32(lib):
    with pytest.raises(idg.IDGError) as ei:
        _create(fft_mode=idg.FFT_TC_SPLIT)                 # L = 16
    assert ei.value.status == 6 and "subgrid size 32" in str(ei.value)
    with pytest.raises(idg.IDGError) as ei:
        _create(fft_mode=5)
    assert ei.value.status == 1 and "fft_mode" in str(ei.value)
    wl = syn.make_small(seed=1, n_st=4, n_t=8, n_chan=2, L=32, N=128, with_vis=False, aterms="identity")
    p = idg.plan_from_workload(wl, fft_mode=idg.FFT_TC_SPLIT)
    assert p.stats.subgrid_size == 32


def test_no_alloc_refuses_the_compensated_adder(lib):
    # the compensated adder needs a grid-sized buffer that the no-allocation call
    # cannot take: refused before anything is enqueued (and before device checks)
    p = _create(adder_mode=idg.ADDER_COMPENSATED)
    st = lib.idg_grid_no_alloc(p.handle, ctypes.c_void_p(16), None, None, None, ctypes.c_void_p(16), None)
    assert st == 6
    assert b"compensated" in lib.idg_last_error()


def test_kernel_choice_is_per_plan(lib):
    wl = syn.make_small(seed=1, n_st=4, n_t=8, n_chan=2, L=32, N=128, with_vis=False, aterms="identity")
    a, b = idg.plan_from_workload(wl), idg.plan_from_workload(wl)
    n = len(idg.kernel_variants("gridder", 32))
    assert n >= 2
    assert idg.plan_get_kernel_variant(a, "gridder") == idg.get_kernel_variant("gridder", 32) == 0
    idg.plan_set_kernel_variant(a, "gridder", 1)
    assert idg.plan_get_kernel_variant(a, "gridder") == 1
    assert idg.plan_get_kernel_variant(b, "gridder") == 0          # the other plan keeps its choice
    assert idg.get_kernel_variant("gridder", 32) == 0              # and so does the process
    try:
        idg.set_kernel_variant("gridder", 32, n - 1)                # process-wide default moves b, not a
        assert idg.plan_get_kernel_variant(b, "gridder") == n - 1
        assert idg.plan_get_kernel_variant(a, "gridder") == 1
        idg.plan_set_kernel_variant(a, "gridder", -1)                # back to following the process
        assert idg.plan_get_kernel_variant(a, "gridder") == n - 1
    finally:
        idg.set_kernel_variant("gridder", 32, 0)
    with pytest.raises(idg.IDGError):
        idg.plan_set_kernel_variant(a, "gridder", n)
    with pytest.raises(idg.IDGError):
        idg.plan_set_kernel_variant(a, "adder", 0)


def header_enums():
    """Every enumerator of include/idg.h with its value (implicit ones counted on)."""
    text = open(os.path.join(ROOT, "include", "idg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    values = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            name, _, val = (x.strip() for x in item.partition("="))
            nxt = int(val) if val else nxt
            values[name] = nxt
            nxt += 1
    return values


def test_binding_constants_match_the_header():
    e = header_enums()
    for py in ("PHASOR_SINCOS", "PHASOR_RECURRENCE", "FFT_FP32", "FFT_TC_SPLIT", "ADDER_ATOMIC",
               "ADDER_COMPENSATED", "ADDER_SORTED", "TAPER_PSWF", "TAPER_IDG_OPTIMAL", "BATCH_GRAPH"):
        assert getattr(idg, py) == e["IDG_" + py], py
    assert idg.STATUS_NAMES == {v: k for k, v in e.items() if k == "IDG_OK" or k.startswith("IDG_ERR_")}
    kernels = sorted((v, k) for k, v in e.items() if k.startswith("IDG_KERNEL_") and k != "IDG_KERNEL_COUNT")
    assert idg.KERNELS == [k[len("IDG_KERNEL_"):].lower() for _, k in kernels]
    assert e["IDG_KERNEL_COUNT"] == len(idg.KERNELS)
    desc = sorted((v, k) for k, v in e.items() if k.startswith("IDG_DESC_"))
    assert [v for v, _ in desc] == list(range(idg.DESC_FIELDS))
    assert [k for _, k in desc][:2] == ["IDG_DESC_BASELINE", "IDG_DESC_SLOT"]
