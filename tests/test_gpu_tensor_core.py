"""GPU parity of the tensor-core gridder (tcgen05, L = 32) against the FP64 oracle.

The variant forms the phasors on the CUDA cores, splits phasors and
visibilities into FP16 hi + lo parts (visibilities after a power-of-two scale
per subgrid) and sums three FP16 products per term with FP32 accumulation in
tensor memory.  The cases probe what that design can get wrong: visibility
magnitudes far outside the FP16 range (the per-subgrid scale), a wide dynamic
range inside one subgrid, the W term, ragged groups of eight visibilities,
fully flagged subgrids, and the full grid pipeline.  Same bar as every other
kernel: relative RMS <= 1e-5 against the oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07226_gb300 import idg
from paper_1909_07226_gb300 import synthetic as syn
from tests.gpu_util import dev, parity, workload_to_device

pytestmark = pytest.mark.gpu

TC = "tcgen05_fp16x3_nt256"


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_07226_gb300 import build
    build.build()
    idg.load()


@pytest.fixture
def tc_selected():
    names = idg.kernel_variants("gridder", 32)
    assert TC in names
    idg.set_kernel_variant("gridder", 32, names.index(TC))
    yield
    idg.set_kernel_variant("gridder", 32, 0)


def small32(**kw):
    args = dict(seed=1032, n_st=5, n_t=48, n_chan=5, L=32, N=128, max_t=48, n_slots=1, flag_p=0.1,
                diameter_m=3000.0)
    args.update(kw)
    return syn.make_small(**args)


def _scaled(wl, f):
    wl.vis = (wl.vis * np.float32(f)).astype(np.complex64)
    return wl


def _outliers(wl):
    # noise with 1% of the visibilities 10^4 times larger
    rng = np.random.default_rng(77)
    v = syn.gaussian_noise(rng, wl.vis.shape, 1.0)
    big = rng.random(wl.vis.shape[:3]) < 0.01
    v[big] *= np.float32(1e4)
    wl.vis = v
    return wl


CASES = {
    "points_flags_aterms": lambda: small32(),
    "tiny_magnitudes": lambda: _scaled(small32(), 1e-9),
    "huge_magnitudes": lambda: _scaled(small32(), 1e9),
    "outliers": lambda: _outliers(small32()),
    "w_layers": lambda: small32(w_step=20.0, diameter_m=20000.0, n_t=24, max_t=12),
    "ragged_groups": lambda: small32(n_chan=3, n_t=37, max_t=37, flag_p=0.0),
    "ragged_batches": lambda: small32(n_t=47, n_chan=5, max_t=47),
    # K_p = 2048 as in the LOFAR configuration: 8 folds of the hh | hl accumulators
    "long_kp": lambda: small32(n_t=128, n_chan=16, max_t=128, n_st=4, df=0.25e6),
    "wide_channels": lambda: small32(aterms="identity", n_chan=16, diameter_m=30000.0, df=4e6),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_tc_gridder_stage(case, tc_selected):
    import torch
    wl = CASES[case]()
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    n = p.n_subgrids
    sub = torch.zeros((n, 32, 32, 4), dtype=torch.complex64, device="cuda")
    idg.grid_subgrids(p, 0, n, d["vis"], d["flags"], d["aterms"], d["taper"], sub)
    idg.device_errors()
    parity(sub.cpu().numpy(), O.subgrid_images(wl, op), f"tc gridder {case}")


def test_tc_gridder_kp_spans_batches(tc_selected):
    # K_p above 128 (several staged batches) and not a multiple of 8
    wl = small32(n_t=47, n_chan=5, max_t=47)
    op = O.plan(wl)
    kp = op.desc[:, O.D_KP]
    assert kp.max() > 128 and np.any(kp % 8 != 0)


def test_tc_gridder_all_flagged_is_zero(tc_selected):
    import torch
    wl = small32(flag_p=0.0)
    wl.flags = np.ones(wl.vis.shape[:3], dtype=np.uint8)
    p = idg.plan_from_workload(wl)
    d = workload_to_device(wl)
    n = p.n_subgrids
    sub = torch.full((n, 32, 32, 4), 3.0 + 3.0j, dtype=torch.complex64, device="cuda")
    idg.grid_subgrids(p, 0, n, d["vis"], d["flags"], d["aterms"], d["taper"], sub)
    idg.device_errors()
    assert not torch.any(sub != 0).item()


def test_tc_full_grid(tc_selected):
    import torch
    wl = small32(w_step=20.0, diameter_m=20000.0, n_t=24, max_t=12)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    idg.device_errors()
    parity(g.cpu().numpy(), O.grid(wl, op), "tc grid")


def test_tc_gridder_lofar_slice_sampled(tc_selected):
    # a LOFAR slice (48 stations, 16 channels, 64 timesteps): every subgrid is
    # gridded in one launch; a strided sample of 96 is checked against the oracle
    import torch
    wl = syn.make_lofar(n_t=64, slot_len=64, name="lofar-tc")
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    n = p.n_subgrids
    sub = torch.zeros((n, 32, 32, 4), dtype=torch.complex64, device="cuda")
    idg.grid_subgrids(p, 0, n, d["vis"], d["flags"], d["aterms"], d["taper"], sub)
    idg.device_errors()
    ids = np.linspace(0, n - 1, 96).round().astype(np.int32)
    parity(sub[torch.from_numpy(ids).long().cuda()].cpu().numpy(), O.subgrid_images(wl, op, ids=ids),
           "tc gridder LOFAR slice, sampled")
