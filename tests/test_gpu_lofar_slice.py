"""Full parity of the composite path the benchmark times, on the LOFAR-like
workload cut to its first 256 timesteps (1128 baselines x 256 x 16 channels =
4.6 M visibilities, 3206 subgrids of 32 x 32, A-terms every 128 timesteps,
4096^2 x 4 grid).

At this size the plan is separable, so idg_grid and idg_degrid each run one
fused separable tensor-core launch, exactly as on the full workload.  Every
pixel of the grid and every visibility is compared with the FP64 oracle
(about half a minute of oracle time per direction on 16 host cores).  The same
grid is then rebuilt from two plan-order ranges, as two ranks of the sharded
form would (idg_grid_range, summed), and through the host-buffer call.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07226_gb300 import idg
from paper_1909_07226_gb300 import synthetic as syn
from tests.gpu_util import dev, parity, workload_to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sl():
    from paper_1909_07226_gb300 import build
    build.build()
    idg.load()
    wl = syn.make_lofar(n_t=256)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    assert np.array_equal(p.export(), op.desc)
    assert p.stats.separable == 1
    return dict(wl=wl, p=p, op=op, d=workload_to_device(wl), ref=O.grid(wl, op))


def test_slice_grid_every_pixel(sl):
    import torch
    wl, p, d = sl["wl"], sl["p"], sl["d"]
    idg.profile_enable(True)
    idg.profile_read(reset=True)
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    prof = idg.profile_read(reset=True)
    idg.profile_enable(False)
    idg.device_errors()
    # one launch, no adder: the fused separable kernel
    assert prof["gridder"]["launches"] == 1 and prof["adder"]["launches"] == 0 and prof["fft"]["launches"] == 0
    parity(g.cpu().numpy(), sl["ref"], "LOFAR slice composite grid (fused separable), every pixel")


def test_slice_degrid_every_visibility(sl):
    import torch
    wl, p, op, d = sl["wl"], sl["p"], sl["op"], sl["d"]
    G = syn.random_grid(np.random.default_rng(256), p.n_w_layers, wl.grid_size)
    idg.profile_enable(True)
    idg.profile_read(reset=True)
    v = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")
    idg.degrid(p, dev(G), d["flags"], d["aterms"], d["taper"], v)
    prof = idg.profile_read(reset=True)
    idg.profile_enable(False)
    idg.device_errors()
    assert prof["degridder"]["launches"] == 1 and prof["splitter"]["launches"] == 0
    parity(v.cpu().numpy(), O.degrid(wl, op, G), "LOFAR slice composite degrid (fused separable), every visibility")


def test_slice_two_ranges_and_host_call(sl):
    import torch
    wl, p, d = sl["wl"], sl["p"], sl["d"]
    from paper_1909_07226_gb300 import shard
    (f0, c0), (f1, c1) = shard.shard_ranges(p.export()[:, idg.DESC_FIELDS - 1], 2)
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    part = torch.zeros_like(g)
    for f, c in ((f0, c0), (f1, c1)):
        part.zero_()
        idg.grid_range(p, f, c, d["vis"], d["flags"], d["aterms"], d["taper"], part)
        g += part
    parity(g.cpu().numpy(), sl["ref"], "LOFAR slice, two shard ranges summed")
    gh = np.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=np.complex64)
    idg.grid_host(p, wl.vis, wl.flags, wl.aterms, wl.taper.astype(np.float32), gh)
    parity(gh, sl["ref"], "LOFAR slice, host-buffer grid")
