"""GPU parity of the separable tensor-core kernels at L = 24 and 16 (the plans of
the small, narrow-field workloads below pass the remainder bound, so the
composite calls run the fused separable gridder and degridder), against the
FP64 oracle on the same seeded inputs: relative RMS <= 1e-5
(tests.gpu_util.parity).

Cases: subgrids of up to 1024 visibilities (two staged batches and two
accumulation periods of the gridder), W-layers, no A-terms, flags, and
subgrids of at most 32 visibilities.  Where most visibilities lie in subgrids
of fewer than 64, the degridder takes the unfused splitter, transform and
packed kernel, as at L = 32."""
import numpy as np
import pytest

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
    "long_kp": dict(seed=81, n_st=5, n_t=128, n_chan=16, L=24, N=128, max_t=128, n_slots=2, flag_p=0.1,
                    diameter_m=2500.0, df=0.25e6),
    "w_layers": dict(seed=82, n_st=5, n_t=96, n_chan=8, L=24, N=128, max_t=96, n_slots=1, flag_p=0.05,
                     diameter_m=2500.0, df=0.25e6, w_step=20.0),
    "no_aterms": dict(seed=85, n_st=5, n_t=96, n_chan=8, L=24, N=128, max_t=96, n_slots=1, flag_p=0.0,
                      diameter_m=2500.0, df=0.25e6, aterms="identity"),
    "short_kp": dict(seed=83, n_st=6, n_t=48, n_chan=4, L=24, N=128, max_t=8, n_slots=2, flag_p=0.1,
                     diameter_m=2500.0, df=0.25e6),
    "L16_long_kp": dict(seed=91, n_st=5, n_t=128, n_chan=16, L=16, N=128, max_t=128, n_slots=2, flag_p=0.1,
                        diameter_m=1200.0, df=0.25e6),
    "L16_w_layers": dict(seed=92, n_st=5, n_t=96, n_chan=8, L=16, N=128, max_t=96, n_slots=1, flag_p=0.05,
                         diameter_m=1200.0, df=0.25e6, w_step=20.0),
    "L16_short_kp": dict(seed=93, n_st=6, n_t=48, n_chan=4, L=16, N=128, max_t=8, n_slots=2, flag_p=0.1,
                         diameter_m=1200.0, df=0.25e6),
}


def _launches(prof):
    return {k: v["launches"] for k, v in prof.items() if v["launches"]}


@pytest.mark.parametrize("case", sorted(CASES))
def test_separable_l24_grid_and_degrid(case):
    import torch
    wl = syn.make_small(**CASES[case])
    p = idg.plan_from_workload(wl)
    assert p.stats.separable == 1
    op = O.plan(wl)
    d = workload_to_device(wl)
    aterms = None if case == "no_aterms" else d["aterms"]
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    idg.profile_enable(True)
    try:
        idg.profile_read(reset=True)
        idg.grid(p, d["vis"], d["flags"], aterms, d["taper"], g)
        grid_launches = _launches(idg.profile_read(reset=True))
        G = syn.random_grid(np.random.default_rng(13), p.n_w_layers, wl.grid_size)
        v = torch.full(wl.vis.shape, 5.0 + 5.0j, dtype=torch.complex64, device="cuda")
        idg.degrid(p, dev(G), d["flags"], aterms, d["taper"], v)
        degrid_launches = _launches(idg.profile_read(reset=True))
    finally:
        idg.profile_enable(False)
    idg.device_errors()
    assert grid_launches == {"gridder": 1}          # one fused separable launch
    # the degridder fuses when at least half the visibilities lie in subgrids of 64 or more
    kp = p.export()[:, O.D_KP]
    if 2 * kp[kp < 64].sum() <= kp.sum():
        assert degrid_launches == {"degridder": 1}
    else:
        assert "splitter" in degrid_launches and "fft" in degrid_launches
    if case in ("long_kp", "L16_long_kp"):
        assert degrid_launches == {"degridder": 1}
    # (no_aterms: the workload's A-terms are the identity, which the oracle applies)
    parity(g.cpu().numpy(), O.grid(wl, op), f"separable grid {case}")
    parity(v.cpu().numpy(), O.degrid(wl, op, G), f"separable degrid {case}")


def test_separable_l24_accumulates_and_flags_zero():
    import torch
    wl = syn.make_small(**CASES["long_kp"])
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    g0 = syn.random_grid(np.random.default_rng(17), p.n_w_layers, wl.grid_size)
    g = dev(g0)
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    idg.device_errors()
    parity(g.cpu().numpy(), g0 + O.grid(wl, op), "separable L=24 grid added into a filled grid")
    # every visibility flagged: nothing is added, and the model visibilities are zero
    flags = torch.ones(wl.vis.shape[:3], dtype=torch.uint8, device="cuda")
    g2 = torch.zeros_like(g)
    idg.grid(p, d["vis"], flags, d["aterms"], d["taper"], g2)
    v = torch.full(wl.vis.shape, 1.0 + 1.0j, dtype=torch.complex64, device="cuda")
    idg.degrid(p, dev(g0), flags, d["aterms"], d["taper"], v)
    idg.device_errors()
    torch.cuda.synchronize()
    assert float(g2.abs().max()) == 0.0
    assert float(v.abs().max()) == 0.0


def test_separable_l24_stage_and_composite_agree():
    # the separable composite call against the unfused stage kernels (packed FP32) of the
    # same plan: both against the oracle, and against each other
    import torch
    wl = syn.make_small(**CASES["w_layers"])
    p = idg.plan_from_workload(wl)
    d = workload_to_device(wl)
    n = p.n_subgrids
    shape = (p.n_w_layers, wl.grid_size, wl.grid_size, 4)
    g_comp = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g_comp)
    sub = torch.zeros((n, wl.subgrid_size, wl.subgrid_size, 4), dtype=torch.complex64, device="cuda")
    g_stage = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    idg.grid_subgrids(p, 0, n, d["vis"], d["flags"], d["aterms"], d["taper"], sub)
    idg.fft_subgrids(p, n, -1, sub)
    idg.add_subgrids(p, 0, n, sub, g_stage)
    idg.device_errors()
    parity(g_comp.cpu().numpy(), g_stage.cpu().numpy(), "separable L=24 composite vs stage kernels")
