"""GPU parity of plans whose subgrids meet the separable remainder bound only in
part (0 < n_sep_subgrids < n_subgrids): the composite calls grid and degrid the
subgrids within the bound with the separable tensor-core kernels and the rest with
the direct kernels, in separate launches into the same grid (visibilities), and
take subgrids outside the bound as pieces (blocks of their timesteps and channels,
each within the bound with its own w offset) where the plan splits them.  Also
through a plan-order range (the direct kernels take a range whose separable
subgrids do not come first), the compensated adder (no pieces: the separable head
and the direct rest), the host-buffer call and a batch.  Against the FP64
oracle, relative RMS <= 1e-5 (tests.gpu_util.parity)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07226_gb300 import idg
from paper_1909_07226_gb300 import synthetic as syn
from tests.gpu_util import dev, parity, workload_to_device

pytestmark = pytest.mark.gpu

CASES = {
    # long K_p: every subgrid outside the bound is split into pieces (one fused separable
    # launch per direction)
    "L32": dict(seed=91, n_st=5, n_t=128, n_chan=16, L=32, N=512, max_t=128, n_slots=2, flag_p=0.1,
                diameter_m=300.0, cell=8e-4, df=0.25e6),
    "L24": dict(seed=91, n_st=5, n_t=128, n_chan=16, L=24, N=384, max_t=128, n_slots=2, flag_p=0.1,
                diameter_m=800.0, cell=8e-4, df=0.25e6),
    "L16": dict(seed=91, n_st=5, n_t=128, n_chan=16, L=16, N=256, max_t=128, n_slots=2, flag_p=0.1,
                diameter_m=800.0, cell=1.2e-3, df=0.25e6),
    # W-layers and short K_p: some subgrids stay with the direct kernels (too short to
    # split), and the degridder's parts run unfused
    "L32_w_layers": dict(seed=91, n_st=5, n_t=64, n_chan=8, L=32, N=512, max_t=32, n_slots=2, flag_p=0.1,
                         diameter_m=800.0, cell=8e-4, df=0.5e6, w_step=5.0),
    "L24_w_layers": dict(seed=91, n_st=5, n_t=64, n_chan=8, L=24, N=384, max_t=32, n_slots=2, flag_p=0.1,
                         diameter_m=800.0, cell=8e-4, df=0.5e6, w_step=10.0),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_07226_gb300 import build
    build.build()
    idg.load()


def _mixed(case):
    wl = syn.make_small(**CASES[case])
    p = idg.plan_from_workload(wl)
    assert 0 < p.stats.n_sep_subgrids < p.n_subgrids and p.stats.separable == 0
    return wl, p


@pytest.mark.parametrize("case", sorted(CASES))
def test_mixed_plan_composite(case):
    import torch
    wl, p = _mixed(case)
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
    st = p.stats
    if wl.subgrid_size == 16:
        assert st.n_split_subgrids == 0                 # the direct kernels are as fast at L = 16
    else:
        assert st.n_split_subgrids > 0 and st.n_pieces >= 2 * st.n_split_subgrids
    if st.n_sep_subgrids + st.n_split_subgrids == p.n_subgrids:
        assert launches == {"gridder": 1}               # separable subgrids and pieces in one launch
    elif wl.subgrid_size == 32:
        assert launches == {"gridder": 2}               # the separable and the direct fused launch
    else:
        assert launches["gridder"] >= 2 and launches["adder"] >= 1
    G = syn.random_grid(np.random.default_rng(31), p.n_w_layers, wl.grid_size)
    v = torch.full(wl.vis.shape, complex(3.0, -7.0), dtype=torch.complex64, device="cuda")
    idg.degrid(p, dev(G), d["flags"], d["aterms"], d["taper"], v)
    idg.device_errors()
    parity(g.cpu().numpy(), O.grid(wl, op), f"mixed plan grid {case}")
    parity(v.cpu().numpy(), O.degrid(wl, op, G), f"mixed plan degrid {case}")


@pytest.mark.parametrize("case", ["L32", "L24"])
def test_mixed_plan_ranges(case):
    # plan-order ranges (separable and direct subgrids interleaved): each range alone
    # matches the oracle's range, and the ranges sum to the whole plan
    import torch
    wl, p = _mixed(case)
    op = O.plan(wl)
    d = workload_to_device(wl)
    n = p.n_subgrids
    cut = n // 3
    g_all = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    for f, c in ((0, cut), (cut, n - cut)):
        g = torch.zeros_like(g_all)
        idg.grid_range(p, f, c, d["vis"], d["flags"], d["aterms"], d["taper"], g)
        parity(g.cpu().numpy(), O.grid(wl, op, ids=np.arange(f, f + c)), f"mixed {case} grid range [{f}, {f + c})")
        g_all += g
    idg.device_errors()
    parity(g_all.cpu().numpy(), O.grid(wl, op), f"mixed {case} grid ranges summed")
    G = syn.random_grid(np.random.default_rng(37), p.n_w_layers, wl.grid_size)
    v = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")
    for f, c in ((0, cut), (cut, n - cut)):
        idg.degrid_range(p, f, c, dev(G), d["flags"], d["aterms"], d["taper"], v)
    idg.device_errors()
    parity(v.cpu().numpy(), O.degrid(wl, op, G), f"mixed {case} degrid ranges")


@pytest.mark.parametrize("case", ["L32", "L24"])
def test_mixed_plan_compensated_adder(case):
    # unfused: the separable subgrids first, then the direct ones, through the scratch
    import torch
    wl = syn.make_small(**CASES[case])
    p = idg.plan_from_workload(wl, adder_mode=1)
    assert 0 < p.stats.n_sep_subgrids < p.n_subgrids
    op = O.plan(wl)
    d = workload_to_device(wl)
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    idg.device_errors()
    parity(g.cpu().numpy(), O.grid(wl, op), f"mixed {case} compensated adder")


@pytest.mark.parametrize("case", ["L32_w_layers", "L16", "L24"])
def test_mixed_plan_host_buffers(case):
    # the host-buffer call: each span lists its separable subgrids first
    wl, p = _mixed(case)
    op = O.plan(wl)
    G = syn.random_grid(np.random.default_rng(41), p.n_w_layers, wl.grid_size)
    g = np.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=np.complex64)
    v = np.zeros(wl.vis.shape, dtype=np.complex64)
    idg.grid_degrid_host(p, wl.vis.astype(np.complex64), G.astype(np.complex64), wl.flags, wl.aterms.astype(np.complex64),
                         wl.taper.astype(np.float32), g, v)
    idg.device_errors()
    parity(g, O.grid(wl, op), f"mixed {case} host-buffer grid")
    parity(v, O.degrid(wl, op, G), f"mixed {case} host-buffer degrid")


def test_mixed_plans_in_a_batch():
    # mixed plans of three sizes and one fully separable plan in one batch: each L's
    # work list splits into a separable class (separable subgrids and pieces) and a
    # direct class (the subgrids left)
    import torch
    wls = [syn.make_small(**CASES[c]) for c in ("L32", "L24", "L16", "L32_w_layers")]
    wls.append(syn.make_small(seed=93, n_st=5, n_t=96, n_chan=8, L=24, N=256, max_t=96, n_slots=2, flag_p=0.1,
                              diameter_m=1500.0))
    plans = [idg.plan_from_workload(w) for w in wls]
    assert [int(0 < p.stats.n_sep_subgrids < p.n_subgrids) for p in plans] == [1, 1, 1, 1, 0]
    assert plans[4].stats.separable == 1
    classes = set()
    for p in plans:
        st = p.stats
        classes.add((st.subgrid_size, 1))
        if st.n_sep_subgrids + st.n_split_subgrids < p.n_subgrids:
            classes.add((st.subgrid_size, 0))
    assert (32, 0) in classes                   # the W-layer job keeps direct subgrids
    ops = [O.plan(w) for w in wls]
    rng = np.random.default_rng(43)
    jobs, models = [], []
    for w, p in zip(wls, plans):
        d = workload_to_device(w)
        models.append(syn.random_grid(rng, p.n_w_layers, w.grid_size))
        jobs.append(dict(vis=d["vis"], flags=d["flags"], aterms=d["aterms"], taper=d["taper"],
                         grid=torch.zeros((p.n_w_layers, w.grid_size, w.grid_size, 4), dtype=torch.complex64,
                                          device="cuda"),
                         vis_out=torch.zeros(w.vis.shape, dtype=torch.complex64, device="cuda")))
    b = idg.Batch(plans, jobs)
    assert b.info()["n_launches"] == len(classes)
    b.grid()
    idg.device_errors()
    for i, (w, op, j) in enumerate(zip(wls, ops, jobs)):
        parity(j["grid"].cpu().numpy(), O.grid(w, op), f"mixed batch grid job {i}")
    bd = idg.Batch(plans, [dict(j, grid=dev(m), vis=None) for j, m in zip(jobs, models)])
    bd.degrid()
    idg.device_errors()
    for i, (w, op, j, m) in enumerate(zip(wls, ops, jobs, models)):
        parity(j["vis_out"].cpu().numpy(), O.degrid(w, op, m), f"mixed batch degrid job {i}")
