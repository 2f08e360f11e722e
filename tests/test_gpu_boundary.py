"""GPU checks of the boundary: the default taper of a NULL taper argument, the
per-plan kernel choice, the plan-order range calls (the unit of a partition of
the subgrids), and the failure path of the bounded device waits.

Parity as everywhere: against the FP64 oracle on the same seeded inputs,
relative RMS <= 1e-5 (tests.gpu_util.parity)."""
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


def zeros(shape):
    import torch
    return torch.zeros(shape, dtype=torch.complex64, device="cuda")


def _pswf_taper(L, beta):
    # the window the library documents for a NULL taper, from its own window call
    a, _ = idg.taper_window(L, beta, idg.TAPER_PSWF)
    return np.outer(a, a).astype(np.float32)


CASES = {
    "L24_packed": dict(seed=71, n_st=5, n_t=48, n_chan=5, L=24, N=128, max_t=48, n_slots=2, flag_p=0.1),
    "L32_separable_fused": dict(seed=72, n_st=5, n_t=96, n_chan=8, L=32, N=128, max_t=96, n_slots=1, flag_p=0.1,
                                diameter_m=2500.0, df=0.25e6),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_null_taper_is_the_plans_pswf(case):
    import torch
    wl = syn.make_small(**CASES[case])
    p = idg.plan_from_workload(wl)
    if case.startswith("L32"):
        assert p.stats.separable == 1
    op = O.plan(wl)
    taper = _pswf_taper(wl.subgrid_size, float(wl.kernel_size))
    d = workload_to_device(wl)
    g = zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4))
    idg.grid(p, d["vis"], d["flags"], d["aterms"], None, g)
    parity(g.cpu().numpy(), O.grid(wl, op, taper=taper), f"{case} grid, NULL taper")
    G = syn.random_grid(np.random.default_rng(3), p.n_w_layers, wl.grid_size)
    v = zeros(wl.vis.shape)
    idg.degrid(p, dev(G), d["flags"], d["aterms"], None, v)
    parity(v.cpu().numpy(), O.degrid(wl, op, G, taper=taper), f"{case} degrid, NULL taper")
    # host-buffer calls take the same default
    gh = np.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=np.complex64)
    idg.grid_host(p, wl.vis, wl.flags, wl.aterms, None, gh)
    parity(gh, O.grid(wl, op, taper=taper), f"{case} grid_host, NULL taper")
    # and an explicit copy of the default gives the same result
    g2 = zeros(g.shape)
    idg.grid(p, d["vis"], d["flags"], d["aterms"], dev(taper), g2)
    torch.cuda.synchronize()
    parity(g2.cpu().numpy(), g.cpu().numpy(), f"{case} explicit vs NULL taper", tol=1e-6)


def test_autotune_writes_only_into_its_plan():
    import torch
    wl = syn.make_small(seed=73, n_st=5, n_t=100, n_chan=16, L=32, N=128, max_t=96, n_slots=1, flag_p=0.1)
    a, b = idg.plan_from_workload(wl), idg.plan_from_workload(wl)
    d = workload_to_device(wl)
    before = idg.get_kernel_variant("gridder", 32), idg.get_kernel_variant("degridder", 32)
    scratch = zeros(wl.vis.shape)
    res = idg.autotune(a, d["vis"], d["flags"], d["aterms"], d["taper"], scratch, max_subgrids=64)
    assert (idg.get_kernel_variant("gridder", 32), idg.get_kernel_variant("degridder", 32)) == before
    assert idg.plan_get_kernel_variant(b, "gridder") == before[0]
    assert idg.plan_get_kernel_variant(a, "gridder") == res["gridder"]["chosen"]
    # a plan forced to a non-default variant still gives the oracle's grid, and the
    # default plan next to it is unaffected
    op = O.plan(wl)
    ref = O.grid(wl, op)
    idg.plan_set_kernel_variant(a, "gridder", len(idg.kernel_variants("gridder", 32)) - 1)
    for plan, name in ((a, "plan a (last variant)"), (b, "plan b (process default)")):
        g = zeros((plan.n_w_layers, wl.grid_size, wl.grid_size, 4))
        idg.grid(plan, d["vis"], d["flags"], d["aterms"], d["taper"], g)
        torch.cuda.synchronize()
        parity(g.cpu().numpy(), ref, name)


@pytest.mark.parametrize("case", sorted(CASES))
def test_range_calls_partition_the_composite(case):
    import torch
    wl = syn.make_small(**dict(CASES[case], w_step=0.0))
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    n = p.n_subgrids
    cut = n // 3
    # two ranges summed = the whole plan; each range alone = the oracle's range
    g_all = zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4))
    for f, c in ((0, cut), (cut, n - cut)):
        g = zeros(g_all.shape)
        idg.grid_range(p, f, c, d["vis"], d["flags"], d["aterms"], d["taper"], g)
        parity(g.cpu().numpy(), O.grid(wl, op, ids=np.arange(f, f + c)), f"{case} grid range [{f}, {f + c})")
        g_all += g
    parity(g_all.cpu().numpy(), O.grid(wl, op), f"{case} grid ranges summed")
    # degrid of a range writes its visibilities and nothing else
    G = syn.random_grid(np.random.default_rng(9), p.n_w_layers, wl.grid_size)
    sentinel = complex(3.0, -7.0)
    v = torch.full(wl.vis.shape, sentinel, dtype=torch.complex64, device="cuda")
    idg.degrid_range(p, cut, n - cut, dev(G), d["flags"], d["aterms"], d["taper"], v)
    got = v.cpu().numpy()
    mask = np.zeros(wl.vis.shape[:3], dtype=bool)
    for dsc in op.desc[cut:]:
        mask[dsc[0], dsc[2]:dsc[2] + dsc[3], dsc[4]:dsc[4] + dsc[5]] = True
    ref = O.degrid(wl, op, G, ids=np.arange(cut, n))
    parity(got[mask], ref[mask], f"{case} degrid range")
    assert np.all(got[~mask] == np.complex64(sentinel))
    # an empty range does nothing; a range outside the plan is refused
    idg.grid_range(p, n, 0, d["vis"], d["flags"], d["aterms"], d["taper"], g_all)
    with pytest.raises(idg.IDGError) as ei:
        idg.grid_range(p, 1, n, d["vis"], d["flags"], d["aterms"], d["taper"], g_all)
    assert ei.value.status == 1


def test_bounded_wait_timeout_is_reported_and_the_device_recovers():
    import torch
    idg.device_errors()                                 # clear any earlier state
    idg.selftest_wait_timeout(4096)
    with pytest.raises(idg.IDGError) as ei:
        idg.device_errors()
    assert ei.value.status == 4
    idg.device_errors()                                 # the words were cleared
    # the tensor memory was released: the separable kernels (which take all 512
    # columns of an SM) run next and match the oracle
    wl = syn.make_small(**CASES["L32_separable_fused"])
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    g = zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4))
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    idg.device_errors()
    parity(g.cpu().numpy(), O.grid(wl, op), "separable grid after the self-test")
    with pytest.raises(idg.IDGError):
        idg.selftest_wait_timeout(0)
    torch.cuda.synchronize()


@pytest.mark.parametrize("case", sorted(CASES))
def test_grid_degrid_host_in_one_call(case):
    # both directions on host buffers in one pipelined call, against the oracle
    wl = syn.make_small(**CASES[case])
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    G = syn.random_grid(np.random.default_rng(21), p.n_w_layers, wl.grid_size).astype(np.complex64)
    gout = np.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=np.complex64)
    vout = np.full(wl.vis.shape, 7.0 + 7.0j, dtype=np.complex64)
    idg.grid_degrid_host(p, wl.vis, G, wl.flags, wl.aterms, wl.taper.astype(np.float32), gout, vout)
    parity(gout, O.grid(wl, op), f"{case} grid_degrid_host: grid")
    parity(vout, O.degrid(wl, op, G), f"{case} grid_degrid_host: visibilities")
