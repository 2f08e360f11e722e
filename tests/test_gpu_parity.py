"""GPU parity: every stage and both composite operations of the CUDA path,
called through the C ABI, against the FP64 oracle on the same seeded inputs.

Tolerance: relative RMS <= 1e-5 for grids, subgrids and visibilities (FP32
arithmetic with FP64 coordinate offsets); the max error relative to the
largest reference value is reported and bounded by 1e-3.  Sizes span several
visibility batches per subgrid with a ragged tail, every compiled L, flags,
random A-terms and W-layers.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07226_gb300 import idg
from paper_1909_07226_gb300 import synthetic as syn
from tests.gpu_util import dev, parity, workload_to_device

pytestmark = pytest.mark.gpu

SIZES = [8, 16, 24, 32, 48, 64]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_07226_gb300 import build
    build.build()
    idg.load()


def small(L, **kw):
    args = dict(seed=100 + L, n_st=5, n_t=48, n_chan=5, L=L, N=max(4 * L, 64), max_t=48, n_slots=2, flag_p=0.1,
                diameter_m=3000.0)
    args.update(kw)
    return syn.make_small(**args)


def torch_zeros(shape, dtype=None):
    import torch
    return torch.zeros(shape, dtype=dtype or torch.complex64, device="cuda")


@pytest.mark.parametrize("L", SIZES)
def test_gridder_stage(L):
    wl = small(L, n_slots=1)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    n = p.n_subgrids
    assert int(op.desc[:, O.D_KP].max()) > 128          # several shared-memory batches
    ref = O.subgrid_images(wl, op)
    for v, name in enumerate(idg.kernel_variants("gridder", L)):      # every compiled tile shape
        idg.set_kernel_variant("gridder", L, v)
        sub = torch_zeros((n, L, L, 4))
        idg.grid_subgrids(p, 0, n, d["vis"], d["flags"], d["aterms"], d["taper"], sub)
        idg.device_errors()
        parity(sub.cpu().numpy(), ref, f"gridder L={L} {name}")
    idg.set_kernel_variant("gridder", L, 0)


@pytest.mark.parametrize("L", SIZES)
@pytest.mark.parametrize("direction", [-1, 1])
def test_fft_stage(L, direction):
    wl = small(L, n_t=8, max_t=8)
    p = idg.plan_from_workload(wl)
    rng = np.random.default_rng(L)
    x = (rng.normal(size=(37, L, L, 4)) + 1j * rng.normal(size=(37, L, L, 4))).astype(np.complex64)
    t = dev(x)
    idg.fft_subgrids(p, 37, direction, t)
    parity(t.cpu().numpy(), O.dft2(x, direction), f"fft L={L} dir={direction}")


@pytest.mark.parametrize("L", [16, 32])
def test_adder_and_splitter_stages(L):
    wl = small(L, diameter_m=1000.0)       # short baselines: many overlapping subgrids
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    n = p.n_subgrids
    rng = np.random.default_rng(7)
    x = (rng.normal(size=(n, L, L, 4)) + 1j * rng.normal(size=(n, L, L, 4))).astype(np.complex64)
    g0 = syn.random_grid(rng, p.n_w_layers, wl.grid_size)
    g = dev(g0)
    idg.add_subgrids(p, 0, n, dev(x), g)
    ref = O.add(wl, op, x.astype(np.complex128), grid=g0.astype(np.complex128))
    parity(g.cpu().numpy(), ref, f"adder L={L}")
    sub = torch_zeros((n, L, L, 4))
    idg.split_subgrids(p, 0, n, dev(g0), sub)
    assert np.array_equal(sub.cpu().numpy(), O.split(wl, op, g0).astype(np.complex64))   # a copy: exact


@pytest.mark.parametrize("L", SIZES)
def test_degridder_stage(L):
    wl = small(L, n_chan=16, n_t=100, max_t=96, n_slots=1)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    assert int(op.desc[:, O.D_KP].max()) > 1024         # several passes of the visibility lanes
    assert int(op.desc[:, O.D_KP].min()) < 128          # and subgrids split into pixel groups
    d = workload_to_device(wl)
    n = p.n_subgrids
    rng = np.random.default_rng(11)
    img = (rng.normal(size=(n, L, L, 4)) + 1j * rng.normal(size=(n, L, L, 4))).astype(np.complex64)
    ref = O.degrid_images(wl, op, img.astype(np.complex128))
    for v, name in enumerate(idg.kernel_variants("degridder", L)):    # every compiled tile shape
        idg.set_kernel_variant("degridder", L, v)
        out = torch_zeros(wl.vis.shape)
        idg.degrid_subgrids(p, 0, n, dev(img), d["flags"], d["aterms"], d["taper"], out)
        parity(out.cpu().numpy(), ref, f"degridder L={L} {name}")
    idg.set_kernel_variant("degridder", L, 0)


CASES = {
    "tiny": lambda: syn.make_tiny(),
    "L16_flags_aterms": lambda: small(16),
    "L24_wlayers": lambda: small(24, w_step=20.0, diameter_m=20000.0, n_t=24, max_t=12),
    "L32_identity_wide": lambda: small(32, aterms="identity", n_chan=16, diameter_m=30000.0, df=4e6),
    "L48_noflags": lambda: small(48, flag_p=0.0, n_t=24),
    "L64_dropped": lambda: small(64, cell=1.2e-3, diameter_m=6000.0, n_t=24),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_grid_and_degrid(case):
    import torch
    wl = CASES[case]()
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    g = torch_zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4))
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    parity(g.cpu().numpy(), O.grid(wl, op), f"grid {case}")
    rng = np.random.default_rng(3)
    g_in = syn.random_grid(rng, p.n_w_layers, wl.grid_size)
    v = torch.full(wl.vis.shape, 7.0 + 7.0j, dtype=torch.complex64, device="cuda")   # must be overwritten
    idg.degrid(p, dev(g_in), d["flags"], d["aterms"], d["taper"], v)
    parity(v.cpu().numpy(), O.degrid(wl, op, g_in), f"degrid {case}")


def test_adjointness_on_gpu():
    # <degrid(G), V> = <G, grid(V)> holds for the FP32 path to FP32 rounding
    import torch
    wl = small(24, w_step=15.0, diameter_m=20000.0, n_t=24, max_t=12)
    p = idg.plan_from_workload(wl)
    d = workload_to_device(wl)
    rng = np.random.default_rng(5)
    G = syn.random_grid(rng, p.n_w_layers, wl.grid_size)
    g = torch_zeros(G.shape)
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    v = torch_zeros(wl.vis.shape)
    idg.degrid(p, dev(G), d["flags"], d["aterms"], d["taper"], v)
    lhs = np.vdot(v.cpu().numpy().astype(np.complex128), wl.vis.astype(np.complex128))
    rhs = np.vdot(G.astype(np.complex128), g.cpu().numpy().astype(np.complex128))
    assert abs(lhs - rhs) / abs(rhs) < 1e-5


def test_flat_grid_identity_on_gpu():
    import torch
    wl = small(32, aterms="identity", flag_p=0.0)
    wl.aterms = None
    p = idg.plan_from_workload(wl)
    g = np.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=np.complex64)
    g[..., 0] = 1.0
    g[..., 3] = 1.0
    v = torch_zeros(wl.vis.shape)
    idg.degrid(p, dev(g), None, None, dev(wl.taper), v)
    y = v.cpu().numpy()
    mask = np.zeros(y.shape[:3], dtype=bool)
    for d in p.export():
        mask[d[0], d[2]:d[2] + d[3], d[4]:d[4] + d[5]] = True
    assert mask.sum() > 0 and p.stats.n_vis_dropped == int((~mask).sum())
    ym = y[mask]
    assert np.max(np.abs(ym[:, 0] - 1)) < 2e-6 and np.max(np.abs(ym[:, 3] - 1)) < 2e-6
    assert np.max(np.abs(ym[:, 1:3])) < 2e-6
    assert np.all(y[~mask] == 0)            # dropped visibilities are set to 0


def test_empty_plan_and_all_flagged():
    import torch
    # every visibility off the grid: an empty plan grids nothing and degrids zeros
    wl = small(16, cell=5e-3, diameter_m=50000.0, n_t=6)
    p = idg.plan_from_workload(wl)
    assert p.n_subgrids == 0 and p.stats.n_vis_dropped == wl.n_vis
    d = workload_to_device(wl)
    g = torch_zeros((1, wl.grid_size, wl.grid_size, 4))
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    assert int(torch.count_nonzero(g)) == 0
    v = torch.ones(wl.vis.shape, dtype=torch.complex64, device="cuda")
    idg.degrid(p, g, d["flags"], d["aterms"], d["taper"], v)
    assert int(torch.count_nonzero(v)) == 0
    # all flagged: zero grid, zero visibilities
    wl = small(16, n_t=8)
    wl.flags = np.ones_like(wl.flags)
    p = idg.plan_from_workload(wl)
    d = workload_to_device(wl)
    g = torch_zeros((1, wl.grid_size, wl.grid_size, 4))
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    assert int(torch.count_nonzero(g)) == 0
    v = torch.ones(wl.vis.shape, dtype=torch.complex64, device="cuda")
    idg.degrid(p, dev(syn.random_grid(np.random.default_rng(1), 1, wl.grid_size)), d["flags"], d["aterms"],
               d["taper"], v)
    assert int(torch.count_nonzero(v)) == 0


def test_single_visibility_subgrids():
    # T_max = 1 and one channel: every subgrid holds exactly one visibility
    wl = small(16, n_chan=1, max_t=1, n_t=12)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    assert np.all(op.desc[:, O.D_KP] == 1)
    d = workload_to_device(wl)
    g = torch_zeros((1, wl.grid_size, wl.grid_size, 4))
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    parity(g.cpu().numpy(), O.grid(wl, op), "grid K_p=1")


def test_device_call_errors():
    import torch
    wl = small(16, n_t=8)
    p = idg.plan_from_workload(wl)
    lib = idg.load()
    st = lib.idg_grid(p.handle, None, None, None, None, None, None)
    assert st == 1 and b"NULL" in lib.idg_last_error()
    with pytest.raises(ValueError):
        idg.grid(p, torch_zeros((1, 2, 3, 4)), None, None, dev(wl.taper), torch_zeros((1, 4, 4, 4)))
    with pytest.raises(idg.IDGError):
        idg.fft_subgrids(p, 4, 0, torch_zeros((4, 16, 16, 4)))


def test_autotune_selects_a_variant_and_results_hold():
    import torch
    wl = small(32, n_chan=16, n_t=100, max_t=96, n_slots=1)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    scratch = torch_zeros(wl.vis.shape)
    res = idg.autotune(p, d["vis"], d["flags"], d["aterms"], d["taper"], scratch, max_subgrids=64)
    assert all(ms > 0 for ms in res["gridder"]["ms"].values())
    assert len(res["degridder"]["ms"]) == len(idg.kernel_variants("degridder", 32))
    g = torch_zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4))
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    parity(g.cpu().numpy(), O.grid(wl, op), "grid after autotune")
    for k in ("gridder", "degridder"):
        idg.set_kernel_variant(k, 32, 0)


REC_CASES = {
    "tiny": lambda: syn.make_tiny(),
    "L8": lambda: small(8, n_chan=9, n_t=24, dt=5.0),
    "L16_flags_aterms_13ch": lambda: small(16, n_chan=13, n_t=24, max_t=24, n_slots=1),
    "L24_wlayers": lambda: small(24, w_step=20.0, diameter_m=20000.0, n_t=24, max_t=12, n_chan=11),
    "L32_wide": lambda: small(32, n_chan=16, diameter_m=30000.0, df=2e6, n_t=40),
    "L48_1ch": lambda: small(48, n_chan=1, n_t=30),
    "L64": lambda: small(64, n_chan=6, n_t=16),
}


@pytest.mark.parametrize("case", sorted(REC_CASES))
def test_recurrence_form_grid_and_degrid(case):
    # precision form: phasors advanced along channels, re-anchored every 8
    # channels; compared with the same FP64 oracle at the same tolerance
    import torch
    wl = REC_CASES[case]()
    p = idg.plan_from_workload(wl, precision_mode=idg.PHASOR_RECURRENCE)
    op = O.plan(wl)
    assert np.array_equal(p.export(), op.desc)
    d = workload_to_device(wl)
    g = torch_zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4))
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    parity(g.cpu().numpy(), O.grid(wl, op), f"recurrence grid {case}")
    g_in = syn.random_grid(np.random.default_rng(8), p.n_w_layers, wl.grid_size)
    v = torch.full(wl.vis.shape, 3.0 + 3.0j, dtype=torch.complex64, device="cuda")
    idg.degrid(p, dev(g_in), d["flags"], d["aterms"], d["taper"], v)
    parity(v.cpu().numpy(), O.degrid(wl, op, g_in), f"recurrence degrid {case}")


def test_compensated_adder_reduces_summation_error():
    # thousands of short-baseline subgrids pile up on the uv centre, where the
    # FP32 summation error of plain atomics dominates; the compensated adder
    # (exact TwoSum errors folded back) must be closer to the FP64 oracle there
    import torch
    wl = small(16, n_st=10, n_t=600, max_t=2, n_chan=2, N=64, diameter_m=300.0, flag_p=0.0, aterms="identity",
               n_slots=1)
    op = O.plan(wl)
    assert op.n_sub > 2000
    ref = O.grid(wl, op)
    d = workload_to_device(wl)
    errs = {}
    for mode in (idg.ADDER_ATOMIC, idg.ADDER_COMPENSATED):
        p = idg.plan_from_workload(wl, adder_mode=mode)
        g = torch_zeros((1, wl.grid_size, wl.grid_size, 4))
        idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
        got = g.cpu().numpy().astype(np.complex128)
        c = wl.grid_size // 2
        win = (slice(None), slice(c - 8, c + 8), slice(c - 8, c + 8))
        errs[mode] = np.linalg.norm((got - ref)[win]) / np.linalg.norm(ref[win])
        parity(got, ref, f"grid adder_mode={mode}")
    print(f"centre error: atomic {errs[0]:.3e} compensated {errs[1]:.3e}")
    assert errs[1] < errs[0]


# ---------------------------------------------------------------------------
# host-buffer calls: copies pipelined over spans of whole baselines

HOST_CASES = {
    "tiny": lambda: syn.make_tiny(),
    "L16_flags_aterms": lambda: small(16),
    "L24_wlayers": lambda: small(24, w_step=20.0, diameter_m=20000.0, n_t=24, max_t=12),
    "L32_identity_wide": lambda: small(32, aterms="identity", n_chan=16, diameter_m=30000.0, df=4e6),
    "L64_dropped": lambda: small(64, cell=1.2e-3, diameter_m=6000.0, n_t=24),
    "L32_many_baselines": lambda: small(32, n_st=12, n_t=16, max_t=16),
    # K_p = 2048: the spans take the fused tensor-core degridder as well
    "L32_long_kp": lambda: small(32, n_t=128, n_chan=16, max_t=128, n_st=4, df=0.25e6),
}


@pytest.mark.parametrize("case", sorted(HOST_CASES))
def test_grid_and_degrid_host_buffers(case):
    import torch
    wl = HOST_CASES[case]()
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    taper = wl.taper.astype(np.float32)
    # pinned host buffers, as a streaming caller would hold them
    vis = torch.from_numpy(wl.vis).pin_memory()
    flags = None if wl.flags is None else torch.from_numpy(wl.flags).pin_memory()
    aterms = None if wl.aterms is None else torch.from_numpy(wl.aterms).pin_memory()
    g = torch.full((p.n_w_layers, wl.grid_size, wl.grid_size, 4), 9.0 + 9.0j, dtype=torch.complex64).pin_memory()
    idg.grid_host(p, vis.numpy(), None if flags is None else flags.numpy(), None if aterms is None else aterms.numpy(),
                  taper, g.numpy())
    idg.device_errors()
    parity(g.numpy(), O.grid(wl, op), f"grid_host {case}")          # overwritten, not accumulated
    rng = np.random.default_rng(3)
    g_in = syn.random_grid(rng, p.n_w_layers, wl.grid_size)
    v = np.full(wl.vis.shape, 7.0 + 7.0j, dtype=np.complex64)         # pageable memory works too
    idg.degrid_host(p, g_in, wl.flags, wl.aterms, taper, v)
    idg.device_errors()
    parity(v, O.degrid(wl, op, g_in), f"degrid_host {case}")


def test_host_buffers_compensated_adder():
    wl = small(32, w_step=20.0, diameter_m=20000.0, n_t=24, max_t=12)
    p = idg.plan_from_workload(wl, adder_mode=idg.ADDER_COMPENSATED)
    op = O.plan(wl)
    g = np.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=np.complex64)
    idg.grid_host(p, wl.vis, wl.flags, wl.aterms, wl.taper.astype(np.float32), g)
    parity(g, O.grid(wl, op), "grid_host compensated")
