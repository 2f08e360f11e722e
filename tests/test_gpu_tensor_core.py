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

TC_VARIANTS = ["tcgen05_separable", "tcgen05_tmemA_ws_nt288"]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_07226_gb300 import build
    build.build()
    idg.load()


@pytest.fixture(params=TC_VARIANTS)
def tc_selected(request):
    names = idg.kernel_variants("gridder", 32)
    assert request.param in names
    idg.set_kernel_variant("gridder", 32, names.index(request.param))
    yield request.param
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
    # wide field with the separable remainder phase just under its bound (1.34e-3 rad)
    "wide_field_near_bound": lambda: small32(N=256, cell=1.2e-3, diameter_m=500.0),
    # wide field far over the bound (1.4e-2 rad): the separable choice falls back to the direct kernel
    "wide_field_direct": lambda: small32(N=512, cell=1e-3, diameter_m=800.0),
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
    parity(sub.cpu().numpy(), O.subgrid_images(wl, op), f"{tc_selected} {case}")


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
    parity(g.cpu().numpy(), O.grid(wl, op), f"{tc_selected} grid")


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
           f"{tc_selected} LOFAR slice, sampled")


# ---------------------------------------------------------------------------
# subgrid transform on the tensor cores (fft_mode = FFT_TC_SPLIT)

def _tc_plan(wl):
    return idg.plan_from_workload(wl, fft_mode=idg.FFT_TC_SPLIT)


@pytest.mark.parametrize("direction", [-1, 1])
@pytest.mark.parametrize("case", ["gaussian", "huge", "tiny", "mixed_rows", "zero_and_delta"])
def test_tc_transform_stage(direction, case):
    wl = small32(n_t=8, max_t=8)
    p = _tc_plan(wl)
    rng = np.random.default_rng(500 + direction)
    n = 41
    x = (rng.normal(size=(n, 32, 32, 4)) + 1j * rng.normal(size=(n, 32, 32, 4)))
    if case == "huge":
        x *= 1e12
    elif case == "tiny":
        x *= 1e-12
    elif case == "mixed_rows":
        x *= 10.0 ** rng.uniform(-6, 6, size=(n, 32, 1, 1))     # dynamic range inside a subgrid
    elif case == "zero_and_delta":
        x[0] = 0.0
        x[1] = 0.0
        x[1, 3, 29, 2] = 5.0 - 2.0j
    x = x.astype(np.complex64)
    t = dev(x)
    idg.fft_subgrids(p, n, direction, t)
    idg.device_errors()
    out = t.cpu().numpy()
    ref = O.dft2(x, direction)
    if case == "zero_and_delta":
        assert not np.any(out[0])
    parity(out, ref, f"tc transform {case} dir={direction}")


def test_tc_transform_inverse_pair():
    # forward then backward returns the input scaled by L^-2 (both carry 1/L^2)
    wl = small32(n_t=8, max_t=8)
    p = _tc_plan(wl)
    rng = np.random.default_rng(9)
    x = (rng.normal(size=(16, 32, 32, 4)) + 1j * rng.normal(size=(16, 32, 32, 4))).astype(np.complex64)
    t = dev(x)
    idg.fft_subgrids(p, 16, -1, t)
    idg.fft_subgrids(p, 16, 1, t)
    idg.device_errors()
    parity(t.cpu().numpy() * 1024.0, x, "tc transform round trip")


@pytest.mark.parametrize("case", ["points_flags_aterms", "w_layers", "long_kp"])
def test_tc_transform_in_grid_and_degrid(case):
    import torch
    wl = CASES[case]()
    p = _tc_plan(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    idg.device_errors()
    parity(g.cpu().numpy(), O.grid(wl, op), f"grid with tc transform, {case}")
    rng = np.random.default_rng(3)
    g_in = syn.random_grid(rng, p.n_w_layers, wl.grid_size)
    v = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")
    idg.degrid(p, dev(g_in), d["flags"], d["aterms"], d["taper"], v)
    idg.device_errors()
    parity(v.cpu().numpy(), O.degrid(wl, op, g_in), f"degrid with tc transform, {case}")


def test_tc_transform_rejected_by_batches():
    wl = small32(n_t=8, max_t=8)
    p = _tc_plan(wl)
    d = workload_to_device(wl)
    import torch
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(idg.IDGError):
        idg.Batch([p], [dict(vis=d["vis"], vis_out=None, flags=d["flags"], aterms=d["aterms"], taper=d["taper"],
                             grid=g)])


# ---------------------------------------------------------------------------
# tensor-core degridder

TCD_VARIANTS = ["tcgen05_separable", "tcgen05_tmemA_ws_nt288"]


@pytest.fixture(params=TCD_VARIANTS)
def tcd_selected(request):
    names = idg.kernel_variants("degridder", 32)
    assert request.param in names
    prev = idg.get_kernel_variant("degridder", 32)
    idg.set_kernel_variant("degridder", 32, names.index(request.param))
    yield request.param
    idg.set_kernel_variant("degridder", 32, prev)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("image", ["gaussian", "huge", "tiny"])
def test_tc_degridder_stage(case, image, tcd_selected):
    import torch
    wl = CASES[case]()
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    n = p.n_subgrids
    rng = np.random.default_rng(31)
    img = rng.normal(size=(n, 32, 32, 4)) + 1j * rng.normal(size=(n, 32, 32, 4))
    img *= {"gaussian": 1.0, "huge": 1e12, "tiny": 1e-12}[image]
    img = img.astype(np.complex64)
    out = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")   # dropped samples stay 0
    idg.degrid_subgrids(p, 0, n, dev(img), d["flags"], d["aterms"], d["taper"], out)
    idg.device_errors()
    parity(out.cpu().numpy(), O.degrid_images(wl, op, img.astype(np.complex128)), f"tc degridder {case} {image}")


def test_tc_degrid_full(tcd_selected):
    import torch
    wl = small32(w_step=20.0, diameter_m=20000.0, n_t=24, max_t=12)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    rng = np.random.default_rng(3)
    g_in = syn.random_grid(rng, p.n_w_layers, wl.grid_size)
    v = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")
    idg.degrid(p, dev(g_in), d["flags"], d["aterms"], d["taper"], v)
    idg.device_errors()
    parity(v.cpu().numpy(), O.degrid(wl, op, g_in), "tc degrid")


def test_tc_degridder_lofar_slice_sampled(tcd_selected):
    import torch
    wl = syn.make_lofar(n_t=64, slot_len=64, name="lofar-tc")
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    n = p.n_subgrids
    rng = np.random.default_rng(41)
    ids = np.linspace(0, n - 1, 64).round().astype(np.int32)
    img = (rng.normal(size=(n, 32, 32, 4)) + 1j * rng.normal(size=(n, 32, 32, 4))).astype(np.complex64)
    out = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")
    idg.degrid_subgrids(p, 0, n, dev(img), d["flags"], d["aterms"], d["taper"], out)
    idg.device_errors()
    # the visibilities of the sampled subgrids, against the oracle on those subgrids alone
    ref = O.degrid_images(wl, op, img[ids].astype(np.complex128), ids=ids)
    desc = op.desc[ids]
    sel = np.zeros(wl.vis.shape[:3], dtype=bool)
    for row in desc:
        bl, t0, nt, c0, nc = row[O.D_BL], row[O.D_T0], row[O.D_NT], row[O.D_C0], row[O.D_NC]
        sel[bl, t0:t0 + nt, c0:c0 + nc] = True
    parity(out.cpu().numpy()[sel], ref[sel], "tc degridder LOFAR slice, sampled")


# ---------------------------------------------------------------------------
# fused tensor-core kernels: with the default choices at L = 32 (FP32
# transform, direct phasors, plain adder) a composite call grids each subgrid
# in one CTA (gridder, transform and adder) and degrids it in one CTA
# (splitter, transform and degridder) when most of its visibilities lie in
# subgrids of K_p >= 64 (separable plans; 512 for the direct kernels).  The
# launch counters show which path ran.

def _no_aterms(wl):
    wl.aterms = None
    return wl


FUSED_CASES = {
    "long_kp": CASES["long_kp"],
    # no A-terms: the separable degridder fetches none and waits for none
    "long_kp_no_aterms": lambda: _no_aterms(CASES["long_kp"]()),
    # four w layers, K_p 96 .. 2048: fused degridder
    "long_kp_w_layers": lambda: small32(n_t=128, n_chan=16, max_t=128, n_st=4, df=0.25e6, w_step=50.0),
    # two A-term slots and two w layers, K_p 8 .. 768: fused degridder, ragged groups
    "long_kp_slots_layers": lambda: small32(n_t=192, n_chan=8, max_t=96, n_st=4, df=0.25e6, n_slots=2,
                                            w_step=100.0, diameter_m=2000.0),
    # many small subgrids (K_p <= 160, half of the visibilities in subgrids of 64 or more)
    "short_kp_w_layers": lambda: small32(n_t=128, n_chan=16, max_t=128, n_st=4, df=0.25e6, w_step=20.0,
                                         diameter_m=20000.0),
    # subgrids of at most 32 visibilities: fused gridder, separate degridding stages
    "tiny_kp": lambda: small32(n_t=64, n_chan=8, max_t=4, n_st=4),
    "points_flags_aterms": CASES["points_flags_aterms"],
    "huge_magnitudes": CASES["huge_magnitudes"],
}


def _launches(prof):
    return {k: v["launches"] for k, v in prof.items() if v["launches"]}


def _kp_mostly_long(p):
    kp = p.export()[:, O.D_KP]
    kmin = 64 if p.stats.separable else 512
    return 2 * kp[kp < kmin].sum() <= kp.sum()


@pytest.mark.parametrize("case", sorted(FUSED_CASES))
def test_fused_grid_and_degrid(case):
    import torch
    wl = FUSED_CASES[case]()
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    idg.profile_enable(True)
    try:
        idg.profile_read(reset=True)
        idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
        grid_launches = _launches(idg.profile_read(reset=True))
        rng = np.random.default_rng(5)
        g_in = syn.random_grid(rng, p.n_w_layers, wl.grid_size)
        v = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")
        idg.degrid(p, dev(g_in), d["flags"], d["aterms"], d["taper"], v)
        degrid_launches = _launches(idg.profile_read(reset=True))
    finally:
        idg.profile_enable(False)
    idg.device_errors()
    assert grid_launches == {"gridder": 1}
    if _kp_mostly_long(p):
        assert degrid_launches == {"degridder": 1}
    else:
        assert "splitter" in degrid_launches and "fft" in degrid_launches
    parity(g.cpu().numpy(), O.grid(wl, op), f"fused grid {case}")
    parity(v.cpu().numpy(), O.degrid(wl, op, g_in), f"fused degrid {case}")


def test_fused_grid_accumulates_into_the_grid():
    # the fused adder adds into what the grid holds, as the separate adder does
    import torch
    wl = CASES["long_kp"]()
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    rng = np.random.default_rng(9)
    g0 = syn.random_grid(rng, p.n_w_layers, wl.grid_size)
    g = dev(g0)
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    idg.device_errors()
    parity(g.cpu().numpy(), O.grid(wl, op) + g0, "fused grid accumulated")


def test_stage_calls_stay_unfused():
    # grid_subgrids writes subgrid images: the fused kernels never serve it
    import torch
    wl = CASES["long_kp"]()
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    n = p.n_subgrids
    sub = torch.zeros((n, 32, 32, 4), dtype=torch.complex64, device="cuda")
    idg.grid_subgrids(p, 0, n, d["vis"], d["flags"], d["aterms"], d["taper"], sub)
    idg.device_errors()
    parity(sub.cpu().numpy(), O.subgrid_images(wl, op), "stage gridder, long K_p")


def test_separable_flag_follows_the_bound():
    near = idg.plan_from_workload(CASES["wide_field_near_bound"]())
    far = idg.plan_from_workload(CASES["wide_field_direct"]())
    assert near.stats.separable == 1 and 1.2e-3 < near.stats.sep_phase <= 1.38e-3
    assert far.stats.separable == 0 and far.stats.sep_phase > 1e-2
