"""Full-size parity on the LOFAR-like workload (48 stations, 1128 baselines,
4096 x 1 s, 16 channels: 73.9 M visibilities, 4096^2 x 4 grid, L = 32, A-terms
every 128 timesteps) in the launch configuration the benchmark times.

The oracle cannot redo the whole job in seconds, so it checks sampled subgrids
one by one (gridder stage; degridded visibilities, which belong to exactly one
subgrid each), and the full composite outputs are checked through properties
that hold at any size: the sum of the grid equals, per subgrid, the taper and
A-terms at the subgrid centre applied to the sum of its visibilities (the
centred DFT of a subgrid sums to its centre pixel, where every phasor is 1),
and adjointness of the two composite operations.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07226_gb300 import idg
from paper_1909_07226_gb300 import synthetic as syn
from tests.gpu_util import dev, parity, workload_to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lofar():
    from paper_1909_07226_gb300 import build
    import torch
    build.build()
    wl = syn.make_lofar(with_vis=True)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    d = workload_to_device(wl)
    rng = np.random.default_rng(2024)
    ranges = sorted({int(s) for s in rng.integers(0, p.n_subgrids - 8, size=16)})
    ids = np.concatenate([np.arange(s, s + 8) for s in ranges]).astype(np.int32)
    ids = np.unique(ids)
    G = syn.random_grid(np.random.default_rng(77), p.n_w_layers, wl.grid_size)
    g = torch.zeros(G.shape, dtype=torch.complex64, device="cuda")
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    v = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")
    idg.degrid(p, dev(G), d["flags"], d["aterms"], d["taper"], v)
    torch.cuda.synchronize()
    return dict(wl=wl, p=p, op=op, d=d, ids=ids, G=G, g=g, v=v)


def test_lofar_plan_shape(lofar):
    p, wl = lofar["p"], lofar["wl"]
    assert wl.n_vis == 1128 * 4096 * 16
    assert p.stats.n_vis_planned + p.stats.n_vis_dropped == wl.n_vis
    assert p.n_subgrids >= 36096


def test_lofar_gridder_sampled_subgrids(lofar):
    import torch
    p, wl, op, d, ids = lofar["p"], lofar["wl"], lofar["op"], lofar["d"], lofar["ids"]
    L = wl.subgrid_size
    got = []
    i = 0
    while i < len(ids):           # contiguous runs of plan indices
        j = i
        while j + 1 < len(ids) and ids[j + 1] == ids[j] + 1:
            j += 1
        cnt = j - i + 1
        sub = torch.zeros((cnt, L, L, 4), dtype=torch.complex64, device="cuda")
        idg.grid_subgrids(p, int(ids[i]), cnt, d["vis"], d["flags"], d["aterms"], d["taper"], sub)
        got.append(sub.cpu().numpy())
        i = j + 1
    parity(np.concatenate(got), O.subgrid_images(wl, op, ids), "lofar gridder (sampled subgrids)")


def test_lofar_grid_sum_identity(lofar):
    import torch
    wl, op, g = lofar["wl"], lofar["op"], lofar["g"]
    L = wl.subgrid_size
    c = L // 2
    got = g.to(torch.complex128).sum(dim=(0, 1, 2)).cpu().numpy()
    tw = float(wl.taper[c, c])
    ref = np.zeros(4, dtype=np.complex128)
    scale = 0.0
    for dsc in op.desc:
        b, a, t0, nt, c0, nc = (int(x) for x in dsc[:6])
        s = wl.vis[b, t0:t0 + nt, c0:c0 + nc].astype(np.complex128).sum(axis=(0, 1)).reshape(2, 2)
        pst, qst = wl.baselines[b]
        Ap = wl.aterms[a, pst, c, c].astype(np.complex128).reshape(2, 2)
        Aq = wl.aterms[a, qst, c, c].astype(np.complex128).reshape(2, 2)
        m = tw * (np.conj(Ap.T) @ s @ Aq)
        ref += m.reshape(4)
        scale += np.abs(m).sum()
    err = np.max(np.abs(got - ref)) / scale
    print(f"grid sum identity: err/sum|terms| = {err:.3e}")
    assert err < 1e-6


def test_lofar_degrid_sampled_subgrids(lofar):
    wl, op, ids, G, v = lofar["wl"], lofar["op"], lofar["ids"], lofar["G"], lofar["v"]
    ref = O.degrid(wl, op, G, ids=ids)
    got = v.cpu().numpy()
    mask = np.zeros(wl.vis.shape[:3], dtype=bool)
    for dsc in op.desc[ids]:
        mask[dsc[0], dsc[2]:dsc[2] + dsc[3], dsc[4]:dsc[4] + dsc[5]] = True
    parity(got[mask], ref[mask], "lofar degrid (sampled subgrids)")


def test_lofar_adjointness(lofar):
    import torch
    wl, G, g, v = lofar["wl"], lofar["G"], lofar["g"], lofar["v"]
    lhs = torch.vdot(v.reshape(-1).to(torch.complex128), dev(wl.vis).reshape(-1).to(torch.complex128)).item()
    rhs = torch.vdot(dev(G).reshape(-1).to(torch.complex128), g.reshape(-1).to(torch.complex128)).item()
    print(f"adjointness: |lhs-rhs|/|rhs| = {abs(lhs - rhs) / abs(rhs):.3e}")
    assert abs(lhs - rhs) / abs(rhs) < 1e-5


def _grid_sum_reference(wl, op):
    L = wl.subgrid_size
    c = L // 2
    tw = float(wl.taper[c, c])
    ref = np.zeros(4, dtype=np.complex128)
    scale = 0.0
    for dsc in op.desc:
        b, a, t0, nt, c0, nc = (int(x) for x in dsc[:6])
        s = wl.vis[b, t0:t0 + nt, c0:c0 + nc].astype(np.complex128).sum(axis=(0, 1)).reshape(2, 2)
        pst, qst = wl.baselines[b]
        Ap = wl.aterms[a, pst, c, c].astype(np.complex128).reshape(2, 2)
        Aq = wl.aterms[a, qst, c, c].astype(np.complex128).reshape(2, 2)
        m = tw * (np.conj(Ap.T) @ s @ Aq)
        ref += m.reshape(4)
        scale += np.abs(m).sum()
    return ref, scale


def test_lofar_recurrence_form_sampled(lofar):
    # the channel-recurrence precision form at full size: sampled subgrid images
    # and sampled degridded visibilities against the oracle, and the grid-sum
    # identity for its full grid
    import torch
    wl, op, ids, G, d = lofar["wl"], lofar["op"], lofar["ids"], lofar["G"], lofar["d"]
    L = wl.subgrid_size
    pr = idg.plan_from_workload(wl, precision_mode=idg.PHASOR_RECURRENCE)
    got = []
    i = 0
    while i < len(ids):
        j = i
        while j + 1 < len(ids) and ids[j + 1] == ids[j] + 1:
            j += 1
        cnt = j - i + 1
        sub = torch.zeros((cnt, L, L, 4), dtype=torch.complex64, device="cuda")
        idg.grid_subgrids(pr, int(ids[i]), cnt, d["vis"], d["flags"], d["aterms"], d["taper"], sub)
        got.append(sub.cpu().numpy())
        i = j + 1
    parity(np.concatenate(got), O.subgrid_images(wl, op, ids), "lofar recurrence gridder (sampled subgrids)")
    g = torch.zeros(G.shape, dtype=torch.complex64, device="cuda")
    idg.grid(pr, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    ref, scale = _grid_sum_reference(wl, op)
    err = np.max(np.abs(g.to(torch.complex128).sum(dim=(0, 1, 2)).cpu().numpy() - ref)) / scale
    print(f"recurrence grid sum identity: err/sum|terms| = {err:.3e}")
    assert err < 1e-6
    v = torch.zeros(wl.vis.shape, dtype=torch.complex64, device="cuda")
    idg.degrid(pr, dev(G), d["flags"], d["aterms"], d["taper"], v)
    ref = O.degrid(wl, op, G, ids=ids)
    mask = np.zeros(wl.vis.shape[:3], dtype=bool)
    for dsc in op.desc[ids]:
        mask[dsc[0], dsc[2]:dsc[2] + dsc[3], dsc[4]:dsc[4] + dsc[5]] = True
    parity(v.cpu().numpy()[mask], ref[mask], "lofar recurrence degrid (sampled subgrids)")


def test_lofar_fused_grid_on_sampled_ranges(lofar):
    # the fused separable gridder the benchmark times, on sampled plan-order
    # ranges of the full plan (idg_grid_range runs the same kernel), every pixel
    # of the resulting grid against the oracle's grid of the same subgrids
    import torch
    wl, p, op, d, ids = lofar["wl"], lofar["p"], lofar["op"], lofar["d"], lofar["ids"]
    assert p.stats.separable == 1
    g = torch.zeros((p.n_w_layers, wl.grid_size, wl.grid_size, 4), dtype=torch.complex64, device="cuda")
    i = 0
    while i < len(ids):
        j = i
        while j + 1 < len(ids) and ids[j + 1] == ids[j] + 1:
            j += 1
        idg.grid_range(p, int(ids[i]), j - i + 1, d["vis"], d["flags"], d["aterms"], d["taper"], g)
        i = j + 1
    idg.device_errors()
    parity(g.cpu().numpy(), O.grid(wl, op, ids=ids), "lofar fused grid (sampled ranges, every pixel)")
