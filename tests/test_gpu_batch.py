"""Batched form: several jobs with different subgrid and grid sizes gridded and
degridded together (per subgrid size one work class, or two when some subgrids
take the separable kernels and others the direct ones: one persistent launch,
or tensor-core launches per job; subgrids kept in shared memory), each job
checked against the FP64 oracle; the same with the launch sequence captured in
a CUDA graph and replayed."""
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


def jobs_mix():
    return [
        syn.make_small(seed=301, n_st=5, n_t=40, n_chan=6, L=16, N=64, max_t=20, flag_p=0.1),
        syn.make_small(seed=302, n_st=6, n_t=30, n_chan=4, L=24, N=192, max_t=30, n_slots=3),
        syn.make_small(seed=303, n_st=6, n_t=48, n_chan=16, L=32, N=256, max_t=48, diameter_m=4000.0),
        syn.make_small(seed=304, n_st=4, n_t=24, n_chan=5, L=24, N=128, w_step=15.0, diameter_m=15000.0),
        syn.make_small(seed=305, n_st=5, n_t=20, n_chan=3, L=8, N=64, dt=5.0),
        syn.make_small(seed=306, n_st=6, n_t=20, n_chan=4, L=16, N=64, cell=6e-4, diameter_m=8000.0),  # drops
    ]


@pytest.mark.parametrize("graph", [False, True])
def test_batch_grid_and_degrid_match_the_oracle(graph):
    import torch
    wls = jobs_mix()
    plans = [idg.plan_from_workload(w) for w in wls]
    ops = [O.plan(w) for w in wls]
    assert any(p.stats.n_vis_dropped > 0 for p in plans)
    rng = np.random.default_rng(12)
    jobs, models = [], []
    for w, p in zip(wls, plans):
        d = workload_to_device(w)
        grid = torch.zeros((p.n_w_layers, w.grid_size, w.grid_size, 4), dtype=torch.complex64, device="cuda")
        models.append(syn.random_grid(rng, p.n_w_layers, w.grid_size))
        jobs.append(dict(vis=d["vis"], flags=d["flags"], aterms=d["aterms"], taper=d["taper"], grid=grid,
                         vis_out=torch.full(w.vis.shape, 5.0 + 5.0j, dtype=torch.complex64, device="cuda")))
    b = idg.Batch(plans, jobs, graph=graph)
    info = b.info()
    # one work class per subgrid size
    assert info["n_launches"] == 4 and info["n_items"] == sum(p.n_subgrids for p in plans)
    for rep in range(2):                 # second pass replays the captured graph
        for j in jobs:
            j["grid"].zero_()
        b.grid()
        torch.cuda.synchronize()
        for i, (w, op, j) in enumerate(zip(wls, ops, jobs)):
            parity(j["grid"].cpu().numpy(), O.grid(w, op), f"batch grid job {i} pass {rep}")
    # degrid from model grids: a degrid-only batch bound to the model grids
    djobs = [dict(j, grid=dev(m), vis=None) for j, m in zip(jobs, models)]
    bd = idg.Batch(plans, djobs, graph=graph)
    for rep in range(2):
        bd.degrid()
        torch.cuda.synchronize()
        for i, (w, op, j, m) in enumerate(zip(wls, ops, djobs, models)):
            parity(j["vis_out"].cpu().numpy(), O.degrid(w, op, m), f"batch degrid job {i} pass {rep}")


def test_batch_rejects_unsupported_jobs():
    wl = syn.make_small(seed=311, n_st=4, n_t=8, n_chan=2, L=64, N=256)
    p = idg.plan_from_workload(wl)
    d = workload_to_device(wl)
    with pytest.raises(idg.IDGError) as ei:
        idg.Batch([p], [dict(vis=d["vis"], taper=d["taper"])])
    assert ei.value.status == 6
    wl = syn.make_small(seed=312, n_st=4, n_t=8, n_chan=2, L=16, N=64)
    p = idg.plan_from_workload(wl, precision_mode=idg.PHASOR_RECURRENCE)
    d = workload_to_device(wl)
    with pytest.raises(idg.IDGError):
        idg.Batch([p], [dict(vis=d["vis"], taper=d["taper"])])


def _big_l32_jobs():
    # L = 32 jobs with K_p up to 1024, so the class runs on the tensor-core path
    # (the W-layered job adds partial tiles: 28 % of the class's visibilities lie in subgrids below 512)
    return [syn.make_small(seed=320 + i, n_st=5 + i, n_t=64, n_chan=16, L=32, N=256, max_t=64, flag_p=0.05 * i,
                           diameter_m=3000.0 + 1000.0 * i, w_step=20.0 * (i == 2), n_slots=2) for i in range(3)]


@pytest.mark.parametrize("graph", [False, True])
def test_batch_tensor_core_class_matches_the_oracle(graph):
    import torch
    wls = _big_l32_jobs()
    plans = [idg.plan_from_workload(w) for w in wls]
    ops = [O.plan(w) for w in wls]
    rng = np.random.default_rng(21)
    jobs, models = [], []
    for w, p in zip(wls, plans):
        d = workload_to_device(w)
        models.append(syn.random_grid(rng, p.n_w_layers, w.grid_size))
        jobs.append(dict(vis=d["vis"], flags=d["flags"], aterms=d["aterms"], taper=d["taper"],
                         grid=torch.zeros((p.n_w_layers, w.grid_size, w.grid_size, 4), dtype=torch.complex64,
                                          device="cuda"),
                         vis_out=torch.full(w.vis.shape, 5.0 + 5.0j, dtype=torch.complex64, device="cuda")))
    b = idg.Batch(plans, jobs, graph=graph)
    assert b.info()["n_launches"] == 1       # the fused tensor-core kernel, one CTA per work item
    for rep in range(2):
        for j in jobs:
            j["grid"].zero_()
        b.grid()
        idg.device_errors()
        for i, (w, op, j) in enumerate(zip(wls, ops, jobs)):
            parity(j["grid"].cpu().numpy(), O.grid(w, op), f"tc batch grid job {i} pass {rep}")
    djobs = [dict(j, grid=dev(m), vis=None) for j, m in zip(jobs, models)]
    bd = idg.Batch(plans, djobs, graph=graph)
    for rep in range(2):
        bd.degrid()
        idg.device_errors()
        for i, (w, op, j, m) in enumerate(zip(wls, ops, djobs, models)):
            parity(j["vis_out"].cpu().numpy(), O.degrid(w, op, m), f"tc batch degrid job {i} pass {rep}")


def test_batch_separable_and_direct_l32_classes():
    # two L = 32 jobs: one whose plan takes the separable kernels and one wide-field job over
    # the remainder bound (the direct tensor-core kernels); each forms its own class
    import torch
    wls = [_big_l32_jobs()[0],
           syn.make_small(seed=777, n_st=4, n_t=128, n_chan=16, L=32, N=512, max_t=128, n_slots=1, flag_p=0.05,
                          diameter_m=800.0, cell=1e-3, df=0.25e6)]
    plans = [idg.plan_from_workload(w) for w in wls]
    assert [p.stats.separable for p in plans] == [1, 0]
    ops = [O.plan(w) for w in wls]
    rng = np.random.default_rng(23)
    jobs, models = [], []
    for w, p in zip(wls, plans):
        d = workload_to_device(w)
        models.append(syn.random_grid(rng, p.n_w_layers, w.grid_size))
        jobs.append(dict(vis=d["vis"], flags=d["flags"], aterms=d["aterms"], taper=d["taper"],
                         grid=torch.zeros((p.n_w_layers, w.grid_size, w.grid_size, 4), dtype=torch.complex64,
                                          device="cuda"),
                         vis_out=torch.zeros(w.vis.shape, dtype=torch.complex64, device="cuda")))
    b = idg.Batch(plans, jobs)
    assert b.info()["n_launches"] == 2
    b.grid()
    idg.device_errors()
    for i, (w, op, j) in enumerate(zip(wls, ops, jobs)):
        parity(j["grid"].cpu().numpy(), O.grid(w, op), f"l32 classes grid job {i}")
    bd = idg.Batch(plans, [dict(j, grid=dev(m), vis=None) for j, m in zip(jobs, models)])
    bd.degrid()
    idg.device_errors()
    for i, (w, op, j, m) in enumerate(zip(wls, ops, jobs, models)):
        parity(j["vis_out"].cpu().numpy(), O.degrid(w, op, m), f"l32 classes degrid job {i}")


def test_batch_autotune_keeps_results():
    # the batch's autotuner times every persistent shape of every class, keeps the
    # fastest, and the batch (graph recorded again) still matches the oracle
    import torch
    wls = jobs_mix()
    plans = [idg.plan_from_workload(w) for w in wls]
    ops = [O.plan(w) for w in wls]
    jobs = []
    for w, p in zip(wls, plans):
        d = workload_to_device(w)
        jobs.append(dict(vis=d["vis"], flags=d["flags"], aterms=d["aterms"], taper=d["taper"],
                         grid=torch.zeros((p.n_w_layers, w.grid_size, w.grid_size, 4), dtype=torch.complex64,
                                          device="cuda"),
                         vis_out=torch.zeros(w.vis.shape, dtype=torch.complex64, device="cuda")))
    b = idg.Batch(plans, jobs, graph=True)
    b.grid()                                 # records the graph with the default shapes
    trials = b.autotune()
    assert len(trials) >= 4 and all(t > 0 for t in trials)
    for j in jobs:
        j["grid"].zero_()
    b.grid()
    torch.cuda.synchronize()
    for i, (w, op, j) in enumerate(zip(wls, ops, jobs)):
        parity(j["grid"].cpu().numpy(), O.grid(w, op), f"batch grid job {i} after autotune")


@pytest.mark.parametrize("graph", [False, True])
def test_batch_jobs_adding_into_one_grid(graph):
    # three separable L = 32 jobs of one grid size gridded into the same grid by one batch:
    # their per-job launches may overlap (programmatic dependent launches) and add into
    # the grid together; the result is the sum of the three oracle grids
    import torch
    wls = [syn.make_small(seed=410 + i, n_st=5, n_t=96, n_chan=8, L=32, N=256, max_t=96, n_slots=1, flag_p=0.05,
                          diameter_m=2500.0 + 500.0 * i) for i in range(3)]
    plans = [idg.plan_from_workload(w) for w in wls]
    assert all(p.stats.separable == 1 for p in plans)
    grid = torch.zeros((1, 256, 256, 4), dtype=torch.complex64, device="cuda")
    jobs = []
    for w in wls:
        d = workload_to_device(w)
        jobs.append(dict(vis=d["vis"], flags=d["flags"], aterms=d["aterms"], taper=d["taper"], grid=grid,
                         vis_out=None))
    b = idg.Batch(plans, jobs, graph=graph)
    for rep in range(2):
        grid.zero_()
        b.grid()
        idg.device_errors()
        ref = sum(O.grid(w, O.plan(w)) for w in wls)
        parity(grid.cpu().numpy(), ref, f"three jobs into one grid, pass {rep}")
