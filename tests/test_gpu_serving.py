"""Serving engine: each job's results are the same alone and in a mix with
other jobs that arrive while it runs (continuous batching), within the parity
tolerance; the mix really shares launches."""
import numpy as np
import pytest

from paper_1909_07226_gb300 import idg, serving
from paper_1909_07226_gb300 import synthetic as syn
from tests.gpu_util import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_07226_gb300 import build
    build.build()
    idg.load()


def test_same_result_alone_and_in_the_mix():
    wls = syn.make_batched_jobs(6, seed=21, scale_t=0.1)
    kinds = ("cycle",)
    # alone
    alone = serving.make_trace(wls[:1], 1e5, kinds, seed=4, n_cycles=3)
    eng = serving.Engine(budget_bytes=64 << 30, keep=True)
    eng.run(alone)
    a = alone[0]
    ref_model = a.data.model.cpu().numpy()
    ref_resid = a.data.residual.cpu().numpy()
    ref_work = a.data.work.cpu().numpy()
    # in the mix: the same job first, five more arriving while it runs
    mix = serving.make_trace(wls, 1e5, kinds, seed=4, n_cycles=3)
    mix[0].seed = a.seed
    eng2 = serving.Engine(budget_bytes=64 << 30, keep=True)
    eng2.run(mix)
    m = mix[0]
    assert max(n for n, _ in eng2.launch_sets) > 1          # batched together with other jobs
    parity(m.data.residual.cpu().numpy(), ref_resid, "serving residual grid alone vs mix", tol=1e-6)
    parity(m.data.work.cpu().numpy(), ref_work, "serving residual visibilities alone vs mix", tol=1e-6)
    assert np.array_equal(m.data.model.cpu().numpy(), ref_model)  # model updates do not depend on the mix


def test_serving_matches_plain_per_job():
    wls = syn.make_batched_jobs(4, seed=22, scale_t=0.1)
    kinds = ("cycle", "grid", "degrid")
    t1 = serving.make_trace(wls, 1000.0, kinds, seed=9, n_cycles=2)
    serving.Engine(budget_bytes=64 << 30, keep=True).run(t1)
    t2 = serving.make_trace(wls, 1000.0, kinds, seed=9, n_cycles=2)
    serving.run_plain_fifo(t2, keep=True)
    for a, b in zip(t1, t2):
        assert a.kind == b.kind
        if a.kind in ("cycle", "grid"):
            parity(a.data.residual.cpu().numpy(), b.data.residual.cpu().numpy(), f"serving vs plain grid job {a.id}",
                   tol=1e-6)
        if a.kind in ("cycle", "degrid"):
            parity(a.data.work.cpu().numpy(), b.data.work.cpu().numpy(), f"serving vs plain vis job {a.id}", tol=1e-6)


def test_served_cycle_job_matches_the_oracle():
    # A "cycle" job served inside a mix, checked against the FP64 oracle's
    # composition of the residual formulation (Sect. 2): after 3 major cycles the
    # model is m2 = 0.75 truth (m0 = 0, m <- m + (truth - m) / 2), the residual
    # visibilities are observed - degrid(m2) (flagged and dropped ones: the model
    # is 0 there) and the residual grid is grid(residual) over unflagged samples.
    from oracle import oracle as O
    wls = syn.make_batched_jobs(6, seed=23, scale_t=0.1)
    trace = serving.make_trace(wls, 1e5, ("cycle",), seed=5, n_cycles=3)
    eng = serving.Engine(budget_bytes=64 << 30, keep=True)
    eng.run(trace)
    assert max(n for n, _ in eng.launch_sets) > 1          # the job shared launches with others
    job = min(trace, key=lambda j: j.wl.n_vis)               # the smallest keeps the oracle quick
    wl, dd = job.wl, job.data
    observed = dd.observed.cpu().numpy().astype(np.complex128)
    flags = dd.flags.cpu().numpy()
    m2 = 0.75 * dd.truth.cpu().numpy().astype(np.complex128)
    op = O.plan(wl)
    assert np.array_equal(job.plan.export(), op.desc)
    model_vis = O.degrid(wl, op, m2, flags=flags)
    resid = observed - model_vis
    parity(dd.work.cpu().numpy(), resid, f"served job {job.id}: residual visibilities vs oracle")
    ref_grid = O.grid(wl, op, vis=resid.astype(np.complex64), flags=flags)
    parity(dd.residual.cpu().numpy(), ref_grid, f"served job {job.id}: residual grid vs oracle")
