"""Serving form: a request loop with continuous batching over the batched kernels.

Jobs (imaging requests) arrive over time.  Each job is one of
  "cycle"   n major cycles of  degrid(model grid) -> residual = observed - model
            -> grid(residual) -> model update  (the residual formulation of the
            gradient, Sect. 2 of the paper, as used by deconvolution major cycles)
  "grid"    one gridding of the observed visibilities
  "degrid"  one degridding of the model grid
Admission control keeps a device-memory budget and a maximum number of slots.
The engine advances every admitted job by one step per iteration: all
pending degrids run as ONE batch (idg_batch_degrid: one persistent launch per
subgrid size across all those jobs), then all pending grids as one batch.
Jobs arriving while others run are admitted at the next iteration if a slot
and memory are free, so their work shares the same launches (continuous
batching); a job's grids stay resident on the device across its cycles.

The model update of "cycle" jobs is synthetic: model <- model + 0.5 (truth - model)
for a fixed seeded truth grid.  Device arithmetic outside gridding/degridding
(the residual and the model update) is a single elementwise torch operation.
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import time
from typing import Dict, List, Optional

import numpy as np

from . import idg


# ---------------------------------------------------------------------------
# admission (host only, testable without a GPU)

@dataclasses.dataclass
class Admission:
    """Device-memory and slot accounting.  `need` is a job's resident bytes."""
    budget_bytes: int
    max_slots: int
    used_bytes: int = 0
    active: Dict[int, int] = dataclasses.field(default_factory=dict)

    def fits(self, need: int) -> bool:
        return len(self.active) < self.max_slots and self.used_bytes + need <= self.budget_bytes

    def admit(self, job_id: int, need: int) -> bool:
        if job_id in self.active or not self.fits(need):
            return False
        self.active[job_id] = need
        self.used_bytes += need
        return True

    def release(self, job_id: int):
        need = self.active.pop(job_id)
        self.used_bytes -= need


def job_bytes(wl, n_w: int = 1) -> int:
    """Resident device bytes of a job: observed and work visibilities, flags,
    model, residual and truth grids, taper."""
    vis = wl.n_vis * 32
    grid = n_w * wl.grid_size * wl.grid_size * 32
    return 2 * vis + wl.n_vis + 3 * grid + wl.subgrid_size ** 2 * 4


# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Job:
    id: int
    kind: str
    wl: object
    arrival: float                 # seconds from the start of the trace
    n_cycles: int = 5
    seed: int = 0
    plan: Optional[object] = None
    bufs: Optional[dict] = None
    step: int = 0                  # completed steps
    done_at: Optional[float] = None
    admitted_at: Optional[float] = None
    need: int = 0
    data: Optional[object] = None

    @property
    def n_steps(self):
        return self.n_cycles if self.kind == "cycle" else 1

    @property
    def vis_passes(self):
        # visibilities processed: a cycle is one degrid and one grid pass
        return self.wl.n_vis * (2 * self.n_cycles if self.kind == "cycle" else 1)


def make_trace(workloads, rate_per_s: float, kinds=("cycle",), seed: int = 1913, n_cycles: int = 5) -> List[Job]:
    """Poisson arrivals at rate_per_s; the kind of each request drawn from kinds."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for i, wl in enumerate(workloads):
        t += float(rng.exponential(1.0 / rate_per_s))
        jobs.append(Job(i, str(rng.choice(list(kinds))), wl, t, n_cycles=n_cycles, seed=int(rng.integers(1 << 30))))
    return jobs


class JobData:
    """Device buffers of a job (observed visibilities drawn on the device)."""

    def __init__(self, job: Job, device, plan):
        import torch
        wl = job.wl
        gen = torch.Generator(device=device)
        gen.manual_seed(job.seed)
        shape = (wl.n_bl, wl.n_t, wl.n_chan, 4)
        gshape = (plan.n_w_layers, wl.grid_size, wl.grid_size, 4)
        self.observed = torch.randn(shape, dtype=torch.complex64, device=device, generator=gen)
        self.work = torch.zeros(shape, dtype=torch.complex64, device=device)
        p = getattr(wl, "flag_p", 0.0)
        self.flags = (torch.rand(shape[:3], device=device, generator=gen) < p).to(torch.uint8)
        self.truth = torch.randn(gshape, dtype=torch.complex64, device=device, generator=gen)
        self.model = torch.zeros(gshape, dtype=torch.complex64, device=device)
        self.residual = torch.zeros(gshape, dtype=torch.complex64, device=device)
        self.taper = torch.from_numpy(wl.taper).to(device)
        if wl.aterms is not None:
            self.aterms = torch.from_numpy(wl.aterms).to(device)
        else:
            self.aterms = None

    def degrid_buffers(self):
        return dict(vis=None, vis_out=self.work, flags=self.flags, aterms=self.aterms, taper=self.taper,
                    grid=self.model)

    def grid_buffers(self, source):
        return dict(vis=source, vis_out=None, flags=self.flags, aterms=self.aterms, taper=self.taper,
                    grid=self.residual)


class Engine:
    """Continuous-batching request loop on one GPU stream."""

    def __init__(self, budget_bytes: int = 150 << 30, max_slots: int = 32, graph: bool = True,
                 host_threads: int = 4, device=None, keep: bool = False):
        import torch
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.current_stream(self.device)
        self.adm = Admission(budget_bytes, max_slots)
        self.graph = graph
        self.pool = concurrent.futures.ThreadPoolExecutor(host_threads)
        self._batches = {}
        self.iterations = 0
        self.launch_sets = []
        self.keep = keep           # keep the device buffers of finished jobs (tests)
        self.max_active = 0
        self.host_batch_s = 0.0    # host time spent building batches

    def _batch(self, jobs, kind):
        key = (kind, tuple(j.id for j in jobs))
        b = self._batches.get(key)
        if b is None:
            t0 = time.perf_counter()
            if kind == "degrid":
                bufs = [j.data.degrid_buffers() for j in jobs]
            else:
                bufs = [j.data.grid_buffers(j.data.work if j.kind == "cycle" else j.data.observed) for j in jobs]
            b = idg.Batch([j.plan for j in jobs], bufs, graph=self.graph)
            self._batches[key] = b
            self.host_batch_s += time.perf_counter() - t0
        return b

    def _drop_batches(self, job_id):
        for k in [k for k in self._batches if job_id in k[1]]:
            self._batches.pop(k).destroy()

    def run(self, jobs: List[Job], clock=time.perf_counter) -> dict:
        """Serve the trace in real time; returns latency and throughput stats."""
        import torch
        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
        planning = {}
        active: List[Job] = []
        t0 = clock()
        waiting = collections.deque()
        while pending or waiting or planning or active:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                j = pending.popleft()
                waiting.append(j)
                planning[j.id] = self.pool.submit(idg.plan_from_workload, j.wl)
            # admit in arrival order while slots and memory allow
            while waiting and planning[waiting[0].id].done():
                j = waiting[0]
                j.plan = planning[j.id].result()
                j.need = job_bytes(j.wl, j.plan.n_w_layers)
                if not self.adm.admit(j.id, j.need):
                    break
                waiting.popleft()
                planning.pop(j.id)
                j.data = JobData(j, self.device, j.plan)
                j.admitted_at = clock() - t0
                active.append(j)
            if not active:
                nxt = pending[0].arrival if pending else None
                if nxt is not None and not waiting:
                    time.sleep(max(0.0, min(0.01, nxt - (clock() - t0))))
                else:
                    time.sleep(0.0005)
                continue
            # one iteration: all degrids, residuals, all grids, model updates
            self.iterations += 1
            self.max_active = max(self.max_active, len(active))
            deg = [j for j in active if j.kind in ("cycle", "degrid")]
            grd = [j for j in active if j.kind in ("cycle", "grid")]
            self.launch_sets.append((len(deg), len(grd)))
            if deg:
                self._batch(deg, "degrid").degrid(self.stream)
            for j in active:
                if j.kind == "cycle":
                    torch.sub(j.data.observed, j.data.work, out=j.data.work)   # residual visibilities
                    j.data.residual.zero_()
                elif j.kind == "grid":
                    j.data.residual.zero_()
            if grd:
                self._batch(grd, "grid").grid(self.stream)
            for j in active:
                if j.kind == "cycle":
                    j.data.model.lerp_(j.data.truth, 0.5)      # synthetic model update
            torch.cuda.synchronize(self.device)
            t_done = clock() - t0
            still = []
            for j in active:
                j.step += 1
                if j.step >= j.n_steps:
                    j.done_at = t_done
                    self.adm.release(j.id)
                    self._drop_batches(j.id)
                    if not self.keep:
                        j.data = None
                else:
                    still.append(j)
            active = still
        makespan = clock() - t0
        return summarize(jobs, makespan)


def summarize(jobs: List[Job], makespan: float) -> dict:
    lat = np.array([j.done_at - j.arrival for j in jobs])
    passes = float(sum(j.vis_passes for j in jobs))
    # a "visibility pass" is one visibility gridded or degridded once; a grid +
    # degrid pair of passes counts as one visibility in the grid+degrid metric
    return {"jobs": len(jobs), "makespan_s": makespan, "mvis_passes_per_s": passes / makespan / 1e6,
            "grid_degrid_mvis_per_s": 0.5 * passes / makespan / 1e6,
            "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "latency_mean_s": float(lat.mean()), "vis_passes": passes}


def run_plain_fifo(jobs: List[Job], device=None, clock=time.perf_counter, keep: bool = False) -> dict:
    """Per-job plain form on the same trace: one job at a time in arrival order
    with idg_grid / idg_degrid."""
    import torch
    device = device or torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(device)
    t0 = clock()
    for j in sorted(jobs, key=lambda j: j.arrival):
        while clock() - t0 < j.arrival:
            time.sleep(0.0005)
        plan = idg.plan_from_workload(j.wl)
        d = JobData(j, device, plan)
        for _ in range(j.n_steps):
            if j.kind in ("cycle", "degrid"):
                idg.degrid(plan, d.model, d.flags, d.aterms, d.taper, d.work, stream)
            if j.kind == "cycle":
                torch.sub(d.observed, d.work, out=d.work)
            if j.kind in ("cycle", "grid"):
                d.residual.zero_()
                idg.grid(plan, d.work if j.kind == "cycle" else d.observed, d.flags, d.aterms, d.taper,
                         d.residual, stream)
            if j.kind == "cycle":
                d.model.lerp_(d.truth, 0.5)
        torch.cuda.synchronize(device)
        j.done_at = clock() - t0
        if keep:
            j.data, j.plan = d, plan
    return summarize(jobs, clock() - t0)
