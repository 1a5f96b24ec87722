"""Continuous-batching server of shock-bubble jobs on one GPU.

Jobs (workloads.Job: arrival time, grid edge, steps, bubble and shock
parameters) arrive over time. The server keeps every admitted job's state
resident on the device and advances all resident jobs together, one batched
launch per kernel (m2c_batch), in slices of at most `slice_steps` steps that
end when the next job finishes. Between slices it evicts finished jobs
(copying their state to the host) and admits waiting jobs in arrival order
while free device memory, less a reserve, covers their state and workspace.
Every grid keeps its own time step and reinitialisation schedule, so a job's
result is the same alone and in any mix.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Optional

from . import m2c as M
from . import workloads as WL

BYTES_PER_CELL_STATE = 6 * 8  # W (5 doubles) and phi


@dataclass
class JobResult:
    job_id: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    cells: int
    status: int
    err_cell: int = -1
    W: Optional[object] = None
    phi: Optional[object] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Resident:
    job: WL.Job
    grid: M.Grid
    remaining: int
    admitted: float


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    wall_s: float = 0.0
    cell_updates: int = 0
    slices: int = 0
    max_resident: int = 0

    def latencies(self):
        return sorted(r.latency for r in self.results)

    def percentile(self, q: float) -> float:
        xs = self.latencies()
        if not xs:
            return float("nan")
        k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
        return xs[k]


def job_setup(job: WL.Job, water=WL.WATER_SG):
    q = job.params
    return WL.Setup(f"job{job.job_id}_{q.edge}^3", (q.edge,) * 3, 1.0 / q.edge, (water, WL.AIR_PG),
                    (WL.BC_TRANSMISSIVE,) * 6, None, None,
                    {WL.AMBIENT: (1000.0, 0.0, 0.0, 0.0, 1e5), WL.BUBBLE: (1.2, 0.0, 0.0, 0.0, 1e5)},
                    shock=(q.p_shock, WL.AMBIENT), steps=q.steps)


def make_job_grid(job: WL.Job, precision, water=WL.WATER_SG, device="cuda"):
    """A context for a job with its initial state built on the device."""
    s = job_setup(job, water)
    q = job.params
    phi, region = WL.shock_bubble_device(q.edge, q.radius, q.centre, q.p_shock, device=device)
    amb = s.prims_by_region[WL.AMBIENT]
    r1, u1, _ = M.m2c_shock_state(water, (amb[0], amb[1], amb[4]), q.p_shock)
    P = WL.prims_device(region, s.prims_by_region, (r1, u1), q.p_shock)
    g = M.Grid(s.n, s.h, s.bc, s.eos, precision=precision, cfl=s.cfl, reinit_every=s.reinit_every,
               reinit_iters=s.reinit_iters, device=device)
    g.set_prims(P, phi)
    return g


def warm_up(precision, water=WL.WATER_SG, device="cuda"):
    """Builds and steps one small job once, untimed, before a server takes jobs: the first job
    set-ups in a process (the device-side construction with PyTorch's elementwise and indexing
    kernels) carry a one-time cost, measured at about 12 s over the first 16 jobs on a fresh
    GB300 machine and none once they have run, which belongs to the server's start, not to the
    latency of the jobs it serves."""
    import torch
    job = WL.Job(-1, 0.0, WL.InstanceParams(edge=16, radius=0.15, centre=(0.5, 0.5, 0.5), p_shock=1e9, steps=2))
    g = make_job_grid(job, precision, water, device=device)
    b = M.Batch([g], (8, 0, 0, 0))
    b.step(2)
    g.sync_status()
    torch.cuda.synchronize()
    del b, g


def job_bytes(edge: int, precision) -> int:
    return M.m2c_workspace_bytes(edge, edge, edge, precision) + BYTES_PER_CELL_STATE * edge ** 3 + (1 << 20)


class Server:
    def __init__(self, precision=M.MIXED, slice_steps: int = 25, reserve_bytes: int = 4 << 30,
                 tuning=(8, 0, 0, 0), water=WL.WATER_SG, keep_results: bool = False, free_bytes_fn=None,
                 max_resident: int = 0, on_admit=None, warm: bool = True):
        import torch
        self.torch = torch
        self.precision = precision
        self.slice_steps = slice_steps
        self.reserve = reserve_bytes
        self.tuning = tuning
        self.water = water
        self.keep = keep_results
        self.free_bytes_fn = free_bytes_fn or self._free_bytes
        self.max_resident = max_resident
        self.on_admit = on_admit  # test hook: called with (job, grid) after a job's state is built
        self.warm = warm          # run warm_up() once, before the first trace's clock starts

    def _free_bytes(self) -> int:
        torch = self.torch
        free, _ = torch.cuda.mem_get_info()
        return free + torch.cuda.memory_reserved() - torch.cuda.memory_allocated()

    def run(self, jobs, realtime: bool = True) -> ServeStats:
        """Serves a trace of jobs (sorted by arrival); arrival times are honoured in wall time
        when realtime, else every job is available at once."""
        torch = self.torch
        if self.warm:
            warm_up(self.precision, self.water)
            self.warm = False
        pending = sorted(jobs, key=lambda j: j.arrival)
        queue, resident = [], []
        st = ServeStats()
        batch = None
        dirty = True
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        while pending or queue or resident:
            t = now()
            while pending and (not realtime or pending[0].arrival <= t):
                queue.append(pending.pop(0))
            # admission in arrival order while memory allows
            while queue and (not self.max_resident or len(resident) < self.max_resident):
                need = job_bytes(queue[0].params.edge, self.precision)
                if self.free_bytes_fn() - need < self.reserve:
                    break
                job = queue.pop(0)
                try:
                    g = make_job_grid(job, self.precision, self.water)
                except M.M2CError as err:
                    st.results.append(JobResult(job.job_id, job.arrival, now(), now(), job.params.steps,
                                                job.params.edge ** 3, err.code))
                    continue
                if self.on_admit is not None:
                    self.on_admit(job, g)
                resident.append(_Resident(job, g, job.params.steps, now()))
                g = None  # the resident list is the only owner, so eviction frees the memory
                dirty = True
            st.max_resident = max(st.max_resident, len(resident))
            if not resident:
                # with nothing resident, no eviction can free memory for the head of the queue
                if queue:
                    raise RuntimeError(f"job {queue[0].job_id} does not fit in device memory")
                if pending and realtime:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now())))
                continue
            if dirty:
                batch = None
                batch = M.Batch([r.grid for r in resident], self.tuning)
                dirty = False
            n = min(self.slice_steps, min(r.remaining for r in resident))
            batch.step(n)
            torch.cuda.synchronize()
            st.slices += 1
            done = []
            for r in resident:
                r.remaining -= n
                st.cell_updates += n * r.grid.N
                if r.remaining == 0:
                    done.append(r)
            if done:
                t_fin = now()
                for r in done:
                    code, cell = r.grid.sync_status()
                    res = JobResult(r.job.job_id, r.job.arrival, r.admitted, t_fin, r.job.params.steps,
                                    r.grid.N, code, cell)
                    if self.keep:
                        res.W = r.grid.W.cpu()
                        res.phi = r.grid.phi.cpu()
                    st.results.append(res)
                    resident.remove(r)
                batch = None
                dirty = True
                for r in done:
                    del r.grid
        st.wall_s = now()
        return st


def serve_serial(jobs, precision=M.FP64, realtime: bool = True, water=WL.WATER_SG, warm: bool = True) -> ServeStats:
    """Baseline: one job at a time in arrival order, each stepped alone with m2c_step (after the
    same warm-up as the server's)."""
    import torch
    if warm:
        warm_up(precision, water)
    st = ServeStats()
    t0 = time.perf_counter()
    for job in sorted(jobs, key=lambda j: j.arrival):
        if realtime:
            wait = job.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        t_adm = time.perf_counter() - t0
        g = make_job_grid(job, precision, water)
        g.step(job.params.steps)
        code, cell = g.sync_status()
        torch.cuda.synchronize()
        t_fin = time.perf_counter() - t0
        st.results.append(JobResult(job.job_id, job.arrival, t_adm, t_fin, job.params.steps, g.N, code, cell))
        st.cell_updates += job.params.steps * g.N
        del g
    st.wall_s = time.perf_counter() - t0
    return st
