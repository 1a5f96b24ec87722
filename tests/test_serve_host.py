"""Host logic of the continuous-batching server with the device parts replaced by fakes (no GPU):
admission in arrival order while free memory allows, the resident cap, slices that never step a
job past its step count, failure of one job at admission isolated from the others, the
too-large-job error, and the accounting of cell updates and times."""
import math
import time
import types

import pytest

from paper_2508_16387_gb300 import m2c as M
from paper_2508_16387_gb300 import serve as S
from paper_2508_16387_gb300 import workloads as WL


class FakeGrid:
    def __init__(self, job):
        self.job = job
        self.N = job.params.edge ** 3
        self.steps = 0

    def sync_status(self):
        return 0, -1


class FakeBatch:
    log = []

    def __init__(self, grids, tuning):
        self.grids = list(grids)

    def step(self, n):
        FakeBatch.log.append((tuple(g.job.job_id for g in self.grids), n))
        for g in self.grids:
            g.steps += n


def _jobs(spec):
    return [WL.Job(i, 0.01 * i, WL.InstanceParams(edge, 0.1, (0.5, 0.5, 0.5), 1e9, steps))
            for i, (edge, steps) in enumerate(spec)]


@pytest.fixture
def fake_device(monkeypatch):
    FakeBatch.log = []
    grids = {}

    def make_job_grid(job, precision, water=WL.WATER_SG, device="cuda"):
        if job.params.edge == 13:   # a job whose state cannot be built
            raise M.M2CError(M.M2C_EINVAL, "m2c_init_grid", "bad job")
        grids[job.job_id] = FakeGrid(job)
        return grids[job.job_id]
    monkeypatch.setattr(S, "make_job_grid", make_job_grid)
    monkeypatch.setattr(S.M, "Batch", FakeBatch)
    monkeypatch.setattr(S, "job_bytes", lambda edge, precision: edge ** 3)
    return grids


def _server(free, **kw):
    srv = S.Server(free_bytes_fn=lambda: free[0], reserve_bytes=0, warm=False, **kw)
    srv.torch = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))
    return srv


def test_every_job_steps_exactly_its_count_in_slices(fake_device):
    jobs = _jobs([(4, 60), (5, 25), (6, 100), (4, 7)])
    st = _server([10 ** 9], slice_steps=20).run(jobs, realtime=False)
    assert sorted(r.job_id for r in st.results) == [0, 1, 2, 3]
    for j in jobs:
        assert fake_device[j.job_id].steps == j.params.steps
    # every slice is at most slice_steps long (and no job was stepped past its count, above)
    for ids, n in FakeBatch.log:
        assert 1 <= n <= 20
    assert st.cell_updates == sum(j.params.steps * j.params.edge ** 3 for j in jobs)
    assert st.slices == len(FakeBatch.log)
    for r in st.results:   # not realtime: every job is available at once, whatever its arrival
        assert r.status == 0 and r.admitted <= r.finished


def test_admission_in_arrival_order_while_memory_allows(fake_device):
    """Device memory for two of these jobs at a time (a job holds its memory from admission to
    completion): the third waits for the first to finish and the fourth never overtakes it."""
    jobs = _jobs([(10, 30), (10, 50), (10, 20), (4, 10)])

    def free():
        live = [g for g in fake_device.values() if g.steps < g.job.params.steps]
        return 2 * 1000 - sum(g.N for g in live)
    srv = S.Server(free_bytes_fn=free, reserve_bytes=0, slice_steps=100, warm=False)
    srv.torch = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))
    st = srv.run(jobs, realtime=False)
    batches = [ids for ids, _ in FakeBatch.log]
    assert batches[0] == (0, 1)
    first_with_2 = next(i for i, b in enumerate(batches) if 2 in b)
    assert all(0 not in b for b in batches[first_with_2:])      # job 2 waited for job 0
    first_with_3 = next(i for i, b in enumerate(batches) if 3 in b)
    assert first_with_3 >= first_with_2                        # and job 3 did not overtake it
    assert st.max_resident == 2
    assert len(st.results) == 4 and all(r.status == 0 for r in st.results)


def test_resident_cap(fake_device):
    jobs = _jobs([(4, 10)] * 6)
    st = _server([10 ** 9], slice_steps=5, max_resident=2).run(jobs, realtime=False)
    assert st.max_resident == 2
    assert all(len(ids) <= 2 for ids, _ in FakeBatch.log)
    assert len(st.results) == 6


def test_a_job_failing_at_admission_does_not_stop_the_others(fake_device):
    jobs = _jobs([(4, 10), (13, 10), (5, 10)])
    st = _server([10 ** 9], slice_steps=10).run(jobs, realtime=False)
    by_id = {r.job_id: r for r in st.results}
    assert by_id[1].status == M.M2C_EINVAL
    assert by_id[0].status == 0 and by_id[2].status == 0
    assert all(1 not in ids for ids, _ in FakeBatch.log)


def test_a_job_that_can_never_fit_is_an_error(fake_device):
    with pytest.raises(RuntimeError):
        _server([100], slice_steps=10).run(_jobs([(10, 10)]), realtime=False)


def test_a_job_that_can_never_fit_fails_at_once_in_real_time(fake_device):
    """With nothing resident the error comes when the job is queued, not after the later jobs of
    the trace have arrived (their arrival frees no memory)."""
    jobs = _jobs([(10, 10), (4, 10)])
    jobs[1] = WL.Job(1, 30.0, jobs[1].params)   # arrives 30 s later
    t0 = time.perf_counter()
    with pytest.raises(RuntimeError, match="job 0"):
        _server([100], slice_steps=10).run(jobs, realtime=True)
    assert time.perf_counter() - t0 < 5.0


def test_percentiles_of_latency():
    st = S.ServeStats()
    for k, lat in enumerate([5.0, 1.0, 3.0, 2.0, 4.0]):
        st.results.append(S.JobResult(k, 0.0, 0.0, lat, 1, 1, 0))
    assert st.percentile(50) == 3.0 and st.percentile(0) == 1.0 and st.percentile(100) == 5.0
    assert math.isnan(S.ServeStats().percentile(50))   # no results
