"""Continuous-batching server: jobs of different grid sizes arriving over time
are admitted by free device memory, advanced together, and each job's result
is the same alone and in the mix (bit for bit: every grid keeps its own time
step and schedule). A job whose state is broken fails alone."""
import numpy as np
import pytest

from paper_2508_16387_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_16387_gb300 import m2c as M
    from paper_2508_16387_gb300 import serve as S
    M.lib()
    return M, S, torch


def small_trace(n=6):
    jobs = WL.served_trace(n_jobs=n, rate=200.0, seed=9, edge_range=(16, 28), steps_range=(8, 23))
    return jobs


def alone(S, M, job, prec):
    g = S.make_job_grid(job, prec)
    g.step(job.params.steps)
    code, _ = g.sync_status()
    return code, g.W.cpu().numpy(), g.phi.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_served_results_equal_alone(env, prec):
    M, S, torch = env
    jobs = small_trace()
    st = S.Server(precision=prec, slice_steps=5, keep_results=True).run(jobs, realtime=True)
    assert len(st.results) == len(jobs)
    assert st.max_resident >= 2          # the jobs overlapped on the device
    for r in st.results:
        job = jobs[r.job_id]
        code, W, phi = alone(S, M, job, prec)
        assert r.status == code == 0
        assert np.array_equal(r.W.numpy(), W)
        assert np.array_equal(r.phi.numpy(), phi)
        assert r.latency >= 0


def test_admission_by_free_memory(env):
    M, S, torch = env
    jobs = small_trace(4)
    for j in jobs:
        j.params.edge = 24               # equal sizes: the budget below holds exactly one job
    biggest = max(S.job_bytes(j.params.edge, 1) for j in jobs)
    base = torch.cuda.memory_allocated()
    budget = int(1.5 * biggest)          # room for one job at a time

    def free():
        return budget - (torch.cuda.memory_allocated() - base)
    st = S.Server(precision=1, slice_steps=50, reserve_bytes=0, free_bytes_fn=free, keep_results=True).run(
        jobs, realtime=False)
    assert st.max_resident == 1 and len(st.results) == 4
    for r in st.results:
        code, W, _ = alone(S, M, jobs[r.job_id], 1)
        assert np.array_equal(r.W.numpy(), W)


def test_broken_job_fails_alone(env):
    M, S, torch = env
    jobs = small_trace(4)

    def poison(job, grid):
        if job.job_id == 2:
            grid.W[0, 3, 3, 3] = float("nan")
    st = S.Server(precision=1, slice_steps=5, keep_results=True, on_admit=poison).run(jobs, realtime=False)
    by_id = {r.job_id: r for r in st.results}
    assert by_id[2].status != 0
    for j in (0, 1, 3):
        code, W, _ = alone(S, M, jobs[j], 1)
        assert by_id[j].status == 0
        assert np.array_equal(by_id[j].W.numpy(), W)
