"""World-size-2 gloo run of the multi-rank host logic (CPU only): the timing
collective takes the max over ranks and the round-robin shards cover every
item exactly once."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2508_16387_gb300 import dist as D
    from paper_2508_16387_gb300 import workloads as WL
    ws, r, _ = D.rank_env()
    assert (ws, r) == (world, rank)
    t = D.max_over_ranks(10.0 + rank)
    jobs = WL.served_trace(n_jobs=11, seed=4)
    mine = [j.job_id for j in D.shard(jobs, r, ws)]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    dist.barrier()
    out[rank] = (t, sorted(sum(gathered, [])))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        t, ids = out[rank]
        assert t == 11.0                  # max over the ranks' times
        assert ids == list(range(11))     # every job on exactly one rank
