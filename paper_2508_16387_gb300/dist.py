"""Multi-GPU host logic of the benchmark and the server: one process per GPU,
each running its own grids (the workloads are independent grids, so there is
no data-path exchange); the only collectives are a barrier and the max of the
per-rank times."""
from __future__ import annotations

import os


def rank_env():
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float) -> float:
    """The largest x over all ranks (x itself without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(items, rank: int, world: int):
    """Round-robin share of `items` (e.g. jobs of a trace, grids of a batch) for one rank."""
    return [it for i, it in enumerate(items) if i % world == rank]
