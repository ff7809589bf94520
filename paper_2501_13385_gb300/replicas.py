"""Host-side logic of the multi-GPU launch: one process per GPU, each solving
its own independent replicas of the workload (PRGD problems do not exchange
data, so no collective sits on the data path).  Only the timing uses the
process group: the slowest rank's time, taken with a MAX all-reduce, prices
the whole job."""
from __future__ import annotations

from typing import List


def replica_seeds(rank: int, batch: int) -> List[int]:
    """Seeds of the problems rank `rank` solves: `batch` consecutive seeds,
    disjoint across ranks, so the job's problems are the same whatever the
    number of ranks that share them."""
    return [rank * batch + i for i in range(batch)]


def max_over_ranks(value: float, world: int) -> float:
    """MAX of `value` over the ranks of the default process group (the
    identity when world == 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, batch: int, units_per_problem: int, steps: int, total_ms: float) -> float:
    """Units all ranks processed per second: world x batch problems, each
    processing `units_per_problem` units per step, over `steps` steps that
    took `total_ms` on the slowest rank."""
    return world * batch * units_per_problem * steps / (total_ms / 1e3)
