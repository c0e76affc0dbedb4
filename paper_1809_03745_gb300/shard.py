"""Host logic for running independent solves on several GPUs (one process per GPU).

The path shards by independent problems: every rank solves its own instances
and no collective touches the data path.  Two host pieces remain:

  * shard(): a deterministic greedy partition of instances over ranks by
    cost (largest first onto the least loaded rank), so each rank gets about
    the same number of cells;
  * job_time(): the whole job's time is the slowest rank's (max over ranks),
    and its throughput is all ranks' units over that time.

Both run over any torch.distributed backend (gloo on CPU in the tests).
"""
from __future__ import annotations


def shard(costs, world: int):
    """Instance indices per rank: greedy longest-processing-time partition,
    ties to the lower rank; deterministic for equal inputs."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]


def job_time(local_ms: float, group=None) -> float:
    """Max over ranks of each rank's measured time (ms); the local value
    when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(local_ms)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def throughput(units_per_rank, world: int, ms: float) -> float:
    """Whole-job units per second: every rank's units over the job time."""
    return units_per_rank * world / (ms / 1000.0)
