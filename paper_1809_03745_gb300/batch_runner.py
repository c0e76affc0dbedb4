"""Batched solves sharded over the ranks of a multi-GPU job (one GPU per rank).

The batched workload is a set of independent problems, so it splits across
GPUs without any exchange on the data path: every rank takes its share of the
seeded instances by `shard.shard` (largest first onto the least loaded rank,
by cell count), builds their geometry and hierarchies on its own GPU and
solves them in batched persistent launches (`eb_poisson_solve_batched`).  The
job's time is the slowest rank's and its throughput counts every rank's cells
(`shard.job_time`, `shard.throughput`); the only collectives are that max and
the gathering of the per-rank reports on the host.

Usage (one process per GPU):
    python -m torch.distributed.run --nproc-per-node N --master-addr 127.0.0.1 \
        -m paper_1809_03745_gb300.batch_runner [--count 64] [--steps 3]
"""
from __future__ import annotations

import argparse
import json
import os
import time

from . import shard as S
from . import workloads as W


def plan(rank: int, world: int, count: int = 64, max_cells=None):
    """This rank's instance indices and their descriptions/inputs."""
    inst = W.batched_instances(count=count, max_cells=max_cells)
    costs = [float(W.ncells(d)) for d, _, _ in inst]
    mine = S.shard(costs, world)[rank]
    return mine, [inst[i] for i in mine]


def solve_local(instances, device, steps: int = 3):
    """Solves this rank's instances in one batched launch per step (mixed
    precision, tol 1e-10); returns (median ms per step, statuses, max V-cycles)."""
    import statistics

    import torch

    from . import ebpoisson as E
    if not instances:
        return 0.0, [], 0
    P = [E.Poisson(E.Geometry(d, device=device), precision="mixed", tol=1e-10, max_cycles=600)
         for d, _, _ in instances]
    rhs = [torch.from_numpy(S_).to(device) for _, S_, _ in instances]
    sig = [torch.from_numpy(s).to(device) for _, _, s in instances]
    E.solve_batched(P, rhs, sig)  # warm-up
    ms, infos = [], []
    for _ in range(steps):
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        _, infos = E.solve_batched(P, rhs, sig)
        torch.cuda.synchronize(device)
        ms.append((time.perf_counter() - t0) * 1e3)
    return statistics.median(ms), sorted(set(i["status"] for i in infos)), max(i["vcycles"] for i in infos)


def run(count: int = 64, steps: int = 3, solve: bool = True, max_cells=None) -> dict:
    """One rank's part of the job inside an initialised process group; the
    report of every rank, gathered on every rank, plus the job figures."""
    import torch.distributed as dist
    rank, world = dist.get_rank(), dist.get_world_size()
    mine, inst = plan(rank, world, count, max_cells)
    cells = sum(W.ncells(d) for d, _, _ in inst)
    local_ms, statuses, vmax = 0.0, [], 0
    if solve:
        import torch
        local = int(os.environ.get("LOCAL_RANK", rank))
        torch.cuda.set_device(local)
        local_ms, statuses, vmax = solve_local(inst, torch.device("cuda", local), steps)
    report = {"rank": rank, "instances": mine, "cells": cells, "ms": local_ms, "statuses": statuses,
              "max_vcycles": vmax}
    reports = [None] * world
    dist.all_gather_object(reports, report)
    job_ms = S.job_time(local_ms)
    total = sum(r["cells"] for r in reports)
    return {"reports": reports, "job_ms": job_ms, "cells": total,
            "cells_per_s": total / (job_ms / 1e3) if job_ms > 0 else None, "world": world}


def main():
    import torch
    import torch.distributed as dist
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=64)
    ap.add_argument("--steps", type=int, default=3)
    args = ap.parse_args()
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    try:
        out = run(args.count, args.steps, solve=torch.cuda.is_available())
        if dist.get_rank() == 0:
            print(json.dumps({"workload": f"{args.count} seeded batched instances, sharded by cells, mixed, tol 1e-10",
                              "scaling": "strong: the instances are split over the ranks, no collective on "
                                         "the data path",
                              **out}), flush=True)
    finally:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
