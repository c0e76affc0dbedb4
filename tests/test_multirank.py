"""The multi-rank host path on CPU with gloo, world size 2: each rank solves
its own instances (no data-path collective), the job time is the max over
ranks and the throughput counts every rank's units; the instance partition is
balanced, complete and deterministic."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1809_03745_gb300 import shard as S
from paper_1809_03745_gb300 import workloads as W


def test_shard_balanced_complete_deterministic():
    inst = W.batched_instances(count=64)
    costs = [W.ncells(d) for d, _, _ in inst]
    parts = S.shard(costs, 4)
    assert sorted(i for p in parts for i in p) == list(range(64))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) <= sum(costs) / 4 + max(costs)  # greedy LPT bound: mean load plus the largest item
    assert min(loads) >= sum(costs) / 4 - max(costs)
    assert S.shard(costs, 4) == parts
    assert S.shard(costs, 1) == [list(range(64))]
    assert S.shard([5.0], 3) == [[0], [], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inst_costs = [float(W.ncells(d)) for d, _, _ in W.batched_instances(count=10, max_cells=50000)]
        mine = S.shard(inst_costs, world)[rank]
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        ms = S.job_time(local_ms)
        objs = [None] * world
        dist.all_gather_object(objs, mine)
        q.put((rank, ms, S.throughput(1000, world, ms), objs))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_gloo_job_time_and_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=100) for _ in range(2)]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, ms, thr, objs in res:
        assert ms == 15.0  # the slowest rank's time
        assert thr == pytest.approx(2 * 1000 / 0.015)
        assert sorted(objs[0] + objs[1]) == list(range(10)) and not set(objs[0]) & set(objs[1])


def _runner_worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_1809_03745_gb300 import batch_runner as R
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, R.run(count=12, solve=False, max_cells=50000)))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_batch_runner_ranks_receive_and_report_their_shards():
    """The sharded batched runner on two gloo ranks (planning and reporting;
    the solves themselves need the GPU): every rank gets the shard that
    shard() gives it, the reports gathered on each rank cover all instances
    exactly once, and the job's cells are their sum."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_runner_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=100) for _ in range(2))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    inst = W.batched_instances(count=12, max_cells=50000)
    parts = S.shard([float(W.ncells(d)) for d, _, _ in inst], 2)
    for rank in (0, 1):
        out = res[rank]
        assert out["world"] == 2
        reps = {r["rank"]: r for r in out["reports"]}
        assert reps[0]["instances"] == parts[0] and reps[1]["instances"] == parts[1]
        assert sorted(reps[0]["instances"] + reps[1]["instances"]) == list(range(12))
        assert out["cells"] == sum(W.ncells(d) for d, _, _ in inst)
        assert reps[rank]["cells"] == sum(W.ncells(inst[i][0]) for i in parts[rank])
