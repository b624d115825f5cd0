"""Multi-rank host logic on CPU (gloo, world size 2): stream sharding of the batched form and the
max-over-ranks timing / sum-over-ranks unit reduction the benchmark uses."""

import os
import socket

import pytest

from paper_2308_16395_gb300.sharding import assign_streams, stream_cost
from workloads import batched_streams


def test_assignment_is_a_balanced_partition():
    specs = batched_streams(nstreams=64, steps=100)
    costs = [stream_cost(s.spatial) for s, _ in specs]
    for ws in (1, 2, 3, 4, 8):
        parts = assign_streams(costs, ws)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: no rank exceeds the ideal share by more than the largest single stream
        assert max(loads) <= sum(costs) / ws + max(costs)
        assert assign_streams(costs, ws) == parts          # deterministic


def test_assignment_edge_cases():
    assert assign_streams([], 2) == [[], []]
    assert assign_streams([5], 3) == [[0], [], []]
    assert assign_streams([3, 3, 3, 3], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        assign_streams([1], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2308_16395_gb300.sharding import assign_streams, max_over_ranks, sum_over_ranks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [7, 3, 9, 1, 4, 4, 8, 2]
        mine = assign_streams(costs, world)[rank]
        # every rank computed the same partition: gather and compare
        got = [None] * world
        dist.all_gather_object(got, mine)
        ms = 10.0 + rank          # per-rank elapsed time
        units = len(mine)
        q.put((rank, got, max_over_ranks(ms), sum_over_ranks(units)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_partition_and_reductions():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    parts = res[0][1]
    assert res[1][1] == parts
    assert sorted(i for p in parts for i in p) == list(range(8))
    for _, _, mx, total in res:
        assert mx == 11.0                     # max over ranks
        assert total == 8.0                   # every stream counted once
