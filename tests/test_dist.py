"""Host logic of the multi-GPU path, run as 2 gloo ranks on CPU: every rank
derives the same partition of independent images, the partition is disjoint,
complete and balanced, and timings combine as max over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1107_4617_gb300 import dist as bdist
from paper_1107_4617_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, costs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bdist.shard(costs, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        seconds = 1.0 + rank  # rank 1 is the slowest
        units = float(sum(costs[i] for i in mine))
        tp = bdist.throughput(units, seconds)
        mx = bdist.max_over_ranks(float(rank * 10))
        q.put((rank, gathered, tp, mx))
    finally:
        dist.destroy_process_group()


def test_shard_is_deterministic_partition():
    costs = [s["H"] * s["W"] for s in synth.batch_specs(64, seed=3)]
    parts = [bdist.shard(costs, r, 4) for r in range(4)]
    allidx = sorted(i for p in parts for i in p)
    assert allidx == list(range(64))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) <= 1.15 * min(loads)
    assert bdist.shard(costs, 2, 4) == parts[2]
    with pytest.raises(ValueError):
        bdist.shard(costs, 4, 4)


def test_two_gloo_ranks():
    world = 2
    costs = [s["H"] * s["W"] for s in synth.batch_specs(32, seed=5)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    g0, g1 = res[0][1], res[1][1]
    assert g0 == g1  # every rank sees the same partition
    assert sorted(g0[0] + g0[1]) == list(range(len(costs)))
    assert not set(g0[0]) & set(g0[1])
    total = float(sum(costs))
    for _, _, tp, mx in res:
        assert tp == pytest.approx(total / 2.0)  # all units over the slowest rank's 2 s
        assert mx == 10.0
