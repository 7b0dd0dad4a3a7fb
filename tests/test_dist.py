"""Host logic of the multi-GPU path, run as gloo ranks on CPU:
- independent images: every rank derives the same partition, the partition is
  disjoint, complete and balanced, and timings combine as max over ranks;
- one image in row bands: with the FP64 oracle as each rank's filter, the
  halo exchange reproduces the whole-image output, dL/df and dL/dgamma."""
import os
import socket

import math

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
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


def _band_worker(rank, world, port, f, g, r, N, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        gam = math.pi / 2
        y0, y1 = bdist.band(f.shape[0], rank, world)
        lf = torch.from_numpy(f[y0:y1].copy())
        lg = torch.from_numpy(g[y0:y1].copy())
        out = bdist.banded_forward(
            lf, r, lambda e: torch.from_numpy(oracle.bilateral(e.numpy(), r, gam, N)), rank, world)
        gi = bdist.banded_gradient(
            lf, lg, r, lambda e, h: torch.from_numpy(oracle.bilateral_grad(e.numpy(), h.numpy(), r,
                                                                           gam, N)[0]),
            rank, world)
        dgam = bdist.banded_scalar_grad(
            lf, lg, r, lambda e, h: oracle.bilateral_grad(e.numpy(), h.numpy(), r, gam, N)[1],
            rank, world)
        q.put((rank, y0, y1, out.numpy(), gi.numpy(), dgam))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,H,r", [(2, 40, 3), (3, 61, 4), (4, 64, 2)])
def test_row_bands_reproduce_whole_image(world, H, r):
    W, N = 23, 11
    f = synth.rectangles(H, W, seed=world).astype(np.float64)
    g = synth.weights((H, W), seed=world + 1).astype(np.float64)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_band_worker, args=(k, world, port, f, g, r, N, q))
             for k in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gam = math.pi / 2
    out_ref = oracle.bilateral(f, r, gam, N)
    gi_ref, dgam_ref = oracle.bilateral_grad(f, g, r, gam, N)
    out = np.concatenate([x[3] for x in res])
    gi = np.concatenate([x[4] for x in res])
    assert [x[1] for x in res] == [bdist.band(H, k, world)[0] for k in range(world)]
    np.testing.assert_allclose(out, out_ref, rtol=0, atol=1e-13)
    np.testing.assert_allclose(gi, gi_ref, rtol=0, atol=1e-12)
    for x in res:  # every rank holds the all-reduced sum
        assert x[5] == pytest.approx(dgam_ref, rel=1e-11, abs=1e-12)


def test_band_split_and_short_bands():
    assert [bdist.band(10, k, 3) for k in range(3)] == [(0, 3), (3, 6), (6, 10)]
    assert bdist.band(7, 0, 1) == (0, 7)
    with pytest.raises(ValueError):
        bdist.band(10, 3, 3)
    t = torch.zeros((3, 5))
    with pytest.raises(ValueError):
        bdist.exchange_halo(t, 4, 0, 2)  # a band shorter than its halo
    ext, top = bdist.exchange_halo(t, 4, 0, 1)  # one rank: nothing to exchange
    assert ext is t and top == 0
