"""Multi-GPU orchestration (one process per GPU).

Independent images: the filter has no exchange step between images, so each
rank filters its own images and no collective touches the data path. Ranks
only meet to time a run (a barrier before and after, then the slowest rank's
time).

One image in row bands: rank k owns rows [y0, y1) of the image. An output row
depends on input rows within r of it, so the forward needs a halo of r rows
from each neighbouring band, exchanged point to point before the filter. The
adjoint's dL/df at a row depends on dL/dout, den and out within r rows, whose
forward values depend on f within 2r: a 2r halo of f and an r halo of dL/dout.
dL/dsigma_r (a sum over the image) takes one scalar all-reduce. Restricting
the haloed result to the band's own rows reproduces the whole-image result:
the windows kept never reach the halo's edge, except at the image's own
border, where the truncation is the image's.

These helpers work with any torch.distributed backend (NCCL on GPUs, gloo on
CPU for the tests).
"""
from __future__ import annotations

import heapq


def shard(costs, rank: int, world: int):
    """Indices of the items rank `rank` of `world` processes, assigned by
    longest-processing-time-first: items sorted by decreasing cost, each given
    to the currently least-loaded rank (ties to the lowest rank). Deterministic,
    so every rank computes the same partition without communicating."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return sorted(mine)


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def throughput(units_this_rank: float, seconds_this_rank: float, device=None) -> float:
    """Whole-job throughput: units processed by all ranks over the slowest
    rank's time."""
    total = sum_over_ranks(units_this_rank, device)
    slowest = max_over_ranks(seconds_this_rank, device)
    return total / slowest if slowest > 0 else 0.0


def band(H: int, rank: int, world: int):
    """Rows [y0, y1) of rank `rank` when H rows are split into `world` near-equal
    bands (the first bands are the shorter ones when H % world != 0)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    return rank * H // world, (rank + 1) * H // world


def exchange_halo(local, halo: int, rank: int, world: int, group=None):
    """This rank's band `local` ([rows, W], CPU or CUDA) with `halo` rows of the
    neighbouring bands above and below, exchanged point to point. Returns
    (extended band, rows added on top); the first and last bands get no halo on
    the image side. Every band must have at least `halo` rows."""
    import torch
    import torch.distributed as dist
    rows, W = local.shape
    if halo < 0:
        raise ValueError("halo must be >= 0")
    if world > 1 and halo > 0 and rows < halo:
        raise ValueError(f"band of {rows} rows is shorter than the halo of {halo}")
    if world == 1 or halo == 0:
        return local, 0
    up, down = rank > 0, rank < world - 1
    top = torch.empty((halo if up else 0, W), dtype=local.dtype, device=local.device)
    bot = torch.empty((halo if down else 0, W), dtype=local.dtype, device=local.device)
    reqs = []
    if up:
        reqs.append(dist.isend(local[:halo].contiguous(), rank - 1, group=group))
        reqs.append(dist.irecv(top, rank - 1, group=group))
    if down:
        reqs.append(dist.isend(local[rows - halo:].contiguous(), rank + 1, group=group))
        reqs.append(dist.irecv(bot, rank + 1, group=group))
    for q in reqs:
        q.wait()
    return torch.cat([top, local, bot]), top.shape[0]


def banded_forward(local, r: int, filt, rank: int, world: int, group=None):
    """Forward of one image split in row bands: `filt` maps an [h, W] image to
    its filtered [h, W] image (any implementation of the same filter); the
    result is this band's rows of the whole image's output."""
    ext, top = exchange_halo(local, r, rank, world, group)
    return filt(ext)[top:top + local.shape[0]]


def banded_gradient(local_f, local_g, r: int, grad_fn, rank: int, world: int, group=None):
    """dL/df on this band for L = sum(g * out) over the whole image, with f and
    g split in row bands. grad_fn(f, g) returns dL/df of sum(g * filter(f)) for
    an [h, W] frame. The frame is f with a 2r halo and g with an r halo, g being
    0 beyond it, so that every output the band's pixels feed is formed from its
    true window."""
    import torch
    ext_f, top2 = exchange_halo(local_f, 2 * r, rank, world, group)
    ext_g, top1 = exchange_halo(local_g, r, rank, world, group)
    g_frame = torch.zeros_like(ext_f, dtype=local_g.dtype)
    g_frame[top2 - top1:top2 - top1 + ext_g.shape[0]] = ext_g
    return grad_fn(ext_f, g_frame)[top2:top2 + local_f.shape[0]]


def banded_scalar_grad(local_f, local_g, r: int, scalar_fn, rank: int, world: int, group=None,
                       device=None) -> float:
    """dL/d(a scalar parameter of the filter, e.g. sigma_r) for L = sum(g * out)
    over the whole image: each rank differentiates only its own rows' outputs
    (f with an r halo, g on its own rows and 0 in the halo, so no output is
    counted twice), then one all-reduce sums the parts. scalar_fn(f, g) returns
    that derivative for an [h, W] frame."""
    import torch
    ext_f, top = exchange_halo(local_f, r, rank, world, group)
    g_frame = torch.zeros_like(ext_f, dtype=local_g.dtype)
    g_frame[top:top + local_g.shape[0]] = local_g
    return sum_over_ranks(float(scalar_fn(ext_f, g_frame)), device)
