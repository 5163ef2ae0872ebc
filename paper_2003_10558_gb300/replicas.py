"""Replicas across GPUs: the rasterizer has no exchange step (views and
tiles are independent), so N GPUs run N independent replicas.  This module
holds the host-side logic: which views a rank renders and how per-rank
throughput is combined (units summed, time = the slowest rank's).  It uses
torch.distributed only for these two host-level reductions; no data-path
collective exists."""
from __future__ import annotations


def shard_views(sizes, rank, world):
    """Assign views to ranks, balancing their pixel counts: greedy largest
    first onto the least-loaded rank, ties to the lower rank.  Returns the
    indices (ascending) of the views `rank` renders; every view goes to
    exactly one rank and the result is the same on every rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    owner = [0] * len(sizes)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += sizes[i]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def combine(units, seconds, group=None):
    """Whole-job throughput of replicas: (sum of units over ranks, max of the
    ranks' seconds).  Without an initialised process group, the local
    values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units, seconds
    dev = torch.device("cpu")
    if dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()), float(t.item())
