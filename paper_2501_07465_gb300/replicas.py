"""Several GPUs, one process each: independent simulations only.

The method has no exchange step between independent simulations, so more
GPUs run more of them: either replicas of one workload (the throughput line
of the benchmark) or a share of a sweep of independent jobs.  Nothing here
moves simulation data between ranks; the only collectives are on the host's
bookkeeping (the slowest rank's time, the units all ranks processed).

Jobs are shared by a cost model (cells plus particles, times steps): largest
first, each to the rank with the least work so far.
"""
from __future__ import annotations

import heapq


def job_cost(wl, particles=None):
    """Work of one simulation job: (cells + particles) x steps.  particles
    defaults to cells x the species' particles per cell over the material."""
    g = wl["grid"]
    cells = 1
    for a in range(g["dims"]):
        cells *= g["n"][a]
    if particles is None:
        mat = int(wl["mask"].sum()) if wl.get("mask") is not None else cells
        particles = sum(sp["ppc"] * mat for sp in wl["species"])
    return (cells + particles) * wl["steps"]


def shard(costs, world):
    """Assign job indices to `world` ranks: largest cost first, each to the
    least-loaded rank (ties to the lower rank).  Returns one sorted index
    list per rank; every job appears exactly once."""
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def slowest(seconds, group=None, device=None):
    """The largest of every rank's time (the job is done when the slowest
    rank is); the rank's own value without a process group."""
    import torch
    import torch.distributed as dist
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def total(units, group=None, device=None):
    """Sum of every rank's processed units (particle-steps, simulations)."""
    import torch
    import torch.distributed as dist
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return float(units)
    t = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
