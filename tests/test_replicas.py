"""Several ranks, independent simulations: the job split and the host-side
reductions, on CPU with the gloo backend (world size 2)."""
import os
import socket

import numpy as np
import pytest

from paper_2501_07465_gb300 import inputs as I
from paper_2501_07465_gb300 import replicas as R


def test_shard_covers_every_job_once_and_balances():
    rng = np.random.default_rng(5)
    costs = list(rng.lognormal(10, 1, size=257))
    for world in (1, 2, 3, 8):
        parts = R.shard(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # largest-first greedy: no rank exceeds the mean by more than the largest job
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9


def test_job_cost_counts_cells_and_particles():
    wl = I.batch2d(count=3)[0]
    g = wl["grid"]
    cells = g["n"][0] * g["n"][1]
    mat = int(wl["mask"].sum())
    ppc = sum(sp["ppc"] for sp in wl["species"])
    assert R.job_cost(wl) == (cells + ppc * mat) * wl["steps"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [5.0, 1.0, 4.0, 2.0, 3.0, 3.0]
        mine = R.shard(costs, world)[rank]
        seconds = 1.0 + rank  # rank 1 is slower
        units = sum(costs[i] for i in mine)
        q.put((rank, mine, R.slowest(seconds), R.total(units)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_slowest_time_and_total_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (_, m0, t0, u0), (_, m1, t1, u1) = out
    assert sorted(m0 + m1) == list(range(6))
    assert not set(m0) & set(m1)
    assert t0 == t1 == 2.0
    assert u0 == u1 == 18.0


def test_without_a_process_group_the_values_are_the_ranks_own():
    assert R.slowest(1.5) == 1.5
    assert R.total(7) == 7.0
