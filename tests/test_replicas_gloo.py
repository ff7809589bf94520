"""The multi-GPU launch on CPU: two `gloo` ranks, each solving its own
replicas.  Checks that the shards are disjoint and rank-independent (a
problem's PRGD iterate does not depend on which rank computes it, the oracle
standing in for the GPU path), and that the timing reduction and the
whole-job rate follow the one-process-per-GPU contract."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as o
from paper_2501_13385_gb300 import workloads as w
from paper_2501_13385_gb300.replicas import max_over_ranks, replica_seeds, whole_job_rate

SHAPE = dict(n=[7, 6, 5], r=[1, 2, 2, 1], count=120)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _digest(seed):
    P = w.random_problem(seed, SHAPE["n"], SHAPE["r"], SHAPE["count"], init_rel=0.1)
    cores, _ = o.prgd_step(P.init, P.idx, P.y, P.n, P.r)
    return float(sum(np.sum(c * c) for c in cores))


def _rank(rank, world, port, batch, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = replica_seeds(rank, batch)
        digests = [_digest(s) for s in seeds]
        gathered = [None] * world
        dist.all_gather_object(gathered, (seeds, digests))
        slowest = max_over_ranks(10.0 + rank, world)
        q.put((rank, gathered, slowest))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_shard_without_exchange():
    world, batch = 2, 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, batch, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    g0 = out[0][1]
    assert g0 == out[1][1]
    seeds = [s for sh, _ in g0 for s in sh]
    assert len(set(seeds)) == world * batch and sorted(seeds) == list(range(world * batch))
    # every rank's iterate equals the one computed here, in one process
    for sh, dg in g0:
        for s, d in zip(sh, dg):
            assert d == _digest(s)
    # the slowest rank prices the job
    assert all(slow == 11.0 for _, _, slow in out)


def test_whole_job_rate_and_single_rank():
    assert max_over_ranks(3.5, 1) == 3.5
    # 2 ranks x 4 problems x 1000 entries x 10 steps in 20 ms
    assert whole_job_rate(2, 4, 1000, 10, 20.0) == pytest.approx(4.0e6)
    assert replica_seeds(0, 4) == [0, 1, 2, 3] and replica_seeds(1, 4) == [4, 5, 6, 7]
