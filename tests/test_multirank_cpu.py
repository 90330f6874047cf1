"""The N > 1 path of bench.py on CPU: two gloo ranks (the launch torchrun makes,
with the data path replaced by given durations).  Each rank solves its own
instance of the same shape (weak scaling, no collective on the data path); the
job's duration is the slowest rank's and its rate counts every rank's units;
the reference arm runs on rank 0 alone."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, durations, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        tmax, rate = bench.whole_job(durations[rank], 10.0, world, dist, "cpu")
        dist.barrier()
        q.put((rank, tmax, rate))
    finally:
        dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    durations = [1.5, 4.0]
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, durations, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, tmax, rate in got:
        assert tmax == 4.0                 # the slowest rank's time
        assert rate == 2 * 10.0 / 4.0      # both ranks' units in that time


def test_whole_job_single_rank():
    import bench
    assert bench.whole_job(2.0, 8.0, 1) == (2.0, 4.0)


def test_rank_systems_weak_scaling():
    import bench
    from paper_1609_00061_gb300 import workloads as W
    a, b = bench.rank_system(W, 0), bench.rank_system(W, 1)
    assert a.axes == b.axes and a.exposed == b.exposed
    assert [r.vars for r in a.rels] == [r.vars for r in b.rels]
    assert any(not np.array_equal(x.coeffs, y.coeffs) for x, y in zip(a.rels, b.rels))


def test_reference_arm_other_ranks_do_nothing():
    import bench

    class Args:
        steps, warmup = 1, 0

    assert bench.run_reference(Args, 1) is None
