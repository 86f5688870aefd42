"""The multi-rank path of bench.py on CPU: two gloo ranks, each timing its
own independent problem, combine into one whole-job rate over the slowest
rank (weak scaling, no collective on the data path)."""

import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_by_rank, units, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rate, ms = bench.whole_job_rate(units, world, ms_by_rank[rank], dist)
        out[rank] = (rate, ms)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_over_the_slowest_rank():
    world, units = 2, 435603 * 10
    ms_by_rank = [412.5, 433.0]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, ms_by_rank, units, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    expect = world * units / (max(ms_by_rank) * 1e-3)
    for r in range(world):
        rate, ms = out[r]
        assert ms == max(ms_by_rank)
        assert rate == pytest.approx(expect, rel=1e-15)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    rate, ms = bench.whole_job_rate(1000, 1, 2.0)
    assert ms == 2.0 and rate == pytest.approx(5e5)
