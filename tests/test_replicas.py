"""Replica runs at N > 1 (independent runs, one per rank, no data-path
collective): the whole-job rate is the units all ranks processed over the
slowest rank's time.  Checked with world_size-2 gloo process groups on CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, units, seconds, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.replica_throughput(units[rank], seconds[rank], dist, "cpu")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("units,seconds", [([1000, 1000], [2.0, 4.0]), ([3e9, 1e9], [1.5, 0.5])])
def test_two_rank_replica_rate(units, seconds):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), units, seconds, out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    want = sum(units) / max(seconds)
    for r in (0, 1):
        value, tmax = res[r]
        assert value == pytest.approx(want, rel=1e-12)
        assert tmax == max(seconds)


def test_one_rank_is_plain_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(500, 2.0) == (250.0, 2.0)


def test_replicas_draw_different_seeds():
    sys.path.insert(0, ROOT)
    import bench
    seeds = {bench.make_workload(r).params.seed for r in range(4)}
    assert len(seeds) == 4
