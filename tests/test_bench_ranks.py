"""bench.py's multi-rank aggregation on CPU ranks (gloo, world size 2).

The match runs as independent replicas, one per GPU; the whole-job rate is
the work summed over ranks divided by the slowest rank's time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [2.0, 3.0]
    work = [600.0, 900.0]
    rate, tmax = bench.across_ranks(times[rank], work[rank], world)
    out[rank] = (rate, tmax)
    dist.barrier()
    dist.destroy_process_group()


def test_rate_is_total_work_over_slowest_rank():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in range(2):
        rate, tmax = out[rank]
        assert tmax == 3.0
        assert rate == pytest.approx((600.0 + 900.0) / 3.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.across_ranks(2.0, 10.0, 1) == (5.0, 2.0)
