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


@pytest.mark.parametrize("n_ids,dim,part,complex_pack,encrypted,want", [
    (6144, 128, 16, True, False, "deferred"),      # face: 2 groups < 8 parts
    (6144, 128, 16, False, False, "deferred"),     # 3 groups < 8 parts
    (6144, 128, 16, True, True, "fused"),          # encrypted gallery: no deferred division
    (65536, 16, 4, True, False, "fused"),          # finger: 4 groups, 4 parts
    (1 << 20, 128, 4, True, False, "fused"),       # 64 groups, 32 parts
    (1024, 16, 16, True, False, "hoisted"),        # one part: no fused forms
    (6144, 128, 2, True, False, "hoisted"),        # 64 parts: beyond the fused forms' 32
])
def test_best_expansion_form(n_ids, dim, part, complex_pack, encrypted, want):
    """bench.py's default form: the deferred division when the gallery has fewer
    groups than parts (plaintext galleries), else the fused expansion, and the
    plain hoisted sum outside 2..32 parts; explicit forms pass through."""
    import bench
    assert bench.resolve_expansion("best", n_ids, dim, part, complex_pack, 1 << 15, encrypted) == want
    assert bench.resolve_expansion("fused", n_ids, dim, part, complex_pack, 1 << 15, encrypted) == "fused"
