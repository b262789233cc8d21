"""Gallery sharding by pack (Sec. 3.4's clusters as ranks): the partition is whole
packs, and the score ciphertexts gathered from a 2-way split (gloo, two CPU ranks,
each running the oracle's match on its shard) equal the unsharded match bit for bit."""
import os
import socket

import numpy as np
import pytest

from paper_2408_06167_gb300 import shard

torch = pytest.importorskip("torch")

CASE = dict(name="small4", m=16, s=4, R=9000)     # complex packing: 4096 identities a pack, 3 packs


def test_shards_are_whole_packs_and_cover_the_gallery():
    slots = 2048
    for world in (1, 2, 3, 4, 5):
        got = [shard.shard_range(9000, slots, 4, True, True, r, world) for r in range(world)]
        assert got[0][0] == 0 and got[-1][1] == 9000
        for (a, b), (c, d) in zip(got, got[1:]):
            assert b == c                       # contiguous
        for a, b in got:
            assert a % 4096 == 0                # every shard starts at a pack
    # without compression the unit is a group (512 identities real, 1024 complex)
    assert shard.ids_per_unit(2048, 4, False, False) == 512
    assert shard.ids_per_unit(2048, 4, True, False) == 1024
    assert shard.ids_per_unit(2048, 4, True, True) == 4096


def _oracle_outputs(lo, hi, feats, query):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from helpers_oracle import OracleMatch
    om = OracleMatch(CASE["name"], CASE["m"], CASE["s"], hi - lo, 1, feats=feats[lo:hi], complex_pack=True,
                     hoisted="fused", hoisted_tail=True, double_hoisted=True)
    om.queries = query
    out, packed = om.match(om.encrypt(0))
    assert packed
    return out[None]                                 # [queries][packs][2][1][N]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2408_06167_gb300 import workload as wl
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    feats = wl.gallery(CASE["R"], CASE["m"])
    query, _ = wl.queries(feats, 1)
    lo, hi = shard.shard_range(CASE["R"], 2048, CASE["s"], True, True, rank, world)
    local = _oracle_outputs(lo, hi, feats, query) if hi > lo else None
    got = shard.gather_outputs(local, rank, world)
    if rank == 0:
        out["got"] = got
    dist.barrier()
    dist.destroy_process_group()


def test_gathered_shards_equal_the_unsharded_match():
    import torch.multiprocessing as mp
    from paper_2408_06167_gb300 import workload as wl
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    feats = wl.gallery(CASE["R"], CASE["m"])
    query, _ = wl.queries(feats, 1)
    want = _oracle_outputs(0, CASE["R"], feats, query)
    assert out["got"].shape == want.shape == (1, 3, 2, 1, 4096)
    assert np.array_equal(out["got"], want)
