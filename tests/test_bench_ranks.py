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


def test_roofline_bound_is_the_binding_roof():
    """The line's roofline takes the roof the dominant class is closer to: HBM for a
    class moving bytes at a larger fraction of the copy bandwidth than its multiplies
    reach of the integer peak, the ALU otherwise; both views are reported."""
    import bench
    # 3 launches of 1 ms: 8 GB and 10 T mul32 in total -> 2.67 TB/s, 3.33 T mul32/s
    r = bench.roofline_of("ks_ip", 3.0, 8e9, 10e12 / 1e3, 6669.5, "measured", 20.137, 68.6e6)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 68.6e6
    assert abs(r["frac"] - (8e9 / 3e-3 / 1e9) / 6669.5) < 1e-12
    assert r["alu_view"]["frac"] < r["frac"] == r["hbm_view"]["frac"]
    r = bench.roofline_of("moddown", 1.0, 1e9, 15e9, 6669.5, "measured", 20.137, None)
    assert r["bound"] == "alu" and r["unit"] == "Tmul32/s" and abs(r["frac"] - 15.0 / 20.137) < 1e-12
    r = bench.roofline_of("copy", 1.0, 5e9, 0, 6669.5, "measured", 20.137, None)
    assert r["bound"] == "hbm" and "alu_view" not in r


def test_traffic_record_own_proxy_and_stale(tmp_path, monkeypatch):
    """The line's `traffic`: the workload's own ncu record; for a workload only a
    smaller case's record stands for, that record's DRAM bytes per launch scaled by
    the ratio of algorithmic bytes per launch; nothing for another schedule, and
    nothing once the kernel sources differ from those the counters were taken on."""
    import json
    import bench
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES", ["k.cu"])
    csv_path = tmp_path / "l.csv"
    csv_path.write_text('"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
                        '"0","void k_ks_f4s<8>()","dram__bytes_read.sum","Mbyte","80"\n'
                        '"0","void k_ks_f4s<8>()","dram__bytes_write.sum","Mbyte","20"\n'
                        '"1","void k_ks_f4s<8>()","dram__bytes_read.sum","Mbyte","200"\n'
                        '"1","void k_ks_f4s<8>()","dram__bytes_write.sum","byte","0"\n'
                        '"2","void k_mac<1, 2>()","dram__bytes_read.sum","Gbyte","1"\n'
                        '"2","void k_mac<1, 2>()","dram__bytes_write.sum","byte","0"\n')
    plain = tmp_path / "plain.json"
    plain.write_text(json.dumps({"kernel_breakdown": {"ks_ip": {"launches": 2, "alg_GB_per_step": 0.3},
                                                      "mac": {"launches": 1, "alg_GB_per_step": 2.0}}}) + "\n")
    cfg = {"part": 16, "tail": "fused"}
    bench.write_traffic_record(str(csv_path), "small", cfg, "ncu ...", str(plain), ["big"])
    rec = json.load(open(tmp_path / "profiles" / "roofline_traffic.json"))["records"][0]
    assert rec["dram_bytes_per_launch"]["ks_ip"] == pytest.approx(150e6)
    assert rec["alg_bytes_per_launch"]["ks_ip"] == pytest.approx(150e6)
    assert bench.measured_traffic("ks_ip", "small", cfg) == (pytest.approx(150e6), "ncu capture of this workload")
    b, why = bench.measured_traffic("ks_ip", "big", cfg, 600e6)
    assert b == pytest.approx(600e6) and "scaled" in why
    assert bench.measured_traffic("mac", "big", cfg, 4e9)[0] == pytest.approx(2e9)
    assert bench.measured_traffic("ks_ip", "big", {"part": 4, "tail": "fused"}, 600e6) == (None, None)
    assert bench.measured_traffic("ks_ip", "other", cfg, 600e6) == (None, None)
    src.write_text("kernel v2")
    assert bench.measured_traffic("ks_ip", "small", cfg) == (None, None)
