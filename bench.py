#!/usr/bin/env python
"""Benchmark of the encrypted 1:N match (Blind-Match, Sec. 3.3) on the GPU.

One step = one bm_match call: Algorithm 1 on the encrypted query, HE-C^3 over
every gallery group, compression, score ciphertexts resident on the device.
Default workload: ring 2^16 RNS-CKKS, 6,144 identities x 128-dim features in
parts of 16, one tiled query (the paper's Table 2 gallery size).  Features are
seeded synthetic L2-normalised Gaussians (paper_2408_06167_gb300.workload).

Prints one JSON line: matches/s with the query resident in HBM (`value`),
the same through host buffers (`e2e`), p50/p99 step latency, the roofline of
the dominant kernel class, and the CPU oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--part S] [--no-cpu-baseline] [--no-tune]
  python bench.py --sweep-part [--workload NAME]      N_in sweep vs the cost model
  python bench.py --serve [--auto-part] [--rate R]    serving mix
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted 1:N template matches/sec @128-dim, ring 2^16; p50/p99 query latency"
UNIT = "matches/s"
KEY_SEED, ENC_SEED, TEMPLATE_SEED = 3, 4, 6
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2, written between timed steps


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="face-128d-6144")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--write-traffic", default="",
                    help="write the DRAM-traffic record of --workload (its default forms) from this ncu CSV "
                         "(dram__bytes_read.sum, dram__bytes_write.sum per launch) and exit")
    ap.add_argument("--traffic-command", default="", help="--write-traffic: the ncu command the CSV came from")
    ap.add_argument("--traffic-plain", default="",
                    help="--write-traffic: the bench line of the same command without ncu (algorithmic bytes)")
    ap.add_argument("--traffic-stands-for", default="",
                    help="--write-traffic: comma-separated larger workloads the record is scaled to")
    ap.add_argument("--cpu-extrapolate", action="store_true",
                    help="the oracle on the batched configurations, sampled and scaled (a labelled extrapolation)")
    ap.add_argument("--cpu-sample-ids", type=int, default=32768,
                    help="--cpu-extrapolate: identities of the sampled gallery")
    ap.add_argument("--serve", action="store_true",
                    help="serving mix: Poisson arrivals against four resident galleries through bm_server_*")
    ap.add_argument("--rate", default="200", help="serving: arrivals per second (comma-separated: one line each)")
    ap.add_argument("--rate-too", action="store_true", help="serving: the Poisson rates as well as --closed-loop")
    ap.add_argument("--closed-loop", default="0",
                    help="serving: K clients, each submitting its next query when its previous result is back "
                         "(in place of Poisson arrivals)")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of arrivals")
    ap.add_argument("--executors", type=int, default=2)
    ap.add_argument("--serve-warmup", type=float, default=5.0,
                    help="serving: seconds of closed-loop requests before each measured window (plans built)")
    ap.add_argument("--max-batch", type=int, default=256)
    ap.add_argument("--part", type=int, default=0, help="part size (default: the workload's)")
    ap.add_argument("--shard", action="store_true",
                    help="with N ranks: the gallery split by whole packs over the ranks (strong scaling: each "
                         "rank matches the same queries against its shard); without: N replicas")
    ap.add_argument("--sweep-part", action="store_true",
                    help="N_in sweep: every part size of the workload, measured beside the cost model's prediction")
    ap.add_argument("--sweep-limit", type=float, default=4.0,
                    help="sweep: measure only part sizes predicted within this factor of the best")
    ap.add_argument("--auto-part", action="store_true",
                    help="serving: each gallery's part size chosen by the cost model (bm_choose_part)")
    ap.add_argument("--no-tune", action="store_true", help="skip the rotation kernel-shape tuner")
    ap.add_argument("--tune-dnum", action="store_true",
                    help="also report the cost model's choice of key-switching digits for the workload (the line "
                         "itself keeps the configuration's dnum)")
    ap.add_argument("--expansion", default="best",
                    choices=["doubling", "hoisted", "fused", "deferred", "best", "auto"],
                    help="form of Algorithm 1: the printed doubling order, the hoisted sum, the hoisted sum "
                         "with its key switches and rescale fused, or that with its division moved past HE-C^3's "
                         "products (best: deferred when the gallery has fewer groups than parts, else fused; "
                         "auto: serving picks per gallery by the cost model)")
    ap.add_argument("--tail", default="fused", choices=["printed", "hoisted", "double", "fused"],
                    help="Algorithm 2's rotate-and-sum and the compression: the printed sequential forms, "
                         "rounds of hoisted rotations, the same rounds with one ModDown per output "
                         "(double hoisting), or that with the rotate-and-sum's last round and the "
                         "compression in one round per pack (one ModDown a pack)")
    ap.add_argument("--gallery", default="plain", choices=["plain", "encrypted"],
                    help="gallery of plaintexts, or of ciphertexts enrolled on the server (Sec. 3.2)")
    ap.add_argument("--packing", default="complex", choices=["real", "complex"],
                    help="gallery slot packing (complex: a second identity in the imaginary parts)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def _oracle_match(wname, form, n_ids=None, tail="fused"):
    """The oracle's match of one query of the workload, in the forms the GPU line runs:
    Algorithm 1 hoisted with its key switches fused (form "fused"), or also with its
    division moved past HE-C^3's products ("deferred"); double-hoisted rotate-and-sum
    and compression (tail "fused": the rotate-and-sum's last round and the compression
    in one round per pack); complex packing.  n_ids < the workload's: the first n_ids
    identities (whole groups), for a sampled run."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from helpers_oracle import OracleMatch
    from paper_2408_06167_gb300 import workload as wl
    W = wl.WORKLOADS[wname]
    return W, OracleMatch(W.preset, W.dim, W.part, n_ids or W.n_ids, 1, complex_pack=True, hoisted=form,
                          hoisted_tail=True, double_hoisted=True, fused_compress=tail == "fused")


def _oracle_expand(om, ct, form):
    from oracle import schedule as sch
    return (sch.expand_query_ext if form == "deferred" else sch.expand_query_fused)(om.ev, ct, om.m, om.s)


def _oracle_groups(om, ct, parts, groups, form, rotsum=True):
    """HE-C^3 (the products over the parts and their division or rescale) and (rotsum)
    the rotate-and-sum for the given groups; returns (accs, mac_s, rotsum_s)."""
    from oracle import schedule as sch
    ev, accs, tm, tr = om.ev, [], 0.0, 0.0
    for g in groups:
        t0 = time.perf_counter()
        if form == "deferred":
            acc = ev.hec3_deferred(parts, om.gal[g], ct)
        else:
            acc = ev.mul_plain(parts[0], om.gal[g][0])
            for i in range(1, len(parts)):
                acc = ev.add(acc, ev.mul_plain(parts[i], om.gal[g][i]))
            acc = ev.rescale(acc)
        t1 = time.perf_counter()
        if rotsum:
            acc = sch.rotsum_hoisted(ev, acc, om.s, double=True)
        accs.append(acc)
        tm += t1 - t0
        tr += time.perf_counter() - t1
    return accs, tm, tr


_WORKER = {}


def _worker_init(wname, form, n_ids, tail):
    _WORKER["om"] = _oracle_match(wname, form, n_ids, tail)[1]


def _worker_groups(ct, parts, groups, form, rotsum):
    return _oracle_groups(_WORKER["om"], ct, parts, groups, form, rotsum)


class OracleRun:
    """The oracle's match of one query (keys, gallery and query prepared once), timed
    by stage -- expansion (Algorithm 1), HE-C^3 products, rotate-and-sum, compression
    (with tail "fused" the last two are one round per pack, timed as compression) --
    single-threaded, or with the groups spread over `cores` worker processes (each
    holding its own copy of the keys and gallery; the expanded query goes to them)."""

    def __init__(self, wname, form, cores=1, n_ids=None, tail="fused"):
        from oracle import schedule as sch
        self.form, self.cores, self.tail = form, cores, tail
        self.W, self.om = _oracle_match(wname, form, n_ids, tail)
        self.n_ids = n_ids or self.W.n_ids
        self.cts = self.om.encrypt(0)
        self.groups = len(self.om.gal)
        self.pool = None
        # the staged composition is the oracle's own match
        outs = self._run()[0]
        want, _ = self.om.match(self.cts)
        assert np.array_equal(self.om.ct_array(outs), want), "staged oracle run differs from its match"
        if cores > 1 and self.groups > 1:
            import concurrent.futures
            import multiprocessing
            self.pool = concurrent.futures.ProcessPoolExecutor(
                max_workers=min(cores, self.groups), mp_context=multiprocessing.get_context("spawn"),
                initializer=_worker_init, initargs=(wname, form, n_ids, tail))
            list(self.pool.map(_noop, range(min(cores, self.groups))))     # workers set up before timing
        self._sch = sch

    def _run(self):
        from oracle import schedule as sch
        ct = self.cts[0]
        t0 = time.perf_counter()
        parts = _oracle_expand(self.om, ct, self.form)
        t1 = time.perf_counter()
        rotsum = self.tail != "fused"
        if self.pool is None:
            accs, tm, tr = _oracle_groups(self.om, ct, parts, range(self.groups), self.form, rotsum)
        else:
            w = min(self.cores, self.groups)
            chunks = [list(range(k, self.groups, w)) for k in range(w)]
            res = list(self.pool.map(_worker_groups, [ct] * w, [parts] * w, chunks, [self.form] * w, [rotsum] * w))
            accs = [None] * self.groups
            for ch, (a, _, _) in zip(chunks, res):
                for g, x in zip(ch, a):
                    accs[g] = x
            tm, tr = max(r[1] for r in res), max(r[2] for r in res)
        t2 = time.perf_counter()
        if rotsum:
            packs = sch.compress(self.om.ev, accs, self.om.cmask, self.om.s, hoisted="double")
        else:
            packs = sch.rotsum_compress(self.om.ev, accs, self.om.cmask, self.om.s)
        t3 = time.perf_counter()
        return packs, {"expansion": t1 - t0, "hec3_products": tm, "rotate_and_sum": tr, "compression": t3 - t2,
                       "groups_wall": t2 - t1, "total": t3 - t0}

    def step(self):
        return self._run()[1]

    def close(self):
        if self.pool is not None:
            self.pool.shutdown()


def _noop(_):
    return 0


def oracle_form(wname):
    from paper_2408_06167_gb300 import workload as wl
    W = wl.WORKLOADS[wname]
    return resolve_expansion("best", W.n_ids, W.dim, W.part, True, (1 << (16 if W.preset == "ring16" else 12)) // 2)


def cpu_baseline(wname, tail="fused"):
    """The oracle on the host cores: one query of the workload in the GPU line's forms,
    by stage single-threaded, then with its groups spread over the host cores."""
    form = oracle_form(wname)
    cores = os.cpu_count() or 1
    single = OracleRun(wname, form, tail=tail)
    st = single.step()
    multi = OracleRun(wname, form, cores=cores, tail=tail) if single.groups > 1 and cores > 1 else None
    mt = multi.step() if multi else st
    if multi:
        multi.close()
    used = min(cores, single.groups) if multi else 1
    return {"value": single.n_ids / mt["total"], "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"one query x {single.n_ids} identities ({wname}), full match: Algorithm 1, then the "
                      f"{single.groups} groups' HE-C^3{'' if tail == 'fused' else ' and rotate-and-sum'} over "
                      f"{used} processes, then {'rotate-and-sum and ' if tail == 'fused' else ''}compression",
            "host_cpus": cores, "forms": f"{form} Algorithm 1, double-hoisted rotate-and-sum and compression"
                                        f"{' in one round per pack' if tail == 'fused' else ''}, "
                                        f"complex packing (the GPU line's)",
            "single_thread_value": single.n_ids / st["total"],
            "stages_s_single_thread": {k: st[k] for k in ("expansion", "hec3_products", "rotate_and_sum",
                                                          "compression", "total")},
            "stages_s": {k: mt[k] for k in ("expansion", "groups_wall", "compression", "total")}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    form = oracle_form(args.workload)
    cores = os.cpu_count() or 1
    run = OracleRun(args.workload, form, cores=cores, tail=args.tail)
    for _ in range(args.warmup):
        run.step()
    stages = [run.step() for _ in range(args.steps)]
    run.close()
    times = [x["total"] for x in stages]
    total = sum(times)
    value = args.steps * run.n_ids / total
    used = min(cores, run.groups) if run.pool else 1
    W = run.W
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": W.name, "ring": "2^16" if W.preset == "ring16" else W.preset,
                   "n_ids": W.n_ids, "dim": W.dim, "part": W.part, "queries_per_step": 1, "packing": "complex",
                   "expansion": form, "tail": args.tail, "gallery": "plain"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "host_cpus": cores,
                         "sample": f"each step: one query x {run.n_ids} identities, full oracle match in the GPU "
                                   f"line's forms, the {run.groups} groups over {used} processes"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "latency_ms": {"p50": 1e3 * statistics.median(times), "p99": 1e3 * max(times)},
        "stages_s": {k: statistics.median(x[k] for x in stages) for k in stages[0]},
    }
    print(json.dumps(line))


def run_cpu_extrapolate(args):
    """The oracle on the batched configurations, sampled and scaled (a labelled
    extrapolation, not a run of the whole configuration): per query, Algorithm 1 once;
    HE-C^3, rotate-and-sum and compression over the first `--cpu-sample-ids`
    identities (whole groups), scaled by the gallery's groups; x the queries of a
    batch.  Single-threaded and over the host cores."""
    out = {}
    cores = os.cpu_count() or 1
    for wname in ("finger-16d-65536-q64", "large-128d-1m-q256"):
        from paper_2408_06167_gb300 import workload as wl
        W = wl.WORKLOADS[wname]
        form = oracle_form(wname)
        n = min(W.n_ids, args.cpu_sample_ids)
        for c in (1, cores):
            run = OracleRun(wname, form, cores=c, n_ids=n, tail=args.tail)
            st = run.step()
            run.close()
            full_groups = -(-W.n_ids // (n // run.groups if run.groups else 1))
            scale = full_groups / run.groups
            per_query = st["expansion"] + scale * (st["groups_wall"] + st["compression"])
            out.setdefault(wname, {})[f"cores_{min(c, run.groups) if c > 1 else 1}"] = {
                "sampled_ids": n, "sampled_groups": run.groups, "scale_to_groups": full_groups,
                "stages_s_sample": st, "query_s_extrapolated": per_query,
                "batch_s_extrapolated": per_query * W.n_queries,
                "matches_per_s_extrapolated": W.n_ids / per_query, "forms": form}
    print(json.dumps({"cpu_extrapolation": out, "host_cpus": cores}))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Integer-multiply peak of the NTT passes: 152 SMs x 64 32-bit multiply results per
# clock per SM (the integer multiply-add rate of the SM, half its 128 FP32 lanes)
# x the maximum SM clock.  A 64-bit Shoup butterfly needs 16 such results: the
# high 64 bits of x*w' (four 32x32-bit products, low and high halves) and the low
# 64 bits of x*w and of floor(x*w'/2^64)*q (four each).
SM_COUNT = 152
INT32_MUL_PER_CLK_PER_SM = 64


def alu_peak_tops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        mhz = 2070.0
    return SM_COUNT * INT32_MUL_PER_CLK_PER_SM * mhz * 1e6 / 1e12


def measured_traffic(kernel_class, workload, config, alg_bytes_per_launch=None):
    """DRAM bytes per launch of a kernel class from the committed ncu record of the
    workload, or None when there is none for this schedule, or when the kernel sources
    have changed since the counters were taken.  A workload too large to capture under
    ncu is covered by the record of a smaller case of the same schedule that names it in
    `stands_for`: its DRAM bytes per launch scaled by the ratio of algorithmic bytes per
    launch (traffic taken to grow in proportion to the units a launch processes).
    Returns (bytes, source) or (None, None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            doc = json.load(f)
        own = [r for r in doc["records"] if r["workload"] == workload]
        proxy = [r for r in doc["records"] if workload in r.get("stands_for", [])]
        for rec in own + proxy:
            if any(rec["config"].get(k) != config.get(k) for k in rec["config"]):
                continue
            if _sources_sha1(rec["sources"]) != rec["sources_sha1"]:
                return None, None
            b = float(rec["dram_bytes_per_launch"][kernel_class])
            if rec["workload"] == workload:
                return b, "ncu capture of this workload"
            ref = rec.get("alg_bytes_per_launch", {}).get(kernel_class)
            if not ref or not alg_bytes_per_launch:
                return None, None
            return b * alg_bytes_per_launch / ref, ("ncu capture of %s scaled by algorithmic bytes per launch"
                                                    % rec["workload"])
    except (OSError, KeyError, ValueError, TypeError):
        pass
    return None, None


class L2Flush:
    """Between timed steps: a 512 MiB write (larger than the 129 MB L2), then a 512 MiB
    read of another buffer, which writes the dirty lines back before the step starts
    (so the next step neither finds its data in L2 nor pays for that write-back)."""

    def __init__(self):
        import torch
        self.w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        self.r = torch.ones(L2_FLUSH_BYTES // 8, dtype=torch.int64, device="cuda")

    def __call__(self):
        self.w.zero_()
        self.r.sum()


# kernel classes of the library's launches by kernel name (the classes the roofline
# can name as dominant; NTT passes also run inside other classes and are left out)
TRAFFIC_CLASSES = {"ks_ip": ("k_ks_f4s<", "k_ks_f4h<", "k_ks_f4<"),
                   "mac": ("k_mac<", "k_mac_ct<", "k_mac_circ<", "k_mac_circ_ntt<"),
                   "moddown": ("k_ks_f5<",), "modup": ("k_ks_f3<", "k_ks_f3r<", "k_ks_f0c<"),
                   "ks_combine": ("k_ks_f6<", "k_ks_f6u<")}
TRAFFIC_SOURCES = ["paper_2408_06167_gb300/csrc/kernels.cu", "paper_2408_06167_gb300/csrc/ks_fused.cu",
                   "paper_2408_06167_gb300/csrc/ntt_reg.cuh", "paper_2408_06167_gb300/csrc/bm_math.cuh"]


def _sources_sha1(srcs):
    import hashlib
    h = hashlib.sha1()
    for src in srcs:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def write_traffic_record(csv_path, workload, config, command, plain_json=None, stands_for=None):
    """Adds (or replaces) the record of `workload` in profiles/roofline_traffic.json from
    an ncu CSV with dram__bytes_read.sum and dram__bytes_write.sum per launch: DRAM
    bytes per launch of each kernel class, keyed by the workload, its schedule config
    and the SHA-1 of the kernel sources.  With `plain_json` (the bench line of the same
    command run without ncu) the record keeps the algorithmic bytes per launch of each
    class, so that it can stand for the larger workloads listed in `stands_for`."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    hi = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    h = rows[hi]
    ki, mi, ui, vi, ii = (h.index(x) for x in ("Kernel Name", "Metric Name", "Metric Unit", "Metric Value", "ID"))
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    per = {}
    for r in rows[hi + 1:]:
        if len(r) > vi and r[mi] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            d = per.setdefault(r[ii], {"k": r[ki], "b": 0.0})
            d["b"] += float(r[vi].replace(",", "")) * scale[r[ui]]
    cls = {}
    for d in per.values():
        kind = next((c for c, pats in TRAFFIC_CLASSES.items() if any(p in d["k"] for p in pats)), None)
        if kind:
            cls.setdefault(kind, []).append(d["b"])
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        doc = json.load(open(path))
        recs = [r for r in doc.get("records", []) if r.get("workload") != workload]
    except (OSError, ValueError):
        recs = []
    rec = {"workload": workload, "config": config,
           "dram_bytes_per_launch": {k: sum(v) / len(v) for k, v in sorted(cls.items())},
           "launches": {k: len(v) for k, v in sorted(cls.items())}, "command": command,
           "sources": TRAFFIC_SOURCES, "sources_sha1": _sources_sha1(TRAFFIC_SOURCES)}
    if plain_json:
        line = json.loads([x for x in open(plain_json) if x.startswith("{")][-1])
        rec["alg_bytes_per_launch"] = {k: v["alg_GB_per_step"] * 1e9 / v["launches"]
                                       for k, v in sorted(line["kernel_breakdown"].items()) if k in cls}
    if stands_for:
        rec["stands_for"] = list(stands_for)
    recs.append(rec)
    with open(path, "w") as f:
        json.dump({"records": recs}, f, indent=1)
        f.write("\n")


def across_ranks(total_s, work, world):
    """Whole-job rate: work summed over ranks / the slowest rank's time.  Returns (rate, max_time)."""
    if world == 1:
        return work / total_s, total_s
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([total_s], dtype=torch.float64, device=dev)
    w = torch.tensor([work], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(w.item()) / float(t.item()), float(t.item())


def percentile(xs, p):
    xs = sorted(xs)
    k = min(len(xs) - 1, max(0, int(round(p / 100.0 * (len(xs) - 1)))))
    return xs[k]


SERVE_GALLERIES = [("finger-1k", 1024, 16, 4), ("face-6k", 6144, 128, 16), ("finger-64k", 65536, 16, 4),
                   ("face-1m", 1 << 20, 128, 16)]
ARRIVAL_SEED = 5


def run_serving(args):
    """Poisson arrivals (seed 5) at --rate for --duration seconds, each query against a
    uniformly chosen resident gallery; requests are served by the continuous-batching
    server.  Reports p50/p99 submit-to-completion latency and matches/s, beside the same
    mix served one query per bm_match call (the plain unbatched form)."""
    import numpy as np
    import torch
    from paper_2408_06167_gb300 import binding as bm
    from paper_2408_06167_gb300 import workload as wl
    ctx = bm.bm_context_create("ring16", 0)
    wide = None if args.no_tune else bm.bm_autotune_keyswitch(ctx)
    ntt_shapes = None if args.no_tune else bm.bm_autotune_ntt(ctx)
    costs = bm.bm_measure_op_costs(ctx) if args.auto_part else None
    keys, gals, parts = {}, [], {}
    packing = bm.BM_PACK_COMPLEX if args.packing == "complex" else bm.BM_PACK_REAL
    expansions = {}
    for gi, (name, R, m, s) in enumerate(SERVE_GALLERIES):
        if args.expansion == "auto":
            forms = [(e, t) for e in ("doubling", "hoisted", "fused", "deferred") for t in ("printed", "hoisted", "double", "fused")]
        elif args.expansion == "best" and costs is not None:
            forms = [("fused", args.tail), ("deferred", args.tail)]   # the part size decides: the model picks
        else:
            forms = [(resolve_expansion(args.expansion, R, m, s, packing == bm.BM_PACK_COMPLEX, ctx.n // 2),
                      args.tail)]
        if costs is not None:
            # the cost model's part size (and, with --expansion auto, hoisted forms) for a
            # typical batch of 16 queries
            best = min(((bm.bm_choose_part("ring16", costs, R, m, 16, 32 << 30, packing | sched_flags(bm, *f)[1]), f)
                        for f in forms), key=lambda x: x[0][1])
            (s, _), form = best
        else:
            form = forms[0] if args.expansion != "auto" else ("doubling", "printed")
        if form[0] in ("fused", "deferred") and not 2 <= m // s <= 32:
            form = ("hoisted", form[1])   # the fused forms need 2..32 parts: the plain hoisted sum
        flags, _ = sched_flags(bm, *form)
        parts[name] = s
        expansions[name] = "+".join(x for x, on in (("hoisted-expansion", flags & 1), ("hoisted-rotsum", flags & 2),
                                                    ("hoisted-compression", flags & 4), ("double-hoisted", flags & 8),
                                                    ("fused-expansion", flags & 16), ("deferred-division", flags & 32))
                                    if on) or "printed"
        if (m, s) not in keys:
            keys[(m, s)] = bm.bm_keygen_ex(ctx, KEY_SEED, m, s, bm.BM_KEYS_HOISTED)
        feats = wl.gallery(R, m, seed=10 + gi)
        qs, _ = wl.queries(feats, 64, seed=20 + gi)
        sk, pk, ek = keys[(m, s)]
        cts = [bm.bm_encrypt_query(ctx, pk, q, m, s, bm.BM_QUERY_TILED, ENC_SEED, i) for i, q in enumerate(qs)]
        g = bm.bm_encode_gallery_packed(ctx, feats, m, s, packing)
        bm.bm_gallery_set_schedule(g, flags)
        gals.append(dict(name=name, R=R, g=g, ek=ek, cts=cts))
    # plain unbatched form: one query per bm_match, per gallery
    stream = torch.cuda.current_stream()
    single_ms = []
    for G in gals:
        bm.bm_match(ctx, G["ek"], G["g"], [G["cts"][0]], stream.cuda_stream)
        t = []
        for i in range(3):
            t0 = time.perf_counter()
            bm.bm_match(ctx, G["ek"], G["g"], [G["cts"][i]], stream.cuda_stream)
            t.append(time.perf_counter() - t0)
        single_ms.append(1e3 * min(t))
    mean_single_s = sum(single_ms) / len(single_ms) / 1e3        # uniform gallery choice
    unbatched_rate = 1.0 / mean_single_s
    unbatched_mps = sum(G["R"] for G in gals) / len(gals) * unbatched_rate
    closed = [int(k) for k in str(args.closed_loop).split(",") if int(k) > 0]
    settings = [("closed", k) for k in closed]
    if not closed or args.rate_too:
        settings += [("poisson", float(r)) for r in str(args.rate).split(",")]
    for kind, amount in settings:
        args.closed_loop_n = amount if kind == "closed" else 0
        args.rate_v = amount if kind == "poisson" else 0.0
        srv = bm.bm_server_create(ctx, 160 << 30, max_batch=args.max_batch, executors=args.executors)
        gids = [bm.bm_server_add_gallery(srv, G["g"], G["ek"]) for G in gals]
        import queue
        import threading
        errors = []
        lock = threading.Lock()

        def closed_loop(K, dur, choice):
            # K clients, each submitting its next query as soon as its previous result is back
            t_end = time.perf_counter() + dur

            def client(k):
                rng_k = np.random.default_rng([ARRIVAL_SEED, k, int(dur * 1000)])
                i = 0
                while time.perf_counter() < t_end:
                    gi = int(rng_k.integers(0, len(gals)))
                    G = gals[gi]
                    try:
                        t = bm.bm_server_submit(srv, gids[gi], G["cts"][(k + i) % len(G["cts"])])
                        bm.bm_server_wait(srv, t, 3600 * 1000)
                    except bm.BlindMatchError as e:
                        with lock:
                            errors.append(str(e))
                    with lock:
                        choice.append(gi)
                    i += 1

            threads = [threading.Thread(target=client, args=(k,)) for k in range(K)]
            for th in threads:
                th.start()
            for th in threads:
                th.join()

        # untimed warm-up: the plans the setting uses are built before the window opens
        if args.serve_warmup > 0:
            closed_loop(max(args.closed_loop_n, 16), args.serve_warmup, [])
            bm.bm_server_reset_stats(srv)
            errors.clear()
        start = time.perf_counter()
        sampler = ClockSampler(0)
        sampler.start()
        choice = []
        if args.closed_loop_n:
            closed_loop(args.closed_loop_n, args.duration, choice)
            n = len(choice)
        else:
            # Poisson arrivals; a waiter collects (and drops) each result as it completes
            rng = np.random.default_rng(ARRIVAL_SEED)
            n = int(args.rate_v * args.duration)
            arrivals = np.cumsum(rng.exponential(1.0 / args.rate_v, size=n))
            choice = list(rng.integers(0, len(gals), size=n))
            tickets = queue.Queue()

            def waiter():
                while True:
                    t = tickets.get()
                    if t is None:
                        return
                    try:
                        bm.bm_server_wait(srv, t, 3600 * 1000)
                    except bm.BlindMatchError as e:
                        errors.append(str(e))

            wt = threading.Thread(target=waiter)
            wt.start()
            for k in range(n):
                delay = start + arrivals[k] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                G = gals[choice[k]]
                tickets.put(bm.bm_server_submit(srv, gids[choice[k]], G["cts"][k % len(G["cts"])]))
            tickets.put(None)
            wt.join()
        wall = time.perf_counter() - start
        clocks = sampler.stop()
        st = bm.bm_server_stats(srv)
        matches = sum(gals[c]["R"] for c in choice)
        line = {
            "metric": METRIC, "value": st["matches_per_s"], "unit": UNIT, "n_gpus": 1, "steps": n, "warmup": 0,
            "ms_per_step": 1e3 * wall / n, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": "serving-mix", "ring": "2^16",
                       "arrivals": (f"closed loop, {args.closed_loop_n} clients" if args.closed_loop_n
                                    else f"Poisson, {args.rate_v:g} per s"),
                       "arrivals_per_s": n / wall,
                       "duration_s": args.duration, "galleries": [g[0] for g in SERVE_GALLERIES],
                       "executors": args.executors, "max_batch": args.max_batch, "parts": parts,
                       "part_choice": "cost model (bm_choose_part, 16 queries)" if costs is not None else "fixed",
                       "packing": args.packing, "expansion": expansions,
                       "ks_wide_batch": wide, "ntt_shapes": ntt_shapes},
            "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"]},
            "server": {k: st[k] for k in ("submitted", "completed", "failed", "batches", "mean_batch",
                                          "workspace_bytes")},
            "errors": errors[:3],
            "wall_s": wall, "matches": matches,
            "unbatched": {"single_query_ms": dict(zip([g[0] for g in SERVE_GALLERIES], single_ms)),
                          "sustainable_queries_per_s": unbatched_rate, "matches_per_s": unbatched_mps},
            "clocks": clocks,
        }
        print(json.dumps(line))
        del srv


def resolve_expansion(expansion, n_ids, dim, part, complex_pack, slots, encrypted=False):
    """'best': the deferred division when the gallery has fewer groups than parts (one
    division per group instead of one per part; plaintext galleries only), else the
    fused expansion; the plain hoisted sum outside the fused forms' 2..32 parts."""
    if expansion != "best":
        return expansion
    if not 2 <= dim // part <= 32:
        return "hoisted"
    groups = -(-n_ids // ((2 if complex_pack else 1) * (slots // part)))
    return "deferred" if groups < dim // part and not encrypted else "fused"


def roofline_of(kernel, ms, alg_bytes, alg_mul32, peak_gbs, peak_src, peak_tmul, traffic):
    """The dominant kernel class against both of its roofs -- algorithmic bytes / time
    against the measured copy bandwidth, algorithmic 32-bit multiplies / time against
    the derived integer-multiply peak -- with the binding one (the larger fraction)
    as the line's `bound`; both views are kept."""
    secs = ms / 1e3
    gbs = alg_bytes / secs / 1e9 if secs > 0 else 0.0
    hbm = {"bound": "hbm", "achieved": gbs, "peak": peak_gbs, "unit": "GB/s", "frac": gbs / peak_gbs,
           "peak_source": peak_src}
    views = {"hbm_view": {"achieved_gbs": gbs, "peak_gbs": peak_gbs, "frac": gbs / peak_gbs, "peak_source": peak_src}}
    best = hbm
    if alg_mul32 > 0:
        tmul = alg_mul32 / secs / 1e12 if secs > 0 else 0.0
        alu = {"bound": "alu", "achieved": tmul, "peak": peak_tmul, "unit": "Tmul32/s", "frac": tmul / peak_tmul,
               "peak_source": "derived: 152 SMs x 64 int32 mul/clk x max SM clock"}
        views["alu_view"] = {"achieved_tmul32": tmul, "peak_tmul32": peak_tmul, "frac": tmul / peak_tmul}
        if alu["frac"] >= hbm["frac"]:
            best = alu
    # neither roof near: the kernel's time is set by latency (launch ramp, dependent
    # memory round trips, barriers), which the fraction of the nearer roof states
    regime = "at a roof" if best["frac"] >= 0.5 else "latency-bound (below half of both roofs)"
    return {"kernel": kernel, **best, "regime": regime, "traffic": traffic, **views}


def sched_flags(bm, expansion, tail):
    """(gallery schedule flags, model layout flags) of the chosen forms."""
    if expansion == "best":       # resolved per gallery where its size is known
        expansion = "fused"
    f = bm.BM_SCHED_HOISTED_EXPANSION if expansion in ("hoisted", "fused", "deferred") else 0
    if expansion in ("fused", "deferred"):
        f |= bm.BM_SCHED_FUSED_EXPANSION
    if expansion == "deferred":
        f |= bm.BM_SCHED_DEFERRED_DIVISION
    if tail in ("hoisted", "double", "fused"):
        f |= bm.BM_SCHED_HOISTED_ROTSUM | bm.BM_SCHED_HOISTED_COMPRESSION
    if tail in ("double", "fused"):
        f |= bm.BM_SCHED_DOUBLE_HOISTED
    if tail == "fused":
        f |= bm.BM_SCHED_FUSED_COMPRESSION
    lay = ((bm.BM_LAYOUT_HOISTED if f & 1 else 0) | (bm.BM_LAYOUT_HOISTED_ROTSUM if f & 2 else 0)
           | (bm.BM_LAYOUT_HOISTED_COMPRESSION if f & 4 else 0) | (bm.BM_LAYOUT_DOUBLE_HOISTED if f & 8 else 0)
           | (bm.BM_LAYOUT_FUSED_EXPANSION if f & 16 else 0) | (bm.BM_LAYOUT_DEFERRED_DIVISION if f & 32 else 0)
           | (bm.BM_LAYOUT_FUSED_COMPRESSION if f & 64 else 0))
    return f, lay


def run_sweep(args):
    """Sec. 4 on this GPU: the match of the workload at every part size (N_in =
    dim / part), each measured (CUDA events, L2 flushed between steps) beside
    the time the cost model predicts from per-launch times measured on the same
    GPU, and the model's choice (bm_choose_part).  Part sizes whose plan does not
    fit in 80% of free device memory, or predicted slower than --sweep-limit x
    the best prediction, are listed with their prediction only."""
    import torch
    from paper_2408_06167_gb300 import binding as bm
    from paper_2408_06167_gb300 import workload as wl
    W = wl.WORKLOADS[args.workload]
    ctx = bm.bm_context_create(W.preset, 0)
    wide = None if args.no_tune else bm.bm_autotune_keyswitch(ctx)
    ntt_shapes = None if args.no_tune else bm.bm_autotune_ntt(ctx)
    costs = bm.bm_measure_op_costs(ctx)
    budget = int(0.8 * torch.cuda.mem_get_info()[0])
    feats = wl.gallery(W.n_ids, W.dim)
    qs, _ = wl.queries(feats_all, W.n_queries)
    ref0 = wl.plaintext_scores(feats, qs[0])
    mode = bm.BM_QUERY_TILED if W.query_mode == "tiled" else bm.BM_QUERY_EXPANDED
    parts = [p for p in (128, 64, 32, 16, 8, 4, 2, 1) if p <= W.dim]
    packing = bm.BM_PACK_COMPLEX if args.packing == "complex" else bm.BM_PACK_REAL
    flags, lay = sched_flags(bm, args.expansion, args.tail)
    hoisted = flags != 0
    packing |= lay
    pred = {p: bm.bm_predict_match(W.preset, costs, W.n_ids, W.dim, p, W.n_queries, packing) for p in parts}
    fitting = [p for p in parts if pred[p][1] <= budget]
    best_pred = min(pred[p][0] for p in fitting)
    model_part, _ = bm.bm_choose_part(W.preset, costs, W.n_ids, W.dim, W.n_queries, budget, packing)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    flush = L2Flush()
    sampler = ClockSampler(0)
    sampler.start()
    rows = []
    for p in parts:
        ops, nbytes = bm.bm_plan_estimate(W.preset, W.n_ids, W.dim, p, W.n_queries, packing)
        rot = {}
        for o in ops:
            if o["op"] == "rotate":
                rot[o["level"]] = rot.get(o["level"], 0) + o["count"] / W.n_queries
        row = {"part": p, "n_in": W.dim // p, "predicted_ms": pred[p][0], "plan_GB": nbytes / 1e9,
               "rotations_per_query": {f"level{k}": v for k, v in sorted(rot.items())}}
        if nbytes > budget:
            row["skipped"] = "plan larger than 80% of free device memory"
        elif pred[p][0] > args.sweep_limit * best_pred:
            row["skipped"] = f"predicted over {args.sweep_limit:g}x the best"
        if "skipped" in row:
            rows.append(row)
            continue
        sk, pk, ek = bm.bm_keygen_ex(ctx, KEY_SEED, W.dim, p, bm.BM_KEYS_HOISTED if hoisted else 0)
        gal = bm.bm_encode_gallery_packed(ctx, feats, W.dim, p, packing & 0xff)
        bm.bm_gallery_set_schedule(gal, flags)
        cts = [bm.bm_encrypt_query(ctx, pk, q, W.dim, p, mode, ENC_SEED, i) for i, q in enumerate(qs)]
        for ct in cts:
            bm.bm_ciphertext_upload(ct, sptr)
        r = bm.bm_match(ctx, ek, gal, cts, sptr)
        scores, rank1, _ = bm.bm_decrypt_scores(ctx, sk, r, 0, W.n_ids)
        del r
        steps = max(2, min(args.steps, int(2000.0 / max(pred[p][0], 1e-3))))
        for _ in range(max(1, min(args.warmup, steps))):
            bm.bm_match(ctx, ek, gal, cts, sptr)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush()
            ev[k][0].record(stream)
            r = bm.bm_match(ctx, ek, gal, cts, sptr)
            ev[k][1].record(stream)
            del r
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        row.update({"measured_ms": ms, "steps": steps, "matches_per_s": W.n_ids * W.n_queries / (ms / 1e3),
                    "predicted_over_measured": pred[p][0] / ms,
                    "max_abs_score_err_vs_fp64": float(abs(scores - ref0).max()),
                    "rank1_equal_fp64": int(rank1) == int(ref0.argmax())})
        rows.append(row)
        del gal, ek, sk, pk, cts
    clocks = sampler.stop()
    measured = [r for r in rows if "measured_ms" in r]
    best = min(measured, key=lambda r: r["measured_ms"])
    line = {
        "metric": METRIC, "value": best["matches_per_s"], "unit": UNIT, "n_gpus": 1, "steps": best["steps"],
        "warmup": args.warmup, "ms_per_step": best["measured_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": W.name, "mode": "part-sweep", "ring": "2^16" if W.preset == "ring16" else W.preset,
                   "n_ids": W.n_ids, "dim": W.dim, "queries_per_step": W.n_queries,
                   "l2": "flushed between steps (512 MiB write, then 512 MiB read)", "packing": args.packing,
                   "expansion": args.expansion, "tail": args.tail, "ks_wide_batch": wide, "ntt_shapes": ntt_shapes},
        "sweep": rows, "model_part": model_part, "measured_best_part": best["part"],
        "model_part_measured_ms": next((r.get("measured_ms") for r in rows if r["part"] == model_part), None),
        "clocks": clocks,
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.cpu_extrapolate:
        return run_cpu_extrapolate(args)
    if args.write_traffic:
        from paper_2408_06167_gb300 import workload as wl
        W = wl.WORKLOADS[args.workload]
        part = args.part or W.part
        exp = resolve_expansion(args.expansion, W.n_ids, W.dim, part, args.packing == "complex",
                                (1 << (16 if W.preset == "ring16" else 12)) // 2, args.gallery == "encrypted")
        cfg = {"part": part, "packing": args.packing, "gallery": args.gallery, "expansion": exp, "tail": args.tail}
        return write_traffic_record(args.write_traffic, W.name, cfg, args.traffic_command,
                                    args.traffic_plain or None,
                                    [w for w in args.traffic_stands_for.split(",") if w] or None)
    if args.serve:
        return run_serving(args)
    if args.sweep_part:
        return run_sweep(args)
    rank, world, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2408_06167_gb300 import binding as bm
    from paper_2408_06167_gb300 import workload as wl

    W = wl.WORKLOADS[args.workload]
    part = args.part or W.part
    ctx = bm.bm_context_create(W.preset, local)
    args.expansion = resolve_expansion(args.expansion, W.n_ids, W.dim, part, args.packing == "complex", ctx.n // 2,
                                       args.gallery == "encrypted")
    wide = None if args.no_tune else bm.bm_autotune_keyswitch(ctx)
    ntt_shapes = None if args.no_tune else bm.bm_autotune_ntt(ctx)
    packing = bm.BM_PACK_COMPLEX if args.packing == "complex" else bm.BM_PACK_REAL
    feats_all = wl.gallery(W.n_ids, W.dim)
    lo, hi = 0, W.n_ids
    if args.shard and world > 1:
        from paper_2408_06167_gb300 import shard
        lay = bm.bm_gallery_layout_packed(ctx, W.n_ids, W.dim, part, packing)
        lo, hi = shard.shard_range(W.n_ids, ctx.n // 2, part, packing == bm.BM_PACK_COMPLEX, bool(lay["compressed"]),
                                   rank, world)
        assert hi > lo, "more ranks than packs"
    feats = feats_all[lo:hi]
    n_local = hi - lo
    enroll = None
    if args.gallery == "encrypted":
        # the client encrypts every template (one GPU batch), the server enrolls them
        sk, pk, ek = bm.bm_keygen_ex(ctx, KEY_SEED, W.dim, part, bm.BM_KEYS_ENCRYPTED_GALLERY)
        t0 = time.perf_counter()
        temps = bm.bm_encrypt_batch(ctx, pk, feats, W.dim, part, bm.BM_QUERY_TEMPLATE, TEMPLATE_SEED, 0,
                                    bm.BM_ENC_KEEP_DEVICE)
        t1 = time.perf_counter()
        gal = bm.bm_enroll_encrypted(ctx, ek, temps, W.dim, part)
        t2 = time.perf_counter()
        del temps
        enroll = {"encrypt_templates_s": t1 - t0, "enroll_s": t2 - t1}
    else:
        flags, _ = sched_flags(bm, args.expansion if W.query_mode == "tiled" else "doubling", args.tail)
        sk, pk, ek = bm.bm_keygen_ex(ctx, KEY_SEED, W.dim, part, bm.BM_KEYS_HOISTED if flags else 0)
        gal = bm.bm_encode_gallery_packed(ctx, feats, W.dim, part, packing)
        bm.bm_gallery_set_schedule(gal, flags)
    qs, _ = wl.queries(feats_all, W.n_queries)
    mode = bm.BM_QUERY_TILED if W.query_mode == "tiled" else bm.BM_QUERY_EXPANDED
    cts = [bm.bm_encrypt_query(ctx, pk, q, W.dim, part, mode, ENC_SEED, i) for i, q in enumerate(qs)]
    host_cts = [bm.bm_encrypt_query(ctx, pk, q, W.dim, part, mode, ENC_SEED, i) for i, q in enumerate(qs)]
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    for ct in cts:
        bm.bm_ciphertext_upload(ct, sptr)
    flush = L2Flush()
    matches_per_step = n_local * W.n_queries

    # correctness guard on the benchmarked configuration: decrypted Rank-1 vs FP64
    r = bm.bm_match(ctx, ek, gal, cts, sptr)
    scores, rank1, _ = bm.bm_decrypt_scores(ctx, sk, r, 0, n_local)
    ref = wl.plaintext_scores(feats, qs[0])
    max_err = float(abs(scores - ref).max())
    assert max_err < 1e-5, max_err
    del r

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        r = bm.bm_match(ctx, ek, gal, cts, sptr)
        del r
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    bm.bm_profile_control(0, 1)
    # bm_match_async: every step enqueued without a host wait, so each event pair holds
    # the step's device work only (no host wake-up inside it)
    for k in range(args.steps):
        flush()
        ev[k][0].record(stream)
        r = bm.bm_match_async(ctx, ek, gal, cts, sptr)
        ev[k][1].record(stream)
        del r
    torch.cuda.synchronize()
    launches_timed = sum(bm.bm_profile_read(kind)[0] for kind in bm.KERNEL_KINDS)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, total_s = across_ranks(sum(step_ms) / 1e3, matches_per_step * args.steps, world)
    total_ms = total_s * 1e3

    # per-class device time over the same number of steps (event pair per launch)
    bm.bm_profile_control(1, 1)
    for k in range(args.steps):
        flush()
        r = bm.bm_match(ctx, ek, gal, cts, sptr)
        del r
    torch.cuda.synchronize()
    prof = {kind: bm.bm_profile_read(kind) for kind in bm.KERNEL_KINDS}
    bm.bm_profile_control(0, 1)
    dom = max(prof, key=lambda k: prof[k][1])
    n_l, ms_l, by_l, ops_l = prof[dom]
    peak_hbm, peak_src = load_peaks()
    traffic_cfg = {"part": part, "packing": args.packing, "gallery": args.gallery, "expansion": args.expansion,
                   "tail": args.tail}
    traffic, traffic_src = measured_traffic(dom, W.name, traffic_cfg, by_l / max(n_l, 1))
    roofline = roofline_of(dom, ms_l, by_l, ops_l, peak_hbm, peak_src, alu_peak_tops(), traffic)
    if traffic_src:
        roofline["traffic_source"] = traffic_src
    roofline.update({"launches_per_step": n_l / args.steps, "avg_launch_us": 1e3 * ms_l / max(n_l, 1),
                     "alg_bytes_per_launch": by_l / max(n_l, 1), "alg_mul32_per_launch": ops_l / max(n_l, 1),
                     "share_of_kernel_time": ms_l / max(sum(v[1] for v in prof.values()), 1e-12)})
    breakdown = {k: {"launches": v[0] // args.steps, "ms_per_step": v[1] / args.steps,
                     "alg_GB_per_step": v[2] / args.steps / 1e9} for k, v in prof.items() if v[0]}

    # end to end: host ciphertexts in (page-locked), score ciphertexts out to page-locked
    # host buffers, every step
    n_out_e = bm.bm_result_info(bm.bm_match(ctx, ek, gal, cts, sptr))[1]
    host_out = [torch.empty(n_out_e * 2 * ctx.n, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
                for _ in range(W.n_queries)]
    # (a) one step at a time: the match enqueued, then each query's score ciphertexts read
    # back (the export waits for the match itself), a host wait before the next step
    e2e_s = []
    for k in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = bm.bm_match_async(ctx, ek, gal, host_cts, sptr)
        for qi in range(W.n_queries):
            bm.bm_result_export(r, qi, host_out[qi])
        torch.cuda.synchronize()
        e2e_s.append(time.perf_counter() - t0)
        del r
    # (b) back to back, as a client with two requests in flight: step k is enqueued before
    # step k - 1's scores are read back, so the library's copy of step k's query (its own
    # copy stream, double-buffered) runs while step k - 1 matches; every step still copies
    # its query from page-locked host memory and its scores back to host memory
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prev = None
    for k in range(args.steps):
        r = bm.bm_match_async(ctx, ek, gal, host_cts, sptr)
        if prev is not None:
            for qi in range(W.n_queries):
                bm.bm_result_export(prev, qi, host_out[qi])
        prev = r
    for qi in range(W.n_queries):
        bm.bm_result_export(prev, qi, host_out[qi])
    torch.cuda.synchronize()
    e2e_total = time.perf_counter() - t0
    del prev
    r_ref = bm.bm_match(ctx, ek, gal, cts, sptr)
    for qi in range(W.n_queries):   # the last back-to-back step's scores: the same ciphertexts
        assert np.array_equal(host_out[qi], bm.bm_result_export(r_ref, qi).ravel()), "e2e scores differ"
    n_q, n_out, _ = bm.bm_result_info(r_ref)
    del r_ref
    ncts, lvl = bm.bm_ciphertext_info(host_cts[0])
    h2d = W.n_queries * ncts * 2 * (lvl + 1) * ctx.n * 8
    d2h = W.n_queries * n_out * 2 * ctx.n * 8
    e2e_value, _ = across_ranks(e2e_total, matches_per_step * args.steps, world)
    e2e_serial, _ = across_ranks(sum(e2e_s), matches_per_step * args.steps, world)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if args.shard else "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": W.name, "ring": "2^16" if W.preset == "ring16" else W.preset, "n_ids": W.n_ids,
                   "dim": W.dim, "part": part, "queries_per_step": W.n_queries,
                   "l2": "flushed between steps (512 MiB write, then 512 MiB read)",
                   "parallelism": ("gallery shards by pack" if args.shard else "replicas") if world > 1 else "single",
                   "packing": args.packing, "gallery": args.gallery, "expansion": args.expansion,
                   "tail": args.tail, "ks_wide_batch": wide, "ntt_shapes": ntt_shapes},
        "latency_ms": {"p50": percentile(step_ms, 50), "p99": percentile(step_ms, 99)},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps_in_flight": 2,
                "l2": "steps back to back, no flush between them: a step's distinct operands (%.2f GB by the "
                      "library's byte model) exceed the 129 MB L2" % sum(v["alg_GB_per_step"] for v in breakdown.values()),
                "one_step_at_a_time": {"value": e2e_serial, "latency_ms": {"p50": 1e3 * percentile(e2e_s, 50),
                                                                           "p99": 1e3 * percentile(e2e_s, 99)}}},
        "gpu_launches": launches_timed,
        "roofline": roofline,
        "kernel_breakdown": breakdown,
        "clocks": clocks,
        "check": {"max_abs_score_err_vs_fp64": max_err, "rank1": rank1, "rank1_fp64": int(ref.argmax())},
    }
    if enroll:
        line["enrollment"] = enroll
    if args.tune_dnum:
        flags_l = sched_flags(bm, args.expansion, args.tail)[1] | packing
        d, ms = bm.bm_choose_dnum(W.preset, W.n_ids, W.dim, part, W.n_queries, flags_l, local)
        line["dnum_model"] = {"chosen": d, "predicted_ms_by_dnum": {str(k + 1): v for k, v in enumerate(ms) if v > 0},
                              "line_dnum": ctx.dnum}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.tail)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
