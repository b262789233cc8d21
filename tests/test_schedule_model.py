"""The library's schedule model (host only, no GPU): the launches bm_plan_estimate
lists are the operations of the oracle's schedule (Algorithm 1, HE-C^3,
compression) counted by its CountingEvaluator, per op and level; the plan's
bytes are its buffers; the predicted time is the sum the cost table gives each
launch; and the part-size choice is the argmin over the powers of two (Sec. 4's
choice of N_in by the cost model F)."""
import collections
import math

import numpy as np
import pytest

bm = pytest.importorskip("paper_2408_06167_gb300.binding")
from oracle import schedule as sch  # noqa: E402

PRESET = {"toy": (12, 2), "small4": (12, 4), "ring16": (16, 4)}   # log_n, n_q


def oracle_counts(preset, R, dim, part):
    """(op, level) -> count for one query, from the oracle's schedule."""
    log_n, n_q = PRESET[preset]
    L, slots = n_q - 1, 1 << (log_n - 1)
    tiled = L >= 3
    n_in = dim // part
    groups = sch.n_groups(R, part, slots)
    ev = sch.CountingEvaluator()
    q = [sch.SymCt(L)] if tiled else [sch.SymCt(L) for _ in range(n_in)]
    lg = L - 1 if tiled else L
    compress_mask = object() if lg >= 2 else None
    sch.match(ev, q, [[None] * n_in for _ in range(groups)], [None] * n_in, compress_mask, dim, part,
              expanded=not tiled)
    return ev.counts(), lg, tiled, groups


def library_counts(ops):
    c = collections.Counter()
    for o in ops:
        if o["op"] == "mac":
            c[("MAC", o["level"])] += o["queries"] * o["count"] * o["parts"]
        else:
            c[(o["op"], o["level"])] += o["count"]
    return c


CASES = [
    ("toy", 512, 16, 4, 1), ("toy", 700, 16, 4, 3), ("toy", 5000, 16, 2, 2),
    ("small4", 2500, 128, 16, 1), ("small4", 2500, 128, 16, 5), ("small4", 9000, 16, 4, 2),
    ("small4", 100, 8, 1, 1), ("small4", 1, 16, 16, 1), ("small4", 3000, 32, 32, 2),
    ("ring16", 6144, 128, 16, 1), ("ring16", 65536, 16, 4, 64), ("ring16", 1 << 20, 128, 16, 256),
    ("ring16", 1 << 20, 128, 4, 7), ("ring16", 1 << 20, 128, 1, 1), ("ring16", 1024, 16, 4, 3),
]


@pytest.mark.parametrize("preset,R,dim,part,Q", CASES)
def test_launches_are_the_oracle_schedule_operations(preset, R, dim, part, Q):
    ops, _ = bm.bm_plan_estimate(preset, R, dim, part, Q)
    lib = library_counts(ops)
    orc, lg, tiled, groups = oracle_counts(preset, R, dim, part)
    log_n, n_q = PRESET[preset]
    L = n_q - 1
    for (op, level), k in orc.items():
        if op == "Rot":
            assert lib[("rotate", level)] == Q * k, (op, level)
        elif op == "Res":
            assert lib[("rescale", level)] == Q * k, (op, level)
        elif op == "MulP" and level == lg:
            assert lib[("MAC", level)] == Q * k, (op, level)      # HE-C^3 products
        elif op == "MulP":
            assert lib[("mul_plain", level)] == Q * k, (op, level)   # Algorithm-1 and compression masks
    # nothing the oracle does not do
    kinds = {("rotate", "Rot"), ("rescale", "Res"), ("mul_plain", "MulP")}
    for (op, level), k in lib.items():
        if op in ("ntt", "intt", "copy", "MAC"):
            continue
        oname = dict(kinds)[op]
        assert orc.get((oname, level), 0) * Q == k, (op, level)
    # ingest and egress transforms: every limb of the queries, both limbs of every output
    n_in = dim // part
    n_out = -(-groups // part) if lg >= 2 else groups
    assert lib[("ntt", 0)] == Q * (1 if tiled else n_in) * 2 * (L + 1)
    assert lib[("intt", 0)] == Q * n_out * 2
    # rotations and rescales run in batches of at most 128 ciphertexts
    assert all(o["count"] <= 128 for o in ops if o["op"] in ("rotate", "rescale"))


def test_query_staging_buffers_up_to_256_mib():
    """Host queries are staged through two buffers of the plan's input size while that
    input is at most 256 MiB (64 top-level ring-2^16 queries): one query more drops
    both buffers, so the 65-query plan is smaller than the 64-query one by about two
    staging buffers (less the 65th query's own share)."""
    mib = 1 << 20
    per_q = 2 * 4 * (8 << 16)                       # one query at level 3: 2 x 4 limbs of 512 KiB
    b64 = bm.bm_plan_estimate("ring16", 65536, 16, 4, 64)[1]
    b65 = bm.bm_plan_estimate("ring16", 65536, 16, 4, 65)[1]
    b32 = bm.bm_plan_estimate("ring16", 65536, 16, 4, 32)[1]
    assert b64 - b65 > 2 * 64 * per_q - 200 * mib
    # 32 more queries: their own buffers plus twice their share of the staging
    assert b64 - b32 > 3 * 32 * per_q


def test_plan_bytes_are_its_buffers():
    # face gallery, one query: query ct (L = 3) and its two staging copies, Algorithm-1 outputs
    # at 3 and 2, accumulators at 2 and 1 for 3 groups, one score ct, key-switch scratch for 8
    # ciphertexts at level 2
    ops, nbytes = bm.bm_plan_estimate("ring16", 6144, 128, 16, 1)
    limb = 8 << 16
    buffers = (3 * 8 + 8 * 8 + 8 * 6 + 3 * 6 + 3 * 4 + 2) * limb
    ks_scratch = 8 * (2 * 3 + 2 * 5 + 2 * 5 + 2 * 3) * limb
    pointers = nbytes - buffers - ks_scratch
    assert 0 < pointers < 4096, pointers


def synthetic_costs(a, b):
    """t = a[op] + b[op][level] * units at every sample point."""
    units = np.array([[(8.0 if op == bm.OPS["mac"] else 1.0) * (1 << k) for k in range(bm.BM_COST_POINTS)]
                      for op in range(bm.BM_OP_KINDS)])
    t = np.zeros((bm.BM_OP_KINDS, bm.BM_MAX_Q, bm.BM_COST_POINTS))
    for op in range(bm.BM_OP_KINDS):
        for lv in range(bm.BM_MAX_Q):
            t[op, lv] = a[op] + b[op][lv] * units[op]
    return bm.bm_op_costs.from_arrays(units, t)


@pytest.mark.parametrize("preset,R,dim,part,Q", CASES[:12])
def test_prediction_is_the_sum_over_launches(preset, R, dim, part, Q):
    rng = np.random.default_rng(R + dim + part + Q)
    b = rng.uniform(0.5, 5.0, size=(bm.BM_OP_KINDS, bm.BM_MAX_Q))
    # per-unit costs only: the prediction is units x cost summed over the oracle's operations
    costs = synthetic_costs(np.zeros(bm.BM_OP_KINDS), b)
    ms, _ = bm.bm_predict_match(preset, costs, R, dim, part, Q)
    orc, lg, tiled, groups = oracle_counts(preset, R, dim, part)
    L = PRESET[preset][1] - 1
    n_in = dim // part
    want = 0.0
    for (op, level), k in orc.items():
        if op == "Rot":
            want += b[bm.OPS["rotate"], level] * Q * k
        elif op == "Res":
            want += b[bm.OPS["rescale"], level] * Q * k
        elif op == "MulP" and level != lg:
            want += b[bm.OPS["mul_plain"], level] * Q * k
    # HE-C^3 products, per launch (one per chunk of groups): one gallery read serves 4
    # queries, units = ceil(Q/4) x groups x parts, and below the first sample point
    # (8 units) a launch costs the first point's time
    ops, _ = bm.bm_plan_estimate(preset, R, dim, part, Q)
    macs = [o for o in ops if o["op"] == "mac"]
    assert sum(o["count"] for o in macs) == groups
    for o in macs:
        want += b[bm.OPS["mac"], lg] * max(8, math.ceil(Q / 4) * o["count"] * n_in)
    n_out = -(-groups // part) if lg >= 2 else groups
    want += b[bm.OPS["ntt"], 0] * Q * (1 if tiled else n_in) * 2 * (L + 1)
    want += b[bm.OPS["intt"], 0] * Q * n_out * 2
    if lg < 2:
        want += b[bm.OPS["copy"], 0] * Q * groups
    assert ms * 1000 == pytest.approx(want, rel=1e-9)
    # a fixed cost per launch only: the prediction counts the launches
    a = rng.uniform(1.0, 3.0, size=bm.BM_OP_KINDS)
    costs = synthetic_costs(a, np.zeros((bm.BM_OP_KINDS, bm.BM_MAX_Q)))
    ms, _ = bm.bm_predict_match(preset, costs, R, dim, part, Q)
    assert ms * 1000 == pytest.approx(sum(a[bm.OPS[o["op"]]] for o in ops), rel=1e-9)


def test_interpolation_between_and_beyond_the_sample_points():
    # rotation launches of 1..128 ciphertexts (on and between the points) and a
    # mask-product launch of 160 (beyond the last point)
    units = np.array([[(1 << k) for k in range(bm.BM_COST_POINTS)]] * bm.BM_OP_KINDS, dtype=float)
    t = np.zeros((bm.BM_OP_KINDS, bm.BM_MAX_Q, bm.BM_COST_POINTS))
    t[bm.OPS["rotate"], 1] = [10, 11, 13, 17, 25, 41, 73, 137]     # 9 + units, but 10 at one
    costs = bm.bm_op_costs.from_arrays(units, t)
    # small4, one identity, dim = part = 2: 1 rotation at level 1 per query (a4), no compression
    # rotation (groups = 1 < 2 to pair); Q queries -> one launch of Q ciphertexts
    for Q, want in [(1, 10.0), (3, 12.0), (100, 109.0), (128, 137.0)]:
        ops, _ = bm.bm_plan_estimate("small4", 1, 2, 2, Q)
        rot = [o for o in ops if o["op"] == "rotate"]
        assert [(o["level"], o["count"]) for o in rot] == [(1, Q)]
        ms, _ = bm.bm_predict_match("small4", costs, 1, 2, 2, Q)
        assert ms * 1000 == pytest.approx(want)
    t = np.zeros((bm.BM_OP_KINDS, bm.BM_MAX_Q, bm.BM_COST_POINTS))
    t[bm.OPS["mul_plain"], 3] = [5, 6, 8, 12, 20, 36, 68, 132]     # 4 + units: 164 at 160
    costs = bm.bm_op_costs.from_arrays(units, t)
    ops, _ = bm.bm_plan_estimate("small4", 1, 16, 1, 10)        # Algorithm 1: 10 queries x 16 masks
    assert [(o["level"], o["count"]) for o in ops if o["op"] == "mul_plain"][0] == (3, 160)
    ms, _ = bm.bm_predict_match("small4", costs, 1, 16, 1, 10)
    compression = [o for o in ops if o["op"] == "mul_plain" and o["level"] != 3]
    assert all(o["level"] == 1 for o in compression)                # costs 0 at level 1
    assert ms * 1000 == pytest.approx(164.0)


@pytest.mark.parametrize("R,dim,Q", [(6144, 128, 1), (1 << 20, 128, 256), (65536, 16, 64), (1024, 16, 1)])
def test_choice_is_the_argmin_within_the_budget(R, dim, Q):
    rng = np.random.default_rng(7)
    b = rng.uniform(0.5, 5.0, size=(bm.BM_OP_KINDS, bm.BM_MAX_Q))
    b[bm.OPS["rotate"]] *= 40                                      # rotations dominate, as on the GPU
    costs = synthetic_costs(np.full(bm.BM_OP_KINDS, 2.0), b)
    parts = [p for p in (1, 2, 4, 8, 16, 32, 64, 128) if p <= dim]
    pred = {p: bm.bm_predict_match("ring16", costs, R, dim, p, Q) for p in parts}
    best = min(parts, key=lambda p: (pred[p][0], -p))
    part, ms = bm.bm_choose_part("ring16", costs, R, dim, Q)
    assert part == best and ms == pytest.approx(pred[best][0])
    # a budget just below the best plan's bytes excludes it
    budget = pred[best][1] - 1
    fits = [p for p in parts if pred[p][1] <= budget]
    if fits:
        part2, _ = bm.bm_choose_part("ring16", costs, R, dim, Q, budget)
        assert part2 == min(fits, key=lambda p: (pred[p][0], -p))
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_choose_part("ring16", costs, R, dim, Q, 1 << 20)
    assert e.value.status == 7


def test_large_gallery_trade_off_matches_sec4():
    # Sec. 4: more parts cost more expansion rotations (N_in log N_in) and fewer
    # per-group rotations (log s per group plus s - 1 per pack); at a million
    # identities the minimum moves far below parts of 16
    rot = {}
    for part in (1, 2, 4, 8, 16, 32, 64, 128):
        ops, _ = bm.bm_plan_estimate("ring16", 1 << 20, 128, part, 1)
        rot[part] = sum(o["count"] for o in ops if o["op"] == "rotate")
        n_in = 128 // part
        groups = (1 << 20) * part // (1 << 15)
        packs = -(-groups // part)
        s_log = int(math.log2(part))
        assert rot[part] == n_in * int(math.log2(n_in)) + groups * s_log + packs * (part - 1)
    assert min(rot, key=rot.get) == 2 and rot[4] < rot[16] / 4


def test_errors():
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_plan_estimate("ring16", 100, 128, 3, 1)
    assert e.value.status == 5
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_plan_estimate("ring16", 100, 128, 16, 0)
    assert e.value.status == 1


def test_model_counts_halve_with_complex_packing():
    # Algorithm 1 is per query; HE-C^3 rotations and compression are per group and pack
    ops_r, _ = bm.bm_plan_estimate("ring16", 1 << 20, 128, 16, 1)
    ops_c, _ = bm.bm_plan_estimate("ring16", 1 << 20, 128, 16, 1, packing=bm.BM_PACK_COMPLEX)
    def rot(ops, lv):
        return sum(o["count"] for o in ops if o["op"] == "rotate" and o["level"] == lv)
    assert rot(ops_c, 2) == rot(ops_r, 2) == 24
    assert rot(ops_c, 1) == 256 * 4 + 16 * 15 and rot(ops_r, 1) == 512 * 4 + 32 * 15


@pytest.mark.parametrize("preset,R,dim,part,Q", [("small4", 2500, 128, 16, 3), ("ring16", 1 << 20, 128, 4, 40),
                                                 ("ring16", 6144, 128, 32, 1), ("small4", 300, 16, 1, 2),
                                                 ("small4", 300, 16, 16, 2)])
def test_hoisted_launches_are_the_oracle_hoisted_schedule(preset, R, dim, part, Q):
    """Algorithm 1 in hoisted form: one basis extension per query, N_in - 1 rotations
    from it, N_in x N_in mask products per query, then the same HE-C^3 and compression."""
    ops, _ = bm.bm_plan_estimate(preset, R, dim, part, Q, packing=bm.BM_LAYOUT_HOISTED)
    log_n, n_q = PRESET[preset]
    L, slots = n_q - 1, 1 << (log_n - 1)
    n_in = dim // part
    ev = sch.CountingEvaluator()
    groups = sch.n_groups(R, part, slots)
    sch.match(ev, [sch.SymCt(L)], [[None] * n_in for _ in range(groups)], [None] * n_in, object(), dim, part,
              hoisted=True)
    orc = ev.counts()
    lib = library_counts(ops)
    assert lib[("modup", L)] == Q * orc.get(("ModUp", L), 0) == (Q if n_in > 1 else 0)
    assert lib[("rot_hoisted", L)] == Q * orc.get(("RotH", L), 0) == Q * (n_in - 1)
    circ = sum(o["queries"] * o["count"] * o["parts"] for o in ops if o["op"] == "mac_circ")
    assert circ == Q * n_in * n_in == Q * orc.get(("MulP", L), 0)
    assert lib[("rescale", L)] == Q * orc[("Res", L)] == Q * n_in
    assert lib[("rotate", L - 1)] == 0                     # no doubling rotations at the Algorithm-2 level
    for lv in range(L - 1):
        assert lib[("rotate", lv)] == Q * orc.get(("Rot", lv), 0)


@pytest.mark.parametrize("preset,R,dim,part,Q", [("small4", 2500, 128, 16, 3), ("ring16", 1 << 20, 128, 4, 40),
                                                 ("ring16", 6144, 128, 16, 1), ("small4", 3000, 32, 32, 2),
                                                 ("toy", 1500, 16, 4, 2)])
def test_every_hoisted_form_matches_the_oracle_counts(preset, R, dim, part, Q):
    kind = bm.BM_LAYOUT_HOISTED | bm.BM_LAYOUT_HOISTED_ROTSUM | bm.BM_LAYOUT_HOISTED_COMPRESSION
    ops, _ = bm.bm_plan_estimate(preset, R, dim, part, Q, packing=kind)
    log_n, n_q = PRESET[preset]
    L, slots = n_q - 1, 1 << (log_n - 1)
    tiled = L >= 3
    lg = L - 1 if tiled else L
    n_in = dim // part
    groups = sch.n_groups(R, part, slots)
    ev = sch.CountingEvaluator()
    q = [sch.SymCt(L)] if tiled else [sch.SymCt(L) for _ in range(n_in)]
    sch.match(ev, q, [[None] * n_in for _ in range(groups)], [None] * n_in, object() if lg >= 2 else None, dim, part,
              expanded=not tiled, hoisted=tiled, hoisted_rotsum=True, hoisted_compress=True)
    orc = ev.counts()
    lib = library_counts(ops)
    for lv in range(L + 1):
        assert lib[("modup", lv)] == Q * orc.get(("ModUp", lv), 0), lv
        assert lib[("rot_hoisted", lv)] == Q * orc.get(("RotH", lv), 0), lv
        assert lib[("rotate", lv)] == Q * orc.get(("Rot", lv), 0) == 0, lv
    # every rotated copy is summed into its target
    assert sum(o["count"] for o in ops if o["op"] == "accum") == sum(
        o["count"] for o in ops if o["op"] == "rot_hoisted" and o["level"] < lg)


@pytest.mark.parametrize("preset,R,dim,part,Q", [("small4", 2500, 128, 16, 3), ("ring16", 1 << 20, 128, 4, 40),
                                                 ("ring16", 6144, 128, 16, 1), ("small4", 3000, 32, 32, 2),
                                                 ("toy", 1500, 16, 4, 2)])
def test_double_hoisted_forms_match_the_oracle_counts(preset, R, dim, part, Q):
    """One ModDown per round output: the plan's key-switch products and ModDowns
    are the oracle's and no rotated copies are summed afterwards."""
    single = bm.BM_LAYOUT_HOISTED | bm.BM_LAYOUT_HOISTED_ROTSUM | bm.BM_LAYOUT_HOISTED_COMPRESSION
    ops, _ = bm.bm_plan_estimate(preset, R, dim, part, Q, packing=single | bm.BM_LAYOUT_DOUBLE_HOISTED)
    log_n, n_q = PRESET[preset]
    L, slots = n_q - 1, 1 << (log_n - 1)
    tiled = L >= 3
    lg = L - 1 if tiled else L
    n_in = dim // part
    groups = sch.n_groups(R, part, slots)
    ev = sch.CountingEvaluator()
    q = [sch.SymCt(L)] if tiled else [sch.SymCt(L) for _ in range(n_in)]
    sch.match(ev, q, [[None] * n_in for _ in range(groups)], [None] * n_in, object() if lg >= 2 else None, dim, part,
              expanded=not tiled, hoisted=tiled, hoisted_rotsum=True, hoisted_compress=True, double_hoisted=True)
    orc = ev.counts()
    lib = library_counts(ops)
    for lv in range(L + 1):
        assert lib[("modup", lv)] == Q * orc.get(("ModUp", lv), 0), lv
        assert lib[("ip_sum", lv)] == Q * orc.get(("IPH", lv), 0), lv
        assert lib[("moddown", lv)] == Q * orc.get(("ModDown", lv), 0), lv
        assert lib[("rotate", lv)] == 0, lv
        if lv < lg:
            assert lib[("rot_hoisted", lv)] == 0, lv          # the tail's rotations are all summed
    assert not any(o["op"] == "accum" for o in ops)


@pytest.mark.parametrize("preset,R,dim,part,Q", [("small4", 2500, 128, 16, 3), ("ring16", 1 << 20, 128, 4, 40),
                                                 ("ring16", 6144, 128, 16, 1), ("small4", 3000, 32, 32, 2),
                                                 ("ring16", 65536, 16, 4, 64)])
def test_fused_compression_matches_the_oracle_counts(preset, R, dim, part, Q):
    """The rotate-and-sum's last round and the compression in one round per pack: one
    ModDown per pack at the compression level, one key-switch product per rotated term
    (the unrotated term of each group is none), no second round and no mask product."""
    kind = (bm.BM_LAYOUT_HOISTED | bm.BM_LAYOUT_HOISTED_ROTSUM | bm.BM_LAYOUT_HOISTED_COMPRESSION
            | bm.BM_LAYOUT_DOUBLE_HOISTED | bm.BM_LAYOUT_FUSED_COMPRESSION)
    ops, _ = bm.bm_plan_estimate(preset, R, dim, part, Q, packing=kind)
    log_n, n_q = PRESET[preset]
    L, slots = n_q - 1, 1 << (log_n - 1)
    lg, n_in = L - 1, dim // part
    groups = sch.n_groups(R, part, slots)
    packs = -(-groups // part)
    ev = sch.CountingEvaluator()
    sch.match(ev, [sch.SymCt(L)], [[None] * n_in for _ in range(groups)], [None] * n_in, object(), dim, part,
              hoisted=True, hoisted_rotsum=True, hoisted_compress=True, double_hoisted=True, fused_compress=True)
    orc = ev.counts()
    lib = library_counts(ops)
    lc = lg - 1
    b, g = sch.bsgs_split(part, double=True)
    count = g if g > 1 else b
    assert lib[("moddown", lc)] == Q * orc[("ModDown", lc)] == Q * (packs + (groups if g > 1 else 0))
    assert lib[("ip_sum", lc)] == Q * orc[("IPH", lc)]
    rotated = sum(1 for k in range(count) for o in range(part) if (b if g > 1 else 1) * k != o)
    full = groups // part
    assert orc[("IPH", lc)] >= full * rotated
    assert ("MulP", lc) not in orc
    assert lib[("mul_plain", lc)] == 0
    for lv in range(L + 1):
        assert lib[("modup", lv)] == Q * orc.get(("ModUp", lv), 0), lv


@pytest.mark.parametrize("preset,R,dim,part,Q", [("small4", 2500, 128, 16, 3), ("ring16", 6144, 128, 16, 1),
                                                 ("ring16", 1 << 20, 128, 4, 40), ("small4", 3000, 16, 4, 2)])
def test_deferred_division_matches_the_oracle_counts(preset, R, dim, part, Q):
    """The fused Algorithm 1 with its division moved past HE-C^3's products: no
    division per part, one division by q_(L-1) q_L P per (query, group) and no rescale
    at the HE-C^3 level; HE-C^3's products run on the L + 1 + alpha limbs of Q_L u P."""
    kind = (bm.BM_LAYOUT_HOISTED | bm.BM_LAYOUT_FUSED_EXPANSION | bm.BM_LAYOUT_DEFERRED_DIVISION
            | bm.BM_LAYOUT_HOISTED_ROTSUM | bm.BM_LAYOUT_HOISTED_COMPRESSION | bm.BM_LAYOUT_DOUBLE_HOISTED)
    ops, plan_bytes = bm.bm_plan_estimate(preset, R, dim, part, Q, packing=kind)
    _, fused_bytes = bm.bm_plan_estimate(preset, R, dim, part, Q, packing=kind & ~bm.BM_LAYOUT_DEFERRED_DIVISION)
    log_n, n_q = PRESET[preset]
    L, slots = n_q - 1, 1 << (log_n - 1)
    n_in = dim // part
    groups = sch.n_groups(R, part, slots)
    ev = sch.CountingEvaluator()
    sch.match(ev, [sch.SymCt(L)], [[None] * n_in for _ in range(groups)], [None] * n_in, object(), dim, part,
              hoisted="deferred", hoisted_rotsum=True, hoisted_compress=True, double_hoisted=True)
    orc = ev.counts()
    lib = library_counts(ops)
    assert lib[("modup", L)] == Q * orc[("ModUp", L)] == Q
    assert lib[("ip_sum", L)] == Q * orc[("IPH", L)] == Q * (n_in - 1)
    assert ("ModDownRes", L) not in orc
    assert lib[("moddown", L)] == Q * orc[("ModDownRes2", L)] == Q * groups
    alpha = bm.bm_params_preset(preset).n_p
    assert lib[("MAC", L + alpha)] == Q * orc[("MulPExt", L)] == Q * groups * n_in    # on the limbs of Q_L u P
    assert lib[("rescale", L)] == lib[("rescale", L - 1)] == 0
    assert ("Res", L - 1) not in orc
    # the rest of the schedule (rotate-and-sum, compression) is the fused form's
    assert lib[("ip_sum", L - 2)] == Q * orc[("IPH", L - 2)]
    assert plan_bytes > 0 and fused_bytes > 0


@pytest.mark.parametrize("preset,R,dim,part,Q", [("small4", 2500, 128, 16, 3), ("ring16", 6144, 128, 16, 1),
                                                 ("ring16", 10000, 128, 16, 2)])
def test_deferred_division_with_fused_compression_matches_the_oracle_counts(preset, R, dim, part, Q):
    """The bench's default forms on the host-only schedule (the estimate of a context
    with no device tables): the deferred division hands the fused tail its extension, so
    the tail's ModUp is recorded with the division's launches and the counts stay the
    oracle's -- one division per (query, group), one ModUp per group at the compression
    level, one ModDown per pack."""
    kind = (bm.BM_LAYOUT_HOISTED | bm.BM_LAYOUT_FUSED_EXPANSION | bm.BM_LAYOUT_DEFERRED_DIVISION
            | bm.BM_LAYOUT_HOISTED_ROTSUM | bm.BM_LAYOUT_HOISTED_COMPRESSION | bm.BM_LAYOUT_DOUBLE_HOISTED
            | bm.BM_LAYOUT_FUSED_COMPRESSION)
    ops, plan_bytes = bm.bm_plan_estimate(preset, R, dim, part, Q, packing=kind)
    log_n, n_q = PRESET[preset]
    L, slots = n_q - 1, 1 << (log_n - 1)
    n_in = dim // part
    groups = sch.n_groups(R, part, slots)
    packs = -(-groups // part)
    ev = sch.CountingEvaluator()
    sch.match(ev, [sch.SymCt(L)], [[None] * n_in for _ in range(groups)], [None] * n_in, object(), dim, part,
              hoisted="deferred", hoisted_rotsum=True, hoisted_compress=True, double_hoisted=True,
              fused_compress=True)
    orc = ev.counts()
    lib = library_counts(ops)
    assert lib[("moddown", L)] == Q * orc[("ModDownRes2", L)] == Q * groups
    assert lib[("modup", L - 2)] == Q * orc[("ModUp", L - 2)] == Q * groups
    assert lib[("moddown", L - 2)] == Q * orc[("ModDown", L - 2)] == Q * packs
    assert lib[("ip_sum", L - 2)] == Q * orc[("IPH", L - 2)]
    assert plan_bytes > 0


@pytest.mark.parametrize("preset,R,dim,part,Q", [("small4", 2500, 128, 16, 3), ("ring16", 6144, 128, 16, 1),
                                                 ("ring16", 1 << 20, 128, 4, 40), ("small4", 3000, 16, 4, 2)])
def test_fused_expansion_matches_the_oracle_counts(preset, R, dim, part, Q):
    """Algorithm 1 with ModDown and Rescale fused: one basis extension and N_in - 1
    key-switch products per query, N_in fused divisions, no rescale at the top level."""
    kind = (bm.BM_LAYOUT_HOISTED | bm.BM_LAYOUT_FUSED_EXPANSION | bm.BM_LAYOUT_HOISTED_ROTSUM
            | bm.BM_LAYOUT_HOISTED_COMPRESSION | bm.BM_LAYOUT_DOUBLE_HOISTED)
    ops, _ = bm.bm_plan_estimate(preset, R, dim, part, Q, packing=kind)
    log_n, n_q = PRESET[preset]
    L, slots = n_q - 1, 1 << (log_n - 1)
    n_in = dim // part
    groups = sch.n_groups(R, part, slots)
    ev = sch.CountingEvaluator()
    sch.match(ev, [sch.SymCt(L)], [[None] * n_in for _ in range(groups)], [None] * n_in, object(), dim, part,
              hoisted="fused", hoisted_rotsum=True, hoisted_compress=True, double_hoisted=True)
    orc = ev.counts()
    lib = library_counts(ops)
    assert lib[("modup", L)] == Q * orc[("ModUp", L)] == Q
    assert lib[("ip_sum", L)] == Q * orc[("IPH", L)] == Q * (n_in - 1)
    assert lib[("moddown", L)] == Q * orc[("ModDownRes", L)] == Q * n_in
    assert lib[("rescale", L)] == 0 and ("Res", L) not in orc
    assert lib[("rot_hoisted", L)] == 0


def test_products_on_more_limbs_than_measured_are_priced_by_their_limbs():
    """The deferred division's HE-C^3 products run on the L + 1 + alpha limbs of
    Q_L u P, above the levels the cost model measures: the model prices them at the
    top measured level's cost scaled by the limbs (a MAC's cost is proportional to
    them)."""
    preset, R, dim, part, Q = "ring16", 6144, 128, 16, 1
    L = PRESET[preset][1] - 1
    mac = bm.OPS["mac"]
    c = 0.25
    b = np.zeros((bm.BM_OP_KINDS, bm.BM_MAX_Q))
    b[mac, : L + 1] = c * np.arange(1, L + 2)           # proportional to the limbs; nothing above L
    costs = synthetic_costs(np.zeros(bm.BM_OP_KINDS), b)
    kind = (bm.BM_PACK_COMPLEX | bm.BM_LAYOUT_HOISTED | bm.BM_LAYOUT_FUSED_EXPANSION | bm.BM_LAYOUT_DEFERRED_DIVISION
            | bm.BM_LAYOUT_HOISTED_ROTSUM | bm.BM_LAYOUT_HOISTED_COMPRESSION | bm.BM_LAYOUT_DOUBLE_HOISTED)
    ops, _ = bm.bm_plan_estimate(preset, R, dim, part, Q, packing=kind)
    macs = [o for o in ops if o["op"] == "mac"]
    assert macs and all(o["level"] > L for o in macs)
    want = sum(c * (o["level"] + 1) * math.ceil(o["queries"] / 4) * o["count"] * o["parts"] for o in macs)
    ms, _ = bm.bm_predict_match(preset, costs, R, dim, part, Q, packing=kind)
    assert ms * 1000 == pytest.approx(want, rel=1e-9)
