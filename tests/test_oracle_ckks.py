"""Pins of the oracle's CKKS layer and match schedule.

Encoding against brute-force evaluation of the polynomial at the slot roots,
decryption against the encoded message, rotation against a slot permutation
(Sec. 2's Rot), the Algorithm-1 and Algorithm-2 slot invariants, the final
scores against the FP64 plaintext cosine with its Rank-1, and the schedule's
operation counts against the paper's cost model F(N_in) (Sec. 4, Table 1).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import ckks
from oracle import schedule as sch
from paper_2408_06167_gb300 import workload as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_cost_model.json")


def test_encoding_evaluates_to_slots_at_the_5j_roots():
    ctx = ckks.Context(ckks.Params(8, (50,), (), dnum=1))
    rng = np.random.default_rng(0)
    z = rng.normal(size=ctx.slots) + 1j * rng.normal(size=ctx.slots)
    scale = 2.0 ** 40
    m = ctx.encode_int(z, scale).astype(np.float64) / scale
    n = ctx.n
    for j in range(ctx.slots):
        root = np.exp(1j * np.pi * pow(5, j, 2 * n) / n)
        val = np.polyval(m[::-1], root)
        assert abs(val - z[j]) < 1e-9, j


@pytest.mark.parametrize("name", ["toy", "ring16"])
def test_decode_inverts_encode(name):
    ctx = ckks.Context(name)
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, size=ctx.slots)
    c = ctx.encode_int(z, ctx.scale)
    assert np.abs(ctx.decode(c.tolist(), ctx.scale) - z).max() < 2.0 ** -30


@pytest.mark.parametrize("name", ["toy", "small4"])
def test_encrypt_decrypt_and_rotation_permutes_slots(name):
    ctx = ckks.Context(name)
    sk, pk, rks = ckks.keygen(ctx, 3, [1, 5, -1, -6])
    rng = np.random.default_rng(2)
    z = rng.uniform(-1, 1, size=ctx.slots)
    ct = ckks.encrypt(ctx, pk, ctx.encode(z, ctx.scale, ctx.L), 4, 0)
    assert np.abs(ckks.decrypt_decode(ctx, ct, sk) - z).max() < 1e-6
    ev = ckks.Evaluator(ctx, rks)
    for r in [1, 5, -1, -6]:
        d = ckks.decrypt_decode(ctx, ev.rotate(ct, r), sk)
        assert np.abs(d - np.roll(z, -r)).max() < 1e-6, r
    # a rotation at every level down to 0 (the toy's HE-C^3 runs at level 0)
    c = ct
    while c.level > 0:
        pt = ctx.encode(np.ones(ctx.slots), ctx.q[c.level], c.level)
        c = ev.rescale(ev.mul_plain(c, pt))
        d = ckks.decrypt_decode(ctx, ev.rotate(c, 1), sk)
        assert np.abs(d - np.roll(z, -1)).max() < 1e-6, c.level


def _setup(name, m, s, R, seed=3, extra_rots=()):
    ctx = ckks.Context(name)
    n_in = m // s
    rots = ([s << j for j in range(sch.log2i(n_in))] + [1 << t for t in range(sch.log2i(s))]
            + [-(1 << t) for t in range(sch.log2i(s))] + list(extra_rots))
    sk, pk, rks = ckks.keygen(ctx, seed, rots)
    return ctx, sk, pk, ckks.Evaluator(ctx, rks)


@pytest.mark.parametrize("m,s,R", [(128, 16, 2500), (16, 4, 3000)])
def test_match_invariants_and_scores_small4(m, s, R):
    ctx, sk, pk, ev = _setup("small4", m, s, R)
    S, L, n_in = ctx.slots, ctx.L, m // s
    feats = wl.gallery(R, m)
    qs, _ = wl.queries(feats, 1)
    q = qs[0]
    ct = ckks.encrypt(ctx, pk, ctx.encode(sch.tiled_query_slots(q, S), ctx.scale, L), 4, 0)
    masks = [ctx.encode(sch.alg1_mask_slots(m, s, i, S), ctx.q[L], L) for i in range(n_in)]
    cu = sch.expand_query(ev, ct, masks, m, s)
    # Algorithm 1 invariant: part i replicated at period s in every slot
    for i in range(n_in):
        d = ckks.decrypt_decode(ctx, cu[i], sk).real
        assert np.abs(d - np.array(sch.expanded_query_slots(q, s, i, S))).max() < 1e-6
    ng = sch.n_groups(R, s, S)
    gal = [[ctx.encode(sch.gallery_slots(feats, g, i, s, S), ctx.q[L - 1], L - 1) for i in range(n_in)]
           for g in range(ng)]
    accs = [sch.hec3(ev, cu, gal[g], s) for g in range(ng)]
    # Algorithm 2 invariant: slot u*s of group g holds <q, g_(gG+u)>
    G = S // s
    ref = wl.plaintext_scores(feats, q)
    d = ckks.decrypt_decode(ctx, accs[1], sk).real
    for u in range(0, min(G, R - G), 7):
        assert abs(d[u * s] - ref[G + u]) < 1e-6
    mm = ctx.encode(sch.compression_mask_slots(s, S), ctx.q[L - 2], L - 2)
    packs = sch.compress(ev, accs, mm, s)
    assert len(packs) == -(-ng // s) and packs[0].level == 0
    dec = [ckks.decrypt_decode(ctx, p, sk).real for p in packs]
    got = np.array([dec[o][slot] for o, slot, _ in (sch.identity_slot(i, s, S, True) for i in range(R))])
    assert np.abs(got - ref).max() < 1e-5
    top2 = np.sort(ref)[-2:]
    if top2[1] - top2[0] > 2e-5:
        assert got.argmax() == ref.argmax()
    # masked slots of the packs carry nothing: only slots u*s + r (r < groups in pack) are set
    assert np.abs(dec[-1][np.arange(S) % s >= ng - s * (len(packs) - 1)]).max() < 1e-6


def test_linear_compression_and_per_part_rescale_agree_with_default():
    m, s, R = 16, 4, 2100
    ctx, sk, pk, ev = _setup("small4", m, s, R, extra_rots=[-3])
    S, L, n_in = ctx.slots, ctx.L, m // s
    feats = wl.gallery(R, m)
    q = wl.queries(feats, 1)[0][0]
    ct = ckks.encrypt(ctx, pk, ctx.encode(sch.tiled_query_slots(q, S), ctx.scale, L), 4, 0)
    masks = [ctx.encode(sch.alg1_mask_slots(m, s, i, S), ctx.q[L], L) for i in range(n_in)]
    gal = [[ctx.encode(sch.gallery_slots(feats, g, i, s, S), ctx.q[L - 1], L - 1) for i in range(n_in)]
           for g in range(sch.n_groups(R, s, S))]
    mm = ctx.encode(sch.compression_mask_slots(s, S), ctx.q[L - 2], L - 2)
    ref = wl.plaintext_scores(feats, q)
    for kw in [dict(tree=False), dict(rescale_each_part=True)]:
        outs, packed = sch.match(ev, [ct], gal, masks, mm, m, s, **kw)
        dec = [ckks.decrypt_decode(ctx, p, sk).real for p in outs]
        got = np.array([dec[o][slot] for o, slot, _ in (sch.identity_slot(i, s, S, packed) for i in range(R))])
        assert np.abs(got - ref).max() < 1e-5, kw


@pytest.mark.parametrize("m,s,R", [(16, 4, 3000), (128, 16, 5000), (16, 16, 2100)])
def test_complex_slot_packing_scores(m, s, R):
    """Complex packing: identities u and G+u of a group share slot window u (real and
    imaginary parts); every score is still the FP64 cosine within 1e-5, the real and
    imaginary parts carry their own identities, and the groups halve."""
    ctx, sk, pk, ev = _setup("small4", m, s, R)
    S, L, n_in = ctx.slots, ctx.L, m // s
    feats = wl.gallery(R, m)
    q = wl.queries(feats, 1)[0][0]
    ct = ckks.encrypt(ctx, pk, ctx.encode(sch.tiled_query_slots(q, S), ctx.scale, L), 4, 0)
    masks = [ctx.encode(sch.alg1_mask_slots(m, s, i, S), ctx.q[L], L) for i in range(n_in)]
    ng = sch.n_groups(R, s, S, complex_pack=True)
    assert ng == -(-R // (2 * (S // s)))
    gal = [[ctx.encode(sch.gallery_slots_complex(feats, g, i, s, S), ctx.q[L - 1], L - 1) for i in range(n_in)]
           for g in range(ng)]
    # the plaintext of group 0, part 0 evaluates to A + iB at the slot roots
    z = ctx.decode(ctx.crt(gal[0][0].limbs, ctx.q[:L]), ctx.q[L - 1])
    G = S // s
    assert abs(z[0].real - feats[0][0]) < 1e-9 and abs(z[0].imag - feats[G][0]) < 1e-9
    mm = ctx.encode(sch.compression_mask_slots(s, S), ctx.q[L - 2], L - 2)
    outs, packed = sch.match(ev, [ct], gal, masks, mm, m, s)
    dec = [ckks.decrypt_decode(ctx, p, sk) for p in outs]
    got = np.array([dec[o][slot].imag if im else dec[o][slot].real
                    for o, slot, im in (sch.identity_slot(i, s, S, packed, complex_pack=True) for i in range(R))])
    ref = wl.plaintext_scores(feats, q)
    assert np.abs(got - ref).max() < 1e-5
    assert got.argmax() == ref.argmax() or np.sort(ref)[-1] - np.sort(ref)[-2] < 2e-5


def test_toy_expanded_queries_match_plaintext_cosine():
    """Toy ring 2^12 (one rescale prime): client-expanded query, HE-C^3 at level 1 -> 0."""
    m, s, R = 16, 4, 512
    ctx, sk, pk, ev = _setup("toy", m, s, R)
    S, n_in = ctx.slots, m // s
    feats = wl.gallery(R, m)
    qs, _ = wl.queries(feats, 8)
    gal = [[ctx.encode(sch.gallery_slots(feats, 0, i, s, S), ctx.q[1], 1) for i in range(n_in)]]
    for qi, q in enumerate(qs[:3]):
        cts = [ckks.encrypt(ctx, pk, ctx.encode(sch.expanded_query_slots(q, s, i, S), ctx.scale, 1), 4,
                            qi * 256 + i) for i in range(n_in)]
        outs, packed = sch.match(ev, cts, gal, None, None, m, s, expanded=True)
        assert not packed and outs[0].level == 0
        d = ckks.decrypt_decode(ctx, outs[0], sk).real
        got = d[np.arange(R) * s]
        ref = wl.plaintext_scores(feats, q)
        assert np.abs(got - ref).max() < 1e-5
        assert got.argmax() == ref.argmax()


# ------------------------------------------------------------- cost model


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("n_in", [2, 4, 8, 16, 32])
def test_schedule_op_counts_reproduce_cost_model(n_in):
    """The printed schedule's (op, level) counts weighted by Table 1 give F(N_in) of Sec. 4."""
    g = _golden()
    st = g["setting"]
    counts = sch.paper_literal_ops(st["n_slots"], st["m"], st["R_per_cluster"], n_in, st["level"])
    total = sum(c * g["table1_ms"][str(lvl)][op] for (op, lvl), c in counts.items())
    assert round(total, 2) == pytest.approx(g["F_ms"][str(n_in)], abs=1e-9)


def test_identities_per_ciphertext_example():
    ex = _golden()["vectors_per_ciphertext_example"]
    s = ex["m"] // ex["n_in"]
    assert ex["n_slots"] // s == ex["value"]        # (N * N_in) / m vectors per ciphertext


@pytest.fixture(scope="module")
def enrolled():
    """small4, 16-dim parts of 4: 12 encrypted templates placed by the server-side
    enrollment of Sec. 3.2 (mask, rescale, right rotation by powers of two, add)."""
    m, s, R = 16, 4, 12
    ctx = ckks.Context("small4")
    S, L, n_in = ctx.slots, ctx.L, m // s
    rots = ([s << j for j in range(sch.log2i(n_in))] + [1 << t for t in range(sch.log2i(s))]
            + [-(1 << t) for t in range(sch.log2i(s))] + sch.enroll_rotations(s, S))
    sk, pk, rks = ckks.keygen(ctx, 3, rots)
    ev = ckks.Evaluator(ctx, rks, ckks.keygen_relin(ctx, 3, sk))
    feats = wl.gallery(R, m)
    temps = [ckks.encrypt(ctx, pk, ctx.encode(sch.template_slots(f, S), ctx.scale, L), 6, k)
             for k, f in enumerate(feats)]
    emasks = [ctx.encode(sch.enroll_mask_slots(s, i, S), ctx.q[L], L) for i in range(n_in)]
    gal = sch.enroll(ev, temps, emasks, s, S)
    return dict(ctx=ctx, sk=sk, pk=pk, ev=ev, feats=feats, gal=gal, m=m, s=s, R=R)


def test_enrollment_places_each_template_in_its_window(enrolled):
    ctx, gal, s = enrolled["ctx"], enrolled["gal"], enrolled["s"]
    S, L = ctx.slots, ctx.L
    assert len(gal) == 1 and all(c.level == L - 1 and c.scale == ctx.scale for c in gal[0])
    for i, c in enumerate(gal[0]):
        d = ckks.decrypt_decode(ctx, c, enrolled["sk"]).real
        want = np.array(sch.gallery_slots(enrolled["feats"], 0, i, s, S))
        assert np.abs(d - want).max() < 1e-6, i


def test_encrypted_gallery_match_scores(enrolled):
    ctx, ev, s, m = enrolled["ctx"], enrolled["ev"], enrolled["s"], enrolled["m"]
    S, L, n_in = ctx.slots, ctx.L, m // s
    feats = enrolled["feats"]
    q = wl.queries(feats, 1)[0][0]
    ct = ckks.encrypt(ctx, enrolled["pk"], ctx.encode(sch.tiled_query_slots(q, S), ctx.scale, L), 4, 0)
    masks = [ctx.encode(sch.alg1_mask_slots(m, s, i, S), ctx.q[L], L) for i in range(n_in)]
    mm = ctx.encode(sch.compression_mask_slots(s, S), ctx.q[L - 2], L - 2)
    ref = wl.plaintext_scores(feats, q)
    for lazy in (True, False):
        cu = sch.expand_query(ev, ct, masks, m, s)
        accs = [sch.hec3(ev, cu, g, s, encrypted_gallery=True, lazy_relin=lazy) for g in enrolled["gal"]]
        outs = sch.compress(ev, accs, mm, s)
        # ct x ct at level L-1 then one rescale: the output scale is Delta^2 / q_(L-1)
        assert outs[0].level == 0 and outs[0].scale == pytest.approx(ctx.scale ** 2 / ctx.q[L - 1], rel=1e-15)
        dec = [ckks.decrypt_decode(ctx, o, enrolled["sk"]).real for o in outs]
        got = np.array([dec[o][slot] for o, slot, _ in (sch.identity_slot(i, s, S, True) for i in range(len(feats)))])
        assert np.abs(got - ref).max() < 1e-5, lazy


@pytest.mark.parametrize("m,s", [(16, 4), (128, 16), (16, 1)])
def test_hoisted_expansion_gives_algorithm1_outputs(m, s):
    """The hoisted form of Algorithm 1 (N_in - 1 rotations of the query sharing one
    basis extension, products with the rotated masks) decrypts to the same parts as
    the printed doubling form: part i replicated with period s in every slot."""
    ctx, sk, pk, ev = _setup("small4", m, s, 1, extra_rots=[j * s for j in range(1, m // s)])
    S, L, n_in = ctx.slots, ctx.L, m // s
    q = wl.queries(wl.gallery(3, m), 1)[0][0]
    ct = ckks.encrypt(ctx, pk, ctx.encode(sch.tiled_query_slots(q, S), ctx.scale, L), 4, 0)
    masks = [ctx.encode(sch.alg1_mask_slots(m, s, i, S), ctx.q[L], L) for i in range(n_in)]
    hoisted = sch.expand_query_hoisted(ev, ct, masks, m, s)
    for i in range(n_in):
        assert hoisted[i].level == L - 1 and hoisted[i].scale == ctx.scale
        d = ckks.decrypt_decode(ctx, hoisted[i], sk).real
        assert np.abs(d - np.array(sch.expanded_query_slots(q, s, i, S))).max() < 1e-6, i


def test_hoisted_rotation_permutes_slots():
    ctx = ckks.Context("small4")
    sk, pk, rks = ckks.keygen(ctx, 3, [1, 5, -3, 100])
    ev = ckks.Evaluator(ctx, rks)
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, ctx.slots)
    for level in (3, 2):
        ct = ckks.encrypt(ctx, pk, ctx.encode(z, ctx.scale, ctx.L), 5, 0)
        while ct.level > level:
            ct = ckks.Ciphertext(ct.c0[:-1].copy(), ct.c1[:-1].copy(), ct.level - 1, ct.scale)
        outs = ev.rotate_hoisted(ct, [1, 5, -3, 100])
        for r, o in zip([1, 5, -3, 100], outs):
            d = ckks.decrypt_decode(ctx, o, sk).real
            assert np.abs(d - np.roll(z, -r)).max() < 1e-6, (level, r)


@pytest.mark.parametrize("m,s,R", [(128, 16, 2500), (16, 4, 3000), (32, 32, 700), (16, 8, 3000)])
def test_hoisted_rotate_and_sum_and_compression_scores(m, s, R):
    """Algorithm 2's rotate-and-sum as two rounds of hoisted rotations and the
    linear compression with hoisted rotations give the FP64 scores."""
    b, g = sch.bsgs_split(s)
    extra = [k for k in range(1, b)] + [b * k for k in range(1, g)] + [-r for r in range(1, s)]
    ctx, sk, pk, ev = _setup("small4", m, s, R, extra_rots=extra)
    S, L, n_in = ctx.slots, ctx.L, m // s
    feats = wl.gallery(R, m)
    q = wl.queries(feats, 1)[0][0]
    ct = ckks.encrypt(ctx, pk, ctx.encode(sch.tiled_query_slots(q, S), ctx.scale, L), 4, 0)
    masks = [ctx.encode(sch.alg1_mask_slots(m, s, i, S), ctx.q[L], L) for i in range(n_in)]
    gal = [[ctx.encode(sch.gallery_slots(feats, gg, i, s, S), ctx.q[L - 1], L - 1) for i in range(n_in)]
           for gg in range(sch.n_groups(R, s, S))]
    mm = ctx.encode(sch.compression_mask_slots(s, S), ctx.q[L - 2], L - 2)
    ref = wl.plaintext_scores(feats, q)
    outs, packed = sch.match(ev, [ct], gal, masks, mm, m, s, hoisted_rotsum=True, hoisted_compress=True)
    dec = [ckks.decrypt_decode(ctx, o, sk).real for o in outs]
    got = np.array([dec[o][slot] for o, slot, _ in (sch.identity_slot(i, s, S, packed) for i in range(R))])
    assert np.abs(got - ref).max() < 1e-5


def _centred(x, q):
    x = x.astype(object) % q
    return np.where(x > q // 2, x - q, x).astype(np.int64)


def test_double_hoisted_single_term_is_the_hoisted_rotation():
    """With one rotated term the sum before ModDown is that term's inner product,
    so rotate_sum_hoisted(base, [(ct, r)]) is base + rotate_hoisted(ct, [r]) bit
    for bit; an unrotated term adds its ciphertext exactly."""
    ctx = ckks.Context("small4")
    sk, pk, rks = ckks.keygen(ctx, 3, [1, -5, 7])
    ev = ckks.Evaluator(ctx, rks)
    rng = np.random.default_rng(8)
    a = ckks.encrypt(ctx, pk, ctx.encode(rng.uniform(-1, 1, ctx.slots), ctx.scale, ctx.L), 5, 0)
    b = ckks.encrypt(ctx, pk, ctx.encode(rng.uniform(-1, 1, ctx.slots), ctx.scale, ctx.L), 5, 1)
    zero = ckks.Ciphertext(np.zeros_like(a.c0), np.zeros_like(a.c1), a.level, a.scale)
    for r in (1, -5, 7):
        want = ev.rotate_hoisted(a, [r])[0]
        got = ev.rotate_sum_hoisted(zero, [(a, r)])
        assert np.array_equal(got.c0, want.c0) and np.array_equal(got.c1, want.c1), r
        got_b = ev.rotate_sum_hoisted(b, [(a, r), (a, 0)])
        want_b = ev.add(ev.add(b, want), a)
        assert np.array_equal(got_b.c0, want_b.c0) and np.array_equal(got_b.c1, want_b.c1), r


@pytest.mark.parametrize("level", [3, 1])
def test_double_hoisted_sum_decrypts_and_differs_only_by_rounding(level):
    """Several terms over two ciphertexts: the message is base + the rotated
    messages, and the ciphertext differs from base + the single hoisted
    rotations by a small integer polynomial -- the same integer in every limb --
    bounded by the roundings of ModDown: floor(sum Y/P) - sum floor(Y/P) lies in
    [0, T) for T terms, and each fast base conversion adds e in [0, alpha)."""
    ctx = ckks.Context("small4")
    rots = [1, 2, 3, -4, 9]
    sk, pk, rks = ckks.keygen(ctx, 3, rots)
    ev = ckks.Evaluator(ctx, rks)
    rng = np.random.default_rng(9)
    zs = [rng.uniform(-1, 1, ctx.slots) for _ in range(3)]
    cts = []
    for k, z in enumerate(zs):
        ct = ckks.encrypt(ctx, pk, ctx.encode(z, ctx.scale, ctx.L), 5, k)
        cts.append(ckks.Ciphertext(ct.c0[:level + 1].copy(), ct.c1[:level + 1].copy(), level, ct.scale))
    base, a, b = cts
    terms = [(a, 1), (a, 2), (a, 3), (b, -4), (b, 9), (b, 0)]
    got = ev.rotate_sum_hoisted(base, terms)
    d = ckks.decrypt_decode(ctx, got, sk).real
    want_z = zs[0] + np.roll(zs[1], -1) + np.roll(zs[1], -2) + np.roll(zs[1], -3) + np.roll(zs[2], 4) \
        + np.roll(zs[2], -9) + zs[2]
    assert np.abs(d - want_z).max() < 1e-6
    single = base
    for ct, r in terms:
        single = ev.add(single, ev.rotate_hoisted(ct, [r])[0] if r else ct)
    T, alpha = sum(1 for _, r in terms if r), len(ctx.p)
    for comp in ("c0", "c1"):
        diffs = [_centred(getattr(got, comp)[j].astype(object) - getattr(single, comp)[j].astype(object), ctx.q[j])
                 for j in range(level + 1)]
        for j in range(1, level + 1):
            assert np.array_equal(diffs[j], diffs[0]), (comp, j)
        assert np.abs(diffs[0]).max() <= T * (alpha + 1) + alpha, comp
        assert np.abs(diffs[0]).max() > 0, comp          # the roundings saved change the bits


@pytest.mark.parametrize("m,s,R", [(128, 16, 2500), (16, 4, 3000), (16, 8, 3000), (64, 32, 2000)])
def test_double_hoisted_tail_scores(m, s, R):
    """Rotate-and-sum and linear compression with one ModDown per round output
    give the FP64 scores (a single round of rotations up to s = 16, baby and giant
    steps above)."""
    b, g = sch.bsgs_split(s, double=True)
    assert (b, g) == ((s, 1) if s <= 16 else sch.bsgs_split(s))
    extra = [k for k in range(1, b)] + [b * k for k in range(1, g)] + [-r for r in range(1, s)]
    ctx, sk, pk, ev = _setup("small4", m, s, R, extra_rots=extra)
    S, L, n_in = ctx.slots, ctx.L, m // s
    feats = wl.gallery(R, m)
    q = wl.queries(feats, 1)[0][0]
    ct = ckks.encrypt(ctx, pk, ctx.encode(sch.tiled_query_slots(q, S), ctx.scale, L), 4, 0)
    masks = [ctx.encode(sch.alg1_mask_slots(m, s, i, S), ctx.q[L], L) for i in range(n_in)]
    gal = [[ctx.encode(sch.gallery_slots(feats, gg, i, s, S), ctx.q[L - 1], L - 1) for i in range(n_in)]
           for gg in range(sch.n_groups(R, s, S))]
    mm = ctx.encode(sch.compression_mask_slots(s, S), ctx.q[L - 2], L - 2)
    ref = wl.plaintext_scores(feats, q)
    outs, packed = sch.match(ev, [ct], gal, masks, mm, m, s, hoisted_rotsum=True, hoisted_compress=True,
                             double_hoisted=True)
    dec = [ckks.decrypt_decode(ctx, o, sk).real for o in outs]
    got = np.array([dec[o][slot] for o, slot, _ in (sch.identity_slot(i, s, S, packed) for i in range(R))])
    assert np.abs(got - ref).max() < 1e-5


def test_rotated_plaintext_decodes_to_the_rotated_message():
    """The Galois image of a plaintext's coefficients decodes to its message rotated
    by r slots (left for r > 0, as Sec. 2's Rot), against numpy's roll of the encoded
    vector."""
    ctx = ckks.Context("small4")
    rng = np.random.default_rng(21)
    z = rng.uniform(-1, 1, ctx.slots)
    pt = ctx.encode(z, ctx.q[1], 1)
    for r in (1, -1, 3, -7, 0):
        rp = ckks.rotate_plaintext(ctx, pt, r)
        got = ctx.decode(ctx.crt(rp.limbs, ctx.q[:2]), pt.scale).real
        assert np.abs(got - np.roll(z, -r)).max() < 1e-6, r


def test_masked_rotate_sum_with_the_unit_plaintext_is_the_double_hoisted_sum():
    """With one group and the plaintext 1 (the constant polynomial) the masked sum is
    rotate_sum_hoisted on a zero base, bit for bit: the terms' products summed in Q_l u P
    and one ModDown, an unrotated term entering as P * ct (exact under ModDown)."""
    ctx = ckks.Context("small4")
    sk, pk, rks = ckks.keygen(ctx, 3, [1, 2, -3])
    ev = ckks.Evaluator(ctx, rks)
    rng = np.random.default_rng(22)
    lvl = 2
    ct = ckks.encrypt(ctx, pk, ctx.encode(rng.uniform(-1, 1, ctx.slots), ctx.scale, ctx.L), 5, 0)
    a = ckks.Ciphertext(ct.c0[:lvl + 1].copy(), ct.c1[:lvl + 1].copy(), lvl, ct.scale)
    one = ckks.Plaintext(np.stack([np.eye(1, ctx.n, 0, dtype=np.uint64)[0] for _ in range(lvl + 1)]), lvl, 1.0)
    zero = ckks.Ciphertext(np.zeros_like(a.c0), np.zeros_like(a.c1), lvl, a.scale)
    terms = [(a, 1), (a, 0), (a, 2), (a, -3)]
    got = ev.masked_rotate_sums([(one, terms)])
    want = ev.rotate_sum_hoisted(zero, terms)
    assert np.array_equal(got.c0, want.c0) and np.array_equal(got.c1, want.c1)


@pytest.mark.parametrize("m,s,R,complex_pack", [(128, 16, 2500, False), (16, 4, 3000, False),
                                                (64, 32, 2000, False), (16, 8, 1100, True)])
def test_fused_rotate_and_sum_and_compression_scores(m, s, R, complex_pack):
    """The rotate-and-sum's last round and the linear compression in one round per
    pack (the mask rotated by each group's offset, one ModDown a pack) give the FP64
    scores, and every pack decrypts to the message of the double-hoisted compression
    of the double-hoisted rotate-and-sum (ragged last packs, s > 16 with baby steps
    first, complex packing)."""
    b, g = sch.bsgs_split(s, double=True)
    extra = [k for k in range(1, b)] + [b * k for k in range(1, g)] + [-r for r in range(1, s)]
    extra += [b * k - o for k in range(g) for o in range(s)]
    ctx, sk, pk, ev = _setup("small4", m, s, R, extra_rots=sorted(set(r for r in extra if r)))
    S, L, n_in = ctx.slots, ctx.L, m // s
    feats = wl.gallery(R, m)
    q = wl.queries(feats, 1)[0][0]
    ct = ckks.encrypt(ctx, pk, ctx.encode(sch.tiled_query_slots(q, S), ctx.scale, L), 4, 0)
    masks = [ctx.encode(sch.alg1_mask_slots(m, s, i, S), ctx.q[L], L) for i in range(n_in)]
    slots_of = sch.gallery_slots_complex if complex_pack else sch.gallery_slots
    gal = [[ctx.encode(slots_of(feats, gg, i, s, S), ctx.q[L - 1], L - 1) for i in range(n_in)]
           for gg in range(sch.n_groups(R, s, S, complex_pack))]
    mm = ctx.encode(sch.compression_mask_slots(s, S), ctx.q[L - 2], L - 2)
    ref = wl.plaintext_scores(feats, q)
    kw = dict(hoisted_rotsum=True, hoisted_compress=True, double_hoisted=True)
    outs, packed = sch.match(ev, [ct], gal, masks, mm, m, s, fused_compress=True, **kw)
    assert packed and len(outs) == -(-len(gal) // s)
    dec = [ckks.decrypt_decode(ctx, o, sk) for o in outs]
    got = []
    for i in range(R):
        o, slot, im = sch.identity_slot(i, s, S, packed, complex_pack)
        got.append(dec[o][slot].imag if im else dec[o][slot].real)
    assert np.abs(np.array(got) - ref).max() < 1e-5
    plain, _ = sch.match(ev, [ct], gal, masks, mm, m, s, **kw)
    for o, p in zip(outs, plain):
        assert o.level == p.level and o.scale == p.scale
        assert np.abs(ckks.decrypt_decode(ctx, o, sk) - ckks.decrypt_decode(ctx, p, sk)).max() < 1e-6


def test_moddown_rescale_is_the_floor_up_to_the_conversion_error():
    """Big-integer pin of the fused ModDown + Rescale: for the integer E (CRT over
    Q_L u P) of each coefficient and S = q_L * P, the output is floor(E / S) - u
    with the same u in {0, ..., |S| - 1} on every target prime (the fast base
    conversion returns [E]_S + u S)."""
    ctx = ckks.Context("small4")
    L = ctx.L
    ext = ctx.ext_index(L)
    rng = np.random.default_rng(21)
    e = np.stack([np.stack([rng.integers(0, ctx.primes[gi], ctx.n, dtype=np.uint64) for gi in ext])
                  for _ in range(2)])
    c0, c1 = ckks.moddown_rescale(ctx, e, L)
    prims = [ctx.primes[gi] for gi in ext]
    S = ctx.q[L] * ctx.P
    spec = 1 + len(ctx.p)
    for comp, out in enumerate((c0, c1)):
        x = np.stack([ctx.intt(e[comp, jj], gi) for jj, gi in enumerate(ext)])
        Q = math.prod(prims)
        E = [v % Q for v in ctx.crt(x, prims)]
        fl = [v // S for v in E]
        for k in range(0, ctx.n, 97):
            us = {(fl[k] - int(out[j][k])) % ctx.q[j] for j in range(L)}
            assert len(us) == 1 and us.pop() < spec, (comp, k)


def test_moddown_rescale_two_primes_is_the_floor_up_to_the_conversion_error():
    """Big-integer pin of the division by S = q_(L-1) * q_L * P (two q-primes and P
    dropped): for the integer E (CRT over Q_L u P) of each coefficient the output on
    q_0..q_(L-2) is floor(E / S) - u, with the same u in {0, ..., |S| - 1} on every
    target prime."""
    ctx = ckks.Context("small4")
    L = ctx.L
    ext = ctx.ext_index(L)
    rng = np.random.default_rng(22)
    e = np.stack([np.stack([rng.integers(0, ctx.primes[gi], ctx.n, dtype=np.uint64) for gi in ext])
                  for _ in range(2)])
    c0, c1 = ckks.moddown_rescale(ctx, e, L, drop=2)
    assert c0.shape == (L - 1, ctx.n) and c1.shape == (L - 1, ctx.n)
    prims = [ctx.primes[gi] for gi in ext]
    S = ctx.q[L - 1] * ctx.q[L] * ctx.P
    spec = 2 + len(ctx.p)
    for comp, out in enumerate((c0, c1)):
        x = np.stack([ctx.intt(e[comp, jj], gi) for jj, gi in enumerate(ext)])
        E = [v % math.prod(prims) for v in ctx.crt(x, prims)]
        fl = [v // S for v in E]
        for k in range(0, ctx.n, 89):
            us = {(fl[k] - int(out[j][k])) % ctx.q[j] for j in range(L - 1)}
            assert len(us) == 1 and us.pop() < spec, (comp, k)


def test_extend_plaintext_reduces_the_same_integers():
    """A gallery plaintext at level L - 1 extended to Q_L u P: its own limbs come back
    unchanged (so the centred q_0 residues are its integer coefficients), and every
    limb, brought back to coefficient form, holds those integers mod its prime."""
    ctx = ckks.Context("small4")
    L, S, m, s = ctx.L, ctx.slots, 128, 16
    feats = wl.gallery(300, m)
    pt = ctx.encode(sch.gallery_slots_complex(feats, 0, 3, s, S), ctx.q[L - 1], L - 1)
    X = ckks.extend_plaintext(ctx, pt, L)
    ext = ctx.ext_index(L)
    assert len(X) == L + 1 + len(ctx.p)
    ints = [_centred(pt.limbs[0].astype(object), ctx.q[0])[k] for k in range(ctx.n)]
    assert max(abs(v) for v in ints) < ctx.q[0] // 4
    for jj, gi in enumerate(ext):
        coef = ctx.intt(X[jj], gi)
        if jj < L:
            assert np.array_equal(coef, pt.limbs[jj]), jj
        t = ctx.primes[gi]
        assert all(int(coef[k]) == ints[k] % t for k in range(0, ctx.n, 61)), jj


@pytest.mark.parametrize("m,s,R", [(16, 4, 3000), (128, 16, 2500)])
def test_deferred_division_gives_the_fused_hec3_outputs(m, s, R):
    """HE-C^3 on the undivided parts of the fused Algorithm 1, divided once by
    q_(L-1) q_L P, decrypts to the same group sums as HE-C^3 on the fused parts
    (level L - 2, the same scale), and differs from it by a small integer polynomial,
    the same in every limb, bounded by the roundings moved:
    3 * N_in * N * max|pt| / q_(L-1) + 4."""
    ctx, sk, pk, ev = _setup("small4", m, s, R, extra_rots=[j * s for j in range(1, m // s)])
    S, L, n_in = ctx.slots, ctx.L, m // s
    feats = wl.gallery(R, m)
    q = wl.queries(feats, 1)[0][0]
    ct = ckks.encrypt(ctx, pk, ctx.encode(sch.tiled_query_slots(q, S), ctx.scale, L), 4, 0)
    gal = [ctx.encode(sch.gallery_slots_complex(feats, 0, i, s, S), ctx.q[L - 1], L - 1) for i in range(n_in)]
    e_parts = sch.expand_query_ext(ev, ct, m, s)
    fused = sch.expand_query_fused(ev, ct, m, s)
    want = sch.hec3(ev, fused, gal, s)
    got = sch.hec3_deferred(ev, e_parts, gal, s, ct)
    assert got.level == want.level == L - 2 and got.scale == want.scale
    dw = ckks.decrypt_decode(ctx, want, sk)
    dg = ckks.decrypt_decode(ctx, got, sk)
    assert np.abs(dg - dw).max() < 1e-6
    pmax = max(int(np.abs(_centred(p.limbs[0].astype(object), ctx.q[0])).max()) for p in gal)
    bound = 3 * n_in * ctx.n * pmax // ctx.q[L - 1] + 4
    # before the rotate-and-sum: the products and the division alone
    a_w = ev.mul_plain(fused[0], gal[0])
    for i in range(1, n_in):
        a_w = ev.add(a_w, ev.mul_plain(fused[i], gal[i]))
    a_w = ev.rescale(a_w)
    a_g = ev.hec3_deferred(e_parts, gal, ct)
    for comp in ("c0", "c1"):
        diffs = [_centred(getattr(a_g, comp)[j].astype(object) - getattr(a_w, comp)[j].astype(object), ctx.q[j])
                 for j in range(L - 1)]
        for j in range(1, L - 1):
            assert np.array_equal(diffs[j], diffs[0]), (comp, j)
        assert np.abs(diffs[0]).max() <= bound, (comp, int(np.abs(diffs[0]).max()), bound)


@pytest.mark.parametrize("m,s", [(16, 4), (128, 16), (16, 1)])
def test_fused_expansion_gives_algorithm1_outputs(m, s):
    """Algorithm 1 with the key switches and the rescale fused decrypts to the same
    parts as the printed form, and differs from the hoisted form by a small integer
    polynomial -- the same in every limb -- bounded by the roundings moved:
    3 * N_in * N * max|mask| / q_L + 4."""
    ctx, sk, pk, ev = _setup("small4", m, s, 1, extra_rots=[j * s for j in range(1, m // s)])
    S, L, n_in = ctx.slots, ctx.L, m // s
    q = wl.queries(wl.gallery(3, m), 1)[0][0]
    ct = ckks.encrypt(ctx, pk, ctx.encode(sch.tiled_query_slots(q, S), ctx.scale, L), 4, 0)
    masks = [ctx.encode(sch.alg1_mask_slots(m, s, i, S), ctx.q[L], L) for i in range(n_in)]
    fused = sch.expand_query_fused(ev, ct, m, s)
    hoisted = sch.expand_query_hoisted(ev, ct, masks, m, s)
    mmax = max(int(np.abs(ctx.encode_int(sch.alg1_mask_slots(m, s, i, S), ctx.q[L])).max()) for i in range(n_in))
    bound = 3 * n_in * ctx.n * mmax // ctx.q[L] + 4
    for i in range(n_in):
        assert fused[i].level == L - 1 and fused[i].scale == ctx.scale
        d = ckks.decrypt_decode(ctx, fused[i], sk).real
        assert np.abs(d - np.array(sch.expanded_query_slots(q, s, i, S))).max() < 1e-6, i
        for comp in ("c0", "c1"):
            diffs = [_centred(getattr(fused[i], comp)[j].astype(object) - getattr(hoisted[i], comp)[j].astype(object),
                              ctx.q[j]) for j in range(L)]
            for j in range(1, L):
                assert np.array_equal(diffs[j], diffs[0]), (i, comp, j)
            assert np.abs(diffs[0]).max() <= bound, (i, comp, int(np.abs(diffs[0]).max()), bound)
