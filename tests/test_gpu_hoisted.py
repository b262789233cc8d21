"""Algorithm 1 in hoisted form on the GPU against the oracle: the basis
extension of each query's c1 computed once, N_in - 1 rotations taken from it
(the Galois image of each extended limb is a permutation of its NTT slots),
the circulant mask products (up to 32 parts as a cyclic convolution by
transforms over the parts, beyond that the direct sum) and one rescale per part
-- bit-exact against the oracle's hoisted expansion, then the same HE-C^3 and
compression; end to end, the scores equal those of the printed (doubling) form
within the tolerance."""
import numpy as np
import pytest

from helpers_oracle import KEY_SEED, OracleMatch
from paper_2408_06167_gb300 import workload as wl

pytestmark = pytest.mark.gpu

bm = pytest.importorskip("paper_2408_06167_gb300.binding")

_CTX = {}


def gctx(name):
    if name not in _CTX:
        _CTX[name] = bm.bm_context_create(name)
    return _CTX[name]


@pytest.mark.parametrize("name,m,s,R,nq", [
    ("small4", 128, 16, 2500, 2),     # N_in = 8: 7 hoisted rotations per query
    ("small4", 16, 4, 3000, 3),       # N_in = 4, three queries in one chunk
    ("small4", 16, 1, 2100, 1),       # N_in = 16, part size 1
    ("small4", 16, 16, 100, 1),       # N_in = 1: no rotations, the query times its mask
    ("small4", 128, 4, 600, 1),       # N_in = 32: the largest convolution by transforms over the parts
    ("small4", 128, 2, 300, 1),       # N_in = 64: the direct circulant sum (masks in shared memory)
])
def test_hoisted_match_is_bit_exact(name, m, s, R, nq):
    c = gctx(name)
    om = OracleMatch(name, m, s, R, nq, hoisted=True)
    _, _, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_HOISTED)
    g = bm.bm_gallery_import(c, om.pts_array(), om.masks_array(), om.cmask_array(), R, m, s)
    bm.bm_gallery_set_expansion(g, bm.BM_EXPAND_HOISTED)
    ocs = [om.encrypt(qi) for qi in range(nq)]
    qs = [bm.bm_ciphertext_import(c, om.ct_array(cts), om.ctx.L) for cts in ocs]
    res = bm.bm_match(c, ek, g, qs)
    for qi in range(nq):
        want, opacked = om.match(ocs[qi])
        got = bm.bm_result_export(res, qi)
        assert np.array_equal(got, want), f"query {qi}: ciphertexts differ"
        ref = wl.plaintext_scores(om.feats, om.queries[qi])
        assert np.abs(om.scores(got, opacked) - ref).max() < 1e-5


@pytest.mark.parametrize("form", ["fused", "deferred"])
@pytest.mark.parametrize("name,m,s,R,nq", [
    ("small4", 128, 16, 2500, 2),     # N_in = 8
    ("small4", 16, 4, 3000, 3),       # N_in = 4, three queries
    ("small4", 16, 1, 2100, 1),       # N_in = 16
    ("small4", 128, 4, 600, 1),       # N_in = 32
])
def test_fused_expansion_match_is_bit_exact(name, m, s, R, nq, form):
    """Algorithm 1 with ModDown and Rescale fused (rotations kept on Q_L u P, the
    circulant there, one division by q_L P per part), then every hoisted tail
    form: bit-exact against the oracle's same-order evaluation.  form="deferred":
    the parts left undivided, HE-C^3's products on Q_L u P against the gallery
    plaintexts extended there, one division by q_(L-1) q_L P per (query, group)."""
    c = gctx(name)
    om = OracleMatch(name, m, s, R, nq, hoisted=form, hoisted_tail=True, double_hoisted=True)
    _, _, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_HOISTED)
    g = bm.bm_gallery_import(c, om.pts_array(), om.masks_array(), om.cmask_array(), R, m, s)
    flags = bm.BM_SCHED_ALL | bm.BM_SCHED_DOUBLE_HOISTED | bm.BM_SCHED_FUSED_EXPANSION
    if form == "deferred":
        flags |= bm.BM_SCHED_DEFERRED_DIVISION
    bm.bm_gallery_set_schedule(g, flags)
    ocs = [om.encrypt(qi) for qi in range(nq)]
    qs = [bm.bm_ciphertext_import(c, om.ct_array(cts), om.ctx.L) for cts in ocs]
    res = bm.bm_match(c, ek, g, qs)
    for qi in range(nq):
        want, opacked = om.match(ocs[qi])
        got = bm.bm_result_export(res, qi)
        assert np.array_equal(got, want), f"query {qi}: ciphertexts differ"
        ref = wl.plaintext_scores(om.feats, om.queries[qi])
        assert np.abs(om.scores(got, opacked) - ref).max() < 1e-5


@pytest.mark.parametrize("mode", ["fused", "deferred"])
def test_fused_expansion_pipeline_ring16(mode):
    """Ring 2^16 end to end with the fused Algorithm 1 (and with its division moved
    past HE-C^3's products): scores within 1e-5 of FP64, the FP64 Rank-1."""
    c = gctx("ring16")
    m, s, R = 128, 16, 6144
    feats = wl.gallery(R, m)
    qs, _ = wl.queries(feats, 2)
    sk, pk, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_HOISTED)
    g = bm.bm_encode_gallery_packed(c, feats, m, s, bm.BM_PACK_COMPLEX)
    bm.bm_gallery_set_expansion(g, bm.BM_EXPAND_FUSED if mode == "fused" else bm.BM_EXPAND_DEFERRED)
    cts = bm.bm_encrypt_batch(c, pk, qs, m, s, bm.BM_QUERY_TILED, 4, 0)
    res = bm.bm_match(c, ek, g, cts)
    for qi in range(2):
        ref = wl.plaintext_scores(feats, qs[qi])
        scores, rank1, _ = bm.bm_decrypt_scores(c, sk, res, qi, R)
        assert np.abs(scores - ref).max() < 1e-5
        if np.sort(ref)[-1] - np.sort(ref)[-2] > 2e-5:
            assert rank1 == int(ref.argmax())


@pytest.mark.parametrize("double", [False, True])
@pytest.mark.parametrize("name,m,s,R,nq,tail_only", [
    ("small4", 128, 16, 2500, 2, False),   # every hoisted form: rotate-and-sum 4 x 4, compression 15 rotations
    ("small4", 16, 4, 3000, 3, False),     # rotate-and-sum 2 x 2, partial packs
    ("small4", 32, 32, 700, 1, True),      # rotate-and-sum 8 x 4 after the printed Algorithm 1
    ("small4", 16, 8, 2100, 1, False),     # rotate-and-sum 4 x 2
    ("toy", 16, 4, 1500, 2, True),         # client-expanded queries, per-group outputs (no compression)
])
def test_hoisted_schedule_is_bit_exact(name, m, s, R, nq, tail_only, double):
    """Every hoisted form; double=True: each round's rotations into one output
    summed before a single ModDown (double hoisting)."""
    c = gctx(name)
    om = OracleMatch(name, m, s, R, nq, hoisted=not tail_only and name != "toy", hoisted_tail=True,
                     double_hoisted=double)
    _, _, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_HOISTED)
    g = bm.bm_gallery_import(c, om.pts_array(), om.masks_array(), om.cmask_array(), R, m, s)
    flags = bm.BM_SCHED_HOISTED_ROTSUM | bm.BM_SCHED_HOISTED_COMPRESSION
    if double:
        flags |= bm.BM_SCHED_DOUBLE_HOISTED
    if om.hoisted:
        flags |= bm.BM_SCHED_HOISTED_EXPANSION
    bm.bm_gallery_set_schedule(g, flags)
    ocs = [om.encrypt(qi) for qi in range(nq)]
    qs = [bm.bm_ciphertext_import(c, om.ct_array(cts), om.ctx.L) for cts in ocs]
    res = bm.bm_match(c, ek, g, qs)
    for qi in range(nq):
        want, opacked = om.match(ocs[qi])
        got = bm.bm_result_export(res, qi)
        assert np.array_equal(got, want), f"query {qi}: ciphertexts differ"
        ref = wl.plaintext_scores(om.feats, om.queries[qi])
        assert np.abs(om.scores(got, opacked) - ref).max() < 1e-5


@pytest.mark.parametrize("name,m,s,R,nq,expansion", [
    ("small4", 128, 16, 2500, 2, "deferred"),  # one round of 16 terms a group, 2 groups in one pack
    ("small4", 16, 4, 3000, 3, "fused"),       # packs of 4 groups, a ragged last pack, three queries
    ("small4", 32, 32, 700, 1, "printed"),     # baby steps first, the giant round fused (s > 16)
    ("small4", 16, 8, 2100, 1, "hoisted"),     # one round of 8 terms a group
    ("small4", 16, 1, 2100, 1, "hoisted"),     # parts of 1: each pack one group, its masked term alone
    ("ring16", 16, 4, 20000, 1, "fused"),      # ring 2^16, one pack of 3 groups split over two thread groups
    ("ring16", 128, 16, 5000, 2, "deferred"),  # ring 2^16, 3 groups of 2 queries: the division hands the extension on
])
def test_fused_compression_is_bit_exact(name, m, s, R, nq, expansion):
    """The rotate-and-sum's last round and the compression as one round per pack
    (each group's rotations shifted by its offset, the rotated compression masks
    applied before one ModDown a pack): bit-exact against the oracle's same-order
    evaluation, after each form of Algorithm 1."""
    c = gctx(name)
    hoisted = {"printed": False, "hoisted": True}.get(expansion, expansion)
    om = OracleMatch(name, m, s, R, nq, hoisted=hoisted, hoisted_tail=True, double_hoisted=True,
                     fused_compress=True)
    _, _, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_HOISTED)
    g = bm.bm_gallery_import(c, om.pts_array(), om.masks_array(), om.cmask_array(), R, m, s)
    flags = (bm.BM_SCHED_HOISTED_ROTSUM | bm.BM_SCHED_HOISTED_COMPRESSION | bm.BM_SCHED_DOUBLE_HOISTED
             | bm.BM_SCHED_FUSED_COMPRESSION)
    if expansion != "printed":
        flags |= bm.BM_SCHED_HOISTED_EXPANSION
    if expansion in ("fused", "deferred"):
        flags |= bm.BM_SCHED_FUSED_EXPANSION
    if expansion == "deferred":
        flags |= bm.BM_SCHED_DEFERRED_DIVISION
    bm.bm_gallery_set_schedule(g, flags)
    ocs = [om.encrypt(qi) for qi in range(nq)]
    qs = [bm.bm_ciphertext_import(c, om.ct_array(cts), om.ctx.L) for cts in ocs]
    res = bm.bm_match(c, ek, g, qs)
    for qi in range(nq):
        want, opacked = om.match(ocs[qi])
        got = bm.bm_result_export(res, qi)
        assert np.array_equal(got, want), f"query {qi}: ciphertexts differ"
        ref = wl.plaintext_scores(om.feats, om.queries[qi])
        assert np.abs(om.scores(got, opacked) - ref).max() < 1e-5


def test_fused_compression_flag_needs_the_double_hoisted_tail():
    c = gctx("small4")
    om = OracleMatch("small4", 16, 4, 300, 1)
    g = bm.bm_gallery_import(c, om.pts_array(), om.masks_array(), om.cmask_array(), 300, 16, 4)
    with pytest.raises(bm.BlindMatchError):
        bm.bm_gallery_set_schedule(g, bm.BM_SCHED_HOISTED_ROTSUM | bm.BM_SCHED_FUSED_COMPRESSION)


@pytest.mark.parametrize("double", [False, True])
@pytest.mark.parametrize("m,s,R,nq", [(128, 16, 6144, 1), (128, 4, 20000, 3)])
def test_hoisted_and_doubling_forms_give_the_same_scores_ring16(m, s, R, nq, double):
    c = gctx("ring16")
    feats = wl.gallery(R, m)
    qs, _ = wl.queries(feats, nq)
    sk, pk, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_HOISTED)
    gd = bm.bm_encode_gallery(c, feats, m, s)
    gh = bm.bm_encode_gallery(c, feats, m, s)
    bm.bm_gallery_set_schedule(gh, bm.BM_SCHED_ALL | (bm.BM_SCHED_DOUBLE_HOISTED if double else 0))
    cts = bm.bm_encrypt_batch(c, pk, qs, m, s, bm.BM_QUERY_TILED, 4, 0)
    rd, rh = bm.bm_match(c, ek, gd, cts), bm.bm_match(c, ek, gh, cts)
    for qi in range(nq):
        ref = wl.plaintext_scores(feats, qs[qi])
        sd, r1d, _ = bm.bm_decrypt_scores(c, sk, rd, qi, R)
        sh, r1h, _ = bm.bm_decrypt_scores(c, sk, rh, qi, R)
        assert np.abs(sh - ref).max() < 1e-5 and np.abs(sd - ref).max() < 1e-5
        assert r1h == r1d
        assert not np.array_equal(bm.bm_result_export(rd, qi), bm.bm_result_export(rh, qi))


def test_expansion_errors():
    c = gctx("toy")
    g = bm.bm_encode_gallery(c, wl.gallery(100, 16), 16, 4)
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_gallery_set_expansion(g, bm.BM_EXPAND_HOISTED)    # client-expanded queries: no Algorithm 1
    assert e.value.status == 1
    c4 = gctx("small4")
    _, pk, ek = bm.bm_keygen(c4, KEY_SEED, 16, 4)                 # doubling keys only
    g4 = bm.bm_encode_gallery(c4, wl.gallery(100, 16), 16, 4)
    bm.bm_gallery_set_expansion(g4, bm.BM_EXPAND_HOISTED)
    ct = bm.bm_encrypt_query(c4, pk, wl.gallery(1, 16)[0], 16, 4, bm.BM_QUERY_TILED, 4, 0)
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_match(c4, ek, g4, [ct])                             # rotation by 3 parts has no key
    assert e.value.status == 4
    with pytest.raises(bm.BlindMatchError):
        bm.bm_gallery_set_expansion(g4, 7)
    g1 = bm.bm_encode_gallery(c4, wl.gallery(100, 16), 16, 16)   # one part: no rotations to fuse
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_gallery_set_expansion(g1, bm.BM_EXPAND_FUSED)
    assert e.value.status == 1
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_gallery_set_expansion(g1, bm.BM_EXPAND_DEFERRED)
    assert e.value.status == 1
    with pytest.raises(bm.BlindMatchError) as e:                # the deferred division without the fused form
        bm.bm_gallery_set_schedule(g4, bm.BM_SCHED_HOISTED_EXPANSION | bm.BM_SCHED_DEFERRED_DIVISION)
    assert e.value.status == 1


def test_async_match_gives_the_synchronous_results():
    """bm_match_async enqueues the match and returns: back-to-back calls on one stream
    give the same score ciphertexts as bm_match, export and decryption wait for the
    result themselves, and a result destroyed before its stream has passed it is
    freed in stream order."""
    import torch
    c = gctx("small4")
    m, s, R = 16, 4, 3000
    feats = wl.gallery(R, m)
    qs, _ = wl.queries(feats, 3)
    sk, pk, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_HOISTED)
    g = bm.bm_encode_gallery_packed(c, feats, m, s, bm.BM_PACK_COMPLEX)
    bm.bm_gallery_set_expansion(g, bm.BM_EXPAND_DEFERRED)
    cts = [bm.bm_encrypt_query(c, pk, q, m, s, bm.BM_QUERY_TILED, 4, i) for i, q in enumerate(qs)]
    want = [bm.bm_result_export(bm.bm_match(c, ek, g, [ct]), 0) for ct in cts]
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    dropped = bm.bm_match_async(c, ek, g, [cts[0]], sp)
    res = [bm.bm_match_async(c, ek, g, [ct], sp) for ct in cts]
    del dropped
    for i, r in enumerate(res):
        assert np.array_equal(bm.bm_result_export(r, 0), want[i]), i
        scores, rank1, _ = bm.bm_decrypt_scores(c, sk, r, 0, R)
        ref = wl.plaintext_scores(feats, qs[i])
        assert np.abs(scores - ref).max() < 1e-5
    stream.synchronize()


def test_interleaved_async_matches_keep_each_query():
    """A client with two matches in flight on one stream -- match k enqueued, then the
    scores of match k - 1 read back -- as bench.py's end-to-end loop runs them: host
    queries go through the plan's two staging buffers on its own copy stream while the
    previous match runs, so each result must still be its own query's (different
    queries in turn, every staging buffer reused several times)."""
    import torch
    c = gctx("small4")
    m, s, R = 16, 4, 3000
    feats = wl.gallery(R, m)
    qs, _ = wl.queries(feats, 3)
    sk, pk, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_HOISTED)
    g = bm.bm_encode_gallery_packed(c, feats, m, s, bm.BM_PACK_COMPLEX)
    bm.bm_gallery_set_expansion(g, bm.BM_EXPAND_DEFERRED)
    cts = [bm.bm_encrypt_query(c, pk, q, m, s, bm.BM_QUERY_TILED, 4, i) for i, q in enumerate(qs)]
    want = [bm.bm_result_export(bm.bm_match(c, ek, g, [ct]), 0) for ct in cts]
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    prev = None
    for qi in [0, 1, 2, 1, 0, 2, 2, 0, 1]:
        r = bm.bm_match_async(c, ek, g, [cts[qi]], sp)
        if prev is not None:
            assert np.array_equal(bm.bm_result_export(prev[0], 0), want[prev[1]]), prev[1]
        prev = (r, qi)
    assert np.array_equal(bm.bm_result_export(prev[0], 0), want[prev[1]])
    stream.synchronize()
