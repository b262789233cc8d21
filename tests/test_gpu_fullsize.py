"""Parity at the benchmarked sizes, in the launch configuration the bench times.

* 6,144 identities x 128 dims, parts of 16, one query (the bench's default line,
  its default forms, through bm_match_async): the score ciphertext is bit-exact
  against the oracle's evaluation in the same order.
* 65,536 identities x 16 dims, parts of 4, 64 queries matched in one batched
  call, in the printed forms and in the bench's forms: the score ciphertexts of
  sampled queries are bit-exact against the oracle's match of the same
  plaintexts and query ciphertexts.
* 1,048,576 identities x 128 dims, parts of 16, 256 queries in one call (too
  large for the oracle): for sampled queries every one of the million
  decrypted scores is within 1e-5 of the FP64 cosine and Rank-1 is the FP64
  argmax -- with the plaintext gallery as configured, and with the cost
  model's part size, complex packing and the hoisted Algorithm 1.
"""
import numpy as np
import pytest

from helpers_oracle import KEY_SEED, OracleMatch
from paper_2408_06167_gb300 import workload as wl

pytestmark = pytest.mark.gpu

bm = pytest.importorskip("paper_2408_06167_gb300.binding")


@pytest.fixture(scope="module")
def ring16():
    return bm.bm_context_create("ring16")


def test_finger_batched_full_size_is_bit_exact(ring16):
    c = ring16
    W = wl.WORKLOADS["finger-16d-65536-q64"]
    om = OracleMatch("ring16", W.dim, W.part, W.n_ids, W.n_queries)
    _, _, ek = bm.bm_keygen(c, KEY_SEED, W.dim, W.part)
    g = bm.bm_gallery_import(c, om.pts_array(), om.masks_array(), om.cmask_array(), W.n_ids, W.dim, W.part)
    ocs = [om.encrypt(qi) for qi in range(W.n_queries)]
    qs = [bm.bm_ciphertext_import(c, om.ct_array(cts), om.ctx.L) for cts in ocs]
    res = bm.bm_match(c, ek, g, qs)
    assert bm.bm_result_info(res)[:2] == (W.n_queries, 2)
    for qi in (0, W.n_queries - 1):
        want, packed = om.match(ocs[qi])
        got = bm.bm_result_export(res, qi)
        assert np.array_equal(got, want), f"query {qi}: ciphertexts differ"
        ref = wl.plaintext_scores(om.feats, om.queries[qi])
        assert np.abs(om.scores(got, packed) - ref).max() < 1e-5


@pytest.mark.parametrize("part,packing,hoisted", [(16, 0, False), (4, 1, True)])
def test_large_batched_full_size_scores(ring16, part, packing, hoisted):
    c = ring16
    W = wl.WORKLOADS["large-128d-1m-q256"]
    feats = wl.gallery(W.n_ids, W.dim)
    qs, _ = wl.queries(feats, W.n_queries)
    sk, pk, ek = bm.bm_keygen_ex(c, KEY_SEED, W.dim, part, bm.BM_KEYS_HOISTED if hoisted else 0)
    g = bm.bm_encode_gallery_packed(c, feats, W.dim, part, packing)
    if hoisted:
        bm.bm_gallery_set_expansion(g, bm.BM_EXPAND_HOISTED)
    cts = bm.bm_encrypt_batch(c, pk, qs, W.dim, part, bm.BM_QUERY_TILED, 4, 0, bm.BM_ENC_KEEP_DEVICE)
    res = bm.bm_match(c, ek, g, cts)
    for qi in (0, 131, W.n_queries - 1):
        ref = wl.plaintext_scores(feats, qs[qi])
        scores, rank1, top = bm.bm_decrypt_scores(c, sk, res, qi, W.n_ids)
        assert np.abs(scores - ref).max() < 1e-5, qi
        srt = np.sort(ref)
        if srt[-1] - srt[-2] > 2e-5:
            assert rank1 == int(ref.argmax()), qi


@pytest.mark.parametrize("fused_compress", [True, False])
def test_face_full_size_default_forms_are_bit_exact(ring16, fused_compress):
    """The bench's default line: 6,144 identities x 128 dims, parts of 16, one query,
    complex packing, the fused Algorithm 1 with the deferred division and the
    double-hoisted tail (its last round and the compression in one round per pack, or
    the two rounds), matched through bm_match_async as the bench times it: the score
    ciphertext is bit-exact against the oracle's same-order evaluation."""
    c = ring16
    W = wl.WORKLOADS["face-128d-6144"]
    om = OracleMatch("ring16", W.dim, W.part, W.n_ids, 1, complex_pack=True, hoisted="deferred", hoisted_tail=True,
                     double_hoisted=True, fused_compress=fused_compress)
    _, _, ek = bm.bm_keygen_ex(c, KEY_SEED, W.dim, W.part, bm.BM_KEYS_HOISTED)
    g = bm.bm_gallery_import_packed(c, om.pts_array(), om.masks_array(), om.cmask_array(), W.n_ids, W.dim, W.part,
                                    bm.BM_PACK_COMPLEX)
    bm.bm_gallery_set_schedule(g, bm.BM_SCHED_ALL | bm.BM_SCHED_DOUBLE_HOISTED | bm.BM_SCHED_FUSED_EXPANSION
                               | bm.BM_SCHED_DEFERRED_DIVISION
                               | (bm.BM_SCHED_FUSED_COMPRESSION if fused_compress else 0))
    cts = om.encrypt(0)
    q = bm.bm_ciphertext_import(c, om.ct_array(cts), om.ctx.L)
    res = bm.bm_match_async(c, ek, g, [q])
    got = bm.bm_result_export(res, 0)
    want, packed = om.match(cts)
    assert np.array_equal(got, want), "score ciphertexts differ"
    ref = wl.plaintext_scores(om.feats, om.queries[0])
    assert np.abs(om.scores(got, packed) - ref).max() < 1e-5


def test_finger_full_size_default_forms_are_bit_exact(ring16):
    """The finger line's forms: 65,536 identities x 16 dims, parts of 4, 64 queries in
    one call, complex packing, the fused Algorithm 1 (4 groups, 4 parts) and the
    double-hoisted tail with its last round and the compression in one round per pack:
    sampled queries bit-exact against the oracle."""
    c = ring16
    W = wl.WORKLOADS["finger-16d-65536-q64"]
    om = OracleMatch("ring16", W.dim, W.part, W.n_ids, W.n_queries, complex_pack=True, hoisted="fused",
                     hoisted_tail=True, double_hoisted=True, fused_compress=True)
    _, _, ek = bm.bm_keygen_ex(c, KEY_SEED, W.dim, W.part, bm.BM_KEYS_HOISTED)
    g = bm.bm_gallery_import_packed(c, om.pts_array(), om.masks_array(), om.cmask_array(), W.n_ids, W.dim, W.part,
                                    bm.BM_PACK_COMPLEX)
    bm.bm_gallery_set_schedule(g, bm.BM_SCHED_ALL | bm.BM_SCHED_DOUBLE_HOISTED | bm.BM_SCHED_FUSED_EXPANSION
                               | bm.BM_SCHED_FUSED_COMPRESSION)
    ocs = [om.encrypt(qi) for qi in range(W.n_queries)]
    qs = [bm.bm_ciphertext_import(c, om.ct_array(cts), om.ctx.L) for cts in ocs]
    res = bm.bm_match_async(c, ek, g, qs)
    for qi in (0, W.n_queries - 1):
        want, packed = om.match(ocs[qi])
        got = bm.bm_result_export(res, qi)
        assert np.array_equal(got, want), f"query {qi}: ciphertexts differ"
        ref = wl.plaintext_scores(om.feats, om.queries[qi])
        assert np.abs(om.scores(got, packed) - ref).max() < 1e-5
