"""Complex slot packing on the GPU against the oracle: the match of a gallery
whose groups carry a second identity in the imaginary parts is bit-exact
against the oracle's match of the same plaintexts and query ciphertexts, the
library's complex encoder agrees with the oracle's up to rounding, and the
decrypted scores are the FP64 cosine within 1e-5 with the same Rank-1."""
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
    ("small4", 128, 16, 5000, 2),     # 40 real groups -> 20 complex groups -> 2 packs, second partial
    ("small4", 16, 4, 3000, 1),       # 6 -> 3 complex groups, one partial pack; last group half imaginary
    ("small4", 16, 16, 700, 1),       # one complex group, imaginary part partly empty
    ("toy", 16, 4, 1500, 2),          # client-expanded queries, per-group outputs
])
def test_complex_packed_match_is_bit_exact(name, m, s, R, nq):
    c = gctx(name)
    om = OracleMatch(name, m, s, R, nq, complex_pack=True)
    _, _, ek = bm.bm_keygen(c, KEY_SEED, m, s)
    g = bm.bm_gallery_import_packed(c, om.pts_array(), om.masks_array(), om.cmask_array(), R, m, s,
                                    bm.BM_PACK_COMPLEX)
    lo = bm.bm_gallery_layout_packed(c, R, m, s, bm.BM_PACK_COMPLEX)
    assert lo["groups"] == om.groups
    ocs = [om.encrypt(qi) for qi in range(nq)]
    qs = [bm.bm_ciphertext_import(c, om.ct_array(cts), om.ctx.L) for cts in ocs]
    res = bm.bm_match(c, ek, g, qs)
    for qi in range(nq):
        want, opacked = om.match(ocs[qi])
        got = bm.bm_result_export(res, qi)
        assert np.array_equal(got, want), f"query {qi}: ciphertexts differ"
        ref = wl.plaintext_scores(om.feats, om.queries[qi])
        assert np.abs(om.scores(got, opacked) - ref).max() < 1e-5


def test_complex_encoder_matches_oracle_up_to_rounding():
    c = gctx("small4")
    om = OracleMatch("small4", 16, 4, 3000, 1, complex_pack=True)
    g = bm.bm_encode_gallery_packed(c, om.feats, 16, 4, bm.BM_PACK_COMPLEX)
    pts, _, _ = bm.bm_gallery_export(g)
    want = om.pts_array()
    assert pts.shape == want.shape
    q = om.ctx.q
    for j in range(pts.shape[2]):
        d = (pts[:, :, j].astype(object) - want[:, :, j].astype(object)) % q[j]
        d = np.where(d > q[j] // 2, d - q[j], d).astype(np.int64)
        assert np.abs(d).max() <= 1 and (d != 0).mean() < 0.05


@pytest.mark.parametrize("name,m,s,R", [("ring16", 128, 16, 6144), ("ring16", 16, 4, 65536)])
def test_complex_packed_pipeline_scores_and_rank1(name, m, s, R):
    c = gctx(name)
    feats = wl.gallery(R, m)
    qs, _ = wl.queries(feats, 2)
    sk, pk, ek = bm.bm_keygen(c, KEY_SEED, m, s)
    g = bm.bm_encode_gallery_packed(c, feats, m, s, bm.BM_PACK_COMPLEX)
    gr = bm.bm_encode_gallery(c, feats, m, s)
    cts = [bm.bm_encrypt_query(c, pk, q, m, s, bm.BM_QUERY_TILED, 4, i) for i, q in enumerate(qs)]
    res = bm.bm_match(c, ek, g, cts)
    res_r = bm.bm_match(c, ek, gr, cts)
    assert bm.bm_result_info(res)[1] <= bm.bm_result_info(res_r)[1]
    for qi in range(2):
        ref = wl.plaintext_scores(feats, qs[qi])
        scores, rank1, top = bm.bm_decrypt_scores(c, sk, res, qi, R)
        assert np.abs(scores - ref).max() < 1e-5
        gap = np.sort(ref)[-1] - np.sort(ref)[-2]
        assert top == pytest.approx(ref.max(), abs=1e-5)
        if gap > 2e-5:
            assert rank1 == int(ref.argmax())
        scores_r, rank1_r, _ = bm.bm_decrypt_scores(c, sk, res_r, qi, R)
        assert rank1_r == rank1 and np.abs(scores_r - scores).max() < 2e-5

