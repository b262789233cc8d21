"""Encrypted gallery (Sec. 3.2 enrollment, Algorithm 2 with Mul of two
ciphertexts) on the GPU against the oracle.

Bit-exact: the relinearisation key, the server-side enrollment of encrypted
templates (mask, rescale, right rotations by powers of two, sums into the group
ciphertexts), and the match against a gallery of ciphertexts (tensor products
summed over the parts, one relinearisation, rescale, rotate-and-sum,
compression).  End to end through the library: decrypted scores within 1e-5 of
the FP64 cosine with the same Rank-1."""
import numpy as np
import pytest

from helpers_oracle import KEY_SEED, OracleMatch, octx, schedule_rotations
from oracle import ckks
from oracle import schedule as sch
from paper_2408_06167_gb300 import workload as wl

pytestmark = pytest.mark.gpu

bm = pytest.importorskip("paper_2408_06167_gb300.binding")

_CTX = {}


def gctx(name):
    if name not in _CTX:
        _CTX[name] = bm.bm_context_create(name)
    return _CTX[name]


def test_encrypted_key_set_has_enrollment_rotations():
    c, o = gctx("small4"), octx("small4")
    _, _, ek = bm.bm_keygen_ex(c, KEY_SEED, 16, 4, bm.BM_KEYS_ENCRYPTED_GALLERY)
    have = {o.galois_left(r) for r in bm.bm_eval_keys_rotations(ek)}
    assert {o.galois_left(r) for r in sch.enroll_rotations(4, o.slots)} <= have
    # the relinearisation key itself is checked through the bit-exact matches below


@pytest.mark.parametrize("m,s,R,first", [
    (16, 4, 12, 0),        # one group (G = 512), 4 parts
    (16, 4, 540, 1),       # second group: identities 512..539 (checked against the oracle)
    (128, 128, 40, 0),     # N_in = 1, G = 16: three groups, enrollment chunks span groups
    (128, 16, 20, 0),      # 8 parts, shifts up to 7 rotations
])
def test_enrollment_is_bit_exact(m, s, R, first):
    """small4: server-side enrollment of R encrypted templates; group `first`
    onwards compared with the oracle's enrollment of the same templates."""
    c, o = gctx("small4"), octx("small4")
    S, L, n_in = o.slots, o.L, m // s
    G = S // s
    feats = wl.gallery(R, m)
    sk, pk, rks = ckks.keygen(o, KEY_SEED, schedule_rotations(o, m, s) + sch.enroll_rotations(s, S))
    ev = ckks.Evaluator(o, rks)
    temps = [ckks.encrypt(o, pk, o.encode(sch.template_slots(f, S), o.scale, L), 6, k) for k, f in enumerate(feats)]
    _, _, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_ENCRYPTED_GALLERY)
    lib_t = [bm.bm_ciphertext_import(c, np.stack([np.stack([t.c0, t.c1])]), L) for t in temps]
    g = bm.bm_enroll_encrypted(c, ek, lib_t, m, s)
    got, _, _ = bm.bm_gallery_export(g)
    assert got.shape[:3] == (-(-R // G), n_in, 2)
    emasks = [o.encode(sch.enroll_mask_slots(s, i, S), o.q[L], L) for i in range(n_in)]
    # a group's ciphertexts only involve its own identities, so the oracle enrolls
    # from the first checked group on (its windows are the same: idx mod G)
    want = sch.enroll(ev, temps[first * G:], emasks, s, S)
    for k, row in enumerate(want):
        for i, ct in enumerate(row):
            gi = first + k
            assert np.array_equal(got[gi, i, 0], ct.c0) and np.array_equal(got[gi, i, 1], ct.c1), (gi, i)


@pytest.mark.parametrize("name,m,s,R,nq", [
    ("small4", 16, 4, 1300, 2),       # 3 groups of ciphertexts -> 1 partial pack
    ("small4", 128, 16, 2500, 1),     # 20 groups -> 2 packs
    ("small4", 16, 16, 100, 1),       # N_in = 1: one product per group
])
def test_encrypted_gallery_match_is_bit_exact(name, m, s, R, nq):
    c = gctx(name)
    om = OracleMatch(name, m, s, R, nq, encrypted=True)
    sk, _, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_ENCRYPTED_GALLERY)
    g = bm.bm_gallery_import_encrypted(c, om.pts_array(), om.masks_array(), om.cmask_array(), R, m, s)
    assert bm.bm_gallery_info(g) == (True, bm.BM_PACK_REAL)
    ocs = [om.encrypt(qi) for qi in range(nq)]
    qs = [bm.bm_ciphertext_import(c, om.ct_array(cts), om.ctx.L) for cts in ocs]
    res = bm.bm_match(c, ek, g, qs)
    for qi in range(nq):
        want, opacked = om.match(ocs[qi])
        got = bm.bm_result_export(res, qi)
        assert np.array_equal(got, want), f"query {qi}: ciphertexts differ"
        ref = wl.plaintext_scores(om.feats, om.queries[qi])
        assert np.abs(om.scores(got, opacked) - ref).max() < 1e-5
        # the library decrypts with the product's scale
        scores, rank1, _ = bm.bm_decrypt_scores(c, sk, res, qi, R)
        assert np.abs(scores - ref).max() < 1e-5


@pytest.mark.parametrize("name,m,s,R,batch", [("small4", 16, 4, 1500, False), ("ring16", 128, 16, 2500, True)])
def test_encrypted_gallery_pipeline(name, m, s, R, batch):
    """Templates encrypted by the client library (one by one, or as one GPU batch
    kept on the device), enrolled by the server, matched."""
    c = gctx(name)
    feats = wl.gallery(R, m)
    qs, _ = wl.queries(feats, 2)
    sk, pk, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_ENCRYPTED_GALLERY)
    if batch:
        temps = bm.bm_encrypt_batch(c, pk, feats, m, s, bm.BM_QUERY_TEMPLATE, 6, 0, bm.BM_ENC_KEEP_DEVICE)
    else:
        temps = [bm.bm_encrypt_query(c, pk, f, m, s, bm.BM_QUERY_TEMPLATE, 6, k) for k, f in enumerate(feats)]
    g = bm.bm_enroll_encrypted(c, ek, temps, m, s)
    cts = [bm.bm_encrypt_query(c, pk, q, m, s, bm.BM_QUERY_TILED, 4, i) for i, q in enumerate(qs)]
    res = bm.bm_match(c, ek, g, cts)
    for qi in range(2):
        ref = wl.plaintext_scores(feats, qs[qi])
        scores, rank1, _ = bm.bm_decrypt_scores(c, sk, res, qi, R)
        assert np.abs(scores - ref).max() < 1e-5
        if np.sort(ref)[-1] - np.sort(ref)[-2] > 2e-5:
            assert rank1 == int(ref.argmax())


def test_encrypted_gallery_errors():
    c = gctx("toy")
    _, pk, ek = bm.bm_keygen_ex(c, KEY_SEED, 16, 4, bm.BM_KEYS_ENCRYPTED_GALLERY)
    t = bm.bm_encrypt_query(c, pk, np.ones(16) / 4, 16, 4, bm.BM_QUERY_TEMPLATE, 6, 0)
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_enroll_encrypted(c, ek, [t], 16, 4)          # toy chain: one rescale prime
    assert e.value.status == 3
    c4 = gctx("small4")
    _, pk4, ek_plain = bm.bm_keygen(c4, KEY_SEED, 16, 4)
    t4 = bm.bm_encrypt_query(c4, pk4, np.ones(16) / 4, 16, 4, bm.BM_QUERY_TEMPLATE, 6, 0)
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_enroll_encrypted(c4, ek_plain, [t4], 16, 4)  # no relinearisation key
    assert e.value.status == 4


@pytest.mark.parametrize("name,m,s,mode", [("small4", 128, 16, 0), ("toy", 16, 4, 1), ("small4", 16, 4, 2),
                                           ("ring16", 128, 16, 0)])
def test_batch_encryption_equals_single_encryptions(name, m, s, mode):
    """GPU-drawn noise: every ciphertext of a batch is bit-identical to the same
    vector encrypted alone (same seed and query id), and its c1 (which holds no
    encoding) is bit-exact against the oracle's encryption."""
    c, o = gctx(name), octx(name)
    feats = wl.gallery(70, m, seed=9)
    sk, pk, _ = bm.bm_keygen(c, KEY_SEED, m, s)
    batch = bm.bm_encrypt_batch(c, pk, feats, m, s, mode, 11, first_id=5)
    assert len(batch) == 70
    osk, opk, _ = ckks.keygen(o, KEY_SEED, [])
    S, L = o.slots, o.L
    for k in (0, 33, 69):
        single = bm.bm_encrypt_query(c, pk, feats[k], m, s, mode, 11, 5 + k)
        a, b = bm.bm_ciphertext_export(batch[k]), bm.bm_ciphertext_export(single)
        assert np.array_equal(a, b), k
        if mode == 0:
            z = sch.tiled_query_slots(feats[k], S)
        elif mode == 2:
            z = sch.template_slots(feats[k], S)
        else:
            z = sch.expanded_query_slots(feats[k], s, 0, S)
        want = ckks.encrypt(o, opk, o.encode(z, o.scale, L), 11, (5 + k) * 256)
        assert np.array_equal(a[0, 1], want.c1)
    # device copies kept on request
    kept = bm.bm_encrypt_batch(c, pk, feats[:3], m, s, mode, 11, first_id=5, flags=bm.BM_ENC_KEEP_DEVICE)
    assert np.array_equal(bm.bm_ciphertext_export(kept[1]), bm.bm_ciphertext_export(batch[1]))
