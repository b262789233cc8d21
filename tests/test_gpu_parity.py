"""GPU path vs the CPU oracle, through the C-ABI.

Integer results (keys, products, rotations, rescales, match outputs) must be
bit-exact; encodings (FP64) may differ by one unit on rare coefficients, so
the ciphertext parity cases feed the oracle's plaintexts and ciphertexts into
the library.  Decrypted scores must be within 1e-5 of the FP64 cosine with
the same Rank-1 when the top-2 gap exceeds 2e-5.
"""
import numpy as np
import pytest

from helpers_oracle import ENC_SEED, KEY_SEED, OracleMatch, octx, schedule_rotations
from oracle import ckks
from paper_2408_06167_gb300 import workload as wl

pytestmark = pytest.mark.gpu

bm = pytest.importorskip("paper_2408_06167_gb300.binding")

_CTX = {}


def gctx(name):
    if name not in _CTX:
        _CTX[name] = bm.bm_context_create(name)
    return _CTX[name]


def centred_diff(a, b, primes):
    """(a - b) per limb lifted to (-q/2, q/2]; a, b: [..., limbs, N]."""
    out = np.zeros(a.shape, dtype=np.int64)
    for j, q in enumerate(primes):
        d = (a[..., j, :].astype(object) - b[..., j, :].astype(object)) % q
        d = np.where(d > q // 2, d - q, d)
        out[..., j, :] = d.astype(np.int64)
    return out


@pytest.mark.parametrize("name", ["toy", "small4", "ring16"])
def test_primes_agree_with_oracle(name):
    assert bm.bm_context_primes(gctx(name)) == octx(name).primes


@pytest.mark.parametrize("name", ["toy", "ring16"])
def test_negacyclic_product_matches_oracle(name):
    c, o = gctx(name), octx(name)
    rng = np.random.default_rng(5)
    a = np.stack([rng.integers(0, q, size=o.n, dtype=np.uint64) for q in o.primes])
    b = np.stack([rng.integers(0, q, size=o.n, dtype=np.uint64) for q in o.primes])
    b[0, :] = 0
    b[0, 3] = 1                       # edge: a monomial
    got = bm.bm_poly_mul(c, a, b)
    want = np.stack([o.mul(a[j], b[j], j) for j in range(len(o.primes))])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("name,m,s", [("toy", 16, 4), ("small4", 128, 16), ("small4", 16, 4)])
def test_keys_are_bit_exact(name, m, s):
    c, o = gctx(name), octx(name)
    sk, pk, ek = bm.bm_keygen(c, KEY_SEED, m, s)
    rots = schedule_rotations(o, m, s)
    assert bm.bm_eval_keys_rotations(ek) == sorted(set(rots))
    osk, opk, ork = ckks.keygen(o, KEY_SEED, rots)
    assert np.array_equal(bm.bm_secret_key_export(sk), osk.coeffs)
    pkx = bm.bm_public_key_export(pk)
    assert np.array_equal(pkx[0], opk.b) and np.array_equal(pkx[1], opk.a)
    for r in rots:
        assert np.array_equal(bm.bm_eval_keys_export(ek, r), ork[o.galois_left(r)].data), r


def test_ring16_rotation_key_is_bit_exact():
    c, o = gctx("ring16"), octx("ring16")
    _, _, ek = bm.bm_keygen(c, KEY_SEED, 128, 16)
    osk = ckks.sample_secret(o, KEY_SEED)
    for r in [16, -8]:
        want = ckks.keygen_rotation(o, KEY_SEED, osk, o.galois_left(r)).data
        assert np.array_equal(bm.bm_eval_keys_export(ek, r), want)


@pytest.mark.parametrize("name,m,s,mode", [("toy", 16, 4, 1), ("small4", 128, 16, 0), ("ring16", 128, 16, 0)])
def test_encryption_matches_up_to_encoding_rounding(name, m, s, mode):
    c, o = gctx(name), octx(name)
    sk, pk, _ = bm.bm_keygen(c, KEY_SEED, m, s)
    q = wl.queries(wl.gallery(64, m), 2)[0][1]
    ct = bm.bm_ciphertext_export(bm.bm_encrypt_query(c, pk, q, m, s, mode, ENC_SEED, 1))
    opk = ckks.keygen_public(o, KEY_SEED, ckks.sample_secret(o, KEY_SEED))
    S, L = o.slots, o.L
    from oracle import schedule as sch
    zs = ([sch.tiled_query_slots(q, S)] if mode == 0
          else [sch.expanded_query_slots(q, s, i, S) for i in range(m // s)])
    assert ct.shape[0] == len(zs)
    for k, z in enumerate(zs):
        oct_ = ckks.encrypt(o, opk, o.encode(z, o.scale, L), ENC_SEED, 256 + k)
        assert np.array_equal(ct[k, 1], oct_.c1)                 # c1 = v*a + e1: no encoding inside
        d = centred_diff(ct[k, 0], oct_.c0, o.q)
        assert np.abs(d).max() <= 1 and (d != 0).mean() < 0.05  # c0 carries the FP64 encoding


@pytest.mark.parametrize("name,m,s,R", [("toy", 16, 4, 300), ("small4", 128, 16, 2500)])
def test_gallery_encoding_matches_up_to_rounding(name, m, s, R):
    c = gctx(name)
    om = OracleMatch(name, m, s, R, 1)
    g = bm.bm_encode_gallery(c, om.feats, m, s)
    pts, masks, cmask = bm.bm_gallery_export(g)
    o = om.ctx
    for got, want, lvl in [(pts, om.pts_array(), om.level), (masks, om.masks_array(), o.L),
                           (cmask, om.cmask_array(), om.level - 1)]:
        if want is None:
            assert got is None
            continue
        d = centred_diff(got.reshape(-1, lvl + 1, o.n), want.reshape(-1, lvl + 1, o.n), o.q[:lvl + 1])
        assert np.abs(d).max() <= 1 and (d != 0).mean() < 0.05


def _random_ct(o, level, n_cts, seed):
    rng = np.random.default_rng(seed)
    return np.stack([np.stack([np.stack([rng.integers(0, o.q[j], size=o.n, dtype=np.uint64)
                                         for j in range(level + 1)]) for _ in range(2)]) for _ in range(n_cts)])


@pytest.mark.parametrize("level", [0, 1, 2, 3])
@pytest.mark.parametrize("rot", [1, 16, 64, -8])
def test_rotation_is_bit_exact_small4(level, rot):
    c, o = gctx("small4"), octx("small4")
    _, _, ek = bm.bm_keygen(c, KEY_SEED, 128, 16)
    osk = ckks.sample_secret(o, KEY_SEED)
    key = ckks.keygen_rotation(o, KEY_SEED, osk, o.galois_left(rot))
    ev = ckks.Evaluator(o, {key.galois: key})
    data = _random_ct(o, level, 3, 10 * level + (rot % 7))
    got = bm.bm_ciphertext_export(bm.bm_ct_rotate(c, ek, bm.bm_ciphertext_import(c, data, level), rot))
    for b in range(3):
        want = ev.rotate(ckks.Ciphertext(data[b, 0], data[b, 1], level, 1.0), rot)
        assert np.array_equal(got[b, 0], want.c0) and np.array_equal(got[b, 1], want.c1), b


@pytest.mark.parametrize("name,level,rot", [("toy", 0, 1), ("toy", 1, 2), ("ring16", 2, 32), ("ring16", 1, 1)])
def test_rotation_is_bit_exact_other_rings(name, level, rot):
    c, o = gctx(name), octx(name)
    m, s = (16, 4) if name == "toy" else (128, 16)
    _, _, ek = bm.bm_keygen(c, KEY_SEED, m, s)
    key = ckks.keygen_rotation(o, KEY_SEED, ckks.sample_secret(o, KEY_SEED), o.galois_left(rot))
    ev = ckks.Evaluator(o, {key.galois: key})
    data = _random_ct(o, level, 1, 99)
    if o.galois_left(rot) not in [o.galois_left(r) for r in bm.bm_eval_keys_rotations(ek)]:
        pytest.skip("rotation not in the schedule's key set")
    got = bm.bm_ciphertext_export(bm.bm_ct_rotate(c, ek, bm.bm_ciphertext_import(c, data, level), rot))
    want = ev.rotate(ckks.Ciphertext(data[0, 0], data[0, 1], level, 1.0), rot)
    assert np.array_equal(got[0, 0], want.c0) and np.array_equal(got[0, 1], want.c1)


@pytest.mark.parametrize("name,level", [("small4", 1), ("small4", 2), ("small4", 3), ("toy", 1), ("ring16", 3)])
def test_rescale_is_bit_exact(name, level):
    c, o = gctx(name), octx(name)
    data = _random_ct(o, level, 2, level)
    got = bm.bm_ciphertext_export(bm.bm_ct_rescale(c, bm.bm_ciphertext_import(c, data, level)))
    for b in range(2):
        want = ckks.Evaluator(o, {}).rescale(ckks.Ciphertext(data[b, 0], data[b, 1], level, 1.0))
        assert np.array_equal(got[b, 0], want.c0) and np.array_equal(got[b, 1], want.c1)


def _match_parity(name, m, s, R, n_queries, check_queries=None):
    c = gctx(name)
    om = OracleMatch(name, m, s, R, n_queries)
    _, _, ek = bm.bm_keygen(c, KEY_SEED, m, s)
    g = bm.bm_gallery_import(c, om.pts_array(), om.masks_array(), om.cmask_array(), R, m, s)
    ocs = [om.encrypt(qi) for qi in range(n_queries)]
    qs = [bm.bm_ciphertext_import(c, om.ct_array(cts), om.ctx.L) for cts in ocs]
    res = bm.bm_match(c, ek, g, qs)
    nq, n_out, packed = bm.bm_result_info(res)
    assert nq == n_queries and packed == om.compress
    for qi in (check_queries if check_queries is not None else range(n_queries)):
        want, opacked = om.match(ocs[qi])
        got = bm.bm_result_export(res, qi)
        assert got.shape == want.shape
        assert np.array_equal(got, want), f"query {qi}: ciphertexts differ"
        sc = om.scores(got, opacked)
        ref = wl.plaintext_scores(om.feats, om.queries[qi])
        assert np.abs(sc - ref).max() < 1e-5
    return om, res


@pytest.mark.parametrize("name,m,s,R,nq", [
    ("toy", 16, 4, 512, 8),            # toy ring, client-expanded queries, one full group
    ("toy", 16, 4, 700, 2),            # ragged second group, per-group outputs
    ("small4", 128, 16, 2500, 2),      # 20 groups -> 2 packs, second pack partial
    ("small4", 16, 4, 3000, 3),        # 6 groups -> 2 packs of 4 and 2
    ("small4", 16, 16, 100, 1),        # N_in = 1: no Algorithm-1 rotations, one group
    ("small4", 16, 1, 2100, 1),        # part size 1: no HE-C^3 rotations, one group per pack
    ("small4", 64, 4, 1, 1),           # a single identity
])
def test_match_is_bit_exact(name, m, s, R, nq):
    _match_parity(name, m, s, R, nq)


def test_match_face_ring16_is_bit_exact():
    """Ring 2^16, 6,144 identities x 128 dims, parts of 16, one tiled query."""
    _match_parity("ring16", 128, 16, 6144, 1)


def test_library_pipeline_scores_and_rank1():
    """Keys, gallery, encryption, match and decryption all through the library."""
    c = gctx("small4")
    m, s, R = 128, 16, 3000
    feats = wl.gallery(R, m)
    qs, _ = wl.queries(feats, 3)
    sk, pk, ek = bm.bm_keygen(c, 7, m, s)
    g = bm.bm_encode_gallery(c, feats, m, s)
    cts = [bm.bm_encrypt_query(c, pk, q, m, s, bm.BM_QUERY_TILED, 11, i) for i, q in enumerate(qs)]
    res = bm.bm_match(c, ek, g, cts)
    for i, q in enumerate(qs):
        scores, rank1, best = bm.bm_decrypt_scores(c, sk, res, i, R)
        ref = wl.plaintext_scores(feats, q)
        assert np.abs(scores - ref).max() < 1e-5
        top2 = np.sort(ref)[-2:]
        if top2[1] - top2[0] > 2e-5:
            assert rank1 == int(ref.argmax())
        assert best == scores[rank1]


def test_errors_are_reported():
    c = gctx("small4")
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_keygen(c, 1, 24, 4)
    assert e.value.status == 5           # BM_E_DIM
    sk, pk, ek = bm.bm_keygen(c, 1, 16, 4)
    g = bm.bm_encode_gallery(c, wl.gallery(10, 16), 16, 4)
    ct = bm.bm_encrypt_query(c, pk, wl.gallery(1, 16)[0], 16, 4, bm.BM_QUERY_EXPANDED, 1, 0)
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_match(c, ek, g, [ct])
    assert e.value.status == 3           # BM_E_LEVEL: expanded query against a tiled gallery
    _, _, ek2 = bm.bm_keygen(c, 1, 16, 2)
    ct2 = bm.bm_encrypt_query(c, pk, wl.gallery(1, 16)[0], 16, 4, bm.BM_QUERY_TILED, 1, 0)
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_match(c, ek2, g, [ct2])
    assert e.value.status == 4           # BM_E_KEY_MISSING


DNUM4 = ckks.Params(12, (60, 40, 40, 40), (60, 60), dnum=4, secret_hw=192)


def dnum4_ctx():
    """The 4-prime chain with one prime a key-switching digit (four digits at the top
    level: the plain and hoisted key switches sum four products a word)."""
    if "small4-dnum4" not in _CTX:
        p = bm.bm_params_preset("small4")
        p.dnum = 4
        _CTX["small4-dnum4"] = bm.bm_context_create(p)
    return _CTX["small4-dnum4"]


@pytest.mark.parametrize("level,rot", [(0, 1), (1, -8), (2, 16), (3, 16), (3, 64)])
def test_rotation_four_digits_is_bit_exact(level, rot):
    c, o = dnum4_ctx(), octx(DNUM4)
    _, _, ek = bm.bm_keygen(c, KEY_SEED, 128, 16)
    key = ckks.keygen_rotation(o, KEY_SEED, ckks.sample_secret(o, KEY_SEED), o.galois_left(rot))
    ev = ckks.Evaluator(o, {key.galois: key})
    data = _random_ct(o, level, 2, 40 + level)
    got = bm.bm_ciphertext_export(bm.bm_ct_rotate(c, ek, bm.bm_ciphertext_import(c, data, level), rot))
    for b in range(2):
        want = ev.rotate(ckks.Ciphertext(data[b, 0], data[b, 1], level, 1.0), rot)
        assert np.array_equal(got[b, 0], want.c0) and np.array_equal(got[b, 1], want.c1), b


@pytest.mark.parametrize("form", ["fused", "deferred"])
def test_match_four_digits_is_bit_exact(form):
    """The bench's forms (fused Algorithm 1 with or without the deferred division,
    double-hoisted tail with its last round and the compression in one round per pack,
    complex packing) with four digits: the hoisted sums of the top level take four
    digits a word."""
    c = dnum4_ctx()
    m, s, R = 128, 16, 700
    om = OracleMatch(DNUM4, m, s, R, 1, complex_pack=True, hoisted=form, hoisted_tail=True, double_hoisted=True,
                     fused_compress=True)
    _, _, ek = bm.bm_keygen_ex(c, KEY_SEED, m, s, bm.BM_KEYS_HOISTED)
    g = bm.bm_gallery_import_packed(c, om.pts_array(), om.masks_array(), om.cmask_array(), R, m, s, bm.BM_PACK_COMPLEX)
    flags = (bm.BM_SCHED_ALL | bm.BM_SCHED_DOUBLE_HOISTED | bm.BM_SCHED_FUSED_EXPANSION
             | bm.BM_SCHED_FUSED_COMPRESSION)
    if form == "deferred":
        flags |= bm.BM_SCHED_DEFERRED_DIVISION
    bm.bm_gallery_set_schedule(g, flags)
    cts = om.encrypt(0)
    res = bm.bm_match(c, ek, g, [bm.bm_ciphertext_import(c, om.ct_array(cts), om.ctx.L)])
    want, packed = om.match(cts)
    got = bm.bm_result_export(res, 0)
    assert np.array_equal(got, want)
    assert np.abs(om.scores(got, packed) - wl.plaintext_scores(om.feats, om.queries[0])).max() < 1e-5
