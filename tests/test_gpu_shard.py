"""Gallery sharding by pack on one GPU: the shards of a 2- and a 3-way split,
each encoded and matched on its own (independent problems run one after the
other), concatenated in rank order, equal the unsharded match bit for bit."""
import numpy as np
import pytest

from helpers_oracle import ENC_SEED, KEY_SEED
from paper_2408_06167_gb300 import shard
from paper_2408_06167_gb300 import workload as wl

pytestmark = pytest.mark.gpu

bm = pytest.importorskip("paper_2408_06167_gb300.binding")


@pytest.mark.parametrize("world", [2, 3])
def test_shards_equal_the_unsharded_match(world):
    ctx = bm.bm_context_create("small4")
    m, s, R = 16, 4, 9000
    feats = wl.gallery(R, m)
    q, _ = wl.queries(feats, 2)
    sk, pk, ek = bm.bm_keygen_ex(ctx, KEY_SEED, m, s, bm.BM_KEYS_HOISTED)
    cts = [bm.bm_encrypt_query(ctx, pk, x, m, s, bm.BM_QUERY_TILED, ENC_SEED, i) for i, x in enumerate(q)]
    flags = bm.BM_SCHED_ALL | bm.BM_SCHED_DOUBLE_HOISTED | bm.BM_SCHED_FUSED_EXPANSION

    def run(lo, hi):
        g = bm.bm_encode_gallery_packed(ctx, feats[lo:hi], m, s, bm.BM_PACK_COMPLEX)
        bm.bm_gallery_set_schedule(g, flags)
        r = bm.bm_match(ctx, ek, g, cts)
        return np.stack([bm.bm_result_export(r, i) for i in range(len(cts))])

    want = run(0, R)
    lay = bm.bm_gallery_layout_packed(ctx, R, m, s, bm.BM_PACK_COMPLEX)
    parts = []
    for rank in range(world):
        lo, hi = shard.shard_range(R, ctx.n // 2, s, True, bool(lay["compressed"]), rank, world)
        if hi > lo:
            parts.append(run(lo, hi))
    got = np.concatenate(parts, axis=1)
    assert got.shape == want.shape and np.array_equal(got, want)
    # and the client reads every identity's score from the gathered ciphertexts
    res = bm.bm_match(ctx, ek, bm.bm_encode_gallery_packed(ctx, feats, m, s, bm.BM_PACK_COMPLEX), cts[:1])
    scores, rank1, _ = bm.bm_decrypt_scores(ctx, sk, res, 0, R)
    assert np.abs(scores - wl.plaintext_scores(feats, q[0])).max() < 1e-5
