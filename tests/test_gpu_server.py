"""Continuous-batching server: every result is the same alone and in a mixed
stream of requests (bit-exact: all match arithmetic is exact integer work per
query), requests for the same gallery are batched, and the admission,
timeout and cancellation paths report their errors."""
import time

import numpy as np
import pytest

from paper_2408_06167_gb300 import workload as wl

pytestmark = pytest.mark.gpu

bm = pytest.importorskip("paper_2408_06167_gb300.binding")

GiB = 1 << 30


@pytest.fixture(scope="module")
def setup():
    ctx = bm.bm_context_create("small4")
    out = {"ctx": ctx, "gal": {}}
    for name, (m, s, R) in {"face": (128, 16, 2500), "finger": (16, 4, 3000)}.items():
        feats = wl.gallery(R, m)
        qs, _ = wl.queries(feats, 4)
        sk, pk, ek = bm.bm_keygen(ctx, 5, m, s)
        g = bm.bm_encode_gallery(ctx, feats, m, s)
        cts = [bm.bm_encrypt_query(ctx, pk, q, m, s, bm.BM_QUERY_TILED, 9, i) for i, q in enumerate(qs)]
        out["gal"][name] = dict(feats=feats, qs=qs, sk=sk, ek=ek, g=g, cts=cts, R=R)
    return out


def test_result_alone_equals_result_in_mix_and_direct_match(setup):
    ctx = setup["ctx"]
    srv = bm.bm_server_create(ctx, 8 * GiB, max_batch=8, executors=2)
    gids = {n: bm.bm_server_add_gallery(srv, d["g"], d["ek"]) for n, d in setup["gal"].items()}
    alone = {}
    for n, d in setup["gal"].items():
        for i, ct in enumerate(d["cts"]):
            r = bm.bm_server_wait(srv, bm.bm_server_submit(srv, gids[n], ct))
            alone[(n, i)] = bm.bm_result_export(r, 0)
            direct = bm.bm_result_export(bm.bm_match(ctx, d["ek"], d["g"], [ct]), 0)
            assert np.array_equal(alone[(n, i)], direct), (n, i)
    before = bm.bm_server_stats(srv)
    # a burst: every query three times, interleaved over the two galleries
    order = [(n, i) for _ in range(3) for i in range(4) for n in ("face", "finger")]
    tickets = [(key, bm.bm_server_submit(srv, gids[key[0]], setup["gal"][key[0]]["cts"][key[1]])) for key in order]
    for key, t in tickets:
        r = bm.bm_server_wait(srv, t)
        assert np.array_equal(bm.bm_result_export(r, 0), alone[key]), key
        if key[1] == 0:
            d = setup["gal"][key[0]]
            scores, rank1, _ = bm.bm_decrypt_scores(ctx, d["sk"], r, 0, d["R"])
            ref = wl.plaintext_scores(d["feats"], d["qs"][0])
            assert np.abs(scores - ref).max() < 1e-5
    st = bm.bm_server_stats(srv)
    assert st["completed"] == 8 + len(order) and st["failed"] == 0
    burst_batches = st["batches"] - before["batches"]
    assert burst_batches < len(order)                  # requests were batched
    assert st["p99_ms"] >= st["p50_ms"] > 0 and st["matches_per_s"] > 0


def test_workspace_over_budget_is_rejected(setup):
    d = setup["gal"]["face"]
    srv = bm.bm_server_create(setup["ctx"], 1 << 20, max_batch=4, executors=1)
    gid = bm.bm_server_add_gallery(srv, d["g"], d["ek"])
    t = bm.bm_server_submit(srv, gid, d["cts"][0])
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_server_wait(srv, t)
    assert e.value.status == 7                         # BM_E_HBM_BUDGET
    assert bm.bm_server_stats(srv)["failed"] == 1


def test_timeout_cancel_and_layout_errors(setup):
    ctx = setup["ctx"]
    d = setup["gal"]["face"]
    srv = bm.bm_server_create(ctx, 8 * GiB, max_batch=2, executors=1)
    gid = bm.bm_server_add_gallery(srv, d["g"], d["ek"])
    first = bm.bm_server_submit(srv, gid, d["cts"][0])
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_server_wait(srv, first, 0)               # cannot be done yet: the plan is still being built
    assert e.value.status == 9                         # BM_E_TIMEOUT
    time.sleep(0.02)
    later = [bm.bm_server_submit(srv, gid, ct) for ct in d["cts"][1:]]
    try:
        bm.bm_server_cancel(srv, later[-1])
        cancelled = True
    except bm.BlindMatchError as err:
        assert err.status == 1                         # already taken by the executor
        cancelled = False
    bm.bm_server_wait(srv, first)
    for t in later[:-1]:
        bm.bm_server_wait(srv, t)
    if cancelled:
        with pytest.raises(bm.BlindMatchError) as e:
            bm.bm_server_wait(srv, later[-1])
        assert e.value.status == 10                    # BM_E_CANCELLED
    else:
        bm.bm_server_wait(srv, later[-1])
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_server_wait(srv, first)                  # already collected
    assert e.value.status == 1
    g16 = setup["gal"]["finger"]
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_server_add_gallery(srv, g16["g"], d["ek"])   # keys of another (dim, part)
    assert e.value.status == 4
    _, pk, _ = bm.bm_keygen(ctx, 5, 128, 16)
    expanded = bm.bm_encrypt_query(ctx, pk, d["qs"][0], 128, 16, bm.BM_QUERY_EXPANDED, 1, 0)
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_server_submit(srv, gid, expanded)
    assert e.value.status == 3                         # BM_E_LEVEL


def test_destroy_with_requests_in_flight(setup):
    d = setup["gal"]["finger"]
    srv = bm.bm_server_create(setup["ctx"], 8 * GiB, max_batch=4, executors=2)
    gid = bm.bm_server_add_gallery(srv, d["g"], d["ek"])
    for ct in d["cts"] * 4:
        bm.bm_server_submit(srv, gid, ct)
    del srv                                             # cancels what is pending, joins the executors
