"""The allocation-free rotation entry point gives the same ciphertexts as bm_ct_rotate.

bm_ct_rotate_noalloc exists for callers that cannot let the library allocate
device memory (a host whose GPU memory belongs to its own pool allocator, or a
serving loop that forbids allocation after start-up).  It keeps its
temporaries in one shared file-scope device array, so it is called twice in a
row here to show that what an earlier call leaves in that array does not leak
into the next result.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bm = pytest.importorskip("paper_2408_06167_gb300.binding")


def _random_cts(n, primes, level, n_cts, seed):
    rng = np.random.default_rng(seed)
    return np.stack([np.stack([np.stack([rng.integers(0, primes[j], size=n, dtype=np.uint64)
                                         for j in range(level + 1)]) for _ in range(2)]) for _ in range(n_cts)])


def _device(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


@pytest.mark.parametrize("preset,dim,part,level,n_cts,rots", [
    ("small4", 128, 16, 2, 3, [16, 1]),
    ("ring16", 128, 16, 3, 1, [32, -4]),
])
def test_noalloc_rotation_equals_allocating_rotation(preset, dim, part, level, n_cts, rots):
    ctx = bm.bm_context_create(preset)
    _, _, ek = bm.bm_keygen(ctx, 3, dim, part)
    primes = bm.bm_context_primes(ctx)
    stream = torch.cuda.current_stream()
    for call, rot in enumerate(rots):          # two calls in a row on the shared scratch
        data = _random_cts(ctx.n, primes, level, n_cts, seed=call)
        want = bm.bm_ciphertext_export(bm.bm_ct_rotate(ctx, ek, bm.bm_ciphertext_import(ctx, data, level), rot))
        d_in = _device(data)
        d_out = torch.full_like(d_in, -1)       # the call must overwrite every word
        bm.bm_ct_rotate_noalloc(ctx, ek, d_in.data_ptr(), n_cts, level, rot, d_out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint64).reshape(want.shape)
        assert np.array_equal(got, want), (preset, call)
        assert np.array_equal(d_in.cpu().numpy().view(np.uint64).reshape(data.shape), data)   # input untouched


def test_noalloc_rejects_requests_beyond_its_scratch():
    ctx = bm.bm_context_create("ring16")
    _, _, ek = bm.bm_keygen(ctx, 3, 128, 16)
    d = torch.zeros(2 * 2 * 4 * ctx.n, dtype=torch.int64, device="cuda")
    with pytest.raises(bm.BlindMatchError) as e:
        bm.bm_ct_rotate_noalloc(ctx, ek, d.data_ptr(), 2, 3, 1, d.data_ptr() + 0, None)
    assert e.value.status == 1 and "limit" in str(e.value)
