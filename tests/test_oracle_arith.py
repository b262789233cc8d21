"""Pins of the oracle's integer core against facts it cannot fake.

Each check reaches outside the oracle: sympy primality, Python big-integer
brute force (schoolbook negacyclic products, direct evaluation, exact CRT),
numpy's Philox4x64 bit generator, decimal high-precision Gaussian CDF, and
closed forms that hold at full ring size.
"""
import decimal
import math

import numpy as np
import pytest
import sympy

from oracle import ckks, micro

PRESET_NAMES = ["toy", "small4", "ring16"]


def _small_prime(log_n, bits=50):
    q, _ = ckks.gen_chain(log_n, (bits,), ())
    return q[0], ckks.lib().orc_find_psi(q[0], log_n)


# ------------------------------------------------------------------ primes


@pytest.mark.parametrize("name", PRESET_NAMES)
def test_primes_are_the_largest_ntt_friendly_primes(name):
    ctx = ckks.Context(name)
    two_n = 2 * ctx.n
    bits = list(ctx.params.q_bits) + list(ctx.params.p_bits)
    chosen = []
    for prime, b in zip(ctx.primes, bits):
        assert sympy.isprime(prime)
        assert prime % two_n == 1
        assert prime < (1 << b) and prime.bit_length() == b
        # every larger candidate below 2^b is composite or already taken earlier in the chain
        c = prime + two_n
        while c < (1 << b):
            assert c in chosen or not sympy.isprime(c), (name, c)
            c += two_n
        chosen.append(prime)
    assert len(set(ctx.primes)) == len(ctx.primes)


@pytest.mark.parametrize("name", PRESET_NAMES)
def test_psi_is_primitive_2n_root_from_smallest_generator(name):
    ctx = ckks.Context(name)
    for q, psi in zip(ctx.primes, ctx.psi):
        assert pow(psi, ctx.n, q) == q - 1          # order exactly 2N (2N is a power of two)
        e = (q - 1) // (2 * ctx.n)
        g = next(g for g in range(2, 1000) if pow(pow(g, e, q), ctx.n, q) == q - 1)
        assert psi == pow(g, e, q)


# --------------------------------------------------------------------- NTT


@pytest.mark.parametrize("log_n", [2, 3, 4, 5])
def test_ntt_is_evaluation_at_odd_powers_of_psi(log_n):
    q, psi = _small_prime(log_n)
    rng = np.random.default_rng(log_n)
    n = 1 << log_n
    a = [int(x) for x in rng.integers(0, q, size=n, dtype=np.uint64)]
    got = ckks.ntt(np.array(a, dtype=np.uint64), log_n, q, psi)
    want = [micro.evaluate(a, pow(psi, 2 * i + 1, q), q) for i in range(n)]
    assert [int(x) for x in got] == want


@pytest.mark.parametrize("log_n", [3, 5, 8])
def test_ntt_product_equals_schoolbook_negacyclic(log_n):
    q, psi = _small_prime(log_n, 60)
    rng = np.random.default_rng(100 + log_n)
    n = 1 << log_n
    a = rng.integers(0, q, size=n, dtype=np.uint64)
    b = rng.integers(0, q, size=n, dtype=np.uint64)
    got = ckks.poly_mul(a, b, log_n, q, psi)
    want = micro.schoolbook_negacyclic([int(x) for x in a], [int(x) for x in b], q)
    assert [int(x) for x in got] == want


@pytest.mark.parametrize("name", ["toy", "ring16"])
def test_full_size_products_closed_forms(name):
    """X^a * X^b = +-X^((a+b) mod N) and f * X = negacyclic shift of f, at full ring size."""
    ctx = ckks.Context(name)
    n, gi = ctx.n, 0
    q = ctx.primes[gi]
    for a, b in [(0, 0), (1, n - 1), (n - 1, n - 1), (12345 % n, 777)]:
        xa = np.zeros(n, dtype=np.uint64)
        xb = np.zeros(n, dtype=np.uint64)
        xa[a] = 1
        xb[b] = 1
        got = ctx.mul(xa, xb, gi)
        want = np.zeros(n, dtype=np.uint64)
        e = a + b
        want[e % n] = 1 if e < n else q - 1
        assert np.array_equal(got, want)
    rng = np.random.default_rng(7)
    f = rng.integers(0, q, size=n, dtype=np.uint64)
    x = np.zeros(n, dtype=np.uint64)
    x[1] = 1
    shifted = np.empty(n, dtype=np.uint64)
    shifted[0] = (q - int(f[-1])) % q
    shifted[1:] = f[:-1]
    assert np.array_equal(ctx.mul(f, x, gi), shifted)


@pytest.mark.parametrize("name", ["toy", "ring16"])
def test_ntt_roundtrip_identity(name):
    ctx = ckks.Context(name)
    rng = np.random.default_rng(1)
    for gi, q in enumerate(ctx.primes):
        a = rng.integers(0, q, size=ctx.n, dtype=np.uint64)
        assert np.array_equal(ctx.intt(ctx.ntt(a, gi), gi), a)


# ------------------------------------------------------------ automorphism


@pytest.mark.parametrize("log_n,k", [(3, 5), (4, 3), (5, 25), (5, 63)])
def test_automorphism_is_substitution(log_n, k):
    q, _ = _small_prime(log_n)
    rng = np.random.default_rng(k)
    a = [int(x) for x in rng.integers(0, q, size=1 << log_n, dtype=np.uint64)]
    got = ckks.automorphism(np.array(a, dtype=np.uint64), log_n, k, q)
    assert [int(x) for x in got] == micro.substitute(a, k, q)


def test_automorphism_composes_and_is_a_ring_map():
    ctx = ckks.Context("toy")
    q, n = ctx.q[0], ctx.n
    rng = np.random.default_rng(3)
    a = rng.integers(0, q, size=n, dtype=np.uint64)
    b = rng.integers(0, q, size=n, dtype=np.uint64)
    k1, k2 = 5, pow(5, 7, 2 * n)
    s1 = ckks.automorphism(ckks.automorphism(a, ctx.log_n, k1, q), ctx.log_n, k2, q)
    s2 = ckks.automorphism(a, ctx.log_n, (k1 * k2) % (2 * n), q)
    assert np.array_equal(s1, s2)
    lhs = ckks.automorphism(ctx.mul(a, b, 0), ctx.log_n, k1, q)
    rhs = ctx.mul(ckks.automorphism(a, ctx.log_n, k1, q), ckks.automorphism(b, ctx.log_n, k1, q), 0)
    assert np.array_equal(lhs, rhs)


# ------------------------------------------------------------------ Philox


@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (0, 0, 0, 0)),
    ((2**64 - 1, 2**64 - 1), (2**64 - 1, 2**64 - 1, 2**64 - 1, 2**64 - 1)),
    ((3, 4), (17, 2, 65535, 0)),
    ((0x243F6A8885A308D3, 0x13198A2E03707344), (0xA4093822299F31D0, 0x082EFA98EC4E6C89,
                                                 0x452821E638D01377, 0xBE5466CF34E90C6C)),
])
def test_philox_matches_numpy_bit_generator(key, ctr):
    # numpy's Philox (4x64, 10 rounds) increments the 256-bit counter before each block
    c = sum(int(x) << (64 * i) for i, x in enumerate(ctr))
    prev = (c - 1) % (1 << 256)
    words = np.array([(prev >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=words)
    want = [int(x) for x in bg.random_raw(4)]
    assert ckks.philox4x64(key[0], key[1], ctr) == want


# ---------------------------------------------------------------- samplers


def test_cdt_table_matches_high_precision_cdf():
    sigma, kmax = 3.2, 19
    decimal.getcontext().prec = 60
    D = decimal.Decimal
    rho = [(-D(k * k) / (2 * D(sigma) ** 2)).exp() for k in range(kmax + 1)]
    z = rho[0] + 2 * sum(rho[1:])
    table = ckks.cdt_table(sigma, kmax)
    acc = D(0)
    for k in range(kmax + 1):
        acc += rho[k] * (1 if k == 0 else 2)
        exact = acc / z * (D(2) ** 63)
        assert abs(D(table[k]) - exact) <= D(2) ** 12, k   # double precision: 53 of 63 bits
    assert table[-1] == 1 << 63
    assert all(a < b for a, b in zip(table, table[1:]))


def test_gaussian_sampler_moments():
    ctx = ckks.Context("ring16")
    e = np.concatenate([ckks.sample_gauss(ctx, 11, ckks.TAG_PK_E, obj) for obj in range(4)])
    n = e.size
    var = 3.2 ** 2
    assert abs(e.mean()) < 5 * math.sqrt(var / n)
    assert abs(e.var() - var) < 5 * var * math.sqrt(2.0 / n)
    assert np.abs(e).max() <= 19
    p0 = 1.0 / sum(math.exp(-k * k / (2 * var)) * (1 if k == 0 else 2) for k in range(20))
    assert abs((e == 0).mean() - p0) < 5 * math.sqrt(p0 * (1 - p0) / n)
    assert abs((e > 0).mean() - (e < 0).mean()) < 5 / math.sqrt(n)


def test_hamming_weight_secret():
    ctx = ckks.Context("ring16")
    s = ckks.sample_secret(ctx, 3).coeffs
    assert np.count_nonzero(s) == 192
    assert set(np.unique(s).tolist()) == {-1, 0, 1}
    assert np.array_equal(s, ckks.sample_secret(ctx, 3).coeffs)
    assert not np.array_equal(s, ckks.sample_secret(ctx, 4).coeffs)


def test_zo_sampler_frequencies():
    ctx = ckks.Context("ring16")
    v = ckks.sample_zo(ctx, 5, ckks.TAG_ENC_V, 0)
    n = v.size
    for val, p in [(0, 0.5), (1, 0.25), (-1, 0.25)]:
        assert abs((v == val).mean() - p) < 5 * math.sqrt(p * (1 - p) / n)


def test_uniform_sampler_range_and_mean():
    ctx = ckks.Context("small4")
    for gi, q in enumerate(ctx.primes):
        a = ckks.sample_uniform(ctx, 9, ckks.TAG_RK_A, 1, gi)
        assert int(a.max()) < q
        mean = a.astype(np.float64).mean() / q
        assert abs(mean - 0.5) < 5 * math.sqrt(1 / 12 / a.size)
    assert not np.array_equal(ckks.sample_uniform(ctx, 9, ckks.TAG_RK_A, 1, 0),
                              ckks.sample_uniform(ctx, 9, ckks.TAG_RK_A, 2, 0))


# ---------------------------------------------------- base conversion, rescale


@pytest.mark.parametrize("src_idx,dst_idx", [([0, 1], [4, 5, 2]), ([2, 3], [0, 1, 4, 5]), ([4, 5], [0, 1, 2, 3]),
                                             ([2], [0, 1, 4, 5])])
def test_bconv_is_x_plus_small_multiple_of_B(src_idx, dst_idx):
    ctx = ckks.Context("small4")
    rng = np.random.default_rng(sum(src_idx))
    n = 64
    src = [ctx.primes[i] for i in src_idx]
    B = math.prod(src)
    xs = [int(rng.integers(0, 2**62)) * int(rng.integers(0, 2**62)) % B for _ in range(n)]
    xs[:4] = [0, 1, B - 1, B // 2]
    limbs = np.array([[x % p for x in xs] for p in src], dtype=np.uint64)
    for t_i in dst_idx:
        t = ctx.primes[t_i]
        y = ckks.bconv(limbs, src, t)
        for c in range(n):
            es = [e for e in range(len(src)) if (xs[c] + e * B) % t == int(y[c])]
            assert es, (c, xs[c])


@pytest.mark.parametrize("level", [1, 2, 3])
def test_rescale_is_exact_rounding_division(level):
    ctx = ckks.Context("small4")
    rng = np.random.default_rng(level)
    n = 256
    primes = ctx.q[: level + 1]
    Q = math.prod(primes)
    xs = [int(rng.integers(0, 2**63)) ** 3 % Q for _ in range(n)]
    ql = primes[-1]
    xs[:3] = [0, ql // 2, ql // 2 + 1]
    limbs = np.array([[x % p for x in xs] for p in primes], dtype=np.uint64)
    out = ckks.rescale_poly(limbs, ctx.q, level)
    Qd = Q // ql
    for c in range(n):
        x = xs[c] - Q if xs[c] > Q // 2 else xs[c]
        want = (2 * x + ql) // (2 * ql)         # round(x / ql), no ties (ql odd)
        got = micro.crt([int(out[j][c]) for j in range(level)], primes[:level])
        assert (got - want) % Qd == 0, c


# ------------------------------------------------------------ key switching


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_keyswitch_output_decrypts_to_c_times_rotated_secret(level):
    """KS(c) = (d0, d1) with d0 + d1*s = c * sigma_k(s) + (small) mod Q_level."""
    ctx = ckks.Context("small4")
    sk = ckks.sample_secret(ctx, 3)
    k = ctx.galois_left(3)
    key = ckks.keygen_rotation(ctx, 3, sk, k)
    rng = np.random.default_rng(level)
    c = np.stack([rng.integers(0, ctx.q[j], size=ctx.n, dtype=np.uint64) for j in range(level + 1)])
    d0, d1 = ckks.keyswitch(ctx, c, level, key)
    diff = np.zeros((level + 1, ctx.n), dtype=np.uint64)
    for j in range(level + 1):
        qj = ctx.q[j]
        s_j = sk.limb(qj)
        s_rot = ckks.automorphism(s_j, ctx.log_n, k, qj)
        lhs = ckks.add_mod(d0[j], ctx.mul(d1[j], s_j, j), qj)
        diff[j] = ckks.sub_mod(lhs, ctx.mul(c[j], s_rot, j), qj)
    err = ctx.crt(diff, ctx.q[: level + 1])
    # noise: ModDown rounding (<= alpha*(1 + ||s||_1)) + digit*e/P terms, far below 2^20
    assert max(abs(e) for e in err) < 2**20, max(abs(e) for e in err)


@pytest.mark.parametrize("level", [1, 2, 3])
def test_relinearisation_output_decrypts_to_c_times_s_squared(level):
    """KS with the relinearisation key: d0 + d1*s = c * s^2 + (small) mod Q_level."""
    ctx = ckks.Context("small4")
    sk = ckks.sample_secret(ctx, 3)
    key = ckks.keygen_relin(ctx, 3, sk)
    rng = np.random.default_rng(10 + level)
    c = np.stack([rng.integers(0, ctx.q[j], size=ctx.n, dtype=np.uint64) for j in range(level + 1)])
    d0, d1 = ckks.keyswitch(ctx, c, level, key)
    diff = np.zeros((level + 1, ctx.n), dtype=np.uint64)
    for j in range(level + 1):
        qj = ctx.q[j]
        s_j = sk.limb(qj)
        lhs = ckks.add_mod(d0[j], ctx.mul(d1[j], s_j, j), qj)
        diff[j] = ckks.sub_mod(lhs, ctx.mul(c[j], ctx.mul(s_j, s_j, j), j), qj)
    err = ctx.crt(diff, ctx.q[: level + 1])
    assert max(abs(e) for e in err) < 2**20, max(abs(e) for e in err)


def test_tensor_product_decrypts_to_the_product_of_messages():
    """(d0 + d1 s + d2 s^2) = (a0 + a1 s)(b0 + b1 s) exactly in Z_Q[X]/(X^N + 1):
    both sides as centred integers, the right side a schoolbook negacyclic product."""
    ctx = ckks.Context(ckks.Params(6, (50, 40, 40), (50,), dnum=1))
    sk = ckks.sample_secret(ctx, 5)
    ev = ckks.Evaluator(ctx, {})
    rng = np.random.default_rng(3)
    lv = 2
    rnd = lambda: np.stack([rng.integers(0, ctx.q[j], size=ctx.n, dtype=np.uint64) for j in range(lv + 1)])
    a = ckks.Ciphertext(rnd(), rnd(), lv, 1.0)
    b = ckks.Ciphertext(rnd(), rnd(), lv, 1.0)
    t = ev.tensor(a, b)
    Q = math.prod(ctx.q[: lv + 1])
    s = [int(x) for x in sk.coeffs]
    dec = lambda c0, c1: [x % Q for x in ctx.crt(np.stack([ckks.add_mod(c0[j], ctx.mul(c1[j], sk.limb(ctx.q[j]), j),
                                                                        ctx.q[j]) for j in range(lv + 1)]),
                                               ctx.q[: lv + 1])]
    ma, mb = dec(a.c0, a.c1), dec(b.c0, b.c1)
    want = micro.schoolbook_negacyclic(ma, mb, Q)
    # d0 + d1 s + d2 s^2 with big integers
    ci = lambda x: [v % Q for v in ctx.crt(x, ctx.q[: lv + 1])]
    d0, d1, d2 = ci(t.d0), ci(t.d1), ci(t.d2)
    s2 = micro.schoolbook_negacyclic(s, s, Q)
    got = [(x + y + z) % Q for x, y, z in zip(d0, micro.schoolbook_negacyclic(d1, s, Q),
                                              micro.schoolbook_negacyclic(d2, s2, Q))]
    assert got == want
