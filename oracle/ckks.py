"""RNS-CKKS oracle (TEST INFRASTRUCTURE ONLY).

Plain CPU CKKS for the Blind-Match match path, written from the paper's
definitions (Sec. 2 "Homomorphic Encryption": Add, Mul(P), Rot, Res) with the
readings the paper leaves open fixed explicitly:

* primes: the largest primes below 2^bits with q = 1 (mod 2N); the paper is
  silent on moduli (Sec. 5.1 names only N = 8192, log PQ ~ 158, l = 3);
* slot j <-> the root zeta^(5^j) (zeta = exp(i*pi/N)), so Rot(v, r) with r > 0
  is the left rotation of Sec. 2 ("(v_r, v_(r+1), ...)");
* rescale rounds to nearest (centred lift of the dropped limb);
* rotation = Galois automorphism sigma_(5^r) followed by hybrid key switching
  (ModUp with the non-centred fast base conversion, inner product with the
  rotation key, ModDown), digits of the modulus chain, automorphism applied
  before ModUp;
* randomness from Philox4x64-10 with the samplers documented in ckks_oracle.c.

Ciphertexts and plaintexts are kept in coefficient form, one uint64 row per
RNS limb; products go through the C core's NTT.  Only tests, the smoke check
and the benchmark's CPU-baseline leg may import this module.
"""
import ctypes
import math
from dataclasses import dataclass, field

import numpy as np

from . import build_oracle

# Philox key tags (key = (seed, tag)); see the samplers in ckks_oracle.c.
TAG_SECRET = 1
TAG_PK_A = 2
TAG_PK_E = 3
TAG_RK_A = 4
TAG_RK_E = 5
TAG_ENC_V = 6
TAG_ENC_E0 = 7
TAG_ENC_E1 = 8
TAG_RLK_A = 9
TAG_RLK_E = 10

_U64P = ctypes.POINTER(ctypes.c_uint64)
_I64P = ctypes.POINTER(ctypes.c_int64)
_LIB = None


def lib():
    """Load (building if needed) the oracle's C core."""
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(build_oracle.build())
        u64, u32, i32, dbl = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
        sig = {
            "orc_powmod": (u64, [u64, u64, u64]),
            "orc_invmod": (u64, [u64, u64]),
            "orc_is_prime": (i32, [u64]),
            "orc_gen_primes": (i32, [u32, u32, u32, _U64P, u32, _U64P]),
            "orc_find_psi": (u64, [u64, u32]),
            "orc_ntt": (None, [_U64P, u32, u64, u64]),
            "orc_intt": (None, [_U64P, u32, u64, u64]),
            "orc_pointwise_mul": (None, [_U64P, _U64P, _U64P, u64, u64]),
            "orc_scalar_mul": (None, [_U64P, u64, _U64P, u64, u64]),
            "orc_poly_mul": (None, [_U64P, _U64P, _U64P, u32, u64, u64]),
            "orc_automorphism": (None, [_U64P, _U64P, u32, u64, u64]),
            "orc_bconv": (None, [_U64P, _U64P, u32, u64, _U64P, u64]),
            "orc_rescale": (None, [_U64P, _U64P, u32, _U64P, u64]),
            "orc_philox4x64": (None, [u64, u64, _U64P, _U64P]),
            "orc_sample_uniform": (None, [u64, u64, u64, u64, u64, _U64P, u64]),
            "orc_cdt_table": (None, [dbl, u32, _U64P]),
            "orc_sample_gauss": (None, [u64, u64, u64, dbl, u32, _I64P, u64]),
            "orc_sample_zo": (None, [u64, u64, u64, _I64P, u64]),
            "orc_sample_hw": (None, [u64, u64, u32, u32, _I64P]),
            "orc_signed_to_mod": (None, [_I64P, u64, _U64P, u64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _p(a):
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.uint64:
        return a.ctypes.data_as(_U64P)
    if a.dtype == np.int64:
        return a.ctypes.data_as(_I64P)
    raise TypeError(a.dtype)


def _u64(shape):
    return np.zeros(shape, dtype=np.uint64)


# ---------------------------------------------------------------------------
# scalar helpers on the C core
# ---------------------------------------------------------------------------

def is_prime(n):
    return bool(lib().orc_is_prime(n))


def philox4x64(k0, k1, ctr):
    c = np.array(ctr, dtype=np.uint64)
    out = _u64(4)
    lib().orc_philox4x64(k0, k1, _p(c), _p(out))
    return [int(x) for x in out]


def cdt_table(sigma, kmax):
    t = _u64(kmax + 1)
    lib().orc_cdt_table(sigma, kmax, _p(t))
    return [int(x) for x in t]


def ntt(a, log_n, q, psi):
    out = np.ascontiguousarray(a, dtype=np.uint64).copy()
    lib().orc_ntt(_p(out), log_n, q, psi)
    return out


def intt(a, log_n, q, psi):
    out = np.ascontiguousarray(a, dtype=np.uint64).copy()
    lib().orc_intt(_p(out), log_n, q, psi)
    return out


def pointwise_mul(a, b, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    out = np.empty_like(a)
    lib().orc_pointwise_mul(_p(a), _p(b), _p(out), a.size, q)
    return out


def scalar_mul(a, c, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.empty_like(a)
    lib().orc_scalar_mul(_p(a), c % q, _p(out), a.size, q)
    return out


def poly_mul(a, b, log_n, q, psi):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    out = np.empty_like(a)
    lib().orc_poly_mul(_p(a), _p(b), _p(out), log_n, q, psi)
    return out


def automorphism(a, log_n, k, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.empty_like(a)
    lib().orc_automorphism(_p(a), _p(out), log_n, k, q)
    return out


def bconv(x, src_primes, t):
    """Fast base conversion of the limbs x (len(src_primes), n) to prime t."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    src = np.array(src_primes, dtype=np.uint64)
    out = _u64(x.shape[1])
    lib().orc_bconv(_p(x), _p(src), len(src_primes), t, _p(out), x.shape[1])
    return out


def rescale_poly(x, primes, level):
    """Res on one polynomial with limbs q_0..q_level -> limbs q_0..q_(level-1)."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    pr = np.array(primes, dtype=np.uint64)
    out = _u64((level, x.shape[1]))
    lib().orc_rescale(_p(x), _p(pr), level, _p(out), x.shape[1])
    return out


def add_mod(a, b, q):
    s = a + b
    return np.where(s >= np.uint64(q), s - np.uint64(q), s)


def sub_mod(a, b, q):
    return np.where(a >= b, a - b, a + np.uint64(q) - b)


def neg_mod(a, q):
    return np.where(a == 0, a, np.uint64(q) - a)


def signed_to_mod(v, q):
    v = np.ascontiguousarray(v, dtype=np.int64)
    out = _u64(v.size)
    lib().orc_signed_to_mod(_p(v), q, _p(out), v.size)
    return out


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Params:
    """RNS-CKKS parameter set.

    q_bits[0] is the base prime, q_bits[1:] the rescale primes (dropped in the
    order q_L, q_(L-1), ...); p_bits are the special primes of key switching;
    dnum is the number of key-switching digits; secret_hw = 0 selects the
    ZO(1/2) ternary secret, otherwise a ternary secret of that Hamming weight.
    """
    log_n: int
    q_bits: tuple
    p_bits: tuple
    dnum: int
    log_scale: int = 40
    secret_hw: int = 0
    sigma: float = 3.2
    kmax: int = 19


PRESETS = {
    # Toy, not secure: ring 2^12, q0 50-bit + one 40-bit rescale prime, one 50-bit special prime.
    "toy": Params(12, (50, 40), (50,), dnum=2, secret_hw=0),
    # Face/fingerprint scale: ring 2^16, 60 + 3x40-bit chain, 2x60-bit special primes, dnum 2, HW 192.
    "ring16": Params(16, (60, 40, 40, 40), (60, 60), dnum=2, secret_hw=192),
    # The ring16 modulus layout on a 2^12 ring: same level plan, fast enough for CPU tests.
    "small4": Params(12, (60, 40, 40, 40), (60, 60), dnum=2, secret_hw=192),
}


def gen_chain(log_n, q_bits, p_bits):
    """Q primes in q_bits order, then P primes; each the largest unused prime < 2^bits, = 1 mod 2N."""
    used = []
    out = []
    for bits in list(q_bits) + list(p_bits):
        excl = np.array(used if used else [0], dtype=np.uint64)
        got = _u64(1)
        n = lib().orc_gen_primes(log_n, bits, 1, _p(excl), len(used), _p(got))
        if n != 1:
            raise ValueError(f"no prime of {bits} bits for N=2^{log_n}")
        used.append(int(got[0]))
        out.append(int(got[0]))
    return out[: len(q_bits)], out[len(q_bits):]


class Context:
    """Primes, roots and derived constants of one parameter set."""

    def __init__(self, params):
        if isinstance(params, str):
            params = PRESETS[params]
        self.params = params
        self.log_n = params.log_n
        self.n = 1 << params.log_n
        self.slots = self.n // 2
        self.q, self.p = gen_chain(params.log_n, params.q_bits, params.p_bits)
        self.L = len(self.q) - 1
        self.alpha = len(self.p)
        self.primes = self.q + self.p                 # full basis Q_L u P
        self.psi = [lib().orc_find_psi(x, self.log_n) for x in self.primes]
        self.dnum = params.dnum
        dsize = -(-(self.L + 1) // self.dnum)
        self.digits = [list(range(d * dsize, min((d + 1) * dsize, self.L + 1)))
                       for d in range(self.dnum)]
        self.P = math.prod(self.p)
        self.scale = float(1 << params.log_scale)
        self.slot_exp = np.array([pow(5, j, 2 * self.n) for j in range(self.slots)], dtype=np.int64)

    # index helpers -----------------------------------------------------
    def level_primes(self, level):
        return self.q[: level + 1]

    def ext_index(self, level):
        """Global basis indices of Q_level u P (the extended basis of key switching)."""
        return list(range(level + 1)) + list(range(self.L + 1, self.L + 1 + self.alpha))

    def galois_left(self, r):
        """Galois element of the left rotation by r slots (negative r: right)."""
        return pow(5, r % self.slots, 2 * self.n)

    # NTT on a prime of the full basis -------------------------------------
    def ntt(self, a, gi):
        return ntt(a, self.log_n, self.primes[gi], self.psi[gi])

    def intt(self, a, gi):
        return intt(a, self.log_n, self.primes[gi], self.psi[gi])

    def mul(self, a, b, gi):
        return poly_mul(a, b, self.log_n, self.primes[gi], self.psi[gi])

    # encoding (canonical embedding on the slots zeta^(5^j)) -----------------
    def encode_int(self, z, scale):
        """Integer coefficients round(scale * tau^{-1}(z)), round half away from zero."""
        n = self.n
        z = np.asarray(z, dtype=np.complex128)
        assert z.shape == (self.slots,)
        v = np.zeros(n, dtype=np.complex128)
        e = self.slot_exp
        v[(e - 1) // 2] = z                           # value at zeta^(5^j)
        v[(2 * n - e - 1) // 2] = np.conj(z)          # value at zeta^(-5^j)
        k = np.arange(n)
        # v[t] = m(zeta^(2t+1)) = sum_k (m_k zeta^k) omega^(tk), omega = zeta^2
        w = np.fft.fft(v) / n                          # = m_k zeta^k
        m = (w * np.exp(-1j * np.pi * k / n)).real * float(scale)
        r = np.where(m >= 0, np.floor(m + 0.5), -np.floor(-m + 0.5))
        return r.astype(np.int64)

    def encode(self, z, scale, level):
        """Plaintext limbs (level+1, N) of z at the given scale."""
        c = self.encode_int(z, scale)
        return Plaintext(np.stack([signed_to_mod(c, self.q[j]) for j in range(level + 1)]),
                         level, float(scale))

    def decode(self, coeffs, scale):
        """Slots z_j = m(zeta^(5^j)) / scale of integer coefficients (any ints)."""
        n = self.n
        p = np.array([float(c) for c in coeffs], dtype=np.float64) / float(scale)
        k = np.arange(n)
        w = p * np.exp(1j * np.pi * k / n)
        v = np.fft.ifft(w) * n
        return v[(self.slot_exp - 1) // 2]

    # exact integers from residues ------------------------------------------
    def crt(self, limbs, primes):
        """Centred integers (python ints) of the residues limbs[j] mod primes[j]."""
        Q = math.prod(primes)
        acc = np.zeros(limbs.shape[1], dtype=object)
        for j, qj in enumerate(primes):
            hat = Q // qj
            coef = hat * pow(hat % qj, -1, qj)
            acc = acc + limbs[j].astype(object) * coef
        acc = acc % Q
        return [int(x) - Q if x > Q // 2 else int(x) for x in acc]


@dataclass
class Plaintext:
    limbs: np.ndarray       # (level+1, N) coefficient form
    level: int
    scale: float


@dataclass
class Ciphertext:
    c0: np.ndarray          # (level+1, N) coefficient form
    c1: np.ndarray
    level: int
    scale: float

    def copy(self):
        return Ciphertext(self.c0.copy(), self.c1.copy(), self.level, self.scale)


@dataclass
class SecretKey:
    coeffs: np.ndarray      # int64 ternary, length N

    def limb(self, q):
        return signed_to_mod(self.coeffs, q)


@dataclass
class PublicKey:
    b: np.ndarray           # (L+1, N)
    a: np.ndarray


@dataclass
class RotationKey:
    galois: int
    data: np.ndarray                          # (dnum, 2, L+1+alpha, N) coefficient form
    ntt_data: np.ndarray = field(default=None, repr=False)


# ---------------------------------------------------------------------------
# sampling
# ---------------------------------------------------------------------------

def sample_uniform(ctx, seed, tag, obj, gi):
    out = _u64(ctx.n)
    lib().orc_sample_uniform(seed, tag, obj, gi, ctx.primes[gi], _p(out), ctx.n)
    return out


def sample_gauss(ctx, seed, tag, obj):
    out = np.zeros(ctx.n, dtype=np.int64)
    lib().orc_sample_gauss(seed, tag, obj, ctx.params.sigma, ctx.params.kmax, _p(out), ctx.n)
    return out


def sample_zo(ctx, seed, tag, obj):
    out = np.zeros(ctx.n, dtype=np.int64)
    lib().orc_sample_zo(seed, tag, obj, _p(out), ctx.n)
    return out


def sample_secret(ctx, seed):
    out = np.zeros(ctx.n, dtype=np.int64)
    if ctx.params.secret_hw:
        lib().orc_sample_hw(seed, TAG_SECRET, ctx.params.secret_hw, ctx.log_n, _p(out))
    else:
        lib().orc_sample_zo(seed, TAG_SECRET, 0, _p(out), ctx.n)
    return SecretKey(out)


# ---------------------------------------------------------------------------
# keys, encryption, decryption (Sec. 3.1: the client keeps sk, sends pk and evk)
# ---------------------------------------------------------------------------

def keygen_public(ctx, seed, sk):
    """pk = (-a*s + e, a) mod Q_L; a uniform (tag PK_A, object 0), e Gaussian (tag PK_E)."""
    e = sample_gauss(ctx, seed, TAG_PK_E, 0)
    b = _u64((ctx.L + 1, ctx.n))
    a = _u64((ctx.L + 1, ctx.n))
    for j in range(ctx.L + 1):
        qj = ctx.q[j]
        a[j] = sample_uniform(ctx, seed, TAG_PK_A, 0, j)
        b[j] = add_mod(neg_mod(ctx.mul(a[j], sk.limb(qj), j), qj), signed_to_mod(e, qj), qj)
    return PublicKey(b, a)


def rotation_key_object(galois, digit):
    return galois * 16 + digit


def keygen_rotation(ctx, seed, sk, galois):
    """Hybrid key-switching key from sigma_k(s) to s, one component pair per digit d:
    b_d = -a_d*s + e_d + P * [Q_hat_d * (Q_hat_d^{-1} mod Q_d)] * sigma_k(s)  mod P*Q_L,
    a_d uniform.  The gadget factor is P mod q_j on the limbs of digit d and 0 elsewhere."""
    nb = ctx.L + 1 + ctx.alpha
    data = _u64((ctx.dnum, 2, nb, ctx.n))
    s_rot = None
    for d, dl in enumerate(ctx.digits):
        obj = rotation_key_object(galois, d)
        e = sample_gauss(ctx, seed, TAG_RK_E, obj)
        for gi in range(nb):
            t = ctx.primes[gi]
            s_t = sk.limb(t)
            a = sample_uniform(ctx, seed, TAG_RK_A, obj, gi)
            b = add_mod(neg_mod(ctx.mul(a, s_t, gi), t), signed_to_mod(e, t), t)
            if gi in dl:
                s_rot = automorphism(s_t, ctx.log_n, galois, t)
                b = add_mod(b, scalar_mul(s_rot, ctx.P % t, t), t)
            data[d, 0, gi] = b
            data[d, 1, gi] = a
    key = RotationKey(galois, data)
    key.ntt_data = np.stack([np.stack([np.stack([ctx.ntt(data[d, c, gi], gi) for gi in range(nb)])
                                       for c in range(2)]) for d in range(ctx.dnum)])
    return key


def keygen_relin(ctx, seed, sk):
    """Relinearisation key (the evaluation key of Mul, Sec. 3.1): the hybrid
    key-switching key from s^2 to s -- the rotation-key construction with
    sigma_k(s) replaced by s^2 (tags RLK_A / RLK_E, object = digit)."""
    nb = ctx.L + 1 + ctx.alpha
    data = _u64((ctx.dnum, 2, nb, ctx.n))
    for d, dl in enumerate(ctx.digits):
        e = sample_gauss(ctx, seed, TAG_RLK_E, d)
        for gi in range(nb):
            t = ctx.primes[gi]
            s_t = sk.limb(t)
            a = sample_uniform(ctx, seed, TAG_RLK_A, d, gi)
            b = add_mod(neg_mod(ctx.mul(a, s_t, gi), t), signed_to_mod(e, t), t)
            if gi in dl:
                b = add_mod(b, scalar_mul(ctx.mul(s_t, s_t, gi), ctx.P % t, t), t)
            data[d, 0, gi] = b
            data[d, 1, gi] = a
    key = RotationKey(1, data)
    key.ntt_data = np.stack([np.stack([np.stack([ctx.ntt(data[d, c, gi], gi) for gi in range(nb)])
                                       for c in range(2)]) for d in range(ctx.dnum)])
    return key


def keygen(ctx, seed, rotations):
    """sk, pk and the rotation keys for the given left-rotation amounts (negative = right)."""
    sk = sample_secret(ctx, seed)
    pk = keygen_public(ctx, seed, sk)
    rks = {}
    for r in rotations:
        k = ctx.galois_left(r)
        if k not in rks:
            rks[k] = keygen_rotation(ctx, seed, sk, k)
    return sk, pk, rks


def encrypt(ctx, pk, pt, seed, obj):
    """ct = (v*b + e0 + m, v*a + e1) mod Q_L with v ~ ZO(1/2), e0, e1 Gaussian (object `obj`)."""
    assert pt.level == ctx.L
    v = sample_zo(ctx, seed, TAG_ENC_V, obj)
    e0 = sample_gauss(ctx, seed, TAG_ENC_E0, obj)
    e1 = sample_gauss(ctx, seed, TAG_ENC_E1, obj)
    c0 = _u64((ctx.L + 1, ctx.n))
    c1 = _u64((ctx.L + 1, ctx.n))
    for j in range(ctx.L + 1):
        qj = ctx.q[j]
        vj = signed_to_mod(v, qj)
        c0[j] = add_mod(add_mod(ctx.mul(vj, pk.b[j], j), signed_to_mod(e0, qj), qj), pt.limbs[j], qj)
        c1[j] = add_mod(ctx.mul(vj, pk.a[j], j), signed_to_mod(e1, qj), qj)
    return Ciphertext(c0, c1, ctx.L, pt.scale)


def decrypt_int(ctx, ct, sk):
    """Centred integer coefficients of c0 + c1*s mod Q_level."""
    m = _u64((ct.level + 1, ctx.n))
    for j in range(ct.level + 1):
        qj = ctx.q[j]
        m[j] = add_mod(ct.c0[j], ctx.mul(ct.c1[j], sk.limb(qj), j), qj)
    return ctx.crt(m, ctx.q[: ct.level + 1])


def decrypt_decode(ctx, ct, sk):
    return ctx.decode(decrypt_int(ctx, ct, sk), ct.scale)


# ---------------------------------------------------------------------------
# evaluator: Add, Mul(P), Res, Rot (Sec. 2)
# ---------------------------------------------------------------------------

@dataclass
class Ciphertext3:
    """Tensor product (d0, d1, d2) of two ciphertexts: decrypts as d0 + d1*s + d2*s^2."""
    d0: np.ndarray
    d1: np.ndarray
    d2: np.ndarray
    level: int
    scale: float


class Evaluator:
    """Exact RNS-CKKS evaluator on coefficient-form ciphertexts."""

    def __init__(self, ctx, rot_keys, relin_key=None):
        self.ctx = ctx
        self.keys = rot_keys
        self.relin_key = relin_key

    def zero_like(self, ct, level=None):
        """Encryption of zero: the identity of add (Algorithm 2 starts from it)."""
        return None

    def add(self, a, b):
        if a is None:
            return b.copy()
        if b is None:
            return a.copy()
        assert a.level == b.level and a.scale == b.scale
        c0 = np.stack([add_mod(a.c0[j], b.c0[j], self.ctx.q[j]) for j in range(a.level + 1)])
        c1 = np.stack([add_mod(a.c1[j], b.c1[j], self.ctx.q[j]) for j in range(a.level + 1)])
        return Ciphertext(c0, c1, a.level, a.scale)

    def mul_plain(self, ct, pt):
        assert ct.level == pt.level
        c0 = np.stack([self.ctx.mul(ct.c0[j], pt.limbs[j], j) for j in range(ct.level + 1)])
        c1 = np.stack([self.ctx.mul(ct.c1[j], pt.limbs[j], j) for j in range(ct.level + 1)])
        return Ciphertext(c0, c1, ct.level, ct.scale * pt.scale)

    def tensor(self, a, b):
        """(a0 + a1 s)(b0 + b1 s) = a0 b0 + (a0 b1 + a1 b0) s + a1 b1 s^2, per limb."""
        assert a.level == b.level
        m = self.ctx.mul
        lv, q = a.level, self.ctx.q
        d0 = np.stack([m(a.c0[j], b.c0[j], j) for j in range(lv + 1)])
        d1 = np.stack([add_mod(m(a.c0[j], b.c1[j], j), m(a.c1[j], b.c0[j], j), q[j]) for j in range(lv + 1)])
        d2 = np.stack([m(a.c1[j], b.c1[j], j) for j in range(lv + 1)])
        return Ciphertext3(d0, d1, d2, lv, a.scale * b.scale)

    def add3(self, x, y):
        if x is None:
            return y
        q = self.ctx.q
        f = lambda u, v: np.stack([add_mod(u[j], v[j], q[j]) for j in range(x.level + 1)])
        return Ciphertext3(f(x.d0, y.d0), f(x.d1, y.d1), f(x.d2, y.d2), x.level, x.scale)

    def relinearize(self, t):
        """(d0, d1, d2) -> (d0 + KS(d2)_0, d1 + KS(d2)_1) with the key from s^2 to s."""
        ctx, lv = self.ctx, t.level
        k0, k1 = keyswitch(ctx, t.d2, lv, self.relin_key)
        c0 = np.stack([add_mod(t.d0[j], k0[j], ctx.q[j]) for j in range(lv + 1)])
        c1 = np.stack([add_mod(t.d1[j], k1[j], ctx.q[j]) for j in range(lv + 1)])
        return Ciphertext(c0, c1, lv, t.scale)

    def mul_cipher(self, a, b):
        """Mul of two ciphertexts (Sec. 2): tensor product, then relinearisation."""
        return self.relinearize(self.tensor(a, b))

    def rescale(self, ct):
        assert ct.level >= 1
        ql = self.ctx.q[ct.level]
        c0 = rescale_poly(ct.c0, self.ctx.q, ct.level)
        c1 = rescale_poly(ct.c1, self.ctx.q, ct.level)
        return Ciphertext(c0, c1, ct.level - 1, ct.scale / ql)

    def rotate(self, ct, r):
        """Rot(ct, r): left rotation by r slots (right for r < 0)."""
        if r % self.ctx.slots == 0:
            return ct.copy()
        return self.apply_galois(ct, self.ctx.galois_left(r))

    def rotate_hoisted(self, ct, rs):
        """Rot(ct, r) for every r in rs, sharing one basis extension of c1: the
        extended limbs of c1 (ModUp, NTT form) are computed once; each rotation
        takes their Galois image (an exact permutation of the NTT slots,
        computed here as NTT(sigma_k(INTT(.)))), the inner product with its key,
        ModDown, and adds sigma_k(c0).  Same messages as rotate(); the bits
        differ from it because ModUp runs before the automorphism."""
        ctx, lvl = self.ctx, ct.level
        ext_idx = ctx.ext_index(lvl)
        ext = modup_ntt(ctx, ct.c1, lvl)
        outs = []
        for r in rs:
            if r % ctx.slots == 0:
                outs.append(ct.copy())
                continue
            k = ctx.galois_left(r)
            key = self.keys[k]
            acc = np.zeros((2, len(ext_idx), ctx.n), dtype=np.uint64)
            for d, f_d in ext.items():
                for jj, gi in enumerate(ext_idx):
                    t = ctx.primes[gi]
                    fk = ctx.ntt(automorphism(ctx.intt(f_d[jj], gi), ctx.log_n, k, t), gi)
                    for comp in range(2):
                        acc[comp, jj] = add_mod(acc[comp, jj], pointwise_mul(fk, key.ntt_data[d, comp, gi], t), t)
            d0, d1 = moddown(ctx, acc, lvl)
            c0s = np.stack([automorphism(ct.c0[j], ctx.log_n, k, ctx.q[j]) for j in range(lvl + 1)])
            c0 = np.stack([add_mod(c0s[j], d0[j], ctx.q[j]) for j in range(lvl + 1)])
            outs.append(Ciphertext(c0, d1, lvl, ct.scale))
        return outs

    def rotate_sum_hoisted(self, base, terms):
        """base + sum over terms (ct, r) of Rot(ct, r), every ciphertext at one
        level, with ONE ModDown for the whole sum (double hoisting, Bossuat,
        Mouchet, Troncoso-Pastoriza and Hubaux, Eurocrypt 2021): the c1 of each
        distinct ciphertext is extended once (ModUp, NTT form); the Galois image
        of a term's extension times the term's key is summed over all terms in
        Q_l u P; that sum is moved down once; then base and every term's
        sigma_k(c0) are added.  Adding sigma_k(c0) after ModDown gives the same
        residues as adding P * sigma_k(c0) to the q-limbs before it, since
        ModDown(P*x + y) = x + ModDown(y) exactly.  A term with r = 0 (mod slots)
        adds its ciphertext unrotated.  Same message as base plus the single
        rotations; the bits differ from those by the roundings saved."""
        ctx, lvl = self.ctx, base.level
        ext_idx = ctx.ext_index(lvl)
        c0 = [base.c0[j].copy() for j in range(lvl + 1)]
        c1 = [base.c1[j].copy() for j in range(lvl + 1)]
        acc = np.zeros((2, len(ext_idx), ctx.n), dtype=np.uint64)
        exts = {}
        rotated = False
        for ct, r in terms:
            assert ct.level == lvl
            if r % ctx.slots == 0:
                for j in range(lvl + 1):
                    c0[j] = add_mod(c0[j], ct.c0[j], ctx.q[j])
                    c1[j] = add_mod(c1[j], ct.c1[j], ctx.q[j])
                continue
            rotated = True
            k = ctx.galois_left(r)
            key = self.keys[k]
            if id(ct) not in exts:
                exts[id(ct)] = modup_ntt(ctx, ct.c1, lvl)
            for d, f_d in exts[id(ct)].items():
                for jj, gi in enumerate(ext_idx):
                    t = ctx.primes[gi]
                    fk = ctx.ntt(automorphism(ctx.intt(f_d[jj], gi), ctx.log_n, k, t), gi)
                    for comp in range(2):
                        acc[comp, jj] = add_mod(acc[comp, jj], pointwise_mul(fk, key.ntt_data[d, comp, gi], t), t)
            for j in range(lvl + 1):
                c0[j] = add_mod(c0[j], automorphism(ct.c0[j], ctx.log_n, k, ctx.q[j]), ctx.q[j])
        if rotated:
            d0, d1 = moddown(ctx, acc, lvl)
            for j in range(lvl + 1):
                c0[j] = add_mod(c0[j], d0[j], ctx.q[j])
                c1[j] = add_mod(c1[j], d1[j], ctx.q[j])
        return Ciphertext(np.stack(c0), np.stack(c1), lvl, base.scale)

    def rotate_plaintext(self, pt, r):
        return rotate_plaintext(self.ctx, pt, r)

    def masked_rotate_sums(self, groups):
        """sum over groups (pt, terms) of pt * (sum over terms (ct, r) of Rot(ct, r)),
        every ciphertext at one level, with ONE ModDown for the whole sum: each group's
        rotations are taken in the extended basis Q_l u P before ModDown
        (hoisted_products_ext: sum_d sigma_k(ext_d) * key_k,d + P * sigma_k(c0), a term
        with r = 0 entering as P * ct), summed, multiplied there by the group's plaintext
        (its integer coefficients reduced on every prime of Q_l u P, extend_plaintext),
        summed over the groups and moved down once.  Multiplication by a plaintext is
        slot-wise and the key-switch sums are linear, so the message is that of
        sum_g pt_g * (sum of the single rotations); the plaintext multiplies the sum
        before the rounding of ModDown instead of after it."""
        ctx = self.ctx
        lvl = groups[0][1][0][0].level
        ext_idx = ctx.ext_index(lvl)
        acc = np.zeros((2, len(ext_idx), ctx.n), dtype=np.uint64)
        scale = None
        for pt, terms in groups:
            by_ct = {}
            for ct, r in terms:
                assert ct.level == lvl
                by_ct.setdefault(id(ct), (ct, []))[1].append(r)
                scale = ct.scale * pt.scale
            S = np.zeros_like(acc)
            for ct, rs in by_ct.values():
                E = self.hoisted_products_ext(ct, rs)
                for r in rs:
                    for jj, gi in enumerate(ext_idx):
                        t = ctx.primes[gi]
                        for comp in range(2):
                            S[comp, jj] = add_mod(S[comp, jj], E[r][comp, jj], t)
            X = extend_plaintext(ctx, pt, lvl)
            for jj, gi in enumerate(ext_idx):
                t = ctx.primes[gi]
                for comp in range(2):
                    acc[comp, jj] = add_mod(acc[comp, jj], pointwise_mul(S[comp, jj], X[jj], t), t)
        d0, d1 = moddown(ctx, acc, lvl)
        return Ciphertext(d0, d1, lvl, scale)

    def hoisted_products_ext(self, ct, rs):
        """The rotations of ct by every r in rs kept in the extended basis Q_l u P,
        before ModDown, NTT form: {r: E_r} with E_r[comp] of shape (|Q_l u P|, N).
        E_r = (sum_d sigma_k(ext_d) * key_k,d) + (P * sigma_k(c0) on the q-limbs of
        the first component), so that ModDown(E_r) is Rot(ct, r) of rotate_hoisted;
        r = 0 gives P * ct on the q-limbs and 0 on the special limbs.  One basis
        extension of c1 serves every r."""
        ctx, lvl = self.ctx, ct.level
        ext_idx = ctx.ext_index(lvl)
        ext = modup_ntt(ctx, ct.c1, lvl)
        out = {}
        for r in rs:
            E = np.zeros((2, len(ext_idx), ctx.n), dtype=np.uint64)
            if r % ctx.slots == 0:
                for jj, gi in enumerate(ext_idx[: lvl + 1]):
                    t = ctx.primes[gi]
                    E[0, jj] = ctx.ntt(scalar_mul(ct.c0[gi], ctx.P % t, t), gi)
                    E[1, jj] = ctx.ntt(scalar_mul(ct.c1[gi], ctx.P % t, t), gi)
                out[r] = E
                continue
            k = ctx.galois_left(r)
            key = self.keys[k]
            for d, f_d in ext.items():
                for jj, gi in enumerate(ext_idx):
                    t = ctx.primes[gi]
                    fk = ctx.ntt(automorphism(ctx.intt(f_d[jj], gi), ctx.log_n, k, t), gi)
                    for comp in range(2):
                        E[comp, jj] = add_mod(E[comp, jj], pointwise_mul(fk, key.ntt_data[d, comp, gi], t), t)
            for jj, gi in enumerate(ext_idx[: lvl + 1]):
                t = ctx.primes[gi]
                c0k = automorphism(ct.c0[gi], ctx.log_n, k, t)
                E[0, jj] = add_mod(E[0, jj], ctx.ntt(scalar_mul(c0k, ctx.P % t, t), gi), t)
            out[r] = E
        return out

    def expand_query_fused(self, ct, n_in, s, mask_slots):
        """Algorithm 1 with its key switches and rescale fused: T_i =
        moddown_rescale(e_i) for the e_i of expand_query_ext, the parts of Algorithm 1
        at level L - 1."""
        L = ct.level
        return [Ciphertext(*moddown_rescale(self.ctx, e, L), L - 1, ct.scale)
                for e in self.expand_query_ext(ct, n_in, s, mask_slots)]

    def expand_query_ext(self, ct, n_in, s, mask_slots):
        """Algorithm 1 up to its division, in the extended basis: E_j =
        hoisted_products_ext(ct, j*s) for j < n_in, the masks mask_slots(i) encoded
        at scale q_L with their integer coefficients reduced on every prime of
        Q_L u P, and e_i = sum_j E_j * mask_((i-j) mod n_in) there (NTT form,
        e_i[comp] of shape (|Q_L u P|, N)); e_i / (q_L * P) is part i."""
        ctx, L = self.ctx, ct.level
        ext_idx = ctx.ext_index(L)
        E = self.hoisted_products_ext(ct, [s * j for j in range(n_in)])
        masks = []
        for i in range(n_in):
            c = ctx.encode_int(mask_slots(i), ctx.q[L])
            masks.append([ctx.ntt(signed_to_mod(c, ctx.primes[gi]), gi) for gi in ext_idx])
        outs = []
        for i in range(n_in):
            e = np.zeros((2, len(ext_idx), ctx.n), dtype=np.uint64)
            for j in range(n_in):
                M = masks[(i - j) % n_in]
                for jj, gi in enumerate(ext_idx):
                    t = ctx.primes[gi]
                    for comp in range(2):
                        e[comp, jj] = add_mod(e[comp, jj], pointwise_mul(E[s * j][comp, jj], M[jj], t), t)
            outs.append(e)
        return outs

    def hec3_deferred(self, e_parts, pts, ct):
        """HE-C^3's sum of products on the parts of Algorithm 1 before their division:
        sum_i e_i * pt_i on Q_L u P (L = ct.level; the plaintexts' integer
        coefficients reduced on every prime there, extend_plaintext), divided once by
        q_(L-1) * q_L * P (moddown_rescale with two q-primes dropped): the product of
        Algorithm 2 and its rescale, at level L - 2."""
        ctx, L = self.ctx, ct.level
        ext_idx = ctx.ext_index(L)
        acc = np.zeros((2, len(ext_idx), ctx.n), dtype=np.uint64)
        for e, pt in zip(e_parts, pts):
            X = extend_plaintext(ctx, pt, L)
            for jj, gi in enumerate(ext_idx):
                t = ctx.primes[gi]
                for comp in range(2):
                    acc[comp, jj] = add_mod(acc[comp, jj], pointwise_mul(e[comp, jj], X[jj], t), t)
        c0, c1 = moddown_rescale(ctx, acc, L, drop=2)
        return Ciphertext(c0, c1, L - 2, ct.scale * pts[0].scale / ctx.q[L - 1])

    def apply_galois(self, ct, k):
        ctx, lvl = self.ctx, ct.level
        key = self.keys[k]
        c0s = np.stack([automorphism(ct.c0[j], ctx.log_n, k, ctx.q[j]) for j in range(lvl + 1)])
        c1s = np.stack([automorphism(ct.c1[j], ctx.log_n, k, ctx.q[j]) for j in range(lvl + 1)])
        d0, d1 = keyswitch(ctx, c1s, lvl, key)
        c0 = np.stack([add_mod(c0s[j], d0[j], ctx.q[j]) for j in range(lvl + 1)])
        return Ciphertext(c0, d1, lvl, ct.scale)


def modup_ntt(ctx, c, level):
    """ModUp of c (limbs q_0..q_level, coefficient form) per digit, NTT form:
    {digit: [limb of Q_level u P]} -- the digit's own limbs kept, every other limb
    the fast base conversion of them (as in keyswitch)."""
    ext = ctx.ext_index(level)
    out = {}
    for d, dl in enumerate(ctx.digits):
        dl = [j for j in dl if j <= level]
        if not dl:
            continue
        src_primes = [ctx.q[j] for j in dl]
        src = np.stack([c[j] for j in dl])
        out[d] = [ctx.ntt(c[gi] if gi in dl else bconv(src, src_primes, ctx.primes[gi]), gi) for gi in ext]
    return out


def moddown(ctx, acc, level):
    """(x - Conv_P->q_j([x]_P)) * P^{-1} mod q_j for both components of the inner
    product acc[comp][limb of Q_level u P] (NTT form); coefficient-form outputs."""
    ext = ctx.ext_index(level)
    out = []
    for comp in range(2):
        x = np.stack([ctx.intt(acc[comp, jj], gi) for jj, gi in enumerate(ext)])
        xp = x[level + 1:]
        res = _u64((level + 1, ctx.n))
        for j in range(level + 1):
            qj = ctx.q[j]
            conv = bconv(xp, ctx.p, qj)
            p_inv = pow(ctx.P % qj, -1, qj)
            res[j] = scalar_mul(sub_mod(x[j], conv, qj), p_inv, qj)
        out.append(res)
    return out[0], out[1]


def moddown_rescale(ctx, e, level, drop=1):
    """ModDown and Rescale in one step: e[comp] (limbs of Q_level u P, NTT form) divided
    by S = q_(level-drop+1) * ... * q_level * P with the special set {q_(level-drop+1),
    ..., q_level} u P, out_j = (x_j - Conv_S->q_j([x]_S)) * S^{-1} mod q_j for
    j <= level - drop (coefficient form).  The same fast base conversion as moddown;
    e / S carries the message of e / P rescaled by the dropped q-primes."""
    ext = ctx.ext_index(level)
    nt = level + 1 - drop                                                    # target limbs
    spec = list(range(nt, level + 1 + ctx.alpha))                            # positions in ext
    sp_primes = [ctx.primes[ext[j]] for j in spec]
    S = math.prod(sp_primes)
    out = []
    for comp in range(2):
        x = np.stack([ctx.intt(e[comp, jj], gi) for jj, gi in enumerate(ext)])
        xs = np.stack([x[j] for j in spec])
        res = _u64((nt, ctx.n))
        for j in range(nt):
            qj = ctx.q[j]
            conv = bconv(xs, sp_primes, qj)
            s_inv = pow(S % qj, -1, qj)
            res[j] = scalar_mul(sub_mod(x[j], conv, qj), s_inv, qj)
        out.append(res)
    return out[0], out[1]


def rotate_plaintext(ctx, pt, r):
    """The plaintext of Rot(message, r): the Galois automorphism sigma_(5^r) (left by r,
    right for r < 0) applied to every limb's coefficients -- an exact signed permutation
    of the integer coefficients, the same one the rotation of a ciphertext applies."""
    if r % ctx.slots == 0:
        return Plaintext(pt.limbs.copy(), pt.level, pt.scale)
    k = ctx.galois_left(r)
    limbs = np.stack([automorphism(pt.limbs[j], ctx.log_n, k, ctx.q[j]) for j in range(pt.level + 1)])
    return Plaintext(limbs, pt.level, pt.scale)


def extend_plaintext(ctx, pt, level):
    """The integer coefficients of pt -- the centred residues of its q_0 limb, exact
    while they lie within q_0 / 2 -- reduced on every prime of Q_level u P, NTT form
    (one row per prime of ctx.ext_index(level))."""
    q0 = ctx.q[0]
    v = np.asarray(pt.limbs[0], dtype=np.uint64)
    c = v.astype(np.int64)
    c[v > np.uint64(q0 // 2)] -= np.int64(q0)
    return [ctx.ntt(signed_to_mod(c, ctx.primes[gi]), gi) for gi in ctx.ext_index(level)]


def keyswitch(ctx, c, level, key):
    """Hybrid key switching of the polynomial c (limbs q_0..q_level, coefficient form).

    ModUp: per digit d (limbs of Q_d at or below `level`), the digit's own limbs
    are kept and every other limb of Q_level u P is the fast base conversion
    of those limbs.  Inner product with the key's digit-d pair in the NTT
    domain, summed over digits.  ModDown: out_j = (x_j - Conv_P->q_j([x]_P)) * P^{-1}.
    Returns the two output polynomials (limbs q_0..q_level)."""
    ext = ctx.ext_index(level)                     # global basis indices
    acc = np.zeros((2, len(ext), ctx.n), dtype=np.uint64)
    for d, f_d in modup_ntt(ctx, c, level).items():
        for jj, gi in enumerate(ext):
            t = ctx.primes[gi]
            for comp in range(2):
                acc[comp, jj] = add_mod(acc[comp, jj], pointwise_mul(f_d[jj], key.ntt_data[d, comp, gi], t), t)
    return moddown(ctx, acc, level)
