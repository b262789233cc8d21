/*
 * ckks_oracle.c -- integer core of the CPU oracle for the Blind-Match encrypted
 * 1:N match (RNS-CKKS, Sec. 2 "Homomorphic Encryption" and Sec. 3.3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the GPU path is compared against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, tables or headers with the GPU library.
 *
 * Everything here is plain scalar C with 128-bit products reduced by `%`.
 * Polynomials are arrays of N = 2^log_n residues in [0, q), coefficient
 * order, one array per RNS limb.  The NTT used here is the textbook one:
 * evaluation of a(X) at the odd powers psi^(2i+1), natural output order,
 * computed as a psi-twist followed by a radix-2 cyclic DFT.  The ring
 * operations the paper uses (Add, Mul(P), Rot, Res; Sec. 2) are assembled
 * from these primitives in oracle.py.
 *
 * The randomness conventions (Philox4x64-10 from Salmon et al., SC'11, and
 * the samplers built on it) are the ones both sides implement independently;
 * the paper is silent on all of them (Sec. 3.1 only says keys are generated).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* scalar modular arithmetic                                           */
/* ------------------------------------------------------------------ */

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * b) % q);
}
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t s = a + b;           /* a, b < q < 2^62: no overflow */
    return s >= q ? s - q : s;
}
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : a + q - b;
}
uint64_t orc_powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}
/* inverse modulo a prime q (Fermat) */
uint64_t orc_invmod(uint64_t a, uint64_t q) { return orc_powmod(a, q - 2, q); }

/* Deterministic Miller-Rabin for n < 2^64 (bases 2..37). */
int orc_is_prime(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = orc_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int k = 1; k < r; k++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/*
 * The `count` largest primes p < 2^bits with p = 1 (mod 2N), skipping the
 * ones listed in `excl`, in descending order.  Returns the number found.
 */
int orc_gen_primes(uint32_t log_n, uint32_t bits, uint32_t count,
                   const uint64_t* excl, uint32_t n_excl, uint64_t* out) {
    uint64_t two_n = 2ull << log_n;
    uint64_t p = ((1ull << bits) - 1) / two_n * two_n + 1; /* largest 1 mod 2N below 2^bits */
    if (p >= (1ull << bits)) p -= two_n;
    uint32_t found = 0;
    while (found < count && p > two_n) {
        int skip = 0;
        for (uint32_t i = 0; i < n_excl; i++) if (excl[i] == p) skip = 1;
        if (!skip && orc_is_prime(p)) out[found++] = p;
        p -= two_n;
    }
    return (int)found;
}

/* psi = g^((q-1)/2N) for the smallest g >= 2 with psi^N = -1 (so psi has order 2N). */
uint64_t orc_find_psi(uint64_t q, uint32_t log_n) {
    uint64_t n = 1ull << log_n;
    for (uint64_t g = 2; g < q; g++) {
        uint64_t psi = orc_powmod(g, (q - 1) / (2 * n), q);
        if (orc_powmod(psi, n, q) == q - 1) return psi;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* NTT: A[i] = a(psi^(2i+1)), natural order                             */
/* ------------------------------------------------------------------ */

static void bit_reverse_permute(uint64_t* a, uint64_t n) {
    for (uint64_t i = 1, j = 0; i < n; i++) {
        uint64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

/* In-place cyclic DFT of length n over Z_q with root omega (order n). */
static void cyclic_dft(uint64_t* a, uint64_t n, uint64_t q, uint64_t omega) {
    uint64_t* pw = (uint64_t*)malloc(sizeof(uint64_t) * (n / 2 + 1));
    pw[0] = 1;
    for (uint64_t j = 1; j <= n / 2; j++) pw[j] = mulmod(pw[j - 1], omega, q);
    bit_reverse_permute(a, n);
    for (uint64_t len = 2; len <= n; len <<= 1) {
        uint64_t half = len / 2, step = n / len;
        for (uint64_t i = 0; i < n; i += len) {
            for (uint64_t j = 0; j < half; j++) {
                uint64_t u = a[i + j];
                uint64_t v = mulmod(a[i + j + half], pw[j * step], q);
                a[i + j] = addmod(u, v, q);
                a[i + j + half] = submod(u, v, q);
            }
        }
    }
    free(pw);
}

void orc_ntt(uint64_t* a, uint32_t log_n, uint64_t q, uint64_t psi) {
    uint64_t n = 1ull << log_n, t = 1;
    for (uint64_t k = 0; k < n; k++) { a[k] = mulmod(a[k], t, q); t = mulmod(t, psi, q); }
    cyclic_dft(a, n, q, mulmod(psi, psi, q));
}

void orc_intt(uint64_t* a, uint32_t log_n, uint64_t q, uint64_t psi) {
    uint64_t n = 1ull << log_n;
    uint64_t psi_inv = orc_invmod(psi, q);
    cyclic_dft(a, n, q, mulmod(psi_inv, psi_inv, q));
    uint64_t n_inv = orc_invmod(n % q, q), t = n_inv;
    for (uint64_t k = 0; k < n; k++) { a[k] = mulmod(a[k], t, q); t = mulmod(t, psi_inv, q); }
}

/* out[i] = a[i] * b[i] mod q (pointwise; used on NTT images) */
void orc_pointwise_mul(const uint64_t* a, const uint64_t* b, uint64_t* out, uint64_t n, uint64_t q) {
    for (uint64_t i = 0; i < n; i++) out[i] = mulmod(a[i], b[i], q);
}

/* out[i] = a[i] * c mod q */
void orc_scalar_mul(const uint64_t* a, uint64_t c, uint64_t* out, uint64_t n, uint64_t q) {
    for (uint64_t i = 0; i < n; i++) out[i] = mulmod(a[i], c, q);
}

/* Negacyclic product in Z_q[X]/(X^N+1): out = a*b (via NTT, pointwise, iNTT). */
void orc_poly_mul(const uint64_t* a, const uint64_t* b, uint64_t* out,
                  uint32_t log_n, uint64_t q, uint64_t psi) {
    uint64_t n = 1ull << log_n;
    uint64_t* fa = (uint64_t*)malloc(8 * n);
    uint64_t* fb = (uint64_t*)malloc(8 * n);
    memcpy(fa, a, 8 * n);
    memcpy(fb, b, 8 * n);
    orc_ntt(fa, log_n, q, psi);
    orc_ntt(fb, log_n, q, psi);
    orc_pointwise_mul(fa, fb, out, n, q);
    orc_intt(out, log_n, q, psi);
    free(fa);
    free(fb);
}

/*
 * Galois automorphism sigma_k: a(X) -> a(X^k) in Z_q[X]/(X^N+1), k odd,
 * coefficient domain: coefficient n moves to n*k mod 2N, negated when that
 * exponent is >= N (X^N = -1).
 */
void orc_automorphism(const uint64_t* a, uint64_t* out, uint32_t log_n, uint64_t k, uint64_t q) {
    uint64_t n = 1ull << log_n, two_n = 2 * n;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t e = (uint64_t)(((u128)i * k) % two_n);
        if (e < n) out[e] = a[i];
        else out[e - n] = a[i] == 0 ? 0 : q - a[i];
    }
}

/* ------------------------------------------------------------------ */
/* RNS base conversion and rescale                                      */
/* ------------------------------------------------------------------ */

/*
 * Fast base conversion from basis B = {b_0..b_{k-1}} to a target prime t
 * (the "full-RNS" approximate conversion of Cheon-Han-Kim-Kim-Song 2018):
 *   y = sum_i [x_i * (B/b_i)^{-1}]_{b_i} * (B/b_i mod t)  mod t,
 * which equals x + e*B (mod t) for the integer x in [0, B) and some
 * 0 <= e < k.  x is given as k limbs of length n (x[i*n + c]); the
 * output is one limb of length n.
 */
void orc_bconv(const uint64_t* x, const uint64_t* src, uint32_t k,
               uint64_t t, uint64_t* out, uint64_t n) {
    uint64_t* hat_inv = (uint64_t*)malloc(8 * k);   /* (B/b_i)^{-1} mod b_i */
    uint64_t* hat_t = (uint64_t*)malloc(8 * k);     /* (B/b_i) mod t */
    for (uint32_t i = 0; i < k; i++) {
        uint64_t h = 1, ht = 1;
        for (uint32_t j = 0; j < k; j++) {
            if (j == i) continue;
            h = mulmod(h, src[j] % src[i], src[i]);
            ht = mulmod(ht, src[j] % t, t);
        }
        hat_inv[i] = orc_invmod(h, src[i]);
        hat_t[i] = ht;
    }
    for (uint64_t c = 0; c < n; c++) {
        uint64_t y = 0;
        for (uint32_t i = 0; i < k; i++) {
            uint64_t v = mulmod(x[(uint64_t)i * n + c], hat_inv[i], src[i]);
            y = addmod(y, mulmod(v % t, hat_t[i], t), t);
        }
        out[c] = y;
    }
    free(hat_inv);
    free(hat_t);
}

/*
 * Rescale (Res in Sec. 2): drop the last prime q_l of a polynomial with
 * limbs q_0..q_l (coefficient form, x[j*n + c]):
 *   out_j = (x_j - r) * q_l^{-1} mod q_j,  r = x_l lifted to (-q_l/2, q_l/2),
 * i.e. out = round(x / q_l) exactly (q_l odd, so there is no tie).
 */
void orc_rescale(const uint64_t* x, const uint64_t* primes, uint32_t level,
                 uint64_t* out, uint64_t n) {
    uint64_t ql = primes[level];
    const uint64_t* last = x + (uint64_t)level * n;
    for (uint32_t j = 0; j < level; j++) {
        uint64_t qj = primes[j];
        uint64_t inv = orc_invmod(ql % qj, qj);
        for (uint64_t c = 0; c < n; c++) {
            uint64_t v = last[c];
            uint64_t r;                 /* centred residue of v, reduced mod q_j */
            if (v > ql / 2) r = submod(0, (ql - v) % qj, qj);
            else r = v % qj;
            out[(uint64_t)j * n + c] = mulmod(submod(x[(uint64_t)j * n + c], r, qj), inv, qj);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11)                                          */
/* ------------------------------------------------------------------ */

void orc_philox4x64(uint64_t k0, uint64_t k1, const uint64_t ctr_in[4], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += W0; k1 += W1; }
        u128 p0 = (u128)M0 * c0;
        u128 p1 = (u128)M1 * c2;
        uint64_t n0 = (uint64_t)(p1 >> 64) ^ c1 ^ k0;
        uint64_t n1 = (uint64_t)p1;
        uint64_t n2 = (uint64_t)(p0 >> 64) ^ c3 ^ k1;
        uint64_t n3 = (uint64_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_words(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, uint64_t c,
                         uint64_t w[4]) {
    uint64_t ctr[4] = {a, b, c, 0};
    orc_philox4x64(seed, tag, ctr, w);
}

/*
 * Uniform residues mod q for object `id`, limb index `limb` (index in the
 * full basis Q_L u P):  coefficient i draws (w0, w1) from
 * Philox(key=(seed, tag), ctr=(id, limb, i, 0)) and takes (w1*2^64 + w0) mod q.
 */
void orc_sample_uniform(uint64_t seed, uint64_t tag, uint64_t id, uint64_t limb,
                        uint64_t q, uint64_t* out, uint64_t n) {
    uint64_t w[4];
    for (uint64_t i = 0; i < n; i++) {
        philox_words(seed, tag, id, limb, i, w);
        u128 x = ((u128)w[1] << 64) | w[0];
        out[i] = (uint64_t)(x % q);
    }
}

/*
 * Cumulative table of |e| for the discrete Gaussian of width sigma, cut at
 * |e| <= kmax:  T[k] = floor(2^63 * P(|e| <= k)) for k < kmax, T[kmax] = 2^63,
 * with P(|e| = 0) = rho(0)/Z, P(|e| = k) = 2 rho(k)/Z, rho(k) = exp(-k^2/(2 sigma^2)),
 * Z = rho(0) + 2 sum_{k=1..kmax} rho(k); sums are taken in increasing k.
 */
void orc_cdt_table(double sigma, uint32_t kmax, uint64_t* table) {
    double rho[64];
    double z = 0.0;
    for (uint32_t k = 0; k <= kmax; k++) {
        rho[k] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        z += (k == 0 ? 1.0 : 2.0) * rho[k];
    }
    double acc = 0.0;
    for (uint32_t k = 0; k <= kmax; k++) {
        acc += (k == 0 ? 1.0 : 2.0) * rho[k];
        if (k == kmax) table[k] = 1ull << 63;
        else table[k] = (uint64_t)(acc / z * 9223372036854775808.0);
    }
}

/*
 * Discrete Gaussian coefficients (signed) for object `id`: coefficient i takes
 * w0 of Philox(key=(seed, tag), ctr=(id, 0, i, 0)); |e| = min{k : (w0 >> 1) < T[k]},
 * negative when the low bit of w0 is set.
 */
void orc_sample_gauss(uint64_t seed, uint64_t tag, uint64_t id, double sigma, uint32_t kmax,
                      int64_t* out, uint64_t n) {
    uint64_t table[64];
    uint64_t w[4];
    orc_cdt_table(sigma, kmax, table);
    for (uint64_t i = 0; i < n; i++) {
        philox_words(seed, tag, id, 0, i, w);
        uint64_t u = w[0] >> 1;
        int64_t k = 0;
        while (u >= table[k]) k++;
        out[i] = (w[0] & 1) ? -k : k;
    }
}

/*
 * Ternary ZO(1/2): coefficient i takes w0 of Philox(key=(seed, tag), ctr=(id, 0, i, 0));
 * w0 & 3 in {0, 1} -> 0, 2 -> +1, 3 -> -1.
 */
void orc_sample_zo(uint64_t seed, uint64_t tag, uint64_t id, int64_t* out, uint64_t n) {
    uint64_t w[4];
    for (uint64_t i = 0; i < n; i++) {
        philox_words(seed, tag, id, 0, i, w);
        uint64_t b = w[0] & 3;
        out[i] = b < 2 ? 0 : (b == 2 ? 1 : -1);
    }
}

/*
 * Ternary secret of exact Hamming weight h: draw n = 0, 1, 2, ... takes (w0, w1)
 * of Philox(key=(seed, tag), ctr=(0, 0, n, 0)); position = w0 >> (64 - log_n);
 * if that position is still zero it becomes +1 (w1 even) or -1 (w1 odd).
 * Stops when h positions are set.
 */
void orc_sample_hw(uint64_t seed, uint64_t tag, uint32_t h, uint32_t log_n, int64_t* out) {
    uint64_t n = 1ull << log_n, w[4];
    memset(out, 0, 8 * n);
    uint32_t filled = 0;
    for (uint64_t draw = 0; filled < h; draw++) {
        philox_words(seed, tag, 0, 0, draw, w);
        uint64_t pos = w[0] >> (64 - log_n);
        if (out[pos] == 0) {
            out[pos] = (w[1] & 1) ? -1 : 1;
            filled++;
        }
    }
}

/* signed integers -> residues mod q */
void orc_signed_to_mod(const int64_t* a, uint64_t q, uint64_t* out, uint64_t n) {
    for (uint64_t i = 0; i < n; i++) {
        int64_t v = a[i];
        out[i] = v >= 0 ? (uint64_t)v % q : (q - ((uint64_t)(-v) % q)) % q;
    }
}
