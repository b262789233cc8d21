// bm_math.cuh -- 64-bit modular arithmetic shared by the host and device code
// of the Blind-Match GPU library (RNS-CKKS, Sec. 2 of the paper).
//
// Residues live in 64-bit words, moduli are primes below 2^61.
//  * Shoup multiplication by a constant w with companion w' = floor(w*2^64/q)
//    (V. Shoup, NTL): one high and two low 64-bit products, result in [0, 2q)
//    for any x < 2^64.
//  * Montgomery multiplication with R = 2^64 (P. Montgomery, 1985): used for
//    variable x variable products where one operand is stored pre-multiplied
//    by R (rotation keys, plaintexts), result in [0, 2q) when a*b < q*2^64.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define BM_HD __host__ __device__ __forceinline__
#else
#define BM_HD inline
#endif

namespace bm {

BM_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// x * w mod q, lazily in [0, 2q); w' = floor(w * 2^64 / q).
BM_HD uint64_t shoup_lazy(uint64_t x, uint64_t w, uint64_t wsh, uint64_t q) {
    return x * w - mulhi64(x, wsh) * q;
}
BM_HD uint64_t shoup(uint64_t x, uint64_t w, uint64_t wsh, uint64_t q) {
    uint64_t r = shoup_lazy(x, w, wsh, q);
    return r >= q ? r - q : r;
}

// a * b * 2^-64 mod q, lazily in [0, 2q); qneg = -q^{-1} mod 2^64.
BM_HD uint64_t mont_lazy(uint64_t a, uint64_t b, uint64_t q, uint64_t qneg) {
    uint64_t lo = a * b;
    uint64_t hi = mulhi64(a, b);
    uint64_t m = lo * qneg;
    return hi + mulhi64(m, q) + (lo != 0);
}
BM_HD uint64_t mont(uint64_t a, uint64_t b, uint64_t q, uint64_t qneg) {
    uint64_t r = mont_lazy(a, b, q, qneg);
    return r >= q ? r - q : r;
}

// Sums of products, reduced once: the 128-bit sum t of products a*b (a < 4q, b < q,
// q < 2^62, so the high word of a*b is below q) is
// kept below q * 2^64 by subtracting q from its high word whenever that word
// reaches q (t changes by a multiple of q * 2^64, so t mod q does not); one
// Montgomery reduction then gives t * 2^-64 mod q -- the same residue as the sum
// of the Montgomery products, for one reduction instead of one per product.
struct Acc128 {
    uint64_t lo = 0, hi = 0;
};
BM_HD void mul_acc(Acc128& t, uint64_t a, uint64_t b, uint64_t q) {
    const uint64_t lo = a * b, hi = mulhi64(a, b);   // hi < 4q^2 / 2^64 < q
    t.lo += lo;
    t.hi += hi + (t.lo < lo);                        // < 2q
    if (t.hi >= q) t.hi -= q;
}
BM_HD uint64_t redc(const Acc128& t, uint64_t q, uint64_t qneg) {   // t < q * 2^64
    const uint64_t m = t.lo * qneg;
    const uint64_t r = t.hi + mulhi64(m, q) + (t.lo != 0);         // (t + m q) / 2^64 < 2q
    return r >= q ? r - q : r;
}

// Sums of products without a reduction per product: t += a * b as a 128-bit sum
// (a, b < 2^61, so each product is below 2^122 and 64 of them stay below 2^128).
// On the device the full 64 x 64 -> 128-bit product is added by three carry
// chains of 32 x 32-bit multiply-adds (eight multiply-adds, two carry adds);
// reduce_hi keeps longer sums in range, redc_wide reduces the sum once.
BM_HD void mad128(Acc128& t, uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    uint32_t a0, a1, b0, b1, t0, t1, t2, t3;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(a0), "=r"(a1) : "l"(a));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(b0), "=r"(b1) : "l"(b));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(t0), "=r"(t1) : "l"(t.lo));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(t2), "=r"(t3) : "l"(t.hi));
    asm("mad.lo.cc.u32 %0, %4, %6, %0;\n\t"     // low halves: a0 b0 @0, a0 b1 @32, a1 b1 @64
        "madc.lo.cc.u32 %1, %4, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"
        "addc.u32 %3, %3, 0;\n\t"
        "mad.hi.cc.u32 %1, %4, %6, %1;\n\t"      // high halves: a0 b0 @32, a0 b1 @64, a1 b1 @96
        "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
        "madc.hi.u32 %3, %5, %7, %3;\n\t"
        "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"      // a1 b0: low half @32, high half @64
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3)
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(t.lo) : "r"(t0), "r"(t1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(t.hi) : "r"(t2), "r"(t3));
#else
    const unsigned __int128 s = ((unsigned __int128)t.hi << 64 | t.lo) + (unsigned __int128)a * b;
    t.lo = (uint64_t)s;
    t.hi = (uint64_t)(s >> 64);
#endif
}
// the high word reduced below q (t changes by a multiple of q * 2^64, so t mod q
// and its Montgomery reduction do not); rsh = floor(2^64 / q)
BM_HD void reduce_hi(Acc128& t, uint64_t q, uint64_t rsh) {
    uint64_t h = t.hi - mulhi64(t.hi, rsh) * q;        // [0, 2q)
    t.hi = h >= q ? h - q : h;
}
// t * 2^-64 mod q for any 128-bit t
BM_HD uint64_t redc_wide(Acc128 t, uint64_t q, uint64_t qneg, uint64_t rsh) {
    reduce_hi(t, q, rsh);
    return redc(t, q, qneg);
}

// Sums of products by 30-bit pieces, for a, b < q < 2^60: a = a1 * 2^30 + a0 with
// a0, a1 < 2^30, and the sum t = hi * 2^60 + mid * 2^30 + lo held as three 64-bit
// sums of 32 x 32-bit products, one multiply-add each: lo gains a0*b0 < 2^60, mid
// a0*b1 + a1*b0 < 2^61, hi a1*b1 < q^2 / 2^60 < q per product.  fold60 every
// kFold60Every = 8 products moves lo's and mid's bits above 30 up a sum (lo then
// stays below 2^63, mid below 2^64 - 2^34) and keeps hi below 8q by subtracting 8q
// (hi below 16q < 2^64 before the fold), i.e. q * 2^63 from t, which leaves t mod q
// unchanged.
constexpr int kFold60Every = 8;
struct Piece30 {
    uint32_t l, h;
};
BM_HD Piece30 piece30(uint64_t a) { return {(uint32_t)a & 0x3fffffffu, (uint32_t)(a >> 30)}; }
// the pieces stored in one word (low piece in bits 0..29, high piece in bits 32..63)
BM_HD uint64_t pack30(uint64_t a) { return ((a >> 30) << 32) | (a & 0x3fffffffull); }
BM_HD Piece30 unpack30(uint64_t w) { return {(uint32_t)w, (uint32_t)(w >> 32)}; }
struct Acc60 {
    uint64_t lo = 0, mid = 0, hi = 0;
};
// acc += a * b (32 x 32 -> 64 bits).  On the device as the low and high halves of
// the product added through the carry flag (two full-rate integer multiply-adds,
// measured about 1.25x the throughput of one 64-bit-result multiply-add).
BM_HD void mac32(uint64_t& acc, uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    uint32_t lo = (uint32_t)acc, hi = (uint32_t)(acc >> 32);
    asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;" : "+r"(lo), "+r"(hi) : "r"(a), "r"(b));
    acc = ((uint64_t)hi << 32) | lo;
#else
    acc += (uint64_t)a * b;
#endif
}
BM_HD void mul_add(Acc60& t, Piece30 a, Piece30 b) {
    mac32(t.lo, a.l, b.l);
    mac32(t.mid, a.l, b.h);
    mac32(t.mid, a.h, b.l);
    mac32(t.hi, a.h, b.h);
}
BM_HD void fold60(Acc60& t, uint64_t q8) {
    t.mid += t.lo >> 30;
    t.lo &= 0x3fffffffull;
    t.hi += t.mid >> 30;
    t.mid &= 0x3fffffffull;
    if (t.hi >= q8) t.hi -= q8;
}
// t * 2^-64 mod q: after a fold, t < 8q * 2^60 + 2^60 + 2^30, so the high word of the
// 128-bit value is below q
BM_HD uint64_t redc(Acc60 t, uint64_t q, uint64_t qneg) {
    fold60(t, 8 * q);
    Acc128 r;
    const uint64_t top = t.hi << 60;
    r.lo = t.lo + (t.mid << 30);                 // < 2^60 + 2^30: no carry
    r.lo += top;
    r.hi = (t.hi >> 4) + (r.lo < top);
    return redc(r, q, qneg);
}

BM_HD uint64_t reduce2(uint64_t x, uint64_t q) { return x >= q ? x - q : x; }
BM_HD uint64_t addm(uint64_t a, uint64_t b, uint64_t q) { return reduce2(a + b, q); }
BM_HD uint64_t subm(uint64_t a, uint64_t b, uint64_t q) { return a >= b ? a - b : a + q - b; }
BM_HD uint64_t negm(uint64_t a, uint64_t q) { return a ? q - a : 0; }

// ---- host-only helpers (128-bit integer arithmetic) ----
inline uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((unsigned __int128)a * b) % q);
}
inline uint64_t h_powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    for (; e; e >>= 1) {
        if (e & 1) r = h_mulmod(r, a, q);
        a = h_mulmod(a, a, q);
    }
    return r;
}
inline uint64_t h_invmod(uint64_t a, uint64_t q) { return h_powmod(a, q - 2, q); }
inline uint64_t h_shoup_companion(uint64_t w, uint64_t q) {
    return (uint64_t)(((unsigned __int128)w << 64) / q);
}
// -q^{-1} mod 2^64 by Newton iteration (q odd).
inline uint64_t h_mont_qneg(uint64_t q) {
    uint64_t inv = q;                 // correct to 3 bits for odd q
    for (int i = 0; i < 6; i++) inv *= 2 - q * inv;
    return (uint64_t)0 - inv;
}
// a^{-1} mod m for odd a and m a power of two (m <= 2^63)
inline uint64_t h_invmod_pow2(uint64_t a, uint64_t m) {
    uint64_t inv = a;
    for (int i = 0; i < 6; i++) inv *= 2 - a * inv;
    return inv & (m - 1);
}
// 2^64 mod q, 2^128 mod q
inline uint64_t h_r1(uint64_t q) { return (uint64_t)(((unsigned __int128)1 << 64) % q); }
inline uint64_t h_r2(uint64_t q) { return h_mulmod(h_r1(q), h_r1(q), q); }

}  // namespace bm
