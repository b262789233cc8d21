// host.cpp -- client-side number theory, randomness and encoding of the
// Blind-Match library (host code; the match path itself runs in kernels.cu).
//
//  * NTT-friendly primes: the largest primes below 2^bits with q = 1 (mod 2N),
//    by deterministic Miller-Rabin; psi of order 2N from the smallest base g
//    whose power g^((q-1)/2N) is a root of X^N + 1.
//  * Philox4x64-10 (Salmon et al., "Parallel random numbers: as easy as 1, 2, 3",
//    SC'11) keyed by (seed, tag), counter (object, limb, coefficient, 0), and the
//    samplers on top of it: uniform residues (128 bits reduced mod q), discrete
//    Gaussian by cumulative table on 63 bits with a sign bit, ZO(1/2) ternary,
//    ternary of fixed Hamming weight by rejection of occupied positions.
//  * CKKS canonical embedding (Sec. 2: batches of real -- or complex -- values in the slots):
//    slot j is the evaluation at zeta^(5^j), zeta = exp(i*pi/N).  Encoding maps
//    the slots to the N odd powers of zeta and applies one length-N inverse DFT,
//    computed by an iterative radix-2 FFT.
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "bm_internal.h"

namespace bm {

using u128 = unsigned __int128;

static bool mr_witness(uint64_t n, uint64_t a, uint64_t d, int r) {
    uint64_t x = h_powmod(a, d, n);
    if (x == 1 || x == n - 1) return false;
    for (int i = 1; i < r; i++) {
        x = h_mulmod(x, x, n);
        if (x == n - 1) return false;
    }
    return true;   // a proves n composite
}

bool is_prime_u64(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t p : small) {
        if (n == p) return true;
        if (n % p == 0) return false;
    }
    uint64_t d = n - 1;
    int r = 0;
    while (!(d & 1)) { d >>= 1; r++; }
    for (uint64_t a : small)
        if (mr_witness(n, a, d, r)) return false;
    return true;
}

bool gen_primes(uint32_t log_n, const std::vector<uint32_t>& bits, std::vector<uint64_t>& out) {
    const uint64_t step = 2ull << log_n;
    out.clear();
    for (uint32_t b : bits) {
        uint64_t top = (1ull << b) - 1;
        uint64_t cand = top - (top % step) + 1;   // largest value = 1 mod 2N not above 2^b - 1 ...
        if (cand > top) cand -= step;             // ... kept strictly below 2^b
        bool found = false;
        for (; cand > step; cand -= step) {
            bool used = false;
            for (uint64_t u : out) used |= (u == cand);
            if (!used && is_prime_u64(cand)) { found = true; break; }
        }
        if (!found) return false;
        out.push_back(cand);
    }
    return true;
}

uint64_t find_psi(uint64_t q, uint32_t log_n) {
    const uint64_t n = 1ull << log_n;
    const uint64_t e = (q - 1) / (2 * n);
    for (uint64_t g = 2; g < 1000000; g++) {
        uint64_t w = h_powmod(g, e, q);
        if (h_powmod(w, n, q) == q - 1) return w;
    }
    return 0;
}

void philox4x64_10(uint64_t k0, uint64_t k1, const uint64_t ctr[4], uint64_t out[4]) {
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    for (int round = 0; round < 10; ++round) {
        u128 m0 = (u128)0xD2E7470EE14C6C93ull * x0;
        u128 m1 = (u128)0xCA5A826395121157ull * x2;
        uint64_t y0 = (uint64_t)(m1 >> 64) ^ x1 ^ k0;
        uint64_t y2 = (uint64_t)(m0 >> 64) ^ x3 ^ k1;
        x1 = (uint64_t)m1;
        x3 = (uint64_t)m0;
        x0 = y0;
        x2 = y2;
        k0 += 0x9E3779B97F4A7C15ull;   // key schedule (Weyl sequence)
        k1 += 0xBB67AE8584CAA73Bull;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static inline void draw(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, uint64_t c, uint64_t w[4]) {
    const uint64_t ctr[4] = {a, b, c, 0};
    philox4x64_10(seed, tag, ctr, w);
}

void sample_uniform(uint64_t seed, uint64_t tag, uint64_t obj, uint64_t limb, uint64_t q,
                    uint64_t* out, uint32_t n) {
    uint64_t w[4];
    for (uint32_t i = 0; i < n; i++) {
        draw(seed, tag, obj, limb, i, w);
        out[i] = (uint64_t)((((u128)w[1]) << 64 | w[0]) % q);
    }
}

void cdt_table(double sigma, uint32_t kmax, uint64_t* table) {
    std::vector<double> weight(kmax + 1);
    double total = 0;
    for (uint32_t k = 0; k <= kmax; k++) {
        weight[k] = (k ? 2.0 : 1.0) * std::exp(-double(k) * double(k) / (2.0 * sigma * sigma));
        total += weight[k];
    }
    double run = 0;
    for (uint32_t k = 0; k <= kmax; k++) {
        run += weight[k];
        table[k] = (k == kmax) ? (1ull << 63) : (uint64_t)(run / total * 9223372036854775808.0);
    }
}

void sample_gauss(uint64_t seed, uint64_t tag, uint64_t obj, double sigma, int64_t* out, uint32_t n) {
    const uint32_t kmax = 19;
    uint64_t table[kmax + 1];
    cdt_table(sigma, kmax, table);
    uint64_t w[4];
    for (uint32_t i = 0; i < n; i++) {
        draw(seed, tag, obj, 0, i, w);
        const uint64_t u = w[0] >> 1;
        int64_t mag = 0;
        while (u >= table[mag]) mag++;
        out[i] = (w[0] & 1) ? -mag : mag;
    }
}

void sample_zo(uint64_t seed, uint64_t tag, uint64_t obj, int64_t* out, uint32_t n) {
    static const int64_t lut[4] = {0, 0, 1, -1};
    uint64_t w[4];
    for (uint32_t i = 0; i < n; i++) {
        draw(seed, tag, obj, 0, i, w);
        out[i] = lut[w[0] & 3];
    }
}

void sample_secret(uint64_t seed, uint32_t hw, uint32_t log_n, int64_t* out) {
    const uint32_t n = 1u << log_n;
    if (hw == 0) {
        sample_zo(seed, TAG_SECRET, 0, out, n);
        return;
    }
    std::memset(out, 0, sizeof(int64_t) * n);
    uint64_t w[4];
    uint32_t placed = 0;
    for (uint64_t k = 0; placed < hw; k++) {
        draw(seed, TAG_SECRET, 0, 0, k, w);
        const uint64_t pos = w[0] >> (64 - log_n);
        if (out[pos] != 0) continue;
        out[pos] = (w[1] & 1) ? -1 : 1;
        placed++;
    }
}

// ---- FFT-based encoder ----

using cplx = std::complex<double>;

void encoder_tables(Context& ctx) {
    const uint32_t n = ctx.n;
    EncoderTables& T = ctx.enc;
    T.root.resize(n / 2);
    for (uint32_t k = 0; k < n / 2; k++) T.root[k] = std::polar(1.0, 2.0 * M_PI * double(k) / double(n));
    T.brv.resize(n);
    for (uint32_t i = 0; i < n; i++) {
        uint32_t r = 0;
        for (uint32_t b = 0; b < ctx.log_n; b++) r |= ((i >> b) & 1u) << (ctx.log_n - 1 - b);
        T.brv[i] = r;
    }
    T.zeta.resize(n);
    for (uint32_t k = 0; k < n; k++) T.zeta[k] = std::polar(1.0, M_PI * double(k) / double(n));
    // slot j <-> odd exponent 5^j mod 2N = 2t+1 (and its conjugate -5^j)
    T.pos.resize(ctx.slots);
    T.cpos.resize(ctx.slots);
    const uint64_t two_n = 2ull * n;
    uint64_t e = 1;
    for (uint32_t j = 0; j < ctx.slots; j++) {
        T.pos[j] = (uint32_t)((e - 1) / 2);
        T.cpos[j] = (uint32_t)((two_n - e - 1) / 2);
        e = (e * 5) % two_n;
    }
}

// In-place iterative radix-2 DFT: X[k] = sum_t x[t] exp(sign * 2 pi i t k / n).
static void fft(const EncoderTables& T, cplx* a, uint32_t n, int sign) {
    for (uint32_t i = 0; i < n; i++)
        if (i < T.brv[i]) std::swap(a[i], a[T.brv[i]]);
    for (uint32_t len = 2; len <= n; len <<= 1) {
        const uint32_t half = len / 2, step = n / len;
        for (uint32_t i = 0; i < n; i += len)
            for (uint32_t k = 0; k < half; k++) {
                const cplx w = sign > 0 ? T.root[k * step] : std::conj(T.root[k * step]);
                const cplx u = a[i + k], v = a[i + k + half] * w;
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
    }
}

void encode_real(const Context& ctx, const double* z, double scale, int64_t* out) {
    const uint32_t n = ctx.n;
    const EncoderTables& T = ctx.enc;
    // values at zeta^(2t+1): m(zeta^(2t+1)) = sum_k (m_k zeta^k) w^(tk), w = exp(2 pi i / N)
    std::vector<cplx> v(n);
    for (uint32_t j = 0; j < ctx.slots; j++) {
        v[T.pos[j]] = cplx(z[j], 0.0);
        v[T.cpos[j]] = cplx(z[j], 0.0);   // conjugate of a real value
    }
    fft(T, v.data(), n, -1);   // sum_t v_t w^(-tk) = N * m_k zeta^k
    for (uint32_t k = 0; k < n; k++) {
        const double x = (v[k] * std::conj(T.zeta[k])).real() / double(n) * scale;
        out[k] = (int64_t)(x >= 0 ? std::floor(x + 0.5) : -std::floor(-x + 0.5));
    }
}

void encode_complex(const Context& ctx, const std::complex<double>* z, double scale, int64_t* out) {
    const uint32_t n = ctx.n;
    const EncoderTables& T = ctx.enc;
    std::vector<cplx> v(n);
    for (uint32_t j = 0; j < ctx.slots; j++) {
        v[T.pos[j]] = z[j];
        v[T.cpos[j]] = std::conj(z[j]);   // the conjugate root takes the conjugate value: real coefficients
    }
    fft(T, v.data(), n, -1);
    for (uint32_t k = 0; k < n; k++) {
        const double x = (v[k] * std::conj(T.zeta[k])).real() / double(n) * scale;
        out[k] = (int64_t)(x >= 0 ? std::floor(x + 0.5) : -std::floor(-x + 0.5));
    }
}

void decode_complex(const Context& ctx, const double* coeffs, double scale, std::complex<double>* z) {
    const uint32_t n = ctx.n;
    const EncoderTables& T = ctx.enc;
    std::vector<cplx> w(n);
    for (uint32_t k = 0; k < n; k++) w[k] = T.zeta[k] * (coeffs[k] / scale);
    fft(T, w.data(), n, +1);
    for (uint32_t j = 0; j < ctx.slots; j++) z[j] = w[T.pos[j]];
}

void decode_real(const Context& ctx, const double* coeffs, double scale, double* z) {
    const uint32_t n = ctx.n;
    const EncoderTables& T = ctx.enc;
    std::vector<cplx> w(n);
    for (uint32_t k = 0; k < n; k++) w[k] = T.zeta[k] * (coeffs[k] / scale);
    fft(T, w.data(), n, +1);   // value at zeta^(2t+1)
    for (uint32_t j = 0; j < ctx.slots; j++) z[j] = w[T.pos[j]].real();
}

// ---- page-locked host memory (caching pool) ----
namespace {
struct PinnedPool {
    std::mutex mu;
    std::unordered_map<size_t, std::vector<void*>> free_blocks;   // exact size -> blocks
    std::unordered_map<void*, bool> pageable;                     // fallback blocks from malloc
    size_t cached = 0;
    static constexpr size_t kMaxCached = (size_t)2 << 30;
};
PinnedPool& pool() {
    static PinnedPool* p = new PinnedPool();   // never destroyed: blocks may be freed during exit
    return *p;
}
}  // namespace

void* pinned_alloc(size_t bytes) {
    if (bytes == 0) bytes = 1;
    PinnedPool& P = pool();
    {
        std::lock_guard<std::mutex> g(P.mu);
        auto it = P.free_blocks.find(bytes);
        if (it != P.free_blocks.end() && !it->second.empty()) {
            void* p = it->second.back();
            it->second.pop_back();
            P.cached -= bytes;
            return p;
        }
    }
    void* p = nullptr;
    // portable: page-locked for every device's context of the process, not only the
    // one current at the allocation
    if (cudaHostAlloc(&p, bytes, cudaHostAllocPortable) == cudaSuccess) return p;
    cudaGetLastError();   // clear the failed call's error
    p = std::malloc(bytes);
    if (!p) throw std::bad_alloc();
    std::lock_guard<std::mutex> g(P.mu);
    P.pageable[p] = true;
    return p;
}

void pinned_free(void* p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 1;
    PinnedPool& P = pool();
    {
        std::lock_guard<std::mutex> g(P.mu);
        auto pg = P.pageable.find(p);
        if (pg != P.pageable.end()) {
            P.pageable.erase(pg);
            std::free(p);
            return;
        }
        if (P.cached + bytes <= PinnedPool::kMaxCached) {
            P.free_blocks[bytes].push_back(p);
            P.cached += bytes;
            return;
        }
    }
    cudaFreeHost(p);
}

}  // namespace bm
