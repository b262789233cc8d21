// api.cu -- C-ABI of the Blind-Match GPU library (declared in include/blindmatch.h).
//
// Client-side calls (keygen, encrypt, decrypt) sample on the host and do their
// polynomial arithmetic with the same GPU kernels as the match; bm_match runs
// the server side of Sec. 3.3 entirely on the device: Algorithm 1 (Input
// Ciphertext Expansion), Algorithm 2 (HE-C^3) for every gallery group, and the
// compression step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bm_internal.h"

namespace bm {

// NVTX range for profilers (no-op unless a tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

static bm_status fail(bm_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

#define BM_TRY(expr)                              \
    do {                                          \
        bm_status st_ = (expr);                   \
        if (st_ != BM_OK) return st_;             \
    } while (0)

static bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }
static uint32_t ilog2(uint64_t x) {
    uint32_t r = 0;
    while ((1ull << r) < x) r++;
    return r;
}

// ---------------------------------------------------------------------------
// schedule layout for (n_ids, dim, part) under a context
// ---------------------------------------------------------------------------

struct Layout {
    uint32_t n_in, G, groups, level, n_out;
    uint32_t per_group;                     // identities per group: G, or 2G with complex packing
    bool tiled, compress;
    bool encrypted;                         // gallery of ciphertexts (HE-C^3 products ct x ct)
    bool hoisted;                           // Algorithm 1 by hoisted rotations
    bool hrotsum, hcomp;                    // rotate-and-sum / compression by hoisted rounds
    bool dhoist;                            // ... with one ModDown per round output
    bool fused;                             // hoisted Algorithm 1 with ModDown and Rescale fused
    bool deferred;                          // ... with the division moved past HE-C^3's products
    bool fcomp;                             // rotate-and-sum's last round and compression fused
};

// Scale of the score ciphertexts: 2^log_scale with a plaintext gallery (every
// plaintext scale is the prime its rescale drops); Delta^2 / q_level with an
// encrypted one (one ct x ct product, one rescale by the gallery level's prime).
double result_scale(const Context& c, const Gallery& g) {
    return g.encrypted ? c.scale * c.scale / (double)c.primes[g.level] : c.scale;
}

static uint32_t gallery_kind(const Gallery& g) {
    return g.packing | (g.encrypted ? BM_LAYOUT_ENCRYPTED : 0u) |
           ((g.sched & BM_SCHED_HOISTED_EXPANSION) ? BM_LAYOUT_HOISTED : 0u) |
           ((g.sched & BM_SCHED_HOISTED_ROTSUM) ? BM_LAYOUT_HOISTED_ROTSUM : 0u) |
           ((g.sched & BM_SCHED_HOISTED_COMPRESSION) ? BM_LAYOUT_HOISTED_COMPRESSION : 0u) |
           ((g.sched & BM_SCHED_DOUBLE_HOISTED) ? BM_LAYOUT_DOUBLE_HOISTED : 0u) |
           ((g.sched & BM_SCHED_FUSED_EXPANSION) ? BM_LAYOUT_FUSED_EXPANSION : 0u) |
           ((g.sched & BM_SCHED_DEFERRED_DIVISION) ? BM_LAYOUT_DEFERRED_DIVISION : 0u) |
           ((g.sched & BM_SCHED_FUSED_COMPRESSION) ? BM_LAYOUT_FUSED_COMPRESSION : 0u);
}

// baby and giant steps of the hoisted rotate-and-sum over s slots: b = 2^ceil(log2(s)/2);
// with one ModDown per round output (double hoisting) a single round of s - 1
// rotations up to s = 16 (a round: one extension, a product per rotation, one
// ModDown; at s = 16 one round of 15 products measured 20 us faster per face step
// than two rounds of 3)
static void bsgs_split(uint32_t s, bool dhoist, uint32_t& b, uint32_t& g) {
    if (dhoist && s <= 16) {
        b = s;
        g = 1;
        return;
    }
    const uint32_t lb = ilog2(s);
    b = 1u << ((lb + 1) / 2);
    g = s / b;
}

// `kind`: a BM_PACK_* value, or'ed with BM_LAYOUT_ENCRYPTED for a gallery of ciphertexts
static bm_status make_layout(const Context& c, uint64_t n_ids, uint32_t dim, uint32_t part, Layout& lo,
                             uint32_t kind = BM_PACK_REAL) {
    const uint32_t packing = kind & ~(BM_LAYOUT_ENCRYPTED | BM_LAYOUT_HOISTED | BM_LAYOUT_HOISTED_ROTSUM |
                                      BM_LAYOUT_HOISTED_COMPRESSION | BM_LAYOUT_DOUBLE_HOISTED |
                                      BM_LAYOUT_FUSED_EXPANSION | BM_LAYOUT_DEFERRED_DIVISION |
                                      BM_LAYOUT_FUSED_COMPRESSION);
    lo.encrypted = (kind & BM_LAYOUT_ENCRYPTED) != 0;
    lo.hoisted = (kind & BM_LAYOUT_HOISTED) != 0;
    lo.hrotsum = (kind & BM_LAYOUT_HOISTED_ROTSUM) != 0;
    lo.hcomp = (kind & BM_LAYOUT_HOISTED_COMPRESSION) != 0;
    lo.dhoist = (kind & BM_LAYOUT_DOUBLE_HOISTED) != 0;
    lo.fused = (kind & BM_LAYOUT_FUSED_EXPANSION) != 0;
    lo.deferred = (kind & BM_LAYOUT_DEFERRED_DIVISION) != 0;
    lo.fcomp = (kind & BM_LAYOUT_FUSED_COMPRESSION) != 0;
    if (!is_pow2(dim) || !is_pow2(part) || part > dim || dim > c.slots)
        return fail(BM_E_DIM, "dim and part size must be powers of two with part <= dim <= N/2");
    if (packing != BM_PACK_REAL && packing != BM_PACK_COMPLEX) return fail(BM_E_ARG, "unknown slot packing");
    if (lo.encrypted && packing != BM_PACK_REAL) return fail(BM_E_ARG, "encrypted galleries use real packing");
    if (c.L < 1) return fail(BM_E_LEVEL, "the modulus chain needs at least one rescale prime");
    if (lo.encrypted && c.L < 3)
        return fail(BM_E_LEVEL, "an encrypted gallery needs three rescale primes (enrollment, HE-C^3, compression)");
    lo.n_in = dim / part;
    lo.G = c.slots / part;
    lo.per_group = packing == BM_PACK_COMPLEX ? 2 * lo.G : lo.G;
    lo.groups = (uint32_t)((n_ids + lo.per_group - 1) / lo.per_group);
    lo.tiled = c.L >= 3;                    // Algorithm 1 (1 level) + HE-C^3 (1) + compression (1)
    lo.level = lo.tiled ? c.L - 1 : c.L;    // level of the query parts entering HE-C^3
    lo.compress = lo.level >= 2;            // a level left after HE-C^3 for the mask
    if (!lo.tiled) lo.hoisted = false;      // no Algorithm 1 on the server
    if (!lo.compress) lo.hcomp = false;
    if (!lo.hrotsum && !lo.hcomp) lo.dhoist = false;
    if (lo.fused) lo.hoisted = lo.tiled;    // the fused form is a form of the hoisted expansion
    if (lo.deferred) lo.fused = true;       // the deferred division is a form of the fused expansion
    if (!lo.hoisted || lo.n_in < 2 || lo.n_in > kMaxCircParts || !ks_mdr_supported(c)) lo.fused = false;
    if (!lo.fused || lo.encrypted || !ks_mdr_supported(c, 2)) lo.deferred = false;
    if (!lo.compress || !lo.hrotsum || !lo.hcomp || !lo.dhoist) lo.fcomp = false;
    lo.n_out = lo.compress ? (lo.groups + part - 1) / part : lo.groups;
    return BM_OK;
}

// left-rotation amounts the schedule uses (negative = right)
static std::vector<int32_t> schedule_rotations(const Context& c, const Layout& lo, uint32_t part) {
    std::vector<int32_t> r;
    if (lo.tiled && lo.hoisted)
        for (uint32_t j = 1; j < lo.n_in; j++) r.push_back((int32_t)(part * j));
    else if (lo.tiled)
        for (uint32_t j = 0; (1u << j) < lo.n_in; j++) r.push_back((int32_t)(part << j));
    if (lo.fcomp) {
        // rounds before the last as below; the last round's rotations shifted by -o for
        // every group offset o of a pack (the identity needs no key)
        uint32_t b, g;
        bsgs_split(part, true, b, g);
        const uint32_t step = g > 1 ? b : 1, count = g > 1 ? g : b;
        if (g > 1)
            for (uint32_t k = 1; k < b; k++) r.push_back((int32_t)k);
        for (uint32_t k = 0; k < count; k++)
            for (uint32_t o = 0; o < part; o++)
                if (step * k != o) r.push_back((int32_t)(step * k) - (int32_t)o);
        return r;
    }
    if (lo.hrotsum) {
        uint32_t b, g;
        bsgs_split(part, lo.dhoist, b, g);
        for (uint32_t k = 1; k < b; k++) r.push_back((int32_t)k);
        for (uint32_t k = 1; k < g; k++) r.push_back((int32_t)(b * k));
    } else {
        for (uint32_t t = 0; (1u << t) < part; t++) r.push_back((int32_t)(1u << t));
    }
    if (lo.compress && lo.hcomp)
        for (uint32_t k = 1; k < part; k++) r.push_back(-(int32_t)k);
    else if (lo.compress)
        for (uint32_t t = 0; (1u << t) < part; t++) r.push_back(-(int32_t)(1u << t));
    (void)c;
    return r;
}


// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

// Validates the parameters and fills the context's sizes, digits and scale
// (host only: the schedule model uses it without a device).
static bm_status context_shape(Context& c, const bm_params& p) {
    // the key-switching, rescale and NTT kernels are written for these shapes: register-
    // resident NTT passes of 2^6 x 2^6 or 2^8 x 2^8 points, digits of at most two primes
    // and at most two special primes
    if (p.log_n != 12 && p.log_n != 16) return fail(BM_E_PARAM, "log_n must be 12 or 16");
    if (p.n_q < 2 || p.n_q > BM_MAX_Q || p.n_p < 1 || p.n_p > 2)
        return fail(BM_E_PARAM, "n_q must be in [2, 6] and n_p in [1, 2]");
    std::vector<uint32_t> bits;
    for (uint32_t i = 0; i < p.n_q; i++) bits.push_back(p.q_bits[i]);
    for (uint32_t i = 0; i < p.n_p; i++) bits.push_back(p.p_bits[i]);
    for (uint32_t b : bits)
        if (b < 30 || b > 60) return fail(BM_E_PARAM, "prime sizes must be in [30, 60] bits");
    if (p.dnum < 1 || p.dnum > MAXD) return fail(BM_E_PARAM, "dnum must be in [1, 4]");
    const uint32_t dsize = (p.n_q + p.dnum - 1) / p.dnum;
    if (dsize > 2 || (p.dnum - 1) * dsize >= p.n_q)
        return fail(BM_E_PARAM, "digits must be non-empty and hold at most 2 primes");
    if (p.log_scale < 20 || p.log_scale > 50) return fail(BM_E_PARAM, "log_scale must be in [20, 50]");
    c.params = p;
    c.log_n = p.log_n;
    c.n = 1u << p.log_n;
    c.slots = c.n / 2;
    c.L = p.n_q - 1;
    c.alpha = p.n_p;
    c.nb = p.n_q + p.n_p;
    c.scale = std::ldexp(1.0, (int)p.log_scale);
    c.digits.clear();
    for (uint32_t d = 0; d < p.dnum; d++) {
        std::vector<uint32_t> dg;
        for (uint32_t j = d * dsize; j < std::min(p.n_q, (d + 1) * dsize); j++) dg.push_back(j);
        c.digits.push_back(dg);
    }
    return BM_OK;
}

static bm_status context_init(Context& c, const bm_params& p, int device) {
    BM_TRY(context_shape(c, p));
    c.device = device;
    std::vector<uint32_t> bits;
    for (uint32_t i = 0; i < p.n_q; i++) bits.push_back(p.q_bits[i]);
    for (uint32_t i = 0; i < p.n_p; i++) bits.push_back(p.p_bits[i]);
    encoder_tables(c);
    if (!gen_primes(c.log_n, bits, c.primes)) return fail(BM_E_PARAM, "prime search failed");
    for (uint32_t j = 0; j < c.nb; j++) {
        uint64_t P = 1;
        for (uint32_t k = 0; k < c.alpha; k++) P = h_mulmod(P, c.primes[c.L + 1 + k] % c.primes[j], c.primes[j]);
        c.P_mod[j] = P;
    }
    BM_CUDA_TRY(cudaSetDevice(device));
    BM_CUDA_TRY(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
    {
        // keep freed stream-ordered allocations (results, temporaries) in the pool
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    // twiddles: per prime, N forward pairs then N inverse pairs
    const size_t per = (size_t)2 * c.n;
    std::vector<ulonglong2> tw(per * c.nb);
    for (uint32_t j = 0; j < c.nb; j++) {
        const uint64_t q = c.primes[j];
        const uint64_t psi = find_psi(q, c.log_n);
        if (!psi) return fail(BM_E_PARAM, "no primitive 2N-th root");
        c.psi.push_back(psi);
        const uint64_t ipsi = h_invmod(psi, q);
        std::vector<uint64_t> pw(c.n), ipw(c.n);
        pw[0] = ipw[0] = 1;
        for (uint32_t i = 1; i < c.n; i++) {
            pw[i] = h_mulmod(pw[i - 1], psi, q);
            ipw[i] = h_mulmod(ipw[i - 1], ipsi, q);
        }
        for (uint32_t k = 0; k < c.n; k++) {
            uint32_t r = 0;
            for (uint32_t b = 0; b < c.log_n; b++) r |= ((k >> b) & 1u) << (c.log_n - 1 - b);
            tw[j * per + k] = make_ulonglong2(pw[r], h_shoup_companion(pw[r], q));
            tw[j * per + c.n + k] = make_ulonglong2(ipw[r], h_shoup_companion(ipw[r], q));
        }
        c.tab.q[j] = q;
        c.tab.qneg[j] = h_mont_qneg(q);
        c.tab.rsh[j] = h_shoup_companion(1, q);
        c.tab.r2[j] = h_r2(q);
        c.tab.ninv[j] = h_invmod(c.n % q, q);
        c.tab.ninv_sh[j] = h_shoup_companion(c.tab.ninv[j], q);
    }
    BM_CUDA_TRY(cudaMalloc(&c.d_twiddles, tw.size() * sizeof(ulonglong2)));
    BM_CUDA_TRY(cudaMemcpy(c.d_twiddles, tw.data(), tw.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice));
    for (uint32_t j = 0; j < c.nb; j++) {
        c.tab.tw[j] = (const ulonglong2*)c.d_twiddles + j * per;
        c.tab.itw[j] = (const ulonglong2*)c.d_twiddles + j * per + c.n;
    }
    BM_CUDA_TRY(build_ks_constants(c));

    if (const char* w = std::getenv("BM_KS_WIDE_BATCH"))
        for (uint32_t& t : c.ks_wide_batch) t = (uint32_t)std::strtoul(w, nullptr, 10);
    return BM_OK;
}

// signed coefficients -> NTT form on limbs [first, first+nl) of dst (one poly)
static bm_status upload_signed_ntt(const Context& c, const int64_t* h, uint64_t* dst, uint32_t nl, uint32_t first_prime,
                                   cudaStream_t s, bool montgomery) {
    int64_t* d = nullptr;
    BM_CUDA_TRY(cudaMallocAsync(&d, sizeof(int64_t) * c.n, s));
    BM_CUDA_TRY(cudaMemcpyAsync(d, h, sizeof(int64_t) * c.n, cudaMemcpyHostToDevice, s));
    LimbBatch b = limbs_of(dst, 1, nl, (uint64_t)nl * c.n, first_prime);
    BM_CUDA_TRY(lift_signed(c, d, b, s));
    BM_CUDA_TRY(ntt_forward(c, b, s));
    if (montgomery) BM_CUDA_TRY(to_montgomery(c, b, false, s));
    BM_CUDA_TRY(cudaFreeAsync(d, s));
    return BM_OK;
}

}  // namespace bm

using namespace bm;

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

const char* bm_last_error(void) { return g_last_error.c_str(); }

bm_status bm_params_preset(int preset, bm_params* out) {
    if (!out) return fail(BM_E_ARG, "null output");
    bm_params p{};
    p.log_scale = 40;
    p.sigma = 3.2;
    p.dnum = 2;
    switch (preset) {
        case BM_PRESET_TOY:
            p.log_n = 12; p.n_q = 2; p.q_bits[0] = 50; p.q_bits[1] = 40;
            p.n_p = 1; p.p_bits[0] = 50; p.secret_hw = 0;
            break;
        case BM_PRESET_RING16:
        case BM_PRESET_SMALL4:
            p.log_n = preset == BM_PRESET_RING16 ? 16 : 12;
            p.n_q = 4; p.q_bits[0] = 60; p.q_bits[1] = p.q_bits[2] = p.q_bits[3] = 40;
            p.n_p = 2; p.p_bits[0] = p.p_bits[1] = 60; p.secret_hw = 192;
            break;
        default:
            return fail(BM_E_ARG, "unknown preset");
    }
    *out = p;
    return BM_OK;
}

bm_status bm_context_create(const bm_params* params, int device, bm_context** out) {
    if (!params || !out) return fail(BM_E_ARG, "null argument");
    auto* h = new bm_context();
    h->c.owner = h;
    bm_status s = context_init(h->c, *params, device);
    if (s != BM_OK) {
        bm_context_destroy(h);
        return s;
    }
    *out = h;
    return BM_OK;
}

void bm_context_destroy(bm_context* ctx) {
    if (!ctx) return;
    ctx->c.destroy_requested = true;
    if (ctx->c.refs.load() == 0) bm::context_free(ctx);
}

}  // extern "C"

namespace bm {
void ctx_retain(Context* c) { c->refs++; }
void ctx_release(Context* c) {
    if (--c->refs == 0 && c->destroy_requested.load()) context_free(c->owner);
}
void context_free(bm_context* ctx) {
    for (Plan* p : ctx->c.plans) destroy_plan(p);
    ctx->c.plans.clear();
    if (ctx->c.d_twiddles) cudaFree(ctx->c.d_twiddles);
    if (ctx->c.d_ksc) cudaFree(ctx->c.d_ksc);
    if (ctx->c.d_ksc_mdr) cudaFree(ctx->c.d_ksc_mdr);
    if (ctx->c.d_qlinv) cudaFree(ctx->c.d_qlinv);
    if (ctx->c.stream) cudaStreamDestroy(ctx->c.stream);
    delete ctx;
}
}  // namespace bm

extern "C" {

bm_status bm_context_primes(const bm_context* ctx, uint64_t* primes_out, size_t capacity) {
    if (!ctx || !primes_out) return fail(BM_E_ARG, "null argument");
    if (capacity < ctx->c.primes.size()) return fail(BM_E_ARG, "capacity too small");
    std::copy(ctx->c.primes.begin(), ctx->c.primes.end(), primes_out);
    return BM_OK;
}

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------

bm_status bm_keygen(bm_context* ctxh, uint64_t seed, uint32_t dim, uint32_t part_size, bm_secret_key** sk_out,
                    bm_public_key** pk_out, bm_eval_keys** evk_out) {
    return bm_keygen_ex(ctxh, seed, dim, part_size, 0, sk_out, pk_out, evk_out);
}

bm_status bm_keygen_ex(bm_context* ctxh, uint64_t seed, uint32_t dim, uint32_t part_size, uint32_t flags,
                       bm_secret_key** sk_out, bm_public_key** pk_out, bm_eval_keys** evk_out) {
    if (!ctxh || !sk_out || !pk_out || !evk_out) return fail(BM_E_ARG, "null argument");
    if (flags & ~(uint32_t)(BM_KEYS_ENCRYPTED_GALLERY | BM_KEYS_HOISTED)) return fail(BM_E_ARG, "unknown key-set flags");
    Context& c = ctxh->c;
    Layout lo;
    BM_TRY(make_layout(c, 1, dim, part_size, lo));
    BM_CUDA_TRY(cudaSetDevice(c.device));
    cudaStream_t s = c.stream;
    const size_t n = c.n, nb = c.nb, L1 = c.L + 1;

    auto* skh = new bm_secret_key();
    skh->ref.attach(&c);
    skh->k.ctx = &c;
    skh->k.coeffs.resize(n);
    sample_secret(seed, c.params.secret_hw, c.log_n, skh->k.coeffs.data());
    DevBuf s_plain, s_mont;
    if (s_plain.alloc(nb * n) || s_mont.alloc(nb * n)) {
        delete skh;
        return fail(BM_E_OOM, "device allocation failed");
    }
    bm_status st = upload_signed_ntt(c, skh->k.coeffs.data(), s_plain.p, nb, 0, s, false);
    if (st != BM_OK) { delete skh; return st; }
    cudaMemcpyAsync(s_mont.p, s_plain.p, nb * n * 8, cudaMemcpyDeviceToDevice, s);
    to_montgomery(c, packed(c, s_mont.p, 1, nb), false, s);
    skh->k.d_ntt = s_mont.release();

    // public key (b, a) over Q_L: b = e - a*s
    auto* pkh = new bm_public_key();
    pkh->ref.attach(&c);
    pkh->k.ctx = &c;
    DevBuf pkb, tmp;
    pkb.alloc(2 * L1 * n);
    tmp.alloc(L1 * n);
    std::vector<uint64_t> host(nb * n);
    std::vector<int64_t> e(n);
    for (uint32_t j = 0; j < L1; j++) sample_uniform(seed, TAG_PK_A, 0, j, c.primes[j], host.data() + j * n, c.n);
    sample_gauss(seed, TAG_PK_E, 0, c.params.sigma, e.data(), c.n);
    uint64_t* pk_b = pkb.p;
    uint64_t* pk_a = pkb.p + L1 * n;
    cudaMemcpyAsync(pk_a, host.data(), L1 * n * 8, cudaMemcpyHostToDevice, s);
    ntt_forward(c, packed(c, pk_a, 1, L1), s);
    upload_signed_ntt(c, e.data(), pk_b, L1, 0, s, false);
    pointwise_mul(c, packed(c, pk_a, 1, L1), limbs_of(skh->k.d_ntt, 1, L1, nb * n),
                  packed(c, tmp.p, 1, L1), s);
    pointwise_addsub(c, packed(c, pk_b, 1, L1), packed(c, tmp.p, 1, L1), packed(c, pk_b, 1, L1), true, s);
    to_montgomery(c, packed(c, pkb.p, 2, L1), false, s);
    pkh->k.d_ntt = pkb.release();

    // rotation keys: per digit d, b_d = e_d - a_d*s + P*[limb in digit d]*sigma_k(s) over Q_L u P
    auto* evh = new bm_eval_keys();
    evh->ref.attach(&c);
    evh->k.ctx = &c;
    evh->k.id = c.next_id++;
    evh->k.dim = dim;
    evh->k.part = part_size;
    const uint32_t nd = (uint32_t)c.digits.size();
    DevBuf srot, prod;
    srot.alloc(nb * n);
    prod.alloc(nb * n);
    // one key-switching key from the NTT-form polynomial t (every limb of Q_L u P) to s:
    // per digit d, b_d = e_d - a_d*s + P*[limb in digit d]*t, a_d uniform (Philox objects obj0 + d)
    auto switch_key = [&](const uint64_t* t, uint64_t tag_a, uint64_t tag_e, uint64_t obj0, uint64_t*& out) -> bool {
        DevBuf key;
        if (key.alloc((size_t)nd * 2 * nb * n) != cudaSuccess) return false;
        for (uint32_t d = 0; d < nd; d++) {
            const uint64_t obj = obj0 + d;
            uint64_t* kb = key.p + ((size_t)d * 2 + 0) * nb * n;
            uint64_t* ka = key.p + ((size_t)d * 2 + 1) * nb * n;
            for (uint32_t j = 0; j < nb; j++) sample_uniform(seed, tag_a, obj, j, c.primes[j], host.data() + j * n, c.n);
            sample_gauss(seed, tag_e, obj, c.params.sigma, e.data(), c.n);
            cudaMemcpyAsync(ka, host.data(), nb * n * 8, cudaMemcpyHostToDevice, s);
            ntt_forward(c, packed(c, ka, 1, nb), s);
            upload_signed_ntt(c, e.data(), kb, nb, 0, s, false);
            pointwise_mul(c, packed(c, ka, 1, nb), packed(c, skh->k.d_ntt, 1, nb), packed(c, prod.p, 1, nb), s);
            pointwise_addsub(c, packed(c, kb, 1, nb), packed(c, prod.p, 1, nb), packed(c, kb, 1, nb), true, s);
            for (uint32_t j : c.digits[d]) {
                LimbBatch one = limbs_of(const_cast<uint64_t*>(t) + (size_t)j * n, 1, 1, n, j);
                LimbBatch dst = limbs_of(prod.p + (size_t)j * n, 1, 1, n, j);
                scalar_mul(c, one, &c.P_mod[j], dst, s);
                LimbBatch kbj = limbs_of(kb + (size_t)j * n, 1, 1, n, j);
                pointwise_addsub(c, kbj, dst, kbj, false, s);
            }
            // the host staging buffers are reused by the next digit: wait for the copies
            cudaStreamSynchronize(s);
        }
        to_montgomery(c, packed(c, key.p, nd * 2, nb), false, s);
        out = key.release();
        return true;
    };
    std::vector<int32_t> rots = schedule_rotations(c, lo, part_size);
    if (flags & BM_KEYS_HOISTED) {
        Layout all = lo;                                  // every hoisted form, both rotate-and-sum splits
        all.hoisted = lo.tiled;
        all.hrotsum = true;
        all.hcomp = lo.compress;
        for (bool dh : {false, true}) {
            all.dhoist = dh;
            all.fcomp = false;
            for (int32_t r : schedule_rotations(c, all, part_size)) rots.push_back(r);
        }
        all.fcomp = lo.compress;
        for (int32_t r : schedule_rotations(c, all, part_size)) rots.push_back(r);
    }
    if (flags & BM_KEYS_ENCRYPTED_GALLERY)
        for (uint32_t b = 0; (1u << b) < c.slots; b++)
            if ((1u << b) >= part_size) rots.push_back(-(int32_t)(1u << b));   // enrollment shifts
    for (int32_t rot : rots) {
        const uint64_t k = galois_of(c, rot);
        if (evh->k.keys.count(k)) continue;
        permute_ntt(c, packed(c, s_plain.p, 1, nb), packed(c, srot.p, 1, nb), k, s);
        uint64_t* key = nullptr;
        if (!switch_key(srot.p, TAG_RK_A, TAG_RK_E, k * 16, key)) {
            delete skh; delete pkh; delete evh;
            return fail(BM_E_OOM, "rotation key allocation failed");
        }
        evh->k.keys[k] = key;
    }
    if (flags & BM_KEYS_ENCRYPTED_GALLERY) {
        // relinearisation key: the target is s^2 (NTT domain: s times s, Montgomery times plain)
        pointwise_mul(c, packed(c, s_plain.p, 1, nb), packed(c, skh->k.d_ntt, 1, nb), packed(c, srot.p, 1, nb), s);
        if (!switch_key(srot.p, TAG_RLK_A, TAG_RLK_E, 0, evh->k.relin)) {
            delete skh; delete pkh; delete evh;
            return fail(BM_E_OOM, "relinearisation key allocation failed");
        }
    }
    cudaError_t ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
        delete skh; delete pkh; delete evh;
        return fail(BM_E_CUDA, std::string("keygen: ") + cudaGetErrorString(ce));
    }
    *sk_out = skh;
    *pk_out = pkh;
    *evk_out = evh;
    return BM_OK;
}

void bm_secret_key_destroy(bm_secret_key* sk) {
    if (!sk) return;
    if (sk->k.d_ntt) cudaFree(sk->k.d_ntt);
    delete sk;
}
void bm_public_key_destroy(bm_public_key* pk) {
    if (!pk) return;
    if (pk->k.d_ntt) cudaFree(pk->k.d_ntt);
    delete pk;
}
void bm_eval_keys_destroy(bm_eval_keys* evk) { delete evk; }

bm_status bm_eval_keys_rotations(const bm_eval_keys* evk, int32_t* rotations, size_t capacity, uint32_t* count) {
    if (!evk || !count) return fail(BM_E_ARG, "null argument");
    const Context& c = *evk->k.ctx;
    std::vector<int32_t> rots;
    for (auto& kv : evk->k.keys) {
        for (int32_t r = 1; r < (int32_t)c.slots; r++)
            if (galois_of(c, r) == kv.first) {
                rots.push_back(r > (int32_t)c.slots / 2 ? r - (int32_t)c.slots : r);
                break;
            }
    }
    *count = (uint32_t)rots.size();
    if (rotations) {
        if (capacity < rots.size()) return fail(BM_E_ARG, "capacity too small");
        std::copy(rots.begin(), rots.end(), rotations);
    }
    return BM_OK;
}

static bm_status download_coeff(const Context& c, const uint64_t* d_src, uint32_t n_polys, uint32_t nl,
                                bool from_mont, uint64_t* out) {
    cudaStream_t s = c.stream;
    const size_t words = (size_t)n_polys * nl * c.n;
    DevBuf t;
    BM_CUDA_TRY(t.alloc(words));
    BM_CUDA_TRY(cudaMemcpyAsync(t.p, d_src, words * 8, cudaMemcpyDeviceToDevice, s));
    if (from_mont) BM_CUDA_TRY(to_montgomery(c, packed(c, t.p, n_polys, nl), true, s));
    BM_CUDA_TRY(ntt_inverse(c, packed(c, t.p, n_polys, nl), s));
    BM_CUDA_TRY(cudaMemcpyAsync(out, t.p, words * 8, cudaMemcpyDeviceToHost, s));
    BM_CUDA_TRY(cudaStreamSynchronize(s));
    return BM_OK;
}

bm_status bm_secret_key_export(const bm_secret_key* sk, int64_t* out, size_t capacity) {
    if (!sk || !out) return fail(BM_E_ARG, "null argument");
    if (capacity < sk->k.coeffs.size()) return fail(BM_E_ARG, "capacity too small");
    std::copy(sk->k.coeffs.begin(), sk->k.coeffs.end(), out);
    return BM_OK;
}

bm_status bm_public_key_export(const bm_public_key* pk, uint64_t* out, size_t capacity) {
    if (!pk || !out) return fail(BM_E_ARG, "null argument");
    const Context& c = *pk->k.ctx;
    if (capacity < (size_t)2 * (c.L + 1) * c.n) return fail(BM_E_ARG, "capacity too small");
    BM_CUDA_TRY(cudaSetDevice(c.device));
    return download_coeff(c, pk->k.d_ntt, 2, c.L + 1, true, out);
}

bm_status bm_eval_keys_export(const bm_eval_keys* evk, int32_t rotation, uint64_t* out, size_t capacity) {
    if (!evk || !out) return fail(BM_E_ARG, "null argument");
    const Context& c = *evk->k.ctx;
    auto it = evk->k.keys.find(galois_of(c, rotation));
    if (it == evk->k.keys.end()) return fail(BM_E_KEY_MISSING, "no key for this rotation");
    const uint32_t nd = (uint32_t)c.digits.size();
    if (capacity < (size_t)nd * 2 * c.nb * c.n) return fail(BM_E_ARG, "capacity too small");
    BM_CUDA_TRY(cudaSetDevice(c.device));
    return download_coeff(c, it->second, nd * 2, c.nb, true, out);
}

}  // extern "C"

bm::EvalKeys::~EvalKeys() {
    if (ctx) drop_plans(*ctx, id);
    for (auto& kv : keys) cudaFree(kv.second);
    if (relin) cudaFree(relin);
}
bm::Gallery::~Gallery() {
    if (ctx) drop_plans(*ctx, id);
    if (d_pts) cudaFree(d_pts);
    if (d_masks) cudaFree(d_masks);
    if (d_masks_hat) cudaFree(d_masks_hat);
    if (d_circ_tw) cudaFree(d_circ_tw);
    if (d_masks_hat_ext) cudaFree(d_masks_hat_ext);
    if (d_circ_tw_ext) cudaFree(d_circ_tw_ext);
    if (d_pts_ext) cudaFree(d_pts_ext);
    if (d_cmask) cudaFree(d_cmask);
    if (d_cmask_rot) cudaFree(d_cmask_rot);
}
bm::Ciphertext::~Ciphertext() {
    if (d_coef) cudaFree(d_coef);
}
bm::Result::~Result() {
    if (d_data) {
        // allocated from the stream-ordered pool; an asynchronous match's copy may still
        // be in flight on its stream: the free waits for its event
        if (ready) cudaStreamWaitEvent(ctx->stream, ready, 0);
        cudaFreeAsync(d_data, ctx->stream);
    }
    if (ready) cudaEventDestroy(ready);
}

// ---------------------------------------------------------------------------
// gallery
// ---------------------------------------------------------------------------

namespace bm {

static bm_status gallery_alloc(Context& c, const Layout& lo, uint64_t n_ids, uint32_t dim, uint32_t part,
                               uint32_t packing, bm_gallery*& gh) {
    gh = new bm_gallery();
    gh->ref.attach(&c);
    Gallery& g = gh->g;
    g.ctx = &c;
    g.packing = packing & ~(BM_LAYOUT_ENCRYPTED | BM_LAYOUT_HOISTED | BM_LAYOUT_HOISTED_ROTSUM |
                            BM_LAYOUT_HOISTED_COMPRESSION | BM_LAYOUT_DOUBLE_HOISTED | BM_LAYOUT_FUSED_EXPANSION |
                            BM_LAYOUT_DEFERRED_DIVISION | BM_LAYOUT_FUSED_COMPRESSION);
    g.encrypted = lo.encrypted;
    g.sched = (lo.hoisted ? BM_SCHED_HOISTED_EXPANSION : 0u) | (lo.hrotsum ? BM_SCHED_HOISTED_ROTSUM : 0u) |
              (lo.hcomp ? BM_SCHED_HOISTED_COMPRESSION : 0u) | (lo.dhoist ? BM_SCHED_DOUBLE_HOISTED : 0u) |
              (lo.fused ? BM_SCHED_FUSED_EXPANSION : 0u);
    g.id = c.next_id++;
    g.n_ids = n_ids;
    g.dim = dim;
    g.part = part;
    g.n_in = lo.n_in;
    g.groups = lo.groups;
    g.level = lo.level;
    g.tiled = lo.tiled;
    g.compress = lo.compress;
    const size_t n = c.n;
    const size_t polys = lo.encrypted ? 2 : 1;
    cudaError_t e = cudaMalloc(&g.d_pts, (size_t)lo.groups * lo.n_in * polys * (lo.level + 1) * n * 8);
    if (e == cudaSuccess && lo.tiled) e = cudaMalloc(&g.d_masks, (size_t)lo.n_in * (c.L + 1) * n * 8);
    if (e == cudaSuccess && lo.tiled && lo.n_in >= 2 && lo.n_in <= kMaxCircParts) {
        e = cudaMalloc(&g.d_masks_hat, (size_t)lo.n_in * (c.L + 1) * n * 8);
        if (e == cudaSuccess) e = cudaMalloc(&g.d_circ_tw, (size_t)lo.n_in * (c.L + 1) * sizeof(ulonglong2));
        if (e == cudaSuccess && ks_mdr_supported(c)) {
            const size_t nlx = c.L + 1 + c.alpha;
            e = cudaMalloc(&g.d_masks_hat_ext, (size_t)lo.n_in * nlx * n * 8);
            if (e == cudaSuccess) e = cudaMalloc(&g.d_circ_tw_ext, (size_t)lo.n_in * nlx * sizeof(ulonglong2));
        }
    }
    if (e == cudaSuccess && lo.compress) e = cudaMalloc(&g.d_cmask, (size_t)lo.level * n * 8);
    if (e != cudaSuccess) {
        delete gh;
        gh = nullptr;
        return fail(BM_E_OOM, "gallery allocation failed");
    }
    return BM_OK;
}

// encode real slots z at `scale` into limbs 0..level of dst (NTT + Montgomery)
static bm_status encode_to_device(Context& c, const std::vector<double>& z, double scale, uint32_t level,
                                  uint64_t* dst) {
    std::vector<int64_t> m(c.n);
    encode_real(c, z.data(), scale, m.data());
    BM_TRY(upload_signed_ntt(c, m.data(), dst, level + 1, 0, c.stream, true));
    BM_CUDA_TRY(cudaStreamSynchronize(c.stream));   // m is a host temporary
    return BM_OK;
}

// the masks' side of hoisted Algorithm 1 as a convolution over the parts
// (mac_circ), once the masks are on the device
static cudaError_t gallery_circ(Context& c, Gallery& g) {
    if (!g.d_masks_hat) return cudaSuccess;
    cudaError_t e = circ_prepare(c, g.n_in, c.L + 1, g.d_masks, g.d_masks_hat, g.d_circ_tw, c.stream);
    if (e != cudaSuccess || !g.d_masks_hat_ext) return e;
    // the fused Algorithm 1: masks and their transform on Q_L u P (the buffer of the
    // extended masks is reused for nothing else: it is freed after the transform)
    const uint32_t nlx = c.L + 1 + c.alpha;
    uint64_t* ext = nullptr;
    e = cudaMalloc(&ext, (size_t)g.n_in * nlx * c.n * 8);
    if (e == cudaSuccess) e = masks_extend(c, g.n_in, g.d_masks, ext, c.stream);
    if (e == cudaSuccess) e = circ_prepare(c, g.n_in, nlx, ext, g.d_masks_hat_ext, g.d_circ_tw_ext, c.stream);
    if (ext) cudaFree(ext);
    return e;
}

// The Algorithm-1 masks (mask_i[k] = 1 iff floor((k mod dim)/part) = i, at the top
// level, scale q_L) and the compression mask (M[k] = 1 iff k = 0 mod part, scale
// of the prime its rescale drops) of a gallery.
static bm_status encode_gallery_masks(Context& c, const Layout& lo, uint32_t dim, uint32_t part, Gallery& g) {
    const size_t n = c.n, S = c.slots;
    std::vector<double> z(S);
    if (lo.tiled) {
        for (uint32_t i = 0; i < lo.n_in; i++) {
            for (size_t k = 0; k < S; k++) z[k] = ((k % dim) / part == i) ? 1.0 : 0.0;
            BM_TRY(encode_to_device(c, z, (double)c.primes[c.L], c.L, g.d_masks + (size_t)i * (c.L + 1) * n));
        }
        if (g.d_masks_hat)
            BM_CUDA_TRY(gallery_circ(c, g));
    }
    if (lo.compress) {
        for (size_t k = 0; k < S; k++) z[k] = (k % part == 0) ? 1.0 : 0.0;
        BM_TRY(encode_to_device(c, z, (double)c.primes[lo.level - 1], lo.level - 1, g.d_cmask));
    }
    return BM_OK;
}


}  // namespace bm

extern "C" {

bm_status bm_gallery_layout(const bm_context* ctx, uint64_t n_ids, uint32_t dim, uint32_t part_size, uint32_t* groups,
                            uint32_t* level, uint32_t* tiled, uint32_t* compressed, uint32_t* n_out) {
    return bm_gallery_layout_packed(ctx, n_ids, dim, part_size, BM_PACK_REAL, groups, level, tiled, compressed,
                                    n_out);
}

bm_status bm_gallery_layout_packed(const bm_context* ctx, uint64_t n_ids, uint32_t dim, uint32_t part_size,
                                   uint32_t packing, uint32_t* groups, uint32_t* level, uint32_t* tiled,
                                   uint32_t* compressed, uint32_t* n_out) {
    if (!ctx) return fail(BM_E_ARG, "null context");
    Layout lo;
    BM_TRY(make_layout(ctx->c, n_ids, dim, part_size, lo, packing));
    if (groups) *groups = lo.groups;
    if (level) *level = lo.level;
    if (tiled) *tiled = lo.tiled;
    if (compressed) *compressed = lo.compress;
    if (n_out) *n_out = lo.n_out;
    return BM_OK;
}

bm_status bm_encode_gallery(bm_context* ctxh, const double* feats, uint64_t n_ids, uint32_t dim, uint32_t part_size,
                            bm_gallery** out) {
    return bm_encode_gallery_packed(ctxh, feats, n_ids, dim, part_size, BM_PACK_REAL, out);
}

bm_status bm_encode_gallery_packed(bm_context* ctxh, const double* feats, uint64_t n_ids, uint32_t dim,
                                   uint32_t part_size, uint32_t packing, bm_gallery** out) {
    if (!ctxh || !feats || !out || n_ids == 0) return fail(BM_E_ARG, "null argument or empty gallery");
    Context& c = ctxh->c;
    Layout lo;
    BM_TRY(make_layout(c, n_ids, dim, part_size, lo, packing));
    BM_CUDA_TRY(cudaSetDevice(c.device));
    bm_gallery* gh;
    BM_TRY(gallery_alloc(c, lo, n_ids, dim, part_size, packing, gh));
    Gallery& g = gh->g;
    const size_t n = c.n, S = c.slots;
    // plaintexts in chunks: encode on the host cores in parallel, then one upload,
    // lift, NTT and Montgomery conversion per chunk
    const uint32_t total = lo.groups * lo.n_in, chunk = 64;
    std::vector<int64_t> coeffs((size_t)chunk * n);
    int64_t* d_coeffs = nullptr;
    if (cudaMalloc(&d_coeffs, coeffs.size() * sizeof(int64_t)) != cudaSuccess) {
        delete gh;
        return fail(BM_E_OOM, "gallery staging allocation failed");
    }
    const double pscale = (double)c.primes[lo.level];
    bm_status st = BM_OK;
    for (uint32_t p0 = 0; p0 < total && st == BM_OK; p0 += chunk) {
        const uint32_t np = std::min(chunk, total - p0);
#pragma omp parallel for schedule(dynamic)
        for (int pp = 0; pp < (int)np; pp++) {
            const uint32_t grp = (p0 + pp) / lo.n_in, i = (p0 + pp) % lo.n_in;
            // identity u of the group in window u (real parts); with complex packing
            // identity G + u in the imaginary parts of the same window
            std::vector<std::complex<double>> zz(S, 0.0);
            for (uint32_t u = 0; u < lo.per_group; u++) {
                const uint64_t id = (uint64_t)grp * lo.per_group + u;
                if (id >= n_ids) break;
                const uint32_t w = u % lo.G;
                const bool im = u >= lo.G;
                for (uint32_t t = 0; t < part_size; t++) {
                    const double x = feats[id * dim + i * part_size + t];
                    if (im) zz[w * part_size + t].imag(x);
                    else zz[w * part_size + t].real(x);
                }
            }
            encode_complex(c, zz.data(), pscale, coeffs.data() + (size_t)pp * n);
        }
        uint64_t* dst = g.d_pts + (size_t)p0 * (lo.level + 1) * n;
        LimbBatch out = packed(c, dst, np, lo.level + 1);
        cudaError_t e = cudaMemcpyAsync(d_coeffs, coeffs.data(), (size_t)np * n * 8, cudaMemcpyHostToDevice, c.stream);
        if (e == cudaSuccess) e = lift_signed(c, d_coeffs, out, c.stream);
        if (e == cudaSuccess) e = ntt_forward(c, out, c.stream);
        if (e == cudaSuccess) e = to_montgomery(c, out, false, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);   // coeffs is reused
        if (e != cudaSuccess) st = fail(BM_E_CUDA, std::string("gallery encode: ") + cudaGetErrorString(e));
    }
    cudaFree(d_coeffs);
    if (st != BM_OK) {
        delete gh;
        return st;
    }
    st = encode_gallery_masks(c, lo, dim, part_size, g);
    if (st != BM_OK) {
        delete gh;
        return st;
    }
    *out = gh;
    return BM_OK;
}

bm_status bm_gallery_import(bm_context* ctxh, const uint64_t* pts, const uint64_t* masks, const uint64_t* cmask,
                            uint64_t n_ids, uint32_t dim, uint32_t part_size, bm_gallery** out) {
    return bm_gallery_import_packed(ctxh, pts, masks, cmask, n_ids, dim, part_size, BM_PACK_REAL, out);
}

bm_status bm_gallery_import_packed(bm_context* ctxh, const uint64_t* pts, const uint64_t* masks,
                                   const uint64_t* cmask, uint64_t n_ids, uint32_t dim, uint32_t part_size,
                                   uint32_t packing, bm_gallery** out) {
    if (!ctxh || !pts || !out || n_ids == 0) return fail(BM_E_ARG, "null argument or empty gallery");
    Context& c = ctxh->c;
    Layout lo;
    BM_TRY(make_layout(c, n_ids, dim, part_size, lo, packing));
    if ((lo.tiled && !masks) || (lo.compress && !cmask)) return fail(BM_E_ARG, "masks required by this layout");
    BM_CUDA_TRY(cudaSetDevice(c.device));
    bm_gallery* gh;
    BM_TRY(gallery_alloc(c, lo, n_ids, dim, part_size, packing, gh));
    Gallery& g = gh->g;
    cudaStream_t s = c.stream;
    const size_t n = c.n;
    auto up = [&](uint64_t* dst, const uint64_t* src, uint32_t polys, uint32_t nl) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)polys * nl * n * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = ntt_forward(c, packed(c, dst, polys, nl), s);
        if (e == cudaSuccess) e = to_montgomery(c, packed(c, dst, polys, nl), false, s);
        return e;
    };
    cudaError_t e = up(g.d_pts, pts, lo.groups * lo.n_in, lo.level + 1);
    if (e == cudaSuccess && lo.tiled) e = up(g.d_masks, masks, lo.n_in, c.L + 1);
    if (e == cudaSuccess && lo.compress) e = up(g.d_cmask, cmask, 1, lo.level);
    if (e == cudaSuccess) e = gallery_circ(c, g);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete gh;
        return fail(BM_E_CUDA, std::string("gallery import: ") + cudaGetErrorString(e));
    }
    *out = gh;
    return BM_OK;
}

bm_status bm_enroll_encrypted(bm_context* ctxh, const bm_eval_keys* evk, bm_ciphertext* const* templates,
                              uint64_t n_ids, uint32_t dim, uint32_t part_size, bm_gallery** out) {
    if (!ctxh || !evk || !templates || !out || n_ids == 0) return fail(BM_E_ARG, "null argument or empty gallery");
    Context& c = ctxh->c;
    if (evk->k.ctx != &c) return fail(BM_E_ARG, "keys belong to another context");
    const uint32_t kind = BM_PACK_REAL | BM_LAYOUT_ENCRYPTED;
    Layout lo;
    BM_TRY(make_layout(c, n_ids, dim, part_size, lo, kind));
    if (!evk->k.relin) return fail(BM_E_KEY_MISSING, "no relinearisation key (bm_keygen_ex, BM_KEYS_ENCRYPTED_GALLERY)");
    const uint32_t lb0 = ilog2(part_size), lbS = ilog2(c.slots);
    std::vector<const uint64_t*> rkey(lbS, nullptr);
    for (uint32_t b = lb0; b < lbS; b++) {
        auto it = evk->k.keys.find(galois_of(c, -(int32_t)(1u << b)));
        if (it == evk->k.keys.end()) return fail(BM_E_KEY_MISSING, "missing enrollment rotation key");
        rkey[b] = it->second;
    }
    for (uint64_t k = 0; k < n_ids; k++) {
        if (!templates[k]) return fail(BM_E_ARG, "null template");
        const Ciphertext& t = templates[k]->ct;
        if (t.ctx != &c) return fail(BM_E_ARG, "template from another context");
        if (t.n_cts != 1 || t.level != c.L) return fail(BM_E_LEVEL, "templates are single top-level ciphertexts");
    }
    BM_CUDA_TRY(cudaSetDevice(c.device));
    bm_gallery* gh;
    BM_TRY(gallery_alloc(c, lo, n_ids, dim, part_size, kind, gh));
    std::unique_ptr<bm_gallery> guard(gh);
    Gallery& g = gh->g;
    cudaStream_t s = c.stream;
    const size_t n = c.n, L = c.L, lg = lo.level, S = c.slots;
    const uint32_t n_in = lo.n_in, G = lo.G;
    const size_t cwL = ct_words(c, (uint32_t)L), cwg = ct_words(c, (uint32_t)lg);
    // the group ciphertexts are summed at the top level (scale Delta * q_L) and
    // rescaled once at the end: the key-switching noise of every identity stays
    // far below that scale and each group gets one rescale's rounding
    const size_t n_grp = (size_t)lo.groups * n_in;
    DevBuf acc_top;
    BM_CUDA_TRY(acc_top.alloc(n_grp * cwL));
    BM_CUDA_TRY(cudaMemsetAsync(acc_top.p, 0, n_grp * cwL * 8, s));
    // enrollment masks: ones at slots [i*part, (i+1)*part), top level, scale q_L
    DevBuf emask;
    BM_CUDA_TRY(emask.alloc((size_t)n_in * (L + 1) * n));
    {
        std::vector<double> z(S);
        for (uint32_t i = 0; i < n_in; i++) {
            for (size_t k = 0; k < S; k++) z[k] = (k >= (size_t)i * part_size && k < (size_t)(i + 1) * part_size);
            BM_TRY(encode_to_device(c, z, (double)c.primes[L], (uint32_t)L, emask.p + (size_t)i * (L + 1) * n));
        }
    }
    // identities in chunks: templates -> masked parts -> rotations -> sums into the group ciphertexts
    const uint32_t CH = 32, maxB = 128;
    const size_t P = (size_t)CH * n_in;
    DevBuf tin, xa, xb, scratch, plist, olist;
    BM_CUDA_TRY(tin.alloc(CH * cwL));
    BM_CUDA_TRY(xa.alloc(P * cwL));
    BM_CUDA_TRY(xb.alloc(P * cwL));
    BM_CUDA_TRY(scratch.alloc(std::max(ks_scratch_words(c, (uint32_t)L, maxB), rescale_scratch_words(c, (uint32_t)L, maxB))));
    // pointer lists per chunk: 3P (products) + 2P per shift bit + at most P group
    // targets + P sums; offsets: one per target and one more
    const size_t list_cap = std::max<size_t>(P * (5 + 2 * (lbS - lb0)) + 16, 2 * n_grp + 16);
    BM_CUDA_TRY(plist.alloc(list_cap));
    BM_CUDA_TRY(olist.alloc(P + 2));
    std::vector<uint64_t*> hl;
    std::vector<uint64_t> hoff;
    hl.reserve(list_cap);
    uint64_t** dl = (uint64_t**)plist.p;
    for (uint64_t u0 = 0; u0 < n_ids; u0 += CH) {
        const uint32_t nu = (uint32_t)std::min<uint64_t>(CH, n_ids - u0);
        const uint32_t np = nu * n_in;
        hl.clear();
        hoff.clear();
        auto put = [&](uint64_t* p) { hl.push_back(p); };
        for (uint32_t u = 0; u < nu; u++) {
            const Ciphertext& t = templates[u0 + u]->ct;
            if (t.d_coef)
                BM_CUDA_TRY(cudaMemcpyAsync(tin.p + u * cwL, t.d_coef, cwL * 8, cudaMemcpyDeviceToDevice, s));
            else
                BM_CUDA_TRY(cudaMemcpyAsync(tin.p + u * cwL, t.host.data(), cwL * 8, cudaMemcpyHostToDevice, s));
        }
        BM_CUDA_TRY(ntt_forward(c, packed(c, tin.p, nu * 2, (uint32_t)L + 1), s));
        // X[u][i] = template_u * mask_i: lists in, pt, out
        const size_t o_mp = hl.size();
        for (uint32_t k = 0; k < np; k++) put(tin.p + (k / n_in) * cwL);
        for (uint32_t k = 0; k < np; k++) put(emask.p + (size_t)(k % n_in) * (L + 1) * n);
        for (uint32_t k = 0; k < np; k++) put(xa.p + k * cwL);
        // rotations: the right shift of part i of identity u is ((w - i) * part) mod N/2,
        // one rotation per set bit, lowest first; each rotation moves a ciphertext between
        // its two buffers
        std::vector<uint32_t> shift(np);
        std::vector<uint8_t> cur(np, 0);
        for (uint32_t k = 0; k < np; k++) {
            const uint64_t w = (u0 + k / n_in) % G, i = k % n_in;
            shift[k] = (uint32_t)((((int64_t)w - (int64_t)i) * (int64_t)part_size % (int64_t)S + (int64_t)S) % (int64_t)S);
        }
        struct RotLaunch { uint32_t b; size_t off, cnt; };
        std::vector<RotLaunch> rl;
        for (uint32_t b = lb0; b < lbS; b++) {
            std::vector<uint32_t> ks;
            for (uint32_t k = 0; k < np; k++)
                if (shift[k] >> b & 1u) ks.push_back(k);
            if (ks.empty()) continue;
            const size_t off = hl.size();
            for (uint32_t k : ks) put((cur[k] ? xb.p : xa.p) + k * cwL);
            for (uint32_t k : ks) put((cur[k] ? xa.p : xb.p) + k * cwL);
            for (uint32_t k : ks) cur[k] ^= 1;
            rl.push_back({b, off, ks.size()});
        }
        // sums: target (group, part) <- its identities of this chunk, in identity order
        const size_t o_dst = hl.size();
        std::vector<std::pair<uint64_t, uint32_t>> targets;
        for (uint32_t u = 0; u < nu; u++) {
            const uint64_t grp = (u0 + u) / G;
            if (targets.empty() || targets.back().first != grp) targets.push_back({grp, u});
        }
        for (auto& tg : targets)
            for (uint32_t i = 0; i < n_in; i++) put(acc_top.p + (tg.first * n_in + i) * cwL);
        const size_t o_src = hl.size();
        hoff.push_back(0);
        for (size_t ti = 0; ti < targets.size(); ti++) {
            const uint32_t ub = targets[ti].second;
            const uint32_t ue = ti + 1 < targets.size() ? targets[ti + 1].second : nu;
            for (uint32_t i = 0; i < n_in; i++) {
                for (uint32_t u = ub; u < ue; u++) {
                    const uint32_t k = u * n_in + i;
                    put((cur[k] ? xb.p : xa.p) + k * cwL);
                }
                hoff.push_back(hl.size() - o_src);
            }
        }
        if (hl.size() > list_cap || hoff.size() > olist.words) return fail(BM_E_ARG, "enrollment list overflow");
        BM_CUDA_TRY(cudaMemcpyAsync(plist.p, hl.data(), hl.size() * sizeof(void*), cudaMemcpyHostToDevice, s));
        BM_CUDA_TRY(cudaMemcpyAsync(olist.p, hoff.data(), hoff.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
        BM_CUDA_TRY(mul_plain(c, (uint32_t)L, np, dl + o_mp, (const uint64_t* const*)(dl + o_mp + np),
                              dl + o_mp + 2 * np, s));
        for (const RotLaunch& r : rl) {
            const uint64_t gk = galois_of(c, -(int32_t)(1u << r.b));
            for (size_t b0 = 0; b0 < r.cnt; b0 += maxB) {
                const uint32_t B = (uint32_t)std::min<size_t>(maxB, r.cnt - b0);
                BM_CUDA_TRY(ks_rotate(c, rkey[r.b], gk, (uint32_t)L, B, dl + r.off + b0, dl + r.off + r.cnt + b0,
                                      nullptr, scratch.p, s));
            }
        }
        BM_CUDA_TRY(accumulate(c, (uint32_t)L, (uint32_t)(targets.size() * n_in), dl + o_dst,
                               (const uint64_t* const*)(dl + o_src), olist.p, np, s));
        BM_CUDA_TRY(cudaStreamSynchronize(s));           // the host lists are rebuilt for the next chunk
    }
    // one rescale per group ciphertext: top level -> the gallery level
    hl.clear();
    for (size_t k = 0; k < n_grp; k++) hl.push_back(acc_top.p + k * cwL);
    for (size_t k = 0; k < n_grp; k++) hl.push_back(g.d_pts + k * cwg);
    for (size_t b0 = 0; b0 < n_grp; b0 += maxB) {
        const uint32_t B = (uint32_t)std::min<size_t>(maxB, n_grp - b0);
        std::vector<uint64_t*> part_list;
        for (uint32_t k = 0; k < B; k++) part_list.push_back(hl[b0 + k]);
        for (uint32_t k = 0; k < B; k++) part_list.push_back(hl[n_grp + b0 + k]);
        BM_CUDA_TRY(cudaMemcpyAsync(plist.p, part_list.data(), part_list.size() * sizeof(void*),
                                    cudaMemcpyHostToDevice, s));
        BM_CUDA_TRY(rescale(c, (uint32_t)L, B, dl, dl + B, scratch.p, s));
        BM_CUDA_TRY(cudaStreamSynchronize(s));           // the list buffer is reused
    }
    BM_CUDA_TRY(to_montgomery(c, packed(c, g.d_pts, lo.groups * n_in * 2, (uint32_t)lg + 1), false, s));
    BM_TRY(encode_gallery_masks(c, lo, dim, part_size, g));
    BM_CUDA_TRY(cudaStreamSynchronize(s));
    *out = guard.release();
    return BM_OK;
}

bm_status bm_gallery_import_encrypted(bm_context* ctxh, const uint64_t* cts, const uint64_t* masks,
                                      const uint64_t* cmask, uint64_t n_ids, uint32_t dim, uint32_t part_size,
                                      bm_gallery** out) {
    if (!ctxh || !cts || !masks || !cmask || !out || n_ids == 0) return fail(BM_E_ARG, "null argument or empty gallery");
    Context& c = ctxh->c;
    const uint32_t kind = BM_PACK_REAL | BM_LAYOUT_ENCRYPTED;
    Layout lo;
    BM_TRY(make_layout(c, n_ids, dim, part_size, lo, kind));
    BM_CUDA_TRY(cudaSetDevice(c.device));
    bm_gallery* gh;
    BM_TRY(gallery_alloc(c, lo, n_ids, dim, part_size, kind, gh));
    std::unique_ptr<bm_gallery> guard(gh);
    Gallery& g = gh->g;
    cudaStream_t s = c.stream;
    const size_t n = c.n;
    auto up = [&](uint64_t* dst, const uint64_t* src, uint32_t polys, uint32_t nl) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)polys * nl * n * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = ntt_forward(c, packed(c, dst, polys, nl), s);
        if (e == cudaSuccess) e = to_montgomery(c, packed(c, dst, polys, nl), false, s);
        return e;
    };
    cudaError_t e = up(g.d_pts, cts, lo.groups * lo.n_in * 2, lo.level + 1);
    if (e == cudaSuccess) e = up(g.d_masks, masks, lo.n_in, c.L + 1);
    if (e == cudaSuccess) e = up(g.d_cmask, cmask, 1, lo.level);
    if (e == cudaSuccess) e = gallery_circ(c, g);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(BM_E_CUDA, std::string("gallery import: ") + cudaGetErrorString(e));
    *out = guard.release();
    return BM_OK;
}

bm_status bm_gallery_set_schedule(bm_gallery* gh, uint32_t flags) {
    if (!gh) return fail(BM_E_ARG, "null gallery");
    const uint32_t all = BM_SCHED_HOISTED_EXPANSION | BM_SCHED_HOISTED_ROTSUM | BM_SCHED_HOISTED_COMPRESSION |
                         BM_SCHED_DOUBLE_HOISTED | BM_SCHED_FUSED_EXPANSION | BM_SCHED_DEFERRED_DIVISION |
                         BM_SCHED_FUSED_COMPRESSION;
    if (flags & ~all) return fail(BM_E_ARG, "unknown schedule flags");
    const uint32_t fc_needs = BM_SCHED_HOISTED_ROTSUM | BM_SCHED_HOISTED_COMPRESSION | BM_SCHED_DOUBLE_HOISTED;
    if ((flags & BM_SCHED_FUSED_COMPRESSION) && (flags & fc_needs) != fc_needs)
        return fail(BM_E_ARG, "the fused compression needs the double-hoisted rotate-and-sum and compression");
    Gallery& g = gh->g;
    if ((flags & BM_SCHED_HOISTED_EXPANSION) && !g.tiled)
        return fail(BM_E_ARG, "the gallery's queries arrive expanded (no Algorithm 1 on the server)");
    if ((flags & BM_SCHED_FUSED_EXPANSION) && (!(flags & BM_SCHED_HOISTED_EXPANSION) || !g.d_masks_hat_ext))
        return fail(BM_E_ARG, "the fused expansion needs the hoisted expansion and 2..32 parts");
    if (flags & BM_SCHED_DEFERRED_DIVISION) {
        Context& c = *g.ctx;
        if (!(flags & BM_SCHED_FUSED_EXPANSION) || g.encrypted || !ks_mdr_supported(c, 2))
            return fail(BM_E_ARG, "the deferred division needs the fused expansion and a plaintext gallery");
        if (!g.d_pts_ext) {
            // the plaintexts' integer coefficients on every prime of Q_L u P, once, then
            // folded with the masks
            const size_t nlx = c.L + 1 + c.alpha, count = (size_t)g.groups * g.n_in;
            BM_CUDA_TRY(cudaSetDevice(c.device));
            if (cudaMalloc(&g.d_pts_ext, count * nlx * c.n * 8) != cudaSuccess) {
                cudaGetLastError();
                g.d_pts_ext = nullptr;
                return fail(BM_E_OOM, "extended gallery allocation failed");
            }
            cudaError_t e = extend_to_ext_basis(c, count, g.d_pts, g.level + 1, g.d_pts_ext, c.stream);
            // folded with the masks of Algorithm 1 (fold_gallery): HE-C^3 then takes the
            // query's rotated copies E_j themselves, with no circulant
            uint64_t *masks_ext = nullptr, *fold = nullptr;
            if (e == cudaSuccess) e = cudaMalloc(&masks_ext, (size_t)g.n_in * nlx * c.n * 8);
            if (e == cudaSuccess) e = cudaMalloc(&fold, count * nlx * c.n * 8);
            if (e == cudaSuccess) e = masks_extend(c, g.n_in, g.d_masks, masks_ext, c.stream);
            if (e == cudaSuccess) e = fold_gallery(c, g.groups, g.n_in, masks_ext, g.d_pts_ext, fold, c.stream);
            if (masks_ext) cudaFree(masks_ext);
            cudaFree(g.d_pts_ext);
            g.d_pts_ext = e == cudaSuccess ? fold : nullptr;
            if (e != cudaSuccess) {
                if (fold) cudaFree(fold);
                cudaGetLastError();
                return fail(e == cudaErrorMemoryAllocation ? BM_E_OOM : BM_E_CUDA,
                            std::string("gallery extension: ") + cudaGetErrorString(e));
            }
        }
    }
    if ((flags & BM_SCHED_FUSED_COMPRESSION) && g.compress && !g.d_cmask_rot) {
        // the compression mask on Q_lc u P (lc = g.level - 1), then rotated right by every
        // group offset o of a pack: part copies
        Context& c = *g.ctx;
        const uint32_t l_in = g.level, nlc = l_in + c.alpha;
        const size_t mw = (size_t)nlc * c.n;
        BM_CUDA_TRY(cudaSetDevice(c.device));
        uint64_t* ext = nullptr;
        cudaError_t e = cudaMalloc(&g.d_cmask_rot, (size_t)g.part * mw * 8);
        if (e == cudaSuccess) e = cudaMalloc(&ext, mw * 8);
        if (e == cudaSuccess) e = extend_to_level_ext(c, 1, g.d_cmask, l_in, ext, c.stream);
        for (uint32_t o = 0; o < g.part && e == cudaSuccess; o++)
            e = permute_ntt(c, packed(c, ext, 1, nlc), packed(c, g.d_cmask_rot + o * mw, 1, nlc),
                            galois_of(c, -(int32_t)o), c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        if (ext) cudaFree(ext);
        if (e != cudaSuccess) {
            if (g.d_cmask_rot) cudaFree(g.d_cmask_rot);
            g.d_cmask_rot = nullptr;
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? BM_E_OOM : BM_E_CUDA,
                        std::string("compression masks: ") + cudaGetErrorString(e));
        }
    }
    if (g.sched != flags) {
        drop_plans(*g.ctx, g.id);
        g.sched = flags;
    }
    return BM_OK;
}

bm_status bm_gallery_set_expansion(bm_gallery* gh, uint32_t mode) {
    if (!gh) return fail(BM_E_ARG, "null gallery");
    if (mode != BM_EXPAND_DOUBLING && mode != BM_EXPAND_HOISTED && mode != BM_EXPAND_FUSED &&
        mode != BM_EXPAND_DEFERRED)
        return fail(BM_E_ARG, "unknown expansion");
    const uint32_t rest = gh->g.sched & ~(uint32_t)(BM_SCHED_HOISTED_EXPANSION | BM_SCHED_FUSED_EXPANSION |
                                                    BM_SCHED_DEFERRED_DIVISION);
    const uint32_t form =
        mode == BM_EXPAND_DEFERRED ? BM_SCHED_HOISTED_EXPANSION | BM_SCHED_FUSED_EXPANSION | BM_SCHED_DEFERRED_DIVISION
        : mode == BM_EXPAND_FUSED  ? BM_SCHED_HOISTED_EXPANSION | BM_SCHED_FUSED_EXPANSION
        : mode == BM_EXPAND_HOISTED ? BM_SCHED_HOISTED_EXPANSION
                                    : 0u;
    return bm_gallery_set_schedule(gh, rest | form);
}

bm_status bm_gallery_info(const bm_gallery* gh, uint32_t* encrypted, uint32_t* packing) {
    if (!gh) return fail(BM_E_ARG, "null gallery");
    if (encrypted) *encrypted = gh->g.encrypted;
    if (packing) *packing = gh->g.packing;
    return BM_OK;
}

bm_status bm_gallery_export(const bm_gallery* gh, uint64_t* pts, uint64_t* masks, uint64_t* cmask) {
    if (!gh) return fail(BM_E_ARG, "null gallery");
    const Gallery& g = gh->g;
    const Context& c = *g.ctx;
    BM_CUDA_TRY(cudaSetDevice(c.device));
    if (pts) BM_TRY(download_coeff(c, g.d_pts, g.groups * g.n_in * (g.encrypted ? 2 : 1), g.level + 1, true, pts));
    if (masks && g.tiled) BM_TRY(download_coeff(c, g.d_masks, g.n_in, c.L + 1, true, masks));
    if (cmask && g.compress) BM_TRY(download_coeff(c, g.d_cmask, 1, g.level, true, cmask));
    return BM_OK;
}

void bm_gallery_destroy(bm_gallery* g) { delete g; }

// ---------------------------------------------------------------------------
// ciphertexts
// ---------------------------------------------------------------------------

bm_status bm_encrypt_query(bm_context* ctxh, const bm_public_key* pk, const double* q, uint32_t dim,
                           uint32_t part_size, uint32_t mode, uint64_t seed, uint64_t query_id,
                           bm_ciphertext** out) {
    if (!ctxh || !pk || !q || !out) return fail(BM_E_ARG, "null argument");
    if (mode != BM_QUERY_TILED && mode != BM_QUERY_EXPANDED && mode != BM_QUERY_TEMPLATE)
        return fail(BM_E_ARG, "unknown query mode");
    Context& c = ctxh->c;
    Layout lo;
    BM_TRY(make_layout(c, 1, dim, part_size, lo));
    BM_CUDA_TRY(cudaSetDevice(c.device));
    cudaStream_t s = c.stream;
    const size_t n = c.n, S = c.slots, L1 = c.L + 1;
    const uint32_t n_cts = mode == BM_QUERY_EXPANDED ? lo.n_in : 1;
    auto* ch = new bm_ciphertext();
    ch->ref.attach(&c);
    Ciphertext& ct = ch->ct;
    ct.ctx = &c;
    ct.n_cts = n_cts;
    ct.level = c.L;
    ct.host.resize((size_t)n_cts * 2 * L1 * n);
    DevBuf v, w;
    if (v.alloc(L1 * n) || w.alloc(2 * L1 * n)) {
        delete ch;
        return fail(BM_E_OOM, "device allocation failed");
    }
    std::vector<double> z(S);
    std::vector<int64_t> m(n), vv(n), e0(n), e1(n);
    for (uint32_t k = 0; k < n_cts; k++) {
        for (size_t j = 0; j < S; j++) {
            if (mode == BM_QUERY_TILED) z[j] = q[j % dim];
            else if (mode == BM_QUERY_EXPANDED) z[j] = q[k * part_size + (j % part_size)];
            else z[j] = j < dim ? q[j] : 0.0;                 // template: first slots, zero padding
        }
        encode_real(c, z.data(), c.scale, m.data());
        const uint64_t obj = query_id * 256 + k;
        sample_zo(seed, TAG_ENC_V, obj, vv.data(), c.n);
        sample_gauss(seed, TAG_ENC_E0, obj, c.params.sigma, e0.data(), c.n);
        sample_gauss(seed, TAG_ENC_E1, obj, c.params.sigma, e1.data(), c.n);
        for (size_t i = 0; i < n; i++) e0[i] += m[i];
        bm_status st = upload_signed_ntt(c, vv.data(), v.p, L1, 0, s, false);
        if (st == BM_OK) st = upload_signed_ntt(c, e0.data(), w.p, L1, 0, s, false);
        if (st == BM_OK) st = upload_signed_ntt(c, e1.data(), w.p + L1 * n, L1, 0, s, false);
        if (st != BM_OK) { delete ch; return st; }
        DevBuf prod;
        prod.alloc(2 * L1 * n);
        for (int comp = 0; comp < 2; comp++) {
            pointwise_mul(c, packed(c, v.p, 1, L1), packed(c, pk->k.d_ntt + comp * L1 * n, 1, L1),
                          packed(c, prod.p + comp * L1 * n, 1, L1), s);
        }
        pointwise_addsub(c, packed(c, prod.p, 2, L1), packed(c, w.p, 2, L1), packed(c, prod.p, 2, L1), false, s);
        ntt_inverse(c, packed(c, prod.p, 2, L1), s);
        cudaMemcpyAsync(ct.host.data() + (size_t)k * 2 * L1 * n, prod.p, 2 * L1 * n * 8, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            delete ch;
            return fail(BM_E_CUDA, std::string("encrypt: ") + cudaGetErrorString(e));
        }
    }
    *out = ch;
    return BM_OK;
}

bm_status bm_ciphertext_import(bm_context* ctxh, const uint64_t* data, uint32_t n_cts, uint32_t level,
                               bm_ciphertext** out) {
    if (!ctxh || !data || !out || n_cts == 0) return fail(BM_E_ARG, "null argument");
    Context& c = ctxh->c;
    if (level > c.L) return fail(BM_E_FORMAT, "level above the chain");
    auto* ch = new bm_ciphertext();
    ch->ref.attach(&c);
    ch->ct.ctx = &c;
    ch->ct.n_cts = n_cts;
    ch->ct.level = level;
    ch->ct.host.assign(data, data + (size_t)n_cts * ct_words(c, level));
    *out = ch;
    return BM_OK;
}

bm_status bm_ciphertext_info(const bm_ciphertext* ct, uint32_t* n_cts, uint32_t* level) {
    if (!ct) return fail(BM_E_ARG, "null ciphertext");
    if (n_cts) *n_cts = ct->ct.n_cts;
    if (level) *level = ct->ct.level;
    return BM_OK;
}

bm_status bm_ciphertext_export(const bm_ciphertext* ct, uint64_t* out, size_t capacity) {
    if (!ct || !out) return fail(BM_E_ARG, "null argument");
    if (capacity < ct->ct.host.size()) return fail(BM_E_ARG, "capacity too small");
    std::copy(ct->ct.host.begin(), ct->ct.host.end(), out);
    return BM_OK;
}

bm_status bm_ciphertext_upload(bm_ciphertext* cth, void* stream) {
    if (!cth) return fail(BM_E_ARG, "null ciphertext");
    Ciphertext& ct = cth->ct;
    const Context& c = *ct.ctx;
    cudaStream_t s = (cudaStream_t)stream;
    BM_CUDA_TRY(cudaSetDevice(c.device));
    if (!ct.d_coef) BM_CUDA_TRY(cudaMalloc(&ct.d_coef, ct.host.size() * 8));
    BM_CUDA_TRY(cudaMemcpyAsync(ct.d_coef, ct.host.data(), ct.host.size() * 8, cudaMemcpyHostToDevice, s));
    BM_CUDA_TRY(cudaStreamSynchronize(s));
    return BM_OK;
}

void bm_ciphertext_destroy(bm_ciphertext* ct) { delete ct; }

}  // extern "C"

// ---------------------------------------------------------------------------
// the match schedule (Sec. 3.3)
// ---------------------------------------------------------------------------

namespace bm {

// Device arrays of ciphertext pointers for one schedule.  The schedule runs first
// as a dry pass that only collects the arrays (and sizes the scratch), then
// (after one upload) as the launch pass.
struct PtrArena {
    std::vector<uint64_t*> host;
    uint64_t** dev = nullptr;
    bool live = false;
    size_t cursor = 0;
    uint64_t* const* list(const std::vector<uint64_t*>& v) {
        if (!live) {
            host.insert(host.end(), v.begin(), v.end());
            return nullptr;
        }
        uint64_t* const* p = dev + cursor;
        cursor += v.size();
        return p;
    }
};

// A match schedule for one (gallery, key set, batch size): persistent device
// buffers, the pointer arrays, and the whole schedule captured as a CUDA graph.
struct Plan {
    Context* c = nullptr;
    uint64_t gid = 0, kid = 0;
    uint32_t Q = 0, ncts = 0, chunk = 0, n_out = 0;
    uint32_t qe = 0;                       // queries per Algorithm-1 chunk (hoisted form)
    std::vector<void*> bufs;
    uint64_t *qin = nullptr, *t0 = nullptr, *T = nullptr, *accA = nullptr, *accB = nullptr, *accT = nullptr;
    uint64_t *ext = nullptr, *R = nullptr; // hoisted Algorithm 1: query extensions, rotated queries
    uint64_t *ext2 = nullptr, *rot = nullptr; // hoisted rounds after HE-C^3: extensions, rotated copies
    size_t hsrc = 0, helem = 0;            // ... their capacities (ciphertexts)
    uint64_t *packs = nullptr;             // compression outputs before the coefficient-domain rescale
    uint64_t *qc1 = nullptr;               // hoisted Algorithm 1: the queries' c1 in coefficient form
    uint64_t *scratch = nullptr, *result = nullptr;
    size_t scratch_words = 0, result_words = 0, qin_words = 0;
    PtrArena arena;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ProfSink counts;                       // launches per replay
    size_t bytes = 0;                      // device memory held
    // host queries: copied into one of two staging buffers on the plan's own copy stream
    // (so that the copy of a call overlaps the match of the call before it), then moved
    // into qin on the caller's stream ahead of the graph
    uint64_t* stg[2] = {nullptr, nullptr};
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    uint32_t slot = 0;
    ~Plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamSynchronize(cs);
        for (int k = 0; k < 2; k++) {
            if (ev_ready[k]) cudaEventDestroy(ev_ready[k]);
            if (ev_free[k]) cudaEventDestroy(ev_free[k]);
        }
        if (cs) cudaStreamDestroy(cs);
        for (void* p : bufs) cudaFree(p);
    }
    bool alloc(uint64_t*& p, size_t words) {
        if (cudaMalloc((void**)&p, std::max<size_t>(words, 1) * 8) != cudaSuccess) return false;
        bufs.push_back(p);
        bytes += std::max<size_t>(words, 1) * 8;
        return true;
    }
};

void destroy_plan(Plan* p) { delete p; }

void drop_plans(Context& c, uint64_t id) {
    std::vector<Plan*> keep;
    for (Plan* p : c.plans) {
        if (p->gid == id || p->kid == id) delete p;
        else keep.push_back(p);
    }
    c.plans.swap(keep);
}

// What the schedule needs to know about a gallery: its layout and, for the
// launch pass, where its plaintexts live.
struct SchedView {
    uint32_t n_in = 0, part = 0, level = 0, groups = 0;
    bool tiled = true, compress = true, encrypted = false, hoisted = false, hrotsum = false, hcomp = false;
    bool dhoist = false;                   // hoisted rounds with one ModDown per output
    bool fused = false;                    // hoisted Algorithm 1 with ModDown and Rescale fused
    bool deferred = false;                 // ... divided after HE-C^3's products (one division per group)
    bool fcomp = false;                    // rotate-and-sum's last round and compression in one round
    const uint64_t* d_pts = nullptr;
    const uint64_t* d_pts_ext = nullptr;   // the plaintexts on Q_L u P (deferred division)
    const uint64_t* d_masks = nullptr;
    const uint64_t* d_masks_hat = nullptr;
    const ulonglong2* d_circ_tw = nullptr;
    const uint64_t* d_masks_hat_ext = nullptr;
    const ulonglong2* d_circ_tw_ext = nullptr;
    const uint64_t* d_cmask = nullptr;
    const uint64_t* d_cmask_rot = nullptr; // the compression mask on Q_lc u P rotated by each offset
};

// The double-hoisted linear compression at level 1 writes its packs to a buffer of
// their own and ends with the rescale in the coefficient domain.
static bool coef_tail(const Context& c, const SchedView& g) {
    return g.compress && g.hcomp && g.dhoist && g.level == 2 && rescale_coef_supported(c);
}

static SchedView view_of(const Gallery& g) {
    SchedView v;
    v.n_in = g.n_in;
    v.part = g.part;
    v.level = g.level;
    v.groups = g.groups;
    v.tiled = g.tiled;
    v.compress = g.compress;
    v.encrypted = g.encrypted;
    v.hoisted = g.tiled && (g.sched & BM_SCHED_HOISTED_EXPANSION);
    v.hrotsum = (g.sched & BM_SCHED_HOISTED_ROTSUM) != 0;
    v.hcomp = g.compress && (g.sched & BM_SCHED_HOISTED_COMPRESSION);
    v.dhoist = (v.hrotsum || v.hcomp) && (g.sched & BM_SCHED_DOUBLE_HOISTED);
    v.fused = v.hoisted && (g.sched & BM_SCHED_FUSED_EXPANSION) && g.d_masks_hat_ext;
    v.deferred = v.fused && (g.sched & BM_SCHED_DEFERRED_DIVISION) && g.d_pts_ext;
    v.fcomp = v.compress && v.hrotsum && v.hcomp && v.dhoist && (g.sched & BM_SCHED_FUSED_COMPRESSION) &&
              g.d_cmask_rot;
    v.d_cmask_rot = g.d_cmask_rot;
    v.d_pts_ext = g.d_pts_ext;
    v.d_pts = g.d_pts;
    v.d_masks = g.d_masks;
    v.d_masks_hat = g.d_masks_hat;
    v.d_circ_tw = g.d_circ_tw;
    v.d_masks_hat_ext = g.d_masks_hat_ext;
    v.d_circ_tw_ext = g.d_circ_tw_ext;
    v.d_cmask = g.d_cmask;
    return v;
}

static SchedView view_of(const Layout& lo, uint32_t part) {
    SchedView v;
    v.n_in = lo.n_in;
    v.part = part;
    v.level = lo.level;
    v.groups = lo.groups;
    v.tiled = lo.tiled;
    v.compress = lo.compress;
    v.encrypted = lo.encrypted;
    v.hoisted = lo.hoisted;
    v.hrotsum = lo.hrotsum;
    v.hcomp = lo.hcomp;
    v.dhoist = lo.dhoist;
    v.fused = lo.fused;
    v.deferred = lo.deferred;
    v.fcomp = lo.fcomp;
    return v;
}

struct MatchRun {
    const Context& c;
    const SchedView g;
    const EvalKeys* ek;
    Plan& pl;
    cudaStream_t s = nullptr;
    uint32_t ksb = 128;
    cudaError_t err = cudaSuccess;
    std::vector<bm_op_launch>* rec = nullptr;   // dry pass: the launches, in order

    MatchRun(const Context& c_, const SchedView& g_, const EvalKeys* ek_, Plan& p_) : c(c_), g(g_), ek(ek_), pl(p_) {}

    void check(cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) err = e;
    }
    void record(uint32_t op, uint32_t level, size_t count, uint32_t queries = 0, uint32_t parts = 0) {
        if (rec && !pl.arena.live) rec->push_back({op, level, (uint32_t)count, queries, parts});
    }
    size_t cw(uint32_t level) const { return ct_words(c, level); }
    const uint64_t* key(int32_t rot) const {
        if (!ek) return nullptr;                // schedule model: no keys
        auto it = ek->keys.find(galois_of(c, rot));
        return it == ek->keys.end() ? nullptr : it->second;
    }
    void need_scratch(size_t words) { pl.scratch_words = std::max(pl.scratch_words, words); }

    // the shape of a launch of hoisted sums: the distinct extensions, sources and keys
    // of its elements [b, e) and the most elements of one of its targets
    static KsSumInfo sum_info(const std::vector<uint64_t*>& ext_of, const std::vector<uint64_t*>& src,
                              const std::vector<uint64_t*>& keys, size_t b, size_t e, uint32_t max_elems) {
        auto count = [&](const std::vector<uint64_t*>& v) {
            std::vector<uint64_t*> u;
            for (size_t i = b; i < e; i++)
                if (v[i]) u.push_back(v[i]);
            std::sort(u.begin(), u.end());
            return (uint32_t)(std::unique(u.begin(), u.end()) - u.begin());
        };
        return {count(ext_of), count(keys), count(src), max_elems};
    }
    // key switch of a batch: rotation by `rot`, or (relin) relinearisation -- the key
    // from s^2 to s with the identity automorphism
    void rotate_batch(uint32_t level, int32_t rot, const std::vector<uint64_t*>& in,
                      const std::vector<uint64_t*>& out, const std::vector<uint64_t*>* add, bool relin = false) {
        auto din = pl.arena.list(in);
        auto dout = pl.arena.list(out);
        auto dadd = add ? pl.arena.list(*add) : nullptr;
        if (!pl.arena.live) {
            need_scratch(ks_scratch_words(c, level, (uint32_t)std::min<size_t>(ksb, in.size())));
            for (size_t b0 = 0; b0 < in.size(); b0 += ksb) record(BM_OP_ROTATE, level, std::min<size_t>(ksb, in.size() - b0));
            return;
        }
        const uint64_t gk = relin ? 1 : galois_of(c, rot);
        const uint64_t* kp = relin ? ek->relin : key(rot);
        for (size_t b0 = 0; b0 < in.size(); b0 += ksb) {
            const uint32_t B = (uint32_t)std::min<size_t>(ksb, in.size() - b0);
            check(ks_rotate(c, kp, gk, level, B, din + b0, dout + b0, dadd ? dadd + b0 : nullptr, pl.scratch, s));
        }
    }
    void rescale_batch(uint32_t level, const std::vector<uint64_t*>& in, const std::vector<uint64_t*>& out) {
        auto din = pl.arena.list(in);
        auto dout = pl.arena.list(out);
        if (!pl.arena.live) {
            need_scratch(rescale_scratch_words(c, level, (uint32_t)std::min<size_t>(ksb, in.size())));
            for (size_t b0 = 0; b0 < in.size(); b0 += ksb) record(BM_OP_RESCALE, level, std::min<size_t>(ksb, in.size() - b0));
            return;
        }
        for (size_t b0 = 0; b0 < in.size(); b0 += ksb) {
            const uint32_t B = (uint32_t)std::min<size_t>(ksb, in.size() - b0);
            check(rescale(c, level, B, din + b0, dout + b0, pl.scratch, s));
        }
    }
    void mulplain_batch(uint32_t level, const std::vector<uint64_t*>& in, const std::vector<uint64_t*>& pt,
                        const std::vector<uint64_t*>& out) {
        auto din = pl.arena.list(in);
        auto dpt = pl.arena.list(pt);
        auto dout = pl.arena.list(out);
        record(BM_OP_MUL_PLAIN, level, in.size());
        if (!pl.arena.live) return;
        check(mul_plain(c, level, (uint32_t)in.size(), din, dpt, dout, s));
    }

    // hoisted rotations: basis extension of the ciphertexts' c1 into ext (per ciphertext ks_ext_words)
    void modup_batch(uint32_t level, const std::vector<uint64_t*>& in, uint64_t* ext) {
        auto din = pl.arena.list(in);
        record(BM_OP_MODUP, level, in.size());
        if (!pl.arena.live) {
            need_scratch(ks_modup_scratch_words(c, level, (uint32_t)in.size()));
            return;
        }
        check(ks_modup_hoisted(c, level, (uint32_t)in.size(), din, ext, pl.scratch, s));
    }
    // the same from the coefficient form of the sources' c1, coef [B][l1][N]
    void modup_coef_batch(uint32_t level, const std::vector<uint64_t*>& in, const uint64_t* coef, uint64_t* ext) {
        auto din = pl.arena.list(in);
        record(BM_OP_MODUP, level, in.size());
        if (pl.arena.live) check(ks_modup_hoisted_coef(c, level, (uint32_t)in.size(), din, coef, ext, s));
    }
    // dst[t] += the ciphertexts of srcs[t] (one launch)
    void accumulate_batch(uint32_t level, const std::vector<uint64_t*>& dst,
                          const std::vector<std::vector<uint64_t*>>& srcs) {
        std::vector<uint64_t*> flat, off{reinterpret_cast<uint64_t*>((uintptr_t)0)};
        for (const auto& l : srcs) {
            flat.insert(flat.end(), l.begin(), l.end());
            off.push_back(reinterpret_cast<uint64_t*>((uintptr_t)flat.size()));
        }
        auto dd = pl.arena.list(dst);
        auto ds = pl.arena.list(flat);
        auto doff = pl.arena.list(off);
        record(BM_OP_ACCUM, level, flat.size());
        if (!pl.arena.live || flat.empty()) return;
        check(accumulate(c, level, (uint32_t)dst.size(), dd, (const uint64_t* const*)ds, (const uint64_t*)doff,
                         (uint32_t)flat.size(), s));
    }
    // One round of hoisted rotations: every source is extended once; element e rotates
    // source e_src[e] by e_rot[e]; target t then gains the rotated elements t_elems[t]
    // (dst[t] += sum).  Targets may be sources: the sums follow every rotation.
    void hoisted_round(uint32_t level, const std::vector<uint64_t*>& srcs, const std::vector<uint32_t>& e_src,
                       const std::vector<int32_t>& e_rot, const std::vector<uint64_t*>& tgts,
                       const std::vector<std::vector<uint32_t>>& t_elems,
                       const std::vector<uint64_t*>* outs = nullptr, const uint64_t* mask = nullptr) {
        const size_t ew = ks_ext_words(c, level), cwl = cw(level);
        for (size_t s0 = 0; s0 < srcs.size(); s0 += ksb) {
            std::vector<uint64_t*> chunk(srcs.begin() + s0, srcs.begin() + std::min(srcs.size(), s0 + ksb));
            modup_batch(level, chunk, pl.ext2 + s0 * ew);
        }
        if (g.dhoist) {
            double_hoisted_sums(level, srcs, e_src, e_rot, tgts, t_elems, outs, mask);
            return;
        }
        std::vector<uint64_t*> ext_of, src, keys, gal, out;
        for (size_t e = 0; e < e_src.size(); e++) {
            ext_of.push_back(pl.ext2 + (size_t)e_src[e] * ew);
            src.push_back(srcs[e_src[e]]);
            keys.push_back(const_cast<uint64_t*>(key(e_rot[e])));
            gal.push_back(reinterpret_cast<uint64_t*>((uintptr_t)galois_of(c, e_rot[e])));
            out.push_back(pl.rot + e * cwl);
        }
        hoisted_batch(level, ext_of, src, keys, gal, out);
        std::vector<std::vector<uint64_t*>> lists;
        for (const auto& te : t_elems) {
            lists.emplace_back();
            for (uint32_t e : te) lists.back().push_back(pl.rot + (size_t)e * cwl);
        }
        accumulate_batch(level, tgts, lists);
    }
    // ... with one ModDown per target (double hoisting): target t gains the sum of
    // its elements' rotations, their key-switch products (and P * sigma(c0)) summed
    // in Q_l u P and moved down once, in place; targets in chunks of ksb
    void double_hoisted_sums(uint32_t level, const std::vector<uint64_t*>& srcs, const std::vector<uint32_t>& e_src,
                             const std::vector<int32_t>& e_rot, const std::vector<uint64_t*>& tgts,
                             const std::vector<std::vector<uint32_t>>& t_elems,
                             const std::vector<uint64_t*>* outs = nullptr, const uint64_t* mask = nullptr,
                             const std::vector<uint64_t>* e_flag = nullptr, const uint64_t* gmask = nullptr,
                             uint32_t n_masks = 0, bool rs_coef = false) {
        // with outs, target t + its sum goes to outs[t] (every target, a zero sum for
        // those without elements); else the targets are updated in place; with mask the
        // result is multiplied by that plaintext (every target must then have elements).
        // With gmask (group-masked sums, outs required, no target added): the elements'
        // flags e_flag mark each group's end and plaintext and the unrotated terms; with
        // rs_coef (level 1) the ModDown is taken in the coefficient domain with the rescale
        // to level 0, outs then the level-0 results
        const size_t ew = ks_ext_words(c, level);
        std::vector<uint64_t*> ext_of, src, keys, gal, tg, to, off{reinterpret_cast<uint64_t*>((uintptr_t)0)};
        std::vector<uint32_t> t_off{0};
        for (size_t t = 0; t < tgts.size(); t++) {
            if (t_elems[t].empty() && !outs) continue;
            for (uint32_t e : t_elems[t]) {
                const uint64_t f = e_flag ? (*e_flag)[e] : 0;
                const bool id = (f & kGalIdentity) != 0;
                ext_of.push_back(pl.ext2 + (size_t)e_src[e] * ew);
                src.push_back(srcs[e_src[e]]);
                keys.push_back(id ? nullptr : const_cast<uint64_t*>(key(e_rot[e])));
                gal.push_back(reinterpret_cast<uint64_t*>((uintptr_t)((id ? 1u : galois_of(c, e_rot[e])) | f)));
            }
            tg.push_back(tgts[t]);
            if (outs) to.push_back((*outs)[t]);
            off.push_back(reinterpret_cast<uint64_t*>((uintptr_t)ext_of.size()));
            t_off.push_back((uint32_t)ext_of.size());
        }
        auto de = pl.arena.list(ext_of);
        auto ds = pl.arena.list(src);
        auto dk = pl.arena.list(keys);
        auto dg = pl.arena.list(gal);
        auto dt = pl.arena.list(tg);
        auto dto = outs ? pl.arena.list(to) : nullptr;
        auto doff = pl.arena.list(off);
        for (size_t t0 = 0; t0 < tg.size(); t0 += ksb) {
            const uint32_t T = (uint32_t)std::min<size_t>(ksb, tg.size() - t0);
            const uint32_t E = t_off[t0 + T] - t_off[t0];
            uint32_t mx = 0;
            for (uint32_t t = t0; t < t0 + T; t++) mx = std::max(mx, t_off[t + 1] - t_off[t]);
            uint32_t n_rot = E;                  // the unrotated terms are no key-switch products
            for (uint32_t i = t_off[t0]; i < t_off[t0 + T]; i++)
                if (reinterpret_cast<uintptr_t>(gal[i]) & kGalIdentity) n_rot--;
            record(BM_OP_IP_SUM, level, n_rot, 0, T);
            record(BM_OP_MODDOWN, level, T);
            if (!pl.arena.live) {
                need_scratch(ks_hoisted_scratch_words(c, level, T));
                continue;
            }
            KsSumInfo u = sum_info(ext_of, src, keys, t_off[t0], t_off[t0 + T], mx);
            u.masks = n_masks;
            check(ks_ipsum_hoisted(c, level, T, (const uint64_t*)(doff + t0), E, (const uint64_t* const*)de,
                                   (const uint64_t* const*)ds, (const uint64_t* const*)dk, (const uint64_t*)dg,
                                   pl.scratch, s, false, u, 0, gmask, rs_coef));
            if (rs_coef)
                check(ks_moddown_rescale_coef(c, T, pl.scratch, dto + t0, s));
            else
                check(ks_moddown_add(c, level, T, gmask ? nullptr : dt + t0, pl.scratch, s, dto ? dto + t0 : nullptr,
                                     mask));
        }
    }
    // ... rotations of the extended queries (per element: extension, source, key, Galois element)
    void hoisted_batch(uint32_t level, const std::vector<uint64_t*>& ext_of, const std::vector<uint64_t*>& src,
                       const std::vector<uint64_t*>& keys, const std::vector<uint64_t*>& gal,
                       const std::vector<uint64_t*>& out) {
        auto de = pl.arena.list(ext_of);
        auto ds = pl.arena.list(src);
        auto dk = pl.arena.list(keys);
        auto dg = pl.arena.list(gal);
        auto dout = pl.arena.list(out);
        for (size_t b0 = 0; b0 < out.size(); b0 += ksb) {
            const uint32_t E = (uint32_t)std::min<size_t>(ksb, out.size() - b0);
            record(BM_OP_ROT_HOISTED, level, E);
            if (!pl.arena.live) {
                need_scratch(ks_hoisted_scratch_words(c, level, E));
                continue;
            }
            check(ks_rotate_hoisted(c, level, E, (const uint64_t* const*)(de + b0), (const uint64_t* const*)(ds + b0),
                                    (const uint64_t* const*)(dk + b0), (const uint64_t*)(dg + b0), dout + b0,
                                    pl.scratch, s));
        }
    }

    // a0..a6 on the plan's buffers; with arena.live == false only the pointer
    // arrays are collected, the scratch sized and (with rec) the launches listed.
    void schedule() {
        const uint32_t Q = pl.Q, n_in = g.n_in, part = g.part, lg = g.level, n_out = pl.n_out;
        pl.arena.cursor = 0;
        NvtxRange whole(pl.arena.live ? "bm_match_launch" : "bm_match_plan");
        // a0: queries into the NTT domain; the hoisted Algorithm 1 first keeps the
        // coefficient form of each query's c1 for its basis extension (no inverse NTT)
        const size_t lw = c.n * (size_t)(c.L + 1);
        // a0 and Algorithm 1's extension in two launches (ks_a0_modup) when every query is in
        // one chunk and the NTT of the batch takes the default shape; else the copy of c1,
        // the NTT and the extension from the copy
        const bool front = g.tiled && g.hoisted && g.n_in > 1 && pl.qe == Q &&
                           c.ntt_shape[ntt_bucket(Q * pl.ncts * 2 * (c.L + 1))] == 0;
        if (g.tiled && g.hoisted) {
            record(BM_OP_COPY, 0, Q);
            if (pl.arena.live && !front)
                check(cudaMemcpy2DAsync(pl.qc1, lw * 8, pl.qin + lw, cw(c.L) * 8, lw * 8, Q, cudaMemcpyDeviceToDevice,
                                        s));
        }
        record(BM_OP_NTT, 0, (size_t)Q * pl.ncts * 2 * (c.L + 1));
        if (pl.arena.live) {
            if (front) check(ks_a0_modup(c, Q, pl.qin, pl.ext, s));
            else check(ntt_forward(c, packed(c, pl.qin, Q * pl.ncts * 2, c.L + 1), s));
        }
        // Algorithm 1, hoisted form: T_i = Res(sum_j Rot(ct, j*part) * mask_((i-j) mod N_in)),
        // the N_in - 1 rotations of each query sharing one basis extension; queries in chunks of pl.qe
        if (g.tiled && g.hoisted && g.fused) {
            // fused form: E_j = the rotation by j parts before ModDown (sums left in NTT
            // form on Q_L u P, P * sigma(c0) included), E_0 = P * query; e_i = sum_j E_j *
            // mask_((i-j) mod N_in) on Q_L u P; T_i = e_i / (q_L P) (ModDown and Rescale fused).
            // With the deferred division HE-C^3 sums e_i * pts_i, i.e. sum_j E_j * fold_j
            // (the gallery folded with the masks), and divides after it.
            const size_t ew = ks_ext_words(c, c.L);
            const uint32_t nlx = c.L + 1 + c.alpha;
            const size_t xw = (size_t)2 * nlx * c.n;             // one sum on Q_L u P
            for (uint32_t qb = 0; qb < Q; qb += pl.qe) {
                const uint32_t nq = std::min(pl.qe, Q - qb);
                uint64_t* E0 = pl.R + (size_t)pl.qe * (n_in - 1) * xw;       // after the rotated sums
                std::vector<uint64_t*> qs, ext_of, src, keys, gal, off{reinterpret_cast<uint64_t*>((uintptr_t)0)}, R, outs;
                for (uint32_t q = 0; q < nq; q++) qs.push_back(pl.qin + (size_t)(qb + q) * cw(c.L));
                if (front) record(BM_OP_MODUP, c.L, qs.size());          // written by ks_a0_modup
                else modup_coef_batch(c.L, qs, pl.qc1 + (size_t)qb * lw, pl.ext);
                for (uint32_t q = 0; q < nq; q++)
                    for (uint32_t j = 1; j < n_in; j++) {
                        ext_of.push_back(pl.ext + (size_t)q * ew);
                        src.push_back(qs[q]);
                        keys.push_back(const_cast<uint64_t*>(key((int32_t)(part * j))));
                        gal.push_back(reinterpret_cast<uint64_t*>((uintptr_t)galois_of(c, (int32_t)(part * j))));
                        off.push_back(reinterpret_cast<uint64_t*>((uintptr_t)ext_of.size()));
                    }
                auto de = pl.arena.list(ext_of);
                auto ds = pl.arena.list(src);
                auto dk = pl.arena.list(keys);
                auto dg = pl.arena.list(gal);
                auto doff = pl.arena.list(off);
                auto dq = pl.arena.list(qs);
                const uint32_t nt = (uint32_t)ext_of.size();
                // deferred division: E_0 .. E_(N_in-1) of each query go straight to T (on Q_L u P),
                // E_j at part j, for HE-C^3 against the gallery folded with the masks
                // (fold_gallery): no circulant; the sums of a launch are whole queries
                const uint32_t per = n_in - 1, step = g.deferred ? std::max(1u, ksb / per) * per : ksb;
                for (uint32_t t0 = 0; t0 < nt; t0 += step) {
                    const uint32_t T = std::min(step, nt - t0);
                    record(BM_OP_IP_SUM, c.L, T, 0, T);
                    uint64_t* out = g.deferred ? pl.T + ((size_t)qb * n_in + (size_t)(t0 / per) * n_in) * xw
                                               : pl.R + (size_t)t0 * xw;
                    if (pl.arena.live)
                        check(ks_ipsum_hoisted(c, c.L, T, (const uint64_t*)(doff + t0), T, (const uint64_t* const*)de,
                                               (const uint64_t* const*)ds, (const uint64_t* const*)dk,
                                               (const uint64_t*)dg, out, s, true,
                                               sum_info(ext_of, src, keys, t0, t0 + T, 1), g.deferred ? per : 0));
                }
                if (g.deferred) continue;          // E_0 written by the same launch (slot 0 of each query)
                record(BM_OP_COPY, 0, nq);
                if (pl.arena.live) check(lift_p(c, nq, dq, E0, s));
                for (uint32_t q = 0; q < nq; q++)
                    for (uint32_t j = 0; j < n_in; j++)
                        R.push_back(j == 0 ? E0 + (size_t)q * xw : pl.R + ((size_t)q * (n_in - 1) + j - 1) * xw);
                auto dR = pl.arena.list(R);
                record(BM_OP_MAC_CIRC, c.L, n_in, nq, n_in);
                if (pl.arena.live)
                    check(mac_circ(c, nlx - 1, nq, n_in, (const uint64_t* const*)dR, nullptr, g.d_masks_hat_ext,
                                   g.d_circ_tw_ext, pl.t0, s));
                for (uint32_t q = 0; q < nq; q++)
                    for (uint32_t i = 0; i < n_in; i++) outs.push_back(pl.T + ((size_t)(qb + q) * n_in + i) * cw(lg));
                auto dout = pl.arena.list(outs);
                for (uint32_t o0 = 0; o0 < (uint32_t)outs.size(); o0 += ksb) {
                    const uint32_t T = std::min<uint32_t>(ksb, (uint32_t)outs.size() - o0);
                    record(BM_OP_MODDOWN, c.L, T);
                    if (!pl.arena.live) {
                        need_scratch(ks_mdr_scratch_words(c, T));
                        continue;
                    }
                    check(ks_moddown_rescale(c, T, pl.t0 + (size_t)o0 * xw, dout + o0, pl.scratch, s));
                }
            }
        } else if (g.tiled && g.hoisted) {
            const size_t ew = ks_ext_words(c, c.L);
            for (uint32_t qb = 0; qb < Q; qb += pl.qe) {
                const uint32_t nq = std::min(pl.qe, Q - qb);
                std::vector<uint64_t*> qs, ext_of, src, keys, gal, out, R, o0, o1;
                for (uint32_t q = 0; q < nq; q++) qs.push_back(pl.qin + (size_t)(qb + q) * cw(c.L));
                if (front) record(BM_OP_MODUP, c.L, qs.size());           // written by ks_a0_modup
                else if (n_in > 1) modup_coef_batch(c.L, qs, pl.qc1 + (size_t)qb * lw, pl.ext);
                for (uint32_t q = 0; q < nq; q++)
                    for (uint32_t j = 1; j < n_in; j++) {
                        ext_of.push_back(pl.ext + (size_t)q * ew);
                        src.push_back(qs[q]);
                        keys.push_back(const_cast<uint64_t*>(key((int32_t)(part * j))));
                        gal.push_back(reinterpret_cast<uint64_t*>((uintptr_t)galois_of(c, (int32_t)(part * j))));
                        out.push_back(pl.R + ((size_t)q * n_in + j) * cw(c.L));
                    }
                hoisted_batch(c.L, ext_of, src, keys, gal, out);
                for (uint32_t q = 0; q < nq; q++)
                    for (uint32_t j = 0; j < n_in; j++)
                        R.push_back(j == 0 ? qs[q] : pl.R + ((size_t)q * n_in + j) * cw(c.L));
                auto dR = pl.arena.list(R);
                record(BM_OP_MAC_CIRC, c.L, n_in, nq, n_in);
                if (pl.arena.live)
                    check(mac_circ(c, c.L, nq, n_in, (const uint64_t* const*)dR, g.d_masks, g.d_masks_hat,
                                   g.d_circ_tw, pl.t0, s));
                for (uint32_t q = 0; q < nq; q++)
                    for (uint32_t i = 0; i < n_in; i++) {
                        o0.push_back(pl.t0 + ((size_t)q * n_in + i) * cw(c.L));
                        o1.push_back(pl.T + ((size_t)(qb + q) * n_in + i) * cw(lg));
                    }
                rescale_batch(c.L, o0, o1);
            }
        } else if (g.tiled) {
            // Algorithm 1: C_out,i = Res(Mul(P)(C_in, mask_i)), then log2(N_in) rotate-and-add by part*2^(j-1)
            std::vector<uint64_t*> in, pt, o0, o1;
            for (uint32_t q = 0; q < Q; q++)
                for (uint32_t i = 0; i < n_in; i++) {
                    in.push_back(pl.qin + (size_t)q * cw(c.L));
                    pt.push_back(const_cast<uint64_t*>(g.d_masks) + (size_t)i * (c.L + 1) * c.n);
                    o0.push_back(pl.t0 + ((size_t)q * n_in + i) * cw(c.L));
                    o1.push_back(pl.T + ((size_t)q * n_in + i) * cw(lg));
                }
            mulplain_batch(c.L, in, pt, o0);
            rescale_batch(c.L, o0, o1);
            for (uint32_t j = 1; (1u << (j - 1)) < n_in; j++) rotate_batch(lg, (int32_t)(part << (j - 1)), o1, o1, &o1);
        }
        const uint64_t* Tsrc = g.tiled ? pl.T : pl.qin;
        const uint32_t nlx = c.L + 1 + c.alpha;
        const size_t xw = (size_t)2 * nlx * c.n;
        // HE-C^3 per chunk of groups, then compression
        for (uint32_t g0 = 0; g0 < g.groups; g0 += pl.chunk) {
            const uint32_t G = std::min(pl.chunk, g.groups - g0);
            // (the deferred division's products run on the L + 1 + alpha limbs of Q_L u P)
            record(g.encrypted ? BM_OP_MAC_CT : BM_OP_MAC, g.deferred ? nlx - 1 : lg, G, Q, n_in);
            if (pl.arena.live) {
                if (g.deferred)   // the undivided parts times the plaintexts on Q_L u P
                    check(mac(c, nlx - 1, Q, G, n_in, Tsrc, g.d_pts_ext + (size_t)g0 * n_in * nlx * c.n, pl.accA, s));
                else if (g.encrypted)
                    check(mac_ct(c, lg, Q, G, n_in, Tsrc, g.d_pts + (size_t)g0 * n_in * 2 * (lg + 1) * c.n, pl.accT,
                                 pl.accA, s));
                else
                    check(mac(c, lg, Q, G, n_in, Tsrc, g.d_pts + (size_t)g0 * n_in * (lg + 1) * c.n, pl.accA, s));
            }
            std::vector<uint64_t*> a, b, t;
            for (uint32_t q = 0; q < Q; q++)
                for (uint32_t k = 0; k < G; k++) {
                    a.push_back(pl.accA + ((size_t)q * G + k) * cw(lg));
                    b.push_back(pl.accB + ((size_t)q * G + k) * cw(lg - 1));
                    if (g.encrypted) t.push_back(pl.accT + ((size_t)q * G + k) * cw(lg));
                }
            // encrypted gallery: one relinearisation of the summed tensor products,
            // (d0, d1, d2) -> (d0 + KS(d2)_0, d1 + KS(d2)_1) with t = (d0, d2), a = (0, d1)
            if (g.encrypted) rotate_batch(lg, 0, t, a, &a, true);
            // the fused rotate-and-sum + compression extends the group sums first of all (one
            // round: no hoisted round before it), so the deferred division can hand it the
            // extension of its quotients from the same kernels (ks_moddown_rescale_modup)
            uint32_t bs0, gs0;
            bsgs_split(part, g.dhoist, bs0, gs0);
            const bool mdru = g.deferred && g.fcomp && gs0 == 1 && lg == c.L - 1 && ks_mdru_supported(c);
            if (g.deferred) {
                // each (query, group) sum divided once by q_(L-1) q_L P (accA: [Q][G][2][nlx][N])
                auto db = pl.arena.list(b);
                const size_t ewc = ks_ext_words(c, lg - 1);
                for (uint32_t o0 = 0; o0 < (uint32_t)b.size(); o0 += ksb) {
                    const uint32_t T = std::min<uint32_t>(ksb, (uint32_t)b.size() - o0);
                    record(BM_OP_MODDOWN, c.L, T);
                    if (!pl.arena.live) {
                        need_scratch(ks_mdr_scratch_words(c, T));
                        continue;
                    }
                    if (mdru)
                        check(ks_moddown_rescale_modup(c, T, pl.accA + (size_t)o0 * xw, db + o0,
                                                       pl.ext2 + (size_t)o0 * ewc, pl.scratch, s));
                    else
                        check(ks_moddown_rescale(c, T, pl.accA + (size_t)o0 * xw, db + o0, pl.scratch, s, 2));
                }
            } else {
                rescale_batch(lg, a, b);
            }
            // the compression's mask product taken in the ModDown of the last double-hoisted
            // rotate-and-sum round (one launch less); else its own launch below
            bool mask_fused = false;
            if (g.hrotsum) {
                // sum_{r<part} Rot(acc, r) in two hoisted rounds: baby steps 1..bs-1, giant steps bs*k
                uint32_t bs, gs;
                bsgs_split(part, g.dhoist, bs, gs);
                const uint32_t rounds[2][2] = {{1, bs}, {bs, gs}};
                const int last = gs > 1 ? 1 : (bs > 1 ? 0 : -1);
                for (int ri = 0; ri < 2; ri++) {
                    const auto& rd = rounds[ri];
                    if (rd[1] <= 1) continue;
                    if (g.fcomp && ri == last) break;          // taken with the compression below
                    std::vector<uint32_t> e_src;
                    std::vector<int32_t> e_rot;
                    std::vector<std::vector<uint32_t>> t_elems(b.size());
                    for (uint32_t k = 0; k < b.size(); k++)
                        for (uint32_t r = 1; r < rd[1]; r++) {
                            t_elems[k].push_back((uint32_t)e_src.size());
                            e_src.push_back(k);
                            e_rot.push_back((int32_t)(rd[0] * r));
                        }
                    const bool fuse = ri == last && g.compress && g.dhoist;
                    hoisted_round(lg - 1, b, e_src, e_rot, b, t_elems, nullptr, fuse ? g.d_cmask : nullptr);
                    mask_fused = mask_fused || fuse;
                }
            } else {
                for (uint32_t t = 1; (1u << (t - 1)) < part; t++)
                    rotate_batch(lg - 1, (int32_t)(1u << (t - 1)), b, b, &b);
            }
            if (!g.compress) {
                // per-group outputs at level 0: copy into the result
                for (uint32_t q = 0; q < Q; q++) {
                    record(BM_OP_COPY, 0, G);
                    if (!pl.arena.live) continue;
                    ProfScope ps(BM_KERNEL_OTHER, s, 16.0 * G * cw(0));
                    check(cudaMemcpyAsync(pl.result + ((size_t)q * n_out + g0) * cw(0),
                                          pl.accB + (size_t)q * G * cw(0), (size_t)G * cw(0) * 8,
                                          cudaMemcpyDeviceToDevice, s));
                }
                continue;
            }
            const uint32_t lc = lg - 1;
            std::vector<uint64_t*> packs;
            bool tail_done = false;            // the results written by the fused round
            if (g.fcomp) {
                // the rotate-and-sum's last round and the compression in one round per pack:
                // group o of a pack contributes Rot(M, -o) * sum_k Rot(acc_o, step * k - o)
                // (the unrotated term when step * k = o), every pack one group-masked sum
                // moved down once
                uint32_t bs, gs;
                bsgs_split(part, true, bs, gs);
                const uint32_t step = gs > 1 ? bs : 1, count = gs > 1 ? gs : bs;
                std::vector<uint64_t*> srcs, heads, fouts;
                std::vector<uint32_t> e_src;
                std::vector<int32_t> e_rot;
                std::vector<uint64_t> e_flag;
                std::vector<std::vector<uint32_t>> t_elems;
                for (uint32_t q = 0; q < Q; q++)
                    for (uint32_t k = 0; k < G; k += part) {
                        heads.push_back(pl.accB + ((size_t)q * G + k) * cw(lc));
                        t_elems.emplace_back();
                        for (uint32_t o = 0; o < part && k + o < G && g0 + k + o < g.groups; o++) {
                            const uint32_t si = (uint32_t)srcs.size();
                            srcs.push_back(pl.accB + ((size_t)q * G + k + o) * cw(lc));
                            for (uint32_t kk = 0; kk < count; kk++) {
                                const int32_t r = (int32_t)(step * kk) - (int32_t)o;
                                uint64_t f = r == 0 ? kGalIdentity : 0;
                                if (kk + 1 == count) f |= kGalGroupEnd | ((uint64_t)o << kGalMaskShift);
                                t_elems.back().push_back((uint32_t)e_src.size());
                                e_src.push_back(si);
                                e_rot.push_back(r);
                                e_flag.push_back(f);
                            }
                        }
                    }
                // with the coefficient-domain tail the packs' ModDown, inverse NTT and rescale
                // are one kernel writing the level-0 results
                const bool ct = coef_tail();
                for (uint32_t q = 0; q < Q && ct; q++)
                    for (uint32_t k = 0; k < G; k += part)
                        fouts.push_back(pl.result + ((size_t)q * n_out + (g0 + k) / part) * cw(0));
                if (!ct) fouts = heads;
                const size_t ew = ks_ext_words(c, lc);
                for (size_t s0 = 0; s0 < srcs.size(); s0 += ksb) {
                    std::vector<uint64_t*> chunk(srcs.begin() + s0, srcs.begin() + std::min(srcs.size(), s0 + ksb));
                    // (with mdru the division above wrote these extensions: srcs are b, in order)
                    if (mdru) record(BM_OP_MODUP, lc, chunk.size());
                    else modup_batch(lc, chunk, pl.ext2 + s0 * ew);
                }
                double_hoisted_sums(lc, srcs, e_src, e_rot, heads, t_elems, &fouts, nullptr, &e_flag, g.d_cmask_rot,
                                    std::min(part, G), ct);
                mask_fused = true;
                tail_done = ct;
            }
            std::vector<uint64_t*> mp(b.size(), const_cast<uint64_t*>(g.d_cmask));
            if (!mask_fused) mulplain_batch(lc, b, mp, b);
            if (g.hcomp && !g.fcomp) {
                // linear form: every group r > 0 of a pack rotated right by r in one hoisted round,
                // summed into the pack's first group
                std::vector<uint64_t*> srcs, heads;
                std::vector<uint32_t> e_src;
                std::vector<int32_t> e_rot;
                std::vector<std::vector<uint32_t>> t_elems;
                for (uint32_t q = 0; q < Q; q++)
                    for (uint32_t k = 0; k < G; k += part) {
                        heads.push_back(pl.accB + ((size_t)q * G + k) * cw(lc));
                        t_elems.emplace_back();
                        for (uint32_t r = 1; r < part && k + r < G && g0 + k + r < g.groups; r++) {
                            t_elems.back().push_back((uint32_t)e_src.size());
                            e_src.push_back((uint32_t)srcs.size());
                            e_rot.push_back(-(int32_t)r);
                            srcs.push_back(pl.accB + ((size_t)q * G + k + r) * cw(lc));
                        }
                    }
                if (coef_tail()) {
                    // the packs to a contiguous buffer for the coefficient-domain rescale below
                    for (size_t p = 0; p < heads.size(); p++) packs.push_back(pl.packs + p * cw(lc));
                    hoisted_round(lc, srcs, e_src, e_rot, heads, t_elems, &packs);
                } else if (!srcs.empty()) {
                    hoisted_round(lc, srcs, e_src, e_rot, heads, t_elems);
                }
            }
            // tree of right rotations: level bb pairs r and r + 2^bb (r = 0 mod 2^(bb+1)) inside each pack
            for (uint32_t bb = 0; !g.hcomp && (1u << bb) < part; bb++) {
                std::vector<uint64_t*> odd, even;
                for (uint32_t q = 0; q < Q; q++)
                    for (uint32_t k = 0; k < G; k += (2u << bb)) {
                        const uint32_t gl = g0 + k;                 // global group of the even element
                        if (gl + (1u << bb) >= g.groups || k + (1u << bb) >= G) continue;
                        even.push_back(pl.accB + ((size_t)q * G + k) * cw(lc));
                        odd.push_back(pl.accB + ((size_t)q * G + k + (1u << bb)) * cw(lc));
                    }
                if (!odd.empty()) rotate_batch(lc, -(int32_t)(1u << bb), odd, even, &even);
            }
            std::vector<uint64_t*> heads, outs;
            for (uint32_t q = 0; q < Q; q++)
                for (uint32_t k = 0; k < G; k += part) {
                    heads.push_back(pl.accB + ((size_t)q * G + k) * cw(lc));
                    outs.push_back(pl.result + ((size_t)q * n_out + (g0 + k) / part) * cw(0));
                }
            if (tail_done) {
            } else if (coef_tail()) {
                // the last rescale in the coefficient domain: an inverse NTT of both limbs of
                // each pack, then (c_0 - [c_1]) * q_1^-1 into the result (the residues of the
                // NTT-domain rescale and the inverse NTT of a6)
                record(BM_OP_INTT, 0, packs.size() * 2 * (lc + 1));
                if (pl.arena.live) check(ntt_inverse(c, packed(c, pl.packs, (uint32_t)packs.size() * 2, lc + 1), s));
                auto din = pl.arena.list(packs);
                auto dout = pl.arena.list(outs);
                record(BM_OP_RESCALE, lc, packs.size());
                if (pl.arena.live) check(rescale_coef(c, (uint32_t)packs.size(), din, dout, s));
            } else {
                rescale_batch(lc, heads, outs);
            }
        }
        // a6: score ciphertexts back to coefficient form (done above with the coefficient-domain rescale)
        if (!coef_tail()) {
            record(BM_OP_INTT, 0, (size_t)Q * n_out * 2);
            if (pl.arena.live) check(ntt_inverse(c, limbs_of(pl.result, Q * n_out * 2, 1, c.n), s));
        }
    }
    bool coef_tail() const { return bm::coef_tail(c, g); }
};

// Buffer sizes of a plan (words) and its group chunk: whole packs, bounded by
// an 8 GiB temporary budget.
static void plan_dims(const Context& c, const SchedView& g, uint32_t n_out, uint32_t Q, Plan& pl) {
    pl.Q = Q;
    pl.ncts = g.tiled ? 1 : g.n_in;
    pl.n_out = n_out;
    const uint32_t lg = g.level;
    // hoisted rounds after HE-C^3: sources and rotated copies per group of a query
    uint32_t per_src = 0;
    if (g.hrotsum) {
        uint32_t bs, gs;
        bsgs_split(g.part, g.dhoist, bs, gs);
        per_src = std::max(bs, gs) - 1;
    }
    if (g.hcomp) per_src = std::max<uint32_t>(per_src, 1);
    // double hoisting sums the rotations in the key-switch scratch: no rotated copies
    const uint32_t copies = g.dhoist ? 0 : per_src;
    const size_t hold = per_src ? ks_ext_words(c, lg - 1) + (size_t)copies * ct_words(c, lg - 1) : 0;
    const size_t acc_words = g.deferred ? (size_t)2 * (c.L + 1 + c.alpha) * c.n : ct_words(c, lg);
    const size_t per_group = (size_t)Q * ((g.encrypted ? 2 : 1) * acc_words + ct_words(c, lg - 1) + hold) * 8;
    const size_t budget = (size_t)8 << 30;
    uint32_t chunk = (uint32_t)std::max<size_t>(1, budget / std::max<size_t>(per_group, 1));
    if (g.compress) chunk = std::max(g.part, chunk / g.part * g.part);
    pl.chunk = std::min(chunk, g.groups);
    pl.hsrc = per_src ? (size_t)Q * pl.chunk : 0;
    pl.helem = pl.hsrc * copies;
    pl.qin_words = (size_t)Q * pl.ncts * ct_words(c, c.L);
    pl.result_words = (size_t)Q * n_out * ct_words(c, 0);
    // hoisted Algorithm 1: rotated copies and products of a chunk of queries within ~4 GiB
    pl.qe = Q;
    if (g.tiled && g.hoisted) {
        const size_t sw = g.fused ? (size_t)2 * (c.L + 1 + c.alpha) * c.n : ct_words(c, c.L);
        const size_t per_q = ((size_t)2 * g.n_in * sw + ks_ext_words(c, c.L)) * 8;
        pl.qe = (uint32_t)std::min<size_t>(Q, std::max<size_t>(1, ((size_t)4 << 30) / per_q));
    }
}

// The plan's device buffers: field and words, the same list for the allocation
// (plan_build) and the host-side estimate (plan_shape).
struct BufSpec {
    uint64_t** field;
    size_t words;
};
// host queries of a plan whose input is at most this many words (256 MiB: 64 top-level
// ring-2^16 queries) are staged through two buffers of that size (plan_run); larger
// batches are copied into qin directly
constexpr size_t kStageWords = (size_t)32 << 20;
static std::vector<BufSpec> plan_buffers(const Context& c, const SchedView& g, Plan& pl) {
    const uint32_t Q = pl.Q, lg = g.level;
    std::vector<BufSpec> b{{&pl.qin, pl.qin_words}, {&pl.result, pl.result_words}};
    const size_t stage = pl.qin_words <= kStageWords ? pl.qin_words : 0;
    b.push_back({&pl.stg[0], stage});
    b.push_back({&pl.stg[1], stage});
    if (g.tiled) {
        // the fused Algorithm 1 keeps its sums on Q_L u P
        const size_t sw = g.fused ? (size_t)2 * (c.L + 1 + c.alpha) * c.n : ct_words(c, c.L);
        // deferred division: the undivided parts of every query in T, no t0
        b.push_back({&pl.t0, g.deferred ? 0 : (size_t)pl.qe * g.n_in * sw});
        b.push_back({&pl.T, (size_t)Q * g.n_in * (g.deferred ? sw : ct_words(c, lg))});
        if (g.hoisted) {
            b.push_back({&pl.qc1, (size_t)Q * (c.L + 1) * c.n});
            b.push_back({&pl.ext, (size_t)pl.qe * ks_ext_words(c, c.L)});
            b.push_back({&pl.R, (size_t)pl.qe * g.n_in * sw});
        }
    }
    b.push_back({&pl.accA, (size_t)Q * pl.chunk *
                               (g.deferred ? (size_t)2 * (c.L + 1 + c.alpha) * c.n : ct_words(c, lg))});
    b.push_back({&pl.accB, (size_t)Q * pl.chunk * ct_words(c, lg - 1)});
    if (g.encrypted) b.push_back({&pl.accT, (size_t)Q * pl.chunk * ct_words(c, lg)});
    if (coef_tail(c, g)) b.push_back({&pl.packs, (size_t)Q * ((pl.chunk + g.part - 1) / g.part) * ct_words(c, 1)});
    if (pl.hsrc) {
        b.push_back({&pl.ext2, pl.hsrc * ks_ext_words(c, lg - 1)});
        b.push_back({&pl.rot, pl.helem * ct_words(c, lg - 1)});
    }
    return b;
}

static size_t words_bytes(size_t w) { return std::max<size_t>(w, 1) * 8; }

// Device bytes of every buffer the plan allocates (the same sizes, in the same
// roles, as plan_build), with the launches of its schedule when rec != nullptr.
static size_t plan_shape(const Context& c, const SchedView& g, uint32_t n_out, uint32_t Q,
                         std::vector<bm_op_launch>* rec) {
    Plan pl;
    plan_dims(c, g, n_out, Q, pl);
    MatchRun run(c, g, nullptr, pl);
    run.rec = rec;
    run.schedule();
    size_t bytes = 0;
    for (const BufSpec& b : plan_buffers(c, g, pl)) bytes += words_bytes(b.words);
    bytes += words_bytes(pl.scratch_words) + words_bytes(pl.arena.host.size());
    return bytes;
}

size_t plan_estimate_bytes(const Context& c, const Gallery& g, uint32_t Q) {
    Layout lo;
    if (make_layout(c, g.n_ids, g.dim, g.part, lo, gallery_kind(g)) != BM_OK) return 0;
    return plan_shape(c, view_of(g), lo.n_out, Q, nullptr);
}

bm_status schedule_launches(const bm_params& p, uint64_t n_ids, uint32_t dim, uint32_t part, uint32_t packing,
                            uint32_t Q, std::vector<bm_op_launch>* ops, size_t* bytes) {
    if (Q == 0 || n_ids == 0) return fail(BM_E_ARG, "empty gallery or batch");
    Context c;
    BM_TRY(context_shape(c, p));
    Layout lo;
    BM_TRY(make_layout(c, n_ids, dim, part, lo, packing));
    const size_t b = plan_shape(c, view_of(lo, part), lo.n_out, Q, ops);
    if (bytes) *bytes = b;
    return BM_OK;
}

bm_status plan_build(Context& c, const Gallery& g, const EvalKeys& ek, uint32_t Q, cudaStream_t cs, Plan*& out) {
    auto* pl = new Plan();
    std::unique_ptr<Plan> guard(pl);
    Layout lo;
    BM_TRY(make_layout(c, g.n_ids, g.dim, g.part, lo, gallery_kind(g)));
    const SchedView v = view_of(g);
    pl->c = &c;
    pl->gid = g.id;
    pl->kid = ek.id;
    plan_dims(c, v, lo.n_out, Q, *pl);
    bool ok = true;
    for (const BufSpec& b : plan_buffers(c, v, *pl)) ok = ok && pl->alloc(*b.field, b.words);
    if (!ok) return fail(BM_E_OOM, "match workspace allocation failed");
    MatchRun run(c, v, &ek, *pl);
    run.schedule();                                     // dry pass
    uint64_t* arr = nullptr;
    ok = pl->alloc(pl->scratch, pl->scratch_words) && pl->alloc(arr, std::max<size_t>(pl->arena.host.size(), 1));
    if (!ok) return fail(BM_E_OOM, "match scratch allocation failed");
    pl->arena.dev = (uint64_t**)arr;
    BM_CUDA_TRY(cudaMemcpy(arr, pl->arena.host.data(), pl->arena.host.size() * sizeof(void*), cudaMemcpyHostToDevice));
    pl->arena.live = true;
    // capture the launch pass once
    BM_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    prof_set_sink(&pl->counts);
    run.s = cs;
    run.schedule();
    prof_set_sink(nullptr);
    cudaError_t e = cudaStreamEndCapture(cs, &pl->graph);
    if (run.err != cudaSuccess) return fail(BM_E_CUDA, std::string("match capture: ") + cudaGetErrorString(run.err));
    BM_CUDA_TRY(e);
    BM_CUDA_TRY(cudaGraphInstantiate(&pl->exec, pl->graph, 0));
    out = guard.release();
    return BM_OK;
}

size_t plan_bytes(const Plan* p) { return p->bytes; }
uint32_t plan_queries(const Plan* p) { return p->Q; }
uint32_t plan_outputs(const Plan* p) { return p->n_out; }
const uint64_t* plan_result(const Plan* p) { return p->result; }

bm_status plan_run(Context& c, const Gallery& g, const EvalKeys& ek, Plan* pl, const Ciphertext* const* queries,
                   uint32_t nq, cudaStream_t s) {
    if (nq == 0 || nq > pl->Q) return fail(BM_E_ARG, "batch larger than the plan");
    // a0: the queries' coefficient-form limbs into the plan's input buffer (padded with the last)
    const size_t per_q = (size_t)pl->ncts * ct_words(c, c.L);
    bool from_host = false;
    for (uint32_t i = 0; i < nq; i++) from_host = from_host || !queries[i]->d_coef;
    if (!from_host || pl->qin_words > kStageWords) {
        // device queries (or a batch too large to stage): straight into qin on s
        for (uint32_t i = 0; i < pl->Q; i++) {
            const Ciphertext& ct = *queries[std::min(i, nq - 1)];
            uint64_t* dst = pl->qin + (size_t)i * per_q;
            if (ct.d_coef) BM_CUDA_TRY(cudaMemcpyAsync(dst, ct.d_coef, per_q * 8, cudaMemcpyDeviceToDevice, s));
            else BM_CUDA_TRY(cudaMemcpyAsync(dst, ct.host.data(), per_q * 8, cudaMemcpyHostToDevice, s));
        }
    } else {
        // host queries: H2D into a staging buffer on the copy stream, which waits only until
        // the move out of that buffer two calls ago has run (so this copy overlaps the
        // previous call's match), then one device-to-device move into qin on s
        if (!pl->cs) {
            BM_CUDA_TRY(cudaStreamCreateWithFlags(&pl->cs, cudaStreamNonBlocking));
            for (int k = 0; k < 2; k++) {
                BM_CUDA_TRY(cudaEventCreateWithFlags(&pl->ev_ready[k], cudaEventDisableTiming));
                BM_CUDA_TRY(cudaEventCreateWithFlags(&pl->ev_free[k], cudaEventDisableTiming));
            }
        }
        const uint32_t k = pl->slot;
        pl->slot ^= 1;
        BM_CUDA_TRY(cudaStreamWaitEvent(pl->cs, pl->ev_free[k], 0));
        for (uint32_t i = 0; i < pl->Q; i++) {
            const Ciphertext& ct = *queries[std::min(i, nq - 1)];
            uint64_t* dst = pl->stg[k] + (size_t)i * per_q;
            if (ct.d_coef) BM_CUDA_TRY(cudaMemcpyAsync(dst, ct.d_coef, per_q * 8, cudaMemcpyDeviceToDevice, pl->cs));
            else BM_CUDA_TRY(cudaMemcpyAsync(dst, ct.host.data(), per_q * 8, cudaMemcpyHostToDevice, pl->cs));
        }
        BM_CUDA_TRY(cudaEventRecord(pl->ev_ready[k], pl->cs));
        BM_CUDA_TRY(cudaStreamWaitEvent(s, pl->ev_ready[k], 0));
        BM_CUDA_TRY(cudaMemcpyAsync(pl->qin, pl->stg[k], pl->Q * per_q * 8, cudaMemcpyDeviceToDevice, s));
        BM_CUDA_TRY(cudaEventRecord(pl->ev_free[k], s));
    }
    if (prof_timing()) {
        // per-launch timing: run the same launches eagerly so each gets its event pair
        MatchRun run(c, view_of(g), &ek, *pl);
        run.s = s;
        run.schedule();
        if (run.err != cudaSuccess) return fail(BM_E_CUDA, std::string("match: ") + cudaGetErrorString(run.err));
    } else {
        BM_CUDA_TRY(cudaGraphLaunch(pl->exec, s));
        prof_add(pl->counts);
    }
    return BM_OK;
}

static Plan* find_plan(Context& c, uint64_t gid, uint64_t kid, uint32_t Q) {
    for (Plan* p : c.plans)
        if (p->gid == gid && p->kid == kid && p->Q == Q) return p;
    return nullptr;
}

}  // namespace bm

extern "C" {

bm_status bm_plan_estimate(const bm_params* params, uint64_t n_ids, uint32_t dim, uint32_t part_size,
                           uint32_t packing, uint32_t n_queries, bm_op_launch* ops, size_t ops_cap,
                           size_t* n_ops, uint64_t* plan_bytes_out) {
    if (!params) return fail(BM_E_ARG, "null parameters");
    std::vector<bm_op_launch> v;
    size_t bytes = 0;
    BM_TRY(schedule_launches(*params, n_ids, dim, part_size, packing, n_queries, &v, &bytes));
    if (ops) std::copy(v.begin(), v.begin() + std::min(ops_cap, v.size()), ops);
    if (n_ops) *n_ops = v.size();
    if (plan_bytes_out) *plan_bytes_out = bytes;
    return BM_OK;
}

namespace bm {
// bm_match and bm_match_async: with sync, returns once the result is complete; else
// the result carries an event recorded on the stream after its copy
static bm_status match_impl(bm_context* ctxh, const bm_eval_keys* evk, const bm_gallery* gal,
                            bm_ciphertext* const* queries, uint32_t n_queries, void* stream, bm_result** out,
                            bool sync) {
    if (!ctxh || !evk || !gal || !queries || !out || n_queries == 0) return fail(BM_E_ARG, "null argument");
    Context& c = ctxh->c;
    const Gallery& g = gal->g;
    if (g.ctx != &c || evk->k.ctx != &c) return fail(BM_E_ARG, "handles belong to another context");
    const uint32_t ncts = g.tiled ? 1 : g.n_in;
    for (uint32_t i = 0; i < n_queries; i++) {
        if (!queries[i]) return fail(BM_E_ARG, "null query");
        if (queries[i]->ct.n_cts != ncts || queries[i]->ct.level != c.L)
            return fail(BM_E_LEVEL, "query layout does not match the gallery's schedule");
    }
    Layout lo;
    BM_TRY(make_layout(c, g.n_ids, g.dim, g.part, lo, gallery_kind(g)));
    for (int32_t r : schedule_rotations(c, lo, g.part))
        if (!evk->k.keys.count(galois_of(c, r))) return fail(BM_E_KEY_MISSING, "missing rotation key");
    BM_CUDA_TRY(cudaSetDevice(c.device));
    NvtxRange range("bm_match");
    cudaStream_t s = (cudaStream_t)stream;
    Plan* pl = find_plan(c, g.id, evk->k.id, n_queries);
    if (!pl) {
        BM_TRY(plan_build(c, g, evk->k, n_queries, c.stream, pl));
        c.plans.push_back(pl);
    }
    std::vector<const Ciphertext*> qs(n_queries);
    for (uint32_t i = 0; i < n_queries; i++) qs[i] = &queries[i]->ct;
    BM_TRY(plan_run(c, g, evk->k, pl, qs.data(), n_queries, s));
    auto* rh = new bm_result();
    rh->ref.attach(&c);
    Result& res = rh->r;
    res.ctx = &c;
    res.n_queries = n_queries;
    res.n_out = lo.n_out;
    res.n_ids = g.n_ids;
    res.dim = g.dim;
    res.part = g.part;
    res.packed = g.compress;
    res.packing = g.packing;
    res.scale = result_scale(c, g);
    cudaError_t e = cudaMallocAsync((void**)&res.d_data, pl->result_words * 8, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res.d_data, pl->result, pl->result_words * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && sync) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && !sync) {
        e = cudaEventCreateWithFlags(&res.ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(res.ready, s);
    }
    if (e != cudaSuccess) {
        if (!sync) cudaStreamSynchronize(s);   // nothing of the result may still be in flight
        delete rh;
        return fail(BM_E_CUDA, std::string("match: ") + cudaGetErrorString(e));
    }
    *out = rh;
    return BM_OK;
}
}  // namespace bm

bm_status bm_match(bm_context* ctxh, const bm_eval_keys* evk, const bm_gallery* gal, bm_ciphertext* const* queries,
                   uint32_t n_queries, void* stream, bm_result** out) {
    return match_impl(ctxh, evk, gal, queries, n_queries, stream, out, true);
}

bm_status bm_match_async(bm_context* ctxh, const bm_eval_keys* evk, const bm_gallery* gal,
                         bm_ciphertext* const* queries, uint32_t n_queries, void* stream, bm_result** out) {
    return match_impl(ctxh, evk, gal, queries, n_queries, stream, out, false);
}

bm_status bm_result_info(const bm_result* r, uint32_t* n_queries, uint32_t* n_out, uint32_t* packed_out) {
    if (!r) return fail(BM_E_ARG, "null result");
    if (n_queries) *n_queries = r->r.n_queries;
    if (n_out) *n_out = r->r.n_out;
    if (packed_out) *packed_out = r->r.packed;
    return BM_OK;
}

bm_status bm_result_export(const bm_result* r, uint32_t query_index, uint64_t* out, size_t capacity) {
    if (!r || !out) return fail(BM_E_ARG, "null argument");
    const Result& res = r->r;
    const Context& c = *res.ctx;
    if (query_index >= res.n_queries) return fail(BM_E_ARG, "query index out of range");
    const size_t words = (size_t)res.n_out * ct_words(c, 0);
    if (capacity < words) return fail(BM_E_ARG, "capacity too small");
    BM_CUDA_TRY(cudaSetDevice(c.device));
    if (res.ready) BM_CUDA_TRY(cudaEventSynchronize(res.ready));
    // on the context's non-blocking stream: the copy does not wait for work the caller
    // has enqueued since (a later match), as one on the legacy stream would
    BM_CUDA_TRY(cudaMemcpyAsync(out, res.d_data + (size_t)query_index * words, words * 8, cudaMemcpyDeviceToHost,
                                c.stream));
    BM_CUDA_TRY(cudaStreamSynchronize(c.stream));
    return BM_OK;
}

void bm_result_destroy(bm_result* r) { delete r; }

bm_status bm_decrypt_scores(bm_context* ctxh, const bm_secret_key* sk, const bm_result* r, uint32_t query_index,
                            double* scores, uint64_t n_ids, int64_t* rank1, double* rank1_score) {
    if (!ctxh || !sk || !r || !scores) return fail(BM_E_ARG, "null argument");
    Context& c = ctxh->c;
    const Result& res = r->r;
    if (query_index >= res.n_queries) return fail(BM_E_ARG, "query index out of range");
    if (n_ids != res.n_ids) return fail(BM_E_ARG, "n_ids does not match the gallery");
    BM_CUDA_TRY(cudaSetDevice(c.device));
    cudaStream_t s = c.stream;
    if (res.ready) BM_CUDA_TRY(cudaStreamWaitEvent(s, res.ready, 0));
    const size_t n = c.n, nout = res.n_out;
    DevBuf t;
    BM_CUDA_TRY(t.alloc(nout * 2 * n));
    BM_CUDA_TRY(cudaMemcpyAsync(t.p, res.d_data + (size_t)query_index * nout * 2 * n, nout * 2 * n * 8,
                                cudaMemcpyDeviceToDevice, s));
    // m = c0 + c1 * s  (mod q_0)
    LimbBatch c1 = limbs_of(t.p + n, (uint32_t)nout, 1, 2 * n);
    BM_CUDA_TRY(ntt_forward(c, c1, s));
    BM_CUDA_TRY(pointwise_mul(c, c1, limbs_of(sk->k.d_ntt, (uint32_t)nout, 1, 0), c1, s));
    BM_CUDA_TRY(ntt_inverse(c, c1, s));
    LimbBatch c0 = limbs_of(t.p, (uint32_t)nout, 1, 2 * n);
    BM_CUDA_TRY(pointwise_addsub(c, c0, c1, c0, false, s));
    std::vector<uint64_t> h(nout * 2 * n);
    BM_CUDA_TRY(cudaMemcpyAsync(h.data(), t.p, h.size() * 8, cudaMemcpyDeviceToHost, s));
    BM_CUDA_TRY(cudaStreamSynchronize(s));
    const uint64_t q0 = c.primes[0];
    const uint32_t part = res.part, G = c.slots / part;
    const bool cplx = res.packing == BM_PACK_COMPLEX;
    const uint64_t per_group = cplx ? 2ull * G : G;
    std::vector<double> coef(n);
    std::vector<std::complex<double>> slots(c.slots);
    std::vector<std::vector<std::complex<double>>> dec(nout);
    for (size_t o = 0; o < nout; o++) {
        for (size_t i = 0; i < n; i++) {
            const uint64_t v = h[o * 2 * n + i];
            coef[i] = v > q0 / 2 ? -(double)(q0 - v) : (double)v;
        }
        decode_complex(c, coef.data(), res.scale > 0 ? res.scale : c.scale, slots.data());
        dec[o] = slots;
    }
    int64_t best = -1;
    double best_score = -INFINITY;
    for (uint64_t id = 0; id < n_ids; id++) {
        // group, window and part (real / imaginary) of the identity; packed outputs
        // hold group g at offset g mod part of pack g / part
        const uint64_t grp = id / per_group, w = id % per_group, u = w % G;
        const bool im = w >= G;
        const std::complex<double> z = res.packed ? dec[grp / part][u * part + grp % part] : dec[grp][u * part];
        const double v = im ? z.imag() : z.real();
        scores[id] = v;
        if (v > best_score) {
            best_score = v;
            best = (int64_t)id;
        }
    }
    if (rank1) *rank1 = best;
    if (rank1_score) *rank1_score = best_score;
    return BM_OK;
}

// ---------------------------------------------------------------------------
// single operations
// ---------------------------------------------------------------------------

bm_status bm_poly_mul(bm_context* ctxh, const uint64_t* a, const uint64_t* b, uint64_t* out, uint32_t n_limbs) {
    if (!ctxh || !a || !b || !out) return fail(BM_E_ARG, "null argument");
    Context& c = ctxh->c;
    if (n_limbs == 0 || n_limbs > c.nb) return fail(BM_E_ARG, "n_limbs out of range");
    BM_CUDA_TRY(cudaSetDevice(c.device));
    cudaStream_t s = c.stream;
    const size_t w = (size_t)n_limbs * c.n;
    DevBuf da, db;
    BM_CUDA_TRY(da.alloc(w));
    BM_CUDA_TRY(db.alloc(w));
    BM_CUDA_TRY(cudaMemcpyAsync(da.p, a, w * 8, cudaMemcpyHostToDevice, s));
    BM_CUDA_TRY(cudaMemcpyAsync(db.p, b, w * 8, cudaMemcpyHostToDevice, s));
    BM_CUDA_TRY(ntt_forward(c, packed(c, da.p, 1, n_limbs), s));
    BM_CUDA_TRY(ntt_forward(c, packed(c, db.p, 1, n_limbs), s));
    BM_CUDA_TRY(to_montgomery(c, packed(c, db.p, 1, n_limbs), false, s));
    BM_CUDA_TRY(pointwise_mul(c, packed(c, da.p, 1, n_limbs), packed(c, db.p, 1, n_limbs), packed(c, da.p, 1, n_limbs), s));
    BM_CUDA_TRY(ntt_inverse(c, packed(c, da.p, 1, n_limbs), s));
    BM_CUDA_TRY(cudaMemcpyAsync(out, da.p, w * 8, cudaMemcpyDeviceToHost, s));
    BM_CUDA_TRY(cudaStreamSynchronize(s));
    return BM_OK;
}

static bm_status ct_op(bm_context* ctxh, const bm_ciphertext* in, int op, const bm_eval_keys* evk, int32_t rot,
                       bm_ciphertext** out) {
    if (!ctxh || !in || !out) return fail(BM_E_ARG, "null argument");
    Context& c = ctxh->c;
    const Ciphertext& ct = in->ct;
    const uint32_t l = ct.level, B = ct.n_cts;
    const uint32_t lo = op == 1 ? l - 1 : l;
    if (op == 1 && l == 0) return fail(BM_E_LEVEL, "cannot rescale at level 0");
    const uint64_t* key = nullptr;
    if (op == 0) {
        auto it = evk->k.keys.find(galois_of(c, rot));
        if (it == evk->k.keys.end()) return fail(BM_E_KEY_MISSING, "no key for this rotation");
        key = it->second;
    }
    BM_CUDA_TRY(cudaSetDevice(c.device));
    cudaStream_t s = c.stream;
    DevBuf din, dout, scr, lists;
    BM_CUDA_TRY(din.alloc(ct.host.size()));
    BM_CUDA_TRY(dout.alloc((size_t)B * ct_words(c, lo)));
    BM_CUDA_TRY(scr.alloc(std::max(ks_scratch_words(c, l, B), l ? rescale_scratch_words(c, l, B) : 0)));
    std::vector<uint64_t*> h;
    for (uint32_t b = 0; b < B; b++) h.push_back(din.p + (size_t)b * ct_words(c, l));
    for (uint32_t b = 0; b < B; b++) h.push_back(dout.p + (size_t)b * ct_words(c, lo));
    BM_CUDA_TRY(lists.alloc(h.size()));
    BM_CUDA_TRY(cudaMemcpyAsync(lists.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice, s));
    BM_CUDA_TRY(cudaMemcpyAsync(din.p, ct.host.data(), ct.host.size() * 8, cudaMemcpyHostToDevice, s));
    BM_CUDA_TRY(ntt_forward(c, packed(c, din.p, B * 2, l + 1), s));
    uint64_t* const* lin = (uint64_t* const*)lists.p;
    uint64_t* const* lout = lin + B;
    if (op == 0) BM_CUDA_TRY(ks_rotate(c, key, galois_of(c, rot), l, B, lin, lout, nullptr, scr.p, s));
    else BM_CUDA_TRY(rescale(c, l, B, lin, lout, scr.p, s));
    BM_CUDA_TRY(ntt_inverse(c, packed(c, dout.p, B * 2, lo + 1), s));
    auto* ch = new bm_ciphertext();
    ch->ref.attach(&c);
    ch->ct.ctx = &c;
    ch->ct.n_cts = B;
    ch->ct.level = lo;
    ch->ct.host.resize((size_t)B * ct_words(c, lo));
    cudaError_t e = cudaMemcpyAsync(ch->ct.host.data(), dout.p, ch->ct.host.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete ch;
        return fail(BM_E_CUDA, std::string("ct op: ") + cudaGetErrorString(e));
    }
    *out = ch;
    return BM_OK;
}

bm_status bm_ct_rotate(bm_context* ctx, const bm_eval_keys* evk, const bm_ciphertext* in, int32_t rotation,
                       bm_ciphertext** out) {
    if (!evk) return fail(BM_E_ARG, "null keys");
    return ct_op(ctx, in, 0, evk, rotation, out);
}

bm_status bm_ct_rescale(bm_context* ctx, const bm_ciphertext* in, bm_ciphertext** out) {
    return ct_op(ctx, in, 1, nullptr, 0, out);
}

bm_status bm_ntt_forward(bm_context* ctxh, uint64_t* d_data, uint32_t n_polys, uint32_t n_limbs, void* stream) {
    if (!ctxh || !d_data || n_limbs == 0 || n_limbs > ctxh->c.nb) return fail(BM_E_ARG, "bad argument");
    BM_CUDA_TRY(ntt_forward(ctxh->c, packed(ctxh->c, d_data, n_polys, n_limbs), (cudaStream_t)stream));
    return BM_OK;
}

bm_status bm_ntt_inverse(bm_context* ctxh, uint64_t* d_data, uint32_t n_polys, uint32_t n_limbs, void* stream) {
    if (!ctxh || !d_data || n_limbs == 0 || n_limbs > ctxh->c.nb) return fail(BM_E_ARG, "bad argument");
    BM_CUDA_TRY(ntt_inverse(ctxh->c, packed(ctxh->c, d_data, n_polys, n_limbs), (cudaStream_t)stream));
    return BM_OK;
}

}  // extern "C"
