// bm_internal.h -- internal types of the Blind-Match GPU library.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <complex>
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "blindmatch.h"
#include "bm_math.cuh"

namespace bm {

// Page-locked host memory from a caching pool: cudaHostAlloc (portable) on a miss, freed
// blocks kept by exact size (up to 2 GiB in all) for the next request of that
// size, so a host ciphertext is copied to and from the device by DMA without a
// page-locking call per object.  Pageable memory when page-locking fails (no
// device).  Thread-safe.
void* pinned_alloc(size_t bytes);
void pinned_free(void* p, size_t bytes);
template <class T>
struct PinnedAlloc {
    using value_type = T;
    PinnedAlloc() = default;
    template <class U>
    PinnedAlloc(const PinnedAlloc<U>&) {}
    T* allocate(size_t n) { return static_cast<T*>(pinned_alloc(n * sizeof(T))); }
    void deallocate(T* p, size_t n) { pinned_free(p, n * sizeof(T)); }
    template <class U>
    bool operator==(const PinnedAlloc<U>&) const { return true; }
    template <class U>
    bool operator!=(const PinnedAlloc<U>&) const { return false; }
};
using HostWords = std::vector<uint64_t, PinnedAlloc<uint64_t>>;

constexpr int MAXB = BM_MAX_Q + BM_MAX_P;   // primes in the full basis Q_L u P
constexpr int MAXD = 4;                     // key-switching digits
constexpr int MAXDS = 3;                    // limbs per digit
constexpr int MAXSP = BM_MAX_P + 1;         // special limbs of a fused division (P and up to two q-primes)
constexpr int kMdrDrops = 2;                // fused divisions: by q_L P, and by q_(L-1) q_L P

// Per-prime constants and twiddle tables, passed to kernels by value.
struct DevTables {
    uint64_t q[MAXB];
    uint64_t qneg[MAXB];        // -q^{-1} mod 2^64 (Montgomery)
    uint64_t rsh[MAXB];         // floor(2^64 / q): reduces any 64-bit word with one mulhi
    uint64_t r2[MAXB];          // 2^128 mod q: mont(x, r2) = x * 2^64 mod q
    uint64_t ninv[MAXB], ninv_sh[MAXB];
    const ulonglong2* tw[MAXB];     // forward: (psi^brv(k), Shoup companion), k < N
    const ulonglong2* itw[MAXB];    // inverse: (psi^-brv(k), companion)
};

// A set of limbs: n_polys polynomials at base + poly*poly_stride (words); limb k of
// each (k < nl) starts at (limb_off + k) * N and uses prime prime(k) (4-bit fields
// of `pk`, so kernels read them with shifts instead of indexing an array).
struct LimbBatch {
    uint64_t* base;
    uint32_t n_polys;
    uint64_t poly_stride;
    uint32_t limb_off;
    uint32_t nl;
    uint64_t pk;
    __host__ __device__ __forceinline__ int prime(uint32_t k) const { return (int)((pk >> (4 * k)) & 15); }
    __host__ __device__ __forceinline__ void set(uint32_t k, uint32_t p) {
        pk = (pk & ~(15ull << (4 * k))) | ((uint64_t)p << (4 * k));
    }
};

// Constants of key switching at one level (device table, one entry per level).
struct KsLevelConst {
    uint32_t nd, nlx;                          // digits present; limbs of Q_l u P
    uint32_t dstart[MAXD], dsz[MAXD];          // Q-limb range of each digit at this level
    ulonglong2 up_hinv[MAXD][MAXDS];           // (D/d_i)^-1 mod d_i            (Shoup pairs)
    ulonglong2 up_hat[MAXD][MAXDS][MAXB];      // (D/d_i) mod t_jj, jj over Q_l u P
    ulonglong2 dn_hinv[MAXSP];                 // N^-1 (P/p_i)^-1 mod p_i
    ulonglong2 dn_hat[MAXSP][MAXB];            // (P/p_i) mod q_j
    ulonglong2 pinv[MAXB];                     // P^-1 mod q_j
    uint64_t pmont[MAXB];                      // P * 2^64 mod q_j (Montgomery form of P)
};

// A match schedule for one (gallery, key set, batch size): persistent device
// buffers and the whole schedule captured as a CUDA graph (api.cu).
struct Plan;
void destroy_plan(Plan* p);

// Precomputed tables of the canonical-embedding encoder (host.cpp).
struct EncoderTables {
    std::vector<std::complex<double>> root;   // exp(2 pi i k / N), k < N/2
    std::vector<uint32_t> brv;                // bit reversal of log N bits
    std::vector<std::complex<double>> zeta;   // exp(i pi k / N), k < N
    std::vector<uint32_t> pos, cpos;          // slot j -> index t of 5^j = 2t+1, and of -5^j
};

// Batch buckets of the standalone NTT: bucket k holds batches of 2^(k-1) + 1 .. 2^k limbs
// (bucket 0: one limb; the last: 2^(kNttBuckets-2) + 1 limbs and more).
constexpr int kNttBuckets = BM_NTT_BUCKETS;
inline int ntt_bucket(uint32_t limbs) {
    int k = 0;
    while (k + 1 < kNttBuckets && (1u << k) < limbs) k++;
    return k;
}
constexpr int kNttShapes = 3;

struct Context {
    bm_params params{};
    int device = 0;
    uint32_t log_n = 0, n = 0, slots = 0, L = 0, alpha = 0, nb = 0;
    std::vector<uint64_t> primes;             // q_0..q_L, p_0..p_(alpha-1)
    std::vector<uint64_t> psi;
    std::vector<std::vector<uint32_t>> digits;   // Q-limb indices of each digit
    DevTables tab{};
    void* d_twiddles = nullptr;
    cudaStream_t stream = nullptr;            // for client-side helpers (keygen, encrypt)
    uint64_t P_mod[MAXB]{};                   // P mod each prime
    double scale = 0;
    EncoderTables enc;
    std::vector<KsLevelConst> h_ksc;          // key-switching constants per level (host copy)
    KsLevelConst* d_ksc = nullptr;            // ... and on the device
    KsLevelConst h_ksc_mdr[kMdrDrops]{};      // ModDown + Rescale at the top level, [d - 1]: special set
    KsLevelConst* d_ksc_mdr = nullptr;        //   {q_(L-d+1)..q_L} u P (only nlx, dn_hinv, dn_hat, pinv set)
    ulonglong2* d_qlinv = nullptr;            // [level][j]: q_level^-1 mod q_j (Shoup pairs), for rescale
    uint32_t ks_wide_batch[BM_MAX_Q] = {1u << 30, 1u << 30, 1u << 30, 1u << 30, 1u << 30, 1u << 30};
                                              // per level: key-switch batches of at least this many
                                              // ciphertexts use 16 coefficients per thread (set by
                                              // bm_autotune_keyswitch / bm_set_ks_wide_batch / BM_KS_WIDE_BATCH)
    uint8_t ntt_shape[kNttBuckets] = {};      // standalone NTT shape per batch bucket (ntt_bucket):
                                              // set by bm_autotune_ntt / bm_set_ntt_shape
    uint64_t next_id = 1;                     // ids of galleries and key sets (plan cache keys)
    std::vector<Plan*> plans;
    // lifetime: every handle made from the context holds a reference; the context
    // is freed when it was destroyed and its last handle is gone
    std::atomic<int> refs{0};
    std::atomic<bool> destroy_requested{false};
    struct bm_context* owner = nullptr;
};
void ctx_retain(Context* c);
void context_free(struct bm_context* ctx);
void ctx_release(Context* c);   // frees a destroyed context with its last handle

// Reference to the context a handle was made from; declared first in each
// handle so that it is released after the handle's own resources.
struct CtxRef {
    Context* c = nullptr;
    CtxRef() = default;
    CtxRef(const CtxRef&) = delete;
    CtxRef& operator=(const CtxRef&) = delete;
    void attach(Context* x) {
        c = x;
        ctx_retain(c);
    }
    ~CtxRef() {
        if (c) ctx_release(c);
    }
};
// destroys every cached plan that uses the gallery or key set `id`
void drop_plans(Context& c, uint64_t id);
struct Gallery;
struct EvalKeys;
struct Ciphertext;
bm_status plan_build(Context& c, const Gallery& g, const EvalKeys& ek, uint32_t Q, cudaStream_t capture,
                     Plan*& out);
// enqueues the match of nq <= Q queries on s (graph replay; eager when profiling
// with timing); the score ciphertexts land in plan_result(), [Q][n_out][2][N]
bm_status plan_run(Context& c, const Gallery& g, const EvalKeys& ek, Plan* p, const Ciphertext* const* queries,
                   uint32_t nq, cudaStream_t s);
size_t plan_bytes(const Plan* p);
// scale of the score ciphertexts of a match against g
double result_scale(const Context& c, const Gallery& g);
// device bytes the plan of Q queries for this gallery will hold (host only)
size_t plan_estimate_bytes(const Context& c, const Gallery& g, uint32_t Q);
// host only: the launches and plan bytes of a match for (params, n_ids, dim, part, Q)
bm_status schedule_launches(const bm_params& p, uint64_t n_ids, uint32_t dim, uint32_t part, uint32_t packing,
                            uint32_t Q, std::vector<bm_op_launch>* ops, size_t* bytes);
uint32_t plan_queries(const Plan* p);
uint32_t plan_outputs(const Plan* p);
const uint64_t* plan_result(const Plan* p);

struct SecretKey {
    Context* ctx;
    std::vector<int64_t> coeffs;             // ternary, length N
    uint64_t* d_ntt = nullptr;                // NTT(s) on every prime of the full basis, Montgomery form
};

struct PublicKey {
    Context* ctx;
    uint64_t* d_ntt = nullptr;                // [2][L+1][N] NTT + Montgomery
};

struct EvalKeys {
    Context* ctx;
    uint64_t id = 0;
    uint32_t dim = 0, part = 0;
    std::map<uint64_t, uint64_t*> keys;       // galois element -> [dnum][2][nb][N] NTT + Montgomery
    uint64_t* relin = nullptr;                // key from s^2 to s, same layout (encrypted galleries)
    ~EvalKeys();
};

struct Gallery {
    Context* ctx;
    uint64_t id = 0;
    uint64_t n_ids = 0;
    uint32_t dim = 0, part = 0, n_in = 0, groups = 0, level = 0;  // level of the gallery pts
    bool tiled = true;                        // queries arrive tiled (Algorithm 1 on the server)
    bool compress = true;                     // outputs are masked and packed
    uint32_t packing = BM_PACK_REAL;          // BM_PACK_COMPLEX: a second identity in the imaginary parts
    bool encrypted = false;                   // d_pts holds ciphertexts [groups][n_in][2][level+1][N]
    uint32_t sched = 0;                       // hoisted forms of the schedule (BM_SCHED_* flags)
    uint64_t* d_pts = nullptr;                // [groups][n_in][level+1][N] NTT + Montgomery
    uint64_t* d_masks = nullptr;              // [n_in][L+1][N] Algorithm-1 masks (tiled only)
    uint64_t* d_masks_hat = nullptr;          // [n_in][L+1][N] their transform over the parts (circ_prepare)
    ulonglong2* d_circ_tw = nullptr;          // [L+1][n_in] twiddles of that transform
    uint64_t* d_masks_hat_ext = nullptr;      // [n_in][L+1+alpha][N] the same on Q_L u P (fused Algorithm 1)
    uint64_t* d_pts_ext = nullptr;            // [groups][n_in][L+1+alpha][N] d_pts on Q_L u P (deferred division)
    ulonglong2* d_circ_tw_ext = nullptr;      // [L+1+alpha][n_in]
    uint64_t* d_cmask = nullptr;              // [level][N] compression mask at level-1
    // [part][level+alpha][N]: the compression mask on Q_(level-1) u P rotated right by each
    // group offset o of a pack (BM_SCHED_FUSED_COMPRESSION), NTT + Montgomery
    uint64_t* d_cmask_rot = nullptr;
    ~Gallery();
};

struct Ciphertext {
    Context* ctx;
    uint32_t n_cts = 1, level = 0;
    HostWords host;                           // [n_cts][2][level+1][N] coefficient form, page-locked
    uint64_t* d_coef = nullptr;               // optional staged device copy, coefficient form
    ~Ciphertext();
};

struct Result {
    Context* ctx;
    uint32_t n_queries = 0, n_out = 0;
    uint64_t n_ids = 0;
    uint32_t dim = 0, part = 0;
    bool packed = true;
    uint32_t packing = BM_PACK_REAL;          // slot packing of the gallery the result came from
    double scale = 0;                         // scale of the score ciphertexts
    uint64_t* d_data = nullptr;               // [n_queries][n_out][2][N] coefficient form, level 0
    cudaEvent_t ready = nullptr;              // asynchronous match: recorded after d_data's copy
    ~Result();
};

// Galois element 5^r mod 2N of a left rotation by r slots (negative r: right).
inline uint64_t galois_of(const Context& c, int32_t rot) {
    int64_t r = rot % (int64_t)c.slots;
    if (r < 0) r += c.slots;
    return h_powmod(5, (uint64_t)r, 2ull * c.n);
}
// words of one ciphertext at `level`: [2][level+1][N]
inline size_t ct_words(const Context& c, uint32_t level) { return (size_t)2 * (level + 1) * c.n; }

// RAII device buffer
struct DevBuf {
    uint64_t* p = nullptr;
    size_t words = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t w) {
        words = w;
        return cudaMalloc(&p, std::max<size_t>(w, 1) * sizeof(uint64_t));
    }
    uint64_t* release() {
        uint64_t* r = p;
        p = nullptr;
        return r;
    }
};

inline LimbBatch limbs_of(uint64_t* base, uint32_t n_polys, uint32_t nl, uint64_t poly_stride,
                          uint32_t first_prime = 0, uint32_t limb_off = 0) {
    LimbBatch b{base, n_polys, poly_stride, limb_off, nl, {}};
    for (uint32_t k = 0; k < nl; k++) b.set(k, (uint8_t)(first_prime + k));
    return b;
}
// polys of `nl` consecutive limbs starting at prime 0, packed
inline LimbBatch packed(const Context& c, uint64_t* base, uint32_t n_polys, uint32_t nl) {
    return limbs_of(base, n_polys, nl, (uint64_t)nl * c.n);
}


// ---- error reporting ----
void set_error(const std::string& msg);
#define BM_CUDA_TRY(expr)                                                              \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            ::bm::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));       \
            return BM_E_CUDA;                                                          \
        }                                                                              \
    } while (0)

// ---- host-side number theory, randomness, encoding (host.cpp) ----
bool is_prime_u64(uint64_t n);
bool gen_primes(uint32_t log_n, const std::vector<uint32_t>& bits, std::vector<uint64_t>& out);
uint64_t find_psi(uint64_t q, uint32_t log_n);
void philox4x64_10(uint64_t k0, uint64_t k1, const uint64_t ctr[4], uint64_t out[4]);
enum : uint64_t {
    TAG_SECRET = 1, TAG_PK_A = 2, TAG_PK_E = 3, TAG_RK_A = 4, TAG_RK_E = 5,
    TAG_ENC_V = 6, TAG_ENC_E0 = 7, TAG_ENC_E1 = 8, TAG_RLK_A = 9, TAG_RLK_E = 10
};
void sample_uniform(uint64_t seed, uint64_t tag, uint64_t obj, uint64_t limb, uint64_t q,
                    uint64_t* out, uint32_t n);
void sample_gauss(uint64_t seed, uint64_t tag, uint64_t obj, double sigma, int64_t* out, uint32_t n);
void sample_zo(uint64_t seed, uint64_t tag, uint64_t obj, int64_t* out, uint32_t n);
void sample_secret(uint64_t seed, uint32_t hw, uint32_t log_n, int64_t* out);
void cdt_table(double sigma, uint32_t kmax, uint64_t* table);
void encoder_tables(Context& ctx);
// round(scale * tau^{-1}(z)) for real slot values z[slots]; coefficients out[N]
void encode_real(const Context& ctx, const double* z, double scale, int64_t* out);
// slots of integer coefficients / scale (real parts)
void decode_real(const Context& ctx, const double* coeffs, double scale, double* z);
// the same for complex slot values
void encode_complex(const Context& ctx, const std::complex<double>* z, double scale, int64_t* out);
void decode_complex(const Context& ctx, const double* coeffs, double scale, std::complex<double>* z);

// ---- launch accounting (profile.cpp) ----
// Every launcher brackets its kernel with a ProfScope: launches and algorithmic
// bytes are always counted per kernel class; with timing enabled a CUDA event
// pair is recorded around the launch on its stream.
// 32-bit multiply results of the modular arithmetic (the accounting of the
// roofline): a Shoup product with a precomputed companion = the high half of
// x*w' (four 32x32 partial products, both halves: 8) and the low halves of x*w
// and of the quotient times q (4 each) = 16, as one butterfly; a sum of products
// reduced once = 8 per product (the full 128-bit product, or four 32 x 32 -> 64
// multiply-adds of 30-bit pieces, two multiplies each) plus one Montgomery
// reduction per sum (the low half of t*(-q^-1), 4, and the high half of m*q, 8) = 12.
constexpr double kShoupMul = 16, kProdMul = 8, kRedcMul = 12;

struct ProfScope {
    ProfScope(int kind, cudaStream_t s, double alg_bytes, double alg_ops = 0, uint32_t launches = 1);
    ~ProfScope();
    int kind;
    cudaStream_t s;
    int slot;
};
// Launch counts of a captured graph: while a sink is set on this thread, ProfScope
// adds to it instead of the global counters (and records no events); each replay
// of the graph then adds the sink's counts with prof_add.
struct ProfSink {
    uint64_t launches[BM_KERNEL_KINDS] = {};
    double bytes[BM_KERNEL_KINDS] = {};
    double ops[BM_KERNEL_KINDS] = {};
};
void prof_set_sink(ProfSink* sink);
void prof_add(const ProfSink& counts);
bool prof_timing();

// ---- kernel launchers (kernels.cu) ----
cudaError_t ntt_forward(const Context& c, const LimbBatch& b, cudaStream_t s);
cudaError_t ntt_inverse(const Context& c, const LimbBatch& b, cudaStream_t s);
// the same in a given shape (0..kNttShapes-1), whatever the context's choice
cudaError_t ntt_dispatch_shape(const Context& c, const LimbBatch& b, bool inv, int shape, cudaStream_t s);
// x -> x * 2^64 mod q (Montgomery form) / back, on a limb batch
cudaError_t to_montgomery(const Context& c, const LimbBatch& b, bool inverse, cudaStream_t s);
// out[poly][k][i] = signed v[poly][i] mod q_k on each limb (v: device int64[n_polys][N])
cudaError_t lift_signed(const Context& c, const int64_t* d_v, const LimbBatch& out, cudaStream_t s);

// Rotation (automorphism + hybrid key switch) of B ciphertexts at `level`, NTT form:
// out[b] = Rot(in[b]) (+ add[b] if add != nullptr).  in/out/add are device arrays of
// B pointers to [2][level+1][N] ciphertexts; out may alias add, not in.
cudaError_t ks_rotate(const Context& c, const uint64_t* key, uint64_t galois, uint32_t level,
                      uint32_t B, uint64_t* const* d_in, uint64_t* const* d_out,
                      uint64_t* const* d_add, uint64_t* scratch, cudaStream_t s);
size_t ks_scratch_words(const Context& c, uint32_t level, uint32_t B);
// the same rotation in six fused kernels (ks_fused.cu), for rings 2^12 and 2^16
bool ks_fused_supported(const Context& c);
cudaError_t ks_rotate_fused(const Context& c, const uint64_t* key, uint64_t galois, uint32_t level,
                            uint32_t B, uint64_t* const* d_in, uint64_t* const* d_out,
                            uint64_t* const* d_add, uint64_t* scratch, cudaStream_t s);
// the same with the kernel shape forced: wide = 16 coefficients per thread
// (only where ks_has_wide), else 4
bool ks_has_wide(const Context& c);
cudaError_t ks_rotate_fused_shape(const Context& c, bool wide, const uint64_t* key, uint64_t galois,
                                  uint32_t level, uint32_t B, uint64_t* const* d_in, uint64_t* const* d_out,
                                  uint64_t* const* d_add, uint64_t* scratch, cudaStream_t s);
// Hoisted rotations (rings 2^12 and 2^16): the basis extension of c1 of B ciphertexts
// at `level`, every extended limb in NTT order -- ext [B][nd][nlx][N] (ks_ext_words
// per ciphertext; scratch ks_modup_scratch_words) -- then E rotations, element e
// rotating src[e] by Galois element gal_of[e] with key key_of[e] from its
// extension ext_of[e] into out[e] (scratch ks_hoisted_scratch_words).  The same
// messages as ks_rotate; the bits differ (the automorphism follows ModUp).
size_t ks_ext_words(const Context& c, uint32_t level);
size_t ks_modup_scratch_words(const Context& c, uint32_t level, uint32_t B);
size_t ks_hoisted_scratch_words(const Context& c, uint32_t level, uint32_t E);
cudaError_t ks_modup_hoisted(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in, uint64_t* ext,
                             uint64_t* scratch, cudaStream_t s);
// the same extension from c1's coefficient form coef [B][l1][N] (d_in[b]: the NTT-form
// ciphertexts, for the own-digit limbs); no scratch
cudaError_t ks_modup_hoisted_coef(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in,
                                  const uint64_t* coef, uint64_t* ext, cudaStream_t s);
cudaError_t ks_rotate_hoisted(const Context& c, uint32_t level, uint32_t E, const uint64_t* const* ext_of,
                              const uint64_t* const* src, const uint64_t* const* key_of, const uint64_t* gal_of,
                              uint64_t* const* d_out, uint64_t* scratch, cudaStream_t s);
// Sums of hoisted rotations with one ModDown each (double hoisting), in two
// calls on the same scratch (ks_hoisted_scratch_words(c, level, T)):
// ks_ipsum_hoisted sums, for each of T targets, the key-switch products of its
// elements e in [off[t], off[t+1]) (rotation of src_of[e] by gal_of[e] with key
// key_of[e] from the extension ext_of[e]; off on the device, absolute element
// indices) with P * sigma(c0); ks_moddown_add moves the sums down and adds them
// to tgt[t] in place (or writes tgt[t] + the result to d_out[t]).  Targets may be sources.
// (ntt_out: the sums left in NTT form on every limb, written to scratch as [T][2][nlx][N])
// The shape of one such launch as the schedule knows it on the host: the distinct
// extensions, keys and source ciphertexts of its elements (for the algorithmic byte
// count: each is read once, its other uses are re-reads of the same words) and the
// most elements of one target (the depth of the kernel's copy pipeline); zero =
// unknown (every element its own operands; a deep pipeline).
struct KsSumInfo {
    uint32_t ext = 0, keys = 0, srcs = 0, max_elems = 0, masks = 0;
};
// Group-masked sums (gmask != nullptr): a target's elements come group by group, and
// each group's key-switch sum is multiplied by its own plaintext before the target sums
// the groups.  Flags in the high bits of gal_of[e] (the low 32 bits are the Galois element):
constexpr uint64_t kGalGroupEnd = 1ull << 63;  // last element of its group
constexpr uint64_t kGalIdentity = 1ull << 62;  // the unrotated source: P * (c0, c1) on the q-limbs
constexpr int kGalMaskShift = 40;              // the group's plaintext: gmask + index * nlx * N
constexpr uint64_t kGalMaskBits = 0xffffull;
cudaError_t ks_ipsum_hoisted(const Context& c, uint32_t level, uint32_t T, const uint64_t* off, uint32_t E,
                             const uint64_t* const* ext_of, const uint64_t* const* src_of,
                             const uint64_t* const* key_of, const uint64_t* gal_of, uint64_t* scratch,
                             cudaStream_t s, bool ntt_out = false, KsSumInfo u = {}, uint32_t tpad = 0,
                             const uint64_t* gmask = nullptr, bool inv_all = false);
// ModDown of T level-1 sums in scratch (F4s with inv_all: every limb after its inverse
// row pass) taken in the coefficient domain, with the rescale to level 0 after it:
// out[t] [2][1][N] coefficient form = Res((x - Conv_P(x)) * P^-1), the residues of F5 + F6,
// the inverse NTT and rescale_coef (needs rescale_coef_supported)
cudaError_t ks_moddown_rescale_coef(const Context& c, uint32_t T, uint64_t* scratch, uint64_t* const* d_out,
                                    cudaStream_t s);
// ModDown and Rescale fused at the top level: e [T][2][L+1+alpha][N] (NTT form, every
// limb; the special limbs are transformed in place) divided by q_(L-drop+1)..q_L * P
// into out[t] (level L - drop, drop 1 or 2); scratch ks_mdr_scratch_words(c, T);
// needs ks_mdr_supported(c, drop)
bool ks_mdr_supported(const Context& c, uint32_t drop = 1);
size_t ks_mdr_scratch_words(const Context& c, uint32_t T);
cudaError_t ks_moddown_rescale(const Context& c, uint32_t T, uint64_t* e, uint64_t* const* d_out, uint64_t* scratch,
                               cudaStream_t s, uint32_t drop = 1);
// The deferred division (drop 2) of T sums e [T][2][L+1+alpha][N] (NTT form, every limb
// transformed in place) into out[t] at level L - 2, with the quotient's hoisted ModUp at
// that level written to ext + t * ks_ext_words(c, L - 2) -- the residues of
// ks_moddown_rescale(drop 2) followed by ks_modup_hoisted, in three launches; scratch
// ks_mdr_scratch_words(c, T); needs ks_mdru_supported(c)
bool ks_mdru_supported(const Context& c);
// a0 and Algorithm 1's extension together: Q top-level queries qin [Q][2][L+1][N] from
// coefficient to NTT form in place, and the extension of their c1 into ext (the layout
// and residues of ks_modup_hoisted_coef), in two launches
cudaError_t ks_a0_modup(const Context& c, uint32_t Q, uint64_t* qin, uint64_t* ext, cudaStream_t s);
cudaError_t ks_moddown_rescale_modup(const Context& c, uint32_t T, uint64_t* e, uint64_t* const* d_out,
                                     uint64_t* ext, uint64_t* scratch, cudaStream_t s);
cudaError_t ks_moddown_add(const Context& c, uint32_t level, uint32_t T, uint64_t* const* d_tgt, uint64_t* scratch,
                           cudaStream_t s, uint64_t* const* d_out = nullptr, const uint64_t* mask = nullptr);
// rescale in three fused kernels (rings 2^12 and 2^16)
cudaError_t rescale_fused(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in,
                          uint64_t* const* d_out, uint64_t* scratch, cudaStream_t s);
// inverse column pass alone (the second half of an inverse NTT)
cudaError_t ntt_col_inverse(const Context& c, const LimbBatch& b, cudaStream_t s);
// fills c.h_ksc / c.d_ksc
cudaError_t build_ks_constants(Context& c);
// out[b] = Res(in[b]); in at level, out at level-1 (no aliasing)
cudaError_t rescale(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in,
                    uint64_t* const* d_out, uint64_t* scratch, cudaStream_t s);
size_t rescale_scratch_words(const Context& c, uint32_t level, uint32_t B);
// out[b] = in[b] * pt[b] (pt Montgomery, [level+1][N]); out may alias in
cudaError_t mul_plain(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in,
                      const uint64_t* const* d_pt, uint64_t* const* d_out, cudaStream_t s);
// acc[q][g] = sum_i T[q][i] * P[g][i]  (T: [Q][n_in][2][level+1][N], P: [G][n_in][level+1][N])
cudaError_t mac(const Context& c, uint32_t level, uint32_t Q, uint32_t G, uint32_t n_in,
                const uint64_t* T, const uint64_t* P, uint64_t* acc, cudaStream_t s);
// hoisted Algorithm 1: t0[q][i] = sum_j R[q*n_in + j] * masks[(i - j) mod n_in] (t0 [Q][n_in] cts);
// with hat and tw from circ_prepare (2 <= n_in <= kMaxCircParts) as a cyclic
// convolution over the parts by length-n_in transforms, else the direct sum
constexpr uint32_t kMaxCircParts = 32;
cudaError_t mac_circ(const Context& c, uint32_t level, uint32_t Q, uint32_t n_in, const uint64_t* const* R,
                     const uint64_t* masks, const uint64_t* hat, const ulonglong2* tw, uint64_t* t0,
                     cudaStream_t s);
// the masks' side of that convolution on the first l1 primes of the basis: tw
// [l1][n_in] twiddles (host-built, copied), hat [n_in][l1][N] = transformed masks /
// n_in (Montgomery form); synchronises s
cudaError_t circ_prepare(const Context& c, uint32_t n_in, uint32_t l1, const uint64_t* masks, uint64_t* hat,
                         ulonglong2* tw, cudaStream_t s);
// masks [n_in][L+1][N] (NTT + Montgomery) extended to Q_L u P: ext [n_in][L+1+alpha][N],
// the special limbs from the centred integer coefficients of the q_0 limb; synchronises s
cudaError_t masks_extend(const Context& c, uint32_t n_in, const uint64_t* masks, uint64_t* ext, cudaStream_t s);
// plaintexts in [count][l_in][N] (NTT + Montgomery, primes q_0..q_(l_in-1)) extended to
// Q_L u P: out [count][L+1+alpha][N], limbs l_in.. from the centred integer
// coefficients of the q_0 limb (exact while they lie within q_0 / 2); synchronises s
cudaError_t extend_to_ext_basis(const Context& c, size_t count, const uint64_t* in, uint32_t l_in, uint64_t* out,
                                cudaStream_t s);
// ... to the key-switching basis of their own level, Q_(l_in-1) u P: out [count][l_in+alpha][N]
cudaError_t extend_to_level_ext(const Context& c, size_t count, const uint64_t* in, uint32_t l_in, uint64_t* out,
                                cudaStream_t s);
// the last rescale in the coefficient domain: in[b] level-1 ciphertexts (coefficient
// form) -> out[b] at level 0, the residues of rescale + inverse NTT (needs q_1 < q_0)
bool rescale_coef_supported(const Context& c);
cudaError_t rescale_coef(const Context& c, uint32_t B, uint64_t* const* in, uint64_t* const* out, cudaStream_t s);
// E0[q] = P * in[q] on Q_L u P (special limbs 0): in[q] [2][L+1][N], E0 + q * stride holds
// [2][L+1+alpha][N] (stride in words; 0 = packed), NTT form
cudaError_t lift_p(const Context& c, uint32_t Q, uint64_t* const* in, uint64_t* E0, cudaStream_t s,
                   size_t stride = 0);
// The gallery of the deferred division folded with the masks of the fused Algorithm 1:
// fold[g][j] = sum_i mask_((i - j) mod n_in) * pts[g][i] on every limb of Q_L u P (masks
// and plaintexts NTT + Montgomery; the result Montgomery too), so HE-C^3 on the rotated
// copies E_j of the query gives the sum over the parts of the circulant's e_i times the
// plaintexts: sum_j E_j fold_j = sum_i (sum_j E_j mask_(i-j)) pts_i, mod q.
// pts, fold [groups][n_in][L+1+alpha][N]; masks_ext [n_in][L+1+alpha][N]
cudaError_t fold_gallery(const Context& c, size_t groups, uint32_t n_in, const uint64_t* masks_ext,
                         const uint64_t* pts, uint64_t* fold, cudaStream_t s);
// dst[t] += sum of src[off[t] .. off[t+1]) (ciphertexts at `level`; off and the lists on the device)
cudaError_t accumulate(const Context& c, uint32_t level, uint32_t n_targets, uint64_t* const* dst,
                       const uint64_t* const* src, const uint64_t* off, uint32_t n_src, cudaStream_t s);
// encrypted gallery: A[q][g] = (d0, d2), B[q][g] = (0, d1) of sum_i T[q][i] (x) C[g][i]
// (C: [G][n_in][2][level+1][N] Montgomery form)
cudaError_t mac_ct(const Context& c, uint32_t level, uint32_t Q, uint32_t G, uint32_t n_in, const uint64_t* T,
                   const uint64_t* C, uint64_t* A, uint64_t* B, cudaStream_t s);
// plain products a*b on each limb (NTT form, b Montgomery)
cudaError_t pointwise_mul(const Context& c, const LimbBatch& a, const LimbBatch& b,
                          const LimbBatch& out, cudaStream_t s);
// out = a + b, a - b on each limb
cudaError_t pointwise_addsub(const Context& c, const LimbBatch& a, const LimbBatch& b,
                             const LimbBatch& out, bool sub, cudaStream_t s);
// NTT-domain automorphism: out[i] = in[perm_k(i)] on each limb
cudaError_t permute_ntt(const Context& c, const LimbBatch& in, const LimbBatch& out,
                        uint64_t galois, cudaStream_t s);
// out = in * c (per-limb constants c[k], plain form) on each limb
cudaError_t scalar_mul(const Context& c, const LimbBatch& in, const uint64_t* cst,
                       const LimbBatch& out, cudaStream_t s);

}  // namespace bm

// opaque handle types of the C-ABI
struct bm_context { bm::Context c; };
struct bm_secret_key { bm::CtxRef ref; bm::SecretKey k; };
struct bm_public_key { bm::CtxRef ref; bm::PublicKey k; };
struct bm_eval_keys { bm::CtxRef ref; bm::EvalKeys k; };
struct bm_gallery { bm::CtxRef ref; bm::Gallery g; };
struct bm_ciphertext { bm::CtxRef ref; bm::Ciphertext ct; };
struct bm_result { bm::CtxRef ref; bm::Result r; };
