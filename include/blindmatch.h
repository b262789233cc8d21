/*
 * blindmatch.h -- C ABI of the GB300 Blind-Match library: encrypted 1:N
 * cosine-similarity matching of biometric templates under RNS-CKKS
 * (Choi, Kim, Song, Woo: "Blind-Match", CIKM 2024, arXiv 2408.06167).
 *
 * The calls follow the paper's statement of the protocol:
 *   bm_keygen          Sec. 3.1 Key Generation and Management
 *   bm_encode_gallery  Sec. 3.2 Enrollment (layout: identity u of a group at slots [u*s, u*s+s))
 *   bm_encrypt_query   Sec. 3.3 Recognition (client encrypts the query feature vector)
 *   bm_match           Sec. 3.3: Algorithm 1 (Input Ciphertext Expansion), Algorithm 2 (HE-C^3)
 *                      and the compression step, on the GPU
 *   bm_decrypt_scores  Sec. 3.3 Decryption (client decrypts, takes the argmax = Rank-1)
 *
 * Conventions shared by every call:
 *  - A ciphertext at level l has the RNS limbs q_0..q_l; its wire layout is
 *    [2][l+1][N] uint64 residues in coefficient order (c0 then c1).
 *  - Slot j of a plaintext is its value at the root zeta^(5^j), zeta = exp(i*pi/N);
 *    a rotation by r > 0 is the left rotation of Sec. 2 (slot j <- slot j + r).
 *  - Handles are opaque and owned by the caller once returned; free each with its
 *    _destroy call.  Inputs passed by pointer are borrowed for the duration of the
 *    call and copied.  Calls on one context are not thread-safe.
 *  - Every call returns a bm_status; on failure bm_last_error() (thread-local)
 *    describes the cause and no output handle is written.
 *  - Device memory is allocated with the CUDA runtime on the context's device.
 */
#ifndef BLINDMATCH_H
#define BLINDMATCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bm_status {
    BM_OK = 0,
    BM_E_ARG = 1,          /* null pointer, size mismatch, index out of range */
    BM_E_PARAM = 2,        /* parameter set not supported (ring size, prime sizes, digits) */
    BM_E_LEVEL = 3,        /* not enough levels for the requested schedule / mode */
    BM_E_KEY_MISSING = 4,  /* no rotation key for a needed Galois element */
    BM_E_DIM = 5,          /* dim or part size not a power of two, part does not divide dim,
                              or dim larger than the slot count (Sec. 3.2) */
    BM_E_OOM = 6,          /* device or host allocation failed */
    BM_E_HBM_BUDGET = 7,   /* request exceeds the configured device-memory budget */
    BM_E_CUDA = 8,         /* a CUDA runtime call failed */
    BM_E_TIMEOUT = 9,      /* a bounded wait expired */
    BM_E_CANCELLED = 10,   /* the request was cancelled */
    BM_E_FORMAT = 11       /* malformed import data (level, sizes) */
} bm_status;

#define BM_MAX_Q 6   /* primes in the ciphertext modulus chain q_0..q_L */
#define BM_MAX_P 3   /* special primes of key switching */

/* RNS-CKKS parameters.  The primes are derived deterministically: q_0 is the
 * largest prime below 2^q_bits[0] with q = 1 (mod 2N); each later prime (the
 * rescale primes, then the special primes) is the largest such prime below
 * 2^bits not used before it.  The paper fixes none of this (Sec. 5.1 names only
 * N = 8192, log PQ ~ 158, l = 3, under Lattigo). */
typedef struct bm_params {
    uint32_t log_n;               /* ring degree N = 2^log_n: 12 or 16 (the register-resident
                                     NTT passes: 2^6 x 2^6 or 2^8 x 2^8 points) */
    uint32_t n_q;                 /* primes in Q (L = n_q - 1), 2 <= n_q <= BM_MAX_Q */
    uint32_t q_bits[BM_MAX_Q];    /* q_bits[0]: base prime; then rescale primes; each 30..60 */
    uint32_t n_p;                 /* special primes, 1 <= n_p <= 2 */
    uint32_t p_bits[BM_MAX_P];    /* 30..60 */
    uint32_t dnum;                /* key-switching digits (ceil(n_q/dnum) <= 2), 1..4 */
    uint32_t log_scale;           /* encoding scale Delta = 2^log_scale */
    uint32_t secret_hw;           /* 0: ZO(1/2) ternary secret; else ternary of this Hamming weight */
    double sigma;                 /* discrete Gaussian width of the errors (3.2) */
} bm_params;

enum {
    BM_PRESET_TOY = 0,     /* N = 2^12, q 50 + 40 bits, p 50 bits, dnum 2, ZO secret: not secure */
    BM_PRESET_RING16 = 1,  /* N = 2^16, q 60 + 3x40 bits, p 2x60 bits, dnum 2, HW-192 secret */
    BM_PRESET_SMALL4 = 2   /* the RING16 chain on N = 2^12 (test size) */
};

/* Query layouts of bm_encrypt_query (Sec. 3.3). */
enum {
    BM_QUERY_TILED = 0,    /* one ciphertext, q tiled with period dim; the server runs Algorithm 1 */
    BM_QUERY_EXPANDED = 1, /* dim/part ciphertexts, part i tiled with period part (client-side
                              expansion; required when the chain has fewer than 3 rescale primes) */
    BM_QUERY_TEMPLATE = 2  /* one ciphertext, the vector in the first dim slots and zeros after:
                              an enrollment template (Sec. 3.2) for bm_enroll_encrypted */
};

typedef struct bm_context bm_context;
typedef struct bm_secret_key bm_secret_key;
typedef struct bm_public_key bm_public_key;
typedef struct bm_eval_keys bm_eval_keys;
typedef struct bm_gallery bm_gallery;
typedef struct bm_ciphertext bm_ciphertext;
typedef struct bm_result bm_result;

/* Thread-local description of the last failure on this thread ("" if none). */
const char* bm_last_error(void);
/* Fills *out with a preset (BM_PRESET_*).  BM_E_ARG for an unknown preset. */
bm_status bm_params_preset(int preset, bm_params* out);

/* Creates a context on CUDA device `device`: derives primes and roots, uploads the
 * NTT tables.  BM_E_PARAM if the parameters are outside the ranges above or a prime
 * cannot be found; BM_E_CUDA if the device cannot be used. */
bm_status bm_context_create(const bm_params* params, int device, bm_context** out);
void bm_context_destroy(bm_context* ctx);
/* Writes the n_q + n_p primes (q_0..q_L, then p_0..) to primes_out. */
bm_status bm_context_primes(const bm_context* ctx, uint64_t* primes_out, size_t capacity);

/* Sec. 3.1: samples the secret key, the public key and the rotation keys that the
 * match schedule for (dim, part_size) needs -- left rotations by part*2^j
 * (Algorithm 1, tiled schedule only), left rotations by 2^t (Algorithm 2) and right
 * rotations by 2^t (compression, when the chain has a level for it).  All randomness
 * comes from Philox4x64-10 keyed by `seed`.  Keys stay resident on the device.
 * BM_E_DIM for an invalid (dim, part_size). */
bm_status bm_keygen(bm_context* ctx, uint64_t seed, uint32_t dim, uint32_t part_size,
                    bm_secret_key** sk, bm_public_key** pk, bm_eval_keys** evk);
/* Key sets beyond the plaintext-gallery schedule. */
enum {
    BM_KEYS_ENCRYPTED_GALLERY = 1,  /* also the relinearisation key (the key-switching key from s^2
                                       to s, for Mul of two ciphertexts, Sec. 3.1) and the right
                                       rotations by every power of two from part_size below N/2
                                       that enrollment uses (Sec. 3.2) */
    BM_KEYS_HOISTED = 2             /* also the rotations of the hoisted forms (BM_SCHED_*): left by
                                       j*part_size, 0 < j < dim/part_size (Algorithm 1), left by the
                                       baby and giant steps of the rotate-and-sum, right by 1 .. part_size-1
                                       (linear compression) */
};
/* bm_keygen with extra key sets (BM_KEYS_* flags); flags = 0 is bm_keygen.  The
 * relinearisation key is sampled like a rotation key with s^2 in place of
 * sigma_k(s) (Philox tags 9 and 10, object = digit). */
bm_status bm_keygen_ex(bm_context* ctx, uint64_t seed, uint32_t dim, uint32_t part_size, uint32_t flags,
                       bm_secret_key** sk, bm_public_key** pk, bm_eval_keys** evk);
void bm_secret_key_destroy(bm_secret_key* sk);
void bm_public_key_destroy(bm_public_key* pk);
void bm_eval_keys_destroy(bm_eval_keys* evk);
/* Number of rotation keys and their left-rotation amounts (negative = right). */
bm_status bm_eval_keys_rotations(const bm_eval_keys* evk, int32_t* rotations, size_t capacity,
                                 uint32_t* count);
/* Coefficient-form copies for checking: secret key (N signed values), public key
 * [2][L+1][N], rotation key of a left rotation `rotation` [dnum][2][n_q+n_p][N]
 * (component 0 = b, 1 = a; limbs over q_0..q_L then p_0..).  BM_E_KEY_MISSING if
 * the rotation has no key; BM_E_ARG if `capacity` (words) is too small. */
bm_status bm_secret_key_export(const bm_secret_key* sk, int64_t* out, size_t capacity);
bm_status bm_public_key_export(const bm_public_key* pk, uint64_t* out, size_t capacity);
bm_status bm_eval_keys_export(const bm_eval_keys* evk, int32_t rotation, uint64_t* out,
                              size_t capacity);

/* Slot packing of a gallery.  Sec. 3.2 gives each identity of a group one window
 * of `part` slots; CKKS slots are complex and the query is real, so a second
 * identity can ride in the imaginary parts of the same window: every product,
 * sum, rotation and mask of the match acts on both parts alike, and the score of
 * identity u sits in the real part and that of identity G+u in the imaginary
 * part of the same output slot.  Groups (and all per-group work) halve. */
enum {
    BM_PACK_REAL = 0,     /* G = (N/2)/part identities per group, real parts only */
    BM_PACK_COMPLEX = 1   /* 2G per group: identity u (u < G) in the real parts of window u,
                             identity G+u in its imaginary parts */
};

/* Sec. 3.2 (enrollment, with a plaintext gallery): feats is n_ids x dim row-major
 * float64, L2-normalised.  Identities are grouped G = (N/2)/part_size per group;
 * identity u of group g fills slots [u*part, u*part+part) of the group's plaintext
 * for part i (its i-th sub-vector), zero past the last identity.  Also encodes the
 * Algorithm-1 masks (mask_i[k] = 1 iff floor((k mod dim)/part) = i) and the
 * compression mask (M[k] = 1 iff k = 0 mod part).  Everything stays resident on
 * the device.  BM_E_DIM for an invalid (dim, part_size); BM_E_LEVEL if the chain
 * is too short for any schedule (n_q < 2). */
bm_status bm_encode_gallery(bm_context* ctx, const double* feats, uint64_t n_ids, uint32_t dim,
                            uint32_t part_size, bm_gallery** out);
/* The same with a slot packing (BM_PACK_*); bm_encode_gallery is BM_PACK_REAL.
 * BM_E_ARG for an unknown packing. */
bm_status bm_encode_gallery_packed(bm_context* ctx, const double* feats, uint64_t n_ids, uint32_t dim,
                                   uint32_t part_size, uint32_t packing, bm_gallery** out);
/* Same gallery from coefficient-form plaintexts produced elsewhere:
 * pts [groups][dim/part][level+1][N], masks [dim/part][n_q][N] (tiled schedule; NULL
 * otherwise), cmask [level][N] (when compressing; NULL otherwise), where `level`
 * and the schedule are those bm_gallery_layout reports. */
bm_status bm_gallery_import(bm_context* ctx, const uint64_t* pts, const uint64_t* masks,
                            const uint64_t* cmask, uint64_t n_ids, uint32_t dim,
                            uint32_t part_size, bm_gallery** out);
bm_status bm_gallery_import_packed(bm_context* ctx, const uint64_t* pts, const uint64_t* masks,
                                   const uint64_t* cmask, uint64_t n_ids, uint32_t dim,
                                   uint32_t part_size, uint32_t packing, bm_gallery** out);
/* Layout of a gallery for (n_ids, dim, part_size) under this context: number of
 * groups, level of the gallery plaintexts, tiled (1) or expanded (0) queries,
 * compressed (1) or per-group (0) outputs, output ciphertexts per query. */
bm_status bm_gallery_layout(const bm_context* ctx, uint64_t n_ids, uint32_t dim,
                            uint32_t part_size, uint32_t* groups, uint32_t* level,
                            uint32_t* tiled, uint32_t* compressed, uint32_t* n_out);
bm_status bm_gallery_layout_packed(const bm_context* ctx, uint64_t n_ids, uint32_t dim,
                                   uint32_t part_size, uint32_t packing, uint32_t* groups,
                                   uint32_t* level, uint32_t* tiled, uint32_t* compressed,
                                   uint32_t* n_out);
/* Coefficient-form copies of the resident plaintexts (layouts as in the import;
 * pass NULL to skip a part).  For an encrypted gallery `pts` receives its
 * ciphertexts [groups][dim/part][2][level+1][N]. */
bm_status bm_gallery_export(const bm_gallery* g, uint64_t* pts, uint64_t* masks, uint64_t* cmask);

/* Encrypted gallery (Sec. 3.2 as the paper runs it: the server never sees a
 * template in the clear).  templates[k] is identity k's BM_QUERY_TEMPLATE
 * ciphertext at the top level.  Identity k goes to group g = k / G, window
 * w = k mod G (G = (N/2)/part_size); for each part i the server multiplies the
 * template by mask_i (ones at slots [i*part, (i+1)*part)), rescales, rotates the
 * product right by (w - i)*part slots -- as one rotation per set bit of that
 * amount mod N/2, lowest bit first -- and adds it into the group ciphertext
 * C[g][i].  The gallery ciphertexts sit at level L-1 (the Algorithm-2 level) and
 * HE-C^3 multiplies them with the expanded query (ciphertext x ciphertext), sums
 * the tensor products over the parts and relinearises once per group.  Needs
 * evk from bm_keygen_ex(..., BM_KEYS_ENCRYPTED_GALLERY) and a chain with at
 * least three rescale primes (BM_E_LEVEL otherwise); real packing only. */
bm_status bm_enroll_encrypted(bm_context* ctx, const bm_eval_keys* evk, bm_ciphertext* const* templates,
                              uint64_t n_ids, uint32_t dim, uint32_t part_size, bm_gallery** out);
/* The same gallery from ciphertexts made elsewhere: cts [groups][dim/part][2][L][N]
 * (level L-1, scale 2^log_scale), masks and cmask as in bm_gallery_import. */
bm_status bm_gallery_import_encrypted(bm_context* ctx, const uint64_t* cts, const uint64_t* masks,
                                      const uint64_t* cmask, uint64_t n_ids, uint32_t dim,
                                      uint32_t part_size, bm_gallery** out);
/* 1 if the gallery holds ciphertexts, 0 if plaintexts; its packing. */
bm_status bm_gallery_info(const bm_gallery* g, uint32_t* encrypted, uint32_t* packing);

/* How the server runs Algorithm 1 (Input Ciphertext Expansion) for this gallery:
 *  BM_EXPAND_DOUBLING  the printed form: per part i, mask, rescale, then log2(N_in)
 *                      rotate-and-add steps by part*2^(j-1) (N_in log2 N_in rotations)
 *  BM_EXPAND_HOISTED   the same sum reordered: T_i = Res(sum_j Rot(ct, j*part) *
 *                      mask_((i-j) mod N_in)) -- since rotating a masked ciphertext by j
 *                      parts equals rotating the ciphertext and using the mask of part
 *                      i-j -- so N_in - 1 rotations of the one query ciphertext, which
 *                      share its basis extension (hoisting), and N_in^2 plaintext products.
 * Both decrypt to the same parts; the ciphertext bits differ.  Needs the rotation
 * keys by j*part for j < N_in (bm_keygen_ex with BM_KEYS_HOISTED).  Plans of the
 * gallery built before the call are dropped; call it before registering the
 * gallery with a server.  BM_E_ARG for an unknown mode or a gallery without
 * Algorithm 1 (client-expanded queries). */
enum {
    BM_EXPAND_DOUBLING = 0,
    BM_EXPAND_HOISTED = 1,
    BM_EXPAND_FUSED = 2,     /* hoisted, with the key switches and the rescale fused (below) */
    BM_EXPAND_DEFERRED = 3   /* fused, with the division moved past HE-C^3's products (below) */
};
bm_status bm_gallery_set_expansion(bm_gallery* g, uint32_t mode);

/* The schedule's hoisted forms, as a set of flags (the same messages as the
 * printed forms; the ciphertext bits differ, and each is bit-exact against the
 * oracle's evaluation in the same order):
 *  BM_SCHED_HOISTED_EXPANSION    Algorithm 1 as above (= BM_EXPAND_HOISTED)
 *  BM_SCHED_HOISTED_ROTSUM       Algorithm 2's rotate-and-sum over a part of s
 *                                slots, sum_{r<s} Rot(acc, r), as two rounds of
 *                                hoisted rotations: acc += Rot(acc, r) for 0 < r < b,
 *                                then acc += Rot(acc, b*k) for 0 < k < s/b, with
 *                                b = 2^ceil(log2(s)/2) (log2(s) sequential
 *                                rotations otherwise)
 *  BM_SCHED_HOISTED_COMPRESSION  the compression in its linear form, every group
 *                                r > 0 of a pack rotated right by r in one round of
 *                                hoisted rotations (a radix-2 tree otherwise)
 *  BM_SCHED_FUSED_EXPANSION      with the hoisted expansion: the N_in - 1 rotations
 *                                kept in the extended basis Q_L u P (before ModDown),
 *                                the circulant mask products there, and each part
 *                                divided once by q_L * P -- one fused ModDown and
 *                                Rescale per part instead of a ModDown per rotation
 *                                and a rescale per part (2 <= N_in <= 32)
 *  BM_SCHED_DEFERRED_DIVISION    with the fused expansion: the parts kept undivided
 *                                on Q_L u P, HE-C^3's products summed there against
 *                                the gallery plaintexts extended to Q_L u P, and each
 *                                (query, group) sum divided once by q_(L-1) q_L P --
 *                                one division per group instead of one per part and
 *                                the rescale after the products; the gallery keeps a
 *                                second copy of its plaintexts on Q_L u P (twice the
 *                                limbs).  Fewer divisions when a gallery has fewer
 *                                groups than parts.
 *  BM_SCHED_DOUBLE_HOISTED       with either of the two above: each round's
 *                                rotations into one output summed in the extended
 *                                basis Q_l u P and moved down once (one ModDown per
 *                                output instead of one per rotation; double
 *                                hoisting, Bossuat et al., Eurocrypt 2021); the
 *                                rotate-and-sum over s <= 16 slots then takes a
 *                                single round of the s - 1 rotations
 *  BM_SCHED_FUSED_COMPRESSION    with the three above (hoisted rotate-and-sum and
 *                                compression, double hoisting): the rotate-and-sum's
 *                                last round and the compression as one round per pack.
 *                                The compression places group o of a pack (o its
 *                                offset) at Rot(M * acc_o, -o) = Rot(M, -o) *
 *                                Rot(acc_o, -o), and Rot(acc_o, -o) is the last
 *                                round's sum with every rotation shifted by -o, so
 *                                each pack is the sum over its groups of the mask
 *                                rotated by -o times the group's shifted rotations,
 *                                taken in Q_l u P and moved down once: one ModDown per
 *                                pack instead of one per group plus the compression
 *                                round.  The mask multiplies the key-switch sums
 *                                before ModDown's rounding, not after it.  A gallery
 *                                without compression ignores the flag.
 * Needs the keys of bm_keygen_ex(..., BM_KEYS_HOISTED).  Plans of the gallery
 * built before the call are dropped; call it before registering the gallery
 * with a server.  BM_E_ARG for unknown flags, or the expansion flag on a gallery
 * without Algorithm 1. */
enum {
    BM_SCHED_HOISTED_EXPANSION = 1,
    BM_SCHED_HOISTED_ROTSUM = 2,
    BM_SCHED_HOISTED_COMPRESSION = 4,
    BM_SCHED_DOUBLE_HOISTED = 8,
    BM_SCHED_FUSED_EXPANSION = 16,
    BM_SCHED_DEFERRED_DIVISION = 32,
    BM_SCHED_FUSED_COMPRESSION = 64
};
bm_status bm_gallery_set_schedule(bm_gallery* g, uint32_t flags);
void bm_gallery_destroy(bm_gallery* g);

/* Sec. 3.3: encrypts the L2-normalised query q[dim] under pk at the top level
 * with scale 2^log_scale: ct = (v*pk0 + e0 + m, v*pk1 + e1), v ~ ZO(1/2), e0, e1
 * Gaussian, drawn from Philox4x64-10 keyed by `seed`, object query_id*256 + part.
 * mode BM_QUERY_TILED gives one ciphertext, BM_QUERY_EXPANDED dim/part_size.
 * The ciphertext is host-resident (coefficient form, the client-to-server message). */
bm_status bm_encrypt_query(bm_context* ctx, const bm_public_key* pk, const double* q, uint32_t dim,
                           uint32_t part_size, uint32_t mode, uint64_t seed, uint64_t query_id,
                           bm_ciphertext** out);
/* Wraps n_cts coefficient-form ciphertexts [n_cts][2][level+1][N].  BM_E_FORMAT for
 * a level above L. */
/* Batched encryption: vectors is n_vec x dim row-major; out[k] (n_vec handles)
 * is vectors[k] encrypted as bm_encrypt_query(..., mode, seed, first_id + k)
 * would encrypt it -- bit for bit: the noise is drawn from the same counter-based
 * Philox words, on the GPU, and the encoding runs on the host cores in parallel.
 * flags BM_ENC_KEEP_DEVICE also keeps a device copy of each ciphertext (as after
 * bm_ciphertext_upload). */
#define BM_ENC_KEEP_DEVICE 1u
bm_status bm_encrypt_batch(bm_context* ctx, const bm_public_key* pk, const double* vectors, uint64_t n_vec,
                           uint32_t dim, uint32_t part_size, uint32_t mode, uint64_t seed, uint64_t first_id,
                           uint32_t flags, bm_ciphertext** out);
bm_status bm_ciphertext_import(bm_context* ctx, const uint64_t* data, uint32_t n_cts,
                               uint32_t level, bm_ciphertext** out);
bm_status bm_ciphertext_info(const bm_ciphertext* ct, uint32_t* n_cts, uint32_t* level);
bm_status bm_ciphertext_export(const bm_ciphertext* ct, uint64_t* out, size_t capacity);
/* Stages the ciphertext on the device (H2D, coefficient form) on `stream` (a
 * cudaStream_t, NULL for the legacy default stream) and waits for the copy; later
 * bm_match calls copy it device-to-device instead of from the host. */
bm_status bm_ciphertext_upload(bm_ciphertext* ct, void* stream);
void bm_ciphertext_destroy(bm_ciphertext* ct);

/* Sec. 3.3, the server side, on the GPU.  The first call for a (gallery, key set,
 * n_queries) triple builds a plan -- persistent device buffers and the whole
 * schedule captured as a CUDA graph -- kept until the gallery, the key set or the
 * context is destroyed; later calls copy the queries in, replay the graph and
 * copy the score ciphertexts into a new result.  For each query, Algorithm 1 (tiled
 * queries), then for every group HE-C^3 (Algorithm 2: ct x pt products summed
 * over the parts, one rescale, log2(part) rotate-and-add steps), then the
 * compression step (mask, pack `part` groups per ciphertext by a tree of right
 * rotations, rescale).  Scores end at slot u*part + r of pack floor(g/part) for
 * identity u of group g = pack*part + r (packed), or at slot u*part of the group's
 * output (per-group).  Runs on `stream` and returns after the result is complete;
 * the score ciphertexts stay on the device in *out.  BM_E_LEVEL if a query's
 * mode/level does not match the gallery; BM_E_KEY_MISSING if evk lacks a rotation. */
bm_status bm_match(bm_context* ctx, const bm_eval_keys* evk, const bm_gallery* gallery,
                   bm_ciphertext* const* queries, uint32_t n_queries, void* stream,
                   bm_result** out);
/* bm_match without the wait: the match and the copy of its score ciphertexts are
 * enqueued on `stream` and the call returns; the result is complete when the stream
 * reaches the end of that work (the caller synchronises the stream, or records an
 * event after the call).  bm_result_export and bm_decrypt_scores wait for it
 * themselves, and bm_result_destroy may be called at any time (the free is ordered
 * after the copy).  Host ciphertexts are copied from their page-locked host memory
 * while the call's work runs: keep them alive until the stream has passed it.  For
 * plans of up to 256 MiB of queries (64 top-level ring-2^16 queries) that copy runs on
 * the plan's own stream into one of two staging buffers, waiting only for the call
 * before the previous one to have moved its queries out: a call issued while the
 * previous call's match still runs copies its queries during that match, so a client
 * that enqueues the next match before reading back the last result keeps the copies
 * off the critical path.  Calls that share a plan (same gallery, key set and
 * n_queries) must be issued on one stream, or serialised by the caller: the plan's
 * buffers are reused by every call.  The same plans, errors and results as bm_match. */
bm_status bm_match_async(bm_context* ctx, const bm_eval_keys* evk, const bm_gallery* gallery,
                         bm_ciphertext* const* queries, uint32_t n_queries, void* stream, bm_result** out);
bm_status bm_result_info(const bm_result* r, uint32_t* n_queries, uint32_t* n_out,
                         uint32_t* packed);
/* Score ciphertexts of one query: [n_out][2][N] coefficient form at level 0.  Waits
 * for the result's match, then copies on the context's own non-blocking stream: work
 * enqueued after that match (the next bm_match_async) is not waited for. */
bm_status bm_result_export(const bm_result* r, uint32_t query_index, uint64_t* out,
                           size_t capacity);
/* Frees the result; call it before destroying the result's context. */
void bm_result_destroy(bm_result* r);
/* Sec. 3.3 Decryption: decrypts the score ciphertexts of one query with sk and maps
 * slots back to identities: scores[u] ~ <q, g_u> (the cosine similarity of unit
 * vectors; with BM_PACK_COMPLEX galleries the real or imaginary part of the
 * identity's slot).  rank1 = argmax (lowest id on ties), rank1_score its score; the caller
 * applies its own threshold to reject unenrolled users. */
bm_status bm_decrypt_scores(bm_context* ctx, const bm_secret_key* sk, const bm_result* r,
                            uint32_t query_index, double* scores, uint64_t n_ids,
                            int64_t* rank1, double* rank1_score);

/* ---- serving: continuous batching over resident galleries ---- */

typedef struct bm_server bm_server;
typedef struct bm_server_stats_t {
    uint64_t submitted, completed, failed, cancelled;
    uint64_t batches;         /* batched matches executed */
    double mean_batch;        /* queries per executed batch */
    double p50_ms, p99_ms;    /* submit-to-completion latency of the completed requests */
    double matches_per_s;     /* identities scored per second, first submit to last completion */
    uint64_t workspace_bytes; /* device memory held by the executors' match plans */
} bm_server_stats_t;

/* A match server on ctx (Sec. 3.3 recognition, many clients at once).  Requests
 * wait in arrival order; `executors` threads (1..16), each with its own CUDA
 * stream and match plans, repeatedly take the oldest request together with the
 * other pending requests for the same gallery (at most max_batch) and run them as
 * one batched bm_match, so requests that arrive while others run join the next
 * batch and batches of different executors overlap on the GPU.  A batch runs the
 * plan of the largest power of two of queries it holds (so plans are reused and no
 * plan runs padding); the rest go back to the front of the queue.  Match workspaces
 * are admitted against hbm_budget_bytes of device memory: an executor evicts its
 * own idle plans first, then halves its batch; a single query that does not fit
 * fails with BM_E_HBM_BUDGET.  Galleries and key sets are borrowed and must
 * outlive the server. */
bm_status bm_server_create(bm_context* ctx, uint64_t hbm_budget_bytes, uint32_t max_batch, uint32_t executors,
                           bm_server** out);
/* Stops the executors after their current batch; pending requests are cancelled
 * and uncollected results freed. */
void bm_server_destroy(bm_server* srv);
/* Registers a resident gallery with the rotation keys generated for its
 * (dim, part) (BM_E_KEY_MISSING otherwise); *gid identifies it in submissions. */
bm_status bm_server_add_gallery(bm_server* srv, const bm_gallery* gallery, const bm_eval_keys* evk,
                                uint32_t* gid);
/* Queues one query (copied) against gallery gid; BM_E_LEVEL if its layout does
 * not match the gallery's schedule.  *ticket identifies the request. */
bm_status bm_server_submit(bm_server* srv, uint32_t gid, const bm_ciphertext* query, uint64_t* ticket);
/* Waits up to timeout_ms for the request; BM_E_TIMEOUT leaves it in flight (wait
 * again later).  On completion the ticket is consumed: *out receives the
 * request's result (one query; free it with bm_result_destroy), or the request's
 * own error is returned (BM_E_HBM_BUDGET, BM_E_CANCELLED, ...). */
bm_status bm_server_wait(bm_server* srv, uint64_t ticket, uint32_t timeout_ms, bm_result** out);
/* Cancels a request that has not started; BM_E_ARG if it is running or done. */
bm_status bm_server_cancel(bm_server* srv, uint64_t ticket);
bm_status bm_server_stats(bm_server* srv, bm_server_stats_t* out);
/* Zeroes the counters and latencies bm_server_stats reports (plans and pending
 * requests are kept): a measurement window after a warm-up. */
bm_status bm_server_reset_stats(bm_server* srv);

/* ---- single operations, for checking the kernels against a reference ---- */

/* Negacyclic products out = a * b in Z_q[X]/(X^N+1), limb k on prime k of the full
 * basis (k < n_q + n_p), host arrays [n_limbs][N], through the GPU NTT. */
bm_status bm_poly_mul(bm_context* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out,
                      uint32_t n_limbs);
/* Rot(ct, rotation) (Sec. 2) of every ciphertext in `in` at its level, through the
 * GPU key switch; result is a new host ciphertext. */
bm_status bm_ct_rotate(bm_context* ctx, const bm_eval_keys* evk, const bm_ciphertext* in,
                       int32_t rotation, bm_ciphertext** out);
/* Res (Sec. 2) of every ciphertext in `in`: level l -> l-1.  BM_E_LEVEL at level 0. */
bm_status bm_ct_rescale(bm_context* ctx, const bm_ciphertext* in, bm_ciphertext** out);
/* In-place NTT / inverse NTT of device limbs d_data[n_polys][n_limbs][N]; limb k
 * uses prime k of the full basis.  The forward transform's output order is the
 * library's own (bit-reversed evaluation order); only the inverse undoes it. */
bm_status bm_ntt_forward(bm_context* ctx, uint64_t* d_data, uint32_t n_polys, uint32_t n_limbs,
                         void* stream);
bm_status bm_ntt_inverse(bm_context* ctx, uint64_t* d_data, uint32_t n_polys, uint32_t n_limbs,
                         void* stream);

/* Rot(ct, rotation) like bm_ct_rotate, for callers that cannot let the library
 * allocate device memory (a host whose device memory belongs to its own pool
 * allocator, or a serving loop that forbids allocation after start-up).  The
 * paper has no counterpart to this call.
 *   d_in:  n_cts ciphertexts at `level`, coefficient form, device memory,
 *          layout [n_cts][2][level+1][N]; read only.
 *   d_out: device memory of the same size; receives the rotated ciphertexts in
 *          coefficient form.  Must not overlap d_in.
 * Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default stream)
 * and the call returns without waiting for it.  Temporaries live in one
 * file-scope device array of 32 MiB that every GPU loading the library holds
 * until the process exits; the call performs no cudaMalloc/cudaFree.  Requests
 * needing more (input copy + key-switch temporaries, e.g. more than one ring-2^16
 * ciphertext at level 3) or more than 64 ciphertexts fail with BM_E_ARG and a
 * message giving the limit.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, cached per device for the life of the
 * process: calls after a cudaDeviceReset of that device are not supported);
 * make that first call before any stream capture.  Every call writes its
 * pointer lists on the device with a kernel (no host staging buffer and no
 * host-to-device copy), restores the caller's current device before
 * returning, and does not wait on the stream.
 * All calls share the array: calls whose work overlaps on one GPU (issued on
 * different streams or from different threads) race and must be serialised by
 * the caller.  BM_E_KEY_MISSING if evk has no key for the rotation. */
bm_status bm_ct_rotate_noalloc(bm_context* ctx, const bm_eval_keys* evk, const uint64_t* d_in,
                               uint32_t n_cts, uint32_t level, int32_t rotation, uint64_t* d_out,
                               void* stream);

/* ---- launch accounting (measurement support; no counterpart in the paper) ---- */

/* Kernel classes of the match path. */
enum {
    BM_KERNEL_NTT = 0,        /* forward/inverse NTT passes (column and row pass each count) */
    BM_KERNEL_MODUP = 1,      /* automorphism gather + fast base conversion of one digit */
    BM_KERNEL_KS_IP = 2,      /* inner product with the rotation key */
    BM_KERNEL_MODDOWN = 3,    /* base conversion of the special-prime limbs back to Q */
    BM_KERNEL_KS_COMBINE = 4, /* (x - conv) * P^-1 + sigma(c0) (+ addend) */
    BM_KERNEL_RESCALE = 5,    /* rescale gather, lift and combine */
    BM_KERNEL_MAC = 6,        /* HE-C^3 multiply-accumulate over the parts */
    BM_KERNEL_MUL_PLAIN = 7,  /* ct x pt products (masks) */
    BM_KERNEL_OTHER = 8,      /* copies, conversions, client-side helpers */
    BM_KERNEL_KINDS = 9
};

/* Process-wide counters of kernel launches and of their algorithmic work, per
 * class: bytes (the reads and writes each launch must make, from its operand
 * sizes) and 32-bit multiply operations (for the NTT passes: 16 per 64-bit
 * modular butterfly -- the 32x32-bit partial products of the three 64-bit
 * products of a Shoup multiplication, counting low and high halves).  With
 * timing != 0 every later launch is bracketed by a CUDA event pair on its stream
 * and its device time accumulated (bm_match then runs its plan without the graph).
 * reset != 0 zeroes the counters.  Reading waits for the recorded events. */
bm_status bm_profile_control(uint32_t timing, uint32_t reset);
bm_status bm_profile_read(uint32_t kind, uint64_t* launches, double* device_ms, double* alg_bytes,
                          double* alg_mulops);

/* ---------------------------------------------------------------------------
 * Schedule model and part-size choice (Sec. 4: the cost F(N_in) of the match is
 * a sum over its homomorphic operations -- Propositions 1-3 -- of measured
 * per-operation times, and N_in = dim/part is picked where F is smallest).
 * Here the operations are the library's own launches, each timed on this GPU
 * as a + b * count.
 * ------------------------------------------------------------------------- */
enum {
    BM_OP_ROTATE = 0,     /* rotation (automorphism + key switch) of `count` ciphertexts at `level` */
    BM_OP_RESCALE = 1,    /* rescale of `count` ciphertexts from `level` */
    BM_OP_MUL_PLAIN = 2,  /* ct x pt product of `count` ciphertexts at `level` (masks) */
    BM_OP_MAC = 3,        /* HE-C^3 products: `queries` x `count` groups, `parts` products summed each */
    BM_OP_NTT = 4,        /* forward NTT of `count` limbs (query ingest) */
    BM_OP_INTT = 5,       /* inverse NTT of `count` limbs (score egress) */
    BM_OP_COPY = 6,       /* device copy of `count` level-0 ciphertexts (uncompressed outputs) */
    BM_OP_MAC_CT = 7,     /* HE-C^3 tensor products with an encrypted gallery, as BM_OP_MAC */
    BM_OP_MODUP = 8,      /* hoisted rotations: basis extension of `count` ciphertexts at `level` */
    BM_OP_ROT_HOISTED = 9,/* hoisted rotations: `count` rotations from extended ciphertexts */
    BM_OP_MAC_CIRC = 10,  /* hoisted Algorithm 1: `queries` x `count` outputs of `parts` mask products */
    BM_OP_ACCUM = 11,     /* sums of `count` ciphertexts at `level` into their targets (hoisted rounds) */
    BM_OP_IP_SUM = 12,    /* double-hoisted rounds: key-switch products of `count` rotations summed
                             into `parts` targets before ModDown */
    BM_OP_MODDOWN = 13,   /* double-hoisted rounds: ModDown of `count` sums, added to their targets */
    BM_OP_KINDS = 14
};

/* One kernel launch (or launch group) of a match schedule. */
typedef struct bm_op_launch {
    uint32_t op;          /* BM_OP_* */
    uint32_t level;       /* level of the input ciphertexts (0 for NTT / INTT / COPY; for
                             BM_OP_MAC on Q_L u P, the deferred division's products, L + alpha:
                             the limbs less one) */
    uint32_t count;       /* ciphertexts, limbs or groups, as listed above */
    uint32_t queries;     /* BM_OP_MAC: queries per product set; else 0 */
    uint32_t parts;       /* BM_OP_MAC: N_in; BM_OP_IP_SUM: targets; else 0 */
} bm_op_launch;

/* Per-launch device time of each op kind and input level, sampled at
 * BM_COST_POINTS sizes: t_us[op][level][k] is the time (microseconds) of one
 * launch of units[op][k] units, units increasing.  Units are `count`, except for
 * BM_OP_MAC: ceil(queries / 4) * count * parts (one read of a gallery
 * plaintext serves a tile of four queries; the same for BM_OP_MAC_CT and BM_OP_MAC_CIRC).  Between points the time is
 * interpolated linearly, above the last point extrapolated from the last two,
 * below the first taken as the first.  NTT, INTT and COPY use level 0. */
#define BM_COST_POINTS 8
typedef struct bm_op_costs {
    double units[BM_OP_KINDS][BM_COST_POINTS];
    double t_us[BM_OP_KINDS][BM_MAX_Q][BM_COST_POINTS];
} bm_op_costs;

/* Gallery kinds for the schedule model: a BM_PACK_* value, or'ed with
 * BM_LAYOUT_ENCRYPTED for a gallery of ciphertexts (bm_enroll_encrypted). */
#define BM_LAYOUT_ENCRYPTED 0x100u
/* ... or'ed with BM_LAYOUT_HOISTED for the hoisted form of Algorithm 1 (bm_gallery_set_expansion),
 * BM_LAYOUT_HOISTED_ROTSUM and BM_LAYOUT_HOISTED_COMPRESSION for the other hoisted forms. */
#define BM_LAYOUT_HOISTED 0x200u
#define BM_LAYOUT_HOISTED_ROTSUM 0x400u
#define BM_LAYOUT_HOISTED_COMPRESSION 0x800u
/* ... and BM_LAYOUT_DOUBLE_HOISTED for BM_SCHED_DOUBLE_HOISTED, BM_LAYOUT_FUSED_EXPANSION for
 * BM_SCHED_FUSED_EXPANSION, BM_LAYOUT_DEFERRED_DIVISION for BM_SCHED_DEFERRED_DIVISION,
 * BM_LAYOUT_FUSED_COMPRESSION for BM_SCHED_FUSED_COMPRESSION. */
#define BM_LAYOUT_DOUBLE_HOISTED 0x1000u
#define BM_LAYOUT_FUSED_EXPANSION 0x2000u
#define BM_LAYOUT_DEFERRED_DIVISION 0x4000u
#define BM_LAYOUT_FUSED_COMPRESSION 0x8000u

/* Host only (no device needed): the launches of the match of `n_queries`
 * queries against a gallery of n_ids identities in (dim, part_size, packing) under
 * `params` -- exactly the launches bm_match's plan makes, in order -- and the
 * device memory its plan holds.  Writes up to ops_cap launches to ops (ops may
 * be NULL) and the total to *n_ops; *plan_bytes gets the plan's bytes.
 * BM_E_PARAM / BM_E_DIM / BM_E_LEVEL as for bm_context_create / bm_gallery_layout. */
bm_status bm_plan_estimate(const bm_params* params, uint64_t n_ids, uint32_t dim, uint32_t part_size,
                           uint32_t packing, uint32_t n_queries, bm_op_launch* ops, size_t ops_cap,
                           size_t* n_ops, uint64_t* plan_bytes);

/* Host only: the predicted device time (ms) of that match: the sum over its
 * launches of the time `costs` gives each launch. */
bm_status bm_predict_match(const bm_params* params, const bm_op_costs* costs, uint64_t n_ids, uint32_t dim,
                           uint32_t part_size, uint32_t packing, uint32_t n_queries, double* ms,
                           uint64_t* plan_bytes);

/* Host only: the part size (N_in = dim / part) of smallest predicted time among
 * the powers of two 1..dim whose plan fits in `hbm_budget` bytes (0 = no limit);
 * ties go to the larger part (fewer keys).  BM_E_HBM_BUDGET if none fits. */
bm_status bm_choose_part(const bm_params* params, const bm_op_costs* costs, uint64_t n_ids, uint32_t dim,
                         uint32_t packing, uint32_t n_queries, uint64_t hbm_budget, uint32_t* part_size,
                         double* ms);

/* Times every op kind on this context's device at BM_COST_POINTS sizes per
 * level (1, 2, 4, ..., 128 ciphertexts or limbs; MAC_CIRC: 4 queries x 2^k parts; MAC: 4 queries x 8 parts x
 * 1..128 groups), with seeded random residues as operands (the values do not
 * change the time).  Rotations use the kernel shape the context currently picks
 * for each batch size, so run bm_autotune_keyswitch first.  Takes a few seconds
 * and up to ~9 GB of device memory at ring 2^16.  Levels an op cannot take
 * (rescale from level 0) stay 0. */
bm_status bm_measure_op_costs(bm_context* ctx, bm_op_costs* out);

/* Rotation kernels come in two shapes: 4 coefficients per thread (radix-4
 * register phases, 2 NTT rows per block) and 16 (radix-16 phases, 8 rows per
 * block).  bm_autotune_keyswitch times both at every level for batches of
 * 1, 2, 4, ..., 128 ciphertexts and keeps, per level, the smallest batch size
 * from which the 16-coefficient shape is faster at every larger size
 * (wide_batch_out[level], 2^30 = never; pass NULL to skip).
 * bm_set_ks_wide_batch sets one level's threshold by hand.  Plans built before
 * the change keep their kernels. */
bm_status bm_autotune_keyswitch(bm_context* ctx, uint32_t* wide_batch_out, size_t capacity);
bm_status bm_set_ks_wide_batch(bm_context* ctx, uint32_t level, uint32_t batch);

/* The standalone NTT (the match's ingest and egress transforms, and the transforms
 * of the client-side calls) comes in three shapes: 0 = radix-4 register phases with 2
 * rows or columns a block (ring 2^12: 8), 1 = radix-4 with 4 a block (ring 2^12: 16),
 * 2 = radix-16 phases with 8 a block (ring 2^16 only).  A batch of `limbs` limbs
 * falls in bucket k, the smallest with limbs <= 2^k (the last bucket, k =
 * BM_NTT_BUCKETS - 1, takes every larger batch).  bm_autotune_ntt times a forward
 * and an inverse transform of 2^k limbs in every shape for each bucket and keeps,
 * per bucket, the fastest (shape 0 unless another is 2% faster); shapes_out[k]
 * receives the choice (NULL to skip).  Every shape gives the same residues.
 * bm_set_ntt_shape sets one bucket by hand.  Plans built before keep their kernels.
 * (NTT radix and tile as tuned parameters: no counterpart in the paper, whose cost
 * model of Sec. 4 measures per-operation times the same way.) */
#define BM_NTT_BUCKETS 10
bm_status bm_autotune_ntt(bm_context* ctx, uint8_t* shapes_out, size_t capacity);
bm_status bm_set_ntt_shape(bm_context* ctx, uint32_t bucket, uint32_t shape);

/* Key-switching digits (dnum) chosen by the cost model of Sec. 4: for each dnum in
 * 1..4 that bm_context_create accepts with the other fields of *base, a context on
 * `device` is made, its kernel shapes tuned (bm_autotune_keyswitch, bm_autotune_ntt),
 * its per-operation costs measured (bm_measure_op_costs) and the match of n_queries
 * queries against n_ids identities (dim, part_size, packing: as bm_predict_match)
 * predicted; *dnum_out gets the dnum of least predicted time, ms_out[d - 1] (when not
 * NULL, capacity >= 4) each prediction in ms (0: dnum not taken).  More digits make
 * smaller digit products but more extension limbs and larger keys.  Takes about a
 * minute at ring 2^16.  BM_E_PARAM if no dnum is taken. */
bm_status bm_choose_dnum(const bm_params* base, int device, uint64_t n_ids, uint32_t dim, uint32_t part_size,
                         uint32_t packing, uint32_t n_queries, uint32_t* dnum_out, double* ms_out, size_t capacity);

#ifdef __cplusplus
}
#endif
#endif /* BLINDMATCH_H */
