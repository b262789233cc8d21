// tune.cu -- the match's cost model (Sec. 4) on this GPU.
//
// Sec. 4 writes the time of a match as a sum over its homomorphic operations
// (Propositions 1-3) of per-operation times measured on the target machine
// (Table 1), and picks N_in where that sum is smallest.  Here the operations are
// the library's own launches (bm_plan_estimate lists them), the per-launch times
// are measured on this GPU at several batch sizes, and the part size of least
// predicted time is chosen among the powers of two whose plan fits the memory
// budget.  The same measurements choose, per level, between the two rotation
// kernel shapes (4 or 16 coefficients per thread).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "bm_internal.h"

namespace bm {
namespace {

bm_status fail(bm_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

// Operand filler: word i of a buffer whose limbs (n words each) cycle through
// `period` primes gets a residue mod its limb's prime, from a splitmix64 hash
// of (seed, i).  Only the shapes matter for timing; the values stay in range so
// every kernel sees the inputs it is specified for.
__global__ void k_fill_residues(uint64_t* p, size_t words, uint32_t n, uint32_t period, DevTables tab,
                                uint64_t seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t j = (uint32_t)((i / n) % period);
        uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        p[i] = z % tab.q[j];
    }
}

cudaError_t fill(const Context& c, uint64_t* p, size_t words, uint32_t period, uint64_t seed, cudaStream_t s) {
    k_fill_residues<<<1216, 256, 0, s>>>(p, words, c.n, period, c.tab, seed);
    return cudaGetLastError();
}

// Average device time (us) of one call of f over `reps` calls after `warm`,
// CUDA events on s.
struct Timer {
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaSuccess;
    Timer(cudaStream_t s_) : s(s_) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
    }
    ~Timer() {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    template <class F>
    double us(F&& f, int warm, int reps) {
        for (int i = 0; i < warm; i++) keep(f());
        keep(cudaEventRecord(e0, s));
        for (int i = 0; i < reps; i++) keep(f());
        keep(cudaEventRecord(e1, s));
        keep(cudaEventSynchronize(e1));
        float ms = 0;
        keep(cudaEventElapsedTime(&ms, e0, e1));
        return err == cudaSuccess ? 1000.0 * ms / reps : 0.0;
    }
    void keep(cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) err = e;
    }
};

constexpr uint32_t kMaxB = 1u << (BM_COST_POINTS - 1);   // 128: the schedule's largest batch
constexpr uint32_t kMacQ = 4, kMacParts = 8;

int reps_for(uint32_t B) { return B <= 16 ? 10 : 5; }

// device array of B pointers base + k * stride
struct PtrList {
    DevBuf buf;
    cudaError_t make(uint64_t* base, size_t stride, uint32_t B) {
        std::vector<uint64_t*> h(B);
        for (uint32_t k = 0; k < B; k++) h[k] = base + (size_t)k * stride;
        cudaError_t e = buf.alloc(B);
        if (e != cudaSuccess) return e;
        return cudaMemcpy(buf.p, h.data(), B * sizeof(void*), cudaMemcpyHostToDevice);
    }
    uint64_t* const* get() const { return (uint64_t* const*)buf.p; }
};

double interp(const double* u, const double* t, double x) {
    const int P = BM_COST_POINTS;
    if (x <= u[0]) return t[0];
    for (int k = 0; k + 1 < P; k++)
        if (x <= u[k + 1]) return t[k] + (t[k + 1] - t[k]) * (x - u[k]) / (u[k + 1] - u[k]);
    return t[P - 2] + (t[P - 1] - t[P - 2]) * (x - u[P - 2]) / (u[P - 1] - u[P - 2]);
}

double launch_us(const bm_op_costs& k, const bm_op_launch& l) {
    double units = l.count;
    uint32_t level = l.level;
    double scale = 1.0;
    if (l.op >= BM_OP_KINDS) return 0.0;
    if (l.op == BM_OP_MAC || l.op == BM_OP_MAC_CT || l.op == BM_OP_MAC_CIRC) {
        units = std::ceil(l.queries / 4.0) * l.count * l.parts;
        // products on more limbs than the top measured level (the deferred division's
        // HE-C^3 on Q_L u P): that level's time scaled by the limbs, a MAC's cost
        // being proportional to them
        int top = (int)std::min<uint32_t>(level, BM_MAX_Q - 1);
        while (top > 0 && k.t_us[l.op][top][BM_COST_POINTS - 1] == 0.0) top--;
        if ((uint32_t)top < level) {
            scale = (level + 1.0) / (top + 1.0);
            level = (uint32_t)top;
        }
    }
    if (l.op == BM_OP_NTT || l.op == BM_OP_INTT || l.op == BM_OP_COPY) level = 0;
    if (level >= BM_MAX_Q) return 0.0;
    return scale * interp(k.units[l.op], k.t_us[l.op][level], units);
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" {

bm_status bm_predict_match(const bm_params* params, const bm_op_costs* costs, uint64_t n_ids, uint32_t dim,
                           uint32_t part_size, uint32_t packing, uint32_t n_queries, double* ms,
                           uint64_t* plan_bytes) {
    if (!params || !costs) return fail(BM_E_ARG, "null argument");
    std::vector<bm_op_launch> ops;
    size_t bytes = 0;
    bm_status st = schedule_launches(*params, n_ids, dim, part_size, packing, n_queries, &ops, &bytes);
    if (st != BM_OK) return st;
    double us = 0;
    for (const auto& l : ops) us += launch_us(*costs, l);
    if (ms) *ms = us / 1000.0;
    if (plan_bytes) *plan_bytes = bytes;
    return BM_OK;
}

bm_status bm_choose_part(const bm_params* params, const bm_op_costs* costs, uint64_t n_ids, uint32_t dim,
                         uint32_t packing, uint32_t n_queries, uint64_t hbm_budget, uint32_t* part_size,
                         double* ms) {
    if (!params || !costs || !part_size) return fail(BM_E_ARG, "null argument");
    if (!dim || (dim & (dim - 1))) return fail(BM_E_DIM, "dim must be a power of two");
    double best = 0;
    uint32_t best_part = 0;
    for (uint32_t part = dim; part >= 1; part /= 2) {
        double t = 0;
        uint64_t bytes = 0;
        bm_status st = bm_predict_match(params, costs, n_ids, dim, part, packing, n_queries, &t, &bytes);
        if (st != BM_OK) return st;
        if (hbm_budget && bytes > hbm_budget) continue;
        if (!best_part || t < best) {
            best = t;
            best_part = part;
        }
    }
    if (!best_part) return fail(BM_E_HBM_BUDGET, "no part size fits the device-memory budget");
    *part_size = best_part;
    if (ms) *ms = best;
    return BM_OK;
}

bm_status bm_set_ks_wide_batch(bm_context* ctxh, uint32_t level, uint32_t batch) {
    if (!ctxh) return fail(BM_E_ARG, "null context");
    Context& c = ctxh->c;
    if (level > c.L) return fail(BM_E_ARG, "level above the chain");
    c.ks_wide_batch[level] = batch;
    return BM_OK;
}

bm_status bm_autotune_keyswitch(bm_context* ctxh, uint32_t* wide_batch_out, size_t capacity) {
    if (!ctxh) return fail(BM_E_ARG, "null context");
    Context& c = ctxh->c;
    if (wide_batch_out && capacity < (size_t)c.L + 1) return fail(BM_E_ARG, "capacity below L + 1");
    BM_CUDA_TRY(cudaSetDevice(c.device));
    if (ks_fused_supported(c) && ks_has_wide(c)) {
        const size_t cw = ct_words(c, c.L);
        DevBuf in, out, scratch, key;
        BM_CUDA_TRY(in.alloc(cw * kMaxB));
        BM_CUDA_TRY(out.alloc(cw * kMaxB));
        BM_CUDA_TRY(scratch.alloc(ks_scratch_words(c, c.L, kMaxB)));
        BM_CUDA_TRY(key.alloc((size_t)c.digits.size() * 2 * c.nb * c.n));
        cudaStream_t s = c.stream;
        BM_CUDA_TRY(fill(c, key.p, key.words, c.nb, 11, s));
        const uint64_t gk = galois_of(c, 1);
        Timer tm(s);
        for (uint32_t level = 0; level <= c.L; level++) {
            const size_t cwl = ct_words(c, level);
            BM_CUDA_TRY(fill(c, in.p, cwl * kMaxB, level + 1, 12 + level, s));
            BM_CUDA_TRY(fill(c, out.p, cwl * kMaxB, level + 1, 13 + level, s));
            PtrList pin, pout;
            BM_CUDA_TRY(pin.make(in.p, cwl, kMaxB));
            BM_CUDA_TRY(pout.make(out.p, cwl, kMaxB));
            double t[2][BM_COST_POINTS];
            for (int k = 0; k < BM_COST_POINTS; k++) {
                const uint32_t B = 1u << k;
                for (int w = 0; w < 2; w++)
                    t[w][k] = tm.us([&] { return ks_rotate_fused_shape(c, w == 1, key.p, gk, level, B, pin.get(),
                                                                       pout.get(), pout.get(), scratch.p, s); },
                                    2, reps_for(B));
            }
            BM_CUDA_TRY(tm.err);
            // smallest B from which the wide shape wins (by 2%) at every larger size
            uint32_t thr = 1u << 30;
            for (int k = BM_COST_POINTS - 1; k >= 0 && t[1][k] < 0.98 * t[0][k]; k--) thr = 1u << k;
            c.ks_wide_batch[level] = thr;
        }
    }
    if (wide_batch_out)
        for (uint32_t l = 0; l <= c.L; l++) wide_batch_out[l] = c.ks_wide_batch[l];
    return BM_OK;
}

bm_status bm_set_ntt_shape(bm_context* ctxh, uint32_t bucket, uint32_t shape) {
    if (!ctxh) return fail(BM_E_ARG, "null context");
    if (bucket >= (uint32_t)kNttBuckets || shape >= (uint32_t)kNttShapes)
        return fail(BM_E_ARG, "bucket or shape out of range");
    ctxh->c.ntt_shape[bucket] = (uint8_t)shape;
    return BM_OK;
}

bm_status bm_autotune_ntt(bm_context* ctxh, uint8_t* shapes_out, size_t capacity) {
    if (!ctxh) return fail(BM_E_ARG, "null context");
    Context& c = ctxh->c;
    if (shapes_out && capacity < (size_t)kNttBuckets) return fail(BM_E_ARG, "capacity below BM_NTT_BUCKETS");
    BM_CUDA_TRY(cudaSetDevice(c.device));
    const uint32_t max_limbs = 1u << (kNttBuckets - 1);
    DevBuf buf;
    BM_CUDA_TRY(buf.alloc((size_t)max_limbs * c.n));
    cudaStream_t s = c.stream;
    BM_CUDA_TRY(fill(c, buf.p, buf.words, c.nb, 21, s));
    Timer tm(s);
    const int shapes = c.log_n == 16 ? kNttShapes : 2;
    for (int k = 0; k < kNttBuckets; k++) {
        const uint32_t limbs = 1u << k;
        // limbs cycle through the primes of the full basis (a batch of ciphertext limbs)
        LimbBatch b{buf.p, limbs, (uint64_t)c.n, 0, 1, {}};
        b.set(0, 0);
        double t[kNttShapes] = {};
        for (int sh = 0; sh < shapes; sh++)
            t[sh] = tm.us([&] {
                cudaError_t e = ntt_dispatch_shape(c, b, false, sh, s);
                return e != cudaSuccess ? e : ntt_dispatch_shape(c, b, true, sh, s);
            }, 2, reps_for(limbs));
        BM_CUDA_TRY(tm.err);
        int best = 0;
        for (int sh = 1; sh < shapes; sh++)
            if (t[sh] < 0.98 * t[best]) best = sh;
        c.ntt_shape[k] = (uint8_t)best;
    }
    if (shapes_out)
        for (int k = 0; k < kNttBuckets; k++) shapes_out[k] = c.ntt_shape[k];
    return BM_OK;
}

bm_status bm_choose_dnum(const bm_params* base, int device, uint64_t n_ids, uint32_t dim, uint32_t part_size,
                         uint32_t packing, uint32_t n_queries, uint32_t* dnum_out, double* ms_out, size_t capacity) {
    if (!base || !dnum_out) return fail(BM_E_ARG, "null argument");
    if (ms_out && capacity < (size_t)MAXD) return fail(BM_E_ARG, "capacity below 4");
    double best = 0;
    uint32_t best_d = 0;
    for (uint32_t d = 1; d <= (uint32_t)MAXD; d++) {
        if (ms_out) ms_out[d - 1] = 0;
        bm_params p = *base;
        p.dnum = d;
        bm_context* ctx = nullptr;
        if (bm_context_create(&p, device, &ctx) != BM_OK) continue;   // digits the kernels do not take
        bm_op_costs costs{};
        double ms = 0;
        uint64_t bytes = 0;
        bm_status st = bm_autotune_keyswitch(ctx, nullptr, 0);
        if (st == BM_OK) st = bm_autotune_ntt(ctx, nullptr, 0);
        if (st == BM_OK) st = bm_measure_op_costs(ctx, &costs);
        if (st == BM_OK) st = bm_predict_match(&p, &costs, n_ids, dim, part_size, packing, n_queries, &ms, &bytes);
        bm_context_destroy(ctx);
        if (st != BM_OK) return st;
        if (ms_out) ms_out[d - 1] = ms;
        if (!best_d || ms < best) {
            best = ms;
            best_d = d;
        }
    }
    if (!best_d) return fail(BM_E_PARAM, "no digit count the kernels take for these parameters");
    *dnum_out = best_d;
    return BM_OK;
}

bm_status bm_measure_op_costs(bm_context* ctxh, bm_op_costs* out) {
    if (!ctxh || !out) return fail(BM_E_ARG, "null argument");
    Context& c = ctxh->c;
    BM_CUDA_TRY(cudaSetDevice(c.device));
    std::memset(out, 0, sizeof(*out));
    for (int op = 0; op < BM_OP_KINDS; op++)
        for (int k = 0; k < BM_COST_POINTS; k++)
            out->units[op][k] = op == BM_OP_MAC_CIRC ? (double)(1u << k) * (double)(1u << k)   // 4 queries x (2^k)^2
                                : (op == BM_OP_MAC || op == BM_OP_MAC_CT ? (double)kMacParts : 1.0) * (double)(1u << k);
    cudaStream_t s = c.stream;
    Timer tm(s);
    const uint32_t L = c.L;
    {
        // rotations, rescales, mask products, NTTs, copies: batches of 1..128
        const size_t cw = ct_words(c, L);
        DevBuf in, outb, scratch, key, pt;
        BM_CUDA_TRY(in.alloc(cw * kMaxB));
        BM_CUDA_TRY(outb.alloc(cw * kMaxB));
        BM_CUDA_TRY(scratch.alloc(std::max(ks_scratch_words(c, L, kMaxB), rescale_scratch_words(c, L, kMaxB))));
        BM_CUDA_TRY(key.alloc((size_t)c.digits.size() * 2 * c.nb * c.n));
        BM_CUDA_TRY(pt.alloc((size_t)(L + 1) * c.n));
        BM_CUDA_TRY(fill(c, key.p, key.words, c.nb, 21, s));
        BM_CUDA_TRY(fill(c, pt.p, pt.words, L + 1, 22, s));
        const uint64_t gk = galois_of(c, 1);
        for (uint32_t level = 0; level <= L; level++) {
            const size_t cwl = ct_words(c, level);
            BM_CUDA_TRY(fill(c, in.p, cwl * kMaxB, level + 1, 23 + level, s));
            BM_CUDA_TRY(fill(c, outb.p, cwl * kMaxB, level + 1, 33 + level, s));
            PtrList pin, pout, ppt, pres;
            BM_CUDA_TRY(pin.make(in.p, cwl, kMaxB));
            BM_CUDA_TRY(pout.make(outb.p, cwl, kMaxB));
            BM_CUDA_TRY(ppt.make(pt.p, 0, kMaxB));
            if (level) BM_CUDA_TRY(pres.make(outb.p, ct_words(c, level - 1), kMaxB));
            for (int k = 0; k < BM_COST_POINTS; k++) {
                const uint32_t B = 1u << k;
                const int r = reps_for(B);
                out->t_us[BM_OP_ROTATE][level][k] = tm.us(
                    [&] { return ks_rotate(c, key.p, gk, level, B, pin.get(), pout.get(), pout.get(), scratch.p, s); },
                    2, r);
                if (level)
                    out->t_us[BM_OP_RESCALE][level][k] =
                        tm.us([&] { return rescale(c, level, B, pin.get(), pres.get(), scratch.p, s); }, 2, r);
                out->t_us[BM_OP_MUL_PLAIN][level][k] = tm.us(
                    [&] { return mul_plain(c, level, B, pin.get(), (const uint64_t* const*)ppt.get(), pout.get(), s); },
                    2, r);
                if (level == 0) {
                    // limb counts for the transforms, level-0 ciphertexts for the copies
                    out->t_us[BM_OP_NTT][0][k] = tm.us([&] { return ntt_forward(c, packed(c, outb.p, B, 1), s); }, 2, r);
                    out->t_us[BM_OP_INTT][0][k] = tm.us([&] { return ntt_inverse(c, packed(c, outb.p, B, 1), s); }, 2, r);
                    out->t_us[BM_OP_COPY][0][k] = tm.us(
                        [&] {
                            return cudaMemcpyAsync(in.p, outb.p, (size_t)B * ct_words(c, 0) * 8,
                                                   cudaMemcpyDeviceToDevice, s);
                        },
                        2, r);
                }
            }
            BM_CUDA_TRY(tm.err);
        }
    }
    if (ks_fused_supported(c)) {
        // hoisted rotations at every level: basis extension of 1..128 ciphertexts, 1..128
        // rotations from extensions, sums of 1..128 ciphertexts, 1..128 rotations summed
        // before ModDown (four to a target) and 1..128 such ModDowns; at the top level
        // the circulant products of hoisted Algorithm 1, 4 queries x 2^k parts
        const size_t cw = ct_words(c, L), ew = ks_ext_words(c, L);
        DevBuf in, outb, ext, scratch, key, masks, hat, ctw, t0, plist;
        BM_CUDA_TRY(in.alloc(cw * kMaxB));
        BM_CUDA_TRY(outb.alloc(cw * kMaxB));
        BM_CUDA_TRY(ext.alloc(ew * kMaxB));
        BM_CUDA_TRY(scratch.alloc(std::max(ks_modup_scratch_words(c, L, kMaxB), ks_hoisted_scratch_words(c, L, kMaxB))));
        BM_CUDA_TRY(key.alloc((size_t)c.digits.size() * 2 * c.nb * c.n));
        BM_CUDA_TRY(masks.alloc((size_t)kMaxB * (L + 1) * c.n));
        BM_CUDA_TRY(hat.alloc((size_t)kMaxB * (L + 1) * c.n));
        BM_CUDA_TRY(ctw.alloc((size_t)(L + 1) * kMaxCircParts * 2));   // twiddle pairs of up to 32 parts
        BM_CUDA_TRY(t0.alloc((size_t)kMacQ * kMaxB * cw));
        BM_CUDA_TRY(fill(c, in.p, cw * kMaxB, L + 1, 61, s));
        BM_CUDA_TRY(fill(c, key.p, key.words, c.nb, 62, s));
        BM_CUDA_TRY(fill(c, masks.p, masks.words, L + 1, 63, s));
        BM_CUDA_TRY(fill(c, hat.p, hat.words, L + 1, 64, s));
        BM_CUDA_TRY(fill(c, ctw.p, ctw.words, L + 1, 65, s));
        // element lists: extension, source, key, Galois element (rotation by one slot), output
        std::vector<uint64_t*> h;
        for (uint32_t k = 0; k < kMaxB; k++) h.push_back(ext.p + k * ew);
        for (uint32_t k = 0; k < kMaxB; k++) h.push_back(in.p + k * cw);
        for (uint32_t k = 0; k < kMaxB; k++) h.push_back(key.p);
        for (uint32_t k = 0; k < kMaxB; k++) h.push_back(reinterpret_cast<uint64_t*>((uintptr_t)galois_of(c, 1)));
        for (uint32_t k = 0; k < kMaxB; k++) h.push_back(outb.p + k * cw);
        for (uint32_t k = 0; k < kMacQ * kMaxB; k++) h.push_back(in.p + (k % kMaxB) * cw);   // R lists
        BM_CUDA_TRY(plist.alloc(h.size()));
        BM_CUDA_TRY(cudaMemcpy(plist.p, h.data(), h.size() * sizeof(void*), cudaMemcpyHostToDevice));
        uint64_t* const* dl = (uint64_t* const*)plist.p;
        // accumulation lists: B targets, one source each (offsets 0..B)
        DevBuf offs;
        std::vector<uint64_t> ho(kMaxB + 1);
        for (uint32_t k = 0; k <= kMaxB; k++) ho[k] = k;
        BM_CUDA_TRY(offs.alloc(kMaxB + 1));
        BM_CUDA_TRY(cudaMemcpy(offs.p, ho.data(), (kMaxB + 1) * 8, cudaMemcpyHostToDevice));
        // double-hoisted rounds: 2^k rotations summed four to a target (row k of offs4)
        DevBuf offs4;
        std::vector<uint64_t> h4((size_t)BM_COST_POINTS * (kMaxB + 1));
        for (int k = 0; k < BM_COST_POINTS; k++)
            for (uint32_t t = 0; t <= kMaxB; t++) h4[(size_t)k * (kMaxB + 1) + t] = std::min<uint64_t>(4ull * t, 1ull << k);
        BM_CUDA_TRY(offs4.alloc(h4.size()));
        BM_CUDA_TRY(cudaMemcpy(offs4.p, h4.data(), h4.size() * 8, cudaMemcpyHostToDevice));
        for (uint32_t level = 0; level <= L; level++) {
            for (int k = 0; k < BM_COST_POINTS; k++) {
                const uint32_t B = 1u << k;
                const int r = reps_for(B);
                out->t_us[BM_OP_MODUP][level][k] = tm.us(
                    [&] { return ks_modup_hoisted(c, level, B, (uint64_t* const*)(dl + kMaxB), ext.p, scratch.p, s); },
                    2, r);
                out->t_us[BM_OP_ROT_HOISTED][level][k] = tm.us(
                    [&] {
                        return ks_rotate_hoisted(c, level, B, (const uint64_t* const*)dl,
                                                 (const uint64_t* const*)(dl + kMaxB),
                                                 (const uint64_t* const*)(dl + 2 * kMaxB),
                                                 (const uint64_t*)(dl + 3 * kMaxB), dl + 4 * kMaxB, scratch.p, s);
                    },
                    2, r);
                out->t_us[BM_OP_ACCUM][level][k] = tm.us(
                    [&] {
                        return accumulate(c, level, B, dl + 4 * kMaxB, (const uint64_t* const*)(dl + kMaxB), offs.p,
                                          B, s);
                    },
                    2, r);
                out->t_us[BM_OP_IP_SUM][level][k] = tm.us(
                    [&] {
                        return ks_ipsum_hoisted(c, level, (B + 3) / 4, offs4.p + (size_t)k * (kMaxB + 1), B,
                                                (const uint64_t* const*)dl, (const uint64_t* const*)(dl + kMaxB),
                                                (const uint64_t* const*)(dl + 2 * kMaxB),
                                                (const uint64_t*)(dl + 3 * kMaxB), scratch.p, s);
                    },
                    2, r);
                out->t_us[BM_OP_MODDOWN][level][k] =
                    tm.us([&] { return ks_moddown_add(c, level, B, dl + 4 * kMaxB, scratch.p, s); }, 2, r);
                if (level == L)
                    out->t_us[BM_OP_MAC_CIRC][L][k] = tm.us(
                        [&] {
                            // the schedule's form: the convolution over the parts up to 32 parts
                            return mac_circ(c, L, kMacQ, B, (const uint64_t* const*)(dl + 5 * kMaxB), masks.p, hat.p,
                                            (const ulonglong2*)ctw.p, t0.p, s);
                        },
                        2, r);
            }
            BM_CUDA_TRY(tm.err);
        }
    }
    {
        // HE-C^3 products: 4 queries x 8 parts x 1..128 groups, at the levels a
        // gallery can sit (L - 1 with Algorithm 1 on the server, L without)
        // (and the same with a gallery of ciphertexts: tensor products, two outputs)
        const uint32_t Gmax = kMaxB;
        DevBuf T, P, acc, acc2;
        BM_CUDA_TRY(T.alloc((size_t)kMacQ * kMacParts * ct_words(c, L)));
        BM_CUDA_TRY(P.alloc((size_t)Gmax * kMacParts * ct_words(c, L)));
        BM_CUDA_TRY(acc.alloc((size_t)kMacQ * Gmax * ct_words(c, L)));
        BM_CUDA_TRY(acc2.alloc((size_t)kMacQ * Gmax * ct_words(c, L)));
        for (uint32_t level = (L ? L - 1 : 0); level <= L; level++) {
            BM_CUDA_TRY(fill(c, T.p, (size_t)kMacQ * kMacParts * ct_words(c, level), level + 1, 41 + level, s));
            BM_CUDA_TRY(fill(c, P.p, (size_t)Gmax * kMacParts * ct_words(c, level), level + 1, 51 + level, s));
            for (int k = 0; k < BM_COST_POINTS; k++) {
                const uint32_t G = 1u << k;
                out->t_us[BM_OP_MAC][level][k] =
                    tm.us([&] { return mac(c, level, kMacQ, G, kMacParts, T.p, P.p, acc.p, s); }, 2, reps_for(G));
                out->t_us[BM_OP_MAC_CT][level][k] = tm.us(
                    [&] { return mac_ct(c, level, kMacQ, G, kMacParts, T.p, P.p, acc.p, acc2.p, s); }, 2, reps_for(G));
            }
            BM_CUDA_TRY(tm.err);
        }
    }
    return BM_OK;
}

}  // extern "C"
