// encrypt.cu -- batched client-side encryption (Sec. 3.2 templates, Sec. 3.3
// queries) with the noise drawn on the GPU.
//
// The encryption is the one of bm_encrypt_query, ct = (v*pk0 + e0 + m, v*pk1 + e1)
// with v ~ ZO(1/2) and e0, e1 discrete Gaussian, every coefficient drawn from
// Philox4x64-10 keyed by (seed, tag) at counter (object, 0, coefficient, 0),
// object = vector_id * 256 + part.  Philox is counter based, so the device draws
// the same words as the host samplers: a batch is bit-identical to the same
// vectors encrypted one by one.  The CKKS encoding (FP64 canonical embedding)
// stays on the host, spread over its cores; the products with the public key run
// in the NTT domain over every ciphertext of the batch at once.
#include <cuda_runtime.h>

#include <cstring>
#include <memory>
#include <vector>

#include "bm_internal.h"

namespace bm {
namespace {

bm_status fail(bm_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 64x64->128
// multiplications with the published round multipliers and Weyl key increments.
__device__ __forceinline__ void philox(uint64_t k0, uint64_t k1, uint64_t x0, uint64_t x1, uint64_t x2, uint64_t x3,
                                       uint64_t& w0) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
        const uint64_t hi0 = __umul64hi(m0, x0), lo0 = m0 * x0;
        const uint64_t hi1 = __umul64hi(m1, x2), lo1 = m1 * x2;
        const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x1 = lo1;
        x3 = lo0;
        x0 = y0;
        x2 = y2;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    w0 = x0;
}

struct Cdt {
    uint64_t t[20];   // t[k] = floor(2^63 * P(|e| <= k)), t[kmax] = 2^63
};

// noise of ciphertext k, coefficient i: v (ZO(1/2): w0 & 3 in {0, 1} -> 0, 2 -> +1,
// 3 -> -1), e0 + m, e1 (|e| = min{k : (w0 >> 1) < t[k]}, sign from w0's low bit)
__global__ void k_enc_noise(uint64_t seed, const uint64_t* __restrict__ objs, uint32_t n_cts, uint32_t n, Cdt cdt,
                            uint32_t kmax, const int64_t* __restrict__ m, int64_t* __restrict__ v,
                            int64_t* __restrict__ e0, int64_t* __restrict__ e1) {
    const size_t total = (size_t)n_cts * n;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const uint64_t obj = objs[idx / n], i = idx % n;
        uint64_t w;
        philox(seed, TAG_ENC_V, obj, 0, i, 0, w);
        const uint32_t z = (uint32_t)(w & 3);
        v[idx] = z == 2 ? 1 : (z == 3 ? -1 : 0);
        int64_t g[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            philox(seed, h == 0 ? TAG_ENC_E0 : TAG_ENC_E1, obj, 0, i, 0, w);
            const uint64_t u = w >> 1;
            uint32_t mag = 0;
            while (mag < kmax && u >= cdt.t[mag]) mag++;
            g[h] = (w & 1) ? -(int64_t)mag : (int64_t)mag;
        }
        e0[idx] = g[0] + m[idx];
        e1[idx] = g[1];
    }
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" {

bm_status bm_encrypt_batch(bm_context* ctxh, const bm_public_key* pk, const double* vectors, uint64_t n_vec,
                           uint32_t dim, uint32_t part_size, uint32_t mode, uint64_t seed, uint64_t first_id,
                           uint32_t flags, bm_ciphertext** out) {
    if (!ctxh || !pk || !vectors || !out || n_vec == 0) return fail(BM_E_ARG, "null argument or empty batch");
    if (mode != BM_QUERY_TILED && mode != BM_QUERY_EXPANDED && mode != BM_QUERY_TEMPLATE)
        return fail(BM_E_ARG, "unknown query mode");
    if (flags & ~(uint32_t)BM_ENC_KEEP_DEVICE) return fail(BM_E_ARG, "unknown flags");
    Context& c = ctxh->c;
    if (pk->k.ctx != &c) return fail(BM_E_ARG, "key from another context");
    if (!dim || (dim & (dim - 1)) || !part_size || (part_size & (part_size - 1)) || part_size > dim ||
        dim > c.slots)
        return fail(BM_E_DIM, "dim and part size must be powers of two with part <= dim <= N/2");
    BM_CUDA_TRY(cudaSetDevice(c.device));
    cudaStream_t s = c.stream;
    const uint32_t n = c.n, S = c.slots, L1 = c.L + 1;
    const uint32_t per = mode == BM_QUERY_EXPANDED ? dim / part_size : 1;   // ciphertexts per vector
    const size_t cw = (size_t)2 * L1 * n;
    const uint32_t chunk_v = std::max<uint32_t>(1, 64 / per);              // vectors per chunk
    const uint32_t cmax = chunk_v * per;
    Cdt cdt{};
    const uint32_t kmax = 19;
    cdt_table(c.params.sigma, kmax, cdt.t);
    DevBuf dm, dv, de0, de1, V, CT, P, dobj;
    BM_CUDA_TRY(dm.alloc((size_t)cmax * n));
    BM_CUDA_TRY(dv.alloc((size_t)cmax * n));
    BM_CUDA_TRY(de0.alloc((size_t)cmax * n));
    BM_CUDA_TRY(de1.alloc((size_t)cmax * n));
    BM_CUDA_TRY(V.alloc((size_t)cmax * L1 * n));
    BM_CUDA_TRY(CT.alloc((size_t)cmax * cw));
    BM_CUDA_TRY(P.alloc((size_t)cmax * L1 * n));
    BM_CUDA_TRY(dobj.alloc(cmax));
    uint64_t* pinned = nullptr;
    BM_CUDA_TRY(cudaMallocHost(&pinned, (size_t)cmax * cw * 8));
    std::unique_ptr<uint64_t, decltype(&cudaFreeHost)> pin_guard(pinned, &cudaFreeHost);
    std::vector<int64_t> m((size_t)cmax * n);
    std::vector<uint64_t> objs(cmax);
    std::vector<bm_ciphertext*> made;
    auto cleanup = [&](bm_status st) {
        for (bm_ciphertext* h : made) delete h;
        return st;
    };
#define ENC_TRY(expr)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (expr);                                                                        \
        if (e_ != cudaSuccess) return cleanup(fail(BM_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_))); \
    } while (0)
    for (uint64_t v0 = 0; v0 < n_vec; v0 += chunk_v) {
        const uint32_t nv = (uint32_t)std::min<uint64_t>(chunk_v, n_vec - v0), nc = nv * per;
        // messages on the host cores: the slot layout of the mode, encoded at scale 2^log_scale
#pragma omp parallel for schedule(dynamic)
        for (int k = 0; k < (int)nc; k++) {
            const double* q = vectors + (v0 + k / per) * dim;
            const uint32_t part = k % per;
            std::vector<double> z(S);
            for (uint32_t j = 0; j < S; j++) {
                if (mode == BM_QUERY_TILED) z[j] = q[j % dim];
                else if (mode == BM_QUERY_EXPANDED) z[j] = q[part * part_size + (j % part_size)];
                else z[j] = j < dim ? q[j] : 0.0;
            }
            encode_real(c, z.data(), c.scale, m.data() + (size_t)k * n);
        }
        for (uint32_t k = 0; k < nc; k++) objs[k] = (first_id + v0 + k / per) * 256 + k % per;
        ENC_TRY(cudaMemcpyAsync(dm.p, m.data(), (size_t)nc * n * 8, cudaMemcpyHostToDevice, s));
        ENC_TRY(cudaMemcpyAsync(dobj.p, objs.data(), (size_t)nc * 8, cudaMemcpyHostToDevice, s));
        k_enc_noise<<<1216, 256, 0, s>>>(seed, dobj.p, nc, n, cdt, kmax, (const int64_t*)dm.p, (int64_t*)dv.p,
                                         (int64_t*)de0.p, (int64_t*)de1.p);
        ENC_TRY(cudaGetLastError());
        // v and the two noise polynomials in RNS, NTT domain
        LimbBatch vb = packed(c, V.p, nc, L1);
        LimbBatch c0b = limbs_of(CT.p, nc, L1, cw), c1b = limbs_of(CT.p + (size_t)L1 * n, nc, L1, cw);
        ENC_TRY(lift_signed(c, (const int64_t*)dv.p, vb, s));
        ENC_TRY(lift_signed(c, (const int64_t*)de0.p, c0b, s));
        ENC_TRY(lift_signed(c, (const int64_t*)de1.p, c1b, s));
        ENC_TRY(ntt_forward(c, vb, s));
        ENC_TRY(ntt_forward(c, packed(c, CT.p, 2 * nc, L1), s));
        // c_comp += v * pk_comp (pk in Montgomery form, the same for every ciphertext)
        for (int comp = 0; comp < 2; comp++) {
            LimbBatch pkb = limbs_of(pk->k.d_ntt + (size_t)comp * L1 * n, nc, L1, 0);
            LimbBatch pb = packed(c, P.p, nc, L1);
            ENC_TRY(pointwise_mul(c, vb, pkb, pb, s));
            LimbBatch cb = comp == 0 ? c0b : c1b;
            ENC_TRY(pointwise_addsub(c, cb, pb, cb, false, s));
        }
        ENC_TRY(ntt_inverse(c, packed(c, CT.p, 2 * nc, L1), s));
        ENC_TRY(cudaMemcpyAsync(pinned, CT.p, (size_t)nc * cw * 8, cudaMemcpyDeviceToHost, s));
        for (uint32_t vi = 0; vi < nv; vi++) {
            auto* ch = new bm_ciphertext();
            made.push_back(ch);
            ch->ref.attach(&c);
            Ciphertext& ct = ch->ct;
            ct.ctx = &c;
            ct.n_cts = per;
            ct.level = c.L;
            if (flags & BM_ENC_KEEP_DEVICE) {
                if (cudaMalloc(&ct.d_coef, (size_t)per * cw * 8) != cudaSuccess)
                    return cleanup(fail(BM_E_OOM, "device allocation failed"));
                ENC_TRY(cudaMemcpyAsync(ct.d_coef, CT.p + (size_t)vi * per * cw, (size_t)per * cw * 8,
                                            cudaMemcpyDeviceToDevice, s));
            }
        }
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cleanup(fail(BM_E_CUDA, std::string("encrypt: ") + cudaGetErrorString(e)));
        for (uint32_t vi = 0; vi < nv; vi++) {
            Ciphertext& ct = made[v0 + vi]->ct;
            const uint64_t* src = pinned + (size_t)vi * per * cw;
            ct.host.assign(src, src + (size_t)per * cw);
        }
    }
#undef ENC_TRY
    for (uint64_t k = 0; k < n_vec; k++) out[k] = made[k];
    return BM_OK;
}

}  // extern "C"
