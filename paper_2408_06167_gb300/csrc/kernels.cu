// kernels.cu -- GPU kernels of the Blind-Match match path (sm_103a).
//
// RNS-CKKS operations of Sec. 2 (Add, Mul(P), Rot, Res) on limb-major
// uint64 buffers ([ct][poly][limb][N]), in the NTT domain:
//  * negacyclic NTT (Cooley-Tukey, bit-reversed psi twiddles, natural -> bit-
//    reversed order; Gentleman-Sande inverse) split in two passes over an
//    N1 x N2 view: a column pass for the first log N1 stages and a row pass
//    for the rest, each staged through shared memory;
//  * rotation = Galois automorphism + hybrid key switching: the automorphism is
//    fused into the ModUp gather (coefficient domain) and into the final
//    combine (NTT-domain permutation of c0); ModUp's fast base conversion, the
//    inner product with the rotation key (Montgomery products) and ModDown's
//    conversion and scaling by P^{-1} are one kernel each;
//  * rescale by the last prime with a centred lift (rounding division);
//  * ct x pt products and the HE-C^3 multiply-accumulate over the parts.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

#include "bm_internal.h"

namespace bm {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint32_t brev_bits(uint32_t x, uint32_t bits) {
    return __brev(x) >> (32 - bits);
}

// NTT-domain index of the automorphism X -> X^k: out[i] = in[src(i)].
__device__ __forceinline__ uint32_t ntt_perm_src(uint32_t i, uint32_t log_n, uint64_t galois) {
    const uint32_t mask2n = (2u << log_n) - 1;
    const uint32_t r = brev_bits(i, log_n);
    const uint32_t e = ((2u * r + 1u) * (uint32_t)galois) & mask2n;
    return brev_bits((e - 1u) >> 1, log_n);
}

__device__ __forceinline__ uint64_t* limb_ptr(const LimbBatch& b, uint32_t limb, uint32_t n) {
    const uint32_t poly = limb / b.nl, k = limb % b.nl;
    return b.base + (size_t)poly * b.poly_stride + (size_t)(b.limb_off + k) * n;
}

}  // namespace
}  // namespace bm

#include "ntt_reg.cuh"

namespace bm {
namespace {

// register-resident passes for even pass sizes (ring 2^12: 64 x 64, ring 2^16: 256 x 256)
template <int LA, int LB, int LT, int C, int R>
cudaError_t ntt_launch_reg(const LimbBatch& b, const DevTables& tab, bool inv, cudaStream_t s) {
    const uint32_t limbs = b.n_polys * b.nl;
    if (limbs == 0) return cudaSuccess;
    const dim3 gc(limbs, (1 << LB) / C), gr(limbs, (1 << LA) / R);
    const int tc = C * (1 << (LA - LT)), tr = R * (1 << (LB - LT));
    const double bytes = 16.0 * (1 << (LA + LB)) * limbs;   // each pass reads and writes every limb once
    const double ops_c = 16.0 * (1 << (LA + LB - 1)) * LA * limbs;   // 16 mul ops per butterfly
    const double ops_r = 16.0 * (1 << (LA + LB - 1)) * LB * limbs;
    if (!inv) {
        { ProfScope ps(BM_KERNEL_NTT, s, bytes, ops_c); pdl_launch(nttr::k_col_fwd<LA, LB, LT, C>, gc, tc, 0, s, b, tab); }
        { ProfScope ps(BM_KERNEL_NTT, s, bytes, ops_r); pdl_launch(nttr::k_row_fwd<LA, LB, LT, R>, gr, tr, 0, s, b, tab); }
    } else {
        { ProfScope ps(BM_KERNEL_NTT, s, bytes, ops_r); pdl_launch(nttr::k_row_inv<LA, LB, LT, R>, gr, tr, 0, s, b, tab); }
        { ProfScope ps(BM_KERNEL_NTT, s, bytes, ops_c); pdl_launch(nttr::k_col_inv<LA, LB, LT, C>, gc, tc, 0, s, b, tab); }
    }
    return cudaGetLastError();
}

}  // namespace

// The standalone NTT in one of three shapes (the tuner's choice per batch size, see
// ntt_shape_of): 0 = radix-4 register phases, 2 rows or columns a block (ring 2^12: 8);
// 1 = radix-4, 4 a block (ring 2^12: 16); 2 = radix-16 phases, 8 a block (ring 2^16
// only; ring 2^12 keeps shape 0).  Every shape computes the same transform and ends in
// canonical residues, so the choice never changes a result.
cudaError_t ntt_dispatch_shape(const Context& c, const LimbBatch& b, bool inv, int shape, cudaStream_t s) {
    switch (c.log_n) {
        case 12:
            return shape == 1 ? ntt_launch_reg<6, 6, 2, 16, 16>(b, c.tab, inv, s)
                              : ntt_launch_reg<6, 6, 2, 8, 8>(b, c.tab, inv, s);
        case 16:
            return shape == 2   ? ntt_launch_reg<8, 8, 4, 8, 8>(b, c.tab, inv, s)
                   : shape == 1 ? ntt_launch_reg<8, 8, 2, 4, 4>(b, c.tab, inv, s)
                                : ntt_launch_reg<8, 8, 2, 2, 2>(b, c.tab, inv, s);
        default: return cudaErrorInvalidValue;
    }
}

namespace {

cudaError_t ntt_dispatch(const Context& c, const LimbBatch& b, bool inv, cudaStream_t s) {
    return ntt_dispatch_shape(c, b, inv, c.ntt_shape[ntt_bucket(b.n_polys * b.nl)], s);
}

// ---------------------------------------------------------------------------
// elementwise limb kernels: grid (limbs, chunks of a limb), the limb on x so
// that any number of limbs fits (gridDim.y is limited to 65535)
// ---------------------------------------------------------------------------

// x * 2^-64 mod q (leave Montgomery form)
__global__ void k_from_mont(LimbBatch lb, DevTables tab, uint32_t n) {
    const uint32_t limb = blockIdx.x;
    const int pi = lb.prime(limb % lb.nl);
    uint64_t* a = limb_ptr(lb, limb, n);
    const uint64_t q = tab.q[pi], qn = tab.qneg[pi];
    for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x)
        a[i] = mont(a[i], 1, q, qn);
}

// x * 2^64 mod q (enter Montgomery form): mont(x, 2^128 mod q)
__global__ void k_to_mont(LimbBatch lb, DevTables tab, uint32_t n) {
    const uint32_t limb = blockIdx.x;
    const int pi = lb.prime(limb % lb.nl);
    uint64_t* a = limb_ptr(lb, limb, n);
    const uint64_t q = tab.q[pi], qn = tab.qneg[pi], f = tab.r2[pi];
    for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x)
        a[i] = mont(a[i], f, q, qn);
}

__global__ void k_lift_signed(const int64_t* v, LimbBatch lb, DevTables tab, uint32_t n) {
    const uint32_t limb = blockIdx.x;
    const int pi = lb.prime(limb % lb.nl);
    uint64_t* a = limb_ptr(lb, limb, n);
    const uint64_t q = tab.q[pi];
    const int64_t* src = v + (size_t)(limb / lb.nl) * n;
    for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x) {
        const int64_t x = src[i];
        const uint64_t m = x >= 0 ? (uint64_t)x : (uint64_t)(-x);
        const uint64_t r = reduce2(shoup_lazy(m, 1, tab.rsh[pi], q), q);
        a[i] = x >= 0 ? r : negm(r, q);
    }
}

__global__ void k_pointwise(LimbBatch A, LimbBatch B, LimbBatch O, DevTables tab, uint32_t n, int op) {
    const uint32_t limb = blockIdx.x;
    const int pi = A.prime(limb % A.nl);
    const uint64_t* a = limb_ptr(A, limb, n);
    const uint64_t* b = limb_ptr(B, limb, n);
    uint64_t* o = limb_ptr(O, limb, n);
    const uint64_t q = tab.q[pi], qn = tab.qneg[pi];
    for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x) {
        if (op == 0) o[i] = mont(a[i], b[i], q, qn);
        else if (op == 1) o[i] = addm(a[i], b[i], q);
        else o[i] = subm(a[i], b[i], q);
    }
}

__global__ void k_permute(LimbBatch I, LimbBatch O, uint32_t log_n, uint64_t galois) {
    const uint32_t n = 1u << log_n, limb = blockIdx.x;
    const uint64_t* a = limb_ptr(I, limb, n);
    uint64_t* o = limb_ptr(O, limb, n);
    for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x)
        o[i] = a[ntt_perm_src(i, log_n, galois)];
}

struct ScalarK {
    uint64_t w[MAXB], wsh[MAXB];
};

__global__ void k_scalar(LimbBatch I, LimbBatch O, ScalarK sk, DevTables tab, uint32_t n) {
    const uint32_t limb = blockIdx.x, k = limb % I.nl;
    const int pi = I.prime(k);
    const uint64_t* a = limb_ptr(I, limb, n);
    uint64_t* o = limb_ptr(O, limb, n);
    const uint64_t q = tab.q[pi];
    for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x)
        o[i] = shoup(a[i], sk.w[k], sk.wsh[k], q);
}

// ---------------------------------------------------------------------------
// products
// ---------------------------------------------------------------------------

// grid (B * 2 * (lvl + 1), chunks of a limb): one limb of one ciphertext per x index
// (gridDim.x has room for any batch; gridDim.y is limited to 65535)
__global__ void k_mul_plain(uint64_t* const* in, const uint64_t* const* pt, uint64_t* const* out,
                            uint32_t lvl, DevTables tab, uint32_t n) {
    const uint32_t l1 = lvl + 1;
    const uint32_t y = blockIdx.x, b = y / (2 * l1), c = (y / l1) % 2, j = y % l1;
    const uint64_t q = tab.q[j], qn = tab.qneg[j];
    pdl_wait();
    const uint64_t* s = in[b] + ((size_t)c * l1 + j) * n;
    const uint64_t* m = pt[b] + (size_t)j * n;
    uint64_t* o = out[b] + ((size_t)c * l1 + j) * n;
    for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x)
        o[i] = mont(s[i], m[i], q, qn);
}

// ---------------------------------------------------------------------------
// HE-C^3 products (Algorithm 2's Mul and the sum over the parts).  For one
// coefficient of one limb the products of Q queries with G groups over N_in parts
// form a small Q x N_in by N_in x G product; a thread keeps QT x GT of its sums in
// registers, so each part of a query is read once per GT groups and each gallery
// plaintext once per QT queries.  Blocks are numbered tiles fastest, then
// coefficient chunks, then limbs: the blocks in flight share one coefficient range
// of one limb, and the slices they read stay in L2 while the expanded queries
// stream from HBM once per GT groups.
// ---------------------------------------------------------------------------

constexpr int kMacThreads = 128;

struct MacTile {
    uint32_t q0, g0, j, c;
    uint32_t p;
};
// block order: ciphertext component (kMacPolys of them a block's tile set) fastest,
// then group tiles, query tiles, coefficient chunks, limbs
__device__ __forceinline__ MacTile mac_tile(uint32_t n_qt, uint32_t n_gt, uint32_t chunks, int QT, int GT,
                                            uint32_t n_c) {
    uint32_t b = blockIdx.x;
    MacTile t;
    t.c = b % n_c;
    b /= n_c;
    t.g0 = (b % n_gt) * GT;
    b /= n_gt;
    t.q0 = (b % n_qt) * QT;
    b /= n_qt;
    t.p = (b % chunks) * kMacThreads + threadIdx.x;
    t.j = b / chunks;
    return t;
}

// acc[q][g][c][j] = sum_i T[q][i][c][j] * P[g][i][j] (P in Montgomery form, so the
// single reduction of each sum gives the product in normal form; every operand is
// reduced below q)
template <int QT, int GT>
__global__ void __launch_bounds__(kMacThreads) k_mac(const uint64_t* __restrict__ T, const uint64_t* __restrict__ P,
                                                     uint64_t* __restrict__ acc, uint32_t Qn, uint32_t G,
                                                     uint32_t n_in, uint32_t lvl, DevTables tab, uint32_t log_n,
                                                     uint32_t n_qt, uint32_t n_gt) {
    const uint32_t n = 1u << log_n, l1 = lvl + 1;
    const MacTile t = mac_tile(n_qt, n_gt, n / kMacThreads, QT, GT, 1);
    pdl_wait();
    const uint32_t nq = min((uint32_t)QT, Qn - t.q0), ng = min((uint32_t)GT, G - t.g0);
    const uint64_t q = tab.q[t.j], qn = tab.qneg[t.j], q8 = 8 * q;
    const size_t ln = (size_t)l1 * n;                        // one polynomial at this level
    const size_t t_i = 2 * ln, t_q = (size_t)n_in * t_i;     // strides of T: part, query
    const size_t p_g = (size_t)n_in * ln;                    // stride of P: group (part: ln)
    const uint64_t* tp = T + (size_t)t.q0 * t_q + (size_t)t.j * n + t.p;
    const uint64_t* pp = P + (size_t)t.g0 * p_g + (size_t)t.j * n + t.p;
    // the words of U parts are loaded before their products (U by the tile's registers;
    // deeper prefetch of the 4 x 1 tile measured slower)
    constexpr int W = 2 * QT + GT, U = W * 4 <= 24 ? 4 : (W * 2 <= 12 ? 2 : 1);
    Acc60 a0[QT][GT], a1[QT][GT];
    for (uint32_t i0 = 0; i0 < n_in; i0 += kFold60Every) {
#pragma unroll
        for (int v0 = 0; v0 < kFold60Every; v0 += U) {
            uint64_t xr0[U][QT], xr1[U][QT], yr[U][GT];
#pragma unroll
            for (int v = 0; v < U; v++) {
                const uint32_t i = i0 + v0 + v;
                const bool ok = i < n_in;
#pragma unroll
                for (int k = 0; k < QT; k++) {
                    const uint64_t* r = tp + k * t_q + i * t_i;
                    xr0[v][k] = ok && (uint32_t)k < nq ? r[0] : 0;
                    xr1[v][k] = ok && (uint32_t)k < nq ? r[ln] : 0;
                }
#pragma unroll
                for (int h = 0; h < GT; h++) yr[v][h] = ok && (uint32_t)h < ng ? pp[h * p_g + i * ln] : 0;
            }
#pragma unroll
            for (int v = 0; v < U; v++) {
                if (i0 + v0 + v >= n_in) break;
                Piece30 x0[QT], x1[QT], y[GT];
#pragma unroll
                for (int k = 0; k < QT; k++) {
                    x0[k] = piece30(xr0[v][k]);
                    x1[k] = piece30(xr1[v][k]);
                }
#pragma unroll
                for (int h = 0; h < GT; h++) y[h] = piece30(yr[v][h]);
#pragma unroll
                for (int k = 0; k < QT; k++)
#pragma unroll
                    for (int h = 0; h < GT; h++) {
                        mul_add(a0[k][h], x0[k], y[h]);
                        mul_add(a1[k][h], x1[k], y[h]);
                    }
            }
        }
#pragma unroll
        for (int k = 0; k < QT; k++)
#pragma unroll
            for (int h = 0; h < GT; h++) {
                fold60(a0[k][h], q8);
                fold60(a1[k][h], q8);
            }
    }
#pragma unroll
    for (int k = 0; k < QT; k++)
#pragma unroll
        for (int h = 0; h < GT; h++) {
            if ((uint32_t)k >= nq || (uint32_t)h >= ng) continue;
            const size_t ob = ((size_t)(t.q0 + k) * G + t.g0 + h) * t_i + (size_t)t.j * n + t.p;
            acc[ob] = redc(a0[k][h], q, qn);
            acc[ob + ln] = redc(a1[k][h], q, qn);
        }
}

// HE-C^3 with an encrypted gallery: the tensor products of the expanded query
// parts T[q][i] with the gallery ciphertexts C[g][i] summed over the parts,
//   d0 = sum T0*C0,  d1 = sum T0*C1 + T1*C0,  d2 = sum T1*C1   (C in Montgomery form),
// written as A[q][g] = (d0, d2) -- the input of the relinearising key switch --
// and B[q][g] = (0, d1) -- its addend.  Tiles and block order as k_mac; d1 takes
// two products a part, so the sums are folded every kFold60Every / 2 parts.
template <int QT, int GT>
__global__ void __launch_bounds__(kMacThreads) k_mac_ct(const uint64_t* __restrict__ T, const uint64_t* __restrict__ C,
                                                        uint64_t* __restrict__ A, uint64_t* __restrict__ B,
                                                        uint32_t Qn, uint32_t G, uint32_t n_in, uint32_t lvl,
                                                        DevTables tab, uint32_t log_n, uint32_t n_qt, uint32_t n_gt) {
    const uint32_t n = 1u << log_n, l1 = lvl + 1;
    const MacTile t = mac_tile(n_qt, n_gt, n / kMacThreads, QT, GT, 1);
    pdl_wait();
    const uint32_t nq = min((uint32_t)QT, Qn - t.q0), ng = min((uint32_t)GT, G - t.g0);
    const uint64_t q = tab.q[t.j], qn = tab.qneg[t.j], q8 = 8 * q;
    const size_t ln = (size_t)l1 * n;
    const size_t t_i = 2 * ln, t_q = (size_t)n_in * t_i;     // strides of T and C: part; query / group
    const uint64_t* tp = T + (size_t)t.q0 * t_q + (size_t)t.j * n + t.p;
    const uint64_t* cp = C + (size_t)t.g0 * t_q + (size_t)t.j * n + t.p;
    Acc60 d0[QT][GT], d1[QT][GT], d2[QT][GT];
    for (uint32_t i0 = 0; i0 < n_in; i0 += kFold60Every / 2) {
        const uint32_t i1 = min(n_in, i0 + kFold60Every / 2);
        for (uint32_t i = i0; i < i1; i++) {
            Piece30 x0[QT], x1[QT], y0[GT], y1[GT];
#pragma unroll
            for (int k = 0; k < QT; k++) {
                const uint64_t* r = tp + k * t_q + i * t_i;
                x0[k] = piece30((uint32_t)k < nq ? r[0] : 0);
                x1[k] = piece30((uint32_t)k < nq ? r[ln] : 0);
            }
#pragma unroll
            for (int h = 0; h < GT; h++) {
                const uint64_t* r = cp + h * t_q + i * t_i;
                y0[h] = piece30((uint32_t)h < ng ? r[0] : 0);
                y1[h] = piece30((uint32_t)h < ng ? r[ln] : 0);
            }
#pragma unroll
            for (int k = 0; k < QT; k++)
#pragma unroll
                for (int h = 0; h < GT; h++) {
                    mul_add(d0[k][h], x0[k], y0[h]);
                    mul_add(d1[k][h], x0[k], y1[h]);
                    mul_add(d1[k][h], x1[k], y0[h]);
                    mul_add(d2[k][h], x1[k], y1[h]);
                }
        }
#pragma unroll
        for (int k = 0; k < QT; k++)
#pragma unroll
            for (int h = 0; h < GT; h++) {
                fold60(d0[k][h], q8);
                fold60(d1[k][h], q8);
                fold60(d2[k][h], q8);
            }
    }
#pragma unroll
    for (int k = 0; k < QT; k++)
#pragma unroll
        for (int h = 0; h < GT; h++) {
            if ((uint32_t)k >= nq || (uint32_t)h >= ng) continue;
            const size_t ob = ((size_t)(t.q0 + k) * G + t.g0 + h) * t_i + (size_t)t.j * n + t.p;
            A[ob] = redc(d0[k][h], q, qn);
            A[ob + ln] = redc(d2[k][h], q, qn);
            B[ob] = 0;
            B[ob + ln] = redc(d1[k][h], q, qn);
        }
}

// Algorithm 1 in hoisted form: t0[q][i] = sum_j R[q][j] * mask[(i - j) mod n_in] with
// R[q][j] = Rot(query q, j*part) given by pointer (R[q][0] the query itself),
// masks [n_in][l1][N] Montgomery, t0 [Q][n_in][2][l1][N], n_in a power of two.
// Grid (ceil(n_in / OC) * N / kMacThreads, l1, Q), output chunks fastest so that
// the passes over one coefficient range run together and share its rotated
// copies in L2: a thread computes OC outputs i of one query, limb and
// coefficient, reading each rotated query once per OC outputs.  The block
// stages the query's pointer list and, with SM, its words of every mask (split
// into 30-bit pieces; n_in * kMacThreads words of dynamic shared memory) --
// static gallery data, staged before the wait on the previous kernel.
template <int OC, bool SM>
__global__ void __launch_bounds__(kMacThreads) k_mac_circ(const uint64_t* const* R, const uint64_t* __restrict__ masks,
                                                          uint64_t* __restrict__ t0, uint32_t n_in, uint32_t lvl,
                                                          DevTables tab, uint32_t log_n) {
    extern __shared__ uint64_t sm_mask[];                       // [n_in][kMacThreads] (SM)
    __shared__ const uint64_t* sR[kMacThreads];
    const uint32_t n = 1u << log_n, l1 = lvl + 1, nm = n_in - 1;
    const uint32_t chunks = (n_in + OC - 1) / OC;
    const uint32_t i0 = (blockIdx.x % chunks) * OC;
    const uint32_t p = (blockIdx.x / chunks) * kMacThreads + threadIdx.x;   // < n: the grid covers N exactly
    const uint32_t j = blockIdx.y, qi = blockIdx.z;
    const size_t ln = (size_t)l1 * n;
    const uint64_t* mj = masks + (size_t)j * n + p;               // mask k at mj + k * ln
    if (SM)
        for (uint32_t k = 0; k < n_in; k++) sm_mask[k * kMacThreads + threadIdx.x] = pack30(mj[k * ln]);
    pdl_wait();
    const uint64_t q = tab.q[j], qn = tab.qneg[j], q8 = 8 * q;
    Acc60 s0[OC], s1[OC];
    for (uint32_t b0 = 0; b0 < n_in; b0 += kMacThreads) {
        const uint32_t nb = min(n_in - b0, (uint32_t)kMacThreads);
        __syncthreads();
        if (threadIdx.x < nb) sR[threadIdx.x] = R[(size_t)qi * n_in + b0 + threadIdx.x];
        __syncthreads();
        for (uint32_t u0 = 0; u0 < nb; u0 += kFold60Every) {
            uint64_t rv0[kFold60Every], rv1[kFold60Every];
#pragma unroll
            for (int v = 0; v < kFold60Every; v++) {
                if (u0 + v < nb) {
                    const uint64_t* r = sR[u0 + v] + (size_t)j * n + p;
                    rv0[v] = r[0];
                    rv1[v] = r[ln];
                }
            }
#pragma unroll
            for (int v = 0; v < kFold60Every; v++) {
                if (u0 + v >= nb) break;
                const uint32_t jj = b0 + u0 + v;
                const Piece30 r0 = piece30(rv0[v]), r1 = piece30(rv1[v]);
#pragma unroll
                for (int o = 0; o < OC; o++) {
                    if (i0 + o >= n_in) break;
                    const uint32_t k = (i0 + o - jj) & nm;
                    const Piece30 mk = SM ? unpack30(sm_mask[k * kMacThreads + threadIdx.x]) : piece30(mj[k * ln]);
                    mul_add(s0[o], r0, mk);
                    mul_add(s1[o], r1, mk);
                }
            }
#pragma unroll
            for (int o = 0; o < OC; o++) {
                fold60(s0[o], q8);
                fold60(s1[o], q8);
            }
        }
    }
#pragma unroll
    for (int o = 0; o < OC; o++) {
        const uint32_t i = i0 + o;
        if (i >= n_in) break;
        const size_t ob = ((size_t)qi * n_in + i) * 2 * ln + (size_t)j * n + p;
        t0[ob] = redc(s0[o], q, qn);
        t0[ob + ln] = redc(s1[o], q, qn);
    }
}

// The last rescale of the match in the coefficient domain: in[b] a level-1 ciphertext
// [2][2][N] in coefficient form, out[b] its rescale [2][N] at level 0:
// out = (c_0 - [c_1]_centred) * q_1^-1 mod q_0 -- the residues of the NTT-domain
// rescale followed by the inverse NTT.  Grid (B * 2, chunks of a limb).
__global__ void k_rescale_coef(uint64_t* const* in, uint64_t* const* out, uint64_t q0, uint64_t q1, ulonglong2 q1inv,
                               uint32_t n) {
    const uint32_t b = blockIdx.x / 2, comp = blockIdx.x % 2;
    pdl_wait();
    const uint64_t* c = in[b] + (size_t)comp * 2 * n;
    uint64_t* o = out[b] + (size_t)comp * n;
    const uint64_t half = q1 >> 1;
    for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x) {
        const uint64_t r = c[n + i];                              // [0, q_1), q_1 < q_0
        const uint64_t lift = r > half ? q0 - (q1 - r) : r;       // the centred representative mod q_0
        o[i] = shoup(subm(c[i], lift, q0), q1inv.x, q1inv.y, q0);
    }
}

// E0[q] = P * query q in the extended basis Q_L u P: the q-limbs times P (Montgomery
// product with P * 2^64), the special limbs 0.  in[q]: [2][L+1][N] NTT form; E0
// [Q][2][nlx][N].  Grid (Q * 2 * nlx, chunks of a limb).
__global__ void k_lift_p(const uint64_t* const* in, uint64_t* __restrict__ E0, const KsLevelConst* __restrict__ kc,
                         DevTables tab, uint32_t l1, uint32_t nlx, uint32_t n, size_t stride) {
    const uint32_t y = blockIdx.x, b = y / (2 * nlx), comp = (y / nlx) % 2, jj = y % nlx;
    pdl_wait();
    uint64_t* o = E0 + (size_t)b * stride + ((size_t)comp * nlx + jj) * n;
    if (jj >= l1) {
        for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x) o[i] = 0;
        return;
    }
    const uint64_t q = tab.q[jj], qn = tab.qneg[jj], pm = kc->pmont[jj];
    const uint64_t* a = in[b] + ((size_t)comp * l1 + jj) * n;
    for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x)
        o[i] = mont(a[i], pm, q, qn);
}

// The residues of integer coefficients x on the special primes, from their q_0
// residue v (coefficient form): the centred x = v or v - q_0 (|x| < q_0 / 2 and
// below every special prime), out[k][i] = x mod p_k.  Grid (alpha, chunks).
__global__ void k_centred_to_p(const uint64_t* __restrict__ v0, uint64_t* __restrict__ out, size_t out_stride,
                               uint64_t q0, uint32_t first, DevTables tab, uint32_t n) {
    const uint32_t k = blockIdx.x;
    const uint64_t p = tab.q[first + k], half = q0 / 2;
    uint64_t* o = out + (size_t)k * out_stride;
    for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x) {
        const uint64_t v = v0[i];
        o[i] = v <= half ? v : p - (q0 - v);
    }
}

// ---------------------------------------------------------------------------
// Algorithm 1's hoisted sum as a cyclic convolution over the parts.  For one
// coefficient of one limb, t0[i] = sum_j R[j] * M[(i - j) mod n] is the length-n
// cyclic convolution of the rotated copies with the masks.  With w a primitive
// n-th root of unity mod q (n divides q - 1: every prime is 1 mod 2N) it equals
// DIT_{w^-1}(DIF_w(R) * DIF_w(M) / n): Gentleman-Sande forward (natural order in,
// bit-reversed out), the products in that order, Cooley-Tukey inverse
// (bit-reversed in, natural out).  The masks' side DIF_w(M) / n is computed once
// per gallery (k_circ_prep, kept in Montgomery form); the result has the same
// residues as the direct sum, for (n/2) log2 n butterflies a side -- those with
// twiddle 1 without a product -- and n products instead of n^2.
// Twiddle table per limb j: [j][e] = w^e for e < n/2, then [j][n/2 + e] = w^-e (Shoup pairs).
// ---------------------------------------------------------------------------
template <int NIN>
__device__ __forceinline__ void circ_dif(uint64_t (&x)[NIN], const ulonglong2* fw, uint64_t q) {
#pragma unroll
    for (int len = NIN / 2; len >= 1; len >>= 1)
#pragma unroll
        for (int st = 0; st < NIN; st += 2 * len)
#pragma unroll
            for (int k = 0; k < len; k++) {
                const uint64_t u = x[st + k], v = x[st + k + len];
                x[st + k] = addm(u, v, q);
                const uint64_t d = subm(u, v, q);
                if (k == 0) {
                    x[st + k + len] = d;
                } else {
                    const ulonglong2 w = fw[k * (NIN / (2 * len))];
                    x[st + k + len] = shoup(d, w.x, w.y, q);
                }
            }
}
template <int NIN>
__device__ __forceinline__ void circ_dit(uint64_t (&x)[NIN], const ulonglong2* iw, uint64_t q) {
#pragma unroll
    for (int len = 1; len < NIN; len <<= 1)
#pragma unroll
        for (int st = 0; st < NIN; st += 2 * len)
#pragma unroll
            for (int k = 0; k < len; k++) {
                const uint64_t u = x[st + k];
                uint64_t v = x[st + k + len];
                if (k != 0) {
                    const ulonglong2 w = iw[k * (NIN / (2 * len))];
                    v = shoup(v, w.x, w.y, q);
                }
                x[st + k] = addm(u, v, q);
                x[st + k + len] = subm(u, v, q);
            }
}

struct CircNinv {
    ulonglong2 v[MAXB];   // n^-1 mod q_j (Shoup pairs)
};

// hat[k][j][p] = (DIF_w(masks[.][j][p]))[k] / n; the masks are in Montgomery form
// and so is hat.  Grid (N / kMacThreads, l1).
template <int NIN>
__global__ void __launch_bounds__(kMacThreads) k_circ_prep(const uint64_t* __restrict__ masks,
                                                           uint64_t* __restrict__ hat,
                                                           const ulonglong2* __restrict__ tw, CircNinv ninv,
                                                           uint32_t l1, DevTables tab, uint32_t log_n) {
    __shared__ ulonglong2 stw[NIN];
    const uint32_t n = 1u << log_n, j = blockIdx.y, p = blockIdx.x * kMacThreads + threadIdx.x;
    const size_t ln = (size_t)l1 * n;
    if (threadIdx.x < NIN) stw[threadIdx.x] = tw[(size_t)j * NIN + threadIdx.x];
    __syncthreads();
    const uint64_t q = tab.q[j];
    uint64_t x[NIN];
#pragma unroll
    for (int k = 0; k < NIN; k++) x[k] = masks[k * ln + (size_t)j * n + p];
    circ_dif<NIN>(x, stw, q);
    const ulonglong2 ni = ninv.v[j];
#pragma unroll
    for (int k = 0; k < NIN; k++) hat[k * ln + (size_t)j * n + p] = shoup(x[k], ni.x, ni.y, q);
}

// t0[q][i][c][j][p] = sum_jj R[q][jj][c][j][p] * mask[(i - jj) mod NIN][j][p], by the
// convolution above.  Grid (2 * N / kMacThreads, l1, Q): a thread takes one
// coefficient of one component of one limb of one query (component fastest).
template <int NIN>
__global__ void __launch_bounds__(kMacThreads) k_mac_circ_ntt(const uint64_t* const* R,
                                                              const uint64_t* __restrict__ hat,
                                                              const ulonglong2* __restrict__ tw,
                                                              uint64_t* __restrict__ t0, uint32_t lvl, DevTables tab,
                                                              uint32_t log_n) {
    __shared__ ulonglong2 stw[NIN];
    __shared__ const uint64_t* sR[NIN];
    const uint32_t n = 1u << log_n, l1 = lvl + 1;
    const uint32_t c = blockIdx.x & 1, p = (blockIdx.x >> 1) * kMacThreads + threadIdx.x;
    const uint32_t j = blockIdx.y, qi = blockIdx.z;
    const size_t ln = (size_t)l1 * n;
    if (threadIdx.x < NIN) stw[threadIdx.x] = tw[(size_t)j * NIN + threadIdx.x];   // gallery data: before the wait
    pdl_wait();
    if (threadIdx.x < NIN) sR[threadIdx.x] = R[(size_t)qi * NIN + threadIdx.x];
    __syncthreads();
    const uint64_t q = tab.q[j], qn = tab.qneg[j];
    const size_t off = (size_t)c * ln + (size_t)j * n + p;
    uint64_t x[NIN];
#pragma unroll
    for (int k = 0; k < NIN; k++) x[k] = sR[k][off];
    circ_dif<NIN>(x, stw, q);
    const uint64_t* h = hat + (size_t)j * n + p;
#pragma unroll
    for (int k = 0; k < NIN; k++) x[k] = mont(x[k], h[k * ln], q, qn);
    circ_dit<NIN>(x, stw + NIN / 2, q);
    uint64_t* o = t0 + (size_t)qi * NIN * 2 * ln + off;
#pragma unroll
    for (int i = 0; i < NIN; i++) o[(size_t)i * 2 * ln] = x[i];
}

// dst[t] += sum of src[k], k in [off[t], off[t+1]): ciphertexts [2][l1][N] at one
// level; grid (targets * 2 * l1, chunks of a limb)
__global__ void k_accumulate(uint64_t* const* dst, const uint64_t* const* src, const uint64_t* off, uint32_t l1,
                             DevTables tab, uint32_t n) {
    const uint32_t t = blockIdx.x / (2 * l1), r = blockIdx.x % (2 * l1), j = r % l1;
    const uint64_t q = tab.q[j];
    pdl_wait();
    uint64_t* d = dst[t] + (size_t)r * n;
    const uint64_t k0 = off[t], k1 = off[t + 1];
    for (uint32_t i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x) {
        uint64_t acc = d[i];
        for (uint64_t k = k0; k < k1; k++) acc = addm(acc, src[k][(size_t)r * n + i], q);
        d[i] = acc;
    }
}


}  // namespace

// ===========================================================================
// launchers
// ===========================================================================

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("BM_PDL");
        return !e || std::atoi(e) != 0;
    }();
    return on;
}

cudaError_t ntt_forward(const Context& c, const LimbBatch& b, cudaStream_t s) { return ntt_dispatch(c, b, false, s); }

cudaError_t ntt_col_inverse(const Context& c, const LimbBatch& b, cudaStream_t s) {
    const uint32_t limbs = b.n_polys * b.nl;
    if (limbs == 0) return cudaSuccess;
    const double lw = 16.0 * c.n * limbs, ops = 16.0 * (c.n / 2) * (c.log_n / 2) * limbs;
    ProfScope ps(BM_KERNEL_NTT, s, lw, ops);
    if (c.log_n == 16) pdl_launch(nttr::k_col_inv<8, 8, 2, 2>, dim3(limbs, 256 / 2), 2 * 64, 0, s, b, c.tab);
    else if (c.log_n == 12) pdl_launch(nttr::k_col_inv<6, 6, 2, 8>, dim3(limbs, 64 / 8), 8 * 16, 0, s, b, c.tab);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t build_ks_constants(Context& c) {
    auto pair = [](uint64_t w, uint64_t q) { return make_ulonglong2(w % q, h_shoup_companion(w % q, q)); };
    c.h_ksc.assign(c.L + 1, KsLevelConst{});
    for (uint32_t l = 0; l <= c.L; l++) {
        KsLevelConst& K = c.h_ksc[l];
        const uint32_t l1 = l + 1, nlx = l1 + c.alpha;
        K.nlx = nlx;
        auto xprime = [&](uint32_t jj) { return c.primes[jj < l1 ? jj : c.L + 1 + (jj - l1)]; };
        uint32_t nd = 0;
        for (const auto& dg : c.digits) {
            if (dg.empty() || dg[0] > l) continue;
            uint32_t ds = 0;
            for (uint32_t x : dg) ds += (x <= l);
            K.dstart[nd] = dg[0];
            K.dsz[nd] = ds;
            for (uint32_t i = 0; i < ds; i++) {
                const uint64_t qi = c.primes[dg[0] + i];
                uint64_t hat = 1;
                for (uint32_t k = 0; k < ds; k++)
                    if (k != i) hat = h_mulmod(hat, c.primes[dg[0] + k] % qi, qi);
                K.up_hinv[nd][i] = pair(h_invmod(hat, qi), qi);
                for (uint32_t jj = 0; jj < nlx; jj++) {
                    const uint64_t t = xprime(jj);
                    uint64_t ht = 1;
                    for (uint32_t k = 0; k < ds; k++)
                        if (k != i) ht = h_mulmod(ht, c.primes[dg[0] + k] % t, t);
                    K.up_hat[nd][i][jj] = pair(ht, t);
                }
            }
            nd++;
        }
        K.nd = nd;
        for (uint32_t i = 0; i < c.alpha; i++) {
            const uint64_t pi = c.primes[c.L + 1 + i];
            uint64_t hat = 1;
            for (uint32_t k = 0; k < c.alpha; k++)
                if (k != i) hat = h_mulmod(hat, c.primes[c.L + 1 + k] % pi, pi);
            const uint64_t w = h_mulmod(h_invmod(hat, pi), h_invmod(c.n % pi, pi), pi);
            K.dn_hinv[i] = pair(w, pi);
            for (uint32_t j = 0; j < l1; j++) {
                const uint64_t t = c.primes[j];
                uint64_t ht = 1;
                for (uint32_t k = 0; k < c.alpha; k++)
                    if (k != i) ht = h_mulmod(ht, c.primes[c.L + 1 + k] % t, t);
                K.dn_hat[i][j] = pair(ht, t);
            }
        }
        for (uint32_t j = 0; j < l1; j++) {
            K.pinv[j] = pair(h_invmod(c.P_mod[j], c.primes[j]), c.primes[j]);
            K.pmont[j] = (uint64_t)(((unsigned __int128)c.P_mod[j] << 64) % c.primes[j]);
        }
    }
    cudaError_t e = cudaMalloc(&c.d_ksc, sizeof(KsLevelConst) * c.h_ksc.size());
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(c.d_ksc, c.h_ksc.data(), sizeof(KsLevelConst) * c.h_ksc.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    // ModDown and Rescale fused at the top level, dropping d = 1 or 2 q-primes: special
    // set S = {q_(L-d+1), .., q_L} u P (primes L-d+1 .. L+alpha, contiguous in the
    // basis), targets q_0..q_(L-d); the F5 / F6 fields with S in place of P
    for (uint32_t d = 1; d <= (uint32_t)kMdrDrops; d++) {
        KsLevelConst M{};
        const uint32_t L = c.L, ns = c.alpha + d, nt = L + 1 - d, s0 = nt;
        if (ns > (uint32_t)MAXSP || L < d) break;
        M.nlx = L + 1 + c.alpha;
        for (uint32_t i = 0; i < ns; i++) {
            const uint64_t si = c.primes[s0 + i];
            uint64_t hat = 1;                                     // (S / s_i) mod s_i
            for (uint32_t k = 0; k < ns; k++)
                if (k != i) hat = h_mulmod(hat, c.primes[s0 + k] % si, si);
            M.dn_hinv[i] = pair(h_mulmod(h_invmod(hat, si), h_invmod(c.n % si, si), si), si);
            for (uint32_t j = 0; j < nt; j++) {
                const uint64_t t = c.primes[j];
                uint64_t ht = 1;
                for (uint32_t k = 0; k < ns; k++)
                    if (k != i) ht = h_mulmod(ht, c.primes[s0 + k] % t, t);
                M.dn_hat[i][j] = pair(ht, t);
            }
        }
        for (uint32_t j = 0; j < nt; j++) {
            const uint64_t t = c.primes[j];
            uint64_t smod = c.P_mod[j];                           // S mod q_j
            for (uint32_t k = 0; k < d; k++) smod = h_mulmod(smod, c.primes[s0 + k] % t, t);
            M.pinv[j] = pair(h_invmod(smod, t), t);
        }
        c.h_ksc_mdr[d - 1] = M;
    }
    if (c.L >= 1 && c.alpha + 1 <= (uint32_t)BM_MAX_P) {
        e = cudaMalloc(&c.d_ksc_mdr, sizeof(KsLevelConst) * kMdrDrops);
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(c.d_ksc_mdr, c.h_ksc_mdr, sizeof(KsLevelConst) * kMdrDrops, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    std::vector<ulonglong2> qi((size_t)(c.L + 1) * MAXB, make_ulonglong2(0, 0));
    for (uint32_t l = 1; l <= c.L; l++)
        for (uint32_t j = 0; j < l; j++) qi[(size_t)l * MAXB + j] = pair(h_invmod(c.primes[l] % c.primes[j], c.primes[j]), c.primes[j]);
    e = cudaMalloc(&c.d_qlinv, sizeof(ulonglong2) * qi.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(c.d_qlinv, qi.data(), sizeof(ulonglong2) * qi.size(), cudaMemcpyHostToDevice);
}
cudaError_t ntt_inverse(const Context& c, const LimbBatch& b, cudaStream_t s) { return ntt_dispatch(c, b, true, s); }

cudaError_t to_montgomery(const Context& c, const LimbBatch& b, bool inverse, cudaStream_t s) {
    const uint32_t limbs = b.n_polys * b.nl;
    if (!limbs) return cudaSuccess;
    const dim3 g(limbs, c.n / kThreads / 4);
    ProfScope ps(BM_KERNEL_OTHER, s, 16.0 * c.n * limbs);
    if (inverse) k_from_mont<<<g, kThreads, 0, s>>>(b, c.tab, c.n);
    else k_to_mont<<<g, kThreads, 0, s>>>(b, c.tab, c.n);
    return cudaGetLastError();
}

cudaError_t lift_signed(const Context& c, const int64_t* d_v, const LimbBatch& out, cudaStream_t s) {
    const uint32_t limbs = out.n_polys * out.nl;
    ProfScope ps(BM_KERNEL_OTHER, s, 8.0 * c.n * (limbs + 1));
    k_lift_signed<<<dim3(limbs, c.n / kThreads / 4), kThreads, 0, s>>>(d_v, out, c.tab, c.n);
    return cudaGetLastError();
}

cudaError_t pointwise_mul(const Context& c, const LimbBatch& a, const LimbBatch& b, const LimbBatch& out,
                          cudaStream_t s) {
    ProfScope ps(BM_KERNEL_OTHER, s, 24.0 * c.n * a.n_polys * a.nl);
    k_pointwise<<<dim3(a.n_polys * a.nl, c.n / kThreads / 4), kThreads, 0, s>>>(a, b, out, c.tab, c.n, 0);
    return cudaGetLastError();
}

cudaError_t pointwise_addsub(const Context& c, const LimbBatch& a, const LimbBatch& b, const LimbBatch& out,
                             bool sub, cudaStream_t s) {
    ProfScope ps(BM_KERNEL_OTHER, s, 24.0 * c.n * a.n_polys * a.nl);
    k_pointwise<<<dim3(a.n_polys * a.nl, c.n / kThreads / 4), kThreads, 0, s>>>(a, b, out, c.tab, c.n,
                                                                                 sub ? 2 : 1);
    return cudaGetLastError();
}

cudaError_t permute_ntt(const Context& c, const LimbBatch& in, const LimbBatch& out, uint64_t galois,
                        cudaStream_t s) {
    ProfScope ps(BM_KERNEL_OTHER, s, 16.0 * c.n * in.n_polys * in.nl);
    k_permute<<<dim3(in.n_polys * in.nl, c.n / kThreads / 4), kThreads, 0, s>>>(in, out, c.log_n, galois);
    return cudaGetLastError();
}

cudaError_t scalar_mul(const Context& c, const LimbBatch& in, const uint64_t* cst, const LimbBatch& out,
                       cudaStream_t s) {
    ScalarK sk{};
    for (uint32_t k = 0; k < in.nl; k++) {
        const uint64_t q = c.primes[in.prime(k)];
        sk.w[k] = cst[k] % q;
        sk.wsh[k] = h_shoup_companion(sk.w[k], q);
    }
    ProfScope ps(BM_KERNEL_OTHER, s, 16.0 * c.n * in.n_polys * in.nl);
    k_scalar<<<dim3(in.n_polys * in.nl, c.n / kThreads / 4), kThreads, 0, s>>>(in, out, sk, c.tab, c.n);
    return cudaGetLastError();
}

// ---- key switching ----

size_t ks_scratch_words(const Context& c, uint32_t level, uint32_t B) {
    const size_t n = c.n, l1 = level + 1, nlx = l1 + c.alpha;
    size_t nd = 0;
    for (auto& d : c.digits) nd += (!d.empty() && d[0] <= level);
    return (size_t)B * n * (2 * l1 + nd * nlx + 2 * nlx + 2 * l1);
}

cudaError_t ks_rotate(const Context& c, const uint64_t* key, uint64_t galois, uint32_t level, uint32_t B,
                      uint64_t* const* d_in, uint64_t* const* d_out, uint64_t* const* d_add, uint64_t* scratch,
                      cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    // every context the library creates is one the fused kernels cover (context_shape)
    if (!ks_fused_supported(c)) return cudaErrorInvalidValue;
    return ks_rotate_fused(c, key, galois, level, B, d_in, d_out, d_add, scratch, s);
}

// ---- rescale ----

size_t rescale_scratch_words(const Context& c, uint32_t level, uint32_t B) {
    return (size_t)B * 2 * c.n * (1 + level);
}

cudaError_t rescale(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in, uint64_t* const* d_out,
                    uint64_t* scratch, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    if (!ks_fused_supported(c)) return cudaErrorInvalidValue;
    return rescale_fused(c, level, B, d_in, d_out, scratch, s);
}

cudaError_t mul_plain(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in,
                      const uint64_t* const* d_pt, uint64_t* const* d_out, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ProfScope ps(BM_KERNEL_MUL_PLAIN, s, 8.0 * c.n * B * (level + 1) * 5);
    pdl_launch(k_mul_plain, dim3(B * 2 * (level + 1), c.n / kThreads / 4), kThreads, 0, s, d_in, d_pt, d_out, level, c.tab,
                                                                                   c.n);
    return cudaGetLastError();
}

// Tile of the HE-C^3 products for measurements: BM_MAC_TILE="QxG" (each 1, 2 or 4)
// sets the queries and groups a thread takes (at most 4 pairs for the ct x ct form),
// in place of the default choice.
static void mac_tile_env(int& qt, int& gt, int max_pairs) {
    static const int env = [] {
        int a = 0, b = 0;
        if (const char* e = std::getenv("BM_MAC_TILE"))
            if (std::sscanf(e, "%dx%d", &a, &b) != 2) a = b = 0;
        auto pow2 = [](int v) { return v >= 4 ? 4 : (v >= 2 ? 2 : 1); };
        return a > 0 && b > 0 ? pow2(a) * 8 + pow2(b) : 0;
    }();
    if (!env) return;
    qt = env / 8;
    gt = env % 8;
    while (qt * gt > max_pairs) (gt > 1 ? gt : qt) /= 2;
}

// tile shape of the HE-C^3 products: up to 4 queries and 4 (ct x pt) or 2
// (ct x ct) groups a thread; blocks = tiles x chunks x limbs
static bool mac_grid(const Context& c, uint32_t level, uint32_t Q, uint32_t G, int QT, int GT, uint32_t n_c,
                     uint32_t& n_qt, uint32_t& n_gt, uint32_t& blocks) {
    n_qt = (Q + QT - 1) / QT;
    n_gt = (G + GT - 1) / GT;
    const uint64_t b = (uint64_t)n_c * n_qt * n_gt * (c.n / kMacThreads) * (level + 1);
    blocks = (uint32_t)b;
    return b > 0 && b <= 0x7fffffffull;
}

template <int QT, int GT>
static cudaError_t launch_mac(const Context& c, uint32_t level, uint32_t Q, uint32_t G, uint32_t n_in,
                              const uint64_t* T, const uint64_t* P, uint64_t* acc, cudaStream_t s) {
    uint32_t n_qt, n_gt, blocks;
    if (!mac_grid(c, level, Q, G, QT, GT, 1, n_qt, n_gt, blocks)) return cudaErrorInvalidConfiguration;
    return pdl_launch(k_mac<QT, GT>, dim3(blocks), kMacThreads, 0, s, T, P, acc, Q, G, n_in, level, c.tab, c.log_n,
                      n_qt, n_gt);
}

template <int QT, int GT>
static cudaError_t launch_mac_ct(const Context& c, uint32_t level, uint32_t Q, uint32_t G, uint32_t n_in,
                                 const uint64_t* T, const uint64_t* C, uint64_t* A, uint64_t* B, cudaStream_t s) {
    uint32_t n_qt, n_gt, blocks;
    if (!mac_grid(c, level, Q, G, QT, GT, 1, n_qt, n_gt, blocks)) return cudaErrorInvalidConfiguration;
    return pdl_launch(k_mac_ct<QT, GT>, dim3(blocks), kMacThreads, 0, s, T, C, A, B, Q, G, n_in, level, c.tab,
                      c.log_n, n_qt, n_gt);
}

cudaError_t mac(const Context& c, uint32_t level, uint32_t Q, uint32_t G, uint32_t n_in, const uint64_t* T,
                const uint64_t* P, uint64_t* acc, cudaStream_t s) {
    if (!Q || !G) return cudaSuccess;
    const double lim = (double)c.n * (level + 1);   // coefficients of a polynomial at this level
    ProfScope ps(BM_KERNEL_MAC, s, 8.0 * lim * ((double)Q * n_in * 2 + (double)G * n_in + 2.0 * Q * G),
                 lim * 2.0 * Q * G * (kProdMul * n_in + kRedcMul));
    // (query, group) sums of both components a thread, six registers each: a tile of 4
    // queries x 1 group with many queries (measured best on the batched workloads:
    // the group tiles re-read the query words from L2), else up to 2 x 2 / 1 x 4
    int qt = Q >= 4 ? 4 : (Q >= 2 ? 2 : 1);
    int gt = qt == 4 ? 1 : (qt == 2 ? (G >= 2 ? 2 : 1) : (G >= 3 ? 4 : (G == 2 ? 2 : 1)));
    mac_tile_env(qt, gt, 8);
    switch (qt * 8 + gt) {
        case 4 * 8 + 4:
        case 4 * 8 + 2: return launch_mac<4, 2>(c, level, Q, G, n_in, T, P, acc, s);
        case 4 * 8 + 1: return launch_mac<4, 1>(c, level, Q, G, n_in, T, P, acc, s);
        case 2 * 8 + 4: return launch_mac<2, 4>(c, level, Q, G, n_in, T, P, acc, s);
        case 2 * 8 + 2: return launch_mac<2, 2>(c, level, Q, G, n_in, T, P, acc, s);
        case 2 * 8 + 1: return launch_mac<2, 1>(c, level, Q, G, n_in, T, P, acc, s);
        case 1 * 8 + 4: return launch_mac<1, 4>(c, level, Q, G, n_in, T, P, acc, s);
        case 1 * 8 + 2: return launch_mac<1, 2>(c, level, Q, G, n_in, T, P, acc, s);
        default: return launch_mac<1, 1>(c, level, Q, G, n_in, T, P, acc, s);
    }
}

cudaError_t mac_ct(const Context& c, uint32_t level, uint32_t Q, uint32_t G, uint32_t n_in, const uint64_t* T,
                   const uint64_t* C, uint64_t* A, uint64_t* B, cudaStream_t s) {
    if (!Q || !G) return cudaSuccess;
    const double lim = (double)c.n * (level + 1);
    ProfScope ps(BM_KERNEL_MAC, s, 8.0 * lim * ((double)Q * n_in * 2 + 2.0 * G * n_in + 4.0 * Q * G),
                 lim * (double)Q * G * (4.0 * kProdMul * n_in + 3.0 * kRedcMul));
    // at most 4 (query, group) triples of sums a thread
    int qt = Q >= 4 ? 4 : (Q >= 2 ? 2 : 1), gt = G >= 2 && qt < 4 ? 2 : 1;
    mac_tile_env(qt, gt, 4);
    switch (qt * 8 + gt) {
        case 4 * 8 + 2:
        case 4 * 8 + 1: return launch_mac_ct<4, 1>(c, level, Q, G, n_in, T, C, A, B, s);
        case 2 * 8 + 2: return launch_mac_ct<2, 2>(c, level, Q, G, n_in, T, C, A, B, s);
        case 2 * 8 + 1: return launch_mac_ct<2, 1>(c, level, Q, G, n_in, T, C, A, B, s);
        case 1 * 8 + 2: return launch_mac_ct<1, 2>(c, level, Q, G, n_in, T, C, A, B, s);
        default: return launch_mac_ct<1, 1>(c, level, Q, G, n_in, T, C, A, B, s);
    }
}

cudaError_t accumulate(const Context& c, uint32_t level, uint32_t n_targets, uint64_t* const* dst,
                       const uint64_t* const* src, const uint64_t* off, uint32_t n_src, cudaStream_t s) {
    if (!n_targets) return cudaSuccess;
    ProfScope ps(BM_KERNEL_OTHER, s, 16.0 * c.n * (level + 1) * (n_targets + n_src));
    return pdl_launch(k_accumulate, dim3(n_targets * 2 * (level + 1), c.n / kThreads / 4), kThreads, 0, s, dst, src,
                      off, level + 1, c.tab, c.n);
}

// non-trivial twiddle products of one length-n transform (butterflies with k > 0)
static double circ_products(uint32_t n) {
    double t = 0;
    for (uint32_t len = n / 2; len >= 1; len >>= 1) t += (double)(n / (2 * len)) * (len - 1);
    return t;
}

template <int NIN>
static cudaError_t launch_circ_ntt(const Context& c, uint32_t level, uint32_t Q, const uint64_t* const* R,
                                   const uint64_t* hat, const ulonglong2* tw, uint64_t* t0, cudaStream_t s) {
    return pdl_launch(k_mac_circ_ntt<NIN>, dim3(2 * (c.n / kMacThreads), level + 1, Q), kMacThreads, 0, s, R, hat, tw,
                      t0, level, c.tab, c.log_n);
}

cudaError_t mac_circ(const Context& c, uint32_t level, uint32_t Q, uint32_t n_in, const uint64_t* const* R,
                     const uint64_t* masks, const uint64_t* hat, const ulonglong2* tw, uint64_t* t0,
                     cudaStream_t s) {
    constexpr int OC = 8;
    if (!Q) return cudaSuccess;
    if (Q > 65535) return cudaErrorInvalidConfiguration;
    const double lim = (double)c.n * (level + 1);
    if (hat && tw && n_in >= 2 && n_in <= kMaxCircParts) {
        // two transforms of n_in words and n_in Montgomery products per coefficient,
        // component and query
        ProfScope ps(BM_KERNEL_MAC, s, 8.0 * lim * ((double)Q * n_in * 2 + (double)n_in + 2.0 * Q * n_in),
                     lim * 2.0 * Q * (2.0 * kShoupMul * circ_products(n_in) + (kProdMul + kRedcMul) * n_in));
        switch (n_in) {
            case 2: return launch_circ_ntt<2>(c, level, Q, R, hat, tw, t0, s);
            case 4: return launch_circ_ntt<4>(c, level, Q, R, hat, tw, t0, s);
            case 8: return launch_circ_ntt<8>(c, level, Q, R, hat, tw, t0, s);
            case 16: return launch_circ_ntt<16>(c, level, Q, R, hat, tw, t0, s);
            default: return launch_circ_ntt<32>(c, level, Q, R, hat, tw, t0, s);
        }
    }
    const dim3 g((c.n / kMacThreads) * ((n_in + OC - 1) / OC), level + 1, Q);
    // masks in shared memory up to 64 parts (64 KiB a block)
    constexpr uint32_t kMaxSmParts = 64;
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_mac_circ<OC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(kMaxSmParts * kMacThreads * 8)) == cudaSuccess;
    }();
    ProfScope ps(BM_KERNEL_MAC, s, 8.0 * lim * ((double)Q * n_in * 2 + (double)n_in + 2.0 * Q * n_in),
                 lim * 2.0 * Q * n_in * (kProdMul * n_in + kRedcMul));
    if (attr && n_in <= kMaxSmParts)
        pdl_launch(k_mac_circ<OC, true>, g, kMacThreads, (size_t)n_in * kMacThreads * 8, s, R, masks, t0, n_in, level,
                   c.tab, c.log_n);
    else
        pdl_launch(k_mac_circ<OC, false>, g, kMacThreads, 0, s, R, masks, t0, n_in, level, c.tab, c.log_n);
    return cudaGetLastError();
}

// q_1 < q_0 follows from the bit sizes (a b-bit prime lies in [2^(b-1), 2^b)); the
// host-only plan estimate has the sizes but no primes
bool rescale_coef_supported(const Context& c) { return c.L >= 1 && c.params.q_bits[1] < c.params.q_bits[0]; }

cudaError_t rescale_coef(const Context& c, uint32_t B, uint64_t* const* in, uint64_t* const* out, cudaStream_t s) {
    if (!B) return cudaSuccess;
    if (!rescale_coef_supported(c)) return cudaErrorInvalidValue;
    const uint64_t q0 = c.primes[0], q1 = c.primes[1];
    const uint64_t inv = h_invmod(q1 % q0, q0);
    ProfScope ps(BM_KERNEL_RESCALE, s, 8.0 * c.n * B * 2 * 3, 16.0 * c.n * B * 2);
    return pdl_launch(k_rescale_coef, dim3(B * 2, c.n / kThreads / 4), kThreads, 0, s, in, out, q0, q1,
                      make_ulonglong2(inv, h_shoup_companion(inv, q0)), (uint32_t)c.n);
}

cudaError_t lift_p(const Context& c, uint32_t Q, uint64_t* const* in, uint64_t* E0, cudaStream_t s, size_t stride) {
    if (!Q) return cudaSuccess;
    const uint32_t l1 = c.L + 1, nlx = l1 + c.alpha;
    if (!stride) stride = (size_t)2 * nlx * c.n;
    ProfScope ps(BM_KERNEL_OTHER, s, 8.0 * c.n * Q * 2 * (l1 + nlx), 20.0 * c.n * Q * 2 * l1);
    return pdl_launch(k_lift_p, dim3(Q * 2 * nlx, c.n / kThreads / 4), kThreads, 0, s, (const uint64_t* const*)in, E0,
                      c.d_ksc + c.L, c.tab, l1, nlx, c.n, stride);
}

// fold [groups][n_in][nlx][N]: grid (groups * n_in * nlx, N / (kThreads * 2)); each thread
// two words of one limb of one (group, part j), the sum over the parts i of the
// Montgomery products mask_((i-j) mod n_in) * pts_i, accumulated at 128 bits
__global__ void k_fold_gallery(const uint64_t* __restrict__ masks, const uint64_t* __restrict__ pts,
                               uint64_t* __restrict__ fold, DevTables tab, uint32_t n_in, uint32_t nlx, uint32_t n) {
    const uint32_t y = blockIdx.x, jj = y % nlx, j = (y / nlx) % n_in, g = y / nlx / n_in;
    const uint64_t q = tab.q[jj], qn = tab.qneg[jj];   // limb jj of Q_L u P: prime jj of the basis
    const uint64_t* P = pts + (size_t)g * n_in * nlx * n + (size_t)jj * n;
    for (uint32_t w = blockIdx.y * blockDim.x + threadIdx.x; w < n; w += gridDim.y * blockDim.x) {
        Acc128 a;
        for (uint32_t i = 0; i < n_in; i++) {
            const uint32_t mi = (i + n_in - j) % n_in;
            mul_acc(a, masks[((size_t)mi * nlx + jj) * n + w], P[(size_t)i * nlx * n + w], q);
        }
        fold[(((size_t)g * n_in + j) * nlx + jj) * n + w] = redc(a, q, qn);
    }
}

cudaError_t fold_gallery(const Context& c, size_t groups, uint32_t n_in, const uint64_t* masks_ext,
                         const uint64_t* pts, uint64_t* fold, cudaStream_t s) {
    const uint32_t nlx = c.L + 1 + c.alpha;
    // grid x over (group, part, limb) in chunks below the launch limit
    const size_t per = (size_t)n_in * nlx, max_x = (size_t)1 << 30;
    for (size_t g0 = 0; g0 < groups; g0 += max_x / per) {
        const size_t gn = std::min(groups - g0, max_x / per);
        k_fold_gallery<<<dim3((uint32_t)(gn * per), c.n / kThreads / 2), kThreads, 0, s>>>(
            masks_ext, pts + g0 * per * c.n, fold + g0 * per * c.n, c.tab, n_in, nlx, c.n);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(s);
}

// out [count][nlx][N]: the l_in limbs of in copied, limbs l_in..nlx-1 (the primes of
// index first, first + 1, ... in the basis q_0..q_L, p_0..) from the q_0 limb's integer
// coefficients, centred (NTT + Montgomery like the copied limbs)
static cudaError_t extend_limbs(const Context& c, size_t count, const uint64_t* in, uint32_t l_in, uint32_t nlx,
                                uint32_t first, uint64_t* out, cudaStream_t s) {
    if (l_in == 0 || l_in >= nlx || first + (nlx - l_in) > c.L + 1 + c.alpha) return cudaErrorInvalidValue;
    const uint32_t nx = nlx - l_in;
    const size_t n = c.n;
    uint64_t* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, n * 8);
    if (e != cudaSuccess) return e;
    for (size_t k = 0; k < count && e == cudaSuccess; k++) {
        const uint64_t* src = in + k * l_in * n;
        uint64_t* dst = out + k * nlx * n;
        e = cudaMemcpyAsync(dst, src, l_in * n * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, src, n * 8, cudaMemcpyDeviceToDevice, s);
        LimbBatch t0{tmp, 1, n, 0, 1, 0};
        t0.set(0, 0);
        if (e == cudaSuccess) e = to_montgomery(c, t0, true, s);
        if (e == cudaSuccess) e = ntt_inverse(c, t0, s);
        if (e == cudaSuccess) {
            k_centred_to_p<<<dim3(nx, (uint32_t)(n / kThreads / 4)), kThreads, 0, s>>>(tmp, dst + l_in * n, n,
                                                                                     c.primes[0], first, c.tab,
                                                                                     (uint32_t)n);
            e = cudaGetLastError();
        }
        LimbBatch pb{dst, 1, (uint64_t)nlx * n, l_in, nx, 0};
        for (uint32_t i = 0; i < nx; i++) pb.set(i, first + i);
        if (e == cudaSuccess) e = ntt_forward(c, pb, s);
        if (e == cudaSuccess) e = to_montgomery(c, pb, false, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(tmp);
    return e;
}

cudaError_t extend_to_ext_basis(const Context& c, size_t count, const uint64_t* in, uint32_t l_in, uint64_t* out,
                                cudaStream_t s) {
    return extend_limbs(c, count, in, l_in, c.L + 1 + c.alpha, l_in, out, s);
}

cudaError_t extend_to_level_ext(const Context& c, size_t count, const uint64_t* in, uint32_t l_in, uint64_t* out,
                                cudaStream_t s) {
    return extend_limbs(c, count, in, l_in, l_in + c.alpha, c.L + 1, out, s);
}

cudaError_t masks_extend(const Context& c, uint32_t n_in, const uint64_t* masks, uint64_t* ext, cudaStream_t s) {
    return extend_to_ext_basis(c, n_in, masks, c.L + 1, ext, s);
}

cudaError_t circ_prepare(const Context& c, uint32_t n_in, uint32_t l1, const uint64_t* masks, uint64_t* hat,
                         ulonglong2* tw, cudaStream_t s) {
    if (n_in < 2 || n_in > kMaxCircParts || (n_in & (n_in - 1)) || l1 > MAXB) return cudaErrorInvalidValue;
    std::vector<ulonglong2> h((size_t)l1 * n_in);
    CircNinv ninv{};
    for (uint32_t j = 0; j < l1; j++) {
        const uint64_t q = c.primes[j];
        const uint64_t w = h_powmod(c.psi[j], (2ull << c.log_n) / n_in, q), wi = h_invmod(w, q);
        for (uint32_t e = 0; e < n_in / 2; e++) {
            const uint64_t a = h_powmod(w, e, q), b = h_powmod(wi, e, q);
            h[(size_t)j * n_in + e] = make_ulonglong2(a, h_shoup_companion(a, q));
            h[(size_t)j * n_in + n_in / 2 + e] = make_ulonglong2(b, h_shoup_companion(b, q));
        }
        const uint64_t ni = h_invmod(n_in % q, q);
        ninv.v[j] = make_ulonglong2(ni, h_shoup_companion(ni, q));
    }
    cudaError_t e = cudaMemcpyAsync(tw, h.data(), h.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    const dim3 g(c.n / kMacThreads, l1);
    switch (n_in) {
        case 2: k_circ_prep<2><<<g, kMacThreads, 0, s>>>(masks, hat, tw, ninv, l1, c.tab, c.log_n); break;
        case 4: k_circ_prep<4><<<g, kMacThreads, 0, s>>>(masks, hat, tw, ninv, l1, c.tab, c.log_n); break;
        case 8: k_circ_prep<8><<<g, kMacThreads, 0, s>>>(masks, hat, tw, ninv, l1, c.tab, c.log_n); break;
        case 16: k_circ_prep<16><<<g, kMacThreads, 0, s>>>(masks, hat, tw, ninv, l1, c.tab, c.log_n); break;
        default: k_circ_prep<32><<<g, kMacThreads, 0, s>>>(masks, hat, tw, ninv, l1, c.tab, c.log_n); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the host table must outlive the copy
    return cudaStreamSynchronize(s);
}

}  // namespace bm
