// ks_fused.cu -- rotation (Galois automorphism + hybrid key switching) in six
// fused kernels, for the rings whose NTT passes are register resident (2^12, 2^16).
//
// Rot(ct, r) of Sec. 2 on B ciphertexts (c0, c1) at level l, NTT form:
//   F1  inverse row pass of c1; copy of c0; the digit's own extended limbs as
//       the NTT-domain automorphism of c1 (no transform needed for them)
//   F2  inverse column pass of c1 -> coefficient form
//   F3  per digit: automorphism gather (X^p <- +-X^(p k^-1)) + fast base
//       conversion to each other limb of Q_l u P + forward column pass
//   F4  per extended limb: forward row pass, inner product with the rotation
//       key over the digits, and for the special-prime limbs the inverse row pass
//   F5  inverse column pass of the special-prime limbs, conversion P -> Q_l,
//       forward column pass
//   F6  forward row pass, (acc - conv) * P^-1 + sigma(c0) (+ addend) -> out
// Each kernel reads and writes every coefficient once; the scratch holds
// X0, X1, ext, acc and conv (the same words as the staged kernels).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "bm_internal.h"
#include "ntt_reg.cuh"

namespace bm {
namespace {


__device__ __forceinline__ uint32_t brev_n(uint32_t x, uint32_t bits) { return __brev(x) >> (32 - bits); }

// NTT-domain automorphism: NTT(sigma_k a)[i] = NTT(a)[perm(i)]
__device__ __forceinline__ uint32_t perm_src(uint32_t i, uint32_t log_n, uint32_t galois) {
    const uint32_t r = brev_n(i, log_n);
    const uint32_t e = ((2u * r + 1u) * galois) & ((2u << log_n) - 1);
    return brev_n((e - 1u) >> 1, log_n);
}

__device__ __forceinline__ int ext_prime(int jj, int l1, int L) { return jj < l1 ? jj : L + 1 + (jj - l1); }

__device__ __forceinline__ uint64_t red6(uint64_t y, uint64_t t) {   // [0, 6t) -> [0, 4t)
    return y >= 4 * t ? y - 4 * t : y;
}

constexpr int kMaxDigit = 2;   // limbs per digit and special primes handled by the fused kernels


using nttr::ColBase;
using nttr::first_idx;
using nttr::last_idx;
using nttr::RowBase;
using nttr::row_tw_entries;
using nttr::stage_col_twiddles;
using nttr::stage_row_twiddles;
using nttr::sub_words;
using nttr::SubMem;
using nttr::tw_wait;

// Dynamic shared memory (words) of the column kernel F3: exchange tiles,
// kMaxDigit thread-private staging tiles (each thread reads back only what it
// wrote), staged twiddles.
template <int LA, int LT, int C>
__host__ __device__ constexpr size_t col_smem_words() {
    return (size_t)sub_words<LA, LT>() * C + (size_t)kMaxDigit * (1 << LA) * C + 2 * (size_t)(1 << LA);
}
// ... and of F4: exchange rows, staging, forward and inverse row twiddles.
template <int LB, int LT, int R, int ND>
__host__ __device__ constexpr size_t f4_smem_words() {
    return (size_t)R * sub_words<LB, LT>() + (LT > 2 ? (size_t)ND * R * (1 << LB) : 0) +
           4 * (size_t)row_tw_entries<LB, R>();
}

// ---------------------------------------------------------------------------
// F1: grid (B * l1, N1 / R)
// ---------------------------------------------------------------------------
template <int LA, int LB, int LT, int R>
__global__ void __launch_bounds__(R * (1 << (LB - LT)))
    k_ks_f1(uint64_t* const* in, uint64_t* __restrict__ X0, uint64_t* __restrict__ X1, uint64_t* __restrict__ ext,
            const KsLevelConst* __restrict__ kc, DevTables tab, uint32_t l1, uint32_t galois) {
    constexpr int K = 1 << LT, M = 1 << LB, TH = M >> LT, S = sub_words<LB, LT>(), LOGN = LA + LB, N = 1 << LOGN;
    __shared__ uint64_t sm[R * S];
    __shared__ ulonglong2 tws[row_tw_entries<LB, R>()];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const uint32_t b = blockIdx.x / l1, j = blockIdx.x % l1;
    const int row = blockIdx.y * R + jr;
    const size_t roff = (size_t)row * M;
    const uint64_t q = tab.q[j], q2 = 2 * q;
    const uint64_t* c0 = in[b] + (size_t)j * N + roff;
    const uint64_t* c1 = in[b] + ((size_t)l1 + j) * N;
    const uint32_t nd = kc->nd, nlx = kc->nlx;
    uint32_t d = 0;
    while (d + 1 < nd && j >= kc->dstart[d + 1]) d++;
    uint64_t* x0 = X0 + ((size_t)b * l1 + j) * N + roff;
    uint64_t* eo = ext + (((size_t)b * nd + d) * nlx + j) * N + roff;
    const SubMem sr{sm + jr * S, 1};
    stage_row_twiddles<LA, LB, R, R * TH>(tws, tab.itw[j], blockIdx.y * R);
    pdl_wait();
    uint64_t v[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int c = first_idx<LB, LT>(t, k);
        v[k] = c1[roff + c];
        x0[c] = c0[c];
        eo[c] = c1[perm_src((uint32_t)(roff + c), LOGN, galois)];
    }
    nttr::relayout<LB, LT, 0, LB / LT - 1>(v, sr, t);
    tw_wait();
    nttr::inv_pass<LB, LT>(v, sr, tws, RowBase<R>{jr}, t, q, q2);
    pdl_trigger();
    uint64_t* x1 = X1 + ((size_t)b * l1 + j) * N + roff;
#pragma unroll
    for (int k = 0; k < K; k++) x1[first_idx<LB, LT>(t, k)] = v[k];
}

// forward column pass of y (phase-0 layout in) stored in the last layout to o
template <int LA, int LB, int LT, int C>
__device__ __forceinline__ void col_fwd_store(uint64_t (&y)[1 << LT], uint64_t* sm, const ulonglong2* tws, int t,
                                              int jc, uint64_t q, uint64_t* o) {
    constexpr int N2 = 1 << LB;
    nttr::fwd_pass<LA, LT>(y, SubMem{sm + jc, C}, tws, ColBase{}, t, q, 2 * q);
#pragma unroll
    for (int k = 0; k < (1 << LT); k++) o[(size_t)last_idx<LA, LT>(t, k) * N2] = y[k];
}

// ---------------------------------------------------------------------------
// F3: grid (B * nd * ts_n, N2 / C).  X1 holds c1 in coefficient form.  The digit's
// target limbs (every extended limb but its own) are dealt round-robin to ts_n blocks
// of the same columns, each staging the digit's source limbs itself: ts_n > 1 fills
// the GPU when B * nd column blocks alone would leave SMs idle (one query).
// ---------------------------------------------------------------------------
template <int LA, int LB, int LT, int C>
__global__ void __launch_bounds__(C * (1 << (LA - LT)))
    k_ks_f3(const uint64_t* __restrict__ X1, uint64_t* __restrict__ ext, const KsLevelConst* __restrict__ kc,
            DevTables tab, uint32_t l1, uint32_t L, uint32_t kinv, uint32_t ts_n) {
    constexpr int K = 1 << LT, M = 1 << LA, N2 = 1 << LB, LOGN = LA + LB, N = 1 << LOGN;
    extern __shared__ uint64_t dsm[];
    uint64_t* sm = dsm;                                   // exchange tiles
    // staging [i][k][thread]: thread-private (each thread reads back only what it
    // wrote), thread index fastest so a warp's accesses are free of bank conflicts
    uint64_t* st = sm + sub_words<LA, LT>() * C;
    ulonglong2* tws = (ulonglong2*)(st + kMaxDigit * M * C);
    constexpr int NT = C * (M >> LT);
    const int tid = threadIdx.x, t = tid / C, jc = tid % C;
    const uint32_t nd = kc->nd, nlx = kc->nlx;
    const uint32_t ts = blockIdx.x % ts_n, bd = blockIdx.x / ts_n;
    const uint32_t b = bd / nd, d = bd % nd;
    const int col = blockIdx.y * C + jc;
    const uint32_t ds = kc->dsz[d], d0 = kc->dstart[d];
    pdl_wait();
#pragma unroll 1
    for (uint32_t i = 0; i < ds; i++) {
        const uint64_t qi = tab.q[d0 + i];
        const ulonglong2 h = kc->up_hinv[d][i];
        const uint64_t* src = X1 + ((size_t)b * l1 + d0 + i) * N;
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int r = first_idx<LA, LT>(t, k);
            const uint32_t e = ((uint32_t)r * N2 + col) * kinv & (2u * N - 1);
            uint64_t x = src[e & (N - 1)];
            if (e >= (uint32_t)N) x = negm(x, qi);
            st[(i * K + k) * NT + tid] = shoup(x, h.x, h.y, qi);
        }
    }
    uint32_t ti = 0;                                          // index among the digit's targets
#pragma unroll 1
    for (uint32_t jj = 0; jj < nlx; jj++) {
        if (jj >= d0 && jj < d0 + ds) continue;               // the digit's own limbs come from F1
        if (ti++ % ts_n != ts) continue;                      // another block's target
        const int pi = ext_prime(jj, l1, L);
        const uint64_t tq = tab.q[pi];
        stage_col_twiddles<LA, C * (M >> LT)>(tws, tab.tw[pi]);
        uint64_t y[K];
#pragma unroll
        for (int k = 0; k < K; k++) y[k] = 0;
#pragma unroll 1
        for (uint32_t i = 0; i < ds; i++) {
            const ulonglong2 h = kc->up_hat[d][i][jj];
#pragma unroll
            for (int k = 0; k < K; k++)
                y[k] += shoup_lazy(st[(i * K + k) * NT + tid], h.x, h.y, tq);
        }
#pragma unroll
        for (int k = 0; k < K; k++) y[k] = red6(y[k], tq);
        tw_wait();
        col_fwd_store<LA, LB, LT, C>(y, sm, tws, t, jc, tq, ext + (((size_t)b * nd + d) * nlx + jj) * N + col);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// F4: grid (B * nlx, N1 / R).  acc = sum_d ext_d * key_d (both components), up to
// ND digits (their row-passed extension words in registers, or in shared memory for
// the 16-coefficient shape).
// ---------------------------------------------------------------------------
template <int LA, int LB, int LT, int R, int ND>
__global__ void __launch_bounds__(R * (1 << (LB - LT)), LT <= 2 ? 8 : 4)
    k_ks_f4(const uint64_t* __restrict__ ext, const uint64_t* __restrict__ key, uint64_t* __restrict__ acc,
            const KsLevelConst* __restrict__ kc, DevTables tab, uint32_t l1, uint32_t L, uint32_t nb) {
    constexpr int K = 1 << LT, M = 1 << LB, TH = M >> LT, S = sub_words<LB, LT>(), LOGN = LA + LB, N = 1 << LOGN;
    constexpr int TWN = row_tw_entries<LB, R>();
    constexpr bool REG = LT <= 2;                            // digits held in registers (else shared memory)
    constexpr int NT = R * TH;
    extern __shared__ uint64_t dsm[];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const SubMem sr{dsm + jr * S, 1};                        // exchange row
    uint64_t* st = dsm + R * S;                              // staging (16-coefficient shape): [d][k][tid]
    ulonglong2* twf = (ulonglong2*)(dsm + R * S + (REG ? 0 : ND * R * M));
    ulonglong2* twi = twf + TWN;
    const uint32_t nd = kc->nd, nlx = kc->nlx;
    const uint32_t b = blockIdx.x / nlx, jj = blockIdx.x % nlx;
    const int pi = ext_prime(jj, l1, L);
    const uint64_t q = tab.q[pi], qn = tab.qneg[pi], q2 = 2 * q;
    const int row = blockIdx.y * R + jr;
    const size_t roff = (size_t)row * M;
    const RowBase<R> base{jr};
    stage_row_twiddles<LA, LB, R, R * TH>(twf, tab.tw[pi], blockIdx.y * R);
    if (jj >= l1) stage_row_twiddles<LA, LB, R, R * TH>(twi, tab.itw[pi], blockIdx.y * R);
    tw_wait();
    pdl_wait();
    uint64_t v[K], sv[REG ? ND : 1][REG ? K : 1];
    // extended limb jj of every digit, NTT form, last-phase layout
#pragma unroll 1
    for (uint32_t d = 0; d < nd; d++) {
        const uint64_t* e = ext + (((size_t)b * nd + d) * nlx + jj) * N + roff;
        if (jj >= kc->dstart[d] && jj < kc->dstart[d] + kc->dsz[d]) {
            nttr::load_last<LB, LT>(v, e, t);
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) v[k] = e[first_idx<LB, LT>(t, k)];
            nttr::fwd_pass<LB, LT>(v, sr, twf, base, t, q, q2);
            __syncthreads();
        }
        if constexpr (REG) {
#pragma unroll
            for (int dd = 0; dd < ND; dd++)
                if ((uint32_t)dd == d) {
#pragma unroll
                    for (int k = 0; k < K; k++) sv[dd][k] = v[k];
                }
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) st[(d * K + k) * NT + tid] = v[k];
        }
    }
    // inner product per key component (summed at 128 bits, one reduction), then
    // store (special primes: inverse row pass)
#pragma unroll 1
    for (uint32_t comp = 0; comp < 2; comp++) {
        Acc128 a[K];
#pragma unroll
        for (int d = 0; d < ND; d++) {
            if ((uint32_t)d < nd) {
                uint64_t kv[K];
                nttr::load_last<LB, LT>(kv, key + ((size_t)(d * 2 + comp) * nb + pi) * N + roff, t);
#pragma unroll
                for (int k = 0; k < K; k++) {
                    uint64_t e;
                    if constexpr (REG) e = sv[d][k];
                    else e = st[(d * K + k) * NT + tid];
                    mul_acc(a[k], e, kv[k], q);              // e < 4q after the row pass: allowed
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; k++) v[k] = redc(a[k], q, qn);
        if (jj < l1) {
            nttr::relayout<LB, LT, LB / LT - 1, 0>(v, sr, t);
        } else {
            nttr::inv_pass<LB, LT>(v, sr, twi, base, t, q, q2);
        }
        uint64_t* o = acc + (((size_t)b * 2 + comp) * nlx + jj) * N + roff;
#pragma unroll
        for (int k = 0; k < K; k++) o[first_idx<LB, LT>(t, k)] = v[k];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The queries' forward NTT (a0) and the extension of their c1 for the hoisted Algorithm 1
// in two launches, from the coefficient form in qin ([Q][2][l1][N], qstride words a query):
// F0c, grid (Q * l1 + Q * nd * ts_n, N2 / C): blocks below Q * l1 the forward column pass
// of a c0 limb in place; the others, per (query, digit, slice), the digit's targets --
// every extended limb, its own limbs as they are and the others by the fast base
// conversion of F3 -- each after its forward column pass into ext (qin's c1 is only
// read here, so no copy of it is needed).  F0r, grid (Q * l1 + Q * nd * nlx, N1 / R):
// the forward row pass of the c0 limbs in place and of every limb of ext in place, each
// own limb of a digit written to qin's c1 as well.  The residues of a0's NTT, F3 and F3r.
// ---------------------------------------------------------------------------
template <int LA, int LB, int LT, int C>
__global__ void __launch_bounds__(C * (1 << (LA - LT)))
    k_ks_f0c(uint64_t* __restrict__ qin, uint64_t qstride, uint64_t* __restrict__ ext,
             const KsLevelConst* __restrict__ kc, DevTables tab, uint32_t l1, uint32_t L, uint32_t n0, uint32_t ts_n) {
    constexpr int K = 1 << LT, M = 1 << LA, N2 = 1 << LB, LOGN = LA + LB, N = 1 << LOGN;
    extern __shared__ uint64_t dsm[];
    uint64_t* sm = dsm;
    uint64_t* st = sm + sub_words<LA, LT>() * C;
    ulonglong2* tws = (ulonglong2*)(st + kMaxDigit * M * C);
    constexpr int NT = C * (M >> LT);
    const int tid = threadIdx.x, t = tid / C, jc = tid % C;
    const int col = blockIdx.y * C + jc;
    if (blockIdx.x < n0) {
        // a0, c0 limb j of query b
        const uint32_t b = blockIdx.x / l1, j = blockIdx.x % l1;
        uint64_t* a = qin + (size_t)b * qstride + (size_t)j * N + col;
        const uint64_t q = tab.q[j];
        stage_col_twiddles<LA, NT>(tws, tab.tw[j]);
        pdl_wait();
        uint64_t v[K];
#pragma unroll
        for (int k = 0; k < K; k++) v[k] = a[(size_t)first_idx<LA, LT>(t, k) * N2];
        tw_wait();
        nttr::fwd_pass<LA, LT>(v, SubMem{sm + jc, C}, tws, ColBase{}, t, q, 2 * q);
#pragma unroll
        for (int k = 0; k < K; k++) a[(size_t)last_idx<LA, LT>(t, k) * N2] = v[k];
        return;
    }
    const uint32_t nd = kc->nd, nlx = kc->nlx;
    const uint32_t rb = blockIdx.x - n0, ts = rb % ts_n, bd = rb / ts_n;
    const uint32_t b = bd / nd, d = bd % nd;
    const uint32_t ds = kc->dsz[d], d0 = kc->dstart[d];
    const uint64_t* X1 = qin + (size_t)b * qstride + (size_t)l1 * N;      // c1, coefficient form
    pdl_wait();
#pragma unroll 1
    for (uint32_t i = 0; i < ds; i++) {
        const uint64_t qi = tab.q[d0 + i];
        const ulonglong2 h = kc->up_hinv[d][i];
        const uint64_t* src = X1 + (size_t)(d0 + i) * N + col;
#pragma unroll
        for (int k = 0; k < K; k++)
            st[(i * K + k) * NT + tid] = shoup(src[(size_t)first_idx<LA, LT>(t, k) * N2], h.x, h.y, qi);
    }
#pragma unroll 1
    for (uint32_t jj = ts; jj < nlx; jj += ts_n) {
        const int pi = ext_prime(jj, l1, L);
        const uint64_t tq = tab.q[pi];
        stage_col_twiddles<LA, NT>(tws, tab.tw[pi]);
        uint64_t y[K];
        if (jj >= d0 && jj < d0 + ds) {
            const uint64_t* src = X1 + (size_t)jj * N + col;             // own limb: c1 itself
#pragma unroll
            for (int k = 0; k < K; k++) y[k] = src[(size_t)first_idx<LA, LT>(t, k) * N2];
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) y[k] = 0;
#pragma unroll 1
            for (uint32_t i = 0; i < ds; i++) {
                const ulonglong2 h = kc->up_hat[d][i][jj];
#pragma unroll
                for (int k = 0; k < K; k++) y[k] += shoup_lazy(st[(i * K + k) * NT + tid], h.x, h.y, tq);
            }
#pragma unroll
            for (int k = 0; k < K; k++) y[k] = red6(y[k], tq);
        }
        tw_wait();
        col_fwd_store<LA, LB, LT, C>(y, sm, tws, t, jc, tq, ext + (((size_t)b * nd + d) * nlx + jj) * N + col);
        __syncthreads();
    }
}

template <int LA, int LB, int LT, int R>
__global__ void __launch_bounds__(R * (1 << (LB - LT)))
    k_ks_f0r(uint64_t* __restrict__ qin, uint64_t qstride, uint64_t* __restrict__ ext,
             const KsLevelConst* __restrict__ kc, DevTables tab, uint32_t l1, uint32_t L, uint32_t n0) {
    constexpr int K = 1 << LT, M = 1 << LB, TH = M >> LT, S = sub_words<LB, LT>(), N = 1 << (LA + LB);
    __shared__ uint64_t sm[R * S];
    __shared__ ulonglong2 tws[row_tw_entries<LB, R>()];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const size_t roff = (size_t)(blockIdx.y * R + jr) * M;
    uint64_t *e, *also = nullptr;
    int pi;
    if (blockIdx.x < n0) {
        const uint32_t b = blockIdx.x / l1, j = blockIdx.x % l1;
        e = qin + (size_t)b * qstride + (size_t)j * N + roff;
        pi = (int)j;
    } else {
        const uint32_t nd = kc->nd, nlx = kc->nlx, rb = blockIdx.x - n0;
        const uint32_t jj = rb % nlx, d = (rb / nlx) % nd, b = rb / (nd * nlx);
        e = ext + (size_t)rb * N + roff;
        pi = ext_prime(jj, l1, L);
        if (jj >= kc->dstart[d] && jj < kc->dstart[d] + kc->dsz[d])
            also = qin + (size_t)b * qstride + ((size_t)l1 + jj) * N + roff;      // qin's c1 limb jj
    }
    const uint64_t q = tab.q[pi], q2 = 2 * q;
    stage_row_twiddles<LA, LB, R, R * TH>(tws, tab.tw[pi], blockIdx.y * R);
    pdl_wait();
    uint64_t v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = e[first_idx<LB, LT>(t, k)];
    tw_wait();
    nttr::fwd_pass<LB, LT>(v, SubMem{sm + jr * S, 1}, tws, RowBase<R>{jr}, t, q, q2);
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = nttr::reduce4(v[k], q, q2);
    pdl_trigger();
    nttr::store_last<LB, LT>(v, e, t);
    if (also) nttr::store_last<LB, LT>(v, also, t);
}

// ---------------------------------------------------------------------------
// Hoisted rotations (several rotations of one ciphertext share its basis
// extension).  F3r: grid (B * nd * nlx, N1 / R): forward row pass, in place, of
// the converted limbs F3 left column-transformed, so that every extended limb
// of ext is in NTT order (the digit's own limbs already are, from F1).
// ---------------------------------------------------------------------------
template <int LA, int LB, int LT, int R>
__global__ void __launch_bounds__(R * (1 << (LB - LT)))
    k_ks_f3r(uint64_t* __restrict__ ext, const KsLevelConst* __restrict__ kc, DevTables tab, uint32_t l1, uint32_t L,
             const uint64_t* const* own_src) {
    constexpr int K = 1 << LT, M = 1 << LB, TH = M >> LT, S = sub_words<LB, LT>(), LOGN = LA + LB, N = 1 << LOGN;
    __shared__ uint64_t sm[R * S];
    __shared__ ulonglong2 tws[row_tw_entries<LB, R>()];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const uint32_t nd = kc->nd, nlx = kc->nlx;
    const uint32_t jj = blockIdx.x % nlx, d = (blockIdx.x / nlx) % nd;
    if (jj >= kc->dstart[d] && jj < kc->dstart[d] + kc->dsz[d]) {
        // own limb: NTT form already (F1 wrote it), or copied here from the NTT-form
        // input when the extension started from its coefficient form
        if (!own_src) return;
        const uint32_t b = blockIdx.x / (nd * nlx);
        const size_t roff = (size_t)(blockIdx.y * R + jr) * M;
        const uint64_t* src = own_src[b] + ((size_t)l1 + jj) * N + roff;
        uint64_t* e = ext + (size_t)blockIdx.x * N + roff;
        pdl_wait();
        uint64_t v[K];
#pragma unroll
        for (int k = 0; k < K; k++) v[k] = src[first_idx<LB, LT>(t, k)];
        pdl_trigger();
#pragma unroll
        for (int k = 0; k < K; k++) e[first_idx<LB, LT>(t, k)] = v[k];
        return;
    }
    const int pi = ext_prime(jj, l1, L);
    const uint64_t q = tab.q[pi], q2 = 2 * q;
    const int row = blockIdx.y * R + jr;
    uint64_t* e = ext + (size_t)blockIdx.x * N + (size_t)row * M;
    stage_row_twiddles<LA, LB, R, R * TH>(tws, tab.tw[pi], blockIdx.y * R);
    pdl_wait();
    uint64_t v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = e[first_idx<LB, LT>(t, k)];
    tw_wait();
    nttr::fwd_pass<LB, LT>(v, SubMem{sm + jr * S, 1}, tws, RowBase<R>{jr}, t, q, q2);
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = nttr::reduce4(v[k], q, q2);
    pdl_trigger();
    nttr::store_last<LB, LT>(v, e, t);
}

// F4h: grid (E * nlx, N1 / R).  Element e: acc[e] = sum_d sigma_e(ext_of[e]_d) * key_e,d
// -- the Galois image of an extended limb is a permutation of its NTT slots --
// then, for the special-prime limbs, the inverse row pass (as F4).
template <int LA, int LB, int LT, int R>
__global__ void __launch_bounds__(R * (1 << (LB - LT)), LT <= 2 ? 8 : 4)
    k_ks_f4h(const uint64_t* const* ext_of, const uint64_t* const* key_of, const uint64_t* gal_of,
             uint64_t* __restrict__ acc, const KsLevelConst* __restrict__ kc, DevTables tab, uint32_t l1, uint32_t L,
             uint32_t nb) {
    constexpr int K = 1 << LT, M = 1 << LB, TH = M >> LT, S = sub_words<LB, LT>(), LOGN = LA + LB, N = 1 << LOGN;
    constexpr int TWN = row_tw_entries<LB, R>();
    __shared__ uint64_t sm[R * S];
    __shared__ ulonglong2 twi[TWN];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const SubMem sr{sm + jr * S, 1};
    const uint32_t nd = kc->nd, nlx = kc->nlx;
    const uint32_t e = blockIdx.x / nlx, jj = blockIdx.x % nlx;
    const int pi = ext_prime(jj, l1, L);
    const uint64_t q = tab.q[pi], qn = tab.qneg[pi], q2 = 2 * q;
    const uint32_t galois = (uint32_t)gal_of[e];
    const uint64_t* key = key_of[e];
    const uint64_t* ext = ext_of[e];
    const int row = blockIdx.y * R + jr;
    const size_t roff = (size_t)row * M;
    if (jj >= l1) stage_row_twiddles<LA, LB, R, R * TH>(twi, tab.itw[pi], blockIdx.y * R);
    pdl_wait();
    uint32_t src[K];
#pragma unroll
    for (int k = 0; k < K; k++) src[k] = perm_src((uint32_t)(roff + last_idx<LB, LT>(t, k)), LOGN, galois);
    uint64_t v[K];
#pragma unroll 1
    for (uint32_t comp = 0; comp < 2; comp++) {
        Acc128 a[K];
#pragma unroll 1
        for (uint32_t d = 0; d < nd; d++) {
            const uint64_t* x = ext + ((size_t)d * nlx + jj) * N;
            uint64_t kv[K];
            nttr::load_last<LB, LT>(kv, key + ((size_t)(d * 2 + comp) * nb + pi) * N + roff, t);
#pragma unroll
            for (int k = 0; k < K; k++) mul_acc(a[k], x[src[k]], kv[k], q);
        }
#pragma unroll
        for (int k = 0; k < K; k++) v[k] = redc(a[k], q, qn);
        if (jj < l1) {
            nttr::relayout<LB, LT, LB / LT - 1, 0>(v, sr, t);
        } else {
            if (comp == 0) tw_wait();
            nttr::inv_pass<LB, LT>(v, sr, twi, RowBase<R>{jr}, t, q, q2);
        }
        uint64_t* o = acc + (((size_t)e * 2 + comp) * nlx + jj) * N + roff;
#pragma unroll
        for (int k = 0; k < K; k++) o[first_idx<LB, LT>(t, k)] = v[k];
        __syncthreads();
    }
}

// The Galois image of a limb in NTT form at the four positions i0 .. i0 + 3 (i0 a
// multiple of 4, thread t of the last row layout): for any odd Galois element the
// four source positions perm_src(i0 + k) are an aligned group of four words --
// positions i0 + k and i0 + k + 1 (k even) come from one 16-byte half of the
// group, in either order, and positions i0 + 2, i0 + 3 from the other half -- so
// the group is read as one 32-byte vector and its words put in place by selects.
struct Perm4 {
    uint32_t gb;        // first source word of the group
    uint32_t sel;       // bit 1: the half of positions 0, 1; bit 0: they are swapped; bit 2: 2, 3 swapped
};
__device__ __forceinline__ Perm4 perm4(uint32_t i0, uint32_t log_n, uint32_t galois) {
    const uint32_t p0 = perm_src(i0, log_n, galois), p2 = perm_src(i0 + 2, log_n, galois);
    return {p0 & ~3u, (p0 & 3u) | ((p2 & 1u) << 2)};
}
struct W4 {
    uint64_t w[4];
};
// four consecutive words, one 256-bit load (32-byte aligned)
__device__ __forceinline__ W4 ld256(const uint64_t* p) {
    W4 r;
    asm volatile("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(r.w[0]), "=l"(r.w[1]), "=l"(r.w[2]), "=l"(r.w[3])
                 : "l"(p));
    return r;
}
__device__ __forceinline__ void place4(uint64_t (&o)[4], const W4& g, uint32_t sel) {
    const uint64_t a0 = (sel & 2) ? g.w[2] : g.w[0], a1 = (sel & 2) ? g.w[3] : g.w[1];
    const uint64_t b0 = (sel & 2) ? g.w[0] : g.w[2], b1 = (sel & 2) ? g.w[1] : g.w[3];
    o[0] = (sel & 1) ? a1 : a0;
    o[1] = (sel & 1) ? a0 : a1;
    o[2] = (sel & 4) ? b1 : b0;
    o[3] = (sel & 4) ? b0 : b1;
}

// F4s: grid (T * nlx, N1 / R); a block holds both ciphertext components of R rows of
// one extended limb of one target, so every gathered extension word serves the
// products of both.  Target t sums its elements e in [off[t], off[t+1]) before a
// single ModDown (double hoisting):
//   acc[t] = sum_e ( sum_d sigma_e(ext_of[e]_d) * key_e,d  +  P * sigma_e(c0 of src_of[e]) )
// the last term on the q-limbs of the first component only (ModDown returns it
// exactly: P * x has no special-prime residue and (P * x) * P^-1 = x), taken as P
// times the sum of the gathered c0 words (one product per word, not one per
// element); then, for the special-prime limbs, the inverse row pass (as F4) -- or,
// with ntt_out, every limb left in NTT form (the fused Algorithm 1 multiplies them
// by the masks first).  A thread holds four consecutive words of a row (the last
// row layout) and moves every operand group as one 32-byte vector: its key words of
// each digit and component, the Galois source group of each extension digit and of
// c0.  The products are summed at 128 bits without a reduction per product (the
// high word -- and the c0 sum -- reduced every kFoldElems elements: at most
// ND * kFoldElems < 64 products and kFoldElems < 16 c0 words between reductions)
// and reduced once.  With tpad (only with ntt_out), the sums of each run of tpad
// consecutive targets go to slots 1..tpad of a run of tpad + 1, and slot 0 of the run
// gets P times the run's source ciphertext: E_0, E_1..E_(N_in-1) of a query of the fused
// Algorithm 1 in one launch.  GM: group-masked sums (the fused rotate-and-sum and
// compression; flags in each element's Galois word mark its group's end and mask and the
// unrotated term).  PF (one digit, with GM): the element loop software-pipelined, the next
// element's key words, extension gather and permutation issued before the current
// element's c0 gather and products.
constexpr uint32_t kFoldElems = 12;

// F3's target slices: every target limb of a digit in a block of its own while the
// batch's column blocks (B * nd * column blocks) would not give each SM four, else one
// block for all of a digit's targets (the source limbs staged once)
constexpr uint32_t kF3FillBlocks = 4 * 152;
uint32_t f3_slices(const KsLevelConst& K, uint32_t B, uint32_t col_blocks) {
    if ((uint64_t)B * K.nd * col_blocks >= kF3FillBlocks) return 1;
    uint32_t t = 1;
    for (uint32_t d = 0; d < K.nd; d++) t = std::max(t, K.nlx - K.dsz[d]);
    return t;
}
template <int LA, int LB, int R, int ND, int MINB, bool GM, bool PF = false>
__global__ void __launch_bounds__(R * (1 << (LB - 2)), MINB)
    k_ks_f4s(const uint64_t* const* ext_of, const uint64_t* const* src_of, const uint64_t* const* key_of,
             const uint64_t* gal_of, const uint64_t* off, uint64_t* __restrict__ acc,
             const KsLevelConst* __restrict__ kc, DevTables tab, uint32_t l1, uint32_t L, uint32_t nb,
             bool ntt_out, uint32_t tpad, bool by_target, const uint64_t* __restrict__ gmask, bool inv_all) {
    constexpr int LT = 2, K = 4, M = 1 << LB, TH = M >> LT, SW = sub_words<LB, LT>(), LOGN = LA + LB, N = 1 << LOGN;
    constexpr int TWN = row_tw_entries<LB, R>();
    __shared__ uint64_t sm[R * SW];
    __shared__ ulonglong2 twi[TWN];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const SubMem sr{sm + jr * SW, 1};
    const uint32_t nd = kc->nd, nlx = kc->nlx;
    // by_target: blocks taken target by target (limb fastest, then row), so the many
    // rotations of one source read its permuted extension while it is still in L2;
    // else row by row over all targets (limb fastest, then target), so targets that share
    // a key read each key row while it is in L2
    const uint32_t lin = blockIdx.y * gridDim.x + blockIdx.x, jj = lin % nlx;
    const uint32_t yb = by_target ? (lin / nlx) % gridDim.y : blockIdx.y;
    const uint32_t slot = by_target ? lin / (nlx * gridDim.y) : blockIdx.x / nlx;
    const int pi = ext_prime(jj, l1, L);
    const uint64_t q = tab.q[pi], qn = tab.qneg[pi], rsh = tab.rsh[pi], q2 = 2 * q;
    const uint64_t pm = jj < l1 ? kc->pmont[jj] : 0;
    const int row = yb * R + jr;
    const size_t roff = (size_t)row * M;
    const uint32_t i0 = (uint32_t)roff + (uint32_t)(t << LT);     // last layout: words i0 .. i0 + 3
    // special limbs for F5: inverse row pass (inv_all: every limb, for a ModDown taken in
    // the coefficient domain)
    const bool inv = (jj >= l1 || inv_all) && !ntt_out;
    const bool qlimb = jj < l1;
    // output slot = block's slot; with tpad, slot 0 of each run of tpad + 1 is P * the
    // run's source ciphertext (E_0 of the fused Algorithm 1: P * c on the q-limbs, 0 on
    // the special limbs) and slots 1..tpad the run's targets
    const uint32_t run = tpad ? slot / (tpad + 1) : 0, kk = tpad ? slot % (tpad + 1) : 1;
    const uint32_t tg = tpad ? run * tpad + kk - 1 : slot, tgo = slot;
    if (inv) stage_row_twiddles<LA, LB, R, R * TH>(twi, tab.itw[pi], yb * R);
    pdl_wait();
    if (kk == 0) {
        const uint64_t* src = src_of[off[run * tpad]];
#pragma unroll 1
        for (uint32_t comp = 0; comp < 2; comp++) {
            uint64_t v[K] = {0, 0, 0, 0};
            if (qlimb) {
                const W4 x = ld256(src + ((size_t)comp * l1 + jj) * N + i0);
#pragma unroll
                for (int k = 0; k < K; k++) v[k] = mont(x.w[k], pm, q, qn);
            }
            nttr::store_last<LB, LT>(v, acc + (((size_t)tgo * 2 + comp) * nlx + jj) * N + roff, t);
        }
        return;
    }
    const uint32_t e0 = (uint32_t)off[tg], e1 = (uint32_t)off[tg + 1];
    Acc128 a0[K], a1[K];
    uint64_t cs[K] = {0, 0, 0, 0};
    uint64_t pk0[K] = {0, 0, 0, 0}, pk1[K] = {0, 0, 0, 0};   // GM: the target's sum of masked groups
    if constexpr (PF) {
        // one digit, group-masked sums, elements software-pipelined: the key words and the
        // extension gather of element e + 1 (keys read from DRAM the first time a launch
        // uses them) are in flight while element e gathers its c0 words and runs its products
        static_assert(GM && ND == 1, "the pipelined loop takes one digit and group masks");
        uint64_t gwn = kGalIdentity;
        Perm4 pmn{i0, 0};
        W4 k0n{}, k1n{}, xn{};
        // element f's words: the unrotated source's c1 for an identity element (its c0 is
        // read with the products), else the Galois gather of its extension and its key
        auto issue = [&](uint32_t f) {
            gwn = gal_of[f];
            if (gwn & kGalIdentity) {
                pmn = Perm4{i0, 0};
                if (qlimb) xn = ld256(src_of[f] + ((size_t)l1 + jj) * N + i0);
            } else {
                pmn = perm4(i0, LOGN, (uint32_t)gwn);
                xn = ld256(ext_of[f] + (size_t)jj * N + pmn.gb);
                const uint64_t* key = key_of[f] + (size_t)pi * N + i0;
                k0n = ld256(key);
                k1n = ld256(key + (size_t)nb * N);
            }
        };
        if (e0 < e1) issue(e0);
        uint32_t fold = kFoldElems;                     // elements to the next reduction
#pragma unroll 1
        for (uint32_t e = e0; e < e1; e++) {
            const uint64_t gw = gwn;
            const W4 k0 = k0n, k1 = k1n, xw = xn;
            const bool ident = (gw & kGalIdentity) != 0;
            const Perm4 pm4 = pmn;
            W4 cw;
            if (qlimb) cw = ld256(src_of[e] + (size_t)jj * N + pm4.gb);
            if (e + 1 < e1) issue(e + 1);
            if (ident) {
                // the unrotated source: P * c0 joins the c0 sum, P * c1 the second component
                if (qlimb) {
#pragma unroll
                    for (int k = 0; k < K; k++) {
                        cs[k] += cw.w[k];
                        mad128(a1[k], xw.w[k], pm);
                    }
                }
            } else {
                uint64_t x[K];
                place4(x, xw, pm4.sel);
#pragma unroll
                for (int k = 0; k < K; k++) {
                    mad128(a0[k], x[k], k0.w[k]);
                    mad128(a1[k], x[k], k1.w[k]);
                }
                if (qlimb) {
                    uint64_t c[K];
                    place4(c, cw, pm4.sel);
#pragma unroll
                    for (int k = 0; k < K; k++) cs[k] += c[k];
                }
            }
            if (--fold == 0) {
                fold = kFoldElems;
#pragma unroll
                for (int k = 0; k < K; k++) {
                    reduce_hi(a0[k], q, rsh);
                    reduce_hi(a1[k], q, rsh);
                    const uint64_t r = cs[k] - mulhi64(cs[k], rsh) * q;   // [0, 2q)
                    cs[k] = r >= q ? r - q : r;
                }
            }
            if (gw & kGalGroupEnd) {
                const uint32_t mi = (uint32_t)((gw >> kGalMaskShift) & kGalMaskBits);
                const W4 mw = ld256(gmask + ((size_t)mi * nlx + jj) * N + i0);
#pragma unroll
                for (int k = 0; k < K; k++) {
                    if (qlimb) mad128(a0[k], cs[k], pm);
                    pk0[k] = addm(pk0[k], mont(redc_wide(a0[k], q, qn, rsh), mw.w[k], q, qn), q);
                    pk1[k] = addm(pk1[k], mont(redc_wide(a1[k], q, qn, rsh), mw.w[k], q, qn), q);
                    a0[k] = Acc128{};
                    a1[k] = Acc128{};
                    cs[k] = 0;
                }
            }
        }
    } else {
#pragma unroll 1
    for (uint32_t e = e0; e < e1; e++) {
        const uint64_t gw = gal_of[e];
        if (GM && (gw & kGalIdentity)) {
            // the unrotated source: P * c0 joins the c0 sum, P * c1 the second component
            if (qlimb) {
                const uint64_t* src = src_of[e];
                const W4 x0 = ld256(src + (size_t)jj * N + i0);
                const W4 x1 = ld256(src + ((size_t)l1 + jj) * N + i0);
#pragma unroll
                for (int k = 0; k < K; k++) {
                    cs[k] += x0.w[k];
                    mad128(a1[k], x1.w[k], pm);
                }
            }
        } else {
        const Perm4 pm4 = perm4(i0, LOGN, (uint32_t)gw);
        const uint64_t* key = key_of[e] + (size_t)pi * N + i0;
        const uint64_t* ext = ext_of[e] + (size_t)jj * N + pm4.gb;
        W4 xs[ND], k0s[ND], k1s[ND], cw;
#pragma unroll
        for (int d = 0; d < ND; d++) {
            if (d < (int)nd) {
                xs[d] = ld256(ext + (size_t)d * nlx * N);
                k0s[d] = ld256(key + (size_t)(2 * d) * nb * N);
                k1s[d] = ld256(key + (size_t)(2 * d + 1) * nb * N);
            }
        }
        if (qlimb) cw = ld256(src_of[e] + (size_t)jj * N + pm4.gb);
#pragma unroll
        for (int d = 0; d < ND; d++) {
            if (d < (int)nd) {
                uint64_t x[K];
                place4(x, xs[d], pm4.sel);
#pragma unroll
                for (int k = 0; k < K; k++) {
                    mad128(a0[k], x[k], k0s[d].w[k]);
                    mad128(a1[k], x[k], k1s[d].w[k]);
                }
            }
        }
        if (qlimb) {
            uint64_t c[K];
            place4(c, cw, pm4.sel);
#pragma unroll
            for (int k = 0; k < K; k++) cs[k] += c[k];
        }
        }
        if ((e - e0) % kFoldElems == kFoldElems - 1) {
#pragma unroll
            for (int k = 0; k < K; k++) {
                reduce_hi(a0[k], q, rsh);
                reduce_hi(a1[k], q, rsh);
                const uint64_t r = cs[k] - mulhi64(cs[k], rsh) * q;   // [0, 2q)
                cs[k] = r >= q ? r - q : r;
            }
        }
        if (GM && (gw & kGalGroupEnd)) {
            // the group's sum (with P times its c0 words) reduced, times the group's
            // plaintext (Montgomery form), added to the target's sum; the group
            // accumulators start again from zero
            const uint32_t mi = (uint32_t)((gw >> kGalMaskShift) & kGalMaskBits);
            const W4 mw = ld256(gmask + ((size_t)mi * nlx + jj) * N + i0);
#pragma unroll
            for (int k = 0; k < K; k++) {
                if (qlimb) mad128(a0[k], cs[k], pm);
                pk0[k] = addm(pk0[k], mont(redc_wide(a0[k], q, qn, rsh), mw.w[k], q, qn), q);
                pk1[k] = addm(pk1[k], mont(redc_wide(a1[k], q, qn, rsh), mw.w[k], q, qn), q);
                a0[k] = Acc128{};
                a1[k] = Acc128{};
                cs[k] = 0;
            }
        }
    }
    }
    if (!GM && qlimb) {
#pragma unroll
        for (int k = 0; k < K; k++) mad128(a0[k], cs[k], pm);
    }
#pragma unroll 1
    for (uint32_t comp = 0; comp < 2; comp++) {
        uint64_t v[K];
#pragma unroll
        for (int k = 0; k < K; k++) v[k] = GM ? (comp ? pk1[k] : pk0[k]) : redc_wide(comp ? a1[k] : a0[k], q, qn, rsh);
        uint64_t* o = acc + (((size_t)tgo * 2 + comp) * nlx + jj) * N + roff;
        if (!inv) {
            nttr::store_last<LB, LT>(v, o, t);
        } else {
            if (comp == 0) tw_wait();
            else __syncthreads();
            nttr::inv_pass<LB, LT>(v, sr, twi, RowBase<R>{jr}, t, q, q2);
#pragma unroll
            for (int k = 0; k < K; k++) o[first_idx<LB, LT>(t, k)] = v[k];
        }
    }
}

// ---------------------------------------------------------------------------
// F5: grid (B * 2, N2 / C), GP groups of C columns a block.  conv = Conv_{P -> Q_l}(acc's
// special-prime limbs): the inverse column pass of the ns special limbs (group g takes
// limb g: the passes of a column run side by side), each scaled by N^-1 (P/p_i)^-1 and
// staged in shared memory, then the conversion to the l1 target limbs and their
// forward column passes (group g takes targets g, g + GP, ...).  Groups without a limb
// in a phase only meet its barriers.
// (GP: the most special limbs; the fused divisions call it with the special set
// {q_L} u P -- l1 = L, L - 1 in place of L -- or {q_(L-1), q_L} u P -- l1 = L - 1, L - 2
// in place of L; the special limbs follow the targets in the basis order either way.)
// ---------------------------------------------------------------------------
// the block barriers of one register pass (one per exchange), without its arithmetic: a
// group with nothing to transform meets the barriers of the groups that have
template <int P, int LT>
__device__ __forceinline__ void pass_barriers() {
#pragma unroll
    for (int h = 0; h + 1 < P / LT; h++) __syncthreads();
}
template <int LA, int LT, int C, int GP, int MAXS, bool CD = false>
__host__ __device__ constexpr size_t f5_smem_words() {   // exchange and twiddles of each group, staging
    return (size_t)GP * (sub_words<LA, LT>() * C + 2 * (1 << LA)) +
           (size_t)(MAXS + (CD ? 2 : 0)) * (1 << LT) * C * ((1 << LA) >> LT);
}
// the constants of F5's coefficient-domain forms (RS, MU): N^-1 and the divisor's inverse
// (P^-1, or S^-1 for the deferred division) mod q_0, q_1, and q_1^-1 mod q_0 (Shoup pairs)
struct F5Rs {
    ulonglong2 ninv[2], pinv[2], q1inv;
};
// MU: the quotient's ModUp for the next level's hoisted key switching, taken in the same
// kernel: y [B][2][l1][N] receives the quotient's limbs after their forward column pass,
// ext (stride ext_words a ciphertext) the conversion of its c1 to the level's other
// extended limbs after theirs (the level has one digit, its l1 q-limbs; kcu its constants)
struct F5Mu {
    uint64_t* y;
    uint64_t* ext;
    const KsLevelConst* kcu;
    uint64_t ext_words;
    uint32_t Lc;                 // the context's top level (the special primes follow it)
};
template <int LA, int LB, int LT, int C, int GP, int MAXS, bool RS = false, bool MU = false>
__global__ void __launch_bounds__(GP * C * (1 << (LA - LT)))
    k_ks_f5(const uint64_t* __restrict__ acc, uint64_t* __restrict__ conv, const KsLevelConst* __restrict__ kc,
            DevTables tab, uint32_t l1, uint32_t L, uint32_t ns, uint64_t* const* rs_out, F5Rs rc, F5Mu mu) {
    constexpr bool CD = RS || MU;     // the ModDown in the coefficient domain
    constexpr int K = 1 << LT, M = 1 << LA, N2 = 1 << LB, LOGN = LA + LB, N = 1 << LOGN, TPC = M >> LT, NTG = C * TPC;
    constexpr int SW = sub_words<LA, LT>() * C;
    extern __shared__ uint64_t dsm[];
    const int tid = threadIdx.x, g = tid / NTG, r = tid % NTG, t = r / C, jc = r % C;
    uint64_t* xch = dsm + g * SW;                                   // the group's exchange columns
    uint64_t* st = dsm + GP * SW;                                   // staging [ns][K][NTG]
    uint64_t* fin = st + (size_t)MAXS * K * NTG;                    // CD: the two targets [2][K][NTG]
    ulonglong2* tws = reinterpret_cast<ulonglong2*>(fin + (CD ? (size_t)2 * K * NTG : 0)) + g * M;   // the group's twiddles
    const uint32_t b = blockIdx.x / 2, comp = blockIdx.x % 2;
    const int col = blockIdx.y * C + jc;
    const uint32_t nlx = l1 + ns;
    const SubMem sx{xch + jc, C};
    auto stage_tw = [&](const ulonglong2* tw) {
        for (int i = r; i < M; i += NTG) __pipeline_memcpy_async(tws + i, tw + i, sizeof(ulonglong2));
        __pipeline_commit();
    };
    // phase 1: special limbs g, g + GP, ...
    uint64_t y[K];
#pragma unroll 1
    for (uint32_t i0 = 0; i0 < ns; i0 += GP) {
        const uint32_t i = i0 + g;
        const bool a1 = i < ns;
        const int ps = (int)L + 1 + (int)i;
        const uint64_t p = a1 ? tab.q[ps] : tab.q[0];
        if (a1) stage_tw(tab.itw[ps]);
        if (i0 == 0) pdl_wait();
        if (a1) {
            const uint64_t* src = acc + (((size_t)b * 2 + comp) * nlx + l1 + i) * N + col;
#pragma unroll
            for (int k = 0; k < K; k++) y[k] = src[(size_t)last_idx<LA, LT>(t, k) * N2];
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) y[k] = 0;
        }
        __pipeline_wait_prior(0);
        __syncthreads();
        if (a1) nttr::inv_pass<LA, LT>(y, sx, tws, ColBase{}, t, p, 2 * p);
        else pass_barriers<LA, LT>();
        if (a1) {
            const ulonglong2 h = kc->dn_hinv[i];          // N^-1 * (P/p_i)^-1 mod p_i
#pragma unroll
            for (int k = 0; k < K; k++) st[(i * K + k) * NTG + r] = shoup(y[k], h.x, h.y, p);
        }
        __syncthreads();        // the twiddles are restaged, and the staging read, next
    }
    // phase 2: targets g, g + GP, ...  (CD: the target limb's own inverse column pass
    // instead of the conversion's forward one, the ModDown in the coefficient domain)
#pragma unroll 1
    for (uint32_t j0 = 0; j0 < l1; j0 += GP) {
        const uint32_t j = j0 + g;
        const bool a2 = j < l1;
        const uint64_t q = tab.q[a2 ? j : 0];
        if (a2) stage_tw(CD ? tab.itw[j] : tab.tw[j]);
#pragma unroll
        for (int k = 0; k < K; k++) y[k] = 0;
        if (a2) {
#pragma unroll 1
            for (uint32_t i = 0; i < ns; i++) {
                const ulonglong2 h = kc->dn_hat[i][j];
#pragma unroll
                for (int k = 0; k < K; k++) y[k] += shoup_lazy(st[(i * K + k) * NTG + r], h.x, h.y, q);
            }
        }
#pragma unroll
        for (int k = 0; k < K; k++) y[k] = red6(y[k], q);
        if constexpr (CD) {
            uint64_t x[K];
            if (a2) {
                const uint64_t* src = acc + (((size_t)b * 2 + comp) * nlx + j) * N + col;
#pragma unroll
                for (int k = 0; k < K; k++) x[k] = src[(size_t)last_idx<LA, LT>(t, k) * N2];
            }
            __pipeline_wait_prior(0);
            __syncthreads();
            if (a2) nttr::inv_pass<LA, LT>(x, sx, tws, ColBase{}, t, q, 2 * q);
            else pass_barriers<LA, LT>();
            if (a2) {
                // (N^-1 x - conv) * P^-1: the coefficient form of F6's output
                const ulonglong2 ni = rc.ninv[j], pi = rc.pinv[j];
#pragma unroll
                for (int k = 0; k < K; k++) {
                    uint64_t yr = y[k] >= 2 * q ? y[k] - 2 * q : y[k];           // [0, 4q) -> [0, q)
                    yr = yr >= q ? yr - q : yr;
                    fin[(j * K + k) * NTG + r] = shoup(subm(shoup(x[k], ni.x, ni.y, q), yr, q), pi.x, pi.y, q);
                }
            }
        } else {
            __pipeline_wait_prior(0);
            __syncthreads();
            if (a2) nttr::fwd_pass<LA, LT>(y, sx, tws, ColBase{}, t, q, 2 * q);
            else pass_barriers<LA, LT>();
            if (a2) {
                uint64_t* o = conv + (((size_t)b * 2 + comp) * l1 + j) * N + col;
#pragma unroll
                for (int k = 0; k < K; k++) o[(size_t)last_idx<LA, LT>(t, k) * N2] = y[k];
            }
        }
        __syncthreads();        // the twiddles are restaged for the next targets
    }
    if constexpr (MU) {
        // phase 3, jobs g, g + GP, ...: the forward column pass of each quotient limb (both
        // components) and, for c1, its conversion to each other extended limb of its level
        // (the fast base conversion of the hoisted ModUp, from the coefficient form held in
        // fin) and that limb's forward column pass
        const uint32_t nlu = mu.kcu->nlx, nj = l1 + (comp ? nlu - l1 : 0);
#pragma unroll 1
        for (uint32_t o0 = 0; o0 < nj; o0 += GP) {
            const uint32_t o = o0 + g;
            const bool a3 = o < nj;
            const int pi = o < l1 ? (int)o : (int)mu.Lc + 1 + (int)(o - l1);
            const uint64_t q = tab.q[a3 ? pi : 0];
            if (a3) stage_tw(tab.tw[pi]);
            if (a3) {
                if (o < l1) {
#pragma unroll
                    for (int k = 0; k < K; k++) y[k] = fin[(o * K + k) * NTG + r];
                } else {
#pragma unroll
                    for (int k = 0; k < K; k++) y[k] = 0;
#pragma unroll 1
                    for (uint32_t i = 0; i < l1; i++) {
                        const ulonglong2 hi = mu.kcu->up_hinv[0][i], hh = mu.kcu->up_hat[0][i][o];
                        const uint64_t qi = tab.q[i];
#pragma unroll
                        for (int k = 0; k < K; k++)
                            y[k] += shoup_lazy(shoup(fin[(i * K + k) * NTG + r], hi.x, hi.y, qi), hh.x, hh.y, q);
                    }
#pragma unroll
                    for (int k = 0; k < K; k++) y[k] = red6(y[k], q);
                }
            }
            __pipeline_wait_prior(0);
            __syncthreads();
            if (a3) nttr::fwd_pass<LA, LT>(y, sx, tws, ColBase{}, t, q, 2 * q);
            else pass_barriers<LA, LT>();
            if (a3) {
                uint64_t* dst = o < l1 ? mu.y + (((size_t)b * 2 + comp) * l1 + o) * N + col
                                       : mu.ext + (size_t)b * mu.ext_words + (size_t)o * N + col;
#pragma unroll
                for (int k = 0; k < K; k++) dst[(size_t)last_idx<LA, LT>(t, k) * N2] = y[k];
            }
            __syncthreads();    // the twiddles are restaged for the next jobs
        }
    }
    if constexpr (RS) {
        // the rescale from level 1: (c_0 - [c_1]_centred) * q_1^-1 mod q_0 (q_1 < q_0), in
        // natural coefficient order (the inverse pass leaves its first-phase layout)
        if (g == 0) {
            const uint64_t q0 = tab.q[0], q1 = tab.q[1], half = q1 >> 1;
            uint64_t* o = rs_out[b] + (size_t)comp * N + col;
#pragma unroll
            for (int k = 0; k < K; k++) {
                const uint64_t r1 = fin[(K + k) * NTG + r];
                const uint64_t lift = r1 > half ? q0 - (q1 - r1) : r1;
                o[(size_t)first_idx<LA, LT>(t, k) * N2] =
                    shoup(subm(fin[k * NTG + r], lift, q0), rc.q1inv.x, rc.q1inv.y, q0);
            }
        }
    }
}

// F5 of nb2 = (ciphertexts x 2 components) with ns <= MAXS special limbs: one thread
// group a special limb for the few column blocks of a small batch (latency-bound: the
// limbs' passes side by side), a single group looping over them for a batch that
// already fills the GPU (no idle groups).  Shared memory set once per variant.
template <int LA, int LB, int LT, int C, int GP, int MAXS, bool RS = false, bool MU = false>
cudaError_t f5_variant(uint32_t nb2, const uint64_t* acc, uint64_t* conv, const KsLevelConst* kc,
                       const DevTables& tab, uint32_t l1, uint32_t L, uint32_t ns, cudaStream_t s,
                       uint64_t* const* rs_out = nullptr, F5Rs rc = {}, F5Mu mu = {}) {
    constexpr int threads = GP * C * (1 << (LA - LT));
    constexpr size_t smem = 8 * f5_smem_words<LA, LT, C, GP, MAXS, RS || MU>();
    static const bool attrs = cudaFuncSetAttribute(k_ks_f5<LA, LB, LT, C, GP, MAXS, RS, MU>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                              cudaSuccess;
    (void)attrs;
    return pdl_launch(k_ks_f5<LA, LB, LT, C, GP, MAXS, RS, MU>, dim3(nb2, (1 << LB) / C), threads, smem, s, acc, conv,
                      kc, tab, l1, L, ns, rs_out, rc, mu);
}
constexpr uint32_t kF5SerialFrom = 16;    // ciphertext components from which F5 takes one group
template <int LA, int LB, int LT, int C, int MAXS>
cudaError_t f5_launch(uint32_t nb2, const uint64_t* acc, uint64_t* conv, const KsLevelConst* kc, const DevTables& tab,
                      uint32_t l1, uint32_t L, uint32_t ns, cudaStream_t s) {
    if (ns > (uint32_t)MAXS) return cudaErrorInvalidValue;
    if (nb2 >= kF5SerialFrom) return f5_variant<LA, LB, LT, C, 1, MAXS>(nb2, acc, conv, kc, tab, l1, L, ns, s);
    return f5_variant<LA, LB, LT, C, MAXS, MAXS>(nb2, acc, conv, kc, tab, l1, L, ns, s);
}

// ---------------------------------------------------------------------------
// F6: grid (B * l1, N1 / R).  out = (acc - conv) * P^-1 + sigma(c0) (+ add); without
// X0 and c0_of no sigma(c0) term (the sums of F4s hold it); with mask (a plaintext
// [l1][N], NTT + Montgomery) the result times it, the mask product of the compression
// taken here instead of in a launch of its own
// ---------------------------------------------------------------------------
template <int LA, int LB, int LT, int R>
__global__ void __launch_bounds__(R * (1 << (LB - LT)), LT <= 2 ? 8 : 3)
    k_ks_f6(const uint64_t* __restrict__ conv, const uint64_t* __restrict__ acc, const uint64_t* __restrict__ X0,
            uint64_t* const* out, uint64_t* const* add, const KsLevelConst* __restrict__ kc, DevTables tab,
            uint32_t l1, uint32_t galois, const uint64_t* const* c0_of, const uint64_t* gal_of,
            const uint64_t* __restrict__ mask) {
    constexpr int K = 1 << LT, M = 1 << LB, TH = M >> LT, S = sub_words<LB, LT>(), LOGN = LA + LB, N = 1 << LOGN;
    __shared__ uint64_t sm[R * S];
    __shared__ ulonglong2 tws[row_tw_entries<LB, R>()];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const uint32_t b = blockIdx.x / l1, j = blockIdx.x % l1;
    const uint64_t qn = tab.qneg[j];
    // hoisted rotations: each element has its own Galois element and reads sigma(c0)
    // from its source ciphertext (NTT form) instead of the copy X0
    if (gal_of) galois = (uint32_t)gal_of[b];
    // sums of hoisted rotations (F4s) carry their sigma(c0) terms already: no X0, no c0_of
    const uint64_t* x0 = c0_of ? c0_of[b] + (size_t)j * N : (X0 ? X0 + ((size_t)b * l1 + j) * N : nullptr);
    const uint32_t nlx = kc->nlx;
    const int row = blockIdx.y * R + jr;
    const size_t roff = (size_t)row * M;
    const uint64_t q = tab.q[j], q2 = 2 * q;
    const ulonglong2 pinv = kc->pinv[j];
    const RowBase<R> base{jr};
    const SubMem sr{sm + jr * S, 1};
    stage_row_twiddles<LA, LB, R, R * TH>(tws, tab.tw[j], blockIdx.y * R);
    pdl_wait();
    uint64_t v[K];
#pragma unroll 1
    for (int comp = 0; comp < 2; comp++) {
        const uint64_t* cv = conv + (((size_t)b * 2 + comp) * l1 + j) * N + roff;
#pragma unroll
        for (int k = 0; k < K; k++) v[k] = cv[first_idx<LB, LT>(t, k)];
        if (comp == 0) tw_wait();
        else __syncthreads();
        nttr::fwd_pass<LB, LT>(v, sr, tws, base, t, q, q2);
        uint64_t av[K], ad[K];
        nttr::load_last<LB, LT>(av, acc + (((size_t)b * 2 + comp) * nlx + j) * N + roff, t);
        if (add) nttr::load_last<LB, LT>(ad, add[b] + ((size_t)comp * l1 + j) * N + roff, t);
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int c = last_idx<LB, LT>(t, k);
            uint64_t o = shoup(subm(av[k], nttr::reduce4(v[k], q, q2), q), pinv.x, pinv.y, q);
            if (comp == 0 && x0) o = addm(o, x0[perm_src((uint32_t)(roff + c), LOGN, galois)], q);
            if (add) o = addm(o, ad[k], q);
            if (mask) o = mont(o, mask[(size_t)j * N + roff + c], q, qn);   // the ct x pt product after it
            v[k] = o;
        }
        nttr::relayout<LB, LT, LB / LT - 1, 0>(v, sr, t);
        uint64_t* o = out[b] + ((size_t)comp * l1 + j) * N + roff;
#pragma unroll
        for (int k = 0; k < K; k++) o[first_idx<LB, LT>(t, k)] = v[k];
    }
}

// ---------------------------------------------------------------------------
// F6u: grid (T * (2 l1 + nu), N1 / R), after F5's MU form.  Jobs of ciphertext b: the
// forward row pass of each quotient limb y [b][comp][j] into out[b] (the level-l1-1
// ciphertext in NTT form, the F6 of a plain division) and, for c1, into ext's digit
// limbs as well (the extension's own limbs are the ciphertext's NTT form); then the
// forward row pass of each converted limb of ext in place (as F3r).
// ---------------------------------------------------------------------------
template <int LA, int LB, int LT, int R>
__global__ void __launch_bounds__(R * (1 << (LB - LT)))
    k_ks_f6u(const uint64_t* __restrict__ Y, uint64_t* const* out, uint64_t* __restrict__ ext, uint64_t ext_words,
             DevTables tab, uint32_t l1, uint32_t nlu, uint32_t Lc) {
    constexpr int K = 1 << LT, M = 1 << LB, TH = M >> LT, S = sub_words<LB, LT>(), N = 1 << (LA + LB);
    __shared__ uint64_t sm[R * S];
    __shared__ ulonglong2 tws[row_tw_entries<LB, R>()];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const uint32_t jobs = 2 * l1 + (nlu - l1), b = blockIdx.x / jobs, job = blockIdx.x % jobs;
    const bool quot = job < 2 * l1;
    const uint32_t comp = quot ? job / l1 : 1, j = quot ? job % l1 : l1 + (job - 2 * l1);
    const int pi = j < l1 ? (int)j : (int)Lc + 1 + (int)(j - l1);
    const uint64_t q = tab.q[pi], q2 = 2 * q;
    const size_t roff = (size_t)(blockIdx.y * R + jr) * M;
    uint64_t* e = ext + (size_t)b * ext_words + (size_t)j * N + roff;
    const uint64_t* src = quot ? Y + (((size_t)b * 2 + comp) * l1 + j) * N + roff : e;
    stage_row_twiddles<LA, LB, R, R * TH>(tws, tab.tw[pi], blockIdx.y * R);
    pdl_wait();
    uint64_t v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = src[first_idx<LB, LT>(t, k)];
    tw_wait();
    nttr::fwd_pass<LB, LT>(v, SubMem{sm + jr * S, 1}, tws, RowBase<R>{jr}, t, q, q2);
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = nttr::reduce4(v[k], q, q2);
    pdl_trigger();
    if (quot) nttr::store_last<LB, LT>(v, out[b] + ((size_t)comp * l1 + j) * N + roff, t);
    if (!quot || comp == 1) nttr::store_last<LB, LT>(v, e, t);
}

// ---------------------------------------------------------------------------
// Rescale (Res of Sec. 2) in three kernels: out_j = (c_j - [c_l]_centred) * q_l^-1.
// R1: grid (B * 2, N1 / R): inverse row pass of limb l of each polynomial -> Y
// ---------------------------------------------------------------------------
template <int LA, int LB, int LT, int R>
__global__ void __launch_bounds__(R * (1 << (LB - LT)))
    k_rs_r1(uint64_t* const* in, uint64_t* __restrict__ Y, DevTables tab, uint32_t lvl) {
    constexpr int K = 1 << LT, M = 1 << LB, TH = M >> LT, S = sub_words<LB, LT>(), N = 1 << (LA + LB);
    __shared__ uint64_t sm[R * S];
    __shared__ ulonglong2 tws[row_tw_entries<LB, R>()];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const uint32_t b = blockIdx.x / 2, comp = blockIdx.x % 2;
    const int row = blockIdx.y * R + jr;
    const size_t roff = (size_t)row * M;
    const uint64_t q = tab.q[lvl], q2 = 2 * q;
    const uint64_t* src = in[b] + ((size_t)comp * (lvl + 1) + lvl) * N + roff;
    const SubMem sr{sm + jr * S, 1};
    stage_row_twiddles<LA, LB, R, R * TH>(tws, tab.itw[lvl], blockIdx.y * R);
    pdl_wait();
    uint64_t v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = src[first_idx<LB, LT>(t, k)];
    nttr::relayout<LB, LT, 0, LB / LT - 1>(v, sr, t);
    tw_wait();
    nttr::inv_pass<LB, LT>(v, sr, tws, RowBase<R>{jr}, t, q, q2);
    pdl_trigger();
    uint64_t* o = Y + (size_t)blockIdx.x * N + roff;
#pragma unroll
    for (int k = 0; k < K; k++) o[first_idx<LB, LT>(t, k)] = v[k];
}

// R2: grid (B * 2, N2 / C): inverse column pass -> centred lift -> forward column
// pass on every q_j, j < l -> Rl[b*2+comp][j]
template <int LA, int LB, int LT, int C>
__global__ void __launch_bounds__(C * (1 << (LA - LT)))
    k_rs_r2(const uint64_t* __restrict__ Y, uint64_t* __restrict__ Rl, DevTables tab, uint32_t lvl) {
    constexpr int K = 1 << LT, M = 1 << LA, N2 = 1 << LB, N = 1 << (LA + LB);
    __shared__ uint64_t sm[sub_words<LA, LT>() * C];
    __shared__ ulonglong2 tws[M];
    const int tid = threadIdx.x, t = tid / C, jc = tid % C;
    const int col = blockIdx.y * C + jc;
    const uint64_t ql = tab.q[lvl];
    const uint64_t* src = Y + (size_t)blockIdx.x * N + col;
    stage_col_twiddles<LA, C * (M >> LT)>(tws, tab.itw[lvl]);
    pdl_wait();
    uint64_t c[K];
#pragma unroll
    for (int k = 0; k < K; k++) c[k] = src[(size_t)last_idx<LA, LT>(t, k) * N2];
    tw_wait();
    nttr::inv_pass<LA, LT>(c, SubMem{sm + jc, C}, tws, ColBase{}, t, ql, 2 * ql);
    const uint64_t ni = tab.ninv[lvl], nis = tab.ninv_sh[lvl];
#pragma unroll
    for (int k = 0; k < K; k++) c[k] = shoup(c[k], ni, nis, ql);      // coefficients of limb l, [0, q_l)
    __syncthreads();
#pragma unroll 1
    for (uint32_t j = 0; j < lvl; j++) {
        const uint64_t qj = tab.q[j];
        stage_col_twiddles<LA, C * (M >> LT)>(tws, tab.tw[j]);
        uint64_t y[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const bool neg = c[k] > (ql >> 1);
            const uint64_t mag = neg ? ql - c[k] : c[k];
            const uint64_t r = reduce2(shoup_lazy(mag, 1, tab.rsh[j], qj), qj);
            y[k] = neg ? negm(r, qj) : r;
        }
        tw_wait();
        col_fwd_store<LA, LB, LT, C>(y, sm, tws, t, jc, qj, Rl + ((size_t)blockIdx.x * lvl + j) * N + col);
        __syncthreads();
    }
}

// R3: grid (B * 2 * l, N1 / R): forward row pass of Rl, out_j = (in_j - r_j) * q_l^-1
template <int LA, int LB, int LT, int R>
__global__ void __launch_bounds__(R * (1 << (LB - LT)))
    k_rs_r3(uint64_t* const* in, const uint64_t* __restrict__ Rl, uint64_t* const* out, DevTables tab, uint32_t lvl,
            const ulonglong2* __restrict__ qlinv) {
    constexpr int K = 1 << LT, M = 1 << LB, TH = M >> LT, S = sub_words<LB, LT>(), N = 1 << (LA + LB);
    __shared__ uint64_t sm[R * S];
    __shared__ ulonglong2 tws[row_tw_entries<LB, R>()];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const uint32_t y = blockIdx.x, b = y / (2 * lvl), comp = (y / lvl) % 2, j = y % lvl;
    const int row = blockIdx.y * R + jr;
    const size_t roff = (size_t)row * M;
    const uint64_t q = tab.q[j], q2 = 2 * q;
    const SubMem sr{sm + jr * S, 1};
    stage_row_twiddles<LA, LB, R, R * TH>(tws, tab.tw[j], blockIdx.y * R);
    pdl_wait();
    const uint64_t* r = Rl + ((size_t)(b * 2 + comp) * lvl + j) * N + roff;
    uint64_t v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = r[first_idx<LB, LT>(t, k)];
    tw_wait();
    nttr::fwd_pass<LB, LT>(v, sr, tws, RowBase<R>{jr}, t, q, q2);
    uint64_t x[K];
    nttr::load_last<LB, LT>(x, in[b] + ((size_t)comp * (lvl + 1) + j) * N + roff, t);
    const ulonglong2 w = qlinv[j];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = shoup(subm(x[k], nttr::reduce4(v[k], q, q2), q), w.x, w.y, q);
    nttr::relayout<LB, LT, LB / LT - 1, 0>(v, sr, t);
    pdl_trigger();
    uint64_t* o = out[b] + ((size_t)comp * lvl + j) * N + roff;
#pragma unroll
    for (int k = 0; k < K; k++) o[first_idx<LB, LT>(t, k)] = v[k];
}

template <int LA, int LB, int LT, int C, int R>
cudaError_t rescale_fused_launch(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in,
                                 uint64_t* const* d_out, uint64_t* scratch, cudaStream_t s) {
    constexpr int N1 = 1 << LA, N2 = 1 << LB, N = N1 * N2;
    uint64_t* Y = scratch;                          // [B*2][N]
    uint64_t* Rl = Y + (size_t)B * 2 * N;           // [B*2][level][N]
    const int tr = R * (1 << (LB - LT)), tc = C * (1 << (LA - LT));
    const double lw = 8.0 * N, bf_r = 16.0 * (N / 2) * LB, bf_c = 16.0 * (N / 2) * LA;
    {
        ProfScope ps(BM_KERNEL_RESCALE, s, lw * B * 2 * 2, bf_r * B * 2);
        pdl_launch(k_rs_r1<LA, LB, LT, R>, dim3(B * 2, N1 / R), tr, 0, s, d_in, Y, c.tab, level);
    }
    {
        ProfScope ps(BM_KERNEL_RESCALE, s, lw * B * 2 * (1 + level), bf_c * B * 2 * (1 + level));
        pdl_launch(k_rs_r2<LA, LB, LT, C>, dim3(B * 2, N2 / C), tc, 0, s, Y, Rl, c.tab, level);
    }
    {
        ProfScope ps(BM_KERNEL_RESCALE, s, lw * B * 2 * level * 3, bf_r * B * 2 * level);
        pdl_launch(k_rs_r3<LA, LB, LT, R>, dim3(B * 2 * level, N1 / R), tr, 0, s, d_in, Rl, d_out, c.tab, level,
                                                                          c.d_qlinv + (size_t)level * MAXB);
    }
    return cudaGetLastError();
}

template <int LA, int LB, int LT, int C, int R>
cudaError_t ks_fused_launch(const Context& c, const uint64_t* key, uint64_t galois, uint32_t level, uint32_t B,
                            uint64_t* const* d_in, uint64_t* const* d_out, uint64_t* const* d_add, uint64_t* scratch,
                            cudaStream_t s) {
    constexpr int N1 = 1 << LA, N2 = 1 << LB, N = N1 * N2;
    const KsLevelConst& K = c.h_ksc[level];
    const uint32_t l1 = level + 1, nd = K.nd, nlx = K.nlx, alpha = c.alpha;
    const KsLevelConst* kc = c.d_ksc + level;
    uint64_t* X0 = scratch;
    uint64_t* X1 = X0 + (size_t)B * l1 * N;
    uint64_t* ext = X1 + (size_t)B * l1 * N;
    uint64_t* acc = ext + (size_t)B * nd * nlx * N;
    uint64_t* conv = acc + (size_t)B * 2 * nlx * N;
    const int tr = R * (1 << (LB - LT)), tc = C * (1 << (LA - LT));
    const size_t col_smem = 8 * col_smem_words<LA, LT, C>();
    const size_t f4_smem2 = 8 * f4_smem_words<LB, LT, R, 2>(), f4_smem4 = 8 * f4_smem_words<LB, LT, R, MAXD>();
    static bool attrs = [&] {
        cudaFuncSetAttribute(k_ks_f3<LA, LB, LT, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem);
        cudaFuncSetAttribute(k_ks_f4<LA, LB, LT, R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f4_smem2);
        cudaFuncSetAttribute(k_ks_f4<LA, LB, LT, R, MAXD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)f4_smem4);
        return true;
    }();
    (void)attrs;
    const double lw = 8.0 * N;                                              // bytes of one limb
    const double bf_r = 16.0 * (N / 2) * LB, bf_c = 16.0 * (N / 2) * LA;    // mul ops of one limb pass
    uint32_t targets = 0, gathers = 0;
    for (uint32_t d = 0; d < nd; d++) {
        targets += nlx - K.dsz[d];
        gathers += K.dsz[d] * (nlx - K.dsz[d]);
    }
    {
        ProfScope ps(BM_KERNEL_NTT, s, lw * B * l1 * 6, bf_r * B * l1);
        pdl_launch(k_ks_f1<LA, LB, LT, R>, dim3(B * l1, N1 / R), tr, 0, s, d_in, X0, X1, ext, kc, c.tab, l1,
                                                                     (uint32_t)galois);
    }
    LimbBatch xb{X1, B, (uint64_t)l1 * N, 0, l1, 0};
    for (uint32_t k = 0; k < l1; k++) xb.set(k, k);
    cudaError_t e = ntt_col_inverse(c, xb, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(BM_KERNEL_MODUP, s, lw * B * (gathers + targets),
                     bf_c * B * targets + kShoupMul * N * B * (l1 + gathers));
        const uint32_t kinv = (uint32_t)h_invmod_pow2(galois, 2ull * N);
        const uint32_t ts_n = f3_slices(K, B, N2 / C);
        pdl_launch(k_ks_f3<LA, LB, LT, C>, dim3(B * nd * ts_n, N2 / C), tc, col_smem, s, X1, ext, kc, c.tab, l1, c.L,
                   kinv, ts_n);
    }
    {
        ProfScope ps(BM_KERNEL_KS_IP, s, lw * nlx * ((double)B * nd + 2.0 * nd + 2.0 * B),
                     bf_r * B * (targets + 2.0 * alpha) + N * B * nlx * 2.0 * (kProdMul * nd + kRedcMul));
        if (nd <= 2)
            pdl_launch(k_ks_f4<LA, LB, LT, R, 2>, dim3(B * nlx, N1 / R), tr, f4_smem2, s, ext, key, acc, kc, c.tab, l1,
                       c.L, c.nb);
        else
            pdl_launch(k_ks_f4<LA, LB, LT, R, MAXD>, dim3(B * nlx, N1 / R), tr, f4_smem4, s, ext, key, acc, kc, c.tab,
                       l1, c.L, c.nb);
    }
    {
        ProfScope ps(BM_KERNEL_MODDOWN, s, lw * B * 2 * (alpha + l1),
                     bf_c * B * 2 * (alpha + l1) + kShoupMul * N * B * 2 * (alpha + (double)l1 * alpha));
        f5_launch<LA, LB, LT, C, kMaxDigit>(B * 2, acc, conv, kc, c.tab, l1, c.L, alpha, s);
    }
    {
        ProfScope ps(BM_KERNEL_KS_COMBINE, s, lw * B * l1 * (2 + 2 + 1 + 2 + (d_add ? 2 : 0)),
                     bf_r * B * 2 * l1 + kShoupMul * N * B * 2 * l1);
        pdl_launch(k_ks_f6<LA, LB, LT, R>, dim3(B * l1, N1 / R), tr, 0, s, conv, acc, X0, d_out, d_add, kc, c.tab, l1,
                                                                     (uint32_t)galois, nullptr, nullptr, nullptr);
    }
    return cudaGetLastError();
}

// ModUp of c1 for B ciphertexts, every extended limb in NTT order: ext [B][nd][nlx][N].
// Scratch: X0, X1 ([B][l1][N] each; X0 receives an unused copy of c0).
template <int LA, int LB, int LT, int C, int R>
cudaError_t ks_modup_launch(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in, uint64_t* ext,
                            uint64_t* scratch, cudaStream_t s) {
    constexpr int N1 = 1 << LA, N2 = 1 << LB, N = N1 * N2;
    const KsLevelConst& K = c.h_ksc[level];
    const uint32_t l1 = level + 1, nd = K.nd, nlx = K.nlx;
    const KsLevelConst* kc = c.d_ksc + level;
    uint64_t* X0 = scratch;
    uint64_t* X1 = X0 + (size_t)B * l1 * N;
    const int tr = R * (1 << (LB - LT)), tc = C * (1 << (LA - LT));
    const size_t col_smem = 8 * col_smem_words<LA, LT, C>();
    static bool attrs = [&] {
        cudaFuncSetAttribute(k_ks_f3<LA, LB, LT, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem);
        return true;
    }();
    (void)attrs;
    const double lw = 8.0 * N, bf_r = 16.0 * (N / 2) * LB, bf_c = 16.0 * (N / 2) * LA;
    uint32_t targets = 0, gathers = 0;
    for (uint32_t d = 0; d < nd; d++) {
        targets += nlx - K.dsz[d];
        gathers += K.dsz[d] * (nlx - K.dsz[d]);
    }
    {
        ProfScope ps(BM_KERNEL_NTT, s, lw * B * l1 * 6, bf_r * B * l1);
        pdl_launch(k_ks_f1<LA, LB, LT, R>, dim3(B * l1, N1 / R), tr, 0, s, d_in, X0, X1, ext, kc, c.tab, l1, 1u);
    }
    LimbBatch xb{X1, B, (uint64_t)l1 * N, 0, l1, 0};
    for (uint32_t k = 0; k < l1; k++) xb.set(k, k);
    cudaError_t e = ntt_col_inverse(c, xb, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(BM_KERNEL_MODUP, s, lw * B * (gathers + targets),
                     bf_c * B * targets + kShoupMul * N * B * (l1 + gathers));
        const uint32_t ts_n = f3_slices(K, B, N2 / C);
        pdl_launch(k_ks_f3<LA, LB, LT, C>, dim3(B * nd * ts_n, N2 / C), tc, col_smem, s, X1, ext, kc, c.tab, l1, c.L,
                   1u, ts_n);
    }
    {
        ProfScope ps(BM_KERNEL_MODUP, s, lw * B * targets * 2, bf_r * B * targets);
        pdl_launch(k_ks_f3r<LA, LB, LT, R>, dim3(B * nd * nlx, N1 / R), tr, 0, s, ext, kc, c.tab, l1, c.L,
                   (const uint64_t* const*)nullptr);
    }
    return cudaGetLastError();
}

// The same extension from c1 in coefficient form, coef [B][l1][N] (the input before its
// forward NTT): F3 on coef directly and F3r, whose own-limb blocks copy the
// NTT-form limbs of d_in[b]'s c1 -- no F1 and no inverse column pass.
template <int LA, int LB, int LT, int C, int R>
cudaError_t ks_modup_coef_launch(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in,
                                 const uint64_t* coef, uint64_t* ext, cudaStream_t s) {
    constexpr int N1 = 1 << LA, N2 = 1 << LB, N = N1 * N2;
    const KsLevelConst& K = c.h_ksc[level];
    const uint32_t l1 = level + 1, nd = K.nd, nlx = K.nlx;
    const KsLevelConst* kc = c.d_ksc + level;
    const int tr = R * (1 << (LB - LT)), tc = C * (1 << (LA - LT));
    const size_t col_smem = 8 * col_smem_words<LA, LT, C>();
    static bool attrs = [&] {
        cudaFuncSetAttribute(k_ks_f3<LA, LB, LT, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem);
        return true;
    }();
    (void)attrs;
    const double lw = 8.0 * N, bf_r = 16.0 * (N / 2) * LB, bf_c = 16.0 * (N / 2) * LA;
    uint32_t targets = 0, gathers = 0;
    for (uint32_t d = 0; d < nd; d++) {
        targets += nlx - K.dsz[d];
        gathers += K.dsz[d] * (nlx - K.dsz[d]);
    }
    {
        ProfScope ps(BM_KERNEL_MODUP, s, lw * B * (gathers + targets),
                     bf_c * B * targets + kShoupMul * N * B * (l1 + gathers));
        const uint32_t ts_n = f3_slices(K, B, N2 / C);
        pdl_launch(k_ks_f3<LA, LB, LT, C>, dim3(B * nd * ts_n, N2 / C), tc, col_smem, s, coef, ext, kc, c.tab, l1, c.L,
                   1u, ts_n);
    }
    {
        ProfScope ps(BM_KERNEL_MODUP, s, lw * B * (targets * 2 + 2 * l1), bf_r * B * targets);
        pdl_launch(k_ks_f3r<LA, LB, LT, R>, dim3(B * nd * nlx, N1 / R), tr, 0, s, ext, kc, c.tab, l1, c.L,
                   (const uint64_t* const*)d_in);
    }
    return cudaGetLastError();
}

// E hoisted rotations: out[e] = Rot(src[e]) by Galois element gal_of[e] with key key_of[e],
// from the extension ext_of[e] of src[e]'s c1.  Scratch: acc, conv.
template <int LA, int LB, int LT, int C, int R>
cudaError_t ks_hoisted_launch(const Context& c, uint32_t level, uint32_t E, const uint64_t* const* ext_of,
                              const uint64_t* const* src, const uint64_t* const* key_of, const uint64_t* gal_of,
                              uint64_t* const* d_out, uint64_t* scratch, cudaStream_t s) {
    constexpr int N1 = 1 << LA, N2 = 1 << LB, N = N1 * N2;
    const KsLevelConst& K = c.h_ksc[level];
    const uint32_t l1 = level + 1, nd = K.nd, nlx = K.nlx, alpha = c.alpha;
    const KsLevelConst* kc = c.d_ksc + level;
    uint64_t* acc = scratch;
    uint64_t* conv = acc + (size_t)E * 2 * nlx * N;
    const int tr = R * (1 << (LB - LT));
    const double lw = 8.0 * N, bf_r = 16.0 * (N / 2) * LB, bf_c = 16.0 * (N / 2) * LA;
    {
        ProfScope ps(BM_KERNEL_KS_IP, s, lw * nlx * ((double)E * nd + 2.0 * nd * E + 2.0 * E),
                     bf_r * E * 2.0 * alpha + N * E * nlx * 2.0 * (kProdMul * nd + kRedcMul));
        pdl_launch(k_ks_f4h<LA, LB, LT, R>, dim3(E * nlx, N1 / R), tr, 0, s, ext_of, key_of, gal_of, acc, kc, c.tab, l1, c.L,
                                                                       c.nb);
    }
    {
        ProfScope ps(BM_KERNEL_MODDOWN, s, lw * E * 2 * (alpha + l1),
                     bf_c * E * 2 * (alpha + l1) + kShoupMul * N * E * 2 * (alpha + (double)l1 * alpha));
        f5_launch<LA, LB, LT, C, kMaxDigit>(E * 2, acc, conv, kc, c.tab, l1, c.L, alpha, s);
    }
    {
        ProfScope ps(BM_KERNEL_KS_COMBINE, s, lw * E * l1 * 7, bf_r * E * 2 * l1 + kShoupMul * N * E * 2 * l1);
        pdl_launch(k_ks_f6<LA, LB, LT, R>, dim3(E * l1, N1 / R), tr, 0, s, conv, acc, nullptr, d_out, nullptr, kc, c.tab, l1,
                                                                     0u, src, gal_of, nullptr);
    }
    return cudaGetLastError();
}

// Sums of hoisted rotations before ModDown (double hoisting), F4s: acc[t] for T
// targets, the elements of target t in [off[t], off[t+1]) rotating src_of[e] by
// gal_of[e] with key key_of[e] from the extension ext_of[e] of src_of[e]'s c1.
// Scratch: acc, then conv (ks_moddown_add), of T targets.
template <int LA, int LB, int LT, int C, int R>
cudaError_t ks_ipsum_launch(const Context& c, uint32_t level, uint32_t T, const uint64_t* off, uint32_t E,
                            const uint64_t* const* ext_of, const uint64_t* const* src_of,
                            const uint64_t* const* key_of, const uint64_t* gal_of, uint64_t* scratch, bool ntt_out,
                            KsSumInfo u, uint32_t tpad, const uint64_t* gmask, bool inv_all, cudaStream_t s) {
    constexpr int N1 = 1 << LA, N2 = 1 << LB, N = N1 * N2;
    (void)N2;
    const KsLevelConst& K = c.h_ksc[level];
    const uint32_t l1 = level + 1, nd = K.nd, nlx = K.nlx, alpha = c.alpha;
    const KsLevelConst* kc = c.d_ksc + level;
    const double lw = 8.0 * N, bf_r = 16.0 * (N / 2) * LB;
    // algorithmic bytes: every distinct extension (nd x nlx limbs), key slice (nd x 2 x
    // nlx limbs) and source c0 (l1 limbs) once, and the sums (2 x nlx limbs a target)
    const double ue = u.ext ? u.ext : E, uk = u.keys ? u.keys : E, us = u.srcs ? u.srcs : E;
    // with tpad the E_0 slots: each source's 2 l1 limbs read, 2 nlx written; with group
    // masks each mask's nlx limbs and each source's c1 limbs (its unrotated term)
    const double e0 = tpad ? (double)(T / tpad) * (2.0 * l1 + 2.0 * nlx) : 0.0;
    const double gm = gmask ? (double)u.masks * nlx + us * l1 : 0.0;
    ProfScope ps(BM_KERNEL_KS_IP, s, lw * (nlx * (ue * nd + 2.0 * nd * uk + 2.0 * T) + us * l1 + e0 + gm),
                 (ntt_out ? 0.0 : bf_r * T * 2.0 * alpha) +
                     N * (double)nlx * (2.0 * kProdMul * nd * E + 2.0 * kRedcMul * T) + (double)N * l1 * E * kProdMul);
    // R rows a block (64 threads); digits unrolled up to ND
    constexpr int RF = 256 >> LB;
    const dim3 g((T + (tpad ? T / tpad : 0)) * nlx, N1 / RF), b(RF * (1 << (LB - 2)));
    auto args = [&](auto kernel) {
        return pdl_launch(kernel, g, b, 0, s, ext_of, src_of, key_of, gal_of, off, scratch, kc, c.tab, l1, c.L, c.nb,
                          ntt_out, tpad, u.max_elems > 1, gmask, inv_all);
    };
    cudaError_t e = cudaErrorInvalidValue;
    // one digit, group masks: the software-pipelined loop (PF; the same 128 registers)
    const bool pf = gmask && nd <= 1;
    if (pf) {
        e = args(k_ks_f4s<LA, LB, RF, 1, 8, true, true>);
    } else if (gmask) {
        if (nd <= 1) e = args(k_ks_f4s<LA, LB, RF, 1, 8, true>);
        else if (nd <= 2) e = args(k_ks_f4s<LA, LB, RF, 2, 8, true>);
        else if (nd <= 4) e = args(k_ks_f4s<LA, LB, RF, 4, 4, true>);
    } else {
        if (nd <= 1) e = args(k_ks_f4s<LA, LB, RF, 1, 8, false>);
        else if (nd <= 2) e = args(k_ks_f4s<LA, LB, RF, 2, 8, false>);
        else if (nd <= 4) e = args(k_ks_f4s<LA, LB, RF, 4, 4, false>);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ModDown of the T sums in scratch and tgt[t] += the result, F5 + F6 (in place: F6
// reads each target word before writing it, and no sigma(c0) term -- F4s holds it);
// with d_out the sum tgt[t] + result goes to out[t] instead.
template <int LA, int LB, int LT, int C, int R>
cudaError_t ks_moddown_add_launch(const Context& c, uint32_t level, uint32_t T, uint64_t* const* d_tgt,
                                  uint64_t* const* d_out, uint64_t* scratch, const uint64_t* mask, cudaStream_t s) {
    constexpr int N1 = 1 << LA, N2 = 1 << LB, N = N1 * N2;
    const KsLevelConst& K = c.h_ksc[level];
    const uint32_t l1 = level + 1, nlx = K.nlx, alpha = c.alpha;
    const KsLevelConst* kc = c.d_ksc + level;
    uint64_t* acc = scratch;
    uint64_t* conv = acc + (size_t)T * 2 * nlx * N;
    const int tr = R * (1 << (LB - LT));
    const double lw = 8.0 * N, bf_r = 16.0 * (N / 2) * LB, bf_c = 16.0 * (N / 2) * LA;
    {
        ProfScope ps(BM_KERNEL_MODDOWN, s, lw * T * 2 * (alpha + l1),
                     bf_c * T * 2 * (alpha + l1) + kShoupMul * N * T * 2 * (alpha + (double)l1 * alpha));
        f5_launch<LA, LB, LT, C, kMaxDigit>(T * 2, acc, conv, kc, c.tab, l1, c.L, alpha, s);
    }
    {
        // with the mask: its l1 limbs once more, and a Montgomery product a word (20 mul32)
        ProfScope ps(BM_KERNEL_KS_COMBINE, s, lw * (T * l1 * 8 + (mask ? l1 : 0)),
                     bf_r * T * 2 * l1 + kShoupMul * N * T * 2 * l1 + (mask ? 20.0 * N * T * 2 * l1 : 0.0));
        pdl_launch(k_ks_f6<LA, LB, LT, R>, dim3(T * l1, N1 / R), tr, 0, s, conv, acc, nullptr, d_out ? d_out : d_tgt,
                   d_tgt, kc, c.tab, l1, 0u, nullptr, nullptr, mask);
    }
    return cudaGetLastError();
}

// ModDown and Rescale fused on T sums in the extended basis: e [T][2][nlx][N] (NTT
// form, every limb) divided by S = q_(L-drop+1) .. q_L * P into out[t] (level
// L - drop): the inverse row pass of the special limbs {q_(L-drop+1) .. q_L} u P, F5
// with that special set (l1 = L + 1 - drop targets, the dropped q-primes first among
// the specials) and F6 with S^-1 (constants c.d_ksc_mdr[drop - 1]).  Scratch: conv of T.
// (MAXS: F5's groups, one per special limb, alpha + drop <= MAXS; the fewer groups
// of one dropped prime keep that division's blocks smaller)
template <int LA, int LB, int LT, int C, int R, int MAXS>
cudaError_t ks_mdr_launch(const Context& c, uint32_t T, uint64_t* e, uint64_t* const* d_out, uint64_t* scratch,
                          uint32_t drop, cudaStream_t s) {
    constexpr int N1 = 1 << LA, N2 = 1 << LB, N = N1 * N2;
    const uint32_t nlx = c.L + 1 + c.alpha, ns = c.alpha + drop, L = c.L + 1 - drop;   // L: target limbs
    const KsLevelConst* kc = c.d_ksc_mdr + (drop - 1);
    uint64_t* conv = scratch;
    const int tr = R * (1 << (LB - LT));
    const double lw = 8.0 * N, bf_r = 16.0 * (N / 2) * LB, bf_c = 16.0 * (N / 2) * LA;
    {
        LimbBatch sb{e, T * 2, (uint64_t)nlx * N, L, ns, 0};
        for (uint32_t k = 0; k < ns; k++) sb.set(k, L + k);
        // the prelude of the fused ModDown (the part F4 does for a plain key switch): moddown class
        ProfScope ps(BM_KERNEL_MODDOWN, s, 2 * lw * T * 2 * ns, bf_r * T * 2 * ns);
        pdl_launch(nttr::k_row_inv<LA, LB, LT, R>, dim3(T * 2 * ns, N1 / R), tr, 0, s, sb, c.tab);
    }
    {
        ProfScope ps(BM_KERNEL_MODDOWN, s, lw * T * 2 * (ns + L),
                     bf_c * T * 2 * (ns + L) + kShoupMul * N * T * 2 * (ns + (double)L * ns));
        f5_launch<LA, LB, LT, C, MAXS>(T * 2, e, conv, kc, c.tab, L, L - 1, ns, s);   // special i at prime L + i
    }
    {
        ProfScope ps(BM_KERNEL_KS_COMBINE, s, lw * T * L * 6, bf_r * T * 2 * L + kShoupMul * N * T * 2 * L);
        pdl_launch(k_ks_f6<LA, LB, LT, R>, dim3(T * L, N1 / R), tr, 0, s, conv, e, nullptr, d_out, nullptr, kc, c.tab,
                   L, 0u, nullptr, nullptr, nullptr);
    }
    return cudaGetLastError();
}

// The deferred division (drop 2: S = q_(L-1) q_L P) and the quotient's hoisted ModUp at
// its level in three launches: the inverse row pass of every limb of the T sums (in
// place), F5 in its MU form (the division in the coefficient domain, the quotient's
// forward column passes and its c1's conversion to the level's special primes) and
// F6u (the row passes).  out[t] receives the quotient in NTT form -- the residues of
// ks_moddown_rescale's F5 + F6 -- and ext + t * ks_ext_words(c, L - 2) its extension --
// those of F1, the inverse column pass, F3 and F3r on out[t].  Scratch: y of T.
template <int LA, int LB, int LT, int C, int R>
cudaError_t ks_mdru_launch(const Context& c, uint32_t T, uint64_t* e, uint64_t* const* d_out, uint64_t* ext,
                           uint64_t* scratch, cudaStream_t s) {
    constexpr int N1 = 1 << LA, N2 = 1 << LB, N = N1 * N2;
    constexpr uint32_t drop = 2;
    const uint32_t nlx = c.L + 1 + c.alpha, ns = c.alpha + drop, l1 = c.L + 1 - drop, lc = l1 - 1;
    const KsLevelConst& KU = c.h_ksc[lc];
    const uint32_t nlu = KU.nlx;
    const int tr = R * (1 << (LB - LT));
    const double lw = 8.0 * N, bf_r = 16.0 * (N / 2) * LB, bf_c = 16.0 * (N / 2) * LA;
    {
        LimbBatch sb{e, T * 2, (uint64_t)nlx * N, 0, nlx, 0};
        for (uint32_t k = 0; k < nlx; k++) sb.set(k, (uint8_t)k);
        ProfScope ps(BM_KERNEL_MODDOWN, s, 2 * lw * T * 2 * nlx, bf_r * T * 2 * nlx);
        pdl_launch(nttr::k_row_inv<LA, LB, LT, R>, dim3(T * 2 * nlx, N1 / R), tr, 0, s, sb, c.tab);
    }
    {
        F5Rs rc{};
        for (uint32_t j = 0; j < l1; j++) {
            const uint64_t q = c.primes[j], ni = h_invmod(c.n % q, q);
            rc.ninv[j] = make_ulonglong2(ni, h_shoup_companion(ni, q));
            rc.pinv[j] = c.h_ksc_mdr[drop - 1].pinv[j];
        }
        F5Mu mu{scratch, ext, c.d_ksc + lc, ks_ext_words(c, lc), c.L};
        // reads every limb of the sums; writes the quotient and the converted limbs
        ProfScope ps(BM_KERNEL_MODDOWN, s, lw * T * (2 * nlx + 2 * l1 + (nlu - l1)),
                     bf_c * T * (2 * (ns + l1) + 2 * l1 + (nlu - l1)) +
                         kShoupMul * N * T * (2 * (ns + (double)l1 * ns + 2.0 * l1) + l1 * (1.0 + (nlu - l1))));
        f5_variant<LA, LB, LT, C, MAXSP, MAXSP, false, true>(T * 2, e, nullptr, c.d_ksc_mdr + (drop - 1), c.tab, l1,
                                                            l1 - 1, ns, s, nullptr, rc, mu);
    }
    {
        const uint32_t jobs = 2 * l1 + (nlu - l1);
        ProfScope ps(BM_KERNEL_KS_COMBINE, s, lw * T * (2 * jobs + l1), bf_r * T * jobs);
        pdl_launch(k_ks_f6u<LA, LB, LT, R>, dim3(T * jobs, N1 / R), tr, 0, s, (const uint64_t*)scratch, d_out, ext,
                   (uint64_t)ks_ext_words(c, lc), c.tab, l1, nlu, c.L);
    }
    return cudaGetLastError();
}

// a0 and the extension of the top-level queries' c1 (F0c, F0r): qin [Q][2][L+1][N] in
// coefficient form -> NTT form in place; ext [Q][nd][nlx][N] as ks_modup_hoisted_coef writes it
template <int LA, int LB, int LT, int C, int R>
cudaError_t ks_a0_modup_launch(const Context& c, uint32_t Q, uint64_t* qin, uint64_t* ext, cudaStream_t s) {
    constexpr int N1 = 1 << LA, N2 = 1 << LB, N = N1 * N2;
    const uint32_t level = c.L, l1 = level + 1;
    const KsLevelConst& K = c.h_ksc[level];
    const uint32_t nd = K.nd, nlx = K.nlx, n0 = Q * l1;
    const KsLevelConst* kc = c.d_ksc + level;
    const uint64_t qstride = (uint64_t)ct_words(c, level);
    const int tr = R * (1 << (LB - LT)), tc = C * (1 << (LA - LT));
    const size_t col_smem = 8 * col_smem_words<LA, LT, C>();
    static bool attrs = [&] {
        cudaFuncSetAttribute(k_ks_f0c<LA, LB, LT, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem);
        return true;
    }();
    (void)attrs;
    // every target of a digit in a block of its own while the column blocks alone would
    // not fill the GPU (as F3)
    const uint32_t ts_n = (uint64_t)Q * nd * (N2 / C) >= kF3FillBlocks ? 1 : nlx;
    const double lw = 8.0 * N, bf_r = 16.0 * (N / 2) * LB, bf_c = 16.0 * (N / 2) * LA;
    uint32_t gathers = 0;
    for (uint32_t d = 0; d < nd; d++) gathers += K.dsz[d] * (nlx - K.dsz[d]);
    {
        // c0's column pass; c1 read once per digit slice, every extended limb written
        ProfScope ps(BM_KERNEL_MODUP, s, lw * Q * (2.0 * l1 + l1 + nd * nlx),
                     bf_c * Q * (l1 + (double)nd * nlx) + kShoupMul * N * Q * (l1 + gathers));
        pdl_launch(k_ks_f0c<LA, LB, LT, C>, dim3(n0 + Q * nd * ts_n, N2 / C), tc, col_smem, s, qin, qstride, ext, kc,
                   c.tab, l1, c.L, n0, ts_n);
    }
    {
        ProfScope ps(BM_KERNEL_NTT, s, lw * Q * (2.0 * l1 + 2.0 * nd * nlx + l1), bf_r * Q * (l1 + (double)nd * nlx));
        pdl_launch(k_ks_f0r<LA, LB, LT, R>, dim3(n0 + Q * nd * nlx, N1 / R), tr, 0, s, qin, qstride, ext, kc, c.tab,
                   l1, c.L, n0);
    }
    return cudaGetLastError();
}

}  // namespace

size_t ks_modup_scratch_words(const Context& c, uint32_t level, uint32_t B) {
    return (size_t)2 * B * (level + 1) * c.n;
}
size_t ks_ext_words(const Context& c, uint32_t level) {
    size_t nd = 0;   // digits with a limb at or below the level (host-only contexts have no constants)
    for (auto& d : c.digits) nd += (!d.empty() && d[0] <= level);
    return nd * (level + 1 + c.alpha) * c.n;
}
size_t ks_hoisted_scratch_words(const Context& c, uint32_t level, uint32_t E) {
    const size_t nlx = level + 1 + c.alpha;
    return (size_t)E * c.n * (2 * nlx + 2 * (level + 1));
}

cudaError_t ks_modup_hoisted(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in, uint64_t* ext,
                             uint64_t* scratch, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    if (c.log_n == 16) return ks_modup_launch<8, 8, 2, 2, 2>(c, level, B, d_in, ext, scratch, s);
    if (c.log_n == 12) return ks_modup_launch<6, 6, 2, 8, 8>(c, level, B, d_in, ext, scratch, s);
    return cudaErrorInvalidValue;
}

cudaError_t ks_modup_hoisted_coef(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in,
                                  const uint64_t* coef, uint64_t* ext, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    if (c.log_n == 16) return ks_modup_coef_launch<8, 8, 2, 2, 2>(c, level, B, d_in, coef, ext, s);
    if (c.log_n == 12) return ks_modup_coef_launch<6, 6, 2, 8, 8>(c, level, B, d_in, coef, ext, s);
    return cudaErrorInvalidValue;
}

cudaError_t ks_rotate_hoisted(const Context& c, uint32_t level, uint32_t E, const uint64_t* const* ext_of,
                              const uint64_t* const* src, const uint64_t* const* key_of, const uint64_t* gal_of,
                              uint64_t* const* d_out, uint64_t* scratch, cudaStream_t s) {
    if (E == 0) return cudaSuccess;
    if (c.log_n == 16)
        return ks_hoisted_launch<8, 8, 2, 2, 2>(c, level, E, ext_of, src, key_of, gal_of, d_out, scratch, s);
    if (c.log_n == 12)
        return ks_hoisted_launch<6, 6, 2, 8, 8>(c, level, E, ext_of, src, key_of, gal_of, d_out, scratch, s);
    return cudaErrorInvalidValue;
}

cudaError_t ks_ipsum_hoisted(const Context& c, uint32_t level, uint32_t T, const uint64_t* off, uint32_t E,
                             const uint64_t* const* ext_of, const uint64_t* const* src_of,
                             const uint64_t* const* key_of, const uint64_t* gal_of, uint64_t* scratch,
                             cudaStream_t s, bool ntt_out, KsSumInfo u, uint32_t tpad, const uint64_t* gmask,
                             bool inv_all) {
    if (T == 0) return cudaSuccess;
    if (gmask && (ntt_out || tpad)) return cudaErrorInvalidValue;
    if (inv_all && ntt_out) return cudaErrorInvalidValue;
    if (c.log_n == 16)
        return ks_ipsum_launch<8, 8, 2, 2, 2>(c, level, T, off, E, ext_of, src_of, key_of, gal_of, scratch, ntt_out, u,
                                              tpad, gmask, inv_all, s);
    if (c.log_n == 12)
        return ks_ipsum_launch<6, 6, 2, 8, 8>(c, level, T, off, E, ext_of, src_of, key_of, gal_of, scratch, ntt_out, u,
                                              tpad, gmask, inv_all, s);
    return cudaErrorInvalidValue;
}

bool ks_mdr_supported(const Context& c, uint32_t drop) {
    // staging depth BM_MAX_P for one dropped prime, MAXSP = BM_MAX_P + 1 for two
    return ks_fused_supported(c) && drop >= 1 && drop <= (uint32_t)kMdrDrops && c.alpha + 1 <= BM_MAX_P &&
           c.L >= drop;
}
size_t ks_mdr_scratch_words(const Context& c, uint32_t T) { return (size_t)T * 2 * c.L * c.n; }

cudaError_t ks_moddown_rescale(const Context& c, uint32_t T, uint64_t* e, uint64_t* const* d_out, uint64_t* scratch,
                               cudaStream_t s, uint32_t drop) {
    if (T == 0) return cudaSuccess;
    if (!ks_mdr_supported(c, drop)) return cudaErrorInvalidValue;
    if (c.log_n == 16)
        return drop == 1 ? ks_mdr_launch<8, 8, 2, 2, 2, BM_MAX_P>(c, T, e, d_out, scratch, drop, s)
                         : ks_mdr_launch<8, 8, 2, 2, 2, MAXSP>(c, T, e, d_out, scratch, drop, s);
    if (c.log_n == 12)
        return drop == 1 ? ks_mdr_launch<6, 6, 2, 8, 8, BM_MAX_P>(c, T, e, d_out, scratch, drop, s)
                         : ks_mdr_launch<6, 6, 2, 8, 8, MAXSP>(c, T, e, d_out, scratch, drop, s);
    return cudaErrorInvalidValue;
}

cudaError_t ks_a0_modup(const Context& c, uint32_t Q, uint64_t* qin, uint64_t* ext, cudaStream_t s) {
    if (Q == 0) return cudaSuccess;
    if (c.log_n == 16) return ks_a0_modup_launch<8, 8, 2, 2, 2>(c, Q, qin, ext, s);
    if (c.log_n == 12) return ks_a0_modup_launch<6, 6, 2, 8, 8>(c, Q, qin, ext, s);
    return cudaErrorInvalidValue;
}

bool ks_mdru_supported(const Context& c) {
    // the quotient's level has one digit, its q-limbs, and at most MAXSP extended limbs
    // besides them (F5's thread groups take the conversions side by side); from the
    // digits themselves, so that host-only contexts (schedule estimates) answer too
    if (!ks_mdr_supported(c, 2) || c.L < 2) return false;
    const uint32_t lc = c.L - 2, l1 = lc + 1;
    uint32_t nd = 0, ds = 0, d0 = 0;
    for (const auto& dg : c.digits) {
        if (dg.empty() || dg[0] > lc) continue;
        nd++;
        d0 = dg[0];
        ds = 0;
        for (uint32_t x : dg) ds += (x <= lc);
    }
    return nd == 1 && d0 == 0 && ds == l1 && ds <= 2 && c.alpha <= (uint32_t)MAXSP;
}

cudaError_t ks_moddown_rescale_modup(const Context& c, uint32_t T, uint64_t* e, uint64_t* const* d_out,
                                     uint64_t* ext, uint64_t* scratch, cudaStream_t s) {
    if (T == 0) return cudaSuccess;
    if (!ks_mdru_supported(c)) return cudaErrorInvalidValue;
    if (c.log_n == 16) return ks_mdru_launch<8, 8, 2, 2, 2>(c, T, e, d_out, ext, scratch, s);
    if (c.log_n == 12) return ks_mdru_launch<6, 6, 2, 8, 8>(c, T, e, d_out, ext, scratch, s);
    return cudaErrorInvalidValue;
}

cudaError_t ks_moddown_add(const Context& c, uint32_t level, uint32_t T, uint64_t* const* d_tgt, uint64_t* scratch,
                           cudaStream_t s, uint64_t* const* d_out, const uint64_t* mask) {
    if (T == 0) return cudaSuccess;
    if (!d_tgt && !d_out) return cudaErrorInvalidValue;
    if (c.log_n == 16) return ks_moddown_add_launch<8, 8, 2, 2, 2>(c, level, T, d_tgt, d_out, scratch, mask, s);
    if (c.log_n == 12) return ks_moddown_add_launch<6, 6, 2, 8, 8>(c, level, T, d_tgt, d_out, scratch, mask, s);
    return cudaErrorInvalidValue;
}

cudaError_t ks_moddown_rescale_coef(const Context& c, uint32_t T, uint64_t* scratch, uint64_t* const* d_out,
                                    cudaStream_t s) {
    if (T == 0) return cudaSuccess;
    const uint32_t level = 1, l1 = 2, ns = c.alpha;
    if (!rescale_coef_supported(c) || c.L < level || ns > (uint32_t)kMaxDigit) return cudaErrorInvalidValue;
    F5Rs rc{};
    for (uint32_t j = 0; j < 2; j++) {
        const uint64_t q = c.primes[j], ni = h_invmod(c.n % q, q);
        rc.ninv[j] = make_ulonglong2(ni, h_shoup_companion(ni, q));
        rc.pinv[j] = c.h_ksc[level].pinv[j];
    }
    const uint64_t q0 = c.primes[0], q1i = h_invmod(c.primes[1] % q0, q0);
    rc.q1inv = make_ulonglong2(q1i, h_shoup_companion(q1i, q0));
    const uint32_t nlx = l1 + ns, nb2 = T * 2;
    const double N = (double)c.n, bf_c = 16.0 * (N / 2) * (c.log_n / 2);
    // reads every limb of each sum, writes one limb of each component
    ProfScope ps(BM_KERNEL_MODDOWN, s, 8.0 * N * nb2 * (nlx + 1),
                 bf_c * nb2 * (ns + l1) + kShoupMul * N * nb2 * (ns + (double)l1 * ns + 2.0 * l1 + 1));
    if (c.log_n == 16) {
        if (nb2 >= kF5SerialFrom)
            return f5_variant<8, 8, 2, 2, 1, kMaxDigit, true>(nb2, scratch, nullptr, c.d_ksc + level, c.tab, l1, c.L,
                                                             ns, s, d_out, rc);
        return f5_variant<8, 8, 2, 2, kMaxDigit, kMaxDigit, true>(nb2, scratch, nullptr, c.d_ksc + level, c.tab, l1,
                                                                 c.L, ns, s, d_out, rc);
    }
    if (c.log_n == 12) {
        if (nb2 >= kF5SerialFrom)
            return f5_variant<6, 6, 2, 8, 1, kMaxDigit, true>(nb2, scratch, nullptr, c.d_ksc + level, c.tab, l1, c.L,
                                                             ns, s, d_out, rc);
        return f5_variant<6, 6, 2, 8, kMaxDigit, kMaxDigit, true>(nb2, scratch, nullptr, c.d_ksc + level, c.tab, l1,
                                                                 c.L, ns, s, d_out, rc);
    }
    return cudaErrorInvalidValue;
}

cudaError_t rescale_fused(const Context& c, uint32_t level, uint32_t B, uint64_t* const* d_in,
                          uint64_t* const* d_out, uint64_t* scratch, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    if (c.log_n == 16) return rescale_fused_launch<8, 8, 2, 2, 2>(c, level, B, d_in, d_out, scratch, s);
    if (c.log_n == 12) return rescale_fused_launch<6, 6, 2, 8, 8>(c, level, B, d_in, d_out, scratch, s);
    return cudaErrorInvalidValue;
}

bool ks_fused_supported(const Context& c) {
    if (c.log_n != 12 && c.log_n != 16) return false;
    if (c.alpha > (uint32_t)kMaxDigit) return false;
    for (const auto& d : c.digits)
        if (d.size() > (size_t)kMaxDigit) return false;
    return true;
}

bool ks_has_wide(const Context& c) { return c.log_n == 16; }

cudaError_t ks_rotate_fused_shape(const Context& c, bool wide, const uint64_t* key, uint64_t galois,
                                  uint32_t level, uint32_t B, uint64_t* const* d_in, uint64_t* const* d_out,
                                  uint64_t* const* d_add, uint64_t* scratch, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    if (c.log_n == 16)
        return wide ? ks_fused_launch<8, 8, 4, 8, 8>(c, key, galois, level, B, d_in, d_out, d_add, scratch, s)
                    : ks_fused_launch<8, 8, 2, 2, 2>(c, key, galois, level, B, d_in, d_out, d_add, scratch, s);
    if (c.log_n == 12) return ks_fused_launch<6, 6, 2, 8, 8>(c, key, galois, level, B, d_in, d_out, d_add, scratch, s);
    return cudaErrorInvalidValue;
}

cudaError_t ks_rotate_fused(const Context& c, const uint64_t* key, uint64_t galois, uint32_t level, uint32_t B,
                            uint64_t* const* d_in, uint64_t* const* d_out, uint64_t* const* d_add, uint64_t* scratch,
                            cudaStream_t s) {
    // few ciphertexts: 4 coefficients per thread (more warps hide the latency);
    // many: 16 per thread (fewer shared-memory exchanges) -- the per-level
    // threshold is the tuner's (or the caller's) choice
    const bool wide = level < BM_MAX_Q && B >= c.ks_wide_batch[level];
    return ks_rotate_fused_shape(c, wide, key, galois, level, B, d_in, d_out, d_add, scratch, s);
}

}  // namespace bm
