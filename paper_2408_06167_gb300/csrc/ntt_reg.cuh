// ntt_reg.cuh -- register-resident NTT passes (included by kernels.cu).
//
// The negacyclic NTT of one limb (N = N1 * N2, N1 = 2^LA, N2 = 2^LB) is the
// Cooley-Tukey network with bit-reversed psi twiddles; stage s pairs indices
// j and j + N/2^(s+1) with twiddle W[2^s + j / (N/2^s)].  Stages 0..LA-1 act on
// columns of the N1 x N2 view (a "column pass"), stages LA..log N-1 on rows (a
// "row pass").  Inside a pass each sub-transform has M = 2^P points (P even) and
// is handled by E = 2^(P/2) threads holding E coefficients each:
//   phase 1 (first P/2 stages, pair distance >= E): thread t holds the
//            coefficients t + E*k, k < E ("stride" layout);
//   phase 2 (last P/2 stages, distance < E): thread t holds E*t + k
//            ("consecutive" layout);
// so each pass needs a single exchange through shared memory (padded by one
// word per E so both layouts are bank-conflict free) instead of a barrier per
// stage.  Butterflies are Harvey's lazy forms: forward keeps values in [0, 4q),
// inverse in [0, 2q); the last pass of each transform reduces to [0, q).
#pragma once

#include <cuda_pipeline.h>

namespace bm {

// Programmatic dependent launch (the kernels of the match path are launched with
// pdl_launch): a kernel may be scheduled while the previous kernel of its stream
// drains.  pdl_wait() blocks until that kernel has completed and its writes are
// visible -- every such kernel calls it before its first read of data the
// previous kernels wrote and before its first global write; only constant
// context tables (twiddles, primes) are read before it.  pdl_trigger() lets the
// next kernel be scheduled once every block of this one has reached it; both
// are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// launch with the programmatic-serialization attribute (off with BM_PDL=0)
bool pdl_enabled();
template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

namespace nttr {

__device__ __forceinline__ uint64_t* limb_at(const LimbBatch& b, uint32_t limb, uint32_t n) {
    const uint32_t poly = limb / b.nl, k = limb % b.nl;
    return b.base + (size_t)poly * b.poly_stride + (size_t)(b.limb_off + k) * n;
}

// x, y in [0, 4q) -> x + w y, x - w y in [0, 4q)
__device__ __forceinline__ void ct_bfly(uint64_t& x, uint64_t& y, const ulonglong2 w, uint64_t q, uint64_t q2) {
    const uint64_t a = x >= q2 ? x - q2 : x;
    const uint64_t t = shoup_lazy(y, w.x, w.y, q);
    x = a + t;
    y = a - t + q2;
}

// x, y in [0, 2q) -> x + y, (x - y) w in [0, 2q)
__device__ __forceinline__ void gs_bfly(uint64_t& x, uint64_t& y, const ulonglong2 w, uint64_t q, uint64_t q2) {
    uint64_t a = x + y;
    a = a >= q2 ? a - q2 : a;
    const uint64_t t = x - y + q2;
    x = a;
    y = shoup_lazy(t, w.x, w.y, q);
}

__device__ __forceinline__ uint64_t reduce4(uint64_t x, uint64_t q, uint64_t q2) {
    x = x >= q2 ? x - q2 : x;
    return x >= q ? x - q : x;
}

// One stage, compile-time: pairs (k, k + hk) within blocks of 2*hk registers;
// block blk uses twiddle tw[first + blk].
template <int E, int HK, bool FWD>
__device__ __forceinline__ void stage(uint64_t (&v)[E], const ulonglong2* __restrict__ tw, int first, uint64_t q,
                                      uint64_t q2) {
#pragma unroll
    for (int blk = 0; blk < E / (2 * HK); blk++) {
        const ulonglong2 w = tw[first + blk];
#pragma unroll
        for (int j = 0; j < HK; j++) {
            if constexpr (FWD) ct_bfly(v[blk * 2 * HK + j], v[blk * 2 * HK + j + HK], w, q, q2);
            else gs_bfly(v[blk * 2 * HK + j], v[blk * 2 * HK + j + HK], w, q, q2);
        }
    }
}

// A 2^P-point sub-transform is processed by 2^(P-LT) threads holding 2^LT
// registers each, in P/LT phases of LT stages.  In phase h thread t holds the
// elements pidx(h, t, k) = ((t >> lb) << (lb + LT)) | (k << lb) | (t mod 2^lb),
// lb = P - LT*(h+1), so stage s = LT*h + s' pairs registers k and k + 2^(LT-1-s')
// and its block blk (= k >> (LT - s')) uses twiddle W[base(s) + ((t >> lb) << s') + blk].
// Phase 0 is the "stride" layout (t + 2^(P-LT) k), the last phase the
// "consecutive" one (2^LT t + k).
template <int P, int LT, int h>
__device__ __forceinline__ int pidx(int t, int k) {
    constexpr int lb = P - LT * (h + 1);
    return ((t >> lb) << (lb + LT)) | (k << lb) | (t & ((1 << lb) - 1));
}

// padded shared-memory index (one spare word per 2^LT): keeps every phase layout
// within two wavefronts per warp access
template <int LT>
__device__ __forceinline__ int padx(int x) { return x + (x >> LT); }
template <int P, int LT>
__host__ __device__ constexpr int sub_words() { return (1 << P) + ((1 << P) >> LT); }

// Shared-memory view of one sub-transform: element x at base[padx(x) * stride].
struct SubMem {
    uint64_t* base;
    int stride;
    __device__ __forceinline__ uint64_t& operator[](int px) const { return base[px * stride]; }
};

template <int P, int LT, int h, int S = 0, typename BaseF>
__device__ __forceinline__ void fwd_phase(uint64_t (&v)[1 << LT], const ulonglong2* __restrict__ tw, BaseF base,
                                          int t, uint64_t q, uint64_t q2) {
    if constexpr (S < LT) {
        constexpr int lb = P - LT * (h + 1);
        stage<1 << LT, (1 << (LT - 1 - S)), true>(v, tw, base(LT * h + S) + ((t >> lb) << S), q, q2);
        fwd_phase<P, LT, h, S + 1>(v, tw, base, t, q, q2);
    }
}

template <int P, int LT, int h, int S = LT - 1, typename BaseF>
__device__ __forceinline__ void inv_phase(uint64_t (&v)[1 << LT], const ulonglong2* __restrict__ tw, BaseF base,
                                          int t, uint64_t q, uint64_t q2) {
    if constexpr (S >= 0) {
        constexpr int lb = P - LT * (h + 1);
        stage<1 << LT, (1 << (LT - 1 - S)), false>(v, tw, base(LT * h + S) + ((t >> lb) << S), q, q2);
        inv_phase<P, LT, h, S - 1>(v, tw, base, t, q, q2);
    }
}

// Moves v from phase-h1 layout to phase-h2 layout through shared memory (one
// barrier).  Safe back to back: each thread only overwrites positions it read.
template <int P, int LT, int h1, int h2>
__device__ __forceinline__ void relayout(uint64_t (&v)[1 << LT], const SubMem& sm, int t) {
#pragma unroll
    for (int k = 0; k < (1 << LT); k++) sm[padx<LT>(pidx<P, LT, h1>(t, k))] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < (1 << LT); k++) v[k] = sm[padx<LT>(pidx<P, LT, h2>(t, k))];
}

// All forward stages: v in phase-0 layout on entry, last-phase layout on exit.
template <int P, int LT, int h = 0, typename BaseF>
__device__ __forceinline__ void fwd_pass(uint64_t (&v)[1 << LT], const SubMem& sm, const ulonglong2* __restrict__ tw,
                                         BaseF base, int t, uint64_t q, uint64_t q2) {
    fwd_phase<P, LT, h>(v, tw, base, t, q, q2);
    if constexpr (h + 1 < P / LT) {
        relayout<P, LT, h, h + 1>(v, sm, t);
        fwd_pass<P, LT, h + 1>(v, sm, tw, base, t, q, q2);
    }
}

// All inverse stages: v in last-phase layout on entry, phase-0 layout on exit.
template <int P, int LT, int h = P / LT - 1, typename BaseF>
__device__ __forceinline__ void inv_pass(uint64_t (&v)[1 << LT], const SubMem& sm, const ulonglong2* __restrict__ tw,
                                         BaseF base, int t, uint64_t q, uint64_t q2) {
    inv_phase<P, LT, h>(v, tw, base, t, q, q2);
    if constexpr (h > 0) {
        relayout<P, LT, h, h - 1>(v, sm, t);
        inv_pass<P, LT, h - 1>(v, sm, tw, base, t, q, q2);
    }
}

template <int P, int LT>
__device__ __forceinline__ int first_idx(int t, int k) { return pidx<P, LT, 0>(t, k); }
template <int P, int LT>
__device__ __forceinline__ int last_idx(int t, int k) { return pidx<P, LT, P / LT - 1>(t, k); }

// In the last-phase layout of a pass over 2^P contiguous words (P a multiple of
// LT), thread t holds the 2^LT consecutive words at t * 2^LT: moved as 16-byte
// vectors (the row is 256-byte aligned, so every vector is 16-byte aligned).
template <int P, int LT>
__device__ __forceinline__ void store_last(const uint64_t (&v)[1 << LT], uint64_t* __restrict__ row, int t) {
    static_assert(P % LT == 0, "last phase must start at a multiple of the thread's run");
    ulonglong2* p = reinterpret_cast<ulonglong2*>(row + (t << LT));
#pragma unroll
    for (int k = 0; k < (1 << LT) / 2; k++) p[k] = make_ulonglong2(v[2 * k], v[2 * k + 1]);
}

template <int P, int LT>
__device__ __forceinline__ void load_last(uint64_t (&v)[1 << LT], const uint64_t* __restrict__ row, int t) {
    static_assert(P % LT == 0, "last phase must start at a multiple of the thread's run");
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(row + (t << LT));
#pragma unroll
    for (int k = 0; k < (1 << LT) / 2; k++) {
        const ulonglong2 w = p[k];
        v[2 * k] = w.x;
        v[2 * k + 1] = w.y;
    }
}

// Twiddles a column pass uses: entries 1 .. 2^LA - 1 of the table, copied to
// shared memory (index unchanged) with asynchronous copies issued all at once by
// the T threads of the CTA; wait with tw_wait() before use.
template <int LA, int T>
__device__ __forceinline__ void stage_col_twiddles(ulonglong2* dst, const ulonglong2* __restrict__ tw) {
#pragma unroll
    for (int i0 = 0; i0 < (1 << LA); i0 += T) {
        const int i = i0 + (int)threadIdx.x;
        if (i < (1 << LA)) __pipeline_memcpy_async(dst + i, tw + i, sizeof(ulonglong2));
    }
    __pipeline_commit();
}

// Twiddles of a row pass over rows r0 .. r0+R-1: stage s uses the global entries
// 2^(LA+s) + r*2^s + [0, 2^s), contiguous over the R rows; copied to
// R*(2^s - 1) + (r - r0)*2^s + [0, 2^s).
template <int LA, int LB, int R, int T>
__device__ __forceinline__ void stage_row_twiddles(ulonglong2* dst, const ulonglong2* __restrict__ tw, int r0) {
#pragma unroll
    for (int s = 0; s < LB; s++) {
        const ulonglong2* src = tw + (1 << (LA + s)) + r0 * (1 << s);
        ulonglong2* d = dst + R * ((1 << s) - 1);
#pragma unroll
        for (int i0 = 0; i0 < (R << s); i0 += T) {
            const int i = i0 + (int)threadIdx.x;
            if (i < (R << s)) __pipeline_memcpy_async(d + i, src + i, sizeof(ulonglong2));
        }
    }
    __pipeline_commit();
}

// completes this thread's staged copies and makes every thread's visible
__device__ __forceinline__ void tw_wait() {
    __pipeline_wait_prior(0);
    __syncthreads();
}

template <int LB, int R>
__host__ __device__ constexpr int row_tw_entries() { return R * ((1 << LB) - 1); }

// base(s) of a row pass on staged twiddles, local row jr
template <int R>
struct RowBase {
    int jr;
    __device__ __forceinline__ int operator()(int s) const { return R * ((1 << s) - 1) + jr * (1 << s); }
};
struct ColBase {
    __device__ __forceinline__ int operator()(int s) const { return 1 << s; }
};

// ---------------------------------------------------------------------------
// pass kernels on a LimbBatch; grid (limbs, tiles)
// ---------------------------------------------------------------------------

// Column pass, forward: global stages 0..LA-1 on C columns.  Output lazy [0, 4q).
template <int LA, int LB, int LT, int C>
__global__ void __launch_bounds__(C * (1 << (LA - LT))) k_col_fwd(LimbBatch lb, DevTables tab) {
    constexpr int K = 1 << LT, M = 1 << LA, N2 = 1 << LB;
    __shared__ uint64_t sm[sub_words<LA, LT>() * C];
    __shared__ ulonglong2 tws[M];
    const int tid = threadIdx.x, t = tid / C, j = tid % C;
    const int pi = lb.prime(blockIdx.x % lb.nl);
    uint64_t* a = limb_at(lb, blockIdx.x, M * N2) + blockIdx.y * C + j;
    const uint64_t q = tab.q[pi], q2 = 2 * q;
    stage_col_twiddles<LA, C * (M >> LT)>(tws, tab.tw[pi]);
    pdl_wait();
    uint64_t v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = a[(size_t)first_idx<LA, LT>(t, k) * N2];
    tw_wait();
    fwd_pass<LA, LT>(v, SubMem{sm + j, C}, tws, ColBase{}, t, q, q2);
    pdl_trigger();
#pragma unroll
    for (int k = 0; k < K; k++) a[(size_t)last_idx<LA, LT>(t, k) * N2] = v[k];
}

// Row pass, forward: global stages LA..LA+LB-1 on R rows.  Input [0, 4q), output [0, q).
template <int LA, int LB, int LT, int R>
__global__ void __launch_bounds__(R * (1 << (LB - LT))) k_row_fwd(LimbBatch lb, DevTables tab) {
    constexpr int K = 1 << LT, M = 1 << LB, TH = M >> LT, S = sub_words<LB, LT>();
    __shared__ uint64_t sm[R * S];
    __shared__ ulonglong2 tws[row_tw_entries<LB, R>()];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const int row = blockIdx.y * R + jr;
    const int pi = lb.prime(blockIdx.x % lb.nl);
    uint64_t* a = limb_at(lb, blockIdx.x, (1 << LA) * M) + (size_t)row * M;
    const uint64_t q = tab.q[pi], q2 = 2 * q;
    const SubMem sr{sm + jr * S, 1};
    stage_row_twiddles<LA, LB, R, R * TH>(tws, tab.tw[pi], blockIdx.y * R);
    pdl_wait();
    uint64_t v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = a[first_idx<LB, LT>(t, k)];
    tw_wait();
    fwd_pass<LB, LT>(v, sr, tws, RowBase<R>{jr}, t, q, q2);
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = reduce4(v[k], q, q2);
    relayout<LB, LT, LB / LT - 1, 0>(v, sr, t);
    pdl_trigger();
#pragma unroll
    for (int k = 0; k < K; k++) a[first_idx<LB, LT>(t, k)] = v[k];
}

// Row pass, inverse: global stages LA+LB-1..LA on R rows.  Input [0, 2q), output [0, 2q).
template <int LA, int LB, int LT, int R>
__global__ void __launch_bounds__(R * (1 << (LB - LT))) k_row_inv(LimbBatch lb, DevTables tab) {
    constexpr int K = 1 << LT, M = 1 << LB, TH = M >> LT, S = sub_words<LB, LT>();
    __shared__ uint64_t sm[R * S];
    __shared__ ulonglong2 tws[row_tw_entries<LB, R>()];
    const int tid = threadIdx.x, jr = tid / TH, t = tid % TH;
    const int row = blockIdx.y * R + jr;
    const int pi = lb.prime(blockIdx.x % lb.nl);
    uint64_t* a = limb_at(lb, blockIdx.x, (1 << LA) * M) + (size_t)row * M;
    const uint64_t q = tab.q[pi], q2 = 2 * q;
    const SubMem sr{sm + jr * S, 1};
    stage_row_twiddles<LA, LB, R, R * TH>(tws, tab.itw[pi], blockIdx.y * R);
    pdl_wait();
    uint64_t v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = a[first_idx<LB, LT>(t, k)];
    relayout<LB, LT, 0, LB / LT - 1>(v, sr, t);
    tw_wait();
    inv_pass<LB, LT>(v, sr, tws, RowBase<R>{jr}, t, q, q2);
    pdl_trigger();
#pragma unroll
    for (int k = 0; k < K; k++) a[first_idx<LB, LT>(t, k)] = v[k];
}

// Column pass, inverse: global stages LA-1..0 on C columns, then * N^-1.  Output [0, q).
template <int LA, int LB, int LT, int C>
__global__ void __launch_bounds__(C * (1 << (LA - LT))) k_col_inv(LimbBatch lb, DevTables tab) {
    constexpr int K = 1 << LT, M = 1 << LA, N2 = 1 << LB;
    __shared__ uint64_t sm[sub_words<LA, LT>() * C];
    __shared__ ulonglong2 tws[M];
    const int tid = threadIdx.x, t = tid / C, j = tid % C;
    const int pi = lb.prime(blockIdx.x % lb.nl);
    uint64_t* a = limb_at(lb, blockIdx.x, M * N2) + blockIdx.y * C + j;
    const uint64_t q = tab.q[pi], q2 = 2 * q;
    stage_col_twiddles<LA, C * (M >> LT)>(tws, tab.itw[pi]);
    pdl_wait();
    uint64_t v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = a[(size_t)last_idx<LA, LT>(t, k) * N2];
    tw_wait();
    inv_pass<LA, LT>(v, SubMem{sm + j, C}, tws, ColBase{}, t, q, q2);
    pdl_trigger();
    const uint64_t ni = tab.ninv[pi], nis = tab.ninv_sh[pi];
#pragma unroll
    for (int k = 0; k < K; k++) a[(size_t)first_idx<LA, LT>(t, k) * N2] = shoup(v[k], ni, nis, q);
}

}  // namespace nttr
}  // namespace bm
