// noalloc.cu -- a rotation entry point that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: a host whose device memory
// is owned by its own pool allocator (a framework caching allocator sized to the
// whole GPU, where a foreign cudaMalloc fails or fragments the pool), or a
// latency-critical serving loop that forbids any allocation after start-up,
// where cudaMalloc's implicit synchronisation would stall the device.
// bm_ct_rotate_noalloc serves them: it does the same work as bm_ct_rotate
// (automorphism + hybrid key switch) on device buffers the caller provides,
// and keeps its temporaries in the file-scope array below, which the CUDA
// runtime places on every device that loads this code and keeps until exit.
#include <cuda_runtime.h>

#include <mutex>

#include "bm_internal.h"

namespace bm {
namespace {

// 32 MiB: one ring-2^16 ciphertext at level 3, or proportionally more at lower
// levels / smaller rings (input copy + key-switch temporaries + pointer lists).
constexpr size_t kScratchWords = (size_t)4 << 20;
constexpr uint32_t kMaxCts = 64;
constexpr size_t kListWords = 2 * kMaxCts;     // in/out pointer arrays, 1 KiB (keeps 256-byte alignment)

static __device__ __align__(256) uint64_t g_rotate_scratch[kScratchWords];

std::mutex g_mu;
uint64_t* g_addr[256] = {};

// Device address of g_rotate_scratch on `device` (which must be current); the
// symbol's name in host code is only a host-side stand-in, so its address is
// looked up once per device and cached for the life of the process (a
// cudaDeviceReset reloads the module and may move the array: calls after one
// are not supported).
cudaError_t scratch_address(int device, uint64_t** out) {
    std::lock_guard<std::mutex> g(g_mu);
    if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
    if (!g_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rotate_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = (uint64_t*)p;
    }
    *out = g_addr[device];
    return cudaSuccess;
}

// The in/out pointer lists of the key switch, written on the device from values
// passed by value (no host staging buffer, so nothing is read from host memory
// after the call returns).
__global__ void k_noalloc_lists(uint64_t** lists, uint64_t* work, uint64_t* out, size_t cw, uint32_t n) {
    const uint32_t b = threadIdx.x;
    if (b < n) {
        lists[b] = work + b * cw;
        lists[kMaxCts + b] = out + b * cw;
    }
}

// Restores the caller's current device on every return path.
struct DeviceGuard {
    int prev = -1;
    DeviceGuard() {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" bm_status bm_ct_rotate_noalloc(bm_context* ctxh, const bm_eval_keys* evk, const uint64_t* d_in,
                                          uint32_t n_cts, uint32_t level, int32_t rotation, uint64_t* d_out,
                                          void* stream) {
    if (!ctxh || !evk || !d_in || !d_out || n_cts == 0) {
        set_error("bm_ct_rotate_noalloc: null argument or no ciphertexts");
        return BM_E_ARG;
    }
    const Context& c = ctxh->c;
    if (level > c.L) {
        set_error("bm_ct_rotate_noalloc: level above the modulus chain");
        return BM_E_LEVEL;
    }
    const size_t cw = ct_words(c, level);
    const size_t need = kListWords + (size_t)n_cts * cw + ks_scratch_words(c, level, n_cts);
    if (n_cts > kMaxCts || need > kScratchWords) {
        set_error("bm_ct_rotate_noalloc: " + std::to_string(n_cts) + " ciphertexts at level " +
                  std::to_string(level) + " need " + std::to_string(need * 8) + " bytes of scratch; the limit is " +
                  std::to_string(kScratchWords * 8) + " bytes and " + std::to_string(kMaxCts) + " ciphertexts");
        return BM_E_ARG;
    }
    auto it = evk->k.keys.find(galois_of(c, rotation));
    if (it == evk->k.keys.end()) {
        set_error("bm_ct_rotate_noalloc: no key for this rotation");
        return BM_E_KEY_MISSING;
    }
    cudaStream_t s = (cudaStream_t)stream;
    DeviceGuard keep_device;
    BM_CUDA_TRY(cudaSetDevice(c.device));
    uint64_t* base = nullptr;
    BM_CUDA_TRY(scratch_address(c.device, &base));
    uint64_t** lists = (uint64_t**)base;               // [in pointers][out pointers]
    uint64_t* work = base + kListWords;                // NTT-form copy of the inputs
    uint64_t* ks = work + (size_t)n_cts * cw;          // key-switch temporaries
    k_noalloc_lists<<<1, kMaxCts, 0, s>>>(lists, work, d_out, cw, n_cts);
    BM_CUDA_TRY(cudaGetLastError());
    BM_CUDA_TRY(cudaMemcpyAsync(work, d_in, n_cts * cw * 8, cudaMemcpyDeviceToDevice, s));
    LimbBatch all{work, n_cts * 2, (uint64_t)(level + 1) * c.n, 0, level + 1, {}};
    for (uint32_t k = 0; k <= level; k++) all.set(k, (uint8_t)k);
    BM_CUDA_TRY(ntt_forward(c, all, s));
    BM_CUDA_TRY(ks_rotate(c, it->second, galois_of(c, rotation), level, n_cts, lists, lists + kMaxCts, nullptr, ks, s));
    LimbBatch outb = all;
    outb.base = d_out;
    BM_CUDA_TRY(ntt_inverse(c, outb, s));
    return BM_OK;
}
