// profile.cpp -- per-kernel-class launch accounting of the Blind-Match library.
//
// Counts launches and algorithmic bytes for every kernel class, and (when
// enabled) times each launch with a CUDA event pair on the launching stream;
// read back through bm_profile_read.  Process-wide; meant for one context at a
// time on one device.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "bm_internal.h"

namespace bm {
namespace {

struct Pending {
    int kind;
    cudaEvent_t a, b;
};

struct Profiler {
    std::mutex mu;
    bool timing = false;
    uint64_t launches[BM_KERNEL_KINDS] = {};
    double bytes[BM_KERNEL_KINDS] = {};
    double ops[BM_KERNEL_KINDS] = {};
    double ms[BM_KERNEL_KINDS] = {};
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;

    cudaEvent_t get_event() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void resolve() {
        for (auto& p : pending) {
            float t = 0.f;
            if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess)
                ms[p.kind] += t;
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
};

Profiler& prof() {
    static Profiler p;
    return p;
}

thread_local ProfSink* t_sink = nullptr;

}  // namespace

void prof_set_sink(ProfSink* sink) { t_sink = sink; }

void prof_add(const ProfSink& counts) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    for (int k = 0; k < BM_KERNEL_KINDS; k++) {
        p.launches[k] += counts.launches[k];
        p.bytes[k] += counts.bytes[k];
        p.ops[k] += counts.ops[k];
    }
}

bool prof_timing() {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    return p.timing;
}

ProfScope::ProfScope(int k, cudaStream_t st, double alg_bytes, double alg_ops, uint32_t n)
    : kind(k), s(st), slot(-1) {
    if (t_sink) {
        t_sink->launches[kind] += n;
        t_sink->bytes[kind] += alg_bytes;
        t_sink->ops[kind] += alg_ops;
        return;
    }
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.launches[kind] += n;
    p.bytes[kind] += alg_bytes;
    p.ops[kind] += alg_ops;
    if (p.timing) {
        Pending e{kind, p.get_event(), p.get_event()};
        cudaEventRecord(e.a, s);
        p.pending.push_back(e);
        slot = (int)p.pending.size() - 1;
    }
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    if (slot < (int)p.pending.size()) cudaEventRecord(p.pending[slot].b, s);
}

}  // namespace bm

extern "C" {

bm_status bm_profile_control(uint32_t timing, uint32_t reset) {
    bm::Profiler& p = bm::prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.resolve();
    if (reset) {
        for (int k = 0; k < BM_KERNEL_KINDS; k++) {
            p.launches[k] = 0;
            p.bytes[k] = 0;
            p.ops[k] = 0;
            p.ms[k] = 0;
        }
    }
    p.timing = timing != 0;
    return BM_OK;
}

bm_status bm_profile_read(uint32_t kind, uint64_t* launches, double* device_ms, double* alg_bytes,
                          double* alg_mulops) {
    if (kind >= BM_KERNEL_KINDS) return BM_E_ARG;
    bm::Profiler& p = bm::prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.resolve();
    if (launches) *launches = p.launches[kind];
    if (device_ms) *device_ms = p.ms[kind];
    if (alg_bytes) *alg_bytes = p.bytes[kind];
    if (alg_mulops) *alg_mulops = p.ops[kind];
    return BM_OK;
}

}  // extern "C"
