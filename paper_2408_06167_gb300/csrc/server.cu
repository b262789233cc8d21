// server.cu -- continuous-batching match server over resident galleries.
//
// Requests (one encrypted query against one registered gallery) are queued in
// arrival order.  Each executor thread owns a CUDA stream and its own match
// plans; whenever it is free it takes the oldest pending request and every
// other pending request for the same gallery (up to max_batch), runs them as
// one batched match on its stream and completes them.  Several executors run
// at once, so batches for different galleries (or successive batches for one)
// overlap on the device while new requests keep arriving.  Plan workspaces are
// admitted against a device-memory budget: an executor first evicts its own
// idle plans, then halves its batch; a single query that still does not fit
// fails with BM_E_HBM_BUDGET.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bm_internal.h"

namespace bm {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    uint32_t gid = 0;
    Ciphertext ct;
    Clock::time_point t_submit, t_done;
    bool done = false;
    bm_status status = BM_OK;
    std::string error;
    bm_result* result = nullptr;
};

struct Entry {
    const Gallery* g;
    const EvalKeys* ek;
};

struct ExecPlan {
    uint32_t gid, Q;
    Plan* plan;
    uint64_t last_used;
};

struct Server;

struct Executor {
    Server* srv = nullptr;
    cudaStream_t s = nullptr;
    std::vector<ExecPlan> plans;
    std::thread th;
    uint64_t clock = 0;
};

struct Server {
    Context* c = nullptr;
    uint64_t budget = 0;
    uint32_t max_batch = 1;
    std::vector<Entry> galleries;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> requests;
    std::vector<Executor*> execs;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t plan_bytes_total = 0;
    // statistics
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, batches = 0, batched_queries = 0;
    double matches = 0;
    std::vector<double> latencies_ms;
    Clock::time_point t_first, t_last;
    bool any = false;
};

// the plan size for n pending queries: the largest power of two not above n (and
// max_batch), so a plan never runs padding queries; the surplus goes back to the queue
uint32_t bucket(uint32_t n, uint32_t max_batch) {
    uint32_t b = 1;
    while (2 * b <= n) b <<= 1;
    return std::min(b, max_batch);
}

void finish(Server& S, Request* r, bm_status st, const std::string& err) {
    r->status = st;
    r->error = err;
    r->done = true;
    r->t_done = Clock::now();
    if (st == BM_OK) {
        S.completed++;
        S.latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
        S.t_last = r->t_done;
    } else if (st == BM_E_CANCELLED) {
        S.cancelled++;
    } else {
        S.failed++;
    }
}

// a plan for (gid, Q) on this executor, within the budget; nullptr + status if not possible
bm_status get_plan(Executor& E, uint32_t gid, uint32_t Q, Plan*& out, std::string& err) {
    Server& S = *E.srv;
    for (auto& p : E.plans)
        if (p.gid == gid && p.Q == Q) {
            p.last_used = ++E.clock;
            out = p.plan;
            return BM_OK;
        }
    const Entry& en = S.galleries[gid];
    // admission: the plan's bytes are known before anything is allocated
    const size_t need = plan_estimate_bytes(*S.c, *en.g, Q);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(S.mu);
            if (S.plan_bytes_total + need <= S.budget) {
                S.plan_bytes_total += need;
                break;
            }
        }
        // evict this executor's least recently used plan, if any
        if (E.plans.empty()) {
            err = "the match workspace (" + std::to_string(need) + " bytes) exceeds the device-memory budget";
            return BM_E_HBM_BUDGET;
        }
        auto lru = std::min_element(E.plans.begin(), E.plans.end(),
                                    [](const ExecPlan& a, const ExecPlan& b) { return a.last_used < b.last_used; });
        const size_t freed = plan_bytes(lru->plan);
        destroy_plan(lru->plan);
        E.plans.erase(lru);
        std::lock_guard<std::mutex> lk(S.mu);
        S.plan_bytes_total -= freed;
    }
    Plan* pl = nullptr;
    bm_status st = plan_build(*S.c, *en.g, *en.ek, Q, E.s, pl);
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.plan_bytes_total -= need;
        if (st == BM_OK) S.plan_bytes_total += plan_bytes(pl);
    }
    if (st != BM_OK) {
        err = bm_last_error();
        return st;
    }
    E.plans.push_back({gid, Q, pl, ++E.clock});
    out = pl;
    return BM_OK;
}

void run_batch(Executor& E, std::vector<Request*>& batch) {
    Server& S = *E.srv;
    Context& c = *S.c;
    const uint32_t gid = batch[0]->gid;
    const Entry& en = S.galleries[gid];
    uint32_t Q = bucket((uint32_t)batch.size(), S.max_batch);
    Plan* pl = nullptr;
    std::string err;
    bm_status st;
    for (;;) {
        st = get_plan(E, gid, Q, pl, err);
        if (st != BM_E_HBM_BUDGET || Q == 1) break;
        Q /= 2;                                   // a smaller batch may fit
    }
    if (st == BM_OK && batch.size() > Q) {
        // hand the surplus back, oldest first
        std::lock_guard<std::mutex> lk(S.mu);
        for (size_t i = batch.size(); i-- > Q;) S.pending.push_front(batch[i]);
        batch.resize(Q);
        S.cv_work.notify_all();
    }
    std::vector<bm_result*> results(batch.size(), nullptr);
    if (st == BM_OK) {
        std::vector<const Ciphertext*> qs(batch.size());
        for (size_t i = 0; i < batch.size(); i++) qs[i] = &batch[i]->ct;
        st = plan_run(c, *en.g, *en.ek, pl, qs.data(), (uint32_t)batch.size(), E.s);
        if (st != BM_OK) err = bm_last_error();
    }
    if (st == BM_OK) {
        const uint32_t n_out = plan_outputs(pl);
        const size_t words = (size_t)n_out * ct_words(c, 0);
        for (size_t i = 0; i < batch.size() && st == BM_OK; i++) {
            auto* rh = new bm_result();
            rh->ref.attach(&c);
            Result& r = rh->r;
            r.ctx = &c;
            r.n_queries = 1;
            r.n_out = n_out;
            r.n_ids = en.g->n_ids;
            r.dim = en.g->dim;
            r.part = en.g->part;
            r.packed = en.g->compress;
            r.packing = en.g->packing;
            r.scale = result_scale(c, *en.g);
            cudaError_t e = cudaMallocAsync((void**)&r.d_data, words * 8, E.s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r.d_data, plan_result(pl) + i * words, words * 8, cudaMemcpyDeviceToDevice, E.s);
            if (e != cudaSuccess) {
                st = BM_E_CUDA;
                err = cudaGetErrorString(e);
            }
            results[i] = rh;
        }
        cudaError_t e = cudaStreamSynchronize(E.s);
        if (st == BM_OK && e != cudaSuccess) {
            st = BM_E_CUDA;
            err = cudaGetErrorString(e);
        }
    }
    std::lock_guard<std::mutex> lk(S.mu);
    if (st == BM_OK) {
        S.batches++;
        S.batched_queries += batch.size();
    }
    for (size_t i = 0; i < batch.size(); i++) {
        if (st == BM_OK) {
            batch[i]->result = results[i];
            S.matches += (double)en.g->n_ids;
        } else {
            delete results[i];
        }
        finish(S, batch[i], st, err);
    }
    S.cv_done.notify_all();
}

void executor_loop(Executor* E) {
    Server& S = *E->srv;
    cudaSetDevice(S.c->device);
    for (;;) {
        std::vector<Request*> batch;
        {
            std::unique_lock<std::mutex> lk(S.mu);
            S.cv_work.wait(lk, [&] { return S.stop || !S.pending.empty(); });
            if (S.stop) break;
            const uint32_t gid = S.pending.front()->gid;
            for (auto it = S.pending.begin(); it != S.pending.end() && batch.size() < S.max_batch;) {
                if ((*it)->gid == gid) {
                    batch.push_back(*it);
                    it = S.pending.erase(it);
                } else {
                    ++it;
                }
            }
        }
        run_batch(*E, batch);
    }
    for (auto& p : E->plans) destroy_plan(p.plan);
    E->plans.clear();
}

}  // namespace
}  // namespace bm

struct bm_server { bm::CtxRef ref; bm::Server s; };

using namespace bm;

extern "C" {

bm_status bm_server_create(bm_context* ctx, uint64_t hbm_budget_bytes, uint32_t max_batch, uint32_t executors,
                           bm_server** out) {
    if (!ctx || !out || max_batch == 0 || executors == 0 || executors > 16) {
        set_error("bm_server_create: null argument, zero max_batch, or executors outside 1..16");
        return BM_E_ARG;
    }
    auto* h = new bm_server();
    h->ref.attach(&ctx->c);
    Server& S = h->s;
    S.c = &ctx->c;
    S.budget = hbm_budget_bytes;
    S.max_batch = max_batch;
    if (cudaSetDevice(ctx->c.device) != cudaSuccess) {
        delete h;
        set_error("bm_server_create: cannot use the context's device");
        return BM_E_CUDA;
    }
    for (uint32_t i = 0; i < executors; i++) {
        auto* E = new Executor();
        E->srv = &S;
        if (cudaStreamCreateWithFlags(&E->s, cudaStreamNonBlocking) != cudaSuccess) {
            delete E;
            bm_server_destroy(h);
            set_error("bm_server_create: stream creation failed");
            return BM_E_CUDA;
        }
        S.execs.push_back(E);
    }
    for (Executor* E : S.execs) E->th = std::thread(executor_loop, E);
    *out = h;
    return BM_OK;
}

void bm_server_destroy(bm_server* h) {
    if (!h) return;
    Server& S = h->s;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
        for (Request* r : S.pending) finish(S, r, BM_E_CANCELLED, "server destroyed");
        S.pending.clear();
    }
    S.cv_work.notify_all();
    S.cv_done.notify_all();
    for (Executor* E : S.execs) {
        if (E->th.joinable()) E->th.join();
        if (E->s) cudaStreamDestroy(E->s);
        delete E;
    }
    for (auto& kv : S.requests) {
        if (kv.second->result) bm_result_destroy(kv.second->result);
        delete kv.second;
    }
    delete h;
}

bm_status bm_server_add_gallery(bm_server* h, const bm_gallery* g, const bm_eval_keys* evk, uint32_t* gid) {
    if (!h || !g || !evk || !gid) {
        set_error("bm_server_add_gallery: null argument");
        return BM_E_ARG;
    }
    Server& S = h->s;
    if (g->g.ctx != S.c || evk->k.ctx != S.c) {
        set_error("bm_server_add_gallery: handles belong to another context");
        return BM_E_ARG;
    }
    if (evk->k.dim != g->g.dim || evk->k.part != g->g.part) {
        set_error("bm_server_add_gallery: key set generated for another (dim, part)");
        return BM_E_KEY_MISSING;
    }
    std::lock_guard<std::mutex> lk(S.mu);
    S.galleries.push_back({&g->g, &evk->k});
    *gid = (uint32_t)S.galleries.size() - 1;
    return BM_OK;
}

bm_status bm_server_submit(bm_server* h, uint32_t gid, const bm_ciphertext* query, uint64_t* ticket) {
    if (!h || !query || !ticket) {
        set_error("bm_server_submit: null argument");
        return BM_E_ARG;
    }
    Server& S = h->s;
    const Ciphertext& ct = query->ct;
    auto* r = new Request();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        if (gid >= S.galleries.size()) {
            delete r;
            set_error("bm_server_submit: unknown gallery");
            return BM_E_ARG;
        }
        const Gallery& g = *S.galleries[gid].g;
        if (ct.n_cts != (g.tiled ? 1u : g.n_in) || ct.level != S.c->L) {
            delete r;
            set_error("bm_server_submit: query layout does not match the gallery's schedule");
            return BM_E_LEVEL;
        }
    }
    r->gid = gid;
    r->ct.ctx = ct.ctx;
    r->ct.n_cts = ct.n_cts;
    r->ct.level = ct.level;
    r->ct.host = ct.host;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        r->ticket = S.next_ticket++;
        S.requests[r->ticket] = r;
        S.pending.push_back(r);
        S.submitted++;
        if (!S.any) {
            S.any = true;
            S.t_first = r->t_submit;
        }
        *ticket = r->ticket;
    }
    S.cv_work.notify_one();
    return BM_OK;
}

bm_status bm_server_wait(bm_server* h, uint64_t ticket, uint32_t timeout_ms, bm_result** out) {
    if (!h || !out) {
        set_error("bm_server_wait: null argument");
        return BM_E_ARG;
    }
    Server& S = h->s;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.requests.find(ticket);
    if (it == S.requests.end()) {
        set_error("bm_server_wait: unknown or already collected ticket");
        return BM_E_ARG;
    }
    Request* r = it->second;
    if (!S.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; })) {
        set_error("bm_server_wait: the request did not complete within " + std::to_string(timeout_ms) + " ms");
        return BM_E_TIMEOUT;
    }
    S.requests.erase(it);
    const bm_status st = r->status;
    if (st == BM_OK) *out = r->result;
    else set_error(r->error);
    delete r;
    return st;
}

bm_status bm_server_cancel(bm_server* h, uint64_t ticket) {
    if (!h) {
        set_error("bm_server_cancel: null server");
        return BM_E_ARG;
    }
    Server& S = h->s;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = std::find_if(S.pending.begin(), S.pending.end(), [&](Request* r) { return r->ticket == ticket; });
    if (it == S.pending.end()) {
        set_error("bm_server_cancel: the request is not pending (running, finished or unknown)");
        return BM_E_ARG;
    }
    finish(S, *it, BM_E_CANCELLED, "cancelled by the caller");
    S.pending.erase(it);
    S.cv_done.notify_all();
    return BM_OK;
}

bm_status bm_server_reset_stats(bm_server* h) {
    if (!h) {
        set_error("bm_server_reset_stats: null argument");
        return BM_E_ARG;
    }
    Server& S = h->s;
    std::lock_guard<std::mutex> lk(S.mu);
    S.submitted = S.completed = S.failed = S.cancelled = S.batches = 0;
    S.batched_queries = 0;
    S.matches = 0;
    S.latencies_ms.clear();
    S.any = false;
    return BM_OK;
}

bm_status bm_server_stats(bm_server* h, bm_server_stats_t* out) {
    if (!h || !out) {
        set_error("bm_server_stats: null argument");
        return BM_E_ARG;
    }
    Server& S = h->s;
    std::lock_guard<std::mutex> lk(S.mu);
    bm_server_stats_t st{};
    st.submitted = S.submitted;
    st.completed = S.completed;
    st.failed = S.failed;
    st.cancelled = S.cancelled;
    st.batches = S.batches;
    st.mean_batch = S.batches ? (double)S.batched_queries / (double)S.batches : 0.0;
    st.workspace_bytes = S.plan_bytes_total;
    if (!S.latencies_ms.empty()) {
        std::vector<double> l = S.latencies_ms;
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p / 100.0 * (double)(l.size() - 1) + 0.5))]; };
        st.p50_ms = pct(50);
        st.p99_ms = pct(99);
        const double span = std::chrono::duration<double>(S.t_last - S.t_first).count();
        st.matches_per_s = span > 0 ? S.matches / span : 0.0;
    }
    *out = st;
    return BM_OK;
}

}  // extern "C"
