// Serving engine: continuous batching of MaxSAT instances on one GPU.
//
// A scheduler thread owns the device work.  Requests wait in a FIFO queue;
// the oldest is admitted when a slot is free and its estimated device
// memory fits the budget.  Admission reserves the slot and the bytes and
// hands the request to a pool of builder threads: each builds an ordinary
// context (the host-side CSR work and its upload) with stream-ordered
// allocations on a stream of its own, so building never stalls the compute
// stream and a burst of requests is built in parallel.  All placed
// instances advance together: one iteration of Algorithm 1 for the whole
// slot table is three batched kernels (clause pass, heavy and light
// variable passes) captured once into a CUDA graph, replayed `chunk` times
// per round; the table and the graph are rebuilt only when the slot set
// changes.  An instance that has taken its steps is evaluated once more,
// its best costs and assignment are copied to pinned host memory behind an
// event, and its memory is released in stream order once the copy has
// landed; the freed budget admits queued requests.
// An instance small enough for the single-CTA kernel (state in shared
// memory) skips the slot table: it takes all its steps in one launch on one
// of several side streams as soon as it is built and retires the same
// way, so it is not held back by the large instances of the batch.
//
// Instances share no device state, so each result is bit for bit what the
// same request gives alone through msat_create / msat_step / msat_best.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ctx.cuh"

using namespace msat;
using Clock = std::chrono::steady_clock;

namespace {

struct SrvRequest {
    uint64_t ticket = 0;
    int32_t n = 0, steps = 0;
    int64_t m = 0;
    std::vector<int64_t> off;
    std::vector<int32_t> lits;
    std::vector<int64_t> w;
    uint64_t seed = 1;
    Clock::time_point t_submit;
    size_t est = 0;
    int64_t work = 0;  // literal evaluations of one step: nnz x restarts
};

struct SrvSlot {
    uint64_t ticket = 0;
    msat_ctx *ctx = nullptr;
    int32_t remaining = 0, steps = 0;
    Clock::time_point t_submit, t_admit;
    size_t bytes = 0;
    int64_t work = 0;
};

// A request whose context a builder has made (ctx NULL: creation failed
// and the request is already finished as failed).
struct SrvBuilt {
    SrvRequest req;
    msat_ctx *ctx = nullptr;
    Clock::time_point t_admit;
};

struct SrvFinishing {
    SrvSlot slot;
    cudaEvent_t ev = nullptr;
    int64_t *h_best = nullptr;  // pinned [B]
    uint8_t *h_bits = nullptr;  // pinned [n][B]
    int64_t *h_bstep = nullptr; // pinned [B]
    size_t cap_best = 0, cap_bits = 0, cap_bstep = 0;
};

struct SrvDone {
    msat_result res{};
    std::vector<int64_t> best;
    std::vector<uint8_t> assign;
    std::string error;  // message of a failed request
};

enum { ST_QUEUED = 0, ST_RUNNING = 1, ST_DONE = 2, ST_FAILED = 3 };

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct msat_server {
    msat_server_config cfg{};
    int device = 0;
    cudaStream_t compute = nullptr;
    // small requests run apart from the slot table, round robin over these
    static constexpr int kSmallStreams = 16;
    cudaStream_t small_st[kSmallStreams] = {};
    int small_next = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_build;
    bool stop = false;
    std::deque<SrvRequest> queue;
    // builder pool: requests handed over for context creation, and the
    // contexts made, waiting for the scheduler to place them
    std::vector<std::thread> builders;
    std::vector<cudaStream_t> build_st;
    std::deque<SrvRequest> build_q;
    std::deque<SrvBuilt> ready;
    bool stop_build = false;
    std::unordered_map<uint64_t, int> state;
    std::unordered_map<uint64_t, SrvDone> done;
    uint64_t next_ticket = 1;
    msat_server_stats st{};

    // scheduler-owned
    std::vector<SrvSlot> slots;
    std::vector<SrvFinishing> finishing;
    size_t in_use = 0;   // placed and finishing instances, plus reservations of those being built
    int building = 0;    // requests handed to the builders and not yet placed
    int64_t work = 0;    // step work of the slot table plus that of the requests being built
    int64_t work_cap = 0;
    SlotDesc *d_slots = nullptr;
    int *d_starts = nullptr;          // fwd[max+1], heavy[max+1], light[max+1]
    SlotDesc *h_slots[2] = {nullptr, nullptr};
    int *h_starts[2] = {nullptr, nullptr};
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    int stage_idx = 0;
    cudaGraphExec_t graph = nullptr;
    bool dirty = true;
    int fwd_total = 0, heavy_total = 0, light_total = 0;
    cudaEvent_t round_ev[2] = {nullptr, nullptr};
    bool round_pending[2] = {false, false};
    int round_idx = 0;
    int fwd_vw = 0, stage_vw = 0, task_cap = 0;
    // pinned result buffers are reused (freeing pinned memory synchronises the device)
    std::multimap<size_t, void *> pinned_free;
};

namespace {

// Upper bound of a context's device bytes (the allocations msat_create makes
// with f stored, before repeated literals are dropped).
size_t estimate_bytes(int64_t n, int64_t m, int64_t nnz, bool weighted, int B) {
    size_t b = 0;
    b += 4 * (size_t)(m + 1) + 4 * (size_t)nnz + (weighted ? 8 * (size_t)m : 0);  // clause CSR
    b += 4 * (size_t)(n + 1) + 4 * (size_t)nnz;                                   // transposed CSR
    b += 8 * (size_t)n + 8 * (size_t)(n + 1);                                     // heavy and light tables
    b += 21 * (size_t)n * B;                                                      // x, m, v, t0, t1, best
    b += 4 * ((size_t)m * B / 32 + 2) + 4 * (size_t)m * B;                        // unsat bits, f store
    b += 8 * (size_t)kRep * B + 64 * (size_t)B + 4 * 1216 * (size_t)B;           // step state, partials
    b += 4 * ((size_t)nnz / kChunk + (size_t)n / 512 + 1) * B + 8 * (size_t)n;   // heavy partials
    b += 40 * 256 + (1 << 16);                                                    // rounding slack
    return b;
}

cudaError_t pinned_get(msat_server *S, size_t bytes, void **p, size_t *cap) {
    auto it = S->pinned_free.lower_bound(bytes);
    if (it != S->pinned_free.end()) {
        *cap = it->first;
        *p = it->second;
        S->pinned_free.erase(it);
        return cudaSuccess;
    }
    size_t c = 256;
    while (c < bytes) c <<= 1;
    *cap = c;
    return cudaMallocHost(p, c);
}

void pinned_put(msat_server *S, void *p, size_t cap) {
    if (p) S->pinned_free.emplace(cap, p);
}

void finish_failed(msat_server *S, uint64_t ticket, int code, Clock::time_point t_submit) {
    const std::string msg = msat_last_error();
    std::lock_guard<std::mutex> lk(S->mu);
    SrvDone d;
    d.res.status = code;
    d.error = msg;
    d.res.latency_ms = ms_between(t_submit, Clock::now());
    S->done[ticket] = std::move(d);
    S->state[ticket] = ST_FAILED;
    S->st.failed++;
    S->cv_done.notify_all();
}

// Evaluate a finished instance once more and copy its best costs and
// assignment to pinned host memory behind an event, all on the instance's
// stream; reap() collects it when the event has completed.
cudaError_t start_retire(msat_server *S, const SrvSlot &sl) {
    msat_ctx *c = sl.ctx;
    SrvFinishing fin;
    fin.slot = sl;
    cudaError_t e = ctx_eval_current(c);
    if (!e) e = pinned_get(S, sizeof(int64_t) * (size_t)c->B, (void **)&fin.h_best, &fin.cap_best);
    if (!e) e = pinned_get(S, (size_t)c->n * c->B, (void **)&fin.h_bits, &fin.cap_bits);
    if (!e) e = pinned_get(S, sizeof(int64_t) * (size_t)c->B, (void **)&fin.h_bstep, &fin.cap_bstep);
    if (!e) e = cudaMemcpyAsync(fin.h_bstep, c->D.best_step, sizeof(int64_t) * (size_t)c->B, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(fin.h_best, c->D.best, sizeof(int64_t) * (size_t)c->B, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(fin.h_bits, c->S.bestx, (size_t)c->n * c->B, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaEventCreateWithFlags(&fin.ev, cudaEventDisableTiming);
    if (!e) e = cudaEventRecord(fin.ev, c->stream);
    if (!e) S->finishing.push_back(fin);
    return e;
}

msat_config request_config(const msat_server *S, const SrvRequest &req) {
    msat_config cfg;
    msat_config_default(&cfg);
    cfg.lr = S->cfg.lr;
    cfg.beta1 = S->cfg.beta1;
    cfg.beta2 = S->cfg.beta2;
    cfg.eps = S->cfg.eps;
    cfg.restarts = S->cfg.restarts;
    cfg.seed_x = req.seed;
    cfg.f_mode = MSAT_F_STORE;  // batched kernels use the stored-f path
    cfg.fwd_vw = S->fwd_vw;
    cfg.stage_vw = S->stage_vw;
    return cfg;
}

// Builder thread k: create the context of each handed-over request on
// stream k (the creation ends with that stream synchronised, so the
// context is ready for any stream), then pass it back to the scheduler.
void builder_main(msat_server *S, int k) {
    cudaSetDevice(S->device);
    for (;;) {
        SrvRequest req;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_build.wait(lk, [&] { return S->stop_build || !S->build_q.empty(); });
            if (S->build_q.empty()) return;
            req = std::move(S->build_q.front());
            S->build_q.pop_front();
        }
        const msat_config cfg = request_config(S, req);
        msat_ctx *c = nullptr;
        const int rc = ctx_create(&c, req.n, req.m, req.off.data(), req.lits.data(),
                                  req.w.empty() ? nullptr : req.w.data(), &cfg, S->build_st[(size_t)k], true);
        if (rc) finish_failed(S, req.ticket, rc, req.t_submit);
        SrvBuilt b;
        b.ctx = rc ? nullptr : c;
        b.t_admit = Clock::now();
        b.req.ticket = req.ticket;
        b.req.steps = req.steps;
        b.req.t_submit = req.t_submit;
        b.req.est = req.est;
        b.req.work = req.work;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->ready.push_back(std::move(b));
        }
        S->cv_work.notify_one();
    }
}

// Scheduler side of admission: swap the request's reservation for the
// context's real bytes and start it, either directly (small instances) or
// as a new slot of the batched table.
void place(msat_server *S, SrvBuilt &b) {
    S->building--;
    S->in_use -= b.req.est;
    S->work -= b.req.work;
    msat_ctx *c = b.ctx;
    if (!c) return;  // creation failed; the request is finished already
    const SrvRequest &req = b.req;
    SrvSlot sl;
    sl.ticket = req.ticket;
    sl.ctx = c;
    sl.remaining = req.steps;
    sl.steps = req.steps;
    sl.t_submit = req.t_submit;
    sl.t_admit = b.t_admit;
    sl.bytes = (size_t)c->device_bytes;
    S->in_use += sl.bytes;
    if (small_fits(c->I, c->max_deg)) {
        // a small instance takes all its steps in one single-CTA launch on a
        // side stream (same bits as the batched kernels), then retires
        c->stream = S->small_st[S->small_next];
        S->small_next = (S->small_next + 1) % msat_server::kSmallStreams;
        cudaError_t e = launch_small_steps(c->I, c->S, c->D, req.steps, c->stream);
        if (!e) e = start_retire(S, sl);
        if (e) {
            cuda_fail(e, "msat server: small instance");
            finish_failed(S, req.ticket, MSAT_ECUDA, req.t_submit);
            ctx_destroy_async(c);
            S->in_use -= sl.bytes;
        }
        std::lock_guard<std::mutex> lk(S->mu);
        S->st.small_direct++;
        return;
    }
    c->stream = S->compute;  // every later kernel of this instance runs on the compute stream
    sl.work = req.work;
    S->work += sl.work;
    S->slots.push_back(sl);
    S->dirty = true;
}

int rebuild(msat_server *S) {
    const int n = (int)S->slots.size();
    const int k = S->stage_idx;
    S->stage_idx ^= 1;
    // the staging pair k was last used two rebuilds ago: wait for its copy
    if (S->stage_ev[k]) cudaEventSynchronize(S->stage_ev[k]);
    SlotDesc *hs = S->h_slots[k];
    int *hst = S->h_starts[k];
    const int M = S->cfg.max_slots + 1;
    int f = 0, h = 0, l = 0;
    for (int i = 0; i < n; ++i) {
        msat_ctx *c = S->slots[(size_t)i].ctx;
        if (c->B != S->cfg.restarts || c->I.task_cap != S->task_cap || c->I.fwd_vw != S->fwd_vw ||
            c->I.stage_vw != S->stage_vw || !c->S.fstore)
            return fail(MSAT_ESTATE, "msat server: an instance's launch shape differs from the slot table's");
        hs[i].I = c->I;
        hs[i].S = c->S;
        hs[i].D = c->D;
        hst[i] = f;
        hst[M + i] = h;
        hst[2 * M + i] = l;
        f += c->D.fwd_blocks;
        h += heavy_blocks_of(c->I);
        l += light_blocks_of(c->I);
    }
    hst[n] = f;
    hst[M + n] = h;
    hst[2 * M + n] = l;
    S->fwd_total = f;
    S->heavy_total = h;
    S->light_total = l;
    cudaError_t e = cudaSuccess;
    if (n > 0) e = cudaMemcpyAsync(S->d_slots, hs, sizeof(SlotDesc) * (size_t)n, cudaMemcpyHostToDevice, S->compute);
    if (!e) e = cudaMemcpyAsync(S->d_starts, hst, sizeof(int) * 3 * (size_t)M, cudaMemcpyHostToDevice, S->compute);
    if (!e) e = cudaEventRecord(S->stage_ev[k], S->compute);
    if (e) return cuda_fail(e, "msat server: slot table upload");
    if (S->graph) {
        cudaGraphExecDestroy(S->graph);
        S->graph = nullptr;
    }
    if (n > 0) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(S->compute, cudaStreamCaptureModeThreadLocal);
        if (!e) {
            const cudaError_t le = launch_step_batch(S->d_slots, n, S->d_starts, f, S->d_starts + M, h,
                                                     S->d_starts + 2 * M, l, S->cfg.restarts, S->fwd_vw,
                                                     S->stage_vw, S->task_cap, S->compute);
            e = cudaStreamEndCapture(S->compute, &g);
            if (!e) e = le;
        }
        if (!e) e = cudaGraphInstantiate(&S->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e) return cuda_fail(e, "msat server: step graph capture");
        S->st.graph_captures++;
    }
    S->dirty = false;
    return MSAT_OK;
}

// One scheduling round: advance every slot by R steps, then retire the
// slots that have taken all their steps.
int run_round_body(msat_server *S) {
    if (S->dirty) {
        const int rc = rebuild(S);
        if (rc) return rc;
    }
    int R = S->cfg.chunk;
    for (const SrvSlot &sl : S->slots) R = std::min(R, sl.remaining);
    if (R > 0 && S->graph) {
        const int k = S->round_idx & 1;
        if (S->round_pending[k]) cudaEventSynchronize(S->round_ev[k]);  // at most two rounds queued
        for (int r = 0; r < R; ++r) {
            const cudaError_t e = cudaGraphLaunch(S->graph, S->compute);
            if (e) return cuda_fail(e, "msat server: graph launch");
        }
        cudaEventRecord(S->round_ev[k], S->compute);
        S->round_pending[k] = true;
        S->round_idx++;
        for (SrvSlot &sl : S->slots) sl.remaining -= R;
        std::lock_guard<std::mutex> lk(S->mu);
        S->st.rounds += R;
    }
    // retire
    std::vector<SrvSlot> keep;
    keep.reserve(S->slots.size());
    for (SrvSlot &sl : S->slots) {
        if (sl.remaining > 0) {
            keep.push_back(sl);
            continue;
        }
        const cudaError_t e = start_retire(S, sl);
        if (e) return cuda_fail(e, "msat server: result copy");
        S->work -= sl.work;
        S->dirty = true;
    }
    S->slots.swap(keep);
    return MSAT_OK;
}

int run_round(msat_server *S) {
    nvtxRangePushA("msat server round");
    const int rc = run_round_body(S);
    nvtxRangePop();
    return rc;
}

// Collect finished results (waiting for the first one when block is set).
void reap(msat_server *S, bool block) {
    std::vector<SrvFinishing> pending;
    for (size_t i = 0; i < S->finishing.size(); ++i) {
        SrvFinishing &f = S->finishing[i];
        bool ready = false;
        if (block && i == 0) ready = cudaEventSynchronize(f.ev) == cudaSuccess;
        else ready = cudaEventQuery(f.ev) == cudaSuccess;
        if (!ready) {
            cudaGetLastError();
            pending.push_back(f);
            continue;
        }
        msat_ctx *c = f.slot.ctx;
        const int B = c->B, n = c->n;
        SrvDone d;
        d.best.assign(f.h_best, f.h_best + B);
        int bb = 0;
        for (int b = 1; b < B; ++b)
            if (d.best[(size_t)b] < d.best[(size_t)bb]) bb = b;
        d.assign.resize((size_t)n);
        for (int i2 = 0; i2 < n; ++i2) d.assign[(size_t)i2] = f.h_bits[(size_t)i2 * B + bb];
        const Clock::time_point now = Clock::now();
        d.res.status = 0;
        d.res.best_restart = bb;
        d.res.best_cost = d.best[(size_t)bb];
        d.res.best_step = f.h_bstep[bb];
        d.res.steps = f.slot.steps;
        d.res.n_vars = n;
        d.res.restarts = B;
        d.res.queue_ms = ms_between(f.slot.t_submit, f.slot.t_admit);
        d.res.latency_ms = ms_between(f.slot.t_submit, now);
        ctx_destroy_async(c);  // frees in order on the compute stream
        S->in_use -= f.slot.bytes;
        pinned_put(S, f.h_best, f.cap_best);
        pinned_put(S, f.h_bits, f.cap_bits);
        pinned_put(S, f.h_bstep, f.cap_bstep);
        cudaEventDestroy(f.ev);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->done[f.slot.ticket] = std::move(d);
            S->state[f.slot.ticket] = ST_DONE;
            S->st.completed++;
        }
        S->cv_done.notify_all();
    }
    S->finishing.swap(pending);
}

// A slot is free, the oldest request's estimate fits the budget and its
// step work fits the batch cap (or nothing else is running or being
// built); the caller holds the lock.
bool can_admit(const msat_server *S) {
    if (S->queue.empty()) return false;
    const SrvRequest &r = S->queue.front();
    const bool alone = S->slots.empty() && S->building == 0;
    return (int)S->slots.size() + S->building < S->cfg.max_slots &&
           S->in_use + r.est <= S->cfg.hbm_budget &&
           (S->work_cap <= 0 || alone || S->work + r.work <= S->work_cap);
}

void worker_main(msat_server *S) {
    cudaSetDevice(S->device);
    std::deque<SrvBuilt> got;
    for (;;) {
        bool block_reap = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // admission in FIFO order: reserve a slot and the estimated
            // bytes, and hand the request to the builders
            bool handed = false;
            while (can_admit(S)) {
                SrvRequest &req = S->queue.front();
                S->state[req.ticket] = ST_RUNNING;
                S->in_use += req.est;
                S->work += req.work;
                S->building++;
                S->build_q.push_back(std::move(req));
                S->queue.pop_front();
                handed = true;
            }
            if (handed) S->cv_build.notify_all();
            got.swap(S->ready);
            const bool idle = got.empty() && S->slots.empty();
            if (idle && S->finishing.empty()) {
                if (S->stop && S->queue.empty() && S->building == 0) break;
                S->cv_work.wait(lk, [&] {
                    return (S->stop && S->queue.empty() && S->building == 0) || !S->ready.empty() ||
                           can_admit(S);
                });
                continue;
            }
            if (idle) {
                // only results in flight: wait for them, unless contexts are
                // still being built (then poll, so a built one is placed soon)
                if (S->building > 0)
                    S->cv_work.wait_for(lk, std::chrono::microseconds(200), [&] { return !S->ready.empty(); });
                else
                    block_reap = true;
            }
        }
        for (SrvBuilt &b : got) place(S, b);
        got.clear();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->st.running = (int32_t)S->slots.size();
            S->st.peak_running = std::max(S->st.peak_running, S->st.running);
            S->st.queued = (int32_t)S->queue.size();
            S->st.hbm_in_use = (int64_t)S->in_use;
        }
        if (!S->slots.empty()) {
            const int rc = run_round(S);
            if (rc) {
                // a CUDA failure in the shared loop fails every running request
                for (SrvSlot &sl : S->slots) {
                    finish_failed(S, sl.ticket, rc, sl.t_submit);
                    ctx_destroy_async(sl.ctx);
                    S->in_use -= sl.bytes;
                    S->work -= sl.work;
                }
                S->slots.clear();
                S->dirty = true;
            }
        }
        reap(S, block_reap);
    }
}

}  // namespace

extern "C" int msat_server_config_default(msat_server_config *cfg) {
    if (!cfg) return fail(MSAT_EINVAL, "msat_server_config_default: cfg is NULL");
    memset(cfg, 0, sizeof(*cfg));
    cfg->max_slots = 256;
    cfg->restarts = 8;
    cfg->chunk = 50;
    cfg->batch_mlits = 128;
    cfg->lr = 1e-4;
    cfg->beta1 = 0.9;
    cfg->beta2 = 0.999;
    cfg->eps = 1e-8;
    return MSAT_OK;
}

extern "C" int msat_server_create(msat_server **out, const msat_server_config *cfg_in) {
    if (!out) return fail(MSAT_EINVAL, "msat_server_create: out is NULL");
    *out = nullptr;
    msat_server_config cfg;
    if (cfg_in) cfg = *cfg_in; else msat_server_config_default(&cfg);
    if (cfg.max_slots <= 0) cfg.max_slots = 256;
    if (cfg.chunk <= 0) cfg.chunk = 50;
    if (cfg.batch_mlits == 0) cfg.batch_mlits = 128;
    const int B = cfg.restarts;
    if (B < 1 || B > 1024 || (B & (B - 1)))
        return fail(MSAT_EINVAL, "msat_server_create: restarts must be a power of two in [1, 1024]");
    msat_server *S = new (std::nothrow) msat_server();
    if (!S) return fail(MSAT_ENOMEM, "msat_server_create: host allocation failed");
    cudaGetDevice(&S->device);
    if (cfg.hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = (size_t)8 << 30;
        }
        cfg.hbm_budget = fr / 2;
    }
    S->cfg = cfg;
    S->work_cap = cfg.batch_mlits > 0 ? (int64_t)cfg.batch_mlits * 1000000 : 0;
    // four restarts a thread in the batched clause pass (74 registers, three
    // resident blocks per SM; eight take 92 and two blocks) -- measured on
    // the k in {3,4,5} request stream at B = 8: 69 -> 75 instances/s
    S->fwd_vw = B < 4 ? B : 4;
    // two restarts a leaf task: the batched variable pass then fits four
    // resident blocks per SM (63 registers) instead of two at four restarts
    // (86); launch shapes never change a result bit
    S->stage_vw = B < 2 ? B : 2;
    S->task_cap = std::max(kTaskCap, B / S->stage_vw);
    const int M = cfg.max_slots + 1;
    // builders: half the host's hardware threads, 1 to 8
    const unsigned hc = std::thread::hardware_concurrency();
    const int n_build = (int)std::min(8u, std::max(1u, hc / 2));
    S->build_st.assign((size_t)n_build, nullptr);
    cudaError_t e = cudaStreamCreateWithFlags(&S->compute, cudaStreamNonBlocking);
    for (int k = 0; k < n_build && !e; ++k)
        e = cudaStreamCreateWithFlags(&S->build_st[(size_t)k], cudaStreamNonBlocking);
    for (int k = 0; k < msat_server::kSmallStreams && !e; ++k)
        e = cudaStreamCreateWithFlags(&S->small_st[k], cudaStreamNonBlocking);
    if (!e) e = cudaMalloc(&S->d_slots, sizeof(SlotDesc) * (size_t)cfg.max_slots);
    if (!e) e = cudaMalloc(&S->d_starts, sizeof(int) * 3 * (size_t)M);
    for (int k = 0; k < 2 && !e; ++k) {
        e = cudaMallocHost(&S->h_slots[k], sizeof(SlotDesc) * (size_t)cfg.max_slots);
        if (!e) e = cudaMallocHost(&S->h_starts[k], sizeof(int) * 3 * (size_t)M);
        if (!e) e = cudaEventCreateWithFlags(&S->stage_ev[k], cudaEventDisableTiming);
        if (!e) e = cudaEventCreateWithFlags(&S->round_ev[k], cudaEventDisableTiming);
    }
    if (!e) {
        // keep freed pool memory cached for the next admissions (process-local setting)
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    }
    if (e) {
        const int rc = cuda_fail(e, "msat_server_create");
        msat_server_destroy(S);
        return rc;
    }
    S->st.hbm_budget = (int64_t)cfg.hbm_budget;
    for (int k = 0; k < n_build; ++k) S->builders.emplace_back(builder_main, S, k);
    S->worker = std::thread(worker_main, S);
    *out = S;
    return MSAT_OK;
}

extern "C" void msat_server_destroy(msat_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();  // returns once nothing is queued or being built
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop_build = true;
    }
    S->cv_build.notify_all();
    for (std::thread &t : S->builders)
        if (t.joinable()) t.join();
    if (S->compute) cudaStreamSynchronize(S->compute);
    for (cudaStream_t st : S->small_st)
        if (st) cudaStreamSynchronize(st);
    if (S->graph) cudaGraphExecDestroy(S->graph);
    cudaFree(S->d_slots);
    cudaFree(S->d_starts);
    for (int k = 0; k < 2; ++k) {
        if (S->h_slots[k]) cudaFreeHost(S->h_slots[k]);
        if (S->h_starts[k]) cudaFreeHost(S->h_starts[k]);
        if (S->stage_ev[k]) cudaEventDestroy(S->stage_ev[k]);
        if (S->round_ev[k]) cudaEventDestroy(S->round_ev[k]);
    }
    for (auto &kv : S->pinned_free) cudaFreeHost(kv.second);
    if (S->compute) cudaStreamDestroy(S->compute);
    for (cudaStream_t st : S->build_st)
        if (st) cudaStreamDestroy(st);
    for (cudaStream_t st : S->small_st)
        if (st) cudaStreamDestroy(st);
    delete S;
}

extern "C" int msat_submit(msat_server *S, const msat_request *req, uint64_t *ticket) {
    if (!S || !req || !ticket) return fail(MSAT_EINVAL, "msat_submit: NULL argument");
    const int64_t m = req->n_clauses;
    if (req->n_vars < 1 || m < 0 || req->steps < 0 || !req->clause_off)
        return fail(MSAT_EINVAL, "msat_submit: need n_vars >= 1, n_clauses >= 0, steps >= 0, clause_off");
    if (req->clause_off[0] != 0) return fail(MSAT_EINVAL, "msat_submit: clause_off[0] must be 0");
    for (int64_t j = 0; j < m; ++j)
        if (req->clause_off[j + 1] < req->clause_off[j])
            return fail(MSAT_EINVAL, "msat_submit: clause_off is not non-decreasing");
    const int64_t nnz = req->clause_off[m];
    if (nnz > 0 && !req->lits) return fail(MSAT_EINVAL, "msat_submit: lits is NULL");
    for (int64_t q = 0; q < nnz; ++q)
        if (req->lits[q] == 0 || req->lits[q] > req->n_vars || req->lits[q] < -req->n_vars)
            return fail(MSAT_EINVAL, "msat_submit: literal names no variable");
    if (req->weights)
        for (int64_t j = 0; j < m; ++j)
            if (req->weights[j] < 1) return fail(MSAT_EINVAL, "msat_submit: weight below 1");
    SrvRequest r;
    r.n = req->n_vars;
    r.m = m;
    r.steps = req->steps;
    r.seed = req->seed_x;
    r.off.assign(req->clause_off, req->clause_off + m + 1);
    r.lits.assign(req->lits, req->lits + nnz);
    if (req->weights) r.w.assign(req->weights, req->weights + m);
    r.est = estimate_bytes(r.n, m, nnz, req->weights != nullptr, S->cfg.restarts);
    r.work = nnz * (int64_t)S->cfg.restarts;
    if (r.est > S->cfg.hbm_budget)
        return fail(MSAT_EBUDGET, "msat_submit: the instance needs about " + std::to_string(r.est) +
                                      " device bytes, above the server budget of " +
                                      std::to_string(S->cfg.hbm_budget));
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return fail(MSAT_ESTATE, "msat_submit: the server is shutting down");
        r.ticket = S->next_ticket++;
        *ticket = r.ticket;
        S->state[r.ticket] = ST_QUEUED;
        S->queue.push_back(std::move(r));
        S->st.submitted++;
    }
    S->cv_work.notify_one();
    return MSAT_OK;
}

static int take_result(msat_server *S, uint64_t ticket, msat_result *out, int64_t *best_costs,
                       uint8_t *assign01) {
    auto it = S->state.find(ticket);
    if (it == S->state.end()) return fail(MSAT_EINVAL, "msat_poll: unknown ticket");
    if (it->second == ST_QUEUED || it->second == ST_RUNNING) return MSAT_EAGAIN;
    SrvDone &d = S->done[ticket];
    const int status = d.res.status;
    if (out) *out = d.res;
    if (status == 0) {
        if (best_costs) std::copy(d.best.begin(), d.best.end(), best_costs);
        if (assign01) std::copy(d.assign.begin(), d.assign.end(), assign01);
    }
    const std::string err = d.error;
    S->done.erase(ticket);
    S->state.erase(it);
    if (status) return fail(status, "the request failed: " + err);
    return MSAT_OK;
}

extern "C" int msat_poll(msat_server *S, uint64_t ticket, msat_result *out, int64_t *best_costs,
                         uint8_t *assign01) {
    if (!S) return fail(MSAT_EINVAL, "msat_poll: server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    return take_result(S, ticket, out, best_costs, assign01);
}

extern "C" int msat_wait(msat_server *S, uint64_t ticket, double timeout_s, msat_result *out,
                         int64_t *best_costs, uint8_t *assign01) {
    if (!S) return fail(MSAT_EINVAL, "msat_wait: server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        auto it = S->state.find(ticket);
        if (it == S->state.end()) return fail(MSAT_EINVAL, "msat_wait: unknown ticket");
        if (it->second == ST_DONE || it->second == ST_FAILED)
            return take_result(S, ticket, out, best_costs, assign01);
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto it2 = S->state.find(ticket);
            if (it2 != S->state.end() && (it2->second == ST_DONE || it2->second == ST_FAILED))
                return take_result(S, ticket, out, best_costs, assign01);
            return fail(MSAT_ETIMEOUT, "msat_wait: timed out");
        }
    }
}

extern "C" int msat_cancel(msat_server *S, uint64_t ticket) {
    if (!S) return fail(MSAT_EINVAL, "msat_cancel: server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->state.find(ticket);
    if (it == S->state.end()) return fail(MSAT_EINVAL, "msat_cancel: unknown ticket");
    if (it->second != ST_QUEUED) return fail(MSAT_ESTATE, "msat_cancel: the request is already admitted");
    for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
        if (q->ticket == ticket) {
            S->queue.erase(q);
            break;
        }
    S->state.erase(it);
    S->st.cancelled++;
    return MSAT_OK;
}

extern "C" int msat_server_get_stats(msat_server *S, msat_server_stats *out) {
    if (!S || !out) return fail(MSAT_EINVAL, "msat_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->queued = (int32_t)S->queue.size();
    return MSAT_OK;
}
