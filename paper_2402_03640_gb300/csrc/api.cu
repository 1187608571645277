// C ABI of the MaxSAT gradient engine: context creation (validation, clause
// canonicalisation, CSR and transposed CSR, device upload), the step loop,
// evaluation, best assignment, checkpoint and the differentiable probe.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "msat_internal.cuh"

namespace msat {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return MSAT_ECUDA;
}

}  // namespace msat

using namespace msat;

#include "ctx.cuh"
#include "host_cnf.cuh"

#include <nvtx3/nvToolsExt.h>

// NVTX range over a host call (visible to nsys / ncu --nvtx; no cost
// without an attached tool)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

enum { PROF_FWD = 0, PROF_BWD = 1, PROF_EVAL = 2, PROF_OTHER = 3 };

static void prof_begin(msat_ctx *c, int kind) {
    if (!c->prof_on) return;
    if (2 * c->prof_used + 2 > c->prof_ev.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            cudaGetLastError();
            c->prof_on = false;
            return;
        }
        c->prof_ev.push_back(a);
        c->prof_ev.push_back(b);
        c->prof_kind.push_back(kind);
    }
    c->prof_kind[c->prof_used] = kind;
    cudaEventRecord(c->prof_ev[2 * c->prof_used], c->stream);
}

static void prof_end(msat_ctx *c) {
    if (!c->prof_on) return;
    cudaEventRecord(c->prof_ev[2 * c->prof_used + 1], c->stream);
    ++c->prof_used;
}

static int dalloc(msat_ctx *c, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = c->pool_alloc ? cudaMallocAsync(p, bytes, c->stream) : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(MSAT_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) +
                                     " bytes failed: " + cudaGetErrorString(e));
    }
    c->allocs.push_back(*p);
    c->device_bytes += (int64_t)bytes;
    return MSAT_OK;
}

template <typename T>
static int dalloc_t(msat_ctx *c, T **p, size_t count) {
    return dalloc(c, reinterpret_cast<void **>(p), count * sizeof(T));
}

static void free_all(msat_ctx *c) {
    if (c->graph1) cudaGraphExecDestroy(c->graph1);
    if (c->graphK) cudaGraphExecDestroy(c->graphK);
    c->graph1 = c->graphK = nullptr;
    for (void *p : c->allocs) {
        if (c->pool_alloc) cudaFreeAsync(p, c->stream); else cudaFree(p);
    }
    c->allocs.clear();
    if (c->dense.Xt) cudaFree(c->dense.Xt);
    c->dense.Xt = nullptr;
    c->dense.xt_bytes = 0;
    if (c->dense.ptgt) cudaFree(c->dense.ptgt);
    if (c->dense.pmask) cudaFree(c->dense.pmask);
    if (c->dense.part_cnt) cudaFree(c->dense.part_cnt);
    c->dense.ptgt = nullptr;
    c->dense.pmask = nullptr;
    c->dense.part_cnt = nullptr;
    c->dense.ptgt_slots = c->dense.part_cnts = c->dense.pmask_ntile = 0;
    c->dense.plan_grid = -1;
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    c->prof_kind.clear();
    c->prof_used = 0;
}

extern "C" int msat_config_default(msat_config *cfg) {
    if (!cfg) return fail(MSAT_EINVAL, "msat_config_default: cfg is NULL");
    memset(cfg, 0, sizeof(*cfg));
    cfg->lr = 1e-4;
    cfg->beta1 = 0.9;
    cfg->beta2 = 0.999;
    cfg->eps = 1e-8;
    cfg->restarts = 1;
    cfg->seed_x = 1;
    return MSAT_OK;
}

extern "C" const char *msat_last_error(void) { return g_last_error.c_str(); }

static bool valid_restarts(int32_t B) {
    return B >= 1 && B <= 1024 && (B & (B - 1)) == 0;
}

extern "C" int msat_create(msat_ctx **out, int32_t n_vars, int64_t n_clauses,
                           const int64_t *clause_off, const int32_t *lits, const int64_t *weights,
                           const msat_config *cfg_in, void *stream) {
    return msat::ctx_create(out, n_vars, n_clauses, clause_off, lits, weights, cfg_in,
                            (cudaStream_t)stream, false);
}

int msat::ctx_create(msat_ctx **out, int32_t n_vars, int64_t n_clauses, const int64_t *clause_off,
                     const int32_t *lits, const int64_t *weights, const msat_config *cfg_in,
                     cudaStream_t stream, bool pool_alloc) {
    if (!out) return fail(MSAT_EINVAL, "msat_create: out is NULL");
    *out = nullptr;
    msat_config cfg;
    if (cfg_in) cfg = *cfg_in; else msat_config_default(&cfg);
    if (n_vars < 1 || n_vars >= (1 << 30))
        return fail(MSAT_EINVAL, "msat_create: n_vars must be in [1, 2^30)");
    if (n_clauses < 0 || n_clauses >= (1LL << 30))
        return fail(MSAT_EINVAL, "msat_create: n_clauses must be in [0, 2^30)");
    if (!clause_off) return fail(MSAT_EINVAL, "msat_create: clause_off is NULL");
    if (!valid_restarts(cfg.restarts))
        return fail(MSAT_EINVAL, "msat_create: restarts must be a power of two in [1, 1024]");
    if (n_clauses * (int64_t)cfg.restarts >= (1LL << 31) || (int64_t)n_vars * cfg.restarts >= (1LL << 31))
        return fail(MSAT_EINVAL, "msat_create: m * restarts and n * restarts must stay below 2^31");
    if (!(cfg.lr > 0) || !(cfg.beta1 >= 0 && cfg.beta1 < 1) || !(cfg.beta2 >= 0 && cfg.beta2 < 1) ||
        !(cfg.eps >= 0))
        return fail(MSAT_EINVAL, "msat_create: Adam settings out of range");
    const int64_t m = n_clauses;
    // checks, canonical clauses and the transposed CSR (host_cnf.cu, on the
    // host's cores)
    HostCnf hc;
    {
        const int hrc = build_host_cnf(n_vars, m, clause_off, lits, weights, hc);
        if (hrc) return hrc;
    }
    I32Buf &coff = hc.coff, &lit = hc.lit, &voff = hc.voff, &occ = hc.occ;
    const int64_t nnz = hc.nnz, wsum = hc.wsum;
    const int32_t max_len = hc.max_len, kfix = hc.kfix, max_deg = hc.max_deg;
    if ((int64_t)max_deg > 4095LL * 32 * kChunk)
        return fail(MSAT_EINVAL, "msat_create: a variable occurs more than 4095*32768 times");
    const int32_t B = cfg.restarts;
    const int VW = (B % 4 == 0) ? 4 : (B % 2 == 0 ? 2 : 1);
    const int G = B / VW;
    // launch shapes
    auto pow2_le = [](int32_t v, int32_t cap) { return v >= 1 && v <= cap && (v & (v - 1)) == 0; };
    const int32_t fwd_vw = cfg.fwd_vw ? cfg.fwd_vw : auto_fwd_vw(B);
    const int32_t stage_vw = cfg.stage_vw ? cfg.stage_vw : auto_stage_vw(B);
    if (!pow2_le(fwd_vw, std::min(8, B)) || !pow2_le(stage_vw, std::min(16, B)))
        return fail(MSAT_EINVAL, "msat_create: fwd_vw / stage_vw must be powers of two <= min(8 or 16, B)");
    if ((int64_t)fwd_vw * kThreads < B || (int64_t)stage_vw * kThreads < B)
        return fail(MSAT_EINVAL, "msat_create: B / fwd_vw and B / stage_vw must not exceed 256");
    if (cfg.fwd_blocks < 0 || cfg.light_rows < 0 || (cfg.light_rows > 0 && cfg.light_rows < 16))
        return fail(MSAT_EINVAL, "msat_create: fwd_blocks >= 0 and light_rows 0 or >= 16");
    // a light block holds at most task_cap leaf tasks (32-occurrence leaf x
    // group of stage_vw restarts); a variable with more leaves than fit is
    // split into 1024-occurrence chunks instead (heavy variable)
    const int32_t GS = B / stage_vw;
    int32_t task_cap = cfg.light_rows > 0 ? cfg.light_rows : kTaskCap;
    task_cap = std::max(task_cap, GS);
    if (light_smem_bytes(task_cap, stage_vw) > 48 * 1024)
        return fail(MSAT_EINVAL, "msat_create: light_rows x stage_vw x 4 bytes exceeds 48 KiB");
    if (cfg.f_mode < MSAT_F_AUTO || cfg.f_mode > MSAT_F_EXPANDED)
        return fail(MSAT_EINVAL, "msat_create: unknown f_mode");
    if (cfg.f_mode == MSAT_F_EXPANDED && (kfix != 3 || m >= (1LL << 28)))
        return fail(MSAT_EINVAL, "msat_create: MSAT_F_EXPANDED needs every clause to have 3 literals");
    if (cfg.heavy_deg < 0) return fail(MSAT_EINVAL, "msat_create: heavy_deg < 0");
    if (cfg.loss_norm < MSAT_LOSS_MEAN_UNSAT || cfg.loss_norm > MSAT_LOSS_MEAN_ALL)
        return fail(MSAT_EINVAL, "msat_create: unknown loss_norm");
    if (cfg.row_order < 0 || cfg.row_order > 2) return fail(MSAT_EINVAL, "msat_create: unknown row_order");
    const int32_t leaf_room = 32 * (task_cap / GS);  // occurrences of the longest light variable
    const int32_t heavy_deg = std::min(cfg.heavy_deg > 0 ? cfg.heavy_deg : kLightMaxDeg,
                                       std::min(leaf_room, kLightMaxDeg));
    std::vector<int32_t> hvar, hchunk0(1, 0);
    std::vector<int2> lblk;
    {
        int32_t v0 = -1, cnt = 0, tasks_in = 0;
        for (int32_t i = 0; i < n_vars; ++i) {
            const int32_t d = voff[(size_t)i + 1] - voff[(size_t)i];
            if (d > heavy_deg) {
                hvar.push_back(i);
                hchunk0.push_back(hchunk0.back() + (d + kChunk - 1) / kChunk);
                if (v0 >= 0) lblk.push_back(make_int2(v0, i));
                v0 = -1;
                continue;
            }
            const int32_t tasks = std::max(1, (d + 31) / 32) * GS;
            if (v0 >= 0 && (cnt == kThreads || tasks_in + tasks > task_cap)) {
                lblk.push_back(make_int2(v0, i));
                v0 = -1;
            }
            if (v0 < 0) {
                v0 = i;
                cnt = 0;
                tasks_in = 0;
            }
            ++cnt;
            tasks_in += tasks;
        }
        if (v0 >= 0) lblk.push_back(make_int2(v0, n_vars));
    }
    // f of the clause pass is kept (as w*f of unsat clauses) unless the [m][B]
    // array exceeds 8 GiB; otherwise the variable pass recomputes f
    // the stored w*f costs one [m][B] write and one row gather per
    // occurrence; recomputing gathers the unsat bits and every literal's row
    // of t, which measured slower even when the store does not fit in L2
    const bool auto_store = (double)m * B * sizeof(float) <= 8.0 * (1 << 30) || B <= 2;
    const bool use_fstore = cfg.f_mode == MSAT_F_STORE || (cfg.f_mode == MSAT_F_AUTO && auto_store);
    // recomputing f of 3-literal clauses reads the other two literals from an
    // expanded occurrence record streamed with the occurrence list
    const bool expand = cfg.f_mode == MSAT_F_EXPANDED ||
                        (cfg.f_mode == MSAT_F_AUTO && !use_fstore && kfix == 3 && m < (1LL << 28));
    // rows of the store grouped by the variable pass's light blocks (the
    // occurrence words carry rows; every sum keeps its order): by default
    // when the store is above 32 MiB and so mostly gathered from HBM;
    // never for the serving engine's contexts (their batched kernels read
    // clause order)
    const bool block_rows = use_fstore && !expand && !pool_alloc &&
                            (cfg.row_order == 2 ||
                             (cfg.row_order == 0 && (double)m * B * sizeof(float) > 32.0 * (1 << 20)));
    RowOrder ro;
    if (block_rows) {
        const int rrc = build_block_rows(n_vars, m, kfix, coff, lit, weights, lblk, ro);
        if (rrc) return rrc;
    }
    scatter_occurrences(n_vars, m, hc, block_rows ? &ro.row : nullptr);
    std::vector<int2> occx;
    if (expand) {
        occx.resize((size_t)nnz);
        std::vector<int32_t> fill(voff.begin(), voff.end() - 1);
        for (int64_t j = 0; j < m; ++j)
            for (int32_t p = 0; p < 3; ++p) {
                const int32_t L = lit[(size_t)(3 * j + p)];
                const int32_t slot = fill[(size_t)(L >> 1)]++;
                occ[(size_t)slot] = (int32_t)(j << 3) | (p << 1) | (L & 1);
                const int32_t a = lit[(size_t)(3 * j + (p == 0 ? 1 : 0))];
                const int32_t b = lit[(size_t)(3 * j + (p == 2 ? 1 : 2))];
                occx[(size_t)slot] = make_int2(a, b);
            }
    }

    msat_ctx *c = new (std::nothrow) msat_ctx();
    if (!c) return fail(MSAT_ENOMEM, "msat_create: host allocation failed");
    c->cfg = cfg;
    c->stream = stream;
    c->pool_alloc = pool_alloc;
    cudaGetDevice(&c->device);
    c->n = n_vars;
    c->B = cfg.restarts;
    c->m = m;
    c->nnz = nnz;
    c->kfix = kfix;
    c->max_len = max_len;
    c->max_deg = max_deg;
    c->wsum = wsum;
    c->clen = std::move(hc.clen);
    c->taut = std::move(hc.taut);
    if (weights) c->wts.assign(weights, weights + m);

    const int64_t nB = (int64_t)n_vars * B;
    int rc = MSAT_OK;
    int32_t *d_coff = nullptr, *d_lit = nullptr, *d_voff = nullptr, *d_occ = nullptr;
    int32_t *d_hvar = nullptr, *d_hch = nullptr, *d_hofc = nullptr;
    int2 *d_lblk = nullptr, *d_occx = nullptr;
    int32_t *d_plit = nullptr, *d_pcoff = nullptr;
    int64_t *d_pw = nullptr;
    int64_t *d_w = nullptr;
#define TRY_ALLOC(ptr, count)                          \
    do {                                               \
        rc = dalloc_t(c, &(ptr), (size_t)(count));     \
        if (rc) { free_all(c); delete c; return rc; }  \
    } while (0)
    TRY_ALLOC(d_coff, m + 1);
    TRY_ALLOC(d_lit, nnz);
    if (weights) TRY_ALLOC(d_w, m);
    TRY_ALLOC(d_voff, (int64_t)n_vars + 1);
    TRY_ALLOC(d_occ, nnz);
    TRY_ALLOC(d_hvar, (int64_t)hvar.size());
    TRY_ALLOC(d_hch, (int64_t)hchunk0.size());
    TRY_ALLOC(d_hofc, std::max<int64_t>(1, hchunk0.back()));
    TRY_ALLOC(d_lblk, (int64_t)lblk.size());
    if (expand) TRY_ALLOC(d_occx, nnz);
    if (block_rows) {
        TRY_ALLOC(d_plit, nnz);
        if (kfix == 0) TRY_ALLOC(d_pcoff, m + 1);
        if (weights) TRY_ALLOC(d_pw, m);
    }
    if (use_fstore) TRY_ALLOC(c->S.fstore, m * B);
    TRY_ALLOC(c->S.x, nB);
    TRY_ALLOC(c->S.mom, nB);
    TRY_ALLOC(c->S.vel, nB);
    TRY_ALLOC(c->S.t0, nB);
    TRY_ALLOC(c->S.t1, nB);
    TRY_ALLOC(c->S.ubits, (m * B + 31) / 32 + 1);
    TRY_ALLOC(c->S.bestx, nB);

    DevInst &I = c->I;
    I.n = n_vars;
    I.m = (int32_t)m;
    I.B = B;
    I.kfix = kfix;
    I.coff = d_coff;
    I.lit = d_lit;
    I.w = d_w;
    I.voff = d_voff;
    I.occ = d_occ;
    I.heavy_deg = heavy_deg;
    I.n_heavy = (int32_t)hvar.size();
    I.heavy_chunks = hchunk0.back();
    I.heavy_var = d_hvar;
    I.heavy_chunk0 = d_hch;
    I.heavy_of_chunk = d_hofc;
    I.occ_shift = expand ? 3 : 1;
    I.occx = d_occx;
    I.n_lblk = (int32_t)lblk.size();
    I.task_cap = task_cap;
    I.fwd_vw = fwd_vw;
    I.stage_vw = stage_vw;
    I.lblk = d_lblk;
    I.plit = d_plit;
    I.pcoff = d_pcoff;
    I.pw = d_pw;

    DevStep &D = c->D;
    D.fwd_blocks = cfg.fwd_blocks > 0 ? cfg.fwd_blocks : fwd_grid_blocks(I);
    TRY_ALLOC(D.sc, 1);
    TRY_ALLOC(D.wu_acc, (int64_t)kRep * B);
    TRY_ALLOC(D.cost, B);
    TRY_ALLOC(D.best, B);
    TRY_ALLOC(D.best_step, B);
    TRY_ALLOC(D.improved, B);
    TRY_ALLOC(D.cscale, B);
    TRY_ALLOC(D.loss, B);
    TRY_ALLOC(D.lpart, (int64_t)D.fwd_blocks * B);
    TRY_ALLOC(D.hpart, std::max<int64_t>(1, I.heavy_chunks) * B);
    TRY_ALLOC(D.hcount, std::max<int64_t>(1, (int64_t)hvar.size() * G));
#undef TRY_ALLOC

    cudaStream_t st = c->stream;
    auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        if (bytes == 0) return cudaSuccess;
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    StepScalars sc{};
    sc.counter = 0;
    sc.steps_done = 0;
    sc.p1 = 1.0;
    sc.p2 = 1.0;
    sc.lr = cfg.lr;
    sc.beta1 = cfg.beta1;
    sc.beta2 = cfg.beta2;
    sc.eps = cfg.eps;
    sc.b1f = (float)cfg.beta1;
    sc.b2f = (float)cfg.beta2;
    sc.omb1f = (float)(1.0 - cfg.beta1);
    sc.omb2f = (float)(1.0 - cfg.beta2);
    sc.epsf = (float)cfg.eps;
    sc.dense = 1;
    sc.wsum = wsum;
    sc.loss_norm = cfg.loss_norm;
    std::vector<long long> best((size_t)B, (long long)wsum);
    cudaError_t e = cudaSuccess;
    if (!e) e = up(d_coff, coff.data(), sizeof(int32_t) * coff.size());
    if (!e) e = up(d_lit, lit.data(), sizeof(int32_t) * lit.size());
    if (!e && weights) e = up(d_w, weights, sizeof(int64_t) * (size_t)m);
    if (!e) e = up(d_voff, voff.data(), sizeof(int32_t) * voff.size());
    if (!e) e = up(d_occ, occ.data(), sizeof(int32_t) * occ.size());
    if (!e) e = up(d_hvar, hvar.data(), sizeof(int32_t) * hvar.size());
    if (!e) e = up(d_hch, hchunk0.data(), sizeof(int32_t) * hchunk0.size());
    // the heavy variable of every chunk (one load per chunk block)
    std::vector<int32_t> hofc((size_t)std::max<int32_t>(1, hchunk0.back()), 0);
    for (size_t h = 0; h + 1 < hchunk0.size(); ++h)
        for (int32_t ch = hchunk0[h]; ch < hchunk0[h + 1]; ++ch) hofc[(size_t)ch] = (int32_t)h;
    if (!e) e = up(d_hofc, hofc.data(), sizeof(int32_t) * hofc.size());
    if (!e) e = up(d_lblk, lblk.data(), sizeof(int2) * lblk.size());
    if (!e && expand) e = up(d_occx, occx.data(), sizeof(int2) * occx.size());
    if (!e && block_rows) e = up(d_plit, ro.plit.data(), sizeof(int32_t) * ro.plit.size());
    if (!e && d_pcoff) e = up(d_pcoff, ro.pcoff.data(), sizeof(int32_t) * ro.pcoff.size());
    if (!e && d_pw) e = up(d_pw, ro.pw.data(), sizeof(int64_t) * ro.pw.size());
    if (!e) e = up(D.sc, &sc, sizeof(sc));
    if (!e) e = up(D.best, best.data(), sizeof(long long) * best.size());
    if (!e) e = cudaMemsetAsync(D.best_step, 0, sizeof(long long) * (size_t)B, st);
    if (!e) e = cudaMemsetAsync(D.wu_acc, 0, sizeof(unsigned long long) * (size_t)kRep * B, st);
    if (!e) e = cudaMemsetAsync(D.improved, 0, sizeof(int) * (size_t)B, st);
    if (!e) e = cudaMemsetAsync(D.cost, 0, sizeof(long long) * (size_t)B, st);
    if (!e) e = cudaMemsetAsync(D.loss, 0, sizeof(float) * (size_t)B, st);
    if (!e) e = cudaMemsetAsync(D.hcount, 0, sizeof(unsigned) * std::max<size_t>(1, hvar.size() * (size_t)G), st);
    if (!e) e = cudaMemsetAsync(c->S.ubits, 0, sizeof(uint32_t) * (size_t)((m * B + 31) / 32 + 1), st);
    if (!e) e = launch_init(I, c->S, cfg.seed_x, st);
    if (!e) e = cudaStreamSynchronize(st);  // host vectors above are freed on return
    if (e) {
        rc = cuda_fail(e, "msat_create: upload / init");
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return MSAT_OK;
}

extern "C" void msat_destroy(msat_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

void msat::ctx_destroy_async(msat_ctx *c) {
    if (!c) return;
    free_all(c);  // pool allocations are released in order on the context stream
    delete c;
}

extern "C" int msat_set_stream(msat_ctx *c, void *stream) {
    if (!c) return fail(MSAT_EINVAL, "msat_set_stream: ctx is NULL");
    c->stream = (cudaStream_t)stream;
    return MSAT_OK;
}

// One evaluation of the current x (final evaluation of a msat_step call).
static cudaError_t eval_current(msat_ctx *c);
cudaError_t msat::ctx_eval_current(msat_ctx *c) { return eval_current(c); }

static cudaError_t eval_current(msat_ctx *c) {
    prof_begin(c, PROF_FWD);
    cudaError_t e = launch_forward(c->I, c->S, c->D, FWD_EVAL, nullptr, c->stream);
    prof_end(c);
    if (e) return e;
    prof_begin(c, PROF_BWD);
    e = launch_backward(c->I, c->S, c->D, BWD_BITS_ONLY, nullptr, nullptr, nullptr, c->stream);
    prof_end(c);
    return e;
}

// Graph of k steps (clause pass and variable pass, k times), captured on a
// private non-blocking stream: the kernels take the context's device
// pointers by value, so the graph stays valid for the context's lifetime.
static cudaError_t capture_steps(msat_ctx *c, int k, cudaGraphExec_t *out) {
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e) return e;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (!e) {
        cudaError_t le = cudaSuccess;
        for (int s = 0; s < k && !le; ++s) {
            le = launch_forward(c->I, c->S, c->D, FWD_STEP, nullptr, cs);
            if (!le) le = launch_backward(c->I, c->S, c->D, BWD_UPDATE, nullptr, nullptr, nullptr, cs);
        }
        e = cudaStreamEndCapture(cs, &g);
        if (!e) e = le;
    }
    if (!e) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return e;
}

static constexpr int kGraphSteps = 32;

static cudaError_t graph_steps(msat_ctx *c, int64_t n_steps) {
    cudaError_t e = cudaSuccess;
    if (n_steps >= kGraphSteps && !c->graphK) e = capture_steps(c, kGraphSteps, &c->graphK);
    if (!e && n_steps % kGraphSteps && !c->graph1) e = capture_steps(c, 1, &c->graph1);
    for (int64_t s = 0; s + kGraphSteps <= n_steps && !e; s += kGraphSteps)
        e = cudaGraphLaunch(c->graphK, c->stream);
    for (int64_t s = 0; s < n_steps % kGraphSteps && !e; ++s) e = cudaGraphLaunch(c->graph1, c->stream);
    return e;
}

static cudaError_t plain_steps(msat_ctx *c, int64_t n_steps) {
    cudaError_t e = cudaSuccess;
    for (int64_t s = 0; s < n_steps && !e; ++s) {
        prof_begin(c, PROF_FWD);
        e = launch_forward(c->I, c->S, c->D, FWD_STEP, nullptr, c->stream);
        prof_end(c);
        if (e) break;
        prof_begin(c, PROF_BWD);
        e = launch_backward(c->I, c->S, c->D, BWD_UPDATE, nullptr, nullptr, nullptr, c->stream);
        prof_end(c);
    }
    return e;
}

// k steps by the fastest route that gives the same bits: the single-CTA
// kernel for small instances, captured graphs when asked, else plain
// launches (always plain while kernel timing is on, so every pass is timed).
static cudaError_t run_steps(msat_ctx *c, int64_t k, uint32_t flags) {
    if (c->prof_on) return plain_steps(c, k);
    if (!(flags & MSAT_STEP_PER_PASS) && small_fits(c->I, c->max_deg)) {
        cudaError_t e = cudaSuccess;
        for (int64_t done = 0; done < k && !e; done += (1 << 30))
            e = launch_small_steps(c->I, c->S, c->D, (int)std::min<int64_t>(k - done, 1 << 30), c->stream);
        return e;
    }
    return (flags & MSAT_STEP_GRAPH) ? graph_steps(c, k) : plain_steps(c, k);
}

extern "C" int msat_step_ex(msat_ctx *c, int32_t n_steps, uint32_t flags, float *loss_out,
                            int64_t *cost_out) {
    if (!c) return fail(MSAT_EINVAL, "msat_step: ctx is NULL");
    if (n_steps < 0) return fail(MSAT_EINVAL, "msat_step: n_steps < 0");
    if (flags & ~(MSAT_STEP_NO_FINAL_EVAL | MSAT_STEP_GRAPH | MSAT_STEP_PER_PASS))
        return fail(MSAT_EINVAL, "msat_step: unknown flags");
    NvtxRange nv("msat_step");
    cudaError_t e = run_steps(c, n_steps, flags);
    if (!e && !(flags & MSAT_STEP_NO_FINAL_EVAL)) e = eval_current(c);
    if (e) return cuda_fail(e, "msat_step: kernel launch");
    c->steps_done_host += n_steps;
    if (loss_out)
        MSAT_CUDA_TRY(cudaMemcpyAsync(loss_out, c->D.loss, sizeof(float) * (size_t)c->B,
                                      cudaMemcpyDeviceToHost, c->stream));
    if (cost_out)
        MSAT_CUDA_TRY(cudaMemcpyAsync(cost_out, c->D.cost, sizeof(int64_t) * (size_t)c->B,
                                      cudaMemcpyDeviceToHost, c->stream));
    if (loss_out || cost_out) MSAT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return MSAT_OK;
}

extern "C" int msat_step(msat_ctx *c, int32_t n_steps, float *loss_out, int64_t *cost_out) {
    return msat_step_ex(c, n_steps, 0u, loss_out, cost_out);
}

extern "C" int msat_solve(msat_ctx *c, int64_t max_steps, double time_limit_s, int32_t chunk,
                          int64_t *steps_out, double *elapsed_out, int64_t *trace_cost,
                          double *trace_time, int32_t trace_cap, int32_t *trace_len) {
    if (!c) return fail(MSAT_EINVAL, "msat_solve: ctx is NULL");
    if (max_steps < 0 || chunk < 1 || trace_cap < 0 || !(time_limit_s >= 0.0))
        return fail(MSAT_EINVAL, "msat_solve: max_steps >= 0, chunk >= 1, trace_cap >= 0 and "
                                 "time_limit_s >= 0 required");
    if (trace_cap > 0 && (!trace_cost || !trace_time))
        return fail(MSAT_EINVAL, "msat_solve: trace buffers are NULL");
    NvtxRange nv("msat_solve");
    const auto t0 = std::chrono::steady_clock::now();
    auto seconds = [&] {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    std::vector<long long> best((size_t)c->B);
    int64_t done = 0;
    int32_t tl = 0;
    auto read_best = [&](long long *bmin) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(best.data(), c->D.best, sizeof(long long) * best.size(),
                                        cudaMemcpyDeviceToHost, c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
        *bmin = *std::min_element(best.begin(), best.end());
        return e;
    };
    auto trace = [&](long long bmin) {
        if (tl < trace_cap) {
            trace_cost[tl] = bmin;
            trace_time[tl] = seconds();
            ++tl;
        }
    };
    for (;;) {
        const int64_t k = std::min<int64_t>(chunk, max_steps - done);
        cudaError_t e = cudaSuccess;
        if (k > 0) e = run_steps(c, k, MSAT_STEP_GRAPH);
        done += k;
        long long bmin = 0;
        if (!e) e = read_best(&bmin);
        if (e) return cuda_fail(e, "msat_solve");
        trace(bmin);
        if (done >= max_steps || bmin == 0 || seconds() >= time_limit_s) break;
    }
    // the final x is evaluated once, as msat_step does
    long long bmin = 0;
    cudaError_t e = eval_current(c);
    if (!e) e = read_best(&bmin);
    if (e) return cuda_fail(e, "msat_solve: final evaluation");
    trace(bmin);
    c->steps_done_host += done;
    if (steps_out) *steps_out = done;
    if (elapsed_out) *elapsed_out = seconds();
    if (trace_len) *trace_len = tl;
    return MSAT_OK;
}

extern "C" int msat_profile_enable(msat_ctx *c, int on) {
    if (!c) return fail(MSAT_EINVAL, "msat_profile_enable: ctx is NULL");
    c->prof_on = on != 0;
    return MSAT_OK;
}

extern "C" int msat_profile_read(msat_ctx *c, msat_profile *out, int reset) {
    if (!c || !out) return fail(MSAT_EINVAL, "msat_profile_read: NULL argument");
    memset(out, 0, sizeof(*out));
    if (c->prof_used) MSAT_CUDA_TRY(cudaEventSynchronize(c->prof_ev[2 * c->prof_used - 1]));
    for (size_t k = 0; k < c->prof_used; ++k) {
        float ms = 0.0f;
        MSAT_CUDA_TRY(cudaEventElapsedTime(&ms, c->prof_ev[2 * k], c->prof_ev[2 * k + 1]));
        const int kind = c->prof_kind[k];
        out->launches[kind] += 1;
        out->ms[kind] += ms;
    }
    if (reset) c->prof_used = 0;
    return MSAT_OK;
}

// First use of the dense backend: the clause matrix W^T [m_pad][n_pad] in
// packed e2m1 (two codes a byte, zero padding), per-clause targets -len_j (NaN for padding rows and for
// clauses holding some x and not x, which are never unsat), 32-bit weights
// and the TMA descriptor of W^T.
static int dense_setup(msat_ctx *c) {
    if (c->dense_ready) return MSAT_OK;
    for (int64_t w : c->wts)
        if (w >= (1LL << 25))
            return fail(MSAT_EINVAL, "msat_evaluate: the dense backend needs clause weights below 2^25");
    DenseDev &d = c->dense;
    d.m_pad = (int)std::max<int64_t>(128, (c->m + 127) / 128 * 128);
    d.n_pad = (c->n + kDenseKStep - 1) / kDenseKStep * kDenseKStep;
    const double bytes = (double)d.m_pad * (double)d.n_pad / 2;
    if (bytes > 64.0 * (1LL << 30))
        return fail(MSAT_EINVAL, "msat_evaluate: the dense clause matrix would take " +
                                     std::to_string((long long)(bytes / (1 << 20))) + " MiB (limit 64 GiB)");
    int rc;
    if ((rc = dalloc_t(c, &d.Wt, (size_t)d.m_pad * d.n_pad / 2))) return rc;
    if ((rc = dalloc_t(c, &d.target, (size_t)d.m_pad))) return rc;
    if ((rc = dalloc_t(c, &d.wgt, (size_t)d.m_pad))) return rc;
    if ((rc = dalloc_t(c, &d.errflag, 1))) return rc;
    std::vector<float> tgt((size_t)d.m_pad, std::nanf(""));
    std::vector<uint32_t> w32((size_t)d.m_pad, 0u);
    d.unit_w = true;
    for (int64_t j = 0; j < c->m; ++j) {
        if (!c->taut[(size_t)j]) tgt[(size_t)j] = -(float)c->clen[(size_t)j];
        w32[(size_t)j] = c->wts.empty() ? 1u : (uint32_t)c->wts[(size_t)j];
        d.unit_w = d.unit_w && w32[(size_t)j] == 1u;
    }
    cudaStream_t st = c->stream;
    MSAT_CUDA_TRY(cudaMemsetAsync(d.Wt, 0, (size_t)d.m_pad * d.n_pad / 2, st));
    MSAT_CUDA_TRY(cudaMemsetAsync(d.errflag, 0, sizeof(unsigned), st));
    MSAT_CUDA_TRY(cudaMemcpyAsync(d.target, tgt.data(), sizeof(float) * tgt.size(), cudaMemcpyHostToDevice, st));
    MSAT_CUDA_TRY(cudaMemcpyAsync(d.wgt, w32.data(), sizeof(uint32_t) * w32.size(), cudaMemcpyHostToDevice, st));
    cudaError_t e = launch_dense_fill(c->I, d.Wt, d.n_pad, st);
    if (e) return cuda_fail(e, "msat_evaluate: dense matrix fill");
    MSAT_CUDA_TRY(cudaStreamSynchronize(st));  // host vectors above are freed on return
    if ((rc = dense_encode_a(d))) return rc;
    if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        d.sm_count = 0;
    }
    c->dense_ready = true;
    return MSAT_OK;
}

extern "C" int msat_check(msat_ctx *c) {
    if (!c) return fail(MSAT_EINVAL, "msat_check: ctx is NULL");
    MSAT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->dense.errflag) {
        unsigned flag = 0;
        MSAT_CUDA_TRY(cudaMemcpy(&flag, c->dense.errflag, sizeof(flag), cudaMemcpyDeviceToHost));
        if (flag) {
            MSAT_CUDA_TRY(cudaMemset(c->dense.errflag, 0, sizeof(unsigned)));
            // an aborted launch may have left split-tile counts behind
            if (c->dense.part_cnt)
                MSAT_CUDA_TRY(cudaMemset(c->dense.part_cnt, 0, sizeof(unsigned) * c->dense.part_cnts));
            return fail(MSAT_ETIMEOUT, "a bounded wait in the dense evaluation kernel gave up (flag " +
                                           std::to_string(flag) + ")");
        }
    }
    return MSAT_OK;
}

static int dense_eval(msat_ctx *c, const int8_t *a, const float *x, int32_t nb, int64_t *cost_out);

extern "C" int msat_evaluate(msat_ctx *c, const int8_t *assign_pm1, int32_t nb, int64_t *cost_out,
                             int32_t backend) {
    if (!c) return fail(MSAT_EINVAL, "msat_evaluate: ctx is NULL");
    if (nb < 1 || !assign_pm1 || !cost_out)
        return fail(MSAT_EINVAL, "msat_evaluate: need nb >= 1 and non-NULL buffers");
    if (backend == MSAT_BACKEND_SPARSE) {
        prof_begin(c, PROF_EVAL);
        cudaError_t e = launch_eval_sparse(c->I, assign_pm1, nb, (long long *)cost_out, c->stream);
        prof_end(c);
        if (e) return cuda_fail(e, "msat_evaluate: sparse kernel");
        return MSAT_OK;
    }
    if (backend == MSAT_BACKEND_DENSE) return dense_eval(c, assign_pm1, nullptr, nb, cost_out);
    return fail(MSAT_EINVAL, "msat_evaluate: unknown backend");
}

// Tensor-core evaluation of a batch given as int8 +-1 (a) or as relaxed x
// read through its rounding (x; the current x of the context).
static int dense_eval(msat_ctx *c, const int8_t *a, const float *x, int32_t nb, int64_t *cost_out) {
    NvtxRange nv("msat_evaluate dense");
    int rc = dense_setup(c);
    if (rc) return rc;
    const int rows = dense_rows(nb), ntile = dense_tile_n(nb);
    const size_t need = (size_t)rows * c->dense.n_pad / 2;  // packed 4-bit codes
    if (need > c->dense.xt_bytes) {
        if (c->dense.Xt) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->dense.Xt);
            c->dense.Xt = nullptr;
            c->dense.xt_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&c->dense.Xt, need);
        if (e) {
            cudaGetLastError();
            c->dense.Xt = nullptr;
            return fail(MSAT_ENOMEM, "msat_evaluate: dense assignment buffer allocation failed");
        }
        c->dense.xt_bytes = need;
        c->dense.tmB_rows = 0;
    }
    if (c->dense.tmB_rows != rows || c->dense.tmB_ntile != ntile) {
        rc = dense_encode_b(c->dense, rows, ntile);
        if (rc) return rc;
    }
    {
        // split tiles: per-piece targets (built when the plan changes), the
        // pieces' bit masks and their counters (zeroed once; every launch
        // leaves them zeroed)
        DenseDev &d = c->dense;
        int grid = 0;
        const DenseSched p = dense_plan(d, ntile, &grid);
        if (p.tail > 0) {
            const int slots = p.tail * p.split;
            if (slots > d.ptgt_slots || p.tail > d.part_cnts || ntile != d.pmask_ntile) {
                cudaStreamSynchronize(c->stream);
                if (d.ptgt) cudaFree(d.ptgt);
                if (d.pmask) cudaFree(d.pmask);
                if (d.part_cnt) cudaFree(d.part_cnt);
                d.ptgt = nullptr;
                d.pmask = nullptr;
                d.part_cnt = nullptr;
                d.ptgt_slots = d.part_cnts = d.pmask_ntile = 0;
                d.plan_grid = -1;
                cudaError_t e = cudaMalloc(&d.ptgt, sizeof(float) * (size_t)slots * 128);
                if (!e) e = cudaMalloc(&d.pmask, sizeof(uint32_t) * (size_t)slots * ((ntile + 31) / 32) * 128);
                if (!e) e = cudaMalloc(&d.part_cnt, sizeof(unsigned) * (size_t)p.tail);
                if (!e) e = cudaMemsetAsync(d.part_cnt, 0, sizeof(unsigned) * (size_t)p.tail, c->stream);
                if (e) {
                    cudaGetLastError();
                    return fail(MSAT_ENOMEM, "msat_evaluate: dense split-tile buffer allocation failed");
                }
                d.ptgt_slots = slots;
                d.part_cnts = p.tail;
                d.pmask_ntile = ntile;
            }
            if (grid != d.plan_grid || memcmp(&p, &d.plan, sizeof(p)) != 0) {
                cudaError_t e = launch_dense_piece_targets(c->I, d, p, grid, c->stream);
                if (e) return cuda_fail(e, "msat_evaluate: dense piece targets");
                d.plan = p;
                d.plan_grid = grid;
            }
        }
    }
    prof_begin(c, PROF_OTHER);
    cudaError_t e = x ? launch_dense_convert_x(c->dense, x, c->n, nb, (long long *)cost_out, c->stream)
                      : launch_dense_convert(c->dense, a, c->n, nb, (long long *)cost_out, c->stream);
    prof_end(c);
    if (e) return cuda_fail(e, "msat_evaluate: dense batch conversion");
    prof_begin(c, PROF_EVAL);
    e = launch_dense_gemm(c->dense, nb, (long long *)cost_out, c->stream);
    prof_end(c);
    if (e) return cuda_fail(e, "msat_evaluate: dense tensor-core kernel");
    return MSAT_OK;
}

extern "C" int msat_evaluate_x(msat_ctx *c, int32_t backend, int64_t *cost_out) {
    if (!c || !cost_out) return fail(MSAT_EINVAL, "msat_evaluate_x: NULL argument");
    // the tensor-core operand is built from x directly (rounding and transposition in one kernel)
    if (backend == MSAT_BACKEND_DENSE) return dense_eval(c, nullptr, c->S.x, c->B, cost_out);
    const long long nB = (long long)c->n * c->B;
    if (!c->xpm1) {
        int rc = dalloc_t(c, &c->xpm1, (size_t)nB);
        if (rc) return rc;
    }
    prof_begin(c, PROF_OTHER);
    cudaError_t e = launch_round_pm1(c->S.x, c->xpm1, nB, c->stream);
    prof_end(c);
    if (e) return cuda_fail(e, "msat_evaluate_x: rounding kernel");
    return msat_evaluate(c, c->xpm1, c->B, cost_out, backend);
}

extern "C" int msat_heuristic_gap(msat_ctx *c, int64_t *heur_unsat, int64_t *disagree) {
    if (!c || !heur_unsat || !disagree) return fail(MSAT_EINVAL, "msat_heuristic_gap: NULL argument");
    if (!c->hgap) {
        const int rc = dalloc_t(c, &c->hgap, (size_t)2 * c->B);  // freed with the context
        if (rc) return rc;
    }
    long long *d = c->hgap;
    cudaError_t e = launch_heuristic_gap(c->I, c->S.x, d, d + c->B, c->stream);
    if (!e) e = cudaMemcpyAsync(heur_unsat, d, sizeof(int64_t) * (size_t)c->B, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(disagree, d + c->B, sizeof(int64_t) * (size_t)c->B, cudaMemcpyDeviceToHost,
                                c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(e, "msat_heuristic_gap");
    return MSAT_OK;
}

extern "C" int msat_best(msat_ctx *c, uint8_t *assign01, int64_t *best_cost) {
    if (!c) return fail(MSAT_EINVAL, "msat_best: ctx is NULL");
    if (best_cost)
        MSAT_CUDA_TRY(cudaMemcpyAsync(best_cost, c->D.best, sizeof(int64_t) * (size_t)c->B,
                                      cudaMemcpyDeviceToHost, c->stream));
    std::vector<uint8_t> tmp;
    if (assign01) {
        tmp.resize((size_t)c->n * c->B);
        MSAT_CUDA_TRY(cudaMemcpyAsync(tmp.data(), c->S.bestx, tmp.size(), cudaMemcpyDeviceToHost,
                                      c->stream));
    }
    MSAT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (assign01)
        for (int32_t i = 0; i < c->n; ++i)
            for (int32_t b = 0; b < c->B; ++b)
                assign01[(size_t)b * c->n + i] = tmp[(size_t)i * c->B + b];
    return MSAT_OK;
}

extern "C" int msat_get_x(msat_ctx *c, float *x_host) {
    if (!c || !x_host) return fail(MSAT_EINVAL, "msat_get_x: NULL argument");
    MSAT_CUDA_TRY(cudaMemcpyAsync(x_host, c->S.x, sizeof(float) * (size_t)c->n * c->B,
                                  cudaMemcpyDeviceToHost, c->stream));
    MSAT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return MSAT_OK;
}

extern "C" int msat_get_info(msat_ctx *c, msat_info *info) {
    if (!c || !info) return fail(MSAT_EINVAL, "msat_get_info: NULL argument");
    StepScalars sc;
    MSAT_CUDA_TRY(cudaMemcpyAsync(&sc, c->D.sc, sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
    MSAT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    memset(info, 0, sizeof(*info));
    info->n = c->n;
    info->restarts = c->B;
    info->m = c->m;
    info->nnz = c->nnz;
    info->steps_done = sc.steps_done;
    info->device_bytes = c->device_bytes;
    info->max_clause_len = c->max_len;
    info->max_degree = c->max_deg;
    info->n_heavy = c->I.n_heavy;
    info->uniform_len = c->kfix;
    info->small_kernel = small_fits(c->I, c->max_deg) ? 1 : 0;
    return MSAT_OK;
}

extern "C" int msat_get_state(msat_ctx *c, float *x, float *mom, float *vel, int64_t *best_cost,
                              uint8_t *best_assign, int64_t *steps_done, double *adam_pow) {
    if (!c) return fail(MSAT_EINVAL, "msat_get_state: ctx is NULL");
    const size_t nB = (size_t)c->n * c->B;
    cudaStream_t st = c->stream;
    if (x) MSAT_CUDA_TRY(cudaMemcpyAsync(x, c->S.x, sizeof(float) * nB, cudaMemcpyDeviceToHost, st));
    if (mom) MSAT_CUDA_TRY(cudaMemcpyAsync(mom, c->S.mom, sizeof(float) * nB, cudaMemcpyDeviceToHost, st));
    if (vel) MSAT_CUDA_TRY(cudaMemcpyAsync(vel, c->S.vel, sizeof(float) * nB, cudaMemcpyDeviceToHost, st));
    if (best_cost)
        MSAT_CUDA_TRY(cudaMemcpyAsync(best_cost, c->D.best, sizeof(int64_t) * (size_t)c->B,
                                      cudaMemcpyDeviceToHost, st));
    if (best_assign)
        MSAT_CUDA_TRY(cudaMemcpyAsync(best_assign, c->S.bestx, nB, cudaMemcpyDeviceToHost, st));
    StepScalars sc;
    MSAT_CUDA_TRY(cudaMemcpyAsync(&sc, c->D.sc, sizeof(sc), cudaMemcpyDeviceToHost, st));
    MSAT_CUDA_TRY(cudaStreamSynchronize(st));
    if (steps_done) *steps_done = sc.steps_done;
    if (adam_pow) {
        adam_pow[0] = sc.p1;
        adam_pow[1] = sc.p2;
    }
    return MSAT_OK;
}

extern "C" int msat_set_state(msat_ctx *c, const float *x, const float *mom, const float *vel,
                              const int64_t *best_cost, const uint8_t *best_assign,
                              int64_t steps_done, const double *adam_pow) {
    if (!c || !x || !mom || !vel || !best_cost || !best_assign || !adam_pow)
        return fail(MSAT_EINVAL, "msat_set_state: NULL argument");
    if (steps_done < 0) return fail(MSAT_EINVAL, "msat_set_state: steps_done < 0");
    const size_t nB = (size_t)c->n * c->B;
    cudaStream_t st = c->stream;
    StepScalars sc;
    MSAT_CUDA_TRY(cudaMemcpyAsync(&sc, c->D.sc, sizeof(sc), cudaMemcpyDeviceToHost, st));
    MSAT_CUDA_TRY(cudaStreamSynchronize(st));
    sc.counter = 0;
    sc.steps_done = steps_done;
    sc.p1 = adam_pow[0];
    sc.p2 = adam_pow[1];
    MSAT_CUDA_TRY(cudaMemcpyAsync(c->D.sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, st));
    MSAT_CUDA_TRY(cudaMemcpyAsync(c->S.x, x, sizeof(float) * nB, cudaMemcpyHostToDevice, st));
    MSAT_CUDA_TRY(cudaMemcpyAsync(c->S.mom, mom, sizeof(float) * nB, cudaMemcpyHostToDevice, st));
    MSAT_CUDA_TRY(cudaMemcpyAsync(c->S.vel, vel, sizeof(float) * nB, cudaMemcpyHostToDevice, st));
    // the step of a restored best is not part of a checkpoint: it reads 0 after a restore
    MSAT_CUDA_TRY(cudaMemsetAsync(c->D.best_step, 0, sizeof(int64_t) * (size_t)c->B, st));
    MSAT_CUDA_TRY(cudaMemcpyAsync(c->D.best, best_cost, sizeof(int64_t) * (size_t)c->B,
                                  cudaMemcpyHostToDevice, st));
    MSAT_CUDA_TRY(cudaMemcpyAsync(c->S.bestx, best_assign, nB, cudaMemcpyHostToDevice, st));
    // the forward pass reads tanh(x) from the buffer of the current parity
    float *tcur = (steps_done & 1) ? c->S.t1 : c->S.t0;
    cudaError_t e = launch_tanh(c->S.x, tcur, (int64_t)nB, st);
    if (e) return cuda_fail(e, "msat_set_state: tanh kernel");
    MSAT_CUDA_TRY(cudaStreamSynchronize(st));
    c->steps_done_host = steps_done;
    return MSAT_OK;
}

// ------------------------------------------------------------ probe path

static int ensure_probe(msat_ctx *c) {
    if (c->probe_ready) return MSAT_OK;
    const int32_t B = c->B;
    const int64_t nB = (int64_t)c->n * B;
    c->PS = c->S;
    c->PD = c->D;
    int rc;
    if ((rc = dalloc_t(c, &c->PS.t0, nB))) return rc;
    c->PS.t1 = c->PS.t0;
    if ((rc = dalloc_t(c, &c->PS.ubits, (c->m * B + 31) / 32 + 1))) return rc;
    if ((rc = dalloc_t(c, &c->PD.sc, 1))) return rc;
    if ((rc = dalloc_t(c, &c->PD.wu_acc, (int64_t)kRep * B))) return rc;
    if (c->S.fstore && (rc = dalloc_t(c, &c->PS.fstore, c->m * B))) return rc;
    if ((rc = dalloc_t(c, &c->PD.cost, B))) return rc;
    if ((rc = dalloc_t(c, &c->PD.cscale, B))) return rc;
    if ((rc = dalloc_t(c, &c->PD.lpart, (int64_t)c->PD.fwd_blocks * B))) return rc;
    c->PD.best = nullptr;
    c->PD.best_step = nullptr;
    c->PD.improved = nullptr;
    StepScalars sc;
    MSAT_CUDA_TRY(cudaMemcpyAsync(&sc, c->D.sc, sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
    MSAT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    sc.counter = 0;
    sc.steps_done = 0;
    MSAT_CUDA_TRY(cudaMemcpyAsync(c->PD.sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, c->stream));
    MSAT_CUDA_TRY(cudaMemsetAsync(c->PD.wu_acc, 0, sizeof(unsigned long long) * (size_t)kRep * B, c->stream));
    MSAT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->probe_ready = true;
    return MSAT_OK;
}

extern "C" int msat_forward(msat_ctx *c, const float *x, float *loss, int64_t *cost) {
    if (!c || !x || !loss) return fail(MSAT_EINVAL, "msat_forward: NULL argument");
    int rc = ensure_probe(c);
    if (rc) return rc;
    cudaStream_t st = c->stream;
    const int64_t nB = (int64_t)c->n * c->B;
    cudaError_t e = launch_tanh(x, c->PS.t0, nB, st);
    if (!e) e = launch_forward(c->I, c->PS, c->PD, FWD_PROBE, c->PS.t0, st);
    DevStep d = c->PD;
    d.loss = loss;
    if (!e) e = launch_loss_reduce(d, c->B, st);
    if (!e && cost)
        e = cudaMemcpyAsync(cost, c->PD.cost, sizeof(int64_t) * (size_t)c->B,
                            cudaMemcpyDeviceToDevice, st);
    if (e) return cuda_fail(e, "msat_forward");
    return MSAT_OK;
}

extern "C" int msat_backward(msat_ctx *c, const float *gscale, float *grad) {
    if (!c || !grad) return fail(MSAT_EINVAL, "msat_backward: NULL argument");
    if (!c->probe_ready) return fail(MSAT_ESTATE, "msat_backward: no msat_forward before it");
    // 1 - t^2 comes from the tanh(x) stored by msat_forward
    cudaError_t e = launch_backward(c->I, c->PS, c->PD, BWD_GRAD_ONLY, c->PS.t0, gscale, grad,
                                    c->stream);
    if (e) return cuda_fail(e, "msat_backward");
    return MSAT_OK;
}

extern "C" int msat_selftest_bounded_wait(int64_t spins) {
    if (spins < 0 || spins > (1LL << 24))
        return fail(MSAT_EINVAL, "msat_selftest_bounded_wait: spins must be in [0, 2^24]");
    unsigned int *flag = nullptr;
    cudaError_t e = cudaMalloc(&flag, sizeof(unsigned));
    if (e) return cuda_fail(e, "msat_selftest_bounded_wait: allocation");
    unsigned h = 0;
    e = cudaMemset(flag, 0, sizeof(unsigned));
    if (!e) e = launch_wait_selftest(spins, flag, nullptr);
    if (!e) e = cudaMemcpy(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(flag);
    if (e) return cuda_fail(e, "msat_selftest_bounded_wait");
    if (h)
        return fail(MSAT_ETIMEOUT, "msat_selftest_bounded_wait: the wait gave up after " +
                                       (spins ? std::to_string(spins) + " tries" : std::string("its time limit")) +
                                       " (flag " + std::to_string(h) + ")");
    return MSAT_OK;
}

extern "C" int msat_dense_mma_rate(int32_t n_assign, int32_t iters, double *tflops) {
    if (!tflops) return fail(MSAT_EINVAL, "msat_dense_mma_rate: NULL argument");
    if (n_assign < 16 || n_assign > 256 || n_assign % 16 != 0)
        return fail(MSAT_EINVAL, "msat_dense_mma_rate: n_assign must be a multiple of 16 in [16, 256]");
    if (iters < 1 || iters > (1 << 20)) return fail(MSAT_EINVAL, "msat_dense_mma_rate: iters must be in [1, 2^20]");
    int dev = 0, sms = 0;
    MSAT_CUDA_TRY(cudaGetDevice(&dev));
    MSAT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    unsigned int *flag = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&flag, sizeof(unsigned));
    if (e) return cuda_fail(e, "msat_dense_mma_rate: allocation");
    float ms = 0.0f;
    unsigned h = 0;
    e = cudaMemset(flag, 0, sizeof(unsigned));
    if (!e) e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    if (!e) e = launch_mma_rate(n_assign, iters, sms, flag, nullptr);  // warm-up
    if (!e) e = cudaEventRecord(e0, nullptr);
    if (!e) e = launch_mma_rate(n_assign, iters, sms, flag, nullptr);
    if (!e) e = cudaEventRecord(e1, nullptr);
    if (!e) e = cudaEventSynchronize(e1);
    if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
    if (!e) e = cudaMemcpy(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(flag);
    if (e) return cuda_fail(e, "msat_dense_mma_rate");
    if (h) return fail(MSAT_ETIMEOUT, "msat_dense_mma_rate: a wait gave up (flag " + std::to_string(h) + ")");
    // four MMAs of 128 x n_assign x 64 multiply-adds a stage, on every SM
    const double flops = 2.0 * 128.0 * n_assign * 64.0 * 4.0 * (double)iters * (double)sms;
    *tflops = flops / ((double)ms * 1e-3) / 1e12;
    return MSAT_OK;
}

extern "C" int msat_best_step(msat_ctx *c, int64_t *best_step) {
    if (!c || !best_step) return fail(MSAT_EINVAL, "msat_best_step: NULL argument");
    MSAT_CUDA_TRY(cudaMemcpyAsync(best_step, c->D.best_step, sizeof(int64_t) * (size_t)c->B,
                                  cudaMemcpyDeviceToHost, c->stream));
    MSAT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return MSAT_OK;
}
