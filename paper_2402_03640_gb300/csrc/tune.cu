// Launch-shape autotuner (msat_autotune).
//
// The launch shapes -- restarts per thread of the clause pass (fwd_vw) and
// of the light-variable leaf tasks (stage_vw), leaf tasks per light block
// (light_rows) -- never change a result bit: every sum runs in the order the
// instance fixes.  So the tuner only times.  It builds a scratch context per
// candidate on the caller's stream (stage_vw and light_rows change the
// light-block partition, which is built at creation), runs warm-up steps,
// times n_steps steps with CUDA events and keeps the fastest, one parameter
// at a time: stage_vw, then light_rows, then fwd_vw.  Winners are cached for
// the process by instance shape, so a second create of a like instance does
// not tune again.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ctx.cuh"

using namespace msat;

namespace {

using TuneKey = std::tuple<int, int32_t, int64_t, int64_t, int32_t, int32_t, int32_t, int32_t>;

struct TuneWin {
    int32_t fwd_vw, stage_vw, light_rows;
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneWin> g_tune_cache;

// Milliseconds per step of one launch shape in *ms; a non-zero return is
// the error of creating or stepping the scratch context (message set).
int time_shape(int32_t n, int64_t m, const int64_t *off, const int32_t *lits, const int64_t *w,
               const msat_config &cfg, cudaStream_t st, int32_t n_steps, float *ms) {
    msat_ctx *c = nullptr;
    int rc = ctx_create(&c, n, m, off, lits, w, &cfg, st, false);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    if (e) rc = cuda_fail(e, "msat_autotune: event");
    if (!rc) rc = msat_step_ex(c, 2, MSAT_STEP_NO_FINAL_EVAL, nullptr, nullptr);
    if (!rc && (e = cudaEventRecord(e0, st))) rc = cuda_fail(e, "msat_autotune: event");
    if (!rc) rc = msat_step_ex(c, n_steps, MSAT_STEP_NO_FINAL_EVAL, nullptr, nullptr);
    if (!rc && (e = cudaEventRecord(e1, st))) rc = cuda_fail(e, "msat_autotune: event");
    if (!rc && (e = cudaEventSynchronize(e1))) rc = cuda_fail(e, "msat_autotune: timing");
    if (!rc && (e = cudaEventElapsedTime(ms, e0, e1))) rc = cuda_fail(e, "msat_autotune: timing");
    if (!rc) *ms /= (float)n_steps;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    msat_destroy(c);
    return rc;
}

bool pow2_ok(int32_t v, int32_t B, int32_t cap) {
    return v >= 1 && v <= cap && v <= B && (v & (v - 1)) == 0 && (int64_t)v * kThreads >= B;
}

}  // namespace

extern "C" int msat_autotune(int32_t n_vars, int64_t n_clauses, const int64_t *clause_off,
                             const int32_t *lits, const int64_t *weights, const msat_config *cfg_in,
                             void *stream, int32_t n_steps, msat_config *cfg_out,
                             msat_tune_entry *entries, int32_t cap, int32_t *n_entries) {
    if (!cfg_out || n_steps < 1 || cap < 0 || (cap > 0 && !entries) || !clause_off)
        return fail(MSAT_EINVAL, "msat_autotune: cfg_out, clause_off NULL, n_steps < 1 or bad entries");
    msat_config base;
    if (cfg_in) base = *cfg_in; else msat_config_default(&base);
    base.fwd_vw = base.stage_vw = base.light_rows = base.fwd_blocks = 0;
    const int32_t B = base.restarts;
    if (n_entries) *n_entries = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    int64_t nnz = n_clauses >= 0 ? clause_off[n_clauses] - clause_off[0] : 0;
    const TuneKey key{dev, n_vars, n_clauses, nnz, B, base.f_mode, weights != nullptr, base.heavy_deg};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *cfg_out = base;
            cfg_out->fwd_vw = it->second.fwd_vw;
            cfg_out->stage_vw = it->second.stage_vw;
            cfg_out->light_rows = it->second.light_rows;
            return MSAT_OK;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    int32_t used = 0;
    msat_config best = base;
    float best_ms = -1.0f;
    auto trial = [&](const msat_config &cand) -> int {
        float ms = 0.0f;
        const int rc = time_shape(n_vars, n_clauses, clause_off, lits, weights, cand, st, n_steps, &ms);
        if (rc) return rc;
        if (used < cap) {
            entries[used].fwd_vw = cand.fwd_vw;
            entries[used].stage_vw = cand.stage_vw;
            entries[used].light_rows = cand.light_rows;
            entries[used].ms_per_step = ms;
        }
        ++used;
        if (best_ms < 0.0f || ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
        return MSAT_OK;
    };
    // the automatic shape first: it is the reference every candidate must beat
    msat_config cand = base;
    cand.fwd_vw = auto_fwd_vw(B);
    cand.stage_vw = auto_stage_vw(B);
    cand.light_rows = kTaskCap;
    int rc = trial(cand);
    if (rc) return rc;  // the instance itself was rejected, or the device failed
    for (int32_t sv : {1, 2, 4, 8}) {
        if (!pow2_ok(sv, B, 8) || sv == best.stage_vw) continue;
        cand = best;
        cand.stage_vw = sv;
        if ((rc = trial(cand)) == MSAT_ECUDA) return rc;
    }
    for (int32_t lr : {128, 256, 512}) {
        if (lr == best.light_rows) continue;
        cand = best;
        cand.light_rows = lr;
        if ((rc = trial(cand)) == MSAT_ECUDA) return rc;
    }
    for (int32_t fv : {1, 2, 4, 8}) {
        if (!pow2_ok(fv, B, 8) || fv == best.fwd_vw) continue;
        cand = best;
        cand.fwd_vw = fv;
        if ((rc = trial(cand)) == MSAT_ECUDA) return rc;
    }
    if (n_entries) *n_entries = used < cap ? used : cap;
    *cfg_out = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = TuneWin{best.fwd_vw, best.stage_vw, best.light_rows};
    return MSAT_OK;
}
