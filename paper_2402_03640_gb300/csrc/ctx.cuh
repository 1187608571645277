// Internal: the context object behind msat_ctx, shared by the C ABI
// (api.cu) and the serving engine (server.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "msat_internal.cuh"

// Device memory of one context.  Every buffer is a separate allocation so
// each starts on a 256-byte boundary (vector loads need 16 bytes).
struct msat_ctx {
    bool pool_alloc = false;  // stream-ordered allocations (contexts of the server)
    msat_config cfg;
    cudaStream_t stream = nullptr;
    int device = 0;
    int32_t n = 0, B = 0;
    int64_t m = 0, nnz = 0;
    int32_t kfix = 0, max_len = 0, max_deg = 0;
    int64_t wsum = 0;
    int64_t steps_done_host = 0;
    std::vector<void *> allocs;
    int64_t device_bytes = 0;

    msat::DevInst I{};
    msat::DevState S{};
    msat::DevStep D{};

    // probe (autograd) path, allocated on first use
    bool probe_ready = false;
    msat::DevState PS{};
    msat::DevStep PD{};

    // dense tensor-core evaluation, set up on first use
    std::vector<int32_t> clen;    // canonical clause lengths
    std::vector<uint8_t> taut;    // clause holds some x and not x
    std::vector<int64_t> wts;     // clause weights (empty: all 1)
    bool dense_ready = false;
    msat::DenseDev dense;
    int8_t *xpm1 = nullptr;       // rounded x as a +-1 batch, allocated on first use
    long long *hgap = nullptr;    // [2][B] counts of msat_heuristic_gap, allocated on first use

    // CUDA graphs of 1 and kGraphSteps steps (MSAT_STEP_GRAPH), captured on first use
    cudaGraphExec_t graph1 = nullptr, graphK = nullptr;

    // kernel timing (msat_profile_*): event pairs around each launch
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_kind;
    size_t prof_used = 0;
};

namespace msat {

// msat_create with an explicit stream; pool_alloc: allocate with
// cudaMallocAsync on that stream (freed with cudaFreeAsync in order).
int ctx_create(msat_ctx **out, int32_t n_vars, int64_t n_clauses, const int64_t *clause_off,
               const int32_t *lits, const int64_t *weights, const msat_config *cfg,
               cudaStream_t stream, bool pool_alloc);
// final evaluation of the current x (best update and capture) on c->stream
cudaError_t ctx_eval_current(msat_ctx *c);
// free a context without synchronising (pool contexts: frees ordered on c->stream)
void ctx_destroy_async(msat_ctx *c);

}  // namespace msat
