// msat_objective_noalloc: the clause pass (relaxed objective and exact cost
// of a caller-supplied x) for callers that cannot allocate device memory.
//
// Who needs it: an application that hands this library a fixed device
// memory budget and forbids allocation once its loop runs.  cudaMalloc can
// synchronise the whole device and takes unbounded time, so latency-bound
// serving loops and real-time controllers ban it; hosts whose memory manager
// must account for every byte, and plugins called from contexts where CUDA
// allocation calls are not allowed, cannot call it either.  msat_create
// allocates, so such callers cannot build a context; this entry point takes
// every input and output from the caller and keeps its scratch in a fixed
// array compiled into the library.
//
// Scratch: g_scratch below, kScratchBytes (4 MiB) of device memory that
// every GPU which loads the library holds until the process exits.  All
// calls on a device share it: two calls whose kernels overlap on the GPU
// race on it and give wrong results.  Each call clears the finish counter
// before its kernel; the per-block partials are written in full every call.
//
// The loss is summed in another order than the context path's clause pass
// (per thread in 32-term leaves combined by the dyadic counter, then per
// block, then over the blocks in block order), so it agrees with
// msat_forward's loss to within 1e-5 relative, not bit for bit; the cost is
// an exact integer sum.
//
// The host cannot use the symbol g_scratch as a device address; the first
// call on each device (with that device current) asks the runtime for the
// address with cudaGetSymbolAddress and caches it.  Make that first call
// before any stream capture.

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "msat_internal.cuh"

namespace msat {

namespace {

constexpr size_t kScratchBytes = 4u << 20;
constexpr int kMaxDevices = 64;
constexpr int kNaBlocksMax = 256;  // blocks of one launch: partials fit the scratch for B <= 1024

// [0, 256): finish counter; then uint64 cost partials [blocks][B]; then
// float loss partials [blocks][B].
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Every literal of clause j in order: f by the fixed summation order
// (32-literal leaves, dyadic combination), and whether any literal is true.
// A literal of 0 or naming no variable is skipped.
__device__ __forceinline__ void clause_at(const int64_t *__restrict__ coff,
                                          const int32_t *__restrict__ lits,
                                          const float *__restrict__ x, int n, int B, int b,
                                          long long j, float &f, bool &sat) {
    const long long beg = __ldg(coff + j), end = __ldg(coff + j + 1);
    LeafCounter<31> lc;  // any clause length the offsets can express
    lc.init();
    float leaf = 0.0f;
    int in_leaf = 0;
    sat = false;
    for (long long p = beg; p < end; ++p) {
        const int l = __ldg(lits + p);
        const int v = (l > 0 ? l : -l) - 1;
        if (l == 0 || v >= n) continue;
        const bool neg = l < 0;
        const float xv = __ldg(x + (long long)v * B + b);
        const float t = tanh_fixed(xv);
        const float term = neg ? -t : t;
        leaf = (in_leaf == 0) ? term : leaf + term;
        sat |= ((xv > 0.0f) != neg);
        if (++in_leaf == 32) {
            lc.push(leaf);
            in_leaf = 0;
        }
    }
    if (in_leaf) lc.push(leaf);
    f = lc.finish();
}

// One thread per (clause, restart) item, grid-stride with a stride that is a
// multiple of B, so each thread keeps one restart; block sums per restart go
// to the scratch partials, and the last block to finish adds them in block
// order into cost_out and loss_out.  For B > 256 block k covers the restart
// slice 256 * (k % (B / 256)) .. + 255.  A thread sums its loss terms in
// 32-term leaves combined by the dyadic counter, so the rounding error grows
// with the logarithm of its item count rather than linearly.
__global__ void __launch_bounds__(kThreads)
    k_objective_noalloc(const int64_t *__restrict__ coff, const int32_t *__restrict__ lits,
                        const int64_t *__restrict__ w, const float *__restrict__ x, int n,
                        long long m, int B, unsigned char *__restrict__ scratch,
                        long long *__restrict__ cost_out, float *__restrict__ loss_out) {
    __shared__ unsigned long long s_c[kThreads];
    __shared__ float s_l[kThreads];
    __shared__ int s_last;
    unsigned int *counter = reinterpret_cast<unsigned int *>(scratch);
    unsigned long long *cpart = reinterpret_cast<unsigned long long *>(scratch + 256);
    float *lpart = reinterpret_cast<float *>(cpart + (size_t)gridDim.x * B);

    const long long total = m * B;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(first % B);
    unsigned long long cacc = 0;
    LeafCounter<24> lsum;  // up to 2^24 - 1 leaves of 32 loss terms a thread
    lsum.init();
    float leaf = 0.0f;
    int in_leaf = 0;
    for (long long it = first; it < total; it += stride) {
        const long long j = it / B;
        float f;
        bool sat;
        clause_at(coff, lits, x, n, B, b, j, f, sat);
        if (!sat) {
            const long long wj = w ? __ldg(w + j) : 1ll;
            cacc += (unsigned long long)wj;
            const float term = ((float)wj * f) * f;
            leaf = in_leaf == 0 ? term : leaf + term;
            if (++in_leaf == 32) {
                lsum.push(leaf);
                in_leaf = 0;
            }
        }
    }
    if (in_leaf) lsum.push(leaf);
    const float lacc = lsum.finish();
    s_c[threadIdx.x] = cacc;
    s_l[threadIdx.x] = lacc;
    __syncthreads();
    // threads r and r + B*k of a block share restart (threadIdx.x % B)
    if (threadIdx.x < B) {
        unsigned long long c = 0;
        float l = 0.0f;
        for (int r = threadIdx.x; r < blockDim.x; r += B) {
            c += s_c[r];
            l += s_l[r];
        }
        cpart[(size_t)blockIdx.x * B + b] = c;
        lpart[(size_t)blockIdx.x * B + b] = l;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const unsigned unit = B > kThreads ? (unsigned)(B / kThreads) : 1u;
    for (int r = threadIdx.x; r < B; r += blockDim.x) {
        unsigned long long c = 0;
        float l = 0.0f;
        for (unsigned k = (unsigned)(r / kThreads) % unit; k < gridDim.x; k += unit) {
            c += __ldcg(cpart + (size_t)k * B + r);
            l += __ldcg(lpart + (size_t)k * B + r);
        }
        cost_out[r] = (long long)c;
        loss_out[r] = c > 0 ? l / (float)(long long)c : 0.0f;
    }
}

int scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "msat_objective_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(MSAT_EINVAL, "msat_objective_noalloc: device index beyond 63");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                             "msat_objective_noalloc: cudaGetSymbolAddress(scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return MSAT_OK;
}

}  // namespace

}  // namespace msat

using namespace msat;

extern "C" int msat_objective_noalloc(int32_t n_vars, int64_t n_clauses, const int64_t *clause_off,
                                      const int32_t *lits, const int64_t *weights, const float *x,
                                      int32_t restarts, int64_t *cost_out, float *loss_out,
                                      void *stream) {
    const int32_t B = restarts;
    if (B < 1 || B > 1024 || (B & (B - 1)) != 0)
        return fail(MSAT_EINVAL, "msat_objective_noalloc: restarts must be a power of two in [1, 1024]");
    if (n_vars < 1 || n_clauses < 0 || (int64_t)n_vars * B >= (1LL << 31) ||
        n_clauses * (int64_t)B >= (1LL << 40))
        return fail(MSAT_EINVAL, "msat_objective_noalloc: n_vars >= 1, n_clauses >= 0, n*B < 2^31, m*B < 2^40");
    if (!clause_off || (n_clauses > 0 && !lits) || !x || !cost_out || !loss_out)
        return fail(MSAT_EINVAL, "msat_objective_noalloc: NULL device pointer");
    const long long items = n_clauses * (long long)B;
    long long blocks = (items + kThreads - 1) / kThreads;
    if (blocks > kNaBlocksMax) blocks = kNaBlocksMax;
    if (blocks < 1) blocks = 1;
    // the stride (blocks * kThreads) must be a multiple of B
    const long long unit = B > kThreads ? B / kThreads : 1;
    blocks = (blocks + unit - 1) / unit * unit;
    const size_t need = 256 + (size_t)blocks * B * (sizeof(unsigned long long) + sizeof(float));
    if (need > kScratchBytes)
        return fail(MSAT_EINVAL, "msat_objective_noalloc: " + std::to_string(need) +
                                     " scratch bytes needed, " + std::to_string(kScratchBytes) +
                                     " available");
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(scratch, 0, 256, st);  // finish counter
    if (e != cudaSuccess) return cuda_fail(e, "msat_objective_noalloc: clear counter");
    k_objective_noalloc<<<(unsigned)blocks, kThreads, 0, st>>>(
        clause_off, lits, weights, x, n_vars, n_clauses, B, static_cast<unsigned char *>(scratch),
        reinterpret_cast<long long *>(cost_out), loss_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "msat_objective_noalloc: kernel launch");
    return MSAT_OK;
}
