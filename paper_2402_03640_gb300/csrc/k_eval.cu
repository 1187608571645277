// Exact cost of a batch of +-1 assignments by the clause CSR (sm_103a).
//
// A clause is unsatisfied iff none of its literals is true (the paper's
// test x'.W == -len with x' read as +-1, Sec. 4 "Unsatisfiable Cores").
// Layout: a[i * nb + b] is variable i of assignment b, so the 32 lanes of a
// warp read 32 consecutive assignments of one variable (one 32-byte sector).
// Each warp walks clauses with a stride; per-lane integer sums are combined
// across the block's warps in shared memory and added to cost[b] with one
// 64-bit atomic per (block, assignment) -- integer addition, so the result
// does not depend on the order.

#include <cuda_runtime.h>
#include <stdint.h>

#include "msat_internal.cuh"

namespace msat {

namespace {
constexpr int kEvalWarps = kThreads / 32;
}

__global__ void __launch_bounds__(kThreads)
    k_eval_sparse(DevInst I, const int8_t *__restrict__ a, int nb,
                  unsigned long long *__restrict__ cost) {
    __shared__ unsigned long long s_acc[kEvalWarps][32];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int b = blockIdx.y * 32 + lane;
    const bool live = b < nb;
    unsigned long long acc = 0;
    for (long long j = (long long)blockIdx.x * kEvalWarps + warp; j < I.m;
         j += (long long)gridDim.x * kEvalWarps) {
        int beg, end;
        if (I.kfix > 0) {
            beg = (int)j * I.kfix;
            end = beg + I.kfix;
        } else {
            beg = __ldg(I.coff + j);
            end = __ldg(I.coff + j + 1);
        }
        bool sat = false;
        for (int p = beg; p < end; ++p) {
            const int L = __ldg(I.lit + p);
            const int8_t v = live ? __ldg(a + (long long)(L >> 1) * nb + b) : 0;
            sat |= ((v > 0) != (bool)(L & 1));
        }
        if (!sat) acc += I.w ? (unsigned long long)__ldg(I.w + j) : 1ull;
    }
    s_acc[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long s = 0;
#pragma unroll
        for (int k = 0; k < kEvalWarps; ++k) s += s_acc[k][lane];
        if (live && s) atomicAdd(cost + b, s);
    }
}

cudaError_t launch_eval_sparse(const DevInst &I, const int8_t *a, int nb, long long *cost,
                               cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(cost, 0, sizeof(long long) * (size_t)nb, st);
    if (e != cudaSuccess) return e;
    if (I.m == 0) return cudaSuccess;
    const int gy = (nb + 31) / 32;
    long long gx = (I.m + kEvalWarps - 1) / kEvalWarps;
    long long cap = (152LL * 8 + gy - 1) / gy;  // about 8 blocks per SM in total
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    dim3 grid((unsigned)gx, (unsigned)gy);
    k_eval_sparse<<<grid, kThreads, 0, st>>>(I, a, nb, reinterpret_cast<unsigned long long *>(cost));
    return cudaGetLastError();
}

// Rounded batch of the relaxed variables: a[q] = +1 if x[q] > 0 else -1
// (the de-relaxation of Sec. 4, read as +-1), same [n][B] layout.
__global__ void k_round_pm1(const float *__restrict__ x, int8_t *__restrict__ a, long long count) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        a[q] = __ldg(x + q) > 0.0f ? (int8_t)1 : (int8_t)-1;
}

cudaError_t launch_round_pm1(const float *x, int8_t *a, long long count, cudaStream_t st) {
    long long blocks = (count + kThreads - 1) / kThreads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_round_pm1<<<(unsigned)blocks, kThreads, 0, st>>>(x, a, count);
    return cudaGetLastError();
}

}  // namespace msat
