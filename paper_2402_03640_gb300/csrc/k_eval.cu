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

// The paper's quick reading of a clause as satisfied when f_j > 0 (Sec. 4,
// "Example") against the exact test (some literal true under x > 0).  One
// thread per (clause, restart): f_j in the fixed order of the step (terms in
// literal order, 32-term leaves, dyadic combination) from t = tanh(x);
// counts per restart the clauses read as unsat by the heuristic and those on
// which the two tests disagree.  Integer counts, so the order of the
// additions does not matter.
__global__ void k_heuristic_gap(DevInst I, const float *__restrict__ x,
                                unsigned long long *__restrict__ heur_unsat,
                                unsigned long long *__restrict__ disagree) {
    const int B = I.B;
    const long long total = (long long)I.m * B;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q / B), b = (int)(q - (long long)j * B);
        int beg, end;
        if (I.kfix > 0) {
            beg = j * I.kfix;
            end = beg + I.kfix;
        } else {
            beg = __ldg(I.coff + j);
            end = __ldg(I.coff + j + 1);
        }
        LeafCounter<kClauseLevels> lc;
        lc.init();
        float leaf = 0.0f;
        int in_leaf = 0;
        bool sat = false;
        for (int p = beg; p < end; ++p) {
            const int L = __ldg(I.lit + p);
            const float xv = __ldg(x + (long long)(L >> 1) * B + b);
            const float tv = tanh_fixed(xv);
            const bool neg = L & 1;
            const float term = neg ? -tv : tv;
            leaf = in_leaf == 0 ? term : leaf + term;
            sat |= (xv > 0.0f) != neg;
            if (++in_leaf == 32) {
                lc.push(leaf);
                in_leaf = 0;
            }
        }
        if (in_leaf) lc.push(leaf);
        const float f = lc.finish();
        if (!(f > 0.0f)) atomicAdd(heur_unsat + b, 1ull);
        if ((f > 0.0f) != sat) atomicAdd(disagree + b, 1ull);
    }
}

cudaError_t launch_heuristic_gap(const DevInst &I, const float *x, long long *heur_unsat,
                                 long long *disagree, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(heur_unsat, 0, sizeof(long long) * (size_t)I.B, st);
    if (!e) e = cudaMemsetAsync(disagree, 0, sizeof(long long) * (size_t)I.B, st);
    if (e) return e;
    const long long total = (long long)I.m * I.B;
    long long blocks = (total + kThreads - 1) / kThreads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_heuristic_gap<<<(unsigned)blocks, kThreads, 0, st>>>(I, x, reinterpret_cast<unsigned long long *>(heur_unsat),
                                                           reinterpret_cast<unsigned long long *>(disagree));
    return cudaGetLastError();
}

cudaError_t launch_round_pm1(const float *x, int8_t *a, long long count, cudaStream_t st) {
    long long blocks = (count + kThreads - 1) / kThreads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_round_pm1<<<(unsigned)blocks, kThreads, 0, st>>>(x, a, count);
    return cudaGetLastError();
}

}  // namespace msat
