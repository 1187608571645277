// Step kernels of the MaxSAT gradient engine (sm_103a).
//
//   k_init      random start of x (Alg. 1 line 1), zero Adam moments, tanh(x)
//   k_forward   clause pass: f_j, exact unsat bits, sum_U w and the loss
//               partials per restart; the last block to finish turns them
//               into cost, best, 2/W_U and the Adam step scalars
//   k_backward  variable pass over the transposed CSR: occurrence sum of
//               +-dL/df_j, times 1 - t^2, fused Adam update, best-assignment
//               capture and tanh of the new x.  Variables with more than
//               heavy_deg occurrences are split into 1024-occurrence chunks
//               handled by whole warps and combined in the fixed tree order.
//
// Layouts: x, mom, vel, t are float [n][B] (restart index innermost), so the
// B values of one variable are one contiguous, vector-loadable row.  Each
// thread owns VW consecutive restarts (VW = 4, 2 or 1) of one clause or
// variable.

#include <cuda_runtime.h>
#include <stdint.h>

#include "msat_internal.cuh"

namespace msat {

namespace {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <int VW>
__device__ __forceinline__ void ldv(const float *__restrict__ p, float (&o)[VW]) {
    if constexpr (VW == 4) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else if constexpr (VW == 2) {
        float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = __ldg(p);
    }
}

// plain (coherent) vector load, for arrays this kernel also writes
template <int VW>
__device__ __forceinline__ void ldv_rw(const float *p, float (&o)[VW]) {
    if constexpr (VW == 4) {
        float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else if constexpr (VW == 2) {
        float2 v = *reinterpret_cast<const float2 *>(p);
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = *p;
    }
}

template <int VW>
__device__ __forceinline__ void stv(float *p, const float (&o)[VW]) {
    if constexpr (VW == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (VW == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(o[0], o[1]);
    } else {
        *p = o[0];
    }
}

__device__ __forceinline__ void clause_range(const DevInst &I, int kfix, int j, int &beg, int &end) {
    if (kfix > 0) {
        beg = j * kfix;
        end = beg + kfix;
    } else {
        beg = __ldg(I.coff + j);
        end = __ldg(I.coff + j + 1);
    }
}

// f_j for VW restarts in the fixed order (literal order, 32-literal leaves,
// dyadic combination) and, if WANT_SAT, whether some literal is true.
template <int VW, bool WANT_SAT>
__device__ __forceinline__ void clause_value(const DevInst &I, const float *__restrict__ t,
                                             int beg, int end, int col, float (&f)[VW],
                                             bool (&sat)[VW]) {
    const int B = I.B;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        f[e] = 0.0f;
        sat[e] = false;
    }
    if (end - beg <= 32) {
        for (int p = beg; p < end; ++p) {
            int L = __ldg(I.lit + p);
            bool neg = L & 1;
            float tv[VW];
            ldv<VW>(t + (int64_t)(L >> 1) * B + col, tv);
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                float term = neg ? -tv[e] : tv[e];
                f[e] = (p == beg) ? term : f[e] + term;
                if (WANT_SAT) sat[e] |= ((tv[e] > 0.0f) != neg);
            }
        }
    } else {
        LeafCounter<6> lc[VW];
        float leaf[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) lc[e].init();
        int in_leaf = 0;
        for (int p = beg; p < end; ++p) {
            int L = __ldg(I.lit + p);
            bool neg = L & 1;
            float tv[VW];
            ldv<VW>(t + (int64_t)(L >> 1) * B + col, tv);
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                float term = neg ? -tv[e] : tv[e];
                leaf[e] = (in_leaf == 0) ? term : leaf[e] + term;
                if (WANT_SAT) sat[e] |= ((tv[e] > 0.0f) != neg);
            }
            if (++in_leaf == 32) {
#pragma unroll
                for (int e = 0; e < VW; ++e) lc[e].push(leaf[e]);
                in_leaf = 0;
            }
        }
        if (in_leaf) {
#pragma unroll
            for (int e = 0; e < VW; ++e) lc[e].push(leaf[e]);
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) f[e] = lc[e].finish();
    }
}

// Fixed-length clause (KFIX literals): all literal loads first, then all
// row gathers, so the loads of one clause are in flight together.
template <int VW, int KFIX>
__device__ __forceinline__ void clause_value_fixed(const DevInst &I, const float *__restrict__ t,
                                                   int j, int col, float (&f)[VW],
                                                   bool (&sat)[VW]) {
    const int B = I.B;
    int L[KFIX];
#pragma unroll
    for (int p = 0; p < KFIX; ++p) L[p] = __ldg(I.lit + j * KFIX + p);
    float tv[KFIX][VW];
#pragma unroll
    for (int p = 0; p < KFIX; ++p) ldv<VW>(t + (int64_t)(L[p] >> 1) * B + col, tv[p]);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        sat[e] = false;
#pragma unroll
        for (int p = 0; p < KFIX; ++p) {
            const bool neg = L[p] & 1;
            const float term = neg ? -tv[p][e] : tv[p][e];
            f[e] = (p == 0) ? term : f[e] + term;
            sat[e] |= ((tv[p][e] > 0.0f) != neg);
        }
    }
}

// Occurrence term for VW restarts given the occurrence word o = j << 1 | neg
// and the unsat word covering (j, col): +-((float)w_j * f_j) * (2/W_U) where
// clause j is unsat, +0 elsewhere.  f comes from the clause pass's store when
// there is one, else it is recomputed from the clause in the same order.
template <int VW, int KFIX>
__device__ __forceinline__ void occ_term(const DevInst &I, int kfix, const float *__restrict__ t,
                                         const float *__restrict__ fstore, const float (&cs)[VW],
                                         int o, uint32_t wd, int col, float (&term)[VW]) {
    const int B = I.B;
    const int j = o >> 1;
    const bool neg = o & 1;
    const int64_t qb = (int64_t)j * B + col;
    const uint32_t nib = (wd >> (qb & 31)) & ((1u << VW) - 1u);
#pragma unroll
    for (int e = 0; e < VW; ++e) term[e] = 0.0f;
    if (!nib) return;
    float f[VW];
    if (fstore) {
        ldv<VW>(fstore + qb, f);
    } else {
        bool sat[VW];
        if constexpr (KFIX > 0) {
            clause_value_fixed<VW, KFIX>(I, t, j, col, f, sat);
        } else {
            int beg, end;
            clause_range(I, kfix, j, beg, end);
            clause_value<VW, false>(I, t, beg, end, col, f, sat);
        }
    }
    const float wj = I.w ? (float)__ldg(I.w + j) : 1.0f;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        if ((nib >> e) & 1u) {
            const float g = (wj * f[e]) * cs[e];
            term[e] = neg ? -g : g;
        }
    }
}

// Dyadic tree over the first K lanes' values (lane 0 receives the result).
__device__ __forceinline__ float warp_dyadic(float v, int K, int lane) {
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        float o = __shfl_down_sync(0xffffffffu, v, s);
        if ((lane & (2 * s - 1)) == 0 && lane + s < K) v = v + o;
    }
    return v;
}

struct AdamView {
    float a_t, r_t, b1, b2, omb1, omb2, eps;
};

__device__ __forceinline__ float adam_update(const AdamView &A, float x, float &m, float &v,
                                             float g) {
    float mq = A.b1 * m + A.omb1 * g;
    float vq = A.b2 * v + (A.omb2 * g) * g;
    float den = sqrtf(vq) * A.r_t + A.eps;
    m = mq;
    v = vq;
    return x - (A.a_t * mq) / den;
}

template <int VW>
struct LightLevels {
    // occurrence rows of one light block / 32, rounded up to a power of two
    static constexpr int value = VW == 1 ? 9 : (VW == 2 ? 8 : 7);
};

}  // namespace

// ------------------------------------------------------------------ k_init

__global__ void k_init(int n, int B, uint64_t seed, float *__restrict__ x,
                       float *__restrict__ mom, float *__restrict__ vel,
                       float *__restrict__ t0, uint8_t *__restrict__ bestx) {
    const int64_t total = (int64_t)n * B;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q / B;
        int64_t b = q - i * B;
        uint64_t u = splitmix64_at(seed, (uint64_t)b * (uint64_t)n + (uint64_t)i);
        float k = (float)(uint32_t)(u >> 40);
        float xv = k * 0x1p-23f - 1.0f;
        x[q] = xv;
        mom[q] = 0.0f;
        vel[q] = 0.0f;
        t0[q] = tanh_fixed(xv);
        bestx[q] = 0;
    }
}

cudaError_t launch_init(const DevInst &I, const DevState &S, uint64_t seed, cudaStream_t st) {
    int64_t total = (int64_t)I.n * I.B;
    int blocks = (int)((total + kThreads - 1) / kThreads);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_init<<<blocks, kThreads, 0, st>>>(I.n, I.B, seed, S.x, S.mom, S.vel, S.t0, S.bestx);
    return cudaGetLastError();
}

__global__ void k_tanh(const float *__restrict__ x, float *__restrict__ t, int64_t count) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x)
        t[q] = tanh_fixed(__ldg(x + q));
}

cudaError_t launch_tanh(const float *x, float *t, int64_t count, cudaStream_t st) {
    int blocks = (int)((count + kThreads - 1) / kThreads);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_tanh<<<blocks, kThreads, 0, st>>>(x, t, count);
    return cudaGetLastError();
}

// --------------------------------------------------------------- k_forward
// One item = (clause j, restart group g).  The grid-stride loop is unrolled
// by two (items base + lane and base + stride + lane; the stride is a
// multiple of G, so both belong to the thread's restart group), keeping the
// loads of two clauses in flight; the unsat bits of 32 consecutive items are
// packed with shuffles into whole 32-bit words.

template <int VW, int KFIX>
__global__ void __launch_bounds__(kThreads)
    k_forward(DevInst I, const float *__restrict__ t0, const float *__restrict__ t1,
              const float *__restrict__ t_ovr, DevStep D, uint32_t *__restrict__ ubits,
              float *__restrict__ fstore, int mode) {
    __shared__ unsigned long long s_w[kThreads * VW];
    __shared__ float s_l[kThreads * VW];
    __shared__ int s_last;

    const int B = I.B;
    const int G = B / VW;
    const long long steps = D.sc->steps_done;
    const float *__restrict__ t = t_ovr ? t_ovr : ((steps & 1) ? t1 : t0);
    const int kfix = KFIX > 0 ? KFIX : I.kfix;
    const int lane = threadIdx.x & 31;
    const int g = threadIdx.x % G;
    const int col = g * VW;
    const long long total = (long long)I.m * G;
    const long long stride = (long long)gridDim.x * blockDim.x;

    float lacc[VW];
    unsigned long long wacc[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        lacc[e] = 0.0f;
        wacc[e] = 0ull;
    }
    constexpr int LPW = 32 / VW;  // lanes whose bits share one 32-bit word
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total;
         base += 2 * stride) {
        long long item[2] = {base + lane, base + stride + lane};
        bool act[2] = {item[0] < total, item[1] < total};
        int jj[2] = {act[0] ? (int)(item[0] / G) : 0, act[1] ? (int)(item[1] / G) : 0};
        float f[2][VW];
        bool sat[2][VW];
        if constexpr (KFIX > 0) {
            // both clauses' literals, then both clauses' rows
            int L[2][KFIX];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int p = 0; p < KFIX; ++p) L[h][p] = __ldg(I.lit + jj[h] * KFIX + p);
            float tv[2][KFIX][VW];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int p = 0; p < KFIX; ++p)
                    ldv<VW>(t + (int64_t)(L[h][p] >> 1) * B + col, tv[h][p]);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    sat[h][e] = false;
#pragma unroll
                    for (int p = 0; p < KFIX; ++p) {
                        const bool neg = L[h][p] & 1;
                        const float term = neg ? -tv[h][p][e] : tv[h][p][e];
                        f[h][e] = (p == 0) ? term : f[h][e] + term;
                        sat[h][e] |= ((tv[h][p][e] > 0.0f) != neg);
                    }
                }
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int beg = 0, end = 0;
                if (act[h]) clause_range(I, kfix, jj[h], beg, end);
                clause_value<VW, true>(I, t, beg, end, col, f[h], sat[h]);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            unsigned nib = 0;
            if (act[h]) {
                const long long wj = I.w ? __ldg(I.w + jj[h]) : 1ll;
                const float wf = (float)wj;
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    if (!sat[h][e]) {
                        nib |= 1u << e;
                        wacc[e] += (unsigned long long)wj;
                        lacc[e] += (wf * f[h][e]) * f[h][e];
                    }
                }
                if (fstore) stv<VW>(fstore + (int64_t)jj[h] * B + col, f[h]);
            }
            unsigned word = nib << ((lane % LPW) * VW);
#pragma unroll
            for (int o = 1; o < LPW; o <<= 1) word |= __shfl_xor_sync(0xffffffffu, word, o);
            if (act[h] && (lane % LPW) == 0) ubits[(item[h] * VW) >> 5] = word;
        }
    }

#pragma unroll
    for (int e = 0; e < VW; ++e) {
        s_w[threadIdx.x * VW + e] = wacc[e];
        s_l[threadIdx.x * VW + e] = lacc[e];
    }
    __syncthreads();
    if (threadIdx.x < G) {
        unsigned long long *acc = D.wu_acc + (long long)(blockIdx.x % kRep) * B;
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            unsigned long long sw = 0;
            float sl = 0.0f;
            for (int r = threadIdx.x; r < blockDim.x; r += G) {
                sw += s_w[r * VW + e];
                sl += s_l[r * VW + e];
            }
            const int b = threadIdx.x * VW + e;
            if (sw) atomicAdd(acc + b, sw);
            D.lpart[(long long)blockIdx.x * B + b] = sl;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&D.sc->counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        unsigned long long wu = 0;
        for (int r = 0; r < kRep; ++r) wu += atomicExch(D.wu_acc + (long long)r * B + b, 0ull);
        const long long c = (long long)wu;
        D.cost[b] = c;
        if (mode != FWD_PROBE) {
            const long long bb = D.best[b];
            const int imp = c < bb;
            if (imp) D.best[b] = c;
            D.improved[b] = imp;
        }
        D.cscale[b] = c > 0 ? 2.0f / (float)c : 0.0f;
    }
    if (threadIdx.x == 0) {
        StepScalars *sc = D.sc;
        sc->counter = 0;
        if (mode == FWD_STEP) {
            const double p1 = sc->p1 * sc->beta1;
            const double p2 = sc->p2 * sc->beta2;
            sc->p1 = p1;
            sc->p2 = p2;
            sc->a_t = (float)(sc->lr / (1.0 - p1));
            sc->r_t = (float)(1.0 / sqrt(1.0 - p2));
            sc->steps_done = steps + 1;
        }
    }
}

int fwd_grid_blocks(const DevInst &I) {
    const int VW = (I.B % 4 == 0) ? 4 : (I.B % 2 == 0 ? 2 : 1);
    const long long items = (long long)I.m * (I.B / VW);
    long long blocks = (items + 2 * kThreads - 1) / (2 * kThreads);
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

template <int VW>
static cudaError_t launch_forward_vw(const DevInst &I, const DevState &S, const DevStep &D,
                                     int mode, const float *t_ovr, cudaStream_t st) {
    const int blocks = D.fwd_blocks;
    if (I.kfix == 3)
        k_forward<VW, 3><<<blocks, kThreads, 0, st>>>(I, S.t0, S.t1, t_ovr, D, S.ubits, S.fstore, mode);
    else
        k_forward<VW, 0><<<blocks, kThreads, 0, st>>>(I, S.t0, S.t1, t_ovr, D, S.ubits, S.fstore, mode);
    return cudaGetLastError();
}

cudaError_t launch_forward(const DevInst &I, const DevState &S, const DevStep &D, int mode,
                           const float *t_override, cudaStream_t st) {
    if (I.B % 4 == 0) return launch_forward_vw<4>(I, S, D, mode, t_override, st);
    if (I.B % 2 == 0) return launch_forward_vw<2>(I, S, D, mode, t_override, st);
    return launch_forward_vw<1>(I, S, D, mode, t_override, st);
}

// -------------------------------------------------------------- k_backward
// k_backward_heavy: variables with more occurrences than a light block can
// stage, one warp per (1024-occurrence chunk, restart group); the last warp
// of a (variable, group) combines the chunk partials in the fixed tree order
// and applies the update.
// k_backward_light: one block per range of consecutive light variables.
// Phase 1 spreads the block's (occurrence, restart group) items over all
// threads and stages each occurrence term in shared memory; phase 2 gives
// each (variable, restart group) to one thread, which sums its terms in the
// fixed order and applies 1 - t^2 and Adam.  Block b < B also reduces the
// loss of restart b from the forward partials.

template <int VW, int KFIX>
__global__ void __launch_bounds__(kThreads)
    k_backward_heavy(DevInst I, DevState S, DevStep D, int mode, const float *__restrict__ t_ovr,
                     const float *__restrict__ gscale, float *__restrict__ grad_out) {
    const int B = I.B;
    const int G = B / VW;
    const int kfix = KFIX > 0 ? KFIX : I.kfix;
    const long long steps = D.sc->steps_done;
    const float *tcur;
    float *tnext = nullptr;
    if (mode == BWD_UPDATE) {
        tcur = ((steps - 1) & 1) ? S.t1 : S.t0;
        tnext = (steps & 1) ? S.t1 : S.t0;
    } else {
        tcur = t_ovr;
    }
    const uint32_t *__restrict__ ubits = S.ubits;
    const float *__restrict__ fstore = S.fstore;

    AdamView A;
    {
        const StepScalars *sc = D.sc;
        A.a_t = sc->a_t;
        A.r_t = sc->r_t;
        A.b1 = sc->b1f;
        A.b2 = sc->b2f;
        A.omb1 = sc->omb1f;
        A.omb2 = sc->omb2f;
        A.eps = sc->epsf;
    }

    {
        // ---------------- heavy variables: one warp per (chunk, restart group)
        const int lane = threadIdx.x & 31;
        const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
        const long long nchunks = I.heavy_chunks;
        for (long long it = warp; it < nchunks * G; it += nwarps) {
            const int gg = (int)(it % G);
            const long long cidx = it / G;
            const int col = gg * VW;
            int lo = 0, hi = I.n_heavy - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (__ldg(I.heavy_chunk0 + mid) <= cidx) lo = mid; else hi = mid - 1;
            }
            const int h = lo;
            const int i = __ldg(I.heavy_var + h);
            const int c0 = __ldg(I.heavy_chunk0 + h);
            const int nch = __ldg(I.heavy_chunk0 + h + 1) - c0;
            const int c = (int)(cidx - c0);
            const int vbeg = __ldg(I.voff + i), vend = __ldg(I.voff + i + 1);
            float cs[VW];
#pragma unroll
            for (int e = 0; e < VW; ++e) cs[e] = D.cscale[col + e];
            float leaf[VW];
#pragma unroll
            for (int e = 0; e < VW; ++e) leaf[e] = 0.0f;
            if (mode != BWD_BITS_ONLY) {
                const int lb = vbeg + c * kChunk + lane * 32;
                const int le = min(lb + 32, vend);
                for (int s = lb; s < le; ++s) {
                    const int o = __ldg(I.occ + s);
                    const uint32_t wd = __ldg(ubits + (((int64_t)(o >> 1) * B + col) >> 5));
                    float term[VW];
                    occ_term<VW, KFIX>(I, kfix, tcur, fstore, cs, o, wd, col, term);
#pragma unroll
                    for (int e = 0; e < VW; ++e) leaf[e] = (s == lb) ? term[e] : leaf[e] + term[e];
                }
                const int rem = vend - (vbeg + c * kChunk);
                const int K = min(32, (rem + 31) / 32);
#pragma unroll
                for (int e = 0; e < VW; ++e) leaf[e] = warp_dyadic(leaf[e], K, lane);
                if (lane == 0) {
#pragma unroll
                    for (int e = 0; e < VW; ++e) D.hpart[cidx * B + col + e] = leaf[e];
                }
            }
            __threadfence();
            unsigned prev = 0;
            if (lane == 0) prev = atomicAdd(D.hcount + (long long)h * G + gg, 1u);
            prev = __shfl_sync(0xffffffffu, prev, 0);
            if (prev != (unsigned)(nch - 1)) continue;
            __threadfence();
            // last warp of this (variable, group): combine the chunk partials
            LeafCounter<12> lc[VW];
#pragma unroll
            for (int e = 0; e < VW; ++e) lc[e].init();
            if (mode != BWD_BITS_ONLY) {
                for (int base = 0; base < nch; base += 32) {
                    const int Kc = min(32, nch - base);
                    float v[VW];
#pragma unroll
                    for (int e = 0; e < VW; ++e)
                        v[e] = (lane < Kc) ? __ldcg(D.hpart + (c0 + base + lane) * (long long)B + col + e)
                                           : 0.0f;
#pragma unroll
                    for (int e = 0; e < VW; ++e) {
                        v[e] = warp_dyadic(v[e], Kc, lane);
                        lc[e].push(v[e]);
                    }
                }
            }
            if (lane == 0) {
                D.hcount[(long long)h * G + gg] = 0;
                const int64_t q0 = (int64_t)i * B + col;
                float xv[VW];  // x, or t = tanh(x) in the gradient-only mode
                if (mode == BWD_GRAD_ONLY) ldv<VW>(tcur + q0, xv); else ldv_rw<VW>(S.x + q0, xv);
                if (mode == BWD_BITS_ONLY) {
#pragma unroll
                    for (int e = 0; e < VW; ++e)
                        if (D.improved[col + e]) S.bestx[q0 + e] = xv[e] > 0.0f;
                } else {
                    float gr[VW];
#pragma unroll
                    for (int e = 0; e < VW; ++e) {
                        const float tv = (mode == BWD_GRAD_ONLY) ? xv[e] : tanh_fixed(xv[e]);
                        gr[e] = lc[e].finish() * fmaf(-tv, tv, 1.0f);
                    }
                    if (mode == BWD_GRAD_ONLY) {
#pragma unroll
                        for (int e = 0; e < VW; ++e)
                            grad_out[q0 + e] = gscale ? gr[e] * gscale[col + e] : gr[e];
                    } else {
                        float mv[VW], vv[VW], xn[VW], tn[VW];
                        ldv_rw<VW>(S.mom + q0, mv);
                        ldv_rw<VW>(S.vel + q0, vv);
#pragma unroll
                        for (int e = 0; e < VW; ++e) {
                            xn[e] = xv[e];
                            if (D.cost[col + e] != 0) xn[e] = adam_update(A, xv[e], mv[e], vv[e], gr[e]);
                            if (D.improved[col + e]) S.bestx[q0 + e] = xv[e] > 0.0f;
                            tn[e] = tanh_fixed(xn[e]);
                        }
                        stv<VW>(S.x + q0, xn);
                        stv<VW>(S.mom + q0, mv);
                        stv<VW>(S.vel + q0, vv);
                        stv<VW>(tnext + q0, tn);
                    }
                }
            }
        }
        return;
    }

}

template <int VW, int KFIX>
__global__ void __launch_bounds__(kThreads)
    k_backward_light(DevInst I, DevState S, DevStep D, int mode, const float *__restrict__ t_ovr,
                     const float *__restrict__ gscale, float *__restrict__ grad_out) {
    extern __shared__ float4 dyn_smem[];
    const int B = I.B;
    const int G = B / VW;
    const int kfix = KFIX > 0 ? KFIX : I.kfix;
    const long long steps = D.sc->steps_done;
    const float *tcur;
    float *tnext = nullptr;
    if (mode == BWD_UPDATE) {
        tcur = ((steps - 1) & 1) ? S.t1 : S.t0;
        tnext = (steps & 1) ? S.t1 : S.t0;
    } else {
        tcur = t_ovr;
    }
    const uint32_t *__restrict__ ubits = S.ubits;
    const float *__restrict__ fstore = S.fstore;

    // loss of the evaluated x per restart, from the forward block partials
    if (mode == BWD_UPDATE) {
        __shared__ float s_red[kThreads];
        for (int b = blockIdx.x; b < B; b += gridDim.x) {
            float acc = 0.0f;
            for (int k = threadIdx.x; k < D.fwd_blocks; k += blockDim.x)
                acc += D.lpart[(long long)k * B + b];
            s_red[threadIdx.x] = acc;
            __syncthreads();
            for (int s = blockDim.x / 2; s > 0; s >>= 1) {
                if (threadIdx.x < s) s_red[threadIdx.x] += s_red[threadIdx.x + s];
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                const long long c = D.cost[b];
                D.loss[b] = c > 0 ? s_red[0] / (float)c : 0.0f;
            }
            __syncthreads();
        }
    }

    AdamView A;
    {
        const StepScalars *sc = D.sc;
        A.a_t = sc->a_t;
        A.r_t = sc->r_t;
        A.b1 = sc->b1f;
        A.b2 = sc->b2f;
        A.omb1 = sc->omb1f;
        A.omb2 = sc->omb2f;
        A.eps = sc->epsf;
    }

    // ------------------------------------------------------- light block
    float *sterm = reinterpret_cast<float *>(dyn_smem);
    if ((int)blockIdx.x >= I.n_lblk) return;  // a grid of one block when every variable is heavy
    const int2 rg = I.lblk[blockIdx.x];
    const int v0 = rg.x, v1 = rg.y;
    const int s0 = __ldg(I.voff + v0);
    const int nocc = __ldg(I.voff + v1) - s0;
    const int gshift = __ffs(G) - 1;  // G is a power of two
    const int g = threadIdx.x & (G - 1);
    const int col = g * VW;
    float cs[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) cs[e] = D.cscale[col + e];

    if (mode != BWD_BITS_ONLY) {
        // phase 1: occurrence terms into shared memory, four items per thread in flight
        const int items = nocc << gshift;
        for (int base = threadIdx.x; base < items; base += 4 * kThreads) {
            int o[4];
            uint32_t wd[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int it = base + u * kThreads;
                o[u] = it < items ? __ldg(I.occ + s0 + (it >> gshift)) : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int it = base + u * kThreads;
                wd[u] = it < items ? __ldg(ubits + (((int64_t)(o[u] >> 1) * B + col) >> 5)) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int it = base + u * kThreads;
                if (it < items) {
                    float term[VW];
                    occ_term<VW, KFIX>(I, kfix, tcur, fstore, cs, o[u], wd[u], col, term);
                    float *dst = sterm + (int64_t)(it >> gshift) * B + col;
                    if constexpr (VW == 4) {
                        *reinterpret_cast<float4 *>(dst) = make_float4(term[0], term[1], term[2], term[3]);
                    } else if constexpr (VW == 2) {
                        *reinterpret_cast<float2 *>(dst) = make_float2(term[0], term[1]);
                    } else {
                        dst[0] = term[0];
                    }
                }
            }
        }
        __syncthreads();
    }

    // phase 2: one thread per (variable, restart group)
    const int vloc = threadIdx.x >> gshift;
    const int i = v0 + vloc;
    if (i >= v1) return;
    const int64_t q0 = (int64_t)i * B + col;
    float xv[VW];  // x, or t = tanh(x) in the gradient-only mode
    if (mode == BWD_GRAD_ONLY) ldv<VW>(tcur + q0, xv); else ldv_rw<VW>(S.x + q0, xv);
    if (mode == BWD_BITS_ONLY) {
#pragma unroll
        for (int e = 0; e < VW; ++e)
            if (D.improved[col + e]) S.bestx[q0 + e] = xv[e] > 0.0f;
        return;
    }
    const int rb = __ldg(I.voff + i) - s0, re = __ldg(I.voff + i + 1) - s0;
    LeafCounter<LightLevels<VW>::value> lc[VW];
    float leaf[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        lc[e].init();
        leaf[e] = 0.0f;
    }
    int in_leaf = 0;
    for (int r = rb; r < re; ++r) {
        float term[VW];
        const float *src = sterm + (int64_t)r * B + col;
        if constexpr (VW == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(src);
            term[0] = v.x; term[1] = v.y; term[2] = v.z; term[3] = v.w;
        } else if constexpr (VW == 2) {
            const float2 v = *reinterpret_cast<const float2 *>(src);
            term[0] = v.x; term[1] = v.y;
        } else {
            term[0] = src[0];
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) leaf[e] = (in_leaf == 0) ? term[e] : leaf[e] + term[e];
        if (++in_leaf == 32) {
#pragma unroll
            for (int e = 0; e < VW; ++e) lc[e].push(leaf[e]);
            in_leaf = 0;
        }
    }
    if (in_leaf) {
#pragma unroll
        for (int e = 0; e < VW; ++e) lc[e].push(leaf[e]);
    }
    float gr[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        const float tv = (mode == BWD_GRAD_ONLY) ? xv[e] : tanh_fixed(xv[e]);
        gr[e] = lc[e].finish() * fmaf(-tv, tv, 1.0f);
    }
    if (mode == BWD_GRAD_ONLY) {
#pragma unroll
        for (int e = 0; e < VW; ++e) gr[e] = gscale ? gr[e] * gscale[col + e] : gr[e];
        stv<VW>(grad_out + q0, gr);
        return;
    }
    float mv[VW], vv[VW], xn[VW], tn[VW];
    ldv_rw<VW>(S.mom + q0, mv);
    ldv_rw<VW>(S.vel + q0, vv);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        xn[e] = (D.cost[col + e] != 0) ? adam_update(A, xv[e], mv[e], vv[e], gr[e]) : xv[e];
        if (D.improved[col + e]) S.bestx[q0 + e] = xv[e] > 0.0f;
        tn[e] = tanh_fixed(xn[e]);
    }
    stv<VW>(S.x + q0, xn);
    stv<VW>(S.mom + q0, mv);
    stv<VW>(S.vel + q0, vv);
    stv<VW>(tnext + q0, tn);
}

template <int VW, int KFIX>
static cudaError_t launch_backward_k(const DevInst &I, const DevState &S, const DevStep &D,
                                     int mode, const float *t_ovr, const float *gscale,
                                     float *grad_out, cudaStream_t st) {
    const int G = I.B / VW;
    if (I.n_heavy > 0) {
        const long long warps = I.heavy_chunks * G;  // one warp per (chunk, group)
        long long hblocks = (warps + (kThreads / 32) - 1) / (kThreads / 32);
        if (hblocks > 152 * 8) hblocks = 152 * 8;
        k_backward_heavy<VW, KFIX><<<(unsigned)hblocks, kThreads, 0, st>>>(I, S, D, mode, t_ovr,
                                                                            gscale, grad_out);
        cudaError_t e = cudaGetLastError();
        if (e) return e;
    }
    const long long lblocks = I.n_lblk > 0 ? I.n_lblk : 1;
    const size_t smem = (size_t)I.occ_cap * I.B * sizeof(float);
    k_backward_light<VW, KFIX><<<(unsigned)lblocks, kThreads, smem, st>>>(I, S, D, mode, t_ovr,
                                                                           gscale, grad_out);
    return cudaGetLastError();
}

template <int VW>
static cudaError_t launch_backward_vw(const DevInst &I, const DevState &S, const DevStep &D,
                                      int mode, const float *t_ovr, const float *gscale,
                                      float *grad_out, cudaStream_t st) {
    if (I.kfix == 3) return launch_backward_k<VW, 3>(I, S, D, mode, t_ovr, gscale, grad_out, st);
    return launch_backward_k<VW, 0>(I, S, D, mode, t_ovr, gscale, grad_out, st);
}

cudaError_t launch_backward(const DevInst &I, const DevState &S, const DevStep &D, int mode,
                            const float *t_override, const float *gscale, float *grad_out,
                            cudaStream_t st) {
    if (I.B % 4 == 0) return launch_backward_vw<4>(I, S, D, mode, t_override, gscale, grad_out, st);
    if (I.B % 2 == 0) return launch_backward_vw<2>(I, S, D, mode, t_override, gscale, grad_out, st);
    return launch_backward_vw<1>(I, S, D, mode, t_override, gscale, grad_out, st);
}

// loss per restart from the forward partials (used where no update follows)
__global__ void k_loss_reduce(DevStep D, int B) {
    __shared__ float s_red[kThreads];
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        float acc = 0.0f;
        for (int k = threadIdx.x; k < D.fwd_blocks; k += blockDim.x)
            acc += D.lpart[(long long)k * B + b];
        s_red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) s_red[threadIdx.x] += s_red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const long long c = D.cost[b];
            D.loss[b] = c > 0 ? s_red[0] / (float)c : 0.0f;
        }
        __syncthreads();
    }
}

cudaError_t launch_loss_reduce(const DevStep &D, int B, cudaStream_t st) {
    int blocks = B < 152 * 4 ? B : 152 * 4;
    k_loss_reduce<<<blocks, kThreads, 0, st>>>(D, B);
    return cudaGetLastError();
}

}  // namespace msat
