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

// Occurrence term of clause j (occurrence sign neg) for VW restarts:
// +-((float)w_j * f_j) * (2/W_U) where clause j is unsat, +0 elsewhere.
template <int VW>
__device__ __forceinline__ void occ_term(const DevInst &I, int kfix, const float *__restrict__ t,
                                         const uint32_t *__restrict__ ubits,
                                         const float (&cs)[VW], int o, int col,
                                         float (&term)[VW]) {
    const int B = I.B;
    const int j = o >> 1;
    const bool neg = o & 1;
    const int64_t qb = (int64_t)j * B + col;
    const uint32_t wd = __ldg(ubits + (qb >> 5));
    const uint32_t nib = (wd >> (qb & 31)) & ((1u << VW) - 1u);
#pragma unroll
    for (int e = 0; e < VW; ++e) term[e] = 0.0f;
    if (nib) {
        int beg, end;
        clause_range(I, kfix, j, beg, end);
        float f[VW];
        bool sat[VW];
        clause_value<VW, false>(I, t, beg, end, col, f, sat);
        const float wj = I.w ? (float)__ldg(I.w + j) : 1.0f;
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            if ((nib >> e) & 1u) {
                float g = (wj * f[e]) * cs[e];
                term[e] = neg ? -g : g;
            }
        }
    }
}

// Canonical occurrence sum of a variable with occurrences [beg, end) in one
// thread: 32-term leaves in order, leaves combined by the dyadic counter.
template <int VW>
__device__ __forceinline__ void occ_sum_thread(const DevInst &I, int kfix,
                                               const float *__restrict__ t,
                                               const uint32_t *__restrict__ ubits,
                                               const float (&cs)[VW], int beg, int end, int col,
                                               float (&S)[VW]) {
    LeafCounter<6> lc[VW];
    float leaf[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        lc[e].init();
        leaf[e] = 0.0f;
    }
    int in_leaf = 0;
    for (int s = beg; s < end; ++s) {
        float term[VW];
        occ_term<VW>(I, kfix, t, ubits, cs, __ldg(I.occ + s), col, term);
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
#pragma unroll
    for (int e = 0; e < VW; ++e) S[e] = lc[e].finish();
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

template <int VW, int KFIX>
__global__ void __launch_bounds__(kThreads)
    k_forward(DevInst I, const float *__restrict__ t0, const float *__restrict__ t1,
              const float *__restrict__ t_ovr, DevStep D, uint32_t *__restrict__ ubits, int mode) {
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
         base += stride) {
        const long long item = base + lane;
        const bool active = item < total;
        unsigned nib = 0;
        if (active) {
            const int j = (int)(item / G);
            int beg, end;
            clause_range(I, kfix, j, beg, end);
            float f[VW];
            bool sat[VW];
            clause_value<VW, true>(I, t, beg, end, col, f, sat);
            const long long wj = I.w ? __ldg(I.w + j) : 1ll;
            const float wf = (float)wj;
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                if (!sat[e]) {
                    nib |= 1u << e;
                    wacc[e] += (unsigned long long)wj;
                    lacc[e] += (wf * f[e]) * f[e];
                }
            }
        }
        unsigned word = nib << ((lane % LPW) * VW);
#pragma unroll
        for (int o = 1; o < LPW; o <<= 1) word |= __shfl_xor_sync(0xffffffffu, word, o);
        if (active && (lane % LPW) == 0) ubits[(item * VW) >> 5] = word;
    }

#pragma unroll
    for (int e = 0; e < VW; ++e) {
        s_w[threadIdx.x * VW + e] = wacc[e];
        s_l[threadIdx.x * VW + e] = lacc[e];
    }
    __syncthreads();
    if (threadIdx.x < G) {
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            unsigned long long sw = 0;
            float sl = 0.0f;
            for (int r = threadIdx.x; r < blockDim.x; r += G) {
                sw += s_w[r * VW + e];
                sl += s_l[r * VW + e];
            }
            const int b = threadIdx.x * VW + e;
            if (sw) atomicAdd(D.wu_acc + b, sw);
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
        const long long c = (long long)atomicExch(D.wu_acc + b, 0ull);
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
    long long blocks = (items + kThreads - 1) / kThreads;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

template <int VW>
static cudaError_t launch_forward_vw(const DevInst &I, const DevState &S, const DevStep &D,
                                     int mode, const float *t_ovr, uint32_t *ubits,
                                     cudaStream_t st) {
    const int blocks = D.fwd_blocks;
    if (I.kfix == 3)
        k_forward<VW, 3><<<blocks, kThreads, 0, st>>>(I, S.t0, S.t1, t_ovr, D, ubits, mode);
    else
        k_forward<VW, 0><<<blocks, kThreads, 0, st>>>(I, S.t0, S.t1, t_ovr, D, ubits, mode);
    return cudaGetLastError();
}

cudaError_t launch_forward(const DevInst &I, const DevState &S, const DevStep &D, int mode,
                           const float *t_override, cudaStream_t st) {
    if (I.B % 4 == 0) return launch_forward_vw<4>(I, S, D, mode, t_override, S.ubits, st);
    if (I.B % 2 == 0) return launch_forward_vw<2>(I, S, D, mode, t_override, S.ubits, st);
    return launch_forward_vw<1>(I, S, D, mode, t_override, S.ubits, st);
}

// -------------------------------------------------------------- k_backward

template <int VW, int KFIX>
__global__ void __launch_bounds__(kThreads)
    k_backward(DevInst I, DevState S, DevStep D, int mode, const float *__restrict__ x_ovr,
               const float *__restrict__ t_ovr, const float *__restrict__ gscale,
               float *__restrict__ grad_out, int heavy_blocks) {
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
    const float *xin = x_ovr ? x_ovr : S.x;
    const uint32_t *__restrict__ ubits = S.ubits;

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

    if ((int)blockIdx.x < heavy_blocks) {
        // ---------------- heavy variables: one warp per (chunk, restart group)
        const int lane = threadIdx.x & 31;
        const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const long long nwarps = ((long long)heavy_blocks * blockDim.x) >> 5;
        const long long nchunks = I.n_heavy > 0 ? __ldg(I.heavy_chunk0 + I.n_heavy) : 0;
        for (long long it = warp; it < nchunks * G; it += nwarps) {
            const int gg = (int)(it % G);
            const long long cidx = it / G;
            const int col = gg * VW;
            // heavy variable owning chunk cidx
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
                    float term[VW];
                    occ_term<VW>(I, kfix, tcur, ubits, cs, __ldg(I.occ + s), col, term);
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
                if (mode == BWD_GRAD_ONLY) ldv<VW>(tcur + q0, xv); else ldv_rw<VW>(xin + q0, xv);
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

    // -------------------- light variables: one thread per (variable, group)
    const int lblock = blockIdx.x - heavy_blocks;
    const int lblocks = gridDim.x - heavy_blocks;
    const int g = threadIdx.x % G;
    const int col = g * VW;
    float cs[VW], gsc[VW];
    bool upd[VW], imp[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        cs[e] = D.cscale[col + e];
        gsc[e] = gscale ? gscale[col + e] : 1.0f;
        upd[e] = mode == BWD_UPDATE && D.cost[col + e] != 0;
        imp[e] = mode != BWD_GRAD_ONLY && D.improved[col + e] != 0;
    }
    const long long total = (long long)I.n * G;
    const long long stride = (long long)lblocks * blockDim.x;
    for (long long item = (long long)lblock * blockDim.x + threadIdx.x; item < total; item += stride) {
        const int i = (int)(item / G);
        const int beg = __ldg(I.voff + i), end = __ldg(I.voff + i + 1);
        if (end - beg > I.heavy_deg) continue;
        const int64_t q0 = (int64_t)i * B + col;
        float xv[VW];  // x, or t = tanh(x) in the gradient-only mode
        if (mode == BWD_GRAD_ONLY) ldv<VW>(tcur + q0, xv); else ldv_rw<VW>(xin + q0, xv);
        if (mode == BWD_BITS_ONLY) {
#pragma unroll
            for (int e = 0; e < VW; ++e)
                if (imp[e]) S.bestx[q0 + e] = xv[e] > 0.0f;
            continue;
        }
        float Ssum[VW];
        occ_sum_thread<VW>(I, kfix, tcur, ubits, cs, beg, end, col, Ssum);
        float gr[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            const float tv = (mode == BWD_GRAD_ONLY) ? xv[e] : tanh_fixed(xv[e]);
            gr[e] = Ssum[e] * fmaf(-tv, tv, 1.0f);
        }
        if (mode == BWD_GRAD_ONLY) {
#pragma unroll
            for (int e = 0; e < VW; ++e) gr[e] = gscale ? gr[e] * gsc[e] : gr[e];
            stv<VW>(grad_out + q0, gr);
            continue;
        }
        float mv[VW], vv[VW], xn[VW], tn[VW];
        ldv_rw<VW>(S.mom + q0, mv);
        ldv_rw<VW>(S.vel + q0, vv);
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            xn[e] = upd[e] ? adam_update(A, xv[e], mv[e], vv[e], gr[e]) : xv[e];
            if (imp[e]) S.bestx[q0 + e] = xv[e] > 0.0f;
            tn[e] = tanh_fixed(xn[e]);
        }
        stv<VW>(S.x + q0, xn);
        stv<VW>(S.mom + q0, mv);
        stv<VW>(S.vel + q0, vv);
        stv<VW>(tnext + q0, tn);
    }
}

template <int VW, int KFIX>
static cudaError_t launch_backward_k(const DevInst &I, const DevState &S, const DevStep &D,
                                     int mode, const float *x_ovr, const float *t_ovr,
                                     const float *gscale, float *grad_out, cudaStream_t st) {
    const int G = I.B / VW;
    const long long items = (long long)I.n * G;
    long long lblocks = (items + kThreads - 1) / kThreads;
    if (lblocks > 152 * 8) lblocks = 152 * 8;
    if (lblocks < 1) lblocks = 1;
    long long hblocks = 0;
    if (I.n_heavy > 0) {
        const long long warps = I.heavy_chunks * G;  // one warp per (chunk, group)
        hblocks = (warps + (kThreads / 32) - 1) / (kThreads / 32);
        if (hblocks > 152 * 8) hblocks = 152 * 8;
    }
    k_backward<VW, KFIX><<<(int)(hblocks + lblocks), kThreads, 0, st>>>(
        I, S, D, mode, x_ovr, t_ovr, gscale, grad_out, (int)hblocks);
    return cudaGetLastError();
}

template <int VW>
static cudaError_t launch_backward_vw(const DevInst &I, const DevState &S, const DevStep &D,
                                      int mode, const float *x_ovr, const float *t_ovr,
                                      const float *gscale, float *grad_out, cudaStream_t st) {
    if (I.kfix == 3)
        return launch_backward_k<VW, 3>(I, S, D, mode, x_ovr, t_ovr, gscale, grad_out, st);
    return launch_backward_k<VW, 0>(I, S, D, mode, x_ovr, t_ovr, gscale, grad_out, st);
}

cudaError_t launch_backward(const DevInst &I, const DevState &S, const DevStep &D, int mode,
                            const float *x_override, const float *t_override,
                            const float *gscale, float *grad_out, cudaStream_t st) {
    if (I.B % 4 == 0)
        return launch_backward_vw<4>(I, S, D, mode, x_override, t_override, gscale, grad_out, st);
    if (I.B % 2 == 0)
        return launch_backward_vw<2>(I, S, D, mode, x_override, t_override, gscale, grad_out, st);
    return launch_backward_vw<1>(I, S, D, mode, x_override, t_override, gscale, grad_out, st);
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
