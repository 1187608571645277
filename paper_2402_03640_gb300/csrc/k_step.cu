// Step kernels of the MaxSAT gradient engine (sm_103a).
//
//   k_init            random start of x (Algorithm 1 initialisation), zero Adam moments,
//                     tanh(x)
//   k_forward         clause pass: f_j, exact unsat bits, sum_U w and the
//                     loss partials per restart; the last block to finish
//                     turns them into cost, best, 2/W_U and the Adam scalars
//   k_backward_light  variable pass over the transposed CSR for variables
//                     with few occurrences: occurrence terms staged in shared
//                     memory, then per variable the fixed-order sum, 1 - t^2,
//                     fused Adam update, best-assignment capture and tanh
//   k_backward_heavy  the same for variables with many occurrences, split
//                     into 1024-occurrence chunks combined in the fixed order
//
// Layouts: x, mom, vel, t are float [n][B] (restart index innermost), so the
// B values of one variable are one contiguous, vector-loadable row.  A
// thread owns VW consecutive restarts of one clause, occurrence or variable:
// up to 8 in the clause pass, up to 16 when staging occurrence terms, up to
// 4 in the update (where every restart carries x, m, v, t and the sums).

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "msat_internal.cuh"

namespace msat {

namespace {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// --------------------------------------------------------- vector access
// VW floats at p (16-byte aligned for VW >= 4): read-only (nc) loads,
// coherent loads, streaming (evict-first) loads and stores.  Streaming is
// used for data touched once per pass, so the gathered rows of t, the unsat
// bits and the f store keep their L2 lines.

template <int VW>
__device__ __forceinline__ void ldv(const float *__restrict__ p, float (&o)[VW]) {
    if constexpr (VW >= 4) {
#pragma unroll
        for (int k = 0; k < VW / 4; ++k) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + k);
            o[4 * k] = v.x; o[4 * k + 1] = v.y; o[4 * k + 2] = v.z; o[4 * k + 3] = v.w;
        }
    } else if constexpr (VW == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = __ldg(p);
    }
}

template <int VW>
__device__ __forceinline__ void ldv_rw(const float *p, float (&o)[VW]) {
    if constexpr (VW >= 4) {
#pragma unroll
        for (int k = 0; k < VW / 4; ++k) {
            const float4 v = reinterpret_cast<const float4 *>(p)[k];
            o[4 * k] = v.x; o[4 * k + 1] = v.y; o[4 * k + 2] = v.z; o[4 * k + 3] = v.w;
        }
    } else if constexpr (VW == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = *p;
    }
}

template <int VW>
__device__ __forceinline__ void ldv_stream(const float *p, float (&o)[VW]) {
    if constexpr (VW >= 4) {
#pragma unroll
        for (int k = 0; k < VW / 4; ++k) {
            const float4 v = __ldcs(reinterpret_cast<const float4 *>(p) + k);
            o[4 * k] = v.x; o[4 * k + 1] = v.y; o[4 * k + 2] = v.z; o[4 * k + 3] = v.w;
        }
    } else if constexpr (VW == 2) {
        const float2 v = __ldcs(reinterpret_cast<const float2 *>(p));
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = __ldcs(p);
    }
}

template <int VW>
__device__ __forceinline__ void stv(float *p, const float (&o)[VW]) {
    if constexpr (VW >= 4) {
#pragma unroll
        for (int k = 0; k < VW / 4; ++k)
            reinterpret_cast<float4 *>(p)[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
    } else if constexpr (VW == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(o[0], o[1]);
    } else {
        *p = o[0];
    }
}

template <int VW>
__device__ __forceinline__ void stv_stream(float *p, const float (&o)[VW]) {
    if constexpr (VW >= 4) {
#pragma unroll
        for (int k = 0; k < VW / 4; ++k)
            __stcs(reinterpret_cast<float4 *>(p) + k, make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]));
    } else if constexpr (VW == 2) {
        __stcs(reinterpret_cast<float2 *>(p), make_float2(o[0], o[1]));
    } else {
        __stcs(p, o[0]);
    }
}

// ------------------------------------------------------------ clause sums

__device__ __forceinline__ void clause_range(const DevInst &I, int kfix, int j, int &beg, int &end) {
    if (kfix > 0) {
        beg = j * kfix;
        end = beg + kfix;
    } else {
        beg = __ldg(I.coff + j);
        end = __ldg(I.coff + j + 1);
    }
}

// Dyadic counter of finished 32-literal leaves for clauses longer than 32
// literals (the same binary counter as LeafCounter), on a per-thread array
// indexed at run time: it lives in local memory and is touched once per 32
// literals, so short clauses never use it.
template <int VW>
__device__ __forceinline__ void leaf_push(float (&stk)[kClauseLevels][VW], unsigned &cnt, float (&v)[VW]) {
    unsigned c = cnt;
    int lvl = 0;
    while (c & 1u) {
#pragma unroll
        for (int e = 0; e < VW; ++e) v[e] = stk[lvl][e] + v[e];
        c >>= 1;
        ++lvl;
    }
#pragma unroll
    for (int e = 0; e < VW; ++e) stk[lvl][e] = v[e];
    ++cnt;
}

template <int VW>
__device__ __forceinline__ void leaf_finish(const float (&stk)[kClauseLevels][VW], unsigned cnt, float (&r)[VW]) {
    bool have = false;
    for (int lvl = 0; lvl < kClauseLevels; ++lvl) {
        if (!((cnt >> lvl) & 1u)) continue;
#pragma unroll
        for (int e = 0; e < VW; ++e) r[e] = have ? (stk[lvl][e] + r[e]) : stk[lvl][e];
        have = true;
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
    float stk[kClauseLevels][VW];
    unsigned nleaf = 0;
    int in_leaf = 0;
    if constexpr (WANT_SAT && VW <= 2) {
        // the clause pass with one or two restarts a thread: NB literals at
        // a time -- their loads, then their row gathers, then the terms in
        // literal order (the same additions as one literal at a time)
        constexpr int NB = 8 / VW;
        for (int p0 = beg; p0 < end; p0 += NB) {
            int L[NB];
            float tv[NB][VW];
#pragma unroll
            for (int k = 0; k < NB; ++k) L[k] = p0 + k < end ? __ldg(I.lit + p0 + k) : 0;
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (p0 + k < end) ldv<VW>(t + (int64_t)(L[k] >> 1) * B + col, tv[k]);
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                if (p0 + k >= end) break;
                if (in_leaf == 32) {
                    leaf_push<VW>(stk, nleaf, f);
                    in_leaf = 0;
                }
                const bool neg = L[k] & 1;
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    const float term = neg ? -tv[k][e] : tv[k][e];
                    f[e] = (in_leaf == 0) ? term : f[e] + term;
                    sat[e] |= ((tv[k][e] > 0.0f) != neg);
                }
                ++in_leaf;
            }
        }
    } else {
#pragma unroll 2
        for (int p = beg; p < end; ++p) {
            if (in_leaf == 32) {
                leaf_push<VW>(stk, nleaf, f);
                in_leaf = 0;
            }
            const int L = __ldg(I.lit + p);
            const bool neg = L & 1;
            float tv[VW];
            ldv<VW>(t + (int64_t)(L >> 1) * B + col, tv);
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const float term = neg ? -tv[e] : tv[e];
                f[e] = (in_leaf == 0) ? term : f[e] + term;
                if (WANT_SAT) sat[e] |= ((tv[e] > 0.0f) != neg);
            }
            ++in_leaf;
        }
    }
    if (nleaf) {  // more than 32 literals: the last leaf, then the counter
        leaf_push<VW>(stk, nleaf, f);
        leaf_finish<VW>(stk, nleaf, f);
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

// ------------------------------------------------------- occurrence terms

// Unsat bits of (clause of occurrence word o, restarts col .. col+VW-1)
// from the 32-bit word wd that holds them (flat bit index j*B + col, which
// fits 32 bits: the context rejects m*B >= 2^31).
template <int VW>
__device__ __forceinline__ uint32_t occ_nib(const DevInst &I, int o, uint32_t wd, int col) {
    const uint32_t qb = (uint32_t)(o >> I.occ_shift) * (uint32_t)I.B + (uint32_t)col;
    constexpr uint32_t mask = VW >= 32 ? 0xffffffffu : ((1u << VW) - 1u);
    return (wd >> (qb & 31u)) & mask;
}

__device__ __forceinline__ const uint32_t *ubits_word(const DevInst &I, const uint32_t *ubits,
                                                      int o, int col) {
    return ubits + (((uint32_t)(o >> I.occ_shift) * (uint32_t)I.B + (uint32_t)col) >> 5);
}

// f_j for VW restarts (col .. col+VW-1) of the clause of occurrence word o
// (clause j in the bits above occ_shift, literal sign in bit 0), recomputed
// in the literal order; for 3-literal clauses from the expanded occurrence
// record (position of the variable in bits 1-2 of o, the other two
// literals in ox; own_var is the occurring variable).
template <int VW, int KFIX>
__device__ __forceinline__ void fetch_f(const DevInst &I, int kfix, const float *__restrict__ t,
                                        int o, int2 ox, int own_var, int col, float (&f)[VW]) {
    const int B = I.B;
    const int j = o >> I.occ_shift;
    bool sat[VW];
    if constexpr (KFIX == 3) {
        if (I.occx) {
            const int pos = (o >> 1) & 3;
            const int own = (own_var << 1) | (o & 1);
            int L[3];
            L[0] = pos == 0 ? own : ox.x;
            L[1] = pos == 0 ? ox.x : (pos == 1 ? own : ox.y);
            L[2] = pos == 2 ? own : ox.y;
            float tv[3][VW];
#pragma unroll
            for (int p = 0; p < 3; ++p) ldv<VW>(t + (int64_t)(L[p] >> 1) * B + col, tv[p]);
#pragma unroll
            for (int e = 0; e < VW; ++e) {
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    const float tt = (L[p] & 1) ? -tv[p][e] : tv[p][e];
                    f[e] = (p == 0) ? tt : f[e] + tt;
                }
            }
        } else {
            clause_value_fixed<VW, 3>(I, t, j, col, f, sat);
        }
    } else if constexpr (KFIX > 0) {
        clause_value_fixed<VW, KFIX>(I, t, j, col, f, sat);
    } else {
        int beg, end;
        clause_range(I, kfix, j, beg, end);
        clause_value<VW, false>(I, t, beg, end, col, f, sat);
    }
}

// Occurrence term for VW restarts: +-((float)w_j * f_j) * (2/W_U) where
// clause j is unsat (bit set in nib), +0 elsewhere.
template <int VW>
__device__ __forceinline__ void term_from_f(const DevInst &I, int o, uint32_t nib,
                                            const float (&f)[VW], const float (&cs)[VW],
                                            float (&term)[VW]) {
    const int j = o >> I.occ_shift;
    const bool neg = o & 1;
    const float wj = I.w ? (float)__ldg(I.w + j) : 1.0f;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        term[e] = 0.0f;
        if ((nib >> e) & 1u) {
            const float g = (wj * f[e]) * cs[e];
            term[e] = neg ? -g : g;
        }
    }
}

// Terms of C occurrences (words o, expanded records ox, valid where ok) of
// variable own_var for VW restarts at col, all loads of the C occurrences in
// flight together.  With the clause pass's store, q = (float)w_j * f_j (NaN
// where satisfied) gives the term +-(q * 2/W_U) or +0; otherwise the unsat
// bits select the restarts whose f is recomputed (fetched together with the
// bits when unsat clauses are dense).
template <int VW, int KFIX, int C, bool STORE>
__device__ __forceinline__ void occ_terms(const DevInst &I, const DevState &S, int kfix,
                                          const float *__restrict__ tcur, const int (&o)[C],
                                          const int2 (&ox)[C], const bool (&ok)[C], int own_var,
                                          int col, const float (&cs)[VW], bool dense,
                                          float (&term)[C][VW]) {
    const int B = I.B;
    if constexpr (STORE) {
        float q[C][VW];
#pragma unroll
        for (int u = 0; u < C; ++u) {
            if (ok[u]) {
                ldv<VW>(S.fstore + (int64_t)(o[u] >> I.occ_shift) * B + col, q[u]);
            } else {
#pragma unroll
                for (int e = 0; e < VW; ++e) q[u][e] = 0.0f;
            }
        }
#pragma unroll
        for (int u = 0; u < C; ++u) {
            const bool neg = o[u] & 1;
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const float g = q[u][e] * cs[e];
                term[u][e] = (q[u][e] != q[u][e]) ? 0.0f : (neg ? -g : g);
            }
        }
    } else {
        uint32_t wd[C];
        float f[C][VW];
#pragma unroll
        for (int u = 0; u < C; ++u) {
            wd[u] = ok[u] ? __ldg(ubits_word(I, S.ubits, o[u], col)) : 0u;
            if (dense && ok[u]) fetch_f<VW, KFIX>(I, kfix, tcur, o[u], ox[u], own_var, col, f[u]);
        }
#pragma unroll
        for (int u = 0; u < C; ++u) {
            const uint32_t nib = ok[u] ? occ_nib<VW>(I, o[u], wd[u], col) : 0u;
#pragma unroll
            for (int e = 0; e < VW; ++e) term[u][e] = 0.0f;
            if (nib) {
                if (!dense) fetch_f<VW, KFIX>(I, kfix, tcur, o[u], ox[u], own_var, col, f[u]);
                term_from_f<VW>(I, o[u], nib, f[u], cs, term[u]);
            }
        }
    }
}

// The same terms of C consecutive occurrences of one leaf, added in order
// to the leaf sum (first: the chunk opens the leaf, so its first term
// starts the sum instead of being added to +0).
template <int VW, int KFIX, int C, bool STORE>
__device__ __forceinline__ void occ_accumulate(const DevInst &I, const DevState &S, int kfix,
                                               const float *__restrict__ tcur, const int (&o)[C],
                                               const int2 (&ox)[C], const bool (&ok)[C],
                                               int own_var, int col, const float (&cs)[VW],
                                               bool dense, bool first, float (&leaf)[VW]) {
    const int B = I.B;
    float v[C][VW];
    if constexpr (STORE) {
#pragma unroll
        for (int u = 0; u < C; ++u) {
            if (ok[u]) {
                ldv<VW>(S.fstore + (int64_t)(o[u] >> I.occ_shift) * B + col, v[u]);
            } else {
#pragma unroll
                for (int e = 0; e < VW; ++e) v[u][e] = 0.0f;
            }
        }
#pragma unroll
        for (int u = 0; u < C; ++u) {
            if (!ok[u]) continue;
            const bool neg = o[u] & 1;
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const float g = v[u][e] * cs[e];
                const float term = (v[u][e] != v[u][e]) ? 0.0f : (neg ? -g : g);
                leaf[e] = (first && u == 0) ? term : leaf[e] + term;
            }
        }
    } else {
        uint32_t wd[C];
#pragma unroll
        for (int u = 0; u < C; ++u) {
            wd[u] = ok[u] ? __ldg(ubits_word(I, S.ubits, o[u], col)) : 0u;
            if (dense && ok[u]) fetch_f<VW, KFIX>(I, kfix, tcur, o[u], ox[u], own_var, col, v[u]);
        }
#pragma unroll
        for (int u = 0; u < C; ++u) {
            if (!ok[u]) continue;
            const uint32_t nib = occ_nib<VW>(I, o[u], wd[u], col);
            float term[VW];
#pragma unroll
            for (int e = 0; e < VW; ++e) term[e] = 0.0f;
            if (nib) {
                if (!dense) fetch_f<VW, KFIX>(I, kfix, tcur, o[u], ox[u], own_var, col, v[u]);
                term_from_f<VW>(I, o[u], nib, v[u], cs, term);
            }
#pragma unroll
            for (int e = 0; e < VW; ++e) leaf[e] = (first && u == 0) ? term[e] : leaf[e] + term[e];
        }
    }
}

// Dyadic tree over the first K lanes' values (lane 0 receives the result).
__device__ __forceinline__ float warp_dyadic(float v, int K, int lane) {
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const float o = __shfl_down_sync(0xffffffffu, v, s);
        if ((lane & (2 * s - 1)) == 0 && lane + s < K) v = v + o;
    }
    return v;
}

// --------------------------------------------------------------- update

struct AdamView {
    float a_t, r_t, b1, b2, omb1, omb2, eps;
};

__device__ __forceinline__ AdamView adam_view(const StepScalars *sc) {
    AdamView A;
    A.a_t = sc->a_t;
    A.r_t = sc->r_t;
    A.b1 = sc->b1f;
    A.b2 = sc->b2f;
    A.omb1 = sc->omb1f;
    A.omb2 = sc->omb2f;
    A.eps = sc->epsf;
    return A;
}

__device__ __forceinline__ float adam_update(const AdamView &A, float x, float &m, float &v,
                                             float g) {
    const float mq = A.b1 * m + A.omb1 * g;
    const float vq = A.b2 * v + (A.omb2 * g) * g;
    const float den = sqrtf(vq) * A.r_t + A.eps;
    m = mq;
    v = vq;
    return x - (A.a_t * mq) / den;
}

// Update of one (variable, restart group) from its occurrence sum S: the
// gradient S * (1 - t^2) with t = tanh(x) of the evaluated x, then Adam
// (unless the restart has stopped), the best-assignment capture and tanh of
// the new x; or, in the gradient-only mode, the scaled gradient.
template <int VW>
__device__ __forceinline__ void finish_variable(const DevState &S, const DevStep &D,
                                                const AdamView &A, int mode, int64_t q0,
                                                int col, const float *__restrict__ tcur,
                                                const float (&Ssum)[VW], float *tnext,
                                                const float *__restrict__ gscale,
                                                float *__restrict__ grad_out) {
    if constexpr (VW > 4) {  // slices of four restarts keep the live registers down
#pragma unroll
        for (int h = 0; h < VW; h += 4) {
            float part[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) part[e] = Ssum[h + e];
            finish_variable<4>(S, D, A, mode, q0 + h, col + h, tcur, part, tnext, gscale, grad_out);
        }
        return;
    }
    float tv[VW], gr[VW];
    ldv<VW>(tcur + q0, tv);
#pragma unroll
    for (int e = 0; e < VW; ++e) gr[e] = Ssum[e] * fmaf(-tv[e], tv[e], 1.0f);
    if (mode == BWD_GRAD_ONLY) {
#pragma unroll
        for (int e = 0; e < VW; ++e) gr[e] = gscale ? gr[e] * gscale[col + e] : gr[e];
        stv<VW>(grad_out + q0, gr);
        return;
    }
    float xv[VW], mv[VW], vv[VW], tn[VW];
    ldv_stream<VW>(S.x + q0, xv);
    ldv_stream<VW>(S.mom + q0, mv);
    ldv_stream<VW>(S.vel + q0, vv);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        if (D.improved[col + e]) S.bestx[q0 + e] = xv[e] > 0.0f;
        if (D.cost[col + e] != 0) {
            xv[e] = adam_update(A, xv[e], mv[e], vv[e], gr[e]);
            tn[e] = tanh_fixed(xv[e]);
        } else {
            tn[e] = tv[e];
        }
    }
    stv_stream<VW>(S.x + q0, xv);
    stv_stream<VW>(S.mom + q0, mv);
    stv_stream<VW>(S.vel + q0, vv);
    stv<VW>(tnext + q0, tn);
}

__device__ __forceinline__ void step_buffers(const DevState &S, const DevStep &D, int mode,
                                             const float *t_ovr, const float *&tcur,
                                             float *&tnext) {
    const long long steps = D.sc->steps_done;
    if (mode == BWD_UPDATE) {
        tcur = ((steps - 1) & 1) ? S.t1 : S.t0;
        tnext = (steps & 1) ? S.t1 : S.t0;
    } else {
        tcur = t_ovr ? t_ovr : ((steps & 1) ? S.t1 : S.t0);
        tnext = nullptr;
    }
}

}  // namespace

// ------------------------------------------------------------------ k_init

__global__ void k_init(int n, int B, uint64_t seed, float *__restrict__ x,
                       float *__restrict__ mom, float *__restrict__ vel,
                       float *__restrict__ t0, uint8_t *__restrict__ bestx) {
    const int64_t total = (int64_t)n * B;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / B;
        const int64_t b = q - i * B;
        const uint64_t u = splitmix64_at(seed, (uint64_t)b * (uint64_t)n + (uint64_t)i);
        const float k = (float)(uint32_t)(u >> 40);
        const float xv = k * 0x1p-23f - 1.0f;
        x[q] = xv;
        mom[q] = 0.0f;
        vel[q] = 0.0f;
        t0[q] = tanh_fixed(xv);
        bestx[q] = 0;
    }
}

cudaError_t launch_init(const DevInst &I, const DevState &S, uint64_t seed, cudaStream_t st) {
    const int64_t total = (int64_t)I.n * I.B;
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
// One item = (clause j, restart group g of VW restarts).  For VW <= 4 the
// grid-stride loop is unrolled by two (items base + lane and base + stride +
// lane; the stride is a multiple of G, so both belong to the thread's
// restart group), keeping the loads of two clauses in flight; wider groups
// already have VW/4 row loads per literal in flight.  The unsat bits of 32
// consecutive items are packed with shuffles into whole 32-bit words.

template <int VW, int KFIX>
__device__ __forceinline__ void forward_body(const DevInst &I, const float *__restrict__ t0,
                                             const float *__restrict__ t1,
                                             const float *__restrict__ t_ovr, const DevStep &D,
                                             uint32_t *__restrict__ ubits,
                                             float *__restrict__ fstore, int mode, int blk,
                                             int nblk) {
    constexpr int NU = VW <= 4 ? 2 : 1;  // items per lane per iteration
    __shared__ unsigned long long s_w[kThreads];
    __shared__ float s_l[kThreads];
    __shared__ int s_last;

    const int B = I.B;
    const int G = B / VW;
    const long long steps = D.sc->steps_done;
    const float *__restrict__ t = t_ovr ? t_ovr : ((steps & 1) ? t1 : t0);
    const int kfix = KFIX > 0 ? KFIX : I.kfix;
    const int lane = threadIdx.x & 31;
    const int gshift = __ffs(G) - 1;  // G = B / VW is a power of two
    const int g = threadIdx.x & (G - 1);
    const int col = g * VW;
    const long long total = (long long)I.m * G;
    const long long stride = (long long)nblk * blockDim.x;

    float lacc[VW];
    unsigned long long wacc[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        lacc[e] = 0.0f;
        wacc[e] = 0ull;
    }
    constexpr int LPW = 32 / VW;  // lanes whose bits share one 32-bit word
    for (long long base = (long long)blk * blockDim.x + (threadIdx.x & ~31); base < total;
         base += NU * stride) {
        long long item[NU];
        bool act[NU];
        int jj[NU];
#pragma unroll
        for (int h = 0; h < NU; ++h) {
            item[h] = base + h * stride + lane;
            act[h] = item[h] < total;
            jj[h] = act[h] ? (int)(item[h] >> gshift) : 0;
        }
        float f[NU][VW];
        bool sat[NU][VW];
        if constexpr (KFIX > 0) {
            // every clause's literals, then every clause's rows
            int L[NU][KFIX];
#pragma unroll
            for (int h = 0; h < NU; ++h)
#pragma unroll
                for (int p = 0; p < KFIX; ++p) L[h][p] = __ldg(I.lit + jj[h] * KFIX + p);
            float tv[NU][KFIX][VW];
#pragma unroll
            for (int h = 0; h < NU; ++h)
#pragma unroll
                for (int p = 0; p < KFIX; ++p)
                    ldv<VW>(t + (int64_t)(L[h][p] >> 1) * B + col, tv[h][p]);
#pragma unroll
            for (int h = 0; h < NU; ++h)
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
            for (int h = 0; h < NU; ++h) {
                int beg = 0, end = 0;
                if (act[h]) clause_range(I, kfix, jj[h], beg, end);
                clause_value<VW, true>(I, t, beg, end, col, f[h], sat[h]);
            }
        }
#pragma unroll
        for (int h = 0; h < NU; ++h) {
            unsigned nib = 0;
            if (act[h]) {
                const long long wj = I.w ? __ldg(I.w + jj[h]) : 1ll;
                const float wf = (float)wj;
                float q[VW];
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    q[e] = __int_as_float(0x7fc00000);  // satisfied: NaN marker
                    if (!sat[h][e]) {
                        nib |= 1u << e;
                        wacc[e] += (unsigned long long)wj;
                        q[e] = wf * f[h][e];
                        lacc[e] += q[e] * f[h][e];
                    }
                }
                if (fstore) stv<VW>(fstore + (int64_t)jj[h] * B + col, q);
            }
            if (!fstore) {  // uniform: the variable pass reads the bits only when f is recomputed
                unsigned word = nib << ((lane % LPW) * VW);
#pragma unroll
                for (int o = 1; o < LPW; o <<= 1) word |= __shfl_xor_sync(0xffffffffu, word, o);
                if (act[h] && (lane % LPW) == 0) ubits[(item[h] * VW) >> 5] = word;
            }
        }
    }

    // per restart: block sums.  The threads of restart group g are those
    // with threadIdx.x % G == g (G divides the block).  Lanes of one warp in
    // the same group are combined by xor shuffles, then thread g adds the
    // blockDim / max(G, 32) partials of its group.  The weights are integers
    // (any order is exact); the loss partial's order is free because the
    // loss is reported and never fed back into x.
    unsigned long long *acc = D.wu_acc + (long long)(blk % kRep) * B;
    const int per_group = blockDim.x / (G < 32 ? 32 : G);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        unsigned long long sw = wacc[e];
        float sl = lacc[e];
        for (int o = G; o < 32; o <<= 1) {
            sw += __shfl_xor_sync(0xffffffffu, sw, o);
            sl += __shfl_xor_sync(0xffffffffu, sl, o);
        }
        s_w[threadIdx.x] = sw;
        s_l[threadIdx.x] = sl;
        __syncthreads();
        if (threadIdx.x < G) {
            sw = 0;
            sl = 0.0f;
            const int step = G < 32 ? 32 : G;
            for (int k = 0; k < per_group; ++k) {
                sw += s_w[threadIdx.x + k * step];
                sl += s_l[threadIdx.x + k * step];
            }
            const int b = threadIdx.x * VW + e;
            if (sw) atomicAdd(acc + b, sw);
            D.lpart[(long long)blk * B + b] = sl;
        }
        __syncthreads();
    }
    __threadfence();
    if (threadIdx.x == 0) s_last = (atomicAdd(&D.sc->counter, 1u) == nblk - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long my_tot = 0;  // this thread's restarts' costs
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        // every block's additions are complete (fence before the counter):
        // read the replicas from L2, then clear them for the next pass
        unsigned long long wu = 0;
#pragma unroll 8
        for (int r = 0; r < kRep; ++r) wu += __ldcg(D.wu_acc + (long long)r * B + b);
#pragma unroll 8
        for (int r = 0; r < kRep; ++r) D.wu_acc[(long long)r * B + b] = 0ull;
        const long long c = (long long)wu;
        my_tot += wu;
        D.cost[b] = c;
        if (mode != FWD_PROBE) {
            const long long bb = D.best[b];
            const int imp = c < bb;
            if (imp) {
                D.best[b] = c;
                D.best_step[b] = steps;
            }
            D.improved[b] = imp;
        }
        // g_j = (w_j f_j) * 2 / N with N = W_U (mean over the unsat clauses),
        // 1 (sum over them) or the total weight (mean over all clauses)
        const int ln = D.sc->loss_norm;
        const float den = ln == 1 ? 1.0f : (float)(ln == 2 ? D.sc->wsum : c);
        D.cscale[b] = c > 0 ? 2.0f / den : 0.0f;
    }
    // the sum over the restarts from shared memory (integers: any order is
    // exact); the costs just written to global memory are not read back
    s_w[threadIdx.x] = my_tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        StepScalars *sc = D.sc;
        sc->counter = 0;
        unsigned long long tot = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) tot += s_w[k];
        sc->dense = (double)tot * 16.0 > (double)sc->wsum * (double)B;
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

template <int VW, int KFIX>
__global__ void __launch_bounds__(kThreads)
    k_forward(DevInst I, const float *__restrict__ t0, const float *__restrict__ t1,
              const float *__restrict__ t_ovr, DevStep D, uint32_t *__restrict__ ubits,
              float *__restrict__ fstore, int mode) {
    forward_body<VW, KFIX>(I, t0, t1, t_ovr, D, ubits, fstore, mode, blockIdx.x, gridDim.x);
}

int auto_fwd_vw(int B) { return B < 8 ? B : 8; }
int auto_stage_vw(int B) { return B < 4 ? B : 4; }
int update_vw(int B) { return B < 4 ? B : 4; }

template <int VW>
static int fwd_resident(const DevInst &I) {
    int per_sm = 0;
    cudaError_t e = I.kfix == 3
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forward<VW, 3>, kThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forward<VW, 0>, kThreads, 0);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 2;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 152;
    }
    return per_sm * sms;
}

// One wave of resident blocks (the grid-stride loop covers the rest), or
// fewer when the clauses do not fill it.
int fwd_grid_blocks(const DevInst &I) {
    const int VW = I.fwd_vw;
    const int per_thread = VW <= 4 ? 2 : 1;
    const long long items = (long long)I.m * (I.B / VW);
    long long blocks = (items + per_thread * kThreads - 1) / (per_thread * kThreads);
    int resident;
    switch (VW) {
        case 8: resident = fwd_resident<8>(I); break;
        case 4: resident = fwd_resident<4>(I); break;
        case 2: resident = fwd_resident<2>(I); break;
        default: resident = fwd_resident<1>(I); break;
    }
    if (blocks > resident) blocks = resident;
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

cudaError_t launch_forward(const DevInst &I0, const DevState &S, const DevStep &D, int mode,
                           const float *t_override, cudaStream_t st) {
    // with the store's rows grouped by block, the clause pass walks the
    // clauses in row order (its item index is the row it writes)
    DevInst I = I0;
    if (I0.plit) {
        I.lit = I0.plit;
        I.coff = I0.pcoff ? I0.pcoff : I0.coff;
        I.w = I0.pw;
    }
    switch (I.fwd_vw) {
        case 8: return launch_forward_vw<8>(I, S, D, mode, t_override, st);
        case 4: return launch_forward_vw<4>(I, S, D, mode, t_override, st);
        case 2: return launch_forward_vw<2>(I, S, D, mode, t_override, st);
        default: return launch_forward_vw<1>(I, S, D, mode, t_override, st);
    }
}

// -------------------------------------------------------------- k_backward
// Per restart b < B, block b of the light kernel also reduces the loss of
// the evaluated x from the forward block partials.

__device__ __forceinline__ void reduce_loss(const DevStep &D, int B, int blk, int nblk) {
    __shared__ float s_red[kThreads];
    for (int b = blk; b < B; b += nblk) {
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
            const int ln = D.sc->loss_norm;
            const float den = ln == 1 ? 1.0f : (float)(ln == 2 ? D.sc->wsum : c);
            D.loss[b] = c > 0 ? s_red[0] / den : 0.0f;
        }
        __syncthreads();
    }
}

// k_backward_heavy: one block per (1024-occurrence chunk, restart group of
// VW restarts) of a heavy variable.  The chunk's terms are staged in shared
// memory; 32 leaves of 32 terms are summed in order and combined by the
// dyadic tree; the last chunk block of a (variable, group) combines the
// chunk partials with the same tree and applies the update.
template <int VW, int KFIX, bool STORE>
__device__ __forceinline__ void heavy_body(const DevInst &I, const DevState &S, const DevStep &D,
                                           int mode, const float *__restrict__ t_ovr,
                                           const float *__restrict__ gscale,
                                           float *__restrict__ grad_out, int blk) {
    __shared__ float s_term[kChunk * VW];
    __shared__ int s_last;
    const int B = I.B;
    const int G = B / VW;
    const int kfix = KFIX > 0 ? KFIX : I.kfix;
    const float *tcur;
    float *tnext;
    step_buffers(S, D, mode, t_ovr, tcur, tnext);
    const AdamView A = adam_view(D.sc);
    const int gg = blk % G;
    const long long cidx = blk / G;
    const int col = gg * VW;
    const int h = __ldg(I.heavy_of_chunk + cidx);
    const int i = __ldg(I.heavy_var + h);
    const int c0 = __ldg(I.heavy_chunk0 + h);
    const int nch = __ldg(I.heavy_chunk0 + h + 1) - c0;
    const int c = (int)(cidx - c0);
    const int vbeg = __ldg(I.voff + i), vend = __ldg(I.voff + i + 1);
    const int cb = vbeg + c * kChunk;
    const int cn = min(kChunk, vend - cb);  // occurrences in this chunk
    const int lane = threadIdx.x & 31;
    float cs[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) cs[e] = D.cscale[col + e];

    if (mode != BWD_BITS_ONLY) {
        // phase 1: the chunk's terms into shared memory, four per thread in flight
        const bool dense = D.sc->dense != 0;
        const bool expanded = KFIX == 3 && I.occx != nullptr;
        int o[4];
        int2 ox[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = threadIdx.x + u * kThreads;
            ok[u] = r < cn;
            o[u] = ok[u] ? __ldcs(I.occ + cb + r) : 0;
            ox[u] = (expanded && ok[u]) ? __ldcs(I.occx + cb + r) : make_int2(0, 0);
        }
        float term[4][VW];
        occ_terms<VW, KFIX, 4, STORE>(I, S, kfix, tcur, o, ox, ok, i, col, cs, dense, term);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = threadIdx.x + u * kThreads;
            if (ok[u]) {
#pragma unroll
                for (int e = 0; e < VW; ++e) s_term[r * VW + e] = term[u][e];
            }
        }
        __syncthreads();
        // phase 2: 32 leaves of 32 terms in order, then the dyadic tree
        if (threadIdx.x < 32) {
            float leaf[VW];
#pragma unroll
            for (int e = 0; e < VW; ++e) leaf[e] = 0.0f;
            const int lb = lane * 32, le = min(lb + 32, cn);
#pragma unroll 8
            for (int r = lb; r < le; ++r)
#pragma unroll
                for (int e = 0; e < VW; ++e) leaf[e] = (r == lb) ? s_term[r * VW + e] : leaf[e] + s_term[r * VW + e];
            const int K = (cn + 31) / 32;
#pragma unroll
            for (int e = 0; e < VW; ++e) leaf[e] = warp_dyadic(leaf[e], K, lane);
            if (lane == 0) {
#pragma unroll
                for (int e = 0; e < VW; ++e) D.hpart[cidx * B + col + e] = leaf[e];
            }
        }
    }
    // thread 0 wrote the chunk's partial: it alone fences before counting in
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(D.hcount + (long long)h * G + gg, 1u) == (unsigned)(nch - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last chunk block of this (variable, group): dyadic tree over the chunk
    // partials, kChunk of them per round (a round is a complete dyadic block)
    LeafCounter<8> lc[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) lc[e].init();
    if (mode != BWD_BITS_ONLY) {
        for (int base = 0; base < nch; base += kChunk) {
            const int K = min(kChunk, nch - base);
            __syncthreads();
            for (int r = threadIdx.x; r < K; r += kThreads)
#pragma unroll
                for (int e = 0; e < VW; ++e)
                    s_term[r * VW + e] = __ldcg(D.hpart + (long long)(c0 + base + r) * B + col + e);
            __syncthreads();
            for (int st = 1; st < K; st <<= 1) {
                for (int r = threadIdx.x * 2 * st; r < K; r += kThreads * 2 * st)
                    if (r + st < K)
#pragma unroll
                        for (int e = 0; e < VW; ++e) s_term[r * VW + e] = s_term[r * VW + e] + s_term[(r + st) * VW + e];
                __syncthreads();
            }
            if (threadIdx.x == 0)
#pragma unroll
                for (int e = 0; e < VW; ++e) lc[e].push(s_term[e]);
        }
    }
    if (threadIdx.x != 0) return;
    D.hcount[(long long)h * G + gg] = 0;
    const int64_t q0 = (int64_t)i * B + col;
    if (mode == BWD_BITS_ONLY) {
        float xv[VW];
        ldv_rw<VW>(S.x + q0, xv);
#pragma unroll
        for (int e = 0; e < VW; ++e)
            if (D.improved[col + e]) S.bestx[q0 + e] = xv[e] > 0.0f;
        return;
    }
    float Ssum[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) Ssum[e] = lc[e].finish();
    finish_variable<VW>(S, D, A, mode, q0, col, tcur, Ssum, tnext, gscale, grad_out);
}

template <int VW, int KFIX, bool STORE>
__global__ void __launch_bounds__(kThreads)
    k_backward_heavy(DevInst I, DevState S, DevStep D, int mode, const float *__restrict__ t_ovr,
                     const float *__restrict__ gscale, float *__restrict__ grad_out) {
    heavy_body<VW, KFIX, STORE>(I, S, D, mode, t_ovr, gscale, grad_out, blockIdx.x);
}

// k_backward_light: one block per range of consecutive light variables.
// A task is (variable, 32-occurrence leaf, group of VS restarts); the
// restart group is the fastest index, so the lanes of a warp that share a
// leaf read consecutive columns of the same rows.  A thread sums its leaf's
// terms in the stored order, with the loads of four occurrences in flight
// at a time.  A variable with one leaf (or none) is finished by the same
// thread; the leaves of a longer variable meet in shared memory and the
// thread of its first leaf combines them by the dyadic counter, then
// applies the update.  A thread keeps its restart group for all its tasks
// (the task stride, kThreads, is a multiple of the group count).
template <int VS, int KFIX, bool STORE>
__device__ __forceinline__ void vars_body(const DevInst &I, const DevState &S, const DevStep &D,
                                          int mode, const float *__restrict__ t_ovr,
                                          const float *__restrict__ gscale,
                                          float *__restrict__ grad_out, int blk, int nblk) {
    constexpr int C = 4;  // occurrences in flight per thread
    extern __shared__ float4 dyn_smem[];
    __shared__ int s_voff[kThreads + 1];
    __shared__ int s_lpre[kThreads + 1];
    __shared__ int s_wtot[kThreads / 32];
    const int B = I.B;
    const int kfix = KFIX > 0 ? KFIX : I.kfix;
    const float *tcur;
    float *tnext;
    step_buffers(S, D, mode, t_ovr, tcur, tnext);
    if (mode == BWD_UPDATE) reduce_loss(D, B, blk, nblk);
    if (blk >= I.n_lblk) return;  // a grid of one block when every variable is heavy
    const AdamView A = adam_view(D.sc);
    float *s_leaf = reinterpret_cast<float *>(dyn_smem);
    const int2 rg = I.lblk[blk];
    const int v0 = rg.x, nv = rg.y - rg.x;  // nv <= kThreads

    // occurrence offsets and leaf counts of the block's variables, then the
    // exclusive prefix of the leaf counts (warp scans, then warp totals)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int nl = 0;
    if (threadIdx.x < nv) {
        const int a = __ldg(I.voff + v0 + threadIdx.x);
        const int b = __ldg(I.voff + v0 + threadIdx.x + 1);
        s_voff[threadIdx.x] = a;
        if (threadIdx.x == nv - 1) s_voff[nv] = b;
        nl = mode == BWD_BITS_ONLY ? 1 : max(1, (b - a + 31) >> 5);
    }
    int inc = nl;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_wtot[warp] = inc;
    __syncthreads();
    int before = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) before += w < warp ? s_wtot[w] : 0;
    if (threadIdx.x < nv) s_lpre[threadIdx.x] = before + inc - nl;
    if (threadIdx.x == nv - 1) s_lpre[nv] = before + inc;
    __syncthreads();

    const int GS = B / VS;
    const int gshift = __ffs(GS) - 1;  // GS is a power of two <= kThreads
    const int col = (threadIdx.x & (GS - 1)) * VS;
    const int nleaves = s_lpre[nv];
    const int ntasks = nleaves << gshift;
    float cs[VS];
#pragma unroll
    for (int e = 0; e < VS; ++e) cs[e] = D.cscale[col + e];
    const bool dense = D.sc->dense != 0;
    const bool expanded = KFIX == 3 && I.occx != nullptr;

    const bool one_leaf_each = nleaves == nv;  // uniform: task ti belongs to variable ti
    for (int t = threadIdx.x; t < ntasks; t += kThreads) {
        const int ti = t >> gshift;
        int lo = 0, hi = nv - 1;  // the variable: last vloc with s_lpre[vloc] <= ti
        if (one_leaf_each) lo = ti;
        else
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_lpre[mid] <= ti) lo = mid; else hi = mid - 1;
            }
        const int vloc = lo;
        const int L = ti - s_lpre[vloc];
        const int nleaf = s_lpre[vloc + 1] - s_lpre[vloc];
        const int i = v0 + vloc;
        const int64_t q0 = (int64_t)i * B + col;
        if (mode == BWD_BITS_ONLY) {
            float xv[VS];
            ldv_rw<VS>(S.x + q0, xv);
#pragma unroll
            for (int e = 0; e < VS; ++e)
                if (D.improved[col + e]) S.bestx[q0 + e] = xv[e] > 0.0f;
            continue;
        }
        const int pb = s_voff[vloc] + 32 * L;
        const int pe = min(pb + 32, s_voff[vloc + 1]);
        float leaf[VS];
#pragma unroll
        for (int e = 0; e < VS; ++e) leaf[e] = 0.0f;
        // occurrence words one batch ahead: the next batch's words are in
        // flight while this batch's f values are gathered
        int on[C];
        int2 oxn[C];
#pragma unroll
        for (int u = 0; u < C; ++u) {
            const bool okn = pb + u < pe;
            on[u] = okn ? __ldg(I.occ + pb + u) : 0;
            oxn[u] = (expanded && okn) ? __ldg(I.occx + pb + u) : make_int2(0, 0);
        }
        for (int p = pb; p < pe; p += C) {
            int o[C];
            int2 ox[C];
            bool ok[C];
#pragma unroll
            for (int u = 0; u < C; ++u) {
                ok[u] = p + u < pe;
                o[u] = on[u];
                ox[u] = oxn[u];
                const bool okn = p + C + u < pe;
                on[u] = okn ? __ldg(I.occ + p + C + u) : 0;
                oxn[u] = (expanded && okn) ? __ldg(I.occx + p + C + u) : make_int2(0, 0);
            }
            occ_accumulate<VS, KFIX, C, STORE>(I, S, kfix, tcur, o, ox, ok, i, col, cs, dense, p == pb, leaf);
        }
        if (nleaf == 1) {
            finish_variable<VS>(S, D, A, mode, q0, col, tcur, leaf, tnext, gscale, grad_out);
        } else {
            stv<VS>(s_leaf + (int64_t)ti * B + col, leaf);
        }
    }
    if (mode == BWD_BITS_ONLY || nleaves == nv) return;  // uniform: no variable has two leaves
    __syncthreads();
    for (int t = threadIdx.x; t < ntasks; t += kThreads) {
        const int ti = t >> gshift;
        int lo = 0, hi = nv - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_lpre[mid] <= ti) lo = mid; else hi = mid - 1;
        }
        const int vloc = lo;
        const int nleaf = s_lpre[vloc + 1] - s_lpre[vloc];
        if (ti != s_lpre[vloc] || nleaf == 1) continue;
        LeafCounter<5> lc[VS];  // at most kLightMaxDeg = 512 occurrences: 16 leaves
#pragma unroll
        for (int e = 0; e < VS; ++e) lc[e].init();
        for (int l = 0; l < nleaf; ++l) {
            float v[VS];
            ldv_rw<VS>(s_leaf + (int64_t)(ti + l) * B + col, v);
#pragma unroll
            for (int e = 0; e < VS; ++e) lc[e].push(v[e]);
        }
        float Ssum[VS];
#pragma unroll
        for (int e = 0; e < VS; ++e) Ssum[e] = lc[e].finish();
        const int64_t q0 = (int64_t)(v0 + vloc) * B + col;
        finish_variable<VS>(S, D, A, mode, q0, col, tcur, Ssum, tnext, gscale, grad_out);
    }
}

template <int VS, int KFIX, bool STORE>
__global__ void __launch_bounds__(kThreads)
    k_backward_light(DevInst I, DevState S, DevStep D, int mode, const float *__restrict__ t_ovr,
                     const float *__restrict__ gscale, float *__restrict__ grad_out) {
    vars_body<VS, KFIX, STORE>(I, S, D, mode, t_ovr, gscale, grad_out, blockIdx.x, gridDim.x);
}

// The same pass held to 64 registers a thread, so that four 256-thread
// blocks are resident per SM instead of three: used for the shapes where
// that costs no spills (stored w*f with up to 4 restarts a task, or up to 2
// restarts a task).  The pass is latency-bound on its gathers, so the
// extra resident warps hide more of that latency.
template <int VS, int KFIX, bool STORE>
__global__ void __launch_bounds__(kThreads, 4)
    k_backward_light_occ4(DevInst I, DevState S, DevStep D, int mode, const float *__restrict__ t_ovr,
                          const float *__restrict__ gscale, float *__restrict__ grad_out) {
    vars_body<VS, KFIX, STORE>(I, S, D, mode, t_ovr, gscale, grad_out, blockIdx.x, gridDim.x);
}

// Heavy-variable chunks and light blocks in one launch: blocks [0, hblocks)
// take the chunks (first, so the long variables start early), the rest the
// light blocks.  The two write disjoint variables, so neither waits for the
// other, and each fills the other's last partial wave.
template <int VS, int VU, int KFIX, bool STORE, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
    k_backward_mixed(DevInst I, DevState S, DevStep D, int mode, const float *__restrict__ t_ovr,
                     const float *__restrict__ gscale, float *__restrict__ grad_out, int hblocks,
                     int lblocks) {
    if ((int)blockIdx.x < hblocks)
        heavy_body<VU, KFIX, STORE>(I, S, D, mode, t_ovr, gscale, grad_out, blockIdx.x);
    else
        vars_body<VS, KFIX, STORE>(I, S, D, mode, t_ovr, gscale, grad_out, (int)blockIdx.x - hblocks, lblocks);
}

template <int VS, int VU, int KFIX, bool STORE>
static cudaError_t launch_backward_k(const DevInst &I, const DevState &S, const DevStep &D,
                                     int mode, const float *t_ovr, const float *gscale,
                                     float *grad_out, cudaStream_t st) {
    const long long lblocks = I.n_lblk > 0 ? I.n_lblk : 1;
    const size_t smem = light_smem_bytes(I.task_cap, VS);
    if (I.n_heavy > 0) {
        const long long hblocks = I.heavy_chunks * (I.B / VU);  // one block per (chunk, group)
        if constexpr (STORE && VU <= 2 && VS <= 2) {
            // one launch where that keeps the light blocks' 64-register,
            // four-blocks-per-SM shape without spills
            k_backward_mixed<VS, VU, KFIX, STORE, 4><<<(unsigned)(hblocks + lblocks), kThreads, smem, st>>>(
                I, S, D, mode, t_ovr, gscale, grad_out, (int)hblocks, (int)lblocks);
            return cudaGetLastError();
        }
        k_backward_heavy<VU, KFIX, STORE><<<(unsigned)hblocks, kThreads, 0, st>>>(I, S, D, mode, t_ovr,
                                                                                   gscale, grad_out);
        const cudaError_t e = cudaGetLastError();
        if (e) return e;
    }
    if constexpr ((STORE && VS <= 4) || VS <= 2)
        k_backward_light_occ4<VS, KFIX, STORE><<<(unsigned)lblocks, kThreads, smem, st>>>(I, S, D, mode, t_ovr,
                                                                                      gscale, grad_out);
    else
        k_backward_light<VS, KFIX, STORE><<<(unsigned)lblocks, kThreads, smem, st>>>(I, S, D, mode, t_ovr,
                                                                                     gscale, grad_out);
    return cudaGetLastError();
}

template <int VS, int VU>
static cudaError_t launch_backward_vw(const DevInst &I, const DevState &S, const DevStep &D,
                                      int mode, const float *t_ovr, const float *gscale,
                                      float *grad_out, cudaStream_t st) {
    // f stored by the clause pass, or recomputed from the unsat bits
    if (S.fstore) {
        if (I.kfix == 3) return launch_backward_k<VS, VU, 3, true>(I, S, D, mode, t_ovr, gscale, grad_out, st);
        return launch_backward_k<VS, VU, 0, true>(I, S, D, mode, t_ovr, gscale, grad_out, st);
    }
    if (I.kfix == 3) return launch_backward_k<VS, VU, 3, false>(I, S, D, mode, t_ovr, gscale, grad_out, st);
    return launch_backward_k<VS, VU, 0, false>(I, S, D, mode, t_ovr, gscale, grad_out, st);
}

cudaError_t launch_backward(const DevInst &I, const DevState &S, const DevStep &D, int mode,
                            const float *t_override, const float *gscale, float *grad_out,
                            cudaStream_t st) {
    const int vu = update_vw(I.B);
    switch (I.stage_vw * 8 + vu) {
        case 16 * 8 + 4: return launch_backward_vw<16, 4>(I, S, D, mode, t_override, gscale, grad_out, st);
        case 8 * 8 + 4: return launch_backward_vw<8, 4>(I, S, D, mode, t_override, gscale, grad_out, st);
        case 4 * 8 + 4: return launch_backward_vw<4, 4>(I, S, D, mode, t_override, gscale, grad_out, st);
        case 2 * 8 + 4: return launch_backward_vw<2, 4>(I, S, D, mode, t_override, gscale, grad_out, st);
        case 1 * 8 + 4: return launch_backward_vw<1, 4>(I, S, D, mode, t_override, gscale, grad_out, st);
        case 2 * 8 + 2: return launch_backward_vw<2, 2>(I, S, D, mode, t_override, gscale, grad_out, st);
        case 1 * 8 + 2: return launch_backward_vw<1, 2>(I, S, D, mode, t_override, gscale, grad_out, st);
        case 1 * 8 + 1: return launch_backward_vw<1, 1>(I, S, D, mode, t_override, gscale, grad_out, st);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------ batched step
// One launch of each pass advances every instance of a slot table by one
// iteration of Algorithm 1.  A block finds its slot by binary search in the
// launch's block prefix table and runs the same body on that slot's views
// with its block index inside the slot.

__device__ __forceinline__ int slot_of(const int *__restrict__ start, int nslot, int blk) {
    int lo = 0, hi = nslot - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int VW>
__global__ void __launch_bounds__(kThreads)
    k_forward_batch(const SlotDesc *__restrict__ slots, const int *__restrict__ start, int nslot) {
    const int s = slot_of(start, nslot, blockIdx.x);
    const int b0 = __ldg(start + s), b1 = __ldg(start + s + 1);
    const SlotDesc &sd = slots[s];
    forward_body<VW, 0>(sd.I, sd.S.t0, sd.S.t1, nullptr, sd.D, sd.S.ubits, sd.S.fstore, FWD_STEP,
                        blockIdx.x - b0, b1 - b0);
}

template <int VU>
__global__ void __launch_bounds__(kThreads)
    k_backward_heavy_batch(const SlotDesc *__restrict__ slots, const int *__restrict__ start, int nslot) {
    const int s = slot_of(start, nslot, blockIdx.x);
    const SlotDesc &sd = slots[s];
    heavy_body<VU, 0, true>(sd.I, sd.S, sd.D, BWD_UPDATE, nullptr, nullptr, nullptr,
                      blockIdx.x - __ldg(start + s));
}

template <int VS>
__global__ void __launch_bounds__(kThreads)
    k_backward_light_batch(const SlotDesc *__restrict__ slots, const int *__restrict__ start, int nslot) {
    const int s = slot_of(start, nslot, blockIdx.x);
    const int b0 = __ldg(start + s), b1 = __ldg(start + s + 1);
    const SlotDesc &sd = slots[s];
    vars_body<VS, 0, true>(sd.I, sd.S, sd.D, BWD_UPDATE, nullptr, nullptr, nullptr, blockIdx.x - b0, b1 - b0);
}

int heavy_blocks_of(const DevInst &I) {
    return I.n_heavy > 0 ? (int)(I.heavy_chunks * (I.B / update_vw(I.B))) : 0;
}

int light_blocks_of(const DevInst &I) { return I.n_lblk > 0 ? I.n_lblk : 1; }

template <int VS, int VU>
static cudaError_t launch_batch_bwd(const SlotDesc *slots, int nslot, const int *heavy_start,
                                    int heavy_total, const int *light_start, int light_total,
                                    size_t smem, cudaStream_t st) {
    if (heavy_total > 0) {
        k_backward_heavy_batch<VU><<<(unsigned)heavy_total, kThreads, 0, st>>>(slots, heavy_start, nslot);
        const cudaError_t e = cudaGetLastError();
        if (e) return e;
    }
    k_backward_light_batch<VS><<<(unsigned)light_total, kThreads, smem, st>>>(slots, light_start, nslot);
    return cudaGetLastError();
}

cudaError_t launch_step_batch(const SlotDesc *slots, int nslot, const int *fwd_start, int fwd_total,
                              const int *heavy_start, int heavy_total, const int *light_start,
                              int light_total, int B, int fwd_vw, int stage_vw, int task_cap,
                              cudaStream_t st) {
    if (nslot <= 0) return cudaSuccess;
    switch (fwd_vw) {
        case 8: k_forward_batch<8><<<(unsigned)fwd_total, kThreads, 0, st>>>(slots, fwd_start, nslot); break;
        case 4: k_forward_batch<4><<<(unsigned)fwd_total, kThreads, 0, st>>>(slots, fwd_start, nslot); break;
        case 2: k_forward_batch<2><<<(unsigned)fwd_total, kThreads, 0, st>>>(slots, fwd_start, nslot); break;
        default: k_forward_batch<1><<<(unsigned)fwd_total, kThreads, 0, st>>>(slots, fwd_start, nslot); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    const size_t smem = light_smem_bytes(task_cap, stage_vw);
    const int vu = update_vw(B);
    switch (stage_vw * 8 + vu) {
        case 16 * 8 + 4: return launch_batch_bwd<16, 4>(slots, nslot, heavy_start, heavy_total, light_start, light_total, smem, st);
        case 8 * 8 + 4: return launch_batch_bwd<8, 4>(slots, nslot, heavy_start, heavy_total, light_start, light_total, smem, st);
        case 4 * 8 + 4: return launch_batch_bwd<4, 4>(slots, nslot, heavy_start, heavy_total, light_start, light_total, smem, st);
        case 2 * 8 + 4: return launch_batch_bwd<2, 4>(slots, nslot, heavy_start, heavy_total, light_start, light_total, smem, st);
        case 1 * 8 + 4: return launch_batch_bwd<1, 4>(slots, nslot, heavy_start, heavy_total, light_start, light_total, smem, st);
        case 2 * 8 + 2: return launch_batch_bwd<2, 2>(slots, nslot, heavy_start, heavy_total, light_start, light_total, smem, st);
        case 1 * 8 + 2: return launch_batch_bwd<1, 2>(slots, nslot, heavy_start, heavy_total, light_start, light_total, smem, st);
        case 1 * 8 + 1: return launch_batch_bwd<1, 1>(slots, nslot, heavy_start, heavy_total, light_start, light_total, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

// loss per restart from the forward partials (used where no update follows)
__global__ void k_loss_reduce(DevStep D, int B) { reduce_loss(D, B, blockIdx.x, gridDim.x); }

cudaError_t launch_loss_reduce(const DevStep &D, int B, cudaStream_t st) {
    const int blocks = B < 152 * 4 ? B : 152 * 4;
    k_loss_reduce<<<blocks, kThreads, 0, st>>>(D, B);
    return cudaGetLastError();
}


// ------------------------------------------------------- small instances
// k_small_steps: n_steps iterations of Algorithm 1 for a small instance in
// one launch of one CTA, with x, the Adam moments, t = tanh(x) and the
// clause pass's w*f (NaN where satisfied) held in shared memory; literal
// and occurrence lists are read through L1.  Per step: the clause pass
// (one thread per (clause, restart), the fixed literal order with 32-term
// leaves), the per-restart scalars (cost, best, 2/N, the Adam products in
// double), the variable pass (one thread per (variable, restart), the
// fixed occurrence order with 32-term leaves and the dyadic counter, then
// the same Adam update and tanh), each separated by a block barrier.  Every
// value that enters x is computed with the operations of the per-pass
// kernels, so the trajectory is the same bit for bit; the state left in
// device memory (x, moments, t in the buffer of the step parity, best,
// cost, scalars) is what those kernels leave.  The loss partials are summed
// in another order (the loss is reported, never fed back).

__device__ __forceinline__ float small_clause_f(const DevInst &I, const float *__restrict__ st,
                                                int j, int b, bool &sat) {
    const int B = I.B;
    int beg, end;
    clause_range(I, I.kfix, j, beg, end);
    LeafCounter<kClauseLevels> lc;
    lc.init();
    float leaf = 0.0f;
    int in_leaf = 0;
    sat = false;
    for (int p = beg; p < end; ++p) {
        const int L = __ldg(I.lit + p);
        const bool neg = L & 1;
        const float tv = st[(L >> 1) * B + b];
        const float term = neg ? -tv : tv;
        leaf = in_leaf == 0 ? term : leaf + term;
        sat |= (tv > 0.0f) != neg;
        if (++in_leaf == 32) {
            lc.push(leaf);
            in_leaf = 0;
        }
    }
    if (lc.cnt == 0) return in_leaf ? leaf : 0.0f;  // at most 32 literals: the leaf itself
    if (in_leaf) lc.push(leaf);
    return lc.finish();
}

__global__ void __launch_bounds__(kSmallThreads, 1)
    k_small_steps(DevInst I, DevState S, DevStep D, int n_steps) {
    extern __shared__ float4 small_smem[];
    __shared__ float s_lsum[kSmallMaxB];
    __shared__ float s_lp[kSmallThreads];
    __shared__ unsigned long long s_wp[kSmallThreads];
    __shared__ long long s_cost[kSmallMaxB], s_best[kSmallMaxB], s_bstep[kSmallMaxB];
    __shared__ int s_imp[kSmallMaxB];
    __shared__ float s_cs[kSmallMaxB];
    __shared__ float s_at, s_rt, s_at_next, s_rt_next;
    const int B = I.B;
    const int nB = I.n * B, mB = I.m * B;
    float *sx = reinterpret_cast<float *>(small_smem);
    float *smo = sx + nB, *sve = smo + nB, *st = sve + nB, *sq = st + nB;
    StepScalars *sc = D.sc;
    const long long steps0 = sc->steps_done;
    const float *t_in = (steps0 & 1) ? S.t1 : S.t0;
    for (int q = threadIdx.x; q < nB; q += blockDim.x) {
        sx[q] = S.x[q];
        smo[q] = S.mom[q];
        sve[q] = S.vel[q];
        st[q] = t_in[q];
    }
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        s_best[b] = D.best[b];
        s_bstep[b] = D.best_step[b];
    }
    const AdamView A0 = adam_view(sc);
    const int ln = sc->loss_norm;
    const long long wsum = sc->wsum;
    // Adam scalars of each step from the running products, in double as the
    // clause pass's last block computes them; the last thread computes the
    // next step's while the others run the variable pass
    double p1 = sc->p1, p2 = sc->p2;  // used by the last thread
    double fin_p1 = p1, fin_p2 = p2;  // the products of the last step taken
    float fin_at = 0.0f, fin_rt = 0.0f;
    const int tl = blockDim.x - 1;
    if (threadIdx.x == tl) {
        p1 = p1 * sc->beta1;
        p2 = p2 * sc->beta2;
        s_at = (float)(sc->lr / (1.0 - p1));
        s_rt = (float)(1.0 / sqrt(1.0 - p2));
    }
    __syncthreads();
    for (int step = 0; step < n_steps; ++step) {
        // clause pass: f, exact unsat test, w*f (NaN where satisfied), sums.
        // The item stride (the block) is a multiple of B, so a thread keeps
        // one restart and its loss partial is one float.
        float lpart = 0.0f;
        unsigned long long wpart = 0ull;
        for (int it = threadIdx.x; it < mB; it += blockDim.x) {
            const int j = it / B, b = it - j * B;
            bool sat;
            const float f = small_clause_f(I, st, j, b, sat);
            float q = __int_as_float(0x7fc00000);
            if (!sat) {
                const long long wj = I.w ? __ldg(I.w + j) : 1ll;
                q = (float)wj * f;
                wpart += (unsigned long long)wj;
                lpart += q * f;
            }
            sq[it] = q;
        }
        // loss partials in a fixed order: lanes of a restart by a shuffle
        // tree, then the warp partials in warp order
        for (int o = B; o < 32; o <<= 1) {
            lpart += __shfl_xor_sync(0xffffffffu, lpart, o);
            wpart += __shfl_xor_sync(0xffffffffu, wpart, o);
        }
        s_lp[threadIdx.x] = lpart;
        s_wp[threadIdx.x] = wpart;
        __syncthreads();
        // per-restart sums (integers exact in any order), then the scalars as
        // the clause pass's last block computes them
        for (int b = threadIdx.x; b < B; b += blockDim.x) {
            const int stride = B < 32 ? 32 : B;
            float sum = 0.0f;
            unsigned long long wsm = 0ull;
            for (int k = b; k < (int)blockDim.x; k += stride) {
                sum += s_lp[k];
                wsm += s_wp[k];
            }
            s_lsum[b] = sum;
            const long long c = (long long)wsm;
            const int imp = c < s_best[b];
            if (imp) {
                s_best[b] = c;
                s_bstep[b] = steps0 + step;
            }
            s_cost[b] = c;
            s_imp[b] = imp;
            const float den = ln == 1 ? 1.0f : (float)(ln == 2 ? wsum : c);
            s_cs[b] = c > 0 ? 2.0f / den : 0.0f;
        }
        __syncthreads();
        AdamView A = A0;
        A.a_t = s_at;
        A.r_t = s_rt;
        // variable pass: occurrence sum, gradient, best capture, Adam, tanh
        for (int it = threadIdx.x; it < nB; it += blockDim.x) {
            const int i = it / B, b = it - i * B;
            const int vb = __ldg(I.voff + i), ve = __ldg(I.voff + i + 1);
            const float cs = s_cs[b];
            LeafCounter<10> lc;
            lc.init();
            float leaf = 0.0f;
            int in_leaf = 0;
            for (int p = vb; p < ve; ++p) {
                const int o = __ldg(I.occ + p);
                const float qv = sq[(o >> I.occ_shift) * B + b];
                const float g = qv * cs;
                const float term = (qv != qv) ? 0.0f : ((o & 1) ? -g : g);
                leaf = in_leaf == 0 ? term : leaf + term;
                if (++in_leaf == 32) {
                    lc.push(leaf);
                    in_leaf = 0;
                }
            }
            if (in_leaf) lc.push(leaf);
            const float Ssum = lc.finish();
            const float tv = st[it];
            const float gr = Ssum * fmaf(-tv, tv, 1.0f);
            float xv = sx[it], mv = smo[it], vv = sve[it];
            if (s_imp[b]) S.bestx[it] = xv > 0.0f;
            if (s_cost[b] != 0) {
                xv = adam_update(A, xv, mv, vv, gr);
                sx[it] = xv;
                smo[it] = mv;
                sve[it] = vv;
                st[it] = tanh_fixed(xv);
            }
        }
        if (threadIdx.x == tl) {  // the next step's scalars; read after the barrier
            fin_p1 = p1;
            fin_p2 = p2;
            fin_at = A.a_t;
            fin_rt = A.r_t;
            p1 = p1 * sc->beta1;
            p2 = p2 * sc->beta2;
            s_at_next = (float)(sc->lr / (1.0 - p1));
            s_rt_next = (float)(1.0 / sqrt(1.0 - p2));
        }
        __syncthreads();
        if (threadIdx.x == tl) {
            s_at = s_at_next;
            s_rt = s_rt_next;
        }
    }
    // the state the per-pass kernels leave
    float *t_out = ((steps0 + n_steps) & 1) ? S.t1 : S.t0;
    for (int q = threadIdx.x; q < nB; q += blockDim.x) {
        S.x[q] = sx[q];
        S.mom[q] = smo[q];
        S.vel[q] = sve[q];
        t_out[q] = st[q];
    }
    if (S.fstore)
        for (int q = threadIdx.x; q < mB; q += blockDim.x) S.fstore[q] = sq[q];
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        D.cost[b] = s_cost[b];
        D.best[b] = s_best[b];
        D.best_step[b] = s_bstep[b];
        D.improved[b] = s_imp[b];
        D.cscale[b] = s_cs[b];
        const long long c = s_cost[b];
        const float den = ln == 1 ? 1.0f : (float)(ln == 2 ? wsum : c);
        D.loss[b] = c > 0 ? s_lsum[b] / den : 0.0f;
    }
    if (threadIdx.x == tl) {
        long long tot = 0;
        for (int b = 0; b < B; ++b) tot += s_cost[b];
        sc->dense = (double)tot * 16.0 > (double)wsum * (double)B;
        sc->p1 = fin_p1;
        sc->p2 = fin_p2;
        sc->a_t = fin_at;
        sc->r_t = fin_rt;
        sc->steps_done = steps0 + n_steps;
    }
}

size_t small_smem_bytes(const DevInst &I) {
    return sizeof(float) * (4 * (size_t)I.n * I.B + (size_t)I.m * I.B);
}

bool small_fits(const DevInst &I, int max_deg) {
    return !I.plit && I.B <= kSmallMaxB && small_smem_bytes(I) <= kSmallSmemMax && max_deg <= 32 * 1023 &&
           (long long)I.m * I.B <= (1LL << 30);
}

cudaError_t launch_small_steps(const DevInst &I, const DevState &S, const DevStep &D, int n_steps,
                               cudaStream_t st) {
    if (n_steps <= 0) return cudaSuccess;
    const size_t smem = small_smem_bytes(I);
    cudaError_t e = cudaFuncSetAttribute(k_small_steps, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmallSmemMax);
    if (e) return e;
    // a block of the work's size (a power of two, a multiple of B): the
    // per-step barriers cost less with fewer warps
    const long long items = std::max<long long>((long long)I.m * I.B, (long long)I.n * I.B);
    int threads = 64;
    while (threads < items && threads < kSmallThreads) threads <<= 1;
    k_small_steps<<<1, threads, smem, st>>>(I, S, D, n_steps);
    return cudaGetLastError();
}

}  // namespace msat
