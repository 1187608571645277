// Internal declarations of the GB300 MaxSAT engine: device views of the
// instance and the step state, the fixed-order fp32 arithmetic shared by the
// kernels, and the launchers each kernel file provides.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/msat.h"

namespace msat {

// ------------------------------------------------------------ error plumbing

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define MSAT_CUDA_TRY(expr)                                  \
    do {                                                     \
        cudaError_t e__ = (expr);                            \
        if (e__ != cudaSuccess) return cuda_fail(e__, #expr); \
    } while (0)

// ------------------------------------------------------------- device views

// Clause CSR and its transpose (variable -> occurrences), both in stored
// literal order.  lit = var << 1 | neg; occ = clause << 1 | neg.
struct DevInst {
    int32_t n;
    int32_t m;
    int32_t B;
    int32_t kfix;                 // common clause length (> 0) or 0
    const int32_t *coff;          // [m+1] (unused when kfix > 0)
    const int32_t *lit;           // [nnz]
    const int64_t *w;             // [m] or nullptr (all weights 1)
    const int32_t *voff;          // [n+1]
    const int32_t *occ;           // [nnz]
    int32_t heavy_deg;            // degree above which a variable is split
    int32_t n_heavy;              // number of heavy variables
    long long heavy_chunks;       // total chunks of the heavy variables
    const int32_t *heavy_var;     // [n_heavy] variable ids
    const int32_t *heavy_chunk0;  // [n_heavy+1] prefix of chunk counts
    const int32_t *heavy_of_chunk;  // [heavy_chunks] heavy index h of each chunk
    int32_t occ_shift;            // occ word: clause index above this bit (1, or 3 when
                                  // bits 1-2 hold the variable's position in its clause)
    const int2 *occx;             // [nnz] other two literals of a 3-literal clause, or nullptr
    int32_t n_lblk;               // blocks of the light-variable pass
    int32_t task_cap;             // leaf tasks (32-occurrence leaf x restart group) of
                                  // one light block; sizes its shared leaf partials
    int32_t fwd_vw;               // restarts per thread in the clause pass
    int32_t stage_vw;             // restarts per thread of a light-variable leaf task
    const int2 *lblk;             // [n_lblk] variable range [x, y) of each light block
    // stored w*f with rows grouped by light block (or nullptr: row = clause):
    // the clause arrays in row order, which the clause pass reads instead
    // of lit / coff / w; the occurrence words then carry rows, not clauses
    const int32_t *plit;          // [nnz]
    const int32_t *pcoff;         // [m+1] or nullptr (every clause has kfix literals)
    const int64_t *pw;            // [m] or nullptr (all weights 1)
};

// Scalars of the optimizer step shared by all restarts.
struct StepScalars {
    unsigned int counter;   // finished-block counter of the forward kernel
    int loss_norm;          // MSAT_LOSS_*: normaliser of the loss and of g
    long long steps_done;   // Adam steps taken
    double p1, p2;          // beta1^steps_done, beta2^steps_done (running products)
    float a_t, r_t;         // lr / (1 - p1), 1 / sqrt(1 - p2) of the step in flight
    double lr, beta1, beta2, eps;
    float b1f, b2f, omb1f, omb2f, epsf;
    int dense;              // last evaluation left > 1/16 of the clause weight unsat:
                            // the variable pass fetches f before testing the unsat bits
    long long wsum;         // sum of all clause weights
};

// Per-restart step state plus scratch.
struct DevStep {
    StepScalars *sc;
    unsigned long long *wu_acc;  // [kRep][B] atomic accumulators of sum_U w
    long long *cost;             // [B] cost of the evaluated x
    long long *best;             // [B] best cost so far
    long long *best_step;        // [B] updates taken before the x that gave it (0: x_0)
    int *improved;               // [B] cost < best at the last evaluation
    float *cscale;               // [B] 2 / (float)W_U (0 if W_U = 0)
    float *loss;                 // [B] loss of the last updated x
    float *lpart;                // [fwd_blocks][B] per-block loss partials
    int fwd_blocks;              // blocks of the forward launch
    float *hpart;                // [total heavy chunks][B] heavy chunk partials
    unsigned int *hcount;        // [n_heavy][G] heavy finish counters
};

struct DevState {
    float *x, *mom, *vel;  // [n][B]
    float *t0, *t1;        // double-buffered tanh(x), [n][B]
    uint32_t *ubits;       // unsat bits, flat index row*B + b (row = j unless grouped)
    uint8_t *bestx;        // [n][B] best assignment (0/1)
    float *fstore;         // [m][B] of the last clause pass: (float)w_j * f_j where clause
                           // j is unsat for restart b, NaN where it is satisfied; or
                           // nullptr: the variable pass recomputes f from the unsat bits
};

// Dense tensor-core evaluation (k_dense.cu): clause matrix W^T
// [m_pad][n_pad] in packed e2m1 (n_pad / 2 bytes a row), per-row target
// -len_j (NaN: never unsat), 32-bit weights, the packed e2m1 assignment
// batch X^T [rows][n_pad] and their TMA descriptors.
// Variables per k-step of the dense evaluation (n is padded to a multiple).
constexpr int kDenseKStep = 256;

// Work split of one dense launch: tile t covers clause rows
// (t % tiles_m) * 128 and assignment columns (t / tiles_m) * ntile; CTA c
// takes whole tiles j * grid + c for j < full, then (c < extra) whole tile
// full * grid + c, or (c < tail_ctas) piece c % split of split tile
// c / split: k-steps [piece * kt_count / split, (piece + 1) * kt_count /
// split) of tile full * grid + c / split.  extra and tail are never both
// nonzero.
struct DenseSched {
    int kt_count;   // k-steps (kDenseKStep variables) per tile
    int tiles_m;
    int ntile;      // assignments per tile
    int full;
    int tail;       // split tiles
    int split;      // pieces per split tile
    int tail_ctas;  // tail * split
    int extra;      // CTAs that take one more whole tile
};

struct DenseDev {
    uint8_t *Wt = nullptr;
    float *target = nullptr;
    uint32_t *wgt = nullptr;
    bool unit_w = false;  // every clause weight is 1
    int m_pad = 0, n_pad = 0;
    uint8_t *Xt = nullptr;
    size_t xt_bytes = 0;
    int tmB_rows = 0, tmB_ntile = 0;
    unsigned int *errflag = nullptr;
    // split tiles: per-piece targets [tile][piece][row], the pieces' unsat
    // bits [tile][piece][column / 32][row] and the pieces counted in per
    // tile (kept zeroed); plan and plan_grid: what the targets were made for
    float *ptgt = nullptr;
    uint32_t *pmask = nullptr;
    unsigned int *part_cnt = nullptr;
    int ptgt_slots = 0, part_cnts = 0, pmask_ntile = 0;
    DenseSched plan{};
    int plan_grid = -1;
    int sm_count = 0;
    CUtensorMap tmA, tmB;
};

// One instance of a batched launch (serving): its device views and the
// first block of each pass in the launch grids.  start[] tables of the
// launches are prefix sums of the per-slot block counts.
struct SlotDesc {
    DevInst I;
    DevState S;
    DevStep D;
};

// Kernel modes of the variable pass.
enum { BWD_UPDATE = 0, BWD_BITS_ONLY = 1, BWD_GRAD_ONLY = 2 };

constexpr int kThreads = 256;
constexpr int kRep = 32;                 // replicas of the per-restart cost accumulator
constexpr int kTaskCap = 256;          // default leaf tasks of one light block
constexpr int kLightMaxDeg = 512;      // more occurrences than this: heavy variable
constexpr int kMaxClauseLen = 32767;  // at most 1024 leaves of 32 literals
constexpr int kClauseLevels = 11;     // binary leaf counter of a clause sum (1024 leaves)
constexpr int kChunk = 1024;         // occurrences per heavy-variable chunk (32 leaves)

// Shared memory of a light block: the partial sums of its leaf tasks
// (task_cap x stage_vw floats).  Every launch of the light kernel must use
// the task cap of the partition its blocks were built with.
inline size_t light_smem_bytes(int task_cap, int stage_vw) {
    return (size_t)task_cap * (size_t)stage_vw * sizeof(float);
}

// ------------------------------------------------------- fp32 arithmetic
// Fixed-order float arithmetic of the step.  Every operation is a single
// IEEE operation rounded to nearest; fused multiply-adds appear only where
// written as fmaf (the library is built with -fmad=false).

// e^y - 1 for 0 <= y <= 18: y = k ln2 + r (Cody-Waite split of ln2 with a
// 16-bit-exact high part), e^r - 1 = r + r^2 q(r), q the Taylor series of
// (e^r - 1 - r) / r^2 to degree 6 (terms 1/2! .. 1/8!), Horner with fmaf;
// e^y - 1 = 2^k (e^r - 1) + (2^k - 1).
__device__ __forceinline__ float expm1_fixed(float y) {
    const float kInvLn2 = 1.44269504088896341f;
    const float kLn2Hi = 0.693145751953125f;
    const float kLn2Lo = 1.428606820309417232e-06f;
    float kf = rintf(y * kInvLn2);
    float r = fmaf(-kf, kLn2Hi, y);
    r = fmaf(-kf, kLn2Lo, r);
    float q = 1.0f / 40320.0f;
    q = fmaf(q, r, 1.0f / 5040.0f);
    q = fmaf(q, r, 1.0f / 720.0f);
    q = fmaf(q, r, 1.0f / 120.0f);
    q = fmaf(q, r, 1.0f / 24.0f);
    q = fmaf(q, r, 1.0f / 6.0f);
    q = fmaf(q, r, 0.5f);
    float rr = r * r;
    float em = fmaf(rr, q, r);
    int k = (int)kf;
    if (k == 0) return em;
    float scale = __int_as_float((127 + k) << 23);
    return fmaf(scale, em, scale - 1.0f);
}

// tanh(a) = sign(a) * em1 / (em1 + 2), em1 = e^{2|a|} - 1; 1 for |a| >= 9.
// tanh(a) > 0 exactly when a > 0.
__device__ __forceinline__ float tanh_fixed(float a) {
    float s = fabsf(a);
    float r;
    if (!(s < 9.0f)) {
        r = (s != s) ? s : 1.0f;
    } else {
        float em1 = expm1_fixed(s + s);
        r = em1 / (em1 + 2.0f);
    }
    return copysignf(r, a);
}

// Leaf counter of the fixed summation order: 32-term leaves are summed in
// order by the caller; finished leaves are pushed here and merged into
// dyadic blocks (binary counter), and finish() combines what is left from
// the smallest (rightmost) block to the largest.  LEVELS bounds the leaf
// count to 2^LEVELS - 1.
template <int LEVELS>
struct LeafCounter {
    float blk[LEVELS];
    unsigned cnt;
    __device__ __forceinline__ void init() { cnt = 0; }
    __device__ __forceinline__ void push(float v) {
        bool carry = true;
#pragma unroll
        for (int p = 0; p < LEVELS; ++p) {
            if (carry) {
                if (cnt & (1u << p)) {
                    v = blk[p] + v;
                } else {
                    blk[p] = v;
                    carry = false;
                }
            }
        }
        ++cnt;
    }
    __device__ __forceinline__ float finish() const {
        float r = 0.0f;
        bool have = false;
#pragma unroll
        for (int p = 0; p < LEVELS; ++p) {
            if (cnt & (1u << p)) {
                r = have ? (blk[p] + r) : blk[p];
                have = true;
            }
        }
        return r;
    }
};

// ----------------------------------------------------------------- launchers
// Implemented in k_step.cu / k_eval.cu; each returns a cudaError_t.

cudaError_t launch_init(const DevInst &I, const DevState &S, uint64_t seed, cudaStream_t st);
int fwd_grid_blocks(const DevInst &I);
int auto_fwd_vw(int B);
int auto_stage_vw(int B);
int update_vw(int B);
enum { FWD_STEP = 0, FWD_EVAL = 1, FWD_PROBE = 2 };
cudaError_t launch_forward(const DevInst &I, const DevState &S, const DevStep &D, int mode,
                           const float *t_override, cudaStream_t st);
cudaError_t launch_backward(const DevInst &I, const DevState &S, const DevStep &D, int mode,
                            const float *t_override, const float *gscale, float *grad_out,
                            cudaStream_t st);
cudaError_t launch_tanh(const float *x, float *t, int64_t count, cudaStream_t st);
// Batched step over nslot instances (all with the same B and launch shape,
// f stored by the clause pass; variable-length clause path): fwd_start / heavy_start / light_start are device int[nslot+1]
// block prefixes; totals are the grid sizes.
cudaError_t launch_step_batch(const SlotDesc *slots, int nslot, const int *fwd_start, int fwd_total,
                              const int *heavy_start, int heavy_total, const int *light_start,
                              int light_total, int B, int fwd_vw, int stage_vw, int task_cap,
                              cudaStream_t st);
int heavy_blocks_of(const DevInst &I);
int light_blocks_of(const DevInst &I);
cudaError_t launch_loss_reduce(const DevStep &D, int B, cudaStream_t st);
// Small instances: every step in one single-CTA launch with the state in
// shared memory (same bits as the per-pass kernels).
constexpr int kSmallThreads = 1024;
constexpr int kSmallMaxB = 64;
constexpr size_t kSmallSmemMax = 200 * 1024;
size_t small_smem_bytes(const DevInst &I);
bool small_fits(const DevInst &I, int max_deg);
cudaError_t launch_small_steps(const DevInst &I, const DevState &S, const DevStep &D, int n_steps,
                               cudaStream_t st);
cudaError_t launch_eval_sparse(const DevInst &I, const int8_t *a, int nb, long long *cost,
                               cudaStream_t st);
cudaError_t launch_round_pm1(const float *x, int8_t *a, long long count, cudaStream_t st);
cudaError_t launch_heuristic_gap(const DevInst &I, const float *x, long long *heur_unsat,
                                 long long *disagree, cudaStream_t st);
int dense_tile_n(int nb);
int dense_rows(int nb);
size_t dense_smem_bytes(int ntile);
size_t smem_max_dense();
int dense_encode_a(DenseDev &d);
int dense_encode_b(DenseDev &d, int rows, int ntile);
cudaError_t launch_dense_fill(const DevInst &I, uint8_t *Wt, int n_pad, cudaStream_t st);
cudaError_t launch_dense_convert(const DenseDev &d, const int8_t *a, int n, int nb, long long *cost,
                                 cudaStream_t st);
cudaError_t launch_dense_convert_x(const DenseDev &d, const float *x, int n, int nb, long long *cost,
                                   cudaStream_t st);
DenseSched dense_plan(const DenseDev &d, int ntile, int *grid);
cudaError_t launch_dense_piece_targets(const DevInst &I, const DenseDev &d, const DenseSched &p, int grid,
                                       cudaStream_t st);
cudaError_t launch_dense_gemm(const DenseDev &d, int nb, long long *cost, cudaStream_t st);
cudaError_t launch_wait_selftest(long long spins, unsigned int *errflag, cudaStream_t st);
// k_mma_rate: `iters` stages of four MMAs of the evaluator's shape, N = n.
cudaError_t launch_mma_rate(int n, int iters, int grid, unsigned int *errflag, cudaStream_t st);

}  // namespace msat
