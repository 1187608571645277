/*
 * msat.h -- C ABI of the GB300 MaxSAT gradient engine.
 *
 * The engine runs the solving loop of torchmSAT (arXiv 2402.03640) on one
 * GPU.  The problem statement it serves is the paper's (Sec. 2, Eq. 1): a
 * CNF formula F = c_1 and ... and c_m over n Boolean variables; the answer is
 * an assignment that leaves as few clauses unsatisfied as possible (the
 * cost), optionally weighted (an extension the paper lists as future work in
 * Sec. 6).  Each optimizer step is (Sec. 4, Algorithm 1):
 *
 *   t = tanh(x)                         relaxed variables x in R^n
 *   f_j = sum over literals of c_j of (+t_i for x_i, -t_i for not x_i)
 *   x'_i = [x_i > 0];  clause j is unsat iff no literal is true under x'
 *   cost = sum of w_j over unsat clauses  (exact integer)
 *   best cost / best assignment kept (Alg. 1)
 *   L = sum_{unsat j} w_j f_j^2 / sum_{unsat j} w_j    (masked MSE)
 *   gradient by backpropagation, one Adam step (Sec. 5)
 *   a restart whose cost reaches 0 stops (Alg. 1 stop rule)
 *
 * B independent restarts run side by side ("restarts"); each has its own x,
 * Adam state, unsat set, loss and best assignment.
 *
 * Conventions for every call:
 *   - Return 0 on success or a negative MSAT_E* code; the message of the
 *     last failure on the calling thread is returned by msat_last_error().
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the GPU that was current when the context was made.
 *   - The caller owns every buffer it passes; the library copies what it
 *     keeps.  The context owns its device state and frees it in
 *     msat_destroy().
 *   - Work is issued on the context's stream.  Calls that return results to
 *     host buffers synchronise that stream; calls that only touch device
 *     buffers are asynchronous on it.
 *   - Floating-point arithmetic is IEEE fp32 with a fixed evaluation order
 *     (literal / occurrence order, 32-term leaves summed in order, leaves
 *     combined by the dyadic tree), so results are reproducible run to run.
 */
#ifndef MSAT_H
#define MSAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSAT_OK 0
#define MSAT_EINVAL (-1)   /* bad argument or malformed CNF                      */
#define MSAT_ENOMEM (-2)   /* host or device allocation failed                   */
#define MSAT_EBUDGET (-3)  /* request does not fit the server's memory budget    */
#define MSAT_ETIMEOUT (-4) /* a bounded device wait gave up                      */
#define MSAT_ECUDA (-5)    /* a CUDA runtime call failed                         */
#define MSAT_EAGAIN (-6)   /* result not ready yet (msat_poll)                   */
#define MSAT_ESTATE (-7)   /* call not valid in the object's current state       */

#define MSAT_BACKEND_SPARSE 0 /* clause CSR gather kernel                       */
#define MSAT_BACKEND_DENSE 1  /* tensor-core GEMM of the clause matrix          */

typedef struct msat_ctx msat_ctx;

/* Solver settings.  Fill with msat_config_default() and override. */
typedef struct {
    double lr;        /* Adam learning rate; the paper uses 1e-4 (Sec. 5)      */
    double beta1;     /* Adam first-moment decay (default 0.9)                 */
    double beta2;     /* Adam second-moment decay (default 0.999)              */
    double eps;       /* Adam epsilon (default 1e-8)                           */
    int32_t restarts; /* B: 1, 2, 4, ..., 1024 (a power of two)                */
    int32_t f_mode;   /* how the variable pass gets f_j of unsat clauses:
                         MSAT_F_AUTO (store unless m x B x 4 bytes > 8 GiB),
                         MSAT_F_STORE (the clause pass stores w_j f_j),
                         MSAT_F_RECOMPUTE (recomputed from the clause CSR),
                         MSAT_F_EXPANDED (3-literal clauses: recomputed from
                         occurrence records holding the other two literals) */
    uint64_t seed_x;  /* seed of the random start of x (Alg. 1)                 */
    int32_t heavy_deg; /* occurrences above which a variable's sum is split
                          into 1024-occurrence chunks (0 = automatic)          */
    /* Launch shapes (0 = automatic).  None of them changes a result bit: the
     * order of every sum is fixed by the instance, not by the launch.       */
    int32_t fwd_vw;     /* restarts per thread in the clause pass (1,2,4,8;
                           <= B and >= B/256)                                   */
    int32_t stage_vw;   /* restarts per thread staging occurrence terms
                           (1,2,4,8,16; <= B and >= B/256)                      */
    int32_t fwd_blocks; /* thread blocks of the clause pass                    */
    int32_t light_rows; /* leaf tasks of one light-variable block, a task
                           being one 32-occurrence leaf of a variable for
                           stage_vw restarts (>= 16; light_rows x stage_vw x 4
                           bytes <= 48 KiB; 0 = 256)                            */
    int32_t loss_norm;  /* MSAT_LOSS_MEAN_UNSAT (default), MSAT_LOSS_SUM_UNSAT
                           or MSAT_LOSS_MEAN_ALL; see below                    */
    int32_t row_order;  /* rows of the stored w_j f_j: 0 = automatic (grouped
                           by the variable pass's blocks when the store
                           exceeds 32 MiB, else clause order), 1 = clause
                           order, 2 = grouped by block.  x, costs and best
                           are the same bits either way (the loss is summed
                           in row order, within 1e-5); grouping puts about
                           a third of a block's gathers in one window      */
} msat_config;

/* Normaliser N of the loss L = sum_{j in U} w_j f_j^2 / N and of its
 * gradient (g_j = 2 w_j f_j / N).  Sec. 4 takes the MSE of f against zero
 * over the unsatisfied clauses: N = sum_{j in U} w_j (MEAN_UNSAT, the
 * default).  SUM_UNSAT (N = 1) and MEAN_ALL (N = sum of all weights) are the
 * two other readings, kept for the ablation; Adam is nearly invariant to a
 * per-step scale, so they differ mainly through epsilon. */
#define MSAT_LOSS_MEAN_UNSAT 0
#define MSAT_LOSS_SUM_UNSAT 1
#define MSAT_LOSS_MEAN_ALL 2

#define MSAT_F_AUTO 0
#define MSAT_F_STORE 1
#define MSAT_F_RECOMPUTE 2
#define MSAT_F_EXPANDED 3

/* Write the defaults (lr 1e-4, Adam 0.9/0.999/1e-8, B = 1, seed 1, automatic
 * f mode and heavy threshold).  Every mode gives bit-identical results. */
int msat_config_default(msat_config *cfg);

/*
 * Build a solver context for one CNF (Alg. 1: the clause matrix is built once).
 *   n_vars      n >= 1 (variables are numbered 1..n in lits)
 *   n_clauses   m >= 0
 *   clause_off  host int64[m+1], clause j holds lits[clause_off[j] ..
 *               clause_off[j+1]); clause_off[0] = 0, non-decreasing
 *   lits        host int32[clause_off[m]], DIMACS literals: +(i+1) for x_i,
 *               -(i+1) for not x_i; 0 and |l| > n are rejected
 *   weights     host int64[m] clause weights >= 1, or NULL for all 1
 *   cfg         settings (NULL = defaults)
 *   stream      cudaStream_t to issue work on (NULL = the legacy default
 *               stream)
 * A literal repeated inside a clause is dropped (W has one entry per
 * variable and clause); a clause holding x and not x is kept and is never
 * unsatisfied; an empty clause is always unsatisfied.  Clauses longer than
 * 32767 literals, nnz >= 2^31 and m or n >= 2^30 are rejected (MSAT_EINVAL).
 * x is initialised on the device: x[i][b] = k * 2^-23 - 1 with k the top 24
 * bits of output number b*n + i of the SplitMix64 stream seeded with
 * seed_x; Adam moments are zero; the best cost starts at sum_j w_j.
 */
int msat_create(msat_ctx **out, int32_t n_vars, int64_t n_clauses, const int64_t *clause_off,
                const int32_t *lits, const int64_t *weights, const msat_config *cfg,
                void *stream);

/* Free every resource of the context (NULL is ignored). */
void msat_destroy(msat_ctx *ctx);

/* Issue later work of this context on another cudaStream_t. */
int msat_set_stream(msat_ctx *ctx, void *stream);

/*
 * Run n_steps iterations of Algorithm 1 (evaluate x, keep the best, masked
 * MSE loss, gradient, one Adam step) and then one evaluation of the final x.
 *   loss_out   host float[B]: loss at the last updated x, or NULL
 *   cost_out   host int64[B]: cost of the final x, or NULL
 * With both outputs NULL the call is asynchronous on the context stream.
 * n_steps = 0 only evaluates the current x.
 */
int msat_step(msat_ctx *ctx, int32_t n_steps, float *loss_out, int64_t *cost_out);

/*
 * msat_step with flags.  MSAT_STEP_NO_FINAL_EVAL skips the evaluation of
 * the final x; cost_out then holds the cost of the last x evaluated inside
 * the loop (the x before the last update) and loss_out its loss.  With
 * n_steps = 0 and this flag nothing runs.  MSAT_STEP_GRAPH replays the
 * steps from CUDA graphs of one and of 32 steps, captured on the first such
 * call (on a private stream, so the context stream may be the default
 * stream); the results are bit for bit those of the plain launches.  It is
 * ignored while kernel timing (msat_profile_enable) is on.  A graph holds
 * the context's device pointers; it is released with the context.
 * Small instances (B <= 64, 4 n B + m B floats within 200 KiB of shared
 * memory, no variable with more than 32736 occurrences) run all their steps
 * in one single-CTA launch holding the state in shared memory, again with
 * the same bits; MSAT_STEP_PER_PASS keeps them on the per-pass kernels (for
 * comparison), as does kernel timing.
 */
#define MSAT_STEP_NO_FINAL_EVAL 1u
#define MSAT_STEP_GRAPH 2u
#define MSAT_STEP_PER_PASS 4u
int msat_step_ex(msat_ctx *ctx, int32_t n_steps, uint32_t flags, float *loss_out,
                 int64_t *cost_out);

/*
 * Time-limited solving (Sec. 4: Algorithm 1 takes a wall-clock limit T as
 * input and ends at zero cost or when T is reached).  Runs the steps in chunks of `chunk` steps (CUDA-graph replays
 * unless kernel timing is on) until some restart's best cost is 0,
 * max_steps steps have run, or time_limit_s seconds have passed (checked
 * after each chunk, so a chunk in flight completes); then evaluates the
 * final x once, exactly as msat_step does.  The result after k steps is bit
 * for bit that of msat_step(ctx, k, ...); read it with msat_best.
 *   steps_out, elapsed_out    steps taken and seconds spent (nullable)
 *   trace_cost, trace_time    host buffers of trace_cap entries (nullable
 *                             when trace_cap is 0): after each chunk, and
 *                             after the final evaluation, the best cost over
 *                             all restarts and the seconds since the call began
 *   trace_len                 entries written (nullable)
 * Synchronous.  EINVAL on a NULL ctx, max_steps < 0, chunk < 1, a negative
 * time limit or missing trace buffers; ECUDA on a CUDA failure.
 */
int msat_solve(msat_ctx *ctx, int64_t max_steps, double time_limit_s, int32_t chunk,
               int64_t *steps_out, double *elapsed_out, int64_t *trace_cost, double *trace_time,
               int32_t trace_cap, int32_t *trace_len);

/*
 * Launch-shape autotuner (no counterpart in the paper: it tunes this
 * library's kernels).  The launch shapes -- fwd_vw, stage_vw and light_rows
 * of msat_config -- never change a result bit, so the tuner only times: for
 * each candidate it creates a scratch context for the instance on `stream`
 * (same arguments as msat_create), runs 2 warm-up steps and times n_steps
 * steps with CUDA events, one parameter at a time (stage_vw, then
 * light_rows, then fwd_vw), starting from the automatic shape.  cfg_out
 * receives cfg_in (NULL: defaults) with the fastest shape filled in; pass it
 * to msat_create.  entries (nullable, cap entries) and n_entries report the
 * candidates timed.  The winner is cached for the process per instance
 * shape (device, n, m, nnz, restarts, f_mode, weighted, heavy_deg); a cached
 * call times nothing and reports no entries.  Synchronous; needs memory for
 * one more context of the instance.  Errors: as msat_create (EINVAL for a
 * malformed instance or config, ENOMEM), ECUDA on a device failure.
 */
typedef struct {
    int32_t fwd_vw, stage_vw, light_rows;
    float ms_per_step;
} msat_tune_entry;
int msat_autotune(int32_t n_vars, int64_t n_clauses, const int64_t *clause_off,
                  const int32_t *lits, const int64_t *weights, const msat_config *cfg_in,
                  void *stream, int32_t n_steps, msat_config *cfg_out, msat_tune_entry *entries,
                  int32_t cap, int32_t *n_entries);

/*
 * Exact cost of a batch of assignments (Sec. 4, "Unsatisfiable Cores": a
 * clause is unsatisfied iff x'.W equals -len with x' read as +-1).
 *   assign_pm1  device int8[n][nb], entry (i, b) at i*nb + b: +1 = true,
 *               -1 = false (any value > 0 counts as true)
 *   nb          number of assignments, >= 1
 *   cost_out    device int64[nb]: sum of w_j over clauses with no true literal
 *   backend     MSAT_BACKEND_SPARSE or MSAT_BACKEND_DENSE
 * Asynchronous on the context stream; the result is exact for both
 * backends.  The dense backend multiplies the clause matrix W^T (e2m1,
 * m x n, packed two codes a byte, built on its first use: m_pad * n_pad / 2
 * bytes, rejected above 64 GiB) by the batch on the tensor cores; it needs
 * weights below 2^25.
 */
int msat_evaluate(msat_ctx *ctx, const int8_t *assign_pm1, int32_t nb, int64_t *cost_out,
                  int32_t backend);

/*
 * Exact cost of the context's current x, rounded (x' = [x > 0], Sec. 4) to a
 * +-1 batch of B assignments by a kernel, with either backend.
 *   cost_out   device int64[B]
 * Asynchronous on the context stream.
 */
int msat_evaluate_x(msat_ctx *ctx, int32_t backend, int64_t *cost_out);

/*
 * Wait for the context's stream and report a device-side failure that the
 * asynchronous calls could not return: MSAT_ETIMEOUT when a bounded wait in
 * a kernel (the dense backend's pipeline barriers) gave up; the flag is
 * cleared.  0 otherwise.
 */
int msat_check(msat_ctx *ctx);

/*
 * Failure-detection self-test (no counterpart in the paper).  Every device
 * wait of this library (the mbarrier phases of the tensor-core evaluator)
 * gives up after 200 ms of the GPU's global timer (a phase normally
 * completes within microseconds), records the reason in an error flag and
 * returns, so a phase that never completes is reported by msat_check as
 * MSAT_ETIMEOUT instead of hanging the GPU.  This call runs that path on
 * purpose: one thread waits on a barrier nothing arrives at, for `spins`
 * tries (1 .. 2^24) or, with spins = 0, until the 200 ms limit.  Returns
 * MSAT_ETIMEOUT (the expected result) with the flag in the message; the
 * device stays usable.  Synchronous; allocates and frees one 4-byte flag.
 */
int msat_selftest_bounded_wait(int64_t spins);

/*
 * Measured peak of the dense backend's tensor-core instruction (no
 * counterpart in the paper; a benchmark helper): every SM issues `iters`
 * stages of four block-scaled kind::mxf4 MMAs (M = 128 clauses, N =
 * n_assign assignments, K = 64 e2m1 codes, unit scale factors) on operands
 * resident in shared memory, and the second of two launches is timed with
 * CUDA events on the current device.  The dense evaluator runs the same
 * instructions behind its TMA pipeline, so this rate bounds it.
 *   n_assign   multiple of 16 in [16, 256]
 *   iters      stages per SM, in [1, 2^20]
 *   tflops     host double: 2 * 128 * n_assign * 64 * 4 * iters * SMs
 *              divided by the launch time, in TFLOP/s
 * Synchronous; allocates and frees one 4-byte flag.  EINVAL on bad
 * arguments, ETIMEOUT if the bounded wait for the MMAs gave up.
 */
int msat_dense_mma_rate(int32_t n_assign, int32_t iters, double *tflops);

/*
 * The paper's quick evaluation reads clause j as satisfied when f_j > 0
 * (Sec. 4, "Example": a positive clause value marks a satisfied clause);
 * the exact test is "some literal is true under x > 0" (Sec. 4,
 * "Unsatisfiable Cores").  For the current x this counts, per restart,
 * the clauses the quick reading calls unsatisfied (f_j <= 0) and the
 * clauses on which the two readings disagree, with f_j in the step's fixed
 * summation order.  Diagnostic for the readings ablation.
 *   heur_unsat, disagree   host int64[B]
 * Synchronous; EINVAL on NULL arguments, ECUDA on a CUDA failure.
 */
int msat_heuristic_gap(msat_ctx *ctx, int64_t *heur_unsat, int64_t *disagree);

/*
 * Best assignment and cost seen so far per restart (Alg. 1, best kept).
 *   assign01   host uint8[B][n] (0/1), or NULL
 *   best_cost  host int64[B], or NULL
 */
int msat_best(msat_ctx *ctx, uint8_t *assign01, int64_t *best_cost);

/*
 * Steps to best (Alg. 1 keeps the best assignment; this reports when
 * it was found): for each restart, the number of optimizer steps taken before
 * the x whose cost is the best cost (0: the random start x_0), an index of
 * the cost-vs-step history.  Not part of a checkpoint: reads 0 after
 * msat_set_state.  best_step host int64[B]; synchronous.
 */
int msat_best_step(msat_ctx *ctx, int64_t *best_step);

/* Copy the current relaxed variables to host float[n][B] (entry i*B + b). */
int msat_get_x(msat_ctx *ctx, float *x_host);

/*
 * Relaxed objective and its gradient at a caller-supplied x, without an
 * optimizer step (the differentiable layer of Sec. 4).
 *   x        device float[n][B]
 *   loss     device float[B]   (masked MSE per restart)
 *   cost     device int64[B] or NULL (exact cost of x' = [x > 0])
 * msat_forward keeps tanh(x), the unsat mask and 2/sum_U w in the context;
 * msat_backward then writes
 *   grad     device float[n][B] = dloss/dx, scaled per restart by
 *   gscale   device float[B] (NULL = all ones),
 * for the x of the most recent msat_forward on this context.  The mask is
 * piecewise constant and is not differentiated.  These calls do not touch
 * the context's own x, Adam state or best assignment.
 */
int msat_forward(msat_ctx *ctx, const float *x, float *loss, int64_t *cost);
int msat_backward(msat_ctx *ctx, const float *gscale, float *grad);

/* Sizes and counters of a context. */
typedef struct {
    int32_t n;            /* variables                                         */
    int32_t restarts;     /* B                                                 */
    int64_t m;            /* clauses                                           */
    int64_t nnz;          /* literals after dropping repeats                   */
    int64_t steps_done;   /* optimizer steps taken                             */
    int64_t device_bytes; /* device memory held by the context                 */
    int32_t max_clause_len;
    int32_t max_degree;   /* most occurrences of one variable                  */
    int32_t n_heavy;      /* variables whose occurrence sum is split across warps */
    int32_t uniform_len;  /* common clause length, or 0 if lengths differ      */
    int32_t small_kernel; /* 1: msat_step runs the single-CTA kernel (all steps
                             of a call in one launch, state in shared memory) */
} msat_info;

int msat_get_info(msat_ctx *ctx, msat_info *info);

/*
 * Checkpoint: the full solver state as plain host arrays, so a resumed run
 * continues bit for bit.
 *   x, mom, vel   host float[n][B]
 *   best_cost     host int64[B]
 *   best_assign   host uint8[n][B] (0/1, entry i*B + b)
 *   steps_done    host int64[1]
 *   adam_pow      host double[2]: beta1^steps_done, beta2^steps_done as the
 *                 running products the step kernels use
 * msat_get_state fills them; msat_set_state loads them (any may be NULL in
 * get; all are required in set).
 */
int msat_get_state(msat_ctx *ctx, float *x, float *mom, float *vel, int64_t *best_cost,
                   uint8_t *best_assign, int64_t *steps_done, double *adam_pow);
int msat_set_state(msat_ctx *ctx, const float *x, const float *mom, const float *vel,
                   const int64_t *best_cost, const uint8_t *best_assign, int64_t steps_done,
                   const double *adam_pow);

/*
 * Kernel timing for benchmarks.  While enabled, every kernel the context
 * launches is bracketed by CUDA events recorded on the context stream;
 * msat_profile_read waits for the last event and returns, per kernel kind,
 * the number of launches and their summed duration in milliseconds.
 * Kinds: 0 forward clause pass, 1 backward variable pass (with Adam),
 * 2 evaluation, 3 other (init, tanh, reductions).
 */
typedef struct {
    int64_t launches[4];
    double ms[4];
} msat_profile;

int msat_profile_enable(msat_ctx *ctx, int on);
int msat_profile_read(msat_ctx *ctx, msat_profile *out, int reset);

/*
 * The relaxed objective and exact cost of a caller-supplied x without a
 * context and without allocating device memory.  (This entry point has no
 * counterpart in the paper; it serves callers that may not allocate: hosts
 * that give the library a fixed memory budget, latency-bound loops where
 * cudaMalloc's device synchronisation is not allowed, plugins running where
 * allocation calls are forbidden.)
 *   n_vars, n_clauses   n >= 1, m >= 0
 *   clause_off          device int64[m+1] clause offsets into lits
 *   lits                device int32 DIMACS literals; a literal must not be
 *                       repeated inside its clause (no canonicalisation is
 *                       done here); 0 or |l| > n is skipped
 *   weights             device int64[m] (>= 1) or NULL for all 1
 *   x                   device float[n][B] relaxed variables (entry i*B + b)
 *   restarts            B, a power of two in [1, 1024]
 *   cost_out            device int64[B]: sum of w_j over clauses with no true
 *                       literal under x' = [x > 0]
 *   loss_out            device float[B]: sum_U w f^2 / sum_U w (0 if U empty);
 *                       its sums run in another order than msat_forward's,
 *                       with which it agrees within 1e-5 relative
 *   stream              cudaStream_t (NULL = legacy default stream)
 * Scratch: a 4 MiB array inside the library (held by every GPU that loads
 * it until the process exits); every size in the range above fits, and a
 * size that would not is rejected with MSAT_EINVAL.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * Calls share the array: calls whose kernels overlap on the GPU race and
 * give wrong results.  Asynchronous on the stream; allocates nothing.
 */
int msat_objective_noalloc(int32_t n_vars, int64_t n_clauses, const int64_t *clause_off,
                           const int32_t *lits, const int64_t *weights, const float *x,
                           int32_t restarts, int64_t *cost_out, float *loss_out, void *stream);

/*
 * Serving: a request loop that runs many instances at once (continuous
 * batching).  Requests arrive with msat_submit at any time; a scheduler
 * thread admits them, oldest first, while their device memory fits the
 * budget, a slot is free and the batch's step work stays under its cap; a
 * pool of host threads builds the admitted instances' contexts in parallel.
 * The server keeps every admitted instance's clause arrays and optimizer
 * state resident and advances all of them together: each
 * iteration of Algorithm 1 for the whole slot table is one captured CUDA
 * graph (three batched kernels), replayed chunk by chunk.  An instance that
 * has taken its steps gets one final evaluation; its result is copied out
 * and its memory returned, and queued requests take the freed room.  Each
 * instance's arithmetic is independent of the others, so a result is bit
 * for bit the one msat_create/msat_step(steps)/msat_best gives alone.
 * (Serving is not part of the paper; the per-instance work is Alg. 1.)
 */
typedef struct msat_server msat_server;

typedef struct {
    size_t hbm_budget;  /* device bytes the resident instances may hold
                           (0 = half of the free memory at creation)      */
    int32_t max_slots;  /* instances stepped together (0 = 256)           */
    int32_t restarts;   /* B of every instance (power of two, <= 1024)    */
    int32_t chunk;      /* steps per scheduling round (0 = 50)            */
    int32_t batch_mlits; /* cap on the work of one step of the batch, in
                            millions of literal evaluations (nnz x restarts
                            summed over the instances stepped together and
                            those being admitted); a request waits while it
                            would pass the cap, unless nothing else runs.
                            Past the point where the batch fills the GPU,
                            more instances only slow every one of them
                            (0 = 128, < 0 = no cap)                       */
    double lr, beta1, beta2, eps; /* Adam settings of every instance      */
} msat_server_config;

typedef struct {
    int32_t n_vars;           /* n >= 1                                   */
    int32_t steps;            /* optimizer steps to run (>= 0)            */
    int64_t n_clauses;        /* m >= 0                                   */
    const int64_t *clause_off; /* host int64[m+1]  (copied at submit)     */
    const int32_t *lits;      /* host DIMACS int32 (copied at submit)     */
    const int64_t *weights;   /* host int64[m] or NULL (copied at submit) */
    uint64_t seed_x;          /* seed of the random start                 */
} msat_request;

typedef struct {
    int32_t status;       /* 0 done; MSAT_EAGAIN queued or running; < 0 the
                             request failed with that code               */
    int32_t best_restart; /* restart holding best_cost                   */
    int64_t best_cost;    /* lowest cost over restarts and steps         */
    int64_t steps;        /* optimizer steps taken                       */
    int32_t n_vars;
    int32_t restarts;
    double queue_ms;      /* submit -> admitted and its context built    */
    double latency_ms;    /* submit -> result ready                      */
    int64_t best_step;    /* steps taken before the best restart's best x
                             (steps to best; 0 = the random start)        */
} msat_result;

typedef struct {
    int64_t submitted, completed, failed, cancelled;
    int32_t queued, running, peak_running;
    int32_t small_direct;  /* requests small enough for the single-CTA kernel: they
                              take all their steps in one launch on a side stream
                              as soon as they are admitted, outside the slot table */
    int64_t hbm_in_use, hbm_budget, rounds, graph_captures;
} msat_server_stats;

int msat_server_config_default(msat_server_config *cfg);
int msat_server_create(msat_server **out, const msat_server_config *cfg);
/* Stop accepting requests, finish everything admitted or queued, free all. */
void msat_server_destroy(msat_server *srv);

/* Queue a request (its arrays are copied).  A request that cannot fit the
 * budget even alone, or a malformed one, fails here (MSAT_EBUDGET /
 * MSAT_EINVAL) without a ticket. */
int msat_submit(msat_server *srv, const msat_request *req, uint64_t *ticket);

/* Non-blocking result query.  Returns 0 and fills out (and, when non-NULL,
 * best_costs int64[B] per restart and assign01 uint8[n] of the best
 * restart) once the request is done, after which the ticket is forgotten;
 * MSAT_EAGAIN while it is queued or running; the request's error code if it
 * failed; MSAT_EINVAL for an unknown ticket. */
int msat_poll(msat_server *srv, uint64_t ticket, msat_result *out, int64_t *best_costs,
              uint8_t *assign01);
/* msat_poll that waits up to timeout_s seconds (MSAT_ETIMEOUT after). */
int msat_wait(msat_server *srv, uint64_t ticket, double timeout_s, msat_result *out,
              int64_t *best_costs, uint8_t *assign01);
/* Withdraw a request that is still queued (MSAT_ESTATE once admitted). */
int msat_cancel(msat_server *srv, uint64_t ticket);
int msat_server_get_stats(msat_server *srv, msat_server_stats *out);

/* Message of the last failed call on this thread ("" if none). */
const char *msat_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MSAT_H */
