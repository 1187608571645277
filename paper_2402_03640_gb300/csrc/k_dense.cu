// Dense evaluation of a batch of +-1 assignments on the 5th-generation
// tensor cores (sm_103a): S = W^T X, with W^T the m x n clause matrix
// (W_ij = +1 for x_i in c_j, -1 for not x_i, 0 otherwise; Sec. 4) and X the
// n x nb batch of assignments read as +-1.  Clause j is unsatisfied by
// assignment b iff S_jb = -len_j (the paper's unsat test, Sec. 4
// "Unsatisfiable Cores", with x' read as +-1), and cost_b = sum_j w_j
// [S_jb = -len_j].
//
// tcgen05.mma .kind::i8 is not available on sm_103a, so both operands are
// e2m1 (0, +1, -1 are exact) with fp32 accumulation, which is exact here:
// every partial sum is an integer of magnitude <= n < 2^24.  The MMA kind
// is the block-scaled .kind::mxf4 with every scale factor 1 (ue8m0 code
// 127 = 2^0), so D = A B exactly.  It reads the operands packed, two 4-bit
// codes a byte, the form they have in global memory: HBM, L2, the TMA
// copies and shared memory all carry half a byte per element.  A and B
// pack variable i the same way (low nibble for even i), so the pairing of
// nibbles with k inside the MMA cannot change a dot product.
//
// Tile: 128 clauses x N assignments (N <= 256, a multiple of 16), K = 256
// variables per stage (128 bytes a row).  Warp 0 (one lane) loads A and B
// tiles with TMA into a 4-stage ring of 128B-swizzled shared-memory
// buffers, starting as soon as the barriers exist; warp 1 (one lane)
// issues tcgen05.mma into a TMEM accumulator and releases each stage with
// tcgen05.commit; warps 2-9 write the scale factors into TMEM once, then
// read the accumulator with tcgen05.ld (two warps per TMEM lane quarter,
// alternate 32-column chunks), turn it into hit bits (S_jb = -len_j),
// release it, and count the unsat clauses per column.  With N <= 128 there
// are two accumulators and the next segment accumulates into the other
// one meanwhile; above, the 512 TMEM columns hold one 256-column
// accumulator and the scale factors, and the next segment waits only for
// the bits to be read out.
//
// Schedule: with more tiles than SMs, every CTA of a one-per-SM grid takes
// the same number of whole tiles back to back; leftover tiles that would
// fill at most half a wave are split, each into `split` equal k-step pieces
// on as many CTAs (which take their piece first), and a larger leftover
// runs as one more whole tile on the first CTAs.  Every term of S_jb is -1,
// 0 or +1, so S_jb =
// -len_j exactly when, in every piece, the piece's partial sum equals minus
// the number of the clause's literals whose variable lies in the piece's
// k-range.  A piece therefore tests its own partial sums against those
// per-piece targets, stores one bit per (clause, assignment) and counts
// itself in; the last piece of a tile to arrive ANDs the other pieces' bits
// into its own and counts the unsat clauses.  No CTA waits on another.
//
// Every mbarrier wait gives up after kWaitNs nanoseconds of %globaltimer
// (200 ms; a phase normally completes within microseconds).  On a timeout
// the block records an error flag and stops issuing work; the MMA issuer
// then waits (bounded) until the MMAs it has issued have completed, the
// producer until the copies it has issued have landed, and only then does
// the block free its TMEM.

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "msat_internal.cuh"

namespace msat {

namespace {

constexpr int kTM = 128;            // clauses per tile (MMA M)
constexpr int kTK = kDenseKStep;    // variables per stage (256: 128 bytes a row in shared memory)
constexpr int kRowBytes = kTK / 2;  // packed bytes of a row per stage
constexpr int kSfCols = 32;         // TMEM columns of scale factors (A: first 16, B: last 16)
constexpr uint32_t kSfOne = 0x7F7F7F7Fu;  // four ue8m0 scale factors of 2^0
constexpr int kStages = 4;
constexpr int kAccBufs = 2;         // TMEM accumulators at most (segment j uses j % bufs)
constexpr int kPrefetch = 1;        // clause-matrix k-tiles prefetched into L2 ahead of their loads
constexpr int kDenseThreads = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue (two per lane quarter)
constexpr int kEpiWarps = 8;
constexpr int kHeader = 4096;       // barriers, TMEM address, column sums
constexpr unsigned long long kWaitNs = 200ull * 1000ull * 1000ull;  // 200 ms
// e2m1 codes (sign, 2 exponent bits with bias 1, 1 mantissa bit)
constexpr uint8_t kE2M1One = 0x2, kE2M1MinusOne = 0xA;

struct DenseHeader {
    unsigned long long full[kStages];
    unsigned long long empty[kStages];
    unsigned long long acc_full[kAccBufs];
    unsigned long long acc_empty[kAccBufs];
    uint32_t tmem;
    int abort;
    int epi_fail;  // written only by the epilogue warps, read after their barrier
    int last;      // this CTA finishes the split tile
    unsigned long long drain;  // the MMA issuer's last MMAs completed (abort path)
    unsigned long long colsum[256];
};
static_assert(sizeof(DenseHeader) <= kHeader, "dense header does not fit");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on a barrier phase: false once max_ns nanoseconds of the
// global timer have passed (or after max_tries tries, when max_tries > 0).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, long long max_tries,
                                          unsigned long long max_ns) {
    const unsigned long long t0 = global_ns();
    for (long long i = 0; max_tries <= 0 || i < max_tries; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && global_ns() - t0 > max_ns) return false;
    }
    return false;
}

// The same with the kernel's time limit, giving up early once another
// role of the block has aborted.
__device__ __forceinline__ bool mbar_wait_abort(unsigned long long *bar, uint32_t parity, const int *abort) {
    const unsigned long long t0 = global_ns();
    for (long long i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && (*(volatile const int *)abort || global_ns() - t0 > kWaitNs)) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Programmatic dependent launch: the evaluator is launched to overlap the
// kernel that packs its assignment operand; it waits for that kernel (and
// the visibility of its writes) before its first read of the packed batch
// or write of the costs.  The packing kernels let it start at once.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Named barrier of the eight epilogue warps (256 threads).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Named barrier of the MMA and epilogue warps (warps 1-9, 288 threads).
__device__ __forceinline__ void roles_sync() { asm volatile("bar.sync 2, 288;" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// L2 prefetch of one tile of a tensor map (no shared memory, no barrier):
// the clause-matrix tiles are streamed from HBM once, so fetching them into
// L2 ahead of their TMA loads turns each load's latency into an L2 hit.
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes, 8-row groups 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(16 >> 4) << 16;    // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= 1ull << 46;                   // descriptor version
    d |= 2ull << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor of the block-scaled kind::mxf4: A and B e2m1
// (format 1), both K-major, scale factors ue8m0 (bit 23), scale-factor
// byte 0 of A and of B, M = 128, N = n, dense K = 64 per MMA.
__device__ __forceinline__ uint32_t idesc_mxf4(int n) {
    return (1u << 7) | (1u << 10)         // A, B format e2m1
           | ((uint32_t)(n >> 3) << 17)   // N / 8
           | (1u << 23)                   // scale factors ue8m0
           | ((uint32_t)(kTM >> 4) << 24);  // M / 16
}

// D (+)= (A x SFA) (B x SFB), K = 64 codes (32 bytes of each row).
__device__ __forceinline__ void mma_mxf4(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t tmem_sfa, uint32_t tmem_sfb, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%5], [%6], p;\n\t}" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(tmem_sfa), "r"(tmem_sfb)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
          "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
          "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Issues a load of 32 consecutive columns of the warp's 32 TMEM lanes;
// the registers hold the data only after tmem_wait2 below.
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

// Waits for the warp's outstanding TMEM loads; a and b are tied to the
// wait so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_wait2(uint32_t (&a)[32], uint32_t (&b)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]), "+r"(a[16]), "+r"(a[17]), "+r"(a[18]), "+r"(a[19]), "+r"(a[20]), "+r"(a[21]), "+r"(a[22]), "+r"(a[23]), "+r"(a[24]), "+r"(a[25]), "+r"(a[26]), "+r"(a[27]), "+r"(a[28]), "+r"(a[29]), "+r"(a[30]), "+r"(a[31]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]), "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15]), "+r"(b[16]), "+r"(b[17]), "+r"(b[18]), "+r"(b[19]), "+r"(b[20]), "+r"(b[21]), "+r"(b[22]), "+r"(b[23]), "+r"(b[24]), "+r"(b[25]), "+r"(b[26]), "+r"(b[27]), "+r"(b[28]), "+r"(b[29]), "+r"(b[30]), "+r"(b[31])
                 :
                 : "memory");
}

// Writes v into 32 consecutive columns of the warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_fill32(uint32_t taddr, uint32_t v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
        "r"(v)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Column sums of a 32 x 32 block held one row per lane (x[c] of lane r is
// entry (r, c)): five butterfly rounds, each lane trading half of its
// remaining columns with lane ^ k and adding the other half's partners;
// afterwards lane l holds the sum of column l.  Integer adds, so exact;
// the caller keeps every column sum below 2^32 (32 weights below 2^25).
__device__ __forceinline__ uint32_t column_sums32(uint32_t (&x)[32], int lane) {
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) {
        const bool up = (lane & k) != 0;
#pragma unroll
        for (int i = 0; i < k; ++i) {
            const uint32_t send = up ? x[i] : x[i + k];
            const uint32_t keep = up ? x[i + k] : x[i];
            x[i] = keep + __shfl_xor_sync(0xffffffffu, send, k);
        }
    }
    return x[0];
}

// Transpose of a 32 x 32 bit matrix held one row per lane (bit c of lane
// r's word is entry (r, c)): five butterfly rounds, each exchanging with
// lane ^ j the half of the bits whose position has bit j set; afterwards
// bit r of lane l's word is entry (r, l).
__device__ __forceinline__ uint32_t transpose_bits32(uint32_t x, int lane) {
    uint32_t m = 0x0000FFFFu;
#pragma unroll
    for (int j = 16; j >= 1; j >>= 1, m ^= m << j) {
        const uint32_t t = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? (((t >> j) & m) | (x & ~m)) : ((x & m) | ((t & m) << j));
    }
    return x;
}

// One segment of a CTA's work: k-steps [ka, kb) of tile `tile`; tr is the
// split-tile index (-1 for a whole tile) and piece the part of it.
struct DenseSeg {
    int tile, ka, kb, tr, piece;
};

__device__ __forceinline__ int seg_count(const DenseSched &d, int c) {
    return d.full + (c < d.tail_ctas || c < d.extra ? 1 : 0);
}

// A CTA with a piece of a split tile takes the piece first: the piece's
// bookkeeping (bits stored, counted in, the last piece's combine) then
// overlaps the CTA's whole tiles instead of ending the launch.
__device__ __forceinline__ DenseSeg seg_at(const DenseSched &d, int c, int j) {
    DenseSeg g;
    const bool piece_first = c < d.tail_ctas;
    if (!piece_first || j > 0) {
        if (piece_first) --j;
        g.tile = j * (int)gridDim.x + c;
        g.ka = 0;
        g.kb = d.kt_count;
        g.tr = -1;
        g.piece = 0;
        return g;
    }
    g.tr = c / d.split;
    g.piece = c % d.split;
    g.tile = d.full * (int)gridDim.x + g.tr;
    g.ka = (int)((long long)g.piece * d.kt_count / d.split);
    g.kb = (int)((long long)(g.piece + 1) * d.kt_count / d.split);
    return g;
}

__global__ void __launch_bounds__(kDenseThreads, 1)
    k_dense_eval(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const float *__restrict__ target, const uint32_t *__restrict__ wgt, int unit_w, DenseSched d,
                 int tmem_cols, int nb, unsigned long long *__restrict__ cost, const float *__restrict__ ptgt,
                 uint32_t *__restrict__ pmask, unsigned int *__restrict__ part_cnt,
                 unsigned int *__restrict__ errflag) {
    extern __shared__ uint8_t dsm_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~(uintptr_t)1023);
    DenseHeader *H = reinterpret_cast<DenseHeader *>(base);
    uint8_t *stages = base + kHeader;
    const int ntile = d.ntile;
    const uint32_t a_bytes = kTM * kRowBytes;
    const uint32_t b_bytes = (uint32_t)ntile * kRowBytes;
    // accumulators of tmem_cols columns each, then the scale factors
    const int nbuf = 2 * tmem_cols + kSfCols <= 512 ? kAccBufs : 1;
    const int sf_col = nbuf * tmem_cols;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cta = blockIdx.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&H->full[s], 1);
            mbar_init(&H->empty[s], 1);
        }
        for (int b = 0; b < nbuf; ++b) {
            mbar_init(&H->acc_full[b], 1);
            mbar_init(&H->acc_empty[b], kEpiWarps);  // one arrive per epilogue warp
        }
        mbar_init(&H->drain, 1);
        H->abort = 0;
        H->epi_fail = 0;
        H->last = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int c = threadIdx.x; c < 256; c += blockDim.x) H->colsum[c] = 0ull;
    __syncthreads();  // barriers initialised: the producer may start
    const int nseg = seg_count(d, cta);
    uint32_t tmem = 0;
    if (warp >= 1) {
        // while the first loads are in flight: warps 1-5 allocate TMEM
        // (all 512 columns, one CTA per SM) and write the scale factors,
        // 2^0 in every byte of the scale-factor columns, before the first
        // MMA is issued
        if (warp == 1) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&H->tmem)),
                         "r"(512)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        tc_fence_before();
        roles_sync();
        tc_fence_after();
        tmem = H->tmem;
        if (warp >= 2 && warp < 6) tmem_fill32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)sf_col, kSfOne);
        tc_fence_before();
        roles_sync();
        tc_fence_after();
    }

    if (warp == 0 && lane == 0) {
        // producer: TMA loads of the A (clause rows) and B (assignment rows)
        // tiles of every segment in turn; the A tiles are prefetched into L2
        // kPrefetch k-tiles ahead within a segment (x = kt * 128 bytes,
        // 16-byte aligned)
        int it = 0;
        bool stop = false;
        for (int j = 0; j < nseg && !stop; ++j) {
            const DenseSeg g = seg_at(d, cta, j);
            const int m0 = (g.tile % d.tiles_m) * kTM, n0 = (g.tile / d.tiles_m) * ntile;
            for (int kt = g.ka; kt < g.kb && kt < g.ka + kPrefetch; ++kt) tma_prefetch_2d(&tmA, kt * kRowBytes, m0);
            if (j == 0) grid_dep_wait();  // the clause tiles above need nothing from the packing kernel
            for (int kt = g.ka; kt < g.kb; ++kt) {
                const int s = it % kStages;
                if (kPrefetch > 0 && kt + kPrefetch < g.kb) tma_prefetch_2d(&tmA, (kt + kPrefetch) * kRowBytes, m0);
                if (it >= kStages) {
                    const uint32_t parity = (uint32_t)((it / kStages - 1) & 1);
                    if (*(volatile int *)&H->abort || !mbar_wait(&H->empty[s], parity, 0, kWaitNs)) {
                        H->abort = 1;
                        atomicOr(errflag, 1u);
                        stop = true;
                        break;
                    }
                }
                uint8_t *sa = stages + (size_t)s * stage_bytes;
                mbar_expect_tx(&H->full[s], stage_bytes);
                tma_load_2d(sa, &tmA, kt * kRowBytes, m0, &H->full[s]);
                tma_load_2d(sa + a_bytes, &tmB, kt * kRowBytes, n0, &H->full[s]);
                ++it;
            }
        }
        // every issued copy has landed before the block may exit
        for (int i = (it > kStages ? it - kStages : 0); i < it; ++i)
            if (!mbar_wait(&H->full[i % kStages], (uint32_t)((i / kStages) & 1), 0, kWaitNs)) atomicOr(errflag, 2u);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: segment j accumulates into TMEM buffer j % nbuf once
        // the epilogue has read what segment j - nbuf left there
        const uint32_t idesc = idesc_mxf4(ntile);
        const uint32_t sfa = tmem + (uint32_t)sf_col, sfb = sfa + (uint32_t)(kSfCols / 2);
        int it = 0;
        bool stop = false;
        for (int j = 0; j < nseg && !stop; ++j) {
            const DenseSeg g = seg_at(d, cta, j);
            const int buf = j % nbuf;
            if (j >= nbuf && !mbar_wait_abort(&H->acc_empty[buf], (uint32_t)((j / nbuf - 1) & 1), &H->abort)) {
                H->abort = 1;
                atomicOr(errflag, 1u);
                stop = true;
                break;
            }
            tc_fence_after();
            const uint32_t acc = tmem + (uint32_t)(buf * tmem_cols);
            for (int kt = g.ka; kt < g.kb; ++kt) {
                const int s = it % kStages;
                if (*(volatile int *)&H->abort || !mbar_wait(&H->full[s], (uint32_t)((it / kStages) & 1), 0, kWaitNs)) {
                    H->abort = 1;
                    atomicOr(errflag, 1u);
                    stop = true;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(stages + (size_t)s * stage_bytes);
                const uint64_t adesc = smem_desc_sw128(sa);
                const uint64_t bdesc = smem_desc_sw128(sa + a_bytes);
#pragma unroll
                for (int kk = 0; kk < kRowBytes / 32; ++kk)  // K = 64 codes (32 bytes) per MMA: +2 in the 16-byte address field
                    mma_mxf4(acc, adesc + 2 * kk, bdesc + 2 * kk, idesc, sfa, sfb, (kt != g.ka || kk != 0) ? 1u : 0u);
                mma_commit(&H->empty[s]);
                ++it;
            }
            if (stop) break;
            mma_commit(&H->acc_full[buf]);  // arrives once every MMA of the segment has completed
        }
        if (stop) {
            // MMAs issued before the abort may still be writing TMEM: wait
            // (bounded) until all of them have completed before the block
            // reaches the barrier that precedes the TMEM release
            mma_commit(&H->drain);
            if (!mbar_wait(&H->drain, 0u, 0, kWaitNs)) atomicOr(errflag, 16u);
        }
    } else if (warp >= 2) {
        // epilogue: TMEM lane quarter q (= warp % 4) holds clause rows
        // m0 + 32q .. + 31 of the segment's tile; of the two warps of a
        // quarter, half h takes the 32-column chunks 2 i + h
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const int r = 32 * q + lane;  // row within the tile
        const int etid = threadIdx.x - 64;
        grid_dep_wait();  // the costs were cleared by the packing kernel
        for (int j = 0; j < nseg; ++j) {
            const DenseSeg g = seg_at(d, cta, j);
            const int buf = j % nbuf;
            const bool ok = mbar_wait_abort(&H->acc_full[buf], (uint32_t)((j / nbuf) & 1), &H->abort);
            if (!ok) H->epi_fail = 1;
            epi_sync();
            if (H->epi_fail) {  // the same decision in all eight warps
                if (etid == 0) atomicOr(errflag, 4u);
                H->abort = 1;
                break;
            }
            tc_fence_after();
            const int m0 = (g.tile % d.tiles_m) * kTM, n0 = (g.tile / d.tiles_m) * ntile;
            const uint32_t w = __ldg(wgt + m0 + r);
            const uint32_t acc = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * tmem_cols);
            const int nch = (ntile + 31) / 32;
            // the accumulator as hit masks: bit c of hm[ch] says that
            // column 32 ch + c of the row reached its target -- -len_j for
            // a whole tile (the clause is unsat), the piece's target for a
            // piece of a split tile (every literal of the clause in the
            // piece's k-range is false); columns past ntile never hit
            size_t slot = 0;
            float cmp;
            if (g.tr < 0) {
                cmp = __ldg(target + m0 + r);
            } else {
                slot = (size_t)g.tr * d.split + g.piece;
                cmp = __ldg(ptgt + slot * kTM + r);
            }
            // this half's chunks 2 i + h, two 32-column loads in flight
            // per wait
            uint32_t hm[4];
#pragma unroll
            for (int i = 0; i < 4; i += 2) {
                const int c0 = 2 * i + h, c1 = c0 + 2;
                hm[i] = hm[i + 1] = 0u;
                if (c0 < nch) {
                    uint32_t va[32], vb[32];
                    tmem_ld32_issue(acc + (uint32_t)(32 * c0), va);
                    // past the last chunk: the same columns again (dropped below)
                    tmem_ld32_issue(acc + (uint32_t)(32 * (c1 < nch ? c1 : c0)), vb);
                    tmem_wait2(va, vb);
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        hm[i] |= (__uint_as_float(va[c]) == cmp ? 1u : 0u) << c;
                        hm[i + 1] |= (__uint_as_float(vb[c]) == cmp ? 1u : 0u) << c;
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int live = ntile - 32 * (2 * i + h);
                if (live <= 0) hm[i] = 0u;
                else if (live < 32) hm[i] &= (1u << live) - 1u;
            }
            // every column is read: the accumulator buffer is free for
            // segment j + nbuf while this one is counted
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&H->acc_empty[buf]);
            bool count = true;
            if (g.tr >= 0) {
                // a piece of a split tile: store the bits, count this
                // piece in; the last piece of the tile ANDs the others'
                // bits into its own and counts the tile
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (2 * i + h < nch) pmask[(slot * nch + 2 * i + h) * kTM + r] = hm[i];
                __threadfence();  // this CTA's bits before its count
                epi_sync();
                if (etid == 0) H->last = atomicAdd(part_cnt + g.tr, 1u) == (unsigned)(d.split - 1);
                epi_sync();
                count = H->last != 0;
                if (count) {
                    __threadfence();
                    for (int pc = 0; pc < d.split; ++pc) {
                        if (pc == g.piece) continue;
                        const uint32_t *other = pmask + ((size_t)g.tr * d.split + pc) * nch * kTM + r;
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (2 * i + h < nch) hm[i] &= __ldcg(other + (size_t)(2 * i + h) * kTM);
                    }
                    if (etid == 0) part_cnt[g.tr] = 0u;  // ready for the next launch
                }
            }
            if (count) {
                // unsat count per column over the warp's 32 rows (lane l
                // gets column l), then added over the four quarters: with unit
                // weights the popcount of the transposed hit bits, else
                // the column sums of w [hit]
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int ch = 2 * i + h;
                    if (ch < nch && __any_sync(0xffffffffu, hm[i] != 0u)) {
                        uint32_t sum;
                        if (unit_w) {
                            sum = (uint32_t)__popc(transpose_bits32(hm[i], lane));
                        } else {
                            uint32_t x[32];
#pragma unroll
                            for (int c = 0; c < 32; ++c) x[c] = ((hm[i] >> c) & 1u) ? w : 0u;
                            sum = column_sums32(x, lane);
                        }
                        if (sum) atomicAdd(&H->colsum[32 * ch + lane], (unsigned long long)sum);
                    }
                }
            }
            // add the tile's column sums to the costs
            epi_sync();
            for (int cc = etid; cc < ntile; cc += 32 * kEpiWarps) {
                const unsigned long long cs = H->colsum[cc];
                if (cs) {
                    if (n0 + cc < nb) atomicAdd(cost + n0 + cc, cs);
                    H->colsum[cc] = 0ull;
                }
            }
            epi_sync();
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// Self-test of the bounded waits: one thread waits on an mbarrier that
// nothing arrives at, gives up after `spins` tries (spins = 0: on the
// kernels' own time limit, kWaitNs) and records it in the error flag --
// the path every wait of k_dense_eval takes when a phase never completes.
// Nothing faults and nothing hangs; the context stays usable.
__global__ void k_wait_selftest(long long spins, unsigned int *errflag) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait(&bar, 0u, spins, kWaitNs)) atomicOr(errflag, 8u);
    }
}

// Issue rate of the evaluator's MMA on its own: one CTA per SM issues
// `iters` stages of four kind::mxf4 MMAs (M = 128, N = n, K = 64 codes
// each) on operands resident in shared memory (zero codes, unit scale
// factors), cycling over four stage buffers like the pipeline does, and
// waits (bounded) for them to complete.  The host times the launch: the
// measured peak of this instruction shape, which the evaluator's pipeline
// can approach but not pass.
__global__ void __launch_bounds__(128, 1) k_mma_rate(int n, int iters, unsigned int *__restrict__ errflag) {
    extern __shared__ uint8_t dsm_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint32_t tmem_s;
    __shared__ __align__(8) unsigned long long done;
    const int warp = threadIdx.x >> 5;
    const uint32_t stage_bytes = (uint32_t)(kTM + n) * kRowBytes;
    for (uint32_t i = threadIdx.x; i < kStages * stage_bytes / 4; i += blockDim.x)
        reinterpret_cast<uint32_t *>(base)[i] = 0u;
    if (threadIdx.x == 0) {
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_s;
    const uint32_t sf_col = 256;
    tmem_fill32(tmem + ((uint32_t)(32 * warp) << 16) + sf_col, kSfOne);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeros, for the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_mxf4(n);
        for (int it = 0; it < iters; ++it) {
            const uint32_t sa = smem_u32(base + (size_t)(it % kStages) * stage_bytes);
            const uint64_t adesc = smem_desc_sw128(sa);
            const uint64_t bdesc = smem_desc_sw128(sa + kTM * kRowBytes);
#pragma unroll
            for (int kk = 0; kk < kRowBytes / 32; ++kk)
                mma_mxf4(tmem, adesc + 2 * kk, bdesc + 2 * kk, idesc, tmem + sf_col, tmem + sf_col + kSfCols / 2,
                         (it != 0 || kk != 0) ? 1u : 0u);
        }
        mma_commit(&done);
        if (!mbar_wait(&done, 0u, 0, kWaitNs)) atomicOr(errflag, 32u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// Per-piece targets of the split tiles: for split tile tr, piece p and row
// r, minus the number of the clause's literals whose variable lies in the
// piece's k-range [p * kt / split, (p + 1) * kt / split) x kTK (NaN for
// padding rows and for clauses that never count).
__global__ void k_dense_piece_targets(DevInst I, const float *__restrict__ target, DenseSched d, int grid,
                                      float *__restrict__ ptgt) {
    const int tr = blockIdx.x, r = threadIdx.x;  // kTM threads
    const int tile = d.full * grid + tr;
    const long long j = (long long)(tile % d.tiles_m) * kTM + r;
    float out[4];
    const bool live = j < I.m && !isnan(target[j]);
    for (int p = 0; p < 4; ++p) out[p] = live ? 0.0f : __int_as_float(0x7fc00000);
    if (live) {
        int beg, end;
        if (I.kfix > 0) {
            beg = (int)j * I.kfix;
            end = beg + I.kfix;
        } else {
            beg = I.coff[j];
            end = I.coff[j + 1];
        }
        for (int q = beg; q < end; ++q) {
            const int kt = (I.lit[q] >> 1) / kTK;
            int p = 0;
            while (p + 1 < d.split && (long long)(p + 1) * d.kt_count / d.split <= kt) ++p;
            out[p] -= 1.0f;
        }
    }
    for (int p = 0; p < d.split; ++p) ptgt[((size_t)tr * d.split + p) * kTM + r] = out[p];
}

// W^T in packed e2m1: row j (n_pad / 2 bytes) holds +1 / -1 at the columns
// of the clause's literals, variable i in the low (i even) or high nibble
// of byte i / 2 (the buffer was zeroed).  One thread owns a row, so the
// read-modify-write of a byte shared by two literals is race-free.  A
// clause with x and not x writes both into the same nibble; its target is
// NaN, so it never counts.
__global__ void k_dense_fill(DevInst I, uint8_t *__restrict__ Wt, int n_pad) {
    const long long row_bytes = n_pad / 2;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < I.m;
         j += (long long)gridDim.x * blockDim.x) {
        int beg, end;
        if (I.kfix > 0) {
            beg = (int)j * I.kfix;
            end = beg + I.kfix;
        } else {
            beg = I.coff[j];
            end = I.coff[j + 1];
        }
        uint8_t *row = Wt + j * row_bytes;
        for (int p = beg; p < end; ++p) {
            const int L = I.lit[p];
            const int v = L >> 1, sh = (v & 1) * 4;
            const uint8_t code = (L & 1) ? kE2M1MinusOne : kE2M1One;
            row[v >> 1] = (uint8_t)((row[v >> 1] & ~(0xF << sh)) | (code << sh));
        }
    }
}

// X^T in packed e2m1 (rows = assignments, n_pad / 2 bytes each, zero
// padding) from a batch stored [n][nb]: a block transposes 64 variables x
// 32 assignments through shared memory, reading along the batch and
// writing 32 bytes (64 codes) of each assignment's row.
template <typename T>
__device__ __forceinline__ void pack_transpose(const T *__restrict__ src, int n, int nb, uint8_t *__restrict__ Xt,
                                               int n_pad, int rows) {
    __shared__ uint8_t tile[64][33];
    const int v0 = blockIdx.x * 64, b0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 64; r += blockDim.y) {
        const int v = v0 + r, b = b0 + threadIdx.x;
        uint8_t e = 0;
        if (v < n && b < nb) e = src[(long long)v * nb + b] > (T)0 ? kE2M1One : kE2M1MinusOne;
        tile[r][threadIdx.x] = e;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int b = b0 + r, t = threadIdx.x;
        if (b < rows)
            Xt[(long long)b * (n_pad / 2) + v0 / 2 + t] = (uint8_t)(tile[2 * t][r] | (tile[2 * t + 1][r] << 4));
    }
}

// From the caller's int8 [n][nb] batch (> 0 is true).
__global__ void k_dense_convert(const int8_t *__restrict__ a, int n, int nb, uint8_t *__restrict__ Xt,
                                int n_pad, int rows) {
    grid_dep_launch();
    pack_transpose<int8_t>(a, n, nb, Xt, n_pad, rows);
}

// The same operand straight from the relaxed x (float [n][nb]): x > 0 reads
// as +1, otherwise -1 -- the rounding of Sec. 4 -- without the int8 copy.
__global__ void k_dense_convert_x(const float *__restrict__ x, int n, int nb, uint8_t *__restrict__ Xt,
                                  int n_pad, int rows, long long *__restrict__ cost) {
    grid_dep_launch();
    if (blockIdx.x == 0 && blockIdx.y == 0)  // the GEMM that follows in stream order adds into cost
        for (int b = threadIdx.y * 32 + threadIdx.x; b < nb; b += 32 * blockDim.y) cost[b] = 0;
    pack_transpose<float>(x, n, nb, Xt, n_pad, rows);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2D tensor of packed 4-bit codes [rows][cols] (cols contiguous, cols / 2
// bytes a row; cols a multiple of kTK), copied as bytes: box kRowBytes x
// box_rows, 128B swizzle, landing in shared memory as packed as it is in
// global memory.
int encode_2d(CUtensorMap *map, void *base, long long cols, long long rows, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return fail(MSAT_ECUDA, "dense backend: cuTensorMapEncodeTiled is not available");
    if (cols % kTK != 0) return fail(MSAT_EINVAL, "dense backend: padded variable count is not a multiple of 256");
    const cuuint64_t dims[2] = {(cuuint64_t)(cols / 2), (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(cols / 2)};
    const cuuint32_t box[2] = {(cuuint32_t)kRowBytes, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(MSAT_ECUDA, "dense backend: cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return MSAT_OK;
}

}  // namespace

int dense_tile_n(int nb) {
    const int nb16 = (nb + 15) / 16 * 16;
    return nb16 <= 256 ? nb16 : 256;
}

int dense_rows(int nb) {
    const int nt = dense_tile_n(nb);
    return (nb + nt - 1) / nt * nt;
}

size_t dense_smem_bytes(int ntile) {
    return 1024 + kHeader + (size_t)kStages * ((size_t)kTM + (size_t)ntile) * kRowBytes;
}

int dense_encode_a(DenseDev &d) { return encode_2d(&d.tmA, d.Wt, d.n_pad, d.m_pad, kTM); }

int dense_encode_b(DenseDev &d, int rows, int ntile) {
    d.tmB_rows = rows;
    d.tmB_ntile = ntile;
    return encode_2d(&d.tmB, d.Xt, d.n_pad, rows, ntile);
}

cudaError_t launch_dense_fill(const DevInst &I, uint8_t *Wt, int n_pad, cudaStream_t st) {
    long long blocks = ((long long)I.m + kThreads - 1) / kThreads;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_dense_fill<<<(unsigned)blocks, kThreads, 0, st>>>(I, Wt, n_pad);
    return cudaGetLastError();
}

cudaError_t launch_dense_convert(const DenseDev &d, const int8_t *a, int n, int nb, long long *cost,
                                 cudaStream_t st) {
    dim3 cb(32, 8), cg((unsigned)(d.n_pad / 64), (unsigned)((d.tmB_rows + 31) / 32));
    k_dense_convert<<<cg, cb, 0, st>>>(a, n, nb, d.Xt, d.n_pad, d.tmB_rows);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    return cudaMemsetAsync(cost, 0, sizeof(long long) * (size_t)nb, st);
}

cudaError_t launch_dense_convert_x(const DenseDev &d, const float *x, int n, int nb, long long *cost,
                                   cudaStream_t st) {
    dim3 cb(32, 8), cg((unsigned)(d.n_pad / 64), (unsigned)((d.tmB_rows + 31) / 32));
    k_dense_convert_x<<<cg, cb, 0, st>>>(x, n, nb, d.Xt, d.n_pad, d.tmB_rows, cost);
    return cudaGetLastError();
}

// Whole tiles one per CTA when they fit one wave of one CTA per SM.  With
// more tiles the grid stays one CTA per SM and each CTA streams its tiles
// back to back (the next tile's loads overlap the last one's epilogue):
// equal whole-tile shares, then a leftover of at most half a wave split
// into up to 4 k-step pieces per tile, or a larger leftover as one more
// whole tile on the first CTAs.
DenseSched dense_plan(const DenseDev &d, int ntile, int *grid) {
    DenseSched p{};
    p.kt_count = d.n_pad / kTK;
    p.tiles_m = d.m_pad / kTM;
    p.ntile = ntile;
    p.full = 1;
    p.split = 1;
    const int T = p.tiles_m * (d.tmB_rows / ntile);
    const int G = d.sm_count > 0 ? d.sm_count : 152;
    *grid = T;
    if (T > G) {
        const int full = T / G, rest = T - full * G;
        int split = rest > 0 ? G / rest : 0;
        if (split > 4) split = 4;
        if (split > p.kt_count) split = p.kt_count;
        p.full = full;
        *grid = G;
        if (rest > 0 && split >= 2) {
            p.tail = rest;
            p.split = split;
            p.tail_ctas = rest * split;
        } else {
            p.extra = rest;
        }
    }
    return p;
}

cudaError_t launch_dense_gemm(const DenseDev &d, int nb, long long *cost, cudaStream_t st) {
    const int ntile = d.tmB_ntile;
    cudaError_t e;
    const size_t smem = dense_smem_bytes(ntile);
    e = cudaFuncSetAttribute(k_dense_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max_dense());
    if (e) return e;
    int tmem_cols = 32;  // one accumulator's columns
    while (tmem_cols < ntile) tmem_cols <<= 1;
    int grid = 0;
    const DenseSched p = dense_plan(d, ntile, &grid);
    if (p.tail > 0 && (p.tail * p.split > d.ptgt_slots || p.tail > d.part_cnts || ntile != d.pmask_ntile))
        return cudaErrorInvalidValue;
    // launched to overlap the packing kernel before it in the stream (it
    // waits for that kernel's writes where it needs them)
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(kDenseThreads);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, k_dense_eval, d.tmA, d.tmB, d.target, d.wgt, d.unit_w ? 1 : 0, p, tmem_cols, nb,
                              reinterpret_cast<unsigned long long *>(cost), d.ptgt, d.pmask, d.part_cnt,
                              d.errflag);
}

size_t smem_max_dense() { return dense_smem_bytes(256); }

cudaError_t launch_dense_piece_targets(const DevInst &I, const DenseDev &d, const DenseSched &p, int grid,
                                       cudaStream_t st) {
    if (p.tail <= 0) return cudaSuccess;
    k_dense_piece_targets<<<p.tail, kTM, 0, st>>>(I, d.target, p, grid, d.ptgt);
    return cudaGetLastError();
}

cudaError_t launch_mma_rate(int n, int iters, int grid, unsigned int *errflag, cudaStream_t st) {
    const size_t smem = 1024 + (size_t)kStages * (kTM + n) * kRowBytes;
    cudaError_t e = cudaFuncSetAttribute(k_mma_rate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    k_mma_rate<<<grid, 128, smem, st>>>(n, iters, errflag);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(long long spins, unsigned int *errflag, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(spins, errflag);
    return cudaGetLastError();
}

}  // namespace msat
