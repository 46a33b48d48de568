// Stage 4 on the tcgen05 tensor cores: C_IJ = alpha * sum_{kept K, ascending}
// A_IK B_KJ + beta * C_IJ (Algorithm 1, numeric part), with FP32
// accumulation in tensor memory.
//
// Work unit: one 128 x 256 C tile = TL row leaves x 2 TL column leaves
// (TL = 128 / b), and the tile's steps (K, two half masks) in ascending K
// from the grouping stage.  For every step and every 16-wide K chunk the
// tile needs A's 128 x 16 slice (its row leaves at column leaf K) and B's
// 16 x 256 slice, hi and lo parts; the packs hold them already in the
// no-swizzle K-major layout of tcgen05 (8-row x 16-byte core matrices),
// grouped so that the chunks a tile reads from one operand at one K are
// contiguous runs of pack groups (CG chunks: their high parts, then their
// low parts).  One 1-D bulk copy per operand moves a group into shared
// memory: at b = 64 one step is two copies, with both parts or with the
// high parts alone.  The
// copies, not their bytes, set the pace of the producer (each costs on the
// order of fifty cycles to issue and complete), so fewer and larger copies
// are what keeps the tensor pipe fed.  A 256-wide tile halves the MMA
// instructions per flop compared with 128 x 128: on this part an MMA's
// issue cost, not its arithmetic, dominates at N = 128.
//
// Exactness of the cull: a kept leaf product (x, K, y) must be added and a
// culled one must not.  One MMA over a run of consecutive column leaves
// y0..y0+len-1 that share the same set of kept row leaves uses the MMA's
// disable-output-lane mask to leave the accumulator rows (TMEM lanes) of the
// culled row leaves untouched, so the tensor core adds exactly the kept
// products.  N = len * b (16..256), M = 128.  A step whose products are
// all kept (the common case on dense blocks) skips the run analysis and
// issues unmasked 128 x 256 MMAs.
//
// Precisions: TF32X3 splits each operand into a TF32 high part and a TF32
// low part (a - hi) and adds lo*hi + hi*lo + hi*hi; TF32 uses hi*hi only;
// BF16X3 does the same with bfloat16 parts on kind::f16; F16X3 with fp16
// parts of each operand scaled by a power of two (its largest leaf norm
// just below 2^15), the product scaled back exactly in the epilogue.  All
// accumulate in FP32.  With precision chosen by norm, each step also carries
// the masks of its products whose norm product reaches tau_h: those get all
// three passes, the other kept products hi*hi alone, and a step without any
// such product loads only the high parts of its operands.
//
// Two-level accumulation: the tensor core's FP32 accumulation rounds less
// carefully than an IEEE add, and a C tile can chain thousands of MMAs.  So
// the MMAs of a tile are cut into chunks of at most kChunkIters K-chunks;
// every chunk starts from a zeroed TMEM accumulator, and the epilogue warps
// add the finished chunk into a master FP32 accumulator held in registers
// (one row of 128 values per thread) with round-to-nearest adds.  Chunks are
// added in ascending K, so the result stays deterministic.  The epilogue
// leaves each buffer zero when it has read it (and zeroes both at the
// start), so the MMAs of a chunk accumulate onto zeros without a clearing
// MMA of their own.
//
// Tile order: consecutive work items walk down a group of kGroupRows tile
// rows before moving one tile column right, so the tiles in flight at once
// share A slices (same rows) and B slices (same columns) in L2.
//
// Roles (320 threads): warp 0 lane 0 issues the bulk copies into a ring of
// shared-memory stages (two of 96 KB for 16-bit parts and single TF32, four
// of 48 KB for TF32 hi and lo); warp 1 owns the TMEM allocation (all 512
// columns) and its lane 0 issues the MMAs and commits, a stage's masks read
// at once and its slots unrolled; warps 2-9 move the double-buffered
// 128 x 256 chunk accumulators out of TMEM (two warps per TMEM lane quarter,
// 128 columns each), zero them for the next chunk, sum them, apply
// alpha/beta and store C.  Every wait on
// an mbarrier gives up after one second, raises the timeout status and lets
// the block drain its copies and MMAs, free TMEM and exit.
//
// A launch covers the work items [first, total) of its table: one launch
// for a multiply, or (host entry point) one per band of tile-row groups.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

#include "spamm_internal.cuh"

namespace spamm {
namespace {

constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;
constexpr int kChunkIters = 32;  // K-chunks of 16 per TMEM accumulation chunk
constexpr int kGroupRows = 12;  // tile rows walked together (L2 reuse)
constexpr int kTQ = 16;         // tile-queue entries (producer -> MMA and epilogue)
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s: default bound of the waits

// The bound of the pipeline's waits, set per launch (spamm_set_wait_limit;
// kWaitNs unless a failure-detection test shortens it).  The drains at the
// end of a block always allow kWaitNs.


__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

// Bounded wait: true when the phase completed, false after limit_ns (or
// when another role already gave up).
__device__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                         unsigned int* status, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > limit_ns) {
            *abort_flag = 1;
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
}

// A drain before the block frees its resources: waits out the phase whether
// or not another role gave up, for at most kWaitNs.
__device__ bool wait_drain(uint32_t bar, uint32_t parity, unsigned int* status) {
    const uint64_t t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer() - t0 > kWaitNs) {
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
    return true;
}

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B format (1 = BF16 under
// kind::f16, 2 = TF32 under kind::tf32), both K-major, M x N.
__device__ __forceinline__ constexpr uint32_t make_idesc(uint32_t ab, int M, int N) {
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Work item k -> tile index (row-major over tr x tc tiles), grouped by
// kGroupRows tile rows.
__device__ __forceinline__ int tile_at(int k, int tr, int tc) {
    const int span = kGroupRows * tc;
    const int g = k / span;
    const int rows = min(kGroupRows, tr - g * kGroupRows);
    const int w = k - g * span;
    return (g * kGroupRows + w % rows) * tc + w / rows;
}

// TMEM chunks of a tile with `iters` K-chunk iterations; a tile without
// kept products has none (its epilogue writes beta * C straight away).
__device__ __forceinline__ uint32_t chunks_of(uint32_t iters) {
    return (iters + kChunkIters - 1) / kChunkIters;
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    const uint32_t (&dis)[4], uint32_t acc) {
    if (PREC == SPAMM_PREC_BF16X3 || PREC == SPAMM_PREC_F16X3) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, {%5, %6, %7, %8}, p;\n\t}"
            ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc), "r"(dis[0]), "r"(dis[1]),
            "r"(dis[2]), "r"(dis[3])
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, {%5, %6, %7, %8}, p;\n\t}"
            ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc), "r"(dis[0]), "r"(dis[1]),
            "r"(dis[2]), "r"(dis[3])
            : "memory");
    }
}

// The same MMA without the disable-output-lane operand (every lane written).
template <int PREC>
__device__ __forceinline__ void mma_all(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
    if (PREC == SPAMM_PREC_BF16X3 || PREC == SPAMM_PREC_F16X3) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Zero 32 lanes x 32 columns of tensor memory (this warp's lane quarter).
__device__ __forceinline__ void tmem_zero32(uint32_t taddr) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};"
        ::"r"(taddr), "r"(0u)
        : "memory");
}

template <int PREC>
struct PrecTraits {
    static constexpr bool k16 = PREC == SPAMM_PREC_BF16X3 || PREC == SPAMM_PREC_F16X3;
    static constexpr int kEsize = k16 ? 2 : 4;
    static constexpr int kParts = PREC == SPAMM_PREC_TF32 ? 1 : 2;      // arrays per role
    static constexpr int kSlice = 128 * 16 * kEsize;                   // bytes of one 128x16 slice
    static constexpr int kASlot = kParts * kSlice;                      // A of one K-chunk
    static constexpr int kBSlot = 2 * kParts * kSlice;                  // B of one K-chunk
    static constexpr int kIter = kASlot + kBSlot;                       // A (128) + B (256) rows
    // Stages: 96 KB of four K-chunks (16-bit parts, single TF32) in two
    // stages, or 48 KB of one K-chunk (TF32 hi and lo) in four: measured on
    // the n=7500 workload, each the faster of the two for its precision.
    static constexpr int kSPS = kIter <= 24576 ? 4 : 1;                 // K-chunks per stage
    static constexpr int kStage = kSPS * kIter;
    static constexpr int kStages = 196608 / kStage;
    static constexpr int kKInstr = k16 ? 16 : 8;                        // K per MMA
    static constexpr uint32_t kSBO = 8 * 16 * kEsize;                   // row-group stride
    // operand format of the instruction descriptor: kind::tf32 -> TF32 (2);
    // kind::f16 -> BF16 (1) or F16 (0)
    static constexpr uint32_t kAB = PREC == SPAMM_PREC_BF16X3 ? 1u
                                    : PREC == SPAMM_PREC_F16X3 ? 0u : 2u;
};

// One product of a (possibly one-element) batch, as the host prepares it.
struct TcProd {
    const void* pa[2];
    const void* pb[2];
    int64_t nlp;
    float* C;
    int64_t ldc, n;
    float alpha, beta;
    DevCtl* ctl;
    const uint64_t* pool;
    const uint32_t* off;
    const uint32_t* steps;
    const uint32_t* iters;  // K-chunk iterations per tile
    int tr, tc, S;
    int sl;    // mask pairs per step: 1, or one per K-chunk (sub-leaf cull)
    int base;  // first work item (tile) of this product in the batch
    // sparsified operands (BAND kernels): per K the band of pieces the pack
    // holds, A role over leaf rows [lo, hi] of column K, B role over leaf
    // columns [lo, hi] of row K, and the band's first piece; null if dense
    const int32_t* a_lo;
    const int32_t* a_hi;
    const int64_t* a_off;
    const int32_t* b_lo;
    const int32_t* b_hi;
    const int64_t* b_off;
    // FP16 split: largest squared leaf norms of A and B (their scales)
    const double* gmax;
    // precision chosen by norm: the step list carries a second mask pair per
    // step, the products that keep the full split; the others run hi * hi
    int tier;
};

constexpr int kMaxBatch = 64;

// Passed by value as the kernel parameter (~8 KB), so a launch carries its
// own table: back-to-back launches cannot overwrite each other's, and a graph
// capture records it with the launch.
struct TcBatch {
    TcProd prods[kMaxBatch];
    int count;             // products
    int first;             // first work item of this launch (0 but for banded launches)
    int total;             // work items (tiles) of all products; this launch ends here
    unsigned int* status;  // timeout status word
    unsigned long long wait_ns;  // bound of the pipeline's waits
    unsigned int* ctr;     // work-item counter of the launch (zero at its start)
};

// BAND: at least one operand of the batch is sparsified; its pieces are
// copied from inside their band (the rows or columns of a tile outside the
// band have no kept product and are not loaded).
template <int LEAF, int PREC, bool BAND>
__global__ void __launch_bounds__(kThreads, 1) k_leaf_tc(TcBatch bt) {
    using T = PrecTraits<PREC>;
    constexpr int TL = 128 / LEAF;      // row leaves = column leaves per half
    constexpr int TLC = 2 * TL;         // column leaves of the tile
    constexpr int CHUNKS = LEAF / 16;
    constexpr int ST = T::kStages;
    // K-chunks per pack group (the packs store a group's high parts before
    // its low parts).  A stage is cut into U units: the A region into U
    // 128 x 16 slices, the B region into U 256 x 16 slices.  A group of c
    // chunks takes 2c units with both parts (high c, then low c) or c with
    // the high parts alone, so a stage holds kSPS chunks of full groups or up
    // to U = kParts x kSPS chunks of lean ones.
    constexpr int CG = CHUNKS < T::kSPS ? CHUNKS : T::kSPS;
    constexpr int U = T::kParts * T::kSPS;
    static_assert(CG == pack_group_chunks(LEAF, PREC), "pack group and stage disagree");
    static_assert(T::kSPS % CG == 0, "a stage holds whole pack groups");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[ST], bar_empty[ST], bar_accf[2], bar_acce[2],
        bar_drain;
    __shared__ uint32_t tmem_slot;
    // the groups of each stage: first unit, chunks (and lean flag) packed,
    // the kept masks and, of those, the full-split products
    __shared__ uint32_t st_grp[ST][U];
    __shared__ unsigned long long st_mask[ST][U][2];
    __shared__ unsigned long long st_hmask[ST][U][2];
    __shared__ uint32_t st_count[ST];                        // groups of each stage
    __shared__ volatile int abort_flag;
    // work items in the order the producer took them: full (id written) and
    // empty (taken by the MMA thread and every epilogue warp) barriers
    __shared__ int tq_id[kTQ];
    __shared__ __align__(8) uint64_t bar_tqf[kTQ], bar_tqe[kTQ];
    __shared__ unsigned long long issued_s, consumed_s;
    // per product: step-list offsets in its pool, skip flag, end of its work
    // items.  Everything else is read from the parameter space: pointers that
    // come from there are known to be global, which keeps the MMA issue loop
    // as tight as with a single product.
    __shared__ unsigned long long sp_pk[kMaxBatch], sp_pm[kMaxBatch], sp_ph[kMaxBatch];
    __shared__ int sp_skip[kMaxBatch], sp_end[kMaxBatch];
    __shared__ float2 sp_uns[PREC == SPAMM_PREC_F16X3 ? kMaxBatch : 1];  // 2^-(kA + kB)

    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* stages = base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned int* status = bt.status;
    for (int i = threadIdx.x; i < bt.count; i += kThreads) {
        const TcProd& g = bt.prods[i];
        sp_pk[i] = g.ctl->pk_off;
        sp_pm[i] = g.ctl->pm_off;
        sp_ph[i] = g.ctl->ph_off;
        // a product whose cull failed is left untouched (its status says why)
        sp_skip[i] = (g.ctl->status & (ST_OVERFLOW | ST_NONFINITE)) ? 1 : 0;
        sp_end[i] = g.base + g.tr * g.tc;
        if constexpr (PREC == SPAMM_PREC_F16X3)
            sp_uns[i] = f16_unscale(g.gmax[0], g.gmax[1]);
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bar_accf[b]), 1);
            mbar_init(smem_u32(&bar_acce[b]), kEpiWarps);
        }
        mbar_init(smem_u32(&bar_drain), 1);
        for (int t = 0; t < kTQ; ++t) {
            mbar_init(smem_u32(&bar_tqf[t]), 1);
            mbar_init(smem_u32(&bar_tqe[t]), 1 + kEpiWarps);
        }
        abort_flag = 0;
        issued_s = consumed_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    // work item k -> product index, advancing monotonically (k only grows)
    auto product_of = [&](int k, int& pi) {
        while (pi + 1 < bt.count && k >= sp_end[pi]) ++pi;
    };

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        // The whole warp walks the step list in batches of 32 (each lane
        // loads one step's K and masks; the next batch is prefetched while
        // this one is issued) and lane 0 fills the stages with groups of
        // K-chunks (up to U units per stage, never across tiles).  For every
        // group it adds the group's bytes to the stage's expected transaction
        // count, issues the bulk copies and records the group's first unit,
        // chunk count and masks; closing a stage records its group count and
        // arrives on the full barrier.
        unsigned long long stage_it = 0;
        int fill = 0;   // units of the current stage in use
        int ng = 0;     // groups in the current stage
        int s = 0;
        bool ok = true;
        const size_t piece = (size_t)LEAF * 16 * T::kEsize;
        int pi = 0;
        uint32_t tq = 0;   // work items handed on
        while (ok) {
            // the next work item from the launch's counter (items are taken
            // in ascending order, so tiles in flight on all SMs stay close),
            // handed to the MMA thread and the epilogue through the queue;
            // -1 ends the launch
            int k = -1;
            if (lane == 0) {
                const int w = (int)atomicAdd(bt.ctr, 1u) + bt.first;
                k = w < bt.total ? w : -1;
                const int slot = (int)(tq % kTQ);
                const uint32_t tph = (tq / kTQ) & 1;
                ok = wait_bar(smem_u32(&bar_tqe[slot]), tph ^ 1, &abort_flag, status, bt.wait_ns);
                if (ok) {
                    tq_id[slot] = k;
                    mbar_arrive(smem_u32(&bar_tqf[slot]));
                }
            }
            k = __shfl_sync(0xffffffffu, k, 0);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            ++tq;
            if (k < 0 || !ok) break;
            product_of(k, pi);
            if (sp_skip[pi]) continue;
            const TcProd& q = bt.prods[pi];
            const uint32_t* pk = reinterpret_cast<const uint32_t*>(q.pool + sp_pk[pi]);
            const unsigned long long* pm =
                reinterpret_cast<const unsigned long long*>(q.pool + sp_pm[pi]);
            const unsigned long long* ph =
                reinterpret_cast<const unsigned long long*>(q.pool + sp_ph[pi]);
            const bool tier = q.tier != 0;
            const int u = tile_at(k - q.base, q.tr, q.tc);
            const int64_t srow = (int64_t)(u / q.tc) * TL;
            const int64_t scol = (int64_t)(u % q.tc) * TLC;
            const uint32_t ns = q.steps[u];
            const uint64_t sb = (uint64_t)q.off[u] * q.S;
            // lane 0: the group of m consecutive K-chunks kc0.. of the step at K
            // (a whole pack group, or one chunk with the sub-leaf cull or a
            // sparsified operand) into the units fill.. of the current stage.
            // The dense packs keep a tile's chunks of one K in the same groups
            // (high parts, then low parts) as the stage, so a whole group is
            // one bulk copy per operand, and so are its high parts alone.
            const int64_t ga = srow / TL, gb = scol / TLC;          // tile's pack groups
            int64_t bandK = -1;
            int64_t a_lo = 0, a_hi = -1, a_off = 0, b_lo = 0, b_hi = -1, b_off = 0;
            auto close_stage = [&]() {
                st_count[s] = (uint32_t)ng;
                mbar_arrive(smem_u32(&bar_full[s]));
                issued_s = ++stage_it;
                fill = 0;
                ng = 0;
            };
            // lean: no product of the step keeps the full split (precision
            // chosen by norm), so only the high parts are loaded
            auto issue = [&](int64_t K, int kc0, int m, unsigned long long m0,
                             unsigned long long m1, unsigned long long h0,
                             unsigned long long h1, bool lean) {
                const int parts = lean ? 1 : T::kParts;
                const int need = parts * m;                       // units
                if (fill > 0 && fill + need > U) close_stage();
                if (fill == 0) {
                    s = (int)(stage_it % ST);
                    const uint32_t ph = (uint32_t)((stage_it / ST) & 1);
                    ok = wait_bar(smem_u32(&bar_empty[s]), ph ^ 1, &abort_flag, status, bt.wait_ns);
                }
                if (!ok) return;
                const uint32_t full = smem_u32(&bar_full[s]);
                unsigned char* const stg = stages + (size_t)s * T::kStage;
                // shared memory of unit x of the A and B regions
                auto a_dst = [&](int x) { return stg + (size_t)x * T::kSlice; };
                auto b_dst = [&](int x) {
                    return stg + (size_t)U * T::kSlice + (size_t)x * 2 * T::kSlice;
                };
                // dense operand: the pack group holding chunk kc0, and chunk
                // kc0's part inside it
                const int c0 = kc0 % CG;
                const size_t a_grp =
                    ((size_t)(K * (q.nlp / TL) + ga) * CHUNKS + (kc0 - c0)) * T::kASlot;
                const size_t b_grp =
                    ((size_t)(K * (q.nlp / TLC) + gb) * CHUNKS + (kc0 - c0)) * T::kBSlot;
                const unsigned char* const pa0 = static_cast<const unsigned char*>(q.pa[0]);
                const unsigned char* const pb0 = static_cast<const unsigned char*>(q.pb[0]);
                auto a_src = [&](int part) {
                    return pa0 + a_grp + ((size_t)part * CG + c0) * T::kSlice;
                };
                auto b_src = [&](int part) {
                    return pb0 + b_grp + ((size_t)part * CG + c0) * 2 * T::kSlice;
                };
                if constexpr (BAND) {
                    // m == 1 here: a sparsified operand's chunk comes from
                    // inside its band, one copy per part
                    if (K != bandK) {
                        bandK = K;
                        if (q.a_lo) {
                            a_lo = q.a_lo[K];
                            a_hi = q.a_hi[K];
                            a_off = q.a_off[K];
                        }
                        if (q.b_lo) {
                            b_lo = q.b_lo[K];
                            b_hi = q.b_hi[K];
                            b_off = q.b_off[K];
                        }
                    }
                    uint32_t bytes = 0;
                    int64_t sa = 0, na = TL, da = 0;
                    if (q.a_lo) {
                        const int64_t lo = srow > a_lo ? srow : a_lo;
                        const int64_t hi = srow + TL - 1 < a_hi ? srow + TL - 1 : a_hi;
                        na = hi >= lo ? hi - lo + 1 : 0;
                        sa = a_off + kc0 * (a_hi - a_lo + 1) + (lo - a_lo);
                        da = lo - srow;
                        bytes += (uint32_t)(parts * na * piece);
                    } else {
                        bytes += (uint32_t)(parts * T::kSlice);
                    }
                    int64_t sb2 = 0, nb2 = TLC, db = 0;
                    if (q.b_lo) {
                        const int64_t lo = scol > b_lo ? scol : b_lo;
                        const int64_t hi = scol + TLC - 1 < b_hi ? scol + TLC - 1 : b_hi;
                        nb2 = hi >= lo ? hi - lo + 1 : 0;
                        sb2 = b_off + kc0 * (b_hi - b_lo + 1) + (lo - b_lo);
                        db = lo - scol;
                        bytes += (uint32_t)(parts * nb2 * piece);
                    } else {
                        bytes += (uint32_t)(parts * 2 * T::kSlice);
                    }
                    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(full),
                                 "r"(bytes)
                                 : "memory");
#pragma unroll
                    for (int part = 0; part < T::kParts; ++part) {
                        if (part >= parts) break;
                        if (q.a_lo) {
                            if (na)
                                bulk_g2s(smem_u32(a_dst(fill + part) + da * piece),
                                         static_cast<const unsigned char*>(q.pa[part]) +
                                             (size_t)sa * piece,
                                         (uint32_t)(na * piece), full);
                        } else {
                            bulk_g2s(smem_u32(a_dst(fill + part)), a_src(part),
                                     (uint32_t)T::kSlice, full);
                        }
                        if (q.b_lo) {
                            if (nb2)
                                bulk_g2s(smem_u32(b_dst(fill + part) + db * piece),
                                         static_cast<const unsigned char*>(q.pb[part]) +
                                             (size_t)sb2 * piece,
                                         (uint32_t)(nb2 * piece), full);
                        } else {
                            bulk_g2s(smem_u32(b_dst(fill + part)), b_src(part),
                                     (uint32_t)(2 * T::kSlice), full);
                        }
                    }
                } else if (m == CG) {
                    // a whole pack group: one copy per operand, all parts (or
                    // the high parts alone)
                    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(full),
                                 "r"((uint32_t)(need * 3 * T::kSlice))
                                 : "memory");
                    bulk_g2s(smem_u32(a_dst(fill)), a_src(0), (uint32_t)(need * T::kSlice), full);
                    bulk_g2s(smem_u32(b_dst(fill)), b_src(0), (uint32_t)(need * 2 * T::kSlice),
                             full);
                } else {
                    // one chunk of a group (the sub-leaf cull): one copy per
                    // operand and part
                    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(full),
                                 "r"((uint32_t)(need * 3 * T::kSlice))
                                 : "memory");
                    for (int part = 0; part < parts; ++part) {
                        bulk_g2s(smem_u32(a_dst(fill + part)), a_src(part), (uint32_t)T::kSlice,
                                 full);
                        bulk_g2s(smem_u32(b_dst(fill + part)), b_src(part),
                                 (uint32_t)(2 * T::kSlice), full);
                    }
                }
                st_grp[s][ng] = (uint32_t)fill | ((uint32_t)m << 8);
                st_mask[s][ng][0] = m0;
                st_mask[s][ng][1] = m1;
                st_hmask[s][ng][0] = h0;
                st_hmask[s][ng][1] = h1;
                ++ng;
                fill += need;
                if (fill == U) close_stage();
            };
            if (q.sl == 1) {
                // one mask pair per step, shared by its K-chunks
                uint32_t ck = lane < (int)ns ? pk[sb + lane] : 0u;
                unsigned long long cm0 = lane < (int)ns ? pm[2 * (sb + lane)] : 0ull;
                unsigned long long cm1 = lane < (int)ns ? pm[2 * (sb + lane) + 1] : 0ull;
                unsigned long long ch0 = cm0, ch1 = cm1;
                if (tier) {
                    ch0 = lane < (int)ns ? ph[2 * (sb + lane)] : 0ull;
                    ch1 = lane < (int)ns ? ph[2 * (sb + lane) + 1] : 0ull;
                }
                for (uint32_t base = 0; base < ns && ok; base += 32) {
                    const bool more = base + 32 + lane < ns;
                    const uint32_t nk = more ? pk[sb + base + 32 + lane] : 0u;
                    const unsigned long long nm0 = more ? pm[2 * (sb + base + 32 + lane)] : 0ull;
                    const unsigned long long nm1 = more ? pm[2 * (sb + base + 32 + lane) + 1] : 0ull;
                    unsigned long long nh0 = nm0, nh1 = nm1;
                    if (tier) {
                        nh0 = more ? ph[2 * (sb + base + 32 + lane)] : 0ull;
                        nh1 = more ? ph[2 * (sb + base + 32 + lane) + 1] : 0ull;
                    }
                    const uint32_t cnt = ns - base < 32 ? ns - base : 32;
                    for (uint32_t j = 0; j < cnt && ok; ++j) {
                        const int64_t K = __shfl_sync(0xffffffffu, ck, j);
                        const unsigned long long m0 = __shfl_sync(0xffffffffu, cm0, j);
                        const unsigned long long m1 = __shfl_sync(0xffffffffu, cm1, j);
                        const unsigned long long h0 = __shfl_sync(0xffffffffu, ch0, j);
                        const unsigned long long h1 = __shfl_sync(0xffffffffu, ch1, j);
                        const bool lean = tier && (h0 | h1) == 0ull;
                        // the step's chunks in runs that end at stage boundaries
                        // (one chunk per run when an operand is sparsified)
                        for (int kc = 0; kc < CHUNKS && ok;) {
                            int m = 1;
                            if (lane == 0) {
                                if (!BAND) m = CG;
                                issue(K, kc, m, m0, m1, h0, h1, lean);
                            }
                            m = __shfl_sync(0xffffffffu, m, 0);
                            ok = __shfl_sync(0xffffffffu, ok, 0);
                            kc += m;
                        }
                    }
                    ck = nk;
                    cm0 = nm0;
                    cm1 = nm1;
                    ch0 = nh0;
                    ch1 = nh1;
                }
            } else {
                // sub-leaf cull: a mask pair per (step, K-chunk); chunks whose
                // slice products were all culled are not loaded at all
                // (the full-split masks are per step, shared by its slices)
                const uint32_t nit = ns * CHUNKS;
                auto ld = [&](uint32_t it, uint32_t& kk, unsigned long long& a,
                              unsigned long long& b, unsigned long long& ha,
                              unsigned long long& hb) {
                    if (it < nit) {
                        const uint64_t st = sb + it / CHUNKS;
                        kk = pk[st];
                        a = pm[2 * (st * CHUNKS + it % CHUNKS)];
                        b = pm[2 * (st * CHUNKS + it % CHUNKS) + 1];
                        ha = tier ? ph[2 * st] & a : a;
                        hb = tier ? ph[2 * st + 1] & b : b;
                    } else {
                        kk = 0u;
                        a = b = ha = hb = 0ull;
                    }
                };
                uint32_t ck;
                unsigned long long cm0, cm1, ch0, ch1;
                ld(lane, ck, cm0, cm1, ch0, ch1);
                for (uint32_t base = 0; base < nit && ok; base += 32) {
                    uint32_t nk;
                    unsigned long long nm0, nm1, nh0, nh1;
                    ld(base + 32 + lane, nk, nm0, nm1, nh0, nh1);
                    const uint32_t cnt = nit - base < 32 ? nit - base : 32;
                    for (uint32_t j = 0; j < cnt && ok; ++j) {
                        const int64_t K = __shfl_sync(0xffffffffu, ck, j);
                        const unsigned long long m0 = __shfl_sync(0xffffffffu, cm0, j);
                        const unsigned long long m1 = __shfl_sync(0xffffffffu, cm1, j);
                        const unsigned long long h0 = __shfl_sync(0xffffffffu, ch0, j);
                        const unsigned long long h1 = __shfl_sync(0xffffffffu, ch1, j);
                        if ((m0 | m1) == 0ull) continue;
                        const bool lean = tier && (h0 | h1) == 0ull;
                        if (lane == 0) issue(K, (int)((base + j) % CHUNKS), 1, m0, m1, h0, h1, lean);
                        ok = __shfl_sync(0xffffffffu, ok, 0);
                    }
                    ck = nk;
                    cm0 = nm0;
                    cm1 = nm1;
                    ch0 = nh0;
                    ch1 = nh1;
                }
            }
            // a stage never spans two tiles
            if (lane == 0 && fill > 0) close_stage();
        }
    } else if (warp == 1) {
        // --------------------------------------------------------------- MMA
        // Lane 0 alone: per stage one wait and one commit.  Iteration i of a
        // tile (its i-th loaded K-chunk: every chunk of every step, or with
        // the sub-leaf cull every chunk with a kept slice product) opens a
        // new TMEM chunk when i % kChunkIters == 0 and closes it at the
        // chunk's last iteration; a tile without steps is skipped.
        if (lane == 0) {
            unsigned long long stage_it = 0;
            uint32_t ccount = 0;  // chunks opened so far (selects the TMEM buffer)
            bool ok = true;
            const uint32_t dis0[4] = {0u, 0u, 0u, 0u};
            uint32_t dacc = tmem;
            int pi = 0;
            uint32_t tq = 0;
            while (ok) {
                const int slot = (int)(tq % kTQ);
                const uint32_t tph = (tq / kTQ) & 1;
                if (!wait_bar(smem_u32(&bar_tqf[slot]), tph, &abort_flag, status, bt.wait_ns)) {
                    ok = false;
                    break;
                }
                const int k = tq_id[slot];
                mbar_arrive(smem_u32(&bar_tqe[slot]));
                ++tq;
                if (k < 0) break;
                product_of(k, pi);
                if (sp_skip[pi]) continue;
                const TcProd& q = bt.prods[pi];
                const uint32_t iters = q.iters[tile_at(k - q.base, q.tr, q.tc)];
                if (iters == 0) continue;
                uint32_t i = 0;
                while (i < iters && ok) {
                    const int s = (int)(stage_it % ST);
                    const uint32_t ph = (uint32_t)((stage_it / ST) & 1);
                    if (!wait_bar(smem_u32(&bar_full[s]), ph, &abort_flag, status, bt.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const int ngs = (int)st_count[s];
                    consumed_s = stage_it + 1;
                    const uint32_t sbuf = smem_u32(stages + (size_t)s * T::kStage);
                    constexpr unsigned long long kRep =
                        TL == 8   ? 0x0101010101010101ull
                        : TL == 4 ? 0x0000000001010101ull
                        : TL == 2 ? 0x0000000000000101ull
                                  : 0x0000000000000001ull;
                    constexpr unsigned long long kFull =
                        (unsigned long long)((1u << TL) - 1u) * kRep;
                    // The MMAs of one pass set over the products of masks (r0,
                    // r1), for ngrp groups of c chunks each, the first at unit
                    // u0 and the others every `stride` units: MODE 3 = all three
                    // of the split (lo*hi, hi*lo, hi*hi; hi*hi alone for single
                    // TF32), 1 = hi*hi, 2 = the cross terms.  Chunk j of a group
                    // at unit x has its high parts at unit x + j and its low
                    // parts at unit x + c + j.  Runs of column leaves with the
                    // same kept row leaves: a column y starts a run when its row
                    // mask is non-zero and differs from column y-1's.  Uniform
                    // halves (the common case on dense blocks) give one run
                    // directly.
                    auto passes = [&](unsigned long long r0, unsigned long long r1, auto mode_c,
                                      int u0, int c, int ngrp, int stride) {
                        constexpr int MODE = decltype(mode_c)::value;
                        constexpr bool kCross = PREC != SPAMM_PREC_TF32 && MODE != 1;
                        constexpr bool kHiHi = MODE != 2;
                        // the MMAs of every chunk of the groups over one run: N
                        // = the run's columns, TMEM columns from d, B rows from
                        // boff, lane mask dis
                        auto run_mmas = [&](uint32_t d, uint32_t boff, uint32_t idesc,
                                            const uint32_t (&dis)[4], bool masked) {
                            for (int gq = 0; gq < ngrp; ++gq) {
                                const int x = u0 + gq * stride;
#pragma unroll
                                for (int j = 0; j < CG; ++j) {
                                    if (j >= c) break;
                                    const uint32_t a_hi = sbuf + (uint32_t)(x + j) * T::kSlice;
                                    const uint32_t a_lo = a_hi + (uint32_t)c * T::kSlice;
                                    const uint32_t b_hi = sbuf + (uint32_t)(U * T::kSlice) +
                                                          (uint32_t)(x + j) * 2 * T::kSlice + boff;
                                    const uint32_t b_lo = b_hi + (uint32_t)c * 2 * T::kSlice;
#pragma unroll
                                    for (int kk = 0; kk < 16 / T::kKInstr; ++kk) {
                                        const uint32_t koff = (uint32_t)kk * 256u;
                                        const uint64_t ah = make_desc(a_hi + koff, 128, T::kSBO);
                                        const uint64_t bh = make_desc(b_hi + koff, 128, T::kSBO);
                                        if (kCross) {
                                            const uint64_t al = make_desc(a_lo + koff, 128, T::kSBO);
                                            const uint64_t bl = make_desc(b_lo + koff, 128, T::kSBO);
                                            if (masked) {
                                                mma<PREC>(d, al, bh, idesc, dis, 1u);
                                                mma<PREC>(d, ah, bl, idesc, dis, 1u);
                                            } else {
                                                mma_all<PREC>(d, al, bh, idesc, 1u);
                                                mma_all<PREC>(d, ah, bl, idesc, 1u);
                                            }
                                        }
                                        if (kHiHi) {
                                            if (masked) mma<PREC>(d, ah, bh, idesc, dis, 1u);
                                            else mma_all<PREC>(d, ah, bh, idesc, 1u);
                                        }
                                    }
                                }
                            }
                        };
                        if (r0 == kFull && r1 == kFull) {
                            // every product of the step: one 128 x 256 MMA per
                            // pass, no masks
                            run_mmas(dacc, 0u, make_idesc(T::kAB, 128, 256), dis0, false);
                            return;
                        }
                        const uint32_t x0 = (uint32_t)r0 & 0xFFu;
                        const uint32_t x1 = (uint32_t)r1 & 0xFFu;
                        const bool u0m = r0 == (unsigned long long)x0 * kRep;
                        const bool u1m = r1 == (unsigned long long)x1 * kRep;
                        uint32_t starts, nz;
                        if (u0m && u1m) {
                            starts = (x0 ? 1u : 0u) | ((x1 && x1 != x0) ? (1u << TL) : 0u);
                            nz = (x0 ? (1u << TL) - 1u : 0u) | (x1 ? ((1u << TL) - 1u) << TL : 0u);
                        } else {
                            starts = 0u;
                            nz = 0u;
                            uint32_t prev = 0u;
#pragma unroll
                            for (int yy = 0; yy < TLC; ++yy) {
                                const uint32_t xm =
                                    yy < TL ? (uint32_t)(r0 >> (8 * yy)) & 0xFFu
                                            : (uint32_t)(r1 >> (8 * (yy - TL))) & 0xFFu;
                                if (xm) nz |= 1u << yy;
                                if (xm && xm != prev) starts |= 1u << yy;
                                prev = xm;
                            }
                        }
                        while (starts) {
                            const int y = __ffs(starts) - 1;
                            starts &= starts - 1;
                            const uint32_t stop = (starts | ~nz) & ~((2u << y) - 1u);
                            const int yend = stop ? min(__ffs(stop) - 1, TLC) : TLC;
                            const int len = yend - y;
                            const uint32_t xm = y < TL ? (uint32_t)(r0 >> (8 * y)) & 0xFFu
                                                       : (uint32_t)(r1 >> (8 * (y - TL))) & 0xFFu;
                            // disable-output-lane bits: row r of the tile is
                            // lane r, and a dropped row leaf x masks its b rows
                            uint32_t dis[4];
#pragma unroll
                            for (int w = 0; w < 4; ++w) {
                                uint32_t v = 0;
                                if (LEAF <= 32) {
#pragma unroll
                                    for (int q = 0; q < 32 / LEAF; ++q) {
                                        const int x = w * (32 / LEAF) + q;
                                        if (!((xm >> x) & 1u))
                                            v |= (LEAF == 32 ? 0xFFFFFFFFu : (0xFFFFu << (16 * q)));
                                    }
                                } else {
                                    const int x = (w * 32) / LEAF;
                                    if (!((xm >> x) & 1u)) v = 0xFFFFFFFFu;
                                }
                                dis[w] = v;
                            }
                            run_mmas(dacc + (uint32_t)(y * LEAF), (uint32_t)(y * (LEAF / 8)) * T::kSBO,
                                     make_idesc(T::kAB, 128, len * LEAF), dis, true);
                        }
                    };
                    // a new TMEM chunk at every kChunkIters-th K-chunk of a tile:
                    // wait until the epilogue has drained the buffer and left
                    // it zero (use k of a buffer waits for the (k+1)-th phase of
                    // its barrier: the first is the zeroing at the start)
                    auto open_chunk = [&]() -> bool {
                        const uint32_t ab = ccount & 1, aph = (ccount >> 1) & 1;
                        if (!wait_bar(smem_u32(&bar_acce[ab]), aph, &abort_flag, status, bt.wait_ns))
                            return false;
                        tc_fence_after();
                        dacc = tmem + ab * 256;
                        return true;
                    };
                    // Groups in stage order.  Consecutive groups with the same
                    // masks inside one TMEM chunk share one run analysis: with
                    // the same masks they are both lean or both full and, within
                    // a tile, all groups have the same chunk count, so they sit
                    // at a fixed stride of units.
                    for (int g = 0; g < ngs && ok;) {
                        const uint32_t rec = st_grp[s][g];
                        const int u0 = (int)(rec & 0xFFu), c = (int)((rec >> 8) & 0xFFu);
                        const unsigned long long m0 = st_mask[s][g][0], m1 = st_mask[s][g][1];
                        const unsigned long long h0 = st_hmask[s][g][0], h1 = st_hmask[s][g][1];
                        int g2 = g + 1;
                        int stride = 0;
                        const uint32_t room = kChunkIters - i % kChunkIters;   // chunks left in the TMEM chunk
                        while (g2 < ngs && (uint32_t)((g2 - g + 1) * c) <= room &&
                               st_mask[s][g2][0] == m0 && st_mask[s][g2][1] == m1 &&
                               st_hmask[s][g2][0] == h0 && st_hmask[s][g2][1] == h1) {
                            const int x = (int)(st_grp[s][g2] & 0xFFu);
                            if (g2 == g + 1) stride = x - u0;
                            else if (x - u0 != stride * (g2 - g)) break;
                            ++g2;
                        }
                        if (i % kChunkIters == 0 && !open_chunk()) {
                            ok = false;
                            break;
                        }
                        const int ngrp = g2 - g;
                        if (h0 == m0 && h1 == m1) {
                            passes(m0, m1, std::integral_constant<int, 3>{}, u0, c, ngrp, stride);
                        } else {
                            // precision chosen by norm: hi * hi for every kept
                            // product, the cross terms for the full-split ones
                            passes(m0, m1, std::integral_constant<int, 1>{}, u0, c, ngrp, stride);
                            if ((h0 | h1) != 0ull)
                                passes(h0, h1, std::integral_constant<int, 2>{}, u0, c, ngrp, stride);
                        }
                        i += (uint32_t)(ngrp * c);
                        const uint32_t last = i - 1;
                        if (last % kChunkIters == kChunkIters - 1 || last == iters - 1) {
                            tc_commit(smem_u32(&bar_accf[ccount & 1]));
                            ++ccount;
                        }
                        g = g2;
                    }
                    // the stage's MMAs have read its shared memory once they complete
                    tc_commit(smem_u32(&bar_empty[s]));
                    ++stage_it;
                }
            }
            // drain: every MMA issued so far has completed before TMEM is freed
            tc_commit(smem_u32(&bar_drain));
            wait_drain(smem_u32(&bar_drain), 0, status);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- epilogue
        const int qq = warp & 3;                 // TMEM lane quarter this warp may access
        const int hcol = (warp - 2) >> 2;        // which 128 columns of the 256
        // both chunk buffers start at zero (the MMAs accumulate onto them)
        for (uint32_t ab = 0; ab < 2; ++ab) {
            const uint32_t taddr =
                tmem + ((uint32_t)(qq * 32) << 16) + ab * 256 + (uint32_t)(hcol * 128);
#pragma unroll
            for (int cc = 0; cc < 128; cc += 32) tmem_zero32(taddr + (uint32_t)cc);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(smem_u32(&bar_acce[0]));
            mbar_arrive(smem_u32(&bar_acce[1]));
        }
        uint32_t ccount = 0;
        bool ok = true;
        int pi = 0;
        uint32_t tq = 0;
        while (ok) {
            const int slot = (int)(tq % kTQ);
            const uint32_t tph = (tq / kTQ) & 1;
            int k = -1;
            bool got = true;
            if (lane == 0) {
                got = wait_bar(smem_u32(&bar_tqf[slot]), tph, &abort_flag, status, bt.wait_ns);
                if (got) k = tq_id[slot];
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (!got) {
                ok = false;
                break;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_tqe[slot]));
            ++tq;
            if (k < 0) break;
            product_of(k, pi);
            if (sp_skip[pi]) continue;
            const TcProd& q = bt.prods[pi];
            const int u = tile_at(k - q.base, q.tr, q.tc);
            const uint32_t nch = chunks_of(q.iters[u]);
            if (nch == 0) {
                // no kept product: C = alpha * 0 + beta * C, written row-wise by
                // the 256 epilogue threads (a warp stores 512 contiguous bytes)
                float* const Cp = q.C;
                const int64_t ldc = q.ldc, n = q.n;
                const float alpha = q.alpha, beta = q.beta;
                const int64_t R0 = (int64_t)(u / q.tc) * 128, C0 = (int64_t)(u % q.tc) * 256;
                const int e = (warp - 2) * 32 + lane;
                const bool vec = ((ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(Cp) & 15) == 0);
                const float z = alpha * 0.f;
                for (int idx = e; idx < 128 * 64; idx += kEpiWarps * 32) {
                    const int64_t row = R0 + idx / 64, col = C0 + 4 * (idx % 64);
                    if (row >= n || col >= n) continue;
                    float* dst = Cp + row * ldc + col;
                    if (vec && col + 3 < n) {
                        float4 o = make_float4(z, z, z, z);
                        if (beta != 0.f) {
                            const float4 old = *reinterpret_cast<const float4*>(dst);
                            o.x = fmaf(beta, old.x, z);
                            o.y = fmaf(beta, old.y, z);
                            o.z = fmaf(beta, old.z, z);
                            o.w = fmaf(beta, old.w, z);
                        }
                        *reinterpret_cast<float4*>(dst) = o;
                    } else {
                        for (int c = 0; c < 4 && col + c < n; ++c)
                            dst[c] = beta != 0.f ? fmaf(beta, dst[c], z) : z;
                    }
                }
                continue;
            }
            float master[128];
#pragma unroll
            for (int v = 0; v < 128; ++v) master[v] = 0.f;
            for (uint32_t c = 0; c < nch; ++c, ++ccount) {
                const uint32_t ab = ccount & 1;
                const uint32_t aph = (ccount >> 1) & 1;
                if (!wait_bar(smem_u32(&bar_accf[ab]), aph, &abort_flag, status, bt.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr =
                    tmem + ((uint32_t)(qq * 32) << 16) + ab * 256 + (uint32_t)(hcol * 128);
#pragma unroll
                for (int cc = 0; cc < 128; cc += 32) {
                    uint32_t r[32];
                    tmem_ld32(taddr + (uint32_t)cc, r);
#pragma unroll
                    for (int v = 0; v < 32; ++v) master[cc + v] += __uint_as_float(r[v]);
                    tmem_zero32(taddr + (uint32_t)cc);   // ready for the buffer's next chunk
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bar_acce[ab]));
            }
            if (!ok) break;
            float* const Cp = q.C;
            const int64_t ldc = q.ldc, n = q.n;
            // FP16 split: the products come scaled by 2^(kA + kB); undoing it
            // is exact (powers of two) unless the result leaves the float range
            float alpha = q.alpha;
            if constexpr (PREC == SPAMM_PREC_F16X3) {
                const float2 us = sp_uns[pi];
                alpha *= us.x;
#pragma unroll
                for (int v = 0; v < 128; ++v) master[v] *= us.y;
            }
            const float beta = q.beta;
            const int64_t row = (int64_t)(u / q.tc) * 128 + qq * 32 + lane;
            const int64_t col0 = (int64_t)(u % q.tc) * 256 + hcol * 128;
            if (row < n && col0 < n) {
                float* crow = Cp + row * ldc + col0;
                const bool vec = ((ldc & 3) == 0) &&
                                 ((reinterpret_cast<uintptr_t>(Cp) & 15) == 0) &&
                                 (col0 + 128 <= n);
                if (vec) {
#pragma unroll
                    for (int v = 0; v < 32; ++v) {
                        float4 o = make_float4(alpha * master[4 * v], alpha * master[4 * v + 1],
                                               alpha * master[4 * v + 2],
                                               alpha * master[4 * v + 3]);
                        float4* dst = reinterpret_cast<float4*>(crow) + v;
                        if (beta != 0.f) {
                            const float4 old = *dst;
                            o.x = fmaf(beta, old.x, o.x);
                            o.y = fmaf(beta, old.y, o.y);
                            o.z = fmaf(beta, old.z, o.z);
                            o.w = fmaf(beta, old.w, o.w);
                        }
                        *dst = o;
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < 128; ++v) {
                        if (col0 + v < n) {
                            float o = alpha * master[v];
                            if (beta != 0.f) o = fmaf(beta, crow[v], o);
                            crow[v] = o;
                        }
                    }
                }
            }
        }
    }

    // ------------------------------------------------------------ teardown
    __syncthreads();
    if (abort_flag && threadIdx.x == 0) {
        // stages whose copies were issued but never consumed must land
        // before the block exits
        for (unsigned long long it = consumed_s; it < issued_s; ++it) {
            const int s = (int)(it % ST);
            const uint32_t ph = (uint32_t)((it / ST) & 1);
            const uint64_t t0 = gtimer();
            while (!mbar_try_wait(smem_u32(&bar_full[s]), ph) && gtimer() - t0 < kWaitNs) {
            }
        }
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                     : "memory");
    }
}

template <int LEAF, int PREC, bool BAND>
cudaError_t launch_b(spamm_ctx* ctx, const TcBatch& bt, cudaStream_t stream) {
    using T = PrecTraits<PREC>;
    const size_t smem = 1024 + (size_t)T::kStages * T::kStage;
    cudaError_t e = cudaFuncSetAttribute(k_leaf_tc<LEAF, PREC, BAND>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int items = bt.total - bt.first;
    const int grid = items < ctx->sm_count ? items : ctx->sm_count;
    if (grid <= 0) return cudaSuccess;
    k_leaf_tc<LEAF, PREC, BAND><<<grid, kThreads, smem, stream>>>(bt);
    return cudaGetLastError();
}

template <int LEAF, int PREC>
cudaError_t launch_t(spamm_ctx* ctx, const TcBatch& bt, bool band, cudaStream_t s) {
    return band ? launch_b<LEAF, PREC, true>(ctx, bt, s) : launch_b<LEAF, PREC, false>(ctx, bt, s);
}

}  // namespace

// The launch table for jobs[0, count) (count <= kMaxBatch); returns whether
// any operand is sparsified (the BAND kernels).
static bool fill_batch(spamm_ctx* ctx, const LeafJob* jobs, int count, TcBatch& bt) {
    memset(&bt, 0, sizeof(bt));
    bt.count = count;
    bt.status = &ctx->ctl->status;
    bt.wait_ns = ctx->wait_ns > 0 ? (unsigned long long)ctx->wait_ns : kWaitNs;
    bt.ctr = &ctx->ctl->tile_ctr;
    int base = 0;
    bool band = false;
    for (int i = 0; i < bt.count; ++i) {
        const LeafJob& jb = jobs[i];
        TcProd& q = bt.prods[i];
        for (int h = 0; h < 2; ++h) {
            q.pa[h] = jb.A->packA[h] ? jb.A->packA[h] : jb.A->packA[0];
            q.pb[h] = jb.B->packB[h] ? jb.B->packB[h] : jb.B->packB[0];
        }
        q.nlp = jb.A->nlp;
        q.C = jb.C;
        q.ldc = jb.ldc;
        q.n = jb.A->n;
        q.alpha = jb.alpha;
        q.beta = jb.beta;
        q.ctl = jb.sub->ctl;
        q.pool = jb.sub->pool;
        q.off = jb.sub->tile_off;
        q.steps = jb.sub->tile_steps;
        q.iters = jb.sub->tile_iters;
        q.gmax = jb.sub->need + 2 * jb.A->nb;
        q.tier = ctx->cfg.tier_bits > 0 ? 1 : 0;
        if (jb.A->sparse) {
            const BandView v = band_view(jb.A);
            q.a_lo = v.imin;
            q.a_hi = v.imax;
            q.a_off = v.aoff;
            band = true;
        }
        if (jb.B->sparse) {
            const BandView v = band_view(jb.B);
            q.b_lo = v.kmin;
            q.b_hi = v.kmax;
            q.b_off = v.boff;
            band = true;
        }
        q.sl = (jb.A->slices && jb.B->slices) ? jb.A->slices : 1;
        q.tr = tile_rows(jb.A);
        q.tc = tile_cols(jb.A);
        q.S = jb.sub->last_S;
        q.base = base;
        base += q.tr * q.tc;
    }
    bt.total = base;
    return band;
}

// On stream s; zero_ctr: clear the launch's work-item counter first (the
// per-band counters of a banded launch start at zero with the control block).
static cudaError_t dispatch(spamm_ctx* ctx, const TcBatch& bt, bool band, cudaStream_t s,
                            bool zero_ctr) {
    const int p = ctx->cfg.precision;
    const int b = ctx->cfg.leaf;
    // every launch deals its work items out from a counter that starts at zero
    cudaError_t e = cudaSuccess;
    if (zero_ctr) e = cudaMemsetAsync(bt.ctr, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (b == 16) {
        if (p == SPAMM_PREC_TF32X3) e = launch_t<16, SPAMM_PREC_TF32X3>(ctx, bt, band, s);
        else if (p == SPAMM_PREC_TF32) e = launch_t<16, SPAMM_PREC_TF32>(ctx, bt, band, s);
        else if (p == SPAMM_PREC_BF16X3) e = launch_t<16, SPAMM_PREC_BF16X3>(ctx, bt, band, s);
        else e = launch_t<16, SPAMM_PREC_F16X3>(ctx, bt, band, s);
    } else if (b == 32) {
        if (p == SPAMM_PREC_TF32X3) e = launch_t<32, SPAMM_PREC_TF32X3>(ctx, bt, band, s);
        else if (p == SPAMM_PREC_TF32) e = launch_t<32, SPAMM_PREC_TF32>(ctx, bt, band, s);
        else if (p == SPAMM_PREC_BF16X3) e = launch_t<32, SPAMM_PREC_BF16X3>(ctx, bt, band, s);
        else e = launch_t<32, SPAMM_PREC_F16X3>(ctx, bt, band, s);
    } else if (b == 64) {
        if (p == SPAMM_PREC_TF32X3) e = launch_t<64, SPAMM_PREC_TF32X3>(ctx, bt, band, s);
        else if (p == SPAMM_PREC_TF32) e = launch_t<64, SPAMM_PREC_TF32>(ctx, bt, band, s);
        else if (p == SPAMM_PREC_BF16X3) e = launch_t<64, SPAMM_PREC_BF16X3>(ctx, bt, band, s);
        else e = launch_t<64, SPAMM_PREC_F16X3>(ctx, bt, band, s);
    } else if (b == 128) {
        if (p == SPAMM_PREC_TF32X3) e = launch_t<128, SPAMM_PREC_TF32X3>(ctx, bt, band, s);
        else if (p == SPAMM_PREC_TF32) e = launch_t<128, SPAMM_PREC_TF32>(ctx, bt, band, s);
        else if (p == SPAMM_PREC_BF16X3) e = launch_t<128, SPAMM_PREC_BF16X3>(ctx, bt, band, s);
        else e = launch_t<128, SPAMM_PREC_F16X3>(ctx, bt, band, s);
    } else {
        e = cudaErrorNotSupported;
    }
    return e;
}

// All jobs share the context's leaf size and precision.  At most kMaxBatch
// products go into one launch.
cudaError_t launch_leaf_tc_jobs(spamm_ctx* ctx, const LeafJob* jobs, int count) {
    for (int j0 = 0; j0 < count; j0 += kMaxBatch) {
        TcBatch bt;
        const bool band =
            fill_batch(ctx, jobs + j0, count - j0 < kMaxBatch ? count - j0 : kMaxBatch, bt);
        const cudaError_t e = dispatch(ctx, bt, band, ctx->stream, true);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One product in `bands` launches, each a run of whole tile-row groups (the
// work order walks kGroupRows tile rows at a time), so that after each
// launch the rows of C it finished are final; `done` is told which rows
// (e.g. to start copying them out while the next band computes).  Every
// tile is computed by exactly one launch, as in the single launch, so C is
// the same bit for bit.
cudaError_t launch_leaf_tc_banded(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B,
                                  float alpha, float beta, float* C, int64_t ldc, int bands,
                                  cudaError_t (*done)(void*, int64_t, int64_t, cudaStream_t),
                                  void* user) {
    LeafJob jb{A, B, ctx, alpha, beta, C, ldc};
    TcBatch bt;
    const bool band = fill_batch(ctx, &jb, 1, bt);
    const int tr = bt.prods[0].tr, tc = bt.prods[0].tc;
    const int groups = (tr + kGroupRows - 1) / kGroupRows;
    constexpr int kMaxBands = (int)(sizeof(DevCtl::band_ctr) / sizeof(unsigned int));
    if (bands > groups) bands = groups;
    if (bands > kMaxBands) bands = kMaxBands;
    if (bands < 1) bands = 1;
    // Bands alternate between the context stream and a side stream, so that
    // the next band's blocks take the SMs a band's last wave leaves idle (the
    // bands write disjoint rows of C); each has its own work-item counter.
    cudaStream_t side = ctx->aux[1];
    cudaError_t e = cudaEventRecord(ctx->fork_ev, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ctx->fork_ev, 0);
    if (e != cudaSuccess) return e;
    // band i ends at group ceil(groups (i+1) / bands): the remainder goes to
    // the front, so the last band, whose copy-out nothing hides, is the
    // smallest
    int g0 = 0;
    for (int i = 0; i < bands; ++i) {
        const int g1 = (int)(((int64_t)groups * (i + 1) + bands - 1) / bands);
        cudaStream_t s = (i & 1) ? side : ctx->stream;
        bt.first = g0 * kGroupRows * tc;
        bt.total = (g1 * kGroupRows < tr ? g1 * kGroupRows : tr) * tc;
        bt.ctr = &ctx->ctl->band_ctr[i];
        e = dispatch(ctx, bt, band, s, false);
        if (e != cudaSuccess) return e;
        const int64_t r0 = (int64_t)g0 * kGroupRows * kTileRows;
        const int64_t r1 = std::min<int64_t>((int64_t)g1 * kGroupRows * kTileRows, A->n);
        if (done && r1 > r0) {
            e = done(user, r0, r1, s);
            if (e != cudaSuccess) return e;
        }
        g0 = g1;
    }
    // the context stream continues after every band
    e = cudaEventRecord(ctx->aux_ev[1], side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->aux_ev[1], 0);
    return e;
}

cudaError_t launch_leaf_tc(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B, float alpha,
                           float beta, float* C, int64_t ldc) {
    LeafJob jb{A, B, ctx, alpha, beta, C, ldc};
    return launch_leaf_tc_jobs(ctx, &jb, 1);
}

}  // namespace spamm
