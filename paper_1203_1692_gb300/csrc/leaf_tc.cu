// Stage 4 on the tcgen05 tensor cores: C_IJ = alpha * sum_{kept K, ascending}
// A_IK B_KJ + beta * C_IJ (Algorithm 1, numeric part), with FP32
// accumulation in tensor memory.
//
// Work unit: one 128 x 128 C tile = TL x TL leaf pairs (TL = 128 / b), and the
// tile's steps (K, mask) in ascending K from the grouping stage.  For every
// step and every 16-wide K chunk the tile needs A's 128 x 16 slice (the TL
// row leaves of the tile, column leaf K) and B's 16 x 128 slice; both were
// stored by the norm build as contiguous runs already in the no-swizzle
// K-major layout of tcgen05 (8-row x 16-byte core matrices), so one 1-D bulk
// copy per operand moves them into shared memory.
//
// Exactness of the cull: a kept leaf product (x, K, y) must be added and a
// culled one must not.  One MMA over a run of consecutive column leaves
// y0..y0+len-1 that share the same set of kept row leaves uses the MMA's
// disable-output-lane mask to leave the accumulator rows (TMEM lanes) of the
// culled row leaves untouched, so the tensor core adds exactly the kept
// products.  N = len * b (16..128), M = 128.
//
// Precisions: TF32X3 splits each operand into a TF32 high part and a TF32
// low part (a - hi) and adds lo*hi + hi*lo + hi*hi; TF32 uses hi*hi only;
// BF16X3 does the same with bfloat16 parts on kind::f16.  All accumulate in
// FP32.
//
// Two-level accumulation: the tensor core's FP32 accumulation rounds less
// carefully than an IEEE add, and a C tile can chain thousands of MMAs.  So
// the MMAs of a tile are cut into chunks of at most kChunkIters K-chunks;
// every chunk starts from a zeroed TMEM accumulator, and the epilogue warps
// add the finished chunk into a master FP32 accumulator held in registers
// (one row of 128 values per thread) with round-to-nearest adds.  Chunks are
// added in ascending K, so the result stays deterministic.
//
// Tile order: consecutive work items walk down a group of kGroupRows tile
// rows before moving one tile column right, so the tiles in flight at once
// share A slices (same rows) and B slices (same columns) in L2.
//
// Roles (192 threads): warp 0 lane 0 issues the bulk copies into a ring of
// shared-memory stages; warp 1 owns the TMEM allocation and its lane 0
// issues the MMAs and commits; warps 2-5 move the double-buffered 128 x 128
// chunk accumulators out of TMEM, sum them, apply alpha/beta and store C.  Every wait on an
// mbarrier gives up after one second, raises the timeout status and lets
// the block drain its copies and MMAs, free TMEM and exit.
#include <cuda_bf16.h>

#include "spamm_internal.cuh"

namespace spamm {
namespace {

constexpr int kThreads = 192;
constexpr int kChunkIters = 8;  // K-chunks of 16 per TMEM accumulation chunk
constexpr int kGroupRows = 8;   // tile rows walked together (L2 reuse)
constexpr uint32_t kZeroBytes = 4096;
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s

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
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
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

// Bounded wait: true when the phase completed, false after a timeout (or
// when another role already gave up).
__device__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                         unsigned int* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
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
__device__ __forceinline__ uint32_t make_idesc(uint32_t ab, int M, int N) {
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Work item k -> tile index (row-major over tps x tps tiles), grouped by
// kGroupRows tile rows.
__device__ __forceinline__ int tile_at(int k, int tps) {
    const int span = kGroupRows * tps;
    const int g = k / span;
    const int rows = min(kGroupRows, tps - g * kGroupRows);
    const int w = k - g * span;
    return (g * kGroupRows + w % rows) * tps + w / rows;
}

__device__ __forceinline__ uint32_t chunks_of(uint32_t iters) {
    return iters == 0 ? 1u : (iters + kChunkIters - 1) / kChunkIters;
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    const uint32_t (&dis)[4], uint32_t acc) {
    if (PREC == SPAMM_PREC_BF16X3) {
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

template <int PREC>
struct PrecTraits {
    static constexpr int kEsize = PREC == SPAMM_PREC_BF16X3 ? 2 : 4;
    static constexpr int kParts = PREC == SPAMM_PREC_TF32 ? 1 : 2;      // arrays per role
    static constexpr int kSlice = 128 * 16 * kEsize;                   // bytes of one 128x16 slice
    static constexpr int kStage = 2 * kParts * kSlice;                  // A and B slices
    static constexpr int kStages = PREC == SPAMM_PREC_TF32X3 ? 4 : 6;
    static constexpr int kKInstr = PREC == SPAMM_PREC_BF16X3 ? 16 : 8;  // K per MMA
    static constexpr uint32_t kSBO = 8 * 16 * kEsize;                   // row-group stride
    static constexpr uint32_t kAB = PREC == SPAMM_PREC_BF16X3 ? 1u : 2u;
};

struct TcArgs {
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
    int tps, tiles, S;
};

template <int LEAF, int PREC>
__global__ void __launch_bounds__(kThreads, 1) k_leaf_tc(TcArgs p) {
    using T = PrecTraits<PREC>;
    constexpr int TL = 128 / LEAF;
    constexpr int CHUNKS = LEAF / 16;
    constexpr int ST = T::kStages;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[ST], bar_empty[ST], bar_accf[2], bar_acce[2],
        bar_drain;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    __shared__ unsigned long long issued_s, consumed_s;

    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* zero = base;
    unsigned char* stages = base + kZeroBytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned int* status = &p.ctl->status;
    if (p.ctl->status & (ST_OVERFLOW | ST_NONFINITE)) return;

    for (int i = threadIdx.x; i < (int)(kZeroBytes / 16); i += kThreads)
        reinterpret_cast<uint4*>(zero)[i] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bar_accf[b]), 1);
            mbar_init(smem_u32(&bar_acce[b]), 4);
        }
        mbar_init(smem_u32(&bar_drain), 1);
        abort_flag = 0;
        issued_s = consumed_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(256u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t* pk = reinterpret_cast<const uint32_t*>(p.pool + p.ctl->pk_off);
    const unsigned long long* pm =
        reinterpret_cast<const unsigned long long*>(p.pool + p.ctl->pm_off);

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            unsigned long long it = 0;
            bool ok = true;
            for (int k = blockIdx.x; k < p.tiles && ok; k += gridDim.x) {
                const int u = tile_at(k, p.tps);
                const int64_t srow = (int64_t)(u / p.tps) * TL;
                const int64_t scol = (int64_t)(u % p.tps) * TL;
                const uint32_t ns = p.steps[u];
                const uint64_t sb = (uint64_t)p.off[u] * p.S;
                for (uint32_t st = 0; st < ns && ok; ++st) {
                    const int64_t K = pk[sb + st];
                    for (int kc = 0; kc < CHUNKS && ok; ++kc, ++it) {
                        const int s = (int)(it % ST);
                        const uint32_t ph = (uint32_t)((it / ST) & 1);
                        if (!wait_bar(smem_u32(&bar_empty[s]), ph ^ 1, &abort_flag, status)) {
                            ok = false;
                            break;
                        }
                        const uint32_t full = smem_u32(&bar_full[s]);
                        mbar_expect_tx(full, T::kStage);
                        const int64_t row = (K * CHUNKS + kc) * p.nlp;
                        unsigned char* sbuf = stages + (size_t)s * T::kStage;
                        const size_t piece = (size_t)LEAF * 16 * T::kEsize;
#pragma unroll
                        for (int part = 0; part < T::kParts; ++part) {
                            bulk_g2s(smem_u32(sbuf + part * T::kSlice),
                                     static_cast<const unsigned char*>(p.pa[part]) +
                                         (size_t)(row + srow) * piece,
                                     T::kSlice, full);
                            bulk_g2s(smem_u32(sbuf + (T::kParts + part) * T::kSlice),
                                     static_cast<const unsigned char*>(p.pb[part]) +
                                         (size_t)(row + scol) * piece,
                                     T::kSlice, full);
                        }
                        issued_s = it + 1;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            unsigned long long it = 0;
            uint32_t ccount = 0;  // chunks issued so far (selects the TMEM buffer)
            bool ok = true;
            const uint64_t zdesc = make_desc(smem_u32(zero), 128, 256);
            const uint32_t dis0[4] = {0u, 0u, 0u, 0u};
            for (int k = blockIdx.x; k < p.tiles && ok; k += gridDim.x) {
                const int u = tile_at(k, p.tps);
                const uint32_t ns = p.steps[u];
                const uint64_t sb = (uint64_t)p.off[u] * p.S;
                const uint32_t iters = ns * CHUNKS;
                const uint32_t nch = chunks_of(iters);
                uint32_t st = 0;
                int kc = 0;
                for (uint32_t c = 0; c < nch && ok; ++c, ++ccount) {
                    const uint32_t ab = ccount & 1;
                    const uint32_t aph = (ccount >> 1) & 1;
                    if (!wait_bar(smem_u32(&bar_acce[ab]), aph ^ 1, &abort_flag, status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dacc = tmem + ab * 128;
                    // clear the chunk accumulator: 0 * 0 with the input accumulator off
                    mma<PREC>(dacc, zdesc, zdesc, make_idesc(T::kAB, 128, 128), dis0, 0u);
                    const uint32_t last = min(iters, (c + 1) * kChunkIters);
                    for (uint32_t i = c * kChunkIters; i < last && ok; ++i, ++it) {
                        const unsigned long long mask = pm[sb + st];
                        const int s = (int)(it % ST);
                        const uint32_t ph = (uint32_t)((it / ST) & 1);
                        if (!wait_bar(smem_u32(&bar_full[s]), ph, &abort_flag, status)) {
                            ok = false;
                            break;
                        }
                        consumed_s = it + 1;
                        tc_fence_after();
                        const uint32_t sbuf = smem_u32(stages + (size_t)s * T::kStage);
                        const uint32_t a_hi = sbuf, a_lo = sbuf + T::kSlice;
                        const uint32_t b_hi = sbuf + T::kParts * T::kSlice;
                        const uint32_t b_lo = b_hi + T::kSlice;
                        int y = 0;
                        while (y < TL) {
                            const uint32_t xm = (uint32_t)(mask >> (8 * y)) & 0xFFu;
                            if (!xm) {
                                ++y;
                                continue;
                            }
                            int len = 1;
                            while (y + len < TL &&
                                   ((uint32_t)(mask >> (8 * (y + len))) & 0xFFu) == xm)
                                ++len;
                            uint32_t dis[4];
#pragma unroll
                            for (int w = 0; w < 4; ++w) {
                                uint32_t v = 0;
#pragma unroll
                                for (int q = 0; q < 32 / LEAF; ++q) {
                                    const int x = w * (32 / LEAF) + q;
                                    if (!((xm >> x) & 1u))
                                        v |= (LEAF == 32 ? 0xFFFFFFFFu : (0xFFFFu << (16 * q)));
                                }
                                dis[w] = v;
                            }
                            const uint32_t idesc = make_idesc(T::kAB, 128, len * LEAF);
                            const uint32_t d = dacc + (uint32_t)(y * LEAF);
                            const uint32_t boff = (uint32_t)(y * (LEAF / 8)) * T::kSBO;
#pragma unroll
                            for (int kk = 0; kk < 16 / T::kKInstr; ++kk) {
                                const uint32_t koff = (uint32_t)kk * 256u;
                                const uint64_t ah = make_desc(a_hi + koff, 128, T::kSBO);
                                const uint64_t bh = make_desc(b_hi + boff + koff, 128, T::kSBO);
                                if (PREC != SPAMM_PREC_TF32) {
                                    const uint64_t al = make_desc(a_lo + koff, 128, T::kSBO);
                                    const uint64_t bl =
                                        make_desc(b_lo + boff + koff, 128, T::kSBO);
                                    mma<PREC>(d, al, bh, idesc, dis, 1u);
                                    mma<PREC>(d, ah, bl, idesc, dis, 1u);
                                }
                                mma<PREC>(d, ah, bh, idesc, dis, 1u);
                            }
                            y += len;
                        }
                        tc_commit(smem_u32(&bar_empty[s]));
                        if (++kc == CHUNKS) {
                            kc = 0;
                            ++st;
                        }
                    }
                    if (ok) tc_commit(smem_u32(&bar_accf[ab]));
                }
            }
            // drain: every MMA issued so far has completed before TMEM is freed
            tc_commit(smem_u32(&bar_drain));
            wait_bar(smem_u32(&bar_drain), 0, &abort_flag, status);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        uint32_t ccount = 0;
        bool ok = true;
        for (int k = blockIdx.x; k < p.tiles && ok; k += gridDim.x) {
            const int u = tile_at(k, p.tps);
            const uint32_t nch = chunks_of(p.steps[u] * CHUNKS);
            float master[128];
#pragma unroll
            for (int v = 0; v < 128; ++v) master[v] = 0.f;
            for (uint32_t c = 0; c < nch; ++c, ++ccount) {
                const uint32_t ab = ccount & 1;
                const uint32_t aph = (ccount >> 1) & 1;
                if (!wait_bar(smem_u32(&bar_accf[ab]), aph, &abort_flag, status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + ab * 128;
#pragma unroll
                for (int cc = 0; cc < 128; cc += 32) {
                    uint32_t r[32];
                    tmem_ld32(taddr + (uint32_t)cc, r);
#pragma unroll
                    for (int v = 0; v < 32; ++v) master[cc + v] += __uint_as_float(r[v]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bar_acce[ab]));
            }
            if (!ok) break;
            const int64_t row = (int64_t)(u / p.tps) * 128 + q * 32 + lane;
            const int64_t col0 = (int64_t)(u % p.tps) * 128;
            if (row < p.n) {
                float* crow = p.C + row * p.ldc + col0;
                const bool vec = ((p.ldc & 3) == 0) &&
                                 ((reinterpret_cast<uintptr_t>(p.C) & 15) == 0) &&
                                 (col0 + 128 <= p.n);
                if (vec) {
#pragma unroll
                    for (int v = 0; v < 32; ++v) {
                        float4 o = make_float4(p.alpha * master[4 * v], p.alpha * master[4 * v + 1],
                                               p.alpha * master[4 * v + 2],
                                               p.alpha * master[4 * v + 3]);
                        float4* dst = reinterpret_cast<float4*>(crow) + v;
                        if (p.beta != 0.f) {
                            const float4 old = *dst;
                            o.x = fmaf(p.beta, old.x, o.x);
                            o.y = fmaf(p.beta, old.y, o.y);
                            o.z = fmaf(p.beta, old.z, o.z);
                            o.w = fmaf(p.beta, old.w, o.w);
                        }
                        *dst = o;
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < 128; ++v) {
                        if (col0 + v < p.n) {
                            float o = p.alpha * master[v];
                            if (p.beta != 0.f) o = fmaf(p.beta, crow[v], o);
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
        // copies issued but never consumed must land before the block exits
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                     : "memory");
    }
}

template <int LEAF, int PREC>
cudaError_t launch_t(spamm_ctx* ctx, const TcArgs& a) {
    using T = PrecTraits<PREC>;
    const size_t smem = 1024 + kZeroBytes + (size_t)T::kStages * T::kStage;
    cudaError_t e = cudaFuncSetAttribute(k_leaf_tc<LEAF, PREC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = a.tiles < ctx->sm_count ? a.tiles : ctx->sm_count;
    k_leaf_tc<LEAF, PREC><<<grid, kThreads, smem, ctx->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_leaf_tc(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B, float alpha,
                           float beta, float* C, int64_t ldc) {
    TcArgs a;
    for (int i = 0; i < 2; ++i) {
        a.pa[i] = A->packA[i] ? A->packA[i] : A->packA[0];
        a.pb[i] = B->packB[i] ? B->packB[i] : B->packB[0];
    }
    a.nlp = A->nlp;
    a.C = C;
    a.ldc = ldc;
    a.n = A->n;
    a.alpha = alpha;
    a.beta = beta;
    a.ctl = ctx->ctl;
    a.pool = ctx->pool;
    a.off = ctx->tile_off;
    a.steps = ctx->tile_steps;
    a.tps = tiles_per_side(A);
    a.tiles = a.tps * a.tps;
    a.S = ctx->last_S;
    const int p = A->precision;
    if (A->b == 16) {
        if (p == SPAMM_PREC_TF32X3) return launch_t<16, SPAMM_PREC_TF32X3>(ctx, a);
        if (p == SPAMM_PREC_TF32) return launch_t<16, SPAMM_PREC_TF32>(ctx, a);
        return launch_t<16, SPAMM_PREC_BF16X3>(ctx, a);
    }
    if (A->b == 32) {
        if (p == SPAMM_PREC_TF32X3) return launch_t<32, SPAMM_PREC_TF32X3>(ctx, a);
        if (p == SPAMM_PREC_TF32) return launch_t<32, SPAMM_PREC_TF32>(ctx, a);
        return launch_t<32, SPAMM_PREC_BF16X3>(ctx, a);
    }
    return cudaErrorNotSupported;
}

}  // namespace spamm
