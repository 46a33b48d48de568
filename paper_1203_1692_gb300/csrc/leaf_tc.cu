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
// Roles (192 threads): warp 0 lane 0 issues the bulk copies into a ring of
// shared-memory stages; warp 1 owns the TMEM allocation and its lane 0
// issues the MMAs and commits; warps 2-5 move the double-buffered 128 x 128
// accumulator out of TMEM, apply alpha/beta and store C.  Every wait on an
// mbarrier gives up after one second, raises the timeout status and lets
// the block drain its copies and MMAs, free TMEM and exit.
#include <cuda_bf16.h>

#include "spamm_internal.cuh"

namespace spamm {
namespace {

constexpr int kThreads = 192;
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
            for (int u = blockIdx.x; u < p.tiles && ok; u += gridDim.x) {
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
            uint32_t tcount = 0;
            bool ok = true;
            const uint64_t zdesc = make_desc(smem_u32(zero), 128, 256);
            const uint32_t dis0[4] = {0u, 0u, 0u, 0u};
            for (int u = blockIdx.x; u < p.tiles && ok; u += gridDim.x, ++tcount) {
                const uint32_t ab = tcount & 1;
                const uint32_t aph = (tcount >> 1) & 1;
                if (!wait_bar(smem_u32(&bar_acce[ab]), aph ^ 1, &abort_flag, status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dacc = tmem + ab * 128;
                // clear the accumulator: 0 * 0 with the input accumulator off
                mma<PREC>(dacc, zdesc, zdesc, make_idesc(T::kAB, 128, 128), dis0, 0u);
                const uint32_t ns = p.steps[u];
                const uint64_t sb = (uint64_t)p.off[u] * p.S;
                for (uint32_t st = 0; st < ns && ok; ++st) {
                    const unsigned long long mask = pm[sb + st];
                    for (int kc = 0; kc < CHUNKS; ++kc, ++it) {
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
                            while (y + len < TL && ((uint32_t)(mask >> (8 * (y + len))) & 0xFFu) == xm)
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
                                    const uint64_t bl = make_desc(b_lo + boff + koff, 128, T::kSBO);
                                    mma<PREC>(d, al, bh, idesc, dis, 1u);
                                    mma<PREC>(d, ah, bl, idesc, dis, 1u);
                                }
                                mma<PREC>(d, ah, bh, idesc, dis, 1u);
                            }
                            y += len;
                        }
                        tc_commit(smem_u32(&bar_empty[s]));
                    }
                }
                if (ok) tc_commit(smem_u32(&bar_accf[ab]));
            }
            // drain: every MMA issued so far has completed before TMEM is freed
            tc_commit(smem_u32(&bar_drain));
            wait_bar(smem_u32(&bar_drain), 0, &abort_flag, status);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        uint32_t tcount = 0;
        for (int u = blockIdx.x; u < p.tiles; u += gridDim.x, ++tcount) {
            const uint32_t ab = tcount & 1;
            const uint32_t aph = (tcount >> 1) & 1;
            if (!wait_bar(smem_u32(&bar_accf[ab]), aph, &abort_flag, status)) break;
            tc_fence_after();
            const int64_t row = (int64_t)(u / p.tps) * 128 + q * 32 + lane;
            const int64_t col0 = (int64_t)(u % p.tps) * 128;
            float* crow = p.C + row * p.ldc;
            const bool vec = ((p.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(p.C) & 15) == 0);
#pragma unroll 1
            for (int c = 0; c < 128; c += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + ab * 128 + (uint32_t)c, r);
                if (row < p.n) {
                    const int64_t cb = col0 + c;
                    if (vec && cb + 32 <= p.n) {
#pragma unroll
                        for (int v = 0; v < 8; ++v) {
                            float4 o;
                            o.x = p.alpha * __uint_as_float(r[4 * v + 0]);
                            o.y = p.alpha * __uint_as_float(r[4 * v + 1]);
                            o.z = p.alpha * __uint_as_float(r[4 * v + 2]);
                            o.w = p.alpha * __uint_as_float(r[4 * v + 3]);
                            float4* dst = reinterpret_cast<float4*>(crow + cb + 4 * v);
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
                        for (int v = 0; v < 32; ++v) {
                            if (cb + v < p.n) {
                                float o = p.alpha * __uint_as_float(r[v]);
                                if (p.beta != 0.f) o = fmaf(p.beta, crow[cb + v], o);
                                crow[cb + v] = o;
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_acce[ab]));
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
