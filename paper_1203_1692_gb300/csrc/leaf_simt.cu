// Stage 4, FP32 on the CUDA cores: C_IJ = alpha * sum_{kept K, ascending}
// A_IK B_KJ + beta * C_IJ (Algorithm 1, numeric part).
//
// One block per 128 x 128 half of a C tile, 256 threads, each owning an 8 x 8
// patch (which lies inside one leaf pair (x, y) for b >= 8).  The block
// walks the tile's steps in ascending K, with that half's mask; for each
// step with kept products it stages A's
// 128 x 16 and B's 16 x 128 slices per 16-wide K chunk in shared memory
// (zero outside the n x n matrix) and a thread runs its 8 x 8 x 16 FFMA
// block only when its leaf pair's bit is set.  Like the numeric multiply of
// the method, each leaf product is formed on its own (an FFMA chain over its
// b values of k, starting from zero) and then added to the C block, in
// ascending K: one rounding into C per kept product instead of one per k,
// and a fixed order, so the result is deterministic.  The running sum of the
// C tile lives in shared memory (each thread owns its 8 x 8 patch there),
// which keeps registers low enough for two blocks per SM.
//
// Small products (k_small_fp32): for a product of at most kSmallLeaves leaves
// per side the cull, the grouping and the leaf products run in ONE launch
// instead of one launch per tier and stage.  A block finds its tile's steps
// itself: a leaf triple is kept by the tier-by-tier cull iff its own leaf
// norms pass the SpAMM test, because a parent's squared norm (an FP64 sum of
// its non-negative children) is never below a child's, so the ancestors of
// a passing leaf triple pass too (the same identity that makes the flat
// enumeration of Algorithm 1 equal the recursion).  The blocks also count,
// tier by tier, the tested and kept triples and the tie band as the
// hierarchical cull reports them (a triple is tested iff its parent passes),
// and write the steps in the layout spamm_triples reads.  The leaf products
// are the same code as k_leaf_simt, so C is the same bit for bit.
#include "spamm_internal.cuh"

namespace spamm {

constexpr int kSmallLeaves = 128;   // leaves per side of the fused small path

// The leaf products of one TS x TS block of C (a 128 x 128 tile half, or a
// 64 x 64 quarter of one for the small path) over its steps (K(st),
// mask(st)) in ascending K, and the alpha/beta epilogue.  (TS / P)^2
// threads, each owning a P x P patch (every element is formed the same way
// whatever P is: a k-ordered FFMA chain per leaf product, then one add into
// the block); As is [16][TS + 4], Bs [16][TS], accS [TS][TS + 4].
template <int TS, int P, class StepK, class StepMask>
__device__ __forceinline__ void simt_block(const float* __restrict__ A, int64_t lda,
                                           const float* __restrict__ B, int64_t ldb,
                                           float* __restrict__ C, int64_t ldc, int64_t n, int b,
                                           int64_t R0, int64_t C0, float alpha, float beta,
                                           uint32_t ns, StepK step_k, StepMask step_mask,
                                           float* As, float* Bs, float* accS) {
    constexpr int PT = TS / P;                 // patches per side
    constexpr int THREADS = PT * PT;
    constexpr int LDA = TS + 4, LDS = TS + 4;
    static_assert(P == 4 || P == 8, "patch of 4 or 8");
    const int tid = threadIdx.x;
    const int ty = tid / PT, tx = tid % PT;
    const int x = (P * ty) / b, y = (P * tx) / b;
    const int bit = y * 8 + x;
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
        for (int j = 0; j < P; j += 4)
            *reinterpret_cast<float4*>(&accS[(P * ty + i) * LDS + P * tx + j]) =
                make_float4(0.f, 0.f, 0.f, 0.f);
    // the (step, chunk) pairs with a kept product of this block, in order;
    // the global loads of the next pair are issued before the FFMAs of the
    // current one (software pipelining through registers)
    constexpr int NL = 16 * TS / THREADS;      // elements of each slice per thread
    const int chunks = b >> 4;
    auto next_live = [&](uint32_t st) {
        while (st < ns && step_mask(st) == 0ull) ++st;
        return st;
    };
    float ra[NL], rb[NL];
    auto load = [&](uint32_t st, int ch) {
        const int64_t c0 = step_k(st) * b + 16 * ch;
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            const int e = tid + THREADS * i;
            const int row = e >> 4, col = e & 15;
            const int64_t gr = R0 + row, gc = c0 + col;
            ra[i] = (gr < n && gc < n) ? __ldg(A + gr * lda + gc) : 0.f;
            const int kr = e / TS, cc = e % TS;
            const int64_t gk = c0 + kr, gcol = C0 + cc;
            rb[i] = (gk < n && gcol < n) ? __ldg(B + gk * ldb + gcol) : 0.f;
        }
    };
    uint32_t st = next_live(0);
    int ch = 0;
    if (st < ns) load(st, 0);
    float part[P][P];
    while (st < ns) {
        const bool mine = (step_mask(st) >> bit) & 1ull;
        if (ch == 0) {
#pragma unroll
            for (int i = 0; i < P; ++i)
#pragma unroll
                for (int j = 0; j < P; ++j) part[i][j] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            const int e = tid + THREADS * i;
            As[(e & 15) * LDA + (e >> 4)] = ra[i];
            Bs[(e / TS) * TS + (e % TS)] = rb[i];
        }
        __syncthreads();
        // the next (step, chunk): its loads fly while this one computes
        uint32_t st2 = st;
        int ch2 = ch + 1;
        if (ch2 == chunks) {
            ch2 = 0;
            st2 = next_live(st + 1);
        }
        if (st2 < ns) load(st2, ch2);
        if (mine) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float av[P], bv[P];
#pragma unroll
                for (int q = 0; q < P; q += 4) {
                    const float4 a4 = *reinterpret_cast<const float4*>(&As[k * LDA + P * ty + q]);
                    const float4 b4 = *reinterpret_cast<const float4*>(&Bs[k * TS + P * tx + q]);
                    av[q] = a4.x; av[q + 1] = a4.y; av[q + 2] = a4.z; av[q + 3] = a4.w;
                    bv[q] = b4.x; bv[q + 1] = b4.y; bv[q + 2] = b4.z; bv[q + 3] = b4.w;
                }
#pragma unroll
                for (int i = 0; i < P; ++i)
#pragma unroll
                    for (int j = 0; j < P; ++j) part[i][j] = fmaf(av[i], bv[j], part[i][j]);
            }
        }
        __syncthreads();
        if (mine && ch == chunks - 1) {
            // the leaf product is complete: one rounding into the C block
#pragma unroll
            for (int i = 0; i < P; ++i)
#pragma unroll
                for (int j = 0; j < P; j += 4) {
                    float4* a = reinterpret_cast<float4*>(&accS[(P * ty + i) * LDS + P * tx + j]);
                    float4 v = *a;
                    v.x += part[i][j]; v.y += part[i][j + 1]; v.z += part[i][j + 2];
                    v.w += part[i][j + 3];
                    *a = v;
                }
        }
        st = st2;
        ch = ch2;
    }
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const int64_t gr = R0 + P * ty + i;
        if (gr >= n) break;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int64_t gc = C0 + P * tx + j;
            if (gc < n) {
                float v = alpha * accS[(P * ty + i) * LDS + P * tx + j];
                if (beta != 0.f) v = fmaf(beta, C[gr * ldc + gc], v);
                C[gr * ldc + gc] = v;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_leaf_simt(const float* __restrict__ A, int64_t lda,
                                                   const float* __restrict__ B, int64_t ldb,
                                                   float* __restrict__ C, int64_t ldc, int64_t n,
                                                   int b, int tc, int S, float alpha,
                                                   float beta,
                                                   const DevCtl* __restrict__ ctl,
                                                   const uint64_t* __restrict__ pool,
                                                   const uint32_t* __restrict__ off,
                                                   const uint32_t* __restrict__ steps) {
    __shared__ __align__(16) float As[16][132];  // [k][row]
    __shared__ __align__(16) float Bs[16][128];  // [k][col]
    extern __shared__ __align__(16) float accS[];  // [128][132] running C tile
    if (ctl->status & (ST_OVERFLOW | ST_NONFINITE)) return;
    const uint32_t u = blockIdx.x >> 1;
    const int half = blockIdx.x & 1;
    const int64_t R0 = (int64_t)(u / tc) * kTileRows;
    const int64_t C0 = ((int64_t)(u % tc) * kTileHalves + half) * kTileRows;
    const uint32_t ns = steps[u];
    const uint32_t base = off[u] * (uint32_t)S;
    const uint32_t* pk = reinterpret_cast<const uint32_t*>(pool + ctl->pk_off);
    const unsigned long long* pm = reinterpret_cast<const unsigned long long*>(pool + ctl->pm_off);
    simt_block<128, 8>(A, lda, B, ldb, C, ldc, n, b, R0, C0, alpha, beta, ns,
                    [&](uint32_t st) { return (int64_t)pk[base + st]; },
                    [&](uint32_t st) { return pm[2 * (size_t)(base + st) + half]; }, &As[0][0],
                    &Bs[0][0], accS);
}

cudaError_t launch_leaf_simt(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B,
                             float alpha, float beta, float* C, int64_t ldc) {
    const int tc = tile_cols(A);
    const int tiles = tile_rows(A) * tc;
    const size_t dsm = sizeof(float) * 128 * 132;
    cudaError_t e = cudaFuncSetAttribute(k_leaf_simt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dsm);
    if (e != cudaSuccess) return e;
    k_leaf_simt<<<tiles * kTileHalves, 256, dsm, ctx->stream>>>(A->A, A->lda, B->A, B->lda, C,
                                                    ldc, A->n, A->b, tc, ctx->last_S, alpha, beta,
                                                    ctx->ctl, ctx->pool,
                                                    ctx->tile_off, ctx->tile_steps);
    return cudaGetLastError();
}

// ------------------------------------------------------- small products

struct SmallArgs {
    const float* A;
    int64_t lda;
    const float* B;
    int64_t ldb;
    float* C;
    int64_t ldc;
    int64_t n;
    int b, d, tc, S;
    int64_t nb;            // 2^d leaves per side
    const double* pyrA;
    const double* pyrB;
    Thresh th;
    float alpha, beta;
    DevCtl* ctl;
    uint64_t* pool;
    int write_steps;       // the pool holds tiles x nb step slots
    uint32_t* tile_off;
    uint32_t* tile_steps;
};

// Small blocks: a 128 x 256 tile is cut into eight 64 x 64 blocks, one
// block of 64 threads each, so that a small product spreads over the SMs.
constexpr int kSmallTS = 64;
constexpr int kSmallPatch = 4;
constexpr int kSmallThreads = (kSmallTS / kSmallPatch) * (kSmallTS / kSmallPatch);
constexpr int kSmallBlocksPerTile = (kTileRows / kSmallTS) * (kTileHalves * kTileRows / kSmallTS);

// Kept (x, y) leaf pairs of leaf column K between the staged row leaves
// x0.. of sa (row x at sa[x * nb + K]) and the staged column leaves y0.. of
// sb (sb[K * ldb + y]); nx x ny pairs, the columns in halves of hw leaves,
// bit (y % hw) * 8 + x of mask y / hw.  One warp per K, ORed across the warp.
__device__ __forceinline__ void pair_masks(const double* sa, const double* sb, int ldb, int nb,
                                           int x0, int y0, int nx, int ny, int hw,
                                           const Thresh& th, unsigned long long* m0s,
                                           unsigned long long* m1s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int pairs = nx * ny;
    for (int K = warp; K < nb; K += nwarps) {
        unsigned long long w0 = 0ull, w1 = 0ull;
        for (int p0 = 0; p0 < pairs; p0 += 32) {
            const int pr = p0 + lane;
            const int x = pr % nx, y = pr / nx;
            bool tb;
            // leaves outside the matrix are staged as zero norms: never kept
            const bool keep = pr < pairs &&
                              spamm_keep(sa[(x0 + x) * nb + K], sb[K * ldb + y0 + y], th, &tb);
            const unsigned long long bit = keep ? 1ull << ((y % hw) * 8 + x) : 0ull;
            const unsigned long long b0 = y < hw ? bit : 0ull, b1 = y < hw ? 0ull : bit;
            w0 |= ((unsigned long long)__reduce_or_sync(0xffffffffu, (uint32_t)(b0 >> 32)) << 32) |
                  __reduce_or_sync(0xffffffffu, (uint32_t)b0);
            w1 |= ((unsigned long long)__reduce_or_sync(0xffffffffu, (uint32_t)(b1 >> 32)) << 32) |
                  __reduce_or_sync(0xffffffffu, (uint32_t)b1);
        }
        if (lane == 0) {
            m0s[K] = w0;
            m1s[K] = w1;
        }
    }
}

// The leaf columns with a kept pair, in ascending K (warp 0).
__device__ __forceinline__ void compact_steps(int nb, const unsigned long long* m0s,
                                              const unsigned long long* m1s, uint32_t* sk,
                                              unsigned long long* sm0, unsigned long long* sm1,
                                              uint32_t* nsteps) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    uint32_t cnt = 0;
    for (int base = 0; base < nb; base += 32) {
        const int K = base + lane;
        const bool live = K < nb && (m0s[K] | m1s[K]) != 0ull;
        const unsigned bal = __ballot_sync(0xffffffffu, live);
        if (live) {
            const uint32_t pos = cnt + __popc(bal & ((1u << lane) - 1u));
            sk[pos] = (uint32_t)K;
            sm0[pos] = m0s[K];
            sm1[pos] = m1s[K];
        }
        cnt += __popc(bal);
    }
    if (lane == 0) *nsteps = cnt;
}

__global__ void __launch_bounds__(kSmallThreads) k_small_fp32(SmallArgs a) {
    __shared__ __align__(16) float As[16 * (kSmallTS + 4)];
    __shared__ __align__(16) float Bs[16 * kSmallTS];
    __shared__ __align__(16) float accS[kSmallTS * (kSmallTS + 4)];
    __shared__ unsigned long long m0s[kSmallLeaves], m1s[kSmallLeaves];
    __shared__ unsigned long long sm0[kSmallLeaves], sm1[kSmallLeaves];
    __shared__ uint32_t sk[kSmallLeaves];
    __shared__ uint32_t nsteps;
    extern __shared__ __align__(16) double stage[];   // staged leaf norms of the tile
    const int tid = threadIdx.x, lane = tid & 31;
    const double ra = a.pyrA[0], rb = a.pyrB[0];
    if (!isfinite(ra) || !isfinite(rb)) {
        // Inf/NaN anywhere makes a root non-finite: C is left as it is
        if (blockIdx.x == 0 && tid == 0) {
            a.ctl->status |= ST_NONFINITE;
            a.ctl->tier_cand[0] = 1;
        }
        return;
    }
    const int b = a.b;
    const int64_t n = a.n;
    auto ext = [&](int64_t L) -> unsigned long long {   // rows of leaf L inside the matrix
        const int64_t r = n - L * b;
        return (unsigned long long)(r < b ? (r > 0 ? r : 0) : b);
    };
    // ---- statistics of the tier-by-tier cull: tier t's triples are tested
    // iff their parent passes, and kept iff they pass themselves
    {
        const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
        const unsigned long long gid = (unsigned long long)blockIdx.x * blockDim.x + tid;
        unsigned long long tie = 0, vol = 0;
        if (gid == 0) {
            bool tb;
            const bool k0 = spamm_keep(ra, rb, a.th, &tb);
            a.ctl->tier_cand[0] = 1;
            a.ctl->tier_count[0] = k0 ? 1 : 0;
            tie += tb ? 1 : 0;
            if (k0 && a.d == 0) vol += ext(0) * ext(0) * ext(0);   // the root is the leaf
        }
        for (int t = 1; t <= a.d; ++t) {
            const int64_t w = (int64_t)1 << t, wp = w >> 1;
            const double* na = a.pyrA + ((((int64_t)1 << (2 * t)) - 1) / 3);
            const double* nbb = a.pyrB + ((((int64_t)1 << (2 * t)) - 1) / 3);
            const double* pa = a.pyrA + ((((int64_t)1 << (2 * (t - 1))) - 1) / 3);
            const double* pb = a.pyrB + ((((int64_t)1 << (2 * (t - 1))) - 1) / 3);
            unsigned long long cand = 0, kept = 0;
            const unsigned long long cube = (unsigned long long)(w * w * w);
            constexpr int U4 = 4;                  // items per round: their loads overlap
            for (unsigned long long g0 = gid; g0 < cube; g0 += U4 * stride) {
                double vpa[U4], vpb[U4], vna[U4], vnb[U4];
                int64_t ii[U4], kk[U4], jj[U4];
#pragma unroll
                for (int q = 0; q < U4; ++q) {
                    const unsigned long long g = g0 + q * stride;
                    // (i, k, j) from the bits of g: w is a power of two
                    ii[q] = (int64_t)(g >> (2 * t));
                    kk[q] = (int64_t)((g >> t) & (unsigned long long)(w - 1));
                    jj[q] = (int64_t)(g & (unsigned long long)(w - 1));
                    const bool in = g < cube;
                    vpa[q] = in ? pa[(ii[q] >> 1) * wp + (kk[q] >> 1)] : 0.0;
                    vpb[q] = in ? pb[(kk[q] >> 1) * wp + (jj[q] >> 1)] : 0.0;
                    vna[q] = in ? na[ii[q] * w + kk[q]] : 0.0;
                    vnb[q] = in ? nbb[kk[q] * w + jj[q]] : 0.0;
                }
#pragma unroll
                for (int q = 0; q < U4; ++q) {
                    bool tb;
                    // a zero (or out-of-range) parent is never kept: not tested
                    if (!spamm_keep(vpa[q], vpb[q], a.th, &tb)) continue;
                    ++cand;
                    const bool own = spamm_keep(vna[q], vnb[q], a.th, &tb);
                    tie += tb ? 1 : 0;
                    if (own) {
                        ++kept;
                        if (t == a.d) vol += ext(ii[q]) * ext(kk[q]) * ext(jj[q]);
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                cand += __shfl_xor_sync(0xffffffffu, cand, o);
                kept += __shfl_xor_sync(0xffffffffu, kept, o);
            }
            if (lane == 0 && cand) atomicAdd(&a.ctl->tier_cand[t], cand);
            if (lane == 0 && kept) atomicAdd(&a.ctl->tier_count[t], kept);
        }
        for (int o = 16; o > 0; o >>= 1) {
            tie += __shfl_xor_sync(0xffffffffu, tie, o);
            vol += __shfl_xor_sync(0xffffffffu, vol, o);
        }
        if (lane == 0 && tie) atomicAdd(&a.ctl->tie_band, tie);
        if (lane == 0 && vol) atomicAdd(&a.ctl->clip_vol, vol);
    }
    const uint32_t u = blockIdx.x / kSmallBlocksPerTile;
    const int sub = blockIdx.x % kSmallBlocksPerTile;
    const int sr = sub / (kTileHalves * kTileRows / kSmallTS);
    const int sc = sub % (kTileHalves * kTileRows / kSmallTS);
    const int TL = kTileRows / b;                    // leaves per tile row and column half
    const int SL = kSmallTS / b;                     // leaves per side of this block
    const int64_t tI = (int64_t)(u / a.tc) * TL, tJ = (int64_t)(u % a.tc) * 2 * TL;
    const double* la = a.pyrA + ((((int64_t)1 << (2 * a.d)) - 1) / 3);
    const double* lb = a.pyrB + ((((int64_t)1 << (2 * a.d)) - 1) / 3);
    const int nb = (int)a.nb;
    // the tile's leaf norms in shared memory: A rows tI.. (TL x nb) and B
    // columns tJ.. (nb x 2 TL), zero outside the matrix
    double* sa = stage;
    double* sbn = stage + TL * nb;
#pragma unroll 4
    for (int e = tid; e < TL * nb; e += blockDim.x) {
        const int64_t I = tI + e / nb;
        sa[e] = I < nb ? la[I * nb + e % nb] : 0.0;
    }
#pragma unroll 4
    for (int e = tid; e < nb * 2 * TL; e += blockDim.x) {
        const int64_t J = tJ + e % (2 * TL);
        sbn[e] = J < nb ? lb[(int64_t)(e / (2 * TL)) * nb + J] : 0.0;
    }
    __syncthreads();
    if (sub == 0) {
        // ---- the tile's steps (both column halves) where spamm_triples
        // reads them: tile u owns slots [u nb, u nb + nb) of the pool
        pair_masks(sa, sbn, 2 * TL, nb, 0, 0, TL, 2 * TL, TL, a.th, m0s, m1s);
        __syncthreads();
        compact_steps(nb, m0s, m1s, sk, sm0, sm1, &nsteps);
        __syncthreads();
        const uint32_t ns = nsteps;
        if (a.write_steps) {
            const int64_t tiles = (int64_t)gridDim.x / kSmallBlocksPerTile;
            uint32_t* pk = reinterpret_cast<uint32_t*>(a.pool);
            unsigned long long* pm = reinterpret_cast<unsigned long long*>(a.pool + (tiles * nb + 1) / 2);
            for (uint32_t st = tid; st < ns; st += blockDim.x) {
                pk[(int64_t)u * nb + st] = sk[st];
                pm[2 * ((int64_t)u * nb + st)] = sm0[st];
                pm[2 * ((int64_t)u * nb + st) + 1] = sm1[st];
            }
            if (tid == 0) {
                a.tile_steps[u] = ns;
                a.tile_off[u] = (uint32_t)((int64_t)u * nb / a.S);
                if (u == 0) {
                    a.ctl->pk_off = 0;
                    a.ctl->pm_off = (unsigned long long)((tiles * nb + 1) / 2);
                }
            }
        }
        if (tid == 0 && ns) atomicAdd(&a.ctl->active_steps, (unsigned long long)ns);
        __syncthreads();
    }
    // ---- this block's steps and its leaf products, as k_leaf_simt forms them
    pair_masks(sa, sbn, 2 * TL, nb, sr * SL, sc * SL, SL, SL, SL, a.th, m0s, m1s);
    __syncthreads();
    compact_steps(nb, m0s, m1s, sk, sm0, sm1, &nsteps);
    __syncthreads();
    const int64_t R0 = (int64_t)(u / a.tc) * kTileRows + sr * kSmallTS;
    const int64_t C0 = (int64_t)(u % a.tc) * kTileHalves * kTileRows + sc * kSmallTS;
    simt_block<kSmallTS, kSmallPatch>(a.A, a.lda, a.B, a.ldb, a.C, a.ldc, n, b, R0, C0, a.alpha, a.beta,
                         nsteps, [&](uint32_t st) { return (int64_t)sk[st]; },
                         [&](uint32_t st) { return sm0[st]; }, As, Bs, accS);
}

bool small_path(const spamm_ctx* ctx, const spamm_tree* A) {
    if (ctx->cfg.staged || ctx->cfg.precision != SPAMM_PREC_FP32 || A->nb > kSmallLeaves ||
        A->b > kSmallTS)
        return false;
    const int64_t tiles = (int64_t)tile_rows(A) * tile_cols(A);
    return ctx->pool_words >= tiles * A->nb * 3 + 2;
}

cudaError_t launch_small_fp32(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B, double tau,
                              float alpha, float beta, float* C, int64_t ldc) {
    SmallArgs a;
    a.A = A->A;
    a.lda = A->lda;
    a.B = B->A;
    a.ldb = B->lda;
    a.C = C;
    a.ldc = ldc;
    a.n = A->n;
    a.b = A->b;
    a.d = A->d;
    a.nb = A->nb;
    a.tc = tile_cols(A);
    a.S = ctx->last_S;
    a.pyrA = A->pyr;
    a.pyrB = B->pyr;
    a.th = make_thresh(tau, ctx->cfg.tie_rel);
    a.alpha = alpha;
    a.beta = beta;
    a.ctl = ctx->ctl;
    a.pool = ctx->pool;
    a.write_steps = 1;
    a.tile_off = ctx->tile_off;
    a.tile_steps = ctx->tile_steps;
    const int tiles = tile_rows(A) * a.tc;
    const int TL = kTileRows / A->b;
    const size_t dsm = sizeof(double) * (size_t)(3 * TL) * (size_t)A->nb;   // staged norms
    cudaError_t e = cudaFuncSetAttribute(k_small_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double) * 3 * 8 * kSmallLeaves));
    if (e != cudaSuccess) return e;
    k_small_fp32<<<tiles * kSmallBlocksPerTile, kSmallThreads, dsm, ctx->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace spamm
