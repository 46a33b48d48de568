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

// The leaf products of one 128 x 128 tile half over its steps (K(st),
// mask(st)) in ascending K, and the alpha/beta epilogue.
template <class StepK, class StepMask>
__device__ __forceinline__ void simt_half(const float* __restrict__ A, int64_t lda,
                                          const float* __restrict__ B, int64_t ldb,
                                          float* __restrict__ C, int64_t ldc, int64_t n, int b,
                                          int64_t R0, int64_t C0, float alpha, float beta,
                                          uint32_t ns, StepK step_k, StepMask step_mask,
                                          float (*As)[132], float (*Bs)[128], float* accS) {
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const int x = (8 * ty) / b, y = (8 * tx) / b;
    const int bit = y * 8 + x;
    constexpr int LDS = 132;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float4* a = reinterpret_cast<float4*>(&accS[(8 * ty + i) * LDS + 8 * tx]);
        a[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        a[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int chunks = b >> 4;
    for (uint32_t st = 0; st < ns; ++st) {
        const unsigned long long mask = step_mask(st);
        if (mask == 0ull) continue;  // no kept product of this half at this K
        const int64_t K = step_k(st);
        const bool mine = (mask >> bit) & 1ull;
        float part[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) part[i][j] = 0.f;
        for (int ch = 0; ch < chunks; ++ch) {
            const int64_t c0 = K * b + 16 * ch;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int e = tid + 256 * i;
                const int row = e >> 4, col = e & 15;
                const int64_t gr = R0 + row, gc = c0 + col;
                As[col][row] = (gr < n && gc < n) ? __ldg(A + gr * lda + gc) : 0.f;
                const int kr = e >> 7, cc = e & 127;
                const int64_t gk = c0 + kr, gcol = C0 + cc;
                Bs[kr][cc] = (gk < n && gcol < n) ? __ldg(B + gk * ldb + gcol) : 0.f;
            }
            __syncthreads();
            if (mine) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const float4 a0 = *reinterpret_cast<const float4*>(&As[k][8 * ty]);
                    const float4 a1 = *reinterpret_cast<const float4*>(&As[k][8 * ty + 4]);
                    const float4 b0 = *reinterpret_cast<const float4*>(&Bs[k][8 * tx]);
                    const float4 b1 = *reinterpret_cast<const float4*>(&Bs[k][8 * tx + 4]);
                    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) part[i][j] = fmaf(av[i], bv[j], part[i][j]);
                }
            }
            __syncthreads();
        }
        if (mine) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float4* a = reinterpret_cast<float4*>(&accS[(8 * ty + i) * LDS + 8 * tx]);
                float4 v0 = a[0], v1 = a[1];
                v0.x += part[i][0]; v0.y += part[i][1]; v0.z += part[i][2]; v0.w += part[i][3];
                v1.x += part[i][4]; v1.y += part[i][5]; v1.z += part[i][6]; v1.w += part[i][7];
                a[0] = v0;
                a[1] = v1;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t gr = R0 + 8 * ty + i;
        if (gr >= n) break;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t gc = C0 + 8 * tx + j;
            if (gc < n) {
                float v = alpha * accS[(8 * ty + i) * LDS + 8 * tx + j];
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
    simt_half(A, lda, B, ldb, C, ldc, n, b, R0, C0, alpha, beta, ns,
              [&](uint32_t st) { return (int64_t)pk[base + st]; },
              [&](uint32_t st) { return pm[2 * (size_t)(base + st) + half]; }, As, Bs, accS);
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

__global__ void __launch_bounds__(256) k_small_fp32(SmallArgs a) {
    __shared__ __align__(16) float As[16][132];
    __shared__ __align__(16) float Bs[16][128];
    extern __shared__ __align__(16) float accS[];
    __shared__ unsigned long long m0s[kSmallLeaves], m1s[kSmallLeaves];  // per K: both halves
    __shared__ unsigned long long sm0[kSmallLeaves], sm1[kSmallLeaves];  // compacted steps
    __shared__ uint32_t sk[kSmallLeaves];
    __shared__ uint32_t nsteps;
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
            for (unsigned long long g = gid; g < (unsigned long long)(w * w * w); g += stride) {
                const int64_t i = (int64_t)(g / (unsigned long long)(w * w));
                const int64_t k = (int64_t)((g / (unsigned long long)w) % (unsigned long long)w);
                const int64_t j = (int64_t)(g % (unsigned long long)w);
                bool tb;
                if (!spamm_keep(pa[(i >> 1) * wp + (k >> 1)], pb[(k >> 1) * wp + (j >> 1)], a.th, &tb))
                    continue;                      // the parent was not kept: not tested
                ++cand;
                const bool own = spamm_keep(na[i * w + k], nbb[k * w + j], a.th, &tb);
                tie += tb ? 1 : 0;
                if (own) {
                    ++kept;
                    if (t == a.d) vol += ext(i) * ext(k) * ext(j);
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
    // ---- this tile's steps: for every leaf column K the kept (row leaf,
    // column leaf) pairs of both halves, from the leaf norms alone
    const uint32_t u = blockIdx.x >> 1;
    const int half = blockIdx.x & 1;
    const int TL = kTileRows / b;
    const int64_t I0 = (int64_t)(u / a.tc) * TL;
    const int64_t J0 = (int64_t)(u % a.tc) * 2 * TL;
    const double* la = a.pyrA + ((((int64_t)1 << (2 * a.d)) - 1) / 3);
    const double* lb = a.pyrB + ((((int64_t)1 << (2 * a.d)) - 1) / 3);
    const int nb = (int)a.nb;
    for (int K = tid; K < nb; K += blockDim.x) m0s[K] = m1s[K] = 0ull;
    __syncthreads();
    const int pairs = TL * 2 * TL;                   // (x, y) pairs of one K, both halves
    for (int e = tid; e < pairs * nb; e += blockDim.x) {
        const int K = e / pairs, pr = e % pairs;
        const int x = pr % TL, y = pr / TL;
        const int64_t I = I0 + x, J = J0 + y;
        bool tb;
        const bool keep = I < nb && J < nb && spamm_keep(la[I * nb + K], lb[(int64_t)K * nb + J], a.th, &tb);
        if (keep) {
            const int yy = y < TL ? y : y - TL;
            atomicOr(y < TL ? &m0s[K] : &m1s[K], 1ull << (yy * 8 + x));
        }
    }
    __syncthreads();
    if (tid < 32) {
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
        if (lane == 0) nsteps = cnt;
    }
    __syncthreads();
    const uint32_t ns = nsteps;
    if (half == 0) {
        // the step list where spamm_triples reads it: tile u owns slots
        // [u nb, u nb + nb) of the pool (K, then both halves' masks)
        if (a.write_steps) {
            const int64_t tiles = (int64_t)gridDim.x / 2;
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
    }
    // ---- the leaf products of this half, as k_leaf_simt forms them
    const int64_t R0 = (int64_t)(u / a.tc) * kTileRows;
    const int64_t C0 = ((int64_t)(u % a.tc) * kTileHalves + half) * kTileRows;
    simt_half(a.A, a.lda, a.B, a.ldb, a.C, a.ldc, n, b, R0, C0, a.alpha, a.beta, ns,
              [&](uint32_t st) { return (int64_t)sk[st]; },
              [&](uint32_t st) { return half ? sm1[st] : sm0[st]; }, As, Bs, accS);
}

bool small_path(const spamm_ctx* ctx, const spamm_tree* A) {
    if (ctx->cfg.staged || ctx->cfg.precision != SPAMM_PREC_FP32 || A->nb > kSmallLeaves)
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
    const size_t dsm = sizeof(float) * 128 * 132;
    cudaError_t e = cudaFuncSetAttribute(k_small_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dsm);
    if (e != cudaSuccess) return e;
    k_small_fp32<<<tiles * kTileHalves, 256, dsm, ctx->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace spamm
