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
#include "spamm_internal.cuh"

namespace spamm {

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

    const uint32_t ns = steps[u];
    const uint32_t base = off[u] * (uint32_t)S;
    const uint32_t* pk = reinterpret_cast<const uint32_t*>(pool + ctl->pk_off);
    const unsigned long long* pm = reinterpret_cast<const unsigned long long*>(pool + ctl->pm_off);
    const int chunks = b >> 4;
    for (uint32_t st = 0; st < ns; ++st) {
        const unsigned long long mask = pm[2 * (size_t)(base + st) + half];
        if (mask == 0ull) continue;  // no kept product of this half at this K
        const int64_t K = pk[base + st];
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

}  // namespace spamm
