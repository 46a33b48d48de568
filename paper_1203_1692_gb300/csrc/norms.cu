// Stage 1: the FP64 norm quadtree (Sec. II.A-B, Eq. (norm)) and, for the
// tensor-core precisions, the leaf tiles in tcgen05 shared-memory layout.
//
// Leaf squares: a thread owns four consecutive columns of one leaf row-strip
// and sums (double)a * (double)a (exact) down the strip's b rows; the b/4
// lanes that share a leaf combine their partial sums with a segmented
// xor-shuffle reduction.  The kernel reads each element of A once, with
// 16-byte loads when A and lda allow it, so it is bound by HBM bandwidth.
// With tensor-core packs the same sums come from k_leaf_pack below.
// The upper tiers come from a second kernel that builds five tiers per pass
// in shared memory, each node the sum of its four children in the order
// A11 + A12 + A21 + A22.
//
// Tensor-core tiles (precision != FP32).  The K dimension of a leaf is cut
// into chunks of 16; a "piece" is one leaf x one chunk, b rows x 16 k.
// Inside a piece the rows are grouped by 8: a row group holds the core
// matrices (8 rows x 16 bytes) of the chunk one after another (leading byte
// offset 128 B), and row groups follow each other at the stride-byte offset
// (512 B for TF32, 256 B for BF16): the no-swizzle K-major canonical layout
// of tcgen05.  Pieces are stored with the leaf index innermost:
//     piece(P, Q, kc) at ((P * (b/16) + kc) * nlp + Q) * piece_bytes   (B role)
//     piece(P, Q, kc) at ((Q * (b/16) + kc) * nlp + P) * piece_bytes   (A role)
// so the 128 / b consecutive leaves of one C tile row/column strip form one
// contiguous 8 KB (TF32) / 4 KB (BF16) run that a single bulk copy moves
// into shared memory, already in the layout the MMA reads.  The A role holds
// leaf (I, K) with rows = i (K-major as stored); the B role holds leaf (K, J)
// transposed, rows = j.
#include <cuda_bf16.h>

#include "spamm_internal.cuh"

namespace spamm {

bool precision_uses_tc(int p) { return p != SPAMM_PREC_FP32; }

int pack_arrays_for(int p) { return p == SPAMM_PREC_TF32 ? 1 : 2; }

static int elem_bytes(int p) { return p == SPAMM_PREC_BF16X3 ? 2 : 4; }

size_t pack_bytes_for(int p, int64_t nlp, int b) {
    if (!precision_uses_tc(p)) return 0;
    return (size_t)nlp * b * (size_t)nlp * b * elem_bytes(p);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Leaf squared norms only (FP32 leaf products need no packs).
template <bool VEC>
__global__ void __launch_bounds__(128) k_leaf_norms(const float* __restrict__ A, int64_t n,
                                                    int64_t lda, int b, int64_t nb, int64_t nl,
                                                    double* __restrict__ leaf) {
    const int64_t I = blockIdx.y;                       // leaf row
    const int64_t col0 = (int64_t)blockIdx.x * 512 + 4 * threadIdx.x;
    const int64_t K = col0 / b;                          // leaf column
    const int lanes = b >> 2;                            // lanes per leaf
    double s = 0.0;
    const int64_t r0 = I * b;
    for (int r = 0; r < b; ++r) {
        const int64_t row = r0 + r;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < n) {
            const float* p = A + row * lda + col0;
            if (VEC && col0 + 3 < n) {
                v = __ldg(reinterpret_cast<const float4*>(p));
            } else {
                if (col0 + 0 < n) v.x = __ldg(p + 0);
                if (col0 + 1 < n) v.y = __ldg(p + 1);
                if (col0 + 2 < n) v.z = __ldg(p + 2);
                if (col0 + 3 < n) v.w = __ldg(p + 3);
            }
        }
        const double x = v.x, y = v.y, z = v.z, w = v.w;
        s += x * x;
        s += y * y;
        s += z * z;
        s += w * w;
    }
    // segmented reduction over the lanes of one leaf
    for (int off = lanes >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & (lanes - 1)) == 0 && K < nl) leaf[I * nb + K] = s;
}

// Leaf norms plus tensor-core packs.  A block owns one leaf row-strip (b
// rows) x 128 columns (TL leaves).  It stages the strip in shared memory
// (16-byte loads) while forming the leaf squared norms (FP64), then produces
// the pieces in output order: thread t writes the t-th, (t+128)-th, ...
// 16-byte unit of each piece, reading the elements that unit holds from the
// staged strip (a row quad for the A role, a column quad for the B role),
// splitting them into hi/lo parts and storing both parts.  The A-role
// pieces of one leaf and the B-role pieces of one K-chunk are contiguous in
// HBM, so consecutive threads write consecutive 16-byte units: every global
// store is coalesced.  PK: 1 tf32 hi, 2 tf32 hi+lo, 3 bf16 hi+lo.
template <int PK, int LEAF>
__global__ void __launch_bounds__(128) k_leaf_pack(const float* __restrict__ A, int64_t n,
                                                   int64_t lda, int64_t nb, int64_t nl, int64_t nlp,
                                                   double* __restrict__ leaf,
                                                   void* __restrict__ pa0, void* __restrict__ pa1,
                                                   void* __restrict__ pb0, void* __restrict__ pb1) {
    constexpr int TL = 128 / LEAF;
    constexpr int CH = LEAF / 16;
    constexpr int ES = PK == 3 ? 2 : 4;                  // element bytes
    constexpr int EPU = 16 / ES;                         // elements per 16-byte unit
    constexpr int PIECE = LEAF * 16 * ES;                // bytes of one piece
    constexpr int UPP = PIECE / 16;                      // units per piece
    constexpr int CPC = 16 / EPU;                        // core matrices per 16-wide K chunk
    constexpr int LDS = 128 + 4;                         // padded staging row
    extern __shared__ __align__(16) float raw_dyn[];     // LEAF x LDS staged strip
    float (*raw)[LDS] = reinterpret_cast<float (*)[LDS]>(raw_dyn);
    __shared__ double part[4][TL];
    // leaf rows vary fastest across blocks, so the blocks running at once
    // write neighbouring A-role pieces
    const int64_t I = blockIdx.x;                        // leaf row
    const int64_t Q0 = (int64_t)blockIdx.y * TL;         // first leaf column
    const int64_t r0 = I * LEAF, c0 = Q0 * LEAF;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const bool vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda % 4 == 0);
    const int cq = 4 * lane;
    const int x = cq / LEAF;
    double s = 0.0;
#pragma unroll 4
    for (int r = warp; r < LEAF; r += 4) {
        const int64_t row = r0 + r, col = c0 + cq;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < n) {
            const float* p = A + row * lda + col;
            if (vec && col + 3 < n) {
                v = __ldg(reinterpret_cast<const float4*>(p));
            } else {
                if (col + 0 < n) v.x = __ldg(p + 0);
                if (col + 1 < n) v.y = __ldg(p + 1);
                if (col + 2 < n) v.z = __ldg(p + 2);
                if (col + 3 < n) v.w = __ldg(p + 3);
            }
        }
        const double dx = v.x, dy = v.y, dz = v.z, dw = v.w;
        s += dx * dx;
        s += dy * dy;
        s += dz * dz;
        s += dw * dw;
        *reinterpret_cast<float4*>(&raw[r][cq]) = v;
    }
    // leaf squared norms: lanes of one leaf, then the four warps, fixed order
    constexpr int LPL = LEAF / 4;                        // lanes per leaf
    for (int o = LPL >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((lane % LPL) == 0) part[warp][x] = s;
    __syncthreads();
    if (t < TL) {
        const double v = ((part[0][t] + part[1][t]) + part[2][t]) + part[3][t];
        if (Q0 + t < nl) leaf[I * nb + Q0 + t] = v;
    }
    // pieces, in output order
    constexpr int UNITS = TL * CH * UPP;                 // per role and part
    for (int u = t; u < UNITS; u += 128) {
        const int pc = u / UPP, w = u % UPP;
        // unit w of a piece: row group w / (8 CPC), core (w / 8) % CPC, row w % 8
        const int rg = w / (8 * CPC), core = (w / 8) % CPC, rr = w % 8;
        const int prow = rg * 8 + rr;                    // row of the piece (b of them)
        // ---- A role: piece (leaf xa, chunk kca): rows = i, k contiguous
        {
            const int xa = pc / CH, kca = pc % CH;
            const float* src = &raw[prow][xa * LEAF + kca * 16 + core * EPU];
            const size_t g = ((size_t)((Q0 + xa) * CH + kca) * nlp + I) * PIECE + (size_t)w * 16;
            if (PK != 3) {
                const float4 v = *reinterpret_cast<const float4*>(src);
                uint4 h, l;
                h.x = to_tf32(v.x); l.x = to_tf32(v.x - __uint_as_float(h.x));
                h.y = to_tf32(v.y); l.y = to_tf32(v.y - __uint_as_float(h.y));
                h.z = to_tf32(v.z); l.z = to_tf32(v.z - __uint_as_float(h.z));
                h.w = to_tf32(v.w); l.w = to_tf32(v.w - __uint_as_float(h.w));
                *reinterpret_cast<uint4*>(static_cast<unsigned char*>(pa0) + g) = h;
                if (PK == 2) *reinterpret_cast<uint4*>(static_cast<unsigned char*>(pa1) + g) = l;
            } else {
                const float4 v0 = *reinterpret_cast<const float4*>(src);
                const float4 v1 = *reinterpret_cast<const float4*>(src + 4);
                const float f[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(f[2 * q]);
                    const __nv_bfloat16 h1 = __float2bfloat16_rn(f[2 * q + 1]);
                    const __nv_bfloat16 l0 = __float2bfloat16_rn(f[2 * q] - __bfloat162float(h0));
                    const __nv_bfloat16 l1 = __float2bfloat16_rn(f[2 * q + 1] - __bfloat162float(h1));
                    hw[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                    lw[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                }
                *reinterpret_cast<uint4*>(static_cast<unsigned char*>(pa0) + g) =
                    make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(static_cast<unsigned char*>(pa1) + g) =
                    make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
        }
        // ---- B role: piece (chunk kcb, leaf xb): rows = column j of the leaf,
        //      k = row of the leaf contiguous
        {
            const int kcb = pc / TL, xb = pc % TL;
            const int colj = xb * LEAF + prow;           // staged column
            const int k0 = kcb * 16 + core * EPU;        // staged first row
            const size_t g = ((size_t)(I * CH + kcb) * nlp + (Q0 + xb)) * PIECE + (size_t)w * 16;
            if (PK != 3) {
                float f[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) f[q] = raw[k0 + q][colj];
                uint4 h, l;
                h.x = to_tf32(f[0]); l.x = to_tf32(f[0] - __uint_as_float(h.x));
                h.y = to_tf32(f[1]); l.y = to_tf32(f[1] - __uint_as_float(h.y));
                h.z = to_tf32(f[2]); l.z = to_tf32(f[2] - __uint_as_float(h.z));
                h.w = to_tf32(f[3]); l.w = to_tf32(f[3] - __uint_as_float(h.w));
                *reinterpret_cast<uint4*>(static_cast<unsigned char*>(pb0) + g) = h;
                if (PK == 2) *reinterpret_cast<uint4*>(static_cast<unsigned char*>(pb1) + g) = l;
            } else {
                float f[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) f[q] = raw[k0 + q][colj];
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(f[2 * q]);
                    const __nv_bfloat16 h1 = __float2bfloat16_rn(f[2 * q + 1]);
                    const __nv_bfloat16 l0 = __float2bfloat16_rn(f[2 * q] - __bfloat162float(h0));
                    const __nv_bfloat16 l1 = __float2bfloat16_rn(f[2 * q + 1] - __bfloat162float(h1));
                    hw[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                    lw[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                }
                *reinterpret_cast<uint4*>(static_cast<unsigned char*>(pb0) + g) =
                    make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(static_cast<unsigned char*>(pb1) + g) =
                    make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
        }
    }
}

// Five tiers per pass: a block reduces a (up to) 32 x 32 patch of tier L.
__global__ void __launch_bounds__(256) k_pyramid_up(double* __restrict__ pyr, int L, int levels) {
    __shared__ double sm[32 * 32];
    const int64_t wL = (int64_t)1 << L;
    const int side = wL < 32 ? (int)wL : 32;
    const int64_t bi = blockIdx.y, bj = blockIdx.x;
    const double* src = pyr + (((int64_t)1 << (2 * L)) - 1) / 3;
    for (int e = threadIdx.x; e < side * side; e += blockDim.x) {
        const int i = e / side, j = e % side;
        sm[i * 32 + j] = src[(bi * side + i) * wL + (bj * side + j)];
    }
    __syncthreads();
    int cur = side;
    for (int lv = 1; lv <= levels; ++lv) {
        const int half = cur >> 1;
        const int t = L - lv;
        const int64_t wt = (int64_t)1 << t;
        double* dst = pyr + (((int64_t)1 << (2 * t)) - 1) / 3;
        double v = 0.0;
        int i = 0, j = 0;
        const bool act = threadIdx.x < half * half;
        if (act) {
            i = threadIdx.x / half;
            j = threadIdx.x % half;
            const double a11 = sm[(2 * i) * 32 + 2 * j];
            const double a12 = sm[(2 * i) * 32 + 2 * j + 1];
            const double a21 = sm[(2 * i + 1) * 32 + 2 * j];
            const double a22 = sm[(2 * i + 1) * 32 + 2 * j + 1];
            v = a11 + a12 + a21 + a22;
            dst[(bi * half + i) * wt + (bj * half + j)] = v;
        }
        __syncthreads();
        if (act) sm[i * 32 + j] = v;
        __syncthreads();
        cur = half;
    }
}

cudaError_t launch_build_norms(spamm_tree* t, cudaStream_t s) {
    const int64_t off_leaf = (((int64_t)1 << (2 * t->d)) - 1) / 3;
    double* leaf = t->pyr + off_leaf;
    cudaError_t e = cudaMemsetAsync(leaf, 0, sizeof(double) * t->nb * t->nb, s);
    if (e != cudaSuccess) return e;
    const bool vec = ((reinterpret_cast<uintptr_t>(t->A) & 15) == 0) && (t->lda % 4 == 0);
    void* pa0 = t->packA[0];
    void* pa1 = t->packA[1];
    void* pb0 = t->packB[0];
    void* pb1 = t->packB[1];
    const int pk = t->precision == SPAMM_PREC_FP32    ? 0
                   : t->precision == SPAMM_PREC_TF32  ? 1
                   : t->precision == SPAMM_PREC_TF32X3 ? 2
                                                       : 3;
    if (pk == 0) {
        dim3 grid((unsigned)((t->nl * t->b + 511) / 512), (unsigned)t->nl);
        if (vec)
            k_leaf_norms<true><<<grid, 128, 0, s>>>(t->A, t->n, t->lda, t->b, t->nb, t->nl, leaf);
        else
            k_leaf_norms<false><<<grid, 128, 0, s>>>(t->A, t->n, t->lda, t->b, t->nb, t->nl, leaf);
    } else {
        const int tl = 128 / t->b;
        dim3 grid((unsigned)t->nl, (unsigned)(t->nlp / tl));
        const size_t smem = (size_t)t->b * (128 + 4) * sizeof(float);
#define SPAMM_LP(PKV, LV)                                                                      \
    do {                                                                                       \
        if (smem > 48 * 1024)                                                                  \
            cudaFuncSetAttribute(k_leaf_pack<PKV, LV>,                                         \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
        k_leaf_pack<PKV, LV><<<grid, 128, smem, s>>>(t->A, t->n, t->lda, t->nb, t->nl, t->nlp, \
                                                     leaf, pa0, pa1, pb0, pb1);                \
    } while (0)
#define SPAMM_LP_B(LV)                \
    do {                              \
        if (pk == 1) SPAMM_LP(1, LV); \
        else if (pk == 2) SPAMM_LP(2, LV); \
        else SPAMM_LP(3, LV);         \
    } while (0)
        if (t->b == 16) SPAMM_LP_B(16);
        else if (t->b == 32) SPAMM_LP_B(32);
        else if (t->b == 64) SPAMM_LP_B(64);
        else SPAMM_LP_B(128);
#undef SPAMM_LP_B
#undef SPAMM_LP
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int L = t->d;
    while (L > 0) {
        const int levels = L < 5 ? L : 5;
        const int64_t wL = (int64_t)1 << L;
        const int64_t blocks = wL < 32 ? 1 : wL / 32;
        k_pyramid_up<<<dim3((unsigned)blocks, (unsigned)blocks), 256, 0, s>>>(t->pyr, L, levels);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        L -= levels;
    }
    return cudaSuccess;
}

}  // namespace spamm
