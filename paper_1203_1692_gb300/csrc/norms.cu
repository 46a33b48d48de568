// Stage 1: the FP64 norm quadtree (Sec. II.A-B, Eq. (norm)) and, for the
// tensor-core precisions, the leaf tiles in tcgen05 shared-memory layout.
//
// Leaf squares: a thread owns four consecutive columns of one leaf row-strip
// and sums (double)a * (double)a (exact) down the strip's b rows; the b/4
// lanes that share a leaf combine their partial sums with a segmented
// xor-shuffle reduction.  The kernel reads each element of A once, with
// 16-byte loads when A and lda allow it, so it is bound by HBM bandwidth.
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

// PK: 0 none, 1 tf32 hi, 2 tf32 hi+lo, 3 bf16 hi+lo
template <int PK, bool VEC>
__global__ void __launch_bounds__(128) k_leaf_norms(const float* __restrict__ A, int64_t n,
                                                    int64_t lda, int b, int64_t nb, int64_t nl,
                                                    int64_t nlp, double* __restrict__ leaf,
                                                    void* __restrict__ pa0, void* __restrict__ pa1,
                                                    void* __restrict__ pb0, void* __restrict__ pb1) {
    const int64_t I = blockIdx.y;                       // leaf row
    const int64_t col0 = (int64_t)blockIdx.x * 512 + 4 * threadIdx.x;
    const int64_t K = col0 / b;                          // leaf column
    const int lanes = b >> 2;                            // lanes per leaf
    double s = 0.0;
    const int64_t r0 = I * b;
    const int kk = (int)(col0 - K * b);                  // column inside the leaf
    const int chunks = b >> 4;
    const size_t piece_elems = (size_t)b * 16;
    for (int r = 0; r < b; ++r) {
        const int64_t row = r0 + r;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < n) {
            const float* p = A + row * lda + col0;
            if (VEC) {
                if (col0 + 3 < n) {
                    v = __ldg(reinterpret_cast<const float4*>(p));
                } else {
                    if (col0 + 0 < n) v.x = __ldg(p + 0);
                    if (col0 + 1 < n) v.y = __ldg(p + 1);
                    if (col0 + 2 < n) v.z = __ldg(p + 2);
                }
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
        if (PK != 0 && K < nl) {
            // A role: leaf (I, K), row r, chunk k' = kk.
            const int kc = kk >> 4, kq = kk & 15;
            const size_t pieceA = ((size_t)(K * chunks + kc) * nlp + I) * piece_elems;
            // B role: leaf (K=I, J=K): n-index = kk..kk+3, k index = r.
            const int bkc = r >> 4, bkq = r & 15;
            const size_t pieceB = ((size_t)(I * chunks + bkc) * nlp + K) * piece_elems;
            if (PK == 1 || PK == 2) {
                uint32_t h[4], l[4];
                const float f[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    h[q] = to_tf32(f[q]);
                    l[q] = to_tf32(f[q] - __uint_as_float(h[q]));
                }
                // element offset inside a TF32 piece: row g, k q ->
                // (g%8)*4 + (g/8)*128 + (q%4) + (q/4)*32   (in 4-byte words)
                const size_t offA = pieceA + (r & 7) * 4 + (r >> 3) * 128 + (kq >> 2) * 32;
                reinterpret_cast<uint4*>(pa0)[offA >> 2] = make_uint4(h[0], h[1], h[2], h[3]);
                if (PK == 2)
                    reinterpret_cast<uint4*>(pa1)[offA >> 2] = make_uint4(l[0], l[1], l[2], l[3]);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int nn = kk + q;
                    const size_t offB = pieceB + (nn & 7) * 4 + (nn >> 3) * 128 + (bkq & 3) +
                                        (bkq >> 2) * 32;
                    reinterpret_cast<uint32_t*>(pb0)[offB] = h[q];
                    if (PK == 2) reinterpret_cast<uint32_t*>(pb1)[offB] = l[q];
                }
            } else {  // BF16 hi/lo, core matrix = 8 rows x 8 elements
                __nv_bfloat16 h[4], l[4];
                const float f[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    h[q] = __float2bfloat16_rn(f[q]);
                    l[q] = __float2bfloat16_rn(f[q] - __bfloat162float(h[q]));
                }
                // element offset inside a BF16 piece: row g, k q ->
                // (g%8)*8 + (g/8)*128 + (q%8) + (q/8)*64   (in 2-byte elements)
                const size_t offA = pieceA + (r & 7) * 8 + (r >> 3) * 128 + (kq & 7) + (kq >> 3) * 64;
                uint2 hv, lv;
                hv.x = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
                hv.y = (uint32_t)__bfloat16_as_ushort(h[2]) | ((uint32_t)__bfloat16_as_ushort(h[3]) << 16);
                lv.x = (uint32_t)__bfloat16_as_ushort(l[0]) | ((uint32_t)__bfloat16_as_ushort(l[1]) << 16);
                lv.y = (uint32_t)__bfloat16_as_ushort(l[2]) | ((uint32_t)__bfloat16_as_ushort(l[3]) << 16);
                reinterpret_cast<uint2*>(pa0)[offA >> 2] = hv;
                reinterpret_cast<uint2*>(pa1)[offA >> 2] = lv;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int nn = kk + q;
                    const size_t offB = pieceB + (nn & 7) * 8 + (nn >> 3) * 128 + (bkq & 7) +
                                        (bkq >> 3) * 64;
                    reinterpret_cast<__nv_bfloat16*>(pb0)[offB] = h[q];
                    reinterpret_cast<__nv_bfloat16*>(pb1)[offB] = l[q];
                }
            }
        }
    }
    // segmented reduction over the lanes of one leaf
    for (int off = lanes >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & (lanes - 1)) == 0 && K < nl) leaf[I * nb + K] = s;
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
    dim3 grid((unsigned)((t->nl * t->b + 511) / 512), (unsigned)t->nl);
    void* pa0 = t->packA[0];
    void* pa1 = t->packA[1];
    void* pb0 = t->packB[0];
    void* pb1 = t->packB[1];
#define SPAMM_LN(PK, V)                                                                      \
    k_leaf_norms<PK, V><<<grid, 128, 0, s>>>(t->A, t->n, t->lda, t->b, t->nb, t->nl, t->nlp, \
                                             leaf, pa0, pa1, pb0, pb1)
    const int pk = t->precision == SPAMM_PREC_FP32    ? 0
                   : t->precision == SPAMM_PREC_TF32  ? 1
                   : t->precision == SPAMM_PREC_TF32X3 ? 2
                                                       : 3;
    if (vec) {
        switch (pk) {
            case 0: SPAMM_LN(0, true); break;
            case 1: SPAMM_LN(1, true); break;
            case 2: SPAMM_LN(2, true); break;
            default: SPAMM_LN(3, true); break;
        }
    } else {
        switch (pk) {
            case 0: SPAMM_LN(0, false); break;
            case 1: SPAMM_LN(1, false); break;
            case 2: SPAMM_LN(2, false); break;
            default: SPAMM_LN(3, false); break;
        }
    }
#undef SPAMM_LN
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
