// Stage 1: the FP64 norm quadtree (Sec. II.A-B, Eq. (norm)); and, for the
// tensor-core precisions, the leaf tiles in tcgen05 shared-memory layout,
// written inside a multiply (after the thresholds are known) for the leaves
// that can take part in a kept product only.
//
// Leaf squares: a thread owns four consecutive columns of one leaf row-strip
// and sums their squares down the strip's b rows (exact squares, FP32-pair
// accumulation folded into FP64, see k_leaf_norms); the b/4 lanes that share
// a leaf combine their partial sums with a segmented xor-shuffle reduction.
// The kernel reads each element of A once, with 16-byte loads when A and lda
// allow it, so it is bound by HBM bandwidth.
// The upper tiers come from a second kernel that builds five tiers per pass
// in shared memory, each node the sum of its four children in the order
// A11 + A12 + A21 + A22.
//
// Tensor-core tiles (precision != FP32).  The K dimension of a leaf is cut
// into chunks of 16; a "piece" is one leaf x one chunk, b rows x 16 k.
// Inside a piece the rows are grouped by 8: a row group holds the core
// matrices (8 rows x 16 bytes) of the chunk one after another (leading byte
// offset 128 B), and row groups follow each other at the stride-byte offset
// (512 B for TF32, 256 B for 16-bit parts): the no-swizzle K-major canonical
// layout of tcgen05.  The A role holds leaf (I, K) with rows = i (K-major as
// stored); the B role holds leaf (K, J) transposed, rows = j.  Pieces are
// grouped the way one C tile reads them: a tile's rows are TL = 128 / b
// consecutive leaves, its columns 2 TL, so with G the group size (TL for the
// A role, 2 TL for the B role), P the parts (hi, lo), CH = b / 16 and the
// chunks of a leaf taken CG at a time (pack_group_chunks: the chunks one
// stage of the leaf kernel holds), chunk kc = q CG + c,
//     piece(K, x, kc, part) at (((((K * nlp/G + x/G) * CH/CG + q) * P + part)
//                                 * CG + c) * G + x % G) * piece_bytes
// (K = the shared index, x = the leaf's other index).  The G pieces of one
// group, chunk and part form the 128 x 16 (A) or 256 x 16 (B) operand slice
// of one MMA; the high parts of CG chunks come first, then their low parts,
// and the groups of one K follow each other.  So everything a stage needs
// from one operand is one contiguous run, and its high parts alone (a step
// whose products all run one pass, precision chosen by norm) another, each
// moved by a single bulk copy into shared memory already in the layout the
// MMA reads.  Sparsified trees keep their own banded layout (one array per
// part, see k_leaf_pack).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "spamm_internal.cuh"

namespace spamm {

bool precision_uses_tc(int p) { return p != SPAMM_PREC_FP32; }

int pack_arrays_for(int p) { return p == SPAMM_PREC_TF32 ? 1 : 2; }

static int elem_bytes(int p) {
    return (p == SPAMM_PREC_BF16X3 || p == SPAMM_PREC_F16X3) ? 2 : 4;
}

size_t pack_bytes_for(int p, int64_t nlp, int b) {
    if (!precision_uses_tc(p)) return 0;
    return (size_t)nlp * b * (size_t)nlp * b * elem_bytes(p);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Eight values into hi and lo 16-bit parts, two per word: BF16 (PK 3) as
// they are, FP16 (PK 4) after scaling by the operand's power of two.
template <int PK>
__device__ __forceinline__ void split16(const float (&f)[8], float sc, uint32_t (&hw)[4],
                                        uint32_t (&lw)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if constexpr (PK == 3) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(f[2 * q]);
            const __nv_bfloat16 h1 = __float2bfloat16_rn(f[2 * q + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(f[2 * q] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(f[2 * q + 1] - __bfloat162float(h1));
            hw[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lw[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        } else {
            const float x0 = __fmul_rn(f[2 * q], sc), x1 = __fmul_rn(f[2 * q + 1], sc);
            const __half h0 = __float2half_rn(x0);
            const __half h1 = __float2half_rn(x1);
            const __half l0 = __float2half_rn(__fsub_rn(x0, __half2float(h0)));
            const __half l1 = __float2half_rn(__fsub_rn(x1, __half2float(h1)));
            hw[q] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
            lw[q] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
        }
    }
}

// Leaf squared norms without the FP64 pipe, which is narrow on GB300.
//
// A block covers one leaf row-strip (LEAF rows) x 512 columns; a thread owns
// four consecutive columns.  Its squares are summed in FP32 pairs: with x
// scaled by a power of two to xs in [0, 2), xs^2 = p + e exactly (p = xs*xs,
// e = fma(xs, xs, -p)), p enters the running pair (hi, lo) through an
// error-free two-sum and e goes into lo.  The scale follows the largest
// exponent seen so far (rescaling the pair exactly by a power of two; terms
// 2^-100 below the largest square are far under FP64's resolution of the
// sum).  Every eight rows the pair is folded into an FP64 sum, so a pair
// holds at most 32 terms and the sum's relative error stays near 1e-13, far
// inside the 1e-6 band the cull reports around tau.  The lanes of one leaf
// then combine their FP64 sums with a segmented xor-shuffle reduction.
// Inf or NaN anywhere makes the leaf's norm NaN.
__device__ __forceinline__ float pow2f(int k) {          // 2^k, k in [-127, 127]
    return k >= -126 ? __int_as_float((k + 127) << 23) : __int_as_float(1 << 22);
}

__device__ __forceinline__ double pow2d(int k) {         // 2^k, k in [-1022, 1023]
    return __longlong_as_double((long long)(k + 1023) << 52);
}

struct SqAcc {
    float hi = 0.f, lo = 0.f, sc = 0x1p127f;
    int E = 0;                  // biased exponent of the scale: x = xs * 2^(E - 127)
    bool bad = false;
    double sum = 0.0;

    // explicit round-to-nearest operations: the error-free transformations
    // must not be contracted into fused multiply-adds
    __device__ __forceinline__ void add1(float x) {
        const float xs = __fmul_rn(x, sc);
        const float p = __fmul_rn(xs, xs);
        const float e = fmaf(xs, xs, -p);
        const float t = __fadd_rn(hi, p);
        const float bp = __fsub_rn(t, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ __forceinline__ void add4(float4 v) {
        const int m = max(max((__float_as_int(v.x) >> 23) & 0xff, (__float_as_int(v.y) >> 23) & 0xff),
                          max((__float_as_int(v.z) >> 23) & 0xff, (__float_as_int(v.w) >> 23) & 0xff));
        if (m == 0xff) {
            bad = true;
            return;
        }
        if (m > E) {
            const int k = 2 * (E - m);
            const float f = k >= -126 ? pow2f(k) : 0.f;
            hi = __fmul_rn(hi, f);
            lo = __fmul_rn(lo, f);
            E = m;
            sc = pow2f(127 - E);
        }
        add1(v.x);
        add1(v.y);
        add1(v.z);
        add1(v.w);
    }
    __device__ __forceinline__ void fold() {
        sum = __dadd_rn(sum, __dmul_rn(__dadd_rn((double)hi, (double)lo), pow2d(2 * E - 254)));
        hi = lo = 0.f;
    }
    __device__ __forceinline__ double result() {
        fold();
        return bad ? __longlong_as_double(0x7ff8000000000000ll) : sum;
    }
};

// PAN: also the panel norms of the sub-leaf cull along k (16-wide slices):
// panA[(I nl + K) SL + s] over the b rows of leaf I and the 16 columns of
// slice s of leaf K (the four lanes of a 16-column group), and
// panB[(I SL + s) nl + K] over the 16 rows of slice s of leaf I and the b
// columns of leaf K (a partial per 16 rows, then all the lanes of the leaf).
template <int LEAF, bool VEC, bool PAN>
__global__ void __launch_bounds__(128) k_leaf_norms(const float* __restrict__ A, int64_t n,
                                                    int64_t lda, int64_t nb, int64_t nl,
                                                    double* __restrict__ leaf,
                                                    double* __restrict__ panA,
                                                    double* __restrict__ panB) {
    constexpr int SL = PAN ? LEAF / 16 : 1;              // 16-row groups tracked
    const int64_t I = blockIdx.y;                       // leaf row
    const int64_t col0 = (int64_t)blockIdx.x * 512 + 4 * threadIdx.x;
    const int64_t K = col0 / LEAF;                       // leaf column
    constexpr int lanes = LEAF / 4;                      // lanes per leaf
    const int64_t r0 = I * LEAF;
    const float* base = A + r0 * lda + col0;
    SqAcc acc;
    double rp[SL];                                       // per 16-row group (PAN)
#pragma unroll
    for (int q = 0; q < SL; ++q) rp[q] = 0.0;
    auto group_done = [&](int r) {                       // after row r (0-based)
        if (PAN && (r & 15) == 15) {
            rp[r >> 4] = acc.sum;
            acc.sum = 0.0;
        }
    };
    if (VEC && col0 + 3 < n && r0 + LEAF <= n) {
        for (int r8 = 0; r8 < LEAF; r8 += 8) {
            float4 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                v[q] = __ldg(reinterpret_cast<const float4*>(base + (int64_t)(r8 + q) * lda));
#pragma unroll
            for (int q = 0; q < 8; ++q) acc.add4(v[q]);
            acc.fold();
            group_done(r8 + 7);
        }
    } else {
        int r = 0;
        for (; r < LEAF; ++r) {
            if (r0 + r >= n) break;
            const float* p = base + (int64_t)r * lda;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (col0 + 0 < n) v.x = __ldg(p + 0);
            if (col0 + 1 < n) v.y = __ldg(p + 1);
            if (col0 + 2 < n) v.z = __ldg(p + 2);
            if (col0 + 3 < n) v.w = __ldg(p + 3);
            acc.add4(v);
            if ((r & 7) == 7) acc.fold();
            group_done(r);
        }
        if (PAN && (r & 15) != 0 && r < LEAF) {          // rows ran out mid-group
            acc.fold();
            rp[r >> 4] = acc.sum;
            acc.sum = 0.0;
        }
    }
    double s;
    if (PAN) {
        s = 0.0;
#pragma unroll
        for (int q = 0; q < SL; ++q) s += rp[q];
        if (acc.bad) s = __longlong_as_double(0x7ff8000000000000ll);
        // A-role panel: the four lanes of this 16-column group
        double pa = s;
        pa += __shfl_xor_sync(0xffffffffu, pa, 1);
        pa += __shfl_xor_sync(0xffffffffu, pa, 2);
        if ((threadIdx.x & 3) == 0 && K < nl)
            panA[((int64_t)I * nl + K) * SL + (int)((col0 % LEAF) >> 4)] = pa;
        // B-role panels: every 16-row group over all lanes of the leaf
#pragma unroll
        for (int q = 0; q < SL; ++q) {
            double pb = acc.bad ? __longlong_as_double(0x7ff8000000000000ll) : rp[q];
            for (int off = lanes >> 1; off > 0; off >>= 1)
                pb += __shfl_xor_sync(0xffffffffu, pb, off);
            if ((threadIdx.x & (lanes - 1)) == 0 && K < nl)
                panB[((int64_t)I * SL + q) * nl + K] = pb;
        }
        // leaf norm: the 16-column sums over the remaining lanes
        s = pa;
        for (int off = 4; off < lanes; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    } else {
        s = acc.result();
        // segmented reduction over the lanes of one leaf
        for (int off = lanes >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    }
    if ((threadIdx.x & (lanes - 1)) == 0 && K < nl) leaf[I * nb + K] = s;
}

// Per-K maxima of the leaf squared norms, which bound every leaf product a
// multiply can keep (the SpAMM condition is monotone in each norm):
//   colmaxA[K] = max_I ||A_IK||^2,   rowmaxB[K] = max_J ||B_KJ||^2.
// A piece of A (I, K) can be read only if ||A_IK||^2 * rowmaxB[K] passes the
// condition, a piece of B (K, J) only if colmaxA[K] * ||B_KJ||^2 does.
// blockIdx.y = 0: a block per 32 columns of A, lane = column, the eight
// warps split the rows and combine their maxima in shared memory;
// blockIdx.y = 1: a warp per row K of B.
__global__ void __launch_bounds__(256) k_leaf_max(const double* __restrict__ leafA,
                                                  const double* __restrict__ leafB, int64_t nb,
                                                  int64_t nl, double* __restrict__ colmaxA,
                                                  double* __restrict__ rowmaxB,
                                                  double* __restrict__ gmax) {
    __shared__ double part[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.y == 0) {
        for (int64_t K0 = (int64_t)blockIdx.x * 32; K0 < nl; K0 += (int64_t)gridDim.x * 32) {
            const int64_t K = K0 + lane;
            double m = 0.0;
            if (K < nl) {
#pragma unroll 4
                for (int64_t I = warp; I < nl; I += 8) m = fmax(m, leafA[I * nb + K]);
            }
            part[warp][lane] = m;
            __syncthreads();
            if (warp == 0 && K < nl) {
                double r = part[0][lane];
#pragma unroll
                for (int w = 1; w < 8; ++w) r = fmax(r, part[w][lane]);
                colmaxA[K] = r;
                // largest leaf of A (non-negative doubles order like their bits)
                atomicMax(reinterpret_cast<unsigned long long*>(gmax),
                          (unsigned long long)__double_as_longlong(r));
            }
            __syncthreads();
        }
    } else {
        const int64_t warps = (int64_t)gridDim.x * 8;
        for (int64_t K = (int64_t)blockIdx.x * 8 + warp; K < nl; K += warps) {
            double m = 0.0;
#pragma unroll 4
            for (int64_t J = lane; J < nl; J += 32) m = fmax(m, leafB[K * nb + J]);
            for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) {
                rowmaxB[K] = m;
                atomicMax(reinterpret_cast<unsigned long long*>(gmax + 1),
                          (unsigned long long)__double_as_longlong(m));
            }
        }
    }
}

// Tensor-core packs of the leaves a multiply can read.  A block owns one
// leaf row-strip (b rows) x 128 columns (TL leaves): it decides which of its
// leaves are needed as A-role pieces (rowmaxB given) and as B-role pieces
// (colmaxA given) with the SpAMM condition above, returns at once if none
// is, else stages the strip in shared memory (16-byte loads) and produces
// the needed pieces in output order: with T threads, thread t writes the
// t-th, (t+T)-th, ... 16-byte unit of each piece, reading the elements that unit holds from the
// staged strip (a row quad for the A role, a column quad for the B role),
// splitting them into hi/lo parts and storing both parts.  Every piece is
// a contiguous run of at least 512 bytes and consecutive threads write its
// consecutive 16-byte units: every global store is coalesced.  PK: 1 tf32
// hi, 2 tf32 hi+lo, 3 bf16 hi+lo, 4 scaled fp16 hi+lo.
// BAND: a sparsified tree; the strip comes from the leaf row's slab and the
// pieces go to their place inside the column (A role) or row (B role) band.
// Threads per pack block: 256 for b >= 32, 128 for b = 16 (each the
// faster measured form at n = 7500).
template <int LEAF>
constexpr int pack_threads() { return LEAF >= 32 ? 256 : 128; }

template <int PK, int LEAF, bool BAND>
__global__ void __launch_bounds__(pack_threads<LEAF>()) k_leaf_pack(const float* __restrict__ A, int64_t n,
                                                   int64_t lda, int64_t nb, int64_t nl, int64_t nlp,
                                                   const double* __restrict__ leaf,
                                                   const double* __restrict__ rowmaxB,
                                                   const double* __restrict__ colmaxA, Thresh th,
                                                   void* __restrict__ pa0, void* __restrict__ pa1,
                                                   void* __restrict__ pb0, void* __restrict__ pb1,
                                                   BandView bv, const double* __restrict__ gmax_a,
                                                   const double* __restrict__ gmax_b,
                                                   unsigned long long* __restrict__ packed) {
    constexpr int kPackThreads = pack_threads<LEAF>();
    constexpr int kPackWarps = kPackThreads / 32;
    constexpr int TL = 128 / LEAF;
    constexpr int CH = LEAF / 16;
    constexpr int ES = PK >= 3 ? 2 : 4;                  // element bytes
    constexpr int EPU = 16 / ES;                         // elements per 16-byte unit
    constexpr int PIECE = LEAF * 16 * ES;                // bytes of one piece
    constexpr int UPP = PIECE / 16;                      // units per piece
    constexpr int CPC = 16 / EPU;                        // core matrices per 16-wide K chunk
    constexpr int LDS = 128 + 4;                         // padded staging row
    constexpr int NPART = PK == 1 ? 1 : 2;               // hi (and lo) parts
    // chunks per pack group (high parts of the group, then low parts)
    constexpr int CG = pack_group_chunks(LEAF, PK == 2 ? SPAMM_PREC_TF32X3 : SPAMM_PREC_F16X3);
    extern __shared__ __align__(16) float raw_dyn[];     // LEAF x LDS staged strip
    float (*raw)[LDS] = reinterpret_cast<float (*)[LDS]>(raw_dyn);
    __shared__ int needA[TL], needB[TL], any;
    // leaf rows vary fastest across blocks, so the blocks running at once
    // write neighbouring A-role pieces
    const int64_t I = blockIdx.x;                        // leaf row
    const int64_t Q0 = (int64_t)blockIdx.y * TL;         // first leaf column
    const int64_t r0 = I * LEAF, c0 = Q0 * LEAF;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    if (t == 0) any = 0;
    __syncthreads();
    if (t < TL) {
        const int64_t Q = Q0 + t;
        bool tie;
        const double nq = Q < nl ? leaf[I * nb + Q] : 0.0;
        needA[t] = (rowmaxB && Q < nl && spamm_keep(nq, rowmaxB[Q], th, &tie)) ? 1 : 0;
        needB[t] = (colmaxA && Q < nl && spamm_keep(colmaxA[I], nq, th, &tie)) ? 1 : 0;
        if (needA[t] | needB[t]) atomicOr(&any, 1);
    }
    if (warp == 0) {
        // the leaves this block packs, per role (one atomic per role and block)
        const unsigned ba = __ballot_sync(0xffffffffu, t < TL && needA[t]);
        const unsigned bb = __ballot_sync(0xffffffffu, t < TL && needB[t]);
        if (lane == 0 && ba) atomicAdd(packed, (unsigned long long)__popc(ba));
        if (lane == 0 && bb) atomicAdd(packed + 1, (unsigned long long)__popc(bb));
    }
    __syncthreads();
    if (!any) return;
    // FP16 split: the operand's power-of-two scale, per role
    float sc_a = 1.f, sc_b = 1.f;
    if constexpr (PK == 4) {
        sc_a = ldexpf(1.f, f16_scale_exp(*gmax_a));
        sc_b = ldexpf(1.f, f16_scale_exp(*gmax_b));
    }
    const int cq = 4 * lane;
    if constexpr (BAND) {
        // the slab holds the columns [kmin b, (kmax + 1) b) of this leaf row
        const int kmin = bv.kmin[I], kmax = bv.kmax[I];
        const int64_t w = (int64_t)(kmax - kmin + 1) * LEAF;
        const float* srow = bv.slab + bv.roff[I];
#pragma unroll 4
        for (int r = warp; r < LEAF; r += kPackWarps) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            const int64_t sc = c0 + cq - (int64_t)kmin * LEAF;    // slab column
            if (kmin <= kmax && sc >= 0 && sc + 3 < w)
                v = __ldg(reinterpret_cast<const float4*>(srow + r * w + sc));
            *reinterpret_cast<float4*>(&raw[r][cq]) = v;
        }
    } else {
        const bool vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda % 4 == 0);
#pragma unroll 4
        for (int r = warp; r < LEAF; r += kPackWarps) {
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
            *reinterpret_cast<float4*>(&raw[r][cq]) = v;
        }
    }
    __syncthreads();
    // pieces, in output order
    constexpr int UNITS = TL * CH * UPP;                 // per role and part
    for (int u = t; u < UNITS; u += kPackThreads) {
        const int pc = u / UPP, w = u % UPP;
        // unit w of a piece: row group w / (8 CPC), core (w / 8) % CPC, row w % 8
        const int rg = w / (8 * CPC), core = (w / 8) % CPC, rr = w % 8;
        const int prow = rg * 8 + rr;                    // row of the piece (b of them)
        // ---- A role: piece (leaf xa, chunk kca): rows = i, k contiguous
        bool roleA = pa0 && needA[pc / CH];
        if constexpr (BAND) {
            // a kept leaf lies inside its band; the test keeps every store
            // inside the tree's storage even for norms that do not match the
            // bands (a tree left by a failed re-sparsify)
            const int64_t K = Q0 + pc / CH;
            if (roleA && (I < bv.imin[K] || I > bv.imax[K])) roleA = false;
        }
        if (roleA) {
            const int xa = pc / CH, kca = pc % CH;
            const float* src = &raw[prow][xa * LEAF + kca * 16 + core * EPU];
            size_t g;
            if constexpr (BAND) {
                const int64_t K = Q0 + xa;
                const int64_t len = bv.imax[K] - bv.imin[K] + 1;
                g = (size_t)(bv.aoff[K] + kca * len + (I - bv.imin[K])) * PIECE + (size_t)w * 16;
            } else {
                const int64_t grp = ((Q0 + xa) * (nlp / TL) + I / TL) * (CH / CG) + kca / CG;
                const int64_t slot = grp * NPART * CG + kca % CG;   // its high-part slice
                g = (size_t)(slot * TL + I % TL) * PIECE + (size_t)w * 16;
            }
            if (PK <= 2) {
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
                split16<PK>(f, sc_a, hw, lw);
                *reinterpret_cast<uint4*>(static_cast<unsigned char*>(pa0) + g) =
                    make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(static_cast<unsigned char*>(pa1) + g) =
                    make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
        }
        // ---- B role: piece (chunk kcb, leaf xb): rows = column j of the leaf,
        //      k = row of the leaf contiguous
        if (pb0 && needB[pc % TL]) {
            const int kcb = pc / TL, xb = pc % TL;
            const int colj = xb * LEAF + prow;           // staged column
            const int k0 = kcb * 16 + core * EPU;        // staged first row
            size_t g;
            if constexpr (BAND) {
                if (Q0 + xb < bv.kmin[I] || Q0 + xb > bv.kmax[I]) continue;   // as for A
                const int64_t len = bv.kmax[I] - bv.kmin[I] + 1;
                g = (size_t)(bv.boff[I] + kcb * len + (Q0 + xb - bv.kmin[I])) * PIECE +
                    (size_t)w * 16;
            } else {
                const int64_t grp = (I * (nlp / (2 * TL)) + (Q0 + xb) / (2 * TL)) * (CH / CG) +
                                    kcb / CG;                 // pack group of the chunk
                const int64_t slot = grp * NPART * CG + kcb % CG;   // its high-part slice
                g = (size_t)(slot * (2 * TL) + (Q0 + xb) % (2 * TL)) * PIECE + (size_t)w * 16;
            }
            if (PK <= 2) {
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
                split16<PK>(f, sc_b, hw, lw);
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
    dim3 grid((unsigned)((t->nl * t->b + 511) / 512), (unsigned)t->nl);
#define SPAMM_LN(LV)                                                                         \
    do {                                                                                     \
        if (t->slices) {                                                                     \
            if (vec)                                                                         \
                k_leaf_norms<LV, true, true><<<grid, 128, 0, s>>>(                           \
                    t->A, t->n, t->lda, t->nb, t->nl, leaf, t->panA, t->panB);               \
            else                                                                             \
                k_leaf_norms<LV, false, true><<<grid, 128, 0, s>>>(                          \
                    t->A, t->n, t->lda, t->nb, t->nl, leaf, t->panA, t->panB);               \
        } else {                                                                             \
            if (vec)                                                                         \
                k_leaf_norms<LV, true, false><<<grid, 128, 0, s>>>(                          \
                    t->A, t->n, t->lda, t->nb, t->nl, leaf, nullptr, nullptr);               \
            else                                                                             \
                k_leaf_norms<LV, false, false><<<grid, 128, 0, s>>>(                         \
                    t->A, t->n, t->lda, t->nb, t->nl, leaf, nullptr, nullptr);               \
        }                                                                                    \
    } while (0)
    if (t->b == 16) SPAMM_LN(16);
    else if (t->b == 32) SPAMM_LN(32);
    else if (t->b == 64) SPAMM_LN(64);
    else SPAMM_LN(128);
#undef SPAMM_LN
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_pyramid(t, s);
}

cudaError_t launch_pyramid(spamm_tree* t, cudaStream_t s) {
    int L = t->d;
    while (L > 0) {
        const int levels = L < 5 ? L : 5;
        const int64_t wL = (int64_t)1 << L;
        const int64_t blocks = wL < 32 ? 1 : wL / 32;
        k_pyramid_up<<<dim3((unsigned)blocks, (unsigned)blocks), 256, 0, s>>>(t->pyr, L, levels);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        L -= levels;
    }
    return cudaSuccess;
}

// ------------------------------------------------------- sparsification
// A leaf is kept iff its squared norm passes the SpAMM test against
// norm2_max = max(||A||_F^2, partner_norm2), the largest squared Frobenius
// norm it can meet in a product (the paper's drop tolerance epsilon =
// tau / max ||.||_F in squared form); a dropped leaf's norm and panel norms
// become zero, so no cull ever keeps it.  Then the bands of the kept
// leaves: per leaf row I the first and last kept column (kmin, kmax), per
// leaf column K the first and last kept row (imin, imax); an empty band has
// min > max.  The dense root is read before any leaf changes (it is the leaf
// when d = 0) and recorded in out[1]; a non-finite root drops nothing, so
// the rebuilt tiers keep the Inf/NaN and a multiply reports it.  out[0]
// counts the kept leaves.
__global__ void __launch_bounds__(256) k_sparse_mark(double* leaf, int64_t nb,
                                                     int64_t nl, Thresh th,
                                                     const double* root,   // may be the leaf
                                                     double partner_norm2, int SL,
                                                     double* __restrict__ panA,
                                                     double* __restrict__ panB,
                                                     unsigned long long* __restrict__ out) {
    const double r = *root;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[1] = __double_as_longlong(r);
    if (!isfinite(r)) return;
    const double norm2_max = fmax(r, partner_norm2);
    __syncthreads();   // every thread of block 0 has read the root before a leaf changes
    unsigned long long kept = 0;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nl * nl;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t I = g / nl, K = g % nl;
        bool tie;
        if (spamm_keep(leaf[I * nb + K], norm2_max, th, &tie)) {
            ++kept;
            continue;
        }
        leaf[I * nb + K] = 0.0;
        for (int q = 0; q < SL; ++q) {
            panA[(I * nl + K) * SL + q] = 0.0;
            panB[(I * SL + q) * nl + K] = 0.0;
        }
    }
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    if ((threadIdx.x & 31) == 0 && kept) atomicAdd(out, kept);
}

// A warp per leaf row (blockIdx.y = 0: kmin, kmax) or per leaf column
// (blockIdx.y = 1: imin, imax; strided loads, but every column in flight at
// once rather than one latency-bound walk down each column).
__global__ void __launch_bounds__(256) k_bands(const double* __restrict__ leaf, int64_t nb,
                                               int64_t nl, int32_t* __restrict__ band) {
    const int lane = threadIdx.x & 31;
    const bool rows = blockIdx.y == 0;
    // leaf (L, q) of line L: row L's leaf column q, or column L's leaf row q
    const int64_t s_line = rows ? nb : 1, s_q = rows ? 1 : nb;
    int32_t* lo_out = band + (rows ? 0 : 2 * nl);
    int32_t* hi_out = lo_out + nl;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t L = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); L < nl;
         L += warps) {
        int lo = (int)nl, hi = -1;
        for (int64_t q = lane; q < nl; q += 32)
            if (leaf[L * s_line + q * s_q] > 0.0) {
                lo = min(lo, (int)q);
                hi = max(hi, (int)q);
            }
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            lo_out[L] = lo;
            hi_out[L] = hi;
        }
    }
}

cudaError_t launch_sparsify_mark(spamm_tree* t, double tau, double partner_norm2, double rel,
                                 int32_t* band, unsigned long long* out, cudaStream_t s) {
    const int64_t off_leaf = (((int64_t)1 << (2 * t->d)) - 1) / 3;
    double* leaf = t->pyr + off_leaf;
    const Thresh th = make_thresh(tau, rel);
    const int64_t m = t->nl * t->nl;
    const int blocks = (int)std::min<int64_t>((m + 255) / 256, 4096);
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_sparse_mark<<<std::max(blocks, 1), 256, 0, s>>>(leaf, t->nb, t->nl, th, t->pyr,
                                                      partner_norm2, t->slices, t->panA,
                                                      t->panB, out);
    const int bb = (int)std::max<int64_t>(1, std::min<int64_t>((t->nl + 7) / 8, 4096));
    k_bands<<<dim3(bb, 2), 256, 0, s>>>(leaf, t->nb, t->nl, band);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_pyramid(t, s);
}

// One matrix row per block: the columns of its leaf row's band, kept leaves
// copied and dropped ones zeroed (zero beyond n).
__global__ void __launch_bounds__(256) k_slab_copy(const float* __restrict__ A, int64_t lda,
                                                   int64_t n, int b, int64_t nb,
                                                   const double* __restrict__ leaf, BandView bv,
                                                   float* __restrict__ slab) {
    const int64_t row = blockIdx.x;                     // 0 .. nl * b - 1
    const int64_t I = row / b, r = row % b;
    const int kmin = bv.kmin[I], kmax = bv.kmax[I];
    if (kmin > kmax) return;
    const int64_t w = (int64_t)(kmax - kmin + 1) * b;
    float* dst = slab + bv.roff[I] + r * w;
    for (int64_t c = threadIdx.x; c < w; c += blockDim.x) {
        const int64_t col = (int64_t)kmin * b + c;
        const bool live = row < n && col < n && leaf[I * nb + col / b] > 0.0;
        dst[c] = live ? A[row * lda + col] : 0.f;
    }
}

cudaError_t launch_slab_copy(spamm_tree* t, const float* A, int64_t lda, cudaStream_t s) {
    const int64_t off_leaf = (((int64_t)1 << (2 * t->d)) - 1) / 3;
    const int64_t rows = t->nl * t->b;
    if (rows == 0) return cudaSuccess;
    k_slab_copy<<<(unsigned)rows, 256, 0, s>>>(A, lda, t->n, t->b, t->nb, t->pyr + off_leaf,
                                                band_view(t), t->slab);
    return cudaGetLastError();
}

// Packs for one multiply: the per-K maxima of the two leaf tiers, then the
// needed A-role pieces of A and B-role pieces of B (one pass when A and B are
// the same tree).  `scratch` holds 2 nb doubles.
cudaError_t launch_packs(DevCtl* ctl, const spamm_tree* A, const spamm_tree* B, double tau,
                         double rel, double* scratch, int sm_count, cudaStream_t s) {
    const int64_t off_leaf = (((int64_t)1 << (2 * A->d)) - 1) / 3;
    const double* la = A->pyr + off_leaf;
    const double* lb = B->pyr + off_leaf;
    double* colmaxA = scratch;
    double* rowmaxB = scratch + A->nb;
    double* gmax = scratch + 2 * A->nb;          // largest leaf of A, of B
    const int blocks = (int)std::min<int64_t>((A->nl + 31) / 32 * 4, 8 * (int64_t)sm_count);
    cudaError_t e = cudaMemsetAsync(gmax, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    k_leaf_max<<<dim3((unsigned)std::max(blocks, 1), 2), 256, 0, s>>>(la, lb, A->nb, A->nl,
                                                                        colmaxA, rowmaxB, gmax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const Thresh th = make_thresh(tau, rel);
    const int pk = A->precision == SPAMM_PREC_TF32     ? 1
                   : A->precision == SPAMM_PREC_TF32X3 ? 2
                   : A->precision == SPAMM_PREC_BF16X3 ? 3
                                                       : 4;
    const int tl = 128 / A->b;
    const size_t smem = (size_t)A->b * (128 + 4) * sizeof(float);
    auto one = [&](const spamm_tree* t, const double* rmB, const double* cmA) -> cudaError_t {
        const bool roleA = rmB != nullptr, roleB = cmA != nullptr;
        void* pa0 = roleA ? t->packA[0] : nullptr;
        void* pb0 = roleB ? t->packB[0] : nullptr;
        void* pa1 = nullptr;
        void* pb1 = nullptr;
        if (t->sparse) {
            // banded layout: one array per part
            pa1 = roleA ? t->packA[1] : nullptr;
            pb1 = roleB ? t->packB[1] : nullptr;
        } else if (pk != 1) {
            // grouped layout: the lo parts of a group of CG chunks follow its
            // hi parts
            const size_t slice = (size_t)128 * 16 * (pk >= 3 ? 2 : 4);   // TL pieces
            const size_t cg = (size_t)pack_group_chunks(t->b, t->precision);
            pa1 = pa0 ? static_cast<unsigned char*>(pa0) + cg * slice : nullptr;
            pb1 = pb0 ? static_cast<unsigned char*>(pb0) + 2 * cg * slice : nullptr;
        }
        const double* leaf = t->pyr + off_leaf;
        dim3 grid((unsigned)t->nl, (unsigned)(t->nlp / tl));
#define SPAMM_LP2(PKV, LV, BV)                                                               \
    do {                                                                                     \
        if (smem > 48 * 1024)                                                                \
            cudaFuncSetAttribute(k_leaf_pack<PKV, LV, BV>,                                   \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);    \
        k_leaf_pack<PKV, LV, BV><<<grid, pack_threads<LV>(), smem, s>>>(t->A, t->n, t->lda, t->nb, t->nl,   \
                                                         t->nlp, leaf, rmB, cmA, th, pa0,    \
                                                         pa1, pb0, pb1, band_view(t), gmax,  \
                                                         gmax + 1, &ctl->packed_a);          \
    } while (0)
#define SPAMM_LP(PKV, LV)                                                                    \
    do {                                                                                     \
        if (t->sparse) SPAMM_LP2(PKV, LV, true);                                             \
        else SPAMM_LP2(PKV, LV, false);                                                      \
    } while (0)
#define SPAMM_LP_B(LV)                     \
    do {                                   \
        if (pk == 1) SPAMM_LP(1, LV);      \
        else if (pk == 2) SPAMM_LP(2, LV); \
        else if (pk == 3) SPAMM_LP(3, LV); \
        else SPAMM_LP(4, LV);              \
    } while (0)
        if (t->b == 16) SPAMM_LP_B(16);
        else if (t->b == 32) SPAMM_LP_B(32);
        else if (t->b == 64) SPAMM_LP_B(64);
        else SPAMM_LP_B(128);
#undef SPAMM_LP_B
#undef SPAMM_LP
#undef SPAMM_LP2
        return cudaGetLastError();
    };
    if (A == B) return one(A, rowmaxB, colmaxA);
    e = one(A, rowmaxB, nullptr);
    if (e != cudaSuccess) return e;
    return one(B, nullptr, colmaxA);
}

}  // namespace spamm
