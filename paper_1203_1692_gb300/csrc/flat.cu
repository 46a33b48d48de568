// The paper's flat enumeration of the leaf triples (Sec. III.D.2, Algorithm
// 1): the leaves of A and B are grouped by their k index ("k-value blocks"),
// each group is sorted by descending norm, and for every A leaf of a group
// the B leaves of the same k are walked in descending norm until the norm
// product falls below tau (the early exit).  On the GPU:
//
//   1. k_flat_sort: one block per K sorts column K of A's leaf tier and row
//      K of B's leaf tier by descending squared norm (bitonic sort in shared
//      memory, ties by ascending index so the order is deterministic);
//   2. k_flat_count: one thread per (K, A rank i) finds the length c(i) of
//      the kept prefix of B's sorted row by binary search: the SpAMM test is
//      monotone in each norm, so the kept B leaves of one A leaf are a
//      prefix of the descending order, and c(i) never grows with i (the
//      paper's early exit);
//   3. an exclusive scan of the c(i) gives each (K, i) its output range;
//   4. k_flat_emit writes the triples (I, K, J) of every prefix.
//
// The leaf test is the hierarchical cull's own (squared FP64 norms, NULL
// blocks never kept), and a parent's norm is never below its children's, so
// the flat set equals the set the tier-by-tier cull keeps; spamm_cull_flat
// returns it as an alternative cull and a cross-check of the hierarchy.
#include <algorithm>

#include "spamm_internal.cuh"

namespace spamm {

constexpr int kFlatMax = 2048;  // leaves per side the shared-memory sort holds

// Sort (key desc, index asc) pairs of n <= kFlatMax entries in shared memory.
__device__ void bitonic_desc(double* key, uint32_t* idx, int n_pow2) {
    for (int size = 2; size <= n_pow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < n_pow2 / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                // descending within blocks whose (lo & size) == 0
                const bool desc = (lo & size) == 0;
                const double ka = key[lo], kb = key[hi];
                const uint32_t ia = idx[lo], ib = idx[hi];
                // "a before b": larger key, or equal key and smaller index
                const bool a_first = ka > kb || (ka == kb && ia < ib);
                if (desc != a_first) {
                    key[lo] = kb;
                    key[hi] = ka;
                    idx[lo] = ib;
                    idx[hi] = ia;
                }
            }
            __syncthreads();
        }
    }
}

// Block K: sorted column K of A (norm, row I) and row K of B (norm, col J).
__global__ void __launch_bounds__(512) k_flat_sort(const double* __restrict__ leafA,
                                                   const double* __restrict__ leafB, int64_t nb,
                                                   int nl, int n_pow2, double* __restrict__ sa,
                                                   uint32_t* __restrict__ ia,
                                                   double* __restrict__ sb,
                                                   uint32_t* __restrict__ ib) {
    extern __shared__ unsigned char smem[];
    double* key = reinterpret_cast<double*>(smem);
    uint32_t* idx = reinterpret_cast<uint32_t*>(key + n_pow2);
    const int64_t K = blockIdx.x;
    for (int side = 0; side < 2; ++side) {
        for (int i = threadIdx.x; i < n_pow2; i += blockDim.x) {
            // padding entries sort last (key -1 is below every norm)
            key[i] = i < nl ? (side == 0 ? leafA[(int64_t)i * nb + K] : leafB[K * nb + i]) : -1.0;
            idx[i] = (uint32_t)i;
        }
        __syncthreads();
        bitonic_desc(key, idx, n_pow2);
        double* sk = side == 0 ? sa : sb;
        uint32_t* si = side == 0 ? ia : ib;
        for (int i = threadIdx.x; i < nl; i += blockDim.x) {
            sk[K * nl + i] = key[i];
            si[K * nl + i] = idx[i];
        }
        __syncthreads();
    }
}

// c(K, i): kept prefix length of B's sorted row K for A's i-th leaf of column K.
__global__ void __launch_bounds__(256) k_flat_count(const double* __restrict__ sa,
                                                    const double* __restrict__ sb, int nl,
                                                    Thresh th, uint32_t* __restrict__ cnt) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)nl * nl) return;
    const int64_t K = g / nl;
    const double a = sa[g];
    const double* row = sb + K * nl;
    int lo = 0, hi = nl;                 // first index that is not kept
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        bool tie;
        if (spamm_keep(a, row[mid], th, &tie)) lo = mid + 1;
        else hi = mid;
    }
    cnt[g] = (uint32_t)lo;
}

// Exclusive scan of cnt[0..m) into off[0..m] (off[m] = total), one block.
__global__ void __launch_bounds__(1024) k_flat_scan(const uint32_t* __restrict__ cnt, int64_t m,
                                                    unsigned long long* __restrict__ off) {
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < m; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const unsigned long long v = i < m ? cnt[i] : 0ull;
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned long long t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const unsigned long long pre = (wid ? warp_tot[wid - 1] : 0ull) + carry;
        if (i < m) off[i] = pre + x - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = pre + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[m] = carry;
}

// Triples of each prefix, packed as in the hierarchical cull, into out
// (capacity cap; nothing past cap is written).
__global__ void __launch_bounds__(256) k_flat_emit(const uint32_t* __restrict__ ia,
                                                   const uint32_t* __restrict__ ib,
                                                   const uint32_t* __restrict__ cnt,
                                                   const unsigned long long* __restrict__ off,
                                                   int nl, uint64_t* __restrict__ out,
                                                   unsigned long long cap) {
    const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= (int64_t)nl * nl) return;
    const int64_t K = g / nl;
    const uint32_t I = ia[g];
    const uint32_t c = cnt[g];
    const unsigned long long o = off[g];
    for (uint32_t j = lane; j < c; j += 32)
        if (o + j < cap) out[o + j] = pack_triple(I, (uint64_t)K, ib[K * nl + j]);
}

cudaError_t launch_cull_flat(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B,
                             double tau, uint64_t* out, unsigned long long cap,
                             void* scratch, unsigned long long* total_dev) {
    const int nl = (int)A->nl;
    int n_pow2 = 1;
    while (n_pow2 < nl) n_pow2 <<= 1;
    cudaStream_t s = ctx->stream;
    const int64_t m = (int64_t)nl * nl;
    // scratch: sa, sb (m doubles each), ia, ib, cnt (m u32 each), off (m + 1 u64)
    double* sa = static_cast<double*>(scratch);
    double* sb = sa + m;
    uint32_t* ia = reinterpret_cast<uint32_t*>(sb + m);
    uint32_t* ib = ia + m;
    uint32_t* cnt = ib + m;
    unsigned long long* off = reinterpret_cast<unsigned long long*>(cnt + m + (m & 1));
    const int64_t off_leaf = (((int64_t)1 << (2 * A->d)) - 1) / 3;
    const size_t smem = (size_t)n_pow2 * (sizeof(double) + sizeof(uint32_t));
    cudaError_t e = cudaFuncSetAttribute(k_flat_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_flat_sort<<<nl, 512, smem, s>>>(A->pyr + off_leaf, B->pyr + off_leaf, A->nb, nl, n_pow2, sa,
                                      ia, sb, ib);
    const Thresh th = make_thresh(tau, ctx->cfg.tie_rel);
    k_flat_count<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(sa, sb, nl, th, cnt);
    k_flat_scan<<<1, 1024, 0, s>>>(cnt, m, off);
    k_flat_emit<<<(unsigned)((m + 7) / 8), 256, 0, s>>>(ia, ib, cnt, off, nl, out, cap);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(total_dev, off + m, sizeof(unsigned long long),
                           cudaMemcpyDeviceToDevice, s);
}

size_t flat_scratch_bytes(int64_t nl) {
    const int64_t m = nl * nl;
    return (size_t)m * (2 * sizeof(double) + 3 * sizeof(uint32_t)) + sizeof(uint32_t) +
           (size_t)(m + 1) * sizeof(unsigned long long);
}

int flat_max_leaves() { return kFlatMax; }

}  // namespace spamm
