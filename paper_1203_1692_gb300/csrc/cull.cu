// Stages 2 and 3: the level-by-level SpAMM cull (Eqs. (product) and
// (norm_condition)) and the grouping of the surviving leaf triples by C tile.
//
// Cull.  The frontier of tier t is a list of packed (I, K, J) triples whose
// block product survived at every tier down to t.  One launch per tier
// expands each parent into its 8 children (2I+di, 2K+dk, 2J+dj) and keeps a
// child iff nA2 * nB2 >= tau^2 with both norms non-zero (FP64).  Eight lanes
// of a warp look at the eight children of one parent; the keep bits are
// compacted with a warp ballot and a population count, one atomicAdd per warp
// reserves space, and the kept children are written as one contiguous run,
// so the frontier goes to HBM coalesced.  Frontiers are carved one after
// another out of a single pool; sizes live in device memory, so there is no
// host round trip between tiers.  A frontier that does not fit is truncated
// and the overflow flag is raised.
//
// Grouping.  A C tile is 128 x 128 (TL = 128 / b leaves per side).  Each leaf
// triple is counted per tile, the counts are scanned, the triples are
// scattered into per-tile runs, and one block per tile ORs them into a
// per-K 64-bit mask (bit y * 8 + x) in shared memory and emits the non-zero
// (K, mask) steps in ascending K.  The leaf kernels walk these steps, which
// fixes the accumulation order of every C block.
#include <algorithm>

#include "spamm_internal.cuh"

namespace spamm {

__global__ void k_cull_root(const double* __restrict__ pa, const double* __restrict__ pb,
                            double tau2, double lo2, double hi2, DevCtl* ctl,
                            uint64_t* __restrict__ pool) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double na = pa[0], nb = pb[0];
    ctl->tier_off[0] = 0;
    ctl->tier_cand[0] = 1;
    if (!isfinite(na) || !isfinite(nb)) {
        // Inf/NaN anywhere makes the root sum non-finite.
        ctl->status |= ST_NONFINITE;
        ctl->tier_count[0] = 0;
        return;
    }
    const double p = na * nb;
    const bool keep = na > 0.0 && nb > 0.0 && p >= tau2;
    if (na > 0.0 && nb > 0.0 && p >= lo2 && p <= hi2) ctl->tie_band += 1;
    ctl->tier_count[0] = keep ? 1 : 0;
    if (keep) pool[0] = pack_triple(0, 0, 0);
}

// Expand tier t into tier t + 1.  na/nb are the tier-(t+1) norm grids.
__global__ void __launch_bounds__(256) k_cull_tier(int t, const double* __restrict__ na,
                                                   const double* __restrict__ nb, double tau2,
                                                   double lo2, double hi2, DevCtl* ctl,
                                                   uint64_t* __restrict__ pool,
                                                   unsigned long long cap) {
    const unsigned long long in_off = ctl->tier_off[t];
    const unsigned long long in_cnt = stored_count(ctl, t, cap);
    const unsigned long long out_off = in_off + in_cnt;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->tier_off[t + 1] = out_off;
        ctl->tier_cand[t + 1] = in_cnt * 8;
    }
    const int64_t w = (int64_t)1 << (t + 1);
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long total = in_cnt * 8;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    unsigned long long tie = 0;
    for (unsigned long long base = ((unsigned long long)blockIdx.x * (blockDim.x >> 5) +
                                    (threadIdx.x >> 5)) * 32;
         base < total; base += warps * 32) {
        const unsigned long long g = base + lane;
        bool keep = false;
        uint64_t child = 0;
        if (g < total) {
            const uint64_t par = pool[in_off + (g >> 3)];
            const unsigned q = (unsigned)(g & 7);
            const uint64_t i = 2ull * tri_I(par) + ((q >> 2) & 1);
            const uint64_t k = 2ull * tri_K(par) + ((q >> 1) & 1);
            const uint64_t j = 2ull * tri_J(par) + (q & 1);
            const double a = na[i * w + k];
            const double b = nb[k * w + j];
            const double p = a * b;
            const bool nz = a > 0.0 && b > 0.0;
            keep = nz && p >= tau2;
            tie += (nz && p >= lo2 && p <= hi2) ? 1 : 0;
            child = pack_triple(i, k, j);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (bal == 0) continue;
        unsigned long long start = 0;
        if (lane == 0) start = atomicAdd(&ctl->tier_count[t + 1], (unsigned long long)__popc(bal));
        start = __shfl_sync(0xffffffffu, start, 0);
        if (keep) {
            const unsigned long long pos =
                out_off + start + __popc(bal & ((1u << lane) - 1u));
            if (pos < cap) pool[pos] = child;
        }
    }
    // tie-band count and overflow flag
    for (int off = 16; off > 0; off >>= 1) tie += __shfl_xor_sync(0xffffffffu, tie, off);
    if (lane == 0 && tie) atomicAdd(&ctl->tie_band, tie);
}

__global__ void k_cull_finish(int d, DevCtl* ctl, unsigned long long cap) {
    if (threadIdx.x || blockIdx.x) return;
    for (int t = 0; t <= d; ++t)
        if (ctl->tier_off[t] + ctl->tier_count[t] > cap) ctl->status |= ST_OVERFLOW;
}

cudaError_t launch_cull(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B, double tau) {
    cudaStream_t s = ctx->stream;
    const double tau2 = tau * tau;
    const double rel = ctx->cfg.tie_rel;
    const double lo2 = tau2 * (1.0 - rel) * (1.0 - rel);
    const double hi2 = tau2 * (1.0 + rel) * (1.0 + rel);
    const unsigned long long cap = (unsigned long long)ctx->pool_words;
    k_cull_root<<<1, 32, 0, s>>>(A->pyr, B->pyr, tau2, lo2, hi2, ctx->ctl, ctx->pool);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int blocks = ctx->sm_count * 4;
    for (int t = 0; t < A->d; ++t) {
        const int64_t off = (((int64_t)1 << (2 * (t + 1))) - 1) / 3;
        // Tier t + 1 has at most 8^(t+1) candidates: size small tiers' grids to them.
        int g = blocks;
        if (t + 1 < 7) {
            const int64_t cand = (int64_t)1 << (3 * (t + 1));
            g = (int)std::min<int64_t>(blocks, (cand + 255) / 256);
        }
        k_cull_tier<<<g, 256, 0, s>>>(t, A->pyr + off, B->pyr + off, tau2, lo2, hi2, ctx->ctl,
                                      ctx->pool, cap);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_cull_finish<<<1, 32, 0, s>>>(A->d, ctx->ctl, cap);
    return cudaGetLastError();
}

// ------------------------------------------------------------- grouping

__device__ inline uint32_t tile_of(uint64_t tri, int tl_shift, int tps) {
    return (tri_I(tri) >> tl_shift) * (uint32_t)tps + (tri_J(tri) >> tl_shift);
}

__global__ void __launch_bounds__(256) k_group_count(int d, DevCtl* ctl,
                                                     const uint64_t* __restrict__ pool,
                                                     unsigned long long cap, int tl_shift, int tps,
                                                     uint32_t* __restrict__ tile_cnt) {
    if (ctl->status & (ST_OVERFLOW | ST_NONFINITE)) return;
    const unsigned long long off = ctl->tier_off[d];
    const unsigned long long m = ctl->tier_count[d];
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < m;
         g += (unsigned long long)gridDim.x * blockDim.x)
        atomicAdd(&tile_cnt[tile_of(pool[off + g], tl_shift, tps)], 1u);
}

// Exclusive scan of the tile counts (single block), and the pool layout of
// the grouped arrays behind the leaf frontier.
__global__ void __launch_bounds__(1024) k_group_scan(int d, DevCtl* ctl, unsigned long long cap,
                                                     const uint32_t* __restrict__ cnt,
                                                     uint32_t* __restrict__ off, int tiles) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < tiles; base += 1024) {
        const int i = base + threadIdx.x;
        uint32_t v = i < tiles ? cnt[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            uint32_t t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const uint32_t pre = (wid ? warp_tot[wid - 1] : 0u) + carry;
        if (i < tiles) off[i] = pre + x - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = pre + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[tiles] = carry;
        const unsigned long long m = ctl->tier_count[d];
        const unsigned long long leaf_end = ctl->tier_off[d] + m;
        const unsigned long long half = (m + 1) / 2;  // u32 arrays in 8-byte words
        ctl->ent_off = leaf_end;
        ctl->pk_off = leaf_end + half;
        ctl->pm_off = leaf_end + 2 * half;
        ctl->need_words = leaf_end + 2 * half + m;
        if (ctl->need_words > cap) ctl->status |= ST_OVERFLOW;
    }
}

__global__ void __launch_bounds__(256) k_group_scatter(int d, DevCtl* ctl,
                                                       uint64_t* __restrict__ pool, int tl_shift,
                                                       int tps, const uint32_t* __restrict__ off,
                                                       uint32_t* __restrict__ fill) {
    if (ctl->status & (ST_OVERFLOW | ST_NONFINITE)) return;
    const unsigned long long loff = ctl->tier_off[d];
    const unsigned long long m = ctl->tier_count[d];
    uint32_t* ent = reinterpret_cast<uint32_t*>(pool + ctl->ent_off);
    const uint32_t tmask = (1u << tl_shift) - 1u;
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < m;
         g += (unsigned long long)gridDim.x * blockDim.x) {
        const uint64_t tri = pool[loff + g];
        const uint32_t u = tile_of(tri, tl_shift, tps);
        const uint32_t pos = off[u] + atomicAdd(&fill[u], 1u);
        const uint32_t x = tri_I(tri) & tmask, y = tri_J(tri) & tmask;
        ent[pos] = (tri_K(tri) << 6) | (y << 3) | x;
    }
}

// One block per tile: per-K masks in shared memory over the K range the
// tile touches, then the non-zero steps in ascending K.
__global__ void __launch_bounds__(512) k_group_steps(DevCtl* ctl, const uint64_t* __restrict__ pool,
                                                     const uint32_t* __restrict__ off,
                                                     uint32_t* __restrict__ steps, int nkmax) {
    extern __shared__ unsigned long long smask[];
    __shared__ uint32_t kmin_s, kmax_s, warp_cnt[16], base_s;
    if (ctl->status & (ST_OVERFLOW | ST_NONFINITE)) return;
    const uint32_t u = blockIdx.x;
    const uint32_t e0 = off[u], e1 = off[u + 1];
    const uint32_t* ent = reinterpret_cast<const uint32_t*>(pool + ctl->ent_off);
    uint32_t* pk = reinterpret_cast<uint32_t*>(const_cast<uint64_t*>(pool) + ctl->pk_off);
    unsigned long long* pm =
        reinterpret_cast<unsigned long long*>(const_cast<uint64_t*>(pool) + ctl->pm_off);
    if (e0 == e1) {
        if (threadIdx.x == 0) steps[u] = 0;
        return;
    }
    if (threadIdx.x == 0) {
        kmin_s = 0xffffffffu;
        kmax_s = 0;
    }
    __syncthreads();
    uint32_t lo = 0xffffffffu, hi = 0;
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const uint32_t K = ent[e] >> 6;
        lo = min(lo, K);
        hi = max(hi, K);
    }
    atomicMin(&kmin_s, lo);
    atomicMax(&kmax_s, hi);
    __syncthreads();
    const uint32_t k0 = kmin_s;
    const int span = (int)(kmax_s - k0 + 1);
    // process the K range in windows of nkmax entries
    uint32_t written = 0;
    for (int w0 = 0; w0 < span; w0 += nkmax) {
        const int wn = min(nkmax, span - w0);
        for (int i = threadIdx.x; i < wn; i += blockDim.x) smask[i] = 0ull;
        __syncthreads();
        for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const uint32_t v = ent[e];
            const int kk = (int)((v >> 6) - k0) - w0;
            if (kk >= 0 && kk < wn) atomicOr(&smask[kk], 1ull << (v & 63));
        }
        __syncthreads();
        // ordered compaction of the non-zero masks
        for (int c0 = 0; c0 < wn; c0 += blockDim.x) {
            const int i = c0 + threadIdx.x;
            const unsigned long long m = i < wn ? smask[i] : 0ull;
            const unsigned bal = __ballot_sync(0xffffffffu, m != 0ull);
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            if (lane == 0) warp_cnt[wid] = __popc(bal);
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t acc = written;
                for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                    const uint32_t c = warp_cnt[q];
                    warp_cnt[q] = acc;
                    acc += c;
                }
                base_s = acc;
            }
            __syncthreads();
            if (m) {
                const uint32_t pos = e0 + warp_cnt[wid] + __popc(bal & ((1u << lane) - 1u));
                pk[pos] = k0 + (uint32_t)(w0 + i);
                pm[pos] = m;
            }
            __syncthreads();
            written = base_s;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        steps[u] = written;
        atomicAdd(&ctl->active_steps, (unsigned long long)written);
    }
}

cudaError_t launch_group(spamm_ctx* ctx, const spamm_tree* A) {
    cudaStream_t s = ctx->stream;
    const int tps = tiles_per_side(A);
    const int tiles = tps * tps;
    const int tl = kTileRows / A->b;
    int tl_shift = 0;
    while ((1 << tl_shift) < tl) ++tl_shift;
    const unsigned long long cap = (unsigned long long)ctx->pool_words;
    cudaError_t e = cudaMemsetAsync(ctx->tile_cnt, 0, sizeof(uint32_t) * tiles, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->tile_fill, 0, sizeof(uint32_t) * tiles, s);
    if (e != cudaSuccess) return e;
    const int blocks = ctx->sm_count * 4;
    k_group_count<<<blocks, 256, 0, s>>>(A->d, ctx->ctl, ctx->pool, cap, tl_shift, tps,
                                         ctx->tile_cnt);
    k_group_scan<<<1, 1024, 0, s>>>(A->d, ctx->ctl, cap, ctx->tile_cnt, ctx->tile_off, tiles);
    k_group_scatter<<<blocks, 256, 0, s>>>(A->d, ctx->ctl, ctx->pool, tl_shift, tps,
                                           ctx->tile_off, ctx->tile_fill);
    const int nkmax = 4096;  // 32 KB of masks per window
    k_group_steps<<<tiles, 512, nkmax * sizeof(unsigned long long), s>>>(
        ctx->ctl, ctx->pool, ctx->tile_off, ctx->tile_steps, nkmax);
    return cudaGetLastError();
}

}  // namespace spamm
