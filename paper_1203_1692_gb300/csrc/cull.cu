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
// Grouping.  A C tile is 128 rows x 256 columns: with TL = 128 / b = 2^s it is
// two horizontally adjacent quadtree nodes of tier tt = d - s (its two
// halves).  The tier-by-tier cull therefore stops at tier tt; its triples
// (I', K', J') are counted per tile (I', J' / 2), scanned and scattered as
// entries (K', half), and one block per tile finishes the cull of the last s
// tiers inside the 2^s x 2^s x 2^s sub-cubes of every K' in ascending order:
// a leaf triple survives iff every ancestor below the tile node does, with
// the same FP64 predicate.  The surviving leaf triples of one (tile, K) are
// emitted as one step (K, two 64-bit masks, bit y * 8 + x for row leaf x and
// column leaf y of each half), compacted into a coalesced list in ascending
// K.  This is the leaf-triple list in tile-compressed form; the leaf kernels
// walk it, which fixes the accumulation order of every C block.
#include <algorithm>

#include "spamm_internal.cuh"

namespace spamm {

__global__ void k_cull_root(const double* __restrict__ pa, const double* __restrict__ pb,
                            Thresh th, DevCtl* ctl, uint64_t* __restrict__ pool) {
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
    bool tie;
    const bool keep = spamm_keep(na, nb, th, &tie);
    if (tie) ctl->tie_band += 1;
    ctl->tier_count[0] = keep ? 1 : 0;
    if (keep) pool[0] = pack_triple(0, 0, 0);
}

// Expand tier t into tier t + 1.  na/nb are the tier-(t+1) norm grids.
__global__ void __launch_bounds__(256) k_cull_tier(int t, const double* __restrict__ na,
                                                   const double* __restrict__ nb, Thresh th,
                                                   DevCtl* ctl,
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
            bool tb;
            keep = spamm_keep(na[i * w + k], nb[k * w + j], th, &tb);
            tie += tb ? 1 : 0;
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

__global__ void k_cull_finish(int tt, DevCtl* ctl, unsigned long long cap) {
    if (threadIdx.x || blockIdx.x) return;
    for (int t = 0; t <= tt; ++t)
        if (ctl->tier_off[t] + ctl->tier_count[t] > cap) ctl->status |= ST_OVERFLOW;
}

cudaError_t launch_cull(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B, double tau,
                        int tt) {
    cudaStream_t s = ctx->stream;
    const Thresh th = make_thresh(tau, ctx->cfg.tie_rel);
    const unsigned long long cap = (unsigned long long)ctx->pool_words;
    k_cull_root<<<1, 32, 0, s>>>(A->pyr, B->pyr, th, ctx->ctl, ctx->pool);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int blocks = ctx->sm_count * 4;
    for (int t = 0; t < tt; ++t) {
        const int64_t off = (((int64_t)1 << (2 * (t + 1))) - 1) / 3;
        // Tier t + 1 has at most 8^(t+1) candidates: size small tiers' grids to them.
        int g = blocks;
        if (t + 1 < 7) {
            const int64_t cand = (int64_t)1 << (3 * (t + 1));
            g = (int)std::min<int64_t>(blocks, (cand + 255) / 256);
        }
        k_cull_tier<<<g, 256, 0, s>>>(t, A->pyr + off, B->pyr + off, th, ctx->ctl, ctx->pool,
                                      cap);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_cull_finish<<<1, 32, 0, s>>>(tt, ctx->ctl, cap);
    return cudaGetLastError();
}

// ------------------------------------------------------------- grouping

__device__ inline uint32_t tile_of(uint64_t tri, int tc) {
    return tri_I(tri) * (uint32_t)tc + (tri_J(tri) >> 1);
}

__global__ void __launch_bounds__(256) k_group_count(int tt, DevCtl* ctl,
                                                     const uint64_t* __restrict__ pool, int tc,
                                                     uint32_t* __restrict__ tile_cnt) {
    if (ctl->status & (ST_OVERFLOW | ST_NONFINITE)) return;
    const unsigned long long off = ctl->tier_off[tt];
    const unsigned long long m = ctl->tier_count[tt];
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < m;
         g += (unsigned long long)gridDim.x * blockDim.x)
        atomicAdd(&tile_cnt[tile_of(pool[off + g], tc)], 1u);
}

// Exclusive scan of the tile counts (single block), and the pool layout of
// the grouped arrays behind the tier-tt frontier: entries (u32, one per
// tier-tt triple), then step K (u32) and step masks (2 x u64), S per entry.
__global__ void __launch_bounds__(1024) k_group_scan(int tt, int S, DevCtl* ctl,
                                                     unsigned long long cap,
                                                     const uint32_t* __restrict__ cnt,
                                                     uint32_t* __restrict__ off, int tiles) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < tiles; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < tiles ? cnt[i] : 0u;
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
        const unsigned long long m = ctl->tier_count[tt];
        const unsigned long long end = ctl->tier_off[tt] + m;
        const unsigned long long ms = m * (unsigned long long)S;
        ctl->ent_off = end;
        ctl->pk_off = end + (m + 1) / 2;
        ctl->pm_off = ctl->pk_off + (ms + 1) / 2;
        ctl->need_words = ctl->pm_off + 2 * ms;
        if (ctl->need_words > cap || m >= 0xffffffffull / (unsigned long long)S)
            ctl->status |= ST_OVERFLOW;
    }
}

__global__ void __launch_bounds__(256) k_group_scatter(int tt, DevCtl* ctl,
                                                       uint64_t* __restrict__ pool, int tc,
                                                       const uint32_t* __restrict__ off,
                                                       uint32_t* __restrict__ fill) {
    if (ctl->status & (ST_OVERFLOW | ST_NONFINITE)) return;
    const unsigned long long loff = ctl->tier_off[tt];
    const unsigned long long m = ctl->tier_count[tt];
    uint32_t* ent = reinterpret_cast<uint32_t*>(pool + ctl->ent_off);
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < m;
         g += (unsigned long long)gridDim.x * blockDim.x) {
        const uint64_t tri = pool[loff + g];
        const uint32_t u = tile_of(tri, tc);
        ent[off[u] + atomicAdd(&fill[u], 1u)] = (tri_K(tri) << 1) | (tri_J(tri) & 1u);
    }
}

// Block-wide exclusive scan of one value per thread (blockDim <= 512).
__device__ inline uint32_t block_excl_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t t = lane < nw ? warp_sums[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_sums[lane] = t;
        if (lane == nw - 1) *total = t;
    }
    __syncthreads();
    const uint32_t r = (wid ? warp_sums[wid - 1] : 0u) + x - v;
    __syncthreads();
    return r;
}

// Finish the cull of one tile's sub-cubes (DS = d - tt tiers below the tile
// nodes) and emit its (K, masks) steps in ascending K.  kCullWarps warps per
// block, several blocks per SM so that one tile's barriers overlap another
// tile's work.
//
// One warp evaluates one (K', kk) slice: the S x S leaf pairs (x, y) of
// leaf column K = K' * S + kk in each half whose node has the entry
// (K', half).  A lane tests its leaf triples and all their ancestors below
// the tile node with the FP64 predicate (a leaf survives iff every ancestor
// does, which is the level-by-level cull), and the warp ORs the survivors
// into the two 64-bit masks of that K.  Slices are independent, so no
// block-wide synchronisation is needed between tiers; the masks of a window
// of K values are then compacted in ascending K.
constexpr int kCullWarps = 8;

template <int DS>
__global__ void __launch_bounds__(kCullWarps * 32, 3) k_tile_cull(int tt, const double* __restrict__ pyrA,
                                                   const double* __restrict__ pyrB, Thresh th,
                                                   DevCtl* ctl, uint64_t* __restrict__ pool,
                                                   const uint32_t* __restrict__ off,
                                                   uint32_t* __restrict__ steps, int tc) {
    constexpr int S = 1 << DS;               // K leaves per tier-tt K'
    constexpr int WIN = 1024;                // steps per window (16 KB of masks)
    constexpr int KPW = WIN / S;             // K' per window
    extern __shared__ uint32_t dyn[];        // K' bitmaps of both halves, then the K' list
    __shared__ unsigned long long masks[WIN][2];
    // per-warp staged norms of one sub-cube: levels 1..DS, A side [x][k], B side [k][y]
    __shared__ double nA[kCullWarps][84], nB[kCullWarps][84];
    __shared__ uint32_t warp_sums[16], total_s;
    __shared__ unsigned long long st_cand[4], st_kept[4], st_tie;
    if (ctl->status & (ST_OVERFLOW | ST_NONFINITE)) return;
    const uint32_t u = blockIdx.x;
    const uint32_t e0 = off[u], e1 = off[u + 1];
    if (e0 == e1) {
        if (threadIdx.x == 0) steps[u] = 0;
        return;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t I0 = u / tc, Jp = u % tc;
    const uint32_t* ent = reinterpret_cast<const uint32_t*>(pool + ctl->ent_off);
    uint32_t* pk = reinterpret_cast<uint32_t*>(pool + ctl->pk_off);
    unsigned long long* pm = reinterpret_cast<unsigned long long*>(pool + ctl->pm_off);
    const int words = ((1 << tt) + 31) >> 5;
    uint32_t* bm0 = dyn;
    uint32_t* bm1 = dyn + words;
    uint32_t* klist = dyn + 2 * words;
    for (int w = tid; w < 2 * words; w += blockDim.x) dyn[w] = 0u;
    if (tid < 4) st_cand[tid] = st_kept[tid] = 0ull;
    if (tid == 0) st_tie = 0ull;
    __syncthreads();
    for (uint32_t e = e0 + tid; e < e1; e += blockDim.x) {
        const uint32_t v = ent[e], k = v >> 1;
        atomicOr(&((v & 1u) ? bm1 : bm0)[k >> 5], 1u << (k & 31));
    }
    __syncthreads();
    // ascending list of the K' present in either half
    int nk = 0;
    for (int w0 = 0, base = 0; w0 < words; w0 += blockDim.x) {
        const int w = w0 + tid;
        const uint32_t bits = w < words ? (bm0[w] | bm1[w]) : 0u;
        const uint32_t r = block_excl_scan(__popc(bits), warp_sums, &total_s);
        uint32_t b = bits, pos = base + r;
        while (b) {
            const int q = __ffs(b) - 1;
            b &= b - 1;
            klist[pos++] = (uint32_t)(w * 32 + q);
        }
        base += total_s;
        nk = base;
        __syncthreads();
    }
    const uint32_t obase = e0 * S;
    uint32_t written = 0;
    unsigned long long cand[4] = {0, 0, 0, 0}, kept[4] = {0, 0, 0, 0}, tie = 0;
    for (int kw = 0; kw < nk; kw += KPW) {
        const int kn = min(KPW, nk - kw);
        // phase 1: one warp per (K', half) sub-cube; each tier below the
        // tile node is evaluated once, 8^l triples spread over the lanes,
        // and shared through ballots (bit index (k * side + y) * side + x).
        for (int item = warp; item < 2 * kn; item += kCullWarps) {
            const int g = item >> 1, half = item & 1;
            const uint32_t Kp = klist[kw + g];
            const bool has = half ? ((bm1[Kp >> 5] >> (Kp & 31)) & 1u) != 0
                                  : ((bm0[Kp >> 5] >> (Kp & 31)) & 1u) != 0;
            const uint32_t J0 = Jp * 2 + half;
            unsigned long long prev = has ? 1ull : 0ull;  // tier-tt node kept
            unsigned long long lv2[2] = {0ull, 0ull};    // level-2 bits (64)
#pragma unroll
            for (int l = 1; l <= DS; ++l) {
                const int side = 1 << l;
                const int per = side * side * side;
                const int so = l == 1 ? 0 : l == 2 ? 4 : 20;
                // stage this level's norms ([x][k] for A, [k][y] for B) only if
                // the level above kept something
                const bool any = l == 1 ? prev != 0ull : l == 2 ? prev != 0ull : lv2[0] != 0ull;
                if (any) {
                    const int t = tt + l;
                    const int64_t w = (int64_t)1 << t;
                    const int64_t off_t = (((int64_t)1 << (2 * t)) - 1) / 3;
                    for (int e = lane; e < side * side; e += 32) {
                        const int rr = e / side, cc = e % side;
                        nA[warp][so + e] =
                            pyrA[off_t + (((int64_t)I0 << l) + rr) * w + ((int64_t)Kp << l) + cc];
                        nB[warp][so + e] =
                            pyrB[off_t + (((int64_t)Kp << l) + rr) * w + ((int64_t)J0 << l) + cc];
                    }
                }
                __syncwarp();
#pragma unroll
                for (int r = 0; r < (per + 31) / 32; ++r) {
                    const int idx = lane + 32 * r;
                    const int xi = idx & (side - 1), yi = (idx >> l) & (side - 1),
                              ki = idx >> (2 * l);
                    // parent bit at level l - 1
                    const int ps = side >> 1;
                    const int pidx = ((ki >> 1) * ps + (yi >> 1)) * ps + (xi >> 1);
                    bool par;
                    if (l == 1) par = prev != 0ull;
                    else if (l == 2) par = (prev >> pidx) & 1ull;
                    else par = (lv2[pidx >> 5 >> 1] >> (pidx & 63)) & 1ull;
                    bool ok = false;
                    if (idx < per && par) {
                        bool tb;
                        ok = spamm_keep(nA[warp][so + xi * side + ki], nB[warp][so + ki * side + yi],
                                        th, &tb);
                        cand[l - 1] += 1;
                        kept[l - 1] += ok ? 1 : 0;
                        tie += tb ? 1 : 0;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, ok);
                    if (l == DS) {
                        // leaf level: the mask of leaf column K' * S + ki
                        if (DS == 3) {
                            const int kk = r >> 1;           // uniform across the warp
                            if (lane == 0) {
                                if ((r & 1) == 0) masks[g * S + kk][half] = bal;
                                else masks[g * S + kk][half] |= (unsigned long long)bal << 32;
                            }
                        } else {
                            // remap bit (ki, yi, xi) -> mask of ki, bit yi * 8 + xi
                            const unsigned long long bit = ok ? 1ull << (yi * 8 + xi) : 0ull;
#pragma unroll
                            for (int kq = 0; kq < S; ++kq) {
                                const unsigned long long mine = (idx < per && ki == kq) ? bit : 0ull;
                                const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)mine);
                                const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(mine >> 32));
                                if (r == 0 && lane == 0) masks[g * S + kq][half] = 0ull;
                                if (lane == 0) masks[g * S + kq][half] |= ((unsigned long long)hi << 32) | lo;
                            }
                        }
                    } else if (l == 1) {
                        prev = bal & 0xFFu;
                    } else if (l == 2) {
                        if (r == 0) lv2[0] = bal;
                        else lv2[0] |= (unsigned long long)bal << 32;
                    }
                }
                if (l == 2) prev = lv2[0];
                if (l == 2) lv2[1] = 0ull;
            }
            if (DS == 0) {
                if (lane == 0) masks[g][half] = has ? 1ull : 0ull;
            }
            __syncwarp();  // staged norms are reused by the next sub-cube
        }
        __syncthreads();
        // phase 2: ordered compaction of the window's masks (ascending K)
        for (int c0 = 0; c0 < kn * S; c0 += blockDim.x) {
            const int i = c0 + tid;
            const unsigned long long m0 = i < kn * S ? masks[i][0] : 0ull;
            const unsigned long long m1 = i < kn * S ? masks[i][1] : 0ull;
            const bool any = (m0 | m1) != 0ull;
            const uint32_t r = block_excl_scan(any ? 1u : 0u, warp_sums, &total_s);
            if (any) {
                const int g = i / S, kk = i % S;
                const uint32_t pos = obase + written + r;
                pk[pos] = klist[kw + g] * S + kk;
                pm[2 * (size_t)pos] = m0;
                pm[2 * (size_t)pos + 1] = m1;
            }
            written += total_s;
        }
        __syncthreads();
    }
    // statistics of the tiers below the tile nodes
#pragma unroll
    for (int l = 0; l < DS; ++l) {
        for (int o = 16; o > 0; o >>= 1) {
            cand[l] += __shfl_xor_sync(0xffffffffu, cand[l], o);
            kept[l] += __shfl_xor_sync(0xffffffffu, kept[l], o);
        }
        if (lane == 0 && cand[l]) atomicAdd(&st_cand[l], cand[l]);
        if (lane == 0 && kept[l]) atomicAdd(&st_kept[l], kept[l]);
    }
    for (int o = 16; o > 0; o >>= 1) tie += __shfl_xor_sync(0xffffffffu, tie, o);
    if (lane == 0 && tie) atomicAdd(&st_tie, tie);
    __syncthreads();
    if (tid == 0) {
        steps[u] = written;
        atomicAdd(&ctl->active_steps, (unsigned long long)written);
        for (int l = 0; l < DS; ++l) {
            atomicAdd(&ctl->tier_cand[tt + 1 + l], st_cand[l]);
            atomicAdd(&ctl->tier_count[tt + 1 + l], st_kept[l]);
        }
        if (st_tie) atomicAdd(&ctl->tie_band, st_tie);
    }
}

cudaError_t launch_group(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B, double tau,
                         int tt) {
    cudaStream_t s = ctx->stream;
    const int tc = tile_cols(A);
    const int tiles = tile_rows(A) * tc;
    const int ds = A->d - tt;
    const int S = 1 << ds;
    const unsigned long long cap = (unsigned long long)ctx->pool_words;
    const Thresh th = make_thresh(tau, ctx->cfg.tie_rel);
    cudaError_t e = cudaMemsetAsync(ctx->tile_cnt, 0, sizeof(uint32_t) * tiles, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->tile_fill, 0, sizeof(uint32_t) * tiles, s);
    if (e != cudaSuccess) return e;
    const int blocks = ctx->sm_count * 4;
    k_group_count<<<blocks, 256, 0, s>>>(tt, ctx->ctl, ctx->pool, tc, ctx->tile_cnt);
    k_group_scan<<<1, 1024, 0, s>>>(tt, S, ctx->ctl, cap, ctx->tile_cnt, ctx->tile_off, tiles);
    k_group_scatter<<<blocks, 256, 0, s>>>(tt, ctx->ctl, ctx->pool, tc, ctx->tile_off,
                                           ctx->tile_fill);
    const int words = ((1 << tt) + 31) / 32;
    const size_t dsm = sizeof(uint32_t) * (2 * words + ((size_t)1 << tt));
#define SPAMM_TC(DSV)                                                                          \
    do {                                                                                       \
        cudaFuncSetAttribute(k_tile_cull<DSV>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                             (int)dsm);                                                        \
        cudaFuncSetAttribute(k_tile_cull<DSV>, cudaFuncAttributePreferredSharedMemoryCarveout,  \
                             100);                                                             \
        k_tile_cull<DSV><<<tiles, kCullWarps * 32, dsm, s>>>(tt, A->pyr, B->pyr, th, ctx->ctl,             \
                                                 ctx->pool, ctx->tile_off, ctx->tile_steps,    \
                                                 tc);                                          \
    } while (0)
    switch (ds) {
        case 0: SPAMM_TC(0); break;
        case 1: SPAMM_TC(1); break;
        case 2: SPAMM_TC(2); break;
        default: SPAMM_TC(3); break;
    }
#undef SPAMM_TC
    return cudaGetLastError();
}

}  // namespace spamm
