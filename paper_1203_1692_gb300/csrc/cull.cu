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
//
// Batches.  Every kernel takes a table of products (one for spamm_multiply,
// up to 64 for spamm_multiply_batched) and a flattened grid: product p owns
// the blocks [bbase[p], bbase[p+1]) and works through them as its own grid.
// A batch therefore runs each tier, each grouping step and the tile cull of
// all its products in one launch each, with the blocks of a product sized
// to its share of the work.
#include <algorithm>
#include <cmath>
#include <vector>

#include "spamm_internal.cuh"

namespace spamm {

// One product of a symbolic launch.
struct CullProd {
    const double* pyrA;
    const double* pyrB;
    Thresh th;
    DevCtl* ctl;
    uint64_t* pool;
    unsigned long long cap;    // pool words
    uint32_t* tile_cnt;
    uint32_t* tile_fill;
    uint32_t* tile_off;
    uint32_t* tile_steps;
    uint32_t* tile_iters;      // K-chunk iterations per tile (may be null)
    const double* panA;        // panel norms of the sub-leaf cull (SL > 1)
    const double* panB;
    int tt, tc, tiles, S;
    int SL;                    // mask pairs per step: 1, or the 16-wide slices of a leaf
    int chunks;                // 16-wide K-chunks per leaf (b / 16)
    int nl;                    // leaves per side holding data
    int tier;                  // precision chosen by norm: also emit the full-split masks
    Thresh thh;                // its threshold tau_h
    int64_t n;                 // matrix order (the clipped extent of the ragged leaves)
    int b;                     // leaf size
};

constexpr int kCullBatch = 64;

// Passed by value (the table travels with the launch, also into a graph).
template <int NB>
struct CullBatch {
    CullProd p[NB];
    int bbase[NB + 1];  // first block of each product in the flattened grid
    int count;
};

template <int NB>
__device__ __forceinline__ int product_of_block(const CullBatch<NB>& cb, int b) {
    int lo = 0, hi = cb.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cb.bbase[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// This block's product q, its block index vb and block count vg within it.
#define CULL_RESOLVE(cb)                                       \
    const int pi_ = product_of_block(cb, (int)blockIdx.x);     \
    const CullProd& q = cb.p[pi_];                             \
    const int vb = (int)blockIdx.x - cb.bbase[pi_];            \
    const int vg = cb.bbase[pi_ + 1] - cb.bbase[pi_]

template <int NB>
__global__ void k_cull_root(CullBatch<NB> cb) {
    CULL_RESOLVE(cb);
    (void)vb;
    (void)vg;
    if (threadIdx.x != 0) return;
    DevCtl* ctl = q.ctl;
    const double na = q.pyrA[0], nb = q.pyrB[0];
    ctl->tier_off[0] = 0;
    ctl->tier_cand[0] = 1;
    if (!isfinite(na) || !isfinite(nb)) {
        // Inf/NaN anywhere makes the root sum non-finite.
        ctl->status |= ST_NONFINITE;
        ctl->tier_count[0] = 0;
        return;
    }
    bool tie;
    const bool keep = spamm_keep(na, nb, q.th, &tie);
    if (tie) ctl->tie_band += 1;
    ctl->tier_count[0] = keep ? 1 : 0;
    if (keep) q.pool[0] = pack_triple(0, 0, 0);
}

// Expand tier t into tier t + 1 (the tier-(t+1) norm grids of both trees).
template <int NB>
__global__ void __launch_bounds__(256) k_cull_tier(int t, CullBatch<NB> cb) {
    CULL_RESOLVE(cb);
    DevCtl* ctl = q.ctl;
    uint64_t* __restrict__ pool = q.pool;
    const unsigned long long cap = q.cap;
    const int64_t off_t = (((int64_t)1 << (2 * (t + 1))) - 1) / 3;
    const double* __restrict__ na = q.pyrA + off_t;
    const double* __restrict__ nb = q.pyrB + off_t;
    const Thresh th = q.th;
    const unsigned long long in_off = ctl->tier_off[t];
    const unsigned long long in_cnt = stored_count(ctl, t, cap);
    const unsigned long long out_off = in_off + in_cnt;
    if (vb == 0 && threadIdx.x == 0) {
        ctl->tier_off[t + 1] = out_off;
        ctl->tier_cand[t + 1] = in_cnt * 8;
    }
    const int64_t w = (int64_t)1 << (t + 1);
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long total = in_cnt * 8;
    const unsigned long long warps = (unsigned long long)vg * (blockDim.x >> 5);
    unsigned long long tie = 0;
    for (unsigned long long base = ((unsigned long long)vb * (blockDim.x >> 5) +
                                    (threadIdx.x >> 5)) * 32;
         base < total; base += warps * 32) {
        const unsigned long long g = base + lane;
        bool keep = false;
        uint64_t child = 0;
        if (g < total) {
            const uint64_t par = pool[in_off + (g >> 3)];
            const unsigned qd = (unsigned)(g & 7);
            const uint64_t i = 2ull * tri_I(par) + ((qd >> 2) & 1);
            const uint64_t k = 2ull * tri_K(par) + ((qd >> 1) & 1);
            const uint64_t j = 2ull * tri_J(par) + (qd & 1);
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
    // tie-band count
    for (int o = 16; o > 0; o >>= 1) tie += __shfl_xor_sync(0xffffffffu, tie, o);
    if (lane == 0 && tie) atomicAdd(&ctl->tie_band, tie);
}

template <int NB>
__global__ void k_cull_finish(CullBatch<NB> cb) {
    CULL_RESOLVE(cb);
    (void)vb;
    (void)vg;
    if (threadIdx.x) return;
    for (int t = 0; t <= q.tt; ++t)
        if (q.ctl->tier_off[t] + q.ctl->tier_count[t] > q.cap) q.ctl->status |= ST_OVERFLOW;
}

// ------------------------------------------------------------- grouping

__device__ inline uint32_t tile_of(uint64_t tri, int tc) {
    return tri_I(tri) * (uint32_t)tc + (tri_J(tri) >> 1);
}

template <int NB>
__global__ void __launch_bounds__(256) k_group_zero(CullBatch<NB> cb) {
    CULL_RESOLVE(cb);
    for (int64_t i = (int64_t)vb * blockDim.x + threadIdx.x; i < q.tiles;
         i += (int64_t)vg * blockDim.x) {
        q.tile_cnt[i] = 0u;
        q.tile_fill[i] = 0u;
    }
}

template <int NB>
__global__ void __launch_bounds__(256) k_group_count(CullBatch<NB> cb) {
    CULL_RESOLVE(cb);
    DevCtl* ctl = q.ctl;
    if (ctl->status & (ST_OVERFLOW | ST_NONFINITE)) return;
    const unsigned long long off = ctl->tier_off[q.tt];
    const unsigned long long m = ctl->tier_count[q.tt];
    for (unsigned long long g = (unsigned long long)vb * blockDim.x + threadIdx.x; g < m;
         g += (unsigned long long)vg * blockDim.x)
        atomicAdd(&q.tile_cnt[tile_of(q.pool[off + g], q.tc)], 1u);
}

// Exclusive scan of the tile counts (one block per product), and the pool
// layout of the grouped arrays behind the tier-tt frontier: entries (u32, one
// per tier-tt triple), then step K (u32) and step masks (2 x u64), S per
// entry.
template <int NB>
__global__ void __launch_bounds__(1024) k_group_scan(CullBatch<NB> cb) {
    CULL_RESOLVE(cb);
    (void)vb;
    (void)vg;
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    DevCtl* ctl = q.ctl;
    const uint32_t* __restrict__ cnt = q.tile_cnt;
    uint32_t* __restrict__ off = q.tile_off;
    const int tiles = q.tiles;
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
        const unsigned long long m = ctl->tier_count[q.tt];
        const unsigned long long end = ctl->tier_off[q.tt] + m;
        const unsigned long long ms = m * (unsigned long long)q.S;
        ctl->ent_off = end;
        ctl->pk_off = end + (m + 1) / 2;
        ctl->pm_off = ctl->pk_off + (ms + 1) / 2;
        ctl->ph_off = ctl->pm_off + 2 * ms * (unsigned long long)q.SL;
        ctl->need_words = ctl->ph_off + (q.tier ? 2 * ms : 0ull);
        if (ctl->need_words > q.cap || m >= 0xffffffffull / (unsigned long long)q.S)
            ctl->status |= ST_OVERFLOW;
    }
}

template <int NB>
__global__ void __launch_bounds__(256) k_group_scatter(CullBatch<NB> cb) {
    CULL_RESOLVE(cb);
    DevCtl* ctl = q.ctl;
    if (ctl->status & (ST_OVERFLOW | ST_NONFINITE)) return;
    const unsigned long long loff = ctl->tier_off[q.tt];
    const unsigned long long m = ctl->tier_count[q.tt];
    uint32_t* ent = reinterpret_cast<uint32_t*>(q.pool + ctl->ent_off);
    for (unsigned long long g = (unsigned long long)vb * blockDim.x + threadIdx.x; g < m;
         g += (unsigned long long)vg * blockDim.x) {
        const uint64_t tri = q.pool[loff + g];
        const uint32_t u = tile_of(tri, q.tc);
        ent[q.tile_off[u] + atomicAdd(&q.tile_fill[u], 1u)] = (tri_K(tri) << 1) | (tri_J(tri) & 1u);
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

// SL > 1: the sub-leaf cull along k.  Every leaf triple the cull keeps is
// tested slice by slice with the panel norms (same FP64 condition), and a
// step carries one mask pair per slice; a step none of whose slices
// survives is not written.
template <int DS, int NB, int SL>
__global__ void __launch_bounds__(kCullWarps * 32, 3) k_tile_cull(CullBatch<NB> cb) {
    constexpr int S = 1 << DS;               // K leaves per tier-tt K'
    constexpr int WIN = 1024 / SL;           // steps per window (16 KB of masks)
    constexpr int KPW = WIN / S;             // K' per window
    extern __shared__ uint32_t dyn[];        // K' bitmaps of both halves, then the K' list
    __shared__ unsigned long long masks[WIN][SL][2];
    // products of each step that keep the full split precision (q.tier)
    __shared__ unsigned long long hmasks[WIN][2];
    __shared__ unsigned long long st_slk, st_slt, st_vol, st_nhi, st_tiehi;
    __shared__ uint32_t st_iters;
    // per-warp staged norms of one sub-cube: levels 1..DS, A side [x][k], B side [k][y]
    __shared__ double nA[kCullWarps][84], nB[kCullWarps][84];
    __shared__ uint32_t warp_sums[16], total_s;
    __shared__ unsigned long long st_cand[4], st_kept[4], st_tie;
    CULL_RESOLVE(cb);
    const int tt = q.tt, tc = q.tc;
    const double* __restrict__ pyrA = q.pyrA;
    const double* __restrict__ pyrB = q.pyrB;
    const Thresh th = q.th;
    DevCtl* ctl = q.ctl;
    uint64_t* __restrict__ pool = q.pool;
    const uint32_t* __restrict__ off = q.tile_off;
    uint32_t* __restrict__ steps = q.tile_steps;
    if (ctl->status & (ST_OVERFLOW | ST_NONFINITE)) return;
    const uint32_t u = (uint32_t)vb;
    const uint32_t e0 = off[u], e1 = off[u + 1];
    if (e0 == e1) {
        if (threadIdx.x == 0) {
            steps[u] = 0;
            if (q.tile_iters) q.tile_iters[u] = 0;
        }
        return;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t I0 = u / tc, Jp = u % tc;
    const uint32_t* ent = reinterpret_cast<const uint32_t*>(pool + ctl->ent_off);
    uint32_t* pk = reinterpret_cast<uint32_t*>(pool + ctl->pk_off);
    unsigned long long* pm = reinterpret_cast<unsigned long long*>(pool + ctl->pm_off);
    unsigned long long* ph = reinterpret_cast<unsigned long long*>(pool + ctl->ph_off);
    const int words = ((1 << tt) + 31) >> 5;
    uint32_t* bm0 = dyn;
    uint32_t* bm1 = dyn + words;
    uint32_t* klist = dyn + 2 * words;
    for (int w = tid; w < 2 * words; w += blockDim.x) dyn[w] = 0u;
    if (tid < 4) st_cand[tid] = st_kept[tid] = 0ull;
    if (tid == 0) {
        st_tie = 0ull;
        st_slk = st_slt = 0ull;
        st_vol = st_nhi = st_tiehi = 0ull;
        st_iters = 0u;
    }
    unsigned long long slk = 0, slt = 0;     // kept / tested slice products
    // clipped volume (rows x k x columns inside the matrix) of the kept
    // products, and the precision tier's counts
    unsigned long long vol = 0, nhi = 0, tie_hi = 0;
    const int64_t nn = q.n, lb = q.b;
    auto ext = [&](int64_t L) -> unsigned long long {   // rows of leaf L inside the matrix
        const int64_t r = nn - L * lb;
        return (unsigned long long)(r < lb ? (r > 0 ? r : 0) : lb);
    };
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
                        // leaf level: the clipped extent of every kept leaf
                        // triple and, with the precision tier, whether its
                        // norm product reaches tau_h (the same FP64 test)
                        const int64_t I = ((int64_t)I0 << DS) + xi;
                        const int64_t K = ((int64_t)Kp << DS) + ki;
                        const int64_t J = ((int64_t)J0 << DS) + yi;
                        bool hi = false;
                        if (ok) {
                            if (SL == 1) vol += ext(I) * ext(K) * ext(J);
                            if (q.tier) {
                                bool tb;
                                hi = spamm_keep(nA[warp][so + xi * side + ki],
                                                nB[warp][so + ki * side + yi], q.thh, &tb);
                                tie_hi += tb ? 1 : 0;
                                nhi += hi ? 1 : 0;
                            }
                        }
                        if (q.tier) {
                            if (DS == 3) {
                                const unsigned hb = __ballot_sync(0xffffffffu, hi);
                                const int kk = r >> 1;
                                if (lane == 0) {
                                    if ((r & 1) == 0) hmasks[g * S + kk][half] = hb;
                                    else hmasks[g * S + kk][half] |= (unsigned long long)hb << 32;
                                }
                            } else {
                                const unsigned long long bit = hi ? 1ull << (yi * 8 + xi) : 0ull;
#pragma unroll
                                for (int kq = 0; kq < S; ++kq) {
                                    const unsigned long long mine = (idx < per && ki == kq) ? bit : 0ull;
                                    const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)mine);
                                    const uint32_t hh = __reduce_or_sync(0xffffffffu, (uint32_t)(mine >> 32));
                                    if (r == 0 && lane == 0) hmasks[g * S + kq][half] = 0ull;
                                    if (lane == 0) hmasks[g * S + kq][half] |= ((unsigned long long)hh << 32) | lo;
                                }
                            }
                        }
                    }
                    if (l == DS && SL > 1) {
                        // leaf level with the sub-leaf cull: per slice, the
                        // kept leaf triples whose panels pass, remapped to the
                        // mask of leaf column K' * S + ki, bit yi * 8 + xi
                        const int64_t I = ((int64_t)I0 << DS) + xi;
                        const int64_t K = ((int64_t)Kp << DS) + ki;
                        const int64_t J = ((int64_t)J0 << DS) + yi;
#pragma unroll
                        for (int sl = 0; sl < SL; ++sl) {
                            bool oks = false;
                            if (ok) {
                                bool tb;
                                oks = spamm_keep(q.panA[(I * q.nl + K) * SL + sl],
                                                 q.panB[(K * SL + sl) * q.nl + J], th, &tb);
                                tie += tb ? 1 : 0;
                                slt += 1;
                                slk += oks ? 1 : 0;
                                if (oks) {
                                    const int64_t kr = nn - K * lb - 16 * sl;
                                    vol += ext(I) * ext(J) *
                                           (unsigned long long)(kr < 16 ? (kr > 0 ? kr : 0) : 16);
                                }
                            }
                            const unsigned long long bit = oks ? 1ull << (yi * 8 + xi) : 0ull;
#pragma unroll
                            for (int kq = 0; kq < S; ++kq) {
                                const unsigned long long mine = (idx < per && ki == kq) ? bit : 0ull;
                                const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)mine);
                                const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(mine >> 32));
                                if (r == 0 && lane == 0) masks[g * S + kq][sl][half] = 0ull;
                                if (lane == 0) masks[g * S + kq][sl][half] |= ((unsigned long long)hi << 32) | lo;
                            }
                        }
                    } else if (l == DS) {
                        // leaf level: the mask of leaf column K' * S + ki
                        if (DS == 3) {
                            const int kk = r >> 1;           // uniform across the warp
                            if (lane == 0) {
                                if ((r & 1) == 0) masks[g * S + kk][0][half] = bal;
                                else masks[g * S + kk][0][half] |= (unsigned long long)bal << 32;
                            }
                        } else {
                            // remap bit (ki, yi, xi) -> mask of ki, bit yi * 8 + xi
                            const unsigned long long bit = ok ? 1ull << (yi * 8 + xi) : 0ull;
#pragma unroll
                            for (int kq = 0; kq < S; ++kq) {
                                const unsigned long long mine = (idx < per && ki == kq) ? bit : 0ull;
                                const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)mine);
                                const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(mine >> 32));
                                if (r == 0 && lane == 0) masks[g * S + kq][0][half] = 0ull;
                                if (lane == 0) masks[g * S + kq][0][half] |= ((unsigned long long)hi << 32) | lo;
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
                // the tile node is the leaf (I0, Kp, J0), kept iff it has an
                // entry; its precision tier from the leaf norms
                const unsigned long long rc = has ? ext(I0) * ext(J0) : 0ull;
                if (q.tier && lane == 0) {
                    bool hi = false;
                    if (has) {
                        const int64_t w = (int64_t)1 << tt;
                        const int64_t off_t = (((int64_t)1 << (2 * tt)) - 1) / 3;
                        bool tb;
                        hi = spamm_keep(pyrA[off_t + (int64_t)I0 * w + Kp],
                                        pyrB[off_t + (int64_t)Kp * w + J0], q.thh, &tb);
                        tie_hi += tb ? 1 : 0;
                        nhi += hi ? 1 : 0;
                    }
                    hmasks[g][half] = hi ? 1ull : 0ull;
                }
                if (SL > 1) {
                    // lane sl tests slice sl
                    bool oks = false;
                    if (lane < SL && has) {
                        bool tb;
                        oks = spamm_keep(q.panA[((int64_t)I0 * q.nl + Kp) * SL + lane],
                                         q.panB[((int64_t)Kp * SL + lane) * q.nl + J0], th, &tb);
                        tie += tb ? 1 : 0;
                        slt += 1;
                        slk += oks ? 1 : 0;
                        if (oks) {
                            const int64_t kr = nn - (int64_t)Kp * lb - 16 * lane;
                            vol += rc * (unsigned long long)(kr < 16 ? (kr > 0 ? kr : 0) : 16);
                        }
                    }
                    const unsigned bs = __ballot_sync(0xffffffffu, oks);
                    if (lane == 0)
                        for (int sl = 0; sl < SL; ++sl) masks[g][sl][half] = (bs >> sl) & 1u;
                } else if (lane == 0) {
                    masks[g][0][half] = has ? 1ull : 0ull;
                    vol += rc * ext(Kp);
                }
            }
            __syncwarp();  // staged norms are reused by the next sub-cube
        }
        __syncthreads();
        // phase 2: ordered compaction of the window's masks (ascending K)
        uint32_t it_mine = 0;
        for (int c0 = 0; c0 < kn * S; c0 += blockDim.x) {
            const int i = c0 + tid;
            uint32_t live = 0;                   // slices with a kept product
#pragma unroll
            for (int sl = 0; sl < SL; ++sl)
                if (i < kn * S && (masks[i][sl][0] | masks[i][sl][1]) != 0ull) live |= 1u << sl;
            const bool any = live != 0u;
            const uint32_t r = block_excl_scan(any ? 1u : 0u, warp_sums, &total_s);
            if (any) {
                const int g = i / S, kk = i % S;
                const uint32_t pos = obase + written + r;
                pk[pos] = klist[kw + g] * S + kk;
#pragma unroll
                for (int sl = 0; sl < SL; ++sl) {
                    pm[2 * ((size_t)pos * SL + sl)] = masks[i][sl][0];
                    pm[2 * ((size_t)pos * SL + sl) + 1] = masks[i][sl][1];
                }
                if (q.tier) {
                    ph[2 * (size_t)pos] = hmasks[i][0];
                    ph[2 * (size_t)pos + 1] = hmasks[i][1];
                }
                it_mine += SL > 1 ? (uint32_t)__popc(live) : (uint32_t)q.chunks;
            }
            written += total_s;
        }
        if (it_mine) atomicAdd(&st_iters, it_mine);
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
    for (int o = 16; o > 0; o >>= 1) {
        tie += __shfl_xor_sync(0xffffffffu, tie, o);
        slk += __shfl_xor_sync(0xffffffffu, slk, o);
        slt += __shfl_xor_sync(0xffffffffu, slt, o);
        vol += __shfl_xor_sync(0xffffffffu, vol, o);
        nhi += __shfl_xor_sync(0xffffffffu, nhi, o);
        tie_hi += __shfl_xor_sync(0xffffffffu, tie_hi, o);
    }
    if (lane == 0 && tie) atomicAdd(&st_tie, tie);
    if (lane == 0 && slt) {
        atomicAdd(&st_slk, slk);
        atomicAdd(&st_slt, slt);
    }
    if (lane == 0 && vol) atomicAdd(&st_vol, vol);
    if (lane == 0 && nhi) atomicAdd(&st_nhi, nhi);
    if (lane == 0 && tie_hi) atomicAdd(&st_tiehi, tie_hi);
    __syncthreads();
    if (tid == 0) {
        steps[u] = written;
        if (q.tile_iters) q.tile_iters[u] = st_iters;
        if (st_slt) {
            atomicAdd(&ctl->slice_kept, st_slk);
            atomicAdd(&ctl->slice_tested, st_slt);
        }
        atomicAdd(&ctl->active_steps, (unsigned long long)written);
        if (st_vol) atomicAdd(&ctl->clip_vol, st_vol);
        if (st_nhi) atomicAdd(&ctl->hi_products, st_nhi);
        if (st_tiehi) atomicAdd(&ctl->tie_hi, st_tiehi);
        for (int l = 0; l < DS; ++l) {
            atomicAdd(&ctl->tier_cand[tt + 1 + l], st_cand[l]);
            atomicAdd(&ctl->tier_count[tt + 1 + l], st_kept[l]);
        }
        if (st_tie) atomicAdd(&ctl->tie_band, st_tie);
    }
}

// ------------------------------------------------------------- launches

// Blocks of product p for a grid-stride kernel: its share (by leaf count) of
// `total`, at least one and at most `cap_blocks`.
static void share_blocks(const std::vector<double>& weight, int total, int64_t cap_blocks,
                         std::vector<int>& out) {
    double sum = 0.0;
    for (double w : weight) sum += w;
    out.resize(weight.size());
    for (size_t p = 0; p < weight.size(); ++p) {
        int64_t g = (int64_t)(total * (weight[p] / sum)) + 1;
        g = std::min<int64_t>(g, cap_blocks);
        out[p] = (int)std::max<int64_t>(g, 1);
    }
}

template <int NB>
static int set_bases(CullBatch<NB>& cb, const std::vector<int>& blocks) {
    if (cb.count < 0 || cb.count > NB) return 0;   // callers pass 1..NB products
    int b = 0;
    for (int p = 0; p < cb.count; ++p) {
        cb.bbase[p] = b;
        b += blocks[p];
    }
    cb.bbase[cb.count] = b;
    return b;
}

// Stage 2 for up to NB products: root, one launch per tier, overflow check.
template <int NB>
static cudaError_t cull_stage(const CullProd* prods, const std::vector<double>& weight, int count,
                              int sm_count, cudaStream_t s) {
    CullBatch<NB> cb;
    memset(&cb, 0, sizeof(cb));
    cb.count = count;
    int maxtt = 0;
    for (int p = 0; p < count; ++p) {
        cb.p[p] = prods[p];
        maxtt = std::max(maxtt, prods[p].tt);
    }
    std::vector<int> blocks(count, 1);
    int nb = set_bases(cb, blocks);
    k_cull_root<NB><<<nb, 32, 0, s>>>(cb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int full = sm_count * 4;
    for (int t = 0; t < maxtt; ++t) {
        // tier t + 1 has at most 8^(t+1) candidates: small tiers get small grids
        const int64_t cand_blocks = t + 1 < 7 ? (((int64_t)1 << (3 * (t + 1))) + 255) / 256 : full;
        share_blocks(weight, full, std::min<int64_t>(full, cand_blocks), blocks);
        // a product whose tiles sit above this tier takes no blocks; keep
        // the flattened grid free of them by moving them to the end
        CullBatch<NB> ct;
        memset(&ct, 0, sizeof(ct));
        std::vector<int> bl;
        for (int p = 0; p < count; ++p)
            if (t < prods[p].tt) {
                ct.p[ct.count++] = prods[p];
                bl.push_back(blocks[p]);
            }
        if (ct.count == 0) continue;
        nb = set_bases(ct, bl);
        k_cull_tier<NB><<<nb, 256, 0, s>>>(t, ct);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    std::fill(blocks.begin(), blocks.end(), 1);
    nb = set_bases(cb, blocks);
    k_cull_finish<NB><<<nb, 32, 0, s>>>(cb);
    return cudaGetLastError();
}

// Stage 3 for up to NB products: tile counts, scan, scatter, tile cull.
template <int NB>
static cudaError_t group_stage(const CullProd* prods, const std::vector<double>& weight, int count,
                               int sm_count, cudaStream_t s) {
    CullBatch<NB> cb;
    memset(&cb, 0, sizeof(cb));
    cb.count = count;
    for (int p = 0; p < count; ++p) cb.p[p] = prods[p];
    const int full = sm_count * 4;
    std::vector<int> blocks;
    for (int p = 0; p < count; ++p) blocks.push_back(std::max(1, std::min(64, (prods[p].tiles + 255) / 256)));
    int nb = set_bases(cb, blocks);
    k_group_zero<NB><<<nb, 256, 0, s>>>(cb);
    share_blocks(weight, full, full, blocks);
    nb = set_bases(cb, blocks);
    k_group_count<NB><<<nb, 256, 0, s>>>(cb);
    std::vector<int> ones(count, 1);
    const int nb1 = set_bases(cb, ones);
    k_group_scan<NB><<<nb1, 1024, 0, s>>>(cb);
    nb = set_bases(cb, blocks);
    k_group_scatter<NB><<<nb, 256, 0, s>>>(cb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // tile cull, one launch per depth below the tile nodes (DS = d - tt)
    for (int ds = 0; ds <= 3; ++ds) {
      for (int sl : {1, 2, 4, 8}) {
        CullBatch<NB> ct;
        memset(&ct, 0, sizeof(ct));
        std::vector<int> bl;
        size_t dsm = 0;
        for (int p = 0; p < count; ++p) {
            const int pds = prods[p].S == 1 ? 0 : prods[p].S == 2 ? 1 : prods[p].S == 4 ? 2 : 3;
            if (pds != ds || prods[p].SL != sl) continue;
            ct.p[ct.count++] = prods[p];
            bl.push_back(prods[p].tiles);
            const int words = ((1 << prods[p].tt) + 31) / 32;
            dsm = std::max(dsm, sizeof(uint32_t) * (2 * words + ((size_t)1 << prods[p].tt)));
        }
        if (ct.count == 0) continue;
        nb = set_bases(ct, bl);
        if (nb == 0) continue;
#define SPAMM_TC(DSV, SLV)                                                                    \
    do {                                                                                      \
        cudaFuncSetAttribute(k_tile_cull<DSV, NB, SLV>,                                       \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);          \
        cudaFuncSetAttribute(k_tile_cull<DSV, NB, SLV>,                                       \
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);            \
        k_tile_cull<DSV, NB, SLV><<<nb, kCullWarps * 32, dsm, s>>>(ct);                       \
    } while (0)
        // leaf sizes: b = 16 (SL 1), 32 (SL 2), 64 (SL 4), 128 (SL 8); DS is
        // log2(128 / b) except for products smaller than one tile
        if (sl == 1) {
            switch (ds) {
                case 0: SPAMM_TC(0, 1); break;
                case 1: SPAMM_TC(1, 1); break;
                case 2: SPAMM_TC(2, 1); break;
                default: SPAMM_TC(3, 1); break;
            }
        } else if (sl == 2) {
            switch (ds) {
                case 0: SPAMM_TC(0, 2); break;
                case 1: SPAMM_TC(1, 2); break;
                default: SPAMM_TC(2, 2); break;
            }
        } else if (sl == 4) {
            if (ds == 0) SPAMM_TC(0, 4);
            else SPAMM_TC(1, 4);
        } else {
            SPAMM_TC(0, 8);
        }
#undef SPAMM_TC
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
}

static CullProd make_prod(spamm_ctx* c, const spamm_tree* A, const spamm_tree* B, double tau,
                          double rel, int tt) {
    CullProd q;
    q.pyrA = A->pyr;
    q.pyrB = B->pyr;
    q.th = make_thresh(tau, rel);
    q.ctl = c->ctl;
    q.pool = c->pool;
    q.cap = (unsigned long long)c->pool_words;
    q.tile_cnt = c->tile_cnt;
    q.tile_fill = c->tile_fill;
    q.tile_off = c->tile_off;
    q.tile_steps = c->tile_steps;
    q.tile_iters = c->tile_iters;
    q.panA = A->panA;
    q.panB = B->panB;
    q.tt = tt;
    q.tc = tile_cols(A);
    q.tiles = tile_rows(A) * q.tc;
    q.S = 1 << (A->d - tt);
    q.SL = (A->slices && B->slices) ? A->slices : 1;
    q.chunks = A->b / 16;
    q.nl = (int)A->nl;
    q.tier = c->cfg.tier_bits > 0 ? 1 : 0;
    // tau_h = 2^tier_bits tau, exact (a power-of-two scale), so tau_h^2 is
    // formed as the oracle forms it
    q.thh = make_thresh(q.tier ? ldexp(tau, c->cfg.tier_bits) : tau, rel);
    q.n = A->n;
    q.b = A->b;
    return q;
}

cudaError_t launch_cull(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B, double tau,
                        int tt) {
    const CullProd q = make_prod(ctx, A, B, tau, ctx->cfg.tie_rel, tt);
    return cull_stage<1>(&q, std::vector<double>(1, 1.0), 1, ctx->sm_count, ctx->stream);
}

cudaError_t launch_group(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B, double tau,
                         int tt) {
    const CullProd q = make_prod(ctx, A, B, tau, ctx->cfg.tie_rel, tt);
    return group_stage<1>(&q, std::vector<double>(1, 1.0), 1, ctx->sm_count, ctx->stream);
}

// Stages 2-3 of `count` products, product p in sub-context subs[p] (its
// pool, control block and tile arrays, tile tier subs[p]->last_tt), on
// `stream`, up to kCullBatch products per launch.
cudaError_t launch_symbolic_batched(spamm_ctx* ctx, spamm_ctx* const* subs,
                                    const spamm_tree* const* A, const spamm_tree* const* B,
                                    const double* tau, int count, cudaStream_t stream) {
    for (int c0 = 0; c0 < count; c0 += kCullBatch) {
        const int cnt = std::min(kCullBatch, count - c0);
        std::vector<CullProd> prods;
        std::vector<double> weight;
        for (int i = 0; i < cnt; ++i) {
            const int p = c0 + i;
            prods.push_back(make_prod(subs[p], A[p], B[p], tau[p], ctx->cfg.tie_rel, subs[p]->last_tt));
            weight.push_back((double)A[p]->nl * (double)A[p]->nl);
        }
        cudaError_t e = cull_stage<kCullBatch>(prods.data(), weight, cnt, ctx->sm_count, stream);
        if (e == cudaSuccess)
            e = group_stage<kCullBatch>(prods.data(), weight, cnt, ctx->sm_count, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Control blocks of a batch: zero them (out == nullptr) or gather them into
// one array (out[p] = *ctl[p]) so that a single copy brings them to the host.
struct CtlTable {
    DevCtl* ctl[kCullBatch];
};

__global__ void k_ctl_batch(CtlTable tb, int count, DevCtl* __restrict__ out) {
    constexpr int W = sizeof(DevCtl) / sizeof(unsigned long long);
    static_assert(sizeof(DevCtl) % sizeof(unsigned long long) == 0, "");
    const int p = blockIdx.x;
    if (p >= count) return;
    unsigned long long* src = reinterpret_cast<unsigned long long*>(tb.ctl[p]);
    unsigned long long* dst = out ? reinterpret_cast<unsigned long long*>(out + p) : nullptr;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        if (dst) dst[w] = src[w];
        else src[w] = 0ull;
    }
}

cudaError_t launch_ctl_batch(spamm_ctx* const* subs, int count, DevCtl* out, cudaStream_t s) {
    for (int c0 = 0; c0 < count; c0 += kCullBatch) {
        const int cnt = std::min(kCullBatch, count - c0);
        CtlTable tb;
        memset(&tb, 0, sizeof(tb));
        for (int i = 0; i < cnt; ++i) tb.ctl[i] = subs[c0 + i]->ctl;
        k_ctl_batch<<<cnt, 128, 0, s>>>(tb, cnt, out ? out + c0 : nullptr);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace spamm
