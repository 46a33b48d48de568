// Host side of the C ABI declared in include/spamm.h: argument checks,
// device memory owned by contexts and trees, and the stream-ordered launch
// sequence of a multiply.  All arithmetic runs in the kernels of norms.cu,
// cull.cu, leaf_simt.cu and leaf_tc.cu.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "spamm_internal.cuh"

using namespace spamm;

namespace spamm {

spamm_status set_err(spamm_ctx* ctx, spamm_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return st;
}

spamm_status cuda_err(spamm_ctx* ctx, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SPAMM_OK;
    cudaGetLastError();  // clear a sticky launch error
    const spamm_status st = (e == cudaErrorMemoryAllocation) ? SPAMM_ERR_OOM : SPAMM_ERR_CUDA;
    return set_err(ctx, st, std::string(what) + ": " + cudaGetErrorString(e));
}

int tile_rows(const spamm_tree* t) { return (int)(t->nlp / (kTileRows / t->b)); }

int tile_cols(const spamm_tree* t) {
    return (int)(t->nlp / (kTileHalves * (kTileRows / t->b)));
}

int tile_tier(const spamm_tree* t) {
    int s = 0;
    while ((1 << s) < kTileRows / t->b) ++s;
    return t->d > s ? t->d - s : 0;
}

}  // namespace spamm

namespace {

bool valid_leaf(int b) { return b == 16 || b == 32 || b == 64 || b == 128; }

int depth_for(int64_t n, int b) {
    int d = 0;
    while ((int64_t)b * ((int64_t)1 << d) < n) ++d;
    return d;
}

spamm_status alloc_pool(spamm_ctx* ctx, int64_t bytes) {
    if (ctx->pool) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->pool);
        ctx->pool = nullptr;
        ctx->pool_words = 0;
    }
    bytes = std::max<int64_t>(bytes, 4096);
    bytes = (bytes + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&ctx->pool, (size_t)bytes);
    if (e != cudaSuccess) return cuda_err(ctx, e, "pool allocation");
    ctx->pool_words = bytes / 8;
    return SPAMM_OK;
}

spamm_status ensure_tiles(spamm_ctx* ctx, int64_t tiles) {
    if (tiles <= ctx->tiles_cap) return SPAMM_OK;
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->tile_cnt);
    cudaFree(ctx->tile_fill);
    cudaFree(ctx->tile_off);
    cudaFree(ctx->tile_steps);
    cudaFree(ctx->tile_iters);
    ctx->tile_cnt = ctx->tile_fill = ctx->tile_off = ctx->tile_steps = ctx->tile_iters = nullptr;
    ctx->tiles_cap = 0;
    const int64_t cap = std::max<int64_t>(tiles, 1024);
    cudaError_t e = cudaMalloc(&ctx->tile_cnt, sizeof(uint32_t) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->tile_fill, sizeof(uint32_t) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->tile_off, sizeof(uint32_t) * (cap + 1));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->tile_steps, sizeof(uint32_t) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->tile_iters, sizeof(uint32_t) * cap);
    if (e != cudaSuccess) return cuda_err(ctx, e, "tile arrays");
    ctx->tiles_cap = cap;
    return SPAMM_OK;
}

spamm_status ensure_need(spamm_ctx* ctx, int64_t nb) {
    if (2 * nb + 2 <= ctx->need_cap) return SPAMM_OK;
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->need);
    ctx->need = nullptr;
    ctx->need_cap = 0;
    const int64_t cap = std::max<int64_t>(2 * nb + 2, 1024);
    cudaError_t e = cudaMalloc(&ctx->need, sizeof(double) * cap);
    if (e != cudaSuccess) return cuda_err(ctx, e, "norm maxima");
    ctx->need_cap = cap;
    return SPAMM_OK;
}

void free_tree_storage(spamm_tree* t) {
    cudaFree(t->pyr);
    cudaFree(t->panA);
    cudaFree(t->panB);
    t->panA = t->panB = nullptr;
    cudaFree(t->slab);
    cudaFree(t->band);
    cudaFree(t->offs);
    cudaFree(t->band_new);
    cudaFree(t->sdev);
    cudaFreeHost(t->h_band);
    cudaFreeHost(t->h_offs);
    t->slab = nullptr;
    t->band = nullptr;
    t->offs = nullptr;
    t->band_new = nullptr;
    t->sdev = nullptr;
    t->h_band = nullptr;
    t->h_offs = nullptr;
    t->slab_cap = t->packa_cap = t->packb_cap = 0;
    for (int i = 0; i < 2; ++i) {
        cudaFree(t->packA[i]);
        cudaFree(t->packB[i]);
        t->packA[i] = t->packB[i] = nullptr;
    }
    t->pyr = nullptr;
}

spamm_status check_matrix(spamm_ctx* ctx, const float* A, int64_t n, int64_t lda) {
    if (!A) return set_err(ctx, SPAMM_ERR_INVALID_ARG, "matrix pointer is NULL");
    if (n <= 0) return set_err(ctx, SPAMM_ERR_INVALID_ARG, "n must be positive");
    if (lda < n) return set_err(ctx, SPAMM_ERR_INVALID_ARG, "leading dimension below n");
    return SPAMM_OK;
}

// Pool words a multiply needs: the frontiers of tiers 0..tt, then one u32
// entry per tier-tt triple and S steps (u32 K + SL pairs of u64 masks) per
// entry.
int64_t words_needed(const DevCtl& c, int tt, int S, int SL) {
    unsigned long long s = 0;
    for (int t = 0; t <= tt; ++t) s += c.tier_count[t];
    const unsigned long long m = c.tier_count[tt];
    const unsigned long long ms = m * (unsigned long long)S;
    return (int64_t)(s + (m + 1) / 2 + (ms + 1) / 2 + 2 * ms * (unsigned long long)SL);
}

// Mask pairs per step: one, or one per 16-wide k-slice with the sub-leaf cull.
int slices_of(const spamm_ctx* ctx, int b) { return ctx->cfg.slice ? b / 16 : 1; }

// Pool mask pairs per step: the kept masks, and with the precision tier the
// full-split masks.
int mask_pairs_of(const spamm_ctx* ctx, int b) {
    return slices_of(ctx, b) + (ctx->cfg.tier_bits > 0 ? 1 : 0);
}

bool split_precision(int p) {
    return p == SPAMM_PREC_TF32X3 || p == SPAMM_PREC_BF16X3 || p == SPAMM_PREC_F16X3;
}

// Stats fields of one product from its control block.
void fill_tier_stats(const spamm_ctx* ctx, const DevCtl& c, int64_t leaf_triples,
                     spamm_stats_t* out) {
    out->hi_products = ctx->cfg.tier_bits > 0 ? (int64_t)c.hi_products : leaf_triples;
    out->tie_band_hi = (int64_t)c.tie_hi;
    out->kept_flops_clipped = 2.0 * (double)c.clip_vol;
}

}  // namespace

extern "C" {

void spamm_config_default(spamm_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->leaf = 16;
    cfg->precision = SPAMM_PREC_FP32;
    cfg->tie_rel = 1e-6;
    cfg->pool_bytes = 0;
    cfg->checked = 1;
}

spamm_status spamm_create(spamm_ctx** out, void* stream, const spamm_config* cfg) {
    if (!out) return SPAMM_ERR_INVALID_ARG;
    *out = nullptr;
    spamm_config c;
    if (cfg) c = *cfg; else spamm_config_default(&c);
    if (!valid_leaf(c.leaf)) return SPAMM_ERR_INVALID_ARG;
    if (c.precision < SPAMM_PREC_FP32 || c.precision > SPAMM_PREC_F16X3) return SPAMM_ERR_INVALID_ARG;
    if (!(c.tie_rel >= 0.0 && c.tie_rel < 0.5) || c.pool_bytes < 0) return SPAMM_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i)
        if (c.reserved[i]) return SPAMM_ERR_INVALID_ARG;
    if (c.staged != 0 && c.staged != 1) return SPAMM_ERR_INVALID_ARG;
    if (c.tier_bits < 0 || c.tier_bits > 40) return SPAMM_ERR_INVALID_ARG;
    if (c.tier_bits && !split_precision(c.precision)) return SPAMM_ERR_INVALID_ARG;
    if (c.slice != 0 && c.slice != 16) return SPAMM_ERR_INVALID_ARG;
    if (c.slice && (!precision_uses_tc(c.precision) || c.leaf < 32)) return SPAMM_ERR_UNSUPPORTED;
    spamm_ctx* ctx = new (std::nothrow) spamm_ctx();
    if (!ctx) return SPAMM_ERR_OOM;
    ctx->stream = (cudaStream_t)stream;
    ctx->cfg = c;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->ctl, sizeof(DevCtl));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->ctl_host, sizeof(DevCtl));
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
    if (e != cudaSuccess) {
        spamm_status st = (e == cudaErrorMemoryAllocation) ? SPAMM_ERR_OOM : SPAMM_ERR_CUDA;
        cudaGetLastError();
        spamm_destroy(ctx);
        return st;
    }
    memset(ctx->ctl_host, 0, sizeof(DevCtl));
    spamm_status st = alloc_pool(ctx, c.pool_bytes ? c.pool_bytes : ((int64_t)1 << 30));
    if (st == SPAMM_OK) st = ensure_tiles(ctx, 1024);
    if (st != SPAMM_OK) {
        spamm_destroy(ctx);
        return st;
    }
    ctx->last_status = SPAMM_OK;
    *out = ctx;
    return SPAMM_OK;
}

spamm_status spamm_destroy(spamm_ctx* ctx) {
    if (!ctx) return SPAMM_ERR_INVALID_ARG;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->hostTreeA) spamm_tree_destroy(ctx->hostTreeA);
    if (ctx->hostTreeB) spamm_tree_destroy(ctx->hostTreeB);
    for (spamm_tree* t : ctx->trees) t->ctx = nullptr;
    ctx->trees.clear();
    for (spamm_ctx* sub : ctx->subs) spamm_destroy(sub);
    ctx->subs.clear();
    cudaFree(ctx->pool);
    cudaFree(ctx->ctl);
    if (ctx->ctl_host) cudaFreeHost(ctx->ctl_host);
    cudaFree(ctx->tile_cnt);
    cudaFree(ctx->tile_fill);
    cudaFree(ctx->tile_off);
    cudaFree(ctx->tile_steps);
    cudaFree(ctx->tile_iters);
    cudaFree(ctx->need);
    cudaFree(ctx->dA);
    cudaFree(ctx->dB);
    cudaFree(ctx->dC);
    for (int i = 0; i < 4; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    cudaFree(ctx->bctl);
    if (ctx->bctl_host) cudaFreeHost(ctx->bctl_host);
    if (ctx->aux_ready) {
        for (int i = 0; i < spamm_ctx::kAux; ++i) {
            cudaStreamSynchronize(ctx->aux[i]);
            cudaStreamDestroy(ctx->aux[i]);
            cudaEventDestroy(ctx->aux_ev[i]);
        }
        cudaEventDestroy(ctx->fork_ev);
        cudaStreamSynchronize(ctx->hi);
        cudaStreamDestroy(ctx->hi);
        cudaEventDestroy(ctx->hi_ev);
    }
    cudaGetLastError();
    delete ctx;
    return SPAMM_OK;
}

spamm_status spamm_set_stream(spamm_ctx* ctx, void* stream) {
    if (!ctx) return SPAMM_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)stream;
    return SPAMM_OK;
}

spamm_status spamm_set_checked(spamm_ctx* ctx, int32_t checked) {
    if (!ctx) return SPAMM_ERR_INVALID_ARG;
    ctx->cfg.checked = checked ? 1 : 0;
    return SPAMM_OK;
}

spamm_status spamm_set_wait_limit(spamm_ctx* ctx, int64_t wait_ns) {
    if (!ctx) return SPAMM_ERR_INVALID_ARG;
    ctx->wait_ns = wait_ns > 0 ? wait_ns : 0;
    return SPAMM_OK;
}

spamm_status spamm_reserve(spamm_ctx* ctx, int64_t pool_bytes) {
    if (!ctx || pool_bytes < 0) return SPAMM_ERR_INVALID_ARG;
    if (pool_bytes <= ctx->pool_words * 8) return SPAMM_OK;
    return alloc_pool(ctx, pool_bytes);
}

const char* spamm_last_error(const spamm_ctx* ctx) {
    return ctx ? ctx->err.c_str() : "NULL context";
}

static spamm_status build_into(spamm_ctx* ctx, spamm_tree* t) {
    cudaError_t e = launch_build_norms(t, ctx->stream);
    return cuda_err(ctx, e, "norm build launch");
}

// A tree's shape and norm storage; with packs = true also the dense pack
// arrays.  On failure nothing is left allocated.
static spamm_status new_tree(spamm_ctx* ctx, const float* A, int64_t n, int64_t lda, bool packs,
                             spamm_tree** out) {
    const int b = ctx->cfg.leaf;
    const int d = depth_for(n, b);
    const int64_t nl = (n + b - 1) / b;
    if (nl > kMaxLeavesPerSide || d >= SPAMM_MAX_TIERS - 1)
        return set_err(ctx, SPAMM_ERR_UNSUPPORTED, "more than 2^14 leaves per side");
    const int tl = kTileRows / b;
    spamm_tree* t = new (std::nothrow) spamm_tree();
    if (!t) return SPAMM_ERR_OOM;
    t->ctx = ctx;
    t->A = A;
    t->n = n;
    t->lda = lda;
    t->b = b;
    t->d = d;
    t->nb = (int64_t)1 << d;
    t->nl = nl;
    t->nlp = (nl + 2 * tl - 1) / (2 * tl) * (2 * tl);
    t->nodes = (((int64_t)1 << (2 * (d + 1))) - 1) / 3;
    t->precision = ctx->cfg.precision;
    t->slices = ctx->cfg.slice ? b / ctx->cfg.slice : 0;
    cudaError_t e = cudaMalloc(&t->pyr, sizeof(double) * t->nodes);
    if (e == cudaSuccess && t->slices) {
        const size_t pn = sizeof(double) * (size_t)nl * (size_t)nl * (size_t)t->slices;
        e = cudaMalloc(&t->panA, pn);
        if (e == cudaSuccess) e = cudaMalloc(&t->panB, pn);
    }
    if (e == cudaSuccess && packs && precision_uses_tc(t->precision)) {
        // grouped layout: every part of a role in one array (packA[1] unused)
        t->pack_bytes = pack_bytes_for(t->precision, t->nlp, b);
        const size_t all = t->pack_bytes * (size_t)pack_arrays_for(t->precision);
        e = cudaMalloc(&t->packA[0], all);
        if (e == cudaSuccess) e = cudaMalloc(&t->packB[0], all);
        if (e == cudaSuccess) e = cudaMemsetAsync(t->packA[0], 0, all, ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(t->packB[0], 0, all, ctx->stream);
    }
    if (e != cudaSuccess) {
        const spamm_status st = cuda_err(ctx, e, "tree allocation");
        free_tree_storage(t);
        delete t;
        return st;
    }
    t->bytes = (int64_t)sizeof(double) * t->nodes +
               (t->slices ? 2 * (int64_t)sizeof(double) * nl * nl * t->slices : 0) +
               (int64_t)t->pack_bytes * 2 * (packs && precision_uses_tc(t->precision)
                                                 ? pack_arrays_for(t->precision) : 0);
    *out = t;
    return SPAMM_OK;
}

spamm_status spamm_build_norms(spamm_ctx* ctx, const float* A, int64_t n, int64_t lda,
                               spamm_tree** out) {
    if (!ctx || !out) return SPAMM_ERR_INVALID_ARG;
    *out = nullptr;
    spamm_status st = check_matrix(ctx, A, n, lda);
    if (st != SPAMM_OK) return st;
    spamm_tree* t = nullptr;
    st = new_tree(ctx, A, n, lda, true, &t);
    if (st != SPAMM_OK) return st;
    st = build_into(ctx, t);
    if (st != SPAMM_OK) {
        cudaStreamSynchronize(ctx->stream);
        free_tree_storage(t);
        delete t;
        return st;
    }
    ctx->trees.push_back(t);
    *out = t;
    return SPAMM_OK;
}

// The sparsified storage of A in t (Sec. II.D): dense norms, the drop and
// the bands on the device, one synchronisation to bring the bands to the
// host, the slab and pack layout there, then the offsets, bands and slab
// copy queued on the stream.  Storage already held is reused when the new
// bands fit (grown a quarter beyond the need when they do not), so a
// re-sparsify of a tree in a loop allocates nothing.  On any error the root
// norm is left non-finite, so a multiply with the tree reports NONFINITE
// before it reads bands, offsets or slab that no longer match its norms.
static spamm_status sparsify_fill(spamm_ctx* ctx, spamm_tree* t, const float* A, int64_t lda,
                                  double tau, double partner_norm2) {
    cudaStream_t s = ctx->stream;
    const int64_t nl = t->nl;
    const int b = t->b;
    const size_t nband = (size_t)4 * (size_t)std::max<int64_t>(nl, 1);
    const size_t noffs = (size_t)(3 * nl + 2);
    auto poison = [&](spamm_status st) {
        // a NaN root: every multiply with this tree stops at its root test
        cudaMemsetAsync(t->pyr, 0xff, sizeof(double), s);
        return st;
    };
    cudaError_t e = cudaSuccess;
    if (!t->band) {
        e = cudaMalloc(&t->band, sizeof(int32_t) * nband);
        if (e == cudaSuccess) e = cudaMalloc(&t->band_new, sizeof(int32_t) * nband);
        if (e == cudaSuccess) e = cudaMalloc(&t->offs, sizeof(int64_t) * noffs);
        if (e == cudaSuccess) e = cudaMalloc(&t->sdev, 2 * sizeof(unsigned long long));
        if (e == cudaSuccess)
            e = cudaMallocHost(&t->h_band, sizeof(int32_t) * nband + 2 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMallocHost(&t->h_offs, sizeof(int64_t) * noffs);
        if (e != cudaSuccess) return cuda_err(ctx, e, "sparsify bands");
    }
    // 1. dense norms (and panels) of A; 2. drop, new bands, upper tiers
    t->A = A;
    t->lda = lda;
    e = launch_build_norms(t, s);
    t->A = nullptr;       // the tree holds its own copy of the kept leaves
    t->lda = 0;
    unsigned long long* hw = reinterpret_cast<unsigned long long*>(t->h_band + nband);
    if (e == cudaSuccess)
        e = launch_sparsify_mark(t, tau, partner_norm2, ctx->cfg.tie_rel, t->band_new, t->sdev, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(t->h_band, t->band_new, sizeof(int32_t) * 4 * nl,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hw, t->sdev, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return poison(cuda_err(ctx, e, "sparsify bands"));
    double root;
    memcpy(&root, &hw[1], sizeof(root));
    if (!std::isfinite(root))
        return set_err(ctx, SPAMM_ERR_NONFINITE, "an operand holds Inf or NaN");
    // 3. slab and pack layout (host)
    const int32_t* kmin = t->h_band;
    const int32_t* kmax = kmin + nl;
    const int32_t* imin = kmin + 2 * nl;
    const int32_t* imax = kmin + 3 * nl;
    const int CH = b / 16;
    int64_t* roff = t->h_offs;
    int64_t* aoff = roff + nl;
    int64_t* boff = aoff + nl + 1;
    int64_t slab = 0, pa = 0, pb = 0;
    for (int64_t q = 0; q < nl; ++q) {
        roff[q] = slab;
        aoff[q] = pa;
        boff[q] = pb;
        if (kmin[q] <= kmax[q]) {
            slab += (int64_t)b * (kmax[q] - kmin[q] + 1) * b;
            pb += (int64_t)CH * (kmax[q] - kmin[q] + 1);
        }
        if (imin[q] <= imax[q]) pa += (int64_t)CH * (imax[q] - imin[q] + 1);
    }
    aoff[nl] = pa;
    boff[nl] = pb;
    const int64_t piece =
        (int64_t)b * 16 *
        ((t->precision == SPAMM_PREC_BF16X3 || t->precision == SPAMM_PREC_F16X3) ? 2 : 4);
    const int arrays = pack_arrays_for(t->precision);
    // 4. storage: kept while the new bands fit.  The stream is idle here
    // (synchronised above), so nothing in flight reads what is freed.
    const bool first = t->slab == nullptr;
    auto grown = [&](int64_t need, int64_t floor) {
        return std::max<int64_t>(first ? need : need + need / 4, floor);
    };
    if (slab > t->slab_cap || first) {
        cudaFree(t->slab);
        t->slab = nullptr;
        t->slab_cap = 0;
        const int64_t c = grown(slab, 64);
        e = cudaMalloc(&t->slab, sizeof(float) * (size_t)c);
        if (e != cudaSuccess) return poison(cuda_err(ctx, e, "sparsify storage"));
        t->slab_cap = c;
    }
    auto packs = [&](void** arr, int64_t need, int64_t* cap) -> cudaError_t {
        if (need <= *cap && arr[0]) return cudaSuccess;
        for (int i = 0; i < 2; ++i) {
            cudaFree(arr[i]);
            arr[i] = nullptr;
        }
        *cap = 0;
        const int64_t c = grown(need, 256);
        for (int i = 0; i < arrays; ++i) {
            const cudaError_t ee = cudaMalloc(&arr[i], (size_t)c);
            if (ee != cudaSuccess) return ee;
        }
        *cap = c;
        return cudaSuccess;
    };
    e = packs(t->packA, pa * piece, &t->packa_cap);
    if (e == cudaSuccess) e = packs(t->packB, pb * piece, &t->packb_cap);
    if (e != cudaSuccess) return poison(cuda_err(ctx, e, "sparsify storage"));
    // 5. offsets and bands, then the kept leaves into the slab (queued: the
    // slab copy may still read A when the call returns)
    e = cudaMemcpyAsync(t->offs, t->h_offs, sizeof(int64_t) * noffs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(t->band, t->band_new, sizeof(int32_t) * 4 * nl,
                            cudaMemcpyDeviceToDevice, s);
    t->sparse = 1;
    if (e == cudaSuccess) e = launch_slab_copy(t, A, lda, s);
    if (e != cudaSuccess) return poison(cuda_err(ctx, e, "sparsify storage"));
    t->stored = (int64_t)hw[0];
    t->bytes = (int64_t)sizeof(double) * t->nodes + (int64_t)sizeof(int32_t) * 8 * nl +
               (int64_t)sizeof(int64_t) * (3 * nl + 2) + (int64_t)sizeof(float) * t->slab_cap +
               (int64_t)arrays * (t->packa_cap + t->packb_cap) +
               (t->slices ? 2 * (int64_t)sizeof(double) * nl * nl * t->slices : 0);
    return SPAMM_OK;
}

static spamm_status sparsify_args(spamm_ctx* ctx, double tau, double partner_norm2) {
    if (!(tau >= 0.0) || !std::isfinite(tau) || !(partner_norm2 >= 0.0) ||
        !std::isfinite(partner_norm2))
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "tau and partner_norm2 must be finite and >= 0");
    if (!precision_uses_tc(ctx->cfg.precision))
        return set_err(ctx, SPAMM_ERR_UNSUPPORTED, "sparsified trees need a tensor-core precision");
    return SPAMM_OK;
}

spamm_status spamm_sparsify(spamm_ctx* ctx, const float* A, int64_t n, int64_t lda, double tau,
                            double partner_norm2, spamm_tree** out) {
    if (!ctx || !out) return SPAMM_ERR_INVALID_ARG;
    *out = nullptr;
    spamm_status st = check_matrix(ctx, A, n, lda);
    if (st == SPAMM_OK) st = sparsify_args(ctx, tau, partner_norm2);
    if (st != SPAMM_OK) return st;
    spamm_tree* t = nullptr;
    st = new_tree(ctx, A, n, lda, false, &t);
    if (st != SPAMM_OK) return st;
    st = sparsify_fill(ctx, t, A, lda, tau, partner_norm2);
    if (st != SPAMM_OK) {
        cudaStreamSynchronize(ctx->stream);
        free_tree_storage(t);
        delete t;
        return st;
    }
    ctx->trees.push_back(t);
    *out = t;
    return SPAMM_OK;
}

spamm_status spamm_sparsify_into(spamm_ctx* ctx, spamm_tree* tree, const float* A, int64_t lda,
                                 double tau, double partner_norm2) {
    if (!ctx || !tree) return set_err(ctx, SPAMM_ERR_INVALID_ARG, "NULL argument");
    if (!tree->sparse)
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "not a sparsified tree");
    if (tree->ctx != ctx || tree->precision != ctx->cfg.precision || tree->b != ctx->cfg.leaf)
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "tree built under another configuration");
    spamm_status st = check_matrix(ctx, A, tree->n, lda);
    if (st == SPAMM_OK) st = sparsify_args(ctx, tau, partner_norm2);
    if (st != SPAMM_OK) return st;
    return sparsify_fill(ctx, tree, A, lda, tau, partner_norm2);
}

spamm_status spamm_tree_bytes(const spamm_tree* t, int64_t* bytes, int64_t* stored) {
    if (!t || !bytes) return SPAMM_ERR_INVALID_ARG;
    *bytes = t->bytes;
    if (stored) *stored = t->sparse ? t->stored : -1;
    return SPAMM_OK;
}

spamm_status spamm_tree_rebuild(spamm_ctx* ctx, spamm_tree* t, const float* A, int64_t lda) {
    if (!ctx || !t) return SPAMM_ERR_INVALID_ARG;
    if (t->sparse)
        return set_err(ctx, SPAMM_ERR_UNSUPPORTED, "a sparsified tree is rebuilt by spamm_sparsify");
    spamm_status st = check_matrix(ctx, A, t->n, lda);
    if (st != SPAMM_OK) return st;
    if (t->precision != ctx->cfg.precision || t->b != ctx->cfg.leaf)
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "tree built under another configuration");
    t->A = A;
    t->lda = lda;
    return build_into(ctx, t);
}

spamm_status spamm_tree_destroy(spamm_tree* t) {
    if (!t) return SPAMM_ERR_INVALID_ARG;
    if (t->ctx) {
        cudaStreamSynchronize(t->ctx->stream);
        std::vector<spamm_tree*>& v = t->ctx->trees;
        v.erase(std::remove(v.begin(), v.end(), t), v.end());
    }
    free_tree_storage(t);   // cudaFree waits for work that still uses it
    delete t;
    return SPAMM_OK;
}

spamm_status spamm_tree_footprint(const spamm_ctx* ctx, int64_t n, int64_t* bytes) {
    if (!ctx || !bytes || n <= 0) return SPAMM_ERR_INVALID_ARG;
    const int b = ctx->cfg.leaf;
    const int d = depth_for(n, b);
    const int64_t nl = (n + b - 1) / b;
    if (nl > kMaxLeavesPerSide || d >= SPAMM_MAX_TIERS - 1) return SPAMM_ERR_UNSUPPORTED;
    const int tl = kTileRows / b;
    const int64_t nlp = (nl + 2 * tl - 1) / (2 * tl) * (2 * tl);
    const int64_t nodes = (((int64_t)1 << (2 * (d + 1))) - 1) / 3;
    int64_t total = (int64_t)sizeof(double) * nodes;
    if (precision_uses_tc(ctx->cfg.precision))
        total += 2 * (int64_t)pack_arrays_for(ctx->cfg.precision) *
                 (int64_t)pack_bytes_for(ctx->cfg.precision, nlp, b);
    if (ctx->cfg.slice) total += 2 * (int64_t)sizeof(double) * nl * nl * (b / ctx->cfg.slice);
    *bytes = total;
    return SPAMM_OK;
}

spamm_status spamm_tree_shape(const spamm_tree* t, int32_t* depth, int64_t* nodes) {
    if (!t) return SPAMM_ERR_INVALID_ARG;
    if (depth) *depth = t->d;
    if (nodes) *nodes = t->nodes;
    return SPAMM_OK;
}

spamm_status spamm_tree_norms(spamm_ctx* ctx, const spamm_tree* t, double* host_out,
                              int64_t count) {
    if (!ctx || !t || !host_out || count < t->nodes) return SPAMM_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(host_out, t->pyr, sizeof(double) * t->nodes,
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return cuda_err(ctx, e, "norm copy");
}

// Copy-out hook of the banded leaf launch: rows [r0, r1) of the staged C
// go to the host on aux[0] once the band that finished them (on stream s)
// has run.
static cudaError_t copy_rows_out(void* user, int64_t r0, int64_t r1, cudaStream_t s) {
    spamm_ctx* ctx = static_cast<spamm_ctx*>(user);
    const int64_t n = ctx->last_n;
    cudaError_t e = cudaEventRecord(ctx->aux_ev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->aux[0], ctx->aux_ev[0], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->band_host + r0 * n, ctx->dC + r0 * n,
                            sizeof(float) * (size_t)((r1 - r0) * n), cudaMemcpyDeviceToHost,
                            ctx->aux[0]);
    return e;
}

static spamm_status ensure_aux(spamm_ctx* ctx);

// One multiply on the context stream.  The tensor-core packs depend on the
// leaf norms and tau only, not on the cull, so the cull and grouping run on
// the high-priority side stream beside them: the small latency-bound cull
// launches go ahead of the HBM-bound pack kernel's blocks, and the leaf
// products wait for both.
static spamm_status launch_multiply_once(spamm_ctx* ctx, const spamm_tree* A,
                                         const spamm_tree* B, double tau, float alpha,
                                         float beta, float* C, int64_t ldc) {
    cudaStream_t s = ctx->stream;
    const bool tc = precision_uses_tc(ctx->cfg.precision);
    cudaError_t e = cudaMemsetAsync(ctx->ctl, 0, sizeof(DevCtl), s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[0], s);
    ctx->last_small = small_path(ctx, A);
    if (ctx->last_small) {
        // one launch: cull, grouping and FP32 leaf products of a small product
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[1], s);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[3], s);
        if (e == cudaSuccess) e = launch_small_fp32(ctx, A, B, tau, alpha, beta, C, ldc);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[2], s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s);
        ctx->timed = (e == cudaSuccess);
        return cuda_err(ctx, e, "multiply launch");
    }
    const int tt = tile_tier(A);
    if (tc) {
        // fork: cull + grouping on ctx->hi, packs on the context stream, join
        if (e == cudaSuccess) e = cudaEventRecord(ctx->fork_ev, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->hi, ctx->fork_ev, 0);
        ctx->stream = ctx->hi;
        if (e == cudaSuccess) e = launch_cull(ctx, A, B, tau, tt);
        if (e == cudaSuccess) e = launch_group(ctx, A, B, tau, tt);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[1], ctx->hi);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->hi_ev, ctx->hi);
        ctx->stream = s;
        if (e == cudaSuccess)
            e = launch_packs(ctx->ctl, A, B, tau, ctx->cfg.tie_rel, ctx->need, ctx->sm_count, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->hi_ev, 0);
    } else {
        if (e == cudaSuccess) e = launch_cull(ctx, A, B, tau, tt);
        if (e == cudaSuccess) e = launch_group(ctx, A, B, tau, tt);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[1], s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[3], s);
    if (e == cudaSuccess) {
        if (ctx->cfg.precision == SPAMM_PREC_FP32)
            e = launch_leaf_simt(ctx, A, B, alpha, beta, C, ldc);
        else if (ctx->band_host)
            e = launch_leaf_tc_banded(ctx, A, B, alpha, beta, C, ldc, ctx->band_count,
                                      copy_rows_out, ctx);
        else
            e = launch_leaf_tc(ctx, A, B, alpha, beta, C, ldc);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[2], s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s);
    ctx->timed = (e == cudaSuccess);
    return cuda_err(ctx, e, "multiply launch");
}

static spamm_status status_from_ctl(spamm_ctx* ctx, const DevCtl& c);
static spamm_status status_from_ctl_pub(spamm_ctx* ctx, const DevCtl& c) {
    return status_from_ctl(ctx, c);
}
static spamm_status status_from_ctl(spamm_ctx* ctx, const DevCtl& c) {
    if (c.status & ST_NONFINITE)
        return set_err(ctx, SPAMM_ERR_NONFINITE, "an operand holds Inf or NaN");
    if (c.status & ST_TIMEOUT)
        return set_err(ctx, SPAMM_ERR_TIMEOUT, "a device-side wait timed out");
    if (c.status & ST_OVERFLOW)
        return set_err(ctx, SPAMM_ERR_CAPACITY, "triple pool overflow");
    return SPAMM_OK;
}

spamm_status spamm_multiply(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B,
                            double tau, float alpha, float beta, float* C, int64_t ldc) {
    if (!ctx || !A || !B || !C) return set_err(ctx, SPAMM_ERR_INVALID_ARG, "NULL argument");
    if (!(tau >= 0.0) || !std::isfinite(tau))
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "tau must be finite and >= 0");
    if (A->n != B->n || A->b != B->b || A->precision != B->precision)
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "trees differ in n, leaf or precision");
    if (A->precision != ctx->cfg.precision || A->b != ctx->cfg.leaf)
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "trees built under another configuration");
    if (ldc < A->n) return set_err(ctx, SPAMM_ERR_INVALID_ARG, "ldc below n");
    const int64_t tiles = (int64_t)tile_rows(A) * tile_cols(A);
    spamm_status st = ensure_tiles(ctx, tiles);
    if (st == SPAMM_OK) st = ensure_need(ctx, A->nb);
    if (st == SPAMM_OK && precision_uses_tc(ctx->cfg.precision)) st = ensure_aux(ctx);
    if (st != SPAMM_OK) return st;
    ctx->last_batch = 0;
    ctx->last_d = A->d;
    ctx->last_b = A->b;
    ctx->last_n = A->n;
    ctx->last_prec = A->precision;
    ctx->last_tau = tau;
    ctx->last_tiles = tiles;
    ctx->last_tr = tile_rows(A);
    ctx->last_tc = tile_cols(A);
    ctx->last_tt = tile_tier(A);
    ctx->last_S = 1 << (A->d - ctx->last_tt);
    ctx->last_status = SPAMM_OK;
    for (int attempt = 0;; ++attempt) {
        st = launch_multiply_once(ctx, A, B, tau, alpha, beta, C, ldc);
        if (st != SPAMM_OK) return (spamm_status)(ctx->last_status = st);
        if (!ctx->cfg.checked) return SPAMM_OK;
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return (spamm_status)(ctx->last_status = cuda_err(ctx, e, "multiply"));
        const DevCtl& c = *ctx->ctl_host;
        if ((c.status & ST_OVERFLOW) && !(c.status & (ST_NONFINITE | ST_TIMEOUT)) && attempt < 8) {
            const int64_t need = std::max<int64_t>(words_needed(c, ctx->last_tt, ctx->last_S, mask_pairs_of(ctx, ctx->last_b)),
                                                   2 * ctx->pool_words);
            st = alloc_pool(ctx, need * 8 + need * 2);  // 25% headroom
            if (st != SPAMM_OK) return (spamm_status)(ctx->last_status = st);
            continue;
        }
        return (spamm_status)(ctx->last_status = status_from_ctl(ctx, c));
    }
}

static spamm_status batch_stats(spamm_ctx* ctx, spamm_stats_t* out);

spamm_status spamm_stats(spamm_ctx* ctx, spamm_stats_t* out) {
    if (!ctx || !out) return SPAMM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "stats");
    if (ctx->last_batch > 0) return batch_stats(ctx, out);
    memset(out, 0, sizeof(*out));
    const DevCtl& c = *ctx->ctl_host;
    const int d = ctx->last_d;
    out->depth = d;
    out->n = ctx->last_n;
    out->leaf = ctx->last_b;
    out->precision = ctx->last_prec;
    out->tau = ctx->last_tau;
    for (int t = 0; t <= d && t < SPAMM_MAX_TIERS; ++t) {
        out->tier_candidates[t] = (int64_t)c.tier_cand[t];
        out->tier_kept[t] = (int64_t)c.tier_count[t];
    }
    out->leaf_triples = (int64_t)c.tier_count[d];
    out->tie_band = (int64_t)c.tie_band;
    out->active_steps = (int64_t)c.active_steps;
    out->tiles = ctx->last_tiles;
    const double b = ctx->last_b;
    out->kept_flops = 2.0 * b * b * b * (double)out->leaf_triples;
    out->slice = ctx->cfg.slice;
    out->slice_kept = (int64_t)c.slice_kept;
    out->slice_tested = (int64_t)c.slice_tested;
    out->packed_leaves_a = (int64_t)c.packed_a;
    out->packed_leaves_b = (int64_t)c.packed_b;
    if (ctx->cfg.slice) out->kept_flops = 2.0 * b * b * ctx->cfg.slice * (double)c.slice_kept;
    fill_tier_stats(ctx, c, out->leaf_triples, out);
    out->dense_flops = 2.0 * (double)ctx->last_n * (double)ctx->last_n * (double)ctx->last_n;
    out->pool_bytes = ctx->pool_words * 8;
    out->pool_needed_bytes = words_needed(c, ctx->last_tt, ctx->last_S, mask_pairs_of(ctx, ctx->last_b)) * 8;
    if (ctx->timed) {
        cudaEventElapsedTime(&out->ms_symbolic, ctx->ev[0], ctx->ev[1]);
        cudaEventElapsedTime(&out->ms_pack, ctx->ev[1], ctx->ev[3]);
        cudaEventElapsedTime(&out->ms_numeric, ctx->ev[3], ctx->ev[2]);
        cudaEventElapsedTime(&out->ms_total, ctx->ev[0], ctx->ev[2]);
    }
    spamm_status st = status_from_ctl(ctx, c);
    if (ctx->last_status != SPAMM_OK && st == SPAMM_OK) st = (spamm_status)ctx->last_status;
    out->status = st;
    return st;
}

// spamm_triples and spamm_triples_hi: the tile-compressed steps expanded
// into (I, K, J) rows, all kept triples or (hi, with the precision tier) the
// full-split ones.
static spamm_status expand_triples(spamm_ctx* ctx, int32_t* host_out, int64_t cap,
                                   int64_t* count, bool hi) {
    if (!ctx || !count || cap < 0 || (cap > 0 && !host_out)) return SPAMM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "triples");
    if (ctx->last_batch > 0)
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "the last multiply was batched");
    const DevCtl& c = *ctx->ctl_host;
    const int d = ctx->last_d;
    const int64_t m = (int64_t)c.tier_count[d];
    const int SL = slices_of(ctx, ctx->last_b);
    const bool tier = hi && ctx->cfg.tier_bits > 0;
    *count = tier ? (int64_t)c.hi_products : m;
    if (c.status & (ST_OVERFLOW | ST_NONFINITE)) {
        *count = 0;
        return status_from_ctl_pub(ctx, c);
    }
    if ((cap <= 0 && SL == 1) || *count == 0) return SPAMM_OK;
    // expand the tile-compressed steps (K, mask) into (I, K, J) rows; with the
    // sub-leaf cull, a leaf triple is listed if any of its k-slices is kept
    // (the count is then exact only after the expansion)
    const int64_t tiles = ctx->last_tiles;
    const int tc = ctx->last_tc;
    const int tl = kTileRows / ctx->last_b;
    // the fused small path lists every tile's steps in a slot per leaf column
    const uint64_t msteps = ctx->last_small ? (uint64_t)tiles * ((uint64_t)1 << ctx->last_d)
                                            : (uint64_t)c.tier_count[ctx->last_tt] * ctx->last_S;
    std::vector<uint32_t> off((size_t)tiles + 1), nst((size_t)tiles), pk((size_t)msteps);
    std::vector<uint64_t> pm((size_t)(2 * msteps * SL));
    e = cudaMemcpy(off.data(), ctx->tile_off, sizeof(uint32_t) * (tiles + 1), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(nst.data(), ctx->tile_steps, sizeof(uint32_t) * tiles, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && msteps)
        e = cudaMemcpy(pk.data(), reinterpret_cast<uint32_t*>(ctx->pool + c.pk_off),
                       sizeof(uint32_t) * msteps, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && msteps)
        e = cudaMemcpy(pm.data(), ctx->pool + c.pm_off, sizeof(uint64_t) * 2 * msteps * SL,
                       cudaMemcpyDeviceToHost);
    std::vector<uint64_t> ph(tier ? (size_t)(2 * msteps) : 0);
    if (e == cudaSuccess && msteps && tier)
        e = cudaMemcpy(ph.data(), ctx->pool + c.ph_off, sizeof(uint64_t) * 2 * msteps,
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(ctx, e, "triples copy");
    int64_t k = 0;
    for (int64_t u = 0; u < tiles; ++u) {
        const uint64_t base = (uint64_t)off[u] * ctx->last_S;
        for (uint32_t q = 0; q < nst[u]; ++q) {
            for (int h = 0; h < kTileHalves; ++h) {
                uint64_t mk = 0;
                for (int sl = 0; sl < SL; ++sl) mk |= pm[2 * ((base + q) * SL + sl) + h];
                if (tier) mk &= ph[2 * (base + q) + h];
                while (mk) {
                    const int bit = __builtin_ctzll(mk);
                    mk &= mk - 1;
                    if (k < cap) {
                        host_out[3 * k + 0] = (int32_t)((u / tc) * tl + (bit & 7));
                        host_out[3 * k + 1] = (int32_t)pk[base + q];
                        host_out[3 * k + 2] =
                            (int32_t)(((u % tc) * kTileHalves + h) * tl + (bit >> 3));
                    }
                    ++k;
                }
            }
        }
    }
    *count = k;
    return SPAMM_OK;
}

spamm_status spamm_triples(spamm_ctx* ctx, int32_t* host_out, int64_t cap, int64_t* count) {
    return expand_triples(ctx, host_out, cap, count, false);
}

spamm_status spamm_triples_hi(spamm_ctx* ctx, int32_t* host_out, int64_t cap, int64_t* count) {
    return expand_triples(ctx, host_out, cap, count, true);
}

spamm_status spamm_cull_flat(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B,
                             double tau, int32_t* host_out, int64_t cap, int64_t* count,
                             float* ms) {
    if (!ctx || !A || !B || !count || cap < 0 || (cap > 0 && !host_out))
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "NULL argument");
    if (!(tau >= 0.0) || !std::isfinite(tau))
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "tau must be finite and >= 0");
    if (A->n != B->n || A->b != B->b || A->precision != B->precision ||
        A->precision != ctx->cfg.precision || A->b != ctx->cfg.leaf)
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "trees differ from the configuration");
    if (A->nl > flat_max_leaves())
        return set_err(ctx, SPAMM_ERR_UNSUPPORTED, "flat enumeration: more than 2048 leaves per side");
    *count = 0;
    double roots[2];
    cudaError_t e = cudaMemcpyAsync(&roots[0], A->pyr, sizeof(double), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&roots[1], B->pyr, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "flat enumeration");
    if (!std::isfinite(roots[0]) || !std::isfinite(roots[1]))
        return set_err(ctx, SPAMM_ERR_NONFINITE, "an operand holds Inf or NaN");
    void* scratch = nullptr;
    unsigned long long* total = nullptr;
    uint64_t* out = nullptr;
    e = cudaMalloc(&scratch, flat_scratch_bytes(A->nl));
    if (e == cudaSuccess) e = cudaMalloc(&total, sizeof(unsigned long long));
    const unsigned long long dcap = (unsigned long long)cap;
    if (e == cudaSuccess && dcap) e = cudaMalloc(&out, sizeof(uint64_t) * dcap);
    unsigned long long htotal = 0;
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[0], ctx->stream);
    if (e == cudaSuccess) e = launch_cull_flat(ctx, A, B, tau, out, dcap, scratch, total);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[1], ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&htotal, total, sizeof(htotal), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && ms) e = cudaEventElapsedTime(ms, ctx->ev[0], ctx->ev[1]);
    std::vector<uint64_t> h;
    const unsigned long long got = std::min<unsigned long long>(htotal, dcap);
    if (e == cudaSuccess && got) {
        h.resize((size_t)got);
        e = cudaMemcpy(h.data(), out, sizeof(uint64_t) * got, cudaMemcpyDeviceToHost);
    }
    cudaFree(out);
    cudaFree(total);
    cudaFree(scratch);
    if (e != cudaSuccess) return cuda_err(ctx, e, "flat enumeration");
    // (I, J, K) order, as the tile-grouped list is read row by row
    std::sort(h.begin(), h.end(), [](uint64_t x, uint64_t y) {
        const uint64_t kx = ((uint64_t)tri_I(x) << 42) | ((uint64_t)tri_J(x) << 21) | tri_K(x);
        const uint64_t ky = ((uint64_t)tri_I(y) << 42) | ((uint64_t)tri_J(y) << 21) | tri_K(y);
        return kx < ky;
    });
    for (size_t q = 0; q < h.size(); ++q) {
        host_out[3 * q + 0] = (int32_t)tri_I(h[q]);
        host_out[3 * q + 1] = (int32_t)tri_K(h[q]);
        host_out[3 * q + 2] = (int32_t)tri_J(h[q]);
    }
    *count = (int64_t)htotal;
    return SPAMM_OK;
}

static spamm_status status_of(spamm_ctx* ctx, const DevCtl& c) { return status_from_ctl(ctx, c); }

static spamm_status ensure_aux(spamm_ctx* ctx) {
    if (ctx->aux_ready) return SPAMM_OK;
    cudaError_t e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
    int made = 0;
    for (; made < spamm_ctx::kAux && e == cudaSuccess; ++made) {
        e = cudaStreamCreateWithFlags(&ctx->aux[made], cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&ctx->aux_ev[made], cudaEventDisableTiming);
        if (e != cudaSuccess) break;
    }
    int lo_prio = 0, hi_prio = 0;
    bool hi_made = false;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->hi, cudaStreamNonBlocking, hi_prio);
    if (e == cudaSuccess) {
        hi_made = true;
        e = cudaEventCreateWithFlags(&ctx->hi_ev, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        for (int i = 0; i < made; ++i) {
            cudaStreamDestroy(ctx->aux[i]);
            cudaEventDestroy(ctx->aux_ev[i]);
        }
        if (hi_made) cudaStreamDestroy(ctx->hi);
        cudaEventDestroy(ctx->fork_ev);
        return cuda_err(ctx, e, "side streams");
    }
    ctx->aux_ready = true;
    return SPAMM_OK;
}

// Fork: every side stream waits for the work queued so far on ctx->stream.
static cudaError_t fork_aux(spamm_ctx* ctx) {
    cudaError_t e = cudaEventRecord(ctx->fork_ev, ctx->stream);
    for (int i = 0; i < spamm_ctx::kAux && e == cudaSuccess; ++i)
        e = cudaStreamWaitEvent(ctx->aux[i], ctx->fork_ev, 0);
    return e;
}

// Join: ctx->stream waits for everything queued on the side streams.
static cudaError_t join_aux(spamm_ctx* ctx) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < spamm_ctx::kAux && e == cudaSuccess; ++i) {
        e = cudaEventRecord(ctx->aux_ev[i], ctx->aux[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->aux_ev[i], 0);
    }
    return e;
}

static void note_shape(spamm_ctx* c, const spamm_tree* A, double tau) {
    c->last_batch = 0;
    c->last_d = A->d;
    c->last_b = A->b;
    c->last_n = A->n;
    c->last_prec = A->precision;
    c->last_tau = tau;
    c->last_tiles = (int64_t)tile_rows(A) * tile_cols(A);
    c->last_tr = tile_rows(A);
    c->last_tc = tile_cols(A);
    c->last_tt = tile_tier(A);
    c->last_S = 1 << (A->d - c->last_tt);
    c->last_status = SPAMM_OK;
}

spamm_status spamm_tree_rebuild_batched(spamm_ctx* ctx, int32_t count, spamm_tree* const* trees,
                                        const float* const* A, const int64_t* lda) {
    if (!ctx || count < 0 || (count > 0 && (!trees || !A || !lda)))
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "NULL argument");
    if (count == 0) return SPAMM_OK;
    for (int p = 0; p < count; ++p) {
        spamm_tree* t = trees[p];
        if (!t) return set_err(ctx, SPAMM_ERR_INVALID_ARG, "NULL tree");
        if (t->sparse)
            return set_err(ctx, SPAMM_ERR_UNSUPPORTED, "a sparsified tree is rebuilt by spamm_sparsify");
        const spamm_status st = check_matrix(ctx, A[p], t->n, lda[p]);
        if (st != SPAMM_OK) return st;
        if (t->precision != ctx->cfg.precision || t->b != ctx->cfg.leaf)
            return set_err(ctx, SPAMM_ERR_INVALID_ARG, "tree built under another configuration");
    }
    spamm_status st = ensure_aux(ctx);
    if (st != SPAMM_OK) return st;
    cudaError_t e = fork_aux(ctx);
    for (int p = 0; p < count && e == cudaSuccess; ++p) {
        spamm_tree* t = trees[p];
        t->A = A[p];
        t->lda = lda[p];
        e = launch_build_norms(t, ctx->aux[p % spamm_ctx::kAux]);
    }
    if (e == cudaSuccess) e = join_aux(ctx);
    return cuda_err(ctx, e, "batched norm build launch");
}

spamm_status spamm_multiply_batched(spamm_ctx* ctx, int32_t count, const spamm_tree* const* A,
                                    const spamm_tree* const* B, const double* tau,
                                    const float* alpha, const float* beta, float* const* C,
                                    const int64_t* ldc) {
    if (!ctx || count < 0 || (count > 0 && (!A || !B || !tau || !alpha || !beta || !C || !ldc)))
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "NULL argument");
    if (count == 0) return SPAMM_OK;
    for (int p = 0; p < count; ++p) {
        if (!A[p] || !B[p] || !C[p]) return set_err(ctx, SPAMM_ERR_INVALID_ARG, "NULL argument");
        if (!(tau[p] >= 0.0) || !std::isfinite(tau[p]))
            return set_err(ctx, SPAMM_ERR_INVALID_ARG, "tau must be finite and >= 0");
        if (A[p]->n != B[p]->n || A[p]->b != B[p]->b || A[p]->precision != B[p]->precision ||
            A[p]->precision != ctx->cfg.precision || A[p]->b != ctx->cfg.leaf)
            return set_err(ctx, SPAMM_ERR_INVALID_ARG, "trees differ from the configuration");
        if (ldc[p] < A[p]->n) return set_err(ctx, SPAMM_ERR_INVALID_ARG, "ldc below n");
    }
    // sub-contexts
    while ((int)ctx->subs.size() < count) {
        spamm_config c = ctx->cfg;
        c.checked = 0;
        if (!c.pool_bytes) c.pool_bytes = (int64_t)64 << 20;
        spamm_ctx* sub = nullptr;
        const spamm_status st = spamm_create(&sub, ctx->stream, &c);
        if (st != SPAMM_OK) return set_err(ctx, st, "sub-context creation");
        ctx->subs.push_back(sub);
    }
    spamm_status sta = ensure_aux(ctx);
    if (sta == SPAMM_OK && ctx->bctl_cap < count) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->bctl);
        if (ctx->bctl_host) cudaFreeHost(ctx->bctl_host);
        ctx->bctl = nullptr;
        ctx->bctl_host = nullptr;
        ctx->bctl_cap = 0;
        cudaError_t e = cudaMalloc(&ctx->bctl, sizeof(DevCtl) * (size_t)count);
        if (e == cudaSuccess) e = cudaMallocHost(&ctx->bctl_host, sizeof(DevCtl) * (size_t)count);
        if (e != cudaSuccess) return cuda_err(ctx, e, "batch control blocks");
        ctx->bctl_cap = count;
    }
    if (sta != SPAMM_OK) return sta;
    for (int p = 0; p < count; ++p) {
        spamm_ctx* sub = ctx->subs[p];
        sub->stream = ctx->aux[p % spamm_ctx::kAux];
        spamm_status st = ensure_tiles(sub, (int64_t)tile_rows(A[p]) * tile_cols(A[p]));
        if (st == SPAMM_OK) st = ensure_need(sub, A[p]->nb);
        if (st != SPAMM_OK) return st;
        note_shape(sub, A[p], tau[p]);
    }
    ctx->last_batch = count;
    ctx->last_status = SPAMM_OK;
    std::vector<LeafJob> jobs((size_t)count);
    for (int p = 0; p < count; ++p)
        jobs[p] = LeafJob{A[p], B[p], ctx->subs[p], alpha[p], beta[p], C[p], ldc[p]};
    const bool tc = precision_uses_tc(ctx->cfg.precision);
    for (int attempt = 0;; ++attempt) {
        cudaStream_t s = ctx->stream;
        cudaError_t e = cudaMemsetAsync(ctx->ctl, 0, sizeof(DevCtl), s);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[0], s);
        if (e == cudaSuccess) e = launch_ctl_batch(ctx->subs.data(), count, nullptr, s);
        // the packs depend on the norms alone: side streams, beside the culls
        if (e == cudaSuccess && tc) {
            e = fork_aux(ctx);
            for (int p = 0; p < count && e == cudaSuccess; ++p)
                e = launch_packs(ctx->subs[p]->ctl, A[p], B[p], tau[p], ctx->cfg.tie_rel,
                                 ctx->subs[p]->need,
                                 ctx->sm_count, ctx->subs[p]->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->hi, ctx->fork_ev, 0);
        }
        // stages 2-3 of all products: one launch per tier and grouping step,
        // on the high-priority side stream when packs run beside them
        if (e == cudaSuccess)
            e = launch_symbolic_batched(ctx, ctx->subs.data(), A, B, tau, count,
                                        tc ? ctx->hi : s);
        if (e == cudaSuccess && tc) {
            e = cudaEventRecord(ctx->hi_ev, ctx->hi);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->hi_ev, 0);
            if (e == cudaSuccess) e = join_aux(ctx);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[1], s);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[3], s);
        if (e == cudaSuccess) {
            if (tc) {
                // tensor-core leaf products of all products: one persistent launch
                e = launch_leaf_tc_jobs(ctx, jobs.data(), count);
            } else {
                // FP32 leaf products: one launch per product, on the side streams
                e = fork_aux(ctx);
                for (int p = 0; p < count && e == cudaSuccess; ++p) {
                    spamm_ctx* sub = ctx->subs[p];
                    e = launch_leaf_simt(sub, A[p], B[p], alpha[p], beta[p], C[p], ldc[p]);
                }
                if (e == cudaSuccess) e = join_aux(ctx);
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[2], s);
        if (e == cudaSuccess) e = launch_ctl_batch(ctx->subs.data(), count, ctx->bctl, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->bctl_host, ctx->bctl, sizeof(DevCtl) * (size_t)count,
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s);
        ctx->timed = (e == cudaSuccess);
        if (e != cudaSuccess)
            return (spamm_status)(ctx->last_status = cuda_err(ctx, e, "batched multiply launch"));
        if (!ctx->cfg.checked) return SPAMM_OK;
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return (spamm_status)(ctx->last_status = cuda_err(ctx, e, "batched multiply"));
        bool retry = false;
        for (int p = 0; p < count; ++p) {
            spamm_ctx* sub = ctx->subs[p];
            const DevCtl& c = ctx->bctl_host[p];
            if (c.status & (ST_NONFINITE | ST_TIMEOUT))
                return (spamm_status)(ctx->last_status = status_of(ctx, c));
            if (c.status & ST_OVERFLOW) {
                const int64_t need = std::max<int64_t>(words_needed(c, sub->last_tt, sub->last_S, mask_pairs_of(sub, sub->last_b)),
                                                       2 * sub->pool_words);
                const spamm_status st = alloc_pool(sub, need * 8 + need * 2);
                if (st != SPAMM_OK) return (spamm_status)(ctx->last_status = st);
                retry = true;
            }
        }
        const spamm_status st = status_of(ctx, *ctx->ctl_host);
        if (st != SPAMM_OK) return (spamm_status)(ctx->last_status = st);
        if (retry && attempt < 8) continue;
        if (retry) return (spamm_status)(ctx->last_status = set_err(ctx, SPAMM_ERR_CAPACITY, "pool"));
        return SPAMM_OK;
    }
}

spamm_status spamm_stats_item(spamm_ctx* ctx, int32_t index, spamm_stats_t* out) {
    if (!ctx || !out) return SPAMM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "stats");
    if (index < 0 || index >= ctx->last_batch)
        return set_err(ctx, SPAMM_ERR_INVALID_ARG, "no such product in the last batch");
    memset(out, 0, sizeof(*out));
    spamm_ctx* sub = ctx->subs[index];
    const DevCtl& c = ctx->bctl_host[index];
    const int d = sub->last_d;
    out->depth = d;
    out->n = sub->last_n;
    out->leaf = sub->last_b;
    out->precision = sub->last_prec;
    out->tau = sub->last_tau;
    for (int t = 0; t <= d && t < SPAMM_MAX_TIERS; ++t) {
        out->tier_candidates[t] = (int64_t)c.tier_cand[t];
        out->tier_kept[t] = (int64_t)c.tier_count[t];
    }
    out->leaf_triples = (int64_t)c.tier_count[d];
    out->tie_band = (int64_t)c.tie_band;
    out->active_steps = (int64_t)c.active_steps;
    out->tiles = sub->last_tiles;
    const double b = sub->last_b;
    out->kept_flops = 2.0 * b * b * b * (double)out->leaf_triples;
    out->slice = sub->cfg.slice;
    out->slice_kept = (int64_t)c.slice_kept;
    out->slice_tested = (int64_t)c.slice_tested;
    out->packed_leaves_a = (int64_t)c.packed_a;
    out->packed_leaves_b = (int64_t)c.packed_b;
    if (sub->cfg.slice) out->kept_flops = 2.0 * b * b * sub->cfg.slice * (double)c.slice_kept;
    fill_tier_stats(sub, c, out->leaf_triples, out);
    out->dense_flops = 2.0 * (double)sub->last_n * (double)sub->last_n * (double)sub->last_n;
    out->pool_bytes = sub->pool_words * 8;
    out->pool_needed_bytes = words_needed(c, sub->last_tt, sub->last_S, mask_pairs_of(sub, sub->last_b)) * 8;
    out->status = status_of(ctx, c);
    return (spamm_status)out->status;
}

static spamm_status batch_stats(spamm_ctx* ctx, spamm_stats_t* out) {
    memset(out, 0, sizeof(*out));
    spamm_status worst = status_of(ctx, *ctx->ctl_host);
    for (int p = 0; p < ctx->last_batch && p < (int)ctx->subs.size(); ++p) {
        spamm_ctx* sub = ctx->subs[p];
        const DevCtl& c = ctx->bctl_host[p];
        const int d = sub->last_d;
        for (int t = 0; t <= d && t < SPAMM_MAX_TIERS; ++t) {
            out->tier_candidates[t] += (int64_t)c.tier_cand[t];
            out->tier_kept[t] += (int64_t)c.tier_count[t];
        }
        out->depth = std::max<int32_t>(out->depth, d);
        out->n = std::max<int64_t>(out->n, sub->last_n);
        const int64_t m = (int64_t)c.tier_count[d];
        out->leaf_triples += m;
        out->tie_band += (int64_t)c.tie_band;
        out->active_steps += (int64_t)c.active_steps;
        out->tiles += sub->last_tiles;
        const double b = sub->last_b;
        out->kept_flops += sub->cfg.slice ? 2.0 * b * b * sub->cfg.slice * (double)c.slice_kept
                                          : 2.0 * b * b * b * (double)m;
        out->slice = sub->cfg.slice;
        out->slice_kept += (int64_t)c.slice_kept;
        out->slice_tested += (int64_t)c.slice_tested;
        out->packed_leaves_a += (int64_t)c.packed_a;
        out->packed_leaves_b += (int64_t)c.packed_b;
        spamm_stats_t one{};
        fill_tier_stats(sub, c, m, &one);
        out->hi_products += one.hi_products;
        out->tie_band_hi += one.tie_band_hi;
        out->kept_flops_clipped += one.kept_flops_clipped;
        out->dense_flops += 2.0 * (double)sub->last_n * (double)sub->last_n * (double)sub->last_n;
        out->pool_bytes += sub->pool_words * 8;
        out->pool_needed_bytes += words_needed(c, sub->last_tt, sub->last_S, mask_pairs_of(sub, sub->last_b)) * 8;
        const spamm_status st = status_of(ctx, c);
        if (worst == SPAMM_OK) worst = st;
    }
    out->leaf = ctx->cfg.leaf;
    out->precision = ctx->cfg.precision;
    if (ctx->timed) {
        cudaEventElapsedTime(&out->ms_symbolic, ctx->ev[0], ctx->ev[1]);
        cudaEventElapsedTime(&out->ms_pack, ctx->ev[1], ctx->ev[3]);
        cudaEventElapsedTime(&out->ms_numeric, ctx->ev[3], ctx->ev[2]);
        cudaEventElapsedTime(&out->ms_total, ctx->ev[0], ctx->ev[2]);
    }
    if (ctx->last_status != SPAMM_OK && worst == SPAMM_OK) worst = (spamm_status)ctx->last_status;
    out->status = worst;
    return worst;
}

spamm_status spamm_multiply_host(spamm_ctx* ctx, const float* A, const float* B, int64_t n,
                                 double tau, float alpha, float beta, float* C) {
    if (!ctx || !A || !C || n <= 0) return set_err(ctx, SPAMM_ERR_INVALID_ARG, "bad argument");
    const bool square = (B == nullptr || B == A);
    const int64_t elems = n * n;
    if (elems > ctx->stage_elems) {
        cudaStreamSynchronize(ctx->stream);
        if (ctx->hostTreeA) spamm_tree_destroy(ctx->hostTreeA);
        if (ctx->hostTreeB) spamm_tree_destroy(ctx->hostTreeB);
        ctx->hostTreeA = ctx->hostTreeB = nullptr;
        cudaFree(ctx->dA);
        cudaFree(ctx->dB);
        cudaFree(ctx->dC);
        ctx->dA = ctx->dB = ctx->dC = nullptr;
        ctx->stage_elems = 0;
        cudaError_t e = cudaMalloc(&ctx->dA, sizeof(float) * elems);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->dB, sizeof(float) * elems);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->dC, sizeof(float) * elems);
        if (e != cudaSuccess) return cuda_err(ctx, e, "staging allocation");
        ctx->stage_elems = elems;
    }
    cudaStream_t s = ctx->stream;
    const size_t bytes = sizeof(float) * elems;
    cudaError_t e = cudaMemcpyAsync(ctx->dA, A, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !square) e = cudaMemcpyAsync(ctx->dB, B, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && beta != 0.f) e = cudaMemcpyAsync(ctx->dC, C, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "host to device copy");
    spamm_status st;
    auto tree_for = [&](spamm_tree** slot, const float* dev) -> spamm_status {
        if (*slot && ((*slot)->n != n || (*slot)->precision != ctx->cfg.precision ||
                      (*slot)->b != ctx->cfg.leaf)) {
            spamm_tree_destroy(*slot);
            *slot = nullptr;
        }
        if (*slot) return spamm_tree_rebuild(ctx, *slot, dev, n);
        return spamm_build_norms(ctx, dev, n, n, slot);
    };
    st = tree_for(&ctx->hostTreeA, ctx->dA);
    if (st != SPAMM_OK) return st;
    const spamm_tree* tb = ctx->hostTreeA;
    if (!square) {
        st = tree_for(&ctx->hostTreeB, ctx->dB);
        if (st != SPAMM_OK) return st;
        tb = ctx->hostTreeB;
    }
    // tensor-core path: C leaves in up to eight bands of whole tile-row
    // groups, each copied out (aux[0]) while the later bands compute (the
    // bands themselves overlap on two streams); the FP32 path copies it after
    // the fact
    const bool banded = precision_uses_tc(ctx->cfg.precision);
    if (banded) {
        st = ensure_aux(ctx);
        if (st != SPAMM_OK) return st;
        ctx->band_host = C;
        ctx->band_count = 8;
    }
    st = spamm_multiply(ctx, ctx->hostTreeA, tb, tau, alpha, beta, ctx->dC, n);
    ctx->band_host = nullptr;
    ctx->band_count = 0;
    if (st != SPAMM_OK) {
        if (banded) cudaStreamSynchronize(ctx->aux[0]);
        return st;
    }
    if (banded) {
        e = cudaEventRecord(ctx->aux_ev[1], ctx->aux[0]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->aux_ev[1], 0);
    } else {
        e = cudaMemcpyAsync(C, ctx->dC, bytes, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "device to host copy");
    return status_from_ctl(ctx, *ctx->ctl_host);
}

}  // extern "C"
