// spamm_multiply_static: the FP32 SpAMM product with every scratch buffer in
// one fixed device array, for callers that cannot allocate device memory.
//
// Who needs it: code that runs inside a host framework or plugin which owns
// all device memory through its own allocator or a hard memory cap (a
// cudaMalloc there bypasses its accounting or fails), and latency-critical
// loops that must not pay the implicit device synchronisation of
// cudaMalloc/cudaFree.  Such callers hand in their matrices and C and get
// the same kernels and the same result as spamm_build_norms + spamm_multiply
// with leaf 16 and FP32 leaf products.
//
// The scratch -- both norm quadtrees, the control block, the per-tile arrays
// and the triple pool -- lives in the file-scope array below, sized for the
// worst case (every block product kept) at n <= kStaticMaxN.  Every GPU that
// loads this library holds the array until the process exits.  In host code
// the array's name is only a host-side stand-in, so the host never passes it
// to a kernel: the first call on each device, with that device current,
// looks up its device address with cudaGetSymbolAddress and caches it.  That
// first call per device should therefore come before any stream capture.
// All calls share the array and it keeps the last call's contents; the
// control block and tile counters are cleared on the stream at the start of
// every call.  Calls whose work overlaps on the GPU (other streams, other
// host threads) race on the array: order them on one stream.
#include <cmath>
#include <mutex>

#include "spamm_internal.cuh"

namespace spamm {
namespace {

constexpr int kStaticLeaf = 16;
constexpr int64_t kStaticMaxN = 4096;
constexpr size_t kStaticBytes = (size_t)8 << 20;  // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Bytes the worst case (every triple kept) needs for an n x n product.
struct StaticPlan {
    int d, tt, S;
    int64_t nb, nl, nlp, nodes, tiles, tr, tc;
    size_t off_pyrA, off_pyrB, off_ctl, off_tiles, off_pool, pool_words, total;
};

StaticPlan plan_for(int64_t n) {
    StaticPlan p{};
    int d = 0;
    while ((int64_t)kStaticLeaf * ((int64_t)1 << d) < n) ++d;
    p.d = d;
    p.nb = (int64_t)1 << d;
    p.nl = (n + kStaticLeaf - 1) / kStaticLeaf;
    const int tl = kTileRows / kStaticLeaf;  // 8 leaves per tile half
    p.nlp = (p.nl + 2 * tl - 1) / (2 * tl) * (2 * tl);
    p.nodes = (((int64_t)1 << (2 * (d + 1))) - 1) / 3;
    p.tt = d > 3 ? d - 3 : 0;
    p.S = 1 << (d - p.tt);
    p.tr = p.nlp / tl;
    p.tc = p.nlp / (2 * tl);
    p.tiles = p.tr * p.tc;
    // worst-case pool: every frontier full, every tier-tt entry with S steps
    int64_t words = 0;
    for (int t = 0; t <= p.tt; ++t) words += (int64_t)1 << (3 * t);
    const int64_t m = (int64_t)1 << (3 * p.tt);
    const int64_t ms = m * p.S;
    words += (m + 1) / 2 + (ms + 1) / 2 + 2 * ms;
    p.pool_words = (size_t)words;
    size_t o = 0;
    p.off_pyrA = o; o = align256(o + sizeof(double) * p.nodes);
    p.off_pyrB = o; o = align256(o + sizeof(double) * p.nodes);
    p.off_ctl = o;  o = align256(o + sizeof(DevCtl));
    p.off_tiles = o; o = align256(o + sizeof(uint32_t) * (4 * p.tiles + 1));
    p.off_pool = o; o = align256(o + sizeof(uint64_t) * p.pool_words);
    p.total = o;
    return p;
}

spamm_status device_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return SPAMM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return SPAMM_ERR_CUDA;
        }
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return SPAMM_OK;
}

}  // namespace
}  // namespace spamm

using namespace spamm;

extern "C" spamm_status spamm_multiply_static(const float* A, int64_t lda, const float* B,
                                              int64_t ldb, int64_t n, double tau, float alpha,
                                              float beta, float* C, int64_t ldc, void* stream,
                                              uint32_t* status_dev) {
    if (!A || !B || !C || n <= 0 || lda < n || ldb < n || ldc < n) return SPAMM_ERR_INVALID_ARG;
    if (!(tau >= 0.0) || !std::isfinite(tau)) return SPAMM_ERR_INVALID_ARG;
    if (n > kStaticMaxN) return SPAMM_ERR_UNSUPPORTED;  // beyond the static scratch
    const StaticPlan p = plan_for(n);
    if (p.total > kStaticBytes) return SPAMM_ERR_UNSUPPORTED;
    void* base = nullptr;
    spamm_status st = device_scratch(&base);
    if (st != SPAMM_OK) return st;
    unsigned char* sb = static_cast<unsigned char*>(base);

    spamm_ctx ctx{};
    ctx.stream = (cudaStream_t)stream;
    spamm_config_default(&ctx.cfg);
    if (cudaGetDevice(&ctx.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx.sm_count, cudaDevAttrMultiProcessorCount, ctx.device) !=
            cudaSuccess) {
        cudaGetLastError();
        return SPAMM_ERR_CUDA;
    }
    ctx.pool = reinterpret_cast<uint64_t*>(sb + p.off_pool);
    ctx.pool_words = (int64_t)p.pool_words;
    ctx.ctl = reinterpret_cast<DevCtl*>(sb + p.off_ctl);
    uint32_t* tiles = reinterpret_cast<uint32_t*>(sb + p.off_tiles);
    ctx.tile_cnt = tiles;
    ctx.tile_fill = tiles + p.tiles;
    ctx.tile_steps = tiles + 2 * p.tiles;
    ctx.tile_off = tiles + 3 * p.tiles;
    ctx.tiles_cap = p.tiles;
    ctx.last_S = p.S;
    ctx.last_tt = p.tt;
    ctx.last_tr = (int)p.tr;
    ctx.last_tc = (int)p.tc;

    spamm_tree ta{}, tb{};
    spamm_tree* trees[2] = {&ta, &tb};
    const float* mats[2] = {A, B};
    const int64_t lds[2] = {lda, ldb};
    const size_t pyr_off[2] = {p.off_pyrA, p.off_pyrB};
    for (int i = 0; i < 2; ++i) {
        spamm_tree* t = trees[i];
        t->A = mats[i];
        t->n = n;
        t->lda = lds[i];
        t->b = kStaticLeaf;
        t->d = p.d;
        t->nb = p.nb;
        t->nl = p.nl;
        t->nlp = p.nlp;
        t->pyr = reinterpret_cast<double*>(sb + pyr_off[i]);
        t->nodes = p.nodes;
        t->precision = SPAMM_PREC_FP32;
    }
    cudaStream_t s = ctx.stream;
    cudaError_t e = launch_build_norms(&ta, s);
    if (e == cudaSuccess) e = launch_build_norms(&tb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx.ctl, 0, sizeof(DevCtl), s);
    if (e == cudaSuccess) e = launch_cull(&ctx, &ta, &tb, tau, p.tt);
    if (e == cudaSuccess) e = launch_group(&ctx, &ta, &tb, tau, p.tt);
    if (e == cudaSuccess) e = launch_leaf_simt(&ctx, &ta, &tb, alpha, beta, C, ldc);
    if (e == cudaSuccess && status_dev)
        e = cudaMemcpyAsync(status_dev, &ctx.ctl->status, sizeof(uint32_t),
                            cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SPAMM_ERR_CUDA;
    }
    return SPAMM_OK;
}
