// Internal declarations shared by the CUDA translation units of the engine.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <string>
#include <vector>

#include "../../include/spamm.h"

namespace spamm {

// Triples (I, K, J) at tier t are packed into 64 bits, 21 bits per index.
constexpr int kIdxBits = 21;
constexpr uint64_t kIdxMask = (1ull << kIdxBits) - 1;
__host__ __device__ inline uint64_t pack_triple(uint64_t I, uint64_t K, uint64_t J) {
    return (I << (2 * kIdxBits)) | (K << kIdxBits) | J;
}
__host__ __device__ inline uint32_t tri_I(uint64_t p) { return (uint32_t)(p >> (2 * kIdxBits)); }
__host__ __device__ inline uint32_t tri_K(uint64_t p) { return (uint32_t)((p >> kIdxBits) & kIdxMask); }
__host__ __device__ inline uint32_t tri_J(uint64_t p) { return (uint32_t)(p & kIdxMask); }

// A C tile is 128 rows x 256 columns: TL = 128 / b row leaves and 2 TL
// column leaves, i.e. one quadtree node of TL x TL leaves (tier tt) and its
// right-hand neighbour.  Each grouped (tile, K) step carries two 64-bit
// masks, one per half (node); bit (y * 8 + x) = "the product of row leaf x
// and column leaf y of that half is kept" (only TL x TL bits are used).
constexpr int kTileRows = 128;
constexpr int kTileHalves = 2;
constexpr int kMaxLeavesPerSide = 1 << 14;

// Chunks per pack group: the pieces of a leaf's 16-wide K-chunks are stored
// in groups of this many chunks, the high parts of a group before its low
// parts (norms.cu), so that the K-chunks one leaf-kernel stage holds (four
// for 16-bit parts and single TF32, one for TF32 hi + lo) are one contiguous
// run per part.  At most the chunks of a leaf (b / 16).
__host__ __device__ constexpr int pack_group_chunks(int leaf, int precision) {
    return precision == SPAMM_PREC_TF32X3 ? 1 : (leaf / 16 < 4 ? leaf / 16 : 4);
}

// Device status bits.
constexpr uint32_t ST_OVERFLOW = 1u;
constexpr uint32_t ST_NONFINITE = 2u;
constexpr uint32_t ST_TIMEOUT = 4u;

// Control block in device memory, zeroed before every multiply.  All pool
// offsets are in 8-byte words.
struct DevCtl {
    unsigned long long tier_count[SPAMM_MAX_TIERS];  // true kept count per tier
    unsigned long long tier_cand[SPAMM_MAX_TIERS];
    unsigned long long tier_off[SPAMM_MAX_TIERS + 1];
    unsigned long long tie_band;
    unsigned long long active_steps;
    unsigned long long ent_off;     // u32 K of each tier-tt triple, grouped by tile
    unsigned long long pk_off;      // u32 K of each (tile, K) step
    unsigned long long pm_off;      // two u64 masks (left, right half) of each step
    unsigned long long need_words;  // words the whole multiply needs
    unsigned long long slice_kept;  // kept k-slice products (sub-leaf cull)
    unsigned long long slice_tested;
    unsigned long long packed_a;    // leaves packed in the A role (needed by a kept product)
    unsigned long long packed_b;    // leaves packed in the B role
    unsigned long long ph_off;      // two u64 masks of each step: products that keep the
                                    // full split precision (precision chosen by norm)
    unsigned long long hi_products; // kept leaf products at or above tau_h
    unsigned long long tie_hi;      // kept leaf products in the tie band around tau_h
    unsigned long long clip_vol;    // sum over kept products of rows x k x columns inside
                                    // the n x n matrices
    unsigned int status;
    unsigned int tile_ctr;          // work items taken by the blocks of the running leaf launch
    unsigned int band_ctr[8];       // the same for each band of a banded leaf launch (host
                                    // entry point; the bands may run at the same time)
};

// Words stored for tier t (a frontier that overflowed is truncated).
__device__ inline unsigned long long stored_count(const DevCtl* c, int t, unsigned long long cap) {
    unsigned long long off = c->tier_off[t];
    if (off >= cap) return 0;
    unsigned long long room = cap - off;
    unsigned long long n = c->tier_count[t];
    return n < room ? n : room;
}

// Squared-form thresholds of the SpAMM condition: keep iff fl(nA2 * nB2) >=
// tau2 (FP64) with both norms non-zero; the tie band is [lo2, hi2].
struct Thresh {
    double tau2, lo2, hi2;
    int e_lo, e_hi;  // biased FP64 exponents of lo2 and hi2
};

// FP16 split precision: an operand is scaled by 2^k so that its largest leaf
// norm (an upper bound of every element) lands just below 2^15, inside the
// fp16 range; k from the largest squared leaf norm.  Scaling by a power of
// two is exact, and the product is scaled back by 2^-(kA + kB).  FP32 leaf
// norms stay below 2^136, so k >= -120; k is capped at 126 so that 2^k and
// 2^-k are normal floats (an operand whose largest leaf norm is below
// 2^-111 is then scaled less than fully, into fp16's subnormal range).
// Integer work only (the FP64 pipe is narrow): with gmax2 in [2^E, 2^(E+1)),
// the largest leaf norm sqrt(gmax2) lies below 2^e for e = floor(E/2) + 1.
__device__ inline int f16_scale_exp(double gmax2) {
    if (!(gmax2 > 0.0)) return 0;
    const long long bits = __double_as_longlong(gmax2);
    const int E = (int)((bits >> 52) & 0x7FF) - 1023;   // subnormals: -1023
    const int e = (E >> 1) + 1;
    const int k = 15 - e;
    return k < -126 ? -126 : (k > 126 ? 126 : k);
}

// The unscale 2^-(kA + kB) as two normal floats whose product it is
// (kA + kB lies in [-252, 252], beyond one float's exponent range).
__device__ inline float2 f16_unscale(double gmax2_a, double gmax2_b) {
    const int s = f16_scale_exp(gmax2_a) + f16_scale_exp(gmax2_b);
    const int h = s / 2;
    return make_float2(ldexpf(1.f, -h), ldexpf(1.f, -(s - h)));
}

// Exact keep decision for finite non-negative squared norms a, b, and the
// tie-band flag.  On GB300 the FP64 pipe is narrow, so the exponent fields
// settle every pair whose product lies clearly outside [lo2, hi2] with
// integer operations: 2^(s-1023) <= a*b < 2^(s+1-1023+1) for s = ea + eb -
// 1023.  Only products within a factor of about four of the band are formed
// in FP64, exactly as the oracle forms them.
__device__ __forceinline__ bool spamm_keep(double a, double b, const Thresh& th, bool* tie) {
    const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
    const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
    *tie = false;
    if (ua == 0ull || ub == 0ull) return false;  // a NULL block never multiplies
    const int s = (int)(ua >> 52) + (int)(ub >> 52) - 1023;
    if (s >= 1 && s >= th.e_hi + 1) return true;  // fl(a*b) >= 2^(s-1023) > hi2 >= tau2
    if (s + 2 < th.e_lo) return false;            // fl(a*b) <= 2^(s+2-1023) < lo2 <= tau2
    const double p = a * b;
    *tie = p >= th.lo2 && p <= th.hi2;
    return p >= th.tau2;
}

inline Thresh make_thresh(double tau, double rel) {
    Thresh t;
    t.tau2 = tau * tau;
    t.lo2 = t.tau2 * (1.0 - rel) * (1.0 - rel);
    t.hi2 = t.tau2 * (1.0 + rel) * (1.0 + rel);
    unsigned long long ul, uh;
    static_assert(sizeof(double) == 8, "");
    memcpy(&ul, &t.lo2, 8);
    memcpy(&uh, &t.hi2, 8);
    t.e_lo = (int)(ul >> 52);
    t.e_hi = (int)(uh >> 52);
    return t;
}

}  // namespace spamm

struct spamm_tree {
    spamm_ctx* ctx;
    const float* A;
    int64_t n, lda;
    int b, d;
    int64_t nb;        // 2^d leaves per side (padded grid)
    int64_t nl;        // ceil(n / b) leaves holding data
    int64_t nlp;       // nl rounded up to whole tile widths (2 TL leaves)
    double* pyr;       // squared norms, all tiers
    int64_t nodes;
    int precision;
    // Tensor-core operand tiles, see norms.cu for the layout.  A-role tiles
    // hold leaf (I,K) rows = i; B-role tiles hold leaf (K,J) transposed.
    void* packA[2];    // hi, lo (lo only for split precisions)
    void* packB[2];
    size_t pack_bytes;  // bytes of one pack array
    // sub-leaf cull along k: slices of 16 per leaf (b / 16) and the panel
    // squared norms, A role [I][K][s] (rows of leaf I, columns of slice s of
    // leaf K) and B role [K][s][J] (rows of slice s of leaf K, columns of
    // leaf J), nl leaves per side; null when the cull is off
    int slices;
    double* panA;
    double* panB;
    // sparsified storage (spamm_sparsify): leaf row I keeps the columns of
    // its band of leaves [kmin, kmax] as an FP32 slab (dropped leaves zero),
    // and the packs hold pieces only inside the bands: A role per leaf
    // column K over [imin, imax], B role per leaf row K over [kmin, kmax].
    // Zero for dense trees.
    int sparse;
    float* slab;
    int32_t* band;      // kmin, kmax, imin, imax: 4 x nl (device)
    int64_t* offs;      // roff (nl), aoff (nl + 1), boff (nl + 1) (device)
    int64_t stored;     // leaves kept
    int64_t bytes;      // device bytes the tree holds
    // re-sparsify in place (spamm_sparsify_into): the new bands land in
    // band_new until they are known to fit, the mark kernel's kept count and
    // dense root in sdev[0..1]; pinned host copies of bands and offsets; the
    // capacities of slab (floats) and of each pack array (bytes)
    int32_t* band_new;
    unsigned long long* sdev;
    int32_t* h_band;    // 4 x nl, then the two words of sdev
    int64_t* h_offs;    // 3 nl + 2
    int64_t slab_cap, packa_cap, packb_cap;
};

// Device view of a sparsified tree's bands (see spamm_tree).
struct BandView {
    const float* slab;
    const int32_t* kmin;
    const int32_t* kmax;
    const int32_t* imin;
    const int32_t* imax;
    const int64_t* roff;   // slab element offset of leaf row I
    const int64_t* aoff;   // first A-role piece of leaf column K
    const int64_t* boff;   // first B-role piece of leaf row K
};

inline BandView band_view(const spamm_tree* t) {
    BandView v{};
    if (!t->sparse) return v;
    const int64_t nl = t->nl;
    v.slab = t->slab;
    v.kmin = t->band;
    v.kmax = t->band + nl;
    v.imin = t->band + 2 * nl;
    v.imax = t->band + 3 * nl;
    v.roff = t->offs;
    v.aoff = t->offs + nl;
    v.boff = t->offs + 2 * nl + 1;
    return v;
}

struct spamm_ctx {
    cudaStream_t stream;
    spamm_config cfg;
    int device;
    int sm_count;
    // triple pool
    uint64_t* pool;
    int64_t pool_words;
    // control block (device) and its pinned mirror
    spamm::DevCtl* ctl;
    spamm::DevCtl* ctl_host;
    // per-tile arrays
    uint32_t* tile_cnt;   // entries per tile, then fill cursors
    uint32_t* tile_fill;
    uint32_t* tile_off;   // exclusive scan, tiles + 1
    uint32_t* tile_steps; // (tile, K) steps per tile
    uint32_t* tile_iters; // K-chunk iterations per tile (steps x chunks kept)
    uint32_t* work_ctr;   // persistent-kernel work counter
    int64_t tiles_cap;
    // per-K norm maxima for the packs of a multiply (2 x leaves per side)
    double* need;
    int64_t need_cap;
    // timing
    cudaEvent_t ev[4];
    bool timed;
    // last multiply
    int last_d, last_b, last_prec, last_tt, last_S, last_tr, last_tc;
    int64_t last_n, last_tiles;
    double last_tau;
    int last_status;
    // host staging for spamm_multiply_host
    float* dA; float* dB; float* dC;
    int64_t stage_elems;
    spamm_tree* hostTreeA;
    spamm_tree* hostTreeB;
    // set by spamm_multiply_host around its multiply: copy the rows of C out
    // to this host array band by band, on aux[0], while later bands compute
    float* band_host;
    int band_count;
    // batched multiplies: one sub-context (pool, control block, tile arrays)
    // per product, created on demand and reused
    std::vector<spamm_ctx*> subs;
    int last_batch;  // products in the last multiply (0: a plain multiply)
    // trees built on this context: destroying the context detaches them, so
    // a tree freed later never touches the freed context
    std::vector<spamm_tree*> trees;
    // side streams for the per-product stages of batched calls (fork from
    // and join back into `stream`; inside a graph capture they become
    // parallel branches)
    static constexpr int kAux = 16;
    // gathered control blocks of the last batched multiply (device, pinned host)
    spamm::DevCtl* bctl;
    spamm::DevCtl* bctl_host;
    int bctl_cap;
    cudaStream_t aux[kAux];
    cudaEvent_t aux_ev[kAux];
    cudaEvent_t fork_ev;
    // high-priority side stream: a multiply's cull and grouping, whose small
    // latency-bound launches then go ahead of the concurrent pack kernel
    cudaStream_t hi;
    cudaEvent_t hi_ev;
    bool aux_ready;
    // bound of the leaf kernel's pipeline waits in ns (0: the default 1 s)
    int64_t wait_ns;
    // the last multiply ran the fused small-product path (its step list
    // holds one slot per tile and leaf column)
    bool last_small;
    std::string err;
};

namespace spamm {

spamm_status set_err(spamm_ctx* ctx, spamm_status st, const std::string& msg);
spamm_status cuda_err(spamm_ctx* ctx, cudaError_t e, const char* what);

int tile_rows(const spamm_tree* t);  // nlp / TL
int tile_cols(const spamm_tree* t);  // nlp / (2 TL)

// norms.cu
cudaError_t launch_build_norms(spamm_tree* t, cudaStream_t s);
bool precision_uses_tc(int precision);
size_t pack_bytes_for(int precision, int64_t nlp, int b);
int pack_arrays_for(int precision);  // 1 or 2 per role

// cull.cu
// tt = tier of the tile nodes (a tile is 128 / b leaves per side)
int tile_tier(const spamm_tree* t);
cudaError_t launch_cull(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B, double tau,
                        int tt);
cudaError_t launch_group(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B, double tau,
                         int tt);
// Stages 2-3 of `count` products in sub-contexts subs[p] (tile tier
// subs[p]->last_tt), table-driven launches of up to 64 products each.
cudaError_t launch_symbolic_batched(spamm_ctx* ctx, spamm_ctx* const* subs,
                                    const spamm_tree* const* A, const spamm_tree* const* B,
                                    const double* tau, int count, cudaStream_t stream);
// flat.cu: the flat, norm-sorted enumeration of the leaf triples (Algorithm 1)
cudaError_t launch_cull_flat(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B,
                             double tau, uint64_t* out, unsigned long long cap,
                             void* scratch, unsigned long long* total_dev);
size_t flat_scratch_bytes(int64_t nl);
int flat_max_leaves();

// Zero the control blocks of subs[0..count) (out == nullptr) or gather them
// into out[0..count).
cudaError_t launch_ctl_batch(spamm_ctx* const* subs, int count, DevCtl* out, cudaStream_t s);

// Tensor-core packs of the leaves that can take part in a kept product of
// A x B at tau (norms.cu); scratch holds 2 x (leaves per side) doubles.
cudaError_t launch_packs(DevCtl* ctl, const spamm_tree* A, const spamm_tree* B, double tau,
                         double rel, double* scratch, int sm_count, cudaStream_t s);

// Sparsification (norms.cu): drop the leaves whose product with norm2_max
// fails the SpAMM test at tau (norms and panels zeroed), then the row and
// column bands of the kept leaves (4 x nl int32: kmin, kmax, imin, imax).
cudaError_t launch_sparsify_mark(spamm_tree* t, double tau, double partner_norm2, double rel,
                                 int32_t* band, unsigned long long* out, cudaStream_t s);
// Copy the kept leaves of the dense A into the tree's slab.
cudaError_t launch_slab_copy(spamm_tree* t, const float* A, int64_t lda, cudaStream_t s);
cudaError_t launch_pyramid(spamm_tree* t, cudaStream_t s);

// leaf_simt.cu
cudaError_t launch_leaf_simt(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B,
                             float alpha, float beta, float* C, int64_t ldc);
// The fused small-product path (leaf_simt.cu): FP32 products of at most 128
// leaves per side run their cull, grouping and leaf products in one launch.
bool small_path(const spamm_ctx* ctx, const spamm_tree* A);
cudaError_t launch_small_fp32(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B, double tau,
                              float alpha, float beta, float* C, int64_t ldc);
// leaf_tc.cu
cudaError_t launch_leaf_tc(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B,
                           float alpha, float beta, float* C, int64_t ldc);
// The same product in `bands` launches of whole tile-row groups; after each,
// done(user, row0, row1) is told which rows of C are final.
// `done(user, r0, r1, s)`: rows [r0, r1) of C are final once stream s has
// passed the call.  At most 8 bands.
cudaError_t launch_leaf_tc_banded(spamm_ctx* ctx, const spamm_tree* A, const spamm_tree* B,
                                  float alpha, float beta, float* C, int64_t ldc, int bands,
                                  cudaError_t (*done)(void*, int64_t, int64_t, cudaStream_t),
                                  void* user);
// One product of a batched leaf launch: its trees, the context that ran its
// cull and grouping (pool, control block, tile arrays), and its C.
struct LeafJob {
    const spamm_tree* A;
    const spamm_tree* B;
    spamm_ctx* sub;
    float alpha, beta;
    float* C;
    int64_t ldc;
};
cudaError_t launch_leaf_tc_jobs(spamm_ctx* ctx, const LeafJob* jobs, int count);

}  // namespace spamm
