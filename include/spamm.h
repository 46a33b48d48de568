/*
 * spamm.h -- C ABI of the GB300 SpAMM engine.
 *
 * SpAMM (Sparse Approximate Matrix Multiply, Bock & Challacombe) computes the
 * SGEMM-shaped product C = alpha * A B + beta * C (Sec. II, problem
 * statement) for matrices with decay, skipping every block product whose
 * operand norms satisfy ||A_ik||_F ||B_kj||_F < tau (Eq. (norm_condition))
 * at each tier of a quadtree of Frobenius norms (Eqs. (norm), (product)).
 *
 * The engine runs in four stages, each a CUDA kernel on one GPU:
 *   1. spamm_build_norms: leaf squared norms (FP64) and the upper tiers of the
 *      norm quadtree;
 *   2. spamm_multiply: a level-by-level cull from the root that keeps a block
 *      triple (I,K,J) iff nA2 * nB2 >= tau^2 with both norms non-zero;
 *   3. grouping of the surviving leaf triples by 128 x 256 tile of C with
 *      the kept (row-leaf, column-leaf) pairs of every K as bit masks, and,
 *      for tensor-core precisions, the leaves that can take part in a kept
 *      product repacked into tensor-core leaf tiles;
 *   4. the dense leaf products accumulated into C in ascending K.
 *
 * Conventions for every entry point:
 *   - Matrices are square n x n, FP32, row-major with leading dimension
 *     ld >= n (in elements).  Rectangular shapes are not supported.
 *   - Matrix pointers are DEVICE pointers owned by the caller, except in
 *     spamm_multiply_host, which takes HOST pointers.
 *   - Calls are asynchronous and ordered on the context's stream unless the
 *     comment says they synchronise.
 *   - Errors are returned as spamm_status; no C++ exception crosses the ABI.
 *     spamm_last_error(ctx) gives a message for the last failure on ctx.
 *   - Not thread-safe: one host thread per context at a time.
 */
#ifndef SPAMM_H_
#define SPAMM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPAMM_OK = 0,
    SPAMM_ERR_INVALID_ARG = 1,  /* bad size, stride, pointer, tau or config */
    SPAMM_ERR_NONFINITE = 2,    /* an operand holds Inf or NaN */
    SPAMM_ERR_CAPACITY = 3,     /* the triple pool overflowed; C is not valid */
    SPAMM_ERR_OOM = 4,          /* device or pinned allocation failed */
    SPAMM_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    SPAMM_ERR_UNSUPPORTED = 6,  /* valid request the engine does not support (e.g. rectangular) */
    SPAMM_ERR_CUDA = 7          /* a CUDA runtime call failed */
} spamm_status;

/* Arithmetic of the leaf products (stage 4). */
typedef enum {
    SPAMM_PREC_FP32 = 0,    /* FP32 FFMA on the CUDA cores, FP32 accumulate */
    SPAMM_PREC_TF32X3 = 1,  /* tcgen05 kind::tf32, hi*hi + hi*lo + lo*hi, FP32 accumulate */
    SPAMM_PREC_TF32 = 2,    /* tcgen05 kind::tf32, one pass, FP32 accumulate */
    SPAMM_PREC_BF16X3 = 3,  /* tcgen05 kind::f16 on bf16 hi/lo splits, FP32 accumulate */
    SPAMM_PREC_F16X3 = 4    /* tcgen05 kind::f16 on fp16 hi/lo splits of each operand scaled
                               by a power of two (its largest leaf norm to 2^15), FP32
                               accumulate: 3xTF32-class accuracy with 2-byte operands */
} spamm_precision;

typedef struct {
    int32_t leaf;          /* leaf block size b: 16, 32, 64 or 128 (every
                              precision) */
    int32_t precision;     /* spamm_precision */
    double tie_rel;        /* relative half-width of the band around tau whose
                              triples are counted in spamm_stats (default 1e-6) */
    int64_t pool_bytes;    /* device pool for frontiers and triple lists;
                              0 = 1 GiB, grown on demand in checked mode */
    int32_t checked;       /* 1: spamm_multiply waits for completion, grows the
                              pool and re-runs on overflow, and reports device
                              errors in its return code; 0: fully asynchronous,
                              check spamm_stats */
    int32_t slice;         /* sub-leaf cull along k (the paper's SpAMM(4x4),
                              Sec. III.B, cull finer than storage): 0 = off;
                              16 = inside each kept leaf product, the product
                              of the b x 16 panel of A_IK and the 16 x b panel
                              of B_KJ over each group of 16 k is kept only if
                              their norms pass the SpAMM condition.
                              Tensor-core precisions and leaf >= 32 only. */
    int32_t tier_bits;     /* precision chosen by norm (the SpAMM condition of
                              Eq. (norm_condition) applied a second time, at
                              tau_h = 2^tier_bits tau): 0 = off; 1..40 = a kept
                              leaf product with ||A_IK|| ||B_KJ|| < tau_h
                              (squared, FP64, as the cull) runs one pass on
                              the high parts of the split (hi * hi) instead
                              of three, and the step's low parts are not
                              loaded when none of its products needs them.
                              The dropped cross terms are bounded by
                              (2u + u^2) ||A_IK|| ||B_KJ|| with u = 2^-p, p
                              the high part's significant bits (11 for
                              SPAMM_PREC_F16X3 and SPAMM_PREC_TF32X3, 8 for
                              SPAMM_PREC_BF16X3), so tier_bits = p - 1 keeps
                              each such product's error near tau, like a
                              culled one.  Split precisions only. */
    int32_t staged;        /* 0 (default): an FP32 product of at most 128 leaves
                              per side runs its cull, grouping and leaf
                              products fused in one launch (the same triples,
                              statistics and C as the staged launches);
                              1: always the staged launches (one per tier
                              and stage, with per-stage timings) */
    int32_t reserved[4];   /* must be zero */
} spamm_config;

/* Fill *cfg with the defaults: leaf 16, SPAMM_PREC_FP32, tie_rel 1e-6,
 * pool_bytes 0, checked 1. */
void spamm_config_default(spamm_config *cfg);

typedef struct spamm_ctx spamm_ctx;
typedef struct spamm_tree spamm_tree;

#define SPAMM_MAX_TIERS 32

typedef struct {
    int32_t status;                    /* spamm_status of the last multiply */
    int32_t depth;                     /* d of Eq. (depth) */
    int64_t n;
    int32_t leaf;
    int32_t precision;
    double tau;
    int64_t tier_candidates[SPAMM_MAX_TIERS]; /* triples tested at tier t */
    int64_t tier_kept[SPAMM_MAX_TIERS];       /* triples kept at tier t */
    int64_t leaf_triples;              /* = tier_kept[depth] */
    int64_t tie_band;                  /* tested triples with | ||A|| ||B|| - tau |
                                          <= tie_rel * tau, over all tiers */
    int64_t active_steps;              /* (C tile, K) pairs with >= 1 kept product */
    int64_t tiles;                     /* 128 x 256 C tiles (incl. empty ones) */
    double kept_flops;                 /* 2 b^3 per leaf triple (2 b^2 slice per
                                          kept slice product with slice != 0) */
    double dense_flops;                /* 2 n^3 (Appendix A, square case) */
    int64_t pool_bytes;                /* current pool size */
    int64_t pool_needed_bytes;         /* bytes the last multiply needed */
    float ms_symbolic;                 /* cull + grouping, CUDA events */
    float ms_numeric;                  /* leaf products + C epilogue */
    float ms_total;
    float ms_pack;                     /* tensor-core packs of the needed leaves: the
                                          part not hidden behind the cull, beside
                                          which they run on a side stream */
    int32_t slice;                     /* the config's slice (0: off) */
    int32_t pad;
    int64_t slice_kept;                /* kept k-slice products (slice != 0) */
    int64_t slice_tested;              /* tested k-slice products (slice != 0) */
    int64_t packed_leaves_a;           /* leaves packed as A-role tensor-core operands
                                          (those a kept product can read) */
    int64_t packed_leaves_b;           /* leaves packed as B-role operands */
    int64_t hi_products;               /* with tier_bits: kept leaf products run with
                                          the full split (norm product >= tau_h); the
                                          other leaf_triples - hi_products ran one
                                          pass.  Without tier_bits: leaf_triples */
    int64_t tie_band_hi;               /* kept leaf products with | ||A|| ||B|| - tau_h |
                                          <= tie_rel * tau_h (0 without tier_bits) */
    double kept_flops_clipped;         /* kept_flops counted over each leaf's extent
                                          inside the n x n matrices (rows x columns x k
                                          of the ragged last leaves clipped), i.e.
                                          without the zero padding */
} spamm_stats_t;

/* Create a context bound to the current CUDA device and to `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  cfg NULL = defaults.
 * Allocates the pool and a small control block.  INVALID_ARG for a bad
 * config, OOM, CUDA. */
spamm_status spamm_create(spamm_ctx **ctx, void *stream, const spamm_config *cfg);

/* Release the context and everything it owns (not the trees).  Synchronises
 * the stream. */
spamm_status spamm_destroy(spamm_ctx *ctx);

/* Re-bind the context to another stream (a cudaStream_t). */
spamm_status spamm_set_stream(spamm_ctx *ctx, void *stream);

/* Switch checked mode (see spamm_config.checked) on or off. */
spamm_status spamm_set_checked(spamm_ctx *ctx, int32_t checked);

/* Bound of the tensor-core leaf kernel's pipeline waits (each wait for a
 * stage of operands, for shared memory to refill, or for a TMEM
 * accumulator), in nanoseconds; wait_ns <= 0 restores the default of one
 * second.  A wait that runs out makes the kernel give up: it raises the
 * context's TIMEOUT status, lets the copies and MMAs it issued complete,
 * frees its tensor memory and returns, so the context stays usable; C is
 * not valid after a TIMEOUT.  A short bound exists for failure-detection
 * tests (a wait that nothing satisfies in time), not for production use. */
spamm_status spamm_set_wait_limit(spamm_ctx *ctx, int64_t wait_ns);

/* Grow the triple pool to at least pool_bytes (never shrinks).  Synchronises
 * the stream when it reallocates.  OOM, INVALID_ARG (negative size). */
spamm_status spamm_reserve(spamm_ctx *ctx, int64_t pool_bytes);

/* Message for the last failure on ctx (never NULL; "" when none). */
const char *spamm_last_error(const spamm_ctx *ctx);

/* Stage 1, Sec. II.A-B.  Builds the norm quadtree of the n x n matrix A
 * (device, row-major, leading dimension lda >= n): depth d from Eq. (depth)
 * (the smallest d >= 0 with b 2^d >= n), the matrix zero-padded to
 * n_p = b 2^d, leaf squared norms summed in FP64 from exact FP64 squares,
 * and each upper node the sum of its four children.  For tensor-core
 * precisions it allocates (but does not fill) the leaf tiles in tensor-core
 * layout: spamm_multiply writes those of the leaves that can take part in a
 * kept product, once tau and the other operand are known.  *out is
 * owned by the caller (spamm_tree_destroy).  The tree keeps the pointer A:
 * the caller keeps A alive and unchanged until the last multiply that reads
 * the tree has completed on the stream.  INVALID_ARG (n <= 0, lda < n, NULL
 * pointers), UNSUPPORTED (more than 2^14 leaves per side), OOM, CUDA.
 * Non-finite entries are detected by spamm_multiply (SPAMM_ERR_NONFINITE). */
spamm_status spamm_build_norms(spamm_ctx *ctx, const float *A, int64_t n, int64_t lda,
                               spamm_tree **out);

/* Recompute an existing tree for new contents A (same n, same or larger
 * lda is allowed), reusing its device storage.  Same errors as
 * spamm_build_norms. */
spamm_status spamm_tree_rebuild(spamm_ctx *ctx, spamm_tree *tree, const float *A,
                                int64_t lda);

/* spamm_tree_rebuild for `count` trees at once (host arrays of length
 * count; A[p] device matrices of the trees' n, lda[p] >= n), spread over the
 * same side streams as spamm_multiply_batched and joined back into ctx's
 * stream before the call returns control of it.  Capturable in a CUDA graph.
 * INVALID_ARG, CUDA. */
spamm_status spamm_tree_rebuild_batched(spamm_ctx *ctx, int32_t count, spamm_tree *const *trees,
                                        const float *const *A, const int64_t *lda);

/* Sparsified storage (Sec. II.D: a drop tolerance on the operands).  Like
 * spamm_build_norms, but every leaf whose squared norm times
 * max(||A||_F^2, partner_norm2) fails the SpAMM test at tau is dropped (a
 * NULL block, R3), and the kept leaves are copied into storage of their own:
 * each leaf row keeps the FP32 columns of its band of kept leaves, and the
 * tensor-core packs hold pieces only inside the bands.  For matrices with
 * decay in a locality-preserving order the storage is O(n) (band width
 * times n) instead of O(n^2).  With partner_norm2 = the other operand's
 * squared Frobenius norm this is the paper's epsilon = tau / max(||A||_F,
 * ||B||_F), and spamm_multiply of two trees sparsified at that tau keeps
 * exactly the leaf products of the dense trees (a dropped leaf's product
 * with any leaf is below tau) and gives the same C.  The tree keeps no
 * reference to A: the call synchronises once (to size the bands) and then
 * queues the copy of the kept leaves on ctx's stream, so A must stay
 * unchanged until that stream has passed the call (stream-ordered reuse of
 * A is safe).  Tensor-core precisions only; spamm_tree_rebuild does not
 * apply (UNSUPPORTED).  INVALID_ARG, NONFINITE, UNSUPPORTED, OOM, CUDA. */
spamm_status spamm_sparsify(spamm_ctx *ctx, const float *A, int64_t n, int64_t lda, double tau,
                            double partner_norm2, spamm_tree **out);

/* spamm_sparsify into an existing sparsified tree of this context and
 * configuration, for new contents A of the same n (lda >= n): the tree's
 * device storage is reused whenever the new bands fit in it and grown by a
 * quarter beyond the need when they do not, so re-sparsifying in a loop
 * (Sec. IV's purification iterations) allocates nothing once the bands have
 * settled.  tau and partner_norm2 may differ from the tree's first call.
 * On an error the tree's root norm is left non-finite, so every multiply
 * with it reports NONFINITE until a later spamm_sparsify_into succeeds.
 * INVALID_ARG (NULL, a dense tree, another context or configuration),
 * NONFINITE, OOM, CUDA. */
spamm_status spamm_sparsify_into(spamm_ctx *ctx, spamm_tree *tree, const float *A, int64_t lda,
                                 double tau, double partner_norm2);

/* Device bytes a tree holds, and for a sparsified tree the number of kept
 * leaves (-1 for a dense tree). */
spamm_status spamm_tree_bytes(const spamm_tree *tree, int64_t *bytes, int64_t *stored);

/* Free a tree.  Synchronises its context's stream first. */
spamm_status spamm_tree_destroy(spamm_tree *tree);

/* Device bytes a tree of order n takes under ctx's configuration (norm
 * pyramid plus, for tensor-core precisions, the pack arrays), for admission
 * control before spamm_build_norms.  INVALID_ARG, UNSUPPORTED. */
spamm_status spamm_tree_footprint(const spamm_ctx *ctx, int64_t n, int64_t *bytes);

/* Depth and node count of a tree (no synchronisation). */
spamm_status spamm_tree_shape(const spamm_tree *tree, int32_t *depth, int64_t *nodes);

/* Copy all squared norms of a tree to host memory (count >= nodes doubles;
 * tier t row-major 2^t x 2^t at offset (4^t - 1) / 3).  Synchronises. */
spamm_status spamm_tree_norms(spamm_ctx *ctx, const spamm_tree *tree, double *host_out,
                              int64_t count);

/* Stages 2-4, Eqs. (product) and (norm_condition), Algorithm 1:
 * C = alpha * sum_{(I,K,J) kept} A_IK B_KJ + beta * C over the n x n device
 * matrix C (row-major, ldc >= n).  A product is kept iff
 * ||A_IK||^2 ||B_KJ||^2 >= tau^2 (FP64) with both norms non-zero, and so is
 * every ancestor block product (the cull descends from the root).  Each C
 * block accumulates its kept products in ascending K, so the result is
 * deterministic.  When beta == 0, C is not read.  The two trees must have
 * the same n and leaf size; they may be the same tree (A = B).  In checked
 * mode the call waits for completion; otherwise status arrives through
 * spamm_stats.  INVALID_ARG (tau < 0 or NaN, ldc < n, mismatched trees),
 * NONFINITE, CAPACITY, TIMEOUT, OOM, CUDA. */
spamm_status spamm_multiply(spamm_ctx *ctx, const spamm_tree *A, const spamm_tree *B,
                            double tau, float alpha, float beta, float *C, int64_t ldc);

/* Batched form of spamm_multiply (same Eqs. and algorithm) for `count`
 * independent products of possibly different n:
 *   C[p] = alpha[p] * SpAMM(A[p], B[p]; tau[p]) + beta[p] * C[p],  p < count.
 * All trees must be built under ctx's configuration (leaf size, precision);
 * A[p] and B[p] have the same n.  Stages 2-3 (and the packs) run per
 * product in a sub-context of ctx (own pool, created on first use and kept),
 * the products spread over eight side streams that fork from and join back
 * into ctx's stream, so small products overlap on the device; stage 4 of
 * all products is one persistent launch over the concatenated list of C
 * tiles (up to 64 products per launch) on the tensor-core precisions, one
 * launch per product (on the side streams) for SPAMM_PREC_FP32.  Every product's C is the same,
 * bit for bit, as a single spamm_multiply of it.  Arrays are host arrays of
 * length count; matrices are device memory.  In checked mode the call waits,
 * grows the pool of any product that overflowed and re-runs the batch; with
 * checked == 0 it is asynchronous and can be captured in a CUDA graph once
 * the sub-contexts exist (after a first call).  spamm_stats then reports
 * counts and flops summed over the batch.  INVALID_ARG, NONFINITE, CAPACITY,
 * TIMEOUT, OOM, CUDA. */
spamm_status spamm_multiply_batched(spamm_ctx *ctx, int32_t count, const spamm_tree *const *A,
                                    const spamm_tree *const *B, const double *tau,
                                    const float *alpha, const float *beta, float *const *C,
                                    const int64_t *ldc);

/* The paper's flat enumeration of the leaf triples (Sec. III.D.2, Algorithm
 * 1) on the GPU: per leaf column K the leaves of A (column K) and of B (row
 * K) sorted by descending norm, and for each A leaf the prefix of B leaves
 * whose norm product passes the SpAMM condition (the early exit).  It
 * returns the same set as the hierarchical cull of spamm_multiply (a
 * parent's norm is never below its children's), as an alternative cull and
 * a cross-check.  Trees as for spamm_multiply; at most 2048 leaves per
 * side (UNSUPPORTED beyond).  host_out receives min(count, cap) rows (I, K,
 * J) sorted by (I, J, K); *count the number of triples; *ms (may be NULL)
 * the device time of the enumeration.  Synchronises.  INVALID_ARG,
 * NONFINITE, UNSUPPORTED, OOM, CUDA. */
spamm_status spamm_cull_flat(spamm_ctx *ctx, const spamm_tree *A, const spamm_tree *B,
                             double tau, int32_t *host_out, int64_t cap, int64_t *count,
                             float *ms);

/* Statistics of product `index` of the last spamm_multiply_batched on ctx
 * (same fields as spamm_stats, without the timings).  Synchronises.
 * INVALID_ARG (no such product), or the product's own status. */
spamm_status spamm_stats_item(spamm_ctx *ctx, int32_t index, spamm_stats_t *out);

/* End-to-end form with HOST matrices (row-major, ld = n): copies A and B
 * (and C when beta != 0) to device buffers owned by ctx, builds both trees,
 * multiplies and copies C back.  B may be NULL or equal to A for a square.
 * On the tensor-core precisions the leaf products run in up to eight
 * launches of whole tile-row groups on two side-by-side streams, and each
 * launch's rows of C are copied back (on another side stream of ctx) as
 * soon as it finishes, while the later ones compute; C is the same as from
 * spamm_multiply, bit for bit.  Host buffers may be pageable or pinned
 * (pinned is faster).  Synchronises. */
spamm_status spamm_multiply_host(spamm_ctx *ctx, const float *A, const float *B, int64_t n,
                                 double tau, float alpha, float beta, float *C);

/* spamm_triples restricted to the leaf triples that ran with the full split
 * precision under tier_bits (norm product >= tau_h); all kept triples
 * without tier_bits.  Synchronises. */
spamm_status spamm_triples_hi(spamm_ctx *ctx, int32_t *host_out, int64_t cap, int64_t *count);

/* Statistics of the last multiply on ctx.  Synchronises the stream.  Returns
 * the multiply's own status (e.g. CAPACITY) as well as writing *out. */
spamm_status spamm_stats(spamm_ctx *ctx, spamm_stats_t *out);

/* Copy the surviving leaf triples of the last multiply to host memory as
 * int32 (I, K, J) rows, in no particular order; *count gets the number of
 * triples (also when it exceeds cap, in which case only cap rows are
 * written).  Synchronises. */
spamm_status spamm_triples(spamm_ctx *ctx, int32_t *host_out, int64_t cap, int64_t *count);

/* No counterpart in the paper: a convenience for callers that cannot
 * allocate device memory (a host framework or plugin that owns all device
 * memory through its own allocator or memory cap, or a loop that must not
 * pay cudaMalloc's implicit synchronisation).
 * Computes the same C = alpha * SpAMM(A, B; tau) + beta * C as
 * spamm_build_norms + spamm_multiply with leaf 16 and SPAMM_PREC_FP32, on
 * DEVICE matrices (row-major, lda/ldb/ldc >= n) and the cudaStream_t
 * `stream`, without allocating anything: every scratch buffer lives in one
 * static 8 MiB device array that each GPU loading this library holds until
 * exit, sized for the worst case at n <= 4096.  The first call on each
 * device, with that device current, looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The address is cached for the life of the process: do not call this entry
 * point on a device after cudaDeviceReset (or any teardown of its primary
 * context), since the cached address would then be stale.
 * All calls share the array and it keeps the last call's contents (each
 * call clears what must start at zero); calls that overlap on the GPU race
 * on it, so order them on one stream.  Asynchronous; when status_dev (a
 * device uint32) is not NULL it receives the device status word
 * (0 = OK, 2 = non-finite input).  Returns INVALID_ARG (NULL pointer,
 * n <= 0, leading dimension < n, tau < 0 or not finite), UNSUPPORTED
 * (n > 4096: beyond the static scratch), CUDA. */
spamm_status spamm_multiply_static(const float *A, int64_t lda, const float *B, int64_t ldb,
                                   int64_t n, double tau, float alpha, float beta, float *C,
                                   int64_t ldc, void *stream, uint32_t *status_dev);

#ifdef __cplusplus
}
#endif

#endif /* SPAMM_H_ */
