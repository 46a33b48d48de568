/*
 * FP64 CPU oracle for SpAMM (Bock & Challacombe, "An Optimized Sparse
 * Approximate Matrix Multiply for Matrices with Decay").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links or calls this
 * file; only the tests, the package smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or table with the CUDA path.
 *
 * Every step is written the plain way, in double precision, in the order the
 * paper states it:
 *   - quadtree depth and zero padding ............ Sec. II.A, Eq. (depth)
 *   - per-node Frobenius norms, bottom-up ........ Sec. II.B, Eq. (norm)
 *   - recursive product under the SpAMM condition  Eqs. (product), (norm_condition)
 *   - linear (Morton) index, k-value blocks, norm
 *     sort and convolution of the linkless tree .. Sec. III.D.1-2, Algorithm 1,
 *                                                  Eqs. (linear_index), (convolution)
 *   - numeric multiply C_ij += A_ik B_kj ......... Algorithm 1 (numeric part)
 *   - SGEMM-style alpha/beta epilogue ............ Sec. II (problem statement)
 *
 * Readings taken where the paper is silent (each also listed in the design
 * notes):
 *   R1  a block product is dropped only when ||A_ik|| ||B_kj|| < tau (strict),
 *       so a product exactly at tau is kept;
 *   R2  norms are compared squared, in FP64: keep iff nA2 * nB2 >= tau * tau;
 *   R3  a zero block is a NULL link: it never produces a product, even at
 *       tau = 0;
 *   R4  d = ceil(log2(n / b)) is taken as the smallest d >= 0 with
 *       b * 2^d >= n (so d = 0 when n <= b);
 *   R5  within a C block the kept products are accumulated in ascending k;
 *   R14 the sub-leaf cull (oracle_multiply_sliced) splits the k dimension of
 *       a kept leaf product into slices of g and keeps a slice product iff
 *       the norms of its two panels pass the same condition;
 *   R15 sparsification (oracle_sparsify) drops a leaf iff its product with
 *       the largest operand norm fails the condition (epsilon = tau / max
 *       Frobenius norm, tested in squared form);
 *   R16 precision chosen by norm (oracle_multiply_tiered): the SpAMM
 *       condition applied a second time, at tau_h >= tau, to the kept
 *       products.  A kept product with ||A_ik|| ||B_kj|| >= tau_h is formed
 *       exactly; one below tau_h is formed from its operands rounded to p
 *       significant bits (the high part of a split precision alone).  The
 *       dropped terms are bounded by (2 u + u^2) ||A_ik|| ||B_kj|| with
 *       u = 2^-p, so such a product errs by about tau_h 2^(1-p), the same
 *       order as a culled product when tau_h = tau 2^(p-1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EARG (-1)
#define OR_ECAP (-2)
#define OR_ENOMEM (-3)

/* ------------------------------------------------------------ Eq. (depth) */

int oracle_depth(int64_t n, int64_t b)
{
    if (n <= 0 || b <= 0) return OR_EARG;
    int d = 0;
    while (b * ((int64_t)1 << d) < n) d++;
    return d;
}

int64_t oracle_tier_offset(int t) { return (((int64_t)1 << (2 * t)) - 1) / 3; }

int64_t oracle_pyramid_size(int d) { return oracle_tier_offset(d + 1); }

/* ------------------------------------------------------------- Eq. (norm) */

/* Squared Frobenius norms of every quadtree node, tier t stored row-major as
 * a 2^t x 2^t grid at offset (4^t - 1) / 3.  Leaves: plain row-major sum of
 * squares of the b x b block (elements outside the n x n matrix are the zero
 * padding).  Upper tiers: the sum of the four children, A11 + A12 + A21 + A22,
 * because the squared Frobenius norm is additive over sub-blocks. */
int oracle_build_pyramid(const float *A, int64_t n, int64_t lda, int64_t b,
                         double *pyr)
{
    int d = oracle_depth(n, b);
    if (d < 0 || lda < n) return OR_EARG;
    int64_t nb = (int64_t)1 << d;
    double *leaf = pyr + oracle_tier_offset(d);
    for (int64_t I = 0; I < nb; I++)
        for (int64_t K = 0; K < nb; K++) {
            double s = 0.0;
            for (int64_t r = I * b; r < I * b + b && r < n; r++)
                for (int64_t c = K * b; c < K * b + b && c < n; c++) {
                    double a = (double)A[r * lda + c];
                    s += a * a;
                }
            leaf[I * nb + K] = s;
        }
    for (int t = d - 1; t >= 0; t--) {
        int64_t w = (int64_t)1 << t;
        const double *ch = pyr + oracle_tier_offset(t + 1);
        double *par = pyr + oracle_tier_offset(t);
        for (int64_t i = 0; i < w; i++)
            for (int64_t j = 0; j < w; j++) {
                int64_t cw = 2 * w;
                double a11 = ch[(2 * i) * cw + 2 * j];
                double a12 = ch[(2 * i) * cw + 2 * j + 1];
                double a21 = ch[(2 * i + 1) * cw + 2 * j];
                double a22 = ch[(2 * i + 1) * cw + 2 * j + 1];
                par[i * w + j] = a11 + a12 + a21 + a22;
            }
    }
    return d;
}

/* --------------------------------------------------- Eq. (norm_condition) */

static int keep(double nA2, double nB2, double tau2)
{
    /* R1-R3: keep unless ||A|| ||B|| < tau; NULL (zero) blocks never kept. */
    return nA2 > 0.0 && nB2 > 0.0 && nA2 * nB2 >= tau2;
}

int oracle_keep(double nA2, double nB2, double tau) { return keep(nA2, nB2, tau * tau); }

/* ------------------------------------------- Eq. (product), recursively */

typedef struct {
    const double *pa, *pb;
    int d;
    double tau2;
    int32_t *out;        /* triples (I, K, J) at the leaf tier */
    int64_t cap, count;
    int64_t *cand, *kept; /* per tier t = 0..d */
} rec_state;

static void recurse(rec_state *s, int t, int64_t I, int64_t K, int64_t J)
{
    if (t == s->d) {
        if (s->count < s->cap) {
            s->out[3 * s->count + 0] = (int32_t)I;
            s->out[3 * s->count + 1] = (int32_t)K;
            s->out[3 * s->count + 2] = (int32_t)J;
        }
        s->count++;
        return;
    }
    /* C^t_ij = sum_k A^{t+1}_ik B^{t+1}_kj, each product subject to the
     * SpAMM condition on the children's norms. */
    int64_t w = (int64_t)1 << (t + 1);
    const double *na = s->pa + oracle_tier_offset(t + 1);
    const double *nb = s->pb + oracle_tier_offset(t + 1);
    for (int di = 0; di < 2; di++)
        for (int dj = 0; dj < 2; dj++)
            for (int dk = 0; dk < 2; dk++) {
                int64_t i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
                s->cand[t + 1]++;
                if (keep(na[i * w + k], nb[k * w + j], s->tau2)) {
                    s->kept[t + 1]++;
                    recurse(s, t + 1, i, k, j);
                }
            }
}

/* Leaf triples kept by the recursive SpAMM product.  Returns the number of
 * triples (which may exceed cap; only cap are stored).  cand/kept (length
 * d + 1) receive per-tier candidate and kept counts; tier 0 is the root
 * product itself. */
int64_t oracle_cull_recursive(const double *pyrA, const double *pyrB, int d,
                              double tau, int32_t *out, int64_t cap,
                              int64_t *cand, int64_t *kept)
{
    rec_state s = {pyrA, pyrB, d, tau * tau, out, cap, 0, cand, kept};
    for (int t = 0; t <= d; t++) cand[t] = kept[t] = 0;
    cand[0] = 1;
    if (keep(pyrA[0], pyrB[0], s.tau2)) {
        kept[0] = 1;
        recurse(&s, 0, 0, 0, 0);
    }
    return s.count;
}

/* ---------------------------------------------- Eq. (linear_index) */

/* l = sum_m [ i_m 2^(2m+1) + j_m 2^(2m) ]: row bits on odd positions, column
 * bits on even positions. */
uint64_t oracle_morton(uint32_t i, uint32_t j)
{
    uint64_t l = 0;
    for (int m = 0; m < 32; m++) {
        l |= (uint64_t)((i >> m) & 1u) << (2 * m + 1);
        l |= (uint64_t)((j >> m) & 1u) << (2 * m);
    }
    return l;
}

#define EVEN_BITS 0x5555555555555555ULL /* 0b...010101 */
#define ODD_BITS 0xAAAAAAAAAAAAAAAAULL  /* 0b...101010 */

static uint32_t compress_even(uint64_t x)
{
    uint32_t v = 0;
    for (int m = 0; m < 32; m++) v |= (uint32_t)((x >> (2 * m)) & 1u) << m;
    return v;
}

void oracle_morton_decode(uint64_t l, uint32_t *i, uint32_t *j)
{
    *i = compress_even(l >> 1);
    *j = compress_even(l);
}

/* The masks of Sec. III.D.2: the k digits of l_A(ik) are its even bits and
 * those of l_B(kj) its odd bits; Eq. (convolution) assembles l_C(ij) from
 * the odd bits of l_A and the even bits of l_B. */
uint64_t oracle_k_key_A(uint64_t lA) { return lA & EVEN_BITS; }
uint64_t oracle_k_key_B(uint64_t lB) { return (lB & ODD_BITS) >> 1; }
uint64_t oracle_convolve(uint64_t lA, uint64_t lB) { return (lA & ODD_BITS) | (lB & EVEN_BITS); }

/* ------------------------------------ Algorithm 1: linkless tree, flat */

typedef struct {
    uint64_t l;   /* linear index of the leaf */
    uint64_t k;   /* k digits, aligned to even bits */
    double n2;    /* squared norm */
} key_t_;

static int cmp_k_then_norm(const void *pa, const void *pb)
{
    const key_t_ *a = (const key_t_ *)pa, *b = (const key_t_ *)pb;
    if (a->k != b->k) return a->k < b->k ? -1 : 1;
    if (a->n2 != b->n2) return a->n2 > b->n2 ? -1 : 1; /* descending norm */
    return a->l < b->l ? -1 : (a->l > b->l);
}

/* Flat enumeration of the leaf tier in the manner of Algorithm 1:
 *   1. extract the linear indices of all non-NULL leaves of A and B,
 *   2. sort each list on its k digits into k-value blocks,
 *   3. inside each k-value block sort by descending norm,
 *   4. for every matching pair of k-value blocks convolve: for each A leaf,
 *      walk the B leaves in descending norm and stop at the first one that
 *      fails the SpAMM condition; the C index comes from Eq. (convolution).
 * Emits triples (I, K, J).  Returns the count (may exceed cap). */
int64_t oracle_cull_linkless(const double *pyrA, const double *pyrB, int d,
                             double tau, int32_t *out, int64_t cap)
{
    int64_t nb = (int64_t)1 << d;
    const double *la = pyrA + oracle_tier_offset(d);
    const double *lb = pyrB + oracle_tier_offset(d);
    double tau2 = tau * tau;
    key_t_ *ka = (key_t_ *)malloc(sizeof(key_t_) * (size_t)(nb * nb));
    key_t_ *kb = (key_t_ *)malloc(sizeof(key_t_) * (size_t)(nb * nb));
    if (!ka || !kb) { free(ka); free(kb); return OR_ENOMEM; }
    int64_t na = 0, nbk = 0;
    for (int64_t r = 0; r < nb; r++)
        for (int64_t c = 0; c < nb; c++) {
            uint64_t l = oracle_morton((uint32_t)r, (uint32_t)c);
            if (la[r * nb + c] > 0.0) {
                ka[na].l = l; ka[na].k = oracle_k_key_A(l); ka[na].n2 = la[r * nb + c]; na++;
            }
            if (lb[r * nb + c] > 0.0) {
                kb[nbk].l = l; kb[nbk].k = oracle_k_key_B(l); kb[nbk].n2 = lb[r * nb + c]; nbk++;
            }
        }
    qsort(ka, (size_t)na, sizeof(key_t_), cmp_k_then_norm);
    qsort(kb, (size_t)nbk, sizeof(key_t_), cmp_k_then_norm);
    int64_t count = 0, ia = 0, ib = 0;
    while (ia < na && ib < nbk) {
        if (ka[ia].k < kb[ib].k) { ia++; continue; }
        if (kb[ib].k < ka[ia].k) { ib++; continue; }
        uint64_t k = ka[ia].k;
        int64_t ea = ia, eb = ib;
        while (ea < na && ka[ea].k == k) ea++;
        while (eb < nbk && kb[eb].k == k) eb++;
        for (int64_t x = ia; x < ea; x++)
            for (int64_t y = ib; y < eb; y++) {
                if (!keep(ka[x].n2, kb[y].n2, tau2)) break; /* sorted: rest fail */
                uint64_t lc = oracle_convolve(ka[x].l, kb[y].l);
                uint32_t I, J, I2, K;
                oracle_morton_decode(lc, &I, &J);
                oracle_morton_decode(ka[x].l, &I2, &K);
                if (count < cap) {
                    out[3 * count + 0] = (int32_t)I;
                    out[3 * count + 1] = (int32_t)K;
                    out[3 * count + 2] = (int32_t)J;
                }
                count++;
            }
        ia = ea;
        ib = eb;
    }
    free(ka);
    free(kb);
    return count;
}

/* -------------------------------------- numeric multiply, Algorithm 1 */

/* acc (b x b, row-major, FP64) += A_IK * B_KJ as a naive triple loop, with
 * the zero padding outside the n x n matrices. */
static void leaf_product(const float *A, int64_t lda, const float *B, int64_t ldb,
                         int64_t n, int64_t b, int64_t I, int64_t K, int64_t J,
                         double *acc)
{
    for (int64_t r = 0; r < b; r++) {
        int64_t gr = I * b + r;
        if (gr >= n) break;
        for (int64_t c = 0; c < b; c++) {
            int64_t gc = J * b + c;
            if (gc >= n) break;
            double s = 0.0;
            for (int64_t q = 0; q < b; q++) {
                int64_t gk = K * b + q;
                if (gk >= n) break;
                s += (double)A[gr * lda + gk] * (double)B[gk * ldb + gc];
            }
            acc[r * b + c] += s;
        }
    }
}

static int cmp_ijk(const void *pa, const void *pb)
{
    const int32_t *a = (const int32_t *)pa, *b = (const int32_t *)pb;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1; /* I */
    if (a[2] != b[2]) return a[2] < b[2] ? -1 : 1; /* J */
    return (a[1] > b[1]) - (a[1] < b[1]);          /* K ascending (R5) */
}

/* Full SpAMM: C = alpha * sum_{kept} A_IK B_KJ + beta * C, everything in
 * FP64 (C is an n x n FP64 array, ldc >= n; when beta == 0 its input is not
 * read).  Triples (sorted by I, J, then K) are written to out (3 x cap
 * int32); stats[0..d] get per-tier candidates, stats[d+1..2d+1] per-tier
 * kept counts.  Returns the number of leaf triples or a negative error. */
int64_t oracle_multiply(const float *A, int64_t lda, const float *B, int64_t ldb,
                        int64_t n, int64_t b, double tau, double alpha, double beta,
                        double *C, int64_t ldc, int32_t *out, int64_t cap,
                        int64_t *stats)
{
    int d = oracle_depth(n, b);
    if (d < 0 || lda < n || ldb < n || ldc < n || !(tau >= 0.0)) return OR_EARG;
    int64_t ps = oracle_pyramid_size(d);
    double *pa = (double *)malloc(sizeof(double) * (size_t)ps);
    double *pb = (double *)malloc(sizeof(double) * (size_t)ps);
    if (!pa || !pb) { free(pa); free(pb); return OR_ENOMEM; }
    oracle_build_pyramid(A, n, lda, b, pa);
    oracle_build_pyramid(B, n, ldb, b, pb);
    int64_t cnt = oracle_cull_recursive(pa, pb, d, tau, out, cap, stats, stats + d + 1);
    free(pa);
    free(pb);
    if (cnt > cap) return OR_ECAP;
    qsort(out, (size_t)cnt, 3 * sizeof(int32_t), cmp_ijk);

    int64_t nb = (int64_t)1 << d;
    /* index of the first triple of each C block row I */
    int64_t *rowstart = (int64_t *)calloc((size_t)(nb + 1), sizeof(int64_t));
    if (!rowstart) return OR_ENOMEM;
    for (int64_t t = 0; t < cnt; t++) rowstart[out[3 * t] + 1]++;
    for (int64_t I = 0; I < nb; I++) rowstart[I + 1] += rowstart[I];

    int64_t nbr = (n + b - 1) / b; /* block rows that hold matrix rows */
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t I = 0; I < nbr; I++) {
        double *acc = (double *)malloc(sizeof(double) * (size_t)(b * b * nbr));
        if (!acc) { err = 1; continue; }
        memset(acc, 0, sizeof(double) * (size_t)(b * b * nbr));
        for (int64_t t = rowstart[I]; t < rowstart[I + 1]; t++)
            leaf_product(A, lda, B, ldb, n, b, I, out[3 * t + 1], out[3 * t + 2],
                         acc + out[3 * t + 2] * b * b);
        for (int64_t r = I * b; r < I * b + b && r < n; r++)
            for (int64_t c = 0; c < n; c++) {
                int64_t J = c / b;
                double v = alpha * acc[J * b * b + (r - I * b) * b + (c - J * b)];
                C[r * ldc + c] = beta == 0.0 ? v : v + beta * C[r * ldc + c];
            }
        free(acc);
    }
    free(rowstart);
    return err ? OR_ENOMEM : cnt;
}

/* ------------------------------------------ precision by norm (R16) */

/* x rounded to p significant bits (1 <= p <= 53), to nearest; ties to even,
 * or away from zero when ties_away is set.  The exponent range is
 * unbounded (no overflow, no subnormals): x = m 2^e with 1/2 <= |m| < 1,
 * so m 2^p is exact and rounding it to an integer keeps p bits. */
double oracle_round_sig(double x, int p, int ties_away)
{
    if (x == 0.0 || !isfinite(x) || p >= 53) return x;
    int e;
    double m = frexp(x, &e);
    double s = ldexp(m, p);
    double r = ties_away ? round(s) : nearbyint(s); /* default mode: ties to even */
    return ldexp(r, e - p);
}

/* acc (b x b, FP64) += round(A_IK) round(B_KJ): the leaf product of the
 * operands rounded to p significant bits, naive triple loop, zero padding. */
static void leaf_product_rounded(const float *A, int64_t lda, const float *B, int64_t ldb,
                                 int64_t n, int64_t b, int64_t I, int64_t K, int64_t J,
                                 int p, int ties_away, double *acc)
{
    for (int64_t r = 0; r < b; r++) {
        int64_t gr = I * b + r;
        if (gr >= n) break;
        for (int64_t c = 0; c < b; c++) {
            int64_t gc = J * b + c;
            if (gc >= n) break;
            double s = 0.0;
            for (int64_t q = 0; q < b; q++) {
                int64_t gk = K * b + q;
                if (gk >= n) break;
                s += oracle_round_sig((double)A[gr * lda + gk], p, ties_away) *
                     oracle_round_sig((double)B[gk * ldb + gc], p, ties_away);
            }
            acc[r * b + c] += s;
        }
    }
}

/* SpAMM with the precision of each kept product chosen by its norm (R16):
 * the cull of oracle_multiply at tau, then every kept product with
 * nA2 * nB2 >= tau_h^2 (FP64, squared as in R2) formed exactly, every other
 * kept product formed from its operands rounded to p significant bits (ties
 * to even, or away from zero).  C blocks accumulate in ascending K as in
 * oracle_multiply; with tau_h <= tau (or p >= 53) the result is
 * oracle_multiply's bit for bit.  stats[0] = kept products formed exactly,
 * stats[1] = kept products formed rounded; cull_stats (2 (d + 1), may be
 * NULL) gets the per-tier counts.  Returns the number of kept leaf triples
 * or an error code. */
int64_t oracle_multiply_tiered(const float *A, int64_t lda, const float *B, int64_t ldb,
                               int64_t n, int64_t b, double tau, double tau_h, int p,
                               int ties_away, double alpha, double beta, double *C,
                               int64_t ldc, int64_t *stats)
{
    int d = oracle_depth(n, b);
    if (d < 0 || lda < n || ldb < n || ldc < n || !(tau >= 0.0) || !(tau_h >= 0.0) ||
        p < 1) return OR_EARG;
    int64_t ps = oracle_pyramid_size(d);
    double *pa = (double *)malloc(sizeof(double) * (size_t)ps);
    double *pb = (double *)malloc(sizeof(double) * (size_t)ps);
    int64_t *cs = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(d + 1));
    if (!pa || !pb || !cs) { free(pa); free(pb); free(cs); return OR_ENOMEM; }
    oracle_build_pyramid(A, n, lda, b, pa);
    oracle_build_pyramid(B, n, ldb, b, pb);
    int64_t cnt = oracle_cull_recursive(pa, pb, d, tau, NULL, 0, cs, cs + d + 1);
    int32_t *tri = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(cnt > 0 ? cnt : 1));
    if (!tri) { free(pa); free(pb); free(cs); return OR_ENOMEM; }
    oracle_cull_recursive(pa, pb, d, tau, tri, cnt, cs, cs + d + 1);
    free(cs);
    qsort(tri, (size_t)cnt, 3 * sizeof(int32_t), cmp_ijk);
    int64_t nb = (int64_t)1 << d;
    const double *la = pa + oracle_tier_offset(d);
    const double *lb = pb + oracle_tier_offset(d);
    int64_t nbr = (n + b - 1) / b;
    int64_t exact = 0, rounded = 0;
    double *acc = (double *)malloc(sizeof(double) * (size_t)(b * b * nbr));
    if (!acc) { free(pa); free(pb); free(tri); return OR_ENOMEM; }
    int64_t t = 0;
    for (int64_t I = 0; I < nbr; I++) {
        memset(acc, 0, sizeof(double) * (size_t)(b * b * nbr));
        for (; t < cnt && tri[3 * t] == I; t++) {
            int64_t K = tri[3 * t + 1], J = tri[3 * t + 2];
            if (keep(la[I * nb + K], lb[K * nb + J], tau_h * tau_h)) {
                leaf_product(A, lda, B, ldb, n, b, I, K, J, acc + J * b * b);
                exact++;
            } else {
                leaf_product_rounded(A, lda, B, ldb, n, b, I, K, J, p, ties_away,
                                     acc + J * b * b);
                rounded++;
            }
        }
        for (int64_t r = I * b; r < I * b + b && r < n; r++)
            for (int64_t c = 0; c < n; c++) {
                int64_t J = c / b;
                double v = alpha * acc[J * b * b + (r - I * b) * b + (c - J * b)];
                C[r * ldc + c] = beta == 0.0 ? v : v + beta * C[r * ldc + c];
            }
    }
    free(acc);
    free(tri);
    free(pa);
    free(pb);
    if (stats) {
        stats[0] = exact;
        stats[1] = rounded;
    }
    return cnt;
}

/* Sub-leaf cull along k (the paper's SpAMM(4x4) of Sec. III.B, cull finer
 * than storage, read for tensor cores, reading R14): the leaf triples kept
 * by the recursive product are multiplied slice by slice.  Slice s of leaf
 * column K covers the g columns K*b + s*g .. K*b + s*g + g - 1 of A (the
 * same rows of B); the b x g panel of A_IK and the g x b panel of B_KJ are
 * multiplied only if their Frobenius norms pass the SpAMM condition (R1-R3,
 * squared in FP64, panel norms summed row-major from exact squares).  Each C
 * block accumulates its kept slice products in ascending (K, s).  With
 * tau_h > tau, the precision of every kept leaf product is chosen by its leaf
 * norms as in oracle_multiply_tiered (R16): its slice products are formed
 * exactly if nA2 * nB2 >= tau_h^2, else from operands rounded to p
 * significant bits; tau_h = 0 forms every slice product exactly.
 * stats[0] = kept slice products, stats[1] = tested slice products.
 * Returns the number of kept leaf triples or an error code. */
static double panel_norm2(const float *M, int64_t ld, int64_t n, int64_t r0, int64_t nr,
                          int64_t c0, int64_t nc)
{
    double s = 0.0;
    for (int64_t r = r0; r < r0 + nr && r < n; r++)
        for (int64_t c = c0; c < c0 + nc && c < n; c++) {
            double v = (double)M[r * ld + c];
            s += v * v;
        }
    return s;
}

int64_t oracle_multiply_sliced(const float *A, int64_t lda, const float *B, int64_t ldb,
                               int64_t n, int64_t b, int64_t g, double tau, double tau_h,
                               int p, int ties_away, double alpha, double beta, double *C,
                               int64_t ldc, int64_t *stats)
{
    int d = oracle_depth(n, b);
    if (d < 0 || lda < n || ldb < n || ldc < n || !(tau >= 0.0) || g <= 0 || b % g) return OR_EARG;
    int64_t ps = oracle_pyramid_size(d);
    double *pa = (double *)malloc(sizeof(double) * (size_t)ps);
    double *pb = (double *)malloc(sizeof(double) * (size_t)ps);
    int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(d + 1));
    if (!pa || !pb || !cand) { free(pa); free(pb); free(cand); return OR_ENOMEM; }
    oracle_build_pyramid(A, n, lda, b, pa);
    oracle_build_pyramid(B, n, ldb, b, pb);
    /* count, then collect the kept leaf triples */
    int64_t cnt = oracle_cull_recursive(pa, pb, d, tau, NULL, 0, cand, cand + d + 1);
    int32_t *tri = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(cnt > 0 ? cnt : 1));
    if (!tri) { free(pa); free(pb); free(cand); return OR_ENOMEM; }
    oracle_cull_recursive(pa, pb, d, tau, tri, cnt, cand, cand + d + 1);
    free(cand);
    qsort(tri, (size_t)cnt, 3 * sizeof(int32_t), cmp_ijk);
    int64_t nb = (int64_t)1 << d;
    const double *la = pa + oracle_tier_offset(d);
    const double *lb = pb + oracle_tier_offset(d);
    int64_t nbr = (n + b - 1) / b;
    int64_t kept = 0, tested = 0;
    double *acc = (double *)malloc(sizeof(double) * (size_t)(b * b * nbr));
    if (!acc) { free(tri); return OR_ENOMEM; }
    int64_t t = 0;
    for (int64_t I = 0; I < nbr; I++) {
        memset(acc, 0, sizeof(double) * (size_t)(b * b * nbr));
        for (; t < cnt && tri[3 * t] == I; t++) {
            int64_t K = tri[3 * t + 1], J = tri[3 * t + 2];
            int exact = tau_h <= tau || keep(la[I * nb + K], lb[K * nb + J], tau_h * tau_h);
            for (int64_t s0 = 0; s0 < b; s0 += g) {
                int64_t k0 = K * b + s0;
                double na = panel_norm2(A, lda, n, I * b, b, k0, g);
                double nbv = panel_norm2(B, ldb, n, k0, g, J * b, b);
                tested++;
                if (!keep(na, nbv, tau * tau)) continue;
                kept++;
                double *blk = acc + J * b * b;
                for (int64_t r = 0; r < b && I * b + r < n; r++)
                    for (int64_t c = 0; c < b && J * b + c < n; c++) {
                        double sum = 0.0;
                        for (int64_t q = k0; q < k0 + g && q < n; q++) {
                            double x = (double)A[(I * b + r) * lda + q];
                            double y = (double)B[q * ldb + J * b + c];
                            if (!exact) {
                                x = oracle_round_sig(x, p, ties_away);
                                y = oracle_round_sig(y, p, ties_away);
                            }
                            sum += x * y;
                        }
                        blk[r * b + c] += sum;
                    }
            }
        }
        for (int64_t r = I * b; r < I * b + b && r < n; r++)
            for (int64_t c = 0; c < n; c++) {
                int64_t J = c / b;
                double v = alpha * acc[J * b * b + (r - I * b) * b + (c - J * b)];
                C[r * ldc + c] = beta == 0.0 ? v : v + beta * C[r * ldc + c];
            }
    }
    free(acc);
    free(tri);
    free(pa);
    free(pb);
    if (stats) {
        stats[0] = kept;
        stats[1] = tested;
    }
    return cnt;
}

/* Sparsification with a drop tolerance (Sec. II.D): out = A with every leaf
 * block dropped (zeroed) whose product with the largest norm it can meet
 * fails the SpAMM condition, i.e. ||A_IK||^2 * norm2_max < tau^2 (squared,
 * FP64, R2), and every zero block dropped (R3).  With norm2_max the larger
 * of the two operands' squared Frobenius norms this is the paper's
 * epsilon = tau / max(||A||_F, ||B||_F) (reading R15).  Returns the number
 * of stored (kept, non-zero) leaves; out must hold n * n floats (ld n). */
int64_t oracle_sparsify(const float *A, int64_t lda, int64_t n, int64_t b, double tau,
                        double norm2_max, float *out)
{
    if (n <= 0 || b <= 0 || lda < n || !(tau >= 0.0)) return OR_EARG;
    int64_t nl = (n + b - 1) / b, stored = 0;
    for (int64_t I = 0; I < nl; I++)
        for (int64_t K = 0; K < nl; K++) {
            double s = panel_norm2(A, lda, n, I * b, b, K * b, b);
            int keep_leaf = keep(s, norm2_max, tau * tau);
            stored += keep_leaf;
            for (int64_t r = I * b; r < I * b + b && r < n; r++)
                for (int64_t c = K * b; c < K * b + b && c < n; c++)
                    out[r * n + c] = keep_leaf ? A[r * lda + c] : 0.0f;
        }
    return stored;
}

/* One C block without the epilogue, for spot checks at sizes where the full
 * oracle is too slow: acc = sum over ascending K with the leaf pair kept by
 * the SpAMM condition of A_IK B_KJ.  Testing the leaf pair directly gives
 * the recursive product's set because a parent's norm is never below its
 * children's (checked by the tests against oracle_cull_recursive).  With
 * tau_h > tau each kept product's precision is chosen by its norm as in
 * oracle_multiply_tiered (R16); tau_h = 0 forms every product exactly.
 * Returns the number of kept K. */
int64_t oracle_block(const float *A, int64_t lda, const float *B, int64_t ldb,
                     int64_t n, int64_t b, const double *pyrA, const double *pyrB,
                     double tau, double tau_h, int p, int ties_away, int64_t I, int64_t J,
                     double *acc)
{
    int d = oracle_depth(n, b);
    int64_t nb = (int64_t)1 << d;
    const double *la = pyrA + oracle_tier_offset(d);
    const double *lb = pyrB + oracle_tier_offset(d);
    memset(acc, 0, sizeof(double) * (size_t)(b * b));
    int64_t kept = 0;
    for (int64_t K = 0; K < nb; K++)
        if (keep(la[I * nb + K], lb[K * nb + J], tau * tau)) {
            if (tau_h <= tau || keep(la[I * nb + K], lb[K * nb + J], tau_h * tau_h))
                leaf_product(A, lda, B, ldb, n, b, I, K, J, acc);
            else
                leaf_product_rounded(A, lda, B, ldb, n, b, I, K, J, p, ties_away, acc);
            kept++;
        }
    return kept;
}

/* Many blocks in parallel (for the CPU baseline and sampled checks):
 * blocks[2*q], blocks[2*q+1] = (I, J); acc gets b*b doubles per block. */
int64_t oracle_blocks(const float *A, int64_t lda, const float *B, int64_t ldb,
                      int64_t n, int64_t b, const double *pyrA, const double *pyrB,
                      double tau, double tau_h, int p, int ties_away, const int64_t *blocks,
                      int64_t nblocks, double *acc)
{
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
    for (int64_t q = 0; q < nblocks; q++)
        total += oracle_block(A, lda, B, ldb, n, b, pyrA, pyrB, tau, tau_h, p, ties_away,
                              blocks[2 * q], blocks[2 * q + 1], acc + q * b * b);
    return total;
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
