/*
 * cpd_oracle.c -- FP64 CPU oracle for block-randomized weighted SGD with
 * importance sampling for CP decomposition (BrawsCPD / AdawsCPD,
 * Yu & Li, arXiv 2103.04081).
 *
 * TEST INFRASTRUCTURE. Only the tests, __graft_entry__.smoke() and the
 * bench's CPU-baseline / reference leg load this library. The CUDA product
 * path shares no code, header, table or helper with it, and neither side
 * includes the other.
 *
 * A second build of this same file with -DORC_OMP -fopenmp (liboracle_omp.so)
 * spreads the fiber gather and the rows of the contraction over the host's
 * cores, for CPU-baseline timing only. Its pragmas split independent loop
 * iterations and leave every sum in the order below, so both builds give the
 * same bits; the single-threaded build is the checker.
 *
 * Plain loops in FP64, one function per step of the method, in the order of
 * Alg. 3 (SKRP-ST-I) -> Alg. 1 (SKRP-ST) -> Eq. (11) -> Eq. (12) /
 * Eq. (13a)-(13b) (Alg. 4 / Alg. 5). Built with -ffp-contract=off: the only
 * fused multiply-adds are the explicit fma() calls below.
 *
 * Readings of the paper that this file implements (each also listed in the
 * design notes):
 *  - Gradient normalisation: Eq. (11) is used literally,
 *    G = (1/(B*J_n)) (A Z_S^T D Z_S - X_S D Z_S), D = diag(1/p_f); with
 *    uniform p = 1/J_n this is exactly Alg. 2's BrasCPD gradient (Sec. 2).
 *  - The garbled operand order of Eq. (11) is read as A (Z_S^T D Z_S)
 *    and X_S D Z_S (the only conforming products).
 *  - Leverage probabilities (Eq. (7), Lemma 2) are normalised by
 *    the computed sum of leverage scores W_k (= R at full column rank).
 *  - Per-factor probabilities are recomputed from the current factors at
 *    every draw (Alg. 4/5 take {p_k} as inputs; they are functions of A^(k)).
 *  - Sampling is with replacement (Alg. 3 draws each index independently,
 *    repeats allowed).
 *  - AdaGrad accumulator includes the current gradient (Eq. (13a)).
 *  - Random numbers: Philox4x64-10 (Salmon et al., SC'11); the paper uses
 *    MATLAB randsample, so bit-exact sampling is defined against this
 *    generator and the canonical sampling arithmetic below.
 *
 * Canonical sampling arithmetic (bit-exactness of the sampled indices and
 * of p_f depends on it; a second, independent implementation on the GPU
 * follows the same definitions):
 *  - Euclidean row weight (Def. 5, Lemma 4): w_i = sum_r a_ir^2 as 32 strided
 *    partials (partial p takes r = p, p+32, ... ascending, acc = fma(a, a,
 *    acc) from +0) folded by the fixed tree p += p+off for off = 16,8,4,2,1.
 *  - Leverage row weight (Def. 3): Gram g_rs = sum_i a_ir a_is in the same
 *    32-partial order over i; left-looking Cholesky g = L L^T with k
 *    ascending and inv_j = 1/L_jj; y = L^{-1} a_i by forward substitution
 *    with k ascending; w_i = sum_j y_j^2 (fma, j ascending). A pivot at or
 *    below 2^-40 times its diagonal entry means "degenerate".
 *  - Fixed-point distribution: s = 61 - ceil(log2 I) - floor(log2 max_i w_i),
 *    q_i = floor(w_i 2^s) (exact), Q = sum_i q_i < 2^62, cdf[i] = sum_{j<=i} q_j
 *    as exact 64-bit integers. Rows whose weight is below 2^-(61-ceil(log2 I))
 *    of the largest get q_i = 0 and are never drawn.
 *  - Draw: i = min{ i : floor(x Q / 2^64) < cdf[i] } for the 64-bit Philox
 *    word x (uniform sampling, q_i = 1: i = floor(x I / 2^64)).
 *  - p_k(i) = (double)q_i / (double)Q (both conversions and the quotient
 *    rounded to nearest); p_f = prod_{k != n, k ascending} p_k(i_k).
 *
 * Blocks first, then sampling (Remark 1), when block > 1: the fibers of the
 * mode-n unfolding are grouped, in their Eq. (2) order, into blocks of
 * `block` consecutive columns: an aligned range of the fastest-varying other
 * mode k0 (the first mode other than n) with every other index fixed; block
 * must divide I_1, I_2 and B. The batch is B / block sampled blocks, with
 * replacement. Block beta draws each index of the modes k != n once, from the
 * word of (t, beta, k), by the draw above; for k0 the drawn row stands for its
 * block, so the block is drawn with the sum of its rows' probabilities. The
 * block's fiber u (u < block) takes row (r / block) block + u of k0 and is
 * batch slot beta block + u. Every fiber of a block carries the block's
 * probability p_b (k0's factor q_blk / Q with q_blk the block's exact sum of
 * q_i), and Eq. (11)'s 1/B becomes 1/(B / block), one term per sampled block:
 * E[G] is still the full gradient / J_n. block = 1 is the per-fiber method.
 *
 * Conventions (0-based in code, the paper is 1-based):
 *  - X dense, column-major (first index fastest): entry (i_0..i_{N-1}) at
 *    offset sum_k i_k S_k with S_k = prod_{m<k} I_m.  This is the order in
 *    which Eq. (2) enumerates the columns j of the mode-n unfolding.
 *  - A^(k) row-major I_k x R (double).
 *  - idx is B x N row-major; column n (the drawn mode) is left as -1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 8

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_EDEGENERATE = 6 };
enum { ORC_SAMPLE_EUCLIDEAN = 0, ORC_SAMPLE_LEVERAGE = 1, ORC_SAMPLE_UNIFORM = 2 };
enum { ORC_STEP_FIXED = 0, ORC_STEP_ADAGRAD = 1, ORC_STEP_DECAY = 2 };
enum { ORC_X_F64 = 0, ORC_X_F32 = 1, ORC_X_BF16 = 2 };
enum { ORC_CONSTRAINT_NONE = 0, ORC_CONSTRAINT_NONNEG = 1 };

typedef struct {
    int32_t N;
    int32_t R;
    int32_t B;
    int32_t sampling;
    int32_t step;
    int32_t x_dtype;
    int64_t dims[ORC_MAXN];
    double alpha;  /* fixed step (Eq. (12))                 */
    double eta;    /* AdaGrad eta (Eq. (13a))                  */
    double b;      /* AdaGrad b   (Eq. (13a))                  */
    double beta;   /* decreasing step alpha_t = beta/(t+gamma)  */
    double gamma;  /*   (Thm 9)                                 */
    uint64_t seed;
    int32_t constraint;  /* ORC_CONSTRAINT_*                         */
    int32_t block;       /* Remark 1: fibers per sampled block (1: per fiber) */
} orc_cfg;

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).                   */
/* ------------------------------------------------------------------ */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL; /* golden ratio    */
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL; /* sqrt(3) - 1     */

static uint64_t mulhi64(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t hi0 = mulhi64(PHILOX_M0, c0), lo0 = PHILOX_M0 * c0;
        uint64_t hi1 = mulhi64(PHILOX_M1, c2), lo1 = PHILOX_M1 * c2;
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random word for the draw of fiber f in mode k at iteration t. */
uint64_t orc_fiber_word(uint64_t seed, int64_t t, int64_t f, int k)
{
    uint64_t ctr[4] = {(uint64_t)t, (uint64_t)f, (uint64_t)(k >> 2), 0};
    uint64_t key[2] = {seed, 0};
    uint64_t out[4];
    orc_philox4x64(ctr, key, out);
    return out[k & 3];
}

/* Alg. 4/5: the mode of the iteration is drawn uniformly among the N modes (0-based here). */
int32_t orc_mode_draw(uint64_t seed, int64_t t, int32_t N)
{
    uint64_t ctr[4] = {(uint64_t)t, ~0ULL, 0, 1};
    uint64_t key[2] = {seed, 0};
    uint64_t out[4];
    orc_philox4x64(ctr, key, out);
    return (int32_t)mulhi64(out[0], (uint64_t)N);
}

/* ------------------------------------------------------------------ */
/* Per-factor row weights (Sec. 3.1).                                   */
/* ------------------------------------------------------------------ */

/* Def. 5 / Lemma 4 (beta = 1): w_i = ||A(i,:)||_2^2, canonical tree order. */
void orc_weights_euclidean(const double *A, int64_t I, int32_t R, double *w)
{
    for (int64_t i = 0; i < I; ++i) {
        double part[32];
        for (int p = 0; p < 32; ++p) {
            double acc = 0.0;
            for (int32_t r = p; r < R; r += 32)
                acc = fma(A[i * R + r], A[i * R + r], acc);
            part[p] = acc;
        }
        for (int off = 16; off >= 1; off >>= 1)
            for (int p = 0; p < off; ++p)
                part[p] = part[p] + part[p + off];
        w[i] = part[0];
    }
}

/* Gram entry g_rs = sum_i a_ir a_is in the canonical 32-partial order. */
static double gram_entry(const double *A, int64_t I, int32_t R, int32_t r, int32_t s)
{
    double part[32];
    for (int p = 0; p < 32; ++p) {
        double acc = 0.0;
        for (int64_t i = p; i < I; i += 32)
            acc = fma(A[i * R + r], A[i * R + s], acc);
        part[p] = acc;
    }
    for (int off = 16; off >= 1; off >>= 1)
        for (int p = 0; p < off; ++p)
            part[p] = part[p] + part[p + off];
    return part[0];
}

/*
 * Def. 3: leverage score l_i(A) = ||Q(i,:)||^2 for an orthonormal basis Q of
 * range(A). With A^T A = L L^T (Cholesky), Q = A L^{-T} is such a basis, so
 * l_i = ||L^{-1} a_i||^2. Returns ORC_EDEGENERATE when the Gram matrix is not
 * numerically positive definite -- a Cholesky pivot at or below 2^-40 times
 * its diagonal entry -- i.e. A not of full column rank, the setting Def. 3
 * and Lemma 1 assume.
 */
int orc_weights_leverage(const double *A, int64_t I, int32_t R, double *w)
{
    double *g = (double *)calloc((size_t)R * R, sizeof(double));
    double *L = (double *)calloc((size_t)R * R, sizeof(double));
    double *inv = (double *)calloc((size_t)R, sizeof(double));
    double *y = (double *)calloc((size_t)R, sizeof(double));
    int status = ORC_OK;
    for (int32_t r = 0; r < R; ++r)
        for (int32_t s = r; s < R; ++s) {
            double v = gram_entry(A, I, R, r, s);
            g[r * R + s] = v;
            g[s * R + r] = v;
        }
    for (int32_t j = 0; j < R && status == ORC_OK; ++j) {
        double d = g[j * R + j];
        for (int32_t k = 0; k < j; ++k)
            d = fma(-L[j * R + k], L[j * R + k], d);
        /* Not numerically of full column rank: pivot below 2^-40 g_jj. */
        if (!(d > 0x1.0p-40 * g[j * R + j])) {
            status = ORC_EDEGENERATE;
            break;
        }
        L[j * R + j] = sqrt(d);
        inv[j] = 1.0 / L[j * R + j];
        for (int32_t i = j + 1; i < R; ++i) {
            double v = g[i * R + j];
            for (int32_t k = 0; k < j; ++k)
                v = fma(-L[i * R + k], L[j * R + k], v);
            L[i * R + j] = v * inv[j];
        }
    }
    if (status == ORC_OK) {
        for (int64_t i = 0; i < I; ++i) {
            double acc = 0.0;
            for (int32_t j = 0; j < R; ++j) {
                double v = A[i * R + j];
                for (int32_t k = 0; k < j; ++k)
                    v = fma(-L[j * R + k], y[k], v);
                y[j] = v * inv[j];
                acc = fma(y[j], y[j], acc);
            }
            w[i] = acc;
        }
    }
    free(g); free(L); free(inv); free(y);
    return status;
}

static int ceil_log2_i64(int64_t v)
{
    int L = 0;
    while (((int64_t)1 << L) < v)
        ++L;
    return L;
}

/*
 * Fixed-point sampling distribution of one factor from its row weights:
 * q_i = floor(w_i 2^s) with s = 61 - ceil(log2 I) - floor(log2 max w), and
 * cdf[i] = q_0 + ... + q_i (exact). Returns ORC_EDEGENERATE when a weight is
 * negative or not finite, or when every q_i is 0.
 */
int orc_distribution(const double *w, int64_t I, uint64_t *cdf)
{
    double wmax = 0.0;
    for (int64_t i = 0; i < I; ++i) {
        if (!(w[i] >= 0.0) || isinf(w[i]))
            return ORC_EDEGENERATE;
        if (w[i] > wmax)
            wmax = w[i];
    }
    if (wmax == 0.0)
        return ORC_EDEGENERATE;
    int e;
    frexp(wmax, &e);                 /* wmax in [2^(e-1), 2^e) */
    const int s = 61 - ceil_log2_i64(I) - (e - 1);
    uint64_t acc = 0;
    for (int64_t i = 0; i < I; ++i) {
        acc += (uint64_t)floor(ldexp(w[i], s));
        cdf[i] = acc;
    }
    return acc > 0 ? ORC_OK : ORC_EDEGENERATE;
}

/* Inverse-CDF draw (Def. 2): smallest i with floor(x Q / 2^64) < cdf[i]. */
int64_t orc_draw(const uint64_t *cdf, int64_t I, uint64_t x)
{
    const uint64_t target = mulhi64(x, cdf[I - 1]);
    for (int64_t i = 0; i < I; ++i)
        if (target < cdf[i])
            return i;
    return I - 1;
}

/* p_k(i) = q_i / Q, as doubles. */
double orc_prob(const uint64_t *cdf, int64_t I, int64_t i)
{
    const uint64_t q = cdf[i] - (i > 0 ? cdf[i - 1] : 0);
    return (double)q / (double)cdf[I - 1];
}

/* Row weights of one factor for the configured distribution. */
int orc_weights(int32_t sampling, const double *A, int64_t I, int32_t R, double *w)
{
    if (sampling == ORC_SAMPLE_LEVERAGE)
        return orc_weights_leverage(A, I, R, w);
    if (sampling == ORC_SAMPLE_EUCLIDEAN) {
        orc_weights_euclidean(A, I, R, w);
        return ORC_OK;
    }
    for (int64_t i = 0; i < I; ++i)
        w[i] = 1.0;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Tensor access (Eq. (2)) and the sampled KRP (Alg. 1).                */
/* ------------------------------------------------------------------ */

static double x_at(const void *X, int32_t dtype, int64_t off)
{
    if (dtype == ORC_X_F64)
        return ((const double *)X)[off];
    if (dtype == ORC_X_F32)
        return (double)((const float *)X)[off];
    uint32_t bits = (uint32_t)((const uint16_t *)X)[off] << 16;
    float f;
    memcpy(&f, &bits, sizeof f);
    return (double)f;
}

/* Eq. (2): column j of X_(n) for the multi-index idx (idx[n] ignored). */
int64_t orc_unfold_col(int32_t N, const int64_t *dims, int32_t n, const int64_t *idx)
{
    int64_t j = 0, Jp = 1;
    for (int32_t k = 0; k < N; ++k) {
        if (k == n)
            continue;
        j += idx[k] * Jp;
        Jp *= dims[k];
    }
    return j;
}

/* Alg. 1: the sampled fiber of X through the multi-index idx (mode n free), i.e. one column of X_(n). */
void orc_gather_fiber(const void *X, int32_t dtype, int32_t N, const int64_t *dims,
                      int32_t n, const int64_t *idx, double *x)
{
    int64_t base = 0, S = 1, Sn = 1;
    for (int32_t k = 0; k < N; ++k) {
        if (k == n)
            Sn = S;
        else
            base += idx[k] * S;
        S *= dims[k];
    }
    for (int64_t i = 0; i < dims[n]; ++i)
        x[i] = x_at(X, dtype, base + i * Sn);
}

/* Eq. (3): Z^(n)(j,:) = Hadamard product of A^(k)(i_k,:), k != n. */
void orc_krp_row(int32_t N, int32_t R, int32_t n, const double *const *A,
                 const int64_t *idx, double *z)
{
    for (int32_t r = 0; r < R; ++r)
        z[r] = 1.0;
    for (int32_t k = 0; k < N; ++k) {
        if (k == n)
            continue;
        for (int32_t r = 0; r < R; ++r)
            z[r] = z[r] * A[k][idx[k] * R + r];
    }
}

/* ------------------------------------------------------------------ */
/* Alg. 3 (SKRP-ST-I): draw the mini-batch and its probabilities.       */
/* ------------------------------------------------------------------ */

static int64_t j_count(const orc_cfg *c, int32_t n)
{
    int64_t J = 1;
    for (int32_t k = 0; k < c->N; ++k)
        if (k != n)
            J *= c->dims[k];
    return J;
}

/*
 * Per-factor weights w_k and CDFs cdf_k for every k != n, from the current
 * factors. w and cdf are arrays of N pointers to buffers of I_k doubles.
 */
static int build_distributions(const orc_cfg *c, int32_t n, const double *const *A,
                               double **w, uint64_t **cdf)
{
    for (int32_t k = 0; k < c->N; ++k) {
        if (k == n)
            continue;
        int st = orc_weights(c->sampling, A[k], c->dims[k], c->R, w[k]);
        if (st != ORC_OK)
            return st;
        st = orc_distribution(w[k], c->dims[k], cdf[k]);
        if (st != ORC_OK)
            return st;
    }
    return ORC_OK;
}

/* Blocks (Remark 1): the mode whose rows form the blocks of mode n's fibers. */
static int32_t block_mode(int32_t n) { return n == 0 ? 1 : 0; }

static int32_t block_of(const orc_cfg *c) { return c->block > 1 ? c->block : 1; }

/* Eq. (10): p_f as the product of the per-factor probabilities; with blocks,
 * k0's factor is the probability of the block of rows that holds i_k0. */
static double fiber_probability(const orc_cfg *c, int32_t n, const int64_t *idx,
                                uint64_t *const *cdf)
{
    const int32_t bs = block_of(c), k0 = block_mode(n);
    double p = 1.0;
    for (int32_t k = 0; k < c->N; ++k) {
        if (k == n)
            continue;
        if (bs > 1 && k == k0) {
            const int64_t b = idx[k] / bs;
            const uint64_t hi = cdf[k][(b + 1) * bs - 1];
            const uint64_t lo = b > 0 ? cdf[k][b * bs - 1] : 0;
            p = p * ((double)(hi - lo) / (double)cdf[k][c->dims[k] - 1]);
        } else {
            p = p * orc_prob(cdf[k], c->dims[k], idx[k]);
        }
    }
    return p;
}

/* block > 1 must divide B and the two modes whose rows can form blocks. */
static int blocks_valid(const orc_cfg *c)
{
    const int32_t bs = block_of(c);
    if (c->block < 0)
        return 0;
    return bs == 1 || (c->B % bs == 0 && c->dims[0] % bs == 0 && c->dims[1] % bs == 0);
}

/*
 * Eq. (11) for a given mini-batch:
 *   H = Z_S^T D Z_S (R x R),  M = X_S D Z_S (I_n x R),
 *   G = (A H - M) / (B J_n),  D = diag(1/p_f).
 * Z_S is B x R row-major, X_S is I_n x B with fiber f contiguous (x_S + f*I_n).
 */
static void gradient_eq11(int64_t In, int32_t R, int32_t B, int64_t Bterms, int64_t Jn, const double *An,
                          const double *Zs, const double *Xs, const double *p, double *G);

void orc_gradient(int64_t In, int32_t R, int32_t B, int64_t Jn, const double *An,
                  const double *Zs, const double *Xs, const double *p, double *G)
{
    gradient_eq11(In, R, B, B, Jn, An, Zs, Xs, p, G);
}

/* Eq. (11) over B fibers whose 1/B is 1/Bterms (B / block with blocks). */
static void gradient_eq11(int64_t In, int32_t R, int32_t B, int64_t Bterms, int64_t Jn, const double *An,
                          const double *Zs, const double *Xs, const double *p, double *G)
{
    double *H = (double *)calloc((size_t)R * R, sizeof(double));
    double *M = (double *)calloc((size_t)In * R, sizeof(double));
    /* every entry of H and M sums its terms over f = 0, 1, ..., B-1 in order */
    for (int32_t f = 0; f < B; ++f) {
        double d = 1.0 / p[f];
        for (int32_t r = 0; r < R; ++r)
            for (int32_t s = 0; s < R; ++s)
                H[r * R + s] += Zs[f * R + r] * d * Zs[f * R + s];
    }
#ifdef ORC_OMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < In; ++i)
        for (int32_t f = 0; f < B; ++f) {
            double d = 1.0 / p[f];
            for (int32_t r = 0; r < R; ++r)
                M[i * R + r] += Xs[f * In + i] * d * Zs[f * R + r];
        }
    double scale = 1.0 / ((double)Bterms * (double)Jn);
#ifdef ORC_OMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < In; ++i)
        for (int32_t r = 0; r < R; ++r) {
            double ah = 0.0;
            for (int32_t s = 0; s < R; ++s)
                ah += An[i * R + s] * H[s * R + r];
            G[i * R + r] = (ah - M[i * R + r]) * scale;
        }
    free(H);
    free(M);
}

/*
 * Eq. (12) (fixed alpha, or the decreasing alpha_t = beta/(t+gamma) of
 * Thm 9) and Eq. (13a) / (13b) (AdaGrad-style step, accumulator S
 * including the current gradient).
 *
 * Nonnegative variant (Sec. 5, Table 5 / Fig. 2, generalised "as in" Fu et
 * al.'s BrasCPD, whose constrained step is a projected gradient step): after
 * the step every entry is projected onto the constraint set A >= 0, i.e. the
 * Euclidean projection max(0, a). A NaN stays NaN.
 */
static double project(const orc_cfg *c, double a)
{
    if (c->constraint == ORC_CONSTRAINT_NONNEG && a < 0.0) return 0.0;
    return a;
}

void orc_update(const orc_cfg *c, int64_t t, int64_t In, double *An, double *Sn,
                const double *G)
{
    int32_t R = c->R;
    if (c->step == ORC_STEP_ADAGRAD) {
        for (int64_t q = 0; q < In * R; ++q) {
            Sn[q] = Sn[q] + G[q] * G[q];
            double eta = c->eta / sqrt(c->b + Sn[q]);
            An[q] = project(c, An[q] - eta * G[q]);
        }
        return;
    }
    double alpha = c->alpha;
    if (c->step == ORC_STEP_DECAY)
        alpha = c->beta / ((double)t + c->gamma);
    for (int64_t q = 0; q < In * R; ++q)
        An[q] = project(c, An[q] - alpha * G[q]);
}

/*
 * SKRP-ST + gradient for a GIVEN mini-batch idx (B x N row-major, column n
 * ignored), using the probabilities of the current factors. Writes p (B) and
 * G (I_n x R). Used by the enumeration tests of Thm 5 and Thm 10.
 */
int orc_gradient_for_batch(const orc_cfg *c, int32_t n, const int64_t *idx,
                           const void *X, const double *const *A, double *p, double *G)
{
    int32_t N = c->N, R = c->R, B = c->B;
    if (!blocks_valid(c))
        return ORC_EINVAL;
    int64_t In = c->dims[n];
    double *w[ORC_MAXN] = {0};
    uint64_t *cdf[ORC_MAXN] = {0};
    for (int32_t k = 0; k < N; ++k) {
        w[k] = (double *)malloc((size_t)c->dims[k] * sizeof(double));
        cdf[k] = (uint64_t *)malloc((size_t)c->dims[k] * sizeof(uint64_t));
    }
    int st = build_distributions(c, n, A, w, cdf);
    double *Zs = (double *)malloc((size_t)B * R * sizeof(double));
    double *Xs = (double *)malloc((size_t)B * In * sizeof(double));
    if (st == ORC_OK) {
        for (int32_t f = 0; f < B; ++f) {
            const int64_t *row = idx + (int64_t)f * N;
            p[f] = fiber_probability(c, n, row, cdf);
            orc_krp_row(N, R, n, A, row, Zs + (int64_t)f * R);
            orc_gather_fiber(X, c->x_dtype, N, c->dims, n, row, Xs + (int64_t)f * In);
        }
        gradient_eq11(In, R, B, B / block_of(c), j_count(c, n), A[n], Zs, Xs, p, G);
    }
    free(Zs);
    free(Xs);
    for (int32_t k = 0; k < N; ++k) {
        free(w[k]);
        free(cdf[k]);
    }
    return st;
}

/*
 * Alg. 3 (SKRP-ST-I) followed by Alg. 1 (SKRP-ST) for mode n with the random
 * words of iteration t: the per-factor distributions of the current factors,
 * the B x (N-1) draws, the fiber probabilities p_f (Eq. (10)), the sampled
 * KRP rows Z_S (B x R, Eq. (3)) and the sampled fibers X_S (B x I_n, fiber f
 * contiguous, Eq. (2)). idx is B x N with column n = -1. Z and X may be NULL.
 */
int orc_sample_batch(const orc_cfg *c, int32_t n, int64_t t, const void *X, const double *const *A,
                     int64_t *idx, double *p, double *Zs, double *Xs)
{
    int32_t N = c->N, R = c->R, B = c->B;
    if (N < 2 || N > ORC_MAXN || R < 1 || B < 1 || n < 0 || n >= N || !blocks_valid(c))
        return ORC_EINVAL;
    int64_t In = c->dims[n];
    double *w[ORC_MAXN] = {0};
    uint64_t *cdf[ORC_MAXN] = {0};
    for (int32_t k = 0; k < N; ++k) {
        w[k] = (double *)malloc((size_t)c->dims[k] * sizeof(double));
        cdf[k] = (uint64_t *)malloc((size_t)c->dims[k] * sizeof(uint64_t));
    }
    int st = build_distributions(c, n, A, w, cdf);
    if (st == ORC_OK) {
        /* block beta = f / bs draws once per mode; its fiber u = f % bs takes
         * row u of the drawn block of mode k0 (bs = 1: one draw per fiber) */
        const int32_t bs = block_of(c), k0 = block_mode(n);
        for (int32_t f = 0; f < B; ++f) {
            for (int32_t k = 0; k < N; ++k) {
                if (k == n) {
                    idx[(int64_t)f * N + k] = -1;
                    continue;
                }
                const uint64_t x = orc_fiber_word(c->seed, t, f / bs, k);
                const int64_t r = orc_draw(cdf[k], c->dims[k], x);
                idx[(int64_t)f * N + k] = (bs > 1 && k == k0) ? r / bs * bs + f % bs : r;
            }
        }
#ifdef ORC_OMP
#pragma omp parallel for schedule(static)
#endif
        for (int32_t f = 0; f < B; ++f) {
            const int64_t *row = idx + (int64_t)f * N;
            p[f] = fiber_probability(c, n, row, cdf);
            if (Zs)
                orc_krp_row(N, R, n, A, row, Zs + (int64_t)f * R);
            if (Xs)
                orc_gather_fiber(X, c->x_dtype, N, c->dims, n, row, Xs + (int64_t)f * In);
        }
    }
    for (int32_t k = 0; k < N; ++k) {
        free(w[k]);
        free(cdf[k]);
    }
    return st;
}

/*
 * One iteration of BrawsCPD (Alg. 4) / AdawsCPD (Alg. 5) at iteration t:
 * draw n, draw the mini-batch (Alg. 3), form G (Eq. (11)), update
 * A^(n). A and S (AdaGrad accumulators, may be NULL for the other steps)
 * are arrays of N pointers, updated in place. Optional outputs (NULL to
 * skip): n_out; idx_out (B x N, column n = -1); p_out (B); G_out (I_n x R).
 */
int orc_step(const orc_cfg *c, int64_t t, const void *X, double *const *A,
             double *const *S, int32_t *n_out, int64_t *idx_out, double *p_out,
             double *G_out)
{
    int32_t N = c->N, R = c->R, B = c->B;
    if (N < 2 || N > ORC_MAXN || R < 1 || B < 1 || !blocks_valid(c))
        return ORC_EINVAL;
    if (c->step == ORC_STEP_ADAGRAD && !S)     /* Eq. (13a) needs the accumulators */
        return ORC_EINVAL;
    int32_t n = orc_mode_draw(c->seed, t, N);
    int64_t In = c->dims[n];
    int64_t *idx = (int64_t *)malloc((size_t)B * N * sizeof(int64_t));
    double *p = (double *)malloc((size_t)B * sizeof(double));
    double *G = (double *)malloc((size_t)In * R * sizeof(double));
    double *Zs = (double *)malloc((size_t)B * R * sizeof(double));
    double *Xs = (double *)malloc((size_t)B * In * sizeof(double));
    int st = orc_sample_batch(c, n, t, X, (const double *const *)A, idx, p, Zs, Xs);
    if (st == ORC_OK) {
        gradient_eq11(In, R, B, B / block_of(c), j_count(c, n), A[n], Zs, Xs, p, G);
        orc_update(c, t, In, A[n], S ? S[n] : NULL, G);
        if (n_out)
            *n_out = n;
        if (idx_out)
            memcpy(idx_out, idx, (size_t)B * N * sizeof(int64_t));
        if (p_out)
            memcpy(p_out, p, (size_t)B * sizeof(double));
        if (G_out)
            memcpy(G_out, G, (size_t)In * R * sizeof(double));
    }
    free(Zs);
    free(Xs);
    free(idx);
    free(p);
    free(G);
    return st;
}

/* T consecutive iterations t0 .. t0+T-1. Returns the first failing status. */
int orc_run(const orc_cfg *c, int64_t t0, int64_t T, const void *X, double *const *A,
            double *const *S)
{
    for (int64_t t = t0; t < t0 + T; ++t) {
        int st = orc_step(c, t, X, A, S, NULL, NULL, NULL, NULL);
        if (st != ORC_OK)
            return st;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 5.2: relative error Tol = ||[[A]] - X||_F^2 / ||X||_F^2.        */
/* ------------------------------------------------------------------ */

/* CP model entry x_hat(i) = sum_r prod_k A^(k)(i_k, r) (Sec. 1). */
static double cp_entry(int32_t N, int32_t R, const double *const *A, const int64_t *i)
{
    double s = 0.0;
    for (int32_t r = 0; r < R; ++r) {
        double v = 1.0;
        for (int32_t k = 0; k < N; ++k)
            v = v * A[k][i[k] * R + r];
        s += v;
    }
    return s;
}

/* Direct residual sum over every entry. Writes ||X||^2 to xnorm2 if given. */
double orc_tol(int32_t N, const int64_t *dims, int32_t R, const void *X, int32_t dtype,
               const double *const *A, double *xnorm2)
{
    int64_t i[ORC_MAXN] = {0};
    int64_t total = 1;
    for (int32_t k = 0; k < N; ++k)
        total *= dims[k];
    double res = 0.0, xx = 0.0;
    for (int64_t off = 0; off < total; ++off) {
        double x = x_at(X, dtype, off);
        double d = x - cp_entry(N, R, A, i);
        res += d * d;
        xx += x * x;
        for (int32_t k = 0; k < N; ++k) {
            if (++i[k] < dims[k])
                break;
            i[k] = 0;
        }
    }
    if (xnorm2)
        *xnorm2 = xx;
    return res / xx;
}
