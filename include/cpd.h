/*
 * cpd.h -- C ABI of libcpd, a GB300 (sm_103a) implementation of
 * block-randomized weighted SGD with importance sampling for CP
 * decomposition (BrawsCPD, Alg. 4, and AdawsCPD, Alg. 5, of Yu & Li,
 * arXiv 2103.04081).
 *
 * The problem (Sec. 2, Eq. (5)): given a dense N-way tensor X
 * of size I_1 x ... x I_N and a rank R, find factor matrices A^(k) (I_k x R)
 * minimising 1/2 ||X - [[A^(1), ..., A^(N)]]||_F^2. One iteration draws a
 * mode n, draws B mode-n fibers by Euclidean- or leverage-based importance
 * sampling (Alg. 3, Lemmas 2 and 4), forms the sampled Khatri-Rao rows and
 * fibers (Alg. 1), the weighted stochastic gradient (Eq. (11)) and
 * updates A^(n) with a fixed (Eq. (12)), decreasing (Thm 9) or
 * AdaGrad-style step (Eq. (13a) / (13b)).
 *
 * Conventions for every entry point:
 *  - Indices are 0-based; the paper's are 1-based.
 *  - X is dense and column-major (first index fastest): entry
 *    (i_1, ..., i_N) sits at element offset sum_k i_k * prod_{m<k} I_m,
 *    the order in which Eq. (2) numbers the columns of each unfolding.
 *  - A factor matrix A^(k) is row-major I_k x R (row i contiguous).
 *    Factors are double when x_dtype is CPD_F64 and float otherwise.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy stream).
 *    Calls are ordered on that stream; a call that returns host data
 *    synchronises it first.
 *  - A location flag is CPD_HOST (pageable or pinned host memory) or
 *    CPD_DEVICE (memory of the current CUDA device).
 *  - Every call returns a cpd_status. On failure nothing is half-done
 *    from the caller's point of view, and cpd_last_error() returns a
 *    thread-local message. No C++ exception crosses the ABI.
 *  - The library never falls back to the CPU: without a usable sm_103a
 *    device, cpd_init returns CPD_ECUDA.
 */
#ifndef CPD_H
#define CPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPD_MAX_MODES 8

typedef enum {
    CPD_OK = 0,
    CPD_EINVAL = 1,       /* invalid argument or configuration            */
    CPD_ENOMEM = 2,       /* device allocation failed / over the budget   */
    CPD_ECUDA = 3,        /* CUDA runtime or driver error                 */
    CPD_ETIMEOUT = 4,     /* a bounded device wait gave up                */
    CPD_ENONFINITE = 5,   /* a gradient or factor became NaN / Inf        */
    CPD_EDEGENERATE = 6,  /* a sampling distribution has no mass, or a
                             leverage Gram matrix is not of full rank     */
    CPD_EAGAIN = 7,       /* cpd_poll: request not finished yet           */
    CPD_EBUSY = 8         /* server full; retry later                     */
} cpd_status;

enum { CPD_HOST = 0, CPD_DEVICE = 1 };

/* Importance-sampling distribution of the per-factor row draws (Sec. 3.1). */
enum {
    CPD_SAMPLE_EUCLIDEAN = 0, /* p_k(i) = ||A^(k)(i,:)||^2 / ||A^(k)||_F^2, Lemma 4   */
    CPD_SAMPLE_LEVERAGE = 1,  /* p_k(i) = l_i(A^(k)) / sum_i l_i, Lemma 2           */
    CPD_SAMPLE_UNIFORM = 2    /* p_k(i) = 1 / I_k: BrasCPD / AdasCPD (Alg. 2)       */
};

/* Step rule (Sec. 3.2). */
enum {
    CPD_STEP_FIXED = 0,   /* A -= alpha G                      (Eq. (12))   */
    CPD_STEP_ADAGRAD = 1, /* S += G.^2; A -= eta G ./ sqrt(b + S) (Eq. (13a)/(13b)) */
    CPD_STEP_DECAY = 2    /* A -= beta / (t + gamma) G            (Thm 9)        */
};

/* Storage type of the tensor entries. */
enum { CPD_F64 = 0, CPD_F32 = 1, CPD_BF16 = 2 };

/* Constraint on the factors (Sec. 5, Table 5 / Fig. 2: the nonnegative
 * variant, generalised as in Fu et al.'s BrasCPD): after every step the
 * updated entries are projected onto the constraint set. */
enum {
    CPD_CONSTRAINT_NONE = 0,
    CPD_CONSTRAINT_NONNEG = 1   /* a <- max(0, a) after the step (NaN kept)  */
};

/* Where the sampled fibers are read from (cpd_config.x_layout). */
typedef enum {
    CPD_LAYOUT_REPLICAS = 0,    /* one mode-major replica per mode: every mode-n
                                   fiber contiguous (N copies of X)             */
    CPD_LAYOUT_STRIDED = 1      /* the mode-1 replica alone (X column-major, the
                                   first mode padded to a multiple of 8): a
                                   mode-n fiber (Eq. (2)) is read from it with
                                   stride ld_1 I_2 ... I_{n-1}; CUDA-core engine
                                   only                                         */
} cpd_layout;

typedef struct {
    int32_t N;          /* number of modes, 3 <= N <= CPD_MAX_MODES                 */
    int32_t R;          /* CP rank, 1 <= R <= 256                                   */
    int32_t B;          /* mini-batch size |F_n|, 1 <= B <= 65536                    */
    int32_t sampling;   /* CPD_SAMPLE_*                                             */
    int32_t step;       /* CPD_STEP_*                                               */
    int32_t x_dtype;    /* CPD_F64 / CPD_F32 / CPD_BF16                             */
    int64_t dims[CPD_MAX_MODES]; /* I_1..I_N, each >= 1; leverage needs I_k > R   */
    double alpha;       /* fixed step                                               */
    double eta;         /* AdaGrad eta > 0                                          */
    double b;           /* AdaGrad b >= 0                                           */
    double beta;        /* decreasing step numerator                                */
    double gamma;       /* decreasing step offset (t + gamma > 0)                   */
    uint64_t seed;      /* key of the Philox4x64-10 draws                           */
    int32_t engine;     /* 0 = automatic, 1 = CUDA-core gradient, 2 = tensor-core
                           gradient, one CTA per tile, 3 = tensor-core gradient,
                           one thread-block cluster per fiber group (2 and 3:
                           BF16 tensors, R <= 64; 3: every I_k <= 1024),
                           4 = persistent cluster: one thread-block cluster runs
                           whole calls of cpd_sgd_iters in one launch (BF16
                           tensors, R <= 64, Euclidean or uniform sampling,
                           sum of the I_k <= 4096, ceil(I_max/128) accumulator
                           tiles of <= 64 columns within 512),
                           5 = fused: gradient and step in one launch, one
                           thread-block cluster per 128-row tile of A^(n) whose
                           CTAs split the batch and sum M and H in distributed
                           shared memory in rank order (BF16 tensors, R <= 64,
                           at most 208 fibers per CTA)                          */
    int32_t max_ctas;   /* 0: size the gradient grid for the whole GPU; > 0: use at
                           most about this many CTAs per gradient launch (fewer
                           fiber groups, more fibers per CTA), so that several
                           decompositions share the GPU. Engine 4: the cluster
                           size (1..16; 0 = 8, or less if the device cannot
                           co-schedule 8). Engine 5: the cluster size (0, 1, 2,
                           4, 8 or 16; 0 = the smallest that leaves a CTA at
                           most 64 fibers, up to 16). Part of the arithmetic: the grouping
                           of the batch fixes the summation order of the
                           gradient partials.                                   */
    int32_t constraint; /* CPD_CONSTRAINT_*                                     */
    int32_t x_layout;   /* CPD_LAYOUT_*: replicas (0) or the mode-1 replica alone
                           (1, N times less memory, strided gathers for n > 1)  */
    int32_t tile_rows;  /* rows of A^(n) per gradient CTA (0 = chosen from the
                           shape and max_ctas). CUDA-core engine: a multiple of
                           8 in [8, 512]; tensor-core engines: 0 or 128 (the
                           MMA's M); persistent and fused engines: 0.           */
    int32_t tile_fibers; /* sampled fibers per gradient CTA / fiber group (0 =
                           chosen). CUDA-core engine: [1, B]; tensor-core
                           engines: a multiple of 16 (the MMA's K) in [16, 128]
                           (engine 2) or [16, 256] (engine 3); persistent and
                           fused: 0.
                           Like max_ctas, part of the arithmetic: the fiber
                           groups fix the summation order.                      */
    int32_t block;      /* Remark 1, blocks first and then sampling: 0 or 1 =
                           per-fiber sampling (Alg. 3); bs > 1 = the batch is
                           B / bs sampled blocks of bs consecutive mode-n
                           fibers (Eq. (2) order): an aligned range of bs rows
                           of the first mode other than n, every other index
                           fixed. A block is drawn with the sum of its fibers'
                           probabilities (its row of that mode drawn by
                           Alg. 3 stands for the row's block) and its fibers
                           carry that probability; Eq. (11)'s 1/B becomes
                           1/(B / bs). bs must divide B, I_1 and I_2. Not with
                           the persistent engine, cpd_skrp, cpd_gradients or
                           cpd_grad_variance.                                    */
} cpd_config;

typedef struct cpd_ctx cpd_ctx;

/*
 * cpd_init -- create a decomposition context (the inputs of Alg. 4 / Alg. 5:
 * X, R, |F_n|, A_0, step parameters; Sec. 2 and Sec. 3.2).
 *  cfg   : problem and method parameters (copied).
 *  X     : the dense tensor, column-major, cfg->x_dtype entries, at x_loc.
 *          Copied into device-resident, mode-major replicas owned by the
 *          context (one per mode, so every mode-n fiber is contiguous);
 *          X may be freed after the call returns.
 *  A0    : array of N pointers, A0[k] row-major I_k x R (double for CPD_F64,
 *          float otherwise), at a0_loc. Copied.
 *  out   : receives the context. The iteration counter t starts at 0.
 * Errors: CPD_EINVAL (bad cfg or NULL pointers; nothing is allocated),
 *  CPD_ENOMEM, CPD_ECUDA, CPD_EDEGENERATE (a factor has no sampling mass, or
 *  a leverage Gram matrix is singular). Synchronises `stream` before return.
 */
cpd_status cpd_init(const cpd_config *cfg, const void *X, int x_loc,
                    const void *const *A0, int a0_loc, void *stream, cpd_ctx **out);

/*
 * cpd_sgd_iters -- run `iters` iterations t, t+1, ... of Alg. 4 / Alg. 5
 * (mode draw, SKRP-ST-I of Alg. 3, Eq. (11), the configured step).
 * Asynchronous: enqueued on `stream`; t advances by `iters` on the host
 * immediately. Device-side faults (non-finite values, degenerate
 * distributions) are recorded and reported by the next synchronising call.
 * The random draws of iteration t depend only on (seed, t), so splitting a
 * run into several calls gives bit-identical results.
 */
cpd_status cpd_sgd_iters(cpd_ctx *ctx, int64_t iters, void *stream);

/*
 * cpd_skrp -- Alg. 3 (SKRP-ST-I) followed by Alg. 1 (SKRP-ST), materialised
 * for K mini-batches of mode n: batch b takes the random draws of iteration
 * t0 + b with the mode fixed to n, from the context's current per-factor
 * distributions. Outputs (device memory, each may be NULL):
 *  idx : K*B x N int32, the multi-indices (Eq. (4)), column n = -1;
 *  p   : K*B doubles, p_f of Eq. (10) (FP64, the same bits as the oracle);
 *  Z   : K*B x R floats, the sampled Khatri-Rao rows (Eq. (3)), unweighted;
 *  X   : K*B fibers of the mode-n unfolding (Eq. (2)), fiber f of batch b at
 *        element (b*B + f) * ld_n, ld_n = I_n rounded up to 8 (the padding
 *        entries are 0), in the tensor's storage type.
 * Every SM takes warp blocks of 32 output fibers and streams them in the
 * widest unit (16, 8, 4 or 2 bytes) that divides the fiber length and the
 * addresses of X and the replica: this is the sampled gather on its own, the
 * bandwidth measure of the access pattern. Float factors only (F32 or BF16
 * tensors); X needs only the element alignment of its type.
 * Asynchronous on `stream`. Errors: CPD_EINVAL, CPD_ECUDA.
 */
cpd_status cpd_skrp(cpd_ctx *ctx, int32_t n, int64_t t0, int32_t K, int32_t *idx, double *p, float *Z, void *X,
                    void *stream);

/*
 * cpd_gradients -- K independent mini-batch gradients of mode n at the
 * current factors (Eq. (11), each batch drawn by Alg. 3 from the current
 * per-factor distributions), the samples whose spread Thm 10 and Fig. 3
 * describe. Batch b uses the random draws that iteration t0 + b would use,
 * with the mode fixed to n. G_out: device memory for K x I_n x R floats
 * (batch-major, each gradient row-major). Nothing in the context changes.
 * The batches run concurrently on up to as many thread-block clusters as
 * the device co-schedules; this is also how the fiber gather is measured in
 * bulk (K B fibers per launch). Asynchronous on `stream`. Needs the
 * persistent engine (cpd_config.engine = 4). Errors: CPD_EINVAL, CPD_ENOMEM,
 * CPD_ECUDA.
 */
cpd_status cpd_gradients(cpd_ctx *ctx, int32_t n, int64_t t0, int32_t K, float *G_out, void *stream);

/*
 * cpd_prepare -- capture ahead of time the CUDA graphs that a later
 * cpd_sgd_iters(ctx, iters, stream) replays (chunks of 32 iterations and one
 * chunk per set bit of iters mod 32), so that call pays no capture. Runs no
 * iteration and leaves t unchanged. The paper has no counterpart: graph
 * capture is how this library keeps launch overhead off the iteration loop.
 * Errors: CPD_EINVAL (NULL context, iters < 0), CPD_ECUDA.
 */
cpd_status cpd_prepare(cpd_ctx *ctx, int64_t iters, void *stream);

/*
 * cpd_fit -- relative error of Sec. 5.2, Tol = ||[[A]] - X||_F^2 / ||X||_F^2,
 * by one pass over the whole tensor with FP64 accumulation; fit = 1 - sqrt(Tol).
 * Either output pointer may be NULL. Synchronises `stream`; returns a
 * pending device fault (CPD_ENONFINITE, CPD_EDEGENERATE) if one occurred.
 */
cpd_status cpd_fit(cpd_ctx *ctx, double *fit, double *tol, void *stream);

/*
 * cpd_fit_start / cpd_fit_poll -- the same Tol as cpd_fit without blocking:
 * cpd_fit_start enqueues the full-tensor pass on `stream` and returns;
 * cpd_fit_poll returns CPD_EAGAIN until that pass has finished, then the
 * fit and Tol of the most recent cpd_fit_start (either pointer may be NULL).
 */
cpd_status cpd_fit_start(cpd_ctx *ctx, void *stream);
cpd_status cpd_fit_poll(cpd_ctx *ctx, double *fit, double *tol);

/*
 * cpd_get_factors / cpd_set_factors -- copy the N factor matrices out of / into
 * the context (the output of Alg. 4 / Alg. 5). `A` is an array of N pointers,
 * each I_k x R row-major in the factor type, at `loc`. Setting factors
 * rebuilds every sampling distribution. cpd_get_factors with CPD_HOST
 * synchronises `stream`.
 */
cpd_status cpd_get_factors(cpd_ctx *ctx, void *const *A, int loc, void *stream);
cpd_status cpd_set_factors(cpd_ctx *ctx, const void *const *A, int loc, void *stream);

/*
 * cpd_get_adagrad / cpd_set_adagrad -- the FP64 accumulators S^(k)
 * (I_k x R row-major) of Eq. (13a), for checkpoint and resume.
 */
cpd_status cpd_get_adagrad(cpd_ctx *ctx, double *const *S, int loc, void *stream);
cpd_status cpd_set_adagrad(cpd_ctx *ctx, const double *const *S, int loc, void *stream);

/* cpd_get_iteration / cpd_set_iteration -- the iteration counter t. */
cpd_status cpd_get_iteration(cpd_ctx *ctx, int64_t *t);
cpd_status cpd_set_iteration(cpd_ctx *ctx, int64_t t);

/*
 * cpd_last_sample -- the mini-batch of the most recent iteration (Eq. (4),
 * Eq. (10)): its mode n, idx (B x N row-major int32, column n set
 * to -1) and the fiber probabilities p_f (B doubles). Host outputs; any may
 * be NULL. Synchronises `stream`. Returns CPD_EINVAL before the first
 * iteration.
 */
cpd_status cpd_last_sample(cpd_ctx *ctx, int32_t *n, int32_t *idx, double *p, void *stream);

/*
 * cpd_last_gradient -- G^(n) of the most recent iteration (Eq. (11)),
 * I_n x R row-major in the factor type, copied to host memory `G`.
 * Synchronises `stream`.
 */
cpd_status cpd_last_gradient(cpd_ctx *ctx, void *G, void *stream);

/*
 * cpd_grad_variance -- the exact conditional variance of the mini-batch
 * gradient of mode n at the current factors under the context's own
 * sampling distribution (Thm 10, Table 1; the quantity Fig. 3 follows along
 * a run):
 *   var        = E || G - E[G] ||_F^2 = (S1 - ||M||_F^2) / (B J_n^2),
 *   mean_norm2 = || E[G] ||_F^2        = ||M||_F^2 / J_n^2   (may be NULL),
 * with S1 = sum_j ||r_j||^2 ||z_j||^2 / p_j and M = sum_j r_j z_j^T over all
 * J_n fibers j of the mode-n unfolding with p_j > 0, r_j = A^(n) z_j - x_j
 * (Eq. (11)'s normalisation: the paper's Table 1 is J_n^2 times var).
 * One pass over the mode-n replica: residuals in FP32, sums in FP64. A
 * deferred CDF rebuild is completed first. Synchronises `stream`.
 * Errors: CPD_EINVAL (NULL, n out of range, R > 64), CPD_EDEGENERATE,
 * CPD_ENOMEM, CPD_ECUDA.
 */
cpd_status cpd_grad_variance(cpd_ctx *ctx, int32_t n, double *var, double *mean_norm2, void *stream);

/*
 * cpd_sync -- synchronise `stream` and return a pending device fault, if any
 * (CPD_ENONFINITE, CPD_EDEGENERATE, CPD_ETIMEOUT), clearing it.
 */
cpd_status cpd_sync(cpd_ctx *ctx, void *stream);

/*
 * cpd_profile -- enable (1) or disable (0) per-kernel CUDA-event timing,
 * recorded on the launching stream around the gradient kernel and around the
 * rest of each iteration (update, CDF refresh). cpd_profile_read returns the
 * number of timed iterations and the mean duration (ms) of each part since
 * the last enable, synchronising `stream`. Either output may be NULL.
 */
cpd_status cpd_profile(cpd_ctx *ctx, int enable);
cpd_status cpd_profile_read(cpd_ctx *ctx, int64_t *launches, double *mean_grad_ms,
                            double *mean_update_ms, void *stream);

/*
 * cpd_trace -- enable (1) or disable (0) device-side phase timestamps
 * (%globaltimer, ns) of the iterations that follow; cpd_trace_read copies the
 * 64 stamps of the most recent traced iteration to host memory `out`
 * (synchronising `stream`; 0 = phase not reached). Gradient kernel, first
 * CTA, in the cluster tensor-core engine's order:
 *   0 entry; 1 mbarriers, TMEM and A^(n)-row copy set up; 2 draws done;
 *   26 own fibers' columns and weights; 27 factor-row copies issued;
 *   28 / 10 rows landed; 11 operands built; 22 cluster may exchange;
 *   23 slices sent; 24 partial H formed; 25 / 3 partial-H rows sent;
 *   4 all slices received; 5 gather issued, A^(n) operands converted, owned
 *   H rows summed and sent; 14 all H rows received; 15 H operands converted,
 *   cluster barrier passed; 6 A H_g products issued; 7 accumulator complete;
 *   8 G_g stored; 9 exit.
 * Fused engine (one launch per iteration), first CTA: 0 entry; 15 set up;
 *   1 draws done; 2 columns and weights; 16 X gather issued; 3 operands
 *   built; 4 gather landed; 5 products complete; 6
 *   partials in shared memory; 7 first cluster barrier; 8 owned rows of H
 *   summed; 9 second cluster barrier; 10 H complete; 17 owned rows of M
 *   summed, G and the step written (18 / 19: the first thread's A^(n) H
 *   formed / its M summed); 11 row weights written; 12 / 13 last CTA's
 *   bookkeeping start / end; 14 exit.
 * Every engine's sampler (first CTA): 29 CDFs staged in shared memory, 30
 *   deferred CDF rebuilt; the cluster engine: 31 first fiber's weight.
 * The other gradient engines use slots 0-15 for their own phases in the
 * same spirit. Update kernel: 16 entry, 17 gradient reduced, 18 step
 * applied, 19 row weights written (first CTA); 20 / 21 distribution
 * rebuild start / end (last CTA).
 */
cpd_status cpd_trace(cpd_ctx *ctx, int enable);
cpd_status cpd_trace_read(cpd_ctx *ctx, uint64_t *out, void *stream);

/*
 * cpd_describe -- launch configuration chosen for the context, as a
 * NUL-terminated JSON string in `buf` (at most `len` bytes).
 */
cpd_status cpd_describe(cpd_ctx *ctx, char *buf, size_t len);

/*
 * cpd_tol_noalloc -- the relative error Tol = ||[[A]] - X||_F^2 / ||X||_F^2 of
 * a CP model, computed without allocating any device memory. The paper has no
 * counterpart: this entry point serves callers that cannot call cudaMalloc --
 * a program whose device memory is owned by another allocator (a framework's
 * caching pool, or a service that reserves all memory up front), or a loop
 * that cannot afford the device synchronisation an allocation may cause.
 *  N, dims, R : tensor order, sizes I_1..I_N and rank (3 <= N <= 8, R <= 256).
 *  x_dtype    : CPD_F64 / CPD_F32 / CPD_BF16.
 *  X          : device pointer to the dense tensor, column-major, unpadded.
 *  A          : host array of N device pointers, A[k] row-major I_k x R,
 *               double for CPD_F64 and float otherwise.
 *  tol_out    : device pointer to one double, written in stream order.
 * Limit: at most 1,048,576 mode-1 fibers (I_2 * ... * I_N <= 2^20); larger
 * tensors return CPD_EINVAL (use cpd_fit). Scratch: a 1 MiB array that the
 * library image places in the memory of every GPU that loads it, held until
 * the process exits. Every call looks up that array's device address on the
 * calling device (cudaGetSymbolAddress); the first call on a device may load
 * the library's device code, so make it before any stream capture on the
 * device. Every call reuses the same array, so calls that overlap on the GPU
 * (e.g. on two streams at once) race: serialise them. Each call overwrites
 * every scratch slot it reads. A tensor with ||X|| = 0 has no relative
 * error: tol_out then receives NaN (cpd_init rejects such a tensor).
 */
cpd_status cpd_tol_noalloc(int32_t N, const int64_t *dims, int32_t R, int32_t x_dtype,
                           const void *X, const void *const *A, double *tol_out, void *stream);

/*
 * Serving: many decompositions on one GPU. A server admits submitted
 * requests (each one a full run of Alg. 4 / Alg. 5 until a fit target or an
 * iteration cap, Sec. 5.2 stopping rule) first-fit against a device-memory
 * budget and a limit on concurrent requests, runs every admitted request on
 * a stream of its own so that their kernels overlap, checks each request's
 * fit every fit_every iterations without blocking the others, and frees a
 * request's memory as soon as it stops. A request's results do not depend on
 * what else runs: every kernel's arithmetic is independent of the mix.
 * Throughput: give requests a CTA cap (cpd_config.max_ctas, e.g. 8) so that
 * many fit on the GPU at once, and let the process use 32 hardware work
 * queues (environment CUDA_DEVICE_MAX_CONNECTIONS=32, set before the CUDA
 * context is created); with the default 8, streams share queues and
 * serialise.
 */
typedef struct cpd_server cpd_server;

typedef struct {
    size_t hbm_budget;    /* device bytes admitted requests may hold
                             (0: 85% of the free memory at creation)          */
    int32_t max_active;   /* requests running at once (0: 32)                  */
    int32_t fit_every;    /* iterations between fit checks (0: 250; a multiple
                             of 32 keeps every iteration in replayed graphs)  */
    int32_t no_grouping;  /* 0: requests that use the CUDA-core, per-CTA
                             tensor-core or persistent engine run
                             in grouped launches (cpd_group_*), one group per
                             lane of same-dtype, same-engine requests; others
                             run on streams of their own. 1: every request on
                             a stream of its own.                             */
    int32_t strided_above_mb; /* a request whose mode-major replicas would hold
                             more than this many MiB runs with one strided copy
                             of X on the CUDA-core engine (CPD_LAYOUT_STRIDED;
                             0: only when the replicas exceed the budget)     */
} cpd_server_config;

typedef struct {
    int32_t status;       /* CPD_OK, or the failure that stopped the request   */
    int32_t done;         /* 1 once the request has stopped                    */
    int32_t reached;      /* 1 when the fit target was reached                 */
    int32_t layout;       /* CPD_LAYOUT_* the request runs with (the server
                             falls back to the strided layout, see cpd_submit) */
    int64_t iters;        /* iterations run                                    */
    double fit, tol;      /* at the last check (Sec. 5.2)                      */
    double t_submit, t_start, t_done; /* seconds on the server's clock; t_start:
                             admitted and its own copy of X made (the caller
                             may release X and A0 from then on)               */
} cpd_result;

/* cpd_server_create -- a server on the current CUDA device (one worker thread). */
cpd_status cpd_server_create(const cpd_server_config *cfg, cpd_server **out);

/*
 * cpd_submit -- queue one decomposition: cfg, X and A0 as for cpd_init (X and
 * A0 must stay valid until the request has started: cpd_poll reports
 * t_start > 0); it stops when fit >= stop_fit or after max_iters iterations.
 * Returns its ticket. A request whose mode-major replicas would exceed the
 * budget (or cpd_server_config.strided_above_mb) runs with
 * CPD_LAYOUT_STRIDED on the CUDA-core engine instead (one copy of X; the
 * decision depends only on the request and the server's configuration, so
 * a request's arithmetic never depends on the load).
 * CPD_ENOMEM if the request can never fit the budget.
 */
cpd_status cpd_submit(cpd_server *srv, const cpd_config *cfg, const void *X, int x_loc,
                      const void *const *A0, int a0_loc, double stop_fit, int64_t max_iters,
                      uint64_t *ticket);

/*
 * cpd_poll -- the state of a request; CPD_EAGAIN while it runs or waits (out
 * is still filled). Once done, returns its status and, if A_out is not NULL,
 * copies its N factor matrices into the host buffers A_out[k] (I_k x R).
 */
cpd_status cpd_poll(cpd_server *srv, uint64_t ticket, cpd_result *out, void *const *A_out);

/*
 * cpd_server_stats -- the server's budget, the bytes its admitted requests
 * hold, and how many requests run and wait (any pointer may be NULL).
 */
cpd_status cpd_server_stats(cpd_server *srv, size_t *budget, size_t *held, int32_t *active, int32_t *queued);

/* cpd_server_wait -- block until every submitted request is done, or
 * CPD_EAGAIN after timeout_s seconds (timeout_s <= 0: no limit). */
cpd_status cpd_server_wait(cpd_server *srv, double timeout_s);

/* cpd_server_destroy -- stop the worker (running requests are abandoned) and free. */
cpd_status cpd_server_destroy(cpd_server *srv);

/* cpd_destroy -- free the context and everything it owns. NULL is a no-op. */
cpd_status cpd_destroy(cpd_ctx *ctx);

/*
 * cpd_autotune -- choose the gradient engine, CTA cap and tile shape for a
 * problem by timing. The paper has no counterpart: the launch shape is this
 * library's choice, and it fixes the summation order of the gradient, so it
 * is made once, explicitly, and handed back as a configuration. Runs built
 * from `best` are reproducible; only the choice itself depends on timing.
 *  cfg, X, x_loc, A0, a0_loc: as for cpd_init. If cfg->engine != 0 only
 *    that engine is timed, at cfg->max_ctas, over its tile shapes; otherwise
 *    every applicable engine (CUDA cores; per-CTA and cluster tensor cores
 *    for BF16 tensors with R <= 64; the fused engine with clusters of 4, 8
 *    and 16 CTAs; the persistent cluster engine where it
 *    applies) with a few CTA caps (cluster sizes) and tile shapes (rows and
 *    fibers per CTA; fibers per fiber group).
 *  iters: timed iterations per candidate (after iters / 4 warm-up ones).
 *  best: receives cfg with engine, max_ctas, tile_rows and tile_fibers set to
 *    the fastest candidate;
 *  best_iters_per_s (may be NULL): its measured rate.
 * Creates and destroys one context per candidate on `stream` (device-wide
 * synchronisation). Errors: those of cpd_init for cfg itself; CPD_ECUDA if
 * no candidate ran.
 */
cpd_status cpd_autotune(const cpd_config *cfg, const void *X, int x_loc, const void *const *A0,
                        int a0_loc, int64_t iters, cpd_config *best, double *best_iters_per_s,
                        void *stream);

/*
 * Groups -- advance many decompositions with one gradient launch and one
 * update launch per iteration (batched execution of Alg. 4 / Alg. 5 over
 * independent problems; the paper runs one problem at a time). Every member
 * runs exactly the CTAs, tiling and arithmetic it runs alone, so after
 * cpd_group_iters(g, T) each member's state is bitwise what cpd_sgd_iters(T)
 * on that context alone gives.
 *
 * cpd_group_create -- group G contexts (array of G distinct handles, borrowed:
 *  they must outlive the group). Members must share the tensor dtype and the
 *  gradient engine, which must be the CUDA-core (1), the per-CTA
 *  tensor-core (2) or the persistent (4) engine. Persistent members must
 *  share the cluster size; the group then runs every member's iterations in
 *  ONE launch per call, one thread-block cluster per member. The other
 *  engines use one gradient and one update launch per iteration, plus one
 *  Gram and one leverage-row launch when any member samples by leverage
 *  (members that do not take no CTAs of those). The members' launch state is captured at
 *  creation (later cpd_trace / cpd_profile changes do not reach the group).
 *  Allocates about a kilobyte per member on `stream` and synchronises it.
 *  Errors: CPD_EINVAL (NULL, duplicate or incompatible members), CPD_ENOMEM,
 *  CPD_ECUDA.
 * cpd_group_iters -- run `iters` iterations of every member, enqueued on
 *  `stream` (graph-replayed chunks). Asynchronous. The caller orders this
 *  stream after any work still pending on the members' own streams, and
 *  the members' later calls (cpd_fit, cpd_get_factors, ...) after it.
 * cpd_group_destroy -- synchronise the last stream the group used and free
 *  it; the member contexts are untouched.
 */
typedef struct cpd_group cpd_group;
cpd_status cpd_group_create(cpd_ctx *const *ctxs, int32_t G, void *stream, cpd_group **out);
cpd_status cpd_group_iters(cpd_group *group, int64_t iters, void *stream);
cpd_status cpd_group_destroy(cpd_group *group);

/* Thread-local description of the last failure on this thread. */
const char *cpd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CPD_H */
