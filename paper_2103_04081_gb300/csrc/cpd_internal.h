// Internal declarations of libcpd shared by its translation units.
//
// Device-resident state of one decomposition (all of it lives in HBM for the
// whole run; the host only launches work):
//   rep[k]   mode-k-major replica of X: fiber j of the mode-k unfolding
//            (Eq. (2) numbering) is contiguous at rep[k] + j * ld[k], so
//            every sampled fiber is one contiguous, 16-byte-aligned run.
//   A[k]     factor A^(k), row-major I_k x R, in the factor type T.
//   S[k]     AdaGrad accumulators (FP64), Eq. (13a).
//   w[k]     FP64 row weights (squared row norms or leverage scores).
//   cdf[k]   FP64 inclusive prefix sums of w[k] in the canonical order.
//   t_dev    the iteration counter; every kernel derives the mode n and the
//            random draws of its iteration from (seed, *t_dev), so captured
//            launches replay correctly.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cpd.h"

namespace cpd {

constexpr int kMaxModes = CPD_MAX_MODES;
constexpr int kThreads = 256;

// Device status bits, OR-ed into Problem::status and read at sync points.
enum : int { kStNonFinite = 1, kStDegenerate = 2, kStTimeout = 4 };

// Gradient engines.
enum : int { kEngineSimt = 1, kEngineTensor = 2, kEngineTensorCluster = 3, kEnginePersistent = 4, kEngineFused = 5 };

// Launch tiling of the gradient kernel for one mode n: CTA (gr, gf) handles
// rows [gr*rb, gr*rb+rb) of A^(n) and fibers [gf*fb, gf*fb+fb) of the batch.
struct ModeTile {
    int pr;  // row tiles  = ceil(I_n / rb)
};

template <class T>
struct Problem {
    int N, R, B, sampling, step, x_dtype;
    int constraint;           // CPD_CONSTRAINT_*
    int rb, fb, pf;           // rows per CTA, fibers per CTA, fiber groups
    int cs;                   // CTAs per cluster (clustered tensor-core engine)
    int64_t dims[kMaxModes];
    int64_t ld[kMaxModes];    // fiber stride of replica k (elements, multiple of 8)
    int strided;              // 1: rep[k] is the mode-1 replica for every k (X in
                              // column-major order, the first mode padded to ld[0]);
                              // the other modes' fibers are read from it with a stride
    int block;                // fibers per sampled block (Remark 1; 1: per-fiber sampling)
    int64_t xq[kMaxModes];    // 0-based: prod_{0 < m < n} I_m (1 for modes 0 and 1)
    double Jn[kMaxModes];     // J_n = prod_{k != n} I_k, as a double
    ModeTile tile[kMaxModes];
    const void *rep[kMaxModes];
    T *A[kMaxModes];
    double *S[kMaxModes];
    double *w[kMaxModes];     // FP64 row weights
    unsigned long long *cdf[kMaxModes];  // exact prefix sums of q_i = floor(w_i 2^s)
    float inv_bj[kMaxModes];  // 1 / (B J_n) in FP32
    double alpha, eta, b, beta, gamma;
    unsigned long long seed;
    long long *t_dev;         // iteration counter
    int *n_last;              // mode of the last completed iteration
    int *idx;                 // B x N, last batch (column n = -1)
    double *p;                // B, last batch probabilities
    T *part;                  // gradient partials [pf][I_n][R], one slab per fiber group
    T *G;                     // last gradient, I_n x R row-major
    double *lev_L;            // leverage: Cholesky factor R x R + inverse pivots R
    int *status;              // kSt* bits
    int *dirty;               // mode whose global CDF is stale (-1: none); the next
                              // gradient kernel rebuilds it while staging the CDFs
    int defer_cdf;            // 1: CDF rebuilds are deferred that way
    unsigned *counters;       // last-block arrival counters (zero between launches)
    unsigned long long *trace;  // phase timestamps (cpd_trace), or null
};

// A group of problems advanced by grouped launches: problem g owns CTAs
// [cta_grad[g], cta_grad[g+1]) of the gradient launch and [cta_upd[g],
// cta_upd[g+1]) of the update launch, and runs exactly the CTAs it would run
// alone. All members share T, the tensor dtype and the engine (CUDA-core or
// per-CTA tensor-core), and none samples by leverage.
template <class T>
struct GroupLaunch {
    const Problem<T> *P;      // device array of G problems
    const int *cta_grad;      // device, G + 1 prefix sums
    const int *cta_upd;       // device, G + 1 prefix sums
    const int *cta_gram;      // device, G + 1 prefix sums (leverage members only)
    const int *cta_lev;       // device, G + 1 prefix sums (leverage members only)
    int G, grid_grad, grid_upd, grid_gram, grid_lev, engine, x_dtype;
    size_t smem_grad;         // largest member's dynamic shared memory
    size_t smem_lev;          // largest leverage member's (k_gram / k_lev_rows)
};

// Persistent cluster engine (cpd_pers.cu): one thread-block cluster of cs
// CTAs runs T consecutive iterations of one decomposition in one launch.
// CTA c of the cluster owns fibers [c fpc, c fpc + fpc) of every batch for
// the gather and the tensor-core contraction (all rows of A^(n)), and a
// contiguous range of rows of A^(n) for the reduction and the step.
struct PersArgs {
    Problem<float> P;
    float *Ap[kMaxModes];     // private copies of the factors, row stride R4
    float *part;              // partial M per CTA: [cs][ntile * 128][cst] fp32
    float *hpart;             // partial H per CTA: [cs][64][64] fp32
    long long off[kMaxModes]; // offset of mode k's CDF in the shared staging
    long long sumI;           // sum of the I_k (staging entries)
    int cs, fpc, R4, Npad, cst, ntile;
};

// What a persistent launch does: train (gmode < 0), or form K mini-batch
// gradients of mode gmode at the current factors into gout (K x I_n x R).
struct PersMode {
    int gmode;
    long long t0;
    int K;
    float *gout;
};

// Launchers (cpd_kernels.cu). Every launcher enqueues on `stream` and
// returns the launch error, if any.
template <class T>
cudaError_t launch_iteration(const Problem<T> &P, int grid_grad, int grid_upd,
                             size_t smem_grad, cudaStream_t stream, int engine,
                             cudaEvent_t ev0, cudaEvent_t ev1, cudaEvent_t ev2);
template <class T>
cudaError_t launch_group_iteration(const GroupLaunch<T> &L, cudaStream_t stream);
template <class T>
cudaError_t launch_refresh_mode(const Problem<T> &P, int k, cudaStream_t stream);
template <class T>
cudaError_t launch_sample_probs(const Problem<T> &P, cudaStream_t stream);
template <class T>
cudaError_t launch_flush_dirty(const Problem<T> &P, cudaStream_t stream);
// Gradient-variance diagnostic (cpd_variance.cu): writes {S1, M2} (see there)
// to out2 on the device; scratch from the stream-ordered allocator.
template <class T>
cudaError_t launch_variance(const Problem<T> &P, int n, double *out2, cudaStream_t stream);
template <class T>
cudaError_t launch_fit(const Problem<T> &P, double *partials, int nblocks,
                       double *out2, cudaStream_t stream, int want_xnorm);
cudaError_t launch_build_replica(const void *X, void *rep, int esize, int N,
                                 const int64_t *dims, int n, int64_t ld,
                                 cudaStream_t stream);
template <class T>
size_t grad_smem_bytes(const Problem<T> &P);
int fit_blocks();

// Tensor-core gradient engines (cpd_tc.cu: one CTA per tile; cpd_tcc.cu:
// one cluster per fiber group).
bool tc_supported(int R, int rb);
cudaError_t launch_grad_tc(const Problem<float> &P, int grid, cudaStream_t stream);
cudaError_t launch_grad_tc_group(const GroupLaunch<float> &L, cudaStream_t stream);
size_t tc_smem_bytes(const Problem<float> &P);
cudaError_t launch_grad_tcc(const Problem<float> &P, int grid, cudaStream_t stream);
size_t tcc_smem_bytes(const Problem<float> &P);
int tcc_max_clusters(const Problem<float> &P);
long long tc_stage_cap(const Problem<float> &P);
long long tcc_stage_cap(const Problem<float> &P);
constexpr long long kSimtStageCap = 2048;
size_t lev_smem(int R);   // dynamic shared memory of the leverage kernels

// Fused iteration engine (cpd_fused.cu): one cluster per tile of P.rb =
// 128 or 256 rows of A^(n), gradient and step in one launch; BF16 tensors,
// R <= 64.
constexpr size_t kFusedSmemMax = 226 * 1024;
void fused_plan(int N, int R, int B, int cs_req, int *cs, int *fpc);
bool fused_fits(int N, int R, int B, int cs_req, int tpc);
cudaError_t launch_fused(const Problem<float> &P, int grid, cudaStream_t stream);
size_t fused_smem_bytes(const Problem<float> &P);
long long fused_stage_cap(const Problem<float> &P);
int fused_max_clusters(const Problem<float> &P);

// Tensor-core stop check (cpd_fit_tc.cu): BF16 tensors, float factors, R <= 64.
struct FitTcArgs {
    __nv_bfloat16 *a0op;        // A^(1) hi/lo operand, chunks of 128 rows
    __nv_bfloat16 *ztiles;      // KRP hi/lo operand, tiles of 128 fibers
    float *apad[kMaxModes];     // factors k >= 1 with rows of Kp floats (apad[0] unused)
    double *partials;           // one FP64 partial per CTA
    long long J;                // mode-1 fibers
    int Kp, nchunks;            // R rounded up to 16; chunks of A^(1)
};
bool fit_tc_supported(const Problem<float> &P);
size_t fit_tc_scratch_bytes(const Problem<float> &P);
cudaError_t launch_fit_tc(const Problem<float> &P, void *scratch, double *partials, int sm_count, double *out,
                          cudaStream_t s);
cudaError_t launch_fold(const double *partials, int n, double *out, cudaStream_t s);

// SKRP-ST-I materialised (cpd_skrp.cu).
cudaError_t launch_skrp(const Problem<float> &P, int n, long long t0, int K, int *idx, double *p, float *Z, void *X,
                        int esize, int sm_count, cudaStream_t stream);
size_t skrp_smem_bytes(const Problem<float> &P, int n, int esize);

// Persistent cluster engine (cpd_pers.cu).
bool pers_supported(const cpd_config &cfg);
void pers_fill(PersArgs &a, int cs);        // fpc, R4, Npad, cst, ntile, off, sumI
size_t pers_smem_bytes(const PersArgs &a);
int pers_max_clusters(const PersArgs &a);
cudaError_t launch_pers(const PersArgs &a, long long T, cudaStream_t stream);
cudaError_t launch_pers_group(const PersArgs *dargs, int G, int cs, size_t smem, long long T, cudaStream_t stream);
// K gradients of mode n over `nclusters` clusters; a.part / a.hpart must hold
// nclusters slab sets.
cudaError_t launch_pers_gradients(const PersArgs &a, int n, long long t0, int K, int nclusters, float *gout,
                                  cudaStream_t stream);

}  // namespace cpd
