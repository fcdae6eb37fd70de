// Kernels of one BrawsCPD / AdawsCPD iteration (Alg. 4 / Alg. 5) and the
// full-tensor relative error of Sec. 5.2.
//
// Per iteration (the mode n and all draws follow from (seed, *t_dev)):
//   k_grad_simt   sampling (Alg. 3) + sampled KRP rows (Alg. 1, Eq. (3))
//                 + fiber gather (Alg. 1, Eq. (2)) + weighted gradient partials
//                 (Eq. (11)), split over (row tile, fiber group) CTAs;
//   k_update      fixed-order reduction of the partials, the step
//                 (Eq. (12) / Thm 9 / Eq. (13a)-(13b)), new Euclidean row
//                 weights, and -- in the last CTA to finish -- the canonical
//                 CDF rebuild of mode n and t += 1;
//   k_gram, k_lev_rows   (leverage sampling only) Gram + Cholesky and the new
//                 leverage scores of mode n, then the CDF rebuild and t += 1.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cpd_device.cuh"
#include "cpd_internal.h"

namespace cpd {

namespace {

// Shared-memory carve-up of the gradient kernel (all offsets 16-byte aligned).
template <class T>
struct GradSmem {
    size_t idx, jcol, s, z, At, x, stage, dsm, total;
    __host__ __device__ GradSmem(int N, int R, int rb, int fb)
    {
        size_t o = 0;
        stage = o; o += 2048 * 8;   // CDF staging for the draws
        dsm = o;   o += 2 * kThreads * 8;   // scratch of an in-place CDF rebuild
        idx = o;  o += align_up_h((size_t)fb * N * sizeof(int), 16);
        jcol = o; o += align_up_h((size_t)fb * sizeof(long long), 16);
        s = o;    o += align_up_h((size_t)fb * sizeof(T), 16);
        z = o;    o += align_up_h((size_t)fb * R * sizeof(T), 16);
        At = o;   o += align_up_h((size_t)R * rb * sizeof(T), 16);
        x = o;    o += align_up_h((size_t)fb * rb * sizeof(T), 16);
        total = o;
    }
    __host__ __device__ static size_t align_up_h(size_t v, size_t a) { return (v + a - 1) / a * a; }
};

// Copy rows [r0, r0+rows) of fiber j (contiguous in the mode-n replica) into
// shared memory as T, with 16-byte vector loads (rows are padded to 8).
template <class XT, class T>
__device__ __forceinline__ void gather_rows(const XT *__restrict__ rep, long long ld,
                                            const long long *jcol, int nf, int r0, int rows,
                                            int rb, T *sx)
{
    constexpr int V = 16 / sizeof(XT);
    const int nv = (rows + V - 1) / V;
    for (int e = threadIdx.x; e < nf * nv; e += blockDim.x) {
        const int f = e / nv, q = e % nv;
        const XT *src = rep + jcol[f] * ld + r0 + q * V;
        const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(src));
        const XT *vals = reinterpret_cast<const XT *>(&raw);
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const int i = q * V + u;
            if (i < rows) sx[f * rb + i] = load_x<XT, T>(vals + u);
        }
    }
}

// The strided layout's gather: rows [r0, r0+rows) of the fibers starting at
// start[f] with entries `step` apart, one entry per thread (consecutive
// threads take consecutive rows of a fiber).
template <class XT, class T>
__device__ __forceinline__ void gather_rows_strided(const XT *__restrict__ x, long long step, const long long *start,
                                                    int nf, int r0, int rows, int rb, int bs, T *sx)
{
    if (bs > 1 && nf % bs == 0) {
        // sampled blocks (Remark 1): the bs fibers of a block start at
        // consecutive elements, so consecutive threads take them for one row
        // and each warp reads runs of bs adjacent entries
        for (int e = threadIdx.x; e < nf * rows; e += blockDim.x) {
            const int u = e % bs, rest = e / bs;
            const int i = rest % rows, f = (rest / rows) * bs + u;
            sx[f * rb + i] = load_x<XT, T>(x + start[f] + (long long)(r0 + i) * step);
        }
        return;
    }
    for (int e = threadIdx.x; e < nf * rows; e += blockDim.x) {
        const int f = e / rows, i = e % rows;
        sx[f * rb + i] = load_x<XT, T>(x + start[f] + (long long)(r0 + i) * step);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Gradient partials, residual form. For this CTA's rows i and fibers f:
//   res_if = s_f * (A^(n)(i,:) . z_f - x_f(i))          (one row of A Zs^T - Xs, weighted)
//   part[gf][i][r] = sum_f res_if * z_f(r)
// so that sum over fiber groups gives (A Zs^T D Zs - Xs D Zs) / (B J_n),
// Eq. (11), without the cancellation of forming the two products apart.
// ---------------------------------------------------------------------------
// `bid` is the CTA's index among the CTAs of this problem.
template <class T, class XT>
__device__ __forceinline__ void grad_simt_body(const Problem<T> &P, int bid)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const long long t = *P.t_dev;
    const int N = P.N, R = P.R, rb = P.rb, fb = P.fb;
    const int n = mode_draw(P.seed, t, N);
    const int pr = P.tile[n].pr;
    const int gr = bid % pr, gf = bid / pr;
    if (gf >= P.pf) return;
    const long long In = P.dims[n];
    const int r0 = gr * rb;
    const int rows = (int)((In - r0) < rb ? (In - r0) : rb);
    const int f0 = gf * fb;
    const int nf = (P.B - f0) < fb ? (P.B - f0) : fb;

    const GradSmem<T> L(N, R, rb, fb);
    int *sidx = reinterpret_cast<int *>(smem + L.idx);
    long long *jcol = reinterpret_cast<long long *>(smem + L.jcol);
    T *ss = reinterpret_cast<T *>(smem + L.s);
    T *sz = reinterpret_cast<T *>(smem + L.z);
    T *sAt = reinterpret_cast<T *>(smem + L.At);
    T *sx = reinterpret_cast<T *>(smem + L.x);

    // 1. draws of Alg. 3
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(smem + L.stage);
    draw_indices(P, t, n, f0, nf, sidx, stage, 2048, reinterpret_cast<unsigned long long *>(smem + L.dsm),
                 bid == 0);
    const bool staged = cdfs_staged(P, n, 2048);
    // rows of A^(n) for the residual, transposed (conflict-free reads)
    const T *An = P.A[n];
    for (int e = threadIdx.x; e < rows * R; e += blockDim.x) {
        const int i = e / R, r = e % R;
        sAt[r * rb + i] = An[(long long)(r0 + i) * R + r];
    }
    __syncthreads();

    // 2. fiber column j (Eq. (2)), probability p_f and weight s_f
    for (int f = threadIdx.x; f < nf; f += blockDim.x) {
        const int *row = sidx + f * N;
        long long j = 0, Jp = 1;
        for (int k = 0; k < N; ++k) {
            if (k == n) continue;
            j += (long long)row[k] * Jp;
            Jp *= P.dims[k];
        }
        jcol[f] = (P.strided && n > 0) ? fiber_start(P, n, j) : j;   // strided: the fiber's first entry
        if constexpr (sizeof(T) == 8)
            ss[f] = __ddiv_rn(1.0, __dmul_rn(__dmul_rn((double)(P.B / P.block), P.Jn[n]),
                                             fiber_prob_staged(P, n, row, staged ? stage : nullptr)));
        else
            ss[f] = staged ? fiber_weight_staged(P, n, row, stage) : fiber_weight(P, n, row);
        if (gr == 0)
            for (int k = 0; k < N; ++k) P.idx[(long long)(f0 + f) * N + k] = row[k];
    }
    // 3. sampled KRP rows z_f = Hadamard product of A^(k)(i_k,:), k != n (Alg. 1)
    for (int e = threadIdx.x; e < nf * R; e += blockDim.x) {
        const int f = e / R, r = e % R;
        const int *row = sidx + f * N;
        T z = (T)1;
        for (int k = 0; k < N; ++k) {
            if (k == n) continue;
            z = z * P.A[k][(long long)row[k] * R + r];
        }
        sz[f * R + r] = z;
    }
    __syncthreads();

    // 4. fiber gather from the mode-n replica (Alg. 1, X_(n)(:, F_n))
    if (P.strided && n > 0)
        gather_rows_strided<XT, T>(reinterpret_cast<const XT *>(P.rep[n]), fiber_step(P, n), jcol, nf, r0, rows, rb,
                                   block_mode(n) == 0 ? P.block : 1, sx);
    else
        gather_rows<XT, T>(reinterpret_cast<const XT *>(P.rep[n]), P.ld[n], jcol, nf, r0, rows, rb, sx);
    __syncthreads();

    // 5. weighted residuals
    for (int e = threadIdx.x; e < nf * rows; e += blockDim.x) {
        const int f = e / rows, i = e % rows;
        T acc = (T)0;
        for (int r = 0; r < R; ++r) acc += sAt[r * rb + i] * sz[f * R + r];
        sx[f * rb + i] = ss[f] * (acc - sx[f * rb + i]);
    }
    __syncthreads();

    // 6. partial gradient of this fiber group, layout [gf][i][r] (coalesced rows)
    T *out = P.part + (long long)gf * R * In;
    for (int e = threadIdx.x; e < R * rows; e += blockDim.x) {
        const int i = e / R, r = e % R;
        T acc = (T)0;
        for (int f = 0; f < nf; ++f) acc += sx[f * rb + i] * sz[f * R + r];
        out[(long long)(r0 + i) * R + r] = acc;
    }
}

template <class T, class XT>
__global__ void __launch_bounds__(kThreads) k_grad_simt(const Problem<T> P)
{
    grad_simt_body<T, XT>(P, (int)blockIdx.x);
}

// One launch for a group of problems (see group_member).
template <class T, class XT>
__global__ void __launch_bounds__(kThreads) k_grad_simt_group(const Problem<T> *__restrict__ Ps,
                                                              const int *__restrict__ cta0, int G)
{
    __shared__ __align__(16) Problem<T> sp;
    const int g = group_member(Ps, cta0, G, sp);
    grad_simt_body<T, XT>(sp, (int)blockIdx.x - __ldg(cta0 + g));
}

// ---------------------------------------------------------------------------
// Reduction + step. CTA b owns rows [b*rpc, b*rpc+rpc) of A^(n).
// ---------------------------------------------------------------------------

// Rebuild the fixed-point distribution of mode k from w[k] (one CTA); a
// distribution without mass is flagged.
constexpr int kWStage = 4096;  // doubles of shared staging for the row weights
constexpr int kLevSmemR = 64;  // leverage: L staged in shared memory up to this rank
// dynamic shared memory of the leverage kernels: L (R x R) and the inverse
// pivots when staged, and at least the row-weight staging of a distribution rebuild
inline size_t lev_smem_bytes(int R)
{
    const size_t l = R <= kLevSmemR ? (size_t)(R * R + R) * sizeof(double) : 0;
    const size_t w = (size_t)kWStage * sizeof(double);
    return l > w ? l : w;
}

template <class T>
__device__ void finish_distribution(const Problem<T> &P, int k, unsigned long long *sm, double *wstage)
{
    if (!block_distribution(P.w[k], P.dims[k], P.cdf[k], sm, wstage, kWStage) && threadIdx.x == 0)
        atomicOr(P.status, kStDegenerate);
}

// `bid` / `nblk`: the CTA's index among, and the number of, this problem's CTAs.
template <class T>
__device__ __forceinline__ void update_body(const Problem<T> &P, int bid, unsigned nblk)
{
    __shared__ T s_new[kThreads];
    __shared__ unsigned long long s_dist[2 * kThreads];
    __shared__ __align__(16) double s_w[kWStage];       // last CTA: staged row weights
    const bool tr0 = bid == 0;
    trace_stamp(P.trace, 16, tr0);
    const long long t = *P.t_dev;
    const int N = P.N, R = P.R;
    const int n = mode_draw(P.seed, t, N);
    const long long In = P.dims[n];
    const int rpc = kThreads / R > 0 ? kThreads / R : 1;
    const int li = threadIdx.x / R, r = threadIdx.x % R;
    const long long i = (long long)bid * rpc + li;
    const bool act = li < rpc && i < In;
    T *An = P.A[n];
    if (act) {
        // G(i, r) = sum of the fiber groups' partials in fixed order; the
        // loads are issued in batches of 24 so their latencies overlap.
        T g = (T)0;
        const T *src = P.part + i * R + r;
        const long long slab = (long long)In * R;
        for (int q0 = 0; q0 < P.pf; q0 += 24) {
            T v[24];
#pragma unroll
            for (int u = 0; u < 24; ++u) v[u] = (q0 + u < P.pf) ? __ldcg(src + (q0 + u) * slab) : (T)0;
#pragma unroll
            for (int u = 0; u < 24; ++u)
                if (q0 + u < P.pf) g += v[u];
        }
        P.G[i * R + r] = g;
        trace_stamp(P.trace, 17, tr0 && threadIdx.x == 0);
        T an;
        if (P.step == CPD_STEP_ADAGRAD) {
            // S accumulates in FP64; the step factor eta / sqrt(b + S) is formed
            // in the factor type.
            double *Sp = P.S[n] + i * R + r;
            const double S = __fma_rn((double)g, (double)g, *Sp);
            *Sp = S;
            if constexpr (sizeof(T) == 8)
                an = An[i * R + r] - P.eta * g * rsqrt(P.b + S);
            else
                an = An[i * R + r] - (float)P.eta * g * rsqrtf((float)S + (float)P.b);
        } else {
            const T alpha = (T)((P.step == CPD_STEP_DECAY) ? P.beta / ((double)t + P.gamma) : P.alpha);
            an = An[i * R + r] - alpha * g;
        }
        if (P.constraint == CPD_CONSTRAINT_NONNEG && an < (T)0) an = (T)0;   // projection; NaN kept
        if (!isfinite((double)an) || !isfinite((double)g)) atomicOr(P.status, kStNonFinite);
        An[i * R + r] = an;
        s_new[threadIdx.x] = an;
    }
    __syncthreads();
    trace_stamp(P.trace, 18, tr0);
    if (P.sampling == CPD_SAMPLE_EUCLIDEAN) {
        // one warp per updated row: the canonical tree-ordered squared norm
        const int warp = threadIdx.x >> 5;
        for (int lr = warp; lr < rpc; lr += kThreads / 32) {
            const long long row = (long long)bid * rpc + lr;
            if (row < In) {
                const double wv = warp_row_weight(s_new + lr * R, R);
                if ((threadIdx.x & 31) == 0) P.w[n][row] = wv;
            }
        }
    }
    trace_stamp(P.trace, 19, tr0);
    if (!last_block(P.counters, nblk)) return;
    trace_stamp(P.trace, 20, true);
    if (P.sampling == CPD_SAMPLE_EUCLIDEAN && !P.defer_cdf) finish_distribution(P, n, s_dist, s_w);
    trace_stamp(P.trace, 21, true);
    if (threadIdx.x == 0) {
        P.counters[0] = 0;
        if (P.sampling != CPD_SAMPLE_LEVERAGE) {
            if (P.sampling == CPD_SAMPLE_EUCLIDEAN && P.defer_cdf) *P.dirty = n;
            *P.n_last = n;
            *P.t_dev = t + 1;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_update(const Problem<T> P)
{
    update_body<T>(P, (int)blockIdx.x, gridDim.x);
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_update_group(const Problem<T> *__restrict__ Ps,
                                                           const int *__restrict__ cta0, int G)
{
    __shared__ __align__(16) Problem<T> sp;
    const int g = group_member(Ps, cta0, G, sp);
    const int b0 = __ldg(cta0 + g);
    update_body<T>(sp, (int)blockIdx.x - b0, (unsigned)(__ldg(cta0 + g + 1) - b0));
}

// ---------------------------------------------------------------------------
// Leverage scores (Def. 3) in the canonical order: one warp per Gram entry
// (32 strided partials, shuffle-down tree), the last CTA factors the Gram
// matrix (Cholesky; every entry takes its updates with k ascending) into
// P.lev_L.
// k_mode < 0: the mode of the current iteration; else that mode.
// ---------------------------------------------------------------------------
// `bid` / `nblk`: the CTA's index among, and the number of, this problem's CTAs.
template <class T>
__device__ __forceinline__ void gram_body(const Problem<T> &P, int k_mode, int bid, unsigned nblk)
{
    const long long t = *P.t_dev;
    const int k = k_mode >= 0 ? k_mode : mode_draw(P.seed, t, P.N);
    const int R = P.R;
    const long long I = P.dims[k];
    const T *A = P.A[k];
    double *g = P.lev_L + R * R + R;  // Gram scratch after L and inv
    const int lane = threadIdx.x & 31;
    const int warp_global = (bid * blockDim.x + threadIdx.x) >> 5;
    const int npairs = R * (R + 1) / 2;
    for (int pr = warp_global; pr < npairs; pr += (int)((nblk * blockDim.x) >> 5)) {
        int r = 0, rem = pr;
        while (rem >= R - r) { rem -= R - r; ++r; }
        const int s = r + rem;
        double acc = 0.0;
        for (long long i = lane; i < I; i += 32)
            acc = __fma_rn((double)A[i * R + r], (double)A[i * R + s], acc);
        for (int off = 16; off >= 1; off >>= 1)
            acc = __dadd_rn(acc, __shfl_down_sync(0xffffffffu, acc, off));
        if (lane == 0) {
            g[r * R + s] = acc;
            g[s * R + r] = acc;
        }
    }
    if (!last_block(P.counters + 1, nblk)) return;
    double *Lm = P.lev_L, *inv = P.lev_L + R * R;
    __shared__ int s_bad;
    __shared__ double s_col[256];  // column q of L below the diagonal, contiguous
    __shared__ double s_gd[256];   // g_jj, the pivots' degeneracy thresholds
    // Right-looking order: once column q of L is final, every entry (i, j)
    // with q < j <= i takes its update -L_iq L_jq at once. Each entry still
    // receives the fmas of q = 0, 1, ..., j-1 in ascending order, as in the
    // left-looking form, so L and the inverse pivots are the same bits; the
    // dependent depth per column is one update, one square root and one
    // division instead of a chain of j fmas. Small R: in place in shared
    // memory, then L and the inverse pivots are stored. Large R: in place in
    // P.lev_L (its upper triangle keeps Gram entries nobody reads).
    extern __shared__ __align__(16) double lev_dyn[];
    const bool in_smem = R <= kLevSmemR;
    double *W = in_smem ? lev_dyn : Lm;
    double *wi = in_smem ? lev_dyn + R * R : inv;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) W[e] = __ldcg(g + e);
    for (int j = threadIdx.x; j < R; j += blockDim.x) s_gd[j] = __ldcg(g + j * R + j);
    // pivot j from d, g_jj minus all its updates. The pivots form the only
    // dependent chain of the factorisation (R square roots and reciprocals),
    // so nothing on it goes through memory: the threshold is staged above and
    // d and L_jj stay in registers.
    auto pivot = [&](int j, double d) {
        if (!(d > 0x1.0p-40 * s_gd[j])) {
            s_bad = 1;
            d = 1.0;
        }
        const double ljj = __dsqrt_rn(d);
        W[j * R + j] = ljj;
        wi[j] = __drcp_rn(ljj);  // 1/L_jj, correctly rounded
    };
    __syncthreads();
    if (threadIdx.x == 0) {
        s_bad = 0;
        pivot(0, W[0]);
    }
    __syncthreads();
    static_assert(kThreads >= 64, "the factorisation needs a pivot warp and an update warp");
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int q = 0; q < R; ++q) {
        for (int i = q + 1 + threadIdx.x; i < R; i += blockDim.x) {
            const double l = __dmul_rn(W[i * R + q], wi[q]);
            W[i * R + q] = l;
            s_col[i] = l;
        }
        __syncthreads();
        // row q+1 has one entry left, the diagonal: thread 0 updates it and
        // factors pivot q+1 while warps 1, 2, ... update rows q+2, q+3, ...
        if (warp == 0) {
            if (lane == 0 && q + 1 < R) {
                const double c = s_col[q + 1];
                pivot(q + 1, __fma_rn(-c, c, W[(q + 1) * (R + 1)]));
            }
        } else {
            for (int i = q + 2 + (warp - 1); i < R; i += nwarp - 1) {
                const double li = s_col[i];
                for (int j = q + 1 + lane; j <= i; j += 32) W[i * R + j] = __fma_rn(-li, s_col[j], W[i * R + j]);
            }
        }
        __syncthreads();
    }
    if (in_smem) {
        for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
            const int i = e / R, q = e % R;
            if (q <= i) Lm[e] = W[e];
        }
        for (int j = threadIdx.x; j < R; j += blockDim.x) inv[j] = wi[j];
    }
    if (threadIdx.x == 0) {
        P.counters[1] = 0;
        if (s_bad) atomicOr(P.status, kStDegenerate);
        P.lev_L[R * R + R + R * R] = s_bad ? 1.0 : 0.0;  // flag read by k_lev_rows
    }
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_gram(const Problem<T> P, int k_mode)
{
    gram_body<T>(P, k_mode, (int)blockIdx.x, gridDim.x);
}

// Grouped: the CTAs of problem g are [cta0[g], cta0[g+1]) (none for members
// that do not sample by leverage); each runs its own problem's arithmetic.
template <class T>
__global__ void __launch_bounds__(kThreads) k_gram_group(const Problem<T> *__restrict__ Ps,
                                                         const int *__restrict__ cta0, int G)
{
    __shared__ __align__(16) Problem<T> sp;
    const int g = group_member(Ps, cta0, G, sp);
    const int b0 = __ldg(cta0 + g);
    gram_body<T>(sp, -1, (int)blockIdx.x - b0, (unsigned)(__ldg(cta0 + g + 1) - b0));
}

// l_i = ||L^{-1} a_i||^2 by forward substitution, then the CDF of the mode in
// the last CTA; advance = 1 closes the iteration (t += 1). One warp per row in
// right-looking order: lane j % 32 holds the partial v_j (v_j = a_ij at the
// start); at step q the owner of v_q forms y_q = v_q / L_qq (times the inverse
// pivot), every lane adds y_q^2 to the row's sum, and every v_j with j > q
// takes its fma -L_jq y_q. Each v_j receives the fmas of q = 0, ..., j-1 in
// ascending order and the sum the squares in ascending order, as in the
// sequential form, so l_i is the same bits.
template <class T>
__device__ __forceinline__ void lev_rows_body(const Problem<T> &P, int k_mode, int advance, int bid, unsigned nblk)
{
    const long long t = *P.t_dev;
    const int k = k_mode >= 0 ? k_mode : mode_draw(P.seed, t, P.N);
    const int R = P.R;
    const long long I = P.dims[k];
    const bool bad = __ldcg(P.lev_L + R * R + R + R * R) != 0.0;
    // small R: L transposed (lt[q*R + j] = L_jq, j > q) and the inverse pivots
    // in shared memory (the buffer later serves as the last CTA's weight staging)
    extern __shared__ __align__(16) double lev_dyn[];
    const bool in_smem = R <= kLevSmemR;
    if (in_smem) {
        for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
            const int q = e / R, j = e % R;
            lev_dyn[e] = j > q ? __ldcg(P.lev_L + j * R + q) : 0.0;
        }
        for (int j = threadIdx.x; j < R; j += blockDim.x) lev_dyn[R * R + j] = __ldcg(P.lev_L + R * R + j);
        __syncthreads();
    }
    const double *inv = in_smem ? lev_dyn + R * R : P.lev_L + R * R;
    const int lane = threadIdx.x & 31;
    const long long i = ((long long)bid * blockDim.x + threadIdx.x) >> 5;
    if (!bad && i < I) {
        constexpr int kSlots = 256 / 32;  // v_j of j = lane + 32 s
        const T *a = P.A[k] + i * R;
        double v[kSlots];
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
            const int j = lane + 32 * s;
            v[s] = j < R ? (double)a[j] : 0.0;
        }
        double acc = 0.0;
        for (int q = 0; q < R; ++q) {
            const int qs = q >> 5;
            double vq = 0.0;
#pragma unroll
            for (int s = 0; s < kSlots; ++s)
                if (s == qs) vq = v[s];
            const double y = __shfl_sync(0xffffffffu, __dmul_rn(vq, inv[q]), q & 31);
            acc = __fma_rn(y, y, acc);
#pragma unroll
            for (int s = 0; s < kSlots; ++s) {
                const int j = lane + 32 * s;
                if (s >= qs && j > q && j < R) {
                    const double l = in_smem ? lev_dyn[q * R + j] : __ldg(P.lev_L + (long long)j * R + q);
                    v[s] = __fma_rn(-l, y, v[s]);
                }
            }
        }
        if (lane == 0) P.w[k][i] = acc;
    }
    if (!last_block(P.counters + 2, nblk)) return;
    __shared__ unsigned long long s_dist[2 * kThreads];
    if (!bad) finish_distribution(P, k, s_dist, lev_dyn);
    if (threadIdx.x == 0) {
        P.counters[2] = 0;
        if (advance) {
            *P.n_last = k;
            *P.t_dev = t + 1;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_lev_rows(const Problem<T> P, int k_mode, int advance)
{
    lev_rows_body<T>(P, k_mode, advance, (int)blockIdx.x, gridDim.x);
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_lev_rows_group(const Problem<T> *__restrict__ Ps,
                                                             const int *__restrict__ cta0, int G)
{
    __shared__ __align__(16) Problem<T> sp;
    const int g = group_member(Ps, cta0, G, sp);
    const int b0 = __ldg(cta0 + g);
    lev_rows_body<T>(sp, -1, 1, (int)blockIdx.x - b0, (unsigned)(__ldg(cta0 + g + 1) - b0));
}

// Euclidean or uniform weights of mode k from scratch (initialisation and
// cpd_set_factors), one warp per row, then the distribution.
template <class T>
__global__ void __launch_bounds__(kThreads) k_weights_euclid(const Problem<T> P, int k)
{
    __shared__ unsigned long long s_dist[2 * kThreads];
    const long long I = P.dims[k];
    const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row < I) {
        const double wv = (P.sampling == CPD_SAMPLE_UNIFORM) ? 1.0 : warp_row_weight(P.A[k] + row * P.R, P.R);
        if ((threadIdx.x & 31) == 0) P.w[k][row] = wv;
    }
    if (!last_block(P.counters + 3)) return;
    __shared__ double s_w[kWStage];
    finish_distribution(P, k, s_dist, s_w);
    if (threadIdx.x == 0) P.counters[3] = 0;
}

// Bring a deferred CDF up to date: rebuild the dirty mode's distribution from
// its row weights (the same exact fixed-point CDF the next gradient kernel
// would build) and clear the flag. One CTA.
template <class T>
__global__ void __launch_bounds__(kThreads) k_flush_dirty(const Problem<T> P)
{
    __shared__ unsigned long long s_dist[2 * kThreads];
    __shared__ __align__(16) double s_w[kWStage];
    const int d = *P.dirty;
    if (d < 0) return;
    finish_distribution(P, d, s_dist, s_w);
    __syncthreads();
    if (threadIdx.x == 0) *P.dirty = -1;
}

// p_f of the last batch (Eq. (10), FP64) for its record; the
// distributions of the modes k != n it used have not changed since.
template <class T>
__global__ void k_sample_probs(const Problem<T> P)
{
    const int n = *P.n_last;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < 0 || f >= P.B) return;
    P.p[f] = fiber_prob(P, n, P.idx + (long long)f * P.N);
}

// ---------------------------------------------------------------------------
// Relative error (Sec. 5.2): sum over all entries of (x - x_hat)^2 with
// x_hat(i, j) = A^(1)(i,:) . z_j, z_j the KRP row of mode-1 fiber j, read from
// the mode-1 replica. FP64 accumulation, fixed-order reductions.
// ---------------------------------------------------------------------------
constexpr int kFitFibers = 16;        // fibers per thread per chunk (reuse of each A^(1) entry)
constexpr int kFitStage = 4096;       // staged KRP entries per chunk
constexpr int kFitAtBytes = 48 * 1024;   // A^(1) rows of a CTA's tile, transposed

// Work split of the fit pass. A CTA owns a tile of rt rows of A^(1) (staged
// transposed in shared memory once) and walks its share of the mode-1
// fibers in chunks of F = 16 nblk; thread (row il, block b) forms x_hat for
// its row and 16 fibers. KRP rows are staged at a stride of R rounded up to
// 4 for float factors (128-bit loads).
struct FitTiling {
    int rt, ntile, nblk, F, Rs;
};

__host__ __device__ inline FitTiling fit_tiling(long long I0, int R, int tsize)
{
    FitTiling t;
    t.Rs = tsize == 4 ? (R + 3) / 4 * 4 : R;
    int rmax = kThreads;
    while (rmax > 16 && (long long)rmax * R * tsize > kFitAtBytes) rmax >>= 1;
    t.rt = (int)(I0 < rmax ? I0 : rmax);
    t.ntile = (int)((I0 + t.rt - 1) / t.rt);
    int nblk = kThreads / t.rt;
    const int cap = kFitStage / (kFitFibers * t.Rs);
    if (nblk > cap) nblk = cap;
    if (nblk > kThreads / kFitFibers) nblk = kThreads / kFitFibers;   // one decoding thread per fiber
    if (nblk < 1) nblk = 1;
    t.nblk = nblk;
    t.F = kFitFibers * nblk;
    return t;
}

// Fixed order: a thread's fibers and chunks in order, then the warp tree and
// the CTA's warps; the CTAs' partials are folded by k_fold.
template <class T, class XT>
__global__ void __launch_bounds__(kThreads) k_fit(const Problem<T> P, double *partials, int want_xnorm)
{
    extern __shared__ __align__(16) unsigned char fit_dyn[];
    __shared__ __align__(16) T sz[kFitStage];
    __shared__ int sidx[kThreads * (kMaxModes - 1)];   // the chunk's fibers' indices, modes 1..N-1
    __shared__ double red[kThreads / 32];
    T *sAt = reinterpret_cast<T *>(fit_dyn);           // [R][rt]
    const int N = P.N, R = P.R;
    const long long I0 = P.dims[0];
    long long J = 1;
    for (int k = 1; k < N; ++k) J *= P.dims[k];
    const FitTiling L = fit_tiling(I0, R, (int)sizeof(T));
    const int Rs = L.Rs, rt = L.rt, F = L.F;
    // (tile, fiber group) pairs: one per CTA when the grid covers the tiles,
    // otherwise each CTA walks several tiles with all fibers
    const long long ngroups = (long long)gridDim.x >= L.ntile ? (long long)gridDim.x / L.ntile : 1;
    const long long npairs = (long long)L.ntile * ngroups;
    const int il = threadIdx.x % rt, b = threadIdx.x / rt;
    const int f0 = b * kFitFibers;                     // this thread's fibers in a chunk
    const XT *rep = reinterpret_cast<const XT *>(P.rep[0]);
    double acc = 0.0;
    for (long long pair = blockIdx.x; pair < npairs; pair += gridDim.x) {
        const long long tile = pair % L.ntile, group = pair / L.ntile;
        const long long r0 = tile * rt;
        const int rows = (int)((I0 - r0) < rt ? (I0 - r0) : rt);
        const bool act = b < L.nblk && il < rows;
        __syncthreads();                            // the previous pair's rows are no longer read
        for (int e = threadIdx.x; e < rows * R; e += blockDim.x) {
            const int i = e / R, r = e % R;
            sAt[r * rt + i] = P.A[0][(r0 + i) * R + r];
        }
        for (long long j0 = group * F; j0 < J; j0 += ngroups * F) {
            const int nfib = (J - j0) < F ? (int)(J - j0) : F;
            __syncthreads();
            if (threadIdx.x < nfib) {               // Eq. (2), inverted once per fiber
                long long j = j0 + threadIdx.x;
                for (int k = 1; k < N; ++k) {
                    sidx[threadIdx.x * (kMaxModes - 1) + k - 1] = (int)(j % P.dims[k]);
                    j /= P.dims[k];
                }
            }
            __syncthreads();
#pragma unroll 4
            for (int e = threadIdx.x; e < F * Rs; e += blockDim.x) {   // unrolled: the L2 loads overlap
                const int f = e / Rs, r = e % Rs;
                T z = (T)0;
                if (f < nfib && r < R && !want_xnorm) {
                    z = (T)1;
                    for (int k = 1; k < N; ++k) z = z * P.A[k][(long long)sidx[f * (kMaxModes - 1) + k - 1] * R + r];
                }
                sz[f * Rs + r] = z;
            }
            __syncthreads();
            if (!act) continue;
            T xh[kFitFibers];
#pragma unroll
            for (int f = 0; f < kFitFibers; ++f) xh[f] = (T)0;
            if (!want_xnorm) {
                if constexpr (sizeof(T) == 4) {
                    for (int r = 0; r < Rs; r += 4) {   // staged KRP entries past R are 0
                        const float a0 = sAt[r * rt + il];
                        const float a1 = r + 1 < R ? sAt[(r + 1) * rt + il] : 0.f;
                        const float a2 = r + 2 < R ? sAt[(r + 2) * rt + il] : 0.f;
                        const float a3 = r + 3 < R ? sAt[(r + 3) * rt + il] : 0.f;
#pragma unroll
                        for (int f = 0; f < kFitFibers; ++f) {   // in the stage; used if < nfib
                            const float4 z = *reinterpret_cast<const float4 *>(sz + (f0 + f) * Rs + r);
                            xh[f] += a0 * z.x;
                            xh[f] += a1 * z.y;
                            xh[f] += a2 * z.z;
                            xh[f] += a3 * z.w;
                        }
                    }
                } else {
                    for (int r = 0; r < R; ++r) {
                        const T a = sAt[r * rt + il];
#pragma unroll
                        for (int f = 0; f < kFitFibers; ++f) xh[f] += a * sz[(f0 + f) * Rs + r];
                    }
                }
            }
            const XT *xr = rep + r0 + il;
            if constexpr (sizeof(T) == 8) {
#pragma unroll
                for (int f = 0; f < kFitFibers; ++f) {
                    if (f0 + f < nfib) {
                        const double d = load_x<XT, T>(xr + (j0 + f0 + f) * P.ld[0]) - xh[f];
                        acc = __fma_rn(d, d, acc);
                    }
                }
            } else {
                // this row's (at most 16) squared residuals summed in FP32, the
                // running sum in FP64: one FP64 operation per 16 entries
                float part = 0.f;
#pragma unroll
                for (int f = 0; f < kFitFibers; ++f) {
                    if (f0 + f < nfib) {
                        const float d = load_x<XT, T>(xr + (j0 + f0 + f) * P.ld[0]) - xh[f];
                        part = fmaf(d, d, part);
                    }
                }
                acc += (double)part;
            }
        }
    }
    for (int off = 16; off >= 1; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kThreads) k_fold(const double *partials, int n, double *out)
{
    // fixed order: strided partial sums per thread, then a pairwise tree
    __shared__ double red[kThreads];
    double acc = 0.0;
    for (int q = threadIdx.x; q < n; q += kThreads) acc += partials[q];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// ---------------------------------------------------------------------------
// Mode-n-major replica: X viewed as [I_post][I_n][I_pre] (column-major, i_pre
// fastest) becomes [I_post][I_pre][ld] with i_n fastest, so fiber
// j = i_pre + I_pre * i_post of the mode-n unfolding (Eq. (2)) is contiguous.
// 32 x 32 tiles through shared memory keep both sides coalesced.
// ---------------------------------------------------------------------------
template <class E>
__global__ void k_copy_padded(const E *__restrict__ X, E *__restrict__ Y, long long In, long long J,
                              long long ld)
{
    const long long total = In * J;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / In, i = e % In;
        Y[j * ld + i] = X[e];
    }
}

template <class E>
__global__ void k_replica(const E *__restrict__ X, E *__restrict__ Y, long long Ipre, long long In,
                          long long Ipost, long long ld)
{
    __shared__ E tile[32][33];
    const long long tiles_pre = (Ipre + 31) / 32, tiles_n = (In + 31) / 32;
    const long long ntiles = tiles_pre * tiles_n * Ipost;
    for (long long tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const long long post = tt / (tiles_pre * tiles_n);
        const long long rem = tt % (tiles_pre * tiles_n);
        const long long tn = rem / tiles_pre, tp = rem % tiles_pre;
        __syncthreads();
        for (int y = threadIdx.y; y < 32; y += blockDim.y) {
            const long long in = tn * 32 + y, ip = tp * 32 + threadIdx.x;
            if (in < In && ip < Ipre) tile[y][threadIdx.x] = X[(post * In + in) * Ipre + ip];
        }
        __syncthreads();
        for (int y = threadIdx.y; y < 32; y += blockDim.y) {
            const long long ip = tp * 32 + y, in = tn * 32 + threadIdx.x;
            if (in < In && ip < Ipre) Y[(post * Ipre + ip) * ld + in] = tile[threadIdx.x][y];
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class T>
size_t grad_smem_bytes(const Problem<T> &P)
{
    return GradSmem<T>(P.N, P.R, P.rb, P.fb).total;
}

template <class T, class XT>
static cudaError_t launch_grad_simt(const Problem<T> &P, int grid, size_t smem, cudaStream_t s)
{
    static size_t attr_bytes = 0;
    if (smem > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k_grad_simt<T, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        attr_bytes = smem;
    }
    k_grad_simt<T, XT><<<grid, kThreads, smem, s>>>(P);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_iteration(const Problem<T> &P, int grid_grad, int grid_upd, size_t smem_grad,
                             cudaStream_t s, int engine, cudaEvent_t ev0, cudaEvent_t ev1, cudaEvent_t ev2)
{
    cudaError_t e = cudaSuccess;
    if (ev0) cudaEventRecord(ev0, s);
    if (engine == kEngineTensor || engine == kEngineTensorCluster || engine == kEngineFused) {
        if constexpr (sizeof(T) == 4)
            e = engine == kEngineTensor          ? launch_grad_tc(P, grid_grad, s)
                : engine == kEngineTensorCluster ? launch_grad_tcc(P, grid_grad, s)
                                                 : launch_fused(P, grid_grad, s);
        else
            e = cudaErrorInvalidValue;
    } else {
        if constexpr (sizeof(T) == 8) {
            e = launch_grad_simt<T, double>(P, grid_grad, smem_grad, s);
        } else {
            if (P.x_dtype == CPD_F32) e = launch_grad_simt<T, float>(P, grid_grad, smem_grad, s);
            else e = launch_grad_simt<T, __nv_bfloat16>(P, grid_grad, smem_grad, s);
        }
    }
    if (ev1) cudaEventRecord(ev1, s);
    if (e != cudaSuccess) return e;
    if (engine != kEngineFused) {   // the fused engine applies the step itself
        k_update<T><<<grid_upd, kThreads, 0, s>>>(P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (P.sampling == CPD_SAMPLE_LEVERAGE) {
        const int npairs = P.R * (P.R + 1) / 2;
        k_gram<T><<<(npairs + 7) / 8, kThreads, lev_smem_bytes(P.R), s>>>(P, -1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        long long Imax = 0;
        for (int k = 0; k < P.N; ++k) Imax = P.dims[k] > Imax ? P.dims[k] : Imax;
        k_lev_rows<T><<<(int)((Imax * 32 + kThreads - 1) / kThreads), kThreads, lev_smem_bytes(P.R), s>>>(P, -1, 1);
        e = cudaGetLastError();
    }
    if (ev2) cudaEventRecord(ev2, s);
    return e;
}

template <class T, class XT>
static cudaError_t launch_grad_simt_group(const GroupLaunch<T> &L, cudaStream_t s)
{
    static size_t attr_bytes = 0;
    if (L.smem_grad > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k_grad_simt_group<T, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L.smem_grad);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        attr_bytes = L.smem_grad;
    }
    k_grad_simt_group<T, XT><<<L.grid_grad, kThreads, L.smem_grad, s>>>(L.P, L.cta_grad, L.G);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_group_iteration(const GroupLaunch<T> &L, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (L.engine == kEngineTensor) {
        if constexpr (sizeof(T) == 4) e = launch_grad_tc_group(L, s);
        else e = cudaErrorInvalidValue;
    } else if (L.engine == kEngineSimt) {
        if constexpr (sizeof(T) == 8) {
            e = launch_grad_simt_group<T, double>(L, s);
        } else {
            if (L.x_dtype == CPD_F32) e = launch_grad_simt_group<T, float>(L, s);
            else e = launch_grad_simt_group<T, __nv_bfloat16>(L, s);
        }
    } else {
        e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    k_update_group<T><<<L.grid_upd, kThreads, 0, s>>>(L.P, L.cta_upd, L.G);
    if ((e = cudaGetLastError()) != cudaSuccess || L.grid_gram == 0) return e;
    // leverage members: their modes' Gram factor, then their leverage rows and
    // distribution (which closes their iteration)
    k_gram_group<T><<<L.grid_gram, kThreads, L.smem_lev, s>>>(L.P, L.cta_gram, L.G);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_lev_rows_group<T><<<L.grid_lev, kThreads, L.smem_lev, s>>>(L.P, L.cta_lev, L.G);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_refresh_mode(const Problem<T> &P, int k, cudaStream_t s)
{
    const long long I = P.dims[k];
    const int grid_rows = (int)((I * 32 + kThreads - 1) / kThreads);
    if (P.sampling == CPD_SAMPLE_LEVERAGE) {
        const int npairs = P.R * (P.R + 1) / 2;
        k_gram<T><<<(npairs + 7) / 8, kThreads, lev_smem_bytes(P.R), s>>>(P, k);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_lev_rows<T><<<grid_rows, kThreads, lev_smem_bytes(P.R), s>>>(P, k, 0);
    } else {
        k_weights_euclid<T><<<grid_rows, kThreads, 0, s>>>(P, k);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_sample_probs(const Problem<T> &P, cudaStream_t s)
{
    k_sample_probs<T><<<(P.B + kThreads - 1) / kThreads, kThreads, 0, s>>>(P);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_flush_dirty(const Problem<T> &P, cudaStream_t s)
{
    if (!P.defer_cdf) return cudaSuccess;
    k_flush_dirty<T><<<1, kThreads, 0, s>>>(P);
    return cudaGetLastError();
}

int fit_blocks() { return 4 * 152; }

cudaError_t launch_fold(const double *partials, int n, double *out, cudaStream_t s)
{
    k_fold<<<1, kThreads, 0, s>>>(partials, n, out);
    return cudaGetLastError();
}

// Raise each fit kernel's dynamic shared-memory limit once to the tiling's maximum.
template <class T, class XT>
static cudaError_t launch_fit_kernel(int grid, size_t dyn, cudaStream_t s, const Problem<T> &P, double *partials,
                                     int want_xnorm)
{
    static bool raised = false;   // one flag per kernel instantiation
    void (*kernel)(const Problem<T>, double *, int) = k_fit<T, XT>;
    if (!raised) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFitAtBytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        raised = true;
    }
    kernel<<<grid, kThreads, dyn, s>>>(P, partials, want_xnorm);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_fit(const Problem<T> &P, double *partials, int nblocks, double *out, cudaStream_t s,
                       int want_xnorm)
{
    const FitTiling L = fit_tiling(P.dims[0], P.R, (int)sizeof(T));
    const size_t dyn = (size_t)L.rt * P.R * sizeof(T);
    cudaError_t e;
    if constexpr (sizeof(T) == 8) {
        e = launch_fit_kernel<T, double>(nblocks, dyn, s, P, partials, want_xnorm);
    } else {
        if (P.x_dtype == CPD_F32) e = launch_fit_kernel<T, float>(nblocks, dyn, s, P, partials, want_xnorm);
        else e = launch_fit_kernel<T, __nv_bfloat16>(nblocks, dyn, s, P, partials, want_xnorm);
    }
    if (e != cudaSuccess) return e;
    k_fold<<<1, kThreads, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_build_replica(const void *X, void *rep, int esize, int N, const int64_t *dims, int n,
                                 int64_t ld, cudaStream_t s)
{
    long long pre = 1, post = 1;
    for (int k = 0; k < n; ++k) pre *= dims[k];
    for (int k = n + 1; k < N; ++k) post *= dims[k];
    if (n == 0) {
        const int grid = 152 * 8;
        if (esize == 8)
            k_copy_padded<double><<<grid, 256, 0, s>>>((const double *)X, (double *)rep, dims[0], post, ld);
        else if (esize == 4)
            k_copy_padded<float><<<grid, 256, 0, s>>>((const float *)X, (float *)rep, dims[0], post, ld);
        else
            k_copy_padded<unsigned short><<<grid, 256, 0, s>>>((const unsigned short *)X,
                                                               (unsigned short *)rep, dims[0], post, ld);
        return cudaGetLastError();
    }
    const dim3 block(32, 8);
    const long long ntiles = ((pre + 31) / 32) * ((dims[n] + 31) / 32) * post;
    const int grid = (int)(ntiles < 65535LL * 16 ? ntiles : 65535LL * 16);
    if (esize == 8)
        k_replica<double><<<grid, block, 0, s>>>((const double *)X, (double *)rep, pre, dims[n], post, ld);
    else if (esize == 4)
        k_replica<float><<<grid, block, 0, s>>>((const float *)X, (float *)rep, pre, dims[n], post, ld);
    else
        k_replica<unsigned short><<<grid, block, 0, s>>>((const unsigned short *)X, (unsigned short *)rep,
                                                          pre, dims[n], post, ld);
    return cudaGetLastError();
}

template size_t grad_smem_bytes<float>(const Problem<float> &);
template size_t grad_smem_bytes<double>(const Problem<double> &);
template cudaError_t launch_iteration<float>(const Problem<float> &, int, int, size_t, cudaStream_t, int,
                                             cudaEvent_t, cudaEvent_t, cudaEvent_t);
template cudaError_t launch_iteration<double>(const Problem<double> &, int, int, size_t, cudaStream_t, int,
                                              cudaEvent_t, cudaEvent_t, cudaEvent_t);
size_t lev_smem(int R) { return lev_smem_bytes(R); }

template cudaError_t launch_group_iteration<float>(const GroupLaunch<float> &, cudaStream_t);
template cudaError_t launch_group_iteration<double>(const GroupLaunch<double> &, cudaStream_t);
template cudaError_t launch_refresh_mode<float>(const Problem<float> &, int, cudaStream_t);
template cudaError_t launch_refresh_mode<double>(const Problem<double> &, int, cudaStream_t);
template cudaError_t launch_flush_dirty<float>(const Problem<float> &, cudaStream_t);
template cudaError_t launch_flush_dirty<double>(const Problem<double> &, cudaStream_t);
template cudaError_t launch_sample_probs<float>(const Problem<float> &, cudaStream_t);
template cudaError_t launch_sample_probs<double>(const Problem<double> &, cudaStream_t);
template cudaError_t launch_fit<float>(const Problem<float> &, double *, int, double *, cudaStream_t, int);
template cudaError_t launch_fit<double>(const Problem<double> &, double *, int, double *, cudaStream_t, int);

}  // namespace cpd
