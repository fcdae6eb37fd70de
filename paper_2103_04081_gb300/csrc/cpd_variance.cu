// Gradient-variance diagnostic (Thm 10, Table 1, Fig. 3).
//
// For mode n and the current factors, the mini-batch gradient of Eq. (11)
// is G = (1/(B J_n)) sum_f (1/p_f) r_f z_f^T with r_f = A z_f - x_f
// (the residual column of fiber f, Eq. (2)) and B draws i.i.d. from p. Its
// conditional moments are exact sums over all J_n fibers j:
//   S1 = sum_j ||r_j||^2 ||z_j||^2 / p_j,   M = sum_j r_j z_j^T,
//   E[G] = M / J_n,   E||G - E[G]||_F^2 = (S1 - ||M||_F^2) / (B J_n^2),
// Thm 10 in the normalisation of Eq. (11) (the paper's form is J_n^2
// times this). Fibers with p_j = 0 are never drawn and are left out of both
// sums.
//
// k_variance: CTA (row tile of 256 rows, fiber chunk) walks its chunk of
// fibers 32 at a time. One warp per fiber forms z_j (FP32 products of factor
// rows), ||z_j||^2 (FP64) and p_j (FP64, the sampler's own fixed-point
// distribution); then every thread owns one row i of the tile and adds
// r_ij^2 ||z_j||^2 / p_j to its S1 partial and r_ij z_j to its row of M in
// shared memory (FP64). k_var_fold sums the chunks' M tiles and the S1
// partials in a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cpd_device.cuh"
#include "cpd_internal.h"

namespace cpd {

namespace {

constexpr int kVarRows = kThreads;   // rows of A^(n) per CTA, one per thread
constexpr int kVarFib = 32;          // fibers staged per round
constexpr int kVarMaxR = 64;

size_t var_smem(int R)
{
    return (size_t)R * kVarRows * 8      // M tile, [r][row]
           + (size_t)R * kVarRows * 4    // A^(n) tile, [r][row]
           + (size_t)kVarFib * R * 4     // z of the round's fibers
           + (size_t)kVarFib * 8;        // ||z||^2 / p of the round's fibers
}

template <class XT>
__device__ __forceinline__ float xval(XT v)
{
    if constexpr (sizeof(XT) == 8) return (float)v;
    else return to_float<XT>(v);
}

template <class T, class XT>
__global__ void __launch_bounds__(kThreads) k_variance(const Problem<T> P, int n, int chunks, double *partM,
                                                       double *partS)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = P.R, N = P.N;
    const long long In = P.dims[n];
    const int ntile = (int)((In + kVarRows - 1) / kVarRows);
    const int tile = blockIdx.x % ntile, chunk = blockIdx.x / ntile;
    const long long J = (long long)P.Jn[n];
    const long long j0 = J * chunk / chunks, j1 = J * (chunk + 1) / chunks;
    double *sM = reinterpret_cast<double *>(smem);
    float *sA = reinterpret_cast<float *>(sM + (size_t)R * kVarRows);
    float *sz = sA + (size_t)R * kVarRows;
    double *sw = reinterpret_cast<double *>(sz + (size_t)kVarFib * R);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long row = (long long)tile * kVarRows + threadIdx.x;
    const bool own = row < In;

    for (int r = 0; r < R; ++r) {
        sM[r * kVarRows + threadIdx.x] = 0.0;
        sA[r * kVarRows + threadIdx.x] = own ? (float)P.A[n][row * R + r] : 0.f;
    }
    double S = 0.0;
    const XT *rep = reinterpret_cast<const XT *>(P.rep[n]);
    for (long long jb = j0; jb < j1; jb += kVarFib) {
        const int nf = (int)((j1 - jb) < kVarFib ? (j1 - jb) : kVarFib);
        __syncthreads();
        for (int f = warp; f < nf; f += kThreads / 32) {
            // indices of fiber j (Eq. (2): first mode fastest, mode n skipped)
            int idx[kMaxModes];
            long long rest = jb + f;
            for (int k = 0; k < N; ++k) {
                if (k == n) {
                    idx[k] = -1;
                    continue;
                }
                idx[k] = (int)(rest % P.dims[k]);
                rest /= P.dims[k];
            }
            const double p = fiber_prob(P, n, idx);
            double zz = 0.0;
            for (int r = lane; r < R; r += 32) {
                float z = 1.f;
                for (int k = 0; k < N; ++k)
                    if (k != n) z *= (float)P.A[k][(long long)idx[k] * R + r];
                if (!(p > 0.0)) z = 0.f;
                sz[f * R + r] = z;
                zz += (double)z * (double)z;
            }
            for (int off = 16; off > 0; off >>= 1) zz += __shfl_down_sync(0xffffffffu, zz, off);
            if (lane == 0) sw[f] = p > 0.0 ? zz / p : 0.0;
        }
        __syncthreads();
        if (own) {
            for (int f = 0; f < nf; ++f) {
                const float x = xval<XT>(rep[fiber_start(P, n, jb + f) + row * fiber_step(P, n)]);
                float res = -x;
                for (int r = 0; r < R; ++r) res = fmaf(sA[r * kVarRows + threadIdx.x], sz[f * R + r], res);
                if (sw[f] == 0.0) continue;   // never drawn
                S += sw[f] * ((double)res * (double)res);
                for (int r = 0; r < R; ++r)
                    sM[r * kVarRows + threadIdx.x] += (double)(res * sz[f * R + r]);
            }
        }
    }
    __syncthreads();
    // this chunk's rows of M, [chunk][row][r]
    if (own)
        for (int r = 0; r < R; ++r) partM[((long long)chunk * In + row) * R + r] = sM[r * kVarRows + threadIdx.x];
    // S1 partial: fixed-order block reduction
    __shared__ double s_red[kThreads];
    s_red[threadIdx.x] = S;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s_red[threadIdx.x] += s_red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partS[blockIdx.x] = s_red[0];
}

// out2[0] = S1 (sum of the CTAs' partials in order), out2[1] = ||M||_F^2 with
// M = sum over chunks (in order) of the chunk tiles. One CTA.
__global__ void __launch_bounds__(kThreads) k_var_fold(const double *partM, int chunks, long long entries,
                                                       const double *partS, int nS, double *out2)
{
    __shared__ double s_red[kThreads];
    double acc = 0.0;
    for (long long e = threadIdx.x; e < entries; e += kThreads) {
        double m = 0.0;
        for (int c = 0; c < chunks; ++c) m += partM[(long long)c * entries + e];
        acc += m * m;
    }
    s_red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s_red[threadIdx.x] += s_red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double s1 = 0.0;
        for (int q = 0; q < nS; ++q) s1 += partS[q];
        out2[0] = s1;
        out2[1] = s_red[0];
    }
}

template <class T, class XT>
cudaError_t run_variance(const Problem<T> &P, int n, double *out2, cudaStream_t s)
{
    if (P.R > kVarMaxR) return cudaErrorInvalidValue;
    const long long In = P.dims[n];
    const long long J = (long long)P.Jn[n];
    const int ntile = (int)((In + kVarRows - 1) / kVarRows);
    long long chunks = (2 * 152 + ntile - 1) / ntile;
    if (chunks > J) chunks = J;
    if (chunks < 1) chunks = 1;
    const int grid = ntile * (int)chunks;
    const size_t smem = var_smem(P.R);
    static size_t attr = 0;
    cudaError_t e = cudaSuccess;
    if (smem > attr) {
        e = cudaFuncSetAttribute(k_variance<T, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        attr = smem;
    }
    double *partM = nullptr, *partS = nullptr;
    e = cudaMallocAsync((void **)&partM, (size_t)chunks * In * P.R * sizeof(double), s);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync((void **)&partS, (size_t)grid * sizeof(double), s);
    if (e == cudaSuccess) {
        k_variance<T, XT><<<grid, kThreads, smem, s>>>(P, n, (int)chunks, partM, partS);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_var_fold<<<1, kThreads, 0, s>>>(partM, (int)chunks, In * P.R, partS, grid, out2);
        e = cudaGetLastError();
    }
    cudaFreeAsync(partM, s);
    if (partS) cudaFreeAsync(partS, s);
    return e;
}

}  // namespace

template <class T>
cudaError_t launch_variance(const Problem<T> &P, int n, double *out2, cudaStream_t s)
{
    if constexpr (sizeof(T) == 8) {
        return run_variance<T, double>(P, n, out2, s);
    } else {
        if (P.x_dtype == CPD_F32) return run_variance<T, float>(P, n, out2, s);
        return run_variance<T, __nv_bfloat16>(P, n, out2, s);
    }
}

template cudaError_t launch_variance<float>(const Problem<float> &, int, double *, cudaStream_t);
template cudaError_t launch_variance<double>(const Problem<double> &, int, double *, cudaStream_t);

}  // namespace cpd
