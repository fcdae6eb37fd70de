// SKRP-ST-I materialised (Alg. 3 followed by Alg. 1): for K mini-batches of
// mode n, the sampled multi-indices (Eq. (4)), the fiber probabilities
// p_f (Eq. (10)), the sampled Khatri-Rao rows Z_S (Eq. (3)) and the sampled
// fibers X_S (Eq. (2)), written to device memory. Batch b uses the random
// words of iteration t0 + b with the mode fixed to n, from the context's
// current per-factor distributions.
//
// This is the gather on its own, spread over every SM. The unit of work is a
// warp block of 32 consecutive output fibers, owned by one warp from the
// draws to the last store, so warps never wait on one another: the lanes
// draw their fibers' indices (CDFs staged in shared memory once per CTA),
// form the column and p_f, the warp writes the multi-indices and the KRP rows
// (coalesced), then streams the 32 fibers global -> registers -> global in
// the widest unit the alignment allows, kSkUnroll units per lane in flight.
// With two CTAs (16 warps) per SM the SM holds 16 x 32 x 8 x 16 B = 64 KB of
// loads in flight, about what an SM needs to draw its share of HBM bandwidth
// at the loaded memory latency (the unrolled copy needs 124 registers, so a
// third CTA would spill); a per-CTA staged pipeline with CTA-wide barriers
// kept the loads in a serial chain behind the draws.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "cpd_device.cuh"
#include "cpd_internal.h"

namespace cpd {

namespace {

constexpr int kSkWarps = kThreads / 32;
constexpr long long kSkStageCap = 4096;  // staged CDF entries (modes != n)
constexpr int kSkUnroll = 8;             // copy units in flight per lane

struct SkrpArgs {
    int n, K;
    long long t0;
    int *idx;        // K B x N
    double *p;       // K B
    float *Z;        // K B x R
    void *X;         // K B x ld_n elements
    long long units; // copy units per fiber (ld_n * esize / unit)
    int unit;        // copy unit in bytes: 16, 8, 4 or 2
};

// The 32 fibers of one warp block: fiber u's units [0, units) start at
// rep + jc[u] * units; the output is contiguous. Lane-strided over the flat
// unit index, the (fiber, offset) pair carried along instead of divided out.
// units < 2^26 (the fiber is under 1 GB), so a warp block's flat index fits
// 32 bits.
template <class U>
__device__ __forceinline__ void copy_fibers(const U *__restrict__ rep, const long long *jc, int nf, int units,
                                            U *__restrict__ dst, int lane)
{
    const int total = nf * units;
    int u = 0, r = lane;
    while (r >= units) {
        r -= units;
        ++u;
    }
    for (int base = 0; base < total; base += 32 * kSkUnroll) {
        U v[kSkUnroll];
#pragma unroll
        for (int j = 0; j < kSkUnroll; ++j) {
            if (base + j * 32 + lane < total) v[j] = __ldcs(rep + jc[u] * units + r);
            r += 32;
            while (r >= units) {
                r -= units;
                ++u;
            }
        }
#pragma unroll
        for (int j = 0; j < kSkUnroll; ++j) {
            const int c = base + j * 32 + lane;
            if (c < total) __stcs(dst + c, v[j]);
        }
    }
}

}  // namespace

// kGlobal: a mode's CDFs too long to stage are searched in global memory
// (the warp-cooperative 32-way search, which needs its own 64 registers).
template <bool kGlobal>
__global__ void __launch_bounds__(kThreads, 2) k_skrp(const Problem<float> P, const SkrpArgs s)
{
    extern __shared__ __align__(16) unsigned long long cdfs[];
    __shared__ int sidx_all[kSkWarps][32 * kMaxModes];
    __shared__ long long jc_all[kSkWarps][32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = P.N, R = P.R, n = s.n;
    const long long B = P.B, total = (long long)s.K * B;
    __shared__ long long off[kMaxModes];
    __shared__ int ks[kMaxModes];   // the modes k != n, ascending
    int *sidx = sidx_all[warp];
    long long *jc = jc_all[warp];
    // staged CDFs of the modes k != n (ascending), when they fit
    long long need = 0;
    for (int k = 0; k < N; ++k) {
        if (tid == 0) {
            off[k] = need;
            ks[k - (k > n)] = k;   // k == n writes slot n, which k = n + 1 overwrites
        }
        if (k != n) need += P.dims[k];
    }
    const bool staged = P.sampling != CPD_SAMPLE_UNIFORM && !kGlobal;
    __syncthreads();
    if (staged) {
        for (int k = 0; k < N; ++k)
            if (k != n)
                for (long long i = tid; i < P.dims[k]; i += blockDim.x) cdfs[off[k] + i] = __ldcg(P.cdf[k] + i);
        __syncthreads();
    }
    const long long nwb = (total + 31) / 32;
    for (long long wb = (long long)blockIdx.x * kSkWarps + warp; wb < nwb; wb += (long long)gridDim.x * kSkWarps) {
        const long long fg0 = wb * 32;
        const int nf = (int)((total - fg0) < 32 ? total - fg0 : 32);
        const bool act = lane < nf;
        const long long fg = fg0 + (act ? lane : 0);
        const long long b = fg / B, f = fg % B;
        // draws (Alg. 3): one Philox block per group of four modes
        U64x4 words{};
        for (int k = 0; k < N; ++k) {
            if ((k & 3) == 0)
                words = philox4x64_10((unsigned long long)(s.t0 + b), (unsigned long long)f,
                                      (unsigned long long)(k >> 2), 0ULL, P.seed, 0ULL);
            if (k == n) {
                if (act) sidx[lane * N + k] = -1;
                continue;
            }
            const long long Ik = P.dims[k];
            const int q = k & 3;
            const unsigned long long w = q == 0 ? words.v[0] : q == 1 ? words.v[1] : q == 2 ? words.v[2] : words.v[3];
            const unsigned long long x = act ? w : 0ULL;
            long long i;
            if (P.sampling == CPD_SAMPLE_UNIFORM) {
                i = (long long)__umul64hi(x, (unsigned long long)Ik);
            } else if (!kGlobal) {
                const unsigned long long *c = cdfs + off[k];
                i = warp_search_staged(c, Ik, __umul64hi(x, c[Ik - 1]), act);
            } else {
                const unsigned long long *c = P.cdf[k];
                i = warp_search_cdf(c, Ik, __umul64hi(x, __ldg(c + (Ik - 1))), act);
            }
            if (act) sidx[lane * N + k] = (int)i;
        }
        __syncwarp();
        // column (Eq. (2)) and p_f (Eq. (10), FP64), one lane per fiber
        if (act) {
            const int *row = sidx + lane * N;
            long long j = 0, Jp = 1;
            for (int k = 0; k < N; ++k) {
                if (k == n) continue;
                j += (long long)row[k] * Jp;
                Jp *= P.dims[k];
            }
            jc[lane] = j;
            if (s.p) s.p[fg] = fiber_prob_staged(P, n, row, staged ? cdfs : nullptr);
        }
        __syncwarp();
        // the multi-indices, contiguous for the warp block
        if (s.idx)
            for (int e = lane; e < nf * N; e += 32) s.idx[fg0 * N + e] = sidx[e];
        // sampled KRP rows (Eq. (3)), factor rows multiplied in ascending k;
        // lane-strided over the warp block's nf x R entries, kSkUnroll at a
        // time, two factors at a time so that 2 kSkUnroll loads are in flight
        if (s.Z) {
            const int nk = N - 1;
            const int tot = nf * R;
            int fl = 0, r = lane;
            while (r >= R) {
                r -= R;
                ++fl;
            }
            for (int base = 0; base < tot; base += 32 * kSkUnroll) {
                float z[kSkUnroll];
                int fe[kSkUnroll], re[kSkUnroll];
#pragma unroll
                for (int j = 0; j < kSkUnroll; ++j) {
                    z[j] = 1.f;
                    fe[j] = fl;
                    re[j] = r;
                    r += 32;
                    while (r >= R) {
                        r -= R;
                        ++fl;
                    }
                }
                for (int q = 0; q < nk; q += 2) {
                    const int ka = ks[q], kb = q + 1 < nk ? ks[q + 1] : -1;
                    float va[kSkUnroll], vb[kSkUnroll];
#pragma unroll
                    for (int j = 0; j < kSkUnroll; ++j) {
                        const bool in = base + j * 32 + lane < tot;
                        va[j] = in ? __ldg(P.A[ka] + (long long)sidx[fe[j] * N + ka] * R + re[j]) : 1.f;
                        vb[j] = (in && kb >= 0) ? __ldg(P.A[kb] + (long long)sidx[fe[j] * N + kb] * R + re[j]) : 1.f;
                    }
#pragma unroll
                    for (int j = 0; j < kSkUnroll; ++j) {
                        z[j] = z[j] * va[j];
                        if (kb >= 0) z[j] = z[j] * vb[j];
                    }
                }
#pragma unroll
                for (int j = 0; j < kSkUnroll; ++j) {
                    const int c = base + j * 32 + lane;
                    if (c < tot) s.Z[fg0 * R + c] = z[j];
                }
            }
        }
        // the sampled fibers
        if (s.X) {
            const int ub = (int)s.units;
            char *out = static_cast<char *>(s.X) + (size_t)fg0 * ub * s.unit;
            const char *rep = reinterpret_cast<const char *>(P.rep[n]);
            switch (s.unit) {
            case 16:
                copy_fibers(reinterpret_cast<const uint4 *>(rep), jc, nf, ub, reinterpret_cast<uint4 *>(out), lane);
                break;
            case 8:
                copy_fibers(reinterpret_cast<const uint2 *>(rep), jc, nf, ub, reinterpret_cast<uint2 *>(out), lane);
                break;
            case 4:
                copy_fibers(reinterpret_cast<const unsigned *>(rep), jc, nf, ub, reinterpret_cast<unsigned *>(out),
                            lane);
                break;
            default:
                copy_fibers(reinterpret_cast<const unsigned short *>(rep), jc, nf, ub,
                            reinterpret_cast<unsigned short *>(out), lane);
                break;
            }
        }
        __syncwarp();   // sidx / jc are rewritten by the next warp block
    }
}

size_t skrp_smem_bytes(const Problem<float> &P, int n, int esize)
{
    (void)esize;
    long long need = 0;
    for (int k = 0; k < P.N; ++k)
        if (k != n) need += P.dims[k];
    const bool staged = P.sampling != CPD_SAMPLE_UNIFORM && need <= kSkStageCap;
    return staged ? (size_t)need * 8 : 0;
}

cudaError_t launch_skrp(const Problem<float> &P, int n, long long t0, int K, int *idx, double *p, float *Z, void *X,
                        int esize, int sm_count, cudaStream_t stream)
{
    SkrpArgs a{};
    a.n = n;
    a.K = K;
    a.t0 = t0;
    a.idx = idx;
    a.p = p;
    a.Z = Z;
    a.X = X;
    // the widest unit dividing the fiber length and both base addresses
    // (replica fibers start at multiples of ld_n * esize bytes)
    const unsigned long long fb = (unsigned long long)P.ld[n] * esize;
    const unsigned long long mix = fb | (unsigned long long)(uintptr_t)X | (unsigned long long)(uintptr_t)P.rep[n];
    a.unit = (mix % 16 == 0) ? 16 : (mix % 8 == 0) ? 8 : (mix % 4 == 0) ? 4 : 2;
    a.units = (long long)(fb / a.unit);
    // staged CDFs take at most kSkStageCap * 8 = 32 KB: no opt-in needed
    const size_t smem = skrp_smem_bytes(P, n, esize);
    const bool global = P.sampling != CPD_SAMPLE_UNIFORM && smem == 0;
    const void *fn = global ? (const void *)k_skrp<true> : (const void *)k_skrp<false>;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long long nwb = ((long long)K * P.B + 31) / 32;
    const long long want = (nwb + kSkWarps - 1) / kSkWarps;
    const int grid = (int)std::min<long long>(want, (long long)per_sm * sm_count);
    if (global)
        k_skrp<true><<<grid, kThreads, smem, stream>>>(P, a);
    else
        k_skrp<false><<<grid, kThreads, smem, stream>>>(P, a);
    return cudaGetLastError();
}

}  // namespace cpd
