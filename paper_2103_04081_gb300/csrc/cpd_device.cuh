// Device building blocks of libcpd: the counter-based generator, the
// canonical FP64 sampling arithmetic and the warp-cooperative inverse-CDF
// search. Everything here is the GPU side's own implementation of the
// published definitions cited below.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cpd_internal.h"

namespace cpd {

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplications,
// the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct U64x4 {
    unsigned long long v[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(unsigned long long c0, unsigned long long c1,
                                               unsigned long long c2, unsigned long long c3,
                                               unsigned long long k0, unsigned long long k1)
{
    const unsigned long long m0 = 0xD2E7470EE14C6C93ULL, m1 = 0xCA5A826395121157ULL;
    const unsigned long long w0 = 0x9E3779B97F4A7C15ULL, w1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += w0;
            k1 += w1;
        }
        const unsigned long long h0 = __umul64hi(m0, c0), l0 = m0 * c0;
        const unsigned long long h1 = __umul64hi(m1, c2), l1 = m1 * c2;
        const unsigned long long n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
    }
    U64x4 r;
    r.v[0] = c0; r.v[1] = c1; r.v[2] = c2; r.v[3] = c3;
    return r;
}

// Mode of iteration t (Alg. 4/5: n uniform on the N modes): counter
// (t, 2^64-1, 0, 1), word 0, scaled by a 64x64 multiply-high.
__device__ __forceinline__ int mode_draw(unsigned long long seed, long long t, int N)
{
    const U64x4 x = philox4x64_10((unsigned long long)t, ~0ULL, 0ULL, 1ULL, seed, 0ULL);
    return (int)__umul64hi(x.v[0], (unsigned long long)N);
}

// Random word of the draw of fiber f in mode k at iteration t: counter
// (t, f, k/4, 0), word k%4.
__device__ __forceinline__ unsigned long long fiber_word(unsigned long long seed, long long t,
                                                         long long f, int k)
{
    const U64x4 x = philox4x64_10((unsigned long long)t, (unsigned long long)f,
                                  (unsigned long long)(k >> 2), 0ULL, seed, 0ULL);
    return x.v[k & 3];
}

__device__ __forceinline__ double u53(unsigned long long x)
{
    return __dmul_rn((double)(x >> 11), 0x1.0p-53);
}

// ---------------------------------------------------------------------------
// Warp-cooperative inverse-CDF search (Def. 2 sampling from an FP64 CDF).
// Every lane brings one target; all 32 searches share the CDF c[0..I).
// Each lane ends with min{ i : target < c[i] } (I-1 if no such i).
// One level splits every lane's candidate range into 32 segments: the warp
// issues the 32 draws' segment-end loads back to back (one memory round trip
// per level for all 32 draws) and a ballot per draw picks the segment, so an
// I-entry CDF costs ceil(log32 I) + 1 dependent round trips.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long warp_search_cdf(const double *__restrict__ c, long long I,
                                                     double target, bool active)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const double top = __ldg(c + (I - 1));
    bool done = !active || !(target < top);
    long long result = I - 1;
    long long lo = 0, len = done ? 0 : I;
    while (__any_sync(full, len > 32)) {
        double v[32];
#pragma unroll
        for (int d = 0; d < 32; ++d) {
            const long long lo_d = __shfl_sync(full, lo, d);
            const long long len_d = __shfl_sync(full, len, d);
            if (len_d > 32) {
                const long long step = (len_d + 31) / 32;
                long long end = (long long)(lane + 1) * step;
                end = end < len_d ? end : len_d;
                v[d] = __ldg(c + lo_d + end - 1);
            } else {
                v[d] = 0.0;
            }
        }
#pragma unroll
        for (int d = 0; d < 32; ++d) {
            const long long len_d = __shfl_sync(full, len, d);
            const double tg = __shfl_sync(full, target, d);
            const unsigned m = __ballot_sync(full, tg < v[d]);
            if (len_d > 32 && lane == d) {
                const long long step = (len_d + 31) / 32;
                const int first = __ffs(m) - 1;
                lo += (long long)first * step;
                const long long rest = len - (long long)first * step;
                len = rest < step ? rest : step;
            }
        }
    }
    double v[32];
#pragma unroll
    for (int d = 0; d < 32; ++d) {
        const long long lo_d = __shfl_sync(full, lo, d);
        const long long len_d = __shfl_sync(full, len, d);
        v[d] = (lane < len_d) ? __ldg(c + lo_d + lane) : 0.0;
    }
#pragma unroll
    for (int d = 0; d < 32; ++d) {
        const long long len_d = __shfl_sync(full, len, d);
        const double tg = __shfl_sync(full, target, d);
        const unsigned m = __ballot_sync(full, (lane < len_d) && (tg < v[d]));
        if (lane == d && len_d > 0)
            result = lo + (__ffs(m) - 1);
    }
    return done ? I - 1 : result;
}

// ---------------------------------------------------------------------------
// Canonical inclusive prefix sum ("scan32") of w[0..I) by one CTA: chunks of
// 32 summed sequentially; chunk totals scanned recursively by the same rule;
// offsets added top-down. scratch needs ceil(I/31) + 8 doubles. w is read
// through L2 (other CTAs may have written it in this launch).
// ---------------------------------------------------------------------------
__device__ inline void block_scan32(const double *w, long long I, double *cdf, double *scratch)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    for (long long c = tid; c * 32 < I; c += nt) {
        double acc = 0.0;
        const long long hi = (c + 1) * 32 < I ? (c + 1) * 32 : I;
        for (long long e = c * 32; e < hi; ++e) {
            acc = __dadd_rn(acc, __ldcg(w + e));
            cdf[e] = acc;
        }
    }
    double *lev[12];
    long long levn[12];
    int L = 0;
    const double *src = cdf;
    long long cnt = I;
    double *sp = scratch;
    while (cnt > 32) {
        const long long nc = (cnt + 31) / 32;
        __syncthreads();
        for (long long c = tid; c < nc; c += nt) {
            const long long last = (c + 1) * 32 - 1 < cnt ? (c + 1) * 32 - 1 : cnt - 1;
            sp[c] = src[last];
        }
        __syncthreads();
        for (long long c = tid; c * 32 < nc; c += nt) {
            double acc = 0.0;
            const long long hi = (c + 1) * 32 < nc ? (c + 1) * 32 : nc;
            for (long long e = c * 32; e < hi; ++e) {
                acc = __dadd_rn(acc, sp[e]);
                sp[e] = acc;
            }
        }
        lev[L] = sp;
        levn[L] = nc;
        ++L;
        src = sp;
        sp += nc;
        cnt = nc;
    }
    for (int l = L - 1; l >= 0; --l) {
        __syncthreads();
        double *below = (l == 0) ? cdf : lev[l - 1];
        const long long nb = (l == 0) ? I : levn[l - 1];
        for (long long e = 32 + tid; e < nb; e += nt)
            below[e] = __dadd_rn(lev[l][e / 32 - 1], below[e]);
    }
    __syncthreads();
}

template <class XT>
__device__ __forceinline__ float to_float(XT x);
template <>
__device__ __forceinline__ float to_float<float>(float x) { return x; }
template <>
__device__ __forceinline__ float to_float<__nv_bfloat16>(__nv_bfloat16 x)
{
    return __bfloat162float(x);
}

}  // namespace cpd
