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
// Canonical inclusive prefix sum ("scan32") by one CTA, in place on a[0..I):
// chunks of 32 summed sequentially; chunk totals scanned recursively by the
// same rule; offsets added top-down. `levels` needs ceil(I/31) + 8 doubles.
// ---------------------------------------------------------------------------
__device__ inline void scan32_inplace(double *a, long long I, double *levels)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    for (long long c = tid; c * 32 < I; c += nt) {
        double acc = 0.0;
        const long long hi = (c + 1) * 32 < I ? (c + 1) * 32 : I;
        for (long long e = c * 32; e < hi; ++e) {
            acc = __dadd_rn(acc, a[e]);
            a[e] = acc;
        }
    }
    double *lev[12];
    long long levn[12];
    int L = 0;
    const double *src = a;
    long long cnt = I;
    double *sp = levels;
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
        double *below = (l == 0) ? a : lev[l - 1];
        const long long nb = (l == 0) ? I : levn[l - 1];
        for (long long e = 32 + tid; e < nb; e += nt)
            below[e] = __dadd_rn(lev[l][e / 32 - 1], below[e]);
    }
    __syncthreads();
}

// cdf[0..I) = scan32(w[0..I)). Staged through the shared buffer sm (cap
// doubles) when it fits, else in global memory with `scratch` for the levels.
// w is read through L2 (other CTAs of the launch may have written it).
__device__ inline void block_scan32(const double *w, long long I, double *cdf, double *scratch,
                                    double *sm, int cap)
{
    if (I + I / 31 + 16 <= cap) {
        for (long long e = threadIdx.x; e < I; e += blockDim.x) sm[e] = __ldcg(w + e);
        __syncthreads();
        scan32_inplace(sm, I, sm + I);
        for (long long e = threadIdx.x; e < I; e += blockDim.x) cdf[e] = sm[e];
    } else {
        for (long long e = threadIdx.x; e < I; e += blockDim.x) cdf[e] = __ldcg(w + e);
        __syncthreads();
        scan32_inplace(cdf, I, scratch);
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


// ---------------------------------------------------------------------------
// Sampling steps shared by both gradient engines.
// ---------------------------------------------------------------------------
// Draw the (N-1) x nf indices of this CTA's fibers (Alg. 3 "Randsample(I_k,
// |F_n|, true, p_k)"): warps take 32-fiber chunks per mode k != n and run the
// warp-cooperative search on cdf[k].
template <class T>
__device__ inline void draw_indices(const Problem<T> &P, long long t, int n, int f0, int nf, int *sidx)
{
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
    const int chunks = (nf + 31) / 32;
    for (int job = warp; job < chunks * P.N; job += nwarps) {
        const int k = job / chunks, ch = job % chunks;
        const int fl = ch * 32 + lane;
        const bool act = fl < nf;
        if (k == n) {
            if (act) sidx[fl * P.N + k] = -1;
            continue;
        }
        const long long Ik = P.dims[k];
        unsigned long long x = act ? fiber_word(P.seed, t, (long long)(f0 + fl), k) : 0ULL;
        long long i;
        if (P.sampling == CPD_SAMPLE_UNIFORM) {
            i = (long long)__umul64hi(x, (unsigned long long)Ik);
        } else {
            const double *c = P.cdf[k];
            const double target = __dmul_rn(u53(x), __ldg(c + (Ik - 1)));
            i = warp_search_cdf(c, Ik, target, act);
        }
        if (act) sidx[fl * P.N + k] = (int)i;
    }
}

// p_f (Eq. block_lev_prob, product in ascending k) and the weight
// s_f = 1 / (B J_n p_f) of the fiber's term in Eq. gradient1.
template <class T>
__device__ __forceinline__ double fiber_prob(const Problem<T> &P, int n, const int *row)
{
    double p = 1.0;
    for (int k = 0; k < P.N; ++k) {
        if (k == n) continue;
        if (P.sampling == CPD_SAMPLE_UNIFORM) {
            p = __dmul_rn(p, __ddiv_rn(1.0, (double)P.dims[k]));
        } else {
            const double W = __ldg(P.cdf[k] + (P.dims[k] - 1));
            p = __dmul_rn(p, __ddiv_rn(__ldg(P.w[k] + row[k]), W));
        }
    }
    return p;
}

template <class XT, class T>
__device__ __forceinline__ T load_x(const XT *p) { return (T)to_float<XT>(*p); }
template <>
__device__ __forceinline__ double load_x<double, double>(const double *p) { return *p; }


// Arrival counter: true in exactly one CTA, the last one to finish.
__device__ __forceinline__ bool last_block(unsigned *counter)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}
}  // namespace cpd
