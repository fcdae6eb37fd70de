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

// Phase timestamp (%globaltimer, ns) into P.trace[slot] from one thread of the
// chosen CTA, when tracing is on.
__device__ __forceinline__ void trace_stamp(unsigned long long *trace, int slot, bool cta)
{
    if (trace && cta && threadIdx.x == 0) {
        unsigned long long ns;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
        trace[slot] = ns;
    }
}

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

// ---------------------------------------------------------------------------
// Warp-cooperative inverse-CDF search (Def. 2 sampling). The CDF is exact
// 64-bit fixed point: cdf[i] = q_0 + ... + q_i. Every lane brings one target
// t = floor(x Q / 2^64) and ends with min{ i : t < cdf[i] }. One level splits
// every lane's candidate range into 32 segments: the warp issues the 32
// draws' segment-end loads back to back (one memory round trip per level for
// all 32 draws) and a ballot per draw picks the segment, so an I-entry CDF
// costs ceil(log32 I) + 1 dependent round trips. Kept out of line: its
// unrolled levels are long (about 130 KB of code), run only when the CDFs do
// not fit the staging buffer, and would otherwise sit inside every sampler's
// loop and lengthen the code each launch fetches.
// ---------------------------------------------------------------------------
static __device__ __noinline__ long long warp_search_cdf(const unsigned long long *__restrict__ c, long long I,
                                                     unsigned long long target, bool active)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    long long result = I - 1;
    long long lo = 0, len = active ? I : 0;
    while (__any_sync(full, len > 32)) {
        unsigned long long v[32];
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
                v[d] = 0;
            }
        }
#pragma unroll
        for (int d = 0; d < 32; ++d) {
            const long long len_d = __shfl_sync(full, len, d);
            const unsigned long long tg = __shfl_sync(full, target, d);
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
    unsigned long long v[32];
#pragma unroll
    for (int d = 0; d < 32; ++d) {
        const long long lo_d = __shfl_sync(full, lo, d);
        const long long len_d = __shfl_sync(full, len, d);
        v[d] = (lane < len_d) ? __ldg(c + lo_d + lane) : 0;
    }
#pragma unroll
    for (int d = 0; d < 32; ++d) {
        const long long len_d = __shfl_sync(full, len, d);
        const unsigned long long tg = __shfl_sync(full, target, d);
        const unsigned m = __ballot_sync(full, (lane < len_d) && (tg < v[d]));
        if (lane == d && len_d > 0) result = m ? lo + (__ffs(m) - 1) : I - 1;
    }
    return result;
}

// Warp-cooperative search over a CDF held in shared memory. The first level
// is common to all 32 draws: lane l loads one splitter c[min((l+1)step, I)-1]
// (step = ceil(I/32)), and each lane finds its segment by a binary search
// over the 32 splitters through shuffles; the lane then finishes inside its
// segment (at most step entries) with a binary search of its own.
__device__ __forceinline__ long long warp_search_staged(const unsigned long long *c, long long I,
                                                        unsigned long long target, bool active)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long step = (I + 31) / 32;
    long long e = (long long)(lane + 1) * step;
    e = (e < I ? e : I) - 1;
    const unsigned long long split = c[e];
    // segment = number of splitters <= target (splitter 31 = c[I-1] > target)
    int seg = 0;
#pragma unroll
    for (int half = 16; half >= 1; half >>= 1) {
        const unsigned long long v = __shfl_sync(full, split, seg + half - 1);
        if (v <= target) seg += half;
    }
    long long lo = (long long)seg * step;
    long long len = I - lo < step ? I - lo : step;
    if (!active || len <= 0) return I - 1;
    while (len > 1) {
        const long long h = len >> 1;
        if (target < c[lo + h - 1]) {
            len = h;
        } else {
            lo += h;
            len -= h;
        }
    }
    return lo;
}

// Row weight of the Euclidean distribution (Def. 5, Lemma 4) in the canonical
// order, by one warp: lane l accumulates a_r^2 for r = l, l+32, ... (fma from
// +0), then the shuffle-down tree adds lane l+off into lane l for off =
// 16..1. The FP64 dependency chain is ceil(R/32) + 5 operations long.
template <class T>
__device__ __forceinline__ double warp_row_weight(const T *row, int R)
{
    double acc = 0.0;
    for (int r = threadIdx.x & 31; r < R; r += 32) {
        const double a = (double)row[r];
        acc = __fma_rn(a, a, acc);
    }
    for (int off = 16; off >= 1; off >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(0xffffffffu, acc, off));
    return acc;
}

// floor(w 2^s) for a finite w >= 0, exactly, on the integer pipe: w = M 2^e
// with an integer mantissa M.
__device__ __forceinline__ unsigned long long quantize(double w, int s)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(w);
    const int ef = (int)(bits >> 52);
    const unsigned long long frac = bits & ((1ULL << 52) - 1);
    const unsigned long long M = ef ? (frac | (1ULL << 52)) : frac;
    const int e = (ef ? ef : 1) - 1075;
    const int sh = e + s;
    if (sh >= 0) return M << sh;   // bounded by 2^62 through the choice of s
    if (sh <= -64) return 0;
    return M >> (-sh);
}

// In place: `a` holds the bit patterns of the FP64 row weights w[0..I) on
// entry and the fixed-point CDF (same definition as block_distribution) on
// exit. Each thread transforms a contiguous chunk, reading every weight
// before overwriting it. `sm` holds 2 * kThreads uint64 slots. Returns false
// in every thread when the distribution has no mass. Blocks of kThreads
// threads: the warps' partials are then combined by unrolled loops whose
// shared-memory loads are independent.
__device__ inline bool block_distribution_inplace(unsigned long long *a, long long I, unsigned long long *sm)
{
    constexpr int nt = kThreads, nw = kThreads / 32;
    const int tid = threadIdx.x;
    long long mx = 0;
    int bad = 0;
    for (long long i = tid; i < I; i += nt) {
        const double v = __longlong_as_double((long long)a[i]);
        if (!(v >= 0.0) || isinf(v)) bad = 1;
        const long long b = (long long)a[i];
        mx = b > mx ? b : mx;
    }
    for (int off = 16; off >= 1; off >>= 1) {
        const long long o = __shfl_down_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
    }
    bad = __syncthreads_or(bad);
    if ((tid & 31) == 0) sm[tid >> 5] = (unsigned long long)mx;
    __syncthreads();
    long long gmx = 0;
#pragma unroll
    for (int q = 0; q < nw; ++q) gmx = (long long)sm[q] > gmx ? (long long)sm[q] : gmx;
    __syncthreads();
    const double wmax = __longlong_as_double(gmx);
    if (bad || !(wmax > 0.0)) return false;
    const int ef = (int)((unsigned long long)gmx >> 52);
    const int lg = ef ? ef - 1023 : 63 - __clzll(gmx) - 1074;
    int L = 0;
    while ((1LL << L) < I) ++L;
    const int s = 61 - L - lg;
    const long long chunk = (I + nt - 1) / nt;
    const long long i0 = tid * chunk, i1 = (i0 + chunk < I) ? i0 + chunk : I;
    unsigned long long tot = 0;
    for (long long i = i0; i < i1; ++i) tot += quantize(__longlong_as_double((long long)a[i]), s);
    unsigned long long inc = tot;
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, off);
        if ((tid & 31) >= off) inc += o;
    }
    if ((tid & 31) == 31) sm[nt + (tid >> 5)] = inc;
    __syncthreads();
    unsigned long long acc = 0, Q = 0;
#pragma unroll
    for (int q = 0; q < nw; ++q) {
        const unsigned long long v = sm[nt + q];
        if (q < (tid >> 5)) acc += v;
        Q += v;
    }
    acc += inc - tot;
    for (long long i = i0; i < i1; ++i) {
        acc += quantize(__longlong_as_double((long long)a[i]), s);
        a[i] = acc;
    }
    __syncthreads();
    return Q > 0;
}

// Copy n words from global into shared memory, eight loads in flight a
// thread: a loop that stores each word before loading the next pays one
// memory latency per word it copies. kL2: load through L2 only (words other
// CTAs of the same launch may have written).
template <class W, bool kL2>
__device__ __forceinline__ void stage_words(W *dst, const W *src, long long n)
{
    const long long nt = blockDim.x;
    for (long long i0 = threadIdx.x; i0 < n; i0 += 8 * nt) {
        W v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const long long i = i0 + u * nt;
            v[u] = i < n ? (kL2 ? __ldcg(src + i) : __ldg(src + i)) : W(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const long long i = i0 + u * nt;
            if (i < n) dst[i] = v[u];
        }
    }
}

// ---------------------------------------------------------------------------
// The fixed-point distribution of one factor from its FP64 row weights, by
// one CTA: s = 61 - ceil(log2 I) - floor(log2 max w), q_i = floor(w_i 2^s),
// cdf = inclusive prefix sum of q (exact, so any summation order gives the
// same bits). Returns false (in every thread) when a weight is negative or
// not finite, or when every q_i is 0. `sm` holds 2 * kThreads uint64 slots.
// w is read through L2 (other CTAs of the launch may have written it).
// ---------------------------------------------------------------------------
// Out of line: the iteration kernels call it only where a CDF is rebuilt at
// once (not deferred), and its body would otherwise lengthen their code.
static __device__ __noinline__ bool block_distribution(const double *wg, long long I, unsigned long long *cdf,
                                                       unsigned long long *sm, double *wstage, long long wcap)
{
    constexpr int nt = kThreads, nw = kThreads / 32;   // blocks of kThreads threads
    const int tid = threadIdx.x;
    const double *w = wg;
    if (wstage && I <= wcap) {   // one coalesced pass through L2, then shared memory
        stage_words<double, true>(wstage, wg, I);
        __syncthreads();
        w = wstage;
    }
    // largest weight, through the integer order of non-negative doubles
    long long mx = 0;
    int bad = 0;
    for (long long i = tid; i < I; i += nt) {
        const double v = w == wg ? __ldcg(w + i) : w[i];
        if (!(v >= 0.0) || isinf(v)) bad = 1;
        const long long b = __double_as_longlong(v);
        mx = b > mx ? b : mx;
    }
    for (int off = 16; off >= 1; off >>= 1) {
        const long long o = __shfl_down_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
    }
    bad = __syncthreads_or(bad);
    if ((tid & 31) == 0) sm[tid >> 5] = (unsigned long long)mx;
    __syncthreads();
    long long gmx = 0;
#pragma unroll
    for (int q = 0; q < nw; ++q) gmx = (long long)sm[q] > gmx ? (long long)sm[q] : gmx;
    __syncthreads();
    const double wmax = __longlong_as_double(gmx);
    if (bad || !(wmax > 0.0)) return false;
    // floor(log2 wmax): exponent field for a normal number, leading bit for a subnormal
    const int ef = (int)((unsigned long long)gmx >> 52);
    const int lg = ef ? ef - 1023 : 63 - __clzll(gmx) - 1074;
    int L = 0;
    while ((1LL << L) < I) ++L;
    const int s = 61 - L - lg;
    // exact prefix sum: contiguous chunk per thread, then an exclusive scan of
    // the chunk totals across the CTA
    const long long chunk = (I + nt - 1) / nt;
    const long long i0 = tid * chunk, i1 = (i0 + chunk < I) ? i0 + chunk : I;
    unsigned long long tot = 0;
    for (long long i = i0; i < i1; ++i) tot += quantize(w == wg ? __ldcg(w + i) : w[i], s);
    unsigned long long inc = tot;
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, off);
        if ((tid & 31) >= off) inc += o;
    }
    if ((tid & 31) == 31) sm[nt + (tid >> 5)] = inc;
    __syncthreads();
    unsigned long long base = 0, Q = 0;
#pragma unroll
    for (int q = 0; q < nw; ++q) {
        const unsigned long long v = sm[nt + q];
        if (q < (tid >> 5)) base += v;
        Q += v;
    }
    unsigned long long acc = base + inc - tot;
    for (long long i = i0; i < i1; ++i) {
        acc += quantize(w == wg ? __ldcg(w + i) : w[i], s);
        cdf[i] = acc;
    }
    __syncthreads();
    return Q > 0;
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


// Blocks (Remark 1): the mode whose rows form the blocks of mode n's fibers
// (the first mode other than n: the fastest-varying index of Eq. (2)).
__device__ __forceinline__ int block_mode(int n) { return n == 0 ? 1 : 0; }

// q of row i of a CDF, or of i's whole block of bs rows (its exact sum).
__device__ __forceinline__ unsigned long long row_mass(const unsigned long long *c, long long i, int bs)
{
    const long long b0 = bs > 1 ? i / bs * bs : i, b1 = b0 + bs - 1;
    return c[b1] - (b0 > 0 ? c[b0 - 1] : 0ULL);
}

// ---------------------------------------------------------------------------
// Sampling steps shared by both gradient engines.
// ---------------------------------------------------------------------------
// Draw the (N-1) x nf indices of this CTA's fibers (Alg. 3: for every mode
// k != n, |F_n| independent draws from p_k, with replacement). When the CDFs of the modes k != n fit the shared
// buffer `stage` (cap entries) they are copied there first (one coalesced
// pass) and searched there; otherwise the warp-cooperative multi-level
// search runs on the global copies. Warps take 32-fiber chunks per mode.
//
// When CDF rebuilds are deferred (P.defer_cdf), the mode updated last
// (*P.dirty) has only fresh row weights: its CDF is rebuilt here, in the
// staging buffer, from those weights (scratch: `dsm`, 2 * kThreads uint64),
// and the one CTA of the launch that passes `writer` stores it for later
// iterations.
template <class T>
__device__ inline void draw_indices(const Problem<T> &P, long long t, int n, int f0, int nf, int *sidx,
                                    unsigned long long *stage, long long cap, unsigned long long *dsm,
                                    bool writer)
{
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
    long long need = 0, off[kMaxModes];
    for (int k = 0; k < P.N; ++k) {
        off[k] = need;
        if (k != n) need += P.dims[k];
    }
    const bool staged = P.sampling != CPD_SAMPLE_UNIFORM && stage != nullptr && need <= cap;
    if (staged) {
        const int dirty = P.defer_cdf ? *P.dirty : -1;
        for (int k = 0; k < P.N; ++k) {
            if (k == n) continue;
            if (k == dirty)
                stage_words<unsigned long long, true>(stage + off[k],
                                                      reinterpret_cast<const unsigned long long *>(P.w[k]), P.dims[k]);
            else
                stage_words<unsigned long long, false>(stage + off[k], P.cdf[k], P.dims[k]);
        }
        __syncthreads();
        trace_stamp(P.trace, 29, blockIdx.x == 0);
        if (dirty >= 0 && dirty != n) {
            unsigned long long *c = stage + off[dirty];
            if (!block_distribution_inplace(c, P.dims[dirty], dsm)) {
                if (threadIdx.x == 0) atomicOr(P.status, kStDegenerate);
            } else if (writer) {
                for (long long i = threadIdx.x; i < P.dims[dirty]; i += blockDim.x) P.cdf[dirty][i] = c[i];
            }
        }
        trace_stamp(P.trace, 30, blockIdx.x == 0);
    }
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
        // blocks (Remark 1): block f / bs draws once per mode from the word of
        // (t, f / bs, k); for the blocks' mode k0 the drawn row stands for its
        // block and fiber f takes row f % bs of it (bs = 1: one draw per fiber)
        const int bs = P.block;
        const long long f = (long long)(f0 + fl);
        const unsigned long long x = act ? fiber_word(P.seed, t, bs > 1 ? f / bs : f, k) : 0ULL;
        long long i;
        if (P.sampling == CPD_SAMPLE_UNIFORM) {
            i = (long long)__umul64hi(x, (unsigned long long)Ik);
        } else if (staged) {
            const unsigned long long *c = stage + off[k];
            i = warp_search_staged(c, Ik, __umul64hi(x, c[Ik - 1]), act);
        } else {
            const unsigned long long *c = P.cdf[k];
            i = warp_search_cdf(c, Ik, __umul64hi(x, __ldg(c + (Ik - 1))), act);
        }
        if (bs > 1 && k == block_mode(n)) i = i / bs * bs + f % bs;
        if (act) sidx[fl * P.N + k] = (int)i;
    }
}

// p_f = prod_{k != n, ascending} q_k(i_k) / Q_k in FP64 (Eq. (10)),
// for the record of the last batch; uniform: q = 1, Q = I_k. With blocks,
// k0's factor is the probability of i_k0's block.
template <class T>
__device__ __forceinline__ double fiber_prob(const Problem<T> &P, int n, const int *row)
{
    double p = 1.0;
    for (int k = 0; k < P.N; ++k) {
        if (k == n) continue;
        const int bs = k == block_mode(n) ? P.block : 1;
        if (P.sampling == CPD_SAMPLE_UNIFORM) {
            p = __dmul_rn(p, __ddiv_rn((double)bs, (double)P.dims[k]));
        } else {
            const unsigned long long *c = P.cdf[k];
            const unsigned long long q = row_mass(c, row[k], bs);
            p = __dmul_rn(p, __ddiv_rn(__ull2double_rn(q), __ull2double_rn(c[P.dims[k] - 1])));
        }
    }
    return p;
}

// fiber_prob on the staged CDFs (stage == nullptr: the global ones).
template <class T>
__device__ __forceinline__ double fiber_prob_staged(const Problem<T> &P, int n, const int *row,
                                                    const unsigned long long *stage)
{
    if (!stage) return fiber_prob(P, n, row);
    double p = 1.0;
    long long off = 0;
    for (int k = 0; k < P.N; ++k) {
        if (k == n) continue;
        const unsigned long long *c = stage + off;
        const unsigned long long q = row_mass(c, row[k], k == block_mode(n) ? P.block : 1);
        p = __dmul_rn(p, __ddiv_rn(__ull2double_rn(q), __ull2double_rn(c[P.dims[k] - 1])));
        off += P.dims[k];
    }
    return p;
}

// The fiber's weight in Eq. (11), s_f = 1 / (B J_n p_f), in FP32 (the
// gradient's own precision): (1/(B J_n)) prod_k Q_k / q_k(i_k). With blocks
// of bs fibers, 1 / ((B / bs) J_n p_b): P.inv_bj carries the factor bs and
// k0's q is its block's.
// Out of line: it serves only CDFs too long to stage (see warp_search_cdf).
template <class T>
static __device__ __noinline__ float fiber_weight(const Problem<T> &P, int n, const int *row)
{
    float s = P.inv_bj[n];
    for (int k = 0; k < P.N; ++k) {
        if (k == n) continue;
        const int bs = k == block_mode(n) ? P.block : 1;
        if (P.sampling == CPD_SAMPLE_UNIFORM) {
            s *= (float)P.dims[k] / (float)bs;
        } else {
            const unsigned long long *c = P.cdf[k];
            const long long b0 = bs > 1 ? row[k] / bs * bs : row[k], b1 = b0 + bs - 1;
            const unsigned long long hi = __ldg(c + b1);
            const unsigned long long lo = b0 > 0 ? __ldg(c + b0 - 1) : 0ULL;
            s *= __ull2float_rn(__ldg(c + P.dims[k] - 1)) / __ull2float_rn(hi - lo);
        }
    }
    return s;
}

// s_f from CDFs staged in shared memory by draw_indices (modes k != n in
// ascending order, I_k entries each); same arithmetic as fiber_weight.
template <class T>
__device__ __forceinline__ float fiber_weight_staged(const Problem<T> &P, int n, const int *row,
                                                     const unsigned long long *stage)
{
    float s = P.inv_bj[n];
    long long off = 0;
    for (int k = 0; k < P.N; ++k) {
        if (k == n) continue;
        const int bs = k == block_mode(n) ? P.block : 1;
        if (P.sampling == CPD_SAMPLE_UNIFORM) {
            s *= (float)P.dims[k] / (float)bs;
        } else {
            const unsigned long long *c = stage + off;
            s *= __ull2float_rn(c[P.dims[k] - 1]) / __ull2float_rn(row_mass(c, row[k], bs));
        }
        off += P.dims[k];
    }
    return s;
}

// True when draw_indices staged the CDFs of every mode k != n in `cap` slots.
template <class T>
__device__ __forceinline__ bool cdfs_staged(const Problem<T> &P, int n, long long cap)
{
    long long need = 0;
    for (int k = 0; k < P.N; ++k)
        if (k != n) need += P.dims[k];
    return P.sampling != CPD_SAMPLE_UNIFORM && need <= cap;
}

template <class XT, class T>
__device__ __forceinline__ T load_x(const XT *p) { return (T)to_float<XT>(*p); }

// Element offset of the first entry of mode-n fiber j (Eq. (2) numbering) in
// the storage the problem reads, and the distance between its entries: the
// mode-n replica (fibers contiguous, ld[n] apart), or, with the strided
// layout, the mode-1 replica alone, X in column-major order with the first
// mode padded to ld[0]. There (0-based modes), writing
// j = i_pre + (I_0 ... I_{n-1}) i_post and i_pre = i_0 + I_0 mid, the fiber
// starts at i_0 + ld[0] (mid + q_n I_n i_post) and its entries are ld[0] q_n
// apart, q_n = I_1 ... I_{n-1}.
template <class T>
__device__ __forceinline__ long long fiber_start(const Problem<T> &P, int n, long long j)
{
    if (!P.strided || n == 0) return j * P.ld[n];
    const long long pre = P.dims[0] * P.xq[n];
    const long long ipre = j % pre, ipost = j / pre;
    return (ipre % P.dims[0]) + P.ld[0] * (ipre / P.dims[0] + P.xq[n] * P.dims[n] * ipost);
}

template <class T>
__device__ __forceinline__ long long fiber_step(const Problem<T> &P, int n)
{
    return (P.strided && n > 0) ? P.ld[0] * P.xq[n] : 1;
}
template <>
__device__ __forceinline__ double load_x<double, double>(const double *p) { return *p; }


// Arrival counter: true in exactly one of the nblk CTAs that work on one
// problem, the last one to finish.
__device__ __forceinline__ bool last_block(unsigned *counter, unsigned nblk)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev == nblk - 1);
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

__device__ __forceinline__ bool last_block(unsigned *counter) { return last_block(counter, gridDim.x); }

// Grouped launches: one launch runs the CTAs of G problems back to back;
// problem g owns CTAs [cta0[g], cta0[g+1]). Returns g (binary search by one
// thread) and copies problem g into `sp` for the whole CTA.
template <class T>
__device__ __forceinline__ int group_member(const Problem<T> *__restrict__ Ps, const int *__restrict__ cta0,
                                            int G, Problem<T> &sp)
{
    __shared__ int s_g;
    if (threadIdx.x == 0) {
        int lo = 0, hi = G - 1;
        const int b = (int)blockIdx.x;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(cta0 + mid) <= b) lo = mid;
            else hi = mid - 1;
        }
        s_g = lo;
    }
    __syncthreads();
    const int g = s_g;
    static_assert(sizeof(Problem<T>) % 8 == 0, "Problem is copied in 8-byte words");
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(Ps + g);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(&sp);
    for (int q = threadIdx.x; q < (int)(sizeof(Problem<T>) / 8); q += blockDim.x) dst[q] = __ldg(src + q);
    __syncthreads();
    return g;
}
}  // namespace cpd
