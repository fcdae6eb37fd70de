// Stop check of Sec. 5.2 on the tensor cores (sm_103a): Tol's numerator
// sum_{i,j} (x_ij - x_hat_ij)^2 over the mode-1 unfolding, x_hat_ij =
// A^(1)(i,:) . z_j, z_j the Khatri-Rao row of mode-1 fiber j (Eq. (2), (3)).
//
// For a BF16 tensor the pass is one read of the mode-1 replica, so its bound
// is HBM. Forming x_hat on CUDA cores costs 2 R flops per entry, more than
// the SMs' FP32 rate sustains at HBM speed (R = 50: 100 flops per 2-byte
// entry); on the tensor cores it is hidden under the read. Both operands are
// split into bf16 hi/lo pairs (a = hi + lo, lo = bf16(a - hi)) and
//   x_hat = Z_hi A_hi^T + Z_hi A_lo^T + Z_lo A_hi^T,
// which keeps about 16 significant bits of each product; the dropped lo*lo
// term and the two splitting errors bound |x_hat' - x_hat| by 2^-15
// sum_r |a_ir z_jr| per entry, a few hundred times finer than the stored
// BF16 entries themselves.
//
// Layout. The pass tiles the fibers: tile t = fibers [128 t, 128 t + 128)
// (MMA M = 128, one TMEM lane per fiber), the rows of A^(1) in chunks of 256
// (MMA N <= 256), K = R rounded up to 16. A CTA per SM walks tiles t = b,
// b + grid, ...; its warps take fixed roles:
//   warps 0-7   epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its fibers),
//               warps 0-3 the even 32-row groups of a chunk, 4-7 the odd ones;
//               each thread loads its fiber's 32 entries of a group from the
//               replica (four 16-byte loads, issued for the whole chunk before
//               the accumulator is ready), subtracts x_hat, squares, sums.
//   warps 8-11  producer: the tile's KRP rows (FP32 products of the factor
//               rows, from padded copies with 16-byte rows), split hi/lo into
//               the K-major operand; two stages.
//   warp 12     one thread issues the MMAs: 3 K/16 per (tile, chunk), into one
//               of two 256-column TMEM accumulators.
//   warp 13     one thread loads the A^(1) operand chunks (hi/lo, prepared by
//               k_fit_tc_prep) with bulk copies into two slots; when all
//               chunks fit the two slots they are loaded once.
// Hand-offs are mbarriers; every wait is bounded and a timeout makes every
// role leave its loop (status kStTimeout), so the kernel always returns.
// Sums are in a fixed order: a thread's groups in order (32 squared residuals
// in FP32, then one FP64 add), the warp tree, the CTA's warps, and k_fold over
// the CTAs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "cpd_device.cuh"
#include "cpd_internal.h"
#include "cpd_tcgen05.cuh"

namespace cpd {

namespace {

constexpr int kFtM = 128;           // fibers per tile (MMA M)
constexpr int kFtN = 256;           // rows of A^(1) per chunk (MMA N, largest)
constexpr int kFtThreads = 448;     // 14 warps
constexpr int kFtEpiWarps = 8;
constexpr int kFtProdWarp0 = 8, kFtProdThreads = 128;
constexpr int kFtMmaWarp = 12;      // warp 13 loads the A^(1) chunks
constexpr int kFtColumns = 512;     // TMEM: two 256-column accumulators

// Instruction descriptor of kind::f16, D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_kk(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// bf16 index of element (row, k) in a K-major, no-swizzle operand of Kp
// columns: core matrices of 8 rows x 8 k (16 bytes a row), adjacent in k 128
// bytes apart (LBO), adjacent in rows Kp / 8 * 128 bytes apart (SBO).
__host__ __device__ inline int kmaj(int row, int k, int Kp)
{
    return (((row >> 3) * (Kp >> 3) + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

struct FitTcLayout {
    size_t zst, aslot, z, a, fi, bar, misc, total;
    __host__ __device__ FitTcLayout(int Kp)
    {
        zst = (size_t)kFtM * Kp * 2 * 2;     // one stage: Z hi, Z lo
        aslot = (size_t)kFtN * Kp * 2 * 2;   // one chunk: A hi, A lo
        z = 0;
        a = z + 2 * zst;
        fi = a + 2 * aslot;                  // the tile's fibers' indices, [128][kMaxModes]
        bar = fi + (size_t)kFtM * kMaxModes * 4;
        misc = bar + 128;                    // tmem holder, abort flag, warp sums
        total = misc + 16 + (kFtThreads / 32) * 8;
        // at least 120 KB: one CTA per SM, so the 512-column TMEM
        // allocation never waits for another CTA's
        if (total < 120 * 1024) total = 120 * 1024;
    }
};

enum { kBarZFull = 0, kBarZFree = 2, kBarAFull = 4, kBarAFree = 6, kBarMDone = 8, kBarTFree = 10, kBarDrain = 12 };

__device__ __forceinline__ unsigned long long ft_now()
{
    unsigned long long ns;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
    return ns;
}

// Bounded wait that also gives up when another role has given up. With
// `timed`, the nanoseconds spent waiting are added to `waited_ns` (the trace
// of cpd_trace: where each role of CTA 0 waits).
__device__ __forceinline__ bool ft_wait(uint32_t bar, uint32_t parity, volatile int *abort, bool timed = false,
                                        unsigned long long *waited_ns = nullptr)
{
    const unsigned long long t0 = timed ? ft_now() : 0ULL;
    bool ok = false;
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        if (mbar_try_wait(bar, parity)) {
            ok = true;
            break;
        }
        if ((it & 255u) == 255u && *abort) break;
    }
    if (!ok && !*abort) *abort = 1;
    if (timed) *waited_ns += ft_now() - t0;
    return ok;
}

__device__ __forceinline__ void ft_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void ft_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void ft_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// Columns of chunk c: its rows of A^(1) rounded up to 16 (MMA N), at most 256.
__host__ __device__ inline int chunk_cols(long long I0, int c)
{
    const long long rows = I0 - (long long)c * kFtN;
    const long long n = (rows + 15) / 16 * 16;
    return (int)(n < kFtN ? n : kFtN);
}

// A step of the epilogue: group g = h + 2 u of chunk c of tile t (the
// warpgroup h's u-th group of that chunk), qi = the (tile, chunk) sequence
// number of the CTA. next() skips chunks that hold no group for h (a tail
// chunk of at most 32 rows has none for h = 1); qi still counts them.
struct FtStep {
    long long t, qi;
    int c, u;
    bool valid;
    __device__ __forceinline__ static int groups(long long I0, int c) { return (chunk_cols(I0, c) + 31) / 32; }
    __device__ __forceinline__ void settle(int grid, long long ntile, int nch, int h, long long I0)
    {
        while (valid && h + 2 * u >= groups(I0, c)) {
            u = 0;
            ++qi;
            if (++c == nch) {
                c = 0;
                t += grid;
                if (t >= ntile) valid = false;
            }
        }
    }
    __device__ __forceinline__ void start(long long t0, int grid, long long ntile, int nch, int h, long long I0)
    {
        t = t0;
        qi = 0;
        c = 0;
        u = 0;
        valid = t0 < ntile;
        settle(grid, ntile, nch, h, I0);
    }
    __device__ __forceinline__ void next(int grid, long long ntile, int nch, int h, long long I0)
    {
        ++u;
        settle(grid, ntile, nch, h, I0);
    }
    __device__ __forceinline__ bool last_in_chunk(int h, long long I0) const
    {
        return h + 2 * (u + 1) >= groups(I0, c);
    }
};

// The 32 replica entries of a step for fiber m of its tile, warpgroup h
// (zeros past the tensor's fibers; each 16-byte load lies inside the fiber's
// ld0 entries, the padding past I_1 being zero).
__device__ __forceinline__ void ft_load(uint4 (&x)[4], const FtStep &s, int h, const __nv_bfloat16 *rep, int m,
                                        long long J, long long ld0)
{
#pragma unroll
    for (int w = 0; w < 4; ++w) x[w] = make_uint4(0u, 0u, 0u, 0u);
    if (!s.valid) return;
    const long long j = s.t * kFtM + m;
    if (j >= J) return;
    const long long i0 = (long long)s.c * kFtN + 32 * (h + 2 * s.u);
    const uint4 *p = reinterpret_cast<const uint4 *>(rep + j * ld0 + i0);
#pragma unroll
    for (int w = 0; w < 4; ++w)
        if (i0 + 8 * w < ld0) x[w] = __ldcs(p + w);
}

// v = hi + lo with hi = bf16(v), lo = bf16(v - hi), four entries packed as
// bf16 pairs (element 0 in the low half), by paired conversions.
__device__ __forceinline__ void split4(float4 v, uint2 &hi, uint2 &lo)
{
    const __nv_bfloat162 h01 = __float22bfloat162_rn(make_float2(v.x, v.y));
    const __nv_bfloat162 h23 = __float22bfloat162_rn(make_float2(v.z, v.w));
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    const __nv_bfloat162 l01 = __float22bfloat162_rn(make_float2(v.x - f01.x, v.y - f01.y));
    const __nv_bfloat162 l23 = __float22bfloat162_rn(make_float2(v.z - f23.x, v.w - f23.y));
    hi = make_uint2(*reinterpret_cast<const uint32_t *>(&h01), *reinterpret_cast<const uint32_t *>(&h23));
    lo = make_uint2(*reinterpret_cast<const uint32_t *>(&l01), *reinterpret_cast<const uint32_t *>(&l23));
}

}  // namespace

// A^(1)'s hi/lo operand in chunks of 256 rows (rows past I_1 zero), and the
// factors k >= 2 (in the paper's 1-based numbering: every mode but the first)
// copied with rows of Kp floats, zero-padded.
__global__ void __launch_bounds__(kThreads) k_fit_tc_prep(const Problem<float> P, FitTcArgs a)
{
    const int R = P.R, Kp = a.Kp;
    const long long nA = (long long)a.nchunks * kFtN * Kp;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nA; e += stride) {
        const int c = (int)(e / ((long long)kFtN * Kp));
        const int rem = (int)(e % ((long long)kFtN * Kp));
        const int il = rem / Kp, r = rem % Kp;
        const long long i = (long long)c * kFtN + il;
        const float v = (i < P.dims[0] && r < R) ? P.A[0][i * R + r] : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        __nv_bfloat16 *chunk = a.a0op + (size_t)c * (2 * kFtN * Kp);
        chunk[kmaj(il, r, Kp)] = hi;
        chunk[kFtN * Kp + kmaj(il, r, Kp)] = lo;
    }
    for (int k = 1; k < P.N; ++k) {
        const long long nk = P.dims[k] * Kp;
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nk; e += stride) {
            const long long i = e / Kp;
            const int r = (int)(e % Kp);
            a.apad[k][e] = r < R ? P.A[k][i * R + r] : 0.f;
        }
    }
}

// 14 warps: four to a sub-partition, whose 16K registers cap a thread at 128
__global__ void __launch_bounds__(kFtThreads, 1) k_fit_tc(const Problem<float> P, const FitTcArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int Kp = a.Kp, N = P.N, nch = a.nchunks;
    const FitTcLayout L(Kp);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long I0 = P.dims[0], J = a.J, ld0 = P.ld[0];
    const long long ntile = (J + kFtM - 1) / kFtM;
    int *sfi = reinterpret_cast<int *>(smem + L.fi);
    const uint32_t bar0 = smem_u32(smem + L.bar);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + L.misc);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + L.misc + 4);
    volatile int *pdec = reinterpret_cast<volatile int *>(smem + L.misc + 8);   // producers' verdict
    double *wsum = reinterpret_cast<double *>(smem + L.misc + 16);
    auto bar = [&](int which, int idx) { return bar0 + 8u * (uint32_t)(which + idx); };
    const bool resident = nch <= 2;

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(bar(kBarZFull, s), 1);
            mbar_init(bar(kBarZFree, s), 1);
            mbar_init(bar(kBarAFull, s), 1);
            mbar_init(bar(kBarAFree, s), 1);
            mbar_init(bar(kBarMDone, s), 1);
            mbar_init(bar(kBarTFree, s), kFtEpiWarps);
        }
        mbar_init(bar(kBarDrain, 0), 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(tmem_holder)),
                     "r"(kFtColumns)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_holder;
    double acc = 0.0;
    bool timed_out = false;
    // cpd_trace: CTA 0 records where its roles wait (slots 44-55)
    const bool timed = P.trace != nullptr && blockIdx.x == 0;
    unsigned long long w0 = 0, w1 = 0, w2 = 0;   // the role's wait times (ns)
    trace_stamp(P.trace, 44, blockIdx.x == 0);

    if (warp < kFtEpiWarps) {
        // ---- epilogue ------------------------------------------------------
        // The thread's work is a sequence of steps, one per 32-row group of a
        // (tile, chunk) that its warpgroup owns; the replica entries of step
        // n + 4 are loaded while step n is processed (a ring of four register
        // slots, rotated by unrolling), so loads stay in flight across chunk
        // and tile boundaries.
        const int q = warp & 3, h = warp >> 2, m = 32 * q + lane;
        const __nv_bfloat16 *rep = reinterpret_cast<const __nv_bfloat16 *>(P.rep[0]);
        FtStep ld, pr;
        ld.start(blockIdx.x, gridDim.x, ntile, nch, h, I0);
        pr = ld;
        uint4 xv[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ft_load(xv[k], ld, h, rep, m, J, ld0);
            ld.next(gridDim.x, ntile, nch, h, I0);
        }
        long long waited = -1;   // chunks whose accumulator this warp has waited for
        const long long nseq = ((ntile - 1 - blockIdx.x) / gridDim.x + 1) * nch;
        while (pr.valid && !timed_out) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!pr.valid || timed_out) break;
                while (waited < pr.qi && !timed_out) {   // the step's chunk (and chunks empty for this warp)
                    ++waited;
                    const bool ok = ft_wait(bar(kBarMDone, (int)(waited & 1)), (uint32_t)((waited >> 1) & 1), abort,
                                            timed, &w0);
                    if (!__all_sync(0xffffffffu, ok)) {
                        timed_out = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    if (waited < pr.qi) {
                        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                        __syncwarp();
                        if (lane == 0) ft_arrive(bar(kBarTFree, (int)(waited & 1)));
                    }
                }
                if (timed_out) break;
                const int b = (int)(pr.qi & 1), g = h + 2 * pr.u;
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kFtN + 32 * g), v);
                // No per-entry mask: past I_1 and past the fibers both x (zero
                // padding or skipped loads) and x_hat (zero operand rows) are 0.
                // Only columns at or past the chunk's MMA width Nc hold stale
                // accumulator values: Nc is a multiple of 16, so a group
                // straddling it keeps its first 16 columns.
                const bool half = 32 * g + 32 > chunk_cols(I0, pr.c);
                float p4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    if (w >= 2 && half) break;
                    const uint32_t wd[4] = {xv[k][w].x, xv[k][w].y, xv[k][w].z, xv[k][w].w};
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const uint32_t bits = (e & 1) ? (wd[e >> 1] & 0xffff0000u) : (wd[e >> 1] << 16);
                        const float d = __uint_as_float(bits) - v[8 * w + e];
                        p4[e & 3] = fmaf(d, d, p4[e & 3]);
                    }
                }
                const float part = (p4[0] + p4[1]) + (p4[2] + p4[3]);
                acc += (double)part;
                if (pr.last_in_chunk(h, I0)) {
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    __syncwarp();
                    if (lane == 0) ft_arrive(bar(kBarTFree, b));
                }
                ft_load(xv[k], ld, h, rep, m, J, ld0);
                ld.next(gridDim.x, ntile, nch, h, I0);
                pr.next(gridDim.x, ntile, nch, h, I0);
            }
        }
        while (!timed_out && waited + 1 < nseq) {   // trailing chunks empty for this warp
            ++waited;
            const bool ok = ft_wait(bar(kBarMDone, (int)(waited & 1)), (uint32_t)((waited >> 1) & 1), abort);
            if (!__all_sync(0xffffffffu, ok)) {
                timed_out = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) ft_arrive(bar(kBarTFree, (int)(waited & 1)));
        }
    } else if (warp < kFtMmaWarp) {
        // ---- producer: KRP rows of the tile, hi/lo, K-major ----------------
        const int pt = tid - kFtProdWarp0 * 32;
        const int nq = Kp / 4, tot = kFtM * nq;
        long long tl = 0;
        for (long long t = blockIdx.x; t < ntile && !timed_out; t += gridDim.x, ++tl) {
            const int s = (int)(tl & 1);
            // one thread waits for the stage; its verdict, in shared memory,
            // is read by all 128 after the barrier, so they leave together
            if (pt == 0)
                *pdec = (tl >= 2 && !ft_wait(bar(kBarZFree, s), (uint32_t)(((tl >> 1) + 1) & 1), abort, timed, &w0)) ? 1 : 0;
            asm volatile("bar.sync 1, %0;\n" ::"r"(kFtProdThreads) : "memory");
            if (*pdec) {
                timed_out = true;
                break;
            }
            {   // Eq. (2) inverted once per fiber: i_k = (j / prod_{1<=l<k} I_l) mod I_k
                long long j = t * kFtM + pt;
                int *row = sfi + pt * kMaxModes;
                row[0] = j < J ? 1 : 0;
                for (int k = 1; k < N; ++k) {
                    row[k] = (int)(j % P.dims[k]);
                    j /= P.dims[k];
                }
            }
            asm volatile("bar.sync 1, %0;\n" ::"r"(kFtProdThreads) : "memory");
            unsigned char *zs = smem + L.z + (size_t)s * L.zst;
            uint2 *zhi = reinterpret_cast<uint2 *>(zs);
            uint2 *zlo = reinterpret_cast<uint2 *>(zs + (size_t)kFtM * Kp * 2);
            for (int base = 0; base < tot; base += kFtProdThreads * 8) {
                float4 z[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e4 = base + u * kFtProdThreads + pt;
                    const int f = e4 / nq, r4 = e4 - f * nq;
                    const bool ok = e4 < tot && sfi[f * kMaxModes] != 0;
                    z[u] = ok ? __ldg(reinterpret_cast<const float4 *>(a.apad[1] + (long long)sfi[f * kMaxModes + 1] * Kp) + r4)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                for (int k = 2; k < N; ++k) {   // ascending k, as in Eq. (3)
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int e4 = base + u * kFtProdThreads + pt;
                        const int f = e4 / nq, r4 = e4 - f * nq;
                        if (e4 < tot && sfi[f * kMaxModes] != 0) {
                            const float4 v = __ldg(
                                reinterpret_cast<const float4 *>(a.apad[k] + (long long)sfi[f * kMaxModes + k] * Kp) + r4);
                            z[u].x *= v.x;
                            z[u].y *= v.y;
                            z[u].z *= v.z;
                            z[u].w *= v.w;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e4 = base + u * kFtProdThreads + pt;
                    if (e4 < tot) {
                        const int f = e4 / nq, r4 = e4 - f * nq;
                        const int o = kmaj(f, 4 * r4, Kp) >> 2;   // 4 bf16 = one uint2
                        split4(z[u], zhi[o], zlo[o]);
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("bar.sync 1, %0;\n" ::"r"(kFtProdThreads) : "memory");
            if (pt == 0) ft_arrive(bar(kBarZFull, s));
        }
    } else if (warp == kFtMmaWarp) {
        // ---- MMA issue -----------------------------------------------------
        if (lane == 0) {
            long long qi = 0, tl = 0;
            bool issued = false;
            const uint32_t sbo = (uint32_t)(Kp / 8) * 128u;
            for (long long t = blockIdx.x; t < ntile && !timed_out; t += gridDim.x, ++tl) {
                const int s = (int)(tl & 1);
                if (!ft_wait(bar(kBarZFull, s), (uint32_t)((tl >> 1) & 1), abort, timed, &w0)) {
                    timed_out = true;
                    break;
                }
                const uint32_t zb = smem_u32(smem + L.z + (size_t)s * L.zst);
                for (int c = 0; c < nch; ++c, ++qi) {
                    const int slot = resident ? c : (int)(qi & 1);
                    const uint32_t apar = resident ? 0u : (uint32_t)((qi >> 1) & 1);
                    const int b = (int)(qi & 1);
                    if (!ft_wait(bar(kBarAFull, slot), apar, abort, timed, &w1) ||
                        (qi >= 2 && !ft_wait(bar(kBarTFree, b), (uint32_t)(((qi >> 1) + 1) & 1), abort, timed, &w2))) {
                        timed_out = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const int Nc = chunk_cols(I0, c);
                    const uint32_t idesc = idesc_bf16_kk(kFtM, Nc);
                    const uint32_t ab = smem_u32(smem + L.a + (size_t)slot * L.aslot);
                    const uint32_t d = tmem + (uint32_t)(b * kFtN);
                    for (int ks = 0; ks < Kp / 16; ++ks) {
                        const uint64_t zh = smem_desc(zb + ks * 256u, 128u, sbo);
                        const uint64_t zl = smem_desc(zb + (uint32_t)(kFtM * Kp * 2) + ks * 256u, 128u, sbo);
                        const uint64_t ah = smem_desc(ab + ks * 256u, 128u, sbo);
                        const uint64_t al = smem_desc(ab + (uint32_t)(kFtN * Kp * 2) + ks * 256u, 128u, sbo);
                        ft_mma(d, zh, ah, idesc, ks > 0 ? 1u : 0u);
                        ft_mma(d, zh, al, idesc, 1u);
                        ft_mma(d, zl, ah, idesc, 1u);
                    }
                    issued = true;
                    ft_commit(bar(kBarMDone, b));
                    if (!resident) ft_commit(bar(kBarAFree, slot));
                }
                if (timed_out) break;
                ft_commit(bar(kBarZFree, s));
            }
            if (issued) {   // drain: every MMA and every commit's arrival done before exit
                ft_commit(bar(kBarDrain, 0));
                mbar_wait_bounded(bar(kBarDrain, 0), 0);
            }
        }
    } else {
        // ---- A^(1) operand chunks ------------------------------------------
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)L.aslot;
            if (resident) {
                for (int c = 0; c < nch; ++c) {
                    mbar_expect_tx(bar(kBarAFull, c), bytes);
                    bulk_g2s(smem_u32(smem + L.a + (size_t)c * L.aslot), a.a0op + (size_t)c * (2 * kFtN * Kp), bytes,
                             bar(kBarAFull, c));
                }
                for (int c = 0; c < nch; ++c) mbar_wait_bounded(bar(kBarAFull, c), 0);
            } else {
                long long qi = 0;
                for (long long t = blockIdx.x; t < ntile && !timed_out; t += gridDim.x)
                    for (int c = 0; c < nch; ++c, ++qi) {
                        const int slot = (int)(qi & 1);
                        if (qi >= 2 &&
                            !ft_wait(bar(kBarAFree, slot), (uint32_t)(((qi >> 1) + 1) & 1), abort, timed, &w0)) {
                            timed_out = true;
                            break;
                        }
                        mbar_expect_tx(bar(kBarAFull, slot), bytes);
                        bulk_g2s(smem_u32(smem + L.a + (size_t)slot * L.aslot), a.a0op + (size_t)c * (2 * kFtN * Kp),
                                 bytes, bar(kBarAFull, slot));
                    }
                // the copies in flight land before the CTA's shared memory goes away
                for (long long r = (qi >= 2 ? qi - 2 : 0); r < qi; ++r)
                    mbar_wait_bounded(bar(kBarAFull, (int)(r & 1)), (uint32_t)((r >> 1) & 1));
            }
        }
    }
    if (timed_out && (lane == 0)) atomicOr(P.status, kStTimeout);
    if (timed && lane == 0) {   // one thread per role: epilogue warps 0 and 4, producer, MMA, loader
        if (warp == 0) P.trace[46] = w0;
        if (warp == 4) P.trace[47] = w0;
        if (warp == kFtProdWarp0) P.trace[48] = w0;
        if (warp == kFtMmaWarp) {
            P.trace[49] = w0;
            P.trace[50] = w1;
            P.trace[51] = w2;
        }
        if (warp == kFtMmaWarp + 1) P.trace[52] = w0;
    }
    trace_stamp(P.trace, 45, blockIdx.x == 0);

    // fixed-order sum: warp tree, then the warps in order
    for (int off = 16; off >= 1; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) wsum[warp] = acc;
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int w = 0; w < kFtThreads / 32; ++w) sum += wsum[w];
        a.partials[blockIdx.x] = sum;
    }
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kFtColumns)
                     : "memory");
    }
}

bool fit_tc_supported(const Problem<float> &P)
{
    return P.x_dtype == CPD_BF16 && P.R >= 1 && P.R <= 64;
}

int fit_tc_kp(int R) { return (R + 15) / 16 * 16; }

int fit_tc_chunks(long long I0) { return (int)((I0 + kFtN - 1) / kFtN); }

size_t fit_tc_scratch_bytes(const Problem<float> &P)
{
    const int Kp = fit_tc_kp(P.R);
    size_t b = (size_t)fit_tc_chunks(P.dims[0]) * 2 * kFtN * Kp * 2;
    for (int k = 1; k < P.N; ++k) b += (size_t)P.dims[k] * Kp * 4 + 64;
    return b + 256;
}

void fit_tc_args(const Problem<float> &P, void *scratch, double *partials, FitTcArgs &a)
{
    a.Kp = fit_tc_kp(P.R);
    a.nchunks = fit_tc_chunks(P.dims[0]);
    a.J = 1;
    for (int k = 1; k < P.N; ++k) a.J *= P.dims[k];
    a.partials = partials;
    char *p = static_cast<char *>(scratch);
    a.a0op = reinterpret_cast<__nv_bfloat16 *>(p);
    p += (size_t)a.nchunks * 2 * kFtN * a.Kp * 2;
    a.apad[0] = nullptr;
    for (int k = 1; k < P.N; ++k) {
        a.apad[k] = reinterpret_cast<float *>(p);
        p += ((size_t)P.dims[k] * a.Kp * 4 + 64 + 15) / 16 * 16;
    }
}

cudaError_t launch_fit_tc(const Problem<float> &P, void *scratch, double *partials, int sm_count, double *out,
                          cudaStream_t s)
{
    FitTcArgs a{};
    fit_tc_args(P, scratch, partials, a);
    const FitTcLayout L(a.Kp);
    static size_t raised = 0;
    if (L.total > raised) {
        cudaError_t e = cudaFuncSetAttribute(k_fit_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        raised = L.total;
    }
    k_fit_tc_prep<<<2 * sm_count, kThreads, 0, s>>>(P, a);
    const long long ntile = (a.J + kFtM - 1) / kFtM;
    const int grid = (int)std::min<long long>(ntile, sm_count);
    k_fit_tc<<<grid, kFtThreads, L.total, s>>>(P, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_fold(partials, grid, out, s);
}

}  // namespace cpd
