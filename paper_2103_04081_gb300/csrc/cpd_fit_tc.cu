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
// Three launches. k_fit_tc_prep writes A^(1)'s hi/lo operand in chunks of 128
// rows and copies of the other factors with 16-byte rows; k_fit_tc_z writes
// the hi/lo KRP operand of every tile of 128 fibers (the operand layout of
// the MMA, so one bulk copy moves a tile); k_fit_tc makes the pass.
//
// k_fit_tc: a CTA per SM walks tiles t = b, b + grid, ... (MMA M = 128, one
// TMEM lane per fiber) and, per tile, the chunks of A^(1) (MMA N <= 128,
// K = R rounded up to 16). Warp roles:
//   warp 17     lane 0 loads a tile's KRP operand (bulk copy, two stages)
//               and the A^(1) chunks (bulk copies, two slots, loaded once when
//               all chunks fit); lane 1 loads each (tile, chunk) block of the
//               replica, 128 fibers x 128 entries, by two 2-D tensor copies
//               with the 128-byte swizzle into one of three stages; entries
//               past the fibers or past I_1's padding arrive as zeros.
//   warp 16     one thread issues the 3 K/16 MMAs of a (tile, chunk) into one
//               of four 128-column TMEM accumulators.
//   warps 0-15  epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its fibers)
//               and the 32-row group w / 4 of every chunk; x comes from the
//               swizzled stage (conflict-free 16-byte reads), d = x - x_hat,
//               d^2 summed.
// Hand-offs are mbarriers; every wait is bounded and a timeout makes every
// role leave its loop (status kStTimeout), so the kernel always returns.
// Sums are in a fixed order: a thread's groups in order (32 squared residuals
// in four FP32 partial sums, then one FP64 add), the warp tree, the CTA's
// warps, and k_fold over the CTAs.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "cpd_device.cuh"
#include "cpd_internal.h"
#include "cpd_tcgen05.cuh"

namespace cpd {

namespace {

constexpr int kFtM = 128;           // fibers per tile (MMA M)
constexpr int kFtN = 128;           // rows of A^(1) per chunk (MMA N, largest)
constexpr int kFtThreads = 576;     // 18 warps
constexpr int kFtEpiWarps = 16;
constexpr int kFtMmaWarp = 16, kFtLoadWarp = 17;
constexpr int kFtBufs = 4;          // TMEM accumulators of 128 columns
constexpr int kFtXStages = 3;       // replica blocks in flight
constexpr int kFtColumns = 512;
constexpr uint32_t kFtXBytes = kFtM * kFtN * 2;   // one replica block: 128 fibers x 128 entries

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

// Dynamic shared memory, from a 1024-byte aligned base (the swizzled stages).
struct FitTcLayout {
    size_t zst, aslot, x, z, a, bar, misc, total;
    __host__ __device__ FitTcLayout(int Kp)
    {
        zst = (size_t)kFtM * Kp * 2 * 2;     // a tile's KRP operand: hi, lo
        aslot = (size_t)kFtN * Kp * 2 * 2;   // a chunk of A^(1): hi, lo
        x = 0;                               // kFtXStages replica blocks (1024-aligned)
        z = x + (size_t)kFtXStages * kFtXBytes;
        a = z + 2 * zst;
        bar = a + 2 * aslot;
        misc = bar + 256;                    // tmem holder, abort flag, warp sums
        total = misc + 16 + (kFtThreads / 32) * 8 + 1024;   // + alignment slack
    }
};

enum {
    kBarZFull = 0, kBarZFree = 2, kBarAFull = 4, kBarAFree = 6, kBarXFull = 8, kBarXFree = 11,
    kBarMDone = 14, kBarTFree = 18, kBarDrain = 22
};

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

// 2-D tensor copy global -> shared completing on an mbarrier; x (the
// contiguous coordinate) is a multiple of 64 entries, 128 bytes.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

// Columns of chunk c: its rows of A^(1) rounded up to 16 (MMA N), at most 128.
__host__ __device__ inline int chunk_cols(long long I0, int c)
{
    const long long rows = I0 - (long long)c * kFtN;
    const long long n = (rows + 15) / 16 * 16;
    return (int)(n < kFtN ? n : kFtN);
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

// A^(1)'s hi/lo operand in chunks of 128 rows (rows past I_1 zero), and the
// other factors (modes k >= 1 here; the paper's modes 2..N) copied with rows
// of Kp floats, zero-padded.
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

// The KRP operand of every tile: z_j = A^(2)(i_2,:) * ... * A^(N)(i_N,:) in
// FP32 (factors in ascending order, Eq. (3)), j = t 128 + f, split hi/lo and
// written in the tile's K-major layout; fibers past J are zero. A thread
// forms one 16-byte row of a core matrix (8 entries of z_j), so the fiber's
// indices are decoded once per 8 entries and 8 consecutive threads write a
// core matrix's 128 contiguous bytes.
__global__ void __launch_bounds__(kThreads) k_fit_tc_z(const Problem<float> P, FitTcArgs a)
{
    const int Kp = a.Kp, N = P.N;
    const int per_tile = kFtM * Kp / 8;   // 16-byte rows of a tile's hi (or lo) half
    const long long ntile = (a.J + kFtM - 1) / kFtM;
    const long long total = ntile * per_tile;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long t = e / per_tile;
        const int o = (int)(e - t * per_tile);
        const int cm = o >> 3, kb = cm % (Kp >> 3);
        const int f = (cm / (Kp >> 3)) * 8 + (o & 7);
        const long long j = t * kFtM + f;
        float4 z0 = make_float4(0.f, 0.f, 0.f, 0.f), z1 = z0;
        if (j < a.J) {
            unsigned rest = (unsigned)j;   // Eq. (2) inverted, mode 2 fastest; J < 2^31
            for (int k = 1; k < N; ++k) {
                const unsigned Ik = (unsigned)P.dims[k];
                const unsigned ik = rest % Ik;
                rest /= Ik;
                const float4 *src = reinterpret_cast<const float4 *>(a.apad[k] + (long long)ik * Kp + kb * 8);
                const float4 v0 = __ldg(src), v1 = __ldg(src + 1);
                if (k == 1) {
                    z0 = v0;
                    z1 = v1;
                } else {
                    z0.x *= v0.x; z0.y *= v0.y; z0.z *= v0.z; z0.w *= v0.w;
                    z1.x *= v1.x; z1.y *= v1.y; z1.z *= v1.z; z1.w *= v1.w;
                }
            }
        }
        uint2 h0, l0, h1, l1;
        split4(z0, h0, l0);
        split4(z1, h1, l1);
        uint4 *tile = reinterpret_cast<uint4 *>(a.ztiles + (size_t)t * (2 * kFtM * Kp));
        tile[o] = make_uint4(h0.x, h0.y, h1.x, h1.y);
        tile[per_tile + o] = make_uint4(l0.x, l0.y, l1.x, l1.y);
    }
}

// 18 warps: at most five to a sub-partition, whose 16K registers allow 102 a thread
__global__ void __launch_bounds__(kFtThreads, 1) k_fit_tc(const Problem<float> P, const FitTcArgs a,
                                                          const __grid_constant__ CUtensorMap xmap)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int Kp = a.Kp, nch = a.nchunks;
    const FitTcLayout L(Kp);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long I0 = P.dims[0], J = a.J;
    const long long ntile = (J + kFtM - 1) / kFtM;
    const uint32_t bar0 = smem_u32(smem + L.bar);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + L.misc);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + L.misc + 4);
    double *wsum = reinterpret_cast<double *>(smem + L.misc + 16);
    auto bar = [&](int which, int idx) { return bar0 + 8u * (uint32_t)(which + idx); };
    const bool resident = nch <= 2;

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(bar(kBarZFull, s), 1);
            mbar_init(bar(kBarZFree, s), 1);
            mbar_init(bar(kBarAFull, s), 1);
            mbar_init(bar(kBarAFree, s), 1);
        }
        for (int s = 0; s < kFtXStages; ++s) {
            mbar_init(bar(kBarXFull, s), 1);
            mbar_init(bar(kBarXFree, s), kFtEpiWarps);
        }
        for (int b = 0; b < kFtBufs; ++b) {
            mbar_init(bar(kBarMDone, b), 1);
            mbar_init(bar(kBarTFree, b), kFtEpiWarps);
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
        const int q = warp & 3, g = warp >> 2, m = 32 * q + lane;
        long long qi = 0;   // (tile, chunk) sequence number of the CTA
        for (long long t = blockIdx.x; t < ntile && !timed_out; t += gridDim.x) {
            for (int c = 0; c < nch; ++c, ++qi) {
                const int b = (int)(qi & (kFtBufs - 1)), xs = (int)(qi % kFtXStages);
                // every lane waits; the warp leaves together if any lane gave up
                bool ok = ft_wait(bar(kBarMDone, b), (uint32_t)((qi / kFtBufs) & 1), abort, timed, &w0);
                ok = ok && ft_wait(bar(kBarXFull, xs), (uint32_t)((qi / kFtXStages) & 1), abort, timed, &w1);
                if (!__all_sync(0xffffffffu, ok)) {
                    timed_out = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const int Nc = chunk_cols(I0, c);
                const unsigned char *xst = smem + L.x + (size_t)xs * kFtXBytes;
                if (32 * g < Nc) {   // warp-uniform
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kFtN + 32 * g), v);
                    // No per-entry mask: past I_1 and past the fibers both x
                    // (zero padding or the copies' zero fill) and x_hat (zero
                    // operand rows) are 0. Columns at or past Nc (a multiple of
                    // 16) hold stale accumulator values: a group straddling Nc
                    // keeps its first 16 columns.
                    const bool half = 32 * g + 32 > Nc;
                    // box g / 2 holds rows [64 (g / 2), +64) of the 128 fibers; the
                    // 16-byte chunk k of fiber m's 128-byte row sits at k ^ (m % 8)
                    const unsigned char *row = xst + (size_t)(g >> 1) * (kFtXBytes / 2) + (size_t)m * 128;
                    float p4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        if (w >= 2 && half) break;
                        const int kc = ((g & 1) * 4 + w) ^ (m & 7);
                        const uint4 xv = *reinterpret_cast<const uint4 *>(row + kc * 16);
                        const uint32_t wd[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const uint32_t bits = (e & 1) ? (wd[e >> 1] & 0xffff0000u) : (wd[e >> 1] << 16);
                            const float d = __uint_as_float(bits) - v[8 * w + e];
                            p4[e & 3] = fmaf(d, d, p4[e & 3]);
                        }
                    }
                    acc += (double)((p4[0] + p4[1]) + (p4[2] + p4[3]));
                }
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    ft_arrive(bar(kBarTFree, b));
                    ft_arrive(bar(kBarXFree, xs));
                }
            }
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
                    const int b = (int)(qi & (kFtBufs - 1));
                    if (!ft_wait(bar(kBarAFull, slot), apar, abort, timed, &w1) ||
                        (qi >= kFtBufs &&
                         !ft_wait(bar(kBarTFree, b), (uint32_t)(((qi / kFtBufs) + 1) & 1), abort, timed, &w2))) {
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
        // ---- loads ---------------------------------------------------------
        // lane 0: KRP tiles and A^(1) chunks; lane 1: replica blocks, so that
        // the replica runs ahead while an A^(1) slot waits for its MMAs
        const uint32_t abytes = (uint32_t)L.aslot, zbytes = (uint32_t)L.zst;
        if (lane == 0) {
            if (resident)
                for (int c = 0; c < nch; ++c) {
                    mbar_expect_tx(bar(kBarAFull, c), abytes);
                    bulk_g2s(smem_u32(smem + L.a + (size_t)c * L.aslot), a.a0op + (size_t)c * (2 * kFtN * Kp), abytes,
                             bar(kBarAFull, c));
                }
            long long nz = 0, na = 0;   // copies issued: KRP tiles, A^(1) chunks (ring)
            for (long long t = blockIdx.x; t < ntile && !timed_out; t += gridDim.x) {
                const int s = (int)(nz & 1);
                if (nz >= 2 && !ft_wait(bar(kBarZFree, s), (uint32_t)(((nz >> 1) + 1) & 1), abort, timed, &w0)) {
                    timed_out = true;
                    break;
                }
                mbar_expect_tx(bar(kBarZFull, s), zbytes);
                bulk_g2s(smem_u32(smem + L.z + (size_t)s * L.zst), a.ztiles + (size_t)t * (2 * kFtM * Kp), zbytes,
                         bar(kBarZFull, s));
                ++nz;
                if (resident) continue;
                for (int c = 0; c < nch; ++c) {
                    const int slot = (int)(na & 1);
                    if (na >= 2 && !ft_wait(bar(kBarAFree, slot), (uint32_t)(((na >> 1) + 1) & 1), abort, timed, &w1)) {
                        timed_out = true;
                        break;
                    }
                    mbar_expect_tx(bar(kBarAFull, slot), abytes);
                    bulk_g2s(smem_u32(smem + L.a + (size_t)slot * L.aslot), a.a0op + (size_t)c * (2 * kFtN * Kp),
                             abytes, bar(kBarAFull, slot));
                    ++na;
                }
            }
            // the copies in flight land before the CTA's shared memory goes away
            if (resident)
                for (int c = 0; c < nch; ++c) mbar_wait_bounded(bar(kBarAFull, c), 0);
            for (long long r = (nz >= 2 ? nz - 2 : 0); r < nz; ++r)
                mbar_wait_bounded(bar(kBarZFull, (int)(r & 1)), (uint32_t)((r >> 1) & 1));
            for (long long r = (na >= 2 ? na - 2 : 0); r < na; ++r)
                mbar_wait_bounded(bar(kBarAFull, (int)(r & 1)), (uint32_t)((r >> 1) & 1));
        } else if (lane == 1) {
            long long nx = 0;
            for (long long t = blockIdx.x; t < ntile && !timed_out; t += gridDim.x)
                for (int c = 0; c < nch; ++c) {
                    const int xs = (int)(nx % kFtXStages);
                    if (nx >= kFtXStages &&
                        !ft_wait(bar(kBarXFree, xs), (uint32_t)(((nx / kFtXStages) + 1) & 1), abort, timed, &w2)) {
                        timed_out = true;
                        break;
                    }
                    mbar_expect_tx(bar(kBarXFull, xs), kFtXBytes);
                    const uint32_t dst = smem_u32(smem + L.x + (size_t)xs * kFtXBytes);
                    tma_load_2d(dst, &xmap, c * kFtN, (int)(t * kFtM), bar(kBarXFull, xs));
                    tma_load_2d(dst + kFtXBytes / 2, &xmap, c * kFtN + 64, (int)(t * kFtM), bar(kBarXFull, xs));
                    ++nx;
                }
            for (long long r = (nx >= kFtXStages ? nx - kFtXStages : 0); r < nx; ++r)
                mbar_wait_bounded(bar(kBarXFull, (int)(r % kFtXStages)), (uint32_t)((r / kFtXStages) & 1));
        }
    }
    if (timed_out) atomicOr(P.status, kStTimeout);
    if (timed && lane == 0) {   // one thread per role: epilogue warps 0 and 4, MMA, loader
        if (warp == 0) {
            P.trace[46] = w0;
            P.trace[47] = w1;
        }
        if (warp == 4) P.trace[48] = w0 + w1;
        if (warp == kFtMmaWarp) {
            P.trace[49] = w0;
            P.trace[50] = w1;
            P.trace[51] = w2;
        }
        if (warp == kFtLoadWarp) {
            P.trace[52] = w0;
            P.trace[53] = w1;
        }
    }
    if (timed && warp == kFtLoadWarp && lane == 1) P.trace[54] = w2;
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

namespace {

int fit_tc_kp(int R) { return (R + 15) / 16 * 16; }

int fit_tc_chunks(long long I0) { return (int)((I0 + kFtN - 1) / kFtN); }

long long fit_tc_fibers(const Problem<float> &P)
{
    long long J = 1;
    for (int k = 1; k < P.N; ++k) J *= P.dims[k];
    return J;
}

// cuTensorMapEncodeTiled from the driver, found once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

bool fit_tc_supported(const Problem<float> &P)
{
    // fibers and tile coordinates stay below 2^31 (32-bit copy coordinates)
    // and the copy's row stride (ld_1 entries) is a multiple of 16 bytes
    return P.x_dtype == CPD_BF16 && P.R >= 1 && P.R <= 64 && fit_tc_fibers(P) < (1LL << 31) - kFtM &&
           P.ld[0] % 8 == 0 && encode_tiled() != nullptr;
}

size_t fit_tc_scratch_bytes(const Problem<float> &P)
{
    const int Kp = fit_tc_kp(P.R);
    const long long ntile = (fit_tc_fibers(P) + kFtM - 1) / kFtM;
    size_t b = (size_t)fit_tc_chunks(P.dims[0]) * 2 * kFtN * Kp * 2;
    for (int k = 1; k < P.N; ++k) b += ((size_t)P.dims[k] * Kp * 4 + 64 + 15) / 16 * 16;
    b += (size_t)ntile * 2 * kFtM * Kp * 2;
    return b + 256;
}

static void fit_tc_args(const Problem<float> &P, void *scratch, double *partials, FitTcArgs &a)
{
    a.Kp = fit_tc_kp(P.R);
    a.nchunks = fit_tc_chunks(P.dims[0]);
    a.J = fit_tc_fibers(P);
    a.partials = partials;
    char *p = static_cast<char *>(scratch);
    a.a0op = reinterpret_cast<__nv_bfloat16 *>(p);
    p += (size_t)a.nchunks * 2 * kFtN * a.Kp * 2;
    a.apad[0] = nullptr;
    for (int k = 1; k < P.N; ++k) {
        a.apad[k] = reinterpret_cast<float *>(p);
        p += ((size_t)P.dims[k] * a.Kp * 4 + 64 + 15) / 16 * 16;
    }
    a.ztiles = reinterpret_cast<__nv_bfloat16 *>(p);
}

cudaError_t launch_fit_tc(const Problem<float> &P, void *scratch, double *partials, int sm_count, double *out,
                          cudaStream_t s)
{
    FitTcArgs a{};
    fit_tc_args(P, scratch, partials, a);
    // the mode-1 replica as a 2-D tensor: ld_1 entries (contiguous) x J fibers,
    // boxes of 64 entries (128 bytes, the swizzle span) x 128 fibers
    CUtensorMap xmap;
    const cuuint64_t gdim[2] = {(cuuint64_t)P.ld[0], (cuuint64_t)a.J};
    const cuuint64_t gstride[1] = {(cuuint64_t)P.ld[0] * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)kFtM};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r = encode_tiled()(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(P.rep[0]), gdim,
                                      gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
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
    k_fit_tc_z<<<4 * sm_count, kThreads, 0, s>>>(P, a);
    const long long ntile = (a.J + kFtM - 1) / kFtM;
    const int grid = (int)std::min<long long>(ntile, sm_count);
    k_fit_tc<<<grid, kFtThreads, L.total, s>>>(P, a, xmap);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_fold(partials, grid, out, s);
}

}  // namespace cpd
