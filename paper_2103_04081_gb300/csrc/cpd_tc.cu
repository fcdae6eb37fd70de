// Tensor-core gradient engine for BF16 tensors (sm_103a: tcgen05.mma with the
// accumulator in tensor memory).
//
// Eq. (11) split over fiber groups g (the batch is cut into groups of fb
// fibers, one CTA per (row tile, group)): with Z'_S = D Z_S / (B J_n) (the
// weight s_f folded into each sampled KRP row),
//   M_g = X_S,g Z'_S,g      (I_n x R)  -- tensor cores
//   H_g = Z_S,g^T Z'_S,g    (R x R)    -- CUDA cores, FP32
//   G_g = A^(n) H_g - M_g               -- tensor cores, same accumulator
// and k_update sums the G_g in fixed order. The gathered fibers are BF16
// (exact copies of the stored tensor). Z' is split into a BF16 pair
// hi = bf16(z'), lo = bf16(z' - hi), built negated so that the accumulator
// receives -M_g; A^(n)'s rows and H_g are split the same way and added as
// hi*hi + hi*lo + lo*hi. Each operand keeps ~16 significant bits.
//
// Per CTA (rb = 128 rows of A^(n), fb fibers, fb a multiple of 16):
//   1. draw the fibers (warp-cooperative inverse-CDF search), p_f, s_f;
//   2. 16-byte cp.async copies of rows [r0, r0+128) of every fiber straight
//      into the no-swizzle MN-major operand layout (zero fill past I_n), and
//      the CTA's rows of A^(n) into shared memory;
//   3. z_f and the hi/lo B operands (K-major), zero-padded to N = 64;
//   4. one thread issues 2*fb/16 tcgen05.mma (M=128, N=64, K=16); meanwhile
//      the CTA computes H_g;
//   5. A^(n) rows (MN-major) and H_g (K-major) become bf16 hi/lo operands in
//      the buffers H_g's formation freed; one thread issues the A H_g
//      products and commits every product to an mbarrier;
//   6. tcgen05.ld of G_g, stored as the group's partial.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cpd_device.cuh"
#include "cpd_internal.h"
#include "cpd_tcgen05.cuh"

namespace cpd {

namespace {

constexpr int kTcM = 128;        // rows per CTA (MMA M)
constexpr int kTcN = 64;         // R padded (MMA N)
constexpr int kTcK = 16;         // K of one MMA for 16-bit operands
constexpr int kTcCols = 64;      // TMEM columns allocated (FP32 accumulator, N = 64)
constexpr size_t kAopBytes = (size_t)kTcM * kTcN * 2 * 2;   // A^(n) rows, bf16 hi + lo
constexpr size_t kOpBytes = kAopBytes + (size_t)kTcN * kTcN * 2 * 2;   // + H_g hi + lo

// Shared memory of one CTA (byte offsets; operand tiles 128-byte aligned).
struct TcSmem {
    size_t a, bhi, blo, zs, z, arow, h, rows, s, idx, jcol, bar, tmem, total;
    int lda;  // row stride (floats) of the A^(n) tile: R rounded up to odd
    __host__ __device__ TcSmem(int N, int R, int fb)
    {
        lda = R | 1;
        size_t o = 0;
        a = o;    o += (size_t)fb * kTcM * 2;               // X tile, MN-major bf16
        bhi = o;  o += (size_t)fb * kTcN * 2;               // Z' hi, K-major bf16
        blo = o;  o += (size_t)fb * kTcN * 2;               // Z' lo, K-major bf16
        zs = o;   o += (size_t)fb * kTcN * 4;               // s_f z_f, fp32, 64 wide
        z = o;    o += (size_t)fb * kTcN * 4;               // z_f, fp32, 64 wide
        // [zs, zs + 48 KB) holds the A H_g operands once H_g is formed:
        // A^(n) rows hi / lo (MN-major) then H_g hi / lo (K-major)
        if (o - zs < kOpBytes) o = zs + kOpBytes;
        // [a, arow) is dead once the MMAs are done: it stages the 128 x R
        // G tile of the epilogue, so it must hold at least that much
        if (o - a < (size_t)kTcM * R * 4) o = a + up((size_t)kTcM * R * 4);
        arow = o; o += up((size_t)kTcM * lda * 4);          // A^(n) rows of the tile
        h = o;    o += (size_t)kTcN * kTcN * 4;             // H_g, 64 x 64
        rows = o; o += up((size_t)fb * (N - 1) * R * 4);    // gathered factor rows
        s = o;    o += up((size_t)fb * 4);
        idx = o;  o += up((size_t)fb * N * 4);
        jcol = o; o += up((size_t)fb * 8);
        bar = o;  o += 16;
        tmem = o; o += 16;
        total = o;
    }
    __host__ __device__ static size_t up(size_t v) { return (v + 127) / 128 * 128; }
};

}  // namespace

// `bid` is the CTA's index among the CTAs of this problem.
__device__ __forceinline__ void grad_tc_body(const Problem<float> &P, int bid)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const bool tr0 = bid == 0;
    trace_stamp(P.trace, 0, tr0);
    const long long t = *P.t_dev;
    const int N = P.N, R = P.R, fb = P.fb;
    const int n = mode_draw(P.seed, t, N);
    const int pr = P.tile[n].pr;
    const int gr = bid % pr, gf = bid / pr;
    if (gf >= P.pf) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long In = P.dims[n];
    const int r0 = gr * kTcM;
    const int f0 = gf * fb;
    const int nf = (P.B - f0) < fb ? (P.B - f0) : fb;

    const TcSmem L(N, R, fb);
    unsigned char *sA = smem + L.a;
    __nv_bfloat16 *sBhi = reinterpret_cast<__nv_bfloat16 *>(smem + L.bhi);
    __nv_bfloat16 *sBlo = reinterpret_cast<__nv_bfloat16 *>(smem + L.blo);
    float *szs = reinterpret_cast<float *>(smem + L.zs);
    float *sz = reinterpret_cast<float *>(smem + L.z);
    float *sArow = reinterpret_cast<float *>(smem + L.arow);
    float *sH = reinterpret_cast<float *>(smem + L.h);
    float *sRows = reinterpret_cast<float *>(smem + L.rows);
    float *ss = reinterpret_cast<float *>(smem + L.s);
    int *sidx = reinterpret_cast<int *>(smem + L.idx);
    long long *jcol = reinterpret_cast<long long *>(smem + L.jcol);
    const uint32_t bar = smem_u32(smem + L.bar);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + L.tmem);
    const int lda = L.lda;

    // 0. the tile's rows of A^(n) (independent of the draws): async copies
    {
        const float *An = P.A[n];
        const uint32_t dst0 = smem_u32(sArow);
        const int rows = (In - r0) < kTcM ? (int)(In - r0) : kTcM;
        for (int i = warp; i < rows; i += kThreads / 32) {
            const float *src = An + (long long)(r0 + i) * R;
            for (int q = lane; q < R; q += 32) cp_async4(dst0 + (uint32_t)((i * lda + q) * 4), src + q);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(tmem_holder)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }

    trace_stamp(P.trace, 1, tr0);
    // 1. draws (Alg. 3), fiber columns (Eq. (2)) and weights s_f; the CDFs are
    //    staged over the operand tiles, which are not written before the gather
    const long long cap = (long long)(L.zs - L.a) / 8;
    draw_indices(P, t, n, f0, nf, sidx, reinterpret_cast<unsigned long long *>(sA), cap,
                 reinterpret_cast<unsigned long long *>(szs), bid == 0);
    const bool staged = cdfs_staged(P, n, cap);
    __syncthreads();
    trace_stamp(P.trace, 2, tr0);
    for (int f = threadIdx.x; f < fb; f += blockDim.x) {
        if (f < nf) {
            const int *row = sidx + f * N;
            long long j = 0, Jp = 1;
            for (int k = 0; k < N; ++k) {
                if (k == n) continue;
                j += (long long)row[k] * Jp;
                Jp *= P.dims[k];
            }
            jcol[f] = j;
            ss[f] = staged ? fiber_weight_staged(P, n, row, reinterpret_cast<const unsigned long long *>(sA))
                           : fiber_weight(P, n, row);
            if (gr == 0)
                for (int k = 0; k < N; ++k) P.idx[(long long)(f0 + f) * N + k] = row[k];
        } else {
            jcol[f] = 0;
            ss[f] = 0.f;
        }
    }
    trace_stamp(P.trace, 10, tr0);
    // factor rows A^(k)(i_k, :), k != n, of every fiber: async copies
    {
        // one warp per (fiber, mode) row; 8-byte copies when rows are 8-byte aligned
        const uint32_t dst0 = smem_u32(sRows);
        for (int pr2 = warp; pr2 < nf * (N - 1); pr2 += kThreads / 32) {
            const int f = pr2 / (N - 1), kk = pr2 % (N - 1);
            const int k = kk + (kk >= n ? 1 : 0);
            const float *src = P.A[k] + (long long)sidx[f * N + k] * R;
            const uint32_t dst = dst0 + (uint32_t)(pr2 * R * 4);
            if ((R & 1) == 0) {
                for (int q = lane; q < R / 2; q += 32)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst + q * 8), "l"(src + 2 * q)
                                 : "memory");
            } else {
                for (int q = lane; q < R; q += 32) cp_async4(dst + q * 4, src + q);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    trace_stamp(P.trace, 11, tr0);
    __syncthreads();

    trace_stamp(P.trace, 3, tr0);
    // 2. gather: chunk (f, ig) = rows r0+8ig .. r0+8ig+7 of fiber f, 16 bytes,
    //    to core matrix (f/8, ig) at ((f/8)*16 + ig)*128 + (f%8)*16.
    const __nv_bfloat16 *rep = reinterpret_cast<const __nv_bfloat16 *>(P.rep[n]);
    const long long ld = P.ld[n];
    const uint32_t aBase = smem_u32(sA);
    for (int c = threadIdx.x; c < fb * (kTcM / 8); c += blockDim.x) {
        const int f = c / (kTcM / 8), ig = c % (kTcM / 8);
        const long long i0 = r0 + ig * 8;
        const bool ok = f < nf && i0 < ld;
        const __nv_bfloat16 *src = ok ? rep + jcol[f] * ld + i0 : rep;
        cp_async16(aBase + (uint32_t)((((f >> 3) * (kTcM / 8) + ig) << 7) + ((f & 7) << 4)), src,
                   ok ? 16u : 0u);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");

    trace_stamp(P.trace, 4, tr0);
    // 3. z_f = Hadamard product of the gathered rows (Alg. 1), and the B
    //    operands Z' = s_f z_f as a bf16 hi/lo pair, K-major: element (r, f) at
    //    ((r/8)*(fb/8) + f/8)*64 + (r%8)*8 + f%8. Rows past R are zero.
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // A rows and factor rows landed
    __syncthreads();
    trace_stamp(P.trace, 12, tr0);
    for (int e = threadIdx.x; e < fb * kTcN; e += blockDim.x) {
        const int f = e / kTcN, r = e % kTcN;
        float z = 0.f;
        if (f < nf && r < R) {
            const float *fr = sRows + (long long)f * (N - 1) * R + r;
            z = 1.f;
            for (int kk = 0; kk < N - 1; ++kk) z = z * fr[kk * R];
        }
        const float zp = z * ss[f];
        sz[f * kTcN + r] = z;
        szs[f * kTcN + r] = zp;
        const __nv_bfloat16 hi = __float2bfloat16_rn(-zp);     // -Z': the accumulator gets -M_g
        const __nv_bfloat16 lo = __float2bfloat16_rn(-zp - __bfloat162float(hi));
        const int off = (((r >> 3) * (fb >> 3) + (f >> 3)) << 6) + ((r & 7) << 3) + (f & 7);
        sBhi[off] = hi;
        sBlo[off] = lo;
    }
    trace_stamp(P.trace, 13, tr0);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    const uint32_t tmem = *tmem_holder;
    trace_stamp(P.trace, 5, tr0);

    // 4. M_g = X Z' on the tensor cores (one thread issues), H_g meanwhile
    if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t bhi = smem_u32(sBhi), blo = smem_u32(sBlo);
        const uint32_t idesc = idesc_bf16(kTcM, kTcN);
        const uint32_t sboB = (uint32_t)(fb >> 3) * 128u;
        for (int ks = 0; ks < fb / kTcK; ++ks) {
            const uint64_t da = smem_desc(aBase + ks * 4096u, (kTcM / 8) * 128u, 128u);
            const uint64_t dh = smem_desc(bhi + ks * 256u, 128u, sboB);
            const uint64_t dl = smem_desc(blo + ks * 256u, 128u, sboB);
            const uint32_t acc = ks > 0 ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                "l"(da), "l"(dh), "r"(idesc), "r"(acc)
                : "memory");
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                "l"(da), "l"(dl), "r"(idesc), "r"(1u)
                : "memory");
        }
    }
    {
        // H_g = sum_f (s_f z_f) z_f^T: a 4 x 4 block of the 64 x 64 result per thread
        const int rb = threadIdx.x >> 4, cb = threadIdx.x & 15;
        float hacc[4][4] = {};
        for (int f = 0; f < nf; ++f) {
            const float4 a = *reinterpret_cast<const float4 *>(szs + f * kTcN + 4 * rb);
            const float4 b = *reinterpret_cast<const float4 *>(sz + f * kTcN + 4 * cb);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) hacc[u][v] += av[u] * bv[v];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            *reinterpret_cast<float4 *>(sH + (4 * rb + u) * kTcN + 4 * cb) =
                make_float4(hacc[u][0], hacc[u][1], hacc[u][2], hacc[u][3]);
    }
    __syncthreads();

    // 5. + A H_g on the tensor cores: A^(n) rows -> bf16 hi/lo MN-major (like
    //    X), H_g -> bf16 hi/lo K-major (like Z'), in the buffers H_g freed;
    //    K = R padded to 16. One commit covers every product of this CTA.
    {
        __nv_bfloat16 *aHi = reinterpret_cast<__nv_bfloat16 *>(szs);
        __nv_bfloat16 *aLo = aHi + kTcM * kTcN;
        __nv_bfloat16 *hHi = aLo + kTcM * kTcN;
        __nv_bfloat16 *hLo = hHi + kTcN * kTcN;
        const int rowsA = (In - r0) < kTcM ? (int)(In - r0) : kTcM;
        for (int job = threadIdx.x; job < kTcN * (kTcM / 8); job += blockDim.x) {
            const int r = job % kTcN, ig = job / kTcN;   // K index r, rows 8 ig .. 8 ig + 7
            __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = 8 * ig + u;
                const float a = (i < rowsA && r < R) ? sArow[i * lda + r] : 0.f;
                hi[u] = __float2bfloat16_rn(a);
                lo[u] = __float2bfloat16_rn(a - __bfloat162float(hi[u]));
            }
            const int off = (((r >> 3) * (kTcM >> 3) + ig) << 6) + ((r & 7) << 3);
            *reinterpret_cast<uint4 *>(aHi + off) = *reinterpret_cast<uint4 *>(hi);
            *reinterpret_cast<uint4 *>(aLo + off) = *reinterpret_cast<uint4 *>(lo);
        }
        for (int job = threadIdx.x; job < kTcN * (kTcN / 8); job += blockDim.x) {
            const int c = job % kTcN, rg = job / kTcN;   // column c of H_g, rows 8 rg .. 8 rg + 7
            __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float h = sH[(8 * rg + u) * kTcN + c];
                hi[u] = __float2bfloat16_rn(h);
                lo[u] = __float2bfloat16_rn(h - __bfloat162float(hi[u]));
            }
            const int off = (((c >> 3) * (kTcN >> 3) + rg) << 6) + ((c & 7) << 3);
            *reinterpret_cast<uint4 *>(hHi + off) = *reinterpret_cast<uint4 *>(hi);
            *reinterpret_cast<uint4 *>(hLo + off) = *reinterpret_cast<uint4 *>(lo);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t idesc = idesc_bf16(kTcM, kTcN);
            const uint32_t ah = smem_u32(aHi), al = smem_u32(aLo), bh = smem_u32(hHi), bl = smem_u32(hLo);
            for (int ks = 0; ks < (R + kTcK - 1) / kTcK; ++ks) {
                const uint64_t dah = smem_desc(ah + ks * 4096u, (kTcM / 8) * 128u, 128u);
                const uint64_t dal = smem_desc(al + ks * 4096u, (kTcM / 8) * 128u, 128u);
                const uint64_t dbh = smem_desc(bh + ks * 256u, 128u, (kTcN / 8) * 128u);
                const uint64_t dbl = smem_desc(bl + ks * 256u, 128u, (kTcN / 8) * 128u);
                const uint64_t pa[3] = {dah, dah, dal}, pb[3] = {dbh, dbl, dbh};
#pragma unroll
                for (int u = 0; u < 3; ++u)
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                        "l"(pa[u]), "l"(pb[u]), "r"(idesc), "r"(1u)
                        : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                         : "memory");
        }
    }

    trace_stamp(P.trace, 6, tr0);
    // 6. accumulator -> G_g for row i, columns [32h, 32h+32)
    bool done = mbar_wait_bounded(bar, 0);
    if (!done) {
        if (threadIdx.x == 0) atomicOr(P.status, kStTimeout);
        done = mbar_wait_bounded(bar, 0);
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    trace_stamp(P.trace, 7, tr0);
    if (done) {
        const int q = warp & 3, h = warp >> 2;
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h), v);
        const int il = 32 * q + lane;
        trace_stamp(P.trace, 14, tr0);
        trace_stamp(P.trace, 15, tr0);
        float *tile = reinterpret_cast<float *>(sA);   // operands are dead: stage the 128 x R tile
#pragma unroll
        for (int c = 0; c < 32; ++c)
            if (32 * h + c < R) tile[il * R + 32 * h + c] = v[c];
    }
    __syncthreads();
    if (done) {
        // the tile's rows are contiguous in the partial slab: coalesced stores
        const int rows = (In - r0) < kTcM ? (int)(In - r0) : kTcM;
        float *out = P.part + ((long long)gf * In + r0) * R;
        const float *tile = reinterpret_cast<const float *>(sA);
        for (int e = threadIdx.x; e < rows * R; e += blockDim.x) out[e] = tile[e];
    }
    trace_stamp(P.trace, 8, tr0);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    trace_stamp(P.trace, 9, tr0);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols)
                     : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) k_grad_tc(const Problem<float> P)
{
    grad_tc_body(P, (int)blockIdx.x);
}

// One launch for a group of problems (see group_member).
__global__ void __launch_bounds__(kThreads, 1) k_grad_tc_group(const Problem<float> *__restrict__ Ps,
                                                               const int *__restrict__ cta0, int G)
{
    __shared__ __align__(16) Problem<float> sp;
    const int g = group_member(Ps, cta0, G, sp);
    grad_tc_body(sp, (int)blockIdx.x - __ldg(cta0 + g));
}

cudaError_t launch_grad_tc_group(const GroupLaunch<float> &L, cudaStream_t s)
{
    static size_t attr_bytes = 0;
    if (L.smem_grad > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k_grad_tc_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L.smem_grad);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        attr_bytes = L.smem_grad;
    }
    k_grad_tc_group<<<L.grid_grad, kThreads, L.smem_grad, s>>>(L.P, L.cta_grad, L.G);
    return cudaGetLastError();
}

bool tc_supported(int R, int rb) { return R >= 1 && R <= kTcN && rb == kTcM; }

size_t tc_smem_bytes(const Problem<float> &P) { return TcSmem(P.N, P.R, P.fb).total; }

long long tc_stage_cap(const Problem<float> &P)
{
    const TcSmem L(P.N, P.R, P.fb);
    return (long long)(L.zs - L.a) / 8;
}

cudaError_t launch_grad_tc(const Problem<float> &P, int grid, cudaStream_t s)
{
    static size_t attr_bytes = 0;
    const size_t need = tc_smem_bytes(P);
    if (need > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        attr_bytes = need;
    }
    k_grad_tc<<<grid, kThreads, need, s>>>(P);
    return cudaGetLastError();
}

}  // namespace cpd
