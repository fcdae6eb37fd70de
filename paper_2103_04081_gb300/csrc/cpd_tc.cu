// Tensor-core gradient engine for BF16 tensors (sm_103a: tcgen05.mma with the
// accumulator in tensor memory).
//
// Eq. gradient1 in the M/H form: with Z'_S = D Z_S / (B J_n) (s_f folded into
// the sampled KRP rows),
//   M = X_S Z'_S        (I_n x R)  -- tensor cores, per (row tile, fiber group)
//   H = Z_S^T Z'_S      (R x R)    -- CUDA cores, FP32, reduced in fixed order
//   G = A^(n) H - M                 -- k_update.
// The gathered fibers are BF16 (exact copies of the stored tensor). Z' is
// split into a BF16 pair hi + lo, hi = bf16(z'), lo = bf16(z' - hi), and both
// products accumulate into the same FP32 accumulator, which keeps ~16
// significant bits of Z' instead of 8.
//
// Per CTA (rb = 128 rows of A^(n), fb fibers, fb a multiple of 16):
//   1. draw the fibers (warp-cooperative inverse-CDF search), p_f, s_f;
//   2. 16-byte cp.async copies of rows [r0, r0+128) of every fiber straight
//      into the no-swizzle MN-major operand layout (zero fill past I_n);
//   3. z_f and the hi/lo B operands (K-major), zero-padded to N = 64;
//   4. one thread issues 2*fb/16 tcgen05.mma (M=128, N=64, K=16) and commits
//      to an mbarrier; meanwhile the CTA computes its share of H;
//   5. tcgen05.ld of the accumulator -> M partial [gf][i][r];
//   6. the last CTA to finish reduces the H partials (fixed order).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cpd_device.cuh"
#include "cpd_internal.h"

namespace cpd {

namespace {

constexpr int kTcM = 128;        // rows per CTA (MMA M)
constexpr int kTcN = 64;         // R padded (MMA N)
constexpr int kTcK = 16;         // K of one MMA for 16-bit operands
constexpr int kTcCols = 64;      // TMEM columns allocated (FP32 accumulator, N = 64)
constexpr unsigned kWaitLimit = 1u << 24;

struct TcSmem {
    size_t a, bhi, blo, z, s, idx, jcol, bar, tmem, total;
    __host__ __device__ TcSmem(int N, int R, int fb)
    {
        size_t o = 0;
        a = o;    o += (size_t)fb * kTcM * 2;          // X tile, MN-major
        bhi = o;  o += (size_t)fb * kTcN * 2;          // Z' hi, K-major
        blo = o;  o += (size_t)fb * kTcN * 2;          // Z' lo, K-major
        z = o;    o += up((size_t)fb * R * 4);         // z_f (FP32)
        s = o;    o += up((size_t)fb * 4);             // s_f (FP32)
        idx = o;  o += up((size_t)fb * N * 4);
        jcol = o; o += up((size_t)fb * 8);
        bar = o;  o += 16;
        tmem = o; o += 16;
        // Slack so that every operand read stays inside the allocation even
        // under a transposed reading of the descriptor strides.
        total = o + 32768;
    }
    __host__ __device__ static size_t up(size_t v) { return (v + 127) / 128 * 128; }
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle: start address, leading
// byte offset (core matrices adjacent in K), stride byte offset (adjacent in
// M/N), all >> 4; bits 46-47 carry the descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, A MN-major,
// B K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(addr), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t phase)
{
    for (unsigned it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(addr, phase)) return true;
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) k_grad_tc(const Problem<float> P)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const long long t = *P.t_dev;
    const int N = P.N, R = P.R, fb = P.fb;
    const int n = mode_draw(P.seed, t, N);
    const int pr = P.tile[n].pr;
    const int gr = blockIdx.x % pr, gf = blockIdx.x / pr;
    const bool active = gf < P.pf;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const TcSmem L(N, R, fb);
    unsigned char *sA = smem + L.a;
    __nv_bfloat16 *sBhi = reinterpret_cast<__nv_bfloat16 *>(smem + L.bhi);
    __nv_bfloat16 *sBlo = reinterpret_cast<__nv_bfloat16 *>(smem + L.blo);
    float *sz = reinterpret_cast<float *>(smem + L.z);
    float *ss = reinterpret_cast<float *>(smem + L.s);
    int *sidx = reinterpret_cast<int *>(smem + L.idx);
    long long *jcol = reinterpret_cast<long long *>(smem + L.jcol);
    const uint32_t bar = smem_u32(smem + L.bar);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + L.tmem);

    if (active) {
        const long long In = P.dims[n];
        const int r0 = gr * kTcM;
        const int f0 = gf * fb;
        const int nf = (P.B - f0) < fb ? (P.B - f0) : fb;

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

        // 1. draws, fiber columns, probabilities and weights
        draw_indices(P, t, n, f0, nf, sidx);
        __syncthreads();
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
                const double p = fiber_prob(P, n, row);
                ss[f] = (float)__ddiv_rn(1.0, __dmul_rn(__dmul_rn((double)P.B, P.Jn[n]), p));
                if (gr == 0) {
                    P.p[f0 + f] = p;
                    for (int k = 0; k < N; ++k) P.idx[(long long)(f0 + f) * N + k] = row[k];
                }
            } else {
                jcol[f] = 0;
                ss[f] = 0.f;
            }
        }
        __syncthreads();

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

        // 3. z_f (FP32) and the B operands Z' = s_f z_f as a bf16 hi/lo pair,
        //    K-major: element (r, f) at ((r/8)*(fb/8) + f/8)*64 + (r%8)*8 + f%8.
        for (int e = threadIdx.x; e < fb * kTcN; e += blockDim.x) {
            const int f = e / kTcN, r = e % kTcN;
            float z = 0.f;
            if (f < nf && r < R) {
                const int *row = sidx + f * N;
                z = 1.f;
                for (int k = 0; k < N; ++k) {
                    if (k == n) continue;
                    z = z * P.A[k][(long long)row[k] * R + r];
                }
                sz[f * R + r] = z;
            }
            const float zp = z * ss[f];
            const __nv_bfloat16 hi = __float2bfloat16_rn(zp);
            const __nv_bfloat16 lo = __float2bfloat16_rn(zp - __bfloat162float(hi));
            const int off = (((r >> 3) * (fb >> 3) + (f >> 3)) << 6) + ((r & 7) << 3) + (f & 7);
            sBhi[off] = hi;
            sBlo[off] = lo;
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        const uint32_t tmem = *tmem_holder;

        // 4. MMAs (one thread), H share on the CUDA cores meanwhile
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
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             bar)
                         : "memory");
        }
        const int npairs = R * (R + 1) / 2;
        for (int lp = threadIdx.x; gr + lp * pr < npairs; lp += blockDim.x) {
            int rem = gr + lp * pr, r = 0;
            while (rem >= R - r) {
                rem -= R - r;
                ++r;
            }
            const int s2 = r + rem;
            float acc = 0.f;
            for (int f = 0; f < nf; ++f) acc += ss[f] * sz[f * R + r] * sz[f * R + s2];
            P.hpart[((long long)gf * R + r) * R + s2] = acc;
            P.hpart[((long long)gf * R + s2) * R + r] = acc;
        }

        // 5. accumulator -> M partial rows
        bool done = mbar_wait_bounded(bar, 0);
        if (!done) {
            if (threadIdx.x == 0) atomicOr(P.status, kStTimeout);
            done = mbar_wait_bounded(bar, 0);
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (done) {
            const int q = warp & 3, h = warp >> 2;
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h), v);
            const long long i = r0 + 32 * q + lane;
            if (i < In) {
                float *out = P.part + ((long long)gf * In + i) * R;
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (32 * h + c < R) out[32 * h + c] = v[c];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols)
                         : "memory");
    }

    // 6. the last CTA reduces H over fiber groups in fixed order
    if (!last_block(P.counters + 4)) return;
    const int RR = R * R;
    float *H = P.hpart + (long long)P.pf * RR;
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
        float h = 0.f;
        for (int g = 0; g < P.pf; ++g) h += __ldcg(P.hpart + (long long)g * RR + e);
        H[e] = h;
    }
    if (threadIdx.x == 0) P.counters[4] = 0;
}

bool tc_supported(int R, int rb) { return R >= 1 && R <= kTcN && rb == kTcM; }

size_t tc_smem_bytes(const Problem<float> &P) { return TcSmem(P.N, P.R, P.fb).total; }

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
