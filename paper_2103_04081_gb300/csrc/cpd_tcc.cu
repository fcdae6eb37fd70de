// Tensor-core gradient engine with thread-block clusters (sm_103a).
//
// Same arithmetic as the per-CTA engine (Eq. gradient1 as G_g = A H_g - M_g
// per fiber group g, M_g = X_S,g Z'_S,g on tcgen05, Z' as a bf16 hi/lo pair),
// but one cluster of cs CTAs handles one fiber group: CTA `rank` owns the
// row tile [128 rank, 128 rank + 128) of A^(n) and 1/cs of the group's
// fibers. Everything the row tiles of a group share -- the draws, the
// sampled KRP rows z_f, the B operands and H_g -- is computed once, in
// slices: each CTA draws and builds the operands of its own fibers and
// writes them into every CTA of the cluster through distributed shared
// memory; each CTA forms H over its own fibers, and CTA `rank` sums rows
// r = rank (mod cs) of those partials across the cluster (ascending rank,
// read through DSMEM) and writes the finished rows into every CTA.
//
// Phases of one CTA:
//   0. t, n; async copy of its A^(n) rows; TMEM / mbarrier set-up; early
//      arrival on the cluster barrier.
//   1. draws of its own fibers (Alg. 3), their columns (Eq. map) and weights.
//   2. its fibers' factor rows (async), then z_f, s_f z_f and the hi/lo B
//      operands, stored into all CTAs of the cluster (DSMEM), after the
//      early barrier has completed (every CTA has started).
//   3. cluster barrier: all fibers' columns and operands are everywhere.
//   4. gather of its rows of every fiber (cp.async, MN-major operand layout);
//      its slice of H_g, stored into all CTAs; MMAs; cluster barrier.
//   5. accumulator -> G_g = A H_g - M_g for its rows, staged and stored
//      coalesced as the group's partial.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cpd_device.cuh"
#include "cpd_internal.h"
#include "cpd_tcgen05.cuh"

namespace cpd {

namespace {

constexpr int kM = 128;   // rows per CTA (MMA M)
constexpr int kN = 64;    // R padded (MMA N)
constexpr int kK = 16;    // MMA K for 16-bit operands
constexpr int kCols = 64; // TMEM columns

struct TccSmem {
    size_t a, bhi, blo, zo, zso, hp, arow, h, rows, jcol, s, idx, bar, tmem, total;
    int lda, fpc;
    __host__ __device__ TccSmem(int N, int R, int fb, int cs)
    {
        lda = R | 1;
        fpc = ((fb + cs - 1) / cs + 7) / 8 * 8;   // own fibers per CTA, multiple of 8
        size_t o = 0;
        a = o;    o += (size_t)fb * kM * 2;                 // X tile (also CDF staging)
        bhi = o;  o += (size_t)fb * kN * 2;                 // Z' hi, K-major
        blo = o;  o += (size_t)fb * kN * 2;                 // Z' lo, K-major
        zo = o;   o += up((size_t)fpc * kN * 4);            // own z_f, [fiber][64]
        zso = o;  o += up((size_t)fpc * kN * 4);            // own s_f z_f
        hp = o;   o += (size_t)kN * kN * 4;                 // H over own fibers
        if (o - a < (size_t)kM * R * 4) o = a + up((size_t)kM * R * 4);   // epilogue tile staging
        arow = o; o += up((size_t)kM * lda * 4);            // A^(n) rows of the tile
        h = o;    o += (size_t)kN * kN * 4;                 // H_g
        rows = o; o += up((size_t)fpc * (N - 1) * R * 4);   // own fibers' factor rows
        jcol = o; o += up((size_t)fb * 8);
        s = o;    o += up((size_t)fb * 4);
        idx = o;  o += up((size_t)fpc * N * 4);
        bar = o;  o += 16;
        tmem = o; o += 16;
        total = o;
    }
    __host__ __device__ static size_t up(size_t v) { return (v + 127) / 128 * 128; }
};

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) k_grad_tcc(const Problem<float> P)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const bool tr0 = blockIdx.x == 0;
    trace_stamp(P.trace, 0, tr0);
    const long long t = *P.t_dev;
    const int N = P.N, R = P.R, fb = P.fb, cs = P.cs;
    const int n = mode_draw(P.seed, t, N);
    const int rank = (int)cluster_rank();
    const int gf = blockIdx.x / cs;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long In = P.dims[n];
    const int r0 = rank * kM;
    const bool has_rows = r0 < In;
    const int f0 = gf * fb;
    const int nf = (P.B - f0) < fb ? (P.B - f0) : fb;

    const TccSmem L(N, R, fb, cs);
    unsigned char *sA = smem + L.a;
    float *sArow = reinterpret_cast<float *>(smem + L.arow);
    float *sH = reinterpret_cast<float *>(smem + L.h);
    float *sRows = reinterpret_cast<float *>(smem + L.rows);
    float *sZo = reinterpret_cast<float *>(smem + L.zo);
    float *sZso = reinterpret_cast<float *>(smem + L.zso);
    float *sHp = reinterpret_cast<float *>(smem + L.hp);
    long long *jcol = reinterpret_cast<long long *>(smem + L.jcol);
    float *ss = reinterpret_cast<float *>(smem + L.s);
    int *sidx = reinterpret_cast<int *>(smem + L.idx);
    const uint32_t bar = smem_u32(smem + L.bar);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + L.tmem);
    const int lda = L.lda, fpc = L.fpc;
    const int fo0 = rank * fpc;                                   // own fibers [fo0, fo0+nown)
    const int nown = nf - fo0 < 0 ? 0 : (nf - fo0 < fpc ? nf - fo0 : fpc);

    // 0. own A^(n) rows (async), TMEM and mbarrier, early cluster arrival
    if (has_rows) {
        const float *An = P.A[n];
        const uint32_t dst0 = smem_u32(sArow);
        const int rows = (In - r0) < kM ? (int)(In - r0) : kM;
        for (int i = warp; i < rows; i += kThreads / 32) {
            const float *src = An + (long long)(r0 + i) * R;
            for (int q = lane; q < R; q += 32) cp_async4(dst0 + (uint32_t)((i * lda + q) * 4), src + q);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                             smem_u32(tmem_holder)),
                         "r"(kCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
        }
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
    }
    cluster_arrive();   // no remote store reaches this CTA before everyone has started
    trace_stamp(P.trace, 1, tr0);

    // 1. own fibers: draws (CDFs staged in the X-tile region, written by no
    //    other CTA), columns, weights
    draw_indices(P, t, n, f0 + fo0, nown, sidx, reinterpret_cast<unsigned long long *>(sA),
                 (long long)(fb * kM * 2) / 8);
    __syncthreads();
    trace_stamp(P.trace, 2, tr0);
    const uint32_t jcol_l = smem_u32(jcol), ss_l = smem_u32(ss);
    long long myj = 0;
    float mys = 0.f;
    if (threadIdx.x < nown) {
        const int f = threadIdx.x;
        const int *row = sidx + f * N;
        long long Jp = 1;
        for (int k = 0; k < N; ++k) {
            if (k == n) continue;
            myj += (long long)row[k] * Jp;
            Jp *= P.dims[k];
        }
        mys = fiber_weight(P, n, row);
        for (int k = 0; k < N; ++k) P.idx[(long long)(f0 + fo0 + f) * N + k] = row[k];
    }
    if (threadIdx.x < fpc && fo0 + (int)threadIdx.x < fb) {
        jcol[fo0 + threadIdx.x] = myj;   // local copies for the operand build below
        ss[fo0 + threadIdx.x] = mys;
    }
    {
        // own fibers' factor rows, one warp per (fiber, mode) row
        const uint32_t dst0 = smem_u32(sRows);
        for (int p2 = warp; p2 < nown * (N - 1); p2 += kThreads / 32) {
            const int f = p2 / (N - 1), kk = p2 % (N - 1);
            const int k = kk + (kk >= n ? 1 : 0);
            const float *src = P.A[k] + (long long)sidx[f * N + k] * R;
            const uint32_t dst = dst0 + (uint32_t)(p2 * R * 4);
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
    trace_stamp(P.trace, 10, tr0);
    asm volatile("cp.async.wait_all;\n" ::: "memory");     // A rows and factor rows
    __syncthreads();
    trace_stamp(P.trace, 11, tr0);

    // 2. operands of the own fibers, into every CTA of the cluster
    cluster_wait();
    if (threadIdx.x < fpc && fo0 + (int)threadIdx.x < fb) {
        const int f = fo0 + threadIdx.x;
        for (int d = 0; d < cs; ++d) {
            if (d == rank) continue;
            st_cluster_u64(map_shared(jcol_l + (uint32_t)(f * 8), d), (unsigned long long)myj);
            st_cluster_u32(map_shared(ss_l + (uint32_t)(f * 4), d), __float_as_uint(mys));
        }
    }
    {
        const uint32_t bhi_l = smem_u32(smem + L.bhi), blo_l = smem_u32(smem + L.blo);
        const int nb8 = fpc / 8;
        for (int job = threadIdx.x; job < kN * nb8; job += blockDim.x) {
            const int r = job % kN, b = job / kN;
            if (fo0 + 8 * b >= fb) continue;
            __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int fl = 8 * b + u;
                float v = 0.f;
                if (fl < nown && r < R) {
                    const float *fr = sRows + (long long)fl * (N - 1) * R + r;
                    v = 1.f;
                    for (int kk = 0; kk < N - 1; ++kk) v = v * fr[kk * R];
                }
                const float zs = fl < nown ? v * ss[fo0 + fl] : 0.f;
                sZo[fl * kN + r] = v;
                sZso[fl * kN + r] = zs;
                hi[u] = __float2bfloat16_rn(zs);
                lo[u] = __float2bfloat16_rn(zs - __bfloat162float(hi[u]));
            }
            const int f = fo0 + 8 * b;
            const uint32_t boff = (uint32_t)(((((r >> 3) * (fb >> 3) + (f >> 3)) << 6) + ((r & 7) << 3)) * 2);
            const uint4 vh = *reinterpret_cast<uint4 *>(hi), vl = *reinterpret_cast<uint4 *>(lo);
            for (int d = 0; d < cs; ++d) {
                st_cluster_v4(map_shared(bhi_l + boff, d), vh);
                st_cluster_v4(map_shared(blo_l + boff, d), vl);
            }
        }
    }
    __syncthreads();
    // H over the own fibers: 16 entries (one row, 16 columns) per thread
    {
        const int r = threadIdx.x >> 2, c0 = 16 * (threadIdx.x & 3);
        float acc[16] = {};
        for (int fl = 0; fl < nown; ++fl) {
            const float a = sZso[fl * kN + r];
            const float4 *b4 = reinterpret_cast<const float4 *>(sZo + fl * kN + c0);
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                const float4 y = b4[q4];
                acc[4 * q4 + 0] += a * y.x;
                acc[4 * q4 + 1] += a * y.y;
                acc[4 * q4 + 2] += a * y.z;
                acc[4 * q4 + 3] += a * y.w;
            }
        }
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4)
            *reinterpret_cast<float4 *>(sHp + r * kN + c0 + 4 * q4) =
                make_float4(acc[4 * q4], acc[4 * q4 + 1], acc[4 * q4 + 2], acc[4 * q4 + 3]);
    }
    trace_stamp(P.trace, 3, tr0);
    cluster_arrive();
    cluster_wait();
    trace_stamp(P.trace, 4, tr0);

    // 4. gather of this tile's rows of every fiber
    const uint32_t aBase = smem_u32(sA);
    if (has_rows) {
        const __nv_bfloat16 *rep = reinterpret_cast<const __nv_bfloat16 *>(P.rep[n]);
        const long long ld = P.ld[n];
        for (int c = threadIdx.x; c < fb * (kM / 8); c += blockDim.x) {
            const int f = c / (kM / 8), ig = c % (kM / 8);
            const long long i0 = r0 + ig * 8;
            const bool ok = f < nf && i0 < ld;
            const __nv_bfloat16 *src = ok ? rep + jcol[f] * ld + i0 : rep;
            cp_async16(aBase + (uint32_t)((((f >> 3) * (kM / 8) + ig) << 7) + ((f & 7) << 4)), src,
                       ok ? 16u : 0u);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    // rows r = rank, rank + cs, ... of H_g: the cluster's partials summed in
    // ascending rank, written into every CTA
    {
        const uint32_t h_l = smem_u32(sH), hp_l = smem_u32(sHp);
        const int nrows = (kN - rank + cs - 1) / cs;
        for (int e = threadIdx.x; e < nrows * kN; e += blockDim.x) {
            const int r = rank + cs * (e / kN), c = e % kN;
            const uint32_t off = (uint32_t)((r * kN + c) * 4);
            float acc = 0.f;
            for (int d = 0; d < cs; ++d) acc += ld_cluster_f32(map_shared(hp_l + off, d));
            for (int d = 0; d < cs; ++d) st_cluster_u32(map_shared(h_l + off, d), __float_as_uint(acc));
        }
    }
    trace_stamp(P.trace, 5, tr0);
    uint32_t tmem = 0;
    if (has_rows) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        tmem = *tmem_holder;
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t bhi = smem_u32(smem + L.bhi), blo = smem_u32(smem + L.blo);
            const uint32_t idesc = idesc_bf16(kM, kN);
            const uint32_t sboB = (uint32_t)(fb >> 3) * 128u;
            for (int ks = 0; ks < fb / kK; ++ks) {
                const uint64_t da = smem_desc(aBase + ks * 4096u, (kM / 8) * 128u, 128u);
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
    }
    cluster_arrive();   // H_g slices written
    cluster_wait();
    trace_stamp(P.trace, 6, tr0);

    // 5. G_g = A H_g - M_g for this tile's rows
    if (has_rows) {
        bool done = mbar_wait_bounded(bar, 0);
        if (!done) {
            if (threadIdx.x == 0) atomicOr(P.status, kStTimeout);
            done = mbar_wait_bounded(bar, 0);
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        trace_stamp(P.trace, 7, tr0);
        float *tile = reinterpret_cast<float *>(sA);
        if (done) {
            const int q = warp & 3, hh = warp >> 2;
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * hh), v);
            const int il = 32 * q + lane;
            trace_stamp(P.trace, 14, tr0);
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] = -v[c];
            for (int s2 = 0; s2 < R; ++s2) {
                const float a = sArow[il * lda + s2];
                const float4 *hrow = reinterpret_cast<const float4 *>(sH + s2 * kN + 32 * hh);
#pragma unroll
                for (int c4 = 0; c4 < 8; ++c4) {
                    const float4 hv = hrow[c4];
                    v[4 * c4 + 0] += a * hv.x;
                    v[4 * c4 + 1] += a * hv.y;
                    v[4 * c4 + 2] += a * hv.z;
                    v[4 * c4 + 3] += a * hv.w;
                }
            }
            trace_stamp(P.trace, 15, tr0);
#pragma unroll
            for (int c = 0; c < 32; ++c)
                if (32 * hh + c < R) tile[il * R + 32 * hh + c] = v[c];
        }
        __syncthreads();
        if (done) {
            const int rows = (In - r0) < kM ? (int)(In - r0) : kM;
            float *out = P.part + ((long long)gf * In + r0) * R;
            for (int e = threadIdx.x; e < rows * R; e += blockDim.x) out[e] = tile[e];
        }
        trace_stamp(P.trace, 8, tr0);
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols)
                         : "memory");
    }
    trace_stamp(P.trace, 9, tr0);
}

size_t tcc_smem_bytes(const Problem<float> &P) { return TccSmem(P.N, P.R, P.fb, P.cs).total; }

// The kernel's dynamic shared-memory limit, raised (never lowered) as needed;
// the one place that sets it, so the recorded value is the attribute's.
static cudaError_t ensure_smem_attr(size_t need)
{
    static size_t attr_bytes = 0;
    if (need <= attr_bytes) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k_grad_tcc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    attr_bytes = need;
    return cudaSuccess;
}

cudaError_t launch_grad_tcc(const Problem<float> &P, int grid, cudaStream_t s)
{
    const size_t need = tcc_smem_bytes(P);
    if (cudaError_t e = ensure_smem_attr(need); e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = need;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_grad_tcc, P);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

int tcc_max_clusters(const Problem<float> &P)
{
    const size_t need = tcc_smem_bytes(P);
    if (ensure_smem_attr(need) != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.cs);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = need;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_grad_tcc, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace cpd
