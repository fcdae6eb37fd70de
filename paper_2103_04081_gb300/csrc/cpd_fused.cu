// Fused iteration engine (sm_103a): the gradient of Eq. (11) and the step of
// Eq. (12) / (13a)-(13b) for the drawn mode in ONE kernel, with no partials
// in global memory and no second launch.
//
// One cluster of cs CTAs per tile of 128 tpc rows of A^(n) (tpc = 1 or 2
// MMA tiles of 128 rows; 2 where the tiles of 128 would outnumber the
// clusters the device co-schedules). CTA `rank` of every cluster takes fibers
// [rank fpc, rank fpc + fpc) of the batch, so each cluster holds the whole
// batch and the clusters of a launch never wait on each other:
//   1. the CTA draws its fibers (Alg. 3), forms their columns (Eq. (2)), the
//      weights s_f = 1/(B J_n p_f) (Eq. (10), (11)) and the KRP rows z_f
//      (Eq. (3), Alg. 1);
//   2. it gathers its fibers' entries of the tile's rows into an MN-major
//      bf16 operand and forms its partials on the tensor cores, FP32
//      accumulation in tensor memory:
//        M_c = X_S Z'_S,                 Z' = s_f z_f as a bf16 hi/lo pair;
//        H_c = sum_f z_f (s_f z_f)^T,    z_f and s_f z_f both as hi/lo pairs,
//                                        all four products;
//   3. CTA `rank` owns rows [rank mr, rank mr + mr) of the tile's M and rows
//      [rank hr, rank hr + hr) of H: it sums those rows of every CTA's
//      partial in ascending rank through distributed shared memory, then
//      reads the rest of H from their owners;
//   4. for its own rows of A^(n): G = A^(n) H - M in FP32 (k ascending), the
//      step with the AdaGrad state in FP64, the projection and the rows' new
//      Euclidean weights; the launch's last CTA publishes the iteration
//      (counter, mode, CDF state) as the separate update kernel does.
// Three cluster barriers per launch; every wait on the tensor cores is
// bounded.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cpd_device.cuh"
#include "cpd_internal.h"
#include "cpd_tcgen05.cuh"

namespace cpd {

namespace {

constexpr int kM = 128;     // rows of an MMA tile of A^(n) (MMA M)
constexpr int kN = 64;      // R padded (MMA N)
constexpr int kK = 16;      // MMA K for 16-bit operands
constexpr int kCols = 256;  // TMEM columns: M of MMA tile 0 [0, 64), H products [64, 128) and
                            // [128, 192), M of MMA tile 1 [192, 256)
constexpr int kMs = 68;     // row stride (floats) of the FP32 partials: 16-byte rows, no bank conflicts
constexpr int kMaxCs = 16;

// Instruction descriptor of kind::f16, D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_kk(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// bf16 index of element (row, k) in a K-major, no-swizzle operand of Kp
// columns: core matrices of 8 rows x 8 k (16 bytes a row), adjacent in k 128
// bytes apart, adjacent in rows Kp / 8 * 128 bytes apart.
__device__ __forceinline__ int kmaj(int row, int k, int Kp)
{
    return (((row >> 3) * (Kp >> 3) + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

struct FusedSmem {
    size_t a, bhi, blo, zc, hp, hq, h, arow, srow, snew, jcol, s, idx, bar, tmem, total;
    size_t abytes;
    int fpc, mr, hr;
    __host__ __device__ FusedSmem(int N, int R, int fpc_, int cs, int tpc)
    {
        fpc = fpc_;          // fibers per CTA, multiple of 16
        mr = kM * tpc / cs;  // rows of the cluster's M owned per CTA
        hr = kN / cs;        // rows of H owned per CTA
        const size_t xa = (size_t)fpc * kM * 2 * tpc, mp = (size_t)kM * tpc * kMs * 4;
        abytes = xa > mp ? xa : mp;
        size_t o = 0;
        a = o;    o += up(abytes);                     // CDF stage, then the X tiles (one per MMA tile),
                                                       // then the partial M
        bhi = o;  o += (size_t)fpc * kN * 2;           // Z' hi (K-major, fpc columns)
        blo = o;  o += (size_t)fpc * kN * 2;           // Z' lo
        zc = o;   o += (size_t)fpc * kM * 2;           // z hi (rows 0-63) and z lo (rows 64-127), K-major
        hp = o;   o += up((size_t)kN * kMs * 4);       // draw scratch, then the partial H
        hq = o;   o += up((size_t)kN * kMs * 4);       // the z-lo half of the partial H
        h = o;    o += up((size_t)kN * kMs * 4);       // H: owned rows summed, the rest read from their owners
        arow = o; o += up((size_t)mr * R * 4);         // owned rows of A^(n)
        srow = o; o += up((size_t)mr * R * 8);         // their AdaGrad state
        snew = o; o += up((size_t)mr * R * 4);         // their new values
        jcol = o; o += up((size_t)fpc * 8);
        s = o;    o += up((size_t)fpc * 4);
        idx = o;  o += up((size_t)fpc * N * 4);
        bar = o;  o += 16;
        tmem = o; o += 16;
        total = o;
    }
    __host__ __device__ static size_t up(size_t v) { return (v + 127) / 128 * 128; }
};

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ float4 add4(float4 a, float4 b)
{
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) k_fused(const Problem<float> P)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const long long t = *P.t_dev;
    const int N = P.N, R = P.R, cs = P.cs;
    const int n = mode_draw(P.seed, t, N);
    const long long In = P.dims[n];
    const int rows = P.rb;   // rows per cluster: kM tpc
    const int tpc = rows / kM;
    const int ntiles = (int)((In + rows - 1) / rows);
    const int tile = (int)blockIdx.x / cs;
    if (tile >= ntiles) return;   // the whole cluster: this mode has fewer row tiles
    const bool tr0 = blockIdx.x == 0;
    trace_stamp(P.trace, 0, tr0);
    const int rank = (int)cluster_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = tile * rows;
    const FusedSmem L(N, R, P.fb, cs, tpc);
    const int fpc = L.fpc, mr = L.mr, hr = L.hr;
    const int f0 = rank * fpc;
    const int nown = P.B - f0 < 0 ? 0 : (P.B - f0 < fpc ? P.B - f0 : fpc);
    const long long i_own = (long long)r0 + (long long)rank * mr;   // first owned row
    const int own_rows = In - i_own <= 0 ? 0 : (In - i_own < mr ? (int)(In - i_own) : mr);

    unsigned char *sA = smem + L.a;
    __nv_bfloat16 *sBhi = reinterpret_cast<__nv_bfloat16 *>(smem + L.bhi);
    __nv_bfloat16 *sBlo = reinterpret_cast<__nv_bfloat16 *>(smem + L.blo);
    __nv_bfloat16 *sZc = reinterpret_cast<__nv_bfloat16 *>(smem + L.zc);
    float *sM = reinterpret_cast<float *>(smem + L.a);
    float *sHp = reinterpret_cast<float *>(smem + L.hp);
    float *sHq = reinterpret_cast<float *>(smem + L.hq);
    float *sH = reinterpret_cast<float *>(smem + L.h);
    float *sArow = reinterpret_cast<float *>(smem + L.arow);
    double *sSrow = reinterpret_cast<double *>(smem + L.srow);
    float *sNew = reinterpret_cast<float *>(smem + L.snew);
    long long *jcol = reinterpret_cast<long long *>(smem + L.jcol);
    float *ss = reinterpret_cast<float *>(smem + L.s);
    int *sidx = reinterpret_cast<int *>(smem + L.idx);
    const uint32_t bar_mma = smem_u32(smem + L.bar);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + L.tmem);

    // 0. barrier and tensor memory
    if (threadIdx.x == 0) {
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_holder)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    // 1. own fibers: draws (CDFs staged in the X-tile region), columns, weights
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(sA);
    const long long cap = (long long)(L.abytes / 8);
    trace_stamp(P.trace, 15, tr0);
    draw_indices(P, t, n, f0, nown, sidx, stage, cap, reinterpret_cast<unsigned long long *>(sHp), tr0);
    __syncthreads();
    trace_stamp(P.trace, 1, tr0);
    const bool staged = cdfs_staged(P, n, cap);
    for (int f = threadIdx.x; f < fpc; f += kThreads) {
        long long j = 0;
        float w = 0.f;
        if (f < nown) {
            const int *row = sidx + f * N;
            long long Jp = 1;
            for (int k = 0; k < N; ++k) {
                if (k == n) continue;
                j += (long long)row[k] * Jp;
                Jp *= P.dims[k];
            }
            w = staged ? fiber_weight_staged(P, n, row, stage) : fiber_weight(P, n, row);
            if (tile == 0)
                for (int k = 0; k < N; ++k) P.idx[(long long)(f0 + f) * N + k] = row[k];
        }
        jcol[f] = j;
        ss[f] = w;
    }
    __syncthreads();   // the staged CDFs are dead: the region takes the X tile
    trace_stamp(P.trace, 2, tr0);

    // 2a. the fibers' entries of the cluster's rows -> X operands, one per MMA
    //     tile (MN-major: core matrix (f/8, i/8) at ((f/8) 16 + i/8) 128 bytes,
    //     fiber rows of 16 bytes; tile h at h fpc 256 bytes); in flight while
    //     the operands below are formed
    const uint32_t aBase = smem_u32(sA);
    {
        const __nv_bfloat16 *rep = reinterpret_cast<const __nv_bfloat16 *>(P.rep[n]);
        const long long ld = P.ld[n];
        const int groups = rows / 8;
        for (int c = threadIdx.x; c < fpc * groups; c += kThreads) {
            const int f = c / groups, ig = c % groups;
            const int h = ig / (kM / 8), igl = ig % (kM / 8);
            const long long i0 = r0 + ig * 8;
            const bool inb = f < nown && i0 < ld;
            const __nv_bfloat16 *src = inb ? rep + jcol[f] * ld + i0 : rep;
            cp_async16(aBase + (uint32_t)h * (uint32_t)fpc * 256u +
                           (uint32_t)((((f >> 3) * (kM / 8) + igl) << 7) + ((f & 7) << 4)),
                       src, inb ? 16u : 0u);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    {
        // the owned rows of A^(n) and their AdaGrad state, for the step
        const float *asrc = P.A[n] + i_own * R;
        for (int e = threadIdx.x; e < own_rows * R; e += kThreads) cp_async4(smem_u32(sArow + e), asrc + e);
        if (P.step == CPD_STEP_ADAGRAD) {
            const double *ssrc = P.S[n] + i_own * R;
            for (int e = threadIdx.x; e < own_rows * R; e += kThreads)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(sSrow + e)), "l"(ssrc + e)
                             : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    trace_stamp(P.trace, 16, tr0);

    // 2b. z_f (products of the factor rows, modes ascending) straight from the
    //     factors, and the operands: Z' hi / lo, z hi / lo (K-major, K = fibers).
    //     A thread takes up to kJobs (column r, block of 8 fibers) jobs at once
    //     and issues all their loads of one mode before multiplying, so the
    //     latency is paid once per mode.
    constexpr int kJobs = 4;
    const int njobs = kN * (fpc / 8);
    for (int j0 = 0; j0 < njobs; j0 += kJobs * kThreads) {
        float v[kJobs][8];
#pragma unroll
        for (int jj = 0; jj < kJobs; ++jj) {
            const int job = j0 + jj * kThreads + threadIdx.x;
            const int r = job % kN, b = job / kN;
#pragma unroll
            for (int u = 0; u < 8; ++u) v[jj][u] = (job < njobs && 8 * b + u < nown && r < R) ? 1.f : 0.f;
        }
        for (int k = 0; k < N; ++k) {
            if (k == n) continue;
            const float *Ak = P.A[k];
            float x[kJobs][8];
#pragma unroll
            for (int jj = 0; jj < kJobs; ++jj) {
                const int job = j0 + jj * kThreads + threadIdx.x;
                const int r = job % kN, b = job / kN;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int fl = 8 * b + u;
                    x[jj][u] = (job < njobs && fl < nown && r < R) ? __ldg(Ak + (long long)sidx[fl * N + k] * R + r)
                                                                    : 0.f;
                }
            }
#pragma unroll
            for (int jj = 0; jj < kJobs; ++jj)
#pragma unroll
                for (int u = 0; u < 8; ++u) v[jj][u] = v[jj][u] * x[jj][u];
        }
#pragma unroll
        for (int jj = 0; jj < kJobs; ++jj) {
            const int job = j0 + jj * kThreads + threadIdx.x;
            if (job >= njobs) continue;
            const int r = job % kN, b = job / kN;
            __nv_bfloat16 zh[8], zl[8], ph[8], pl[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float zs = v[jj][u] * ss[8 * b + u];
                zh[u] = __float2bfloat16_rn(v[jj][u]);
                zl[u] = __float2bfloat16_rn(v[jj][u] - __bfloat162float(zh[u]));
                ph[u] = __float2bfloat16_rn(zs);
                pl[u] = __float2bfloat16_rn(zs - __bfloat162float(ph[u]));
            }
            *reinterpret_cast<uint4 *>(sZc + kmaj(r, 8 * b, fpc)) = *reinterpret_cast<uint4 *>(zh);
            *reinterpret_cast<uint4 *>(sZc + kmaj(kN + r, 8 * b, fpc)) = *reinterpret_cast<uint4 *>(zl);
            *reinterpret_cast<uint4 *>(sBhi + kmaj(r, 8 * b, fpc)) = *reinterpret_cast<uint4 *>(ph);
            *reinterpret_cast<uint4 *>(sBlo + kmaj(r, 8 * b, fpc)) = *reinterpret_cast<uint4 *>(pl);
        }
    }
    trace_stamp(P.trace, 3, tr0);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    trace_stamp(P.trace, 4, tr0);

    // 2d. partials on the tensor cores: M_c (columns 0-63, and 192-255 for the
    //     second MMA tile), H_c as z hi/lo (rows 0-63 / 64-127) times Z' hi
    //     (columns 64-127) and Z' lo (columns 128-191)
    const uint32_t tmem = *tmem_holder;
    if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t bh = smem_u32(sBhi), bl = smem_u32(sBlo), zc = smem_u32(sZc);
        const uint32_t sbo = (uint32_t)(fpc >> 3) * 128u;
        const uint32_t id_m = idesc_bf16(kM, kN), id_h = idesc_kk(kM, kN);
        for (int ks = 0; ks < fpc / kK; ++ks) {
            const uint64_t dh = smem_desc(bh + ks * 256u, 128u, sbo);
            const uint64_t dl = smem_desc(bl + ks * 256u, 128u, sbo);
            const uint64_t dz = smem_desc(zc + ks * 256u, 128u, sbo);
            const uint32_t acc = ks > 0 ? 1u : 0u;
            for (int h = 0; h < tpc; ++h) {
                const uint64_t da = smem_desc(aBase + (uint32_t)h * (uint32_t)fpc * 256u + ks * 4096u, (kM / 8) * 128u, 128u);
                const uint32_t dm = tmem + (h ? 192u : 0u);
                mma_f16(dm, da, dh, id_m, acc);
                mma_f16(dm, da, dl, id_m, 1u);
            }
            mma_f16(tmem + 64u, dz, dh, id_h, acc);
            mma_f16(tmem + 128u, dz, dl, id_h, acc);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar_mma)
                     : "memory");
    }
    bool done = mbar_wait_bounded(bar_mma, 0);
    if (!done) {
        if (threadIdx.x == 0) atomicOr(P.status, kStTimeout);
        done = mbar_wait_bounded(bar_mma, 0);   // the products must finish before TMEM is freed
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    trace_stamp(P.trace, 5, tr0);

    // 2e. partials to shared memory (FP32, rows of kMs floats): M_c into the
    //     dead X tile; H_c = (z hi rows) + (z lo rows), each the sum of its
    //     Z' hi and Z' lo products
    {
        const int q = warp & 3, hh = warp >> 2;
        const int row = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        float v[32], w2[32];
        for (int h = 0; h < tpc; ++h) {
            tmem_ld32(lane_base + (h ? 192u : 0u) + (uint32_t)(32 * hh), v);
            if (!done) {
#pragma unroll
                for (int c = 0; c < 32; ++c) v[c] = 0.f;
            }
            float *mrow = sM + (h * kM + row) * kMs + 32 * hh;
#pragma unroll
            for (int c = 0; c < 32; c += 4)
                *reinterpret_cast<float4 *>(mrow + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
        }
        tmem_ld32(lane_base + 64u + (uint32_t)(32 * hh), v);
        tmem_ld32(lane_base + 128u + (uint32_t)(32 * hh), w2);
        float *dst = (q < 2 ? sHp : sHq) + (row & (kN - 1)) * kMs + 32 * hh;
#pragma unroll
        for (int c = 0; c < 32; c += 4)
            *reinterpret_cast<float4 *>(dst + c) =
                done ? make_float4(v[c] + w2[c], v[c + 1] + w2[c + 1], v[c + 2] + w2[c + 2], v[c + 3] + w2[c + 3])
                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols) : "memory");
    for (int e = threadIdx.x; e < kN * (kN / 4); e += kThreads) {
        const int r = e / (kN / 4), c = 4 * (e % (kN / 4));
        float4 *p = reinterpret_cast<float4 *>(sHp + r * kMs + c);
        *p = add4(*p, *reinterpret_cast<const float4 *>(sHq + r * kMs + c));
    }
    trace_stamp(P.trace, 6, tr0);
    cluster_arrive();
    cluster_wait();     // every CTA's partials are in its shared memory
    trace_stamp(P.trace, 7, tr0);

    // 3. owned rows of H: the partials of ranks 0, 1, ..., cs - 1 summed in
    //    that order (float4 columns up to R)
    const int c4 = (R + 3) / 4;
    const uint32_t m_l = smem_u32(sM), hp_l = smem_u32(sHp), h_l = smem_u32(sH);
    for (int e = threadIdx.x; e < hr * c4; e += kThreads) {
        const int rl = e / c4, col = 4 * (e % c4);
        const int row = hr * rank + rl;
        if (row >= R) continue;
        const uint32_t src = hp_l + (uint32_t)((row * kMs + col) * 4);
        float4 part[kMaxCs];
#pragma unroll
        for (int q = 0; q < kMaxCs; ++q)
            if (q < cs) part[q] = ld_cluster_v4(map_shared(src, (uint32_t)q));
        float4 acc = part[0];
#pragma unroll
        for (int q = 1; q < kMaxCs; ++q)
            if (q < cs) acc = add4(acc, part[q]);
        *reinterpret_cast<float4 *>(sH + row * kMs + col) = acc;
    }
    trace_stamp(P.trace, 8, tr0);
    cluster_arrive();
    cluster_wait();     // every owner's rows of H are summed
    trace_stamp(P.trace, 9, tr0);
    {
        // the other rows of H from their owners, up to 4 loads in flight a thread
        constexpr int kPer = (kN * (kN / 4) + kThreads - 1) / kThreads;
        float4 v[kPer];
        int dst[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int e = threadIdx.x + u * kThreads;
            const int row = e / c4, col = 4 * (e % c4);
            dst[u] = -1;
            if (e < R * c4 && row / hr != rank) {
                dst[u] = row * kMs + col;
                v[u] = ld_cluster_v4(map_shared(h_l + (uint32_t)(dst[u] * 4), (uint32_t)(row / hr)));
            }
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u)
            if (dst[u] >= 0) *reinterpret_cast<float4 *>(sH + dst[u]) = v[u];
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    trace_stamp(P.trace, 10, tr0);

    // 4. owned rows, four columns a thread: M summed over the ranks' partials
    //    in ascending rank (loads issued first), G = A^(n) H - M (k ascending),
    //    the step, the projection
    float *An = P.A[n];
    for (int e = threadIdx.x; e < own_rows * c4; e += kThreads) {
        const int rl = e / c4, r4 = 4 * (e % c4);
        const long long i = i_own + rl;
        const uint32_t msrc = m_l + (uint32_t)(((rank * mr + rl) * kMs + r4) * 4);
        float4 part[kMaxCs];
#pragma unroll
        for (int q = 0; q < kMaxCs; ++q)
            if (q < cs) part[q] = ld_cluster_v4(map_shared(msrc, (uint32_t)q));
        const float *arow = sArow + rl * R;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 5
        for (int k = 0; k < R; ++k) {
            const float a = arow[k];
            const float4 h = *reinterpret_cast<const float4 *>(sH + k * kMs + r4);
            acc[0] = __fmaf_rn(a, h.x, acc[0]);
            acc[1] = __fmaf_rn(a, h.y, acc[1]);
            acc[2] = __fmaf_rn(a, h.z, acc[2]);
            acc[3] = __fmaf_rn(a, h.w, acc[3]);
        }
        trace_stamp(P.trace, 18, tr0);
        float4 m = part[0];
#pragma unroll
        for (int q = 1; q < kMaxCs; ++q)
            if (q < cs) m = add4(m, part[q]);
        const float mv[4] = {m.x, m.y, m.z, m.w};
        trace_stamp(P.trace, 19, tr0);
        // the four columns' FP64 AdaGrad updates first, so that their latencies overlap
        float gv[4];
        double Sv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            gv[u] = acc[u] - mv[u];
            Sv[u] = (P.step == CPD_STEP_ADAGRAD && r4 + u < R)
                        ? __fma_rn((double)gv[u], (double)gv[u], sSrow[rl * R + r4 + u])
                        : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r4 + u;
            if (r < R) {
                const int eo = rl * R + r;
                const float g = gv[u];
                P.G[i * R + r] = g;
                float an;
                if (P.step == CPD_STEP_ADAGRAD) {
                    // S accumulates in FP64; the step factor eta / sqrt(b + S) is formed in FP32
                    P.S[n][i * R + r] = Sv[u];
                    an = arow[r] - (float)P.eta * g * rsqrtf((float)Sv[u] + (float)P.b);
                } else {
                    const float alpha =
                        (float)((P.step == CPD_STEP_DECAY) ? P.beta / ((double)t + P.gamma) : P.alpha);
                    an = arow[r] - alpha * g;
                }
                if (P.constraint == CPD_CONSTRAINT_NONNEG && an < 0.f) an = 0.f;   // projection; NaN kept
                if (!isfinite(an) || !isfinite(g)) atomicOr(P.status, kStNonFinite);
                An[i * R + r] = an;
                sNew[eo] = an;
            }
        }
    }
    cluster_arrive();   // no more reads of the other CTAs' shared memory; the barrier completes meanwhile
    __syncthreads();
    trace_stamp(P.trace, 17, tr0);
    // the rows' Euclidean weights, two rows a warp at once, each in the
    // canonical order (lane l: fma over r = l, l + 32, ... from +0, then the
    // shuffle-down tree adding lane l + off into lane l, off = 16 .. 1)
    if (P.sampling == CPD_SAMPLE_EUCLIDEAN)
        for (int rl = warp; rl < own_rows; rl += 2 * (kThreads / 32)) {
            const int rl2 = rl + kThreads / 32;
            const bool two = rl2 < own_rows;
            double w0 = 0.0, w1 = 0.0;
            for (int r = lane; r < R; r += 32) {
                const double a = (double)sNew[rl * R + r];
                w0 = __fma_rn(a, a, w0);
                const double b2 = two ? (double)sNew[rl2 * R + r] : 0.0;
                w1 = __fma_rn(b2, b2, w1);
            }
            for (int off = 16; off >= 1; off >>= 1) {
                w0 = __dadd_rn(w0, __shfl_down_sync(0xffffffffu, w0, off));
                w1 = __dadd_rn(w1, __shfl_down_sync(0xffffffffu, w1, off));
            }
            if (lane == 0) {
                P.w[n][i_own + rl] = w0;
                if (two) P.w[n][i_own + rl2] = w1;
            }
        }
    trace_stamp(P.trace, 11, tr0);

    // 5. the launch's last CTA: the distribution of mode n (unless deferred to
    //    the next draw) and the iteration's bookkeeping
    if (last_block(P.counters, (unsigned)(cs * ntiles))) {
        trace_stamp(P.trace, 12, true);
        if (P.sampling == CPD_SAMPLE_EUCLIDEAN && !P.defer_cdf) {
            // scratch: the partials' regions, dead since the second cluster barrier
            if (!block_distribution(P.w[n], In, P.cdf[n], reinterpret_cast<unsigned long long *>(sHp),
                                    reinterpret_cast<double *>(sA), (long long)(L.abytes / 8)) &&
                threadIdx.x == 0)
                atomicOr(P.status, kStDegenerate);
        }
        if (threadIdx.x == 0) {
            P.counters[0] = 0;
            if (P.sampling != CPD_SAMPLE_LEVERAGE) {
                if (P.sampling == CPD_SAMPLE_EUCLIDEAN && P.defer_cdf) *P.dirty = n;
                *P.n_last = n;
                *P.t_dev = t + 1;
            }
        }
        trace_stamp(P.trace, 13, true);
    }
    cluster_wait();     // no CTA of the cluster reads this one's shared memory any more
    trace_stamp(P.trace, 14, tr0);
}

size_t fused_smem_bytes(const Problem<float> &P) { return FusedSmem(P.N, P.R, P.fb, P.cs, P.rb / kM).total; }

long long fused_stage_cap(const Problem<float> &P)
{
    return (long long)(FusedSmem(P.N, P.R, P.fb, P.cs, P.rb / kM).abytes / 8);
}

// Cluster size and fibers per CTA for a batch of B: the smallest cluster
// (1 to 16 CTAs) that leaves at most 64 fibers to a CTA and fits its shared
// memory, else 16; `cs_req` > 0 forces the cluster size. Fibers per CTA: a
// multiple of 16 (the MMA K).
static int fused_fpc(int B, int cs)
{
    int f = (B + cs - 1) / cs;
    f = (f + kK - 1) / kK * kK;
    return f < kK ? kK : f;
}

void fused_plan(int N, int R, int B, int cs_req, int *cs, int *fpc)
{
    int c = cs_req;
    if (c <= 0) {
        c = 1;
        while (c < kMaxCs && ((B + c - 1) / c > 64 || FusedSmem(N, R, fused_fpc(B, c), c, 1).total > kFusedSmemMax))
            c <<= 1;
    }
    *cs = c;
    *fpc = fused_fpc(B, c);
}

bool fused_fits(int N, int R, int B, int cs_req, int tpc)
{
    int cs, fpc;
    fused_plan(N, R, B, cs_req, &cs, &fpc);
    if (cs < 1 || cs > kMaxCs || (cs & (cs - 1)) || R > kN || kM * tpc / cs < 1) return false;
    return FusedSmem(N, R, fpc, cs, tpc).total <= kFusedSmemMax;
}

static cudaError_t ensure_attrs(size_t need)
{
    static size_t attr_bytes = 0;
    static bool nonportable = false;
    if (!nonportable) {
        const cudaError_t e = cudaFuncSetAttribute(k_fused, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        nonportable = true;
    }
    if (need <= attr_bytes) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    attr_bytes = need;
    return cudaSuccess;
}

static cudaLaunchConfig_t fused_config(const Problem<float> &P, int grid, size_t need, cudaStream_t s,
                                       cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = need;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t launch_fused(const Problem<float> &P, int grid, cudaStream_t s)
{
    const size_t need = fused_smem_bytes(P);
    if (cudaError_t e = ensure_attrs(need); e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = fused_config(P, grid, need, s, attr);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_fused, P);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

int fused_max_clusters(const Problem<float> &P)
{
    const size_t need = fused_smem_bytes(P);
    if (need > kFusedSmemMax || ensure_attrs(need) != cudaSuccess) return 0;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = fused_config(P, P.cs, need, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_fused, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace cpd
