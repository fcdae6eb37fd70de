// Tensor-core gradient engine with thread-block clusters (sm_103a).
//
// Same arithmetic as the per-CTA engine (Eq. (11) as G_g = A H_g - M_g
// per fiber group g, M_g = X_S,g Z'_S,g on tcgen05, Z' as a bf16 hi/lo pair),
// but one cluster of cs CTAs handles one fiber group: CTA `rank` owns the
// row tile [128 rank, 128 rank + 128) of A^(n) and a slice of fpc of the
// group's fb fibers. Everything the row tiles of a group share is computed
// once, in slices, and moved between the CTAs' shared memories by bulk async
// copies (cp.async.bulk shared::cta -> shared::cluster) that complete on the
// receiving CTA's mbarrier:
//   - each CTA draws its fibers (Alg. 3), forms their columns (Eq. (2)),
//     weights and sampled KRP rows (Alg. 1), and the B operands of its slice,
//     and sends the slice (B hi/lo, columns, weights) to every other CTA;
//   - each CTA forms H over its own fibers; CTA d owns rows [d hr, d hr + hr)
//     of H_g, receives those rows of every CTA's partial, sums them in
//     ascending rank and sends the finished rows to every other CTA.
// The A^(n) rows of the tile arrive by one global -> shared bulk copy. One
// cluster barrier after all receptions guarantees that no source buffer is
// reused while a copy could still read it.
//
// The tensor cores form G_g itself: the accumulator receives X (-Z') (the
// B operands are built negated) and then A H_g, with A^(n)'s rows (MN-major,
// like X) and H_g (K-major, like Z') split into bf16 hi/lo pairs
// (hi*hi + hi*lo + lo*hi); the epilogue only reads TMEM and stores.
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
    size_t a, bhi, blo, zo, zso, hp, hrecv, arow, h, hb, rows, jcol, s, idx, bar, tmem, total;
    int fpc, hr;
    __host__ __device__ TccSmem(int N, int R, int fb, int cs)
    {
        fpc = ((fb + cs - 1) / cs + 7) / 8 * 8;   // fiber slots per CTA, multiple of 8
        hr = (kN + cs - 1) / cs;                 // rows of H_g owned per CTA
        size_t o = 0;
        a = o;    o += (size_t)fb * kM * 2;                 // X tile (also CDF staging)
        bhi = o;  o += (size_t)fb * kN * 2;                 // Z' hi, K-major
        blo = o;  o += (size_t)fb * kN * 2;                 // Z' lo, K-major
        zo = o;   o += up((size_t)fpc * kN * 4);            // own z_f, [fiber][64]
        zso = o;  o += up((size_t)fpc * kN * 4);            // own s_f z_f
        hp = o;   o += (size_t)kN * kN * 4;                 // H over own fibers
        hrecv = o; o += up((size_t)cs * hr * kN * 4);       // owned rows of every CTA's partial
        if (o - a < (size_t)kM * R * 4) o = a + up((size_t)kM * R * 4);   // epilogue tile staging
        arow = o; o += up(aop_bytes(R));                    // A^(n) rows of the tile (bulk copy), then
                                                            // their bf16 hi/lo operands in place
        h = o;    o += (size_t)kN * kN * 4;                 // H_g
        hb = o;   o += (size_t)kN * kN * 2 * 2;             // H_g hi / lo (B operands of A H_g)
        rows = o; o += up((size_t)fpc * (N - 1) * R * 4);   // own fibers' factor rows
        jcol = o; o += up((size_t)fb * 8);
        s = o;    o += up((size_t)fb * 4);
        idx = o;  o += up((size_t)fpc * N * 4);
        bar = o;  o += 64;                                  // mbarriers: mma, a, x, hp, h
        tmem = o; o += 16;
        total = o;
    }
    __host__ __device__ static size_t up(size_t v) { return (v + 127) / 128 * 128; }
    __host__ __device__ static size_t aop_bytes(int R)
    {
        const size_t rows = (size_t)kM * R * 4 + 16, ops = (size_t)kM * kN * 2 * 2;
        return rows > ops ? rows : ops;
    }
};

// Fiber slots [c fpc, c fpc + nslot(c)) of CTA c (zero-padded past nf).
__device__ __forceinline__ int nslot(int c, int fpc, int fb)
{
    const int v = fb - c * fpc;
    return v < 0 ? 0 : (v < fpc ? v : fpc);
}

__device__ __forceinline__ int hrows(int d, int hr)
{
    const int v = kN - d * hr;
    return v < 0 ? 0 : (v < hr ? v : hr);
}

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
    const int nrows = has_rows ? ((In - r0) < kM ? (int)(In - r0) : kM) : 0;
    const int f0 = gf * fb;
    const int nf = (P.B - f0) < fb ? (P.B - f0) : fb;

    const TccSmem L(N, R, fb, cs);
    unsigned char *sA = smem + L.a;
    __nv_bfloat16 *sBhi = reinterpret_cast<__nv_bfloat16 *>(smem + L.bhi);
    __nv_bfloat16 *sBlo = reinterpret_cast<__nv_bfloat16 *>(smem + L.blo);
    float *sArow = reinterpret_cast<float *>(smem + L.arow);
    float *sH = reinterpret_cast<float *>(smem + L.h);
    float *sHp = reinterpret_cast<float *>(smem + L.hp);
    float *sHr = reinterpret_cast<float *>(smem + L.hrecv);
    float *sRows = reinterpret_cast<float *>(smem + L.rows);
    float *sZo = reinterpret_cast<float *>(smem + L.zo);
    float *sZso = reinterpret_cast<float *>(smem + L.zso);
    long long *jcol = reinterpret_cast<long long *>(smem + L.jcol);
    float *ss = reinterpret_cast<float *>(smem + L.s);
    int *sidx = reinterpret_cast<int *>(smem + L.idx);
    const uint32_t bar_mma = smem_u32(smem + L.bar), bar_a = bar_mma + 8, bar_x = bar_mma + 16,
                   bar_hp = bar_mma + 24, bar_h = bar_mma + 32;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + L.tmem);
    const int fpc = L.fpc, hr = L.hr;
    const int fo0 = rank * fpc;
    const int myslots = nslot(rank, fpc, fb);
    const int nown = nf - fo0 < 0 ? 0 : (nf - fo0 < fpc ? nf - fo0 : fpc);
    const int nb8 = myslots / 8;

    // 0. mbarriers with the byte counts this CTA will receive; A^(n) rows by
    //    one bulk copy; TMEM; early cluster arrival
    if (threadIdx.x == 0) {
        for (int q = 0; q < 5; ++q) mbar_init(bar_mma + 8 * q, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        uint32_t bx = 0, bh = 0;
        for (int c = 0; c < cs; ++c) {
            if (c == rank) continue;
            bx += 2u * 8u * (uint32_t)(nslot(c, fpc, fb) / 8) * 128u + (uint32_t)nslot(c, fpc, fb) * 12u;
            bh += (uint32_t)hrows(c, hr) * kN * 4u;
        }
        mbar_expect_tx(bar_x, bx);
        mbar_expect_tx(bar_hp, (uint32_t)(cs - 1) * (uint32_t)hrows(rank, hr) * kN * 4u);
        mbar_expect_tx(bar_h, bh);
        if (has_rows) {
            const uint32_t bytes = (uint32_t)((nrows * R * 4 + 15) / 16 * 16);
            mbar_expect_tx(bar_a, bytes);
            bulk_g2s(smem_u32(sArow), P.A[n] + (long long)r0 * R, bytes, bar_a);
        } else {
            mbar_expect_tx(bar_a, 0);
        }
    }
    if (has_rows && warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_holder)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    cluster_arrive();   // released once every CTA's mbarriers are initialised
    trace_stamp(P.trace, 1, tr0);

    // 1. own fibers: draws (CDFs staged in the X-tile region), columns, weights
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(sA);
    const long long cap = (long long)(fb * kM * 2) / 8;
    // the grid's last CTA (the one with the fewest own fibers; no CTA of this
    // kernel returns early) writes the rebuilt CDF back
    draw_indices(P, t, n, f0 + fo0, nown, sidx, stage, cap, reinterpret_cast<unsigned long long *>(sZo),
                 blockIdx.x == gridDim.x - 1);
    __syncthreads();
    trace_stamp(P.trace, 2, tr0);
    const bool staged = cdfs_staged(P, n, cap);
    if (threadIdx.x < myslots) {
        const int f = threadIdx.x;
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
            trace_stamp(P.trace, 31, tr0 && f == 0);
            for (int k = 0; k < N; ++k) P.idx[(long long)(f0 + fo0 + f) * N + k] = row[k];
        }
        jcol[fo0 + f] = j;
        ss[fo0 + f] = w;
    }
    trace_stamp(P.trace, 26, tr0);
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
    trace_stamp(P.trace, 27, tr0);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    trace_stamp(P.trace, 28, tr0);
    __syncthreads();
    trace_stamp(P.trace, 10, tr0);

    // 2. z_f, s_f z_f (own, local) and the own slice of the B operands
    for (int job = threadIdx.x; job < kN * nb8; job += blockDim.x) {
        const int r = job % kN, b = job / kN;
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
            const float zs = v * ss[fo0 + fl];
            sZo[fl * kN + r] = v;
            sZso[fl * kN + r] = zs;
            hi[u] = __float2bfloat16_rn(-zs);           // -Z': the accumulator gets -M_g
            lo[u] = __float2bfloat16_rn(-zs - __bfloat162float(hi[u]));
        }
        // K-major, fiber-block-major: core matrix (r/8, f/8) at ((f/8)*8 + r/8)*128 B,
        // so every CTA's slice of fibers is one contiguous range
        const int f = fo0 + 8 * b;
        const int off = (((f >> 3) * (kN >> 3) + (r >> 3)) << 6) + ((r & 7) << 3);
        *reinterpret_cast<uint4 *>(sBhi + off) = *reinterpret_cast<uint4 *>(hi);
        *reinterpret_cast<uint4 *>(sBlo + off) = *reinterpret_cast<uint4 *>(lo);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    trace_stamp(P.trace, 11, tr0);
    cluster_wait();     // every CTA's mbarriers exist: sends may start
    trace_stamp(P.trace, 22, tr0);
    if (warp == 0 && cs > 1) {
        // own slice -> every other CTA: B hi, B lo (one contiguous range each),
        // columns, weights
        const uint32_t bhi_l = smem_u32(sBhi), blo_l = smem_u32(sBlo);
        const uint32_t j_l = smem_u32(jcol), s_l = smem_u32(ss);
        const int per = 4;
        for (int task = lane; task < (cs - 1) * per; task += 32) {
            const int di = task / per, q = task % per;
            const int d = di + (di >= rank ? 1 : 0);
            const uint32_t mb = map_shared(bar_x, d);
            if (nb8 == 0) continue;
            if (q < 2) {
                const uint32_t base = q == 0 ? bhi_l : blo_l;
                const uint32_t off = (uint32_t)(fo0 >> 3) * (uint32_t)(kN >> 3) * 128u;
                bulk_s2s(map_shared(base + off, d), base + off, (uint32_t)nb8 * (uint32_t)(kN >> 3) * 128u, mb);
            } else if (q == 2) {
                bulk_s2s(map_shared(j_l + fo0 * 8, d), j_l + fo0 * 8, (uint32_t)myslots * 8u, mb);
            } else {
                bulk_s2s(map_shared(s_l + fo0 * 4, d), s_l + fo0 * 4, (uint32_t)myslots * 4u, mb);
            }
        }
    }
    trace_stamp(P.trace, 23, tr0);
    // H over the own fibers (all 64 x 64): a 4 x 4 block per thread; own slots
    // past nown are zero (z_f = 0), so whole groups of 8 are summed
    {
        const int rb = threadIdx.x >> 4, cb = threadIdx.x & 15;
        float acc[4][4] = {};
#pragma unroll 4
        for (int fl = 0; fl < 8 * nb8; ++fl) {
            const float4 a = *reinterpret_cast<const float4 *>(sZso + fl * kN + 4 * rb);
            const float4 b = *reinterpret_cast<const float4 *>(sZo + fl * kN + 4 * cb);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            *reinterpret_cast<float4 *>(sHp + (4 * rb + u) * kN + 4 * cb) =
                make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
    }
    trace_stamp(P.trace, 24, tr0);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    trace_stamp(P.trace, 25, tr0);
    if (warp == 1 && cs > 1) {
        // rows [d hr, d hr + hrows(d)) of the partial -> owner d, slot `rank`
        const uint32_t hp_l = smem_u32(sHp), hr_l = smem_u32(sHr);
        for (int di = lane; di < cs - 1; di += 32) {
            const int d = di + (di >= rank ? 1 : 0);
            const int nr = hrows(d, hr);
            if (nr == 0) continue;
            bulk_s2s(map_shared(hr_l + (uint32_t)(rank * hr * kN * 4), d), hp_l + (uint32_t)(d * hr * kN * 4),
                     (uint32_t)nr * kN * 4u, map_shared(bar_hp, d));
        }
    }
    trace_stamp(P.trace, 3, tr0);

    // 3. fibers' columns and operands of the whole group have arrived: gather
    bool ok = mbar_wait_bounded(bar_x, 0);
    trace_stamp(P.trace, 4, tr0);
    const uint32_t aBase = smem_u32(sA);
    if (has_rows) {
        const __nv_bfloat16 *rep = reinterpret_cast<const __nv_bfloat16 *>(P.rep[n]);
        const long long ld = P.ld[n];
        for (int c = threadIdx.x; c < fb * (kM / 8); c += blockDim.x) {
            const int f = c / (kM / 8), ig = c % (kM / 8);
            const long long i0 = r0 + ig * 8;
            const bool inb = f < nf && i0 < ld;
            const __nv_bfloat16 *src = inb ? rep + jcol[f] * ld + i0 : rep;
            cp_async16(aBase + (uint32_t)((((f >> 3) * (kM / 8) + ig) << 7) + ((f & 7) << 4)), src,
                       inb ? 16u : 0u);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    // A^(n) rows of the tile -> bf16 hi/lo, MN-major like X (K = R padded to
    // kN), in place through registers: operands of the A H_g products
    ok = mbar_wait_bounded(bar_a, 0) && ok;
    __nv_bfloat16 *aHi = reinterpret_cast<__nv_bfloat16 *>(sArow);
    __nv_bfloat16 *aLo = aHi + kM * kN;
    if (has_rows) {
        constexpr int kJobs = kN * (kM / 8) / kThreads;   // 4
        float av[kJobs][8];
#pragma unroll
        for (int jj = 0; jj < kJobs; ++jj) {
            const int job = threadIdx.x + jj * kThreads;
            const int r = job % kN, ig = job / kN;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = 8 * ig + u;
                av[jj][u] = (ok && i < nrows && r < R) ? sArow[i * R + r] : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < kJobs; ++jj) {
            const int job = threadIdx.x + jj * kThreads;
            const int r = job % kN, ig = job / kN;
            __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                hi[u] = __float2bfloat16_rn(av[jj][u]);
                lo[u] = __float2bfloat16_rn(av[jj][u] - __bfloat162float(hi[u]));
            }
            const int off = (((r >> 3) * (kM >> 3) + ig) << 6) + ((r & 7) << 3);
            *reinterpret_cast<uint4 *>(aHi + off) = *reinterpret_cast<uint4 *>(hi);
            *reinterpret_cast<uint4 *>(aLo + off) = *reinterpret_cast<uint4 *>(lo);
        }
    }
    // owned rows of H_g: partials of every CTA summed in ascending rank
    ok = mbar_wait_bounded(bar_hp, 0) && ok;
    {
        const int nr = hrows(rank, hr);
        for (int e = threadIdx.x; e < nr * kN; e += blockDim.x) {
            const int rl = e / kN, c = e % kN, r = rank * hr + rl;
            float acc = 0.f;
            for (int q = 0; q < cs; ++q)
                acc += (q == rank) ? sHp[r * kN + c] : sHr[(q * hr + rl) * kN + c];
            sH[r * kN + c] = acc;
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (warp == 0 && cs > 1 && nr > 0) {
            const uint32_t h_l = smem_u32(sH) + (uint32_t)(rank * hr * kN * 4);
            for (int di = lane; di < cs - 1; di += 32) {
                const int d = di + (di >= rank ? 1 : 0);
                bulk_s2s(map_shared(h_l, d), h_l, (uint32_t)nr * kN * 4u, map_shared(bar_h, d));
            }
        }
    }
    trace_stamp(P.trace, 5, tr0);
    uint32_t tmem = 0;
    __shared__ int s_issued;
    if (threadIdx.x == 0) s_issued = 0;
    if (has_rows) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        tmem = *tmem_holder;
        if (threadIdx.x == 0 && ok) {
            s_issued = 1;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t bhi = smem_u32(sBhi), blo = smem_u32(sBlo);
            const uint32_t idesc = idesc_bf16(kM, kN);
            const uint32_t kstepB = 2u * (uint32_t)(kN >> 3) * 128u;   // 16 fibers = 2 core matrices along K
            for (int ks = 0; ks < fb / kK; ++ks) {
                const uint64_t da = smem_desc(aBase + ks * 4096u, (kM / 8) * 128u, 128u);
                const uint64_t dh = smem_desc(bhi + ks * kstepB, (uint32_t)(kN >> 3) * 128u, 128u);
                const uint64_t dl = smem_desc(blo + ks * kstepB, (uint32_t)(kN >> 3) * 128u, 128u);
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
    }
    ok = mbar_wait_bounded(bar_h, 0) && ok;
    if (!ok && threadIdx.x == 0) atomicOr(P.status, kStTimeout);
    cluster_arrive();   // this CTA has received everything; the barrier completes meanwhile
    trace_stamp(P.trace, 14, tr0);

    // 4. + A H_g on the tensor cores: H_g -> hi/lo, K-major like Z', in its own
    //    buffer; K = R padded to 16.
    __nv_bfloat16 *hHi = reinterpret_cast<__nv_bfloat16 *>(smem + L.hb);
    __nv_bfloat16 *hLo = hHi + kN * kN;
    if (has_rows) {
        for (int job = threadIdx.x; job < kN * (kN / 8); job += blockDim.x) {
            const int c = job % kN, rg = job / kN;  // column c of H, rows 8 rg .. 8 rg + 7 (the K index)
            __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float h = sH[(8 * rg + u) * kN + c];
                hi[u] = __float2bfloat16_rn(h);
                lo[u] = __float2bfloat16_rn(h - __bfloat162float(hi[u]));
            }
            const int off = (((c >> 3) * (kN >> 3) + rg) << 6) + ((c & 7) << 3);
            *reinterpret_cast<uint4 *>(hHi + off) = *reinterpret_cast<uint4 *>(hi);
            *reinterpret_cast<uint4 *>(hLo + off) = *reinterpret_cast<uint4 *>(lo);
        }
    }
    cluster_wait();     // no copy reads our buffers any more
    trace_stamp(P.trace, 15, tr0);
    if (has_rows) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0 && s_issued) {
            if (ok) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t idesc = idesc_bf16(kM, kN);
                const uint32_t ah = smem_u32(aHi), al = smem_u32(aLo), bh = smem_u32(hHi), bl = smem_u32(hLo);
                for (int ks = 0; ks < (R + kK - 1) / kK; ++ks) {
                    const uint64_t dah = smem_desc(ah + ks * 4096u, (kM / 8) * 128u, 128u);
                    const uint64_t dal = smem_desc(al + ks * 4096u, (kM / 8) * 128u, 128u);
                    const uint64_t dbh = smem_desc(bh + ks * 256u, 128u, (kN / 8) * 128u);
                    const uint64_t dbl = smem_desc(bl + ks * 256u, 128u, (kN / 8) * 128u);
                    const uint64_t pa[3] = {dah, dah, dal}, pb[3] = {dbh, dbl, dbh};
#pragma unroll
                    for (int u = 0; u < 3; ++u)
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                            "l"(pa[u]), "l"(pb[u]), "r"(idesc), "r"(1u)
                            : "memory");
                }
            }
            // completes when every product issued above (the M products included) has
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             bar_mma)
                         : "memory");
        }
    }
    trace_stamp(P.trace, 6, tr0);

    // 5. G_g = A H_g - M_g from TMEM for this tile's rows
    if (has_rows) {
        bool done = s_issued && mbar_wait_bounded(bar_mma, 0);
        if (!done && s_issued) {
            if (threadIdx.x == 0) atomicOr(P.status, kStTimeout);
            done = mbar_wait_bounded(bar_mma, 0);
        }
        done = done && ok;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        trace_stamp(P.trace, 7, tr0);
        float *tile = reinterpret_cast<float *>(sA);
        const int q = warp & 3, hh = warp >> 2;
        const int il = 32 * q + lane;
        if (done) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * hh), v);
            // the staging region holds only dead operands (the MMAs are complete)
#pragma unroll
            for (int c = 0; c < 32; ++c)
                if (32 * hh + c < R) tile[il * R + 32 * hh + c] = v[c];
        }
        __syncthreads();
        if (done) {
            float *out = P.part + ((long long)gf * In + r0) * R;
            for (int e = threadIdx.x; e < nrows * R; e += blockDim.x) out[e] = tile[e];
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

long long tcc_stage_cap(const Problem<float> &P) { return (long long)P.fb * kM * 2 / 8; }

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
