// SKRP-ST-I materialised (Alg. 3 followed by Alg. 1): for K mini-batches of
// mode n, the sampled multi-indices (Eq. (4)), the fiber probabilities
// p_f (Eq. (10)), the sampled Khatri-Rao rows Z_S (Eq. (3)) and the sampled
// fibers X_S (Eq. (2)), written to device memory. Batch b uses the random
// words of iteration t0 + b with the mode fixed to n, from the context's
// current per-factor distributions.
//
// This is the gather on its own, spread over every SM: each CTA takes blocks
// of up to 16 fibers; a warp per mode draws them (CDFs staged in shared
// memory), one thread per fiber forms the column and p_f, the CTA forms the
// KRP rows, and the fibers move global -> shared -> global by bulk copies
// (the tensor memory accelerator), double-buffered so a block's stores drain
// while the next block's fibers load.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "cpd_device.cuh"
#include "cpd_internal.h"
#include "cpd_tcgen05.cuh"

namespace cpd {

namespace {

constexpr int kSkFib = 16;               // fibers per block
constexpr long long kSkStageCap = 4096;  // staged CDF entries (modes != n)

struct SkrpArgs {
    int n, K;
    long long t0;
    int *idx;        // K B x N
    double *p;       // K B
    float *Z;        // K B x R
    void *X;         // K B x ld_n elements
    size_t stage_bytes;   // one fiber stage: kSkFib * ld_n * esize
    int esize;
};

__device__ __forceinline__ void bulk_s2g_grp(void *dst, uint32_t src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

}  // namespace

__global__ void __launch_bounds__(kThreads) k_skrp(const Problem<float> P, const SkrpArgs s)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int sidx[kSkFib * kMaxModes];
    __shared__ long long jcol[kSkFib];
    __shared__ __align__(8) unsigned long long bars[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = P.N, R = P.R, n = s.n;
    const long long B = P.B, total = (long long)s.K * B;
    const long long ld = P.ld[n];
    const uint32_t fbytes = (uint32_t)(ld * s.esize);
    // staged CDFs of the modes k != n (ascending), when they fit
    long long need = 0, off[kMaxModes];
    for (int k = 0; k < N; ++k) {
        off[k] = need;
        if (k != n) need += P.dims[k];
    }
    const bool staged = P.sampling != CPD_SAMPLE_UNIFORM && need <= kSkStageCap;
    unsigned long long *cdfs = reinterpret_cast<unsigned long long *>(smem);
    unsigned char *stage0 = smem + (staged ? (size_t)kSkStageCap * 8 : 0);
    if (staged)
        for (int k = 0; k < N; ++k)
            if (k != n)
                for (long long i = tid; i < P.dims[k]; i += blockDim.x) cdfs[off[k] + i] = __ldcg(P.cdf[k] + i);
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const char *rep = reinterpret_cast<const char *>(P.rep[n]);
    unsigned uses[2] = {0u, 0u};
    int local = 0;
    const long long nblk = (total + kSkFib - 1) / kSkFib;
    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x, ++local) {
        const long long fg0 = blk * kSkFib;
        const int nfib = (int)((total - fg0) < kSkFib ? total - fg0 : kSkFib);
        // draws: warp w takes modes w, w + 8, ...; lane = fiber of the block
        for (int k = warp; k < N; k += kThreads / 32) {
            const bool act = lane < nfib;
            const long long fg = fg0 + (act ? lane : 0);
            const long long b = fg / B, f = fg % B;
            if (k == n) {
                if (act) sidx[lane * N + k] = -1;
                continue;
            }
            const long long Ik = P.dims[k];
            const unsigned long long x = act ? fiber_word(P.seed, s.t0 + b, f, k) : 0ULL;
            long long i;
            if (P.sampling == CPD_SAMPLE_UNIFORM) {
                i = (long long)__umul64hi(x, (unsigned long long)Ik);
            } else if (staged) {
                const unsigned long long *c = cdfs + off[k];
                i = warp_search_staged(c, Ik, __umul64hi(x, c[Ik - 1]), act);
            } else {
                const unsigned long long *c = P.cdf[k];
                i = warp_search_cdf(c, Ik, __umul64hi(x, __ldg(c + (Ik - 1))), act);
            }
            if (act) sidx[lane * N + k] = (int)i;
        }
        __syncthreads();
        // column (Eq. (2)), p_f (Eq. (10), FP64), the multi-index
        if (tid < nfib) {
            const int *row = sidx + tid * N;
            long long j = 0, Jp = 1;
            for (int k = 0; k < N; ++k) {
                if (k == n) continue;
                j += (long long)row[k] * Jp;
                Jp *= P.dims[k];
            }
            jcol[tid] = j;
            const long long fg = fg0 + tid;
            if (s.p) s.p[fg] = fiber_prob(P, n, row);
            if (s.idx)
                for (int k = 0; k < N; ++k) s.idx[fg * N + k] = row[k];
        }
        // sampled KRP rows (Eq. (3)), factor rows ascending in k
        if (s.Z) {
            for (int e = tid; e < nfib * R; e += blockDim.x) {
                const int fl = e / R, r = e % R;
                float z = 1.f;
                for (int k = 0; k < N; ++k) {
                    if (k == n) continue;
                    z = z * P.A[k][(long long)sidx[fl * N + k] * R + r];
                }
                s.Z[(fg0 + fl) * R + r] = z;
            }
        }
        __syncthreads();
        // fibers: global -> shared (one bulk copy per fiber) -> global
        if (s.X && warp == 0) {
            const int st = local & 1;
            unsigned char *sb = stage0 + (size_t)st * s.stage_bytes;
            const uint32_t bar = smem_u32(&bars[st]);
            // this lane's store from this stage two blocks ago has read its slot
            asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
            if (lane == 0) mbar_expect_tx(bar, (uint32_t)nfib * fbytes);
            __syncwarp();
            if (lane < nfib)
                bulk_g2s(smem_u32(sb + (size_t)lane * fbytes), rep + jcol[lane] * ld * s.esize, fbytes, bar);
            bool ok = mbar_wait_bounded(bar, uses[st] & 1);
            ++uses[st];
            if (!ok) {
                if (lane == 0) atomicOr(P.status, kStTimeout);
            } else if (lane < nfib) {
                bulk_s2g_grp(static_cast<char *>(s.X) + (size_t)(fg0 + lane) * fbytes,
                             smem_u32(sb + (size_t)lane * fbytes), fbytes);
            }
        }
    }
    // every store has completed before the CTA's shared memory goes away
    if (warp == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

size_t skrp_smem_bytes(const Problem<float> &P, int n, int esize)
{
    long long need = 0;
    for (int k = 0; k < P.N; ++k)
        if (k != n) need += P.dims[k];
    const bool staged = P.sampling != CPD_SAMPLE_UNIFORM && need <= kSkStageCap;
    return (staged ? (size_t)kSkStageCap * 8 : 0) + 2 * (size_t)kSkFib * P.ld[n] * esize;
}

cudaError_t launch_skrp(const Problem<float> &P, int n, long long t0, int K, int *idx, double *p, float *Z, void *X,
                        int esize, int sm_count, cudaStream_t stream)
{
    SkrpArgs a{};
    a.n = n;
    a.K = K;
    a.t0 = t0;
    a.idx = idx;
    a.p = p;
    a.Z = Z;
    a.X = X;
    a.esize = esize;
    a.stage_bytes = (size_t)kSkFib * P.ld[n] * esize;
    const size_t smem = skrp_smem_bytes(P, n, esize);
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(k_skrp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        attr = smem;
    }
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_skrp, kThreads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long long nblk = ((long long)K * P.B + kSkFib - 1) / kSkFib;
    const int grid = (int)std::min<long long>(nblk, (long long)per_sm * sm_count);
    k_skrp<<<grid, kThreads, smem, stream>>>(P, a);
    return cudaGetLastError();
}

}  // namespace cpd
