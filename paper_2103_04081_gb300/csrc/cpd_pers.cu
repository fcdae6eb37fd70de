// Persistent cluster engine (sm_103a): one thread-block cluster runs T
// consecutive iterations of Alg. 4 / Alg. 5 for one decomposition inside a
// single launch, with no grid-wide synchronisation and no launch between
// iterations.
//
// Work split inside the cluster (cs CTAs, CTA `rank`):
//   * fibers: CTA rank owns fibers [rank fpc, rank fpc + fpc) of every batch.
//     It draws them (Alg. 3), forms their columns (Eq. (2)), weights
//     s_f = 1/(B J_n p_f) and sampled KRP rows z_f (Eq. (3)), gathers the
//     whole fibers from the mode-n replica and contracts them on the tensor
//     cores against Z' = s_f z_f (bf16 hi/lo pair, K-major) into a partial
//     M_rank = X_S,rank Z'_S,rank held in tensor memory for every row of
//     A^(n) (one 128-row accumulator tile per 128 rows). The CUDA cores form
//     the partial H_rank = sum_f s_f z_f z_f^T meanwhile.
//   * rows: CTA rank owns a contiguous range of rows of A^(n) (whole groups
//     of 32). The partials of every CTA go to an L2-resident scratch; the
//     owner sums its rows in ascending CTA order, forms G = A H - M
//     (Eq. (11)) and the step (Eq. (12), Thm 9 or Eq. (13a)-(13b)), writes
//     the rows back and sends their new Euclidean weights (Def. 5) to every
//     CTA of the cluster through distributed shared memory.
//   * every CTA keeps the fixed-point CDFs of all modes in shared memory and
//     rebuilds mode n's in place from the gathered weights (the same exact
//     integer CDF as the other engines), so the next iteration draws from
//     the updated factor (Alg. 4 / Alg. 5 take p_k from the current factors).
// Three cluster barriers per iteration order the phases: partials written,
// H rows sent, weights sent. The gather of a CTA streams its fibers in
// chunks of 16 (the MMA K) through a ring of stages filled by 16-byte
// cp.async copies; a chunk's tensor-core products are issued by one thread
// and complete on the stage's mbarrier, which releases the stage.
//
// The factors are mirrored, for the launch, in private copies whose rows
// are padded to a multiple of 4 floats (16-byte aligned rows for the async
// copies); the context's factors are read at the start and written at the
// end, together with the CDFs, t and the last batch.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cpd_device.cuh"
#include "cpd_internal.h"
#include "cpd_tcgen05.cuh"

namespace cpd {

namespace {

constexpr int kPM = 128;          // rows per accumulator tile (MMA M)
constexpr int kPK = 16;           // fibers per chunk (MMA K for 16-bit operands)
constexpr int kPLand = 3;         // landing stages: whole fibers by bulk copies
constexpr int kPOp = 2;           // operand buffers in the MMA layout
constexpr int kPTW = 6;           // transform warps (warps 2..7)
constexpr int kPTT = kPTW * 32;   // transform threads
constexpr int kPHd = 64;          // H is formed 64 x 64 (4 x 4 blocks, upper triangle)
constexpr int kPOwnBlock = 64;    // owned rows handled per pass of the step phase
constexpr long long kPMaxStage = 4096;   // CDF staging entries (sum of all I_k)
constexpr int kPMaxFpc = 1024;    // fibers per CTA
// dynamic shared memory per CTA: the 227 KB a CTA may opt into, less the
// kernel's static copy of its launch arguments and flags
constexpr size_t kPSmemMax = (227 * 1024 - sizeof(PersArgs) - 256) / 1024 * 1024;

__host__ __device__ inline size_t up128(size_t v) { return (v + 127) / 128 * 128; }

// Shared-memory carve-up (byte offsets). The landing stages and operand
// buffers form one region that the phases after the contraction reuse: the
// staging of the partial tiles, then H, the owned rows (A, S, M, new rows),
// the staging of the partial blocks being summed, and the scratch of the
// CDF rebuild.
struct PersLayout {
    size_t cdf, idx, jcol, sw, land, land_bytes, lx, lfr, pitch, op, op_bytes, ox, obh, obl, zf, bar, total;
    size_t region, region_bytes;
    size_t h, own_a, own_m, own_s, own_n, own_g, dsm, red;   // inside the region (step phase)
    int nland;                                        // landing stages (3, or 2 when memory is short)
    int red_slots;                                    // partial blocks staged at once
    __host__ __device__ PersLayout(const PersArgs &a)
    {
        const int N = a.P.N;
        size_t o = 0;
        cdf = o;  o += up128((size_t)a.sumI * 8);
        idx = o;  o += up128((size_t)a.fpc * N * 4);
        jcol = o; o += up128((size_t)a.fpc * 8);
        sw = o;   o += up128((size_t)a.fpc * 4);
        region = o;
        const size_t fixed = o + 2 * (size_t)kPK * kPHd * 4 + 8 * 16;   // + zf, barriers
        // landing pitch of one fiber: 16-byte multiple with pitch / 16 odd, so
        // the 16-byte pieces of 8 consecutive fibers fall in distinct banks
        long long ldmax = 0;
        for (int k = 0; k < N; ++k) ldmax = a.P.ld[k] > ldmax ? a.P.ld[k] : ldmax;
        pitch = (size_t)ldmax * 2;
        if (((pitch / 16) & 1) == 0) pitch += 16;
        lx = 0;
        lfr = up128((size_t)kPK * pitch);
        land_bytes = up128(lfr + (size_t)kPK * (N - 1) * a.R4 * 4);
        ox = 0;
        obh = up128((size_t)kPK * a.ntile * kPM * 2);
        obl = obh + (size_t)kPK * a.Npad * 2;
        op_bytes = up128(obl + (size_t)kPK * a.Npad * 2);
        // step phase inside the region: H, owned rows (A, M, new, S), the
        // CDF-rebuild scratch, then the staged partial blocks
        const size_t blk = (size_t)kPOwnBlock * a.R4 * 4;
        h = 0;
        own_a = h + (size_t)kPHd * kPHd * 4;
        own_m = own_a + up128(blk);
        own_n = own_m + up128(blk);
        own_s = own_n + up128(blk);
        own_g = own_s + up128((size_t)kPOwnBlock * a.P.R * 8 + 16);
        dsm = own_g + up128(blk);
        red = dsm + 2 * kThreads * 8;
        const size_t tiles = 4 * up128((size_t)kPM * a.R4 * 4);   // staged partial tiles
        nland = kPLand;
        size_t base = land_bytes * nland + op_bytes * kPOp;
        if (fixed + (base > red + blk ? base : red + blk) > kPSmemMax) {
            nland = 2;
            base = land_bytes * nland + op_bytes * kPOp;
        }
        const size_t room = kPSmemMax > fixed + red ? kPSmemMax - fixed - red : 0;
        red_slots = (int)(room / blk);
        if (red_slots > a.cs) red_slots = a.cs;
        if (red_slots < 1) red_slots = 1;
        region_bytes = base;
        if (region_bytes < red + blk * red_slots) region_bytes = red + blk * red_slots;
        if (region_bytes < tiles) region_bytes = tiles;
        land = region;
        op = land + land_bytes * nland;
        o += region_bytes;
        zf = o;   o += 2 * (size_t)kPK * kPHd * 4;
        bar = o;  o += 8 * 16;
        total = o;
        // at least half of the SM's shared memory, so one CTA per SM (the
        // tensor-memory allocation assumes it)
        if (total < 120 * 1024) total = 120 * 1024;
    }
};

// Phase timestamp (%globaltimer, ns) from the calling thread, when tracing is on.
__device__ __forceinline__ void stamp_here(unsigned long long *trace, int slot, bool cond)
{
    if (trace && cond) {
        unsigned long long ns;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
        trace[slot] = ns;
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t cluster_nctas()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all()
{
    cluster_arrive();
    cluster_wait();
}

__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;\n" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

// Bulk store shared -> global (async proxy), tracked by a bulk group.
__device__ __forceinline__ void bulk_s2g(void *dst, uint32_t src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// Named barrier of the transform warps.
__device__ __forceinline__ void transform_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(kPTT) : "memory"); }

// One MMA: D(tmem) (+)= A(desc) B(desc), kind::f16 (bf16 in, f32 accumulate).
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

// Wait for the phase of parity `par` unless the CTA gave up already.
__device__ __forceinline__ void wait_or_abort(uint32_t mbar, uint32_t par, volatile int *abort)
{
    if (*abort) return;
    if (!mbar_wait_bounded(mbar, par)) *abort = 1;
}

// s_f = (1/(B J_n)) prod_{k != n, ascending} Q_k / q_k(i_k) in FP32 (the same
// arithmetic as the other engines' fiber_weight), from the staged CDFs.
__device__ __forceinline__ float pers_weight(const PersArgs &a, int n, const int *row,
                                             const unsigned long long *stage)
{
    const Problem<float> &P = a.P;
    float s = P.inv_bj[n];
    for (int k = 0; k < P.N; ++k) {
        if (k == n) continue;
        if (P.sampling == CPD_SAMPLE_UNIFORM) {
            s *= (float)P.dims[k];
        } else {
            const unsigned long long *c = stage + a.off[k];
            const unsigned long long q = c[row[k]] - (row[k] > 0 ? c[row[k] - 1] : 0ULL);
            s *= __ull2float_rn(c[P.dims[k] - 1]) / __ull2float_rn(q);
        }
    }
    return s;
}

// Euclidean weights of up to 8 rows at once by one warp, each in the canonical
// order of warp_row_weight (lane l sums a_r^2 over r = l, l + 32, ... with fma
// from +0; then the shuffle-down tree 16, 8, 4, 2, 1): the 8 rows' chains are
// independent, so the FP64 latencies overlap. Row u is rows + u * stride;
// the weights land in lane 0 of w[u].
__device__ __forceinline__ void warp_row_weights8(const float *rows, int stride, int nrows, int R, double (&w)[8])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int u = 0; u < 8; ++u) w[u] = 0.0;
    for (int r = lane; r < R; r += 32) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (u < nrows) {
                const double v = (double)rows[u * stride + r];
                w[u] = __fma_rn(v, v, w[u]);
            }
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
        for (int u = 0; u < 8; ++u) w[u] = __dadd_rn(w[u], __shfl_down_sync(0xffffffffu, w[u], off));
}

}  // namespace

// Training: one cluster per problem; `one` is used when `many` is null
// (single decomposition), otherwise cluster g runs many[g] for T iterations.
// Gradient mode (md.gmode = n >= 0, `one` only): cluster c forms the mode-n
// mini-batch gradients of batches c, c + #clusters, ... < md.K at the current
// factors (batch b drawn as iteration md.t0 + b would draw it, with the mode
// fixed to n) into md.gout[b] (I_n x R); nothing in the context changes.
//
// Warp roles in the contraction phase: warp 0 lane 0 issues the bulk copies
// of whole fibers (and their factor rows) into the landing stages; warp 1
// lane 0 issues the tensor-core products; warps 2..7 move each landed chunk
// into the MMA operand layout, build its B operands and accumulate H.
__global__ void __launch_bounds__(kThreads, 1) k_pers(const PersArgs one, const PersArgs *__restrict__ many,
                                                      long long T, const PersMode md)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(16) PersArgs sa;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort, s_flags;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cs = (int)cluster_nctas();
    const int rank = (int)cluster_rank();
    const int g = blockIdx.x / cs;
    const bool train = md.gmode < 0;
    const int ncl = gridDim.x / cs;
    {
        static_assert(sizeof(PersArgs) % 8 == 0, "PersArgs is copied in 8-byte words");
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(many ? many + g : &one);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&sa);
        for (int q = tid; q < (int)(sizeof(PersArgs) / 8); q += blockDim.x) dst[q] = src[q];
    }
    if (tid == 0) {
        s_abort = 0;
        s_flags = 0;
    }
    __syncthreads();
    volatile int *abort = &s_abort;
    const PersArgs &a = sa;
    const Problem<float> &P = a.P;
    const int N = P.N, R = P.R, R4 = a.R4, Npad = a.Npad, cst = a.cst, fpc = a.fpc;
    const PersLayout L(a);
    const int rows_all = a.ntile * kPM;     // row extent of a partial slab
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(smem + L.cdf);
    int *sidx = reinterpret_cast<int *>(smem + L.idx);
    long long *jcol = reinterpret_cast<long long *>(smem + L.jcol);
    float *sw = reinterpret_cast<float *>(smem + L.sw);
    unsigned char *region = smem + L.region;
    float *zf = reinterpret_cast<float *>(smem + L.zf);
    float *sH = reinterpret_cast<float *>(region + L.h);
    unsigned long long *dsm = reinterpret_cast<unsigned long long *>(region + L.dsm);
    // mbarriers: land_full[3], land_empty[3], op_full[2], op_empty[2], mma done, step
    const uint32_t bar0 = smem_u32(smem + L.bar);
    const uint32_t b_lfull = bar0, b_lempty = bar0 + 8 * kPLand, b_ofull = bar0 + 16 * kPLand;
    const uint32_t b_oempty = b_ofull + 8 * kPOp, b_mma = b_oempty + 8 * kPOp, b_step = b_mma + 8;
    const bool tr = (g == 0 && rank == 0);
    // scratch of this cluster (gradient mode: one slab set per cluster);
    // CTA c's partial M is slab c (rows_all * cst floats), row-major with
    // row stride R4
    float *const part = a.part + (train ? 0 : (size_t)g * cs * rows_all * cst);
    float *const hpart = a.hpart + (train ? 0 : (size_t)g * cs * kPHd * kPHd);

    // ---- set-up -------------------------------------------------------------
    int tcols = 32;
    while (tcols < a.ntile * cst) tcols <<= 1;
    if (tid == 0) {
        for (int q = 0; q < kPLand; ++q) {
            mbar_init(b_lfull + 8 * q, 1);
            mbar_init(b_lempty + 8 * q, 1);
        }
        for (int q = 0; q < kPOp; ++q) {
            mbar_init(b_ofull + 8 * q, 1);
            mbar_init(b_oempty + 8 * q, 1);
        }
        mbar_init(b_mma, 1);
        mbar_init(b_step, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    // CDFs of every mode (current at launch start: this engine never defers)
    if (P.sampling != CPD_SAMPLE_UNIFORM)
        for (int k = 0; k < N; ++k)
            for (long long i = tid; i < P.dims[k]; i += blockDim.x) stage[a.off[k] + i] = __ldcg(P.cdf[k] + i);
    for (int e = tid; e < 2 * kPK * kPHd; e += blockDim.x) zf[e] = 0.f;
    // factors -> padded private copies, split over the cluster (gradient
    // mode: the host filled them before the launch)
    for (int k = 0; k < N && train; ++k) {
        const long long tot = P.dims[k] * R4;
        for (long long e = (long long)rank * blockDim.x + tid; e < tot; e += (long long)cs * blockDim.x) {
            const long long i = e / R4;
            const int r = (int)(e % R4);
            a.Ap[k][e] = r < R ? __ldcg(P.A[k] + i * R + r) : 0.f;
        }
    }
    // the private factors are read by bulk copies (the async proxy) from now on
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    cluster_sync_all();

    long long t = __ldcg(P.t_dev);
    int n_prev = -1;
    unsigned mma_iters = 0, step_phase = 0;
    long long gq0 = 0;                    // chunks of earlier iterations (barrier phases)
    const int f0 = rank * fpc;
    const int nf = (P.B - f0) < fpc ? ((P.B - f0) > 0 ? P.B - f0 : 0) : fpc;
    const int nchunks = (nf + kPK - 1) / kPK;
    int flags = 0;
    // H: thread tt < 136 of the transform warps owns the 4 x 4 block (hbi, hbj),
    // hbi <= hbj, of the upper triangle of the 64 x 64 grid of blocks
    const int tt = tid - 64;
    int hbi = 0, hbj = 0;
    if (tt >= 0 && tt < 136) {
        int rem = tt;
        while (rem >= 16 - hbi) {
            rem -= 16 - hbi;
            ++hbi;
        }
        hbj = hbi + rem;
    }

    const long long nit = train ? T : (md.K > g ? (md.K - 1 - g) / ncl + 1 : 0);
    for (long long it = 0; it < nit; ++it, ++t, gq0 += nchunks) {
        const long long bt = train ? -1 : g + it * ncl;   // gradient mode: the batch
        if (!train) t = md.t0 + bt;
        const bool last = train && it == T - 1;
        const int n = train ? mode_draw(P.seed, t, N) : md.gmode;
        const long long In = P.dims[n], ld = P.ld[n];
        const int ntile = (int)((In + kPM - 1) / kPM);
        trace_stamp(P.trace, 0, tr);

        // 1. draws of the own fibers (Alg. 3), from the staged CDFs
        {
            const int ch = (nf + 31) / 32;
            for (int job = warp; job < ch * N; job += kThreads / 32) {
                const int k = job / ch, c = job % ch;
                const int fl = 32 * c + lane;
                const bool act = fl < nf;
                if (k == n) {
                    if (act) sidx[fl * N + k] = -1;
                    continue;
                }
                const long long Ik = P.dims[k];
                const unsigned long long x = act ? fiber_word(P.seed, t, (long long)(f0 + fl), k) : 0ULL;
                long long i;
                if (P.sampling == CPD_SAMPLE_UNIFORM) {
                    i = (long long)__umul64hi(x, (unsigned long long)Ik);
                } else {
                    const unsigned long long *c0 = stage + a.off[k];
                    i = warp_search_staged(c0, Ik, __umul64hi(x, c0[Ik - 1]), act);
                }
                if (act) sidx[fl * N + k] = (int)i;
            }
        }
        __syncthreads();
        // columns (Eq. (2)) and weights s_f of the own fibers; padding slots get 0
        for (int fl = tid; fl < nchunks * kPK; fl += blockDim.x) {
            long long j = 0;
            float w = 0.f;
            if (fl < nf) {
                const int *row = sidx + fl * N;
                long long Jp = 1;
                for (int k = 0; k < N; ++k) {
                    if (k == n) continue;
                    j += (long long)row[k] * Jp;
                    Jp *= P.dims[k];
                }
                w = pers_weight(a, n, row, stage);
                if (last)
                    for (int k = 0; k < N; ++k) P.idx[(long long)(f0 + fl) * N + k] = row[k];
            }
            jcol[fl] = j;
            sw[fl] = w;
        }
        __syncthreads();
        trace_stamp(P.trace, 2, tr);

        // 2. gather + tensor-core contraction in chunks of 16 fibers
        const int g8 = ntile * (kPM / 8);          // 16-byte row pieces per fiber in the operand
        const int lpieces = (int)(ld / 8);         // 16-byte pieces of a landed fiber
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
        if (warp == 0) {
            // producer: whole fibers (ld elements) and their factor rows; lane 0
            // announces the bytes, the warp's lanes issue the bulk copies
            // (lane f < 16: fiber f; every lane: a share of the factor rows)
            // rows other CTAs stored (bulk stores, then a cluster barrier) are
            // read by bulk copies below
            asm volatile("fence.proxy.async.global;\n" ::: "memory");
            const __nv_bfloat16 *rep = reinterpret_cast<const __nv_bfloat16 *>(P.rep[n]);
            const uint32_t fbytes = (uint32_t)ld * 2, rbytes = (uint32_t)R4 * 4;
            for (int c = 0; c < nchunks; ++c) {
                const long long gq = gq0 + c;
                const int s = (int)(gq % L.nland);
                const bool trc = tr && c == 3;
                stamp_here(P.trace, 30, trc && lane == 0);
                if (gq >= L.nland) wait_or_abort(b_lempty + 8 * s, (uint32_t)((gq / L.nland - 1) & 1), abort);
                stamp_here(P.trace, 31, trc && lane == 0);
                const uint32_t lb = smem_u32(smem + L.land + (size_t)s * L.land_bytes);
                int nv = nf - c * kPK;
                nv = nv < kPK ? nv : kPK;
                if (lane == 0) mbar_expect_tx(b_lfull + 8 * s, (uint32_t)nv * (fbytes + (uint32_t)(N - 1) * rbytes));
                __syncwarp();
                if (!*abort) {
                    if (lane < nv) {
                        const int fl = c * kPK + lane;
                        bulk_g2s(lb + (uint32_t)(L.lx + lane * L.pitch), rep + jcol[fl] * ld, fbytes, b_lfull + 8 * s);
                    }
                    for (int q = lane; q < nv * (N - 1); q += 32) {
                        const int f = q / (N - 1), kk = q % (N - 1);
                        const int k = kk + (kk >= n ? 1 : 0);
                        const int fl = c * kPK + f;
                        bulk_g2s(lb + (uint32_t)(L.lfr + ((f * (N - 1) + kk) * R4) * 4),
                                 a.Ap[k] + (long long)sidx[fl * N + k] * R4, rbytes, b_lfull + 8 * s);
                    }
                }
                stamp_here(P.trace, 32, trc && lane == 0);
            }
        } else if (warp == 1) {
            // tensor-core products
            if (lane == 0) {
                const uint32_t idesc = idesc_bf16(kPM, Npad);
                for (int c = 0; c < nchunks; ++c) {
                    const long long gq = gq0 + c;
                    const int o = (int)(gq % kPOp);
                    wait_or_abort(b_ofull + 8 * o, (uint32_t)((gq / kPOp) & 1), abort);
                    stamp_here(P.trace, 39, tr && c == 3);
                    if (*abort) continue;
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    unsigned char *ob = smem + L.op + (size_t)o * L.op_bytes;
                    const uint32_t xs = smem_u32(ob + L.ox);
                    const uint64_t dh = smem_desc(smem_u32(ob + L.obh), (uint32_t)(Npad >> 3) * 128u, 128u);
                    const uint64_t dl = smem_desc(smem_u32(ob + L.obl), (uint32_t)(Npad >> 3) * 128u, 128u);
                    for (int m = 0; m < ntile; ++m) {
                        const uint64_t da = smem_desc(xs + (uint32_t)m * 2048u, (uint32_t)g8 * 128u, 128u);
                        const uint32_t d = tmem + (uint32_t)(m * cst);
                        mma_bf16(d, da, dh, idesc, c > 0 ? 1u : 0u);
                        mma_bf16(d, da, dl, idesc, 1u);
                    }
                    mma_commit(b_oempty + 8 * o);
                    stamp_here(P.trace, 43, tr && c == 3);
                }
                if (nchunks > 0 && !*abort) mma_commit(b_mma);
            }
        } else {
            // transform warps
            for (int c = 0; c < nchunks; ++c) {
                const long long gq = gq0 + c;
                const int s = (int)(gq % L.nland), o = (int)(gq % kPOp);
                const bool trc = tr && c == 3 && tt == 0;
                stamp_here(P.trace, 33, trc);
                wait_or_abort(b_lfull + 8 * s, (uint32_t)((gq / L.nland) & 1), abort);
                stamp_here(P.trace, 34, trc);
                if (gq >= kPOp) wait_or_abort(b_oempty + 8 * o, (uint32_t)((gq / kPOp - 1) & 1), abort);
                stamp_here(P.trace, 35, trc);
                const unsigned char *lb = smem + L.land + (size_t)s * L.land_bytes;
                unsigned char *ob = smem + L.op + (size_t)o * L.op_bytes;
                // fibers into the no-swizzle MN-major operand: piece (f, ig) =
                // rows [8 ig, 8 ig + 8) of fiber f at core matrix (f/8, ig),
                // slot f % 8; zero past the fiber and past the valid fibers
                for (int e = tt; e < kPK * g8; e += kPTT) {
                    const int f = (e & 7) | (((e >> 3) & 1) << 3), ig = e >> 4;
                    const int fl = c * kPK + f;
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    if (fl < nf && ig < lpieces)
                        v = *reinterpret_cast<const uint4 *>(lb + L.lx + (size_t)f * L.pitch + (size_t)ig * 16);
                    *reinterpret_cast<uint4 *>(ob + L.ox + ((size_t)((f >> 3) * g8 + ig) << 7) + ((f & 7) << 4)) = v;
                }
                stamp_here(P.trace, 36, trc);
                // z_f (fp32, for H) and Z' = s_f z_f as a bf16 hi/lo pair, K-major:
                // core matrix (f/8, r/8), 8 fibers per 16 bytes
                const float *fr = reinterpret_cast<const float *>(lb + L.lfr);
                __nv_bfloat16 *bh = reinterpret_cast<__nv_bfloat16 *>(ob + L.obh);
                __nv_bfloat16 *bl = reinterpret_cast<__nv_bfloat16 *>(ob + L.obl);
                float *z2 = zf + (gq & 1) * kPK * kPHd;
                for (int job = tt; job < Npad * 2; job += kPTT) {
                    const int r = job % Npad, fb8 = job / Npad;
                    __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int f = 8 * fb8 + u;
                        const int fl = c * kPK + f;
                        float z = 0.f;
                        if (r < R && fl < nf) {
                            const float *row = fr + (size_t)f * (N - 1) * R4 + r;
                            z = 1.f;
                            for (int kk = 0; kk < N - 1; ++kk) z = z * row[kk * R4];
                        }
                        z2[f * kPHd + r] = z;
                        const float zs = z * sw[fl];
                        hi[u] = __float2bfloat16_rn(zs);
                        lo[u] = __float2bfloat16_rn(zs - __bfloat162float(hi[u]));
                    }
                    const int off = ((fb8 * (Npad >> 3) + (r >> 3)) << 6) + ((r & 7) << 3);
                    *reinterpret_cast<uint4 *>(bh + off) = *reinterpret_cast<uint4 *>(hi);
                    *reinterpret_cast<uint4 *>(bl + off) = *reinterpret_cast<uint4 *>(lo);
                }
                fence_async_smem();
                transform_sync();   // the chunk's operands and z_f are complete; the landing stage is read
                stamp_here(P.trace, 37, trc);
                if (tt == 0) {
                    mbar_arrive(b_ofull + 8 * o);
                    mbar_arrive(b_lempty + 8 * s);
                }
                // H over this chunk's fibers: the thread's upper-triangle block
                if (tt < 136) {
                    for (int f = 0; f < kPK; ++f) {
                        const int fl = c * kPK + f;
                        const float sv = fl < nf ? sw[fl] : 0.f;
                        const float4 zr = *reinterpret_cast<const float4 *>(z2 + f * kPHd + 4 * hbi);
                        const float4 zc = *reinterpret_cast<const float4 *>(z2 + f * kPHd + 4 * hbj);
                        const float ar[4] = {zr.x * sv, zr.y * sv, zr.z * sv, zr.w * sv};
                        const float ac[4] = {zc.x, zc.y, zc.z, zc.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int v = 0; v < 4; ++v) acc[u][v] += ar[u] * ac[v];
                    }
                }
                stamp_here(P.trace, 38, trc);
            }
        }
        __syncthreads();
        trace_stamp(P.trace, 3, tr);
        if (nchunks > 0) {
            wait_or_abort(b_mma, mma_iters & 1, abort);
            ++mma_iters;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        trace_stamp(P.trace, 7, tr);

        // 3. partials to the scratch: M tiles staged row-major in shared memory
        //    (four at a time) and stored by bulk copies; H blocks directly
        {
            float *pm = part + (size_t)rank * rows_all * cst;
            const int qd = warp & 3, hh = warp >> 2;
            const bool z0 = nchunks == 0 || *abort;
            const size_t tb = up128((size_t)kPM * R4 * 4);
            for (int m0 = 0; m0 < ntile; m0 += 4) {
                for (int m = m0; m < ntile && m < m0 + 4; ++m) {
                    if (32 * hh >= Npad) break;
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(m * cst + 32 * hh), v);
                    float *tile = reinterpret_cast<float *>(region + (size_t)(m - m0) * tb);
                    const int rl = 32 * qd + lane;
#pragma unroll
                    for (int c = 0; c < 32; ++c)
                        if (32 * hh + c < R4) tile[rl * R4 + 32 * hh + c] = z0 ? 0.f : v[c];
                }
                fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    for (int m = m0; m < ntile && m < m0 + 4; ++m) {
                        const long long r0 = (long long)m * kPM;
                        const long long nr = (In - r0) < kPM ? In - r0 : kPM;
                        bulk_s2g(pm + r0 * R4, smem_u32(region + (size_t)(m - m0) * tb), (uint32_t)(nr * R4 * 4));
                    }
                    bulk_commit();
                    bulk_wait_all();   // written, and the staging may be reused
                }
                __syncthreads();
            }
            if (tt >= 0 && tt < 136) {
                float *ph = hpart + (size_t)rank * kPHd * kPHd;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    *reinterpret_cast<float4 *>(ph + (4 * hbi + u) * kPHd + 4 * hbj) =
                        make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
                    if (hbi != hbj)
#pragma unroll
                        for (int v = 0; v < 4; ++v) ph[(4 * hbj + v) * kPHd + 4 * hbi + u] = acc[u][v];
                }
            }
        }
        if (tid == 0) asm volatile("fence.proxy.async.global;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        trace_stamp(P.trace, 8, tr);
        cluster_sync_all();   // B1: every partial is in the scratch
        trace_stamp(P.trace, 14, tr);

        // 4. owned rows of H: summed in ascending CTA order (loads issued
        //    together, added in order), sent to every CTA
        {
            const int hpc = (R + cs - 1) / cs;
            const int h0 = rank * hpc, h1 = (h0 + hpc) < R ? h0 + hpc : R;
            const uint32_t hbase = smem_u32(sH);
            for (int e = tid; e < (h1 > h0 ? (h1 - h0) * R : 0); e += blockDim.x) {
                const int i = h0 + e / R, c = e % R;
                float pv[16];
#pragma unroll
                for (int src = 0; src < 16; ++src)
                    pv[src] = src < cs ? __ldcg(hpart + (size_t)src * kPHd * kPHd + i * kPHd + c) : 0.f;
                float v = 0.f;
#pragma unroll
                for (int src = 0; src < 16; ++src)
                    if (src < cs) v += pv[src];
                const uint32_t addr = hbase + (uint32_t)((i * kPHd + c) * 4);
                for (int d = 0; d < cs; ++d) st_cluster_f32(map_shared(addr, (uint32_t)d), v);
            }
        }
        cluster_sync_all();   // B2: H complete in every CTA
        trace_stamp(P.trace, 15, tr);

        // 5. owned rows of A^(n), in blocks: A and S rows and the partial
        //    blocks by bulk copies; M summed in ascending CTA order; G = A H - M;
        //    the step; rows and S back by bulk stores; the new weights
        const long long ngroups = (In + 31) / 32;
        const long long gpc = (ngroups + cs - 1) / cs;
        const long long row0 = 32 * gpc * rank;
        const long long row1 = (row0 + 32 * gpc) < In ? row0 + 32 * gpc : In;
        float *sA = reinterpret_cast<float *>(region + L.own_a);
        float *sM = reinterpret_cast<float *>(region + L.own_m);
        float *sN = reinterpret_cast<float *>(region + L.own_n);
        float *sG = reinterpret_cast<float *>(region + L.own_g);
        double *sS = reinterpret_cast<double *>(region + L.own_s);
        const float *red = reinterpret_cast<const float *>(region + L.red);
        const uint32_t wslot = smem_u32(stage + a.off[n]);
        const double alpha = P.step == CPD_STEP_DECAY ? P.beta / ((double)t + P.gamma) : P.alpha;
        const bool ada = train && P.step == CPD_STEP_ADAGRAD;
        for (long long b0 = row0; b0 < row1; b0 += kPOwnBlock) {
            const int nr = (int)((row1 - b0) < kPOwnBlock ? row1 - b0 : kPOwnBlock);
            const uint32_t blkb = (uint32_t)(nr * R4 * 4);
            const size_t blks = (size_t)kPOwnBlock * R4 * 4;
            for (int s0 = 0; s0 < cs; s0 += L.red_slots) {
                const int ns = (cs - s0) < L.red_slots ? cs - s0 : L.red_slots;
                if (tid == 0) {
                    asm volatile("fence.proxy.async.global;\n" ::: "memory");
                    uint32_t bytes = (uint32_t)ns * blkb;
                    if (s0 == 0) bytes += blkb + (ada ? (uint32_t)((nr * R * 8 + 15) / 16 * 16) : 0u);
                    mbar_expect_tx(b_step, bytes);
                    if (!*abort) {
                        if (s0 == 0) {
                            bulk_g2s(smem_u32(sA), a.Ap[n] + b0 * R4, blkb, b_step);
                            if (ada) bulk_g2s(smem_u32(sS), P.S[n] + b0 * R, (uint32_t)((nr * R * 8 + 15) / 16 * 16), b_step);
                        }
                        for (int q = 0; q < ns; ++q)
                            bulk_g2s(smem_u32(region + L.red + q * blks),
                                     part + (size_t)(s0 + q) * rows_all * cst + (size_t)b0 * R4, blkb, b_step);
                    }
                }
                wait_or_abort(b_step, step_phase & 1, abort);
                ++step_phase;
                for (int e = tid; e < nr * R; e += blockDim.x) {
                    const int i = e / R, c = e % R;
                    float v = s0 == 0 ? 0.f : sM[i * R4 + c];
                    for (int q = 0; q < ns; ++q) v += red[q * (blks / 4) + i * R4 + c];
                    sM[i * R4 + c] = v;
                }
                __syncthreads();   // the staged blocks are read
            }
            trace_stamp(P.trace, 40, tr && b0 == row0);
            // A H for a row and 4 consecutive columns per thread (4 independent
            // chains; one broadcast A load and one float4 H load per step)
            const int r4n = R4 / 4;
            for (int e = tid; e < nr * r4n; e += blockDim.x) {
                const int i = e / r4n, r0c = 4 * (e % r4n);
                float ah4[4] = {0.f, 0.f, 0.f, 0.f};
                for (int s = 0; s < R; ++s) {
                    const float av = sA[i * R4 + s];
                    const float4 hv = *reinterpret_cast<const float4 *>(sH + s * kPHd + r0c);
                    ah4[0] += av * hv.x;
                    ah4[1] += av * hv.y;
                    ah4[2] += av * hv.z;
                    ah4[3] += av * hv.w;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) sG[i * R4 + r0c + u] = ah4[u];
            }
            __syncthreads();
            for (int e = tid; e < nr * R; e += blockDim.x) {
                const int i = e / R, r = e % R;
                const long long row = b0 + i;
                const float gr = sG[i * R4 + r] - sM[i * R4 + r];
                if (!train) {
                    md.gout[((size_t)bt * In + row) * R + r] = gr;
                    continue;
                }
                const float aold = sA[i * R4 + r];
                float an;
                if (ada) {
                    const double S2 = __fma_rn((double)gr, (double)gr, sS[i * R + r]);
                    sS[i * R + r] = S2;
                    an = aold - (float)P.eta * gr * rsqrtf((float)S2 + (float)P.b);
                } else {
                    an = aold - (float)alpha * gr;
                }
                if (P.constraint == CPD_CONSTRAINT_NONNEG && an < 0.f) an = 0.f;   // projection; NaN kept
                if (!isfinite(an) || !isfinite(gr)) flags |= kStNonFinite;
                sM[i * R4 + r] = an;   // M(i, r) is read by this thread only; sA stays intact for A H
                sN[i * R + r] = an;
                if (last) P.G[row * R + r] = gr;
            }
            if (R4 > R)   // the stored rows keep their zero padding
                for (int e = tid; e < nr * (R4 - R); e += blockDim.x) sM[(e / (R4 - R)) * R4 + R + e % (R4 - R)] = 0.f;
            fence_async_smem();
            __syncthreads();
            trace_stamp(P.trace, 41, tr && b0 == row0);
            if (train && tid == 0) {
                // rows and S back (the padding columns of the rows are unchanged)
                bulk_s2g(a.Ap[n] + b0 * R4, smem_u32(sM), blkb);
                if (ada && nr * R >= 2) bulk_s2g(P.S[n] + b0 * R, smem_u32(sS), (uint32_t)(nr * R * 8 / 16 * 16));
                bulk_commit();
            }
            if (ada && tid == 0 && ((nr * R) & 1)) P.S[n][(b0 + nr) * R - 1] = sS[nr * R - 1];   // odd tail
            if (train && P.sampling == CPD_SAMPLE_EUCLIDEAN) {
                // eight rows per warp at a time; lanes < cs send the weights
                for (int lr0 = 8 * warp; lr0 < nr; lr0 += 8 * (kThreads / 32)) {
                    const int cnt = (nr - lr0) < 8 ? nr - lr0 : 8;
                    double w[8];
                    warp_row_weights8(sN + lr0 * R, R, cnt, R, w);
                    for (int u = 0; u < cnt; ++u) {
                        const double wv = __shfl_sync(0xffffffffu, w[u], 0);
                        if (lane < cs) {
                            const uint32_t addr = wslot + (uint32_t)((b0 + lr0 + u) * 8);
                            st_cluster_u64(map_shared(addr, (uint32_t)lane),
                                           (unsigned long long)__double_as_longlong(wv));
                        }
                    }
                }
            }
            if (train && tid == 0) bulk_wait_all();   // the stores read the staging before it is reused
            __syncthreads();
            trace_stamp(P.trace, 42, tr && b0 == row0);
        }
        if (tid == 0) asm volatile("fence.proxy.async.global;\n" ::: "memory");
        trace_stamp(P.trace, 18, tr);
        if (!train) {
            // the next batch's partials overwrite the scratch: every CTA has
            // read it (and no H row is still being sent)
            cluster_sync_all();
            continue;
        }
        cluster_sync_all();   // B3: new rows in the private factor, weights in every CTA
        trace_stamp(P.trace, 20, tr);

        // 6. mode n's CDF from its new weights, in place (exact fixed point)
        if (P.sampling == CPD_SAMPLE_EUCLIDEAN) {
            if (!block_distribution_inplace(stage + a.off[n], In, dsm)) flags |= kStDegenerate;
        }
        __syncthreads();
        n_prev = n;
        trace_stamp(P.trace, 21, tr);
    }

    // ---- results back to the context ----------------------------------------
    for (int k = 0; k < N && train; ++k) {
        const long long tot = P.dims[k] * R;
        for (long long e = (long long)rank * blockDim.x + tid; e < tot; e += (long long)cs * blockDim.x) {
            const long long i = e / R;
            const int r = (int)(e % R);
            P.A[k][e] = __ldcg(a.Ap[k] + i * R4 + r);
        }
    }
    if (train && rank == 0) {
        if (P.sampling != CPD_SAMPLE_UNIFORM)
            for (int k = 0; k < N; ++k)
                for (long long i = tid; i < P.dims[k]; i += blockDim.x) P.cdf[k][i] = stage[a.off[k] + i];
        if (tid == 0) {
            *P.t_dev = t;
            if (n_prev >= 0) *P.n_last = n_prev;
            *P.dirty = -1;
        }
    }
    if (flags) atomicOr(&s_flags, flags);
    __syncthreads();
    if (tid == 0) {
        if (s_flags) atomicOr(P.status, s_flags);
        if (*abort) {
            atomicOr(P.status, kStTimeout);
            // products and copies still in flight must finish before the
            // accumulator and the shared memory are released
            mbar_wait_bounded(b_mma, mma_iters & 1);
            for (int q = 0; q < L.nland; ++q) {
                const long long issued = (gq0 + L.nland - 1 - q) / L.nland;   // phases issued on stage q
                if (issued > 0) mbar_wait_bounded(b_lfull + 8 * q, (uint32_t)((issued - 1) & 1));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tcols) : "memory");
    cluster_sync_all();   // no CTA leaves while another may still address its shared memory
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
bool pers_supported(const cpd_config &c)
{
    if (c.x_dtype != CPD_BF16 || c.R > 64 || c.sampling == CPD_SAMPLE_LEVERAGE) return false;
    long long sumI = 0, imax = 0;
    for (int k = 0; k < c.N; ++k) {
        sumI += c.dims[k];
        imax = c.dims[k] > imax ? c.dims[k] : imax;
    }
    const int Npad = (c.R + 15) / 16 * 16;
    const int cst = Npad <= 32 ? 32 : 64;
    return sumI <= kPMaxStage && ((imax + kPM - 1) / kPM) * cst <= 512;
}

void pers_fill(PersArgs &a, int cs)
{
    const Problem<float> &P = a.P;
    a.cs = cs;
    a.fpc = (P.B + cs - 1) / cs;
    a.fpc = (a.fpc + kPK - 1) / kPK * kPK;
    a.R4 = (P.R + 3) / 4 * 4;
    a.Npad = (P.R + 15) / 16 * 16;
    a.cst = a.Npad <= 32 ? 32 : 64;
    long long imax = 0, o = 0;
    for (int k = 0; k < P.N; ++k) {
        a.off[k] = o;
        o += P.dims[k];
        imax = P.dims[k] > imax ? P.dims[k] : imax;
    }
    a.sumI = o;
    a.ntile = (int)((imax + kPM - 1) / kPM);
}

size_t pers_smem_bytes(const PersArgs &a)
{
    if (a.fpc > kPMaxFpc) return (size_t)1 << 30;   // refused by the caller (over the limit)
    const PersLayout L(a);
    return L.total > kPSmemMax ? (size_t)1 << 30 : L.total;
}

static cudaError_t pers_attrs(int cs, size_t smem)
{
    static size_t attr_bytes = 0;
    static bool nonportable = false;
    cudaError_t e = cudaSuccess;
    if (smem > attr_bytes) {
        e = cudaFuncSetAttribute(k_pers, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        attr_bytes = smem;
    }
    if (cs > 8 && !nonportable) {
        e = cudaFuncSetAttribute(k_pers, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        nonportable = true;
    }
    return cudaSuccess;
}

static void pers_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr, int grid, int cs, size_t smem,
                        cudaStream_t s)
{
    cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}

int pers_max_clusters(const PersArgs &a)
{
    const size_t smem = pers_smem_bytes(a);
    if (smem > kPSmemMax || a.cs < 1 || a.cs > 16) return 0;
    if (pers_attrs(a.cs, smem) != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    pers_config(cfg, attr, a.cs, a.cs, smem, nullptr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_pers, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_pers(const PersArgs &a, long long T, cudaStream_t s)
{
    const size_t smem = pers_smem_bytes(a);
    if (cudaError_t e = pers_attrs(a.cs, smem); e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    pers_config(cfg, attr, a.cs, a.cs, smem, s);
    PersMode md{-1, 0, 0, nullptr};
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_pers, a, (const PersArgs *)nullptr, T, md);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

cudaError_t launch_pers_group(const PersArgs *dargs, int G, int cs, size_t smem, long long T, cudaStream_t s)
{
    if (cudaError_t e = pers_attrs(cs, smem); e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    pers_config(cfg, attr, G * cs, cs, smem, s);
    PersArgs dummy{};
    PersMode md{-1, 0, 0, nullptr};
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_pers, dummy, dargs, T, md);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

}  // namespace cpd

namespace cpd {

// Private padded factors from the context's factors (gradient mode).
__global__ void k_pers_pad(const PersArgs a)
{
    const Problem<float> &P = a.P;
    for (int k = 0; k < P.N; ++k) {
        const long long tot = P.dims[k] * a.R4;
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
             e += (long long)gridDim.x * blockDim.x) {
            const long long i = e / a.R4;
            const int r = (int)(e % a.R4);
            a.Ap[k][e] = r < P.R ? P.A[k][i * P.R + r] : 0.f;
        }
    }
}

cudaError_t launch_pers_gradients(const PersArgs &a, int n, long long t0, int K, int nclusters, float *gout,
                                  cudaStream_t s)
{
    const size_t smem = pers_smem_bytes(a);
    if (cudaError_t e = pers_attrs(a.cs, smem); e != cudaSuccess) return e;
    k_pers_pad<<<152, kThreads, 0, s>>>(a);
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    pers_config(cfg, attr, nclusters * a.cs, a.cs, smem, s);
    PersMode md{n, t0, K, gout};
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_pers, a, (const PersArgs *)nullptr, 1LL, md);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

}  // namespace cpd
