// C ABI of libcpd (declared and documented in include/cpd.h).
//
// The context owns every device buffer of one decomposition. Iterations are
// device-driven (mode and draws follow from the device counter t), so chunks
// of 32, 16, 8, 4, 2 and 1 iterations are each captured once into a CUDA
// graph and replayed: any iteration count runs as at most one replay per
// chunk size beyond the whole 32-iteration chunks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cpd.h"
#include "cpd_internal.h"

using namespace cpd;

static thread_local std::string g_err;

static cpd_status fail(cpd_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

static cpd_status cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CPD_ENOMEM : CPD_ECUDA;
}

#define CK(call)                                                      \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);           \
    } while (0)

static constexpr int kGraphChunk = 32;
static constexpr int kGraphSizes = 6;   // chunks of 32, 16, 8, 4, 2, 1 iterations
static constexpr int kProfSlots = 8192;

struct cpd_ctx {
    cpd_config cfg{};
    int fbytes = 4;          // factor element size
    int xbytes = 4;          // tensor element size
    int device = 0;
    int engine = kEngineSimt;
    Problem<float> Pf{};
    Problem<double> Pd{};
    std::vector<void *> allocs;
    int64_t t_host = 0;
    int grid_grad = 0, grid_upd = 0;
    size_t smem_grad = 0;
    double *fit_partials = nullptr, *fit_out = nullptr;
    void *fit_tc = nullptr;  // scratch of the tensor-core stop check (BF16 tensors), or null
    int sm_count = 152;
    double xnorm2 = 0.0;
    int64_t imax = 0;
    // graph replay: graph[q] runs kGraphChunk >> q iterations
    cudaGraphExec_t graph[kGraphSizes] = {};
    cudaStream_t graph_stream = nullptr;
    // profiling
    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    int prof_used = 0;
    bool has_sample = false;
    unsigned long long *trace_buf = nullptr;
    int max_clusters = 0;
    cudaStream_t home = nullptr;     // stream of cpd_init: allocations and frees
    cudaEvent_t fit_event = nullptr; // cpd_fit_start / cpd_fit_poll
    double *fit_host = nullptr;      // pinned copy of the residual sum
    bool fit_started = false;
    PersArgs pers{};                 // persistent engine: launch arguments (P refreshed per launch)
    int64_t prof_iters = 0;          // iterations covered by the profiled launches
    float *gpart = nullptr, *ghpart = nullptr;   // cpd_gradients: scratch of gclusters clusters
    int gclusters = 0;

    template <class F>
    cudaError_t with_problem(F &&f)
    {
        return fbytes == 8 ? f(Pd) : f(Pf);
    }
};

template <class T>
static Problem<T> &problem(cpd_ctx *c);
template <>
Problem<float> &problem<float>(cpd_ctx *c) { return c->Pf; }
template <>
Problem<double> &problem<double>(cpd_ctx *c) { return c->Pd; }

// Device buffers come from the stream-ordered allocator on the context's
// stream, so creating and destroying contexts never synchronises the device
// (other decompositions keep running).
static cudaError_t dmalloc(cpd_ctx *c, void **p, size_t bytes)
{
    cudaError_t e = cudaMallocAsync(p, bytes < 16 ? 16 : bytes, c->home);
    if (e == cudaSuccess) c->allocs.push_back(*p);
    return e;
}

static void drop_graphs(cudaGraphExec_t *g, int n)
{
    for (int q = 0; q < n; ++q)
        if (g[q]) {
            cudaGraphExecDestroy(g[q]);
            g[q] = nullptr;
        }
}

static void free_all(cpd_ctx *c)
{
    drop_graphs(c->graph, kGraphSizes);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->fit_event) cudaEventDestroy(c->fit_event);
    if (c->fit_host) cudaFreeHost(c->fit_host);
    for (void *p : c->allocs) cudaFreeAsync(p, c->home);
    c->allocs.clear();
    cudaStreamSynchronize(c->home);
}

static int64_t round8(int64_t v) { return (v + 7) / 8 * 8; }

static cpd_status validate(const cpd_config *cfg)
{
    if (!cfg) return fail(CPD_EINVAL, "cfg is NULL");
    if (cfg->N < 3 || cfg->N > CPD_MAX_MODES) return fail(CPD_EINVAL, "N must be in [3, 8]");
    if (cfg->R < 1 || cfg->R > 256) return fail(CPD_EINVAL, "R must be in [1, 256]");
    if (cfg->B < 1 || cfg->B > 65536) return fail(CPD_EINVAL, "B must be in [1, 65536]");
    if (cfg->sampling < 0 || cfg->sampling > 2) return fail(CPD_EINVAL, "unknown sampling");
    if (cfg->step < 0 || cfg->step > 2) return fail(CPD_EINVAL, "unknown step");
    if (cfg->x_dtype < 0 || cfg->x_dtype > 2) return fail(CPD_EINVAL, "unknown x_dtype");
    if (cfg->max_ctas < 0) return fail(CPD_EINVAL, "max_ctas must be >= 0");
    if (cfg->constraint != CPD_CONSTRAINT_NONE && cfg->constraint != CPD_CONSTRAINT_NONNEG)
        return fail(CPD_EINVAL, "unknown constraint");
    if (cfg->x_layout != CPD_LAYOUT_REPLICAS && cfg->x_layout != CPD_LAYOUT_STRIDED)
        return fail(CPD_EINVAL, "unknown x_layout");
    if (cfg->x_layout == CPD_LAYOUT_STRIDED && cfg->engine != 0 && cfg->engine != kEngineSimt)
        return fail(CPD_EINVAL, "the strided x_layout runs on the CUDA-core engine (1)");
    if (cfg->engine < 0 || cfg->engine > 5) return fail(CPD_EINVAL, "unknown engine");
    if (cfg->block < 0) return fail(CPD_EINVAL, "block must be >= 0");
    if (cfg->block > 1 && (cfg->B % cfg->block || cfg->dims[0] % cfg->block || cfg->dims[1] % cfg->block))
        return fail(CPD_EINVAL, "block (Remark 1) must divide B, I_1 and I_2");
    if (cfg->block > 1 && cfg->engine == kEnginePersistent)
        return fail(CPD_EINVAL, "the persistent engine samples fibers one by one (block 0 or 1)");
    if (cfg->tile_rows < 0 || cfg->tile_fibers < 0 || cfg->tile_fibers > cfg->B)
        return fail(CPD_EINVAL, "tile_rows and tile_fibers must be >= 0, tile_fibers <= B");
    if (cfg->tile_rows && (cfg->tile_rows % 8 || cfg->tile_rows > 512))
        return fail(CPD_EINVAL, "tile_rows must be a multiple of 8 in [8, 512]");
    if ((cfg->engine == kEnginePersistent || cfg->engine == kEngineFused) && (cfg->tile_rows || cfg->tile_fibers))
        return fail(CPD_EINVAL, "the persistent and fused engines take no tile_rows / tile_fibers");
    if ((cfg->engine == kEngineTensor || cfg->engine == kEngineTensorCluster) &&
        ((cfg->tile_rows && cfg->tile_rows != 128) ||
         (cfg->tile_fibers && (cfg->tile_fibers % 16 ||
                               cfg->tile_fibers > (cfg->engine == kEngineTensor ? 128 : 256)))))
        return fail(CPD_EINVAL, "tensor-core engines: tile_rows 0 or 128, tile_fibers a multiple of 16 "
                                "up to 128 (engine 2) or 256 (engine 3)");
    if (cfg->engine == kEnginePersistent && !pers_supported(*cfg))
        return fail(CPD_EINVAL, "persistent engine needs BF16 tensors, R <= 64, Euclidean or uniform "
                                "sampling, sum of the I_k <= 4096 and ceil(I_max / 128) row tiles in tensor memory");
    if (cfg->engine == kEnginePersistent && cfg->max_ctas > 16)
        return fail(CPD_EINVAL, "persistent engine: max_ctas is the cluster size, at most 16");
    double total = 1.0;
    for (int k = 0; k < cfg->N; ++k) {
        if (cfg->dims[k] < 1 || cfg->dims[k] > (int64_t)1 << 31)
            return fail(CPD_EINVAL, "every dim must be in [1, 2^31]");
        if (cfg->sampling == CPD_SAMPLE_LEVERAGE && cfg->dims[k] <= cfg->R)
            return fail(CPD_EINVAL, "leverage sampling needs I_k > R (Def. 3, Lemma 1)");
        total *= (double)cfg->dims[k];
    }
    if (total > 9.0e15) return fail(CPD_EINVAL, "tensor too large");
    if (cfg->step == CPD_STEP_ADAGRAD && !(cfg->eta > 0.0 && cfg->b >= 0.0))
        return fail(CPD_EINVAL, "AdaGrad needs eta > 0 and b >= 0");
    if (cfg->step == CPD_STEP_DECAY && !(cfg->gamma > 0.0))
        return fail(CPD_EINVAL, "decreasing step needs gamma > 0");
    if ((cfg->engine == kEngineTensor || cfg->engine == kEngineTensorCluster || cfg->engine == kEngineFused) &&
        (cfg->x_dtype != CPD_BF16 || !tc_supported(cfg->R, 128)))
        return fail(CPD_EINVAL, "tensor-core engine needs BF16 tensors and R <= 64");
    if (cfg->engine == kEngineFused &&
        ((cfg->max_ctas & (cfg->max_ctas - 1)) || cfg->max_ctas > 16 || !fused_fits(cfg->N, cfg->R, cfg->B, cfg->max_ctas, 1)))
        return fail(CPD_EINVAL, "fused engine: max_ctas is the cluster size (0 = chosen, or 1, 2, 4, 8, 16) and "
                                "a CTA's share of the batch must fit its shared memory (at most 208 fibers; "
                                "fewer for small clusters and large R)");
    if (cfg->engine == kEngineTensorCluster) {
        int64_t imax = 0;
        for (int k = 0; k < cfg->N; ++k) imax = std::max<int64_t>(imax, cfg->dims[k]);
        if ((imax + 127) / 128 > 8) return fail(CPD_EINVAL, "cluster engine needs every I_k <= 1024");
    }
    return CPD_OK;
}

// Launch tiling: rb rows x fb fibers per CTA, about two waves of CTAs.
template <class T>
static void choose_tiles(cpd_ctx *c, Problem<T> &P, int sm_count)
{
    const cpd_config &g = c->cfg;
    int64_t imax = 0;
    for (int k = 0; k < g.N; ++k) imax = std::max<int64_t>(imax, g.dims[k]);
    c->imax = imax;
    P.cs = 1;
    if (c->engine == kEnginePersistent) {
        if constexpr (sizeof(T) == 4) {
            // one cluster; its size is max_ctas when given, else the largest
            // of 8, 4, 2, 1 that the device can co-schedule with the layout
            PersArgs &pa = c->pers;
            pa.P = P;
            int cs = g.max_ctas > 0 ? g.max_ctas : 8;
            pers_fill(pa, cs);
            while (g.max_ctas == 0 && cs > 1 && pers_max_clusters(pa) < 1) {
                cs >>= 1;
                pers_fill(pa, cs);
            }
            P.rb = 128;
            P.cs = cs;
            P.fb = pa.fpc;
            P.pf = 1;
            for (int k = 0; k < g.N; ++k) P.tile[k].pr = (int)((g.dims[k] + 127) / 128);
            c->grid_grad = cs;
            c->grid_upd = 0;
            c->smem_grad = pers_smem_bytes(pa);
            c->max_clusters = pers_max_clusters(pa);
        }
        return;
    }
    if (c->engine == kEngineFused) {
        if constexpr (sizeof(T) == 4) {
            // one cluster per tile of 128 rows, or of 256 rows (two MMA tiles)
            // where the tiles of 128 would outnumber the clusters the device
            // co-schedules; its CTAs split the batch
            int cs = 1, fpc = 16;
            fused_plan(g.N, g.R, g.B, g.max_ctas, &cs, &fpc);
            P.rb = 128;
            P.cs = cs;
            P.fb = fpc;
            P.pf = 1;
            c->max_clusters = fused_max_clusters(P);
            if (c->max_clusters >= 1 && (imax + 127) / 128 > c->max_clusters && fused_fits(g.N, g.R, g.B, cs, 2)) {
                P.rb = 256;
                const int m2 = fused_max_clusters(P);
                if (m2 >= 1) c->max_clusters = m2;
                else P.rb = 128;
            }
            int maxpr = 0;
            for (int k = 0; k < g.N; ++k) {
                P.tile[k].pr = (int)((g.dims[k] + P.rb - 1) / P.rb);
                maxpr = std::max(maxpr, P.tile[k].pr);
            }
            c->grid_grad = cs * maxpr;
            c->grid_upd = 0;
            c->smem_grad = fused_smem_bytes(P);
            if (c->max_clusters < 1) {   // no such cluster can be co-scheduled
                c->engine = imax <= 1024 ? kEngineTensorCluster : kEngineTensor;
                choose_tiles(c, P, sm_count);
            }
        }
        return;
    }
    if (c->engine == kEngineTensorCluster) {
        if constexpr (sizeof(T) == 4) {
            // one cluster of ceil(I_max / 128) CTAs per fiber group; as many
            // groups as clusters fit at once, fibers per group a multiple of 16
            P.rb = 128;
            P.cs = (int)((imax + P.rb - 1) / P.rb);
            P.fb = 128;
            const int maxc = tcc_max_clusters(P);
            if (maxc < 1) {   // no such cluster can be co-scheduled: per-CTA engine
                c->engine = kEngineTensor;
                choose_tiles(c, P, sm_count);
                return;
            }
            int64_t pf = std::max<int64_t>(1, std::min<int64_t>(maxc, (g.B + 15) / 16));
            if (g.max_ctas > 0) pf = std::max<int64_t>(1, std::min<int64_t>(pf, g.max_ctas / P.cs));
            int64_t fb = (g.B + pf - 1) / pf;
            fb = (fb + 15) / 16 * 16;
            P.fb = (int)std::min<int64_t>(256, std::max<int64_t>(16, fb));
            while (P.fb > 16 && tcc_smem_bytes(P) > 220 * 1024) P.fb -= 16;
            c->max_clusters = maxc;
        }
    } else if (c->engine == kEngineTensor) {
        // 128-row MMA tiles; fibers per CTA a multiple of 16 (the MMA K), about
        // one wave of CTAs.
        P.rb = 128;
        const int64_t pr_max = (imax + P.rb - 1) / P.rb;
        const int64_t ctas = g.max_ctas > 0 ? std::min<int64_t>(g.max_ctas, sm_count) : sm_count;
        const int64_t pf = std::max<int64_t>(1, (ctas + pr_max - 1) / pr_max);
        int64_t fb = (g.B + pf - 1) / pf;
        fb = (fb + 15) / 16 * 16;
        P.fb = (int)std::min<int64_t>(128, std::max<int64_t>(16, fb));
        if constexpr (sizeof(T) == 4)
            while (P.fb > 16 && tc_smem_bytes(P) > 220 * 1024) P.fb -= 16;
    } else {
        // Under a CTA cap (several decompositions share the GPU) a CTA takes
        // whole modes of up to 512 rows, so a fiber group's draws and KRP rows
        // are formed once instead of once per 64-row tile.
        P.rb = (int)std::min<int64_t>(g.max_ctas > 0 ? 512 : 64, round8(imax));
        int64_t pr_max = (imax + P.rb - 1) / P.rb;
        int64_t target = g.max_ctas > 0 ? std::min<int64_t>(g.max_ctas, 2LL * sm_count) : 2LL * sm_count;
        int64_t pf = std::max<int64_t>(1, (target + pr_max - 1) / pr_max);
        pf = std::min<int64_t>(pf, std::max<int64_t>(1, (g.B + 15) / 16));
        P.fb = (int)((g.B + pf - 1) / pf);
        while (grad_smem_bytes(P) > 200 * 1024 && (P.fb > 8 || P.rb > 8)) {
            if (P.fb > 8) P.fb = (P.fb + 1) / 2;
            else P.rb = std::max(8, P.rb / 2);
        }
    }
    // an explicit tile shape (validated per engine; its shared memory is
    // checked after the choice)
    if (g.tile_rows && c->engine == kEngineSimt) P.rb = (int)std::min<int64_t>(g.tile_rows, round8(imax));
    if (g.tile_fibers) P.fb = g.tile_fibers;
    P.pf = (g.B + P.fb - 1) / P.fb;
    int maxpr = 0;
    for (int k = 0; k < g.N; ++k) {
        P.tile[k].pr = (int)((g.dims[k] + P.rb - 1) / P.rb);
        maxpr = std::max(maxpr, P.tile[k].pr);
    }
    c->grid_grad = (c->engine == kEngineTensorCluster ? P.cs : maxpr) * P.pf;
    const int rpc = std::max(1, kThreads / g.R);
    c->grid_upd = (int)((imax + rpc - 1) / rpc);
    if constexpr (sizeof(T) == 4)
        c->smem_grad = c->engine == kEngineTensorCluster ? tcc_smem_bytes(P)
                       : c->engine == kEngineTensor      ? tc_smem_bytes(P)
                                                         : grad_smem_bytes(P);
    else
        c->smem_grad = grad_smem_bytes(P);
}

template <class T>
static cpd_status init_typed(cpd_ctx *c, const void *X, int x_loc, const void *const *A0, int a0_loc,
                             cudaStream_t s)
{
    const cpd_config &g = c->cfg;
    Problem<T> &P = problem<T>(c);
    P.N = g.N; P.R = g.R; P.B = g.B; P.sampling = g.sampling; P.step = g.step; P.x_dtype = g.x_dtype;
    P.constraint = g.constraint;
    P.alpha = g.alpha; P.eta = g.eta; P.b = g.b; P.beta = g.beta; P.gamma = g.gamma;
    P.seed = g.seed;
    P.strided = g.x_layout == CPD_LAYOUT_STRIDED ? 1 : 0;
    P.block = g.block > 1 ? g.block : 1;
    int64_t q = 1;
    for (int k = 0; k < g.N; ++k) {
        P.dims[k] = g.dims[k];
        P.ld[k] = round8(g.dims[k]);
        P.xq[k] = q;                        // prod of dims[1 .. k-1]
        if (k > 0) q *= g.dims[k];
        double J = 1.0;
        for (int m = 0; m < g.N; ++m)
            if (m != k) J *= (double)g.dims[m];
        P.Jn[k] = J;
        P.inv_bj[k] = (float)((double)P.block / ((double)g.B * J));   // 1 / ((B / bs) J_n)
    }
    int sm_count = 152;
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, c->device);
    c->sm_count = sm_count;
    if (g.engine == 0 && P.strided) {
        c->engine = kEngineSimt;
    } else if (g.engine == 0) {
        int64_t imax = 0;
        for (int k = 0; k < g.N; ++k) imax = std::max<int64_t>(imax, g.dims[k]);
        const bool tc = g.x_dtype == CPD_BF16 && tc_supported(g.R, 128) && g.R >= 16;
        c->engine = !tc ? kEngineSimt : ((imax + 127) / 128 <= 8 ? kEngineTensorCluster : kEngineTensor);
    } else {
        c->engine = g.engine;
    }
    choose_tiles(c, P, sm_count);
    if (g.tile_rows || g.tile_fibers) {   // an explicit tile shape must fit the engine
        const size_t lim = c->engine == kEngineSimt ? 200 * 1024 : 220 * 1024;
        if (c->smem_grad > lim || (c->engine == kEngineTensor && P.fb > 128))
            return fail(CPD_EINVAL, "tile_rows / tile_fibers: the tile does not fit the engine's shared memory");
    }

    // Tensor replicas (one per mode), built from a device copy of X.
    int64_t total = 1;
    for (int k = 0; k < g.N; ++k) total *= g.dims[k];
    const size_t xb = (size_t)c->xbytes;
    const void *Xd = X;
    void *staging = nullptr;
    if (x_loc == CPD_HOST) {
        CK(cudaMallocAsync(&staging, total * xb, s));
        CK(cudaMemcpyAsync(staging, X, total * xb, cudaMemcpyHostToDevice, s));
        Xd = staging;
    }
    // the strided layout keeps the mode-1 replica alone and reads every mode from it
    for (int k = 0; k < (P.strided ? 1 : g.N); ++k) {
        const size_t bytes = (size_t)(total / g.dims[k]) * P.ld[k] * xb;
        void *rep;
        cudaError_t e = dmalloc(c, &rep, bytes);
        if (e != cudaSuccess) {
            if (staging) cudaFreeAsync(staging, s);
            return cuda_fail(e, "replica allocation");
        }
        if (P.ld[k] != g.dims[k]) CK(cudaMemsetAsync(rep, 0, bytes, s));
        e = launch_build_replica(Xd, rep, (int)xb, g.N, g.dims, k, P.ld[k], s);
        if (e != cudaSuccess) {
            if (staging) cudaFreeAsync(staging, s);
            return cuda_fail(e, "replica build");
        }
        P.rep[k] = rep;
    }
    for (int k = 1; k < g.N && P.strided; ++k) P.rep[k] = P.rep[0];
    if (staging) CK(cudaFreeAsync(staging, s));

    // Factors, AdaGrad state, distributions.
    for (int k = 0; k < g.N; ++k) {
        const size_t fb = (size_t)g.dims[k] * g.R;
        void *a, *S, *w, *cdf;
        CK(dmalloc(c, &a, fb * sizeof(T) + 64));   // tail room for 16-byte bulk copies of row blocks
        CK(dmalloc(c, &S, fb * sizeof(double) + 64));   // tail room for 16-byte bulk copies of row blocks
        CK(dmalloc(c, &w, g.dims[k] * sizeof(double)));
        CK(dmalloc(c, &cdf, g.dims[k] * sizeof(unsigned long long)));
        CK(cudaMemcpyAsync(a, A0[k], fb * sizeof(T),
                           a0_loc == CPD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(S, 0, fb * sizeof(double), s));
        P.A[k] = (T *)a; P.S[k] = (double *)S; P.w[k] = (double *)w; P.cdf[k] = (unsigned long long *)cdf;
    }
    void *p;
    CK(dmalloc(c, &p, sizeof(long long)));  P.t_dev = (long long *)p;
    CK(dmalloc(c, &p, sizeof(int)));        P.n_last = (int *)p;
    CK(dmalloc(c, &p, (size_t)g.B * g.N * sizeof(int)));  P.idx = (int *)p;
    CK(dmalloc(c, &p, (size_t)g.B * sizeof(double)));     P.p = (double *)p;
    CK(dmalloc(c, &p, (size_t)P.pf * g.R * c->imax * sizeof(T)));  P.part = (T *)p;
    CK(dmalloc(c, &p, (size_t)c->imax * g.R * sizeof(T)));  P.G = (T *)p;
    CK(dmalloc(c, &p, (size_t)(2 * g.R * g.R + g.R + 8) * sizeof(double)));  P.lev_L = (double *)p;
    CK(dmalloc(c, &p, sizeof(int)));  P.status = (int *)p;
    CK(dmalloc(c, &p, sizeof(int)));  P.dirty = (int *)p;
    CK(cudaMemsetAsync(P.dirty, 0xff, sizeof(int), s));
    {
        // CDF rebuilds are deferred to the next gradient kernel when every
        // mode's companions fit its staging buffer
        long long cap = kSimtStageCap;
        if constexpr (sizeof(T) == 4) {
            if (c->engine == kEngineTensor) cap = tc_stage_cap(P);
            if (c->engine == kEngineTensorCluster) cap = tcc_stage_cap(P);
            if (c->engine == kEngineFused) cap = fused_stage_cap(P);
        }
        long long need = 0;
        for (int n = 0; n < g.N; ++n) {
            long long nd = 0;
            for (int k = 0; k < g.N; ++k)
                if (k != n) nd += g.dims[k];
            need = std::max(need, nd);
        }
        P.defer_cdf = (g.sampling == CPD_SAMPLE_EUCLIDEAN && need <= cap) ? 1 : 0;
    }
    if constexpr (sizeof(T) == 4) {
        if (c->engine == kEnginePersistent) {
            PersArgs &pa = c->pers;
            if (c->max_clusters < 1) return fail(CPD_ECUDA, "persistent engine: the cluster cannot be scheduled");
            for (int k = 0; k < g.N; ++k) {
                CK(dmalloc(c, &p, (size_t)g.dims[k] * pa.R4 * sizeof(float)));
                pa.Ap[k] = (float *)p;
            }
            CK(dmalloc(c, &p, (size_t)pa.cs * pa.ntile * 128 * pa.cst * sizeof(float)));
            pa.part = (float *)p;
            CK(dmalloc(c, &p, (size_t)pa.cs * 64 * 64 * sizeof(float)));
            pa.hpart = (float *)p;
            P.defer_cdf = 0;
        }
    }
    CK(dmalloc(c, &p, 16 * sizeof(unsigned)));  P.counters = (unsigned *)p;
    CK(dmalloc(c, &p, (size_t)fit_blocks() * sizeof(double)));  c->fit_partials = (double *)p;
    CK(dmalloc(c, &p, sizeof(double)));  c->fit_out = (double *)p;
    if constexpr (sizeof(T) == 4) {
        if (fit_tc_supported(P)) {
            CK(dmalloc(c, &p, fit_tc_scratch_bytes(P)));
            c->fit_tc = p;
        }
    }
    CK(cudaMemsetAsync(P.t_dev, 0, sizeof(long long), s));
    CK(cudaMemsetAsync(P.n_last, 0xff, sizeof(int), s));
    CK(cudaMemsetAsync(P.status, 0, sizeof(int), s));
    CK(cudaMemsetAsync(P.counters, 0, 16 * sizeof(unsigned), s));
    CK(cudaMemsetAsync(P.G, 0, (size_t)c->imax * g.R * sizeof(T), s));
    for (int k = 0; k < g.N; ++k) CK(launch_refresh_mode(P, k, s));
    CK(launch_fit(P, c->fit_partials, fit_blocks(), c->fit_out, s, 1));
    CK(cudaMemcpyAsync(&c->xnorm2, c->fit_out, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int st = 0;
    CK(cudaMemcpy(&st, P.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & kStDegenerate) return fail(CPD_EDEGENERATE, "a sampling distribution has no mass or a "
                                                         "leverage Gram matrix is singular");
    if (!(c->xnorm2 > 0.0)) return fail(CPD_EINVAL, "X is identically zero");
    return CPD_OK;
}

extern "C" cpd_status cpd_init(const cpd_config *cfg, const void *X, int x_loc, const void *const *A0,
                               int a0_loc, void *stream, cpd_ctx **out)
{
    cpd_status st = validate(cfg);
    if (st != CPD_OK) return st;
    if (!X || !A0 || !out) return fail(CPD_EINVAL, "NULL argument");
    for (int k = 0; k < cfg->N; ++k)
        if (!A0[k]) return fail(CPD_EINVAL, "NULL factor pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int cc_major = 0, cc_minor = 0;
    e = cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    if (cc_major != 10 || cc_minor != 3)
        return fail(CPD_ECUDA, "libcpd is built for sm_103a (GB300); this device is sm_" +
                                   std::to_string(cc_major) + std::to_string(cc_minor));
    cpd_ctx *c = new cpd_ctx();
    c->cfg = *cfg;
    c->device = dev;
    c->fbytes = cfg->x_dtype == CPD_F64 ? 8 : 4;
    c->xbytes = cfg->x_dtype == CPD_F64 ? 8 : (cfg->x_dtype == CPD_F32 ? 4 : 2);
    cudaStream_t s = (cudaStream_t)stream;
    c->home = s;
    st = c->fbytes == 8 ? init_typed<double>(c, X, x_loc, A0, a0_loc, s)
                        : init_typed<float>(c, X, x_loc, A0, a0_loc, s);
    if (st != CPD_OK) {
        cudaStreamSynchronize(s);
        free_all(c);
        delete c;
        return st;
    }
    *out = c;
    return CPD_OK;
}

template <class T>
static cudaError_t run_plain(cpd_ctx *c, int64_t iters, cudaStream_t s)
{
    Problem<T> &P = problem<T>(c);
    for (int64_t q = 0; q < iters; ++q) {
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
        if (c->profiling && c->prof_used < kProfSlots) {
            e0 = c->ev[3 * c->prof_used];
            e1 = c->ev[3 * c->prof_used + 1];
            e2 = c->ev[3 * c->prof_used + 2];
            ++c->prof_used;
            ++c->prof_iters;
        }
        cudaError_t e = launch_iteration(P, c->grid_grad, c->grid_upd, c->smem_grad, s, c->engine, e0, e1, e2);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Capture `len` launches of `launch(stream)` into an executable graph.
template <class F>
static cudaError_t capture_graph(cudaGraphExec_t *out, int len, F &&launch)
{
    cudaStream_t cap;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int q = 0; q < len && e == cudaSuccess; ++q) e = launch(cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(out, g, 0);
            cudaGraphDestroy(g);
        }
    }
    cudaStreamDestroy(cap);
    return e;
}

// `iters` iterations as replays: whole 32-iteration chunks, then one replay
// per set bit of the remainder (16, 8, 4, 2, 1). Graphs are captured on
// first use and kept while the caller's stream stays the same.
// With run = false only the missing graphs are captured (nothing executes).
template <class F>
static cudaError_t replay(cudaGraphExec_t *graphs, cudaStream_t &graph_stream, int64_t iters, cudaStream_t s,
                          F &&launch, bool run = true)
{
    if (graph_stream != s) {
        drop_graphs(graphs, kGraphSizes);
        graph_stream = s;
    }
    for (int q = 0; q < kGraphSizes; ++q) {
        const int len = kGraphChunk >> q;
        const int64_t reps = q == 0 ? iters / kGraphChunk : ((iters & len) ? 1 : 0);
        if (!reps) continue;
        if (!graphs[q]) {
            const cudaError_t e = capture_graph(&graphs[q], len, launch);
            if (e != cudaSuccess) return e;
        }
        for (int64_t r = 0; r < reps && run; ++r) {
            const cudaError_t e = cudaGraphLaunch(graphs[q], s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

template <class T>
static cudaError_t run_graph(cpd_ctx *c, int64_t iters, cudaStream_t s, bool run = true)
{
    Problem<T> &P = problem<T>(c);
    return replay(
        c->graph, c->graph_stream, iters, s,
        [&](cudaStream_t cap) {
            return launch_iteration(P, c->grid_grad, c->grid_upd, c->smem_grad, cap, c->engine, nullptr, nullptr,
                                    nullptr);
        },
        run);
}

extern "C" cpd_status cpd_prepare(cpd_ctx *c, int64_t iters, void *stream)
{
    if (!c || iters < 0) return fail(CPD_EINVAL, "bad context or iteration count");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->engine == kEnginePersistent) return CPD_OK;   // one launch per call, no graph
    const cudaError_t e = c->fbytes == 8 ? run_graph<double>(c, iters, s, false) : run_graph<float>(c, iters, s, false);
    if (e != cudaSuccess) return cuda_fail(e, "cpd_prepare capture");
    return CPD_OK;
}

// Persistent engine: launches of at most 2^20 iterations each (one cluster
// runs them back to back); profiled launches are bracketed by events.
static cudaError_t run_pers(cpd_ctx *c, int64_t iters, cudaStream_t s)
{
    constexpr int64_t kMaxPerLaunch = (int64_t)1 << 20;
    for (int64_t done = 0; done < iters;) {
        const int64_t T = std::min(kMaxPerLaunch, iters - done);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (c->profiling && c->prof_used < kProfSlots) {
            e0 = c->ev[3 * c->prof_used];
            e1 = c->ev[3 * c->prof_used + 1];
            ++c->prof_used;
            c->prof_iters += T;
        }
        c->pers.P = c->Pf;   // current pointers (trace buffer, ...)
        if (e0) cudaEventRecord(e0, s);
        cudaError_t e = launch_pers(c->pers, T, s);
        if (e1) {
            cudaEventRecord(e1, s);
            cudaEventRecord(c->ev[3 * (c->prof_used - 1) + 2], s);
        }
        if (e != cudaSuccess) return e;
        done += T;
    }
    return cudaSuccess;
}

extern "C" cpd_status cpd_gradients(cpd_ctx *c, int32_t n, int64_t t0, int32_t K, float *G_out, void *stream)
{
    if (!c || !G_out || K < 1 || t0 < 0) return fail(CPD_EINVAL, "bad argument");
    if (c->engine != kEnginePersistent) return fail(CPD_EINVAL, "cpd_gradients needs the persistent engine (4)");
    if (n < 0 || n >= c->cfg.N) return fail(CPD_EINVAL, "mode out of range");
    cudaStream_t s = (cudaStream_t)stream;
    PersArgs a = c->pers;
    a.P = c->Pf;
    const int ncl = std::max(1, std::min(K, c->max_clusters));
    if (ncl > c->gclusters) {   // scratch for ncl clusters, kept for later calls
        void *p1 = nullptr, *p2 = nullptr;
        CK(dmalloc(c, &p1, (size_t)ncl * a.cs * a.ntile * 128 * a.cst * sizeof(float)));
        CK(dmalloc(c, &p2, (size_t)ncl * a.cs * 64 * 64 * sizeof(float)));
        c->gpart = (float *)p1;
        c->ghpart = (float *)p2;
        c->gclusters = ncl;
    }
    a.part = c->gpart;
    a.hpart = c->ghpart;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profiling && c->prof_used < kProfSlots) {
        e0 = c->ev[3 * c->prof_used];
        e1 = c->ev[3 * c->prof_used + 1];
        ++c->prof_used;
        c->prof_iters += 1;
    }
    if (e0) cudaEventRecord(e0, s);
    const cudaError_t e = launch_pers_gradients(a, n, t0, K, ncl, G_out, s);
    if (e1) {
        cudaEventRecord(e1, s);
        cudaEventRecord(c->ev[3 * (c->prof_used - 1) + 2], s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cpd_gradients launch");
    return CPD_OK;
}

extern "C" cpd_status cpd_skrp(cpd_ctx *c, int32_t n, int64_t t0, int32_t K, int32_t *idx, double *p, float *Z,
                               void *X, void *stream)
{
    if (!c || K < 1 || t0 < 0) return fail(CPD_EINVAL, "bad argument");
    if (c->fbytes != 4) return fail(CPD_EINVAL, "cpd_skrp takes float factors (F32 or BF16 tensors)");
    if (c->Pf.strided) return fail(CPD_EINVAL, "cpd_skrp reads the mode-major replicas (x_layout 0)");
    if (c->Pf.block > 1) return fail(CPD_EINVAL, "cpd_skrp draws fibers one by one (block 0 or 1)");
    if (n < 0 || n >= c->cfg.N) return fail(CPD_EINVAL, "mode out of range");
    if ((double)K * c->cfg.B > 2.0e9) return fail(CPD_EINVAL, "K B too large");
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaError_t e = launch_flush_dirty(c->Pf, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profiling && c->prof_used < kProfSlots) {
        e0 = c->ev[3 * c->prof_used];
        e1 = c->ev[3 * c->prof_used + 1];
        ++c->prof_used;
        c->prof_iters += 1;
    }
    if (e == cudaSuccess && e0) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_skrp(c->Pf, n, t0, K, idx, p, Z, X, c->xbytes, sms, s);
    if (e == cudaSuccess && e1) {
        e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev[3 * (c->prof_used - 1) + 2], s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cpd_skrp launch");
    return CPD_OK;
}

extern "C" cpd_status cpd_sgd_iters(cpd_ctx *c, int64_t iters, void *stream)
{
    if (!c || iters < 0) return fail(CPD_EINVAL, "bad context or iteration count");
    if (iters == 0) return CPD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (c->engine == kEnginePersistent) {
        e = run_pers(c, iters, s);
    } else if (c->profiling) {
        e = c->fbytes == 8 ? run_plain<double>(c, iters, s) : run_plain<float>(c, iters, s);
    } else {
        e = c->fbytes == 8 ? run_graph<double>(c, iters, s) : run_graph<float>(c, iters, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cpd_sgd_iters launch");
    c->t_host += iters;
    c->has_sample = true;
    return CPD_OK;
}

static cpd_status read_status(cpd_ctx *c, cudaStream_t s)
{
    int *dst = c->fbytes == 8 ? c->Pd.status : c->Pf.status;
    int st = 0;
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(&st, dst, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) CK(cudaMemset(dst, 0, sizeof(int)));
    if (st & kStNonFinite) return fail(CPD_ENONFINITE, "a gradient or factor entry became NaN/Inf");
    if (st & kStDegenerate)
        return fail(CPD_EDEGENERATE, "a sampling distribution lost its mass or a Gram matrix is singular");
    if (st & kStTimeout) return fail(CPD_ETIMEOUT, "a bounded device wait gave up");
    return CPD_OK;
}

extern "C" cpd_status cpd_sync(cpd_ctx *c, void *stream)
{
    if (!c) return fail(CPD_EINVAL, "NULL context");
    return read_status(c, (cudaStream_t)stream);
}

// Tol's numerator into fit_out: on the tensor cores for BF16 tensors (float
// factors, R <= 64), else on CUDA cores.
static cudaError_t launch_tol(cpd_ctx *c, cudaStream_t s)
{
    if (c->fit_tc) return launch_fit_tc(c->Pf, c->fit_tc, c->fit_partials, c->sm_count, c->fit_out, s);
    return c->with_problem([&](auto &P) { return launch_fit(P, c->fit_partials, fit_blocks(), c->fit_out, s, 0); });
}

extern "C" cpd_status cpd_fit(cpd_ctx *c, double *fit, double *tol, void *stream)
{
    if (!c) return fail(CPD_EINVAL, "NULL context");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_tol(c, s);
    if (e != cudaSuccess) return cuda_fail(e, "fit launch");
    double res = 0.0;
    CK(cudaMemcpyAsync(&res, c->fit_out, sizeof(double), cudaMemcpyDeviceToHost, s));
    cpd_status st = read_status(c, s);
    const double tl = res / c->xnorm2;
    if (tol) *tol = tl;
    if (fit) *fit = 1.0 - std::sqrt(tl);
    return st;
}

extern "C" cpd_status cpd_fit_start(cpd_ctx *c, void *stream)
{
    if (!c) return fail(CPD_EINVAL, "NULL context");
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->fit_event) {
        CK(cudaEventCreateWithFlags(&c->fit_event, cudaEventDisableTiming));
        CK(cudaMallocHost((void **)&c->fit_host, 2 * sizeof(double)));   // residual, status word
    }
    cudaError_t e = launch_tol(c, s);
    if (e != cudaSuccess) return cuda_fail(e, "fit launch");
    CK(cudaMemcpyAsync(c->fit_host, c->fit_out, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->fit_host + 1, c->fbytes == 8 ? c->Pd.status : c->Pf.status, sizeof(int),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(c->fit_event, s));
    c->fit_started = true;
    return CPD_OK;
}

extern "C" cpd_status cpd_fit_poll(cpd_ctx *c, double *fit, double *tol)
{
    if (!c) return fail(CPD_EINVAL, "NULL context");
    if (!c->fit_started) return fail(CPD_EINVAL, "no fit was started");
    const cudaError_t q = cudaEventQuery(c->fit_event);
    if (q == cudaErrorNotReady) return CPD_EAGAIN;
    if (q != cudaSuccess) return cuda_fail(q, "fit event");
    const double tl = *c->fit_host / c->xnorm2;
    if (tol) *tol = tl;
    if (fit) *fit = 1.0 - std::sqrt(tl);
    int st = 0;
    std::memcpy(&st, c->fit_host + 1, sizeof(int));
    if (st & kStNonFinite) return fail(CPD_ENONFINITE, "a gradient or factor entry became NaN/Inf");
    if (st & kStDegenerate) return fail(CPD_EDEGENERATE, "a sampling distribution lost its mass");
    if (st & kStTimeout) return fail(CPD_ETIMEOUT, "a bounded device wait gave up");
    return CPD_OK;
}

static cudaMemcpyKind kind_out(int loc) { return loc == CPD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }
static cudaMemcpyKind kind_in(int loc) { return loc == CPD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }

extern "C" cpd_status cpd_get_factors(cpd_ctx *c, void *const *A, int loc, void *stream)
{
    if (!c || !A) return fail(CPD_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < c->cfg.N; ++k) {
        if (!A[k]) return fail(CPD_EINVAL, "NULL factor pointer");
        const void *src = c->fbytes == 8 ? (const void *)c->Pd.A[k] : (const void *)c->Pf.A[k];
        CK(cudaMemcpyAsync(A[k], src, (size_t)c->cfg.dims[k] * c->cfg.R * c->fbytes, kind_out(loc), s));
    }
    if (loc == CPD_HOST) CK(cudaStreamSynchronize(s));
    return CPD_OK;
}

extern "C" cpd_status cpd_set_factors(cpd_ctx *c, const void *const *A, int loc, void *stream)
{
    if (!c || !A) return fail(CPD_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < c->cfg.N; ++k) {
        if (!A[k]) return fail(CPD_EINVAL, "NULL factor pointer");
        void *dst = c->fbytes == 8 ? (void *)c->Pd.A[k] : (void *)c->Pf.A[k];
        CK(cudaMemcpyAsync(dst, A[k], (size_t)c->cfg.dims[k] * c->cfg.R * c->fbytes, kind_in(loc), s));
    }
    for (int k = 0; k < c->cfg.N; ++k) {
        cudaError_t e = c->with_problem([&](auto &P) { return launch_refresh_mode(P, k, s); });
        if (e != cudaSuccess) return cuda_fail(e, "distribution refresh");
    }
    CK(cudaMemsetAsync(c->fbytes == 8 ? c->Pd.dirty : c->Pf.dirty, 0xff, sizeof(int), s));   // all CDFs fresh
    return read_status(c, s);
}

extern "C" cpd_status cpd_get_adagrad(cpd_ctx *c, double *const *S, int loc, void *stream)
{
    if (!c || !S) return fail(CPD_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < c->cfg.N; ++k) {
        const double *src = c->fbytes == 8 ? c->Pd.S[k] : c->Pf.S[k];
        CK(cudaMemcpyAsync(S[k], src, (size_t)c->cfg.dims[k] * c->cfg.R * 8, kind_out(loc), s));
    }
    if (loc == CPD_HOST) CK(cudaStreamSynchronize(s));
    return CPD_OK;
}

extern "C" cpd_status cpd_set_adagrad(cpd_ctx *c, const double *const *S, int loc, void *stream)
{
    if (!c || !S) return fail(CPD_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < c->cfg.N; ++k) {
        double *dst = c->fbytes == 8 ? c->Pd.S[k] : c->Pf.S[k];
        CK(cudaMemcpyAsync(dst, S[k], (size_t)c->cfg.dims[k] * c->cfg.R * 8, kind_in(loc), s));
    }
    CK(cudaStreamSynchronize(s));
    return CPD_OK;
}

extern "C" cpd_status cpd_get_iteration(cpd_ctx *c, int64_t *t)
{
    if (!c || !t) return fail(CPD_EINVAL, "NULL argument");
    *t = c->t_host;
    return CPD_OK;
}

extern "C" cpd_status cpd_set_iteration(cpd_ctx *c, int64_t t)
{
    if (!c || t < 0) return fail(CPD_EINVAL, "bad argument");
    long long v = (long long)t;
    long long *dst = c->fbytes == 8 ? c->Pd.t_dev : c->Pf.t_dev;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(dst, &v, sizeof v, cudaMemcpyHostToDevice));
    c->t_host = t;
    c->has_sample = false;
    return CPD_OK;
}

extern "C" cpd_status cpd_last_sample(cpd_ctx *c, int32_t *n, int32_t *idx, double *p, void *stream)
{
    if (!c) return fail(CPD_EINVAL, "NULL context");
    if (!c->has_sample) return fail(CPD_EINVAL, "no iteration has run since the counter was set");
    cudaStream_t s = (cudaStream_t)stream;
    const bool d = c->fbytes == 8;
    if (n) CK(cudaMemcpyAsync(n, d ? c->Pd.n_last : c->Pf.n_last, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (idx)
        CK(cudaMemcpyAsync(idx, d ? c->Pd.idx : c->Pf.idx, (size_t)c->cfg.B * c->cfg.N * sizeof(int),
                           cudaMemcpyDeviceToHost, s));
    if (p) {
        // p_f is formed on demand from the recorded batch (off the iteration path)
        const cudaError_t e = d ? launch_sample_probs(c->Pd, s) : launch_sample_probs(c->Pf, s);
        if (e != cudaSuccess) return cuda_fail(e, "sample probabilities");
        CK(cudaMemcpyAsync(p, d ? c->Pd.p : c->Pf.p, (size_t)c->cfg.B * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return CPD_OK;
}

extern "C" cpd_status cpd_last_gradient(cpd_ctx *c, void *G, void *stream)
{
    if (!c || !G) return fail(CPD_EINVAL, "NULL argument");
    if (!c->has_sample) return fail(CPD_EINVAL, "no iteration has run since the counter was set");
    cudaStream_t s = (cudaStream_t)stream;
    int n = 0;
    const bool d = c->fbytes == 8;
    CK(cudaMemcpyAsync(&n, d ? c->Pd.n_last : c->Pf.n_last, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (n < 0 || n >= c->cfg.N) return fail(CPD_EINVAL, "no completed iteration");
    const void *src = d ? (const void *)c->Pd.G : (const void *)c->Pf.G;
    CK(cudaMemcpyAsync(G, src, (size_t)c->cfg.dims[n] * c->cfg.R * c->fbytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return CPD_OK;
}

extern "C" cpd_status cpd_profile(cpd_ctx *c, int enable)
{
    if (!c) return fail(CPD_EINVAL, "NULL context");
    if (enable && c->ev.empty()) {
        c->ev.resize(3 * kProfSlots);
        for (auto &e : c->ev) CK(cudaEventCreate(&e));
    }
    c->profiling = enable != 0;
    c->prof_used = 0;
    c->prof_iters = 0;
    return CPD_OK;
}

extern "C" cpd_status cpd_profile_read(cpd_ctx *c, int64_t *launches, double *mean_grad_ms,
                                       double *mean_update_ms, void *stream)
{
    if (!c) return fail(CPD_EINVAL, "NULL context");
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    double tg = 0.0, tu = 0.0;
    for (int q = 0; q < c->prof_used; ++q) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[3 * q], c->ev[3 * q + 1]));
        tg += ms;
        CK(cudaEventElapsedTime(&ms, c->ev[3 * q + 1], c->ev[3 * q + 2]));
        tu += ms;
    }
    // per iteration: a persistent launch covers many iterations (its whole
    // time counts as the gradient part)
    if (launches) *launches = c->prof_iters;
    if (mean_grad_ms) *mean_grad_ms = c->prof_iters ? tg / c->prof_iters : 0.0;
    if (mean_update_ms) *mean_update_ms = c->prof_iters ? tu / c->prof_iters : 0.0;
    return CPD_OK;
}

extern "C" cpd_status cpd_trace(cpd_ctx *c, int enable)
{
    if (!c) return fail(CPD_EINVAL, "NULL context");
    unsigned long long *&tr = c->fbytes == 8 ? c->Pd.trace : c->Pf.trace;
    if (enable && !c->trace_buf) {
        void *p;
        CK(dmalloc(c, &p, 64 * sizeof(unsigned long long)));
        CK(cudaMemset(p, 0, 64 * sizeof(unsigned long long)));
        c->trace_buf = (unsigned long long *)p;
    }
    tr = enable ? c->trace_buf : nullptr;
    drop_graphs(c->graph, kGraphSizes);   // captured launches carry the old pointer
    return CPD_OK;
}

extern "C" cpd_status cpd_trace_read(cpd_ctx *c, uint64_t *out, void *stream)
{
    if (!c || !out) return fail(CPD_EINVAL, "bad argument");
    if (!c->trace_buf) return fail(CPD_EINVAL, "tracing was never enabled");
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    CK(cudaMemcpy(out, c->trace_buf, 64 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    return CPD_OK;
}

extern "C" cpd_status cpd_describe(cpd_ctx *c, char *buf, size_t len)
{
    if (!c || !buf || len == 0) return fail(CPD_EINVAL, "bad argument");
    const int rb = c->fbytes == 8 ? c->Pd.rb : c->Pf.rb;
    const int fb = c->fbytes == 8 ? c->Pd.fb : c->Pf.fb;
    const int pf = c->fbytes == 8 ? c->Pd.pf : c->Pf.pf;
    std::snprintf(buf, len,
                  "{\"engine\": \"%s\", \"rows_per_cta\": %d, \"fibers_per_cta\": %d, \"fiber_groups\": %d, "
                  "\"grad_grid\": %d, \"update_grid\": %d, \"grad_smem\": %zu, \"graph_chunk\": %d, "
                  "\"cluster\": %d, \"max_clusters\": %d, \"deferred_cdf\": %d, "
                  "\"fit_pass\": \"%s\", \"x_layout\": \"%s\", \"block\": %d, \"xnorm2\": %.17g}",
                  c->engine == kEnginePersistent       ? "persistent"
                  : c->engine == kEngineFused         ? "fused"
                  : c->engine == kEngineTensorCluster ? "cluster"
                  : c->engine == kEngineTensor        ? "tensor"
                                                      : "simt",
                  rb, fb, pf, c->grid_grad, c->grid_upd,
                  c->smem_grad, kGraphChunk, c->fbytes == 8 ? 1 : c->Pf.cs, c->max_clusters,
                  c->fbytes == 8 ? c->Pd.defer_cdf : c->Pf.defer_cdf, c->fit_tc ? "tensor" : "cuda_cores",
                  (c->fbytes == 8 ? c->Pd.strided : c->Pf.strided) ? "strided" : "replicas",
                  c->fbytes == 8 ? c->Pd.block : c->Pf.block, c->xnorm2);
    return CPD_OK;
}

extern "C" cpd_status cpd_destroy(cpd_ctx *c)
{
    if (!c) return CPD_OK;
    cudaDeviceSynchronize();
    free_all(c);
    delete c;
    return CPD_OK;
}

// Destroy without a device-wide synchronisation: the caller guarantees that
// all of the context's work was enqueued on its home stream (the server).
namespace cpd {
void destroy_on_home_stream(cpd_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->home);
    free_all(c);
    delete c;
}
}  // namespace cpd

extern "C" const char *cpd_last_error(void) { return g_err.c_str(); }

namespace cpd {
void set_error(const std::string &msg) { g_err = msg; }
int ctx_engine(const cpd_ctx *c) { return c->engine; }
int ctx_cluster(const cpd_ctx *c) { return c->engine == kEnginePersistent ? c->pers.cs : 0; }
}  // namespace cpd

// ---------------------------------------------------------------------------
// Groups: many contexts advanced by one gradient launch and one update
// launch per iteration (each member runs exactly its own CTAs and arithmetic).
// ---------------------------------------------------------------------------
struct cpd_group {
    int fbytes = 4, x_dtype = 0, engine = 0, G = 0;
    std::vector<cpd_ctx *> members;
    void *dP = nullptr;      // device array of the members' Problem structs
    int *dcta = nullptr;     // cta_grad[G + 1] followed by cta_upd[G + 1]
    GroupLaunch<float> Lf{};
    GroupLaunch<double> Ld{};
    cudaStream_t home = nullptr;          // stream of creation: allocation and free
    cudaGraphExec_t graph[kGraphSizes] = {};
    cudaStream_t graph_stream = nullptr;
    cudaStream_t last = nullptr;          // last stream work was enqueued on
    // persistent members: one cluster each, in one launch per call
    PersArgs *dpers = nullptr;
    int pers_cs = 0;
    size_t pers_smem = 0;
};

template <class T>
static GroupLaunch<T> &group_launch(cpd_group *g);
template <>
GroupLaunch<float> &group_launch<float>(cpd_group *g) { return g->Lf; }
template <>
GroupLaunch<double> &group_launch<double>(cpd_group *g) { return g->Ld; }

template <class T>
static cpd_status group_build(cpd_group *g, cudaStream_t s)
{
    std::vector<Problem<T>> hp(g->G);
    const int G1 = g->G + 1;
    std::vector<int> cta(4 * G1, 0);   // gradient, update, Gram, leverage-row CTAs
    size_t smem = 0, smem_lev = 0;
    for (int q = 0; q < g->G; ++q) {
        cpd_ctx *c = g->members[q];
        hp[q] = problem<T>(c);
        cta[q + 1] = cta[q] + c->grid_grad;
        cta[G1 + q + 1] = cta[G1 + q] + c->grid_upd;
        int gram = 0, lev = 0;
        if (c->cfg.sampling == CPD_SAMPLE_LEVERAGE) {   // the grids launch_iteration uses
            gram = (c->cfg.R * (c->cfg.R + 1) / 2 + 7) / 8;
            lev = (int)((c->imax * 32 + kThreads - 1) / kThreads);
            smem_lev = std::max(smem_lev, lev_smem(c->cfg.R));
        }
        cta[2 * G1 + q + 1] = cta[2 * G1 + q] + gram;
        cta[3 * G1 + q + 1] = cta[3 * G1 + q] + lev;
        smem = std::max(smem, c->smem_grad);
    }
    CK(cudaMallocAsync(&g->dP, sizeof(Problem<T>) * g->G, s));
    CK(cudaMallocAsync((void **)&g->dcta, sizeof(int) * cta.size(), s));
    CK(cudaMemcpyAsync(g->dP, hp.data(), sizeof(Problem<T>) * g->G, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(g->dcta, cta.data(), sizeof(int) * cta.size(), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));   // the host staging vectors go out of scope
    GroupLaunch<T> L{};
    L.P = (const Problem<T> *)g->dP;
    L.cta_grad = g->dcta;
    L.cta_upd = g->dcta + G1;
    L.cta_gram = g->dcta + 2 * G1;
    L.cta_lev = g->dcta + 3 * G1;
    L.G = g->G;
    L.grid_grad = cta[g->G];
    L.grid_upd = cta[G1 + g->G];
    L.grid_gram = cta[2 * G1 + g->G];
    L.grid_lev = cta[3 * G1 + g->G];
    L.smem_lev = smem_lev;
    L.engine = g->engine;
    L.x_dtype = g->x_dtype;
    L.smem_grad = smem;
    group_launch<T>(g) = L;
    return CPD_OK;
}

extern "C" cpd_status cpd_group_create(cpd_ctx *const *ctxs, int32_t G, void *stream, cpd_group **out)
{
    if (!ctxs || !out || G < 1) return fail(CPD_EINVAL, "NULL argument or empty group");
    cpd_ctx *c0 = ctxs[0];
    if (!c0) return fail(CPD_EINVAL, "NULL context");
    for (int q = 0; q < G; ++q) {
        cpd_ctx *c = ctxs[q];
        if (!c) return fail(CPD_EINVAL, "NULL context");
        for (int r = 0; r < q; ++r)
            if (ctxs[r] == c) return fail(CPD_EINVAL, "a context appears twice in the group");
        if (c->engine != kEngineSimt && c->engine != kEngineTensor && c->engine != kEnginePersistent)
            return fail(CPD_EINVAL, "grouped launches take CUDA-core, per-CTA tensor-core or persistent contexts");
        if (c->engine == kEnginePersistent && c->pers.cs != c0->pers.cs)
            return fail(CPD_EINVAL, "persistent group members must share the cluster size");
        if (c->engine == kEnginePersistent && c->cfg.sampling == CPD_SAMPLE_LEVERAGE)
            return fail(CPD_EINVAL, "persistent group members do not sample by leverage");
        if (c->fbytes != c0->fbytes || c->cfg.x_dtype != c0->cfg.x_dtype || c->engine != c0->engine ||
            c->device != c0->device)
            return fail(CPD_EINVAL, "group members differ in tensor dtype, engine or device");
    }
    auto *g = new cpd_group();
    g->fbytes = c0->fbytes;
    g->x_dtype = c0->cfg.x_dtype;
    g->engine = c0->engine;
    g->G = G;
    g->members.assign(ctxs, ctxs + G);
    g->home = (cudaStream_t)stream;
    g->last = g->home;
    cpd_status st;
    if (g->engine == kEnginePersistent) {
        // the members' launch arguments, captured now (like the other groups)
        std::vector<PersArgs> hp(G);
        g->pers_cs = c0->pers.cs;
        for (int q = 0; q < G; ++q) {
            hp[q] = ctxs[q]->pers;
            hp[q].P = ctxs[q]->Pf;
            g->pers_smem = std::max(g->pers_smem, ctxs[q]->smem_grad);
        }
        cudaError_t e = cudaMallocAsync((void **)&g->dpers, sizeof(PersArgs) * G, g->home);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->dpers, hp.data(), sizeof(PersArgs) * G, cudaMemcpyHostToDevice, g->home);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->home);
        st = e == cudaSuccess ? CPD_OK : cuda_fail(e, "persistent group set-up");
    } else {
        st = g->fbytes == 8 ? group_build<double>(g, g->home) : group_build<float>(g, g->home);
    }
    if (st != CPD_OK) {
        cudaStreamSynchronize(g->home);
        if (g->dP) cudaFreeAsync(g->dP, g->home);
        if (g->dcta) cudaFreeAsync(g->dcta, g->home);
        if (g->dpers) cudaFreeAsync(g->dpers, g->home);
        cudaStreamSynchronize(g->home);
        delete g;
        return st;
    }
    *out = g;
    return CPD_OK;
}

template <class T>
static cudaError_t group_run(cpd_group *g, int64_t iters, cudaStream_t s)
{
    if (g->engine == kEnginePersistent) {
        constexpr int64_t kMaxPerLaunch = (int64_t)1 << 20;
        for (int64_t done = 0; done < iters;) {
            const int64_t len = std::min(kMaxPerLaunch, iters - done);
            const cudaError_t e = launch_pers_group(g->dpers, g->G, g->pers_cs, g->pers_smem, len, s);
            if (e != cudaSuccess) return e;
            done += len;
        }
        return cudaSuccess;
    }
    const GroupLaunch<T> &L = group_launch<T>(g);
    return replay(g->graph, g->graph_stream, iters, s, [&](cudaStream_t cap) { return launch_group_iteration(L, cap); });
}

extern "C" cpd_status cpd_group_iters(cpd_group *g, int64_t iters, void *stream)
{
    if (!g || iters < 0) return fail(CPD_EINVAL, "bad group or iteration count");
    if (iters == 0) return CPD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const cudaError_t e = g->fbytes == 8 ? group_run<double>(g, iters, s) : group_run<float>(g, iters, s);
    if (e != cudaSuccess) return cuda_fail(e, "cpd_group_iters launch");
    g->last = s;
    for (cpd_ctx *c : g->members) {
        c->t_host += iters;
        c->has_sample = true;
    }
    return CPD_OK;
}

extern "C" cpd_status cpd_group_destroy(cpd_group *g)
{
    if (!g) return CPD_OK;
    cudaStreamSynchronize(g->last);
    drop_graphs(g->graph, kGraphSizes);
    if (g->dP) cudaFreeAsync(g->dP, g->home);
    if (g->dcta) cudaFreeAsync(g->dcta, g->home);
    if (g->dpers) cudaFreeAsync(g->dpers, g->home);
    cudaStreamSynchronize(g->home);
    delete g;
    return CPD_OK;
}

// ---------------------------------------------------------------------------
// Gradient-variance diagnostic (Thm 10, Table 1, Fig. 3).
// ---------------------------------------------------------------------------
template <class T>
static cpd_status variance_typed(cpd_ctx *c, int n, double *var, double *mean_norm2, cudaStream_t s)
{
    Problem<T> &P = problem<T>(c);
    double *d2 = nullptr;
    CK(cudaMallocAsync((void **)&d2, 2 * sizeof(double), s));
    cudaError_t e = launch_flush_dirty(P, s);
    if (e == cudaSuccess) e = launch_variance(P, n, d2, s);
    double h2[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h2, d2, sizeof h2, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d2, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "cpd_grad_variance");
    int st = 0;
    CK(cudaMemcpy(&st, P.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & kStDegenerate) return fail(CPD_EDEGENERATE, "a sampling distribution has no mass");
    const double J = P.Jn[n];
    *var = (h2[0] - h2[1]) / ((double)c->cfg.B * J * J);
    if (mean_norm2) *mean_norm2 = h2[1] / (J * J);
    return CPD_OK;
}

extern "C" cpd_status cpd_grad_variance(cpd_ctx *c, int32_t n, double *var, double *mean_norm2, void *stream)
{
    if (!c || !var) return fail(CPD_EINVAL, "NULL argument");
    if (n < 0 || n >= c->cfg.N) return fail(CPD_EINVAL, "mode out of range");
    if (c->cfg.R > 64) return fail(CPD_EINVAL, "the variance diagnostic takes R <= 64");
    if (c->cfg.block > 1) return fail(CPD_EINVAL, "the variance diagnostic enumerates single fibers (block 0 or 1)");
    cudaStream_t s = (cudaStream_t)stream;
    return c->fbytes == 8 ? variance_typed<double>(c, n, var, mean_norm2, s)
                          : variance_typed<float>(c, n, var, mean_norm2, s);
}

// ---------------------------------------------------------------------------
// Autotuner: time candidate gradient engines and CTA caps on the caller's
// problem and return the fastest configuration.
// ---------------------------------------------------------------------------
extern "C" cpd_status cpd_autotune(const cpd_config *cfg, const void *X, int x_loc, const void *const *A0,
                                   int a0_loc, int64_t iters, cpd_config *best, double *best_iters_per_s,
                                   void *stream)
{
    cpd_status st = validate(cfg);
    if (st != CPD_OK) return st;
    if (!X || !A0 || !best || iters < 1) return fail(CPD_EINVAL, "NULL argument or iters < 1");
    int64_t imax = 0;
    for (int k = 0; k < cfg->N; ++k) imax = std::max<int64_t>(imax, cfg->dims[k]);
    const bool tc_ok = cfg->x_dtype == CPD_BF16 && tc_supported(cfg->R, 128);
    const int cs = (int)((imax + 127) / 128);
    // candidates: (engine, max_ctas, tile_rows, tile_fibers); 0 = the tile
    // chooser's own choice for that cap
    struct Cand {
        int engine, max_ctas, rows, fibers;
    };
    std::vector<Cand> cand;
    const bool fixed = cfg->engine != 0;
    auto want = [&](int e) { return !fixed || cfg->engine == e; };
    if (want(kEngineSimt))
        for (int mc : {0, 16, 64})
            for (int rows : {0, 32, 128})
                for (int fib : {0, 32})
                    if (fib <= cfg->B) cand.push_back({kEngineSimt, fixed ? cfg->max_ctas : mc, rows, fib});
    if (tc_ok && cfg->x_layout == CPD_LAYOUT_REPLICAS) {
        if (want(kEngineTensor))
            for (int mc : {0, 16, 64})
                for (int fib : {0, 32, 64})
                    if (fib <= cfg->B) cand.push_back({kEngineTensor, fixed ? cfg->max_ctas : mc, 0, fib});
        if (cs <= 8 && want(kEngineTensorCluster))
            for (int m : {0, 4, 8, 12})
                for (int fib : {0, 64, 128})
                    if (fib <= cfg->B)
                        cand.push_back({kEngineTensorCluster, fixed ? cfg->max_ctas : m * cs, 0, fib});
    }
    if (tc_ok && cfg->x_layout == CPD_LAYOUT_REPLICAS && want(kEngineFused))
        for (int fcs : {4, 8, 16})
            if (fused_fits(cfg->N, cfg->R, cfg->B, fixed ? cfg->max_ctas : fcs, 1))
                cand.push_back({kEngineFused, fixed ? cfg->max_ctas : fcs, 0, 0});
    if (pers_supported(*cfg) && cfg->x_layout == CPD_LAYOUT_REPLICAS && want(kEnginePersistent))
        for (int mc : {2, 4, 8, 16}) cand.push_back({kEnginePersistent, fixed ? cfg->max_ctas : mc, 0, 0});
    if (cand.empty()) cand.push_back({cfg->engine, cfg->max_ctas, cfg->tile_rows, cfg->tile_fibers});
    // a fixed engine and cap repeat across the caps' loop: keep one of each
    std::vector<Cand> uniq;
    for (const Cand &c : cand) {
        bool dup = false;
        for (const Cand &u : uniq)
            dup = dup || (u.engine == c.engine && u.max_ctas == c.max_ctas && u.rows == c.rows && u.fibers == c.fibers);
        if (!dup) uniq.push_back(c);
    }
    cand.swap(uniq);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best_rate = -1.0;
    cpd_config chosen = *cfg;
    for (const auto &c : cand) {
        cpd_config trial = *cfg;
        trial.engine = c.engine;
        trial.max_ctas = c.max_ctas;
        trial.tile_rows = c.rows;
        trial.tile_fibers = c.fibers;
        cpd_ctx *ctx = nullptr;
        if (cpd_init(&trial, X, x_loc, A0, a0_loc, stream, &ctx) != CPD_OK) continue;   // not applicable
        float ms = 0.f;
        bool ok = cpd_sgd_iters(ctx, std::max<int64_t>(1, iters / 4), stream) == CPD_OK &&
                  cudaEventRecord(e0, s) == cudaSuccess && cpd_sgd_iters(ctx, iters, stream) == CPD_OK &&
                  cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (ok) ok = read_status(ctx, s) == CPD_OK;
        cpd_destroy(ctx);
        if (!ok || !(ms > 0.f)) continue;
        const double rate = (double)iters / (ms * 1e-3);
        if (rate > best_rate) {
            best_rate = rate;
            chosen = trial;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_rate < 0.0) return fail(CPD_ECUDA, "no candidate configuration ran");
    *best = chosen;
    if (best_iters_per_s) *best_iters_per_s = best_rate;
    return CPD_OK;
}
