// Serving loop of libcpd (declared in include/cpd.h): many decompositions on
// one GPU, admitted by a device-memory budget.
//
// One worker thread owns all device work. Per round it
//   1. admits queued requests first-fit while the memory budget and the
//      concurrency limit allow (cpd_init on a fresh non-blocking stream);
//   2. steps the lanes: requests of one class (tensor dtype and engine; for
//      the persistent engine also the cluster size)
//      share a lane whose rounds advance all members with grouped launches
//      (one gradient and one update launch per iteration for the whole
//      lane, or one launch per round for persistent members), then start
//      every member's fit; members leave and join between rounds. Four lanes per class overlap one lane's fits and
//      host work with the others' iterations;
//   3. steps the requests that cannot be grouped, each on its own stream:
//      iterations up to its next check and an asynchronous fit, so every
//      stream has a bounded amount of queued work and the streams overlap;
//   4. retires requests whose check met the target or whose cap is reached:
//      factors copied out, context freed with stream-ordered frees.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cpd.h"
#include "cpd_internal.h"

namespace cpd {
void set_error(const std::string &msg);
void destroy_on_home_stream(cpd_ctx *c);
int ctx_engine(const cpd_ctx *c);
int ctx_cluster(const cpd_ctx *c);
}  // namespace cpd

using namespace cpd;

namespace {

double now_s()
{
    using clk = std::chrono::steady_clock;
    static const clk::time_point t0 = clk::now();
    return std::chrono::duration<double>(clk::now() - t0).count();
}

// Device bytes of a request's copy of X: the mode-major replicas, or the
// single strided copy.
double tensor_bytes(const cpd_config &g)
{
    const double xb = g.x_dtype == CPD_F64 ? 8 : (g.x_dtype == CPD_F32 ? 4 : 2);
    double total = 1.0;
    for (int k = 0; k < g.N; ++k) total *= (double)g.dims[k];
    if (g.x_layout == CPD_LAYOUT_STRIDED)   // the mode-1 replica alone
        return total / (double)g.dims[0] * (double)((g.dims[0] + 7) / 8 * 8) * xb;
    double bytes = 0.0;
    for (int k = 0; k < g.N; ++k) bytes += total / (double)g.dims[k] * (double)((g.dims[k] + 7) / 8 * 8) * xb;
    return bytes;
}

// Device bytes a request may hold: its copy of X, factors and their state,
// the gradient partials (upper bound) and a fixed allowance.
size_t estimate_bytes(const cpd_config &g)
{
    const size_t fb = g.x_dtype == CPD_F64 ? 8 : 4;
    int64_t imax = 0, isum = 0;
    for (int k = 0; k < g.N; ++k) {
        imax = std::max<int64_t>(imax, g.dims[k]);
        isum += g.dims[k];
    }
    double bytes = tensor_bytes(g);
    bytes += (double)isum * g.R * (fb + 8) + (double)isum * 16;
    bytes += 608.0 * g.R * (double)imax * fb;   // partial slabs, bound of the tile chooser
    bytes += 8.0 * 1024 * 1024;
    return (size_t)bytes;
}

struct Request {
    uint64_t ticket = 0;
    cpd_config cfg{};
    const void *X = nullptr;
    int x_loc = 0;
    std::vector<const void *> A0;
    int a0_loc = 0;
    double stop_fit = 1.0;
    int64_t max_iters = 0;
    size_t bytes = 0;
    cpd_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    bool fit_pending = false;
    int64_t next_check = 0;
    cpd_result res{};
    std::vector<std::vector<unsigned char>> factors;
};

}  // namespace

// A lane advances a set of same-class requests (same tensor dtype and
// engine) with grouped launches on its own stream: rounds of `chunk`
// iterations of every member, then every member's asynchronous fit, then an
// event. Members join and leave between rounds.
struct Lane {
    int fbytes = 4, x_dtype = 0, engine = 0, cluster = 0;
    std::vector<std::shared_ptr<Request>> members, joining;
    cpd_group *grp = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false, changed = false;
};

constexpr int kLanesPerClass = 4;

struct cpd_server {
    cpd_server_config cfg{};
    int device = 0;
    size_t budget = 0, used = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> active;   // requests on streams of their own
    std::vector<std::unique_ptr<Lane>> lanes;
    size_t running = 0;                             // admitted and not finished
    std::map<uint64_t, std::shared_ptr<Request>> all;
    size_t unfinished = 0;
    std::thread worker;
};

static void finish(cpd_server *srv, const std::shared_ptr<Request> &r, cpd_status st)
{
    if (r->ctx) {
        if (st == CPD_OK) {
            std::vector<void *> ptrs;
            const size_t fbytes = r->cfg.x_dtype == CPD_F64 ? 8 : 4;
            r->factors.resize(r->cfg.N);
            for (int k = 0; k < r->cfg.N; ++k) {
                r->factors[k].resize((size_t)r->cfg.dims[k] * r->cfg.R * fbytes);
                ptrs.push_back(r->factors[k].data());
            }
            const cpd_status g = cpd_get_factors(r->ctx, ptrs.data(), CPD_HOST, r->stream);
            if (g != CPD_OK) st = g;
        }
        destroy_on_home_stream(r->ctx);
        r->ctx = nullptr;
    }
    if (r->stream) {
        cudaStreamDestroy(r->stream);
        r->stream = nullptr;
    }
    std::lock_guard<std::mutex> lock(srv->mu);
    r->res.status = st;
    r->res.t_done = now_s();
    r->res.done = 1;
    srv->used -= r->bytes;
    --srv->running;
    --srv->unfinished;
    srv->cv_done.notify_all();
}

// The outcome of a finished fit check: true if the request stops. The
// result fields change under the server's lock (cpd_poll reads them).
static bool after_fit(cpd_server *srv, const std::shared_ptr<Request> &r, cpd_status st, double fit, double tol,
                      cpd_status *why)
{
    std::lock_guard<std::mutex> lock(srv->mu);
    r->res.fit = fit;
    r->res.tol = tol;
    *why = st;
    if (st != CPD_OK) return true;
    if (fit >= r->stop_fit) {
        r->res.reached = 1;
        return true;
    }
    return r->res.iters >= r->max_iters;
}

static void add_iters(cpd_server *srv, const std::shared_ptr<Request> &r, int64_t n)
{
    std::lock_guard<std::mutex> lock(srv->mu);
    r->res.iters += n;
}

static Lane *pick_lane(cpd_server *srv, const std::shared_ptr<Request> &r, int engine)
{
    const int fbytes = r->cfg.x_dtype == CPD_F64 ? 8 : 4;
    const int cluster = engine == kEnginePersistent ? ctx_cluster(r->ctx) : 0;
    Lane *best = nullptr;
    int found = 0;
    for (auto &l : srv->lanes) {
        if (l->fbytes != fbytes || l->x_dtype != r->cfg.x_dtype || l->engine != engine || l->cluster != cluster)
            continue;
        ++found;
        if (!best || l->members.size() + l->joining.size() < best->members.size() + best->joining.size())
            best = l.get();
    }
    if (found < kLanesPerClass && (!best || !best->members.empty() || !best->joining.empty())) {
        auto l = std::make_unique<Lane>();
        l->fbytes = fbytes;
        l->x_dtype = r->cfg.x_dtype;
        l->engine = engine;
        l->cluster = cluster;
        if (cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        if (cudaEventCreateWithFlags(&l->done, cudaEventDisableTiming) != cudaSuccess) {
            cudaStreamDestroy(l->stream);
            return nullptr;
        }
        best = l.get();
        srv->lanes.push_back(std::move(l));
    }
    return best;
}

// One scheduling step of a lane; returns true if it changed anything.
static bool step_lane(cpd_server *srv, Lane &l, int fit_every)
{
    if (l.busy) {
        if (cudaEventQuery(l.done) == cudaErrorNotReady) return false;
        l.busy = false;
        for (size_t q = 0; q < l.members.size();) {
            auto m = l.members[q];
            double fit = 0.0, tol = 0.0;
            cpd_status st = cpd_fit_poll(m->ctx, &fit, &tol);
            cpd_status why = CPD_OK;
            if (after_fit(srv, m, st, fit, tol, &why)) {
                finish(srv, m, why);
                l.members.erase(l.members.begin() + q);
                l.changed = true;
            } else {
                ++q;
            }
        }
    }
    if (!l.joining.empty()) {
        l.members.insert(l.members.end(), l.joining.begin(), l.joining.end());
        l.joining.clear();
        l.changed = true;
    }
    if (l.changed && l.grp) {
        cpd_group_destroy(l.grp);
        l.grp = nullptr;
    }
    if (l.members.empty()) {
        l.changed = false;
        return true;
    }
    cpd_status st = CPD_OK;
    if (!l.grp) {
        std::vector<cpd_ctx *> ctxs;
        for (auto &m : l.members) ctxs.push_back(m->ctx);
        st = cpd_group_create(ctxs.data(), (int32_t)ctxs.size(), l.stream, &l.grp);
        l.changed = false;
    }
    int64_t chunk = fit_every;
    for (auto &m : l.members) chunk = std::min<int64_t>(chunk, m->max_iters - m->res.iters);
    if (st == CPD_OK) st = cpd_group_iters(l.grp, chunk, l.stream);
    for (size_t q = 0; q < l.members.size() && st == CPD_OK; ++q) st = cpd_fit_start(l.members[q]->ctx, l.stream);
    if (st == CPD_OK && cudaEventRecord(l.done, l.stream) != cudaSuccess) st = CPD_ECUDA;
    if (st != CPD_OK) {
        cudaStreamSynchronize(l.stream);
        if (l.grp) cpd_group_destroy(l.grp);
        l.grp = nullptr;
        for (auto &m : l.members) finish(srv, m, st);
        l.members.clear();
        return true;
    }
    for (auto &m : l.members) add_iters(srv, m, chunk);
    l.busy = true;
    return true;
}

static void worker_loop(cpd_server *srv)
{
    cudaSetDevice(srv->device);
    const int fit_every = srv->cfg.fit_every > 0 ? srv->cfg.fit_every : 250;
    const size_t max_active = srv->cfg.max_active > 0 ? (size_t)srv->cfg.max_active : 32;
    for (;;) {
        // 1. admission (first fit in submission order)
        std::vector<std::shared_ptr<Request>> admit;
        {
            std::unique_lock<std::mutex> lock(srv->mu);
            if (srv->stop) break;
            if (srv->queue.empty() && srv->running == 0)
                srv->cv_work.wait(lock, [&] { return srv->stop || !srv->queue.empty(); });
            if (srv->stop) break;
            for (auto it = srv->queue.begin(); it != srv->queue.end() && srv->running < max_active;) {
                if (srv->used + (*it)->bytes <= srv->budget) {
                    srv->used += (*it)->bytes;
                    ++srv->running;
                    admit.push_back(*it);
                    it = srv->queue.erase(it);
                } else {
                    ++it;
                }
            }
        }
        for (auto &r : admit) {
            cpd_status st = CPD_OK;
            if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) st = CPD_ECUDA;
            if (st == CPD_OK) st = cpd_init(&r->cfg, r->X, r->x_loc, r->A0.data(), r->a0_loc, r->stream, &r->ctx);
            {
                // cpd_init has copied X and A0 (it synchronises its stream):
                // from here on the caller may release them
                std::lock_guard<std::mutex> lock(srv->mu);
                r->res.t_start = now_s();
            }
            if (st != CPD_OK) {
                finish(srv, r, st);
                continue;
            }
            const int engine = ctx_engine(r->ctx);
            const bool groupable = !srv->cfg.no_grouping &&
                                   (engine == kEngineSimt || engine == kEngineTensor || engine == kEnginePersistent);
            Lane *lane = groupable ? pick_lane(srv, r, engine) : nullptr;
            if (lane) {
                lane->joining.push_back(r);
            } else {
                r->next_check = std::min<int64_t>(fit_every, r->max_iters);
                srv->active.push_back(r);
            }
        }
        bool progressed = !admit.empty();
        // 2. lanes of grouped requests
        for (auto &l : srv->lanes) progressed |= step_lane(srv, *l, fit_every);
        // 3. requests on streams of their own
        for (size_t q = 0; q < srv->active.size();) {
            auto r = srv->active[q];
            bool retire = false;
            cpd_status st = CPD_OK;
            if (r->fit_pending) {
                double fit = 0.0, tol = 0.0;
                const cpd_status ps = cpd_fit_poll(r->ctx, &fit, &tol);
                if (ps == CPD_EAGAIN) {
                    ++q;
                    continue;
                }
                progressed = true;
                r->fit_pending = false;
                retire = after_fit(srv, r, ps, fit, tol, &st);
                if (!retire) r->next_check = std::min<int64_t>(r->res.iters + fit_every, r->max_iters);
            }
            if (!retire && !r->fit_pending) {
                const int64_t chunk = r->next_check - r->res.iters;
                st = cpd_sgd_iters(r->ctx, chunk, r->stream);
                if (st == CPD_OK) st = cpd_fit_start(r->ctx, r->stream);
                if (st != CPD_OK) {
                    retire = true;
                } else {
                    add_iters(srv, r, chunk);
                    r->fit_pending = true;
                    progressed = true;
                }
            }
            if (retire) {
                finish(srv, r, st);
                srv->active.erase(srv->active.begin() + q);
            } else {
                ++q;
            }
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    for (auto &r : srv->active) finish(srv, r, CPD_EBUSY);
    srv->active.clear();
    for (auto &l : srv->lanes) {
        cudaStreamSynchronize(l->stream);
        if (l->grp) cpd_group_destroy(l->grp);
        for (auto &m : l->members) finish(srv, m, CPD_EBUSY);
        for (auto &m : l->joining) finish(srv, m, CPD_EBUSY);
        cudaEventDestroy(l->done);
        cudaStreamDestroy(l->stream);
    }
    srv->lanes.clear();
}

extern "C" cpd_status cpd_server_create(const cpd_server_config *cfg, cpd_server **out)
{
    if (!out) {
        set_error("NULL output");
        return CPD_EINVAL;
    }
    auto *srv = new cpd_server();
    if (cfg) srv->cfg = *cfg;
    if (srv->cfg.strided_above_mb < 0 || srv->cfg.no_grouping < 0 || srv->cfg.no_grouping > 1) {
        delete srv;
        set_error("strided_above_mb must be >= 0 and no_grouping 0 or 1");
        return CPD_EINVAL;
    }
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        delete srv;
        set_error("no CUDA device");
        return CPD_ECUDA;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete srv;
        set_error("cudaMemGetInfo failed");
        return CPD_ECUDA;
    }
    srv->budget = srv->cfg.hbm_budget ? srv->cfg.hbm_budget : (size_t)(0.85 * (double)free_b);
    srv->worker = std::thread(worker_loop, srv);
    *out = srv;
    return CPD_OK;
}

extern "C" cpd_status cpd_submit(cpd_server *srv, const cpd_config *cfg, const void *X, int x_loc,
                                 const void *const *A0, int a0_loc, double stop_fit, int64_t max_iters,
                                 uint64_t *ticket)
{
    if (!srv || !cfg || !X || !A0 || !ticket || max_iters < 1 || cfg->N < 1 || cfg->N > CPD_MAX_MODES) {
        set_error("invalid argument");
        return CPD_EINVAL;
    }
    auto r = std::make_shared<Request>();
    r->cfg = *cfg;
    r->X = X;
    r->x_loc = x_loc;
    r->A0.assign(A0, A0 + cfg->N);
    r->a0_loc = a0_loc;
    r->stop_fit = stop_fit;
    r->max_iters = max_iters;
    r->bytes = estimate_bytes(*cfg);
    const double limit = srv->cfg.strided_above_mb > 0 ? (double)((size_t)srv->cfg.strided_above_mb << 20) : 1e300;
    if (r->cfg.x_layout == CPD_LAYOUT_REPLICAS && (r->bytes > srv->budget || tensor_bytes(r->cfg) > limit)) {
        // the replicas would not fit: one strided copy of X on the CUDA-core
        // engine instead (decided from the request and the configuration)
        r->cfg.x_layout = CPD_LAYOUT_STRIDED;
        r->cfg.engine = 1;
        r->cfg.max_ctas = 0;
        r->bytes = estimate_bytes(r->cfg);
    }
    r->res.layout = r->cfg.x_layout;
    if (r->bytes > srv->budget) {
        set_error("request needs " + std::to_string(r->bytes) + " bytes, over the server budget");
        return CPD_ENOMEM;
    }
    std::lock_guard<std::mutex> lock(srv->mu);
    r->ticket = srv->next_ticket++;
    r->res.t_submit = now_s();
    srv->queue.push_back(r);
    srv->all[r->ticket] = r;
    ++srv->unfinished;
    srv->cv_work.notify_all();
    *ticket = r->ticket;
    return CPD_OK;
}

extern "C" cpd_status cpd_server_stats(cpd_server *srv, size_t *budget, size_t *held, int32_t *active,
                                       int32_t *queued)
{
    if (!srv) {
        set_error("NULL server");
        return CPD_EINVAL;
    }
    std::lock_guard<std::mutex> lock(srv->mu);
    if (budget) *budget = srv->budget;
    if (held) *held = srv->used;
    if (active) *active = (int32_t)srv->running;
    if (queued) *queued = (int32_t)srv->queue.size();
    return CPD_OK;
}

extern "C" cpd_status cpd_poll(cpd_server *srv, uint64_t ticket, cpd_result *out, void *const *A_out)
{
    if (!srv) {
        set_error("NULL server");
        return CPD_EINVAL;
    }
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        auto it = srv->all.find(ticket);
        if (it == srv->all.end()) {
            set_error("unknown ticket");
            return CPD_EINVAL;
        }
        r = it->second;
        if (out) *out = r->res;
        if (!r->res.done) return CPD_EAGAIN;
    }
    if (A_out && r->res.status == CPD_OK)
        for (int k = 0; k < r->cfg.N; ++k)
            if (A_out[k]) std::copy(r->factors[k].begin(), r->factors[k].end(), static_cast<unsigned char *>(A_out[k]));
    return (cpd_status)r->res.status;
}

extern "C" cpd_status cpd_server_wait(cpd_server *srv, double timeout_s)
{
    if (!srv) {
        set_error("NULL server");
        return CPD_EINVAL;
    }
    std::unique_lock<std::mutex> lock(srv->mu);
    auto pred = [&] { return srv->unfinished == 0; };
    if (timeout_s <= 0) {
        srv->cv_done.wait(lock, pred);
        return CPD_OK;
    }
    return srv->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), pred) ? CPD_OK : CPD_EAGAIN;
}

extern "C" cpd_status cpd_server_destroy(cpd_server *srv)
{
    if (!srv) return CPD_OK;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    delete srv;
    return CPD_OK;
}
