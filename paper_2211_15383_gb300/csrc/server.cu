// Request server: whole trace problems (gauge field, mass, hierarchy, deflation,
// target relative error; the estimate of tr(D^{-1}) of Sect. 3.2 with the deflated
// coarsest term of Sect. 2) admitted continuously on one GPU.  The policy that picks
// the next requests is mg::Admission (admission.h); this file holds the footprint
// model, the worker threads (one CUDA stream each) and the C entry points declared
// under "Serving" in include/mgmlmc.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "admission.h"
#include "context.h"
#include "footprint.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double>(b - a).count();
}

thread_local std::string t_server_error;

int fail(int code, const std::string& msg) {
    t_server_error = msg;
    return code;
}

// Level geometry of a request, checked as mgmlmc_set_gauge / mgmlmc_set_hierarchy do.
struct Geometry {
    int L = 0;
    long long sites[MGMLMC_MAX_LEVELS] = {0}, n[MGMLMC_MAX_LEVELS] = {0};
    int d[MGMLMC_MAX_LEVELS] = {0};
};

int geometry(const mgmlmc_request& r, Geometry& g, std::string& why) {
    try {
        mg::check_options(r.opt);
    } catch (const mg::Error& e) {
        why = std::string("request: ") + e.what();
        return e.code;
    }
    if (r.Lx < 2 || r.Lt < 2 || r.Lx % 2 || r.Lt % 2 || (long long)r.Lx * r.Lt > (1LL << 26)) {
        why = "request: Lx, Lt even, >= 2, Lx*Lt <= 2^26";
        return MGMLMC_EINVAL;
    }
    if (r.nlevels < 1 || r.nlevels > MGMLMC_MAX_LEVELS) {
        why = "request: 1 <= nlevels <= 6";
        return MGMLMC_EINVAL;
    }
    g.L = r.nlevels;
    long long lx = r.Lx, lt = r.Lt;
    int d = 2;
    for (int l = 0; l < g.L; ++l) {
        g.sites[l] = lx * lt;
        g.d[l] = d;
        g.n[l] = lx * lt * d;
        if (l == g.L - 1) break;
        const int ax = r.agg_x[l], at = r.agg_t[l], nv = r.nvec[l];
        if (ax < 1 || at < 1 || lx % ax || lt % at) {
            why = "request: aggregates must divide the lattice of their level";
            return MGMLMC_EINVAL;
        }
        if (nv < 1 || nv > 32 || nv > ax * at * d / 2) {
            why = "request: 1 <= nvec <= 32 and nvec <= rows of an aggregate's spin block";
            return MGMLMC_EINVAL;
        }
        lx /= ax;
        lt /= at;
        d = 2 * nv;
    }
    if (r.sum_levels < 0 || r.sum_levels > r.nlevels) {
        why = "request: 0 <= sum_levels <= nlevels";
        return MGMLMC_EINVAL;
    }
    if (g.n[g.L - 1] > 16384) {
        why = "request: the coarsest level is inverted densely (at most 16384 unknowns)";
        return MGMLMC_ENOTIMPL;
    }
    return MGMLMC_OK;
}

int term_levels_of(const mgmlmc_request& r) {
    return (r.sum_levels > 0 && r.sum_levels < r.nlevels) ? r.sum_levels : r.nlevels;
}

// Device bytes a request's context holds at most (mg::footprint_bytes).
size_t footprint_bytes(const mgmlmc_request& r, const Geometry& g) {
    mg::Shape s;
    s.L = g.L;
    s.nterm_levels = term_levels_of(r);
    for (int l = 0; l < g.L; ++l) {
        s.sites[l] = g.sites[l];
        s.n[l] = g.n[l];
        s.d[l] = g.d[l];
        s.nvec[l] = l + 1 < g.L ? r.nvec[l] : 0;
    }
    s.k = r.k;
    s.N = r.opt.max_block_rhs;
    s.m = r.opt.fgmres_restart;
    s.precision = r.opt.mg_precision;
    s.kcycle = r.opt.kcycle_iters;
    return mg::footprint_bytes(s);
}

std::string shape_key(const mgmlmc_request& r) {
    std::string s = std::to_string(r.Lx) + "x" + std::to_string(r.Lt) + "/" + std::to_string(r.nlevels);
    for (int l = 0; l + 1 < r.nlevels; ++l)
        s += ":" + std::to_string(r.agg_x[l]) + "," + std::to_string(r.agg_t[l]) + "," + std::to_string(r.nvec[l]);
    s += "/t" + std::to_string(term_levels_of(r));
    s += "/k" + std::to_string(r.k) + "/p" + std::to_string(r.opt.mg_precision) + "/N" +
         std::to_string(r.opt.max_block_rhs) + "/m" + std::to_string(r.opt.fgmres_restart);
    return s;
}

struct Job {
    uint64_t id = 0;
    mgmlmc_request req{};
    std::vector<double> theta;
    std::vector<std::vector<double>> start;   // start vectors of levels 1..L-1
    std::string shape;
    size_t reserved = 0;
    int retries = 0;
    bool done = false;
    std::atomic<bool> cancel{false};
    Clock::time_point t_submit;
    mgmlmc_request_result res{};
};

// Stream-ordered allocation from the server's pool on the worker's stream.
struct PoolUser {
    cudaMemPool_t pool;
    cudaStream_t stream;
};

void* pool_alloc(void* user, size_t bytes) {
    auto* u = static_cast<PoolUser*>(user);
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, u->pool, u->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pool_free(void* user, void* p) { cudaFreeAsync(p, static_cast<PoolUser*>(user)->stream); }

}  // namespace

struct mgmlmc_server {
    int device = 0;
    cudaMemPool_t pool = nullptr;
    std::unique_ptr<mg::Admission> adm;
    std::mutex mu;
    std::condition_variable cv_work;   // workers: a request was admitted, or stop
    std::condition_variable cv_done;   // waiters: a request finished
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    std::deque<std::shared_ptr<Job>> ready;   // admitted, not yet taken by a worker
    std::map<std::string, size_t> learned;    // largest device peak by request shape
    uint64_t next_id = 1;
    int64_t completed = 0;
    bool stopping = false;
    std::vector<std::thread> workers;
};

namespace {

// Admit what fits; the caller holds srv->mu.
void admit_locked(mgmlmc_server* srv) {
    bool any = false;
    for (const mg::Admission::Item& it : srv->adm->admit()) {
        auto j = srv->jobs.find(it.id);
        if (j == srv->jobs.end()) continue;
        j->second->reserved = it.bytes;
        srv->ready.push_back(j->second);
        any = true;
    }
    if (any) srv->cv_work.notify_all();
}

void finish_locked(mgmlmc_server* srv, Job& j, int status, const std::string& msg) {
    j.res.status = status;
    std::snprintf(j.res.error, sizeof(j.res.error), "%s", msg.c_str());
    j.res.total_s = seconds_between(j.t_submit, Clock::now());
    if (j.res.setup_s == 0 && j.res.estimate_s == 0) j.res.queued_s = j.res.total_s;   // never admitted
    j.res.reserved_bytes = j.reserved;
    j.res.retries = j.retries;
    j.done = true;
    ++srv->completed;
    srv->cv_done.notify_all();
}

// Set-up and estimate of one admitted request on the worker's stream.
int run_job(Job& j, cudaStream_t stream, PoolUser* pu, std::string& msg, size_t& peak) {
    const mgmlmc_request& r = j.req;
    mgmlmc_ctx* ctx = nullptr;
    int rc = MGMLMC_OK;
    auto step = [&](int code, const char* what) {
        if (rc != MGMLMC_OK) return;
        if (code != MGMLMC_OK) {
            rc = code;
            msg = std::string(what) + ": " + (ctx ? mgmlmc_last_error(ctx) : "");
        } else if (j.cancel.load()) {
            rc = MGMLMC_ECANCELLED;
            msg = "cancelled";
        }
    };
    const Clock::time_point t0 = Clock::now();
    j.res.queued_s = seconds_between(j.t_submit, t0);
    step(j.cancel.load() ? MGMLMC_ECANCELLED : MGMLMC_OK, "admission");
    step(rc == MGMLMC_OK ? mgmlmc_create(&ctx, &r.opt, stream, pool_alloc, pool_free, pu) : rc, "create");
    step(rc == MGMLMC_OK ? mgmlmc_set_gauge(ctx, r.Lx, r.Lt, j.theta.data()) : rc, "set_gauge");
    step(rc == MGMLMC_OK ? mgmlmc_set_mass(ctx, r.m0) : rc, "set_mass");
    if (rc == MGMLMC_OK) {
        std::vector<const double*> sv(MGMLMC_MAX_LEVELS, nullptr);
        for (size_t l = 0; l < j.start.size(); ++l) sv[l] = j.start[l].data();
        step(mgmlmc_set_hierarchy(ctx, r.nlevels, r.agg_x, r.agg_t, r.nvec, r.setup_iters, r.setup_tol, sv.data()),
             "set_hierarchy");
    }
    if (rc == MGMLMC_OK && term_levels_of(r) < r.nlevels) {
        // the last levels serve only the solver: the sum ends at level sum_levels
        int skip[MGMLMC_MAX_LEVELS];
        int ns = 0;
        for (int l = term_levels_of(r) + 1; l <= r.nlevels; ++l) skip[ns++] = l;
        step(mgmlmc_set_terms(ctx, ns, skip), "set_terms");
    }
    if (rc == MGMLMC_OK && r.k > 0) {
        // an eigensolver that stops at its iteration cap keeps its factors: the estimate
        // adds the deflated trace of exactly those factors, so it stays unbiased; the
        // result says so instead of failing the request
        int code = mgmlmc_compute_deflation(ctx, r.k, r.defl_tol, r.defl_max_iters);
        j.res.deflation_converged = code == MGMLMC_OK ? 1 : 0;
        if (code == MGMLMC_ENOTCONVERGED) code = MGMLMC_OK;
        step(code, "compute_deflation");
    }
    const Clock::time_point t1 = Clock::now();
    j.res.setup_s = seconds_between(t0, t1);
    if (rc == MGMLMC_OK) {
        mg::Ctx& c = ctx->c;
        bool fixed = false;
        for (int t = 0; t < MGMLMC_MAX_LEVELS; ++t) fixed |= r.costs[t] > 0;
        try {
            mg::mlmc_loop(std::vector<mg::Ctx*>(c.nterms, &c), false, r.rel_tol, r.max_samples, r.seed,
                          fixed ? r.costs : nullptr, &j.res.result, &j.cancel);
        } catch (const mg::Error& e) {
            rc = e.code;
            msg = std::string("estimate_trace: ") + e.what();
        } catch (const std::bad_alloc&) {
            rc = MGMLMC_ENOMEM;
            msg = "estimate_trace: host allocation failed";
        } catch (const std::exception& e) {
            rc = MGMLMC_ECUDA;
            msg = std::string("estimate_trace: ") + e.what();
        }
    }
    j.res.estimate_s = seconds_between(t1, Clock::now());
    if (ctx) {
        peak = ctx->c.peak_bytes;
        mgmlmc_destroy(ctx);   // frees on the stream ...
    }
    cudaStreamSynchronize(stream);   // ... and the memory is back in the pool here
    return rc;
}

void worker_main(mgmlmc_server* srv) {
    cudaSetDevice(srv->device);
    cudaStream_t stream = nullptr;
    const bool stream_ok = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
    PoolUser pu{srv->pool, stream};
    for (;;) {
        std::shared_ptr<Job> job;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] { return srv->stopping || !srv->ready.empty(); });
            if (srv->ready.empty()) break;
            job = srv->ready.front();
            srv->ready.pop_front();
        }
        std::string msg;
        size_t peak = 0;
        int rc = MGMLMC_ECUDA;
        if (stream_ok) {
            rc = run_job(*job, stream, &pu, msg, peak);
        } else {
            msg = "cudaStreamCreateWithFlags failed";
        }
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->adm->finish(job->reserved);
        job->res.peak_bytes = std::max(job->res.peak_bytes, peak);
        const bool others = srv->adm->active() > 0;
        if (rc == MGMLMC_ENOMEM && others && job->retries < 2 && !job->cancel.load() && !srv->stopping) {
            // the device ran short while other requests held memory: queue it again at
            // the head, reserving what it reached (it is not overtaken again)
            ++job->retries;
            job->reserved = std::min(srv->adm->budget(), std::max(job->reserved, peak + peak / 10));
            srv->adm->push_front(job->id, job->reserved);
        } else {
            if (rc == MGMLMC_OK) {
                size_t& lp = srv->learned[job->shape];
                lp = std::max(lp, peak);
            }
            finish_locked(srv, *job, rc, msg);
        }
        admit_locked(srv);
    }
    if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

int mgmlmc_request_footprint(const mgmlmc_request* req, size_t* bytes) {
    if (!req || !bytes) return fail(MGMLMC_EINVAL, "request_footprint: NULL argument");
    Geometry g;
    std::string why;
    const int rc = geometry(*req, g, why);
    if (rc != MGMLMC_OK) return fail(rc, why);
    *bytes = footprint_bytes(*req, g);
    return MGMLMC_OK;
}

int mgmlmc_server_create(mgmlmc_server** out, const mgmlmc_server_options* opt) {
    if (!out) return fail(MGMLMC_EINVAL, "server_create: NULL argument");
    *out = nullptr;
    mgmlmc_server_options o{0, 4, 4};
    if (opt) o = *opt;
    if (o.max_active < 1 || o.max_active > 64 || o.max_bypass < 0)
        return fail(MGMLMC_EINVAL, "server_create: 1 <= max_active <= 64, max_bypass >= 0");
    int dev = 0;
    size_t free_b = 0, total_b = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return fail(MGMLMC_ECUDA, "server_create: no CUDA device");
    }
    const size_t budget = o.hbm_budget ? o.hbm_budget : free_b / 4 * 3;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return fail(MGMLMC_ECUDA, "server_create: cudaMemPoolCreate failed");
    }
    uint64_t keep = budget;   // freed memory stays in the pool for the next requests
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    mgmlmc_server* srv = nullptr;
    try {
        srv = new mgmlmc_server();
        srv->device = dev;
        srv->pool = pool;
        srv->adm.reset(new mg::Admission(budget, o.max_active, o.max_bypass));
        for (int i = 0; i < o.max_active; ++i) srv->workers.emplace_back(worker_main, srv);
    } catch (...) {
        if (srv) {
            {
                std::lock_guard<std::mutex> lk(srv->mu);
                srv->stopping = true;
            }
            srv->cv_work.notify_all();
            for (auto& t : srv->workers) t.join();
            delete srv;
        }
        cudaMemPoolDestroy(pool);
        return fail(MGMLMC_ENOMEM, "server_create: host allocation or thread creation failed");
    }
    *out = srv;
    return MGMLMC_OK;
}

void mgmlmc_server_destroy(mgmlmc_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        for (auto& kv : srv->jobs) {
            Job& j = *kv.second;
            j.cancel.store(true);
            if (!j.done && srv->adm->remove(j.id)) finish_locked(srv, j, MGMLMC_ECANCELLED, "server destroyed");
        }
    }
    srv->cv_work.notify_all();
    for (auto& t : srv->workers) t.join();
    cudaMemPoolDestroy(srv->pool);
    delete srv;
}

int mgmlmc_submit(mgmlmc_server* srv, const mgmlmc_request* req, uint64_t* id) {
    if (!srv || !req || !id) return fail(MGMLMC_EINVAL, "submit: NULL argument");
    const mgmlmc_request& r = *req;
    Geometry g;
    std::string why;
    int rc = geometry(r, g, why);
    if (rc != MGMLMC_OK) return fail(rc, why);
    if (!r.theta) return fail(MGMLMC_EINVAL, "submit: theta is NULL");
    for (int l = 0; l + 1 < r.nlevels; ++l)
        if (!r.start_vectors[l]) return fail(MGMLMC_EINVAL, "submit: missing start vectors");
    if (!(r.rel_tol > 0) || r.max_samples < 1 || r.k < 0 || (r.k > 0 && r.k > g.n[g.L - 1]))
        return fail(MGMLMC_EINVAL, "submit: rel_tol > 0, max_samples >= 1, 0 <= k <= n_L");
    int positive = 0;
    for (int t = 0; t < MGMLMC_MAX_LEVELS; ++t) {
        if (!(r.costs[t] >= 0) || !std::isfinite(r.costs[t])) return fail(MGMLMC_EINVAL, "submit: costs >= 0");
        positive += t < term_levels_of(r) && r.costs[t] > 0;
    }
    if (positive != 0 && positive != term_levels_of(r))   // the allocation divides by every term's cost
        return fail(MGMLMC_EINVAL, "submit: costs all zero (measured) or > 0 for each term");
    std::shared_ptr<Job> job;
    try {
        job = std::make_shared<Job>();
        job->req = r;
        job->theta.assign(r.theta, r.theta + (size_t)r.Lx * r.Lt * 2);
        for (int l = 0; l + 1 < r.nlevels; ++l)
            job->start.emplace_back(r.start_vectors[l], r.start_vectors[l] + (size_t)g.n[l] * r.nvec[l] * 2);
        job->req.theta = nullptr;
        for (auto& p : job->req.start_vectors) p = nullptr;
        job->shape = shape_key(r);
    } catch (const std::bad_alloc&) {
        return fail(MGMLMC_ENOMEM, "submit: host allocation failed");
    }
    job->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stopping) return fail(MGMLMC_ESTATE, "submit: server stopping");
    auto lp = srv->learned.find(job->shape);
    const size_t bytes = lp != srv->learned.end() ? lp->second + lp->second / 10 : footprint_bytes(r, g);
    if (srv->adm->too_large(bytes))
        return fail(MGMLMC_ENOMEM, "submit: footprint " + std::to_string(bytes) + " B exceeds the budget of " +
                                       std::to_string(srv->adm->budget()) + " B");
    job->id = srv->next_id++;
    job->reserved = bytes;
    srv->jobs[job->id] = job;
    srv->adm->push(job->id, bytes);
    admit_locked(srv);
    *id = job->id;
    return MGMLMC_OK;
}

int mgmlmc_poll(mgmlmc_server* srv, uint64_t id, mgmlmc_request_result* out) {
    if (!srv || !out) return fail(MGMLMC_EINVAL, "poll: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(id);
    if (it == srv->jobs.end()) return fail(MGMLMC_EINVAL, "poll: unknown id");
    if (!it->second->done) return MGMLMC_PENDING;
    *out = it->second->res;
    srv->jobs.erase(it);
    return MGMLMC_OK;
}

int mgmlmc_wait(mgmlmc_server* srv, uint64_t id, double timeout_s, mgmlmc_request_result* out) {
    if (!srv || !out) return fail(MGMLMC_EINVAL, "wait: NULL argument");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(id);
    if (it == srv->jobs.end()) return fail(MGMLMC_EINVAL, "wait: unknown id");
    std::shared_ptr<Job> job = it->second;
    if (timeout_s < 0) {
        srv->cv_done.wait(lk, [&] { return job->done; });
    } else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return job->done; })) {
        return MGMLMC_PENDING;
    }
    *out = job->res;
    srv->jobs.erase(id);
    return MGMLMC_OK;
}

int mgmlmc_cancel(mgmlmc_server* srv, uint64_t id) {
    if (!srv) return fail(MGMLMC_EINVAL, "cancel: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(id);
    if (it == srv->jobs.end() || it->second->done) return fail(MGMLMC_EINVAL, "cancel: unknown or finished id");
    Job& j = *it->second;
    j.cancel.store(true);
    if (srv->adm->remove(id)) {
        finish_locked(srv, j, MGMLMC_ECANCELLED, "cancelled while queued");
        admit_locked(srv);
    }
    return MGMLMC_OK;
}

int mgmlmc_get_server_stats(mgmlmc_server* srv, mgmlmc_server_stats* out) {
    if (!srv || !out) return fail(MGMLMC_EINVAL, "get_server_stats: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    out->queued = srv->adm->queued();
    out->active = srv->adm->active();
    out->completed = srv->completed;
    out->max_active_seen = srv->adm->max_active_seen();
    out->budget = srv->adm->budget();
    out->reserved = srv->adm->reserved();
    out->max_reserved = srv->adm->max_reserved();
    return MGMLMC_OK;
}

const char* mgmlmc_server_last_error(const mgmlmc_server*) { return t_server_error.c_str(); }

}  // extern "C"
