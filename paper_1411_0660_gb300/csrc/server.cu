// server.cu -- serving: a request loop with continuous batching and HBM admission.
//
// A context may start a server: `slots` worker threads, each with its own child context (own CUDA
// stream, own scratch) that shares the parent's symbolic analyses (plan cache).  Requests
// (L, h, seed, eps, nev) queue in arrival order; a free worker takes the oldest, builds the sector
// (and, once per L, the plan), estimates the HBM the job will hold from the plan (fronts, factor,
// solve work, Krylov basis, outputs) and waits until that much of the server budget is free.  Jobs
// of different sizes then run side by side on the device, each on its worker's stream; a finished
// job returns its reservation and wakes the waiting workers.  Every job goes through the same
// entry points as a single call (sector build, shift-invert eigensolve, observables), so its
// result is the one it would have alone.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <thread>

#include "factor.h"
#include "krylov.h"
#include "observables.h"

namespace mbl {

// Upper estimate of the device bytes one job holds at its peak (plan of its L known).  A job runs in
// phases: extremal bounds (a Lanczos basis), the numeric factorization (fronts arena at its peak in
// the automatic arena mode, the packed solve factor, the panel operators), then the Krylov iteration
// (solve factor, solve work, Krylov basis, Rayleigh-Ritz and refinement work).  A refactorization
// (shift moved off an eigenvalue, FP64 fallback) runs with the Krylov buffers alive, so they count
// in the factorization phase too.  The sector and the outputs are held throughout.
size_t job_bytes(const Plan &p, int nev, int block, int prec) {
    const double n = (double)p.n, es = prec == MBL_PREC_FP64 ? 8.0 : 4.0;
    const int pb = std::max(1, std::min(32, block));
    const double pad = pb <= 8 ? 8 : (pb <= 16 ? 16 : 32);
    const double ldv = 2.0 * nev + 3.0 * pb;
    const double held = 20.0 * n + 12.0 * (double)p.nnzA      // sector
                        + 8.0 * n * nev + 64.0 * nev;         // outputs
    const double factor_keep = (double)p.sg_elems * es + n * (es + 4.0);  // packed solve factor, D, pivots
    const double krylov = 8.0 * n * (3.0 * ldv + 2.0 * nev + 30.0 * pb)  // Krylov, Rayleigh-Ritz, refinement
                          + 2.0 * (double)p.zwork_elems * pb * es + 2.0 * n * pb * es  // solve work
                          + (double)std::max(p.max_sstep_nrbk, p.max_lvl_nrbk) * SUBS * RBB * pad * es;
    const double bounds = 8.0 * n * 480.0;  // extremal-bounds Lanczos basis
    const double factor = arena_peak_bytes(p, prec, ARENA_AUTO) + factor_keep +
                          (double)std::max<int64_t>(p.wscratch_elems, 1) * 5.0 * es + (double)p.m_elems * es +
                          krylov;  // W21 scratch and the four operand-piece arrays
    const double solve = factor_keep + krylov;
    const double peak = held + std::max(bounds, std::max(factor, solve));
    return (size_t)(1.05 * peak) + ((size_t)128 << 20);
}

namespace {

double now_ms(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

struct Job {
    mbl_request req{};
    std::vector<double> fields;  // explicit disorder (copied at submission), empty = from (h, seed)
    int state = 0;  // 0 queued, 1 running, 2 done
    int status = MBL_OK;
    int factor_reused = 0;
    std::string err;
    int nconv = 0;
    int64_t dim = 0;
    double sigma = 0.0, r_mean = 0.0;
    double t_submit = 0.0, t_admit = 0.0, t_end = 0.0;
    double d_start = 0.0, d_end = 0.0;  // device clock (CUDA events), ms after the server's reference event
    size_t reserved = 0;
    std::vector<double> evals, resid, r, s1p, se, evecs;
};

}  // namespace

// A finished job's sector and live factorization, kept for a later identical request (serving
// residency): same sector shape and fields, target and precision.
struct CacheEntry {
    int L = 0, nup = 0, prec = 0;
    double eps = 0.0;
    std::vector<double> fields;
    mbl_sector *sec = nullptr;
    std::unique_ptr<Factorization> fz;
    size_t bytes = 0;
};

struct Server {
    Ctx *parent = nullptr;
    std::vector<mbl_ctx *> wctx;
    std::vector<std::thread> threads;
    std::mutex mu;
    std::condition_variable cv_work, cv_mem, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Job>> jobs;
    uint64_t next_ticket = 1;
    size_t budget = 0, reserved = 0, peak_reserved = 0;
    int64_t submitted = 0, completed = 0, failed = 0;
    int running = 0;
    bool stop = false;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    cudaEvent_t ref = nullptr;  // recorded at start on the parent stream: origin of the device times
    SolveBatcher *batcher = nullptr;  // shared by the workers (none if batching is off)
    // live factorizations, most recently used first; their bytes count against the budget
    std::list<std::unique_ptr<CacheEntry>> cache;
    size_t cache_bytes = 0, cache_limit = 0;
    int64_t cache_hits = 0;
    void evict_one();  // mu held

    void worker(int i);
    void run(Job &J, mbl_ctx *w);
};

void Server::evict_one() {
    std::unique_ptr<CacheEntry> e = std::move(cache.back());
    cache.pop_back();
    cache_bytes -= e->bytes;
    e->fz.reset();
    mbl_sector_destroy(e->sec);
}

void Server::run(Job &J, mbl_ctx *w) {
    const mbl_request &q = J.req;
    mbl_sector *sec = nullptr;
    bool held = false;
    std::unique_ptr<Factorization> keep;
    try {
        const int nup = q.nup > 0 ? q.nup : q.L / 2;
        int rc = J.fields.empty() ? mbl_build_sector_nup(w, q.L, nup, q.h, q.seed, &sec)
                                  : mbl_build_sector_fields_nup(w, q.L, nup, J.fields.data(), 1.0, &sec);
        if (rc != MBL_OK) fail(rc, mbl_last_error(w));
        if (cache_limit) {
            // a live factorization of the same request: take it (with its sector) out of the cache
            std::unique_ptr<CacheEntry> hit;
            {
                std::lock_guard<std::mutex> lk(mu);
                for (auto it = cache.begin(); it != cache.end(); ++it) {
                    const CacheEntry &e = **it;
                    if (e.L == q.L && e.nup == nup && e.prec == q.precision && e.eps == q.eps &&
                        std::memcmp(e.fields.data(), sec->hfield, sizeof(double) * q.L) == 0) {
                        hit = std::move(*it);
                        cache.erase(it);
                        cache_bytes -= hit->bytes;
                        ++cache_hits;
                        break;
                    }
                }
            }
            if (hit) {
                mbl_sector_destroy(sec);
                sec = hit->sec;
                keep = std::move(hit->fz);
                // the entry was made by another worker: from here on its work runs on this worker's
                // stream (that worker synchronized its stream when the job ended)
                sec->ctx = w;
                keep->ctx = w;
            }
        }
        std::shared_ptr<Plan> plan = get_plan(sec);
        mbl_opts o;
        mbl_opts_default(&o);
        o.precision = q.precision;
        const size_t est = job_bytes(*plan, q.nev, o.block, o.precision);
        {
            std::unique_lock<std::mutex> lk(mu);
            if (est > budget) fail(MBL_ERR_OOM, "request needs more HBM than the server budget");
            for (;;) {  // admit when the job fits beside the running ones, evicting cached factors first
                if (stop || reserved + est + cache_bytes <= budget) break;
                if (!cache.empty()) {
                    evict_one();
                    continue;
                }
                cv_mem.wait(lk);
            }
            if (stop) fail(MBL_ERR_INVALID, "server stopped");
            reserved += est;
            peak_reserved = std::max(peak_reserved, reserved);
            held = true;
            J.reserved = est;
            J.t_admit = now_ms(t0);
        }
        const int64_t n = sec->n;
        const int nev = q.nev;
        J.dim = n;
        struct EvPair {
            cudaEvent_t a = nullptr, b = nullptr;
            ~EvPair() {
                if (a) cudaEventDestroy(a);
                if (b) cudaEventDestroy(b);
            }
        } ev;
        MBL_CUDA(cudaEventCreate(&ev.a));
        MBL_CUDA(cudaEventCreate(&ev.b));
        MBL_CUDA(cudaEventRecord(ev.a, w->stream));
        DVec<double> de, dv, dr, dobs;
        de.alloc(w, nev);
        dv.alloc(w, (size_t)n * nev);
        dr.alloc(w, nev);
        dobs.alloc(w, (size_t)3 * nev + 1);
        int nconv = 0;
        double sigma = 0.0;
        mbl_solve_stats sst{};
        solve_near(sec, q.eps, nev, o, de.data(), dv.data(), dr.data(), &nconv, &sigma, &sst, w->stream,
                   cache_limit ? &keep : nullptr);
        J.factor_reused = sst.factor_reused;
        rc = nconv < nev ? MBL_ERR_NOT_CONVERGED : MBL_OK;
        J.status = rc;
        if (rc != MBL_OK) J.err = "only " + std::to_string(nconv) + " of " + std::to_string(nev) + " eigenpairs reached the tolerance";
        double *d_r = dobs.data(), *d_rm = d_r + nev, *d_s1 = d_rm + 1, *d_se = d_s1 + nev;
        int rc2 = mbl_observables_nup_dev(w, q.L, nup, nev, de.data(), dv.data(), d_r, d_rm, d_s1, d_se, nullptr);
        if (rc2 != MBL_OK) fail(rc2, mbl_last_error(w));
        MBL_CUDA(cudaEventRecord(ev.b, w->stream));
        MBL_CUDA(cudaStreamSynchronize(w->stream));
        float ta = 0.f, tb = 0.f;
        MBL_CUDA(cudaEventElapsedTime(&ta, ref, ev.a));
        MBL_CUDA(cudaEventElapsedTime(&tb, ref, ev.b));
        J.d_start = ta;
        J.d_end = tb;
        J.nconv = nconv;
        J.sigma = sigma;
        J.evals.resize(nev);
        J.resid.resize(nev);
        J.r.resize(std::max(nev - 2, 0));
        J.s1p.resize(nev);
        J.se.resize(nev);
        std::vector<double> obs((size_t)3 * nev + 1);
        MBL_CUDA(cudaMemcpy(J.evals.data(), de.data(), nev * sizeof(double), cudaMemcpyDeviceToHost));
        MBL_CUDA(cudaMemcpy(J.resid.data(), dr.data(), nev * sizeof(double), cudaMemcpyDeviceToHost));
        MBL_CUDA(cudaMemcpy(obs.data(), dobs.data(), obs.size() * sizeof(double), cudaMemcpyDeviceToHost));
        std::copy(obs.begin(), obs.begin() + std::max(nev - 2, 0), J.r.begin());
        J.r_mean = obs[nev];
        std::copy(obs.begin() + nev + 1, obs.begin() + 2 * nev + 1, J.s1p.begin());
        std::copy(obs.begin() + 2 * nev + 1, obs.end(), J.se.begin());
        if (q.want_vectors) {
            J.evecs.resize((size_t)n * nev);
            MBL_CUDA(cudaMemcpy(J.evecs.data(), dv.data(), (size_t)n * nev * sizeof(double), cudaMemcpyDeviceToHost));
        }
    } catch (const Error &e) {
        J.status = e.code;
        J.err = e.msg;
    } catch (const std::exception &e) {
        J.status = MBL_ERR_CUDA;
        J.err = e.what();
    }
    // keep the sector and its live factorization for an identical request, within the cache limit
    if (sec && keep && cache_limit && J.status == MBL_OK && cudaStreamSynchronize(w->stream) == cudaSuccess) {
        auto e = std::make_unique<CacheEntry>();
        e->L = q.L;
        e->nup = q.nup > 0 ? q.nup : q.L / 2;
        e->prec = q.precision;
        e->eps = q.eps;
        e->fields.assign(sec->hfield, sec->hfield + q.L);
        e->bytes = keep->held_bytes() + (size_t)(20 * sec->n + 12 * sec->nnz);
        if (e->bytes <= cache_limit) {
            e->sec = sec;
            e->fz = std::move(keep);
            sec = nullptr;
            std::lock_guard<std::mutex> lk(mu);
            cache_bytes += e->bytes;
            cache.push_front(std::move(e));
            while (cache_bytes > cache_limit) evict_one();
        }
    }
    keep.reset();
    if (sec) mbl_sector_destroy(sec);
    {
        std::lock_guard<std::mutex> lk(mu);
        J.t_end = now_ms(t0);  // before the reservation returns: the next admission comes after it
        if (held) reserved -= J.reserved;
    }
    cv_mem.notify_all();
}

void Server::worker(int i) {
    mbl_ctx *w = wctx[i];
    cudaSetDevice(w->device);
    for (;;) {
        uint64_t t;
        Job *J;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !queue.empty(); });
            if (stop) return;
            t = queue.front();
            queue.pop_front();
            J = jobs[t].get();
            J->state = 1;
            ++running;
        }
        run(*J, w);
        {
            std::lock_guard<std::mutex> lk(mu);
            J->state = 2;
            --running;
            ++completed;
            if (J->status != MBL_OK) ++failed;
        }
        cv_done.notify_all();
    }
}

void server_shutdown(Ctx *ctx) {
    Server *s = ctx->server;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_mem.notify_all();
    for (auto &th : s->threads) th.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        while (!s->cache.empty()) s->evict_one();
    }
    batcher_destroy(s->batcher);
    for (mbl_ctx *w : s->wctx) mbl_ctx_destroy(w);
    if (s->ref) cudaEventDestroy(s->ref);
    ctx->server = nullptr;
    delete s;
}

}  // namespace mbl

using namespace mbl;

namespace {

int srv_report(mbl_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return code;
}

void fill_result(const Job &J, mbl_result *out) {
    out->status = J.status;
    out->nconv = J.nconv;
    out->nev = J.req.nev;
    out->L = J.req.L;
    out->dim = J.dim;
    out->sigma = J.sigma;
    out->r_mean = J.r_mean;
    out->t_submit_ms = J.t_submit;
    out->t_admit_ms = J.t_admit;
    out->t_end_ms = J.t_end;
    out->d_start_ms = J.d_start;
    out->d_end_ms = J.d_end;
    out->reserved_bytes = J.reserved;
    out->factor_reused = J.factor_reused;
    auto put = [](double *dst, const std::vector<double> &v) {
        if (dst && !v.empty()) std::copy(v.begin(), v.end(), dst);
    };
    put(out->evals, J.evals);
    put(out->resid, J.resid);
    put(out->r, J.r);
    put(out->s1p, J.s1p);
    put(out->se, J.se);
    put(out->evecs, J.evecs);
}

}  // namespace

int mbl_server_start(mbl_ctx *ctx, int slots, size_t budget_bytes) {
    if (!ctx) return MBL_ERR_INVALID;
    if (slots < 1 || slots > 64) return srv_report(ctx, MBL_ERR_INVALID, "slots must be in [1, 64]");
    if (ctx->server) return srv_report(ctx, MBL_ERR_INVALID, "server already running");
    try {
        MBL_CUDA(cudaSetDevice(ctx->device));
        size_t fr = 0, tot = 0;
        MBL_CUDA(cudaMemGetInfo(&fr, &tot));
        auto s = std::make_unique<Server>();
        s->parent = ctx;
        s->budget = budget_bytes ? budget_bytes : (size_t)(0.85 * (double)fr);
        if (ctx->budget) s->budget = std::min(s->budget, ctx->budget);
        for (int i = 0; i < slots; ++i) {
            mbl_ctx *w = nullptr;
            int rc = mbl_ctx_create(ctx->device, 0, &w);
            if (rc != MBL_OK) {
                for (mbl_ctx *x : s->wctx) mbl_ctx_destroy(x);
                return srv_report(ctx, rc, "worker context: " + std::string(mbl_last_error(nullptr)));
            }
            w->plans = ctx->plans;
            s->wctx.push_back(w);
        }
        s->cache_limit = ctx->cache_fraction > 0.0 ? (size_t)(ctx->cache_fraction * (double)s->budget) : 0;
        if (ctx->batch_max_jobs > 1 && slots > 1) {
            s->batcher = batcher_create(ctx->device, ctx->batch_max_jobs, ctx->batch_window_us, ctx->batch_lanes);
            for (mbl_ctx *w : s->wctx) w->batcher = s->batcher;
        }
        MBL_CUDA(cudaEventCreate(&s->ref));
        MBL_CUDA(cudaEventRecord(s->ref, ctx->stream));
        MBL_CUDA(cudaEventSynchronize(s->ref));
        Server *raw = s.release();
        ctx->server = raw;
        for (int i = 0; i < slots; ++i) raw->threads.emplace_back([raw, i] { raw->worker(i); });
    } catch (const Error &e) {
        return srv_report(ctx, e.code, e.msg);
    } catch (const std::exception &e) {
        return srv_report(ctx, MBL_ERR_CUDA, e.what());
    }
    return MBL_OK;
}

int mbl_submit(mbl_ctx *ctx, const mbl_request *req, uint64_t *ticket) {
    if (!ctx || !req || !ticket) return MBL_ERR_INVALID;
    Server *s = ctx->server;
    if (!s) return srv_report(ctx, MBL_ERR_INVALID, "no server: call mbl_server_start first");
    if (req->L < 2 || req->L > 22) return srv_report(ctx, MBL_ERR_INVALID, "L must be in 2..22");
    if (req->nup < 0 || req->nup > req->L || (req->nup == 0 && (req->L & 1)))
        return srv_report(ctx, MBL_ERR_INVALID, "nup must be in 1..L (or 0 for the S^z = 0 sector of even L)");
    if (!(req->eps >= 0.0 && req->eps <= 1.0)) return srv_report(ctx, MBL_ERR_INVALID, "eps must be in [0, 1]");
    if (req->h < 0.0 || req->nev < 1) return srv_report(ctx, MBL_ERR_INVALID, "h >= 0 and nev >= 1 required");
    if (req->precision != MBL_PREC_FP32 && req->precision != MBL_PREC_FP64)
        return srv_report(ctx, MBL_ERR_INVALID, "unknown precision");
    auto J = std::make_unique<Job>();
    J->req = *req;
    if (req->fields) J->fields.assign(req->fields, req->fields + req->L);
    J->req.fields = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        J->t_submit = now_ms(s->t0);
        *ticket = s->next_ticket++;
        s->jobs[*ticket] = std::move(J);
        s->queue.push_back(*ticket);
        ++s->submitted;
    }
    s->cv_work.notify_one();
    return MBL_OK;
}

int mbl_poll(mbl_ctx *ctx, uint64_t ticket, mbl_result *out) {
    if (!ctx || !out) return MBL_ERR_INVALID;
    Server *s = ctx->server;
    if (!s) return srv_report(ctx, MBL_ERR_INVALID, "no server");
    std::unique_ptr<Job> J;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return srv_report(ctx, MBL_ERR_INVALID, "unknown ticket");
        if (it->second->state != 2) return MBL_PENDING;
        J = std::move(it->second);
        s->jobs.erase(it);
    }
    fill_result(*J, out);
    if (J->status != MBL_OK) ctx->last_error = J->err;
    return J->status;
}

int mbl_wait(mbl_ctx *ctx, uint64_t ticket, double timeout_s, mbl_result *out) {
    if (!ctx || !out) return MBL_ERR_INVALID;
    Server *s = ctx->server;
    if (!s) return srv_report(ctx, MBL_ERR_INVALID, "no server");
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto ready = [&] {
            auto it = s->jobs.find(ticket);
            return it == s->jobs.end() || it->second->state == 2;
        };
        if (timeout_s > 0) {
            if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return MBL_PENDING;
        } else {
            s->cv_done.wait(lk, ready);
        }
    }
    return mbl_poll(ctx, ticket, out);
}

int mbl_server_stats_get(mbl_ctx *ctx, mbl_server_stats *out) {
    if (!ctx || !out) return MBL_ERR_INVALID;
    Server *s = ctx->server;
    if (!s) return srv_report(ctx, MBL_ERR_INVALID, "no server");
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->running = s->running;
    out->queued = (int)s->queue.size();
    out->slots = (int)s->wctx.size();
    out->budget_bytes = s->budget;
    out->reserved_bytes = s->reserved;
    out->peak_reserved_bytes = s->peak_reserved;
    out->cache_hits = s->cache_hits;
    out->cache_bytes = s->cache_bytes;
    out->solve_batches = out->batched_solves = 0;
    out->batch_ms = out->batch_bytes = out->batch_busy_ms = 0.0;
    if (s->batcher) {
        try {
            batcher_stats(s->batcher, &out->solve_batches, &out->batched_solves, &out->batch_ms, &out->batch_bytes,
                          &out->batch_busy_ms);
        } catch (const Error &e) {
            return srv_report(ctx, e.code, e.msg);
        }
    }
    return MBL_OK;
}

int mbl_server_cache(mbl_ctx *ctx, double fraction) {
    if (!ctx) return MBL_ERR_INVALID;
    if (ctx->server) return srv_report(ctx, MBL_ERR_INVALID, "set the cache before mbl_server_start");
    if (!(fraction >= 0.0 && fraction <= 0.9)) return srv_report(ctx, MBL_ERR_INVALID, "fraction in [0, 0.9]");
    ctx->cache_fraction = fraction;
    return MBL_OK;
}

int mbl_server_batching(mbl_ctx *ctx, int max_jobs, double window_us, int lanes) {
    if (!ctx) return MBL_ERR_INVALID;
    if (ctx->server) return srv_report(ctx, MBL_ERR_INVALID, "set batching before mbl_server_start");
    if (max_jobs < 1 || max_jobs > 64 || !(window_us >= 0.0 && window_us <= 1e6) || lanes < 1 || lanes > 8)
        return srv_report(ctx, MBL_ERR_INVALID, "max_jobs in [1, 64], window_us in [0, 1e6], lanes in [1, 8]");
    ctx->batch_max_jobs = max_jobs;
    ctx->batch_window_us = window_us;
    ctx->batch_lanes = lanes;
    return MBL_OK;
}

int mbl_server_stop(mbl_ctx *ctx) {
    if (!ctx) return MBL_ERR_INVALID;
    server_shutdown(ctx);
    return MBL_OK;
}
