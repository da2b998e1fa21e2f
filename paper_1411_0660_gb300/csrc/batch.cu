// batch.cu -- continuous batching of triangular solves across serving workers.
//
// Jobs of one sector size share one symbolic plan, so their block solves are the same launch
// sequence on different buffers.  A serving worker's solve does not launch that sequence itself:
// it records an event on its stream, hands the request (factorization, right-hand sides, output)
// to the batcher and waits until the batch holding it is launched.  The batcher thread collects
// the requests of one (plan, precision, block width) until every worker inside a solve phase of
// that group has one pending, the oldest has waited `window`, or `max_jobs` are pending; it then
// makes its stream wait for the requests' events, writes the jobs' buffer and right-hand-side
// tables, and replays the graph of the batched sequence for that many jobs (one graph per job
// count, captured on first use): every launch of the sequence covers all jobs (grid z = job).
// Each request's `done` event is recorded after the graph, and the worker's stream waits for it.
// Per-solve work is unchanged; what changes is that K jobs' steps share one launch, so the short,
// latency-bound steps of one solve fill the GPU together.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <tuple>

#include "factor.h"

namespace mbl {

namespace {

constexpr int RING = 16;  // pinned host table slots in flight

using Clock = std::chrono::steady_clock;

struct BatchReq {
    Factorization *fz;
    const double *B;
    int64_t ldb;
    double *X;
    int64_t ldx;
    bool accumulate;
    cudaEvent_t ready, done;
    Clock::time_point t;
    bool launched = false;
    int code = MBL_OK;
    std::string err;
};

struct Group {
    const Plan *plan;
    int prec, p;
    int active = 0;
    std::deque<BatchReq *> pending;
    DevMem tab, io;  // device tables (max_jobs entries)
    char *host = nullptr;  // pinned: RING slots of max_jobs SolveBufs<double> + max_jobs SolveIO
    cudaEvent_t ring_ev[RING] = {};
    int ring_pos = 0;
    std::vector<cudaGraphExec_t> graphs;  // by job count
    std::vector<long long> nodes;
};

struct Timing {
    cudaEvent_t e0, e1;
    double bytes;
};

}  // namespace

struct SolveBatcher {
    mbl_ctx *bctx = nullptr;  // own context: stream and table allocations
    int max_jobs = 16;
    double window_us = 300.0;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_b, cv_w;
    std::map<std::tuple<const Plan *, int, int>, std::unique_ptr<Group>> groups;
    bool stop = false;
    // statistics of the launched batches (tmu: the batcher thread writes them outside mu)
    std::mutex tmu;
    int64_t batches = 0, solves = 0;
    double ms = 0.0, bytes = 0.0;
    std::vector<Timing> timing;
    std::vector<cudaEvent_t> ev_pool;

    Group &group(const Plan *pl, int prec, int p) {
        auto &g = groups[std::make_tuple(pl, prec, p)];
        if (!g) {
            g = std::make_unique<Group>();
            g->plan = pl;
            g->prec = prec;
            g->p = p;
        }
        return *g;
    }
    void loop();
    void launch(Group &g, std::vector<BatchReq *> &reqs);
    void resolve(bool wait);
    cudaEvent_t take_event() {
        if (!ev_pool.empty()) {
            cudaEvent_t e = ev_pool.back();
            ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        MBL_CUDA(cudaEventCreate(&e));
        return e;
    }
};

void SolveBatcher::resolve(bool wait) {
    size_t k = 0;
    for (; k < timing.size(); ++k) {
        Timing &t = timing[k];
        if (!wait && cudaEventQuery(t.e1) != cudaSuccess) break;
        MBL_CUDA(cudaEventSynchronize(t.e1));
        float m = 0.f;
        MBL_CUDA(cudaEventElapsedTime(&m, t.e0, t.e1));
        ms += m;
        bytes += t.bytes;
        ev_pool.push_back(t.e0);
        ev_pool.push_back(t.e1);
    }
    (void)cudaGetLastError();  // a cudaEventQuery of unfinished work reports cudaErrorNotReady
    timing.erase(timing.begin(), timing.begin() + (ptrdiff_t)k);
}

void SolveBatcher::launch(Group &g, std::vector<BatchReq *> &reqs) {
    const unsigned K = (unsigned)reqs.size();
    cudaStream_t st = bctx->stream;
    const size_t es = g.prec == MBL_PREC_FP64 ? sizeof(SolveBufs<double>) : sizeof(SolveBufs<float>);
    if (!g.host) {
        g.tab.alloc(bctx, es * max_jobs);
        g.io.alloc(bctx, sizeof(SolveIO) * max_jobs);
        MBL_CUDA(cudaMallocHost(&g.host, (size_t)RING * max_jobs * (sizeof(SolveBufs<double>) + sizeof(SolveIO))));
        for (auto &e : g.ring_ev) {
            MBL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            MBL_CUDA(cudaEventRecord(e, st));
        }
        g.graphs.assign(max_jobs + 1, nullptr);
        g.nodes.assign(max_jobs + 1, 0);
    }
    for (BatchReq *r : reqs) MBL_CUDA(cudaStreamWaitEvent(st, r->ready, 0));
    const int slot = g.ring_pos++ % RING;
    MBL_CUDA(cudaEventSynchronize(g.ring_ev[slot]));  // its previous copies have left the slot
    char *hb = g.host + (size_t)slot * max_jobs * (sizeof(SolveBufs<double>) + sizeof(SolveIO));
    SolveIO *hio = reinterpret_cast<SolveIO *>(hb + (size_t)max_jobs * sizeof(SolveBufs<double>));
    for (unsigned k = 0; k < K; ++k) {
        const BatchReq &r = *reqs[k];
        if (g.prec == MBL_PREC_FP64) reinterpret_cast<SolveBufs<double> *>(hb)[k] = solve_bufs<double>(*r.fz);
        else reinterpret_cast<SolveBufs<float> *>(hb)[k] = solve_bufs<float>(*r.fz);
        hio[k] = SolveIO{r.B, r.X, r.ldb, r.ldx, 1, 1, r.accumulate ? 1 : 0, 0};
    }
    MBL_CUDA(cudaMemcpyAsync(g.tab.p, hb, es * K, cudaMemcpyHostToDevice, st));
    MBL_CUDA(cudaMemcpyAsync(g.io.p, hio, sizeof(SolveIO) * K, cudaMemcpyHostToDevice, st));
    MBL_CUDA(cudaEventRecord(g.ring_ev[slot], st));
    if (!g.graphs[K]) {
        cudaGraph_t graph;
        const long long before = t_launches;
        MBL_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            enqueue_batched_solve(*g.plan, g.prec, g.tab.p, static_cast<const SolveIO *>(g.io.p), K, g.p, st);
        } catch (...) {
            cudaGraph_t dummy = nullptr;
            cudaStreamEndCapture(st, &dummy);
            if (dummy) cudaGraphDestroy(dummy);
            throw;
        }
        MBL_CUDA(cudaStreamEndCapture(st, &graph));
        g.nodes[K] = t_launches - before;
        t_launches = before;
        g_launches.fetch_sub(g.nodes[K]);  // counted when replayed
        MBL_CUDA(cudaGraphInstantiate(&g.graphs[K], graph, 0));
        cudaGraphDestroy(graph);
    }
    std::lock_guard<std::mutex> tl(tmu);
    Timing t{take_event(), take_event(), 0.0};
    const double es_f = g.prec == MBL_PREC_FP64 ? 8.0 : 4.0;
    t.bytes = K * (2.0 * (double)(g.plan->nnz_l + g.plan->n) * es_f + 16.0 * (double)g.plan->n * g.p);
    MBL_CUDA(cudaEventRecord(t.e0, st));
    MBL_CUDA(cudaGraphLaunch(g.graphs[K], st));
    g_launches.fetch_add(g.nodes[K]);
    MBL_CUDA(cudaEventRecord(t.e1, st));
    timing.push_back(t);
    for (BatchReq *r : reqs) MBL_CUDA(cudaEventRecord(r->done, st));
    batches += 1;
    solves += K;
    if (timing.size() > 256) resolve(false);
}

void SolveBatcher::loop() {
    cudaSetDevice(bctx->device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        if (stop) return;
        Group *ready = nullptr;
        Clock::time_point wake = Clock::time_point::max();
        const auto now = Clock::now();
        for (auto &kv : groups) {
            Group &g = *kv.second;
            if (g.pending.empty()) continue;
            const auto due = g.pending.front()->t + std::chrono::microseconds((int64_t)window_us);
            if ((int)g.pending.size() >= std::max(1, g.active) || (int)g.pending.size() >= max_jobs || due <= now) {
                ready = &g;
                break;
            }
            wake = std::min(wake, due);
        }
        if (!ready) {
            if (wake == Clock::time_point::max()) cv_b.wait(lk);
            else cv_b.wait_until(lk, wake);
            continue;
        }
        std::vector<BatchReq *> reqs;
        while (!ready->pending.empty() && (int)reqs.size() < max_jobs) {
            reqs.push_back(ready->pending.front());
            ready->pending.pop_front();
        }
        lk.unlock();
        int code = MBL_OK;
        std::string err;
        try {
            launch(*ready, reqs);
        } catch (const Error &e) {
            code = e.code;
            err = e.msg;
        } catch (const std::exception &e) {
            code = MBL_ERR_CUDA;
            err = e.what();
        }
        lk.lock();
        for (BatchReq *r : reqs) {
            r->code = code;
            r->err = err;
            r->launched = true;
        }
        cv_w.notify_all();
    }
}

namespace {
// per worker thread: the two events of its (single) outstanding request
struct ThreadEvents {
    cudaEvent_t ready = nullptr, done = nullptr;
    ~ThreadEvents() {
        if (ready) cudaEventDestroy(ready);
        if (done) cudaEventDestroy(done);
    }
};
thread_local ThreadEvents t_ev;
}  // namespace

void batched_solve(SolveBatcher *b, Factorization &fz, const double *B, int64_t ldb, double *X, int64_t ldx, int p,
                   bool accumulate, cudaStream_t st) {
    fz.ensure_solve_work(p);
    if (!t_ev.ready) {
        MBL_CUDA(cudaEventCreateWithFlags(&t_ev.ready, cudaEventDisableTiming));
        MBL_CUDA(cudaEventCreateWithFlags(&t_ev.done, cudaEventDisableTiming));
    }
    BatchReq r{&fz, B, ldb, X, ldx, accumulate, t_ev.ready, t_ev.done, Clock::now()};
    MBL_CUDA(cudaEventRecord(r.ready, st));
    {
        std::unique_lock<std::mutex> lk(b->mu);
        if (b->stop) fail(MBL_ERR_INVALID, "solve batcher stopped");
        b->group(fz.plan.get(), fz.prec, p).pending.push_back(&r);
        b->cv_b.notify_one();
        b->cv_w.wait(lk, [&] { return r.launched || b->stop; });
        if (!r.launched) {
            auto &q = b->group(fz.plan.get(), fz.prec, p).pending;
            q.erase(std::remove(q.begin(), q.end(), &r), q.end());
            fail(MBL_ERR_INVALID, "solve batcher stopped");
        }
    }
    if (r.code != MBL_OK) fail(r.code, "batched solve: " + r.err);
    MBL_CUDA(cudaStreamWaitEvent(st, r.done, 0));
}

void batcher_enter(SolveBatcher *b, const Plan *pl, int prec, int p) {
    if (!b) return;
    std::lock_guard<std::mutex> lk(b->mu);
    b->group(pl, prec, p).active += 1;
}

void batcher_leave(SolveBatcher *b, const Plan *pl, int prec, int p) {
    if (!b) return;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        b->group(pl, prec, p).active -= 1;
    }
    b->cv_b.notify_one();  // the others may now be all there is to wait for
}

SolveBatcher *batcher_create(int device, int max_jobs, double window_us) {
    auto b = std::make_unique<SolveBatcher>();
    b->max_jobs = max_jobs;
    b->window_us = window_us;
    int rc = mbl_ctx_create(device, 0, &b->bctx);
    if (rc != MBL_OK) fail(rc, std::string("solve batcher context: ") + mbl_last_error(nullptr));
    SolveBatcher *raw = b.release();
    raw->th = std::thread([raw] { raw->loop(); });
    return raw;
}

void batcher_destroy(SolveBatcher *b) {
    if (!b) return;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        b->stop = true;
    }
    b->cv_b.notify_all();
    b->cv_w.notify_all();
    if (b->th.joinable()) b->th.join();
    cudaSetDevice(b->bctx->device);
    cudaStreamSynchronize(b->bctx->stream);
    try {
        b->resolve(true);
    } catch (...) {
    }
    for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
    for (auto &kv : b->groups) {
        Group &g = *kv.second;
        for (cudaGraphExec_t x : g.graphs)
            if (x) cudaGraphExecDestroy(x);
        for (cudaEvent_t e : g.ring_ev)
            if (e) cudaEventDestroy(e);
        if (g.host) cudaFreeHost(g.host);
        g.tab.release();
        g.io.release();
    }
    b->groups.clear();
    mbl_ctx_destroy(b->bctx);
    delete b;
}

void batcher_stats(SolveBatcher *b, int64_t *batches, int64_t *solves, double *ms, double *bytes) {
    std::lock_guard<std::mutex> lk(b->tmu);
    b->resolve(true);
    *batches = b->batches;
    *solves = b->solves;
    *ms = b->ms;
    *bytes = b->bytes;
}

}  // namespace mbl
