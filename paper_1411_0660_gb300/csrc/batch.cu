// batch.cu -- continuous batching of triangular solves across serving workers.
//
// Jobs of one sector size share one symbolic plan, so their block solves are the same launch
// sequence on different buffers.  A serving worker's solve does not launch that sequence itself:
// it records an event on its stream, hands the request (factorization, right-hand sides, output)
// to the batcher and waits until the batch holding it is launched.  The batcher thread collects
// the requests of one (plan, precision, block width) and launches them on one of its `lanes`
// streams: when every worker inside a solve phase of that group has one pending, when `max_jobs`
// are pending, or, while a lane of the group is idle, when the oldest has waited `window`.  While
// every lane is executing a batch, new requests could not start earlier by being queued behind one
// of them, so they gather and leave together when a lane completes (a host callback on the lane's
// stream reports that): the batch size follows the arrival rate, as in continuous batching, and
// the lanes let a few batched sequences overlap (one sequence is a chain of short dependent
// launches that does not fill the GPU by itself).  A launch makes the lane's stream wait for the
// requests' events, writes the jobs' buffer and right-hand-side tables, and replays the lane's
// graph of the batched sequence for that many jobs (one graph per job count, captured when the
// lane is first used): every launch of the sequence covers all jobs (grid z = job).  Each
// request's `done` event is recorded after the graph, and the worker's stream waits for it.
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

constexpr int RING = 16;  // pinned host table slots in flight per lane

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

// One lane of a group: its device tables, their pinned staging ring and its graphs.  The tables are
// written and read in the lane's stream order only, so batches queued on one lane never overlap.
struct Lane {
    DevMem tab, io;        // device tables (max_jobs entries)
    char *host = nullptr;  // pinned: RING slots of max_jobs SolveBufs<double> + max_jobs SolveIO
    cudaEvent_t ring_ev[RING] = {};
    int ring_pos = 0;
    std::vector<cudaGraphExec_t> graphs;  // by job count
    std::vector<long long> nodes;
    int inflight = 0;  // batches launched on the lane and not yet completed
};

struct Group {
    const Plan *plan;
    int prec, p;
    int active = 0;
    std::deque<BatchReq *> pending;
    std::vector<Lane> lanes;
    int next = 0;  // round robin when every lane is busy
    int idle_lane() const {
        for (size_t i = 0; i < lanes.size(); ++i)
            if (lanes[i].inflight == 0) return (int)i;
        return -1;
    }
};

struct Timing {
    cudaEvent_t e0, e1;
    double bytes;
};

}  // namespace

struct SolveBatcher {
    mbl_ctx *bctx = nullptr;  // own context: table allocations
    int max_jobs = 16;
    double window_us = 300.0;
    std::vector<cudaStream_t> streams;  // one per lane
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
    // the union of the batches' intervals: start and end of each resolved batch relative to the first
    // batch of the current window (wref, its start event), merged when the window closes
    cudaEvent_t wref = nullptr;
    std::vector<std::pair<float, float>> ivals;
    double busy_ms = 0.0;
    void close_window();

    Group &group(const Plan *pl, int prec, int p) {
        auto &g = groups[std::make_tuple(pl, prec, p)];
        if (!g) {
            g = std::make_unique<Group>();
            g->plan = pl;
            g->prec = prec;
            g->p = p;
            g->lanes.resize(streams.size());
        }
        return *g;
    }
    void loop();
    void launch(Group &g, int lane, std::vector<BatchReq *> &reqs, bool &callback);
    void capture(Group &g, int lane, unsigned k);
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
        float a = 0.f;
        if (!wref) wref = t.e0;  // kept (not returned to the pool) until the window closes
        else MBL_CUDA(cudaEventElapsedTime(&a, wref, t.e0));
        ivals.emplace_back(a, a + m);
        if (t.e0 != wref) ev_pool.push_back(t.e0);
        ev_pool.push_back(t.e1);
    }
    (void)cudaGetLastError();  // a cudaEventQuery of unfinished work reports cudaErrorNotReady
    timing.erase(timing.begin(), timing.begin() + (ptrdiff_t)k);
}

void SolveBatcher::close_window() {
    std::sort(ivals.begin(), ivals.end());
    double end = -1e300;
    for (const auto &iv : ivals) {
        if (iv.first > end) {
            busy_ms += iv.second - iv.first;
            end = iv.second;
        } else if (iv.second > end) {
            busy_ms += iv.second - end;
            end = iv.second;
        }
    }
    ivals.clear();
    if (wref) ev_pool.push_back(wref);
    wref = nullptr;
}

// The graph of the batched launch sequence for k jobs on lane `li` (tables at the lane's tab / io).
void SolveBatcher::capture(Group &g, int li, unsigned k) {
    Lane &ln = g.lanes[li];
    if (ln.graphs[k]) return;
    cudaStream_t st = streams[li];
    cudaGraph_t graph;
    const long long before = t_launches;
    MBL_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
        enqueue_batched_solve(*g.plan, g.prec, ln.tab.p, static_cast<const SolveIO *>(ln.io.p), k, g.p, st);
    } catch (...) {
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(st, &dummy);
        if (dummy) cudaGraphDestroy(dummy);
        throw;
    }
    MBL_CUDA(cudaStreamEndCapture(st, &graph));
    ln.nodes[k] = t_launches - before;
    t_launches = before;
    g_launches.fetch_sub(ln.nodes[k]);  // counted when replayed
    MBL_CUDA(cudaGraphInstantiate(&ln.graphs[k], graph, 0));
    cudaGraphDestroy(graph);
}

namespace {
struct DoneCallback {
    SolveBatcher *b;
    Group *g;
    int lane;
};

// Runs on a driver thread once a batch's work on its lane has completed (no CUDA calls here).
void CUDART_CB batch_done(void *arg) {
    DoneCallback *c = static_cast<DoneCallback *>(arg);
    {
        std::lock_guard<std::mutex> lk(c->b->mu);
        c->g->lanes[c->lane].inflight -= 1;
    }
    c->b->cv_b.notify_one();
    delete c;
}
}  // namespace

void SolveBatcher::launch(Group &g, int li, std::vector<BatchReq *> &reqs, bool &callback) {
    const unsigned K = (unsigned)reqs.size();
    Lane &ln = g.lanes[li];
    cudaStream_t st = streams[li];
    const size_t es = g.prec == MBL_PREC_FP64 ? sizeof(SolveBufs<double>) : sizeof(SolveBufs<float>);
    if (!ln.host) {
        ln.tab.alloc(bctx, es * max_jobs);
        ln.io.alloc(bctx, sizeof(SolveIO) * max_jobs);
        MBL_CUDA(cudaMallocHost(&ln.host, (size_t)RING * max_jobs * (sizeof(SolveBufs<double>) + sizeof(SolveIO))));
        for (auto &e : ln.ring_ev) {
            MBL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            MBL_CUDA(cudaEventRecord(e, st));
        }
        ln.graphs.assign(max_jobs + 1, nullptr);
        ln.nodes.assign(max_jobs + 1, 0);
        // first batch of the lane: capture the graphs of every job count now, so that no later
        // batch pays for a capture in the middle of the jobs' solves
        for (unsigned k = 1; k <= (unsigned)max_jobs; ++k) capture(g, li, k);
    }
    for (BatchReq *r : reqs) MBL_CUDA(cudaStreamWaitEvent(st, r->ready, 0));
    const int slot = ln.ring_pos++ % RING;
    MBL_CUDA(cudaEventSynchronize(ln.ring_ev[slot]));  // its previous copies have left the slot
    char *hb = ln.host + (size_t)slot * max_jobs * (sizeof(SolveBufs<double>) + sizeof(SolveIO));
    SolveIO *hio = reinterpret_cast<SolveIO *>(hb + (size_t)max_jobs * sizeof(SolveBufs<double>));
    for (unsigned k = 0; k < K; ++k) {
        const BatchReq &r = *reqs[k];
        if (g.prec == MBL_PREC_FP64) reinterpret_cast<SolveBufs<double> *>(hb)[k] = solve_bufs<double>(*r.fz);
        else reinterpret_cast<SolveBufs<float> *>(hb)[k] = solve_bufs<float>(*r.fz);
        hio[k] = SolveIO{r.B, r.X, r.ldb, r.ldx, 1, 1, r.accumulate ? 1 : 0, 0};
    }
    MBL_CUDA(cudaMemcpyAsync(ln.tab.p, hb, es * K, cudaMemcpyHostToDevice, st));
    MBL_CUDA(cudaMemcpyAsync(ln.io.p, hio, sizeof(SolveIO) * K, cudaMemcpyHostToDevice, st));
    MBL_CUDA(cudaEventRecord(ln.ring_ev[slot], st));
    std::lock_guard<std::mutex> tl(tmu);
    Timing t{take_event(), take_event(), 0.0};
    const double es_f = g.prec == MBL_PREC_FP64 ? 8.0 : 4.0;
    t.bytes = K * (2.0 * (double)(g.plan->nnz_l + g.plan->n) * es_f + 16.0 * (double)g.plan->n * g.p);
    MBL_CUDA(cudaEventRecord(t.e0, st));
    MBL_CUDA(cudaGraphLaunch(ln.graphs[K], st));
    g_launches.fetch_add(ln.nodes[K]);
    MBL_CUDA(cudaEventRecord(t.e1, st));
    timing.push_back(t);
    for (BatchReq *r : reqs) MBL_CUDA(cudaEventRecord(r->done, st));
    DoneCallback *cb = new DoneCallback{this, &g, li};
    if (cudaLaunchHostFunc(st, batch_done, cb) != cudaSuccess) {
        delete cb;
        fail(MBL_ERR_CUDA, "solve batcher: cudaLaunchHostFunc failed");
    }
    callback = true;
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
        int lane = -1;
        Clock::time_point wake = Clock::time_point::max();
        const auto now = Clock::now();
        for (auto &kv : groups) {
            Group &g = *kv.second;
            if (g.pending.empty()) continue;
            const auto due = g.pending.front()->t + std::chrono::microseconds((int64_t)window_us);
            const int idle = g.idle_lane();
            if ((int)g.pending.size() >= std::max(1, g.active) || (int)g.pending.size() >= max_jobs ||
                (idle >= 0 && due <= now)) {
                ready = &g;
                lane = idle >= 0 ? idle : g.next++ % (int)g.lanes.size();  // busy: queue behind one
                break;
            }
            if (idle >= 0) wake = std::min(wake, due);  // else a completion callback wakes us
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
        ready->lanes[lane].inflight += 1;
        lk.unlock();
        int code = MBL_OK;
        std::string err;
        bool callback = false;
        try {
            launch(*ready, lane, reqs, callback);
        } catch (const Error &e) {
            code = e.code;
            err = e.msg;
        } catch (const std::exception &e) {
            code = MBL_ERR_CUDA;
            err = e.what();
        }
        lk.lock();
        if (!callback) ready->lanes[lane].inflight -= 1;
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

SolveBatcher *batcher_create(int device, int max_jobs, double window_us, int lanes) {
    auto b = std::make_unique<SolveBatcher>();
    b->max_jobs = max_jobs;
    b->window_us = window_us;
    int rc = mbl_ctx_create(device, 0, &b->bctx);
    if (rc != MBL_OK) fail(rc, std::string("solve batcher context: ") + mbl_last_error(nullptr));
    MBL_CUDA(cudaSetDevice(device));
    for (int i = 0; i < std::max(1, lanes); ++i) {
        cudaStream_t s;
        MBL_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        b->streams.push_back(s);
    }
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
    for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);  // the completion callbacks too
    try {
        b->resolve(true);
        b->close_window();
    } catch (...) {
    }
    for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
    for (auto &kv : b->groups) {
        for (Lane &ln : kv.second->lanes) {
            for (cudaGraphExec_t x : ln.graphs)
                if (x) cudaGraphExecDestroy(x);
            for (cudaEvent_t e : ln.ring_ev)
                if (e) cudaEventDestroy(e);
            if (ln.host) cudaFreeHost(ln.host);
            ln.tab.release();
            ln.io.release();
        }
    }
    b->groups.clear();
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    mbl_ctx_destroy(b->bctx);
    delete b;
}

void batcher_stats(SolveBatcher *b, int64_t *batches, int64_t *solves, double *ms, double *bytes, double *busy_ms) {
    std::lock_guard<std::mutex> lk(b->tmu);
    b->resolve(true);
    b->close_window();
    *batches = b->batches;
    *solves = b->solves;
    *ms = b->ms;
    *bytes = b->bytes;
    *busy_ms = b->busy_ms;
}

}  // namespace mbl
