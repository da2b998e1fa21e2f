// capi.cu -- the extern "C" boundary of libmblsi (see include/mblsi.h for the contract).
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <set>

#include "krylov.h"
#include "observables.h"

namespace mbl {

std::atomic<long long> g_launches{0};
thread_local long long t_launches = 0;

// Contexts that are alive: objects that outlive their context (a sector or factorization released
// after mbl_ctx_destroy) free their device memory without touching the dead context.
static std::mutex g_ctx_mu;
static std::set<const Ctx *> &live_ctx() {
    static std::set<const Ctx *> *s = new std::set<const Ctx *>();
    return *s;
}
bool ctx_alive(const Ctx *c) {
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    return c && live_ctx().count(c) != 0;
}

void smem_limit(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> *done = new std::map<std::pair<const void *, int>, size_t>();
    int dev = 0;
    MBL_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t &have = (*done)[{fn, dev}];
    if (have >= bytes) return;
    MBL_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    have = bytes;
}

cudaEvent_t Ctx::take_event() {
    if (!event_pool.empty()) {
        cudaEvent_t e = event_pool.back();
        event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    MBL_CUDA(cudaEventCreate(&e));
    return e;
}

void Ctx::resolve_profile() {
    for (auto &kv : profile) {
        ProfAcc &a = kv.second;
        for (auto &pd : a.pending) {
            MBL_CUDA(cudaEventSynchronize(pd.e1));
            float ms = 0.f;
            MBL_CUDA(cudaEventElapsedTime(&ms, pd.e0, pd.e1));
            a.ms += ms;
            a.work += pd.work;
            a.launches += 1;
            event_pool.push_back(pd.e0);
            event_pool.push_back(pd.e1);
        }
        a.pending.clear();
    }
}

ProfScope::ProfScope(Ctx *c_, const char *name_, double work_, cudaStream_t st_) : c(c_), name(name_), work(work_), st(st_) {
    if (c && c->prof) {
        e0 = c->take_event();
        MBL_CUDA(cudaEventRecord(e0, st));
    }
}

ProfScope::~ProfScope() {
    if (!e0) return;
    cudaEvent_t e1 = c->take_event();
    cudaEventRecord(e1, st);
    c->profile[name].pending.push_back(ProfAcc::Pending{e0, e1, work});
}

DevMem &DevMem::operator=(DevMem &&o) noexcept {
    if (this != &o) {
        release();
        p = o.p;
        bytes = o.bytes;
        ctx = o.ctx;
        o.p = nullptr;
        o.bytes = 0;
        o.ctx = nullptr;
    }
    return *this;
}

// Device memory comes from one stream-ordered pool per device that keeps freed blocks cached
// (release threshold: unlimited): a job's factor, fronts and Krylov basis are reused by the next
// job without cudaMalloc/cudaFree, whose implicit device synchronization would stall the other
// contexts' streams.  mbl_ctx_destroy trims the pool.
static std::mutex g_pool_mu;
static cudaMemPool_t device_pool(int device) {
    static std::map<int, cudaMemPool_t> *pools = new std::map<int, cudaMemPool_t>();
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = pools->find(device);
    if (it != pools->end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool;
    MBL_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t thr = UINT64_MAX;
    MBL_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    (*pools)[device] = pool;
    return pool;
}

void trim_device_pool(int device) { cudaMemPoolTrimTo(device_pool(device), 0); }

void DevMem::alloc(Ctx *c, size_t nbytes) {
    release();
    if (nbytes == 0) nbytes = 16;
    if (c->budget && c->in_use + nbytes > c->budget)
        fail(MBL_ERR_OOM, "allocation of " + std::to_string(nbytes) + " bytes exceeds the context budget");
    cudaError_t e = cudaMallocFromPoolAsync(&p, nbytes, device_pool(c->device), c->stream);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        p = nullptr;
        fail(MBL_ERR_OOM, "device allocation of " + std::to_string(nbytes) + " bytes failed");
    }
    MBL_CUDA(e);
    // a block reused from another stream may still be waited on by that stream's work: settle it
    // before any copy outside this stream touches the block
    MBL_CUDA(cudaStreamSynchronize(c->stream));
    bytes = nbytes;
    ctx = c;
    c->in_use += nbytes;
    if (c->in_use > c->peak) c->peak = c->in_use;
}

void DevMem::release() {
    if (p) {
        const bool live = ctx && ctx_alive(ctx);
        cudaFreeAsync(p, live ? ctx->stream : (cudaStream_t)0);
        if (live) ctx->in_use -= bytes;
    }
    p = nullptr;
    bytes = 0;
}

std::shared_ptr<Plan> get_plan(mbl_sector *sec) {
    Ctx *ctx = sec->ctx;
    std::shared_ptr<PlanCache> cache = ctx->plans;
    std::lock_guard<std::mutex> lk(cache->mu);
    const int ordering = resolve_ordering(cache->ordering, sec->n);
    const int key = plan_key(sec->L, sec->nup, ordering);
    auto it = cache->m.find(key);
    if (it != cache->m.end()) return it->second;
    int64_t n = sec->n;
    std::vector<uint32_t> st(n);
    std::vector<int64_t> rp(n + 1);
    std::vector<int32_t> col(sec->nnz);
    MBL_CUDA(cudaStreamSynchronize(ctx->stream));
    MBL_CUDA(cudaMemcpy(st.data(), sec->states.data(), n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    MBL_CUDA(cudaMemcpy(rp.data(), sec->rowptr.data(), (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    MBL_CUDA(cudaMemcpy(col.data(), sec->col.data(), sec->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
    auto P = build_plan(sec->L, st, rp, col, ordering);
    upload_plan(ctx, *P);
    cache->m[key] = P;
    return P;
}

uint64_t wait_limit_ns(double seconds) {
    if (!(seconds >= 0.0) || seconds > 60.0) fail(MBL_ERR_INVALID, "wait_limit_s must be in [0, 60]");
    if (seconds == 0.0) return 1000000000ull;
    return std::max<uint64_t>(1, (uint64_t)(seconds * 1e9));
}

std::unique_ptr<Factorization> make_factorization(mbl_sector *sec, double sigma, int prec, double hnorm, int tc_mode,
                                                  bool dataflow, uint64_t wait_ns, int arena_mode, double pivot_tiny) {
    if (!(pivot_tiny >= 0.0 && pivot_tiny < 1.0)) fail(MBL_ERR_INVALID, "pivot_tiny must be in [0, 1)");
    if (arena_mode < ARENA_AUTO || arena_mode > ARENA_FULL) fail(MBL_ERR_INVALID, "arena_mode must be 0, 1 or 2");
    if (prec != MBL_PREC_FP64 && prec != MBL_PREC_FP32) fail(MBL_ERR_INVALID, "unknown precision");
    if (tc_mode < 0 || tc_mode > 2) fail(MBL_ERR_INVALID, "tensor_cores must be 0, 1 (3xTF32) or 2 (3xBF16)");
    auto F = std::make_unique<Factorization>();
    F->ctx = sec->ctx;
    F->sec = sec;
    F->plan = get_plan(sec);
    F->sigma = sigma;
    F->prec = prec;
    F->tiny = (pivot_tiny > 0.0 ? pivot_tiny : (prec == MBL_PREC_FP64 ? 1e-12 : 1e-7)) * hnorm;
    F->tc_mode = tc_mode;
    F->dataflow = dataflow;
    F->wait_ns = wait_ns;
    F->allocate(arena_is_lean(*F->plan, prec, arena_mode));
    cudaStream_t st = sec->ctx->stream;
    cudaEvent_t e0, e1;
    MBL_CUDA(cudaEventCreate(&e0));
    MBL_CUDA(cudaEventCreate(&e1));
    tune_schur(*F, st);  // once per plan and tensor-core mode, before the timed factorization
    MBL_CUDA(cudaEventRecord(e0, st));
    {
        ProfScope ps(sec->ctx, prec == MBL_PREC_FP64 ? "factor_fp64" : "factor_fp32", F->plan->flops, st);
        numeric_factor(*F, st);
    }
    MBL_CUDA(cudaEventRecord(e1, st));
    MBL_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    MBL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    F->ms_factor = ms;
    unsigned long long cnt[5];
    MBL_CUDA(cudaMemcpy(cnt, F->counters.data(), sizeof(cnt), cudaMemcpyDeviceToHost));
    F->perturbed = (int64_t)cnt[0];
    F->negative = (int64_t)cnt[1];
    uint32_t ml = (uint32_t)(cnt[3] & 0xffffffffu), md = (uint32_t)(cnt[4] & 0xffffffffu);
    std::memcpy(&F->max_l, &ml, 4);
    std::memcpy(&F->min_d, &md, 4);
    if (cnt[2] != 0) fail(MBL_ERR_TIMEOUT, "tensor-core tile wait timed out in the factorization");
    F->release_scratch();
    return F;
}

}  // namespace mbl

using namespace mbl;

static thread_local std::string g_last_error;

static int report(Ctx *ctx, int code, const std::string &msg) {
    g_last_error = msg;
    if (ctx) ctx->last_error = msg;
    return code;
}

#define API_TRY try {
#define API_CATCH(CTX)                                                               \
    }                                                                                \
    catch (const mbl::Error &e) {                                                    \
        return report((CTX), e.code, e.msg);                                         \
    }                                                                                \
    catch (const std::bad_alloc &) {                                                 \
        return report((CTX), MBL_ERR_OOM, "host allocation failed");                 \
    }                                                                                \
    catch (const std::exception &e) {                                                \
        return report((CTX), MBL_ERR_INVALID, e.what());                             \
    }                                                                                \
    return MBL_OK;

extern "C" {

void mbl_opts_default(mbl_opts *o) {
    if (!o) return;
    o->precision = MBL_PREC_FP32;
    o->block = 8;
    o->ncv = 0;
    o->max_restarts = 60;
    o->tol = 1e-10;
    o->target_tol = 1e-13;
    o->refine_tol = 1e-14;
    o->max_refine = 20;
    o->start_seed = 12345;
    o->tensor_cores = 1;
    o->refine_mode = 1;
    o->gmres_restart = 24;
    o->solve_dataflow = 0;
    o->deflate = 1;
    o->wait_limit_s = 0.0;
    o->arena_mode = 0;
    o->pivot_tiny = 0.0;
}

const char *mbl_version(void) { return "mblsi 0.1 (sm_103a)"; }

const char *mbl_last_error(mbl_ctx *ctx) { return ctx ? ctx->last_error.c_str() : g_last_error.c_str(); }

const char *mbl_status_string(int s) {
    switch (s) {
        case MBL_OK: return "ok";
        case MBL_ERR_INVALID: return "invalid argument";
        case MBL_ERR_OOM: return "out of memory budget";
        case MBL_ERR_SINGULAR: return "singular factorization";
        case MBL_ERR_NOT_CONVERGED: return "not converged";
        case MBL_ERR_TIMEOUT: return "device wait timed out";
        case MBL_ERR_CUDA: return "CUDA error";
        case MBL_PENDING: return "pending";
        default: return "unknown status";
    }
}

int mbl_ctx_create(int device, size_t budget, mbl_ctx **out) {
    if (!out) return report(nullptr, MBL_ERR_INVALID, "out is NULL");
    *out = nullptr;
    mbl_ctx *c = nullptr;
    API_TRY
    int ndev = 0;
    MBL_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) fail(MBL_ERR_INVALID, "no such CUDA device");
    MBL_CUDA(cudaSetDevice(device));
    c = new mbl_ctx();
    c->device = device;
    c->budget = budget;
    MBL_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    MBL_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
    upload_binomials();
    noalloc_setup(device);
    {
        std::lock_guard<std::mutex> lk(g_ctx_mu);
        live_ctx().insert(c);
    }
    *out = c;
    c = nullptr;
    }
    catch (const mbl::Error &e) {
        delete c;
        return report(nullptr, e.code, e.msg);
    }
    return MBL_OK;
}

long long mbl_launch_count(void) { return mbl::g_launches.load(); }

int mbl_ctx_set_profiling(mbl_ctx *ctx, int on) {
    if (!ctx) return report(nullptr, MBL_ERR_INVALID, "ctx is NULL");
    API_TRY
    ctx->resolve_profile();
    ctx->profile.clear();
    ctx->prof = on != 0;
    API_CATCH(ctx)
}

int mbl_ctx_set_ordering(mbl_ctx *ctx, int ordering) {
    if (!ctx) return report(nullptr, MBL_ERR_INVALID, "ctx is NULL");
    if (ordering < MBL_ORDER_BAND || ordering > MBL_ORDER_HYBRID) return report(ctx, MBL_ERR_INVALID, "unknown ordering");
    API_TRY
    std::lock_guard<std::mutex> lk(ctx->plans->mu);
    ctx->plans->ordering = ordering;
    API_CATCH(ctx)
}

int mbl_ctx_profile_get(mbl_ctx *ctx, const char *name, int64_t *launches, double *ms, double *work) {
    if (!ctx || !name) return report(ctx, MBL_ERR_INVALID, "NULL argument");
    API_TRY
    ctx->resolve_profile();
    auto it = ctx->profile.find(name);
    if (launches) *launches = it == ctx->profile.end() ? 0 : it->second.launches;
    if (ms) *ms = it == ctx->profile.end() ? 0.0 : it->second.ms;
    if (work) *work = it == ctx->profile.end() ? 0.0 : it->second.work;
    API_CATCH(ctx)
}

void mbl_ctx_destroy(mbl_ctx *ctx) {
    if (!ctx || !ctx_alive(ctx)) return;
    server_shutdown(ctx);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    try { ctx->resolve_profile(); } catch (...) {}
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    {
        std::lock_guard<std::mutex> lk(ctx->plans->mu);
        if (ctx->plans.use_count() == 1) ctx->plans->m.clear();
    }
    ctx->plans.reset();
    ctx->ent.clear();
    cudaStreamSynchronize(ctx->stream);
    cudaStreamDestroy(ctx->stream);
    {
        std::lock_guard<std::mutex> lk(g_ctx_mu);
        live_ctx().erase(ctx);
    }
    const int dev = ctx->device;
    delete ctx;
    trim_device_pool(dev);
}

int mbl_ctx_synchronize(mbl_ctx *ctx) {
    API_TRY
    MBL_CUDA(cudaStreamSynchronize(ctx->stream));
    API_CATCH(ctx)
}

static int build_common(mbl_ctx *ctx, int L, int nup, const double *h_host, double J, bool from_seed, double h,
                        uint64_t seed, mbl_sector **out) {
    if (!ctx || !out) return report(ctx, MBL_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (L < 2 || L > 22) return report(ctx, MBL_ERR_INVALID, "L must satisfy 2 <= L <= 22");
    if (nup < 0 || nup > L) return report(ctx, MBL_ERR_INVALID, "nup must satisfy 0 <= nup <= L");
    if (from_seed && !(h >= 0.0)) return report(ctx, MBL_ERR_INVALID, "h must be >= 0");
    mbl_sector *s = new mbl_sector();
    API_TRY
    MBL_CUDA(cudaSetDevice(ctx->device));
    s->ctx = ctx;
    s->L = L;
    s->nup = nup;
    s->J = J;
    const int64_t n = host_binom(L, nup);
    s->n = n;
    ProfScope ps(ctx, "sector_build", (double)n, ctx->stream);
    s->d_hfield.alloc(ctx, 32);
    if (from_seed) {
        launch_fields(L, h, seed, s->d_hfield.data(), ctx->stream);
        MBL_CUDA(cudaMemcpyAsync(s->hfield, s->d_hfield.data(), L * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    } else {
        std::memcpy(s->hfield, h_host, L * sizeof(double));
        MBL_CUDA(cudaMemcpyAsync(s->d_hfield.data(), s->hfield, L * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    }
    build_sector_device(s, ctx->stream);
    *out = s;
    s = nullptr;
    }
    catch (const mbl::Error &e) {
        delete s;
        return report(ctx, e.code, e.msg);
    }
    return MBL_OK;
}

int mbl_build_sector(mbl_ctx *ctx, int L, double h, uint64_t seed, mbl_sector **out) {
    if (L & 1) return report(ctx, MBL_ERR_INVALID, "L must be even (mbl_build_sector_nup for other sectors)");
    return build_common(ctx, L, L / 2, nullptr, 1.0, true, h, seed, out);
}

int mbl_build_sector_fields(mbl_ctx *ctx, int L, const double *h_i, double J, mbl_sector **out) {
    if (!h_i) return report(ctx, MBL_ERR_INVALID, "h_i is NULL");
    if (L & 1) return report(ctx, MBL_ERR_INVALID, "L must be even (mbl_build_sector_fields_nup for other sectors)");
    return build_common(ctx, L, L / 2, h_i, J, false, 0.0, 0, out);
}

int mbl_build_sector_nup(mbl_ctx *ctx, int L, int nup, double h, uint64_t seed, mbl_sector **out) {
    return build_common(ctx, L, nup, nullptr, 1.0, true, h, seed, out);
}

int mbl_build_sector_fields_nup(mbl_ctx *ctx, int L, int nup, const double *h_i, double J, mbl_sector **out) {
    if (!h_i) return report(ctx, MBL_ERR_INVALID, "h_i is NULL");
    return build_common(ctx, L, nup, h_i, J, false, 0.0, 0, out);
}

int mbl_sector_shape(const mbl_sector *sec, int *L, int *nup) {
    if (!sec) return report(nullptr, MBL_ERR_INVALID, "sector is NULL");
    if (L) *L = sec->L;
    if (nup) *nup = sec->nup;
    return MBL_OK;
}

void mbl_sector_destroy(mbl_sector *sec) {
    if (!sec) return;
    if (ctx_alive(sec->ctx)) cudaStreamSynchronize(sec->ctx->stream);
    delete sec;
}

int mbl_sector_info(const mbl_sector *sec, int64_t *dim, int64_t *nnz) {
    if (!sec) return report(nullptr, MBL_ERR_INVALID, "sector is NULL");
    if (dim) *dim = sec->n;
    if (nnz) *nnz = sec->nnz;
    return MBL_OK;
}

int mbl_sector_copy_basis(const mbl_sector *sec, uint32_t *states) {
    if (!sec || !states) return report(nullptr, MBL_ERR_INVALID, "NULL argument");
    API_TRY
    MBL_CUDA(cudaStreamSynchronize(sec->ctx->stream));
    MBL_CUDA(cudaMemcpy(states, sec->states.data(), sec->n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    API_CATCH(sec->ctx)
}

int mbl_sector_copy_csr(const mbl_sector *sec, int64_t *rowptr, int32_t *col, double *val) {
    if (!sec) return report(nullptr, MBL_ERR_INVALID, "sector is NULL");
    API_TRY
    MBL_CUDA(cudaStreamSynchronize(sec->ctx->stream));
    if (rowptr) MBL_CUDA(cudaMemcpy(rowptr, sec->rowptr.data(), (sec->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (col) MBL_CUDA(cudaMemcpy(col, sec->col.data(), sec->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (val) MBL_CUDA(cudaMemcpy(val, sec->val.data(), sec->nnz * sizeof(double), cudaMemcpyDeviceToHost));
    API_CATCH(sec->ctx)
}

int mbl_sector_copy_fields(const mbl_sector *sec, double *h_i) {
    if (!sec || !h_i) return report(nullptr, MBL_ERR_INVALID, "NULL argument");
    API_TRY
    MBL_CUDA(cudaStreamSynchronize(sec->ctx->stream));
    std::memcpy(h_i, sec->hfield, sec->L * sizeof(double));
    API_CATCH(sec->ctx)
}

int mbl_sector_rank(const mbl_sector *sec, const uint32_t *states, int64_t count, int64_t *ranks) {
    if (!sec || (count > 0 && (!states || !ranks))) return report(nullptr, MBL_ERR_INVALID, "NULL argument");
    API_TRY
    if (count <= 0) return MBL_OK;
    DVec<uint32_t> ds;
    DVec<int64_t> dr;
    ds.alloc(sec->ctx, count);
    dr.alloc(sec->ctx, count);
    MBL_CUDA(cudaMemcpy(ds.data(), states, count * sizeof(uint32_t), cudaMemcpyHostToDevice));
    launch_rank(sec->L, sec->nup, ds.data(), count, dr.data(), sec->ctx->stream);
    MBL_CUDA(cudaStreamSynchronize(sec->ctx->stream));
    MBL_CUDA(cudaMemcpy(ranks, dr.data(), count * sizeof(int64_t), cudaMemcpyDeviceToHost));
    API_CATCH(sec->ctx)
}

int mbl_spmv(mbl_sector *sec, double shift, const double *x, double *y, int nrhs) {
    if (!sec || !x || !y || nrhs < 1) return report(nullptr, MBL_ERR_INVALID, "bad argument");
    API_TRY
    int64_t n = sec->n;
    DVec<double> dx, dy;
    dx.alloc(sec->ctx, (size_t)n * nrhs);
    dy.alloc(sec->ctx, (size_t)n * nrhs);
    MBL_CUDA(cudaMemcpy(dx.data(), x, (size_t)n * nrhs * sizeof(double), cudaMemcpyHostToDevice));
    launch_spmv(sec, shift, dx.data(), 1, n, dy.data(), 1, n, nrhs, sec->ctx->stream);
    MBL_CUDA(cudaStreamSynchronize(sec->ctx->stream));
    MBL_CUDA(cudaMemcpy(y, dy.data(), (size_t)n * nrhs * sizeof(double), cudaMemcpyDeviceToHost));
    API_CATCH(sec->ctx)
}

int mbl_extremal_bounds(mbl_sector *sec, double *e_min, double *e_max) {
    if (!sec || !e_min || !e_max) return report(nullptr, MBL_ERR_INVALID, "NULL argument");
    API_TRY
    MBL_CUDA(cudaSetDevice(sec->ctx->device));
    extremal_bounds(sec, e_min, e_max);
    API_CATCH(sec->ctx)
}

int mbl_factor(mbl_sector *sec, double sigma, const mbl_opts *opts, mbl_factorization **out) {
    if (!sec || !out) return report(nullptr, MBL_ERR_INVALID, "NULL argument");
    *out = nullptr;
    mbl_opts o;
    mbl_opts_default(&o);
    if (opts) o = *opts;
    API_TRY
    MBL_CUDA(cudaSetDevice(sec->ctx->device));
    double emin, emax;
    extremal_bounds(sec, &emin, &emax);
    double hn = std::max(std::fabs(emin), std::fabs(emax));
    auto F = make_factorization(sec, sigma, o.precision, hn, o.tensor_cores, o.solve_dataflow != 0,
                                wait_limit_ns(o.wait_limit_s), o.arena_mode, o.pivot_tiny);
    mbl_factorization *h = new mbl_factorization();
    h->f = std::move(F);
    *out = h;
    API_CATCH(sec->ctx)
}

int mbl_factor_stats_get(const mbl_factorization *fh, mbl_factor_stats *s) {
    if (!fh || !s) return report(nullptr, MBL_ERR_INVALID, "NULL argument");
    const Factorization &f = *fh->f;
    const Plan &p = *f.plan;
    s->n = p.n;
    s->nnz_l = p.nnz_l;
    s->n_supernodes = p.ns;
    s->max_front = p.max_front;
    s->tree_levels = p.nlevels;
    s->perturbed = f.perturbed;
    s->negative = f.negative;
    s->flops = p.flops;
    s->factor_bytes = (double)(p.nnz_l + p.n) * f.elem_size();
    s->front_bytes = f.lean_used ? (double)p.lean_peak_elems * f.elem_size() : (double)p.arena_elems * f.elem_size();
    const int mode = f.prec == MBL_PREC_FP32 && f.tc_mode >= 1 && f.tc_mode <= 2 ? f.tc_mode : 0;
    for (int c = 0; c < TUNE_CLASSES; ++c) {
        s->tune_choice[c] = mode && p.tuned[mode] ? p.tune_tc[mode][c] : -1;
        s->tune_us_tc[c] = mode ? p.tune_us[mode][c][0] : 0.f;
        s->tune_us_cc[c] = mode ? p.tune_us[mode][c][1] : 0.f;
    }
    s->ms_factor = f.ms_factor;
    s->max_abs_l = f.max_l;
    s->min_abs_d = f.min_d;
    return MBL_OK;
}

int mbl_analyse(mbl_sector *sec, int nev, int block, mbl_plan_stats *s) {
    if (!sec || !s) return report(nullptr, MBL_ERR_INVALID, "NULL argument");
    if (nev < 1 || block < 1 || block > 32) return report(sec->ctx, MBL_ERR_INVALID, "nev >= 1, block in 1..32");
    API_TRY
    MBL_CUDA(cudaSetDevice(sec->ctx->device));
    std::shared_ptr<Plan> P = get_plan(sec);
    const Plan &p = *P;
    s->n = p.n;
    s->nnz_l = p.nnz_l;
    s->n_supernodes = p.ns;
    s->max_front = p.max_front;
    s->tree_levels = p.nlevels;
    s->panel_steps = (int64_t)p.steps.size();
    s->solve_steps = (int64_t)p.ssteps.size();
    s->flops = p.flops;
    s->ms_analyse = p.ms_analyse;
    s->factor_bytes_fp32 = (double)(p.nnz_l + p.n) * 4.0;
    s->factor_bytes_fp64 = (double)(p.nnz_l + p.n) * 8.0;
    s->front_bytes_fp32 = (double)p.arena_elems * 4.0;
    s->front_bytes_fp64 = (double)p.arena_elems * 8.0;
    s->solve_factor_bytes_fp32 = (double)p.sg_elems * 4.0;
    s->front_peak_bytes_fp32 = arena_peak_bytes(p, MBL_PREC_FP32, ARENA_AUTO);
    s->front_peak_bytes_fp64 = arena_peak_bytes(p, MBL_PREC_FP64, ARENA_AUTO);
    s->ordering = p.ordering;
    s->job_peak_bytes_fp32 = (double)job_bytes(p, nev, block, MBL_PREC_FP32);
    s->job_peak_bytes_fp64 = (double)job_bytes(p, nev, block, MBL_PREC_FP64);
    API_CATCH(sec->ctx)
}

int mbl_factor_trace(mbl_factorization *fh, int on) {
    if (!fh) return report(nullptr, MBL_ERR_INVALID, "NULL argument");
    Factorization &f = *fh->f;
    if (f.dataflow && on) return report(f.ctx, MBL_ERR_INVALID, "the launch trace covers the level-by-level solve");
    API_TRY
    if (on && f.trace.size() == 0)
        f.trace.alloc(f.ctx, 2 * (size_t)f.plan->nlevels + f.plan->ssteps.size() + f.plan->bupd.size());
    f.trace_on = on != 0;
    f.graph_p = 0;  // recapture the solve sequence with or without the trace records
    API_CATCH(f.ctx)
}

int mbl_factor_trace_get(mbl_factorization *fh, unsigned long long *t0, unsigned long long *t1, int *kind, int cap,
                         int *count) {
    if (!fh || !count || (cap > 0 && (!t0 || !t1 || !kind))) return report(nullptr, MBL_ERR_INVALID, "NULL argument");
    Factorization &f = *fh->f;
    Ctx *ctx = f.ctx;
    API_TRY
    const int nrec = f.trace_on ? (int)f.trace_kind.size() : 0;
    *count = nrec;
    const int m = std::min(cap, nrec);
    if (m > 0) {
        std::vector<LaunchTrace> h(m);
        MBL_CUDA(cudaStreamSynchronize(ctx->stream));
        MBL_CUDA(cudaMemcpy(h.data(), f.trace.data(), m * sizeof(LaunchTrace), cudaMemcpyDeviceToHost));
        for (int i = 0; i < m; ++i) {
            t0[i] = h[i].t0;
            t1[i] = h[i].t1;
            kind[i] = f.trace_kind[i];
        }
    }
    API_CATCH(ctx)
}

int mbl_factor_solve(mbl_factorization *fh, const double *b, double *x, int nrhs, int refine) {
    if (!fh || !b || !x || nrhs < 1) return report(nullptr, MBL_ERR_INVALID, "bad argument");
    Factorization &f = *fh->f;
    Ctx *ctx = f.ctx;
    API_TRY
    cudaStream_t st = ctx->stream;
    int64_t n = f.plan->n;
    DVec<double> cm, B, X;
    cm.alloc(ctx, (size_t)n * nrhs);
    MBL_CUDA(cudaMemcpy(cm.data(), b, (size_t)n * nrhs * sizeof(double), cudaMemcpyHostToDevice));
    double emin, emax;
    extremal_bounds(f.sec, &emin, &emax);
    double hn = std::max(std::fabs(emin), std::fabs(emax));
    RefinedSolve rs{f.sec, &f, hn + std::fabs(f.sigma), 1e-15, 20};
    rs.gmres = 1;
    for (int c0 = 0; c0 < nrhs; c0 += 32) {
        int p = std::min(32, nrhs - c0);
        B.alloc(ctx, (size_t)n * p);
        X.alloc(ctx, (size_t)n * p);
        // column-major host block -> row-major device block (copy_cols on the transposed view)
        for (int q = 0; q < p; ++q) copy_cols(n, cm.data() + (size_t)(c0 + q) * n, 1, 0, B.data(), p, q, 1, st);
        if (refine) rs.apply(B.data(), p, X.data(), p, st);
        else factor_solve_raw(f, B.data(), p, X.data(), p, p, false, st);
        for (int q = 0; q < p; ++q) copy_cols(n, X.data(), p, q, cm.data() + (size_t)(c0 + q) * n, 1, 0, 1, st);
    }
    MBL_CUDA(cudaStreamSynchronize(st));
    unsigned long long tmo = 0;
    MBL_CUDA(cudaMemcpy(&tmo, f.counters.data() + 2, sizeof(tmo), cudaMemcpyDeviceToHost));
    if (tmo != 0) {
        reset_solve_counters(f, st);
        fail(MBL_ERR_TIMEOUT, "a triangular-solve dependency wait timed out");
    }
    MBL_CUDA(cudaMemcpy(x, cm.data(), (size_t)n * nrhs * sizeof(double), cudaMemcpyDeviceToHost));
    API_CATCH(ctx)
}

int mbl_factor_solve_dev(mbl_factorization *fh, const double *d_b, double *d_x, int nrhs, int refine, void *stream) {
    if (!fh || !d_b || !d_x || nrhs < 1) return report(nullptr, MBL_ERR_INVALID, "bad argument");
    Factorization &f = *fh->f;
    Ctx *ctx = f.ctx;
    API_TRY
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    const int64_t n = f.plan->n;
    if (!refine) {
        for (int c0 = 0; c0 < nrhs; c0 += 32)
            factor_solve_colmajor(f, d_b + (size_t)c0 * n, d_x + (size_t)c0 * n, std::min(32, nrhs - c0), st);
    } else {
        double emin, emax;
        extremal_bounds(f.sec, &emin, &emax);
        const double hn = std::max(std::fabs(emin), std::fabs(emax));
        RefinedSolve rs{f.sec, &f, hn + std::fabs(f.sigma), 1e-15, 20};
        rs.gmres = 1;
        if (f.dev_b.size() < (size_t)n * 32) {
            f.dev_b.alloc(ctx, (size_t)n * 32);
            f.dev_x.alloc(ctx, (size_t)n * 32);
        }
        for (int c0 = 0; c0 < nrhs; c0 += 32) {
            const int p = std::min(32, nrhs - c0);
            for (int q = 0; q < p; ++q) copy_cols(n, d_b + (size_t)(c0 + q) * n, 1, 0, f.dev_b.data(), p, q, 1, st);
            rs.apply(f.dev_b.data(), p, f.dev_x.data(), p, st);
            for (int q = 0; q < p; ++q) copy_cols(n, f.dev_x.data(), p, q, d_x + (size_t)(c0 + q) * n, 1, 0, 1, st);
        }
    }
    MBL_CUDA(cudaStreamSynchronize(st));
    unsigned long long tmo = 0;
    MBL_CUDA(cudaMemcpy(&tmo, f.counters.data() + 2, sizeof(tmo), cudaMemcpyDeviceToHost));
    if (tmo != 0) {
        reset_solve_counters(f, st);
        fail(MBL_ERR_TIMEOUT, "a triangular-solve dependency wait timed out");
    }
    API_CATCH(ctx)
}

int mbl_factor_solve_batch_dev(mbl_factorization *const *fs, int K, const double *const *d_b, double *const *d_x,
                               int nrhs, void *stream) {
    if (!fs || !d_b || !d_x || K < 1 || K > 64 || nrhs < 1) return report(nullptr, MBL_ERR_INVALID, "bad argument");
    for (int k = 0; k < K; ++k)
        if (!fs[k] || !fs[k]->f || !d_b[k] || !d_x[k]) return report(nullptr, MBL_ERR_INVALID, "NULL entry");
    Factorization &f0 = *fs[0]->f;
    Ctx *ctx = f0.ctx;
    API_TRY
    for (int k = 0; k < K; ++k) {
        const Factorization &f = *fs[k]->f;
        if (f.plan.get() != f0.plan.get() || f.prec != f0.prec)
            fail(MBL_ERR_INVALID, "batched solve: every factorization needs the same sector shape and precision");
        if (f.dataflow) fail(MBL_ERR_INVALID, "batched solve: dataflow factorizations are not batched");
        for (int j = 0; j < k; ++j)
            if (fs[j]->f.get() == &f) fail(MBL_ERR_INVALID, "batched solve: a factorization appears twice");
    }
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    const int64_t n = f0.plan->n;
    const size_t es = f0.prec == MBL_PREC_FP64 ? sizeof(SolveBufs<double>) : sizeof(SolveBufs<float>);
    std::vector<char> htab(es * K);
    std::vector<SolveIO> hio(K);
    DevMem dtab, dio;
    dtab.alloc(ctx, es * K);
    dio.alloc(ctx, sizeof(SolveIO) * K);
    for (int c0 = 0; c0 < nrhs; c0 += 32) {
        const int p = std::min(32, nrhs - c0);
        for (int k = 0; k < K; ++k) {
            Factorization &f = *fs[k]->f;
            f.ensure_solve_work(p);
            if (f.prec == MBL_PREC_FP64) reinterpret_cast<SolveBufs<double> *>(htab.data())[k] = solve_bufs<double>(f);
            else reinterpret_cast<SolveBufs<float> *>(htab.data())[k] = solve_bufs<float>(f);
            hio[k] = SolveIO{d_b[k] + (size_t)c0 * n, d_x[k] + (size_t)c0 * n, 1, 1, n, n, 0, 0};
        }
        // pageable sources: the copies complete before the calls return, so the tables can change
        MBL_CUDA(cudaMemcpyAsync(dtab.p, htab.data(), es * K, cudaMemcpyHostToDevice, st));
        MBL_CUDA(cudaMemcpyAsync(dio.p, hio.data(), sizeof(SolveIO) * K, cudaMemcpyHostToDevice, st));
        enqueue_batched_solve(*f0.plan, f0.prec, dtab.p, static_cast<const SolveIO *>(dio.p), (unsigned)K, p, st);
        MBL_CUDA(cudaStreamSynchronize(st));
    }
    API_CATCH(ctx)
}

void mbl_factor_destroy(mbl_factorization *f) {
    if (!f) return;
    if (f->f && ctx_alive(f->f->ctx)) cudaStreamSynchronize(f->f->ctx->stream);
    delete f;
}

int mbl_solve_near_dev(mbl_sector *sec, double eps, int nev, const mbl_opts *opts, double *d_evals, double *d_evecs,
                       double *d_resid, int *nconv, double *sigma_used, mbl_solve_stats *stats, void *stream) {
    if (!sec || !d_evals || !d_evecs || !d_resid || !nconv || !sigma_used)
        return report(nullptr, MBL_ERR_INVALID, "NULL argument");
    mbl_opts o;
    mbl_opts_default(&o);
    if (opts) o = *opts;
    API_TRY
    MBL_CUDA(cudaSetDevice(sec->ctx->device));
    cudaStream_t st = sec->ctx->stream;
    if (stream) {
        // order after the caller's stream, run on the context stream, then make the caller wait
        cudaEvent_t ev;
        MBL_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        MBL_CUDA(cudaEventRecord(ev, (cudaStream_t)stream));
        MBL_CUDA(cudaStreamWaitEvent(st, ev, 0));
        cudaEventDestroy(ev);
    }
    solve_near(sec, eps, nev, o, d_evals, d_evecs, d_resid, nconv, sigma_used, stats, st);
    if (*nconv < nev) fail(MBL_ERR_NOT_CONVERGED, "only " + std::to_string(*nconv) + " of " + std::to_string(nev) +
                                                      " eigenpairs reached the tolerance");
    API_CATCH(sec->ctx)
}

int mbl_solve_near(mbl_sector *sec, double eps, int nev, const mbl_opts *opts, double *evals, double *evecs,
                   double *resid, int *nconv, double *sigma_used, mbl_solve_stats *stats) {
    if (!sec || !evals || !evecs || !resid || !nconv || !sigma_used)
        return report(nullptr, MBL_ERR_INVALID, "NULL argument");
    if (nev < 1 || nev > sec->n) return report(sec->ctx, MBL_ERR_INVALID, "nev must be in [1, dim]");
    int rc = MBL_OK;
    API_TRY
    Ctx *ctx = sec->ctx;
    int64_t n = sec->n;
    DVec<double> de, dv, dr;
    de.alloc(ctx, nev);
    dv.alloc(ctx, (size_t)n * nev);
    dr.alloc(ctx, nev);
    rc = mbl_solve_near_dev(sec, eps, nev, opts, de.data(), dv.data(), dr.data(), nconv, sigma_used, stats, nullptr);
    if (rc != MBL_OK && rc != MBL_ERR_NOT_CONVERGED) return rc;
    std::string keep = ctx->last_error;
    MBL_CUDA(cudaMemcpy(evals, de.data(), nev * sizeof(double), cudaMemcpyDeviceToHost));
    MBL_CUDA(cudaMemcpy(evecs, dv.data(), (size_t)n * nev * sizeof(double), cudaMemcpyDeviceToHost));
    MBL_CUDA(cudaMemcpy(resid, dr.data(), nev * sizeof(double), cudaMemcpyDeviceToHost));
    if (rc != MBL_OK) return report(ctx, rc, keep);
    API_CATCH(sec->ctx)
}

// Observables of nev eigenvectors of the sector (L, nup); the entry points without nup take the
// S^z_tot = 0 sector of even L.
static int obs_dev(mbl_ctx *ctx, int L, int nup, int nev, const double *d_evals, const double *d_evecs, double *d_r,
                   double *d_r_mean, double *d_s1p, double *d_se, void *stream) {
    if (!ctx || !d_evals || !d_evecs || !d_s1p || !d_se || (nev > 2 && !d_r))
        return report(ctx, MBL_ERR_INVALID, "NULL argument");
    if (L < 2 || L > 22 || nup < 0 || nup > L) return report(ctx, MBL_ERR_INVALID, "need 2 <= L <= 22, 0 <= nup <= L");
    API_TRY
    MBL_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    observables_dev(ctx, L, nup, nev, d_evals, d_evecs, d_r, d_r_mean, d_s1p, d_se, st);
    API_CATCH(ctx)
}

static int obs_host(mbl_ctx *ctx, int L, int nup, int nev, const double *evals, const double *evecs, double *r,
                    double *r_mean, double *s1p, double *se) {
    if (!ctx || !evals || !evecs || !s1p || !se || (nev > 2 && !r)) return report(ctx, MBL_ERR_INVALID, "NULL argument");
    if (L < 2 || L > 22 || nup < 0 || nup > L) return report(ctx, MBL_ERR_INVALID, "need 2 <= L <= 22, 0 <= nup <= L");
    API_TRY
    const int64_t n = host_binom(L, nup);
    if (nev < 1 || nev > n) fail(MBL_ERR_INVALID, "nev must be in [1, dim]");
    DVec<double> de, dv, dr, drm, ds, dse;
    de.alloc(ctx, nev);
    dv.alloc(ctx, (size_t)n * nev);
    dr.alloc(ctx, std::max(nev - 2, 1));
    drm.alloc(ctx, 1);
    ds.alloc(ctx, nev);
    dse.alloc(ctx, nev);
    MBL_CUDA(cudaMemcpy(de.data(), evals, nev * sizeof(double), cudaMemcpyHostToDevice));
    MBL_CUDA(cudaMemcpy(dv.data(), evecs, (size_t)n * nev * sizeof(double), cudaMemcpyHostToDevice));
    observables_dev(ctx, L, nup, nev, de.data(), dv.data(), dr.data(), drm.data(), ds.data(), dse.data(), ctx->stream);
    if (nev > 2 && r) MBL_CUDA(cudaMemcpy(r, dr.data(), (nev - 2) * sizeof(double), cudaMemcpyDeviceToHost));
    if (r_mean) MBL_CUDA(cudaMemcpy(r_mean, drm.data(), sizeof(double), cudaMemcpyDeviceToHost));
    MBL_CUDA(cudaMemcpy(s1p, ds.data(), nev * sizeof(double), cudaMemcpyDeviceToHost));
    MBL_CUDA(cudaMemcpy(se, dse.data(), nev * sizeof(double), cudaMemcpyDeviceToHost));
    API_CATCH(ctx)
}

static int obs_extra_dev(mbl_ctx *ctx, int L, int nup, int nev, const double *d_evecs, double q, double *d_kl,
                         double *d_sqp, double *d_fluct, double *d_dynf, void *stream) {
    if (!ctx || !d_evecs || !d_sqp || !d_fluct || !d_dynf || (nev > 1 && !d_kl))
        return report(ctx, MBL_ERR_INVALID, "NULL argument");
    if (L < 2 || L > 22 || nup < 0 || nup > L) return report(ctx, MBL_ERR_INVALID, "need 2 <= L <= 22, 0 <= nup <= L");
    API_TRY
    MBL_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    observables_extra_dev(ctx, L, nup, nev, d_evecs, q, d_kl, d_sqp, d_fluct, d_dynf, st);
    API_CATCH(ctx)
}

static int obs_extra_host(mbl_ctx *ctx, int L, int nup, int nev, const double *evecs, double q, double *kl, double *sqp,
                          double *fluct, double *dynf) {
    if (!ctx || !evecs || !sqp || !fluct || !dynf || (nev > 1 && !kl))
        return report(ctx, MBL_ERR_INVALID, "NULL argument");
    if (L < 2 || L > 22 || nup < 0 || nup > L) return report(ctx, MBL_ERR_INVALID, "need 2 <= L <= 22, 0 <= nup <= L");
    API_TRY
    const int64_t n = host_binom(L, nup);
    if (nev < 1 || nev > n) fail(MBL_ERR_INVALID, "nev must be in [1, dim]");
    DVec<double> dv, dk, dq, df, dd;
    dv.alloc(ctx, (size_t)n * nev);
    dk.alloc(ctx, std::max(nev - 1, 1));
    dq.alloc(ctx, nev);
    df.alloc(ctx, nev);
    dd.alloc(ctx, nev);
    MBL_CUDA(cudaMemcpy(dv.data(), evecs, (size_t)n * nev * sizeof(double), cudaMemcpyHostToDevice));
    observables_extra_dev(ctx, L, nup, nev, dv.data(), q, dk.data(), dq.data(), df.data(), dd.data(), ctx->stream);
    MBL_CUDA(cudaStreamSynchronize(ctx->stream));
    if (nev > 1) MBL_CUDA(cudaMemcpy(kl, dk.data(), (nev - 1) * sizeof(double), cudaMemcpyDeviceToHost));
    MBL_CUDA(cudaMemcpy(sqp, dq.data(), nev * sizeof(double), cudaMemcpyDeviceToHost));
    MBL_CUDA(cudaMemcpy(fluct, df.data(), nev * sizeof(double), cudaMemcpyDeviceToHost));
    MBL_CUDA(cudaMemcpy(dynf, dd.data(), nev * sizeof(double), cudaMemcpyDeviceToHost));
    API_CATCH(ctx)
}

#define MBL_EVEN_L(ctx, L) \
    if ((L) & 1) return report(ctx, MBL_ERR_INVALID, "L must be even (the _nup entry points take other sectors)")

int mbl_observables_dev(mbl_ctx *ctx, int L, int nev, const double *d_evals, const double *d_evecs, double *d_r,
                        double *d_r_mean, double *d_s1p, double *d_se, void *stream) {
    MBL_EVEN_L(ctx, L);
    return obs_dev(ctx, L, L / 2, nev, d_evals, d_evecs, d_r, d_r_mean, d_s1p, d_se, stream);
}

int mbl_observables_nup_dev(mbl_ctx *ctx, int L, int nup, int nev, const double *d_evals, const double *d_evecs,
                            double *d_r, double *d_r_mean, double *d_s1p, double *d_se, void *stream) {
    return obs_dev(ctx, L, nup, nev, d_evals, d_evecs, d_r, d_r_mean, d_s1p, d_se, stream);
}

int mbl_observables(mbl_ctx *ctx, int L, int nev, const double *evals, const double *evecs, double *r, double *r_mean,
                    double *s1p, double *se) {
    MBL_EVEN_L(ctx, L);
    return obs_host(ctx, L, L / 2, nev, evals, evecs, r, r_mean, s1p, se);
}

int mbl_observables_nup(mbl_ctx *ctx, int L, int nup, int nev, const double *evals, const double *evecs, double *r,
                        double *r_mean, double *s1p, double *se) {
    return obs_host(ctx, L, nup, nev, evals, evecs, r, r_mean, s1p, se);
}

int mbl_observables_extra_dev(mbl_ctx *ctx, int L, int nev, const double *d_evecs, double q, double *d_kl,
                              double *d_sqp, double *d_fluct, double *d_dynf, void *stream) {
    MBL_EVEN_L(ctx, L);
    return obs_extra_dev(ctx, L, L / 2, nev, d_evecs, q, d_kl, d_sqp, d_fluct, d_dynf, stream);
}

int mbl_observables_extra_nup_dev(mbl_ctx *ctx, int L, int nup, int nev, const double *d_evecs, double q,
                                  double *d_kl, double *d_sqp, double *d_fluct, double *d_dynf, void *stream) {
    return obs_extra_dev(ctx, L, nup, nev, d_evecs, q, d_kl, d_sqp, d_fluct, d_dynf, stream);
}

int mbl_observables_extra(mbl_ctx *ctx, int L, int nev, const double *evecs, double q, double *kl, double *sqp,
                          double *fluct, double *dynf) {
    MBL_EVEN_L(ctx, L);
    return obs_extra_host(ctx, L, L / 2, nev, evecs, q, kl, sqp, fluct, dynf);
}

int mbl_observables_extra_nup(mbl_ctx *ctx, int L, int nup, int nev, const double *evecs, double q, double *kl,
                              double *sqp, double *fluct, double *dynf) {
    return obs_extra_host(ctx, L, nup, nev, evecs, q, kl, sqp, fluct, dynf);
}

}  // extern "C"

int mbl_entanglement_noalloc_dev(mbl_ctx *ctx, int L, int nev, const double *d_evecs, double *d_se, void *stream) {
    if (!ctx || !d_evecs || !d_se) return report(ctx, MBL_ERR_INVALID, "NULL argument");
    API_TRY
    MBL_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    entanglement_noalloc(ctx, L, nev, d_evecs, d_se, st);
    API_CATCH(ctx)
}
