// mbl_internal.h -- shared declarations of the mblsi library (host C++ and CUDA).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "mblsi.h"

namespace mbl {

struct Error {
    int code;
    std::string msg;
};

[[noreturn]] inline void fail(int code, const std::string &m) { throw Error{code, m}; }

#define MBL_CUDA(x)                                                                            \
    do {                                                                                       \
        cudaError_t e_ = (x);                                                                  \
        if (e_ != cudaSuccess)                                                                 \
            ::mbl::fail(MBL_ERR_CUDA, std::string(#x) + " -> " + cudaGetErrorString(e_) +      \
                                          " at " + __FILE__ + ":" + std::to_string(__LINE__)); \
    } while (0)

// Every kernel launch of the library is followed by exactly one MBL_LAUNCH_CHECK(), which also
// counts it (mbl_launch_count).
extern std::atomic<long long> g_launches;
extern thread_local long long t_launches;  // this thread's share (graph capture counts its own launches)
#define MBL_LAUNCH_CHECK()                                           \
    do {                                                             \
        ::mbl::g_launches.fetch_add(1, std::memory_order_relaxed);   \
        ++::mbl::t_launches;                                         \
        MBL_CUDA(cudaGetLastError());                                \
    } while (0)

// Programmatic dependent launch (sm_90+): a kernel launched with launch_pdl may start while its
// predecessor in the stream is still running.  It must execute pdl_wait() -- which returns once
// the predecessor grid has completed and its writes are visible -- before it touches anything the
// predecessor writes or reads, and on every path before it exits (so that completion stays
// transitive along the stream).  pdl_trigger() lets the successor launch early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Opt-in launch trace of the triangular solves: per launch, the %globaltimer (ns) when its first
// CTA started and when its last CTA finished (thread 0 of each CTA; atomics on two words).
struct LaunchTrace {
    unsigned long long t0, t1;
};
#ifdef __CUDACC__
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
struct TraceScope {
    LaunchTrace *tr;
    __device__ explicit TraceScope(LaunchTrace *t) : tr(t) {
        if (tr && threadIdx.x == 0) atomicMin(&tr->t0, global_ns());
    }
    __device__ ~TraceScope() {
        if (tr && threadIdx.x == 0) atomicMax(&tr->t1, global_ns());
    }
};
#endif

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MBL_CUDA(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
    MBL_LAUNCH_CHECK();
}

struct Ctx;
bool ctx_alive(const Ctx *c);

// Raise kernel fn's dynamic shared-memory limit to `bytes` on the current device, once per
// (kernel, device): function attributes are per device.
void smem_limit(const void *fn, size_t bytes);

// Device allocation accounted against the context budget (admission control).
struct DevMem {
    void *p = nullptr;
    size_t bytes = 0;
    Ctx *ctx = nullptr;
    DevMem() = default;
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    DevMem(DevMem &&o) noexcept { *this = std::move(o); }
    DevMem &operator=(DevMem &&o) noexcept;
    ~DevMem() { release(); }
    void alloc(Ctx *c, size_t nbytes);
    void release();
};

template <class T>
struct DVec {
    DevMem m;
    size_t n = 0;
    T *data() const { return static_cast<T *>(m.p); }
    void alloc(Ctx *c, size_t count) {
        m.alloc(c, count * sizeof(T));
        n = count;
    }
    void release() {
        m.release();
        n = 0;
    }
    size_t size() const { return n; }
};

// Opt-in per-class device timing with CUDA events on the launching stream.
struct ProfAcc {
    struct Pending {
        cudaEvent_t e0, e1;
        double work;
    };
    std::vector<Pending> pending;
    int64_t launches = 0;
    double ms = 0.0, work = 0.0;
};

struct Plan;       // symbolic analysis, symbolic.cpp
struct EntTables;  // entanglement block tables, observables.cu

// Symbolic analyses by L.  Shared by a context and its serving workers; `mu` serializes lookups
// and the (one-off) builds.
// C(n, k) on the host (0 outside 0 <= k <= n)
inline int64_t host_binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// Cache key of a sector (chain length L <= 32, nup up spins)
inline int sector_key(int L, int nup) { return L * 64 + nup; }

struct PlanCache {
    std::mutex mu;
    std::map<int, std::shared_ptr<Plan>> m;  // key: plan_key(L, nup, ordering)
    int ordering = MBL_ORDER_AUTO;           // for plans built from now on
};
inline int plan_key(int L, int nup, int ordering) { return sector_key(L, nup) * 8 + ordering; }
// The ordering MBL_ORDER_AUTO stands for, for a sector of dimension n.
inline int resolve_ordering(int ordering, int64_t n) {
    if (ordering != MBL_ORDER_AUTO) return ordering;
    return n >= 40000 ? MBL_ORDER_MODES : MBL_ORDER_BAND;
}

struct Ctx {
    int device = 0;
    size_t budget = 0;  // 0 = unlimited
    size_t in_use = 0;
    size_t peak = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    std::shared_ptr<PlanCache> plans = std::make_shared<PlanCache>();  // per L; shared with serving workers
    std::map<int, std::shared_ptr<EntTables>> ent;  // per sector (sector_key)
    int sm_count = 0;
    bool prof = false;
    std::map<std::string, ProfAcc> profile;
    std::vector<cudaEvent_t> event_pool;
    struct Server *server = nullptr;  // serving workers (server.cu), if started
    struct SolveBatcher *batcher = nullptr;  // a serving worker's solve batcher (batch.cu), shared
    int batch_max_jobs = 16;                 // server option: jobs per batched solve (1 = no batching)
    double batch_window_us = 300.0;          // server option: longest wait for the other workers
    int batch_lanes = 2;                     // server option: streams of batched solves
    double cache_fraction = 0.25;            // server option: budget share of the live-factor cache
    cudaEvent_t take_event();
    void resolve_profile();
};
void server_shutdown(Ctx *ctx);

// Times the enclosed launches on `st` under class `name` when profiling is on.
struct ProfScope {
    Ctx *c;
    const char *name;
    double work;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr;
    ProfScope(Ctx *c_, const char *name_, double work_, cudaStream_t st_);
    ~ProfScope();
};

}  // namespace mbl

struct mbl_ctx : public mbl::Ctx {};

struct mbl_sector {
    mbl::Ctx *ctx = nullptr;
    int L = 0;
    int nup = 0;  // up spins of every basis state (S^z_tot = nup - L/2)
    int64_t n = 0, nnz = 0;
    double J = 1.0;
    double hfield[32] = {0};
    mbl::DVec<uint32_t> states;
    mbl::DVec<int64_t> rowptr;
    mbl::DVec<int32_t> col;
    mbl::DVec<double> val;
    mbl::DVec<double> d_hfield;
    bool have_bounds = false;
    double emin = 0, emax = 0;
    std::shared_ptr<mbl::Plan> plan;  // lazily attached
};

namespace mbl {

// ---------------- sector.cu ----------------
void upload_binomials();
void launch_fields(int L, double h, uint64_t seed, double *d_out, cudaStream_t st);
void build_sector_device(mbl_sector *sec, cudaStream_t st);
// rank of each state among the L-bit words with nup set bits (-1 if it is not one of them)
void launch_rank(int L, int nup, const uint32_t *d_states, int64_t count, int64_t *d_ranks, cudaStream_t st);
// y[i*ys_r + q*ys_c] = sum_j A_ij x[j*xs_r + q*xs_c] - shift x[i*xs_r + q*xs_c]   (FP64)
void launch_spmv(const mbl_sector *sec, double shift, const double *x, int64_t xs_r, int64_t xs_c,
                 double *y, int64_t ys_r, int64_t ys_c, int p, cudaStream_t st);

// ---------------- dense.cu (FP64 block kernels, small symmetric eigensolver) ----------------
// C[k x p] (row-major, ldc = p) = V[:, c0:c0+k]^T X[:, x0:x0+p], V n x ldv and X n x ldx row-major.
// Uses `work` (>= dense_tn_work doubles) for deterministic partial sums; k * p <= 10240.
size_t dense_tn_work(int64_t n, int k, int p);
void dense_tn(int64_t n, const double *V, int ldv, int c0, int k, const double *X, int ldx, int x0, int p,
              double *C, double *work, cudaStream_t st);
// X -= V[:, c0:c0+k] C  (C k x p row-major)
void dense_nn_sub(int64_t n, const double *V, int ldv, int c0, int k, const double *C, int p, double *X,
                  cudaStream_t st);
// FP32-stored V (the products summed in FP32): dense_tn and dense_nn_sub for preconditioner work.
void dense_tn32(int64_t n, const float *V, int ldv, int c0, int k, const double *X, int ldx, int x0, int p,
                double *C, double *work, cudaStream_t st);
void dense_nn_sub32(int64_t n, const float *V, int ldv, int c0, int k, const double *C, int p, const double *Xin,
                    double *Xout, cudaStream_t st);  // Xout = Xin - V C
// Y[:, 0:m] = V[:, 0:k] S  (S k x m row-major, Y n x ldy row-major starting at column y0)
void dense_nn(int64_t n, const double *V, int ldv, int k, const double *S, int m, double *Y, int ldy,
              int y0, cudaStream_t st);
// Copy columns: dst[:, d0:d0+m] = src[:, s0:s0+m] (row-major, given leading dims)
void copy_cols(int64_t n, const double *src, int lds, int s0, double *dst, int ldd, int d0, int m,
               cudaStream_t st);
// Cholesky-QR of X (n x p row-major) in place; R (p x p row-major, upper) returned on device.
// rank_ok[0] on device set to 0 if the Gram matrix is not numerically positive definite.
void chol_qr(int64_t n, double *X, int p, double *R, double *G, double *work, int *d_flag,
             cudaStream_t st);
// Batched symmetric eigensolver on device: for b in [0, batch): A_b (m_b x m_b, column-major,
// lda_b) -> eigenvalues ascending w_b, eigenvectors (if vecs) overwrite A_b.
// One symmetric m x m FP64 matrix (column-major, m <= 160) -> eigenvectors in place (columns
// ascending) and eigenvalues d_w, by bisection and inverse iteration; d_work >= syev_bisect_work(m).
size_t syev_bisect_work(int m);
void syev_bisect(int m, double *d_A, double *d_w, double *d_work, cudaStream_t st);
// The same method in FP32 arithmetic (FP64 input and output; vectors to FP32 accuracy), as the start
// of a refined decomposition; d_work >= syev_bisect_work(m) / 2 + 1.
void syev_bisect32(int m, double *d_A, double *d_w, double *d_work, cudaStream_t st);
size_t syev_work_doubles(int mmax, bool vecs = true);
// sel (optional, indexed like w): eigenvectors are computed only where sel != 0 (others zero).
constexpr int EIG_SMEM_MAX_M = 160;  // largest order the small eigensolver keeps in shared memory
// fp32: run the reduction and the QL iteration in FP32 (order <= 160; used where FP32 eigenvectors
// are enough, e.g. Krylov-Schur restarts, which are re-orthonormalized in FP64).
void syev_batched(int batch, const int *d_m, const int64_t *d_aoff, const int64_t *d_woff, double *d_A,
                  double *d_w, int vecs, const int *d_sel, int mmax, double *d_work, int *d_info,
                  cudaStream_t st, bool fp32 = false);
// Eigenvalues (ascending) and eigenvectors of the batch's matrices (order <= 160) by the parallel
// cyclic Jacobi method in FP32 on one CTA each, as the start of a refined decomposition; info[b] = 1
// if a matrix did not converge in the sweep limit.
void syev_jacobi32(int batch, const int *d_m, const int64_t *d_aoff, const int64_t *d_woff, double *d_A, double *d_w,
                   int mmax, int *d_info, cudaStream_t st);
// set the small eigensolver's shared-memory attributes on the current device and load its FP32 and
// FP64 kernels now (kernels otherwise load lazily on first launch, taking device memory then)
cudaError_t syev_preload();
// C = alpha op(A) op(B) + beta C for small column-major FP64 matrices
void gemm_small(bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda, const double *B,
                int ldb, double beta, double *C, int ldc, cudaStream_t st);

}  // namespace mbl
