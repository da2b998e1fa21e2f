// factor.h -- numeric factorization object and the raw triangular solve.
#pragma once

#include "plan.h"

namespace mbl {

// Buffers of one factorization's level-sequence triangular solve as the solve kernels read them.
// A launch takes a table of these, one per job (blockIdx.z), so that several factorizations of
// one plan (same pattern, same launch sequence) are solved by one launch sequence.
template <class T>
struct SolveBufs {
    const T *G;          // packed solve factor
    const T *D;          // pivots
    T *Z, *Zs;           // front work rows: gathered, solved
    T *y, *yfw;          // permuted right-hand side / solution; forward result
    T *P;                // backward partial sums
    unsigned int *cnt;   // backward arrival counters (per solve descriptor and column chunk)
};

struct LeanArena;  // physical backing of the memory-lean fronts arena (factor.cu)

// Fronts arena modes: the whole arena allocated at once, or the memory-lean arena (regions backed
// only while their fronts are live).  Automatic: lean when the whole arena would exceed 8 GiB.
constexpr int ARENA_AUTO = 0, ARENA_LEAN = 1, ARENA_FULL = 2;
bool arena_is_lean(const Plan &p, int prec, int mode);
void trim_device_pool(int device);  // release the stream-ordered pool's cached free blocks (capi.cu)
// Device bytes of the fronts arena at its peak in that mode.
double arena_peak_bytes(const Plan &p, int prec, int mode);

struct Factorization {
    Ctx *ctx = nullptr;
    mbl_sector *sec = nullptr;
    std::shared_ptr<Plan> plan;
    double sigma = 0.0;
    int prec = MBL_PREC_FP32;
    double tiny = 0.0;
    DVec<char> arena, D, wscr, cmax, M, zwork, zsolved, ywork, yfw, pwork;
    DVec<char> gpk;           // packed solve factor: every solve panel's G = [M; L21 M] (Plan::sg_elems)
    DVec<int32_t> piv;
    DVec<unsigned int> scnt;  // per (solve panel, column chunk) arrival counters of the backward step
    DVec<int32_t> dfcnt;      // dataflow solve: per-front completion counters (4 ns) and two tickets
    bool dataflow = false;    // solves as one persistent kernel per sweep (else level-by-level launches)
    std::unique_ptr<LeanArena> lean;  // set: the fronts live in the memory-lean arena, not `arena`
    bool lean_used = false;           // the factorization ran in the memory-lean arena
    uint64_t wait_ns = 1000000000ull;  // limit of each bounded dependency wait of the dataflow solve
    // [0] perturbed pivots, [1] negative pivots, [2] wait time-outs, [3] max |l| (float bits, low
    // word), [4] min |d| (float bits, low word)
    DVec<unsigned long long> counters;
    float max_l = 0.f, min_d = 0.f;
    int work_p = 0;
    cudaGraphExec_t graph_exec = nullptr;  // captured solve sequence for block width graph_p
    int graph_p = 0;
    long long graph_nodes = 0;
    int tc_mode = 1;  // FP32 fronts' Schur updates: 0 CUDA cores, 1 tcgen05 3xTF32, 2 tcgen05 3xBF16
    DVec<char> pieces;                    // tensor-core operand pieces of the step's L21 and W21
    int64_t prow = 0;                     // rows of each piece array
    alignas(64) unsigned char tmap[128];  // tensor map over the pieces (TMA-fed Schur update)
    bool tma = false;                     // the pieces and their tensor map are ready
    // launch trace of the level-by-level solve (opt-in; recaptures the solve graph when switched)
    bool trace_on = false;
    DVec<LaunchTrace> trace;
    DVec<double> dev_b, dev_x;  // row-major right-hand-side blocks of refined device solves (n x 32)
    DVec<char> dbufs;           // device SolveBufs<T> of this factorization (one entry)
    std::vector<int> trace_kind;  // per traced launch: 0 forward gather, 1 forward step, 2/3 backward start/update
    int64_t perturbed = 0, negative = 0;
    double ms_factor = 0.0;

    size_t elem_size() const { return prec == MBL_PREC_FP64 ? sizeof(double) : sizeof(float); }
    Factorization();  // out of line: LeanArena is complete only in factor.cu
    size_t held_bytes() const;  // device bytes it holds now (all its buffers)
    ~Factorization();
    void allocate(bool lean_arena = false);
    void release_scratch();
    void ensure_solve_work(int p);
};

// Right-hand side and result of one job of a batched solve (row-major FP64 blocks, row strides).
struct SolveIO {
    const double *B;
    double *X;
    int64_t ldb, ldx;    // row strides
    int64_t ldbq, ldxq;  // right-hand-side (column) strides
    int accumulate;      // X += solution instead of X = solution
    int pad;
};

// Enqueue the solve of K jobs of one plan and precision: tab holds K SolveBufs<T> (T by prec), io
// K SolveIO, both on the device; p right-hand sides per job.  Capturable in a CUDA graph.
void enqueue_batched_solve(const Plan &pl, int prec, const void *tab, const SolveIO *io, unsigned K, int p,
                           cudaStream_t st);

struct SolveBatcher;
// A serving worker's solve through the context's batcher (batch.cu): enqueued on st after the
// work already there; returns once the batch holding it is launched.
void batched_solve(SolveBatcher *b, Factorization &fz, const double *B, int64_t ldb, double *X, int64_t ldx, int p,
                   bool accumulate, cudaStream_t st);
// Workers inside a solve phase of (plan, precision, p): the batcher waits for all of them before
// it launches, up to its window.
void batcher_enter(SolveBatcher *b, const Plan *pl, int prec, int p);
void batcher_leave(SolveBatcher *b, const Plan *pl, int prec, int p);
// A batcher with its own thread, `lanes` streams and context on `device`; batches of at most
// max_jobs.
SolveBatcher *batcher_create(int device, int max_jobs, double window_us, int lanes);
void batcher_destroy(SolveBatcher *b);  // after every worker using it has stopped
// Launched batches, solves in them, their device time (CUDA events) and algorithmic bytes.
void batcher_stats(SolveBatcher *b, int64_t *batches, int64_t *solves, double *ms, double *bytes, double *busy_ms);

// The SolveBufs of a factorization (its solve work allocated).
template <class T>
SolveBufs<T> solve_bufs(const Factorization &fz);

// tcgen05 trailing update of one panel step (FP32 fronts); err counts bounded-wait time-outs.  The
// TMA-fed form reads the operand pieces the panel's trsm wrote (tensor map from encode_pieces_map over
// 4 x prow x NB pieces); the other form splits the raw operands itself.
size_t schur_tc_smem(bool bf16);
bool encode_pieces_map(void *map, void *pieces, int64_t prow, bool bf16);
void launch_schur_tma(const PanelStep &stp, const PanelDesc *d_descs, const int64_t *fo, const int32_t *fsz,
                      float *arena, const void *map, unsigned long long *err, cudaStream_t st, bool bf16);
// Autotuning of the FP32 fronts' trailing update (once per plan and tensor-core mode): for every size
// class of trailing block that the plan's panel steps have, time one update of a synthetic front of
// that class with tcgen05 128 x 128 tiles (TMA-fed) and with CUDA-core 64 x 64 tiles, and keep the
// faster in the plan.
void tune_schur(Factorization &fz, cudaStream_t st);
void launch_schur_tc(const PanelStep &stp, const PanelDesc *d_descs, const Plan &p, float *arena, const float *wscr,
                     unsigned long long *err, cudaStream_t st, bool bf16);

// Both sweeps of a block solve as dataflow kernels (solve_df.cu), between the permutations.
template <class T>
void solve_dataflow(Factorization &fz, int p, cudaStream_t st);

// Enqueue the numeric factorization of H - sigma I (allocate() first).
void numeric_factor(Factorization &fz, cudaStream_t st);
// X (n x p row-major FP64, row stride ldx) (+)= (L D L^T)^-1 B, B row stride ldb; 1 <= p <= 32.
void factor_solve_raw(Factorization &fz, const double *B, int64_t ldb, double *X, int64_t ldx, int p, bool accumulate,
                      cudaStream_t st);
// X = (L D L^T)^-1 B for column-major n x p FP64 blocks (leading dimension n); 1 <= p <= 32.
void factor_solve_colmajor(Factorization &fz, const double *B, double *X, int p, cudaStream_t st);

// Upper estimate of the device bytes one solve_near job holds at its peak (serving admission).
size_t job_bytes(const Plan &p, int nev, int block, int prec);
// Plan of the sector's L (built from the device CSR on first use and cached in the context).
std::shared_ptr<Plan> get_plan(mbl_sector *sec);
// Create, allocate and run a factorization (synchronous; fills stats).
std::unique_ptr<Factorization> make_factorization(mbl_sector *sec, double sigma, int prec, double hnorm,
                                                  int tc_mode = 1, bool dataflow = false,
                                                  uint64_t wait_ns = 1000000000ull, int arena_mode = ARENA_AUTO,
                                                  double pivot_tiny = 0.0);
// Wait-limit option (seconds, 0 = the 1 s default) in nanoseconds.
uint64_t wait_limit_ns(double seconds);
// After a solve reported expired waits: clear the time-out count and the per-chunk arrival counters
// that the stopped CTAs may have left behind, so that the factorization serves later solves.
void reset_solve_counters(Factorization &fz, cudaStream_t st);

}  // namespace mbl

struct mbl_factorization {
    std::unique_ptr<mbl::Factorization> f;
};
