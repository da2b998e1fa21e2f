// factor.h -- numeric factorization object and the raw triangular solve.
#pragma once

#include "plan.h"

namespace mbl {

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
    // [0] perturbed pivots, [1] negative pivots, [2] wait time-outs, [3] max |l| (float bits, low
    // word), [4] min |d| (float bits, low word)
    DVec<unsigned long long> counters;
    float max_l = 0.f, min_d = 0.f;
    int work_p = 0;
    cudaGraphExec_t graph_exec = nullptr;  // captured solve sequence for block width graph_p
    int graph_p = 0;
    long long graph_nodes = 0;
    int tc_mode = 1;  // FP32 fronts' Schur updates: 0 CUDA cores, 1 tcgen05 3xTF32, 2 tcgen05 3xBF16
    // launch trace of the level-by-level solve (opt-in; recaptures the solve graph when switched)
    bool trace_on = false;
    DVec<LaunchTrace> trace;
    DVec<double> dev_b, dev_x;  // row-major right-hand-side blocks of refined device solves (n x 32)
    std::vector<int> trace_kind;  // per traced launch: 0 forward gather, 1 forward step, 2/3 backward start/update
    int64_t perturbed = 0, negative = 0;
    double ms_factor = 0.0;

    size_t elem_size() const { return prec == MBL_PREC_FP64 ? sizeof(double) : sizeof(float); }
    ~Factorization();
    void allocate();
    void release_scratch();
    void ensure_solve_work(int p);
};

// tcgen05 trailing update of one panel step (FP32 fronts); err counts bounded-wait time-outs.
size_t schur_tc_smem(bool bf16);
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
                                                  int tc_mode = 1, bool dataflow = false);

}  // namespace mbl

struct mbl_factorization {
    std::unique_ptr<mbl::Factorization> f;
};
