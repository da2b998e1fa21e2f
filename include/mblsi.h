/*
 * mblsi.h -- C ABI of the GB300 (sm_103a) shift-invert exact-diagonalization library for the
 * random-field Heisenberg chain of Luitz, Laflorencie and Alet (arXiv:1411.0660).
 *
 * Model (Eq. 1, field written as +h_i, periodic chain, J = 1 unless given):
 *     H = J sum_{i=0}^{L-1} S_i . S_{(i+1) mod L} + sum_i h_i S^z_i ,   h_i uniform on [-h, h]
 * restricted to a magnetization sector (numerical-method section: S^z_tot = 0 for even L, the
 * "S^z = 1" sector for odd L).  Site i is bit i of a uint32 state, a set bit is spin up; the basis
 * of the sector with nup up spins is every state with nup set bits in ascending integer order
 * (= the combinatorial number system, rank(s) = sum_t C(p_t, t+1) over the set-bit positions
 * p_0 < p_1 < ...).  Entry points without "nup" in their name take nup = L/2 and even L; the
 * *_nup entry points take any 0 <= nup <= L and either parity of L.
 *
 * Energy target (numerical-method section, read with E_min at eps = 0):
 *     sigma = E_min + eps (E_max - E_min),   ||H|| := max(|E_min|, |E_max|)
 * The method returns the nev eigenpairs nearest sigma through the shift-invert transformation
 * (H - sigma)^-1 (numerical-method section).  Ties in |lambda - sigma| take the lower lambda.
 *
 * Conventions for every entry point
 *   - Return value: MBL_OK or one of the MBL_ERR_* codes; mbl_last_error() gives detail.
 *   - Handles (mbl_ctx, mbl_sector, mbl_factorization) are opaque, owned by the library and released
 *     with the matching *_destroy.  A context is used by one host thread at a time; separate
 *     contexts may run on separate threads.
 *   - Host arrays are caller owned and must hold the stated number of elements.  Entry points
 *     whose name ends in _dev take device pointers (caller owned, on the context's device)
 *     and a cudaStream_t passed as void* (NULL = the context's own stream); they return once
 *     the work is enqueued unless stated otherwise.
 *   - Vectors of the sector are indexed by basis rank.  Blocks of eigenvectors are n x nev
 *     column-major (column j is eigenvector j, unit 2-norm, arbitrary sign).
 */
#ifndef MBLSI_H
#define MBLSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MBL_OK 0
#define MBL_ERR_INVALID 1       /* bad argument: L < 2, L > 22, odd L without nup, nev outside [1, n] ... */
#define MBL_ERR_OOM 2           /* the HBM budget of the context cannot hold the request */
#define MBL_ERR_SINGULAR 3      /* factorization broke down even with FP64 fronts */
#define MBL_ERR_NOT_CONVERGED 4 /* eigenpairs below tolerance not reached; partial results out */
#define MBL_ERR_TIMEOUT 5       /* a bounded device wait expired */
#define MBL_ERR_CUDA 6          /* a CUDA runtime error (text in mbl_last_error) */
#define MBL_PENDING 7           /* serving: the request is not finished yet */

/* Arithmetic of the frontal matrices (dense LDL^T of the multifrontal factorization). */
#define MBL_PREC_FP64 0   /* FP64 fronts and FP64 triangular solves */
#define MBL_PREC_FP32 1   /* FP32 fronts and solves, FP64 iterative refinement */

/* Fill-reducing orderings of the symbolic analysis (nested dissection along the Fourier modes of
 * the magnetization profile; see mbl_ctx_set_ordering). */
#define MBL_ORDER_BAND 0  /* separators = bands of one mode, chosen from the two numbered depth, depth + 1 */
#define MBL_ORDER_COVER 1 /* all modes k <= L/2 searched, separators refined to a minimum vertex cover:
                             the least fill and flops, but more single-column supernodes and a
                             heavier tail of element growth in the unrefined factor */
#define MBL_ORDER_MODES 2 /* all modes k <= L/2 searched, the band separator of the best one */
#define MBL_ORDER_AUTO 3  /* MBL_ORDER_MODES for sectors of dimension >= 40000 (L >= 18 at half filling),
                             where its smaller factor pays; MBL_ORDER_BAND below, where the
                             factorization is bound by the per-level launch chain */
#define MBL_ORDER_HYBRID 4 /* MBL_ORDER_COVER on subgraphs of >= 2000 vertices, MBL_ORDER_MODES on smaller
                              ones: nearly the cover's fill without its single-column leaves */

typedef struct mbl_ctx mbl_ctx;
typedef struct mbl_sector mbl_sector;
typedef struct mbl_factorization mbl_factorization;

/* Options of factor/solve_near.  mbl_opts_default fills the defaults given in brackets. */
typedef struct mbl_opts {
    int precision;        /* MBL_PREC_* of the fronts                               [FP32] */
    int block;            /* block width p of the shift-invert Lanczos, 1..32       [8]    */
    int ncv;              /* Krylov basis size before a restart, 0 = automatic      [0]    */
    int max_restarts;     /* thick restarts before MBL_ERR_NOT_CONVERGED            [60]   */
    double tol;           /* accept when ||H y - theta y|| <= tol ||H||              [1e-10]*/
    double target_tol;    /* converge towards this (the FP64 floor)                  [1e-13]*/
    double refine_tol;    /* refinement stop: ||b - A x|| <= refine_tol (|A||x| + |b|)[1e-14]*/
    int max_refine;       /* refinement steps per application                       [20]   */
    uint64_t start_seed;  /* seed of the random start block                         [12345]*/
    int tensor_cores;     /* FP32 fronts' Schur updates: 0 CUDA cores, 1 tcgen05 3xTF32,      
                             2 tcgen05 3xBF16 (split-BF16 operands, FP32 accumulation)   [1]   */
    int refine_mode;      /* 0: plain iterative refinement, 1: FGMRES with the factor as    */
                          /*    right preconditioner (FP64 Arnoldi per right-hand side)  [1]   */
    int gmres_restart;    /* FGMRES inner dimension before a restart (1..64)          [24]   */
    int solve_dataflow;   /* 1: solves as one persistent dataflow kernel per sweep; 0: one */
                          /*    graph-captured launch per level gather and solve panel  [0]    */
    int deflate;          /* FGMRES preconditioner deflated by the kept Ritz vectors    [1]    */
    double wait_limit_s;  /* limit of each bounded dependency wait of the dataflow solves, */
                          /*    seconds in [0, 60]; 0 = 1 s.  An expired wait stops the   */
                          /*    waiting CTA and the call returns MBL_ERR_TIMEOUT        [0]    */
    int arena_mode;       /* fronts arena: 0 automatic (memory-lean when the whole arena  */
                          /*    would exceed 8 GiB), 1 memory-lean, 2 whole arena       [0]    */
                          /*    Memory-lean: the arena is a reserved virtual range whose */
                          /*    regions (fronts of one tree level with one parent level) */
                          /*    are backed by device memory from their level's assembly */
                          /*    until their parents' assembly; a front's factor columns  */
                          /*    are released once copied to the solve factor.            */
    double pivot_tiny;    /* static pivoting: a pivot below pivot_tiny ||H|| is replaced by  */
                          /*    +-pivot_tiny ||H||; 0 = 1e-7 (FP32 fronts), 1e-12 (FP64)  [0]    */
} mbl_opts;

typedef struct mbl_factor_stats {
    int64_t n;              /* sector dimension */
    int64_t nnz_l;          /* stored entries of the unit lower factor (strictly lower) */
    int64_t n_supernodes;   /* fronts of the assembly tree */
    int64_t max_front;      /* largest front order */
    int64_t tree_levels;    /* levels of the batched schedule */
    int64_t perturbed;      /* pivots replaced by +-tiny (static pivoting) */
    int64_t negative;       /* negative pivots = eigenvalues of H below sigma (if none perturbed) */
    double flops;           /* algorithmic factorization flops (sum over fronts) */
    double factor_bytes;    /* bytes of the stored factor */
    double front_bytes;     /* bytes of the frontal arena (factor + contribution blocks) */
    double ms_factor;       /* device time of the numeric factorization */
    double max_abs_l;       /* largest |L_ij| (element growth of the pivoting) */
    double min_abs_d;       /* smallest |D_jj| */
    /* Autotuned tile shape of the FP32 fronts' trailing update by size class c of the panel step's
     * largest trailing block (64 2^c <= m2 < 64 2^(c+1); class 0 also smaller, class 7 also larger),
     * measured once per sector shape and tensor-core mode on a synthetic front of the class:
     * 1 = tcgen05 128 x 128 tiles, 0 = CUDA-core 64 x 64 tiles, -1 = not tuned (FP64 fronts or CUDA
     * cores requested); the two timings in microseconds (0 where the class has no panel step). */
    int tune_choice[8];
    float tune_us_tc[8], tune_us_cc[8];
} mbl_factor_stats;

typedef struct mbl_solve_stats {
    int restarts;           /* thick restarts done */
    int op_applies;         /* block applications of (H - sigma)^-1 */
    int solves;             /* block triangular solves (applications x refinement steps) */
    int fp64_fallback;      /* 1 if refinement stalled and FP64 fronts were used */
    int krylov_dim;         /* final basis size */
    double max_resid;       /* max ||H y - theta y|| / ||H|| of the returned pairs */
    double ms_total;        /* wall time of solve_near */
    double ms_factor;       /* of which numeric factorization */
    int shift_moves;        /* times the factorization shift moved off an eigenvalue (target on one) */
    int refine_escalations; /* stalls answered with a longer FGMRES instead of FP64 fronts (which would
                               not fit in device memory) */
    int factor_reused;      /* serving: the factorization came from the server's cache of live factors */
    double static_pivot;    /* static pivoting threshold used, relative to ||H|| (0: the precision's
                               default); sqrt(eps_FP32) for FP32 fronts where an FP64 refactorization
                               could not fit in device memory */
} mbl_solve_stats;

void mbl_opts_default(mbl_opts *opts);
const char *mbl_version(void);
const char *mbl_last_error(mbl_ctx *ctx);
const char *mbl_status_string(int status);

/* Number of kernels this library has launched since it was loaded (all contexts). */
long long mbl_launch_count(void);
/* Opt-in device timing by kernel class with CUDA events on the launching stream.  Turning it on
 * or off clears the totals.  Classes: "factor_fp32" / "factor_fp64" (whole numeric factorization,
 * work = algorithmic flops), "schur_fp32" / "schur_fp64" (trailing updates, flops),
 * "trisolve_fp32" / "trisolve_fp64" (forward + backward solve of one block, work = algorithmic
 * bytes: factor read twice plus the right-hand sides), "refine_spmv" (FP64 residual SpMV, bytes),
 * "orth" (block Gram-Schmidt, FP64 flops). */
int mbl_ctx_set_profiling(mbl_ctx *ctx, int on);
int mbl_ctx_profile_get(mbl_ctx *ctx, const char *name, int64_t *launches, double *ms, double *work);

/* Context on CUDA device `device` with a memory budget (0 = no limit) used for admission. */
int mbl_ctx_create(int device, size_t hbm_budget_bytes, mbl_ctx **out);
void mbl_ctx_destroy(mbl_ctx *ctx);
int mbl_ctx_synchronize(mbl_ctx *ctx);

/* Sector of Eq. 1 for (L, h, seed): h_i = h (2 u_i - 1), u_i = (z_i >> 11) 2^-53 with z_i the
 * i-th output of SplitMix64 started at `seed` (the paper names no generator).  Builds the basis
 * (combinadic enumeration) and the CSR Hamiltonian on the device, bit-exactly:
 *   row k: columns ascending, diagonal always stored, value
 *          0.25 J (n_aligned - n_antiparallel) then + (+-0.5) h_i for i = 0..L-1 in order,
 *          one off-diagonal J/2 per antiparallel bond (i, i+1 mod L), summed when two bonds reach
 *          the same state (L = 2 only).
 * L must be even, 2 <= L <= 22, h >= 0. */
int mbl_build_sector(mbl_ctx *ctx, int L, double h, uint64_t seed, mbl_sector **out);
/* Same with explicit fields h_i[L] (host) and coupling J. */
int mbl_build_sector_fields(mbl_ctx *ctx, int L, const double *h_i, double J, mbl_sector **out);
/* The same constructions for the magnetization sector with nup up spins (S^z_tot = nup - L/2):
 * 2 <= L <= 22 of either parity, 0 <= nup <= L, basis = the colex enumeration of nup-subsets of the
 * L sites (dimension C(L, nup)).  The numerical-method section uses S^z = 0 for even L
 * (nup = L/2, what mbl_build_sector builds) and an "S^z = 1" sector for odd L = 15, 17, 19, read as
 * nup - (L - nup) = 1, i.e. nup = (L + 1)/2.  MBL_ERR_INVALID outside these ranges. */
int mbl_build_sector_nup(mbl_ctx *ctx, int L, int nup, double h, uint64_t seed, mbl_sector **out);
int mbl_build_sector_fields_nup(mbl_ctx *ctx, int L, int nup, const double *h_i, double J,
                                mbl_sector **out);
void mbl_sector_destroy(mbl_sector *sec);

int mbl_sector_info(const mbl_sector *sec, int64_t *dim, int64_t *nnz);
/* Chain length and up-spin count of the sector (either pointer may be NULL). */
int mbl_sector_shape(const mbl_sector *sec, int *L, int *nup);
/* Device-to-host copies for inspection: states[dim]; rowptr[dim+1], col[nnz], val[nnz]; h_i[L]. */
int mbl_sector_copy_basis(const mbl_sector *sec, uint32_t *states);
int mbl_sector_copy_csr(const mbl_sector *sec, int64_t *rowptr, int32_t *col, double *val);
int mbl_sector_copy_fields(const mbl_sector *sec, double *h_i);
/* Combinadic rank of `count` states (host arrays) computed on the device; -1 if a state is not
 * in the sector. */
int mbl_sector_rank(const mbl_sector *sec, const uint32_t *states, int64_t count, int64_t *ranks);
/* y = (H - shift) x for nrhs vectors, host arrays n x nrhs column-major (FP64 CSR SpMV). */
int mbl_spmv(mbl_sector *sec, double shift, const double *x, double *y, int nrhs);

/* E_min and E_max of the sector (numerical-method section): block Lanczos on H with full
 * reorthogonalization, converged to 1e-13 ||H||.  Cached on the sector. */
int mbl_extremal_bounds(mbl_sector *sec, double *e_min, double *e_max);

/* Numeric factorization P (H - sigma I) P^T = L D L^T (supernodal multifrontal; ordering and
 * symbolic analysis cached per L in the context).  Diagonal pivoting inside each panel of the
 * fully-summed block; a pivot below tiny = 1e-7 ||H|| (FP32) or 1e-12 ||H|| (FP64) is replaced by
 * +-tiny and counted.  opts may be NULL (defaults). */
int mbl_factor(mbl_sector *sec, double sigma, const mbl_opts *opts, mbl_factorization **out);
int mbl_factor_stats_get(const mbl_factorization *f, mbl_factor_stats *stats);
/* x = (H - sigma)^-1 b for nrhs right-hand sides (host, n x nrhs column-major), with FP64
 * iterative refinement when `refine` is nonzero. */
int mbl_factor_solve(mbl_factorization *f, const double *b, double *x, int nrhs, int refine);
/* Device variant: d_b and d_x are device FP64 arrays, n x nrhs column-major (leading dimension n),
 * owned by the caller and distinct.  The solve is enqueued on `stream` (a cudaStream_t; NULL = the
 * context's stream) and the call returns once it has completed there.  A factorization serves one
 * call at a time.  Unrefined solves (refine = 0) run without device allocation; MBL_ERR_TIMEOUT if
 * a bounded dependency wait of the solve kernels expired. */
int mbl_factor_solve_dev(mbl_factorization *f, const double *d_b, double *d_x, int nrhs, int refine, void *stream);
/* Unrefined solves of K factorizations at once: d_x[k] = (L_k D_k L_k^T)^-1 d_b[k] for k < K, each
 * an n x nrhs column-major device block (leading dimension n), owned by the caller.  All K
 * factorizations must come from sectors of the same (L, nup) -- one symbolic plan -- and the same
 * precision, each at most once, none made with solve_dataflow.  The jobs share every launch of the
 * solve sequence (the same kernels on each factorization's own buffers), so each result is
 * bit-identical to mbl_factor_solve_dev(refine = 0) of its factorization alone.  Enqueued on
 * `stream` (NULL = the first factorization's context stream); returns once complete.  1 <= K <= 64.
 * Not in the paper: the batching pattern for many small jobs of one sector size. */
int mbl_factor_solve_batch_dev(mbl_factorization *const *fs, int K, const double *const *d_b,
                               double *const *d_x, int nrhs, void *stream);
/* Symbolic analysis of the sector's pattern (nested-dissection ordering, supernodes, schedules;
 * numerical-method section: the analysis phase of the direct solver), built on the host on first
 * use for this (L, nup, ordering) and cached in the context, and its predicted fill-in and device footprint.  No
 * numeric factorization runs, so this works for sizes whose fronts would not fit in memory.
 * job_peak_* is the serving admission estimate of one solve_near job with (nev, block). */
typedef struct mbl_plan_stats {
    int64_t n, nnz_l, n_supernodes, max_front, tree_levels, panel_steps, solve_steps;
    double flops;                   /* algorithmic factorization flops */
    double ms_analyse;              /* host time of the analysis when it was built */
    double factor_bytes_fp32, factor_bytes_fp64;  /* entries of L and D */
    double front_bytes_fp32, front_bytes_fp64;    /* the fronts arena (alive during the factorization) */
    double solve_factor_bytes_fp32;               /* packed G of the solve panels (alive with the factor) */
    double job_peak_bytes_fp32, job_peak_bytes_fp64;
    double front_peak_bytes_fp32, front_peak_bytes_fp64;  /* the fronts arena at its peak in the automatic
                                                             arena mode (see mbl_opts.arena_mode) */
    int64_t ordering;               /* the MBL_ORDER_* the plan was built with (MBL_ORDER_AUTO resolved) */
} mbl_plan_stats;
int mbl_analyse(mbl_sector *sec, int nev, int block, mbl_plan_stats *stats);
/* Ordering used by the symbolic analyses built from now on in this context and in the serving
 * workers that share its plans (MBL_ORDER_*, default MBL_ORDER_AUTO).  Plans are cached per
 * (L, nup, ordering), so plans and factorizations made before the call are unaffected.  Any
 * ordering gives the same factorization in exact arithmetic; they differ in fill-in, flops and
 * front sizes (mbl_analyse).  MBL_ERR_INVALID for an unknown value.  Not in the paper, whose
 * direct solver (the MUMPS package) chooses its own ordering. */
int mbl_ctx_set_ordering(mbl_ctx *ctx, int ordering);

/* Launch trace of the level-by-level triangular solve, a diagnostic with no counterpart in the
 * paper.  With on != 0 every later solve of f records, for each kernel launch of its sequence, the
 * device clock (%globaltimer, ns) when the launch's first CTA started and when its last CTA
 * finished; on = 0 stops recording.  Switching recaptures the solve graph.  MBL_ERR_INVALID for a
 * factorization made with solve_dataflow. */
int mbl_factor_trace(mbl_factorization *f, int on);
/* Copies the records of the latest solve: up to cap launches in sequence order into t0[], t1[] and
 * kind[] (0 forward gather, 1 forward panel step, 2 backward level start, 3 backward update);
 * *count = number recorded
 * (0 when tracing is off). */
int mbl_factor_trace_get(mbl_factorization *f, unsigned long long *t0, unsigned long long *t1, int *kind,
                         int cap, int *count);
void mbl_factor_destroy(mbl_factorization *f);

/* The nev eigenpairs of the sector nearest sigma = E_min + eps (E_max - E_min): block
 * shift-invert Lanczos with full reorthogonalization and thick restarts on (H - sigma)^-1,
 * every application refined in FP64 against the CSR, then Rayleigh-Ritz on H.
 * Outputs (host): evals[nev] ascending, evecs[n*nev] column-major, resid[nev] =
 * ||H y - theta y||; *nconv = pairs with resid <= tol ||H||; *sigma_used.  stats may be NULL.
 * Returns MBL_ERR_NOT_CONVERGED (with the partial results written) if nconv < nev. */
int mbl_solve_near(mbl_sector *sec, double eps, int nev, const mbl_opts *opts, double *evals,
                   double *evecs, double *resid, int *nconv, double *sigma_used,
                   mbl_solve_stats *stats);
/* Same with device outputs d_evals[nev], d_evecs[n*nev], d_resid[nev]; returns after the
 * results are written (the host needs them to decide convergence). */
int mbl_solve_near_dev(mbl_sector *sec, double eps, int nev, const mbl_opts *opts,
                       double *d_evals, double *d_evecs, double *d_resid, int *nconv,
                       double *sigma_used, mbl_solve_stats *stats, void *stream);

/* Observables of nev eigenpairs of an L-site sector (characterization section):
 *   r[nev-2]   gap ratios r_k = min(d_k, d_{k+1}) / max(d_k, d_{k+1}), d_k = E_k - E_{k-1},
 *              of the ascending evals (NaN where both gaps are zero, excluded from r_mean);
 *   s1p[nev]   participation entropy -sum_i p_i ln p_i, p_i = y_i^2 / ||y||^2;
 *   se[nev]    half-chain entanglement entropy -Tr rho_A ln rho_A, A = sites 0..L/2-1,
 *              from the eigenvalues of the Gram matrices M M^T of the reshaped vector
 *              (Schmidt weights below 1e-15 count as zero).
 * Host arrays; evecs n x nev column-major. */
int mbl_observables(mbl_ctx *ctx, int L, int nev, const double *evals, const double *evecs,
                    double *r, double *r_mean, double *s1p, double *se);
/* Same on device arrays, enqueued on `stream` (NULL = context stream). */
int mbl_observables_dev(mbl_ctx *ctx, int L, int nev, const double *d_evals,
                        const double *d_evecs, double *d_r, double *d_r_mean, double *d_s1p,
                        double *d_se, void *stream);
/* The same for eigenvectors of the sector (L, nup) of mbl_build_sector_nup: A = sites
 * 0 .. floor(L/2) - 1, B the other L - floor(L/2) sites; the Schmidt blocks are indexed by the up
 * spins n_A of A (n_B = nup - n_A).  The entry points without nup take nup = L/2 and even L. */
int mbl_observables_nup(mbl_ctx *ctx, int L, int nup, int nev, const double *evals,
                        const double *evecs, double *r, double *r_mean, double *s1p, double *se);
int mbl_observables_nup_dev(mbl_ctx *ctx, int L, int nup, int nev, const double *d_evals,
                            const double *d_evecs, double *d_r, double *d_r_mean, double *d_s1p,
                            double *d_se, void *stream);

/* Further eigenvector observables of the characterization section and its supplement, on the
 * columns of evecs (n x nev column-major, host; ascending eigenvalues, so adjacent columns are
 * adjacent eigenstates).  With p_i = y_i^2 / |y|^2 of a column y:
 *   kl[k]    (nev-1) Kullback-Leibler divergence sum_i p_i ln(p_i / q_i) of column k (p) and column
 *            k+1 (q), "level statistics and eigenvectors similarity" paragraph; +infinity if some
 *            q_i = 0 < p_i;
 *   sqp[j]   participation entropy S_q^P = ln(sum_i p_i^q) / (1 - q), q > 0 and q != 1, "Hilbert
 *            space localization" paragraph (q = 1 is the s1p output of mbl_observables);
 *   fluct[j] bipartite fluctuation <(S^z_A)^2> - <S^z_A>^2 of A = sites 0 .. L/2-1, "entanglement
 *            entropy" paragraph;
 *   dynf[j]  dynamic spin fraction 1 - |<M>|^2 / <M^+ M>, M = sum_j S^z_j exp(2 pi i j / L), of the
 *            supplementary section (NaN if <M^+ M> = 0).
 * Errors: MBL_ERR_INVALID for odd L, L outside 2..22, nev outside [1, dim], q <= 0 or q = 1. */
int mbl_observables_extra(mbl_ctx *ctx, int L, int nev, const double *evecs, double q, double *kl,
                          double *sqp, double *fluct, double *dynf);
/* Same on device arrays, enqueued on `stream` (NULL = context stream) without synchronizing: the
 * outputs are complete when the stream reaches this point.  Scratch comes from the context's
 * per-L cache, so calls on one context must not overlap. */
int mbl_observables_extra_dev(mbl_ctx *ctx, int L, int nev, const double *d_evecs, double q,
                              double *d_kl, double *d_sqp, double *d_fluct, double *d_dynf,
                              void *stream);
/* The same for the sector (L, nup); A = sites 0 .. floor(L/2) - 1 in fluct. */
int mbl_observables_extra_nup(mbl_ctx *ctx, int L, int nup, int nev, const double *evecs, double q,
                              double *kl, double *sqp, double *fluct, double *dynf);
int mbl_observables_extra_nup_dev(mbl_ctx *ctx, int L, int nup, int nev, const double *d_evecs,
                                  double q, double *d_kl, double *d_sqp, double *d_fluct,
                                  double *d_dynf, void *stream);

/* Half-chain entanglement entropy (the se output of mbl_observables_dev) computed without any
 * device allocation.  The paper has no counterpart: it exists for callers that cannot allocate
 * device memory (a worker whose admitted jobs already hold the whole HBM budget; a loop that must
 * not trigger the device-wide synchronization of cudaFree).  Its scratch is a fixed 12 MiB device
 * array in the library, whose address is taken once per device when a context is created.  Limits:
 * even L <= 16 and 1 <= nev <= 64 (MBL_ERR_INVALID otherwise).  d_evecs: n x nev column-major
 * device array; d_se: nev device outputs; enqueued on `stream` (NULL = context stream) and
 * complete when the stream reaches it.  The scratch is shared by all callers on the device:
 * overlapping calls race and must be serialized by the caller.  MBL_ERR_CUDA if the scratch
 * address could not be taken on this device. */
int mbl_entanglement_noalloc_dev(mbl_ctx *ctx, int L, int nev, const double *d_evecs, double *d_se,
                                 void *stream);

/* ---- Serving: request loop with continuous batching and HBM admission -------------------
 * Not in the paper, which diagonalizes one realization per batch job; this is the serving
 * pattern for streams of (L, h, seed, eps, nev) requests of mixed L.
 *
 * mbl_server_start creates `slots` worker threads on the context's device, each with its own
 * stream and scratch, sharing the context's symbolic analyses.  Requests start in arrival order as
 * workers free up; before the solve a worker reserves the job's estimated peak HBM (from the
 * symbolic plan of its L) against `budget_bytes` (0 = 85% of the free device memory, capped by the
 * context budget) and waits while it does not fit, so jobs run side by side as memory allows.  A
 * job runs the same steps as mbl_build_sector + mbl_solve_near + mbl_observables and gives the
 * same result as those calls alone.  Errors: MBL_ERR_INVALID (bad slots, server already running). */
typedef struct mbl_request {
    int L;            /* 2..22 (odd L needs nup) */
    double h;         /* disorder strength, fields from the seeded stream (as mbl_build_sector) */
    uint64_t seed;
    const double *fields; /* optional h_i[L] (host, copied at submission; J = 1) instead of (h, seed) */
    double eps;       /* target energy density in [0, 1] */
    int nev;
    int precision;    /* MBL_PREC_FP32 (mixed) or MBL_PREC_FP64 */
    int want_vectors; /* keep the eigenvectors for mbl_poll */
    int nup;          /* up spins of the sector; 0 = L/2 (S^z_tot = 0, even L only) */
} mbl_request;

/* Filled by mbl_poll / mbl_wait.  The array fields are caller-owned outputs set before the call
 * (NULL = not wanted): evals[nev], resid[nev], r[nev-2], s1p[nev], se[nev], evecs[dim*nev]
 * (column-major; only if the request had want_vectors).  Times are host milliseconds since
 * mbl_server_start: submission, admission (HBM reserved, solve starts), completion; d_start_ms and
 * d_end_ms are the device-side (CUDA event) start and end of the job's work on its worker stream,
 * in milliseconds after an event recorded on the context stream at mbl_server_start. */
typedef struct mbl_result {
    int status;       /* MBL_OK, MBL_ERR_NOT_CONVERGED (partial), or the job's error */
    int nconv, nev, L;
    int64_t dim;
    double sigma, r_mean;
    double t_submit_ms, t_admit_ms, t_end_ms;
    double d_start_ms, d_end_ms;
    size_t reserved_bytes;
    double *evals, *resid, *r, *s1p, *se, *evecs;
    int factor_reused;  /* the job's factorization came from the server's cache of live factors */
} mbl_result;

typedef struct mbl_server_stats {
    int64_t submitted, completed, failed;
    int running, queued, slots;
    size_t budget_bytes, reserved_bytes, peak_reserved_bytes;
    int64_t solve_batches;   /* batched triangular-solve launches (see mbl_server_batching) */
    int64_t batched_solves;  /* block solves they held */
    double batch_ms;         /* their device time (CUDA events on the batcher's stream) */
    double batch_bytes;      /* their algorithmic bytes: per block solve the factor read by both
                                sweeps plus the right-hand sides, 2 (nnz_L + n) w + 16 n p */
    int64_t cache_hits;      /* requests served with a cached live factorization */
    size_t cache_bytes;      /* device bytes the cache holds now */
    double batch_busy_ms;    /* time during which at least one batch was executing (the union of the
                                batches' intervals; batches on different lanes overlap, so batch_ms
                                can exceed it) */
} mbl_server_stats;

/* Residency of live factorizations (set before mbl_server_start; default fraction 0.25, 0 = off).
 * A finished job's sector and factorization stay on the device, up to `fraction` of the server
 * budget, most recently used kept first; a later request with the same sector shape, fields (or
 * (h, seed)), eps and precision takes them and skips the sector build, the extremal bounds and the
 * factorization.  Cached bytes count against the budget: admission evicts the least recently used
 * entries before it makes a request wait.  Not in the paper: a serving pattern for repeated targets.
 * MBL_ERR_INVALID while a server runs or for fraction outside [0, 0.9]. */
int mbl_server_cache(mbl_ctx *ctx, double fraction);

/* Continuous batching of the workers' triangular solves (set before mbl_server_start; defaults
 * max_jobs = 16, window_us = 300, lanes = 2).  Jobs of one sector size share a symbolic plan, so
 * their block solves are one launch sequence on different buffers: a worker's solve is handed to a
 * batcher thread, which launches the sequence once for up to max_jobs workers' solves of the same
 * (plan, precision, block width) -- every launch covers all of them -- on one of `lanes` streams:
 * as soon as every worker inside a solve phase of that group has one waiting, or, while a lane is
 * idle, when the oldest has waited window_us microseconds.  While every lane is busy, requests
 * gather until one completes.  Results are the same as unbatched solves (the same kernels on each
 * job's own buffers).  max_jobs = 1 turns batching off.  Not in the paper: a serving pattern for
 * many small jobs.  MBL_ERR_INVALID while a server runs or for max_jobs outside [1, 64], window_us
 * outside [0, 1e6], lanes outside [1, 8]. */
int mbl_server_batching(mbl_ctx *ctx, int max_jobs, double window_us, int lanes);

int mbl_server_start(mbl_ctx *ctx, int slots, size_t budget_bytes);
/* Queue a request; *ticket identifies it.  MBL_ERR_INVALID for bad arguments or no server. */
int mbl_submit(mbl_ctx *ctx, const mbl_request *req, uint64_t *ticket);
/* Non-blocking: MBL_PENDING while queued or running; otherwise fills *out, returns the job's
 * status and forgets the ticket (a second poll gives MBL_ERR_INVALID). */
int mbl_poll(mbl_ctx *ctx, uint64_t ticket, mbl_result *out);
/* Blocking variant; timeout_s <= 0 waits without limit, else MBL_PENDING after timeout_s. */
int mbl_wait(mbl_ctx *ctx, uint64_t ticket, double timeout_s, mbl_result *out);
int mbl_server_stats_get(mbl_ctx *ctx, mbl_server_stats *out);
/* Stop the workers: running jobs finish, queued ones are dropped with their results.  Called by
 * mbl_ctx_destroy.  Must not overlap mbl_wait/mbl_poll on the same context. */
int mbl_server_stop(mbl_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MBLSI_H */
