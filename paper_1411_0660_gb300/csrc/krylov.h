// krylov.h -- block Krylov-Schur engine, refined shift-invert operator, eigen drivers.
#pragma once

#include <functional>

#include "factor.h"

namespace mbl {

constexpr int64_t DENSE_MAX_N = 400;  // sectors up to this size are diagonalized densely on the device

// Op: Y (n x p, ld p) = Op X (X row stride ldx)
using OpFn = std::function<void(const double *X, int ldx, double *Y, cudaStream_t st)>;

struct KrylovSchur {
    Ctx *ctx;
    int64_t n;
    int p, ncv, ldv;
    int m = 0;  // basis columns; the first m - p have been expanded
    DVec<double> V, V2, W, T, C1, C2, R1, R2, Rm, G, work, eigA, eigW, eigWork, res, SK, NS1, NS2, NS3, Ts, Bk;
    DVec<float> V32;  // FP32 copy of V for the first Gram-Schmidt pass
    DVec<int> flag, eigInfo, eigM, keep;
    DVec<int64_t> eigOff;

    KrylovSchur(Ctx *c, int64_t n_, int p_, int ncv_);
    bool full() const { return m + p > ldv; }  // no room for another block
    void start(uint64_t seed, cudaStream_t st);
    void expand(const OpFn &op, cudaStream_t st);
    // Ritz values (ascending) of the expanded part and their Krylov-Schur residual norms
    void ritz(cudaStream_t st, std::vector<double> &theta, std::vector<double> &rnorm);
    // keep the listed Ritz pairs (indices into the last ritz() result) plus the residual block
    void restart(const std::vector<int> &keep_idx, cudaStream_t st);

  private:
    void orthonormalize_new_block(int m, cudaStream_t st, bool *deflated);
};

// (H - sigma)^-1 through the factor with FP64 iterative refinement against the CSR.
struct RefinedSolve {
    mbl_sector *sec;
    Factorization *fz;
    double anorm;      // ||H - sigma|| bound
    double rtol;       // stop when ||b - A x|| <= rtol (anorm ||x|| + ||b||) per column
    int max_refine;
    int solves = 0, applies = 0;
    bool stalled = false;
    double last_rel = 0.0;
    int gmres = 1;     // 1: FGMRES refinement (factor as right preconditioner); 0: plain refinement
    int kmax = 24;     // FGMRES inner dimension
    int max_outer = 4; // FGMRES restarts per application before a stall is declared
    DVec<double> R, part, norms, GV, GZ, GW, Gh, Gy, Gdots;
    // Deflation of the preconditioner (FGMRES mode): with U (n x kd, row stride ldu) approximate
    // eigenvectors nearest sigma and A = H - sigma, the preconditioner is
    //   P = M^-1 (I - A Q) + Q,   Q = U (U^T A U)^-1 U^T,
    // M the factor: the directions where the factor is weakest are solved in span(U) exactly.
    // (U^T A U)^-1 is formed in FP64; U and A U are kept as FP32 copies (n x kd), since the
    // preconditioner needs them only to FP32 accuracy and FP64 products would cost ~20x more.
    int kd = 0;
    DVec<double> AU, Einv, Dc0, Dc1, Dt, Dwork;
    DVec<float> U32, AU32;
    DVec<int> Dflag;
    void apply(const double *X, int ldx, double *Y, int p, cudaStream_t st);
    // Use U[:, 0:k] (k <= 90; k = 0 switches deflation off); U is copied.
    void set_deflation(const double *U_, int ldu_, int k, cudaStream_t st);
    void clear_deflation() { kd = 0; }

  private:
    // true residual R = B - (H - sigma) Y; returns the worst ratio ||r_q|| / (rtol (anorm ||y_q|| + ||b_q||))
    double residual(const double *X, int ldx, double *Y, int p, cudaStream_t st, std::vector<double> *rn = nullptr,
                    std::vector<double> *lim = nullptr);
    void apply_plain(const double *X, int ldx, double *Y, int p, cudaStream_t st);
    void apply_fgmres(const double *X, int ldx, double *Y, int p, cudaStream_t st);
    void precondition(const double *V, double *Z, int p, cudaStream_t st);  // Z = P V (n x p, ld p)
};

// Rayleigh-Ritz of H on the whole basis: the nev Ritz pairs nearest sigma and their residuals.
struct RitzH {
    Ctx *ctx;
    int64_t n;
    int nev;
    unsigned nb = 0;
    DVec<double> HV, Gm, Gs, Gsym, Gr1, Gr2, Gr3, M2, Gw, Gwork, Ctmp, work, SKs, Y, HY, thd, part, nrm;
    DVec<double> Bwork;  // bisection eigensolver scratch
    DVec<int> gm, ginfo, didx;
    DVec<int64_t> goff;
    std::vector<double> evals, resid;
    int nconv = 0;
    double maxres = 0.0;  // max residual / ||H||
    RitzH(Ctx *c, int64_t n_, int ldv, int nev_);
    // writes the normalized Ritz vectors (n x nev column-major) to d_evecs
    void run(mbl_sector *sec, KrylovSchur &ks, double sigma, double hnorm, double tol, double *d_evecs,
             cudaStream_t st);
};

void extremal_bounds(mbl_sector *sec, double *emin, double *emax);
// keep (optional): a live factorization of this request to use instead of factoring (if it matches
// the sector and options), and where the job's factorization is left for reuse afterwards.
void solve_near(mbl_sector *sec, double eps, int nev, const mbl_opts &o, double *d_evals, double *d_evecs,
                double *d_resid, int *nconv, double *sigma_used, mbl_solve_stats *stats, cudaStream_t st,
                std::unique_ptr<Factorization> *keep = nullptr);

}  // namespace mbl
