/*
 * mbl_oracle.h -- plain CPU FP64 reference for the shift-invert exact diagonalization of the
 * random-field Heisenberg chain (Luitz, Laflorencie, Alet, arXiv:1411.0660).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent checker of the GPU path: only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or helper with the GPU library.  Everything is FP64, single threaded
 * and written for readability, not speed.
 *
 * Conventions (the paper leaves them open; each is a stated reading):
 *   - H = J sum_i S_i . S_{i+1 mod L} + sum_i h_i S^z_i   (Eq. 1; field sign as "+h_i")
 *   - site i <-> bit i of a uint32 state, bit set = spin up (S^z = +1/2)
 *   - sector S^z_tot = 0 (popcount = L/2), basis in ascending integer order
 *   - h_i = h (2 u_i - 1), u_i = (z_i >> 11) 2^-53, z_i the i-th SplitMix64 output from seed
 *   - eps = (E - E_min) / (E_max - E_min), sigma = E_min + eps (E_max - E_min)
 *   - half chain A = sites 0 .. L/2-1 (the low bits)
 * Parity unpinned: nothing.  Every function here is checked by the not-gpu tests against
 * closed forms, an independent tensor-product construction, brute force or library routines.
 */
#ifndef MBL_ORACLE_H
#define MBL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Disorder fields h_i (Eq. 1, h_i uniform on [-h, h]) from a SplitMix64 stream.  out[L]. */
void orc_fields(int L, double h, uint64_t seed, double *out);

/* Binomial coefficient C(n, k) as an exact 64-bit integer (0 if k < 0 or k > n). */
int64_t orc_binom(int n, int k);

/* Basis of the sector with nup up spins (2 <= L <= 30, 0 <= nup <= L) by brute force over all 2^L
 * states, ascending.  Returns the count (-1 for invalid arguments); states may be NULL to only count. */
int64_t orc_basis_sector(int L, int nup, uint32_t *states);
/* S^z_tot = 0 basis (even L): orc_basis_sector(L, L/2, states). */
int64_t orc_basis(int L, uint32_t *states);

/* Number of stored entries of H in the sector (diagonal included, duplicates merged). */
int64_t orc_nnz(int L, const uint32_t *states, int64_t n);

/* CSR of H in the sector (Eq. 1).  Columns ascending inside each row; the diagonal is always
 * stored.  The diagonal is 0.25 J (n_aligned - n_anti) followed by the field terms
 * +-0.5 h_i added for i = 0 .. L-1 in that order.  Off-diagonal entries are J/2 per
 * anti-aligned bond (summed if two bonds reach the same state, which happens only at L = 2). */
int orc_csr(int L, const double *hi, double J, const uint32_t *states, int64_t n,
            int64_t *rowptr, int32_t *col, double *val);

/* y = (A - shift I) x for a CSR matrix. */
void orc_spmv(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
              double shift, const double *x, double *y);

/* Dense symmetric eigensolver: Householder tridiagonalization followed by the implicit QL
 * iteration with Wilkinson shift.  A is n x n column-major (full, symmetric); on return w
 * holds the eigenvalues ascending and, if want_vectors, A holds the matching orthonormal
 * eigenvectors (column j for w[j]).  Returns 0, or -1 if the iteration did not converge. */
int orc_syev(int n, double *A, double *w, int want_vectors);

/* Eigenvalues (ascending) and optionally the last components of the eigenvectors of a
 * symmetric tridiagonal matrix with diagonal d[n] and off-diagonal e[n-1]. */
int orc_stev(int n, const double *d, const double *e, double *w, double *zlast);

/* Extremal eigenvalues of H by plain Lanczos with full reorthogonalization, converged to
 * |residual| <= tol * max(|E_min|, |E_max|).  Returns the number of Lanczos steps or < 0. */
int orc_extremal_lanczos(int64_t n, const int64_t *rowptr, const int32_t *col,
                         const double *val, double tol, uint64_t start_seed,
                         double *emin, double *emax);

/* The nev eigenpairs closest to sigma from a full dense diagonalization.  evals ascending,
 * evecs n x nev column-major unit vectors.  Ties in |lambda - sigma| take the lower lambda. */
int orc_nearest_dense(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                      double eps, int nev, double *emin, double *emax, double *sigma,
                      double *evals, double *evecs);

/* ---- sparse shift-invert path (for sizes beyond dense reach) ---- */
typedef struct orc_ldlt orc_ldlt;   /* opaque */

/* Minimum-degree ordering on the graph of the pattern (explicit elimination graph) and the
 * column structure of L.  The numeric LDL^T of A - sigma I without pivoting; a pivot with
 * |d| < tiny is replaced by sign(d) tiny (static perturbation; refinement recovers). */
orc_ldlt *orc_ldlt_analyse(int64_t n, const int64_t *rowptr, const int32_t *col);
int orc_ldlt_factor(orc_ldlt *f, const int64_t *rowptr, const int32_t *col, const double *val,
                    double sigma, double tiny);
void orc_ldlt_solve(const orc_ldlt *f, const double *b, double *x);
int64_t orc_ldlt_nnz(const orc_ldlt *f);
int64_t orc_ldlt_negative(const orc_ldlt *f);   /* inertia: number of negative pivots */
int64_t orc_ldlt_perturbed(const orc_ldlt *f);  /* number of perturbed pivots */
void orc_ldlt_free(orc_ldlt *f);

/* Shift-invert Lanczos (single vector, full reorthogonalization) on (H - sigma)^-1 applied
 * through the factor plus FP64 iterative refinement, then Rayleigh-Ritz on H.  Returns the nev
 * eigenpairs nearest sigma (ascending) with residuals ||H y - theta y||. */
int orc_nearest_shift_invert(int64_t n, const int64_t *rowptr, const int32_t *col,
                             const double *val, double sigma, int nev, double hnorm,
                             double *evals, double *evecs, double *resid);

/* ---- observables ---- */
/* Gap ratio r_k (k = 1 .. nev-2, zero-based middle level) of ascending evals; a ratio whose
 * two gaps are both zero is NaN and excluded from the mean. */
void orc_gap_ratio(int nev, const double *evals, double *r, double *r_mean);
/* Participation entropy S_1^P = -sum p_i ln p_i, p_i = y_i^2 / ||y||^2, 0 ln 0 = 0. */
double orc_s1p(int64_t n, const double *y);
/* Half-chain entanglement entropy (A = sites 0 .. L/2-1) of the sector vector y. */
double orc_entanglement(int L, const uint32_t *states, int64_t n, const double *y);
/* Kullback-Leibler divergence KL = sum_i p_i ln(p_i / q_i) of the weights p of y and q of z
 * ("level statistics and eigenvectors similarity" paragraph); terms with p_i = 0 are 0, a term with
 * p_i > 0 = q_i makes it +infinity. */
double orc_kl(int64_t n, const double *y, const double *z);
/* Participation entropy of order q != 1: S_q^P = ln(sum_i p_i^q) / (1 - q) ("Hilbert space
 * localization" paragraph). */
double orc_sqp(int64_t n, const double *y, double q);
/* Bipartite fluctuation F = <(S^z_A)^2> - <S^z_A>^2 of the half chain A = sites 0 .. L/2-1
 * ("entanglement entropy" paragraph); S^z_A is diagonal in the basis. */
double orc_fluct(int L, const uint32_t *states, int64_t n, const double *y);
/* Dynamic spin fraction f = 1 - |<M>|^2 / <M^dagger M>, M = sum_j S^z_j exp(2 pi i j / L)
 * (supplementary section on the dynamical spin fraction); M is diagonal in the basis.  NaN if
 * <M^dagger M> = 0. */
double orc_dynf(int L, const uint32_t *states, int64_t n, const double *y);

#ifdef __cplusplus
}
#endif
#endif
