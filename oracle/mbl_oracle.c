/*
 * mbl_oracle.c -- plain CPU FP64 reference implementation (test infrastructure only).
 *
 * Luitz, Laflorencie, Alet, "Many-body localization edge in the random-field Heisenberg
 * chain", arXiv:1411.0660.  What is computed follows the paper:
 *   Eq. 1 (model, periodic chain, S^z conserved), the numerical-method section (extremal
 *   energies, energy target, shift-invert spectral transformation, eigenpairs closest to the
 *   target), and the observables of the "characterization" section: gap ratio r^(n),
 *   participation entropy S_1^P, half-chain entanglement entropy S^E.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg use this file.
 * It is deliberately slow and direct: brute-force basis, binary-search CSR, textbook dense
 * Householder + implicit QL, a minimum-degree ordering on an explicit elimination graph,
 * a left-looking sparse LDL^T, and single-vector Lanczos with full reorthogonalization.
 * Compile with -ffp-contract=off so that no multiply-add is fused (the CSR diagonal is
 * compared bit for bit).
 */
#include "mbl_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------
 * Disorder (Eq. 1: h_i uniform on [-h, h]).  The paper does not name its generator; this uses
 * SplitMix64 as published by Steele, Lea and Flood (OOPSLA 2014): add the golden-gamma
 * increment to the state, then two xor-shift-multiply mixing rounds and a final xor-shift.
 * ------------------------------------------------------------------------------------------ */
static uint64_t sm64_next(uint64_t *state) {
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void orc_fields(int L, double h, uint64_t seed, double *out) {
    uint64_t st = seed;
    for (int i = 0; i < L; ++i) {
        uint64_t z = sm64_next(&st);
        double u = (double)(z >> 11) * (1.0 / 9007199254740992.0); /* 2^-53 */
        out[i] = h * (2.0 * u - 1.0);
    }
}

int64_t orc_binom(int n, int k) {
    if (k < 0 || k > n || n < 0) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i; /* stays an exact integer */
    return r;
}

static int popcount32(uint32_t s) {
    int c = 0;
    while (s) { c += (int)(s & 1u); s >>= 1; }
    return c;
}

/* ------------------------------------------------------------------------------------------
 * Basis of a magnetization sector (numerical-method section: the S^z = 0 sector of even L and
 * the S^z = 1 sector of odd L).  Brute force: every integer below 2^L with nup set bits (up
 * spins), in ascending order.  The S^z_tot = 0 sector is nup = L/2.
 * ------------------------------------------------------------------------------------------ */
int64_t orc_basis_sector(int L, int nup, uint32_t *states) {
    if (L < 2 || L > 30 || nup < 0 || nup > L) return -1;
    int64_t n = 0;
    uint32_t top = 1u << L;
    for (uint32_t s = 0; s < top; ++s)
        if (popcount32(s) == nup) {
            if (states) states[n] = s;
            ++n;
        }
    return n;
}

int64_t orc_basis(int L, uint32_t *states) {
    if (L & 1) return -1;
    return orc_basis_sector(L, L / 2, states);
}

static int64_t find_state(const uint32_t *states, int64_t n, uint32_t s) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (states[mid] == s) return mid;
        if (states[mid] < s) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* One row of H: returns the number of distinct entries, columns ascending (Eq. 1). */
static int row_entries(int L, const double *hi, double J, const uint32_t *states, int64_t n,
                       int64_t k, int32_t *cols, double *vals) {
    uint32_t s = states[k];
    int n_al = 0, n_anti = 0;
    int cnt = 0;
    int32_t c_tmp[64];
    double v_tmp[64];
    for (int i = 0; i < L; ++i) {
        int j = (i + 1) % L;
        int bi = (s >> i) & 1, bj = (s >> j) & 1;
        if (bi == bj) { ++n_al; continue; }
        ++n_anti;
        /* S^+_i S^-_j + S^-_i S^+_j exchanges the two antiparallel spins: amplitude J/2 */
        uint32_t t = s ^ (1u << i) ^ (1u << j);
        int64_t c = find_state(states, n, t);
        c_tmp[cnt] = (int32_t)c;
        v_tmp[cnt] = 0.5 * J;
        ++cnt;
    }
    /* diagonal: J S^z_i S^z_j per bond (+1/4 aligned, -1/4 antiparallel), then h_i S^z_i */
    double d = 0.25 * J * (double)(n_al - n_anti);
    for (int i = 0; i < L; ++i) d = d + (((s >> i) & 1u) ? 0.5 : -0.5) * hi[i];
    c_tmp[cnt] = (int32_t)k;
    v_tmp[cnt] = d;
    ++cnt;
    /* insertion sort by column, then merge duplicates (two bonds to one state only at L=2) */
    for (int a = 1; a < cnt; ++a) {
        int32_t cc = c_tmp[a];
        double vv = v_tmp[a];
        int b = a - 1;
        while (b >= 0 && c_tmp[b] > cc) { c_tmp[b + 1] = c_tmp[b]; v_tmp[b + 1] = v_tmp[b]; --b; }
        c_tmp[b + 1] = cc;
        v_tmp[b + 1] = vv;
    }
    int m = 0;
    for (int a = 0; a < cnt; ++a) {
        if (m > 0 && cols[m - 1] == c_tmp[a]) { vals[m - 1] += v_tmp[a]; continue; }
        cols[m] = c_tmp[a];
        vals[m] = v_tmp[a];
        ++m;
    }
    return m;
}

int64_t orc_nnz(int L, const uint32_t *states, int64_t n) {
    double *hz = (double *)calloc((size_t)L, sizeof(double));
    int32_t c[64];
    double v[64];
    int64_t nnz = 0;
    for (int64_t k = 0; k < n; ++k) nnz += row_entries(L, hz, 1.0, states, n, k, c, v);
    free(hz);
    return nnz;
}

int orc_csr(int L, const double *hi, double J, const uint32_t *states, int64_t n,
            int64_t *rowptr, int32_t *col, double *val) {
    int64_t p = 0;
    rowptr[0] = 0;
    for (int64_t k = 0; k < n; ++k) {
        int m = row_entries(L, hi, J, states, n, k, col + p, val + p);
        p += m;
        rowptr[k + 1] = p;
    }
    return 0;
}

void orc_spmv(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
              double shift, const double *x, double *y) {
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val[p] * x[col[p]];
        y[i] = s - shift * x[i];
    }
}

/* ------------------------------------------------------------------------------------------
 * Dense symmetric eigensolver: Householder reduction to tridiagonal form, then the implicit
 * QL iteration with a Wilkinson shift taken from the leading 2x2 of the active block
 * (Golub & Van Loan, Matrix Computations, sections 8.3.1-8.3.3, QL orientation).
 * ------------------------------------------------------------------------------------------ */

/* Apply the rotation J = [[c, s], [-s, c]] in plane (k, k+1) to the columns of Z. */
static void rot_cols(double *Z, int ldz, int zrows, int k, double c, double s) {
    double *zk = Z + (size_t)k * ldz, *zk1 = Z + (size_t)(k + 1) * ldz;
    for (int i = 0; i < zrows; ++i) {
        double a = zk[i], b = zk1[i];
        zk[i] = c * a - s * b;
        zk1[i] = s * a + c * b;
    }
}

/* One implicit QL sweep on the unreduced block lo..hi of (d, e): T <- J^T T J for rotations in
 * planes (hi-1, hi), (hi-2, hi-1), ..., (lo, lo+1).  The first rotation zeroes the upper entry
 * of the last column of T - mu I; each following one chases the bulge at (k, k+2) upward. */
static void ql_sweep(int lo, int hi, double *d, double *e, double *Z, int ldz, int zrows) {
    double delta = 0.5 * (d[lo + 1] - d[lo]);
    double b = e[lo];
    double mu = d[lo] - b * b / (delta + copysign(hypot(delta, b), delta));
    double x = d[hi] - mu, z = e[hi - 1];
    for (int k = hi - 1; k >= lo; --k) {
        double r = hypot(x, z);
        double c = 1.0, s = 0.0;
        if (r != 0.0) { c = x / r; s = z / r; }
        if (k < hi - 1) e[k + 1] = r; /* the bulge has been folded into entry (k+1, k+2) */
        double a = d[k], bb = e[k], dd = d[k + 1];
        d[k] = a * c * c - 2.0 * bb * c * s + dd * s * s;
        d[k + 1] = a * s * s + 2.0 * bb * c * s + dd * c * c;
        e[k] = (a - dd) * c * s + bb * (c * c - s * s);
        if (k > lo) {
            double bulge = s * e[k - 1]; /* new entry at (k-1, k+1) */
            e[k - 1] = c * e[k - 1];
            x = e[k];
            z = bulge;
        }
        if (zrows > 0) rot_cols(Z, ldz, zrows, k, c, s);
    }
}

static int negligible(const double *d, const double *e, int i) {
    return fabs(e[i]) <= DBL_EPSILON * (fabs(d[i]) + fabs(d[i + 1]));
}

static int ql_iterate(int n, double *d, double *e, double *Z, int ldz, int zrows) {
    int lo = 0, iter = 0;
    while (lo < n - 1) {
        if (negligible(d, e, lo)) { e[lo] = 0.0; ++lo; iter = 0; continue; }
        int hi = lo + 1;
        while (hi < n - 1 && !negligible(d, e, hi)) ++hi;
        if (hi < n - 1) e[hi] = 0.0;
        if (++iter > 100) return -1;
        ql_sweep(lo, hi, d, e, Z, ldz, zrows);
    }
    return 0;
}

/* Sort eigenvalues ascending, carrying the columns of Z along (selection sort). */
static void sort_eig(int n, double *w, double *Z, int ldz, int zrows) {
    for (int i = 0; i < n - 1; ++i) {
        int m = i;
        for (int j = i + 1; j < n; ++j) if (w[j] < w[m]) m = j;
        if (m == i) continue;
        double t = w[i]; w[i] = w[m]; w[m] = t;
        for (int r = 0; r < zrows; ++r) {
            double a = Z[r + (size_t)i * ldz];
            Z[r + (size_t)i * ldz] = Z[r + (size_t)m * ldz];
            Z[r + (size_t)m * ldz] = a;
        }
    }
}

int orc_syev(int n, double *A, double *w, int want_vectors) {
    if (n <= 0) return 0;
    if (n == 1) { w[0] = A[0]; if (want_vectors) A[0] = 1.0; return 0; }
    size_t N = (size_t)n;
    double *beta = (double *)calloc(N, sizeof(double));
    double *p = (double *)malloc(N * sizeof(double));
    double *v = (double *)malloc(N * sizeof(double));
    /* Householder: P_k = I - beta_k v v^T with v = [1, v_1, ...] maps A[k+1:, k] onto e_1 */
    for (int k = 0; k + 2 < n; ++k) {
        int m = n - k - 1;
        double *x = A + (size_t)k * N + (k + 1);
        double alpha = 0.0;
        for (int i = 0; i < m; ++i) alpha += x[i] * x[i];
        alpha = sqrt(alpha);
        if (alpha == 0.0) { beta[k] = 0.0; continue; }
        double sgn = x[0] >= 0.0 ? 1.0 : -1.0;
        double v0 = x[0] + sgn * alpha;
        double vtv = 1.0;
        v[0] = 1.0;
        for (int i = 1; i < m; ++i) { v[i] = x[i] / v0; vtv += v[i] * v[i]; }
        double bk = 2.0 / vtv;
        beta[k] = bk;
        /* p = beta A22 v ; w = p - (beta p^T v / 2) v ; A22 -= v w^T + w v^T */
        double *A22 = A + (size_t)(k + 1) * N + (k + 1);
        for (int i = 0; i < m; ++i) p[i] = 0.0;
        for (int j = 0; j < m; ++j) {
            double vj = bk * v[j];
            const double *cj = A22 + (size_t)j * N;
            for (int i = 0; i < m; ++i) p[i] += cj[i] * vj;
        }
        double ptv = 0.0;
        for (int i = 0; i < m; ++i) ptv += p[i] * v[i];
        double K = 0.5 * bk * ptv;
        for (int i = 0; i < m; ++i) p[i] -= K * v[i]; /* p now holds w */
        for (int j = 0; j < m; ++j) {
            double *cj = A22 + (size_t)j * N;
            double vj = v[j], wj = p[j];
            for (int i = 0; i < m; ++i) cj[i] -= v[i] * wj + p[i] * vj;
        }
        x[0] = -sgn * alpha;
        for (int i = 1; i < m; ++i) x[i] = v[i]; /* keep v below the subdiagonal */
    }
    double *d = (double *)malloc(N * sizeof(double));
    double *e = (double *)calloc(N, sizeof(double));
    for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * N + i];
    for (int i = 0; i + 1 < n; ++i) e[i] = A[(size_t)i * N + i + 1];
    double *Q = NULL;
    if (want_vectors) {
        Q = (double *)calloc(N * N, sizeof(double));
        for (int i = 0; i < n; ++i) Q[(size_t)i * N + i] = 1.0;
        /* Q = P_0 P_1 ... P_{n-3}, accumulated from the right end */
        for (int k = n - 3; k >= 0; --k) {
            if (beta[k] == 0.0) continue;
            int m = n - k - 1;
            v[0] = 1.0;
            for (int i = 1; i < m; ++i) v[i] = A[(size_t)k * N + k + 1 + i];
            for (int j = k + 1; j < n; ++j) {
                double *qj = Q + (size_t)j * N + (k + 1);
                double s = 0.0;
                for (int i = 0; i < m; ++i) s += v[i] * qj[i];
                s *= beta[k];
                for (int i = 0; i < m; ++i) qj[i] -= s * v[i];
            }
        }
    }
    int rc = ql_iterate(n, d, e, Q, n, want_vectors ? n : 0);
    for (int i = 0; i < n; ++i) w[i] = d[i];
    sort_eig(n, w, Q, n, want_vectors ? n : 0);
    if (want_vectors) memcpy(A, Q, N * N * sizeof(double));
    free(Q); free(d); free(e); free(beta); free(p); free(v);
    return rc;
}

int orc_stev(int n, const double *d_in, const double *e_in, double *w, double *zlast) {
    if (n <= 0) return 0;
    double *d = (double *)malloc((size_t)n * sizeof(double));
    double *e = (double *)calloc((size_t)n, sizeof(double));
    double *z = (double *)calloc((size_t)n, sizeof(double));
    memcpy(d, d_in, (size_t)n * sizeof(double));
    if (n > 1) memcpy(e, e_in, (size_t)(n - 1) * sizeof(double));
    z[n - 1] = 1.0; /* track the last row of the eigenvector matrix only */
    int rc = ql_iterate(n, d, e, z, 1, 1);
    memcpy(w, d, (size_t)n * sizeof(double));
    sort_eig(n, w, z, 1, 1);
    if (zlast) memcpy(zlast, z, (size_t)n * sizeof(double));
    free(d); free(e); free(z);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Extremal energies E_0, E_max (numerical-method section) by plain Lanczos with full
 * reorthogonalization (two classical Gram-Schmidt passes against every previous vector).
 * ------------------------------------------------------------------------------------------ */
static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static void random_unit(int64_t n, uint64_t seed, double *v) {
    uint64_t st = seed;
    double nrm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double u = (double)(sm64_next(&st) >> 11) * (1.0 / 9007199254740992.0);
        v[i] = 2.0 * u - 1.0;
        nrm += v[i] * v[i];
    }
    nrm = sqrt(nrm);
    for (int64_t i = 0; i < n; ++i) v[i] /= nrm;
}

/* w <- w - V c with c = V^T w, twice; returns the first-pass coefficient on column j0 + the
 * second-pass one (the full projection onto that column). */
static double reorthogonalize(int64_t n, int m, const double *V, double *w, int j0) {
    double proj = 0.0;
    double *c = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    for (int pass = 0; pass < 2; ++pass) {
        for (int j = 0; j < m; ++j) c[j] = dot(n, V + (size_t)j * n, w);
        for (int j = 0; j < m; ++j) {
            const double *vj = V + (size_t)j * n;
            for (int64_t i = 0; i < n; ++i) w[i] -= c[j] * vj[i];
        }
        if (j0 >= 0 && j0 < m) proj += c[j0];
    }
    free(c);
    return proj;
}

int orc_extremal_lanczos(int64_t n, const int64_t *rowptr, const int32_t *col,
                         const double *val, double tol, uint64_t start_seed,
                         double *emin, double *emax) {
    int mmax = n < 1000 ? (int)n : 1000;
    double *V = (double *)malloc((size_t)n * (mmax + 1) * sizeof(double));
    double *w = (double *)malloc((size_t)n * sizeof(double));
    double *al = (double *)calloc((size_t)mmax + 1, sizeof(double));
    double *be = (double *)calloc((size_t)mmax + 1, sizeof(double));
    double *th = (double *)malloc((size_t)mmax * sizeof(double));
    double *zl = (double *)malloc((size_t)mmax * sizeof(double));
    random_unit(n, start_seed, V);
    int steps = -1;
    for (int j = 0; j < mmax; ++j) {
        double *vj = V + (size_t)j * n;
        orc_spmv(n, rowptr, col, val, 0.0, vj, w);
        al[j] = reorthogonalize(n, j + 1, V, w, j);
        double b = sqrt(dot(n, w, w));
        be[j] = b;
        int m = j + 1;
        int check = (m == mmax) || (m >= 8 && (m % 4) == 0);
        double scale = 0.0;
        for (int i = 0; i <= j; ++i) scale = fmax(scale, fabs(al[i]) + be[i]);
        int breakdown = b <= 1e-14 * scale;
        if (check || breakdown) {
            orc_stev(m, al, be, th, zl);
            double hn = fmax(fabs(th[0]), fabs(th[m - 1]));
            double r0 = fabs(b * zl[0]), r1 = fabs(b * zl[m - 1]);
            if (breakdown || (r0 <= tol * hn && r1 <= tol * hn) || m == mmax) {
                *emin = th[0];
                *emax = th[m - 1];
                steps = (breakdown || (r0 <= tol * hn && r1 <= tol * hn)) ? m : -m;
                break;
            }
        }
        double *vn = V + (size_t)(j + 1) * n;
        for (int64_t i = 0; i < n; ++i) vn[i] = w[i] / b;
    }
    free(V); free(w); free(al); free(be); free(th); free(zl);
    return steps;
}

/* Pick the nev values of w[0..m) nearest sigma (ties: lower value first); idx ascending in w. */
static void nearest_indices(int m, const double *w, double sigma, int nev, int *idx) {
    char *used = (char *)calloc((size_t)m, 1);
    for (int t = 0; t < nev; ++t) {
        int best = -1;
        for (int i = 0; i < m; ++i) {
            if (used[i]) continue;
            if (best < 0) { best = i; continue; }
            double di = fabs(w[i] - sigma), db = fabs(w[best] - sigma);
            if (di < db || (di == db && w[i] < w[best])) best = i;
        }
        used[best] = 1;
        idx[t] = best;
    }
    /* ascending order of the selected values */
    for (int a = 1; a < nev; ++a) {
        int x = idx[a], b = a - 1;
        while (b >= 0 && w[idx[b]] > w[x]) { idx[b + 1] = idx[b]; --b; }
        idx[b + 1] = x;
    }
    free(used);
}

int orc_nearest_dense(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                      double eps, int nev, double *emin, double *emax, double *sigma,
                      double *evals, double *evecs) {
    if (nev < 1 || nev > n) return -2;
    size_t N = (size_t)n;
    double *A = (double *)calloc(N * N, sizeof(double));
    double *w = (double *)malloc(N * sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) A[(size_t)col[p] * N + i] = val[p];
    int rc = orc_syev((int)n, A, w, evecs != NULL);
    *emin = w[0];
    *emax = w[n - 1];
    *sigma = w[0] + eps * (w[n - 1] - w[0]);
    int *idx = (int *)malloc((size_t)nev * sizeof(int));
    nearest_indices((int)n, w, *sigma, nev, idx);
    for (int t = 0; t < nev; ++t) {
        evals[t] = w[idx[t]];
        if (evecs) memcpy(evecs + (size_t)t * N, A + (size_t)idx[t] * N, N * sizeof(double));
    }
    free(idx); free(A); free(w);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Sparse LDL^T of A - sigma I (the shift-invert transformation of the numerical-method
 * section; the paper factors with a parallel LU, the factorization is only the means).
 * ------------------------------------------------------------------------------------------ */
struct orc_ldlt {
    int64_t n;
    int64_t *perm;  /* perm[k]: original index eliminated k-th */
    int64_t *iperm; /* iperm[perm[k]] = k */
    int64_t *Lp;    /* strictly lower L, column pointers in elimination order */
    int32_t *Li;    /* row indices (elimination order), ascending per column */
    double *Lx;
    double *D;
    int64_t negative, perturbed;
};

static int popcount64(uint64_t x) { return __builtin_popcountll(x); }

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Minimum-degree ordering on an explicit elimination graph held as one bitset row per vertex:
 * repeatedly eliminate a vertex of least current degree (lowest index on ties), joining its
 * neighbours into a clique.  The neighbour set at elimination time is exactly the row
 * structure of that column of L.  Once the remaining graph is a clique its order is arbitrary. */
orc_ldlt *orc_ldlt_analyse(int64_t n, const int64_t *rowptr, const int32_t *col) {
    size_t W = (size_t)((n + 63) / 64);
    uint64_t *G = (uint64_t *)calloc((size_t)n * W, sizeof(uint64_t));
    if (!G) return NULL;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int64_t j = col[p];
            if (j == i) continue;
            G[(size_t)i * W + (size_t)(j >> 6)] |= 1ULL << (j & 63);
            G[(size_t)j * W + (size_t)(i >> 6)] |= 1ULL << (i & 63);
        }
    int64_t *deg = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    char *alive = (char *)malloc((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (size_t w = 0; w < W; ++w) c += popcount64(G[(size_t)i * W + w]);
        deg[i] = c;
        alive[i] = 1;
    }
    orc_ldlt *f = (orc_ldlt *)calloc(1, sizeof(orc_ldlt));
    f->n = n;
    f->perm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    f->iperm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    f->Lp = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    /* structures recorded as original vertex ids, converted once the order is known */
    size_t cap = (size_t)(16 * n + 16), used = 0;
    int32_t *S = (int32_t *)malloc(cap * sizeof(int32_t));
    int64_t *Sp = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    uint64_t *N = (uint64_t *)malloc(W * sizeof(uint64_t));
    int64_t t = 0;
    Sp[0] = 0;
    while (t < n) {
        int64_t remaining = n - t, v = -1;
        for (int64_t i = 0; i < n; ++i)
            if (alive[i] && (v < 0 || deg[i] < deg[v])) v = i;
        if (deg[v] == remaining - 1) {
            /* clique: eliminate the rest in index order, each column holds all later ones */
            int64_t base = t;
            for (int64_t i = 0; i < n; ++i)
                if (alive[i]) { f->perm[t++] = i; alive[i] = 0; }
            for (int64_t k = base; k < n; ++k) {
                size_t need = used + (size_t)(n - 1 - k);
                if (need > cap) { while (cap < need) cap *= 2; S = (int32_t *)realloc(S, cap * sizeof(int32_t)); }
                for (int64_t q = k + 1; q < n; ++q) S[used++] = (int32_t)f->perm[q];
                Sp[k + 1] = (int64_t)used;
            }
            break;
        }
        f->perm[t] = v;
        memcpy(N, G + (size_t)v * W, W * sizeof(uint64_t));
        size_t need = used + (size_t)deg[v];
        if (need > cap) { while (cap < need) cap *= 2; S = (int32_t *)realloc(S, cap * sizeof(int32_t)); }
        for (size_t w = 0; w < W; ++w) {
            uint64_t bits = N[w];
            while (bits) {
                int b = __builtin_ctzll(bits);
                bits &= bits - 1;
                int64_t u = (int64_t)(w * 64 + (size_t)b);
                S[used++] = (int32_t)u;
                uint64_t *Gu = G + (size_t)u * W;
                int64_t c = 0;
                for (size_t q = 0; q < W; ++q) { Gu[q] |= N[q]; }
                Gu[(size_t)(u >> 6)] &= ~(1ULL << (u & 63));
                Gu[(size_t)(v >> 6)] &= ~(1ULL << (v & 63));
                for (size_t q = 0; q < W; ++q) c += popcount64(Gu[q]);
                deg[u] = c;
            }
        }
        alive[v] = 0;
        ++t;
        Sp[t] = (int64_t)used;
    }
    free(G); free(deg); free(alive); free(N);
    for (int64_t k = 0; k < n; ++k) f->iperm[f->perm[k]] = k;
    f->Li = (int32_t *)malloc((used > 0 ? used : 1) * sizeof(int32_t));
    f->Lx = (double *)calloc(used > 0 ? used : 1, sizeof(double));
    f->D = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t k = 0; k <= n; ++k) f->Lp[k] = Sp[k];
    for (size_t q = 0; q < used; ++q) f->Li[q] = (int32_t)f->iperm[S[q]];
    for (int64_t k = 0; k < n; ++k)
        qsort(f->Li + f->Lp[k], (size_t)(f->Lp[k + 1] - f->Lp[k]), sizeof(int32_t), cmp_i32);
    free(S); free(Sp);
    return f;
}

/* Left-looking column LDL^T: column j gathers A(:, j) - sigma e_j, subtracts L(:, k) D_k L(j, k)
 * for every earlier column k with a nonzero in row j, then divides by the pivot D_j. */
int orc_ldlt_factor(orc_ldlt *f, const int64_t *rowptr, const int32_t *col, const double *val,
                    double sigma, double tiny) {
    int64_t n = f->n;
    double *w = (double *)calloc((size_t)n, sizeof(double));
    int64_t *head = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *next = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *pos = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) head[i] = -1;
    f->negative = 0;
    f->perturbed = 0;
    for (int64_t j = 0; j < n; ++j) {
        int64_t o = f->perm[j];
        for (int64_t p = rowptr[o]; p < rowptr[o + 1]; ++p) {
            int64_t r = f->iperm[col[p]];
            if (r >= j) w[r] += val[p];
        }
        w[j] -= sigma;
        int64_t k = head[j];
        while (k >= 0) {
            int64_t knext = next[k];
            int64_t p = pos[k];
            double t = f->Lx[p] * f->D[k];
            for (int64_t q = p; q < f->Lp[k + 1]; ++q) w[f->Li[q]] -= f->Lx[q] * t;
            pos[k] = p + 1;
            if (p + 1 < f->Lp[k + 1]) {
                int64_t r = f->Li[p + 1];
                next[k] = head[r];
                head[r] = k;
            }
            k = knext;
        }
        double d = w[j];
        w[j] = 0.0;
        if (fabs(d) < tiny) { d = d >= 0.0 ? tiny : -tiny; f->perturbed++; }
        if (d < 0.0) f->negative++;
        f->D[j] = d;
        for (int64_t q = f->Lp[j]; q < f->Lp[j + 1]; ++q) {
            f->Lx[q] = w[f->Li[q]] / d;
            w[f->Li[q]] = 0.0;
        }
        if (f->Lp[j] < f->Lp[j + 1]) {
            pos[j] = f->Lp[j];
            int64_t r = f->Li[f->Lp[j]];
            next[j] = head[r];
            head[r] = j;
        }
    }
    free(w); free(head); free(next); free(pos);
    return 0;
}

void orc_ldlt_solve(const orc_ldlt *f, const double *b, double *x) {
    int64_t n = f->n;
    double *y = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t k = 0; k < n; ++k) y[k] = b[f->perm[k]];
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = f->Lp[j]; q < f->Lp[j + 1]; ++q) y[f->Li[q]] -= f->Lx[q] * y[j];
    for (int64_t j = 0; j < n; ++j) y[j] /= f->D[j];
    for (int64_t j = n - 1; j >= 0; --j) {
        double s = y[j];
        for (int64_t q = f->Lp[j]; q < f->Lp[j + 1]; ++q) s -= f->Lx[q] * y[f->Li[q]];
        y[j] = s;
    }
    for (int64_t k = 0; k < n; ++k) x[f->perm[k]] = y[k];
    free(y);
}

int64_t orc_ldlt_nnz(const orc_ldlt *f) { return f->Lp[f->n]; }
int64_t orc_ldlt_negative(const orc_ldlt *f) { return f->negative; }
int64_t orc_ldlt_perturbed(const orc_ldlt *f) { return f->perturbed; }

void orc_ldlt_free(orc_ldlt *f) {
    if (!f) return;
    free(f->perm); free(f->iperm); free(f->Lp); free(f->Li); free(f->Lx); free(f->D);
    free(f);
}

/* x = (H - sigma)^-1 b with FP64 iterative refinement on the factor. */
static void si_apply(const orc_ldlt *f, int64_t n, const int64_t *rowptr, const int32_t *col,
                     const double *val, double sigma, double anorm, const double *b, double *x,
                     double *r, double *dx) {
    orc_ldlt_solve(f, b, x);
    double bn = sqrt(dot(n, b, b));
    double prev = INFINITY;
    int stall = 0;
    for (int it = 0; it < 30; ++it) {
        orc_spmv(n, rowptr, col, val, sigma, x, r);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double rn = sqrt(dot(n, r, r)), xn = sqrt(dot(n, x, x));
        if (rn <= 1e-15 * (anorm * xn + bn)) break;
        if (rn > 0.5 * prev) { if (++stall >= 2) break; } else stall = 0;
        prev = rn;
        orc_ldlt_solve(f, r, dx);
        for (int64_t i = 0; i < n; ++i) x[i] += dx[i];
    }
}

int orc_nearest_shift_invert(int64_t n, const int64_t *rowptr, const int32_t *col,
                             const double *val, double sigma, int nev, double hnorm,
                             double *evals, double *evecs, double *resid) {
    if (nev < 1 || nev > n) return -2;
    orc_ldlt *f = orc_ldlt_analyse(n, rowptr, col);
    if (!f) return -3;
    orc_ldlt_factor(f, rowptr, col, val, sigma, 1e-8 * hnorm);
    double anorm = hnorm + fabs(sigma);
    int mmax = (int)(n < 4 * (int64_t)nev + 120 ? n : 4 * nev + 120);
    size_t N = (size_t)n;
    double *V = (double *)malloc(N * (size_t)(mmax + 1) * sizeof(double));
    double *w = (double *)malloc(N * sizeof(double));
    double *r = (double *)malloc(N * sizeof(double));
    double *dx = (double *)malloc(N * sizeof(double));
    double *al = (double *)calloc((size_t)mmax + 1, sizeof(double));
    double *be = (double *)calloc((size_t)mmax + 1, sizeof(double));
    double *nu = (double *)malloc((size_t)mmax * sizeof(double));
    double *zl = (double *)malloc((size_t)mmax * sizeof(double));
    random_unit(n, 0x5EEDULL, V);
    int m = 0, converged = 0;
    for (int j = 0; j < mmax; ++j) {
        si_apply(f, n, rowptr, col, val, sigma, anorm, V + (size_t)j * N, w, r, dx);
        al[j] = reorthogonalize(n, j + 1, V, w, j);
        double b = sqrt(dot(n, w, w));
        be[j] = b;
        m = j + 1;
        double scale = 0.0;
        for (int i = 0; i <= j; ++i) scale = fmax(scale, fabs(al[i]) + be[i]);
        int breakdown = b <= 1e-14 * scale;
        if (m >= nev && (breakdown || m == mmax || (m >= nev + 10 && m % 5 == 0))) {
            /* Ritz values nu of the transformed operator: the nev largest |nu| are nearest sigma;
             * ||H y - theta y|| <= ||H - sigma|| * |b s_m| / |nu| */
            orc_stev(m, al, be, nu, zl);
            int ok = 1;
            char *taken = (char *)calloc((size_t)m, 1);
            for (int t = 0; t < nev; ++t) {
                int best = -1;
                for (int i = 0; i < m; ++i)
                    if (!taken[i] && (best < 0 || fabs(nu[i]) > fabs(nu[best]))) best = i;
                taken[best] = 1;
                double est = anorm * fabs(b * zl[best]) / fabs(nu[best]);
                if (est > 1e-13 * hnorm) ok = 0;
            }
            free(taken);
            if (ok || breakdown) { converged = 1; break; }
            if (m == mmax) break;
        }
        double *vn = V + (size_t)(j + 1) * N;
        for (int64_t i = 0; i < n; ++i) vn[i] = w[i] / b;
    }
    /* Rayleigh-Ritz on H in span(V_m): G = V^T H V, G = S diag(theta) S^T, y = V s */
    double *HV = (double *)malloc(N * (size_t)m * sizeof(double));
    for (int j = 0; j < m; ++j) orc_spmv(n, rowptr, col, val, 0.0, V + (size_t)j * N, HV + (size_t)j * N);
    double *G = (double *)malloc((size_t)m * m * sizeof(double));
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c) G[(size_t)c * m + a] = dot(n, V + (size_t)a * N, HV + (size_t)c * N);
    for (int a = 0; a < m; ++a)
        for (int c = a + 1; c < m; ++c) {
            double s = 0.5 * (G[(size_t)c * m + a] + G[(size_t)a * m + c]);
            G[(size_t)c * m + a] = s;
            G[(size_t)a * m + c] = s;
        }
    double *th = (double *)malloc((size_t)m * sizeof(double));
    int rc = orc_syev(m, G, th, 1);
    /* The result is the nev eigenpairs nearest sigma.  Plain Rayleigh-Ritz on H can also give
     * spurious interior Ritz values (mixtures of directions on both sides of sigma) whose pairs are
     * not eigenpairs, so the Ritz values are taken in order of distance to sigma (ties: the lower)
     * and a pair is kept only if its own residual ||H y - theta y|| is at most 1e-8 ||H|| (a
     * converged pair is near 1e-13 ||H||, a spurious one many orders larger). */
    int *order = (int *)malloc((size_t)m * sizeof(int));
    int *idx = (int *)malloc((size_t)nev * sizeof(int));
    double *ys = (double *)malloc(N * (size_t)nev * sizeof(double));
    double *rs = (double *)malloc((size_t)nev * sizeof(double));
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int a = 1; a < m; ++a) {
        int x = order[a], b = a - 1;
        while (b >= 0) {
            double dx_ = fabs(th[x] - sigma), db_ = fabs(th[order[b]] - sigma);
            if (db_ < dx_ || (db_ == dx_ && th[order[b]] <= th[x])) break;
            order[b + 1] = order[b];
            --b;
        }
        order[b + 1] = x;
    }
    int kept = 0;
    for (int t = 0; t < m && kept < nev; ++t) {
        const double *s = G + (size_t)order[t] * m;
        double *y = ys + (size_t)kept * N;
        for (int64_t i = 0; i < n; ++i) y[i] = 0.0;
        for (int a = 0; a < m; ++a) {
            const double *va = V + (size_t)a * N;
            for (int64_t i = 0; i < n; ++i) y[i] += s[a] * va[i];
        }
        double yn = sqrt(dot(n, y, y));
        for (int64_t i = 0; i < n; ++i) y[i] /= yn;
        orc_spmv(n, rowptr, col, val, th[order[t]], y, r);
        double res = sqrt(dot(n, r, r));
        if (res > 1e-8 * hnorm) continue;
        idx[kept] = order[t];
        rs[kept] = res;
        ++kept;
    }
    /* ascending order of the kept eigenvalues */
    for (int t = 0; t < kept; ++t) {
        int best = t;
        for (int u = t + 1; u < kept; ++u)
            if (th[idx[u]] < th[idx[best]]) best = u;
        evals[t] = th[idx[best]];
        resid[t] = rs[best];
        memcpy(evecs + (size_t)t * N, ys + (size_t)best * N, N * sizeof(double));
        if (best != t) {
            int ti = idx[t]; idx[t] = idx[best]; idx[best] = ti;
            double tr = rs[t]; rs[t] = rs[best]; rs[best] = tr;
            memcpy(ys + (size_t)best * N, ys + (size_t)t * N, N * sizeof(double));
        }
    }
    free(order); free(ys); free(rs);
    if (kept < nev) converged = 0;
    free(idx); free(th); free(G); free(HV);
    free(V); free(w); free(r); free(dx); free(al); free(be); free(nu); free(zl);
    orc_ldlt_free(f);
    if (rc != 0) return -4;
    return converged ? m : -m;
}

/* ------------------------------------------------------------------------------------------
 * Observables ("characterization" section).
 * ------------------------------------------------------------------------------------------ */
void orc_gap_ratio(int nev, const double *e, double *r, double *r_mean) {
    double s = 0.0;
    int cnt = 0;
    for (int k = 1; k + 1 < nev; ++k) {
        double d0 = e[k] - e[k - 1], d1 = e[k + 1] - e[k];
        double mx = d0 > d1 ? d0 : d1, mn = d0 > d1 ? d1 : d0;
        if (mx == 0.0) { r[k - 1] = NAN; continue; }
        r[k - 1] = mn / mx;
        s += r[k - 1];
        ++cnt;
    }
    *r_mean = cnt > 0 ? s / cnt : NAN;
}

double orc_s1p(int64_t n, const double *y) {
    double nrm = dot(n, y, y), s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double p = y[i] * y[i] / nrm;
        if (p > 0.0) s -= p * log(p);
    }
    return s;
}

double orc_entanglement(int L, const uint32_t *states, int64_t n, const double *y) {
    /* A = sites 0 .. floor(L/2) - 1; the sector's up-spin count is that of any basis state */
    int LA = L / 2, LB = L - L / 2, nup = n > 0 ? popcount32(states[0]) : 0;
    double nrm = dot(n, y, y), S = 0.0;
    uint32_t *as = (uint32_t *)malloc(sizeof(uint32_t) << LA);
    uint32_t *bs = (uint32_t *)malloc(sizeof(uint32_t) << LB);
    for (int nA = 0; nA <= LA; ++nA) {
        int nB = nup - nA;
        if (nB < 0 || nB > LB) continue;
        int da = 0, db = 0;
        for (uint32_t a = 0; a < (1u << LA); ++a) if (popcount32(a) == nA) as[da++] = a;
        for (uint32_t b = 0; b < (1u << LB); ++b) if (popcount32(b) == nB) bs[db++] = b;
        /* M[a][b] = psi(a + b 2^LA); Schmidt weights are the eigenvalues of G = M M^T */
        double *M = (double *)malloc((size_t)da * db * sizeof(double));
        for (int ia = 0; ia < da; ++ia)
            for (int ib = 0; ib < db; ++ib) {
                int64_t k = find_state(states, n, as[ia] | (bs[ib] << LA));
                M[(size_t)ia * db + ib] = y[k];
            }
        double *G = (double *)calloc((size_t)da * da, sizeof(double));
        for (int i = 0; i < da; ++i)
            for (int j = 0; j < da; ++j) {
                double s = 0.0;
                for (int b = 0; b < db; ++b) s += M[(size_t)i * db + b] * M[(size_t)j * db + b];
                G[(size_t)j * da + i] = s / nrm;
            }
        double *lam = (double *)malloc((size_t)da * sizeof(double));
        orc_syev(da, G, lam, 0);
        for (int i = 0; i < da; ++i)
            if (lam[i] > 1e-15) S -= lam[i] * log(lam[i]);
        free(M); free(G); free(lam);
    }
    free(as); free(bs);
    return S;
}

double orc_kl(int64_t n, const double *y, const double *z) {
    double ny = dot(n, y, y), nz = dot(n, z, z), s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double p = y[i] * y[i] / ny, q = z[i] * z[i] / nz;
        if (p == 0.0) continue;
        if (q == 0.0) return INFINITY;
        s += p * log(p / q);
    }
    return s;
}

double orc_sqp(int64_t n, const double *y, double q) {
    double ny = dot(n, y, y), s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double p = y[i] * y[i] / ny;
        if (p > 0.0) s += pow(p, q);
    }
    return log(s) / (1.0 - q);
}

/* S^z of the sites 0 .. floor(L/2)-1 of a basis state: (#up - #down) / 2 */
static double sz_half(int L, uint32_t s) {
    int up = 0;
    for (int i = 0; i < L / 2; ++i) up += (s >> i) & 1u;
    return 0.5 * (double)(2 * up - L / 2);
}

double orc_fluct(int L, const uint32_t *states, int64_t n, const double *y) {
    double ny = dot(n, y, y), m1 = 0.0, m2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double p = y[i] * y[i] / ny, m = sz_half(L, states[i]);
        m1 += p * m;
        m2 += p * m * m;
    }
    return m2 - m1 * m1;
}

double orc_dynf(int L, const uint32_t *states, int64_t n, const double *y) {
    const double pi = 3.14159265358979323846;
    double ny = dot(n, y, y), re = 0.0, im = 0.0, mm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double p = y[i] * y[i] / ny, mr = 0.0, mi = 0.0;
        for (int j = 0; j < L; ++j) {
            double sz = ((states[i] >> j) & 1u) ? 0.5 : -0.5;
            mr += sz * cos(2.0 * pi * j / L);
            mi += sz * sin(2.0 * pi * j / L);
        }
        re += p * mr;
        im += p * mi;
        mm += p * (mr * mr + mi * mi);
    }
    if (mm == 0.0) return NAN;
    return 1.0 - (re * re + im * im) / mm;
}
