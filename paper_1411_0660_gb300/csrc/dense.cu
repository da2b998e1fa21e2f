// dense.cu -- FP64 block kernels of the Krylov solvers and a batched small symmetric
// eigensolver.
//
// The eigensolver serves the Rayleigh-Ritz steps (projected matrices of the shift-invert
// Lanczos, numerical-method section) and the Schmidt spectra of the half-chain entanglement
// entropy (characterization section (ii)).  One CTA per matrix:
//   1. Householder reduction to tridiagonal form (matrix in shared memory up to order 160);
//   2a. eigenvalues only: every eigenvalue by bisection on Sturm counts, one thread each;
//   2b. with eigenvectors: implicit QL with Wilkinson shifts; one thread generates the rotations
//       of a sweep (the scalar chain) and every thread applies the whole sweep to its rows of Z,
//       so the O(m^3) accumulation runs in parallel without a barrier per rotation;
//   3. back-transformation by the stored reflectors, one warp per vector.
#include <cfloat>

#include <mutex>

#include "mbl_internal.h"

namespace mbl {

// ------------------------------------------------------------------------------------------
// Block kernels on row-major n x ld blocks of vectors.
// ------------------------------------------------------------------------------------------
constexpr int TN_ROWS = 16;   // rows staged per step
constexpr int TN_CHUNKS = 304; // partial-sum chunks (2 x 152 SMs)
constexpr int TN_MAXKP = 8192;  // PER (8) outputs x 1024 threads

size_t dense_tn_work(int64_t n, int k, int p) { return (size_t)TN_CHUNKS * (size_t)k * (size_t)p; }

// Partial sums of C = V^T X over row chunks, in the arithmetic of V's type (X is read as FP64).
template <class TV>
__global__ void k_tn_partial(int64_t n, const TV *__restrict__ V, int ldv, int c0, int k,
                             const double *__restrict__ X, int ldx, int x0, int p, double *__restrict__ work,
                             int64_t rows_per) {
    extern __shared__ __align__(16) unsigned char smraw_tn[];
    TV *sv = reinterpret_cast<TV *>(smraw_tn);  // TN_ROWS x k
    TV *sx = sv + TN_ROWS * k;                  // TN_ROWS x p
    int64_t r0 = (int64_t)blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    int kp = k * p;
    constexpr int PER = 8;
    TV acc[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) acc[u] = TV(0);
    for (int64_t rb = r0; rb < r1; rb += TN_ROWS) {
        int nr = (int)min((int64_t)TN_ROWS, r1 - rb);
        for (int t = threadIdx.x; t < nr * k; t += blockDim.x) {
            int r = t / k, a = t - r * k;
            sv[r * k + a] = V[(rb + r) * ldv + c0 + a];
        }
        for (int t = threadIdx.x; t < nr * p; t += blockDim.x) {
            int r = t / p, q = t - r * p;
            sx[r * p + q] = (TV)X[(rb + r) * ldx + x0 + q];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            int o = threadIdx.x + u * blockDim.x;
            if (o < kp) {
                int a = o / p, q = o - a * p;
                TV s = acc[u];
                for (int r = 0; r < nr; ++r) s = fma(sv[r * k + a], sx[r * p + q], s);
                acc[u] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        int o = threadIdx.x + u * blockDim.x;
        if (o < kp) work[(size_t)blockIdx.x * kp + o] = (double)acc[u];
    }
}

// C[o] = sum_c work[c * kp + o]: one warp per output, lanes over the chunks, a fixed summation order.
__global__ void k_tn_reduce(int nch, int kp, const double *__restrict__ work, double *__restrict__ C) {
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (o >= kp) return;
    double s = 0.0;
    for (int c = lane; c < nch; c += 32) s += work[(size_t)c * kp + o];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) C[o] = s;
}

template <class TV>
static void dense_tn_t(int64_t n, const TV *V, int ldv, int c0, int k, const double *X, int ldx, int x0, int p,
                       double *C, double *work, cudaStream_t st) {
    if (k <= 0 || p <= 0) return;
    if (k * p > TN_MAXKP) fail(MBL_ERR_INVALID, "dense_tn: block too wide");
    int threads = 1024;
    while (threads > 128 && threads * 8 / 2 >= k * p) threads /= 2;
    int64_t rows_per = (n + TN_CHUNKS - 1) / TN_CHUNKS;
    if (rows_per < 1) rows_per = 1;
    int nch = (int)((n + rows_per - 1) / rows_per);
    size_t smem = (size_t)TN_ROWS * (k + p) * sizeof(TV);
    smem_limit((const void *)k_tn_partial<TV>, 200 * 1024);
    k_tn_partial<TV><<<nch, threads, smem, st>>>(n, V, ldv, c0, k, X, ldx, x0, p, work, rows_per);
    MBL_LAUNCH_CHECK();
    k_tn_reduce<<<(unsigned)((k * p + 7) / 8), 256, 0, st>>>(nch, k * p, work, C);
    MBL_LAUNCH_CHECK();
}

void dense_tn(int64_t n, const double *V, int ldv, int c0, int k, const double *X, int ldx, int x0, int p,
              double *C, double *work, cudaStream_t st) {
    dense_tn_t(n, V, ldv, c0, k, X, ldx, x0, p, C, work, st);
}

void dense_tn32(int64_t n, const float *V, int ldv, int c0, int k, const double *X, int ldx, int x0, int p,
                double *C, double *work, cudaStream_t st) {
    dense_tn_t(n, V, ldv, c0, k, X, ldx, x0, p, C, work, st);
}

// Xout = Xin - V C (V row-major n x k at column c0, C k x p row-major; Xin may be Xout); the sum in
// V's type.
template <class TV>
__global__ void k_nn_sub(int64_t n, const TV *__restrict__ V, int ldv, int c0, int k,
                         const double *__restrict__ C, int p, const double *Xin, double *Xout) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t / p;
    int q = (int)(t - i * p);
    if (i >= n) return;
    const TV *v = V + i * ldv + c0;
    TV s = TV(0);
    for (int a = 0; a < k; ++a) s = fma(v[a], (TV)C[a * p + q], s);
    Xout[i * p + q] = Xin[i * p + q] - (double)s;
}

void dense_nn_sub(int64_t n, const double *V, int ldv, int c0, int k, const double *C, int p, double *X,
                  cudaStream_t st) {
    if (k <= 0) return;
    int64_t tot = n * p;
    k_nn_sub<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, V, ldv, c0, k, C, p, X, X);
    MBL_LAUNCH_CHECK();
}

void dense_nn_sub32(int64_t n, const float *V, int ldv, int c0, int k, const double *C, int p, const double *Xin,
                    double *Xout, cudaStream_t st) {
    if (k <= 0) return;
    int64_t tot = n * p;
    k_nn_sub<float><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, V, ldv, c0, k, C, p, Xin, Xout);
    MBL_LAUNCH_CHECK();
}

__global__ void k_nn(int64_t n, const double *__restrict__ V, int ldv, int k, const double *__restrict__ S, int m,
                     double *__restrict__ Y, int ldy, int y0) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t / m;
    int j = (int)(t - i * m);
    if (i >= n) return;
    const double *v = V + i * ldv;
    double s = 0.0;
    for (int a = 0; a < k; ++a) s = fma(v[a], S[a * m + j], s);
    Y[i * ldy + y0 + j] = s;
}

void dense_nn(int64_t n, const double *V, int ldv, int k, const double *S, int m, double *Y, int ldy, int y0,
              cudaStream_t st) {
    if (m <= 0) return;
    int64_t tot = n * m;
    k_nn<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, V, ldv, k, S, m, Y, ldy, y0);
    MBL_LAUNCH_CHECK();
}

__global__ void k_copy_cols(int64_t n, const double *src, int lds, int s0, double *dst, int ldd, int d0, int m) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t / m;
    int j = (int)(t - i * m);
    if (i >= n) return;
    dst[i * ldd + d0 + j] = src[i * lds + s0 + j];
}

void copy_cols(int64_t n, const double *src, int lds, int s0, double *dst, int ldd, int d0, int m,
               cudaStream_t st) {
    if (m <= 0) return;
    int64_t tot = n * m;
    k_copy_cols<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, src, lds, s0, dst, ldd, d0, m);
    MBL_LAUNCH_CHECK();
}

// Cholesky of the p x p Gram matrix G = R^T R (R upper, row-major); flag = 0 if not positive.
__global__ void k_chol(int p, const double *G, double *R, int *flag) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double maxd = 0.0;
    for (int j = 0; j < p; ++j) maxd = fmax(maxd, G[j * p + j]);
    for (int i = 0; i < p * p; ++i) R[i] = 0.0;
    for (int j = 0; j < p; ++j) {
        double s = G[j * p + j];
        for (int l = 0; l < j; ++l) s -= R[l * p + j] * R[l * p + j];
        if (!(s > 1e-28 * maxd) || !(maxd > 0.0)) {
            *flag = 0;
            s = fmax(maxd, 1e-300);  // keep going with a harmless value
        }
        double rjj = sqrt(s);
        R[j * p + j] = rjj;
        for (int c = j + 1; c < p; ++c) {
            double t = G[j * p + c];
            for (int l = 0; l < j; ++l) t -= R[l * p + j] * R[l * p + c];
            R[j * p + c] = t / rjj;
        }
    }
}

// x_row <- x_row R^{-1} for every row
__global__ void k_trsm_rows(int64_t n, double *X, int p, const double *R) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[32];
    for (int j = 0; j < p; ++j) x[j] = X[i * p + j];
    for (int j = 0; j < p; ++j) {
        double s = x[j];
        for (int l = 0; l < j; ++l) s -= x[l] * R[l * p + j];
        x[j] = s / R[j * p + j];
    }
    for (int j = 0; j < p; ++j) X[i * p + j] = x[j];
}

void chol_qr(int64_t n, double *X, int p, double *R, double *G, double *work, int *d_flag, cudaStream_t st) {
    dense_tn(n, X, p, 0, p, X, p, 0, p, G, work, st);
    k_chol<<<1, 32, 0, st>>>(p, G, R, d_flag);
    MBL_LAUNCH_CHECK();
    k_trsm_rows<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, X, p, R);
    MBL_LAUNCH_CHECK();
}

// ------------------------------------------------------------------------------------------
// Batched small symmetric eigensolver.
// ------------------------------------------------------------------------------------------
constexpr int EIG_THREADS = 512;
constexpr int EIG_QL_MAX = 512;  // tridiagonal order kept in shared memory during the QL sweeps
constexpr size_t EIG_SMEM_BYTES = 204800;  // dynamic shared memory of the batched eigensolver

size_t syev_work_doubles(int mmax, bool vecs) {
    // d, e, beta, v, p, e^2 (8m with slack) [+ Z (m*m) + sort scratch (m*m) with eigenvectors]
    size_t m = (size_t)mmax;
    return 8 * m + (vecs ? 2 * m * m : 0) + 64;
}

template <class R>
struct Num;
template <>
struct Num<double> {
    static __device__ __forceinline__ double eps() { return DBL_EPSILON; }
    static __device__ __forceinline__ double tiny() { return DBL_MIN; }
};
template <>
struct Num<float> {
    static __device__ __forceinline__ float eps() { return FLT_EPSILON; }
    static __device__ __forceinline__ float tiny() { return FLT_MIN; }
};

template <class R>
__device__ R block_sum(R v, R *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    R s = R(0);
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
    __syncthreads();
    return s;
}

// Sturm count: number of eigenvalues of T(d, e2) below x.
template <class R>
__device__ int sturm_count(int m, const R *d, const R *e2, R x, R pivmin) {
    int c = 0;
    R q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < R(0);
    for (int i = 1; i < m; ++i) {
        q = (d[i] - x) - e2[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        c += q < R(0);
    }
    return c;
}

// One implicit QL sweep on the unreduced block lo..hi of (d, e), recording the rotations:
// T <- J^T T J with J = [[c, s], [-s, c]] in planes (hi-1, hi), ..., (lo, lo+1); the first rotation
// zeroes the upper entry of the last column of T - mu I, the others chase the bulge upward.
//
// The sweep is one dependent chain, so the entries it carries from one rotation to the next (the
// updated d[k + 1] and e[k], and the chased pair x, z) stay in registers: each rotation loads only the
// entries it meets for the first time, d[k] and e[k - 1], one rotation ahead, and stores each final
// value once.  The arithmetic, and so every result, is the same as with d and e updated in place.
template <class R>
__device__ void ql_sweep_record(int lo, int hi, R *d, R *e, R *cs, R *sn) {
    R delta = R(0.5) * (d[lo + 1] - d[lo]);
    R b = e[lo];
    R mu = d[lo] - b * b / (delta + copysign(hypot(delta, b), delta));
    R dk1 = d[hi];      // d[k + 1] as the sweep has left it
    R ek = e[hi - 1];   // e[k] as the sweep has left it
    R x = dk1 - mu, z = ek;
    R a = d[hi - 1];                          // d[k], not touched yet
    R em = hi - 1 > lo ? e[hi - 2] : R(0);    // e[k - 1], not touched yet
    for (int k = hi - 1; k >= lo; --k) {
        // the entries the next rotation meets first
        const R a_next = k > lo ? d[k - 1] : R(0);
        const R em_next = k - 1 > lo ? e[k - 2] : R(0);
        R r = hypot(x, z);
        R c = R(1), s = R(0);
        if (r != R(0)) {
            R ir = R(1) / r;
            c = x * ir;
            s = z * ir;
        }
        if (k < hi - 1) e[k + 1] = r;
        const R bb = ek, dd = dk1;
        const R dk = a * c * c - R(2) * bb * c * s + dd * s * s;
        d[k + 1] = a * s * s + R(2) * bb * c * s + dd * c * c;
        const R ekn = (a - dd) * c * s + bb * (c * c - s * s);
        if (k > lo) {
            const R bulge = s * em;
            ek = c * em;  // e[k - 1] after this rotation: the next rotation's e[k]
            x = ekn;
            z = bulge;
            e[k] = ekn;   // final unless the next rotation overwrites it with its r
        } else {
            e[k] = ekn;
        }
        dk1 = dk;  // the next rotation's d[k + 1]
        a = a_next;
        em = em_next;
        cs[k] = c;
        sn[k] = s;
    }
    d[lo] = dk1;
}

// Householder reduction of the symmetric m x m matrix a (column-major, lower triangle used, leading
// dimension lda) to tridiagonal form, by the whole block: afterwards the diagonal and subdiagonal are
// on a's diagonals, the reflectors' tails below the subdiagonal and their scalings in beta.
template <class R>
__device__ void householder_tridiag(R *a, int lda, int m, R *beta, R *vv, R *pp, R *red) {
    for (int k = 0; k + 2 < m; ++k) {
        int len = m - k - 1;
        R *x = a + (size_t)k * lda + (k + 1);
        R loc = R(0);
        for (int i = threadIdx.x; i < len; i += blockDim.x) loc += x[i] * x[i];
        R alpha2 = block_sum(loc, red);
        if (alpha2 == R(0)) {
            if (threadIdx.x == 0) beta[k] = R(0);
            __syncthreads();
            continue;
        }
        R x0 = x[0];
        R sgn = x0 >= R(0) ? R(1) : R(-1);
        R alpha = sqrt(alpha2);
        R v0 = x0 + sgn * alpha;
        R iv0 = R(1) / v0;
        loc = R(0);
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            R v = (i == 0) ? R(1) : x[i] * iv0;
            vv[i] = v;
            if (i > 0) loc += v * v;
        }
        R vtv = R(1) + block_sum(loc, red);
        R bk = R(2) / vtv;
        R *A22 = a + (size_t)(k + 1) * lda + (k + 1);
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            R s = R(0);
            for (int j = 0; j < len; ++j) s = fma(A22[(size_t)j * lda + i], vv[j], s);
            pp[i] = bk * s;
        }
        __syncthreads();
        loc = R(0);
        for (int i = threadIdx.x; i < len; i += blockDim.x) loc += pp[i] * vv[i];
        R K = R(0.5) * bk * block_sum(loc, red);
        for (int i = threadIdx.x; i < len; i += blockDim.x) pp[i] -= K * vv[i];
        __syncthreads();
        for (int t = threadIdx.x; t < len * len; t += blockDim.x) {
            int i = t % len, j = t / len;
            A22[(size_t)j * lda + i] -= vv[i] * pp[j] + pp[i] * vv[j];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < len; i += blockDim.x) x[i] = (i == 0) ? -sgn * alpha : vv[i];
        if (threadIdx.x == 0) beta[k] = bk;
        __syncthreads();
    }
}

// A: m x m column-major FP64 (lda = m) at A + aoff[b]; W: eigenvalues (FP64) at W + woff[b];
// vecs: eigenvectors into A (columns ascending); info[b] = 1 if QL did not converge.  The arithmetic
// runs in R (FP32 or FP64); with R = float the matrix must fit in shared memory.
template <class R>
__global__ void __launch_bounds__(EIG_THREADS) k_syev(const int *mv, const int64_t *aoff, const int64_t *woff,
                                                      double *Aall, double *Wall, int vecs, double *workall,
                                                      size_t wstride, int *info, int smem_m, int zsm) {
    extern __shared__ __align__(16) unsigned char smraw[];
    R *sm = reinterpret_cast<R *>(smraw);
    __shared__ R red[EIG_THREADS / 32];
    __shared__ R s_gl, s_gu, s_pivmin, s_atol;
    int b = blockIdx.x;
    int m = mv[b];
    double *Ag = Aall + aoff[b];
    double *W = Wall + woff[b];
    R *work = reinterpret_cast<R *>(workall + (size_t)b * wstride);
    R *d = work, *e = work + m, *beta = work + 2 * m, *vv = work + 3 * m, *pp = work + 4 * m;
    R *e2 = work + 5 * m;
    const bool in_smem = m <= smem_m;  // the launch's dynamic shared memory holds smem_m^2 entries
    // the eigenvectors: in shared memory behind the matrix when the launch holds two of them (the
    // QL rotations update Z one dependent row element after another), else in the work array
    R *Z = (in_smem && zsm) ? sm + (size_t)smem_m * smem_m : work + 8 * m;
    if (threadIdx.x == 0 && info) info[b] = 0;
    if (m <= 0) return;
    if (m == 1) {
        if (threadIdx.x == 0) {
            W[0] = Ag[0];
            if (vecs) Ag[0] = 1.0;
        }
        return;
    }
    R *a;
    if (in_smem) {
        a = sm;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) a[t] = (R)Ag[t];
        __syncthreads();
    } else {
        a = reinterpret_cast<R *>(Ag);  // only instantiated for R = double (checked by the launcher)
    }
    int lda = m;
    // ---- 1. Householder tridiagonalization ----
    householder_tridiag(a, lda, m, beta, vv, pp, red);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        d[i] = a[(size_t)i * lda + i];
        if (i + 1 < m) {
            e[i] = a[(size_t)i * lda + i + 1];
            e2[i] = e[i] * e[i];
        }
    }
    __syncthreads();
    // ---- 2. eigenvalues only: bisection ----
    if (!vecs) {
        if (threadIdx.x == 0) {
            R gl = d[0], gu = d[0], emax2 = R(0);
            for (int i = 0; i < m; ++i) {
                R r = (i > 0 ? fabs(e[i - 1]) : R(0)) + (i + 1 < m ? fabs(e[i]) : R(0));
                gl = fmin(gl, d[i] - r);
                gu = fmax(gu, d[i] + r);
                if (i + 1 < m) emax2 = fmax(emax2, e2[i]);
            }
            R tn = fmax(fabs(gl), fabs(gu));
            gl -= R(2) * Num<R>::eps() * tn * (R)m + Num<R>::tiny();
            gu += R(2) * Num<R>::eps() * tn * (R)m + Num<R>::tiny();
            s_gl = gl;
            s_gu = gu;
            s_pivmin = Num<R>::tiny() * fmax(R(1), emax2);
            s_atol = R(2) * Num<R>::eps() * tn;
        }
        __syncthreads();
        // every eigenvalue to an absolute accuracy of 2 eps ||T|| (LAPACK's choice of ABSTOL for
        // eigenvalues to full accuracy relative to the norm): an eigenvalue near zero -- most of an
        // entanglement spectrum -- is not bisected on to its own relative precision
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            R lo = s_gl, hi = s_gu;
            for (int it = 0; it < 200; ++it) {
                R mid = R(0.5) * (lo + hi);
                if (hi - lo <= R(2) * Num<R>::eps() * fmax(fabs(lo), fabs(hi)) + R(4) * s_pivmin || hi - lo <= s_atol ||
                    mid == lo || mid == hi)
                    break;
                if (sturm_count(m, d, e2, mid, s_pivmin) > j) hi = mid; else lo = mid;
            }
            W[j] = (double)(R(0.5) * (lo + hi));
        }
        return;
    }
    // ---- 3. implicit QL on (d, e) accumulating Z (column-major m x m, starts as identity) ----
    // the sweeps run on one thread as a chain of dependent updates of d, e and the rotation list:
    // keep those in shared memory (global memory would put an L2 round trip in every link)
    __shared__ R q_d[EIG_QL_MAX], q_e[EIG_QL_MAX], q_cs[EIG_QL_MAX], q_sn[EIG_QL_MAX];
    R *cs = pp, *sn = vv;  // reuse the Householder scratch for the sweep's rotations
    {
        if (m <= EIG_QL_MAX) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                q_d[i] = d[i];
                q_e[i] = e[i];
            }
            d = q_d;
            e = q_e;
            cs = q_cs;
            sn = q_sn;
        }
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) Z[t] = ((t / m) == (t % m)) ? R(1) : R(0);
        __shared__ int s_lo, s_hi, s_done, s_fail;
        if (threadIdx.x == 0) { s_lo = 0; s_done = 0; s_fail = 0; }
        __syncthreads();
        int iter = 0;
        while (true) {
            if (threadIdx.x == 0) {
                int lo = s_lo;
                s_hi = -1;
                while (lo < m - 1) {
                    if (fabs(e[lo]) <= Num<R>::eps() * (fabs(d[lo]) + fabs(d[lo + 1]))) {
                        e[lo] = R(0);
                        ++lo;
                        iter = 0;
                        continue;
                    }
                    int hi = lo + 1;
                    while (hi < m - 1 && !(fabs(e[hi]) <= Num<R>::eps() * (fabs(d[hi]) + fabs(d[hi + 1])))) ++hi;
                    if (hi < m - 1) e[hi] = R(0);
                    if (++iter > 100) { s_fail = 1; lo = m; break; }
                    ql_sweep_record(lo, hi, d, e, cs, sn);
                    s_hi = hi;
                    break;
                }
                s_lo = lo;
                if (lo >= m - 1) s_done = 1;
            }
            __syncthreads();
            // every thread takes the exit decision here, between the barriers: thread 0 rewrites
            // s_done (and s_lo, s_hi) as soon as it has passed the barrier below, so a thread
            // reading s_done after that barrier could see the next sweep's value, leave the loop
            // one sweep early and reach the barriers after the loop out of step with the block
            const bool done = s_done != 0;
            if (s_hi >= 0) {
                int lo = s_lo, hi = s_hi;
                // Z is column-major (column k contiguous): thread r walks its row down the sweep,
                // carrying the rotated entry of column k + 1; accesses coalesce across threads
                // (the next rotation's inputs are loaded before this one's store, which the compiler
                // could not otherwise move ahead of it: Z and the rotation list might alias)
                for (int r = threadIdx.x; r < m; r += blockDim.x) {
                    R a1 = Z[(size_t)hi * m + r];
                    R a0 = Z[(size_t)(hi - 1) * m + r];
                    R c = cs[hi - 1], sv = sn[hi - 1];
                    for (int k = hi - 1; k >= lo; --k) {
                        const bool more = k > lo;
                        const R a0n = more ? Z[(size_t)(k - 1) * m + r] : R(0);
                        const R cn = more ? cs[k - 1] : R(0), svn = more ? sn[k - 1] : R(0);
                        Z[(size_t)(k + 1) * m + r] = sv * a0 + c * a1;
                        a1 = c * a0 - sv * a1;
                        a0 = a0n;
                        c = cn;
                        sv = svn;
                    }
                    Z[(size_t)lo * m + r] = a1;
                }
            }
            __syncthreads();
            if (done) break;
        }
        if (threadIdx.x == 0) {
            // selection sort of the eigenvalues; the permutation is kept in cs
            for (int i = 0; i < m; ++i) cs[i] = (R)i;
            for (int i = 0; i < m - 1; ++i) {
                int mi = i;
                for (int j = i + 1; j < m; ++j) if (d[j] < d[mi]) mi = j;
                R t = d[i]; d[i] = d[mi]; d[mi] = t;
                t = cs[i]; cs[i] = cs[mi]; cs[mi] = t;
            }
            if (info) info[b] = s_fail;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += blockDim.x) W[j] = (double)d[j];
        // the columns of Z are put in ascending order at the write-out (the back-transformation acts
        // on each column alone)
    }
    // ---- 4. back-transformation y = H_0 ... H_{m-3} z, one warp per vector ----
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < m; c += nw) {
        R *z = Z + (size_t)c * m;
        for (int k = m - 3; k >= 0; --k) {
            R bk = beta[k];
            if (bk == R(0)) continue;
            const R *vk = a + (size_t)k * lda + (k + 1);
            int len = m - k - 1;
            R s = R(0);
            for (int i = lane; i < len; i += 32) s += (i == 0 ? R(1) : vk[i]) * z[k + 1 + i];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            s *= bk;
            for (int i = lane; i < len; i += 32) z[k + 1 + i] -= s * (i == 0 ? R(1) : vk[i]);
            __syncwarp();
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        const int c = t / m, r = t - c * m;
        Ag[t] = (double)Z[(size_t)(int)cs[c] * m + r];
    }
}

// ------------------------------------------------------------------------------------------
// FP64 eigen-decomposition by bisection and inverse iteration (the classical method of Wilkinson,
// as in LAPACK's dstebz / dstein): Householder tridiagonalization (one CTA), every eigenvalue by
// bisection on Sturm counts (a thread each, several CTAs), every eigenvector by inverse iteration
// with a pivoted tridiagonal LU (a thread each), vectors of clustered eigenvalues re-orthogonalized
// by two classical Gram-Schmidt passes, then the back-transformation (a warp per vector).  All the
// FP64 work is spread over lanes, unlike the QL sweeps, whose rotations form one sequential chain.
// ------------------------------------------------------------------------------------------
size_t syev_bisect_work(int m) { return 8 * (size_t)m + 4 * (size_t)m * m + 64; }

// The arithmetic runs in R (FP64, or FP32 as the start of a refined decomposition); A, W and the
// output vectors are FP64 either way.  work (R): d[m], e[m], e2[m], beta[m], vv[m], pp[m], Z[m x m],
// U[3 m x m].
template <class R>
__global__ void __launch_bounds__(EIG_THREADS) k_bi_tridiag(int m, double *A, R *work) {
    extern __shared__ __align__(16) unsigned char smraw[];
    R *a = reinterpret_cast<R *>(smraw);
    __shared__ R red[EIG_THREADS / 32];
    R *d = work, *e = work + m, *e2 = work + 2 * m, *beta = work + 3 * m, *vv = work + 4 * m, *pp = work + 5 * m;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) a[t] = (R)A[t];
    __syncthreads();
    householder_tridiag<R>(a, m, m, beta, vv, pp, red);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        d[i] = a[(size_t)i * m + i];
        const R ev = i + 1 < m ? a[(size_t)i * m + i + 1] : R(0);
        e[i] = ev;
        e2[i] = ev * ev;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) A[t] = (double)a[t];  // the reflectors
}

// Eigenvalue j (ascending) by bisection to the resolution of R on the Gershgorin interval.
template <class R>
__global__ void k_bi_values(int m, const R *work, double *W) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const R *d = work, *e = work + m, *e2 = work + 2 * m;
    R gl = d[0], gu = d[0], emax2 = R(0);
    for (int i = 0; i < m; ++i) {
        const R r = (i > 0 ? fabs(e[i - 1]) : R(0)) + (i + 1 < m ? fabs(e[i]) : R(0));
        gl = fmin(gl, d[i] - r);
        gu = fmax(gu, d[i] + r);
        if (i + 1 < m) emax2 = fmax(emax2, e2[i]);
    }
    const R tn = fmax(fabs(gl), fabs(gu)), eps = Num<R>::eps(), tiny = Num<R>::tiny();
    gl -= R(2) * eps * tn * (R)m + tiny;
    gu += R(2) * eps * tn * (R)m + tiny;
    const R pivmin = tiny * fmax(R(1), emax2), atol = R(2) * eps * tn;  // absolute accuracy 2 eps ||T||
    R lo = gl, hi = gu;
    for (int it = 0; it < 200; ++it) {
        const R mid = R(0.5) * (lo + hi);
        if (hi - lo <= R(2) * eps * fmax(fabs(lo), fabs(hi)) + R(4) * pivmin || hi - lo <= atol || mid == lo ||
            mid == hi)
            break;
        if (sturm_count<R>(m, d, e2, mid, pivmin) > j) hi = mid; else lo = mid;
    }
    W[j] = (double)(R(0.5) * (lo + hi));
}

// One solve of (T - lambda I) y = x in place (x -> y), Gaussian elimination with partial pivoting:
// U keeps the pivot rows (diagonal, first and second superdiagonal; a pivot below `tiny` becomes
// +-tiny), the eliminations are applied to x as they happen, then back substitution.
template <class R>
__device__ void tridiag_solve_pivoted(int m, const R *d, const R *e, R lambda, R tiny, R *U0, R *U1, R *U2, R *x) {
    R p0 = d[0] - lambda, p1 = m > 1 ? e[0] : R(0), p2 = R(0), xp = x[0];
    for (int i = 0; i + 1 < m; ++i) {
        const R s = e[i], q0 = d[i + 1] - lambda, q1 = i + 2 < m ? e[i + 1] : R(0), xq = x[i + 1];
        R u0, u1, u2, o0, o1, o2, xu, xo;
        if (fabs(p0) >= fabs(s)) {
            u0 = p0; u1 = p1; u2 = p2; xu = xp;
            o0 = s; o1 = q0; o2 = q1; xo = xq;
        } else {
            u0 = s; u1 = q0; u2 = q1; xu = xq;
            o0 = p0; o1 = p1; o2 = p2; xo = xp;
        }
        if (fabs(u0) < tiny) u0 = u0 >= R(0) ? tiny : -tiny;
        const R l = o0 / u0;
        U0[i] = u0;
        U1[i] = u1;
        U2[i] = u2;
        x[i] = xu;
        p0 = o1 - l * u1;
        p1 = o2 - l * u2;
        p2 = R(0);
        xp = xo - l * xu;
    }
    if (fabs(p0) < tiny) p0 = p0 >= R(0) ? tiny : -tiny;
    U0[m - 1] = p0;
    x[m - 1] = xp / p0;
    if (m > 1) x[m - 2] = (x[m - 2] - U1[m - 2] * x[m - 1]) / U0[m - 2];
    for (int i = m - 3; i >= 0; --i) x[i] = (x[i] - U1[i] * x[i + 1] - U2[i] * x[i + 2]) / U0[i];
}

// Eigenvectors of T: thread j iterates on column j of Z (three steps from a fixed pseudo-random
// start, normalized each time); between steps the vectors of each cluster (consecutive eigenvalues
// closer than 1e-3 ||T||) are re-orthogonalized by the block, two classical Gram-Schmidt passes each.
template <class R>
__global__ void __launch_bounds__(EIG_THREADS) k_bi_vectors(int m, const double *W, R *work) {
    __shared__ R red[EIG_THREADS / 32];
    __shared__ R s_h[EIG_SMEM_MAX_M];
    const R *d = work, *e = work + m;
    R *Z = work + 8 * m, *U = Z + (size_t)m * m;
    R tn = R(0);
    for (int i = 0; i < m; ++i) tn = fmax(tn, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : R(0)) + (i + 1 < m ? fabs(e[i]) : R(0)));
    const R tiny = Num<R>::eps() * fmax(tn, Num<R>::tiny());
    const double ortol = 1e-3 * (double)tn;
    const int j = threadIdx.x;
    R *z = Z + (size_t)j * m;
    if (j < m) {
        uint64_t h = 0x9E3779B97F4A7C15ull * (uint64_t)(j + 1);
        for (int i = 0; i < m; ++i) {
            h ^= h >> 33;
            h *= 0xff51afd7ed558ccdull;
            h ^= h >> 33;
            z[i] = (R)((double)(h >> 11) * 0x1.0p-53 - 0.5);
        }
    }
    for (int step = 0; step < 3; ++step) {
        if (j < m) {
            tridiag_solve_pivoted<R>(m, d, e, (R)W[j], tiny, U + (size_t)j * 3 * m, U + (size_t)j * 3 * m + m,
                                     U + (size_t)j * 3 * m + 2 * m, z);
            R nr = R(0);
            for (int i = 0; i < m; ++i) nr += z[i] * z[i];
            nr = R(1) / sqrt(nr);
            for (int i = 0; i < m; ++i) z[i] *= nr;
        }
        __syncthreads();
        if (step == 0) continue;
        // clusters: Gram-Schmidt of each vector against the earlier ones of its cluster (in order)
        for (int c = 1; c < m; ++c) {
            int c0 = c;
            while (c0 > 0 && W[c0] - W[c0 - 1] <= ortol) --c0;
            if (c0 == c) continue;
            R *zc = Z + (size_t)c * m;
            for (int pass = 0; pass < 2; ++pass) {
                for (int k = c0 + (int)threadIdx.x; k < c; k += blockDim.x) {
                    const R *zk = Z + (size_t)k * m;
                    R sdot = R(0);
                    for (int i = 0; i < m; ++i) sdot += zk[i] * zc[i];
                    s_h[k - c0] = sdot;
                }
                __syncthreads();
                for (int i = threadIdx.x; i < m; i += blockDim.x) {
                    R v = zc[i];
                    for (int k = c0; k < c; ++k) v -= s_h[k - c0] * Z[(size_t)k * m + i];
                    zc[i] = v;
                }
                __syncthreads();
            }
            R loc = R(0);
            for (int i = threadIdx.x; i < m; i += blockDim.x) loc += zc[i] * zc[i];
            const R nr = R(1) / sqrt(block_sum(loc, red));
            for (int i = threadIdx.x; i < m; i += blockDim.x) zc[i] *= nr;
            __syncthreads();
        }
    }
}

// z <- H_0 ... H_{m-3} z for the eigenvectors (a warp per vector), reflectors in A and beta; the
// result, in FP64, to X (column-major m x m).
template <class R>
__global__ void k_bi_back(int m, const double *A, R *work, double *X) {
    const R *beta = work + 3 * m;
    R *Z = work + 8 * m;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= m) return;
    R *z = Z + (size_t)c * m;
    for (int k = m - 3; k >= 0; --k) {
        const R bk = beta[k];
        if (bk == R(0)) continue;
        const double *vk = A + (size_t)k * m + (k + 1);
        const int len = m - k - 1;
        R sdot = R(0);
        for (int i = lane; i < len; i += 32) sdot += (i == 0 ? R(1) : (R)vk[i]) * z[k + 1 + i];
        for (int o = 16; o > 0; o >>= 1) sdot += __shfl_xor_sync(0xffffffffu, sdot, o);
        sdot *= bk;
        for (int i = lane; i < len; i += 32) z[k + 1 + i] -= sdot * (i == 0 ? R(1) : (R)vk[i]);
        __syncwarp();
    }
    for (int i = lane; i < m; i += 32) X[(size_t)c * m + i] = (double)z[i];
}

// ------------------------------------------------------------------------------------------
// FP32 eigen-decomposition by the cyclic Jacobi method (Jacobi 1846; the parallel round-robin ordering
// of Brent and Luk, 1985): every round rotates m/2 disjoint index pairs (p, q) at once, each rotation
// chosen to annihilate a_pq; the two-sided update A <- J^T A J is done as the column rotations of all
// pairs, then their row rotations, and V <- V J accumulates the eigenvectors.  m - 1 rounds (m even,
// a dummy index added for odd m) visit every pair once: a sweep.  Sweeps repeat until the
// off-diagonal mass is below FP32 rounding of the diagonal, at most JAC_SWEEPS.  One CTA per matrix,
// A and V in shared memory (leading dimension m | 1, so that the row passes are free of bank
// conflicts).  Unlike the QL sweeps, whose rotations form one chain on one thread, every step is
// spread over the CTA.  A result that did not converge sets info[b] = 1.
// ------------------------------------------------------------------------------------------
constexpr int JAC_SWEEPS = 24;

__global__ void __launch_bounds__(EIG_THREADS) k_syev_jacobi(const int *mv, const int64_t *aoff, const int64_t *woff,
                                                             double *Aall, double *Wall, int *info) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ float s_c[EIG_SMEM_MAX_M / 2 + 1], s_s[EIG_SMEM_MAX_M / 2 + 1];
    __shared__ int s_p[EIG_SMEM_MAX_M / 2 + 1], s_q[EIG_SMEM_MAX_M / 2 + 1];
    __shared__ float red[EIG_THREADS / 32][2];
    __shared__ int s_done;
    const int b = blockIdx.x, m = mv[b], tid = threadIdx.x, nt = blockDim.x;
    double *Ag = Aall + aoff[b];
    double *W = Wall + woff[b];
    if (tid == 0) info[b] = 0;
    if (m <= 0) return;
    const int ld = m | 1, M = (m + 1) & ~1, np = M / 2;
    float *A = reinterpret_cast<float *>(smraw);  // A[c * ld + r]
    float *V = A + (size_t)ld * m;                // V[c * ld + r]
    for (int e = tid; e < m * m; e += nt) {
        const int c = e / m, r = e - c * m;
        A[c * ld + r] = (float)Ag[(size_t)c * m + r];
        V[c * ld + r] = r == c ? 1.f : 0.f;
    }
    if (tid == 0) s_done = 0;
    __syncthreads();
    int sweep = 0;
    float prev_off = 3.0e38f;  // (thread 0) the off-diagonal mass after the previous sweep
    for (; sweep < JAC_SWEEPS; ++sweep) {
        // convergence: the off-diagonal mass at FP32 rounding of the diagonal's (m ulp-sized entries
        // per row), or a sweep that no longer halves it (rounding has been reached)
        float off = 0.f, dia = 0.f;
        for (int e = tid; e < m * m; e += nt) {
            const int c = e / m, r = e - c * m;
            const float v = A[c * ld + r];
            if (r == c) dia += v * v;
            else off += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if ((tid & 31) == 0) {
            red[tid >> 5][0] = off;
            red[tid >> 5][1] = dia;
        }
        __syncthreads();
        if (tid == 0) {
            float o2 = 0.f, d2 = 0.f;
            for (int w = 0; w < nt / 32; ++w) {
                o2 += red[w][0];
                d2 += red[w][1];
            }
            s_done = o2 <= (float)m * 1e-13f * d2 || (sweep >= 3 && o2 > 0.5f * prev_off);
            prev_off = o2;
        }
        __syncthreads();
        if (s_done) break;
        for (int round = 0; round < M - 1; ++round) {
            // pair i: the players at positions i and M - 1 - i (player 0 fixed, the others rotate)
            for (int i = tid; i < np; i += nt) {
                const int ia = i, ib = M - 1 - i;
                const int p = ia == 0 ? 0 : ((ia - 1 + round) % (M - 1)) + 1;
                const int q = ((ib - 1 + round) % (M - 1)) + 1;
                float c = 1.f, sn = 0.f;
                if (p < m && q < m) {
                    const float apq = A[q * ld + p];
                    if (apq != 0.f) {
                        const float app = A[p * ld + p], aqq = A[q * ld + q];
                        const float th = (aqq - app) / (2.f * apq);
                        const float t = copysignf(1.f, th) / (fabsf(th) + sqrtf(th * th + 1.f));
                        c = 1.f / sqrtf(t * t + 1.f);
                        sn = t * c;
                    }
                }
                s_c[i] = c;
                s_s[i] = sn;
                s_p[i] = p;
                s_q[i] = q;
            }
            __syncthreads();
            // columns p, q of A and V: (x_p, x_q) <- (c x_p - s x_q, s x_p + c x_q); a warp per pair,
            // its lanes over the rows
            const int lane = tid & 31, nw = nt >> 5;
            for (int i = tid >> 5; i < np; i += nw) {
                const int p = s_p[i], q = s_q[i];
                if (p >= m || q >= m) continue;
                const float c = s_c[i], sn = s_s[i];
                float *Ap = A + p * ld, *Aq = A + q * ld, *Vp = V + p * ld, *Vq = V + q * ld;
                for (int r = lane; r < m; r += 32) {
                    const float ap = Ap[r], aq = Aq[r];
                    Ap[r] = c * ap - sn * aq;
                    Aq[r] = sn * ap + c * aq;
                    const float vp = Vp[r], vq = Vq[r];
                    Vp[r] = c * vp - sn * vq;
                    Vq[r] = sn * vp + c * vq;
                }
            }
            __syncthreads();
            // rows p, q of A: a warp per pair, its lanes over the columns
            for (int i = tid >> 5; i < np; i += nw) {
                const int p = s_p[i], q = s_q[i];
                if (p >= m || q >= m) continue;
                const float c = s_c[i], sn = s_s[i];
                for (int col = lane; col < m; col += 32) {
                    const float ap = A[col * ld + p], aq = A[col * ld + q];
                    A[col * ld + p] = c * ap - sn * aq;
                    A[col * ld + q] = sn * ap + c * aq;
                }
            }
            __syncthreads();
        }
    }
    if (tid == 0 && !s_done) info[b] = 1;
    // ascending eigenvalues: the rank of each diagonal entry (ties by index), then the vectors to
    // their ranks' columns
    for (int j = tid; j < m; j += nt) {
        const float dj = A[j * ld + j];
        int rank = 0;
        for (int k = 0; k < m; ++k) {
            const float dk = A[k * ld + k];
            rank += (dk < dj || (dk == dj && k < j)) ? 1 : 0;
        }
        W[rank] = (double)dj;
        for (int r = 0; r < m; ++r) Ag[(size_t)rank * m + r] = (double)V[j * ld + r];
    }
}

template <class R>
static void syev_bisect_t(int m, double *d_A, double *d_w, double *d_work, cudaStream_t st) {
    if (m < 1 || m > EIG_SMEM_MAX_M) fail(MBL_ERR_INVALID, "bisection eigensolver: order must be in [1, 160]");
    smem_limit((const void *)k_bi_tridiag<R>, EIG_SMEM_MAX_M * EIG_SMEM_MAX_M * sizeof(R));
    R *work = reinterpret_cast<R *>(d_work);
    // the eigenvectors overwrite A only after the back-transformation has read its reflectors:
    // they go to the U scratch first (3 m^2 entries of R hold m^2 doubles; start rounded up to 16 bytes)
    const size_t xoff = ((8 * (size_t)m + (size_t)m * m) * sizeof(R) + 15) & ~(size_t)15;
    double *X = reinterpret_cast<double *>(reinterpret_cast<char *>(d_work) + xoff);
    k_bi_tridiag<R><<<1, EIG_THREADS, (size_t)m * m * sizeof(R), st>>>(m, d_A, work);
    MBL_LAUNCH_CHECK();
    k_bi_values<R><<<(m + 31) / 32, 32, 0, st>>>(m, work, d_w);
    MBL_LAUNCH_CHECK();
    k_bi_vectors<R><<<1, ((m + 31) / 32) * 32, 0, st>>>(m, d_w, work);
    MBL_LAUNCH_CHECK();
    k_bi_back<R><<<(m + 7) / 8, 256, 0, st>>>(m, d_A, work, X);
    MBL_LAUNCH_CHECK();
    MBL_CUDA(cudaMemcpyAsync(d_A, X, (size_t)m * m * sizeof(double), cudaMemcpyDeviceToDevice, st));
}

void syev_bisect(int m, double *d_A, double *d_w, double *d_work, cudaStream_t st) {
    syev_bisect_t<double>(m, d_A, d_w, d_work, st);
}

void syev_bisect32(int m, double *d_A, double *d_w, double *d_work, cudaStream_t st) {
    syev_bisect_t<float>(m, d_A, d_w, d_work, st);
}

namespace {
// Shared-memory attributes of the batched eigensolver, set once per device (function attributes
// are per device).  Setting them also loads both kernels, which otherwise load lazily on first
// launch and take device memory then.
std::mutex g_syev_mu;
bool g_syev_ready[64] = {};

cudaError_t syev_prepare_current_device() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_syev_mu);
    if (dev >= 0 && dev < 64 && g_syev_ready[dev]) return cudaSuccess;
    cudaFuncAttributes fa;
    e = cudaFuncSetAttribute(k_syev<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_syev<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_syev_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * (EIG_SMEM_MAX_M | 1) * EIG_SMEM_MAX_M * sizeof(float)));
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_syev<double>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_syev<float>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_syev_jacobi);
    if (e == cudaSuccess && dev >= 0 && dev < 64) g_syev_ready[dev] = true;
    return e;
}
}  // namespace

cudaError_t syev_preload() { return syev_prepare_current_device(); }

void syev_batched(int batch, const int *d_m, const int64_t *d_aoff, const int64_t *d_woff, double *d_A,
                  double *d_w, int vecs, const int *d_sel, int mmax, double *d_work, int *d_info, cudaStream_t st,
                  bool fp32) {
    (void)d_sel;
    if (batch <= 0) return;
    MBL_CUDA(syev_prepare_current_device());
    // the matrix in shared memory up to order 160; the eigenvectors beside it when both fit
    const size_t mm = (size_t)mmax * mmax;
    if (fp32) {
        if (mmax > EIG_SMEM_MAX_M) fail(MBL_ERR_INVALID, "FP32 small eigensolver limited to order 160");
        const int zsm = vecs && 2 * mm * sizeof(float) <= EIG_SMEM_BYTES;
        k_syev<float><<<batch, EIG_THREADS, (zsm ? 2 : 1) * mm * sizeof(float), st>>>(
            d_m, d_aoff, d_woff, d_A, d_w, vecs, d_work, syev_work_doubles(mmax, vecs != 0), d_info, mmax, zsm);
    } else {
        const bool sm = mmax <= EIG_SMEM_MAX_M;
        const int zsm = sm && vecs && 2 * mm * sizeof(double) <= EIG_SMEM_BYTES;
        const size_t smem = sm ? (zsm ? 2 : 1) * mm * sizeof(double) : 0;
        k_syev<double><<<batch, EIG_THREADS, smem, st>>>(d_m, d_aoff, d_woff, d_A, d_w, vecs, d_work,
                                                         syev_work_doubles(mmax, vecs != 0), d_info,
                                                         sm ? mmax : 0, zsm);
    }
    MBL_LAUNCH_CHECK();
}

void syev_jacobi32(int batch, const int *d_m, const int64_t *d_aoff, const int64_t *d_woff, double *d_A, double *d_w,
                   int mmax, int *d_info, cudaStream_t st) {
    if (batch <= 0) return;
    if (mmax > EIG_SMEM_MAX_M) fail(MBL_ERR_INVALID, "Jacobi eigensolver limited to order 160");
    MBL_CUDA(syev_prepare_current_device());
    k_syev_jacobi<<<batch, EIG_THREADS, (size_t)2 * (mmax | 1) * mmax * sizeof(float), st>>>(d_m, d_aoff, d_woff, d_A,
                                                                                             d_w, d_info);
    MBL_LAUNCH_CHECK();
}

// C (M x N, column-major ldc) = alpha op(A) op(B) + beta C, op = transpose if the flag is set;
// small FP64 matrices, one thread per output.
__global__ void k_gemm_small(int ta, int tb, int M, int N, int K, double alpha, const double *A, int lda,
                             const double *B, int ldb, double beta, double *C, int ldc) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M * N) return;
    int i = t % M, j = t / M;
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        double a = ta ? A[(size_t)i * lda + k] : A[(size_t)k * lda + i];
        double b = tb ? B[(size_t)k * ldb + j] : B[(size_t)j * ldb + k];
        s = fma(a, b, s);
    }
    C[(size_t)j * ldc + i] = alpha * s + (beta == 0.0 ? 0.0 : beta * C[(size_t)j * ldc + i]);
}

void gemm_small(bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda, const double *B,
                int ldb, double beta, double *C, int ldc, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    k_gemm_small<<<(M * N + 127) / 128, 128, 0, st>>>(ta ? 1 : 0, tb ? 1 : 0, M, N, K, alpha, A, lda, B, ldb, beta, C,
                                                      ldc);
    MBL_LAUNCH_CHECK();
}

}  // namespace mbl
