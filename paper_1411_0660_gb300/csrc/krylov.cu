// krylov.cu -- block Krylov-Schur (symmetric block Lanczos with full reorthogonalization and
// thick restarts), the refined shift-invert operator, extremal bounds and Rayleigh-Ritz on H.
//
// Numerical-method section of arXiv:1411.0660: E_0 and E_max of each sample, then a Krylov
// method on the shift-invert transformation (H - E)^-1 for the eigenpairs nearest the target.
// Here: Krylov-Schur (Stewart 2001) in block form.  The basis V is an n x (ncv + p) row-major FP64
// block on the device; the projected matrix T (= V^T Op V) is kept on the device; every new block
// is orthogonalized twice against the whole basis (classical Gram-Schmidt, FP64) and normalized by
// Cholesky-QR twice.  At a restart the wanted Ritz vectors of T are kept (thick restart) together
// with the residual block.  The operator is either H (extremal energies) or (H - sigma)^-1 applied
// through the LDL^T factor with FP64 iterative refinement against the CSR.  The wanted eigenpairs
// of H are finally extracted by Rayleigh-Ritz of H on the whole basis.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <numeric>

#include <cfloat>

#include "krylov.h"

namespace mbl {

// ------------------------------------------------------------------------------------------
// small kernels
// ------------------------------------------------------------------------------------------
__global__ void k_random_block(int64_t n, int p, uint64_t seed, double *X, int ldx, int x0) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * p) return;
    int64_t i = t / p;
    int q = (int)(t - i * p);
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(t + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    X[i * ldx + x0 + q] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// T(row, col) at T[col * ldt + row].  Column block [j, j+p) against rows [0, m): C1 + C2, mirrored
// into row block [j, j+p).  Within the diagonal block the two computed entries (a, q) and (j + q,
// a - j) are equal only up to rounding; one thread writes both mirror entries with their mean, so no
// entry is written twice with different values (which one landed would depend on warp scheduling).
__global__ void k_write_T_block(double *T, int ldt, int m, int j, int p, const double *C1, const double *C2) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * p) return;
    int a = t / p, q = t % p;
    double v = C1[t] + C2[t];
    if (a >= j && a < j + p) {
        const int qa = a - j;
        if (qa < q) return;  // written by the thread of the mirror entry
        const int u = (j + q) * p + qa;
        if (qa > q) v = 0.5 * (v + (C1[u] + C2[u]));
    }
    T[(size_t)(j + q) * ldt + a] = v;
    T[(size_t)a * ldt + (j + q)] = v;
}

__global__ void k_write_R(double *T, int ldt, int m, int j, int p, const double *R) {
    int t = threadIdx.x;
    if (t >= p * p) return;
    int a = t / p, q = t % p;  // R[a][q], upper
    double v = (q >= a) ? R[a * p + q] : 0.0;
    T[(size_t)(j + q) * ldt + (m + a)] = v;
    T[(size_t)(m + a) * ldt + (j + q)] = v;
}

__global__ void k_zero_R_block(double *T, int ldt, int m, int j, int p) {
    int t = threadIdx.x;
    if (t >= p * p) return;
    int a = t / p, q = t % p;
    T[(size_t)(j + q) * ldt + (m + a)] = 0.0;
    T[(size_t)(m + a) * ldt + (j + q)] = 0.0;
}

// R = R2 R1 (upper triangular, row-major p x p)
__global__ void k_upper_mul(int p, const double *R2, const double *R1, double *R) {
    int t = threadIdx.x;
    if (t >= p * p) return;
    int a = t / p, q = t % p;
    double s = 0.0;
    for (int b = a; b <= q; ++b) s += R2[a * p + b] * R1[b * p + q];
    R[t] = (q >= a) ? s : 0.0;
}

__global__ void k_pack_sym(const double *T, int ldt, int mm, double *A) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= mm * mm) return;
    int r = t % mm, c = t / mm;
    A[t] = 0.5 * (T[(size_t)c * ldt + r] + T[(size_t)r * ldt + c]);
}

// One step of iterative refinement of a symmetric eigendecomposition (Ogita and Aishima, 2018):
// with X the approximate eigenvectors (m x m), G = X^T X and S = X^T A X, the refined eigenvalues are
// lambda_i = S_ii / G_ii and X <- X (I + E) with E_ii = r_ii / 2 and, for |lambda_i - lambda_j| > delta,
// E_ij = (S_ij + lambda_j r_ij) / (lambda_j - lambda_i), where r = I - G; closer pairs (a cluster
// at the current accuracy) take E_ij = r_ij / 2, which refines the cluster's subspace.  delta =
// 2 (||S - diag(lambda)|| + ||A|| ||r||), Frobenius norms and ||A|| ~ max |lambda|.  One CTA.
__global__ void __launch_bounds__(1024) k_oa_step(int m, const double *G, const double *S, double *lam, double *E) {
    __shared__ double red[3][32];
    __shared__ double s_delta;
    const int t = threadIdx.x;
    for (int i = t; i < m; i += blockDim.x) lam[i] = S[(size_t)i * m + i] / G[(size_t)i * m + i];
    __syncthreads();
    double off = 0.0, rr = 0.0, amax = 0.0;
    for (int idx = t; idx < m * m; idx += blockDim.x) {
        const int i = idx % m, j = idx / m;
        const double r = (i == j ? 1.0 : 0.0) - G[idx];
        const double sv = S[idx] - (i == j ? lam[i] : 0.0);
        off += sv * sv;
        rr += r * r;
        if (i == j) amax = fmax(amax, fabs(lam[i]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    if ((t & 31) == 0) {
        red[0][t >> 5] = off;
        red[1][t >> 5] = rr;
        red[2][t >> 5] = amax;
    }
    __syncthreads();
    if (t == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
            c = fmax(c, red[2][w]);
        }
        s_delta = 2.0 * (sqrt(a) + c * sqrt(b));
    }
    __syncthreads();
    const double delta = s_delta;
    for (int idx = t; idx < m * m; idx += blockDim.x) {
        const int i = idx % m, j = idx / m;
        const double r = (i == j ? 1.0 : 0.0) - G[idx];
        double e = 0.5 * r;
        if (i != j && fabs(lam[j] - lam[i]) > delta) e = (S[idx] + lam[j] * r) / (lam[j] - lam[i]);
        E[idx] = e;
    }
}

// Per-column quality of an eigendecomposition after refinement, with G = X^T X and S = X^T A X:
// out[j] = ||e_j - G e_j||, out[m + j] = ||(S - diag(S)) e_j||.  One thread per column.
__global__ void k_oa_colnorms(int m, const double *G, const double *S, double *out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double rr = 0.0, off = 0.0;
    for (int i = 0; i < m; ++i) {
        const double r = (i == j ? 1.0 : 0.0) - G[(size_t)j * m + i];
        rr += r * r;
        if (i != j) off += S[(size_t)j * m + i] * S[(size_t)j * m + i];
    }
    out[j] = sqrt(rr);
    out[m + j] = sqrt(off);
}

// `steps` refinement steps of the eigendecomposition X, lam of the symmetric m x m matrix A
// (all column-major, ld m); G, Q, S are m x m scratch.
static void refine_eig(int m, const double *A, double *X, double *lam, int steps, double *G, double *Q, double *S,
                       cudaStream_t st) {
    for (int it = 0; it < steps; ++it) {
        gemm_small(true, false, m, m, m, 1.0, X, m, X, m, 0.0, G, m, st);
        gemm_small(false, false, m, m, m, 1.0, A, m, X, m, 0.0, Q, m, st);
        gemm_small(true, false, m, m, m, 1.0, X, m, Q, m, 0.0, S, m, st);
        k_oa_step<<<1, 1024, 0, st>>>(m, G, S, lam, Q);  // E into Q
        MBL_LAUNCH_CHECK();
        MBL_CUDA(cudaMemcpyAsync(G, X, (size_t)m * m * sizeof(double), cudaMemcpyDeviceToDevice, st));
        gemm_small(false, false, m, m, m, 1.0, G, m, Q, m, 1.0, X, m, st);  // X += X E
    }
}

// res[i] = || T[mm:mm+p, 0:mm] S[:, i] ||
__global__ void k_ritz_resid(const double *T, int ldt, int mm, int p, const double *S, double *res) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mm) return;
    double ss = 0.0;
    for (int a = 0; a < p; ++a) {
        double v = 0.0;
        for (int b = 0; b < mm; ++b) v += T[(size_t)b * ldt + mm + a] * S[(size_t)i * mm + b];
        ss += v * v;
    }
    res[i] = sqrt(ss);
}

// SK[a * k + c] = S[keep[c] * mm + a]
__global__ void k_gather_S(const double *S, int mm, const int *keep, int k, double *SK) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= mm * k) return;
    int a = t / k, c = t % k;
    SK[t] = S[(size_t)keep[c] * mm + a];
}

// Bk[a * k + c] = sum_b T[mm + a][b] SK[b * k + c]
__global__ void k_Bk(const double *T, int ldt, int mm, int p, const double *SK, int k, double *Bk) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p * k) return;
    int a = t / k, c = t % k;
    double s = 0.0;
    for (int b = 0; b < mm; ++b) s += T[(size_t)b * ldt + mm + a] * SK[(size_t)b * k + c];
    Bk[t] = s;
}

// New T after a thick restart: [[Tk, Bk^T], [Bk, 0]] with Tk (k x k, ld k) symmetrized.
__global__ void k_restart_T(double *T, int ldt, int k, int p, const double *Tk, const double *Bk) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int K = k + p;
    if (t >= K * K) return;
    int r = t % K, c = t / K;
    double v = 0.0;
    if (r < k && c < k) v = 0.5 * (Tk[(size_t)c * k + r] + Tk[(size_t)r * k + c]);
    else if (r >= k && c < k) v = Bk[(r - k) * k + c];
    else if (r < k && c >= k) v = Bk[(c - k) * k + r];
    T[(size_t)c * ldt + r] = v;
}

__global__ void k_zero(double *x, int64_t cnt) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) x[t] = 0.0;
}

// Per-CTA sums over the entries t of a CTA of 256 threads with t mod p = q, in index order: the same
// bits on every run (the decisions that read these norms must not depend on warp scheduling).
// v: K arrays of 256 values in shared memory; out[k * p + q].
template <int K>
__device__ void cta_column_sums(const double (*v)[256], int p, int64_t t0, double *out) {
    const int base = (int)(t0 % p);
    for (int u = threadIdx.x; u < K * p; u += blockDim.x) {
        const int k = u / p, q = u - k * p;
        double sum = 0.0;
        for (int j = (q - base + p) % p; j < 256; j += p) sum += v[k][j];
        out[u] = sum;
    }
}

// R = B - (H - sigma) Y for p columns; per-CTA partial sums of |R_q|^2, |Y_q|^2, |B_q|^2.  256 threads.
__global__ void __launch_bounds__(256) k_refine_resid(int64_t n, const int64_t *__restrict__ rowptr,
                                                      const int32_t *__restrict__ col, const double *__restrict__ val,
                                                      double sigma, const double *__restrict__ B, int ldb,
                                                      const double *__restrict__ Y, double *__restrict__ R, int p,
                                                      double *part) {
    __shared__ double v[3][256];
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x, t = t0 + threadIdx.x;
    int64_t i = t / p;
    int q = (int)(t - i * p);
    double rr = 0.0, yy = 0.0, bb = 0.0;
    if (i < n) {
        double s = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s = fma(val[e], Y[(int64_t)col[e] * p + q], s);
        double y = Y[i * p + q];
        double b = B[i * ldb + q];
        double r = b - (s - sigma * y);
        R[i * p + q] = r;
        rr = r * r;
        yy = y * y;
        bb = b * b;
    }
    v[0][threadIdx.x] = rr;
    v[1][threadIdx.x] = yy;
    v[2][threadIdx.x] = bb;
    __syncthreads();
    cta_column_sums<3>(v, p, t0, part + (size_t)blockIdx.x * 3 * p);
}

// out[u] = sum_b part[b * w + u], u < w: one warp per output, lanes over the partial blocks (all
// loads in flight at once), summed in a fixed order (lane-strided, then a shuffle tree).  Launch
// with reduce_grid(w) blocks of 256 threads.
__global__ void k_reduce_parts(int nb, int w, const double *part, double *out) {
    const int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (u >= w) return;
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += part[(size_t)b * w + u];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[u] = s;
}
static unsigned reduce_grid(int w) { return (unsigned)((w + 7) / 8); }

// per-CTA partial sums of |X_q|^2 and |Y_q - theta_q X_q|^2 for m columns (row-major, ld m), in a
// fixed order (cta_column_sums).  256 threads.
__global__ void __launch_bounds__(256) k_pair_resid(int64_t n, int m, const double *X, const double *HX,
                                                    const double *theta, double *part) {
    __shared__ double v[2][256];
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x, t = t0 + threadIdx.x;
    int64_t i = t / m;
    int q = (int)(t - i * m);
    double xx = 0.0, rr = 0.0;
    if (i < n) {
        double x = X[i * m + q];
        double r = HX[i * m + q] - theta[q] * x;
        xx = x * x;
        rr = r * r;
    }
    v[0][threadIdx.x] = xx;
    v[1][threadIdx.x] = rr;
    __syncthreads();
    cta_column_sums<2>(v, m, t0, part + (size_t)blockIdx.x * 2 * m);
}

__global__ void k_scale_cols_to_cm(int64_t n, int m, const double *Y, const double *nrm2, double *out_cm) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * m) return;
    int64_t i = t / m;
    int q = (int)(t - i * m);
    out_cm[(int64_t)q * n + i] = Y[t] / sqrt(nrm2[q]);
}

__global__ void k_csr_to_dense(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val, double *A) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t c = 0; c < n; ++c) A[c * n + i] = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) A[(int64_t)col[e] * n + i] = val[e];
}

__global__ void k_select_cols_cm(int64_t n, const double *A, const int *idx, int nev, double *out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * nev) return;
    int64_t c = t / n, i = t - c * n;
    out[t] = A[(int64_t)idx[c] * n + i];
}

__global__ void k_cm_to_rm(int64_t n, int m, const double *cm, double *rm) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * m) return;
    int64_t i = t / m;
    int q = (int)(t - i * m);
    rm[t] = cm[(int64_t)q * n + i];
}

static unsigned nblk(int64_t tot, int thr = 256) { return (unsigned)((tot + thr - 1) / thr); }

// ------------------------------------------------------------------------------------------
// Krylov-Schur engine
// ------------------------------------------------------------------------------------------
// dst[:, d0:d0+m] (FP32, row stride ldd) = src[:, s0:s0+m] (row stride lds)
__global__ void k_cols_f32(int64_t n, const double *src, int lds, int s0, float *dst, int ldd, int d0, int m) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * m) return;
    const int64_t i = t / m;
    const int j = (int)(t - i * m);
    dst[i * ldd + d0 + j] = (float)src[i * lds + s0 + j];
}

KrylovSchur::KrylovSchur(Ctx *c, int64_t n_, int p_, int ncv_) : ctx(c), n(n_), p(p_), ncv(ncv_) {
    ldv = ncv + p;
    V.alloc(ctx, (size_t)n * ldv);
    V32.alloc(ctx, (size_t)n * ldv);
    V2.alloc(ctx, (size_t)n * ldv);
    W.alloc(ctx, (size_t)n * p);
    T.alloc(ctx, (size_t)ldv * ldv);
    C1.alloc(ctx, (size_t)ldv * p);
    C2.alloc(ctx, (size_t)ldv * p);
    R1.alloc(ctx, p * p);
    R2.alloc(ctx, p * p);
    Rm.alloc(ctx, p * p);
    G.alloc(ctx, p * p);
    flag.alloc(ctx, 1);
    work.alloc(ctx, std::max(dense_tn_work(n, ldv, p), dense_tn_work(n, ldv, 32)) + 64);
    eigA.alloc(ctx, (size_t)ldv * ldv);
    eigW.alloc(ctx, ldv);
    eigWork.alloc(ctx, syev_work_doubles(ldv));
    eigInfo.alloc(ctx, 1);
    eigM.alloc(ctx, 1);
    eigOff.alloc(ctx, 2);
    res.alloc(ctx, ldv);
    keep.alloc(ctx, ldv);
    SK.alloc(ctx, (size_t)ldv * ldv);
    NS1.alloc(ctx, (size_t)ldv * ldv);
    NS2.alloc(ctx, (size_t)ldv * ldv);
    NS3.alloc(ctx, (size_t)ldv * ldv);
    Ts.alloc(ctx, (size_t)ldv * ldv);
    Bk.alloc(ctx, (size_t)p * ldv);
    int64_t zero2[2] = {0, 0};
    MBL_CUDA(cudaMemcpy(eigOff.data(), zero2, sizeof(zero2), cudaMemcpyHostToDevice));
}

void KrylovSchur::orthonormalize_new_block(int m, cudaStream_t st, bool *deflated) {
    // W -= V[:, 0:m] (V^T W), twice; then Cholesky-QR twice: W = Q R, R = R2 R1
    double *Vd = V.data();
    if (m > 0) {
        dense_tn(n, Vd, ldv, 0, m, W.data(), p, 0, p, C1.data(), work.data(), st);
        dense_nn_sub(n, Vd, ldv, 0, m, C1.data(), p, W.data(), st);
        dense_tn(n, Vd, ldv, 0, m, W.data(), p, 0, p, C2.data(), work.data(), st);
        dense_nn_sub(n, Vd, ldv, 0, m, C2.data(), p, W.data(), st);
    }
    int one = 1;
    MBL_CUDA(cudaMemcpyAsync(flag.data(), &one, sizeof(int), cudaMemcpyHostToDevice, st));
    chol_qr(n, W.data(), p, R1.data(), G.data(), work.data(), flag.data(), st);
    chol_qr(n, W.data(), p, R2.data(), G.data(), work.data(), flag.data(), st);
    k_upper_mul<<<1, 1024, 0, st>>>(p, R2.data(), R1.data(), Rm.data());
    MBL_LAUNCH_CHECK();
    int ok = 1;
    MBL_CUDA(cudaMemcpyAsync(&ok, flag.data(), sizeof(int), cudaMemcpyDeviceToHost, st));
    MBL_CUDA(cudaStreamSynchronize(st));
    *deflated = (ok == 0);
}

void KrylovSchur::start(uint64_t seed, cudaStream_t st) {
    k_zero<<<nblk((int64_t)ldv * ldv), 256, 0, st>>>(T.data(), (int64_t)ldv * ldv);
    MBL_LAUNCH_CHECK();
    for (int attempt = 0; attempt < 4; ++attempt) {
        k_random_block<<<nblk(n * p), 256, 0, st>>>(n, p, seed + 7919ull * attempt, W.data(), p, 0);
        MBL_LAUNCH_CHECK();
        bool defl = false;
        orthonormalize_new_block(0, st, &defl);
        if (!defl) break;
        if (attempt == 3) fail(MBL_ERR_INVALID, "Krylov start block is rank deficient");
    }
    copy_cols(n, W.data(), p, 0, V.data(), ldv, 0, p, st);
    k_cols_f32<<<nblk(n * p), 256, 0, st>>>(n, W.data(), p, 0, V32.data(), ldv, 0, p);
    MBL_LAUNCH_CHECK();
    m = p;
}

void KrylovSchur::expand(const OpFn &op, cudaStream_t st) {
    int j = m - p;  // last (unexpanded) block
    op(V.data() + j, ldv, W.data(), st);
    double *Vd = V.data();
    ProfScope ps(ctx, "orth", 8.0 * (double)n * m * p, st);
    // classical Gram-Schmidt twice.  The first pass's coefficients C1 = V^T W come from the FP32 copy
    // of V in FP32 arithmetic (they only have to make the second pass's input nearly orthogonal);
    // the subtraction W -= V C1 is FP64 on the FP64 basis, so that W = V (C1 + C2) + W' holds to FP64
    // rounding whatever C1's error (the Krylov-Schur relation rests on it); the second pass is FP64
    dense_tn32(n, V32.data(), ldv, 0, m, W.data(), p, 0, p, C1.data(), work.data(), st);
    dense_nn_sub(n, Vd, ldv, 0, m, C1.data(), p, W.data(), st);
    dense_tn(n, Vd, ldv, 0, m, W.data(), p, 0, p, C2.data(), work.data(), st);
    dense_nn_sub(n, Vd, ldv, 0, m, C2.data(), p, W.data(), st);
    k_write_T_block<<<nblk((int64_t)m * p), 256, 0, st>>>(T.data(), ldv, m, j, p, C1.data(), C2.data());
    MBL_LAUNCH_CHECK();
    bool defl = false;
    orthonormalize_new_block(m, st, &defl);
    if (defl) {
        // invariant subspace reached: continue with a fresh random block orthogonal to V, no coupling
        for (int attempt = 0; attempt < 4 && defl; ++attempt) {
            k_random_block<<<nblk(n * p), 256, 0, st>>>(n, p, 0xD1B54A32D192ED03ull + m + attempt, W.data(), p, 0);
            MBL_LAUNCH_CHECK();
            orthonormalize_new_block(m, st, &defl);
        }
        if (defl) fail(MBL_ERR_INVALID, "Krylov basis cannot be extended (sector too small for the basis)");
        k_zero_R_block<<<1, 1024, 0, st>>>(T.data(), ldv, m, j, p);
        MBL_LAUNCH_CHECK();
    } else {
        k_write_R<<<1, 1024, 0, st>>>(T.data(), ldv, m, j, p, Rm.data());
        MBL_LAUNCH_CHECK();
    }
    copy_cols(n, W.data(), p, 0, V.data(), ldv, m, p, st);
    k_cols_f32<<<nblk(n * p), 256, 0, st>>>(n, W.data(), p, 0, V32.data(), ldv, m, p);
    MBL_LAUNCH_CHECK();
    m += p;
}

void KrylovSchur::ritz(cudaStream_t st, std::vector<double> &theta, std::vector<double> &rnorm) {
    int mm = m - p;
    k_pack_sym<<<nblk((int64_t)mm * mm), 256, 0, st>>>(T.data(), ldv, mm, eigA.data());
    MBL_LAUNCH_CHECK();
    k_pack_sym<<<nblk((int64_t)mm * mm), 256, 0, st>>>(T.data(), ldv, mm, Ts.data());
    MBL_LAUNCH_CHECK();
    MBL_CUDA(cudaMemcpyAsync(eigM.data(), &mm, sizeof(int), cudaMemcpyHostToDevice, st));
    const bool fp32 = ldv <= EIG_SMEM_MAX_M;
    {
        ProfScope ps(ctx, "syev_krylov", (double)mm, st);
        // FP32 reduction and QL, then two steps of FP64 refinement of the whole decomposition: a
        // thick restart keeps an invariant subspace of T, so the kept vectors must be accurate to
        // FP64 rounding (an FP32-accurate subspace would cap the attainable residuals near 1e-7).
        // (The FP32 Jacobi start, unchecked here, left an L = 16 job at 48 of 50 pairs.)
        // Bisection and inverse iteration in FP32 are not a usable start here: the small Ritz values
        // of T lie in clusters within which inverse iteration mixes the vectors, the kept block then
        // cuts through such a cluster, and an L = 16 job converged 47 of 50 pairs (three refinement
        // steps did not repair it).
        int info = 0;
        {
            ProfScope ps1(ctx, fp32 ? "syev_fp32" : "syev_fp64", (double)mm, st);
            syev_batched(1, eigM.data(), eigOff.data(), eigOff.data(), eigA.data(), eigW.data(), 1, nullptr, ldv,
                         eigWork.data(), eigInfo.data(), st, fp32);
        }
        MBL_CUDA(cudaMemcpyAsync(&info, eigInfo.data(), sizeof(int), cudaMemcpyDeviceToHost, st));
        MBL_CUDA(cudaStreamSynchronize(st));
        if (fp32 && info != 0) {  // QL did not converge in FP32: redo in FP64
            ProfScope ps2(ctx, "syev_fallback", (double)mm, st);
            k_pack_sym<<<nblk((int64_t)mm * mm), 256, 0, st>>>(T.data(), ldv, mm, eigA.data());
            MBL_LAUNCH_CHECK();
            syev_batched(1, eigM.data(), eigOff.data(), eigOff.data(), eigA.data(), eigW.data(), 1, nullptr, ldv,
                         eigWork.data(), eigInfo.data(), st, false);
        }
        if (fp32) {
            ProfScope ps3(ctx, "oa_refine", (double)mm, st);
            refine_eig(mm, Ts.data(), eigA.data(), eigW.data(), 2, NS1.data(), NS2.data(), NS3.data(), st);
        }
    }
    k_ritz_resid<<<nblk(mm, 128), 128, 0, st>>>(T.data(), ldv, mm, p, eigA.data(), res.data());
    MBL_LAUNCH_CHECK();
    theta.resize(mm);
    rnorm.resize(mm);
    MBL_CUDA(cudaMemcpyAsync(theta.data(), eigW.data(), mm * sizeof(double), cudaMemcpyDeviceToHost, st));
    MBL_CUDA(cudaMemcpyAsync(rnorm.data(), res.data(), mm * sizeof(double), cudaMemcpyDeviceToHost, st));
    MBL_CUDA(cudaStreamSynchronize(st));
}

void KrylovSchur::restart(const std::vector<int> &keep_idx, cudaStream_t st) {
    ProfScope ps_all(ctx, "ks_restart", (double)keep_idx.size(), st);
    int mm = m - p;
    int k = (int)keep_idx.size();
    MBL_CUDA(cudaMemcpyAsync(keep.data(), keep_idx.data(), k * sizeof(int), cudaMemcpyHostToDevice, st));
    // Y = S_keep^T (k x mm, column-major ld k) from the FP32 Ritz vectors
    double *Y = SK.data(), *Y2 = NS1.data(), *Gk = NS2.data(), *Q = NS3.data();
    k_gather_S<<<nblk((int64_t)mm * k), 256, 0, st>>>(eigA.data(), mm, keep.data(), k, Y);
    MBL_LAUNCH_CHECK();
    // Newton-Schulz in FP64: S <- S (3 I - S^T S) / 2, i.e. Y <- 1.5 Y - 0.5 (Y Y^T) Y; two steps take
    // an orthogonality defect of FP32 size (~1e-6) to FP64 rounding
    for (int it = 0; it < 2; ++it) {
        gemm_small(false, true, k, k, mm, 1.0, Y, k, Y, k, 0.0, Gk, k, st);
        MBL_CUDA(cudaMemcpyAsync(Y2, Y, (size_t)k * mm * sizeof(double), cudaMemcpyDeviceToDevice, st));
        gemm_small(false, false, k, mm, k, -0.5, Gk, k, Y, k, 1.5, Y2, k, st);
        std::swap(Y, Y2);
    }
    // exact projection of the expanded T onto the kept vectors: Tk = S^T T S (no diagonal assumed)
    gemm_small(false, true, mm, k, mm, 1.0, T.data(), ldv, Y, k, 0.0, Q, mm, st);
    gemm_small(false, false, k, k, mm, 1.0, Y, k, Q, mm, 0.0, Gk, k, st);
    k_Bk<<<nblk((int64_t)p * k), 256, 0, st>>>(T.data(), ldv, mm, p, Y, k, Bk.data());
    MBL_LAUNCH_CHECK();
    dense_nn(n, V.data(), ldv, mm, Y, k, V2.data(), ldv, 0, st);
    copy_cols(n, V.data(), ldv, mm, V2.data(), ldv, k, p, st);
    std::swap(V, V2);
    k_cols_f32<<<nblk(n * (k + p)), 256, 0, st>>>(n, V.data(), ldv, 0, V32.data(), ldv, 0, k + p);
    MBL_LAUNCH_CHECK();
    k_zero<<<nblk((int64_t)ldv * ldv), 256, 0, st>>>(T.data(), (int64_t)ldv * ldv);
    MBL_LAUNCH_CHECK();
    k_restart_T<<<nblk((int64_t)(k + p) * (k + p)), 256, 0, st>>>(T.data(), ldv, k, p, Gk, Bk.data());
    MBL_LAUNCH_CHECK();
    m = k + p;
}

// ------------------------------------------------------------------------------------------
// refined shift-invert operator
// ------------------------------------------------------------------------------------------
double RefinedSolve::residual(const double *X, int ldx, double *Y, int p, cudaStream_t st, std::vector<double> *rn,
                              std::vector<double> *lim) {
    int64_t n = sec->n;
    unsigned nb = nblk(n * p);
    if (part.size() < (size_t)nb * 3 * p) part.alloc(sec->ctx, (size_t)nb * 3 * p);
    {
        ProfScope ps(sec->ctx, "refine_spmv", 12.0 * (double)sec->nnz + 8.0 * (double)n * (3.0 * p + 1.0), st);
        k_refine_resid<<<nb, 256, 0, st>>>(n, sec->rowptr.data(), sec->col.data(), sec->val.data(), fz->sigma, X, ldx, Y,
                                           R.data(), p, part.data());
        MBL_LAUNCH_CHECK();
    }
    k_reduce_parts<<<reduce_grid(3 * p), 256, 0, st>>>((int)nb, 3 * p, part.data(), norms.data());
    MBL_LAUNCH_CHECK();
    std::vector<double> h(3 * p);
    MBL_CUDA(cudaMemcpyAsync(h.data(), norms.data(), 3 * p * sizeof(double), cudaMemcpyDeviceToHost, st));
    MBL_CUDA(cudaStreamSynchronize(st));
    double worst = 0.0, rmax = 0.0;
    if (rn) rn->assign(p, 0.0);
    if (lim) lim->assign(p, 0.0);
    for (int q = 0; q < p; ++q) {
        double r = std::sqrt(h[q]), yn = std::sqrt(h[p + q]), bn = std::sqrt(h[2 * p + q]);
        double l = rtol * (anorm * yn + bn);
        worst = std::max(worst, l > 0 ? r / l : (r > 0 ? INFINITY : 0.0));
        rmax = std::max(rmax, r / std::max(bn, 1e-300));
        if (rn) (*rn)[q] = r;
        if (lim) (*lim)[q] = l;
    }
    last_rel = rmax;
    return worst;
}

void RefinedSolve::apply(const double *X, int ldx, double *Y, int p, cudaStream_t st) {
    ProfScope ps_all(sec->ctx, "op_apply", (double)p, st);
    int64_t n = sec->n;
    if (R.size() < (size_t)n * p) R.alloc(sec->ctx, (size_t)n * p);
    if (norms.size() < (size_t)3 * 32) norms.alloc(sec->ctx, 3 * 32);
    factor_solve_raw(*fz, X, ldx, Y, p, p, false, st);
    ++solves;
    ++applies;
    if (gmres) apply_fgmres(X, ldx, Y, p, st);
    else apply_plain(X, ldx, Y, p, st);
}

void RefinedSolve::apply_plain(const double *X, int ldx, double *Y, int p, cudaStream_t st) {
    double prev = INFINITY;
    int stall = 0;
    for (int it = 0; it <= max_refine; ++it) {
        double worst = residual(X, ldx, Y, p, st);
        if (worst <= 1.0) break;
        if (it == max_refine) { stalled = true; break; }
        if (last_rel > 0.5 * prev) {
            if (++stall >= 2) { stalled = true; break; }
        } else stall = 0;
        prev = last_rel;
        factor_solve_raw(*fz, R.data(), p, Y, p, p, true, st);
        ++solves;
    }
}

// ---- FGMRES refinement kernels (all p columns in lockstep, each with its own Krylov space) ----
// V blocks are n x p row-major; column q of block i is the i-th Arnoldi vector of right-hand side q.
// part[chunk][i * p + q] = sum over the chunk's rows r of V_i[r][q] W[r][q], i < k1.  Thread t < S
// (S = the largest multiple of p up to the block size) walks the chunk's row-major elements with
// stride S, so its column q = t % p is fixed and the loads coalesce; sixteen V_i at a time are
// accumulated in registers, then the threads of each q are added in shared memory (16 x blockDim).
__global__ void k_gm_dots_part(int64_t n, int k1, int p, const double *V, int64_t vstride, const double *W,
                               double *part, int64_t rows_per) {
    extern __shared__ double red[];
    const int t = threadIdx.x, nt = blockDim.x, S = (nt / p) * p;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    const int64_t e0 = r0 * p, e1 = r1 * p;
    for (int i0 = 0; i0 < k1; i0 += 16) {
        const int ni = min(16, k1 - i0);
        double acc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = 0.0;
        if (t < S) {
            for (int64_t e = e0 + t; e < e1; e += S) {
                const double wv = W[e];
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (i < ni) acc[i] = fma(V[(int64_t)(i0 + i) * vstride + e], wv, acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) red[i * nt + t] = t < S ? acc[i] : 0.0;
        __syncthreads();
        for (int o = t; o < ni * p; o += nt) {
            const int i = o / p, q = o - i * p;
            double sum = 0.0;
            for (int u = q; u < S; u += p) sum += red[i * nt + u];
            part[(size_t)blockIdx.x * k1 * p + (size_t)(i0 + i) * p + q] = sum;
        }
        __syncthreads();
    }
}

__global__ void k_gm_sub(int64_t n, int k1, int p, const double *V, int64_t vstride, const double *h, double *W) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * p) return;
    int q = (int)(t % p);
    double s = 0.0;
    for (int i = 0; i < k1; ++i) s = fma(V[(int64_t)i * vstride + t], h[i * p + q], s);
    W[t] -= s;
}

// normalize W into V_{k+1}; the norms (one per column) come from a dots pass with V = W
__global__ void k_gm_scale(int64_t n, int p, const double *W, const double *nrm2, double *Vn) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * p) return;
    double nn = sqrt(nrm2[t % p]);
    Vn[t] = nn > 0.0 ? W[t] / nn : 0.0;
}

// Hessenberg bookkeeping per column q (one thread each): store column k of H (h1 + h2 from the two
// Gram-Schmidt passes, h_{k+1,k} = |w|), apply the earlier Givens rotations, make a new one, update g.
// Layout per column: Hc[(kmax+1) x kmax] column-major, cs/sn[kmax], g[kmax+1].
__global__ void k_gm_givens(int p, int k, int kmax, const double *h1, const double *h2, const double *nrm2,
                            double *Hall, double *res) {
    int q = threadIdx.x;
    if (q >= p) return;
    const int ld = kmax + 1;
    double *Hc = Hall + (size_t)q * (ld * kmax + 3 * ld);
    double *cs = Hc + ld * kmax, *sn = cs + ld, *g = sn + ld;
    double *col = Hc + (size_t)k * ld;
    for (int i = 0; i <= k; ++i) col[i] = h1[i * p + q] + h2[i * p + q];
    col[k + 1] = sqrt(nrm2[q]);
    for (int i = 0; i < k; ++i) {
        double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    double a = col[k], b = col[k + 1];
    double r = hypot(a, b);
    double c = r > 0.0 ? a / r : 1.0, s_ = r > 0.0 ? b / r : 0.0;
    cs[k] = c;
    sn[k] = s_;
    col[k] = r;
    col[k + 1] = 0.0;
    g[k + 1] = -s_ * g[k];
    g[k] = c * g[k];
    res[q] = fabs(g[k + 1]);
}

__global__ void k_gm_init(int p, int kmax, const double *beta2, double *Hall) {
    int q = threadIdx.x;
    if (q >= p) return;
    const int ld = kmax + 1;
    double *Hc = Hall + (size_t)q * (ld * kmax + 3 * ld);
    double *g = Hc + ld * kmax + 2 * ld;
    for (int i = 0; i < ld; ++i) g[i] = 0.0;
    g[0] = sqrt(beta2[q]);
}

// y = H^{-1} g (upper triangular, k columns), per column q
__global__ void k_gm_solve(int p, int k, int kmax, const double *Hall, double *Y) {
    int q = threadIdx.x;
    if (q >= p) return;
    const int ld = kmax + 1;
    const double *Hc = Hall + (size_t)q * (ld * kmax + 3 * ld);
    const double *g = Hc + ld * kmax + 2 * ld;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int j = i + 1; j < k; ++j) s -= Hc[(size_t)j * ld + i] * Y[j * p + q];
        Y[i * p + q] = Hc[(size_t)i * ld + i] != 0.0 ? s / Hc[(size_t)i * ld + i] : 0.0;
    }
}

// X += sum_i Z_i y_i (per column)
__global__ void k_gm_update(int64_t n, int k, int p, const double *Z, int64_t zstride, const double *y, double *X) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * p) return;
    int q = (int)(t % p);
    double s = 0.0;
    for (int i = 0; i < k; ++i) s = fma(Z[(int64_t)i * zstride + t], y[i * p + q], s);
    X[t] += s;
}

// In-place inverse of a k x k row-major matrix by Gauss-Jordan elimination with partial pivoting
// (one CTA, matrix in shared memory).  *flag = 0 if a pivot vanished.
__global__ void __launch_bounds__(512) k_small_inverse(int k, double *A, int *flag) {
    extern __shared__ double sa[];
    __shared__ int perm[128], s_p;
    __shared__ double s_piv;
    const int t = threadIdx.x;
    for (int i = t; i < k * k; i += blockDim.x) sa[i] = A[i];
    if (t == 0) *flag = 1;
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (t == 0) {
            int p = j;
            double best = fabs(sa[j * k + j]);
            for (int i = j + 1; i < k; ++i)
                if (fabs(sa[i * k + j]) > best) {
                    best = fabs(sa[i * k + j]);
                    p = i;
                }
            s_p = p;
            perm[j] = p;
        }
        __syncthreads();
        const int p = s_p;
        if (p != j)
            for (int c = t; c < k; c += blockDim.x) {
                const double x = sa[j * k + c];
                sa[j * k + c] = sa[p * k + c];
                sa[p * k + c] = x;
            }
        __syncthreads();
        if (t == 0) {
            s_piv = sa[j * k + j];
            if (!(fabs(s_piv) > 1e-300)) {
                *flag = 0;
                s_piv = 1.0;
            }
            sa[j * k + j] = 1.0;
        }
        __syncthreads();
        const double ip = 1.0 / s_piv;
        for (int c = t; c < k; c += blockDim.x) sa[j * k + c] *= ip;
        __syncthreads();
        for (int idx = t; idx < k * k; idx += blockDim.x) {
            const int i = idx / k, c = idx % k;
            if (i == j || c == j) continue;
            sa[i * k + c] -= sa[i * k + j] * sa[j * k + c];
        }
        __syncthreads();
        for (int i = t; i < k; i += blockDim.x)
            if (i != j) sa[i * k + j] = -sa[i * k + j] * sa[j * k + j];
        __syncthreads();
    }
    // the row swaps of the elimination become column swaps of the inverse, undone in reverse order
    for (int j = k - 1; j >= 0; --j) {
        const int p = perm[j];
        if (p != j)
            for (int i = t; i < k; i += blockDim.x) {
                const double x = sa[i * k + j];
                sa[i * k + j] = sa[i * k + p];
                sa[i * k + p] = x;
            }
        __syncthreads();
    }
    for (int i = t; i < k * k; i += blockDim.x) A[i] = sa[i];
}

// dst (n x k row-major, FP32) = src[:, 0:k] (row stride lds)
__global__ void k_cols_to_f32(int64_t n, const double *src, int lds, int k, float *dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * k) return;
    const int64_t i = t / k;
    dst[t] = (float)src[i * lds + (t - i * k)];
}

// ---- deflation products: tall-skinny products with the FP32 copies U32, AU32 (n x kd, kd <= 90) ----
constexpr int DEFL_ROWS = 256;  // rows per CTA of k_defl_tn

// part[b][a][q] = sum over the block's rows r of U[r][a] V[r][q] (FP32 arithmetic, V converted): thread
// a of the CTA owns column a of U (coalesced row reads), the block's rows of V are staged in shared
// memory and read as broadcasts.
template <int PB>
__global__ void __launch_bounds__(128) k_defl_tn(int64_t n, int kd, int p, const float *__restrict__ U,
                                                const double *__restrict__ V, double *__restrict__ part) {
    __shared__ float sv[DEFL_ROWS * PB];
    const int64_t r0 = (int64_t)blockIdx.x * DEFL_ROWS;
    const int nr = (int)min((int64_t)DEFL_ROWS, n - r0);
    for (int e = threadIdx.x; e < nr * PB; e += blockDim.x) {
        const int r = e / PB, q = e - r * PB;
        sv[e] = q < p ? (float)V[(r0 + r) * p + q] : 0.f;
    }
    __syncthreads();
    const int a = threadIdx.x;
    if (a >= kd) return;
    float acc[PB];
#pragma unroll
    for (int q = 0; q < PB; ++q) acc[q] = 0.f;
    const float *u = U + r0 * kd + a;
    for (int r = 0; r < nr; ++r) {
        const float ur = u[(int64_t)r * kd];
#pragma unroll
        for (int q = 0; q < PB; ++q) acc[q] = fmaf(ur, sv[r * PB + q], acc[q]);
    }
    double *out = part + ((size_t)blockIdx.x * kd + a) * p;
#pragma unroll
    for (int q = 0; q < PB; ++q)
        if (q < p) out[q] = (double)acc[q];
}

// c = Einv C (kd x p, row-major; C = U^T v, reduced from the block sums by k_reduce_parts): a thread
// per output.
__global__ void k_defl_coef(int kd, int p, const double *__restrict__ C, const double *__restrict__ Einv,
                            double *__restrict__ c) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= kd * p) return;
    const int a = o / p, q = o - a * p;
    double s = 0.0;
    for (int k = 0; k < kd; ++k) s = fma(Einv[(size_t)a * kd + k], C[k * p + q], s);
    c[o] = s;
}

// Xout[r][q] = Xin[r][q] + sign * sum_a U[r][a] c[a][q] (the sum in FP32): a thread per row, c staged
// in shared memory.  Xin may be Xout.
template <int PB>
__global__ void __launch_bounds__(128) k_defl_apply(int64_t n, int kd, int p, const float *__restrict__ U,
                                                   const double *__restrict__ c, const double *Xin, double *Xout,
                                                   double sign) {
    __shared__ float scf[90 * PB];
    for (int e = threadIdx.x; e < kd * PB; e += blockDim.x) {
        const int a = e / PB, q = e - a * PB;
        scf[e] = q < p ? (float)c[a * p + q] : 0.f;
    }
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float acc[PB];
#pragma unroll
    for (int q = 0; q < PB; ++q) acc[q] = 0.f;
    const float *u = U + r * kd;
    for (int a = 0; a < kd; ++a) {
        const float ua = u[a];
#pragma unroll
        for (int q = 0; q < PB; ++q) acc[q] = fmaf(ua, scf[a * PB + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < PB; ++q)
        if (q < p) Xout[r * p + q] = Xin[r * p + q] + sign * (double)acc[q];
}

void RefinedSolve::set_deflation(const double *U_, int ldu_, int k, cudaStream_t st) {
    kd = 0;
    if (k <= 0) return;
    k = std::min(k, 90);
    const int64_t n = sec->n;
    Ctx *ctx = sec->ctx;
    if (AU.size() < (size_t)n * k) AU.alloc(ctx, (size_t)n * k);
    if (Einv.size() < (size_t)k * k) Einv.alloc(ctx, (size_t)k * k);
    if (Dc0.size() < (size_t)k * 32) Dc0.alloc(ctx, (size_t)k * 32);
    if (Dc1.size() < (size_t)k * 32) Dc1.alloc(ctx, (size_t)k * 32);
    // Dwork: E's partial sums (dense_tn), then the deflation products' per-block partial sums
    const size_t dwork = std::max(dense_tn_work(n, k, std::max(k, 32)),
                                  (size_t)((n + DEFL_ROWS - 1) / DEFL_ROWS) * (size_t)k * 32) + 64;
    if (Dwork.size() < dwork) Dwork.alloc(ctx, dwork);
    if (Dflag.size() < 1) Dflag.alloc(ctx, 1);
    if (U32.size() < (size_t)n * k) U32.alloc(ctx, (size_t)n * k);
    if (AU32.size() < (size_t)n * k) AU32.alloc(ctx, (size_t)n * k);
    // A U, then E = U^T A U (k x k, row-major) and its inverse
    launch_spmv(sec, fz->sigma, U_, ldu_, 1, AU.data(), k, 1, k, st);
    dense_tn(n, U_, ldu_, 0, k, AU.data(), k, 0, k, Einv.data(), Dwork.data(), st);
    smem_limit((const void *)k_small_inverse, 90 * 90 * 8);
    k_small_inverse<<<1, 512, (size_t)k * k * sizeof(double), st>>>(k, Einv.data(), Dflag.data());
    MBL_LAUNCH_CHECK();
    int ok = 0;
    MBL_CUDA(cudaMemcpyAsync(&ok, Dflag.data(), sizeof(int), cudaMemcpyDeviceToHost, st));
    MBL_CUDA(cudaStreamSynchronize(st));
    if (!ok) return;
    k_cols_to_f32<<<nblk(n * k), 256, 0, st>>>(n, U_, ldu_, k, U32.data());
    MBL_LAUNCH_CHECK();
    k_cols_to_f32<<<nblk(n * k), 256, 0, st>>>(n, AU.data(), k, k, AU32.data());
    MBL_LAUNCH_CHECK();
    kd = k;
}

void RefinedSolve::precondition(const double *V, double *Z, int p, cudaStream_t st) {
    if (kd == 0) {
        factor_solve_raw(*fz, V, p, Z, p, p, false, st);
        return;
    }
    const int64_t n = sec->n;
    if (Dt.size() < (size_t)n * p) Dt.alloc(sec->ctx, (size_t)n * p);
    const unsigned nbd = (unsigned)((n + DEFL_ROWS - 1) / DEFL_ROWS);
    const int pb = p <= 8 ? 8 : (p <= 16 ? 16 : 32);
    auto apply = [&](const float *Uf, const double *Xin, double *Xout, double sign) {
        const unsigned g = nblk(n, 128);
        if (pb == 8) k_defl_apply<8><<<g, 128, 0, st>>>(n, kd, p, Uf, Dc1.data(), Xin, Xout, sign);
        else if (pb == 16) k_defl_apply<16><<<g, 128, 0, st>>>(n, kd, p, Uf, Dc1.data(), Xin, Xout, sign);
        else k_defl_apply<32><<<g, 128, 0, st>>>(n, kd, p, Uf, Dc1.data(), Xin, Xout, sign);
        MBL_LAUNCH_CHECK();
    };
    {
        ProfScope ps(sec->ctx, "gm_deflate", 0.0, st);
        // c = E^-1 U^T v  (kd x p, row-major)
        if (pb == 8) k_defl_tn<8><<<nbd, 128, 0, st>>>(n, kd, p, U32.data(), V, Dwork.data());
        else if (pb == 16) k_defl_tn<16><<<nbd, 128, 0, st>>>(n, kd, p, U32.data(), V, Dwork.data());
        else k_defl_tn<32><<<nbd, 128, 0, st>>>(n, kd, p, U32.data(), V, Dwork.data());
        MBL_LAUNCH_CHECK();
        k_reduce_parts<<<reduce_grid(kd * p), 256, 0, st>>>((int)nbd, kd * p, Dwork.data(), Dc0.data());
        MBL_LAUNCH_CHECK();
        k_defl_coef<<<(unsigned)((kd * p + 127) / 128), 128, 0, st>>>(kd, p, Dc0.data(), Einv.data(), Dc1.data());
        MBL_LAUNCH_CHECK();
        // z = M^-1 (v - A U c) + U c
        apply(AU32.data(), V, Dt.data(), -1.0);
    }
    factor_solve_raw(*fz, Dt.data(), p, Z, p, p, false, st);
    ProfScope ps(sec->ctx, "gm_deflate", 0.0, st);
    apply(U32.data(), Z, Z, 1.0);
}

void RefinedSolve::apply_fgmres(const double *X, int ldx, double *Y, int p, cudaStream_t st) {
    const int64_t n = sec->n;
    Ctx *ctx = sec->ctx;
    const int64_t blk = n * p;
    if (GV.size() < (size_t)blk * (kmax + 1)) GV.alloc(ctx, (size_t)blk * (kmax + 1));
    if (GZ.size() < (size_t)blk * kmax) GZ.alloc(ctx, (size_t)blk * kmax);
    if (GW.size() < (size_t)blk) GW.alloc(ctx, blk);
    const int ld = kmax + 1;
    if (Gh.size() < (size_t)p * (ld * kmax + 3 * ld) + 2 * (size_t)ld * p + 3 * 32)
        Gh.alloc(ctx, (size_t)p * (ld * kmax + 3 * ld) + 2 * (size_t)ld * p + 3 * 32);
    const int64_t rows_per = std::max<int64_t>(1, (n + 303) / 304);
    const int nch = (int)((n + rows_per - 1) / rows_per);
    if (Gdots.size() < (size_t)nch * ld * p) Gdots.alloc(ctx, (size_t)nch * ld * p);
    if (Gy.size() < (size_t)kmax * p + 64) Gy.alloc(ctx, (size_t)kmax * p + 64);
    double *Hall = Gh.data();
    double *h1 = Hall + (size_t)p * (ld * kmax + 3 * ld), *h2 = h1 + (size_t)ld * p, *nr = h2 + (size_t)ld * p;
    const unsigned nbk = nblk(blk);
    auto dots = [&](int k1, const double *V, int64_t vstride, const double *W, double *out) {
        k_gm_dots_part<<<nch, 256, 16 * 256 * sizeof(double), st>>>(n, k1, p, V, vstride, W, Gdots.data(), rows_per);
        MBL_LAUNCH_CHECK();
        k_reduce_parts<<<reduce_grid(k1 * p), 256, 0, st>>>(nch, k1 * p, Gdots.data(), out);
        MBL_LAUNCH_CHECK();
    };
    double prev = INFINITY;
    for (int outer = 0; outer < max_outer; ++outer) {
        std::vector<double> rn, lim;
        double worst = residual(X, ldx, Y, p, st, &rn, &lim);
        if (worst <= 1.0) return;
        if (outer > 0 && last_rel > 0.5 * prev) { stalled = true; return; }
        prev = last_rel;
        // V_0 = R / |R|, g = |R| e_1
        dots(1, R.data(), 0, R.data(), nr);
        k_gm_scale<<<nbk, 256, 0, st>>>(n, p, R.data(), nr, GV.data());
        MBL_LAUNCH_CHECK();
        k_gm_init<<<1, 32, 0, st>>>(p, kmax, nr, Hall);
        MBL_LAUNCH_CHECK();
        int k = 0;
        for (; k < kmax; ++k) {
            double *Vk = GV.data() + (size_t)k * blk, *Zk = GZ.data() + (size_t)k * blk;
            // Z_k = M^-1 V_k ; W = (H - sigma) Z_k
            precondition(Vk, Zk, p, st);  // writes all of Z_k
            ++solves;
            {
                ProfScope ps(ctx, "gm_spmv", 0.0, st);
                launch_spmv(sec, fz->sigma, Zk, p, 1, GW.data(), p, 1, p, st);
            }
            ProfScope ps_o(ctx, "gm_orth", 0.0, st);
            // two Gram-Schmidt passes against V_0..V_k (each column its own space)
            dots(k + 1, GV.data(), blk, GW.data(), h1);
            k_gm_sub<<<nbk, 256, 0, st>>>(n, k + 1, p, GV.data(), blk, h1, GW.data());
            MBL_LAUNCH_CHECK();
            dots(k + 1, GV.data(), blk, GW.data(), h2);
            k_gm_sub<<<nbk, 256, 0, st>>>(n, k + 1, p, GV.data(), blk, h2, GW.data());
            MBL_LAUNCH_CHECK();
            dots(1, GW.data(), 0, GW.data(), nr);
            k_gm_givens<<<1, 32, 0, st>>>(p, k, kmax, h1, h2, nr, Hall, nr + 32);
            MBL_LAUNCH_CHECK();
            k_gm_scale<<<nbk, 256, 0, st>>>(n, p, GW.data(), nr, GV.data() + (size_t)(k + 1) * blk);
            MBL_LAUNCH_CHECK();
            std::vector<double> est(p);
            MBL_CUDA(cudaMemcpyAsync(est.data(), nr + 32, p * sizeof(double), cudaMemcpyDeviceToHost, st));
            MBL_CUDA(cudaStreamSynchronize(st));
            bool ok = true;
            for (int q = 0; q < p; ++q) ok = ok && est[q] <= 0.5 * lim[q];
            if (ok) {
                ++k;
                break;
            }
        }
        k_gm_solve<<<1, 32, 0, st>>>(p, k, kmax, Hall, Gy.data());
        MBL_LAUNCH_CHECK();
        k_gm_update<<<nbk, 256, 0, st>>>(n, k, p, GZ.data(), blk, Gy.data(), Y);
        MBL_LAUNCH_CHECK();
    }
    double worst = residual(X, ldx, Y, p, st);
    if (worst > 1.0) stalled = true;
}

// ------------------------------------------------------------------------------------------
// drivers
// ------------------------------------------------------------------------------------------
static void dense_eigen(mbl_sector *sec, bool vecs, DVec<double> &A, DVec<double> &w, cudaStream_t st) {
    int64_t n = sec->n;
    Ctx *ctx = sec->ctx;
    A.alloc(ctx, (size_t)n * n);
    w.alloc(ctx, n);
    k_csr_to_dense<<<nblk(n, 128), 128, 0, st>>>(n, sec->rowptr.data(), sec->col.data(), sec->val.data(), A.data());
    MBL_LAUNCH_CHECK();
    DVec<int> dm, info;
    DVec<int64_t> off;
    DVec<double> work;
    dm.alloc(ctx, 1);
    info.alloc(ctx, 1);
    off.alloc(ctx, 1);
    work.alloc(ctx, syev_work_doubles((int)n));
    int mi = (int)n;
    int64_t z = 0;
    MBL_CUDA(cudaMemcpyAsync(dm.data(), &mi, sizeof(int), cudaMemcpyHostToDevice, st));
    MBL_CUDA(cudaMemcpyAsync(off.data(), &z, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    syev_batched(1, dm.data(), off.data(), off.data(), A.data(), w.data(), vecs ? 1 : 0, nullptr, (int)n, work.data(),
                 info.data(), st);
    int hinfo = 0;
    MBL_CUDA(cudaMemcpyAsync(&hinfo, info.data(), sizeof(int), cudaMemcpyDeviceToHost, st));
    MBL_CUDA(cudaStreamSynchronize(st));
    if (hinfo != 0) fail(MBL_ERR_NOT_CONVERGED, "dense eigensolver did not converge");
}

// ---- single-vector Lanczos for E_min, E_max ----
// alpha_j, beta_j from the two Gram-Schmidt passes and the norm; v_{j+1} = w / beta_j
__global__ void k_lanczos_norm_part(int64_t n, const double *w, double *part) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += w[i] * w[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        part[blockIdx.x] = t;
    }
}

__global__ void k_normalize_first(int64_t n, double *V, int ldv, const double *part, int nb) {
    __shared__ double inv;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[b];
        inv = 1.0 / sqrt(s);
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        V[i * ldv] *= inv;
}

// Plain Lanczos steps of the extremal bounds, over LZ_BLOCKS CTAs of 256 threads with grid-stride
// loops.  Every CTA sums the previous kernel's LZ_BLOCKS partial sums itself, in the same order, so
// all CTAs use identical coefficients and no single-thread launch sits between the steps.
constexpr int LZ_BLOCKS = 304;

__device__ double lz_block_sum(double s) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

// sum of the LZ_BLOCKS partial sums in a fixed order (a warp per CTA, then across the lanes)
__device__ double lz_total(const double *part) {
    __shared__ double tot;
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int b = threadIdx.x; b < LZ_BLOCKS; b += 32) s += part[b];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) tot = s;
    }
    __syncthreads();
    return tot;
}

// dot[b] = partial sums of v^T (w - beta_{j-1} v_prev)
__global__ void k_lz_dot(int64_t n, int j, const double *v, const double *vprev, const double *w, const double *beta,
                         double *dot) {
    const double b = j > 0 ? beta[j - 1] : 0.0;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += v[i] * (w[i] - b * vprev[i]);
    s = lz_block_sum(s);
    if (threadIdx.x == 0) dot[blockIdx.x] = s;
}

// alpha_j = sum(dot); w <- w - beta_{j-1} v_prev - alpha_j v; nrm[b] = partial sums of |w|^2
__global__ void k_lz_update(int64_t n, int j, const double *v, const double *vprev, double *w, const double *dot,
                            double *alpha, const double *beta, double *nrm) {
    const double a = lz_total(dot), b = j > 0 ? beta[j - 1] : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) alpha[j] = a;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = w[i] - b * vprev[i] - a * v[i];
        w[i] = x;
        s += x * x;
    }
    s = lz_block_sum(s);
    if (threadIdx.x == 0) nrm[blockIdx.x] = s;
}

// beta_j = sqrt(sum(nrm)); out = w / beta_j (out may be v_prev: every read of it is done)
__global__ void k_lz_scale(int64_t n, int j, const double *w, const double *nrm, double *beta, double *out) {
    const double b = sqrt(lz_total(nrm));
    if (blockIdx.x == 0 && threadIdx.x == 0) beta[j] = b;
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = w[i] * inv;
}

__device__ int tri_sturm(int m, const double *a, const double *b, double x) {
    const double pivmin = 1e-300;
    int c = 0;
    double q = a[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < 0.0;
    for (int i = 1; i < m; ++i) {
        q = (a[i] - x) - b[i - 1] * b[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        c += q < 0.0;
    }
    return c;
}

// Extreme eigenvalues of the Lanczos tridiagonal T (alpha, beta) by bisection, and the last component
// of their unit eigenvectors by two steps of inverse iteration.  out = {lo, hi, z_lo, z_hi}.
__global__ void k_tridiag_extremes(int m, const double *a, const double *b, double *scratch, double *out) {
    // warp 0 finds the smallest eigenvalue, warp 1 the largest: multisection, each lane one Sturm
    // count per round (32 points split the bracket into 33 parts), then lane 0 inverse-iterates
    const int which = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (which > 1) return;
    double gl = a[0], gu = a[0];
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
        gl = fmin(gl, a[i] - r);
        gu = fmax(gu, a[i] + r);
    }
    const int j = which == 0 ? 0 : m - 1;
    double lo = gl - 1e-12 * (fabs(gl) + fabs(gu)), hi = gu + 1e-12 * (fabs(gl) + fabs(gu));
    for (int it = 0; it < 64; ++it) {
        const double step = (hi - lo) / 33.0;
        const double x = lo + (lane + 1) * step;
        const bool above = x < hi && tri_sturm(m, a, b, x) > j;  // x lies above eigenvalue j
        const unsigned int mask = __ballot_sync(0xffffffffu, above);
        const int first = mask ? __ffs(mask) - 1 : 32;  // first point above it (32: none)
        const double nlo = first == 0 ? lo : lo + first * step;
        const double nhi = first == 32 ? hi : lo + (first + 1) * step;
        if (nlo == lo && nhi == hi) break;  // no progress at this precision
        lo = nlo;
        hi = fmin(nhi, hi);
        if (hi - lo <= 4.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi))) break;
    }
    if (lane != 0) return;
    const double lam = 0.5 * (lo + hi);
    // inverse iteration on T - lam I (LU with partial pivoting of the tridiagonal)
    double *u1 = scratch + (size_t)which * 6 * m, *u2 = u1 + m, *u3 = u2 + m, *l = u3 + m, *x = l + m, *fl = x + m;
    const double tiny = 1e-15 * (fabs(gl) + fabs(gu)) + 1e-300;
    double aa = a[0] - lam, bb = m > 1 ? b[0] : 0.0;
    for (int i = 0; i < m - 1; ++i) {
        double c = b[i], an = a[i + 1] - lam, bn = (i + 1 < m - 1) ? b[i + 1] : 0.0;
        if (fabs(aa) >= fabs(c)) {
            if (aa == 0.0) aa = tiny;
            double mult = c / aa;
            u1[i] = aa; u2[i] = bb; u3[i] = 0.0; l[i] = mult; fl[i] = 0.0;
            aa = an - mult * bb;
            bb = bn;
        } else {
            double mult = aa / c;
            u1[i] = c; u2[i] = an; u3[i] = bn; l[i] = mult; fl[i] = 1.0;
            aa = bb - mult * an;
            bb = -mult * bn;
        }
    }
    if (fabs(aa) < tiny) aa = aa >= 0.0 ? tiny : -tiny;
    u1[m - 1] = aa;
    for (int i = 0; i < m; ++i) x[i] = 1.0 / sqrt((double)m) * ((i & 1) ? 1.0 : 0.7);
    for (int it = 0; it < 3; ++it) {
        for (int i = 0; i < m - 1; ++i) {
            if (fl[i] != 0.0) { double t = x[i]; x[i] = x[i + 1]; x[i + 1] = t; }
            x[i + 1] -= l[i] * x[i];
        }
        x[m - 1] /= u1[m - 1];
        if (m > 1) x[m - 2] = (x[m - 2] - u2[m - 2] * x[m - 1]) / u1[m - 2];
        for (int i = m - 3; i >= 0; --i) x[i] = (x[i] - u2[i] * x[i + 1] - u3[i] * x[i + 2]) / u1[i];
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += x[i] * x[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < m; ++i) x[i] /= nrm;
    }
    out[which] = lam;
    out[2 + which] = x[m - 1];
}

void extremal_bounds(mbl_sector *sec, double *emin, double *emax) {
    if (sec->have_bounds) {
        *emin = sec->emin;
        *emax = sec->emax;
        return;
    }
    cudaStream_t st = sec->ctx->stream;
    Ctx *ctx = sec->ctx;
    int64_t n = sec->n;
    if (n <= DENSE_MAX_N) {
        DVec<double> A, w;
        dense_eigen(sec, false, A, w, st);
        std::vector<double> hw(n);
        MBL_CUDA(cudaMemcpy(hw.data(), w.data(), n * sizeof(double), cudaMemcpyDeviceToHost));
        sec->emin = hw.front();
        sec->emax = hw.back();
        sec->have_bounds = true;
        *emin = sec->emin;
        *emax = sec->emax;
        return;
    }
    ProfScope ps(ctx, "extremal_bounds", 0.0, st);
    // Plain Lanczos (three-term recurrence, no reorthogonalization): only the extreme Ritz values
    // are wanted, and in finite precision those still converge to the extreme eigenvalues; the lost
    // orthogonality only adds copies of converged Ritz values (Paige's analysis of the method).
    const int mmax = (int)std::min<int64_t>(n - 1, 1200);
    const int ldv = mmax + 1;
    DVec<double> V3, W, alpha, beta, part, scr, out;
    V3.alloc(ctx, (size_t)2 * n);
    W.alloc(ctx, n);
    alpha.alloc(ctx, ldv);
    beta.alloc(ctx, ldv);
    part.alloc(ctx, 2 * (size_t)LZ_BLOCKS);
    scr.alloc(ctx, 12 * (size_t)ldv);
    out.alloc(ctx, 4);
    double *v = V3.data(), *vprev = V3.data() + n, *dot = part.data(), *nrm = part.data() + LZ_BLOCKS;
    // v_prev enters the first step multiplied by beta_{-1} = 0: it must hold numbers (0 * NaN is NaN,
    // and pool memory keeps whatever it held before)
    k_zero<<<nblk(2 * n), 256, 0, st>>>(V3.data(), 2 * n);
    MBL_LAUNCH_CHECK();
    k_random_block<<<nblk(n), 256, 0, st>>>(n, 1, 0xB0B5EEDull, v, 1, 0);
    MBL_LAUNCH_CHECK();
    k_lanczos_norm_part<<<LZ_BLOCKS, 256, 0, st>>>(n, v, nrm);
    MBL_LAUNCH_CHECK();
    k_normalize_first<<<LZ_BLOCKS, 256, 0, st>>>(n, v, 1, nrm, LZ_BLOCKS);
    MBL_LAUNCH_CHECK();
    double lo = 0, hi = 0;
    bool done = false;
    for (int j = 0; j < mmax && !done; ++j) {
        // w = H v; alpha_j = v^T (w - beta_{j-1} v_prev); w <- w - beta_{j-1} v_prev - alpha_j v;
        // beta_j = |w|; v_prev <- w / beta_j, then the roles of v and v_prev swap
        launch_spmv(sec, 0.0, v, 1, 1, W.data(), 1, 1, 1, st);
        k_lz_dot<<<LZ_BLOCKS, 256, 0, st>>>(n, j, v, vprev, W.data(), beta.data(), dot);
        MBL_LAUNCH_CHECK();
        k_lz_update<<<LZ_BLOCKS, 256, 0, st>>>(n, j, v, vprev, W.data(), dot, alpha.data(), beta.data(), nrm);
        MBL_LAUNCH_CHECK();
        k_lz_scale<<<LZ_BLOCKS, 256, 0, st>>>(n, j, W.data(), nrm, beta.data(), vprev);
        MBL_LAUNCH_CHECK();
        std::swap(v, vprev);
        const int m = j + 1;
        // convergence checks every 16 steps from m = 32: a check costs a bisection of T on one CTA,
        // several times the Lanczos steps it could save
        if ((m >= 32 && m % 16 == 0) || m == mmax) {
            k_tridiag_extremes<<<1, 64, 0, st>>>(m, alpha.data(), beta.data(), scr.data(), out.data());
            MBL_LAUNCH_CHECK();
            double h[4], bj;
            MBL_CUDA(cudaMemcpyAsync(h, out.data(), 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
            MBL_CUDA(cudaMemcpyAsync(&bj, beta.data() + j, sizeof(double), cudaMemcpyDeviceToHost, st));
            MBL_CUDA(cudaStreamSynchronize(st));
            lo = h[0];
            hi = h[1];
            double hn = std::max(std::fabs(lo), std::fabs(hi));
            if ((std::fabs(bj * h[2]) <= 1e-13 * hn && std::fabs(bj * h[3]) <= 1e-13 * hn) || bj <= 1e-14 * hn) done = true;
        }
    }
    if (!done) fail(MBL_ERR_NOT_CONVERGED, "extremal Lanczos did not converge");
    sec->emin = lo;
    sec->emax = hi;
    sec->have_bounds = true;
    *emin = lo;
    *emax = hi;
}

static std::vector<int> nearest_sorted(const std::vector<double> &th, double sigma, int nev) {
    std::vector<int> idx(th.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        double da = std::fabs(th[a] - sigma), db = std::fabs(th[b] - sigma);
        if (da != db) return da < db;
        return th[a] < th[b];
    });
    idx.resize(nev);
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return th[a] < th[b]; });
    return idx;
}

// Whether an FP64 factorization of the plan could be held at all: its fronts arena at its peak, its
// solve factor and panel scratch against the device's total memory (less a margin for the rest of the
// job) and the context budget.
static bool fp64_fits_plan(const Plan &p, int arena_mode, const Ctx *ctx) {
    const double need = arena_peak_bytes(p, MBL_PREC_FP64, arena_mode) + 8.0 * (double)p.sg_elems +
                        12.0 * (double)p.n + 8.0 * (double)(p.m_elems + p.wscratch_elems);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        (void)cudaGetLastError();
        return true;
    }
    if (ctx->budget && need > (double)ctx->budget) return false;
    return need < 0.9 * (double)tot;
}

// Whether an FP64 refactorization fits in device memory once the FP32 factor fz is freed: the FP64
// fronts arena at its peak, the FP64 solve factor and panel scratch against the free memory plus what
// fz releases, and the context budget.
static bool fp64_fits(const Factorization &fz, int arena_mode) {
    const Plan &p = *fz.plan;
    const double need = arena_peak_bytes(p, MBL_PREC_FP64, arena_mode) + 8.0 * (double)p.sg_elems +
                        12.0 * (double)p.n + 8.0 * (double)(p.m_elems + p.wscratch_elems);
    const double freed = 4.0 * (double)p.sg_elems + 8.0 * (double)p.n;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        (void)cudaGetLastError();
        return true;
    }
    if (fz.ctx->budget && (double)fz.ctx->in_use - freed + need > (double)fz.ctx->budget) return false;
    return need < 0.95 * ((double)fr + freed);
}

void solve_near(mbl_sector *sec, double eps, int nev, const mbl_opts &o, double *d_evals, double *d_evecs,
                double *d_resid, int *nconv, double *sigma_used, mbl_solve_stats *stats, cudaStream_t st,
                std::unique_ptr<Factorization> *keep) {
    auto t0 = std::chrono::steady_clock::now();
    Ctx *ctx = sec->ctx;
    int64_t n = sec->n;
    if (nev < 1 || nev > n) fail(MBL_ERR_INVALID, "nev must be in [1, dim]");
    if (!(eps >= 0.0 && eps <= 1.0)) fail(MBL_ERR_INVALID, "eps must be in [0, 1]");
    double emin, emax;
    extremal_bounds(sec, &emin, &emax);
    double hnorm = std::max(std::fabs(emin), std::fabs(emax));
    double sigma = emin + eps * (emax - emin);
    *sigma_used = sigma;
    mbl_solve_stats S{};
    if (n <= DENSE_MAX_N) {
        // tiny sectors: the whole spectrum on the device, then the nev nearest
        DVec<double> A, w;
        dense_eigen(sec, true, A, w, st);
        std::vector<double> hw(n);
        MBL_CUDA(cudaMemcpy(hw.data(), w.data(), n * sizeof(double), cudaMemcpyDeviceToHost));
        std::vector<int> idx = nearest_sorted(hw, sigma, nev);
        DVec<int> didx;
        didx.alloc(ctx, nev);
        MBL_CUDA(cudaMemcpyAsync(didx.data(), idx.data(), nev * sizeof(int), cudaMemcpyHostToDevice, st));
        k_select_cols_cm<<<nblk(n * nev), 256, 0, st>>>(n, A.data(), didx.data(), nev, d_evecs);
        MBL_LAUNCH_CHECK();
        std::vector<double> ev(nev);
        for (int j = 0; j < nev; ++j) ev[j] = hw[idx[j]];
        MBL_CUDA(cudaMemcpyAsync(d_evals, ev.data(), nev * sizeof(double), cudaMemcpyHostToDevice, st));
        // residuals via SpMV
        DVec<double> Yr, HY, part, nrm, th;
        Yr.alloc(ctx, (size_t)n * nev);
        HY.alloc(ctx, (size_t)n * nev);
        th.alloc(ctx, nev);
        k_cm_to_rm<<<nblk(n * nev), 256, 0, st>>>(n, nev, d_evecs, Yr.data());
        MBL_LAUNCH_CHECK();
        launch_spmv(sec, 0.0, Yr.data(), nev, 1, HY.data(), nev, 1, nev, st);
        MBL_CUDA(cudaMemcpyAsync(th.data(), ev.data(), nev * sizeof(double), cudaMemcpyHostToDevice, st));
        unsigned nb = nblk(n * nev);
        part.alloc(ctx, (size_t)nb * 2 * nev);
        nrm.alloc(ctx, 2 * nev);
        k_pair_resid<<<nb, 256, 0, st>>>(n, nev, Yr.data(), HY.data(), th.data(), part.data());
        MBL_LAUNCH_CHECK();
        k_reduce_parts<<<reduce_grid(2 * nev), 256, 0, st>>>((int)nb, 2 * nev, part.data(), nrm.data());
        MBL_LAUNCH_CHECK();
        std::vector<double> hn2(2 * nev), rr(nev);
        MBL_CUDA(cudaMemcpyAsync(hn2.data(), nrm.data(), 2 * nev * sizeof(double), cudaMemcpyDeviceToHost, st));
        MBL_CUDA(cudaStreamSynchronize(st));
        int nc = 0;
        double mx = 0;
        for (int j = 0; j < nev; ++j) {
            rr[j] = std::sqrt(hn2[nev + j]);
            mx = std::max(mx, rr[j] / hnorm);
            if (rr[j] <= o.tol * hnorm) ++nc;
        }
        MBL_CUDA(cudaMemcpy(d_resid, rr.data(), nev * sizeof(double), cudaMemcpyHostToDevice));
        *nconv = nc;
        S.max_resid = mx;
        S.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (stats) *stats = S;
        return;
    }
    // ---- shift-invert ----
    int p = std::max(1, std::min(32, o.block));
    int ncv = o.ncv > 0 ? o.ncv : 2 * nev + 2 * p;
    ncv = ((ncv + p - 1) / p) * p;
    ncv = std::max(ncv, ((nev + p + p - 1) / p) * p + p);
    if (ncv + p > n) fail(MBL_ERR_INVALID, "Krylov basis larger than the sector");
    if ((ncv + p) * 32 > 8192) fail(MBL_ERR_INVALID, "ncv + block too large (max 256)");
    // A target at the very edge of the spectrum (eps = 0 or 1) sits on an eigenvalue and makes
    // H - sigma singular: factor a hair outside the spectrum instead.  The window is still chosen by
    // distance to sigma; near the edge the nearest eigenvalues are the same.
    double sigma_f = sigma;
    const double guard = 1e-8 * hnorm, nudge = 1e-4 * (emax - emin);
    if (std::fabs(sigma - emin) <= guard) sigma_f = emin - nudge;
    if (std::fabs(sigma - emax) <= guard) sigma_f = emax + nudge;
    auto tf0 = std::chrono::steady_clock::now();
    // Static pivoting threshold of FP32 fronts.  By default 1e-7 ||H||: few pivots are perturbed and the
    // FP64 refactorization backs up a stalled refinement.  Where that refactorization could not fit in
    // device memory (the largest sectors), the FP32 factor must stand on its own: use the static
    // pivoting threshold sqrt(eps_FP32) ||H|| (perturbing more pivots bounds the element growth, and a
    // stable factor of a slightly perturbed matrix is a far better FGMRES preconditioner than an
    // unstable one; at L = 22 the growth falls from 5.5e5 to 4.4e3 and the refinement converges).
    double tiny_rel = o.pivot_tiny;
    if (o.precision == MBL_PREC_FP32 && tiny_rel == 0.0 && !fp64_fits_plan(*get_plan(sec), o.arena_mode, ctx))
        tiny_rel = std::sqrt((double)FLT_EPSILON / 2.0);
    S.static_pivot = tiny_rel;
    std::unique_ptr<Factorization> fz;
    if (keep && *keep && (*keep)->sec == sec && !(*keep)->trace_on &&
        ((*keep)->prec == o.precision || (*keep)->prec == MBL_PREC_FP64) &&
        (*keep)->tc_mode == o.tensor_cores && (*keep)->dataflow == (o.solve_dataflow != 0)) {
        // a live factorization of this very request (serving residency): its shift is the one the
        // earlier run settled on (moved off an eigenvalue, or FP64 after a refinement stall)
        fz = std::move(*keep);
        sigma_f = fz->sigma;
        S.factor_reused = 1;
    } else {
        fz = make_factorization(sec, sigma_f, o.precision, hnorm, o.tensor_cores, o.solve_dataflow != 0,
                                wait_limit_ns(o.wait_limit_s), o.arena_mode, tiny_rel);
    }
    S.ms_factor = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tf0).count();
    RefinedSolve op{sec, fz.get(), hnorm + std::fabs(sigma_f), o.refine_tol, o.max_refine};
    op.gmres = o.refine_mode;
    op.kmax = std::max(1, std::min(64, o.gmres_restart));
    OpFn opfn = [&](const double *X, int ldx, double *Y, cudaStream_t s) { op.apply(X, ldx, Y, p, s); };
    KrylovSchur ks(ctx, n, p, ncv);
    ks.start(o.start_seed, st);
    RitzH rr(ctx, n, ks.ldv, nev);
    std::vector<double> th, rn;
    int k_keep = std::min(ncv - p, nev + (ncv - nev) / 2);
    // The Krylov-Schur residual of a Ritz pair of (H - sigma)^-1 overestimates the residual on H
    // (the refined solves carry forward errors along the wanted directions), so it only screens:
    // convergence is decided by the Rayleigh-Ritz residuals on H.
    double screen = 1e-6;
    int restarts = 0, nc = 0;
    double mxres = INFINITY, prev_rr = INFINITY;
    int nudges = 0;  // moves of the factorization shift off an eigenvalue
    // a serving worker announces its solve phases to the solve batcher, which then waits for its
    // solves before launching a batch of the same plan
    struct BatchPhase {
        SolveBatcher *b;
        const Plan *pl = nullptr;
        int prec = 0, p = 0;
        void enter(const Factorization &f, int p_) {
            if (!b || f.dataflow || pl) return;
            pl = f.plan.get();
            prec = f.prec;
            p = p_;
            batcher_enter(b, pl, prec, p);
        }
        void leave() {
            if (pl) batcher_leave(b, pl, prec, p);
            pl = nullptr;
        }
        ~BatchPhase() { leave(); }
    } phase{ctx->batcher};
    for (;; ++restarts) {
        phase.enter(*fz, p);
        while (!ks.full()) {
            ks.expand(opfn, st);
            if (op.stalled && fz->prec == MBL_PREC_FP32 && !fp64_fits(*fz, o.arena_mode)) {
                // FP64 fronts would not fit beside what the job holds (the largest sectors): keep the FP32
                // factor and give the refinement more room instead (longer and more FGMRES cycles)
                op.stalled = false;
                op.kmax = 64;
                op.max_outer = 16;
                S.refine_escalations += 1;
            }
            if (op.stalled && fz->prec == MBL_PREC_FP32) {
                phase.leave();
                // refinement stalled near the shift: refactor with FP64 fronts.  The Krylov-Schur
                // relation built so far holds only to the accuracy of the stalled solves, and thick
                // restarts would carry that error along for good: start the iteration again.
                auto tf1 = std::chrono::steady_clock::now();
                op.fz = nullptr;
                fz.reset();  // free the FP32 fronts first: the two factors never coexist in HBM
                fz = make_factorization(sec, sigma_f, MBL_PREC_FP64, hnorm, 1, o.solve_dataflow != 0,
                                        wait_limit_ns(o.wait_limit_s), o.arena_mode);
                S.ms_factor += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tf1).count();
                op.fz = fz.get();
                op.stalled = false;
                op.clear_deflation();  // its vectors live in the basis that start() overwrites
                S.fp64_fallback = 1;
                ks.start(o.start_seed, st);
                screen = 1e-6;
                prev_rr = INFINITY;
                phase.enter(*fz, p);
            }
        }
        phase.leave();
        ks.ritz(st, th, rn);
        int mm = (int)th.size();
        if (nudges < 3) {
            // A shift within 1e-2 of the mean level spacing s of an eigenvalue (a target exactly on
            // one, or by chance close to one) makes that Ritz value of (H - sigma)^-1 dominate every
            // solve: the refinement's backward-error bound scales with |x|, which that one component
            // then sets, so the other components, the ones the iteration still needs, are accurate
            // only to about refine_tol * s / distance relative to ||H||.  At 1e-4 s that floor is
            // 1e-10 ||H||, the acceptance bound itself (an L = 16 job at 2.8e-4 s stalled there for
            // 60 restarts with 39 of 50 pairs); at 1e-2 s it is 1e-12.  Factor a tenth of a spacing
            // away from that eigenvalue (an ordinary distance) and start again; the window is still
            // chosen by distance to sigma, and the basis keeps more than nev Ritz pairs around the
            // shift.  A shift that lands on another level moves again.
            const double spacing = (emax - emin) / (double)n;
            double tmax = 0.0, tnear = 0.0;
            for (double t : th)
                if (std::fabs(t) > tmax) tmax = std::fabs(t), tnear = t;
            if (tmax * spacing > 1e2) {
                const double lam = sigma_f + 1.0 / tnear;  // the eigenvalue the shift sits on
                const double side = (sigma_f >= lam ? 1.0 : -1.0) * (nudges == 1 ? -1.0 : 1.0);
                sigma_f = lam + side * (0.1 + 0.05 * nudges) * spacing;
                ++nudges;
                S.shift_moves = nudges;
                const int prec_now = fz->prec;
                op.fz = nullptr;
                fz.reset();
                auto tf1 = std::chrono::steady_clock::now();
                fz = make_factorization(sec, sigma_f, prec_now, hnorm, o.tensor_cores, o.solve_dataflow != 0,
                                        wait_limit_ns(o.wait_limit_s), o.arena_mode,
                                        prec_now == MBL_PREC_FP32 ? tiny_rel : 0.0);
                S.ms_factor += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tf1).count();
                op.fz = fz.get();
                op.anorm = hnorm + std::fabs(sigma_f);
                op.stalled = false;
                op.clear_deflation();
                ks.start(o.start_seed, st);
                screen = 1e-6;
                prev_rr = INFINITY;
                continue;
            }
        }
        std::vector<int> order(mm);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::fabs(th[a]) > std::fabs(th[b]); });
        double worst = 0.0;
        for (int t = 0; t < nev; ++t) {
            int i = order[t];
            worst = std::max(worst, (hnorm + std::fabs(sigma_f)) * rn[i] / std::max(std::fabs(th[i]), 1e-300) / hnorm);
        }
        bool last = restarts >= o.max_restarts;
        if (worst <= screen || last) {
            rr.run(sec, ks, sigma, hnorm, o.tol, d_evecs, st);
            nc = rr.nconv;
            mxres = rr.maxres;
            if (mxres <= o.target_tol || last) break;
            // every pair already meets the acceptance bound and the residuals stopped improving
            // (less than 2x since the previous check): the attainable floor is reached
            if (nc >= nev && prev_rr <= 2.0 * mxres) break;
            prev_rr = mxres;
            screen = std::max(1e-14, std::min(screen, worst) * 0.01);
        }
        std::vector<int> keep(order.begin(), order.begin() + k_keep);
        std::sort(keep.begin(), keep.end());
        ks.restart(keep, st);
        // the kept Ritz vectors approximate the eigenvectors nearest sigma, where the factor is
        // weakest: deflate them from the refinement's preconditioner
        if (op.gmres && o.deflate) op.set_deflation(ks.V.data(), ks.ldv, std::min(k_keep, 90), st);
    }
    {
        unsigned long long tmo = 0;  // bounded waits of the dataflow solves that expired
        MBL_CUDA(cudaMemcpyAsync(&tmo, fz->counters.data() + 2, sizeof(tmo), cudaMemcpyDeviceToHost, st));
        MBL_CUDA(cudaStreamSynchronize(st));
        if (tmo != 0) {
            reset_solve_counters(*fz, st);
            fail(MBL_ERR_TIMEOUT, "a triangular-solve dependency wait timed out");
        }
    }
    MBL_CUDA(cudaMemcpyAsync(d_evals, rr.evals.data(), nev * sizeof(double), cudaMemcpyHostToDevice, st));
    MBL_CUDA(cudaMemcpyAsync(d_resid, rr.resid.data(), nev * sizeof(double), cudaMemcpyHostToDevice, st));
    MBL_CUDA(cudaStreamSynchronize(st));
    *nconv = nc;
    if (keep) *keep = std::move(fz);
    S.restarts = restarts;
    S.op_applies = op.applies;
    S.solves = op.solves;
    S.krylov_dim = ks.m;
    S.max_resid = mxres;
    S.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S;
}

// ------------------------------------------------------------------------------------------
// Rayleigh-Ritz of H on the Krylov basis V[:, 0:m]
// ------------------------------------------------------------------------------------------
RitzH::RitzH(Ctx *c, int64_t n_, int ldv, int nev_) : ctx(c), n(n_), nev(nev_) {
    HV.alloc(ctx, (size_t)n * ldv);
    Gm.alloc(ctx, (size_t)ldv * ldv);
    Gs.alloc(ctx, (size_t)ldv * ldv);
    Gsym.alloc(ctx, (size_t)ldv * ldv);
    Gr1.alloc(ctx, (size_t)ldv * ldv);
    Gr2.alloc(ctx, (size_t)ldv * ldv);
    Gr3.alloc(ctx, (size_t)ldv * ldv);
    M2.alloc(ctx, (size_t)ldv * ldv);
    Gw.alloc(ctx, ldv);
    Gwork.alloc(ctx, syev_work_doubles(ldv));
    if (ldv <= EIG_SMEM_MAX_M) Bwork.alloc(ctx, syev_bisect_work(ldv));
    Ctmp.alloc(ctx, (size_t)ldv * 32);
    work.alloc(ctx, dense_tn_work(n, ldv, 32) + 64);
    gm.alloc(ctx, 1);
    ginfo.alloc(ctx, 1);
    goff.alloc(ctx, 1);
    didx.alloc(ctx, nev);
    SKs.alloc(ctx, (size_t)ldv * nev);
    Y.alloc(ctx, (size_t)n * nev);
    HY.alloc(ctx, (size_t)n * nev);
    thd.alloc(ctx, nev);
    nb = nblk(n * nev);
    part.alloc(ctx, (size_t)nb * 2 * nev);
    nrm.alloc(ctx, 2 * nev);
    evals.assign(nev, 0.0);
    resid.assign(nev, 0.0);
    int64_t z = 0;
    MBL_CUDA(cudaMemcpy(goff.data(), &z, sizeof(int64_t), cudaMemcpyHostToDevice));
}

__global__ void k_copy_diag(int m, const double *S, double *out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) out[j] = S[(size_t)j * m + j];
}

// Residual norms of all Ritz pairs of H on an orthonormal basis V: with M2 = (HV)^T (HV),
// Q = M2 S and the Ritz pair (theta_j, V s_j), ||H V s_j - theta_j V s_j||^2 = s_j^T Q e_j - theta_j^2.
__global__ void k_ritz_all_resid(int m, const double *S, const double *Q, const double *theta, double *out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += S[(size_t)j * m + i] * Q[(size_t)j * m + i];
    out[j] = sqrt(fmax(0.0, s - theta[j] * theta[j]));
}

void RitzH::run(mbl_sector *sec, KrylovSchur &ks, double sigma, double hnorm, double tol, double *d_evecs,
                cudaStream_t st) {
    ProfScope ps_all(ctx, "ritz_h", (double)nev, st);
    int mb = ks.m;
    launch_spmv(sec, 0.0, ks.V.data(), ks.ldv, 1, HV.data(), mb, 1, mb, st);
    for (int c0 = 0; c0 < mb; c0 += 32) {
        int w = std::min(32, mb - c0);
        dense_tn(n, ks.V.data(), ks.ldv, 0, mb, HV.data(), mb, c0, w, Ctmp.data(), work.data(), st);
        copy_cols(mb, Ctmp.data(), w, 0, Gm.data() + (size_t)c0, mb, 0, w, st);
    }
    // M2 = (HV)^T (HV): residuals of every Ritz pair, to keep spurious interior Ritz values (which
    // plain Rayleigh-Ritz produces for a subspace that mixes both sides of sigma) out of the window
    for (int c0 = 0; c0 < mb; c0 += 32) {
        int w = std::min(32, mb - c0);
        dense_tn(n, HV.data(), mb, 0, mb, HV.data(), mb, c0, w, Ctmp.data(), work.data(), st);
        copy_cols(mb, Ctmp.data(), w, 0, M2.data() + (size_t)c0, mb, 0, w, st);
    }
    k_pack_sym<<<nblk((int64_t)mb * mb), 256, 0, st>>>(Gm.data(), mb, mb, Gs.data());
    MBL_LAUNCH_CHECK();
    MBL_CUDA(cudaMemcpyAsync(gm.data(), &mb, sizeof(int), cudaMemcpyHostToDevice, st));
    {
        // FP32 eigensolve (the parallel Jacobi method) refined by three Ogita-Aishima steps and
        // re-orthonormalized (Newton-Schulz) in FP64; accepted only if the nev wanted columns are
        // orthonormal and diagonalize G to FP64 accuracy, otherwise FP64 bisection and inverse
        // iteration run.  The pairs' residuals on H are recomputed below.
        ProfScope ps(ctx, "syev_rr", (double)mb, st);
        const bool fp32 = ks.ldv <= EIG_SMEM_MAX_M;
        // accept eigenvectors X (in Gs) only if the nev wanted columns are orthonormal and diagonalize
        // G to FP64 accuracy: |e_j - X^T X e_j| <= 1e-12, |off(X^T G X) e_j| <= 1e-12 max|lambda|
        // (leaves X^T G X in Gr3)
        auto check_wanted = [&]() {
            gemm_small(true, false, mb, mb, mb, 1.0, Gs.data(), mb, Gs.data(), mb, 0.0, Gr1.data(), mb, st);
            gemm_small(false, false, mb, mb, mb, 1.0, Gsym.data(), mb, Gs.data(), mb, 0.0, Gr2.data(), mb, st);
            gemm_small(true, false, mb, mb, mb, 1.0, Gs.data(), mb, Gr2.data(), mb, 0.0, Gr3.data(), mb, st);
            k_oa_colnorms<<<nblk(mb, 128), 128, 0, st>>>(mb, Gr1.data(), Gr3.data(), Gr2.data());
            MBL_LAUNCH_CHECK();
            std::vector<double> q((size_t)2 * mb), th(mb);
            MBL_CUDA(cudaMemcpyAsync(q.data(), Gr2.data(), q.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
            MBL_CUDA(cudaMemcpyAsync(th.data(), Gw.data(), mb * sizeof(double), cudaMemcpyDeviceToHost, st));
            MBL_CUDA(cudaStreamSynchronize(st));
            double amax = 0.0;
            for (double v : th) amax = std::max(amax, std::fabs(v));
            bool good = true;
            for (int j : nearest_sorted(th, sigma, nev)) good = good && q[j] <= 1e-12 && q[mb + j] <= 1e-12 * amax;
            return good;
        };
        bool ok = false;
        if (fp32) {
            MBL_CUDA(cudaMemcpyAsync(Gsym.data(), Gs.data(), (size_t)mb * mb * sizeof(double), cudaMemcpyDeviceToDevice,
                                     st));
            syev_jacobi32(1, gm.data(), goff.data(), goff.data(), Gs.data(), Gw.data(), ks.ldv, ginfo.data(), st);
            refine_eig(mb, Gsym.data(), Gs.data(), Gw.data(), 3, Gr1.data(), Gr2.data(), Gr3.data(), st);
            for (int it = 0; it < 2; ++it) {  // X <- 1.5 X - 0.5 X (X^T X)
                gemm_small(true, false, mb, mb, mb, 1.0, Gs.data(), mb, Gs.data(), mb, 0.0, Gr1.data(), mb, st);
                MBL_CUDA(cudaMemcpyAsync(Gr2.data(), Gs.data(), (size_t)mb * mb * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
                gemm_small(false, false, mb, mb, mb, -0.5, Gr2.data(), mb, Gr1.data(), mb, 1.5, Gs.data(), mb, st);
            }
            ok = check_wanted();
            if (!ok) {
                // FP64 by bisection and inverse iteration, under the same check
                ProfScope ps2(ctx, "syev_rr_bisect", (double)mb, st);
                MBL_CUDA(cudaMemcpyAsync(Gs.data(), Gsym.data(), (size_t)mb * mb * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
                syev_bisect(mb, Gs.data(), Gw.data(), Bwork.data(), st);
                ok = check_wanted();
            }
            if (ok) {
                // the Ritz values are the Rayleigh quotients of the final vectors: diag(X^T G X)
                k_copy_diag<<<nblk(mb, 128), 128, 0, st>>>(mb, Gr3.data(), Gw.data());
                MBL_LAUNCH_CHECK();
            } else {
                MBL_CUDA(cudaMemcpyAsync(Gs.data(), Gsym.data(), (size_t)mb * mb * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
            }
        }
        if (!ok) {
            ProfScope ps2(ctx, "syev_rr_fp64", (double)mb, st);
            syev_batched(1, gm.data(), goff.data(), goff.data(), Gs.data(), Gw.data(), 1, nullptr, ks.ldv,
                         Gwork.data(), ginfo.data(), st);
        }
    }
    gemm_small(false, false, mb, mb, mb, 1.0, M2.data(), mb, Gs.data(), mb, 0.0, Gr1.data(), mb, st);
    k_ritz_all_resid<<<nblk(mb, 128), 128, 0, st>>>(mb, Gs.data(), Gr1.data(), Gw.data(), Gr2.data());
    MBL_LAUNCH_CHECK();
    std::vector<double> gth(mb), gres(mb);
    MBL_CUDA(cudaMemcpyAsync(gth.data(), Gw.data(), mb * sizeof(double), cudaMemcpyDeviceToHost, st));
    MBL_CUDA(cudaMemcpyAsync(gres.data(), Gr2.data(), mb * sizeof(double), cudaMemcpyDeviceToHost, st));
    MBL_CUDA(cudaStreamSynchronize(st));
    // candidates: Ritz pairs with residual <= 1e-3 ||H|| (a spurious value sits near 0.1 ||H||)
    std::vector<int> cand;
    for (int j = 0; j < mb; ++j)
        if (gres[j] <= 1e-3 * hnorm) cand.push_back(j);
    std::vector<int> idx;
    if ((int)cand.size() >= nev) {
        std::vector<double> cth(cand.size());
        for (size_t u = 0; u < cand.size(); ++u) cth[u] = gth[cand[u]];
        for (int u : nearest_sorted(cth, sigma, nev)) idx.push_back(cand[u]);
    } else {
        idx = nearest_sorted(gth, sigma, nev);
    }
    MBL_CUDA(cudaMemcpyAsync(didx.data(), idx.data(), nev * sizeof(int), cudaMemcpyHostToDevice, st));
    k_gather_S<<<nblk((int64_t)mb * nev), 256, 0, st>>>(Gs.data(), mb, didx.data(), nev, SKs.data());
    MBL_LAUNCH_CHECK();
    dense_nn(n, ks.V.data(), ks.ldv, mb, SKs.data(), nev, Y.data(), nev, 0, st);
    launch_spmv(sec, 0.0, Y.data(), nev, 1, HY.data(), nev, 1, nev, st);
    for (int j = 0; j < nev; ++j) evals[j] = gth[idx[j]];
    MBL_CUDA(cudaMemcpyAsync(thd.data(), evals.data(), nev * sizeof(double), cudaMemcpyHostToDevice, st));
    k_pair_resid<<<nb, 256, 0, st>>>(n, nev, Y.data(), HY.data(), thd.data(), part.data());
    MBL_LAUNCH_CHECK();
    k_reduce_parts<<<reduce_grid(2 * nev), 256, 0, st>>>((int)nb, 2 * nev, part.data(), nrm.data());
    MBL_LAUNCH_CHECK();
    k_scale_cols_to_cm<<<nblk(n * nev), 256, 0, st>>>(n, nev, Y.data(), nrm.data(), d_evecs);
    MBL_LAUNCH_CHECK();
    std::vector<double> hn2(2 * nev);
    MBL_CUDA(cudaMemcpyAsync(hn2.data(), nrm.data(), 2 * nev * sizeof(double), cudaMemcpyDeviceToHost, st));
    MBL_CUDA(cudaStreamSynchronize(st));
    nconv = 0;
    maxres = 0.0;
    for (int j = 0; j < nev; ++j) {
        resid[j] = std::sqrt(hn2[nev + j] / hn2[j]);
        maxres = std::max(maxres, resid[j] / hnorm);
        if (resid[j] <= tol * hnorm) ++nconv;
    }
}

}  // namespace mbl
