// sector.cu -- disorder fields, combinadic basis, CSR Hamiltonian and FP64 SpMV on the device.
//
// Eq. 1 of arXiv:1411.0660 restricted to a magnetization sector (numerical-method section: the
// S^z = 0 sector of even L, the S^z = 1 sector of odd L; here any number nup of up spins).
// All of it is integer bit manipulation plus a fixed-order FP64 diagonal, so the result is
// bit-exact: the basis is the colex enumeration of nup-subsets (the combinatorial number
// system), the column of a flipped state is its combinadic rank, and the diagonal is summed in
// a fixed order with explicitly rounded multiplies and adds (no FMA contraction).
#include "mbl_internal.h"

namespace mbl {

__constant__ uint32_t c_binom[33][33];

void upload_binomials() {
    uint32_t b[33][33] = {{0}};
    for (int n = 0; n <= 32; ++n) {
        b[n][0] = 1;
        for (int k = 1; k <= n; ++k) {
            uint64_t v = (uint64_t)b[n - 1][k - 1] + (k <= n - 1 ? b[n - 1][k] : 0);
            b[n][k] = v > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)v;
        }
    }
    MBL_CUDA(cudaMemcpyToSymbol(c_binom, b, sizeof(b)));
}

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): golden-gamma increment, two xor-shift-multiply
// rounds, final xor-shift.  h_i = h (2 u_i - 1), u_i = (z_i >> 11) 2^-53.
__global__ void k_fields(int L, double h, uint64_t seed, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint64_t st = seed;
    for (int i = 0; i < L; ++i) {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        double u = __dmul_rn((double)(z >> 11), 1.0 / 9007199254740992.0);
        out[i] = __dmul_rn(h, __dsub_rn(__dmul_rn(2.0, u), 1.0));
    }
}

void launch_fields(int L, double h, uint64_t seed, double *d_out, cudaStream_t st) {
    k_fields<<<1, 32, 0, st>>>(L, h, seed, d_out);
    MBL_LAUNCH_CHECK();
}

// rank(s) = sum over set bits (t-th from the bottom, t = 1, 2, ...) at position p of C(p, t)
__device__ __forceinline__ int64_t combinadic_rank(uint32_t s) {
    int64_t r = 0;
    int t = 0;
    while (s) {
        int p = __ffs(s) - 1;
        ++t;
        r += c_binom[p][t];
        s &= s - 1;
    }
    return r;
}

// inverse: the K-subset of {0..L-1} of colex rank r
__device__ __forceinline__ uint32_t combinadic_unrank(int L, int K, int64_t r) {
    uint32_t s = 0;
    int p = L - 1;
    for (int t = K; t >= 1; --t) {
        while ((int64_t)c_binom[p][t] > r) --p;
        s |= 1u << p;
        r -= c_binom[p][t];
        --p;
    }
    return s;
}

__global__ void k_unrank(int L, int nup, int64_t n, uint32_t *states) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) states[k] = combinadic_unrank(L, nup, k);
}

__global__ void k_rank(int L, int nup, const uint32_t *in, int64_t count, int64_t *out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    uint32_t s = in[k];
    bool ok = (L >= 32 || (s >> L) == 0) && __popc(s) == nup;
    out[k] = ok ? combinadic_rank(s) : -1;
}

// The entries of row k (columns ascending, duplicates merged).  Returns the count.
__device__ int row_entries(int L, uint32_t s, int64_t k, const double *hf, double J, int64_t *cols,
                           double *vals) {
    int n_al = 0, n_anti = 0, cnt = 0;
    for (int i = 0; i < L; ++i) {
        int j = (i + 1 == L) ? 0 : i + 1;
        uint32_t bi = (s >> i) & 1u, bj = (s >> j) & 1u;
        if (bi == bj) {
            ++n_al;
            continue;
        }
        ++n_anti;
        cols[cnt] = combinadic_rank(s ^ (1u << i) ^ (1u << j));
        vals[cnt] = __dmul_rn(0.5, J);
        ++cnt;
    }
    double d = __dmul_rn(__dmul_rn(0.25, J), (double)(n_al - n_anti));
    for (int i = 0; i < L; ++i) d = __dadd_rn(d, __dmul_rn(((s >> i) & 1u) ? 0.5 : -0.5, hf[i]));
    cols[cnt] = k;
    vals[cnt] = d;
    ++cnt;
    for (int a = 1; a < cnt; ++a) {
        int64_t cc = cols[a];
        double vv = vals[a];
        int b = a - 1;
        while (b >= 0 && cols[b] > cc) {
            cols[b + 1] = cols[b];
            vals[b + 1] = vals[b];
            --b;
        }
        cols[b + 1] = cc;
        vals[b + 1] = vv;
    }
    int m = 0;
    for (int a = 0; a < cnt; ++a) {
        if (m > 0 && cols[m - 1] == cols[a]) {
            vals[m - 1] = __dadd_rn(vals[m - 1], vals[a]);
            continue;
        }
        cols[m] = cols[a];
        vals[m] = vals[a];
        ++m;
    }
    return m;
}

__global__ void k_row_count(int L, int64_t n, const uint32_t *states, const double *hf, double J,
                            int32_t *counts) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t c[34];
    double v[34];
    counts[k] = row_entries(L, states[k], k, hf, J, c, v);
}

__global__ void k_row_fill(int L, int64_t n, const uint32_t *states, const double *hf, double J,
                           const int64_t *rowptr, int32_t *col, double *val) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t c[34];
    double v[34];
    int m = row_entries(L, states[k], k, hf, J, c, v);
    int64_t p = rowptr[k];
    for (int a = 0; a < m; ++a) {
        col[p + a] = (int32_t)c[a];
        val[p + a] = v[a];
    }
}

// ---- exclusive scan of int32 counts into int64 offsets (three passes) ----
constexpr int SCAN_B = 1024;

__global__ void k_scan_blocksum(const int32_t *in, int64_t n, int64_t *bsum) {
    __shared__ int64_t sh[SCAN_B / 32];
    int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t w = sh[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = w;
    }
}

__global__ void k_scan_serial(int64_t *bsum, int64_t nb) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t run = 0;
    for (int64_t b = 0; b < nb; ++b) {
        int64_t v = bsum[b];
        bsum[b] = run;
        run += v;
    }
    bsum[nb] = run;
}

__global__ void k_scan_apply(const int32_t *in, int64_t n, const int64_t *bsum, int64_t *out) {
    __shared__ int64_t warp_tot[SCAN_B / 32];
    int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t v = i < n ? in[i] : 0, x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = warp_tot[lane], s = t;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_tot[lane] = s - t;
    }
    __syncthreads();
    int64_t excl = bsum[blockIdx.x] + warp_tot[w] + x - v;
    if (i < n) out[i] = excl;
    if (i == n - 1) out[n] = excl + v;
}

void build_sector_device(mbl_sector *sec, cudaStream_t st) {
    Ctx *ctx = sec->ctx;
    int64_t n = sec->n;
    sec->states.alloc(ctx, n);
    sec->rowptr.alloc(ctx, n + 1);
    int thr = 256;
    int64_t g = (n + thr - 1) / thr;
    k_unrank<<<(unsigned)g, thr, 0, st>>>(sec->L, sec->nup, n, sec->states.data());
    MBL_LAUNCH_CHECK();
    DVec<int32_t> counts;
    counts.alloc(ctx, n);
    k_row_count<<<(unsigned)g, thr, 0, st>>>(sec->L, n, sec->states.data(), sec->d_hfield.data(), sec->J,
                                             counts.data());
    MBL_LAUNCH_CHECK();
    int64_t nb = (n + SCAN_B - 1) / SCAN_B;
    DVec<int64_t> bsum;
    bsum.alloc(ctx, nb + 1);
    k_scan_blocksum<<<(unsigned)nb, SCAN_B, 0, st>>>(counts.data(), n, bsum.data());
    MBL_LAUNCH_CHECK();
    k_scan_serial<<<1, 32, 0, st>>>(bsum.data(), nb);
    MBL_LAUNCH_CHECK();
    k_scan_apply<<<(unsigned)nb, SCAN_B, 0, st>>>(counts.data(), n, bsum.data(), sec->rowptr.data());
    MBL_LAUNCH_CHECK();
    MBL_CUDA(cudaMemcpyAsync(&sec->nnz, sec->rowptr.data() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MBL_CUDA(cudaStreamSynchronize(st));
    sec->col.alloc(ctx, sec->nnz);
    sec->val.alloc(ctx, sec->nnz);
    k_row_fill<<<(unsigned)g, thr, 0, st>>>(sec->L, n, sec->states.data(), sec->d_hfield.data(), sec->J,
                                            sec->rowptr.data(), sec->col.data(), sec->val.data());
    MBL_LAUNCH_CHECK();
    MBL_CUDA(cudaStreamSynchronize(st));
}

void launch_rank(int L, int nup, const uint32_t *d_states, int64_t count, int64_t *d_ranks, cudaStream_t st) {
    if (count <= 0) return;
    k_rank<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(L, nup, d_states, count, d_ranks);
    MBL_LAUNCH_CHECK();
}

// One thread per (row, rhs column): the row's (col, val) pairs are read once per warp-row group
// and broadcast; x gathers of one row's p columns are contiguous for row-major blocks.
__global__ void k_spmv(int64_t n, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                       const double *__restrict__ val, double shift, const double *__restrict__ x,
                       int64_t xs_r, int64_t xs_c, double *__restrict__ y, int64_t ys_r, int64_t ys_c, int p) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t / p;
    int q = (int)(t - i * p);
    if (i >= n) return;
    double s = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s = fma(val[e], x[(int64_t)col[e] * xs_r + q * xs_c], s);
    y[i * ys_r + q * ys_c] = s - shift * x[i * xs_r + q * xs_c];
}

void launch_spmv(const mbl_sector *sec, double shift, const double *x, int64_t xs_r, int64_t xs_c, double *y,
                 int64_t ys_r, int64_t ys_c, int p, cudaStream_t st) {
    int64_t tot = sec->n * p;
    if (tot == 0) return;
    k_spmv<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(sec->n, sec->rowptr.data(), sec->col.data(),
                                                          sec->val.data(), shift, x, xs_r, xs_c, y, ys_r,
                                                          ys_c, p);
    MBL_LAUNCH_CHECK();
}

}  // namespace mbl
