// noalloc.cu -- half-chain entanglement entropy with no device allocation.
//
// Same quantity as the S^E output of observables_dev (characterization section: Schmidt weights
// of the half chain A = sites 0..L/2-1 from the Gram matrices M M^T of the reshaped vector, blocks
// by the magnetization n_A of A), for callers that cannot allocate device memory: a caller running
// at the edge of the HBM budget (a serving worker whose admitted jobs hold all of it, where any
// further cudaMalloc fails) or one that must not stall other streams (cudaFree synchronizes the
// whole device).  Its scratch is one file-scope __device__ array of NA_SCRATCH_BYTES (12 MiB),
// enough for L <= 16 and nev <= 64; larger requests are rejected.  The array's address is taken
// with cudaGetSymbolAddress once per device when a context is created.  The index tables that
// observables_dev precomputes on the host are recomputed on the device from the combinatorial
// number system, so nothing is copied in either.  The scratch is shared by every caller on the
// device: overlapping calls (any stream, any thread) race and must be serialized by the caller.
#include <mutex>

#include "observables.h"

namespace mbl {

namespace {

constexpr int NA_MAX_L = 16;
constexpr int NA_MAX_NEV = 64;
constexpr size_t NA_SCRATCH_BYTES = (size_t)12 << 20;

static __device__ __align__(256) unsigned char g_na_scratch[NA_SCRATCH_BYTES];

std::mutex g_na_mu;
void *g_na_addr[64] = {};  // per device; null until set up
bool g_na_tried[64] = {};

// C(p, t) for p <= 16 into a 17 x 9 table
__device__ void fill_binom(int64_t (*B)[9]) {
    for (int t = threadIdx.x; t < 17 * 9; t += blockDim.x) {
        int p = t / 9, k = t % 9;
        int64_t r = 0;
        if (k <= p) {
            r = 1;
            for (int i = 1; i <= k; ++i) r = r * (p - k + i) / i;
        }
        B[p][k] = r;
    }
}

// k-th h-bit word with t set bits in ascending order (colex unranking)
__device__ uint32_t unrank_word(int64_t k, int t, int h, const int64_t (*B)[9]) {
    uint32_t s = 0;
    for (int p = h - 1; p >= 0 && t > 0; --p) {
        if (B[p][t] <= k) {
            s |= 1u << p;
            k -= B[p][t];
            --t;
        }
    }
    return s;
}

// index of an L-bit word with L/2 set bits among all such words in ascending order
__device__ int64_t rank_word(uint32_t s, const int64_t (*B)[9]) {
    int64_t r = 0;
    int t = 0;
    while (s) {
        int p = __ffs(s) - 1;
        ++t;
        r += B[p][t];
        s &= s - 1;
    }
    return r;
}

// per matrix b = j * nb + q: order, Gram offset, eigenvalue offset
__global__ void k_na_meta(int h, int nev, int64_t n, int *m, int64_t *goff, int64_t *woff) {
    __shared__ int64_t B[17][9];
    fill_binom(B);
    __syncthreads();
    const int nb = h + 1;
    for (int b = threadIdx.x; b < nev * nb; b += blockDim.x) {
        const int j = b / nb, q = b % nb;
        int64_t g = (int64_t)j * n, w = (int64_t)j << h;
        for (int qq = 0; qq < q; ++qq) {
            g += B[h][qq] * B[h][qq];
            w += B[h][qq];
        }
        m[b] = (int)B[h][q];
        goff[b] = g;
        woff[b] = w;
    }
}

// CTA (vector j, block q): Gram matrix of the n_A = q block, normalized by |y|^2.  The norm is
// summed in the same order as the participation-entropy kernel so that both entry points agree.
__global__ void __launch_bounds__(256) k_na_gram(int h, int64_t n, const double *Y, const int64_t *goff, double *G) {
    __shared__ int64_t B[17][9];
    __shared__ double Ms[70 * 70];
    __shared__ double ra[32];
    __shared__ double s_inv;
    fill_binom(B);
    const int nb = h + 1;
    const int j = blockIdx.x / nb, q = blockIdx.x % nb;
    const double *y = Y + (int64_t)j * n;
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a = __dadd_rn(a, __dmul_rn(y[i], y[i]));
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) ra[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) A += ra[i];
        s_inv = 1.0 / A;
    }
    const int da = (int)B[h][q];
    for (int t = threadIdx.x; t < da * da; t += blockDim.x) {
        const int ia = t / da, ib = t % da;
        const uint32_t s = unrank_word(ia, q, h, B) | (unrank_word(ib, h - q, h, B) << h);
        Ms[t] = y[rank_word(s, B)];
    }
    __syncthreads();
    const double inv = s_inv;
    double *g = G + goff[blockIdx.x];
    for (int t = threadIdx.x; t < da * da; t += blockDim.x) {
        const int r = t % da, c = t / da;
        if (r < c) continue;
        double sum = 0.0;
        for (int b = 0; b < da; ++b) sum += Ms[r * da + b] * Ms[c * da + b];
        sum *= inv;
        g[(int64_t)c * da + r] = sum;
        g[(int64_t)r * da + c] = sum;
    }
}

// S_E of each vector from its blocks' Schmidt weights; NaN where the eigensolver flagged a block
// as not converged (info != 0), so that a wrong entropy is never returned silently.
__global__ void k_na_entropy(int h, int nev, const int64_t *woff, const double *lam, const int *info, double *se) {
    __shared__ int64_t B[17][9];
    fill_binom(B);
    __syncthreads();
    const int nb = h + 1;
    for (int j = threadIdx.x; j < nev; j += blockDim.x) {
        double S = 0.0;
        bool bad = false;
        for (int q = 0; q < nb; ++q) {
            bad = bad || info[(int64_t)j * nb + q] != 0;
            const double *l = lam + woff[(int64_t)j * nb + q];
            for (int i = 0; i < (int)B[h][q]; ++i)
                if (l[i] > 1e-15) S -= l[i] * log(l[i]);
        }
        se[j] = bad ? nan("") : S;
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Take the scratch address on a device (context creation).  A failure leaves the entry point
// unavailable on that device (it then returns MBL_ERR_CUDA) without failing the context.
void noalloc_setup(int device) {
    if (device < 0 || device >= 64) return;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (g_na_tried[device]) return;
    g_na_tried[device] = true;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    // kernels load lazily on first use, and loading takes device memory: load the ones this path
    // launches now, so that no call allocates
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_meta);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_gram);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_entropy);
    if (e == cudaSuccess) e = syev_preload();
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    g_na_addr[device] = p;
}

void entanglement_noalloc(Ctx *ctx, int L, int nev, const double *d_evecs, double *d_se, cudaStream_t st) {
    if (L < 2 || L > NA_MAX_L || (L & 1)) fail(MBL_ERR_INVALID, "static-scratch entropy: L must be even, 2..16");
    const int h = L / 2, nb = h + 1;
    int64_t n = 1;
    for (int i = 1; i <= h; ++i) n = n * (h + i) / i;
    if (nev < 1 || nev > NA_MAX_NEV || nev > n) fail(MBL_ERR_INVALID, "static-scratch entropy: nev in [1, 64]");
    void *base;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        base = (ctx->device >= 0 && ctx->device < 64) ? g_na_addr[ctx->device] : nullptr;
    }
    if (!base) fail(MBL_ERR_CUDA, "static-scratch entropy: scratch address unavailable on this device");
    int mmax = 1;
    for (int i = 1; i <= h / 2; ++i) mmax = mmax * (h - h / 2 + i) / i;  // C(h, h/2)
    const int64_t batch = (int64_t)nev * nb;
    const size_t wstride = syev_work_doubles(mmax, false);
    size_t off = 0;
    const size_t oG = off;
    off = align256(off + sizeof(double) * (size_t)nev * n);
    const size_t oLam = off;
    off = align256(off + sizeof(double) * ((size_t)nev << h));
    const size_t oWork = off;
    off = align256(off + sizeof(double) * wstride * batch);
    const size_t oM = off;
    off = align256(off + sizeof(int) * batch);
    const size_t oGoff = off;
    off = align256(off + sizeof(int64_t) * batch);
    const size_t oWoff = off;
    off = align256(off + sizeof(int64_t) * batch);
    const size_t oInfo = off;
    off = align256(off + sizeof(int) * batch);
    if (off > NA_SCRATCH_BYTES) fail(MBL_ERR_INVALID, "static-scratch entropy: request exceeds the 12 MiB scratch");
    unsigned char *S = static_cast<unsigned char *>(base);
    double *G = reinterpret_cast<double *>(S + oG), *lam = reinterpret_cast<double *>(S + oLam);
    double *work = reinterpret_cast<double *>(S + oWork);
    int *m = reinterpret_cast<int *>(S + oM), *info = reinterpret_cast<int *>(S + oInfo);
    int64_t *goff = reinterpret_cast<int64_t *>(S + oGoff), *woff = reinterpret_cast<int64_t *>(S + oWoff);
    // the per-matrix convergence flags are the only scratch read before it is written in a call
    MBL_CUDA(cudaMemsetAsync(info, 0, sizeof(int) * batch, st));
    k_na_meta<<<1, 256, 0, st>>>(h, nev, n, m, goff, woff);
    MBL_LAUNCH_CHECK();
    k_na_gram<<<(unsigned)batch, 256, 0, st>>>(h, n, d_evecs, goff, G);
    MBL_LAUNCH_CHECK();
    syev_batched((int)batch, m, goff, woff, G, lam, 0, nullptr, mmax, work, info, st);
    k_na_entropy<<<1, 64, 0, st>>>(h, nev, woff, lam, info, d_se);
    MBL_LAUNCH_CHECK();
}

}  // namespace mbl
