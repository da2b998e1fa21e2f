// observables.cu -- eigenvector observables of arXiv:1411.0660, characterization section:
//   (i)   gap ratio r^(n) = min(d_n, d_{n+1}) / max(d_n, d_{n+1}), d_n = E_n - E_{n-1};
//   (iii) participation entropy S_1^P = -sum_i p_i ln p_i, p_i = |<i|n>|^2 in the S^z basis;
//   (ii)  half-chain entanglement entropy S^E = -Tr rho_A ln rho_A for A = sites 0..L/2-1;
// and, in observables_extra_dev: the Kullback-Leibler divergence KL = sum_i p_i ln(p_i / q_i) of
// adjacent eigenvectors (i), S_q^P = ln(sum_i p_i^q) / (1 - q) (iii), the bipartite fluctuation
// F = <(S^z_A)^2> - <S^z_A>^2 (ii), and the dynamic spin fraction f = 1 - |<M>|^2 / <M^+ M>,
// M = sum_j S^z_j e^{2 pi i j / L}, of the supplementary section.  S^z_A and M are diagonal in the
// S^z basis, so all are reductions over the weights p_i = y_i^2 / |y|^2.
// For S^E the vector is split by the magnetization n_A of the half chain: the block
// M_{n_A}[a][b] = psi(a + b 2^{L/2}) (a with n_A up spins, b with L/2 - n_A) has Gram matrix
// M M^T whose eigenvalues are the Schmidt weights of that block; all blocks of all vectors go to
// one batched eigenvalue launch.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "observables.h"

namespace mbl {

__global__ void k_gap_ratio(int nev, const double *ev, double *r, double *rmean) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    int cnt = 0;
    for (int k = 1; k + 1 < nev; ++k) {
        double d0 = ev[k] - ev[k - 1], d1 = ev[k + 1] - ev[k];
        double mx = d0 > d1 ? d0 : d1, mn = d0 > d1 ? d1 : d0;
        if (mx == 0.0) {
            r[k - 1] = NAN;
            continue;
        }
        r[k - 1] = mn / mx;
        s += r[k - 1];
        ++cnt;
    }
    if (rmean) *rmean = cnt > 0 ? s / cnt : NAN;
}

// One CTA per vector: A = sum y^2, B = sum y^2 ln y^2; S = ln A - B / A.
__global__ void k_s1p(int64_t n, const double *Y, double *s1p, double *nrm2) {
    __shared__ double ra[32], rb[32];
    const double *y = Y + (int64_t)blockIdx.x * n;
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double v = y[i] * y[i];
        a += v;
        if (v > 0.0) b += v * log(v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { ra[w] = a; rb[w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { A += ra[i]; B += rb[i]; }
        s1p[blockIdx.x] = log(A) - B / A;
        nrm2[blockIdx.x] = A;
    }
}

// Gram matrices: CTA (vector j, block q) writes G_q (dA x dA, column-major) normalized by |y|^2.
__global__ void k_gram(int64_t n, int nblk, const double *Y, const double *nrm2, const int32_t *idx,
                       const int64_t *boff, const int32_t *dA, const int32_t *dB, const int64_t *goff, double *G) {
    extern __shared__ double Ms[];
    const int j = blockIdx.x / nblk, q = blockIdx.x % nblk;
    const int da = dA[q], db = dB[q];
    const double *y = Y + (int64_t)j * n;
    const int32_t *ix = idx + boff[q];
    const double inv = 1.0 / nrm2[j];
    double *g = G + goff[(int64_t)j * nblk + q];
    const bool in_smem = (int64_t)da * db <= 12288;
    if (in_smem) {
        for (int t = threadIdx.x; t < da * db; t += blockDim.x) Ms[t] = y[ix[t]];
        __syncthreads();
    }
    for (int t = threadIdx.x; t < da * da; t += blockDim.x) {
        int r = t % da, c = t / da;
        if (r < c) continue;
        double s = 0.0;
        if (in_smem)
            for (int b = 0; b < db; ++b) s += Ms[r * db + b] * Ms[c * db + b];
        else
            for (int b = 0; b < db; ++b) s += y[ix[r * db + b]] * y[ix[c * db + b]];
        s *= inv;
        g[(int64_t)c * da + r] = s;
        g[(int64_t)r * da + c] = s;
    }
}

// S_E of vector j from the Schmidt weights of its nblk blocks; NaN if the eigensolver reported a
// block it did not converge (info != 0), so that a wrong value is never returned silently.
__global__ void k_entropy_sum(int nev, int nblk, const int32_t *dA, const int64_t *woff, const double *lam,
                              const int *info, double *se) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nev) return;
    double S = 0.0;
    bool bad = false;
    for (int q = 0; q < nblk; ++q) {
        bad = bad || info[(int64_t)j * nblk + q] != 0;
        const double *l = lam + woff[(int64_t)j * nblk + q];
        for (int i = 0; i < dA[q]; ++i)
            if (l[i] > 1e-15) S -= l[i] * log(l[i]);
    }
    se[j] = bad ? nan("") : S;
}

static int64_t host_rank(uint32_t s) {
    int64_t r = 0;
    int t = 0;
    while (s) {
        int p = __builtin_ctz(s);
        ++t;
        r += host_binom(p, t);
        s &= s - 1;
    }
    return r;
}

// Per basis state: m_A = S^z of sites 0 .. floor(L/2)-1 and M = sum_j S^z_j e^{2 pi i j / L}.
__global__ void k_state_tables(int64_t n, int L, const uint32_t *states, double *mA, double *Mre, double *Mim) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t s = states[i];
    mA[i] = 0.5 * (double)(2 * __popc(s & ((1u << (L / 2)) - 1u)) - L / 2);
    double mr = 0.0, mi = 0.0;
    for (int j = 0; j < L; ++j) {
        double sj, cj;
        sincospi(2.0 * j / L, &sj, &cj);
        const double sz = ((s >> j) & 1u) ? 0.5 : -0.5;
        mr += sz * cj;
        mi += sz * sj;
    }
    Mre[i] = mr;
    Mim[i] = mi;
}

EntTables &ent_tables(Ctx *ctx, int L, int nup) {
    const int key = sector_key(L, nup);
    auto it = ctx->ent.find(key);
    if (it != ctx->ent.end()) return *it->second;
    auto T = std::make_shared<EntTables>();
    // A = sites 0 .. floor(L/2) - 1 (the low bits), B = the rest
    int LA = L / 2, LB = L - L / 2;
    std::vector<int32_t> idx, da, db;
    std::vector<int64_t> boff;
    for (int nA = 0; nA <= LA; ++nA) {
        int nB = nup - nA;
        if (nB < 0 || nB > LB) continue;
        std::vector<uint32_t> as, bs;
        for (uint32_t a = 0; a < (1u << LA); ++a) if (__builtin_popcount(a) == nA) as.push_back(a);
        for (uint32_t b = 0; b < (1u << LB); ++b) if (__builtin_popcount(b) == nB) bs.push_back(b);
        boff.push_back((int64_t)idx.size());
        da.push_back((int32_t)as.size());
        db.push_back((int32_t)bs.size());
        for (uint32_t a : as)
            for (uint32_t b : bs) idx.push_back((int32_t)host_rank(a | (b << LA)));
    }
    {
        std::vector<uint32_t> st;
        st.reserve((size_t)host_binom(L, nup));
        for (uint32_t s = 0; s < (1u << L); ++s)
            if (__builtin_popcount(s) == nup) st.push_back(s);
        T->d_states.alloc(ctx, st.size());
        MBL_CUDA(cudaMemcpy(T->d_states.data(), st.data(), st.size() * 4, cudaMemcpyHostToDevice));
        T->d_mA.alloc(ctx, st.size());
        T->d_Mre.alloc(ctx, st.size());
        T->d_Mim.alloc(ctx, st.size());
        k_state_tables<<<(unsigned)((st.size() + 255) / 256), 256, 0, ctx->stream>>>((int64_t)st.size(), L,
                                                                                T->d_states.data(), T->d_mA.data(),
                                                                                T->d_Mre.data(), T->d_Mim.data());
        MBL_LAUNCH_CHECK();
        MBL_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    T->nblk = (int)da.size();
    T->dA = da;
    T->dAmax = *std::max_element(da.begin(), da.end());
    T->d_idx.alloc(ctx, idx.size());
    T->d_boff.alloc(ctx, boff.size());
    T->d_dA.alloc(ctx, da.size());
    T->d_dB.alloc(ctx, db.size());
    MBL_CUDA(cudaMemcpy(T->d_idx.data(), idx.data(), idx.size() * 4, cudaMemcpyHostToDevice));
    MBL_CUDA(cudaMemcpy(T->d_boff.data(), boff.data(), boff.size() * 8, cudaMemcpyHostToDevice));
    MBL_CUDA(cudaMemcpy(T->d_dA.data(), da.data(), da.size() * 4, cudaMemcpyHostToDevice));
    MBL_CUDA(cudaMemcpy(T->d_dB.data(), db.data(), db.size() * 4, cudaMemcpyHostToDevice));
    EntTables &ref = *T;
    ctx->ent[key] = T;
    return ref;
}

constexpr int OBS_NS = 7;  // weighted sums per vector: y^2, (y^2)^q, m_A, m_A^2, Re M, Im M, |M|^2

// CTA (chunk c, vector j): partial sums of the chunk's rows, part[(j * nch + c) * OBS_NS + k].
__global__ void __launch_bounds__(256) k_moments_part(int64_t n, int nch, const double *Y, const double *mA,
                                                      const double *Mre, const double *Mim, double q, double *part) {
    __shared__ double red[OBS_NS][8];
    const int j = blockIdx.y, c = blockIdx.x;
    const int64_t per = (n + nch - 1) / nch, r0 = (int64_t)c * per, r1 = min(n, r0 + per);
    const double *y = Y + (int64_t)j * n;
    double v[OBS_NS] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double w = y[i] * y[i];
        const double a = mA[i], mr = Mre[i], mi = Mim[i];
        v[0] += w;
        if (w > 0.0) v[1] += q == 2.0 ? w * w : pow(w, q);
        v[2] += w * a;
        v[3] += w * a * a;
        v[4] += w * mr;
        v[5] += w * mi;
        v[6] += w * (mr * mr + mi * mi);
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < OBS_NS; ++k) {
        double t = v[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) red[k][wp] = t;
    }
    __syncthreads();
    if (threadIdx.x < OBS_NS) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += red[threadIdx.x][i];
        part[((int64_t)j * nch + c) * OBS_NS + threadIdx.x] = t;
    }
}

// Thread j: chunk sums in order, then S_q^P, F, f and |y_j|^2.
__global__ void k_moments_fin(int nev, int nch, const double *part, double q, double *sqp, double *fluct,
                              double *dynf, double *nrm2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nev) return;
    double t[OBS_NS] = {0, 0, 0, 0, 0, 0, 0};
    for (int c = 0; c < nch; ++c)
        for (int k = 0; k < OBS_NS; ++k) t[k] += part[((int64_t)j * nch + c) * OBS_NS + k];
    const double A = t[0];
    sqp[j] = (log(t[1]) - q * log(A)) / (1.0 - q);
    const double m1 = t[2] / A;
    fluct[j] = t[3] / A - m1 * m1;
    dynf[j] = t[6] == 0.0 ? NAN : 1.0 - (t[4] * t[4] + t[5] * t[5]) / (A * t[6]);
    nrm2[j] = A;
}

// CTA (chunk c, pair j = (j, j + 1)): partial sum of y_j^2 (ln y_j^2 - ln y_j+1^2) over the terms with
// y_j != 0, and whether such a term has y_j+1 = 0; part[(j * nch + c) * 2 + {0, 1}].
__global__ void __launch_bounds__(256) k_kl_part(int64_t n, int nch, const double *Y, double *part) {
    __shared__ double red[8];
    __shared__ int rinf[8];
    const int j = blockIdx.y, c = blockIdx.x;
    const int64_t per = (n + nch - 1) / nch, r0 = (int64_t)c * per, r1 = min(n, r0 + per);
    const double *y = Y + (int64_t)j * n, *z = y + n;
    double a = 0.0;
    int inf = 0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double p = y[i] * y[i], qq = z[i] * z[i];
        if (p == 0.0) continue;
        if (qq == 0.0) {
            inf = 1;
            continue;
        }
        a += p * (log(p) - log(qq));
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        inf |= __shfl_down_sync(0xffffffffu, inf, o);
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0) {
        red[wp] = a;
        rinf[wp] = inf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        int f = 0;
        for (int i = 0; i < 8; ++i) {
            t += red[i];
            f |= rinf[i];
        }
        part[((int64_t)j * nch + c) * 2] = t;
        part[((int64_t)j * nch + c) * 2 + 1] = f;
    }
}

// Thread j: KL_j = sum_c part / A_j + ln A_j+1 - ln A_j (+infinity if a chunk flagged q_i = 0 < p_i).
__global__ void k_kl_fin(int npair, int nch, const double *part, const double *nrm2, double *kl) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npair) return;
    double t = 0.0;
    bool f = false;
    for (int c = 0; c < nch; ++c) {
        t += part[((int64_t)j * nch + c) * 2];
        f = f || part[((int64_t)j * nch + c) * 2 + 1] != 0.0;
    }
    kl[j] = f ? INFINITY : t / nrm2[j] + log(nrm2[j + 1]) - log(nrm2[j]);
}

void observables_extra_dev(Ctx *ctx, int L, int nup, int nev, const double *d_evecs, double q, double *d_kl,
                           double *d_sqp, double *d_fluct, double *d_dynf, cudaStream_t st) {
    ProfScope ps_all(ctx, "observables", (double)nev, st);
    const int64_t n = host_binom(L, nup);
    if (nev < 1 || nev > n) fail(MBL_ERR_INVALID, "observables: nev must be in [1, dim]");
    if (!(q > 0.0) || q == 1.0 || !std::isfinite(q)) fail(MBL_ERR_INVALID, "observables: q must be positive and not 1");
    EntTables &E = ent_tables(ctx, L, nup);
    // about two CTAs per SM over all vectors, chunks of at least 2048 rows
    const int nch = (int)std::max<int64_t>(1, std::min<int64_t>((2 * ctx->sm_count + nev - 1) / nev, n / 2048));
    const size_t need_part = (size_t)nev * nch * OBS_NS, need_nrm = (size_t)nev;
    if (E.x_part_cap < need_part) {
        E.x_part.alloc(ctx, need_part);
        E.x_part_cap = need_part;
    }
    if (E.x_nrm_cap < need_nrm) {
        E.x_nrm.alloc(ctx, need_nrm);
        E.x_nrm_cap = need_nrm;
    }
    k_moments_part<<<dim3(nch, nev), 256, 0, st>>>(n, nch, d_evecs, E.d_mA.data(), E.d_Mre.data(), E.d_Mim.data(), q,
                                                   E.x_part.data());
    MBL_LAUNCH_CHECK();
    k_moments_fin<<<(nev + 127) / 128, 128, 0, st>>>(nev, nch, E.x_part.data(), q, d_sqp, d_fluct, d_dynf,
                                                     E.x_nrm.data());
    MBL_LAUNCH_CHECK();
    if (nev > 1) {
        // the moments' partials are consumed: reuse the buffer (2 per pair and chunk <= 7 per vector and chunk)
        k_kl_part<<<dim3(nch, nev - 1), 256, 0, st>>>(n, nch, d_evecs, E.x_part.data());
        MBL_LAUNCH_CHECK();
        k_kl_fin<<<(nev + 126) / 128, 128, 0, st>>>(nev - 1, nch, E.x_part.data(), E.x_nrm.data(), d_kl);
        MBL_LAUNCH_CHECK();
    }
}

void observables_dev(Ctx *ctx, int L, int nup, int nev, const double *d_evals, const double *d_evecs, double *d_r,
                     double *d_rmean, double *d_s1p, double *d_se, cudaStream_t st) {
    ProfScope ps_all(ctx, "observables", (double)nev, st);
    int64_t n = host_binom(L, nup);
    if (nev < 1 || nev > n) fail(MBL_ERR_INVALID, "observables: nev must be in [1, dim]");
    if (nev > 2 || d_rmean) {
        k_gap_ratio<<<1, 32, 0, st>>>(nev, d_evals, d_r, d_rmean);
        MBL_LAUNCH_CHECK();
    }
    DVec<double> nrm2;
    nrm2.alloc(ctx, nev);
    k_s1p<<<nev, 256, 0, st>>>(n, d_evecs, d_s1p, nrm2.data());
    MBL_LAUNCH_CHECK();
    EntTables &E = ent_tables(ctx, L, nup);
    int nb = E.nblk;
    int64_t batch = (int64_t)nev * nb;
    std::vector<int> hm(batch);
    std::vector<int64_t> hg(batch), hw(batch);
    int64_t g = 0, w = 0;
    for (int j = 0; j < nev; ++j)
        for (int q = 0; q < nb; ++q) {
            int64_t b = (int64_t)j * nb + q;
            hm[b] = E.dA[q];
            hg[b] = g;
            hw[b] = w;
            g += (int64_t)E.dA[q] * E.dA[q];
            w += E.dA[q];
        }
    DVec<int> dm, info;
    DVec<int64_t> dgo, dwo;
    DVec<double> G, lam, work;
    dm.alloc(ctx, batch);
    info.alloc(ctx, batch);
    dgo.alloc(ctx, batch);
    dwo.alloc(ctx, batch);
    G.alloc(ctx, g);
    lam.alloc(ctx, w);
    size_t ws = syev_work_doubles(E.dAmax, false);
    work.alloc(ctx, ws * batch);
    MBL_CUDA(cudaMemcpyAsync(dm.data(), hm.data(), batch * sizeof(int), cudaMemcpyHostToDevice, st));
    MBL_CUDA(cudaMemcpyAsync(dgo.data(), hg.data(), batch * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    MBL_CUDA(cudaMemcpyAsync(dwo.data(), hw.data(), batch * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    {
        // function attributes are per device: set once on each device that runs this
        static std::mutex mu;
        static bool ready[64] = {};
        std::lock_guard<std::mutex> lk(mu);
        if (ctx->device < 0 || ctx->device >= 64 || !ready[ctx->device]) {
            MBL_CUDA(cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, 12288 * 8));
            if (ctx->device >= 0 && ctx->device < 64) ready[ctx->device] = true;
        }
    }
    k_gram<<<(unsigned)batch, 256, 12288 * 8, st>>>(n, nb, d_evecs, nrm2.data(), E.d_idx.data(), E.d_boff.data(),
                                                    E.d_dA.data(), E.d_dB.data(), dgo.data(), G.data());
    MBL_LAUNCH_CHECK();
    syev_batched((int)batch, dm.data(), dgo.data(), dwo.data(), G.data(), lam.data(), 0, nullptr, E.dAmax,
                 work.data(), info.data(), st);
    k_entropy_sum<<<(nev + 63) / 64, 64, 0, st>>>(nev, nb, E.d_dA.data(), dwo.data(), lam.data(), info.data(),
                                                   d_se);
    MBL_LAUNCH_CHECK();
    MBL_CUDA(cudaStreamSynchronize(st));
}

}  // namespace mbl
