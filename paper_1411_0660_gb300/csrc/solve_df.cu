// solve_df.cu -- dataflow form of the multifrontal triangular solves.
//
// The same sweeps as the level-by-level launch sequence in factor.cu (forward: gather, then the
// fronts' solve panels z_panel <- M z_panel, z_below -= (L21 M) z_panel; backward: gather, then
// x_panel <- G^T [y_panel; -x_below]), run by one persistent kernel per sweep.  Work items -- a
// gather of GR rows of one front, or one row block of one solve panel -- are listed in a
// topological order of their dependencies (plan: df_fwd, df_bwd) and handed out by an atomic
// ticket.  Before it touches data another item produces, an item waits on per-front completion
// counters:
//   forward  gather of front s   : every child's forward panels are complete;
//            panel step (s, k)   : s's gather is complete and s's panels before k are complete;
//   backward gather of front s   : the parent's backward panels are complete;
//            panel step (s, k)   : s's gather is complete and s's panels after k are complete.
// A CTA only waits on items with smaller tickets, which running CTAs hold, so the oldest unfinished
// item can always proceed: no deadlock, with or without co-residency of the whole grid.  Each wait
// is bounded (%globaltimer); on expiry the CTA counts a time-out in the factorization's error
// counter, settles its copies in flight and stops.  Producers fence their writes before they
// count; consumers read produced data through L2 (ld.cg).
#include "factor.h"
#include "solve_tile.cuh"

namespace mbl {

namespace {

struct DfArgs {
    const SolveItem *items;
    int nitems;
    const SolveDesc *sdescs;
    const int64_t *fo, *zo;
    const int32_t *fsz, *nc, *sn_start, *parent, *ch_ptr, *ch_list;
    const int64_t *rows_off;
    const int32_t *rows;
    const int64_t *fg_dst, *fg_own, *fg_cptr, *fg_src, *fg_off;
    const int32_t *gchunks, *ftotal, *btotal, *fprefix, *bprefix;
    const int64_t *poff;
    int32_t *gcnt, *fcnt, *bgcnt, *bcnt;  // per front
    unsigned int *ticket;
    unsigned int *arrive;  // per (descriptor, column chunk)
    unsigned long long *err;
    uint64_t wait_ns;  // limit of each wait (Factorization::wait_ns)
};

__device__ __forceinline__ uint64_t df_clock() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// thread 0: wait until *c >= v, for at most wait_ns nanoseconds
__device__ bool df_wait(const int32_t *c, int v, unsigned long long *err, uint64_t wait_ns) {
    if (ld_acquire(c) >= v) return true;
    const uint64_t t0 = df_clock();
    while (ld_acquire(c) < v) {
        if (df_clock() - t0 > wait_ns) {
            atomicAdd(err, 1ull);
            return false;
        }
        __nanosleep(128);
    }
    return true;
}

// all threads: make this CTA's writes visible, then count one completion
__device__ __forceinline__ void df_signal(int32_t *c) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(c, 1);
}

// ---------------------------------------------------------------------------------------------
template <class T, int PB>
__global__ void __launch_bounds__(256) k_df_fwd(DfArgs A, const T *Gp, const T *Dg, const T *y, T *Z, T *Zs,
                                                T *yfw, int p) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *zp = reinterpret_cast<T *>(smraw);  // SPW x PB; afterwards the 8 x PB x RBF partials
    __shared__ int s_t, s_ok;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    for (;;) {
        if (tid == 0) s_t = (int)atomicAdd(A.ticket, 1u);
        __syncthreads();
        const int t = s_t;
        if (t >= A.nitems) return;
        const SolveItem it = A.items[t];
        const int s = it.front;
        if (it.kind == 0) {
            // ---- gather GR rows of front s: own right-hand side plus the children's contributions
            if (tid == 0) {
                bool ok = true;
                for (int c = A.ch_ptr[s]; ok && c < A.ch_ptr[s + 1]; ++c) {
                    const int ch = A.ch_list[c];
                    ok = df_wait(A.fcnt + ch, A.ftotal[ch], A.err, A.wait_ns);
                }
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) return;
            const int r0 = GR * it.a, nr = min(GR, A.fsz[s] - r0);
            const int64_t base = A.fg_off[s] + r0;
            for (int o = tid; o < nr * p; o += blockDim.x) {
                const int64_t R = base + o / p;
                const int q = o % p;
                const int64_t own = A.fg_own[R];
                T v = own >= 0 ? y[own * p + q] : T(0);
                for (int64_t c = A.fg_cptr[R]; c < A.fg_cptr[R + 1]; ++c) v += __ldcg(Z + A.fg_src[c] * p + q);
                Z[A.fg_dst[R] * p + q] = v;
            }
            df_signal(A.gcnt + s);
            continue;
        }
        // ---- forward panel step, rows [RBF b, RBF b + RBF) of the panel's column block
        const int qd = it.a;
        const SolveDesc d = A.sdescs[qd];
        const int k0 = d.k0, w = d.w;
        const int r0 = it.b * RBF;
        const int nr = min(RBF, w + d.m2 - r0);
        const int64_t zb = A.zo[s] + k0, ld = sg_ld(w + d.m2);
        constexpr int NH = (SPW + 255) / 256, NPF = sizeof(T) == 4 ? NH : 1;
        const T *g = Gp + d.goff + r0 + lane;
        T lv[NPF][32];
#pragma unroll
        for (int h = 0; h < NPF; ++h) {  // the factor is read-only: load it before waiting
            const int c0 = h * 256 + wp * 32;
            if (lane < nr && c0 + 32 <= w) {
#pragma unroll
                for (int c = 0; c < 32; ++c) lv[h][c] = g[(int64_t)(c0 + c) * ld];
            }
        }
        if (tid == 0)
            s_ok = df_wait(A.gcnt + s, A.gchunks[s], A.err, A.wait_ns) &&
                   df_wait(A.fcnt + s, A.fprefix[qd], A.err, A.wait_ns);
        __syncthreads();
        if (!s_ok) return;
        for (int idx = tid; idx < w * PB; idx += blockDim.x) {
            const int c = idx / PB, q = idx % PB;
            zp[idx] = q < p ? __ldcg(Z + (zb + c) * p + q) : T(0);
        }
        __syncthreads();
        T acc[PB];
#pragma unroll
        for (int q = 0; q < PB; ++q) acc[q] = T(0);
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            const int c0 = h * 256 + wp * 32, c1 = min(w, c0 + 32);
            if (lane >= nr || c0 >= c1) continue;
            if (h < NPF && c1 - c0 == 32) {
#pragma unroll
                for (int c = 0; c < 32; ++c)
#pragma unroll
                    for (int q = 0; q < PB; ++q) acc[q] += lv[h < NPF ? h : 0][c] * zp[(c0 + c) * PB + q];
            } else {
                for (int c = c0; c < c1; ++c) {
                    const T l = g[(int64_t)c * ld];
#pragma unroll
                    for (int q = 0; q < PB; ++q) acc[q] += l * zp[c * PB + q];
                }
            }
        }
        __syncthreads();
        T *red = zp;
#pragma unroll
        for (int q = 0; q < PB; ++q) red[(wp * PB + q) * RBF + lane] = acc[q];
        __syncthreads();
        for (int o = tid; o < RBF * PB; o += blockDim.x) {
            const int i = o % RBF, q = o / RBF;
            if (i >= nr || q >= p) continue;
            T v = T(0);
#pragma unroll
            for (int j = 0; j < 8; ++j) v += red[(j * PB + q) * RBF + i];
            const int rr = r0 + i;
            if (rr < w) {
                const int64_t gr = (int64_t)A.sn_start[s] + k0 + rr;
                Zs[(zb + rr) * p + q] = v;
                yfw[gr * p + q] = v / Dg[gr];
            } else {
                const int64_t zi = (zb + rr) * p + q;
                Z[zi] = __ldcg(Z + zi) - v;
            }
        }
        df_signal(A.fcnt + s);
    }
}

// ---------------------------------------------------------------------------------------------
template <class T, int PB>
__global__ void __launch_bounds__(256) k_df_bwd(DfArgs A, const T *Gp, const T *yfw, T *x, T *Z, T *Zs, T *P,
                                                int p) {
    constexpr int E = 16 / sizeof(T);
    extern __shared__ __align__(16) unsigned char smraw[];
    T *Gs = reinterpret_cast<T *>(smraw);    // RBB columns x bwd_ldg rows
    T *vs = Gs + RBB * bwd_ldg<T>();         // RBK x PB
    T *red = PB == 8 ? Gs : vs + RBK * PB;  // 8 warps x 8 x RBB partial sums
    __shared__ int s_t, s_ok, s_last;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_t = (int)atomicAdd(A.ticket, 1u);
        __syncthreads();
        const int t = s_t;
        if (t >= A.nitems) return;
        const SolveItem it = A.items[t];
        const int s = it.front;
        if (it.kind == 0) {
            // ---- backward gather: forward result of the fully summed rows, ancestors' x below
            if (tid == 0) {
                const int pa = A.parent[s];
                s_ok = pa < 0 || df_wait(A.bcnt + pa, A.btotal[pa], A.err, A.wait_ns);
            }
            __syncthreads();
            if (!s_ok) return;
            const int r0 = GR * it.a, r1 = min(A.fsz[s], r0 + GR), ncs = A.nc[s];
            T *z = Z + A.zo[s] * p;
            const int32_t *rw = A.rows + A.rows_off[s];
            for (int idx = tid; idx < (r1 - r0) * p; idx += blockDim.x) {
                const int r = r0 + idx / p, q = idx % p;
                z[(int64_t)r * p + q] = (r < ncs) ? __ldcg(yfw + ((int64_t)A.sn_start[s] + r) * p + q)
                                                  : __ldcg(x + (int64_t)rw[r] * p + q);
            }
            df_signal(A.bgcnt + s);
            continue;
        }
        // ---- backward panel step: rows [RBK b, ..) x columns [RBB cc, ..) of G
        const int qd = it.a;
        const SolveDesc d = A.sdescs[qd];
        const int k0 = d.k0, w = d.w, ncs = A.nc[s], R = w + d.m2;
        const int ci = it.cc, cc = ci * RBB;
        const int nb = (R + RBK - 1) / RBK;
        const int r0 = it.b * RBK;
        const int nr = min(RBK, R - r0), nrv = (nr + E - 1) / E;
        const int wc = min(RBB, w - cc);
        const int64_t zb = A.zo[s] + k0, ld = sg_ld(R);
        bwd_tile_issue(Gs, Gp + d.goff + (int64_t)cc * ld + r0, ld, wc, nrv);  // read-only: copy before waiting
        if (tid == 0)
            s_ok = df_wait(A.bgcnt + s, A.gchunks[s], A.err, A.wait_ns) &&
                   df_wait(A.bcnt + s, A.bprefix[qd], A.err, A.wait_ns);
        __syncthreads();
        if (!s_ok) {
            cp_async_commit_wait();
            return;
        }
        for (int idx = tid; idx < RBK * PB; idx += blockDim.x) {
            const int i = idx / PB, q = idx % PB;
            T v = T(0);
            if (i < nr && q < p) {
                const int rr = r0 + i;
                if (rr < w) v = __ldcg(Z + (zb + rr) * p + q);
                else if (k0 + rr < ncs) v = -__ldcg(Zs + (zb + rr) * p + q);
                else v = -__ldcg(Z + (zb + rr) * p + q);
            }
            vs[idx] = v;
        }
        cp_async_commit_wait();
        __syncthreads();
        const int64_t tile = (int64_t)RBB * PB;
        T *out = P + (A.poff[qd] + (int64_t)it.b * SUBS + ci) * tile;
        T *zsp = Zs + (zb + cc) * p, *xp = x + ((int64_t)A.sn_start[s] + k0 + cc) * p;
#pragma unroll
        for (int q0 = 0; q0 < PB; q0 += 8) {
            T o2[2];
            bwd_tile_product<T, PB>(Gs, vs, red, nrv * E, q0, o2);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int o = tid + 256 * h, q = q0 + o / RBB, c = o % RBB;
                if (nb == 1) {
                    if (c < wc && q < p) {
                        zsp[c * p + q] = o2[h];
                        xp[c * p + q] = o2[h];
                    }
                } else {
                    out[q * RBB + c] = o2[h];
                }
            }
        }
        if (nb > 1) {
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                const unsigned int prev = atomicAdd(&A.arrive[(size_t)qd * SUBS + ci], 1u);
                s_last = prev == (unsigned int)(nb - 1);
            }
            __syncthreads();
            if (!s_last) continue;
            __threadfence();
            bwd_finish<T, PB>(P + (A.poff[qd] + ci) * tile, (int64_t)SUBS * tile, nb, wc, p, zsp, xp, Gs);
            if (tid == 0) A.arrive[(size_t)qd * SUBS + ci] = 0u;
        }
        df_signal(A.bcnt + s);
    }
}

template <class T, int PB>
size_t df_fwd_smem() { return sizeof(T) * (size_t)SPW * PB; }
template <class T, int PB>
size_t df_bwd_smem() { return bwd_tile_smem<T, PB>(); }

template <class T, int PB>
void df_sweeps(Factorization &fz, int p, cudaStream_t st) {
    Plan &pl = *fz.plan;
    // the persistent sweeps wait on one another's CTAs: every CTA must be resident, so the grid is the
    // occupancy of this device times its SM count
    smem_limit((const void *)k_df_fwd<T, PB>, df_fwd_smem<T, PB>());
    smem_limit((const void *)k_df_bwd<T, PB>, df_bwd_smem<T, PB>());
    int of = 0, ob = 0;
    MBL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&of, k_df_fwd<T, PB>, 256, df_fwd_smem<T, PB>()));
    MBL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, k_df_bwd<T, PB>, 256, df_bwd_smem<T, PB>()));
    const int grid_f = std::max(1, of) * fz.ctx->sm_count;
    const int grid_b = std::max(1, ob) * fz.ctx->sm_count;
    const int ns = pl.ns;
    int32_t *cnt = fz.dfcnt.data();
    MBL_CUDA(cudaMemsetAsync(cnt, 0, ((size_t)4 * ns + 2) * sizeof(int32_t), st));
    DfArgs A;
    A.sdescs = pl.d_sdescs.data();
    A.fo = pl.d_sn_fo.data();
    A.zo = pl.d_sn_zo.data();
    A.fsz = pl.d_sn_f.data();
    A.nc = pl.d_sn_nc.data();
    A.sn_start = pl.d_sn_start.data();
    A.parent = pl.d_sn_parent.data();
    A.ch_ptr = pl.d_ch_ptr.data();
    A.ch_list = pl.d_ch_list.data();
    A.rows_off = pl.d_sn_rows_off.data();
    A.rows = pl.d_rows.data();
    A.fg_dst = pl.d_fg_dst.data();
    A.fg_own = pl.d_fg_own.data();
    A.fg_cptr = pl.d_fg_cptr.data();
    A.fg_src = pl.d_fg_src.data();
    A.fg_off = pl.d_df_fg_off.data();
    A.gchunks = pl.d_df_gchunks.data();
    A.ftotal = pl.d_df_ftotal.data();
    A.btotal = pl.d_df_btotal.data();
    A.fprefix = pl.d_df_fprefix.data();
    A.bprefix = pl.d_df_bprefix.data();
    A.poff = pl.d_df_poff.data();
    A.gcnt = cnt;
    A.fcnt = cnt + ns;
    A.bgcnt = cnt + 2 * ns;
    A.bcnt = cnt + 3 * ns;
    A.arrive = fz.scnt.data();
    A.err = fz.counters.data() + 2;
    A.wait_ns = fz.wait_ns;
    const T *Gp = static_cast<const T *>(fz.gpk.m.p);
    const T *Dg = static_cast<const T *>(fz.D.m.p);
    T *Z = static_cast<T *>(fz.zwork.m.p);
    T *Zs = static_cast<T *>(fz.zsolved.m.p);
    T *y = static_cast<T *>(fz.ywork.m.p);
    T *yfw = static_cast<T *>(fz.yfw.m.p);
    T *P = static_cast<T *>(fz.pwork.m.p);
    A.items = pl.d_df_fwd.data();
    A.nitems = (int)pl.df_fwd.size();
    A.ticket = reinterpret_cast<unsigned int *>(cnt + 4 * ns);
    k_df_fwd<T, PB><<<std::min(grid_f, std::max(1, A.nitems)), 256, df_fwd_smem<T, PB>(), st>>>(
        A, Gp, Dg, y, Z, Zs, yfw, p);
    MBL_LAUNCH_CHECK();
    A.items = pl.d_df_bwd.data();
    A.nitems = (int)pl.df_bwd.size();
    A.ticket = reinterpret_cast<unsigned int *>(cnt + 4 * ns + 1);
    k_df_bwd<T, PB><<<std::min(grid_b, std::max(1, A.nitems)), 256, df_bwd_smem<T, PB>(), st>>>(A, Gp, yfw, y, Z, Zs,
                                                                                                 P, p);
    MBL_LAUNCH_CHECK();
}

}  // namespace

template <class T>
void solve_dataflow(Factorization &fz, int p, cudaStream_t st) {
    const int pb = p <= 8 ? 8 : (p <= 16 ? 16 : 32);
    if (pb == 8) df_sweeps<T, 8>(fz, p, st);
    else if (pb == 16) df_sweeps<T, 16>(fz, p, st);
    else df_sweeps<T, 32>(fz, p, st);
}

template void solve_dataflow<float>(Factorization &, int, cudaStream_t);
template void solve_dataflow<double>(Factorization &, int, cudaStream_t);

}  // namespace mbl
