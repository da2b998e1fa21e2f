// factor.cu -- batched multifrontal LDL^T of H - sigma I and the supernodal triangular solves.
//
// The shift-invert transformation of arXiv:1411.0660 (numerical-method section) needs
// (H - sigma)^-1 applied many times; the paper factors H - sigma with a parallel sparse direct
// solver.  Here the factorization is a supernodal multifrontal LDL^T driven by the static plan
// (plan.h): fronts of one tree level are processed together, panel by panel:
//   assemble   zero the front, scatter the CSR entries (minus sigma on the diagonal) and
//              extend-add the children's contribution blocks (deterministic, no atomics);
//   diag       one CTA factors the NB x NB diagonal block with diagonal pivoting inside it
//              (a pivot below `tiny` is replaced by +-tiny), and inverts its unit-lower factor;
//   trsm       W21 = A21 L11^-T (= L21 D), L21 = W21 D^-1, row blocks in parallel;
//   update     A22 -= L21 W21^T on the lower triangle, 64 x 64 tiles in parallel.
// Pivoting permutes only the variables of the current panel; the rows of earlier panel
// columns keep their order and the solves apply each panel's permutation when they reach it.
#include <cuda.h>

#include <cfloat>
#include <map>
#include <mutex>

#include "factor.h"
#include "solve_tile.cuh"
#include "tc_pieces.cuh"

namespace mbl {

// The driver's virtual-memory calls, resolved through the runtime at first use (the library does
// not link the driver library itself, so it still loads where no driver is installed).
struct VmmApi {
    decltype(&::cuGetErrorString) error_string = nullptr;
    decltype(&::cuMemGetAllocationGranularity) granularity = nullptr;
    decltype(&::cuMemAddressReserve) reserve = nullptr;
    decltype(&::cuMemAddressFree) address_free = nullptr;
    decltype(&::cuMemCreate) create = nullptr;
    decltype(&::cuMemMap) map = nullptr;
    decltype(&::cuMemSetAccess) set_access = nullptr;
    decltype(&::cuMemUnmap) unmap = nullptr;
    decltype(&::cuMemRelease) release = nullptr;
};

static const VmmApi &vmm() {
    static const VmmApi api = [] {
        VmmApi a;
        auto get = [](const char *name, void **fn) {
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion(name, fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess)
                *fn = nullptr;
        };
        get("cuGetErrorString", reinterpret_cast<void **>(&a.error_string));
        get("cuMemGetAllocationGranularity", reinterpret_cast<void **>(&a.granularity));
        get("cuMemAddressReserve", reinterpret_cast<void **>(&a.reserve));
        get("cuMemAddressFree", reinterpret_cast<void **>(&a.address_free));
        get("cuMemCreate", reinterpret_cast<void **>(&a.create));
        get("cuMemMap", reinterpret_cast<void **>(&a.map));
        get("cuMemSetAccess", reinterpret_cast<void **>(&a.set_access));
        get("cuMemUnmap", reinterpret_cast<void **>(&a.unmap));
        get("cuMemRelease", reinterpret_cast<void **>(&a.release));
        (void)cudaGetLastError();
        return a;
    }();
    if (!api.granularity || !api.reserve || !api.address_free || !api.create || !api.map || !api.set_access ||
        !api.unmap || !api.release)
        fail(MBL_ERR_CUDA, "memory-lean arena: the driver's virtual-memory entry points are unavailable");
    return api;
}

#define MBL_CU(x)                                                                                            \
    do {                                                                                                     \
        CUresult r_ = (x);                                                                                   \
        if (r_ != CUDA_SUCCESS) {                                                                            \
            const char *m_ = nullptr;                                                                        \
            if (vmm().error_string) vmm().error_string(r_, &m_);                                             \
            ::mbl::fail(r_ == CUDA_ERROR_OUT_OF_MEMORY ? MBL_ERR_OOM : MBL_ERR_CUDA,                        \
                        std::string(#x) + " -> " + (m_ ? m_ : "?"));                                         \
        }                                                                                                    \
    } while (0)

// Physical backing of the memory-lean fronts arena: the whole arena is one reserved virtual range
// (so that every kernel addresses a front as arena + fo[s], as with the ordinary arena), and each
// region of the plan is backed chunk by chunk (LEAN_CHUNK elements) only while its fronts are live.
struct LeanArena {
    CUdeviceptr base = 0;
    size_t bytes = 0, es = 4;
    Ctx *ctx = nullptr;
    CUmemAllocationProp prop{};
    std::vector<std::vector<CUmemGenericAllocationHandle>> h;  // per region and chunk (0: not backed)

    void reserve(Ctx *c, const Plan &p, size_t es_) {
        ctx = c;
        es = es_;
        prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
        prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
        prop.location.id = c->device;
        size_t gran = 0;
        MBL_CU(vmm().granularity(&gran, &prop, CU_MEM_ALLOC_GRANULARITY_MINIMUM));
        if (gran == 0 || ((size_t)ARENA_ALIGN * es) % gran != 0)
            fail(MBL_ERR_CUDA, "memory-lean arena: allocation granularity does not divide the region alignment");
        bytes = (size_t)p.arena_elems * es;
        MBL_CU(vmm().reserve(&base, bytes, (size_t)ARENA_ALIGN * es, 0, 0));
        h.assign(p.regions.size(), {});
        for (size_t r = 0; r < p.regions.size(); ++r)
            h[r].assign((size_t)((p.regions[r].fo1 - p.regions[r].fo0 + LEAN_CHUNK - 1) / LEAN_CHUNK), 0);
    }
    // byte offset and length of chunk c of region r (the last one rounded up to ARENA_ALIGN elements)
    void chunk(const Plan &p, size_t r, size_t c, size_t &off, size_t &len) const {
        const ArenaRegion &g = p.regions[r];
        const int64_t a0 = g.fo0 + (int64_t)c * LEAN_CHUNK, a1 = std::min(g.fo1, a0 + LEAN_CHUNK);
        off = (size_t)a0 * es;
        len = (size_t)((a1 - a0 + ARENA_ALIGN - 1) / ARENA_ALIGN * ARENA_ALIGN) * es;
    }
    void map_region(const Plan &p, size_t r) {
        CUmemAccessDesc acc{};
        acc.location = prop.location;
        acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
        for (size_t c = 0; c < h[r].size(); ++c) {
            if (h[r][c]) continue;
            size_t off, len;
            chunk(p, r, c, off, len);
            if (ctx->budget && ctx->in_use + len > ctx->budget)
                fail(MBL_ERR_OOM, "memory-lean arena: chunk exceeds the context budget");
            CUmemGenericAllocationHandle hd = 0;
            MBL_CU(vmm().create(&hd, len, &prop, 0));
            CUresult e = vmm().map(base + off, len, 0, hd, 0);
            if (e == CUDA_SUCCESS) e = vmm().set_access(base + off, len, &acc, 1);
            if (e != CUDA_SUCCESS) {
                vmm().unmap(base + off, len);
                vmm().release(hd);
                MBL_CU(e);
            }
            h[r][c] = hd;
            ctx->in_use += len;
            ctx->peak = std::max(ctx->peak, ctx->in_use);
        }
    }
    // the caller has synchronized every stream that used the chunk
    void unmap_chunk(const Plan &p, size_t r, size_t c) {
        if (!h[r][c]) return;
        size_t off, len;
        chunk(p, r, c, off, len);
        MBL_CU(vmm().unmap(base + off, len));
        MBL_CU(vmm().release(h[r][c]));
        h[r][c] = 0;
        ctx->in_use -= len;
    }
    void unmap_region(const Plan &p, size_t r) {
        for (size_t c = 0; c < h[r].size(); ++c) unmap_chunk(p, r, c);
    }
    // (no CUDA error escapes: also run from destructors)
    void release_all(const Plan *p) {
        for (size_t r = 0; r < h.size(); ++r)
            for (size_t c = 0; c < h[r].size(); ++c)
                if (h[r][c]) {
                    size_t off = 0, len = 0;
                    if (p) chunk(*p, r, c, off, len);
                    if (p) vmm().unmap(base + off, len);
                    vmm().release(h[r][c]);
                    h[r][c] = 0;
                    if (ctx && ctx_alive(ctx)) ctx->in_use -= len;
                }
        if (base) vmm().address_free(base, bytes);
        base = 0;
    }
};

template <class T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }
// c - a b, rounded once
__device__ __forceinline__ float fnms(float a, float b, float c) { return __fmaf_rn(-a, b, c); }
__device__ __forceinline__ double fnms(double a, double b, double c) { return __fma_rn(-a, b, c); }

__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int n, int x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// threads of the column-maximum and trsm kernels (one CTA per RB-row block): more than the block's
// rows, so that their loads of the panel are in flight together
constexpr int PANEL_THREADS = 256;

// descriptor whose [off, off + count) range holds `b` (descs of one step are ordered by off)
__device__ __forceinline__ int find_desc2(const PanelDesc *d, int nd, int64_t b) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (d[mid].off2 <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int find_desc3(const PanelDesc *d, int nd, int64_t b) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (d[mid].off3 <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------------------------------
// Numeric factorization kernels
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_assemble(const AsmItem *items, const int64_t *fo, const int32_t *fsz,
                                                  const int32_t *nc, const int32_t *sn_start, const int32_t *ch_ptr,
                                                  const int32_t *ch_list, const int64_t *rel_off,
                                                  const int32_t *relind, const int64_t *amap_ptr,
                                                  const int64_t *amap_src, const int32_t *amap_row,
                                                  const double *val, double sigma, T *arena) {
    AsmItem it = items[blockIdx.x];
    int s = it.front, f = fsz[s], c0 = it.c0, c1 = min(f, c0 + ACOLS);
    T *F = arena + fo[s];
    for (int c = c0; c < c1; ++c)
        for (int r = c + threadIdx.x; r < f; r += blockDim.x) F[(int64_t)c * f + r] = T(0);
    __syncthreads();
    int ncs = nc[s];
    for (int c = c0; c < min(c1, ncs); ++c) {
        int64_t j = sn_start[s] + c;
        for (int64_t e = amap_ptr[j] + threadIdx.x; e < amap_ptr[j + 1]; e += blockDim.x) {
            int r = amap_row[e];
            double v = val[amap_src[e]];
            if (r == c) v -= sigma;
            F[(int64_t)c * f + r] = (T)v;
        }
    }
    __syncthreads();
    for (int q = ch_ptr[s]; q < ch_ptr[s + 1]; ++q) {
        int ch = ch_list[q];
        int fc = fsz[ch], ncc = nc[ch], uc = fc - ncc;
        const int32_t *rel = relind + rel_off[ch];
        const T *C = arena + fo[ch];
        int blo = lower_bound_i32(rel, uc, c0), bhi = lower_bound_i32(rel, uc, c1);
        for (int b = blo; b < bhi; ++b) {
            T *Pcol = F + (int64_t)rel[b] * f;
            const T *Ccol = C + (int64_t)(ncc + b) * fc + ncc;
            for (int a = b + threadIdx.x; a < uc; a += blockDim.x) Pcol[rel[a]] += Ccol[a];
        }
        __syncthreads();
    }
}

// Largest |entry| of each panel column over the rows below the panel (current values), per step
// descriptor: cmax[di * NB + c] (float bits, atomicMax).  Used by the pivot choice of k_panel_diag.
template <class T>
__global__ void __launch_bounds__(PANEL_THREADS) k_panel_colmax(const PanelDesc *descs, int nd, const int64_t *fo,
                                                     const int32_t *fsz, const T *arena, unsigned int *cmax) {
    const int di = find_desc2(descs, nd, blockIdx.x);
    const PanelDesc d = descs[di];
    const int s = d.front, f = fsz[s], k0 = d.k0, w = d.w;
    const int r0 = k0 + w + (int)(blockIdx.x - d.off2) * RB;
    const int nr = min(RB, f - r0);
    const T *F = arena + fo[s];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // warp wp takes columns wp, wp + nw, ...; its lanes cover the block's rows
    for (int c = wp; c < w; c += nw) {
        const T *col = F + (int64_t)(k0 + c) * f + r0;
        float v = 0.f;
        for (int i = lane; i < nr; i += 32) v = fmaxf(v, (float)tabs(col[i]));
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) atomicMax(cmax + (size_t)di * NB + c, __float_as_uint(v));
    }
}

// LDL^T of a panel's w x w diagonal block with symmetric 1x1 pivoting, 128 threads.  The block is
// kept whole (both triangles) in shared memory so that every candidate pivot's off-diagonal entries
// lie in its own row.  A pair of threads owns row t + 1 + i of the trailing block during the update
// of step t (the two threads take alternate columns) and the same index as candidate t + 1 + i in the
// pivot choice of step t + 1, so the largest off-diagonal magnitude that the choice needs falls out
// of the update.  Both mirror entries of the update subtract u_a l_b with one rounding (a the larger
// index, u the unscaled pivot column, l = u / d), so the block stays exactly symmetric.
template <class T>
__global__ void __launch_bounds__(128) k_panel_diag(const PanelDesc *descs, const int64_t *fo, const int32_t *fsz,
                                                    const int32_t *sn_start, T *arena, T *Dg, int32_t *piv,
                                                    double tiny, unsigned long long *counters,
                                                    const unsigned int *cmax) {
    __shared__ T B[NB][NB + 1];
    __shared__ T ucol[NB], lcol[NB], dvec[NB];
    __shared__ int perm[NB];
    __shared__ float cm[NB];
    __shared__ unsigned int s_k1[4], s_k2[4];
    __shared__ int s_jj[4];
    __shared__ unsigned int s_npert, s_nneg;
    static_assert(NB == 64, "two threads per row of a 64-wide block on 128 threads");
    const PanelDesc d = descs[blockIdx.x];
    const int s = d.front, f = fsz[s], k0 = d.k0, w = d.w;
    T *F = arena + fo[s];
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, pi = tid >> 1, h = tid & 1;
    for (int idx = tid; idx < w * w; idx += 128) {
        const int r = idx % w, c = idx / w;
        if (r >= c) {
            const T v = F[(int64_t)(k0 + c) * f + k0 + r];
            B[r][c] = v;
            B[c][r] = v;
        }
    }
    if (tid < w) {
        perm[tid] = tid;
        cm[tid] = __uint_as_float(cmax[(size_t)blockIdx.x * NB + tid]);
    }
    if (tid == 0) s_npert = s_nneg = 0u;
    __syncthreads();
    // off-diagonal magnitude of candidate pi's row over the whole block (step 0)
    float om = 0.f;
    if (pi < w) {
        for (int c = h; c < w; c += 2)
            if (c != pi) om = fmaxf(om, (float)tabs(B[pi][c]));
    }
    om = fmaxf(om, __shfl_xor_sync(0xffffffffu, om, 1));
    for (int t = 0; t < w; ++t) {
        // pivot: the candidate whose diagonal is largest relative to the rest of its column (inside the
        // block and, from before this panel, in the rows below), which bounds the multipliers; order:
        // largest score, then largest |d|, then the smallest index.  Scores and |d| are non-negative
        // floats, so their bit patterns order like their values: a warp's choice is three redux.sync
        // steps (score, then |d| among the best scores, then the smallest index).
        {
            const int j = t + pi;
            const bool valid = j < w;
            unsigned int k1 = 0u, k2 = 0u;
            if (valid) {
                const float o = fmaxf(om, cm[perm[j]]);
                const float dj = (float)tabs(B[j][j]);
                const float sc = o > 0.f ? dj / o : 3.0e38f;
                k1 = __float_as_uint(sc) + 1u;  // 0 marks a lane without a candidate
                k2 = __float_as_uint(dj);
            }
            const unsigned int m1 = __reduce_max_sync(0xffffffffu, k1);
            const unsigned int m2 = __reduce_max_sync(0xffffffffu, k1 == m1 ? k2 : 0u);
            const unsigned int jm =
                __reduce_min_sync(0xffffffffu, (valid && k1 == m1 && k2 == m2) ? (unsigned int)j : (unsigned int)w);
            if (lane == 0) {
                s_k1[wp] = m1;
                s_k2[wp] = m2;
                s_jj[wp] = (int)jm;
            }
        }
        __syncthreads();
        int j = s_jj[0];
        {
            // the warps hold candidates in increasing order: a later warp wins only if strictly better
            unsigned int b1 = s_k1[0], b2 = s_k2[0];
#pragma unroll
            for (int v = 1; v < 4; ++v) {
                const unsigned int k1 = s_k1[v], k2 = s_k2[v];
                if (k1 > b1 || (k1 == b1 && k2 > b2)) {
                    b1 = k1;
                    b2 = k2;
                    j = s_jj[v];
                }
            }
            if (b1 == 0u || j >= w) j = t;
        }
        if (j != t) {
            // symmetric exchange of indices t and j: rows over every column (the computed L rows
            // included), then columns over the trailing rows
            if (tid < w) {
                const T x = B[t][tid];
                B[t][tid] = B[j][tid];
                B[j][tid] = x;
            }
            if (tid == 0) {
                const int pp = perm[t];
                perm[t] = perm[j];
                perm[j] = pp;
            }
            __syncthreads();
            if (tid >= t && tid < w) {
                const T x = B[tid][t];
                B[tid][t] = B[tid][j];
                B[tid][j] = x;
            }
        }
        __syncthreads();
        // the pivot (a tiny one replaced by +-tiny, statically); the column: u keeps the unscaled
        // entries, the column itself becomes L's
        // (B[t][t] itself is left as it is: D goes to dvec)
        T dv = B[t][t];
        const bool pert = !(tabs(dv) >= (T)tiny);
        if (pert) dv = (dv >= T(0)) ? (T)tiny : (T)(-tiny);
        const int r = t + 1 + pi;
        const bool own = r < w;
        T ur = (own && h == 0) ? B[r][t] : T(0);
        ur = __shfl_sync(0xffffffffu, ur, lane & ~1);  // the pair's second thread never reads B[r][t]
        const T lr = own ? ur / dv : T(0);
        if (own && h == 0) {
            B[r][t] = lr;
            ucol[r] = ur;
            lcol[r] = lr;
        }
        if (tid == 0) {
            dvec[t] = dv;
            s_npert += pert ? 1u : 0u;
            s_nneg += dv < T(0) ? 1u : 0u;
        }
        __syncthreads();
        // trailing update of row r over the columns of this thread, both triangles.  The next step's
        // choice reads only the thread's own row, so no barrier closes the step.
        om = 0.f;
        if (own) {
#pragma unroll 4
            for (int c = t + 1 + h; c < w; c += 2) {
                const T v = c <= r ? fnms(ur, lcol[c], B[r][c]) : fnms(ucol[c], lr, B[r][c]);
                B[r][c] = v;
                if (c != r) om = fmaxf(om, (float)tabs(v));
            }
        }
        om = fmaxf(om, __shfl_xor_sync(0xffffffffu, om, 1));
    }
    __syncthreads();
    if (tid == 0) {
        if (s_npert) atomicAdd(&counters[0], (unsigned long long)s_npert);
        if (s_nneg) atomicAdd(&counters[1], (unsigned long long)s_nneg);
    }
    // write L11 (strictly lower), D on the diagonal, pivots
    for (int idx = tid; idx < w * w; idx += 128) {
        const int r = idx % w, c = idx / w;
        if (r >= c) F[(int64_t)(k0 + c) * f + k0 + r] = r == c ? dvec[r] : B[r][c];
    }
    const int64_t g0 = (int64_t)sn_start[s] + k0;
    if (tid < w) {
        Dg[g0 + tid] = dvec[tid];
        piv[g0 + tid] = k0 + perm[tid];
        float lmax = 0.f;
        for (int r = tid + 1; r < w; ++r) lmax = fmaxf(lmax, (float)tabs(B[r][tid]));
        atomicMax(reinterpret_cast<unsigned int *>(counters + 3), __float_as_uint(lmax));
        atomicMin(reinterpret_cast<unsigned int *>(counters + 4), __float_as_uint((float)tabs(dvec[tid])));
    }
}

// W21 = A21 L11^-T by forward substitution (one thread per row, no explicit inverse), then
// L21 = W21 D^-1.  The columns of A21 are read in the panel's pivoted order.
template <class T>
__global__ void __launch_bounds__(PANEL_THREADS) k_panel_trsm(const PanelDesc *descs, int nd, const int64_t *fo,
                                                   const int32_t *fsz, const int32_t *sn_start, T *arena,
                                                   const T *Dg, const int32_t *piv, T *wscr,
                                                   unsigned long long *stats, void *pieces, int64_t prow,
                                                   int pmode) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T(*Lb)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smraw);                      // L11
    T(*As)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smraw + sizeof(T) * NB * (NB + 1));
    __shared__ T Dinv[NB];
    __shared__ int pv[NB];
    const int di = find_desc2(descs, nd, blockIdx.x);
    const PanelDesc d = descs[di];
    const int s = d.front, f = fsz[s], k0 = d.k0, w = d.w, m2 = d.m2;
    const int r0 = k0 + w + (int)(blockIdx.x - d.off2) * RB;
    const int nr = min(RB, f - r0);
    T *F = arena + fo[s];
    const int tid = threadIdx.x;
    const int64_t g0 = (int64_t)sn_start[s] + k0;
    for (int idx = tid; idx < w * w; idx += blockDim.x) {
        int r = idx % w, c = idx / w;
        Lb[r][c] = (r > c) ? F[(int64_t)(k0 + c) * f + k0 + r] : T(0);
    }
    if (tid < w) {
        Dinv[tid] = T(1) / Dg[g0 + tid];
        pv[tid] = piv[g0 + tid];
    }
    __syncthreads();
    for (int idx = tid; idx < nr * w; idx += blockDim.x) {
        int i = idx % nr, k = idx / nr;
        As[i][k] = F[(int64_t)pv[k] * f + r0 + i];
    }
    __syncthreads();
    if (tid < nr) {
        T *a = As[tid];
        for (int t = 1; t < w; ++t) {
            T acc = a[t];
            for (int k = 0; k < t; ++k) acc -= a[k] * Lb[t][k];
            a[t] = acc;
        }
    }
    __syncthreads();
    T *W = wscr + d.woff;
    float lmax = 0.f;
    for (int idx = tid; idx < nr * w; idx += blockDim.x) {
        int i = idx % nr, t = idx / nr;
        T x = As[i][t];
        T l = x * Dinv[t];
        F[(int64_t)(k0 + t) * f + r0 + i] = l;
        W[(int64_t)(r0 - k0 - w + i) + (int64_t)t * m2] = x;
        lmax = fmaxf(lmax, (float)tabs(l));
    }
    if (sizeof(T) == 4 && pmode) {
        // tensor-core operand pieces of this block's rows of L21 and W21 (pieces 0/1 and 2/3), row-major
        // with NB per row, zero past the panel width; rows start at the descriptor's woff / NB
        const int64_t rb = d.woff / NB + (r0 - k0 - w);
        for (int idx = tid; idx < nr * NB; idx += blockDim.x) {
            const int i = idx / NB, t = idx - i * NB;
            const float xv = t < w ? (float)As[i][t] : 0.f;
            const float lv = t < w ? (float)(As[i][t] * Dinv[t]) : 0.f;
            const int64_t e = (rb + i) * NB + t;
            if (pmode == 1) {
                uint32_t *P = static_cast<uint32_t *>(pieces);
                split_tf32(lv, P[e], P[prow * NB + e]);
                split_tf32(xv, P[2 * prow * NB + e], P[3 * prow * NB + e]);
            } else {
                uint16_t *P = static_cast<uint16_t *>(pieces);
                split_bf16(lv, P[e], P[prow * NB + e]);
                split_bf16(xv, P[2 * prow * NB + e], P[3 * prow * NB + e]);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((tid & 31) == 0) atomicMax(reinterpret_cast<unsigned int *>(stats), __float_as_uint(lmax));
}

// Trailing update of one 64 x 64 lower tile: C[i][j] -= sum_t L21[i][t] W21[j][t]
template <class T>
__global__ void __launch_bounds__(256) k_panel_update(const PanelDesc *descs, int nd, const int64_t *fo,
                                                      const int32_t *fsz, T *arena, const T *wscr) {
    constexpr int KC = 16;
    static_assert(RB == NB, "solve kernels share one shared-memory size");
    __shared__ T As[KC][TB + 4];
    __shared__ T Bs[KC][TB + 4];
    const int di = find_desc3(descs, nd, blockIdx.x);
    const PanelDesc d = descs[di];
    const int s = d.front, f = fsz[s], k0 = d.k0, w = d.w, m2 = d.m2;
    int64_t t = (int64_t)blockIdx.x - d.off3;
    int bi = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(bi + 1) * (bi + 2) / 2 <= t) ++bi;
    while ((int64_t)bi * (bi + 1) / 2 > t) --bi;
    const int bj = (int)(t - (int64_t)bi * (bi + 1) / 2);
    const int base = k0 + w;
    const int i0 = base + bi * TB, j0 = base + bj * TB;
    T *F = arena + fo[s];
    const T *W = wscr + d.woff;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int kt = 0; kt < w; kt += KC) {
        for (int idx = tid; idx < KC * TB; idx += 256) {
            int k = idx / TB, i = idx % TB;
            int kk = kt + k;
            int gi = i0 + i, gj = j0 + i;
            As[k][i] = (kk < w && gi < f) ? F[(int64_t)(k0 + kk) * f + gi] : T(0);
            Bs[k][i] = (kk < w && gj < f) ? W[(int64_t)(gj - base) + (int64_t)kk * m2] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[k][ty * 4 + u];
                b[u] = Bs[k][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        int gj = j0 + tx * 4 + v;
        if (gj >= f) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int gi = i0 + ty * 4 + u;
            if (gi >= f || gi < gj) continue;
            F[(int64_t)gj * f + gi] -= acc[u][v];
        }
    }
}

// ------------------------------------------------------------------------------------------
// Triangular solves (row-major n x p blocks, p <= 32) in multifrontal order, SPW-wide solve
// panels.  Per solve panel: forward z_panel <- M z_panel then z_below -= L21 z_panel; backward
// z_panel <- M^T (z_panel - L21^T x_below).  Own rows of a front hold pivoted-order values
// between the two sweeps (Zs / yfw); the backward sweep leaves true-order values.
// ------------------------------------------------------------------------------------------
// B, X: entry (row r, right-hand side q) at r * ld + q * ldq (row-major blocks: ldq = 1;
// column-major: ld = 1, ldq = n).
template <class T>
__global__ void k_perm_in(int64_t n, int p, const int32_t *perm, const double *B, int64_t ldb, int64_t ldbq, T *y) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * p) return;
    int64_t k = idx / p;
    int q = (int)(idx - k * p);
    y[idx] = (T)B[(int64_t)perm[k] * ldb + q * ldbq];
}

template <class T>
__global__ void k_perm_out(int64_t n, int p, const int32_t *perm, const T *x, double *X, int64_t ldx, int64_t ldxq,
                           int accumulate) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * p) return;
    int64_t k = idx / p;
    int q = (int)(idx - k * p);
    double v = (double)x[idx];
    double *dst = X + (int64_t)perm[k] * ldx + q * ldxq;
    *dst = accumulate ? *dst + v : v;
}

__device__ __forceinline__ int find_sdesc_b(const SolveDesc *d, int nd, int64_t b) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (d[mid].offb <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// M of one solve panel, 32 columns per CTA, in FP64: the forward sequence (pivot permutation,
// unit-lower substitution, elimination of the later rows of the panel) applied to unit vectors.
template <class T>
__global__ void __launch_bounds__(256) k_build_m(const SolveDesc *sdescs, const int64_t *fo, const int32_t *fsz,
                                                 const int32_t *sn_start, const T *arena, const int32_t *piv,
                                                 T *Mall) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double(*Zc)[33] = reinterpret_cast<double(*)[33]>(smraw);                          // SPW x 33
    double(*Zp)[33] = reinterpret_cast<double(*)[33]>(smraw + 8 * SPW * 33);           // NB x 33
    double(*Lb)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(smraw + 8 * (SPW + NB) * 33);
    const SolveDesc d = sdescs[blockIdx.x];
    const int c0 = blockIdx.y * 32;
    if (c0 >= d.w) return;
    const int ncol = min(32, d.w - c0), w = d.w, s = d.front, f = fsz[s], k0 = d.k0;
    const T *F = arena + fo[s];
    const int64_t g0 = (int64_t)sn_start[s] + k0;
    for (int idx = threadIdx.x; idx < w * 32; idx += blockDim.x) {
        int r = idx / 32, c = idx % 32;
        Zc[r][c] = (c < ncol && r == c0 + c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int u = 0; u < SUBS; ++u) {
        const int s0 = u * NB;
        if (s0 >= w) break;
        const int ws = min(NB, w - s0);
        for (int idx = threadIdx.x; idx < ws * ws; idx += blockDim.x) {
            int r = idx % ws, c = idx / ws;
            Lb[r][c] = (r > c) ? (double)F[(int64_t)(k0 + s0 + c) * f + k0 + s0 + r] : 0.0;
        }
        for (int idx = threadIdx.x; idx < ws * 32; idx += blockDim.x) {
            int t = idx / 32, c = idx % 32;
            Zp[t][c] = Zc[piv[g0 + s0 + t] - k0][c];
        }
        __syncthreads();
        // forward substitution with the unit-lower L11, one thread per column
        if (threadIdx.x < 32) {
            const int c = threadIdx.x;
            for (int t = 1; t < ws; ++t) {
                double acc = Zp[t][c];
                for (int k = 0; k < t; ++k) acc -= Lb[t][k] * Zp[k][c];
                Zp[t][c] = acc;
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < ws * 32; idx += blockDim.x) {
            int t = idx / 32, c = idx % 32;
            Zc[s0 + t][c] = Zp[t][c];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < (w - s0 - ws) * 32; idx += blockDim.x) {
            int r = s0 + ws + idx / 32, c = idx % 32;
            double acc = 0.0;
            for (int t = 0; t < ws; ++t) acc += (double)F[(int64_t)(k0 + s0 + t) * f + k0 + r] * Zc[s0 + t][c];
            Zc[r][c] -= acc;
        }
        __syncthreads();
    }
    T *M = Mall + d.moff;
    for (int idx = threadIdx.x; idx < ncol * w; idx += blockDim.x) {
        int c = idx / w, r = idx % w;
        M[(int64_t)(c0 + c) * w + r] = (T)Zc[r][c];
    }
}

// G = [M; L21 M] of a solve panel (rows [k0, f) of the front x the panel's w columns) into the
// packed solve factor (column-major, leading dimension sg_ld(f - k0)).  CTA (x: the step's RBB-row
// tiles, y: 256-column halves of the panel) computes a 64 x 256 block of L21 M in 32-deep chunks
// of the contraction (16 x 16 threads, 4 x 16 outputs each); rows of the panel itself take M.
template <class T>
__global__ void __launch_bounds__(256) k_apply_m(const SolveDesc *sdescs, int nd, const int64_t *fo,
                                                 const int32_t *fsz, const T *arena, const T *Mall, T *Gp) {
    constexpr int KC = 32, CW = 256, MSL = CW + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *As = reinterpret_cast<T *>(smraw);  // RBB x (KC + 1): rows of L21, one contraction chunk
    T *Ms = As + RBB * (KC + 1);           // KC x MSL: the chunk of M
    const int di = find_sdesc_b(sdescs, nd, blockIdx.x);
    const SolveDesc d = sdescs[di];
    const int s = d.front, f = fsz[s], k0 = d.k0, w = d.w;
    const int cb = blockIdx.y * CW;  // first column of this half
    if (cb >= w) return;
    const int r0 = (int)(blockIdx.x - d.offb) * RBB;  // first row, relative to k0
    const int nr = min(RBB, w + d.m2 - r0);
    if (nr <= 0) return;
    const T *F = arena + fo[s];
    const T *M = Mall + d.moff;
    T *G = Gp + d.goff;
    const int64_t ld = sg_ld(w + d.m2);
    const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;
    T acc[4][16];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[i][j] = T(0);
    if (r0 + nr > w) {  // the tile has rows of L21
        for (int kc0 = 0; kc0 < w; kc0 += KC) {
            const int kc = min(KC, w - kc0);
            __syncthreads();
            for (int idx = threadIdx.x; idx < RBB * KC; idx += blockDim.x) {
                const int i = idx % RBB, k = idx / RBB;
                As[i * (KC + 1) + k] = (i < nr && k < kc) ? F[(int64_t)(k0 + kc0 + k) * f + k0 + r0 + i] : T(0);
            }
            for (int idx = threadIdx.x; idx < KC * CW; idx += blockDim.x) {
                const int k = idx % KC, c = idx / KC;
                Ms[k * MSL + c] = (k < kc && cb + c < w) ? M[(int64_t)(cb + c) * w + kc0 + k] : T(0);
            }
            __syncthreads();
#pragma unroll 4
            for (int k = 0; k < KC; ++k) {
                T a[4], bv[16];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[(tr + 16 * i) * (KC + 1) + k];
#pragma unroll
                for (int j = 0; j < 16; ++j) bv[j] = Ms[k * MSL + tc + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[i][j] += a[i] * bv[j];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = tr + 16 * i;
        if (row >= nr) continue;
        const int rr = r0 + row;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = cb + tc + 16 * j;
            if (col >= w) continue;
            G[(int64_t)col * ld + rr] = rr < w ? M[(int64_t)col * w + rr] : acc[i][j];
        }
    }
}

// Forward solve step over the row blocks (RBF rows of [k0, f)) of every panel of the step and of
// every job of the launch: a block of job j's panel with z = Z[panel] (PB >= p, zero-padded) gives
// Zs = M z on the panel's own rows and Z -= (L21 M) z on the rows below.  CTAs walk the (job, row
// block) items with a grid stride (the grid is the resident capacity, so there is no tail wave).
// Per item the RBF x w tile of G is copied to shared memory with 16-byte cp.async (issued before the
// wait on the previous step for the first item, since G is read-only); warp j then takes columns
// [32 j, 32 j + 32) and lane i row i, and the eight partial sums meet in shared memory in a fixed
// order (results do not depend on which CTA takes an item).
template <class T>
__host__ __device__ constexpr size_t fwd_gtile_bytes() { return sizeof(T) * (size_t)SPW * RBF; }

template <class T>
__device__ __forceinline__ void fwd_tile_issue(T *Gs, const T *G, int64_t ld, int w, int rows_avail) {
    // 16-byte pieces: column c, rows [4 v, 4 v + 4) of the tile; rows past the padded column end are
    // not copied (their lanes are discarded)
    constexpr int E = 16 / sizeof(T), PPC = RBF / E;
    for (int u = threadIdx.x; u < w * PPC; u += blockDim.x) {
        const int c = u / PPC, v = u - c * PPC;
        if (v * E < rows_avail) cp_async16(Gs + c * RBF + v * E, G + (int64_t)c * ld + v * E);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <class T, int PB>
__global__ void __launch_bounds__(256, PB <= 8 ? 4 : 2)
    k_fwd_step(const SolveDesc *sdescs, const int32_t *blk_desc, int nrb, int K, const int64_t *zo,
               const int32_t *sn_start, const SolveBufs<T> *jb, int p, LaunchTrace *tr) {
    static_assert(SPW == 256 && RBF == 32, "eight warps of 32 columns, a lane per row");
    TraceScope trace_scope(tr);
    extern __shared__ __align__(16) unsigned char smraw[];
    T *Gs = reinterpret_cast<T *>(smraw);                         // SPW columns x RBF rows
    T *zp = reinterpret_cast<T *>(smraw + fwd_gtile_bytes<T>());  // SPW x PB
    T *red = Gs;                                                  // 8 x PB x RBF partials, after the products
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int nit = nrb * K;
    bool waited = false;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const int job = it / nrb, b = it - job * nrb;
        const SolveBufs<T> J = jb[job];
        const int di = blk_desc[b];
        const SolveDesc d = sdescs[di];
        const int s = d.front, k0 = d.k0, w = d.w, R = w + d.m2;
        const int r0 = (b - (int)d.off) * RBF;  // relative to k0
        const int nr = min(RBF, R - r0);
        const int64_t zb = zo[s] + k0, ld = sg_ld(R);
        fwd_tile_issue(Gs, J.G + d.goff + r0, ld, w, (int)(ld - r0));
        // this thread's outputs o = threadIdx.x + 256 u (row i = o % RBF, right-hand side q = o / RBF)
        constexpr int NO = RBF * PB / 256;
        static_assert(NO * 256 == RBF * PB, "outputs per thread");
        T dg[NO], zold[NO];
#pragma unroll
        for (int u = 0; u < NO; ++u) {
            const int o = threadIdx.x + 256 * u, i = o % RBF, q = o / RBF, rr = r0 + i;
            dg[u] = (i < nr && q < p && rr < w) ? J.D[(int64_t)sn_start[s] + k0 + rr] : T(1);
        }
        if (!waited) {
            pdl_wait();
            pdl_trigger();
            waited = true;
        }
        for (int idx = threadIdx.x; idx < w * PB; idx += blockDim.x) {
            const int c = idx / PB, q = idx % PB;
            zp[idx] = q < p ? J.Z[(zb + c) * p + q] : T(0);
        }
#pragma unroll
        for (int u = 0; u < NO; ++u) {
            const int o = threadIdx.x + 256 * u, i = o % RBF, q = o / RBF, rr = r0 + i;
            zold[u] = (i < nr && q < p && rr >= w) ? J.Z[(zb + rr) * p + q] : T(0);
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        T acc[PB];
#pragma unroll
        for (int q = 0; q < PB; ++q) acc[q] = T(0);
        {
            const int c0 = wp * 32, c1 = min(w, c0 + 32);
            if (lane < nr) {
                for (int c = c0; c < c1; ++c) {
                    const T l = Gs[c * RBF + lane];
#pragma unroll
                    for (int q = 0; q < PB; ++q) acc[q] += l * zp[c * PB + q];
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PB; ++q) red[(wp * PB + q) * RBF + lane] = acc[q];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NO; ++u) {
            const int o = threadIdx.x + 256 * u, i = o % RBF, q = o / RBF;
            if (i >= nr || q >= p) continue;
            T v = T(0);
#pragma unroll
            for (int j = 0; j < 8; ++j) v += red[(j * PB + q) * RBF + i];
            const int rr = r0 + i;
            if (rr < w) {
                // a panel row is final here: also its diagonal-scaled value for the backward sweep
                const int64_t gr = (int64_t)sn_start[s] + k0 + rr;
                J.Zs[(zb + rr) * p + q] = v;
                J.yfw[gr * p + q] = v / dg[u];
            } else {
                J.Z[(zb + rr) * p + q] = zold[u] - v;
            }
        }
        __syncthreads();  // Gs, zp and red are reused by the next item
    }
    if (!waited) pdl_wait();
}

// Narrow steps (every panel of the step at most 32 columns wide, e.g. the leaves of the tree): one
// warp per 32-row block (RBF) instead of CTAs of RBF rows x 8 column chunks, most of which would idle.
// Forward: lane c holds z_panel row c; lane r accumulates row r of the block's G z, the z values
// broadcast by shuffles.  The block's rows of G and the panel's pivots are read before the wait on
// the previous step.
template <class T, int PB>
__global__ void __launch_bounds__(256) k_fwd_narrow(const SolveDesc *sdescs, const int32_t *blk_desc, int nblk,
                                                    const int64_t *zo, const int32_t *sn_start,
                                                    const SolveBufs<T> *jb, int p, LaunchTrace *tr) {
    static_assert(RBF == 32, "one warp per row block");
    TraceScope trace_scope(tr);
    const T *Gp = jb[blockIdx.z].G, *Dg = jb[blockIdx.z].D;
    T *Z = jb[blockIdx.z].Z, *Zs = jb[blockIdx.z].Zs, *yfw = jb[blockIdx.z].yfw;
    const int lane = threadIdx.x & 31, item = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (item >= nblk) {
        pdl_wait();
        return;
    }
    const SolveDesc d = sdescs[blk_desc[item]];
    const int s = d.front, k0 = d.k0, w = d.w, R = w + d.m2;
    const int r = (int)(item - d.off) * RBF + lane;  // this lane's row, relative to k0
    const int64_t zb = zo[s] + k0, ld = sg_ld(R), g0 = (int64_t)sn_start[s] + k0;
    const T *G = Gp + d.goff + r;
    T gl[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) gl[c] = (c < w && r < R) ? G[(int64_t)c * ld] : T(0);
    const T dg = r < w ? Dg[g0 + r] : T(1);
    pdl_wait();
    pdl_trigger();
    T zr[PB], zold[PB];
#pragma unroll
    for (int q = 0; q < PB; ++q) {
        zr[q] = (lane < w && q < p) ? Z[(zb + lane) * p + q] : T(0);
        zold[q] = (r >= w && r < R && q < p) ? Z[(zb + r) * p + q] : T(0);
    }
    T acc[PB];
#pragma unroll
    for (int q = 0; q < PB; ++q) acc[q] = T(0);
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        if (c >= w) break;
#pragma unroll
        for (int q = 0; q < PB; ++q) acc[q] += gl[c] * __shfl_sync(0xffffffffu, zr[q], c);
    }
    if (r < R) {
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            if (q >= p) break;
            if (r < w) {
                Zs[(zb + r) * p + q] = acc[q];
                yfw[(g0 + r) * p + q] = acc[q] / dg;
            } else {
                Z[(zb + r) * p + q] = zold[q] - acc[q];
            }
        }
    }
}

// Backward narrow step: lane c accumulates x_panel[c] = sum_r G[r][c] v[r] over 32-row chunks;
// lane j of a chunk reads row j of v (yfw, Zs or the ancestors' x, as in k_bwd_step) and the
// values broadcast by shuffles.  Every panel is handled by one warp, so there are no partial sums.
template <class T, int PB>
__global__ void __launch_bounds__(256) k_bwd_narrow(const SolveDesc *sdescs, int nd, const int64_t *zo,
                                                    const int32_t *nc, const int32_t *sn_start,
                                                    const int64_t *rows_off, const int32_t *rows,
                                                    const SolveBufs<T> *jb, int p, LaunchTrace *tr) {
    TraceScope trace_scope(tr);
    const T *Gp = jb[blockIdx.z].G, *yfw = jb[blockIdx.z].yfw;
    T *Zs = jb[blockIdx.z].Zs, *x = jb[blockIdx.z].y;
    const int lane = threadIdx.x & 31, di = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (di >= nd) {
        pdl_wait();
        return;
    }
    const SolveDesc d = sdescs[di];
    const int s = d.front, k0 = d.k0, w = d.w, R = w + d.m2, ncs = nc[s];
    const int64_t zb = zo[s] + k0, ld = sg_ld(R), g0 = (int64_t)sn_start[s] + k0;
    const T *G = Gp + d.goff + (int64_t)lane * ld;  // this lane's column
    const int32_t *rw = rows + rows_off[s] + k0;
    T gl[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) gl[j] = (lane < w && j < R) ? G[j] : T(0);
    const int rowx = lane < R && k0 + lane >= ncs ? rw[lane] : 0;
    pdl_wait();
    pdl_trigger();
    T acc[PB];
#pragma unroll
    for (int q = 0; q < PB; ++q) acc[q] = T(0);
    for (int rb = 0; rb < R; rb += 32) {
        const int rr = rb + lane;
        T vr[PB];
        {
            const T *sp = nullptr;
            T sg = T(0);
            if (rr < R) {
                if (rr < w) {
                    sp = yfw + (g0 + rr) * p;
                    sg = T(1);
                } else if (k0 + rr < ncs) {
                    sp = Zs + (zb + rr) * p;
                    sg = T(-1);
                } else {
                    sp = x + (int64_t)(rb == 0 ? rowx : rw[rr]) * p;
                    sg = T(-1);
                }
            }
#pragma unroll
            for (int q = 0; q < PB; ++q) vr[q] = (sp && q < p) ? sg * sp[q] : T(0);
        }
        if (rb > 0) {  // this chunk's column entries, all loads in flight before the products
#pragma unroll
            for (int j = 0; j < 32; ++j) gl[j] = (lane < w && rb + j < R) ? G[rb + j] : T(0);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j)
#pragma unroll
            for (int q = 0; q < PB; ++q) acc[q] += gl[j] * __shfl_sync(0xffffffffu, vr[q], j);
    }
    if (lane < w) {
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            if (q >= p) break;
            Zs[(zb + lane) * p + q] = acc[q];
            x[(g0 + lane) * p + q] = acc[q];
        }
    }
}

// Backward update (grid: the launch's (i, j) items x column chunks of panel i): acc_i -= G_i[rows of
// panel j]^T x_j for an earlier panel i of the same front, where x_j = acc_j (in Zs) is final.  The
// RBK x RBB tile of G_i is copied before waiting.  When panel j directly follows panel i this is the
// last contribution to acc_i, which is then written to x as well.  Each accumulator chunk has one
// writer per launch, so the updates are deterministic.
template <class T, int PB>
__global__ void __launch_bounds__(256) k_bwd_update(const SolveDesc *sdescs, const int32_t *items, const int64_t *zo,
                                                    const int32_t *sn_start, const SolveBufs<T> *jb, int p,
                                                    LaunchTrace *tr) {
    TraceScope trace_scope(tr);
    const T *Gp = jb[blockIdx.z].G;
    T *Zs = jb[blockIdx.z].Zs, *x = jb[blockIdx.z].y;
    constexpr int E = 16 / sizeof(T);
    extern __shared__ __align__(16) unsigned char smraw[];
    T *Gs = reinterpret_cast<T *>(smraw);    // RBB columns x bwd_ldg rows
    T *vs = Gs + RBB * bwd_ldg<T>();         // RBK x PB
    T *red = PB == 8 ? Gs : vs + RBK * PB;  // 8 warps x 8 x RBB partial sums
    const SolveDesc di = sdescs[items[2 * blockIdx.x]], dj = sdescs[items[2 * blockIdx.x + 1]];
    const int cc = blockIdx.y * RBB;
    if (cc >= di.w) {
        pdl_wait();
        return;
    }
    const int s = di.front, wc = min(RBB, di.w - cc), wj = dj.w, nrv = (wj + E - 1) / E;
    const int64_t ldi = sg_ld(di.w + di.m2);
    bwd_tile_issue(Gs, Gp + di.goff + (int64_t)cc * ldi + (dj.k0 - di.k0), ldi, wc, nrv);
    const int64_t zi = zo[s] + di.k0 + cc, zj = zo[s] + dj.k0;
    const bool fin = dj.k0 == di.k0 + di.w;
    pdl_wait();
    pdl_trigger();
    {
        static_assert(RBK == 256, "one row of v per thread");
        const int r = threadIdx.x;
        T *vr = vs + r * PB;
#pragma unroll
        for (int q = 0; q < PB; ++q) vr[q] = (r < wj && q < p) ? Zs[(zj + r) * p + q] : T(0);
    }
    // the accumulator entries this thread updates: outputs o = threadIdx.x + 256 h of each 8-wide
    // chunk of right-hand sides (column c = o % RBB, q = q0 + o / RBB)
    constexpr int NQ = PB / 8;
    T old[NQ][2];
#pragma unroll
    for (int u = 0; u < NQ; ++u)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int o = threadIdx.x + 256 * h, q = 8 * u + o / RBB, c = o % RBB;
            old[u][h] = (c < wc && q < p) ? Zs[(zi + c) * p + q] : T(0);
        }
    cp_async_commit_wait();
    __syncthreads();
    T *xp = x + ((int64_t)sn_start[s] + di.k0 + cc) * p;
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
        T o2[2];
        bwd_tile_product<T, PB>(Gs, vs, red, nrv * E, 8 * u, o2);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int o = threadIdx.x + 256 * h, q = 8 * u + o / RBB, c = o % RBB;
            if (c < wc && q < p) {
                const T v = old[u][h] - o2[h];
                Zs[(zi + c) * p + q] = v;
                if (fin) xp[c * p + q] = v;
            }
        }
    }
}

__global__ void k_trace_reset(LaunchTrace *tr, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        tr[i].t0 = ~0ull;
        tr[i].t1 = 0ull;
    }
}

// Forward gather of one level from the row lists: Z[dst] = y[own] (or 0) + the children's
// contributions in tree order; one thread per (row, right-hand side).
template <class T>
__global__ void k_fwd_gather_rows(int64_t nrows, const int64_t *dst, const int64_t *own, const int64_t *cptr,
                                  const int64_t *src, const SolveBufs<T> *jb, int p, LaunchTrace *tr) {
    TraceScope trace_scope(tr);
    const T *y = jb[blockIdx.z].y;
    T *Z = jb[blockIdx.z].Z;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = t / p;
    const int q = (int)(t - row * p);
    int64_t o = -1, d = 0, c0 = 0, c1 = 0;
    if (row < nrows) {
        o = own[row];
        d = dst[row];
        c0 = cptr[row];
        c1 = cptr[row + 1];
    }
    pdl_wait();
    pdl_trigger();
    if (row >= nrows) return;
    T v = o >= 0 ? y[o * p + q] : T(0);
    for (int64_t c = c0; c < c1; ++c) v += Z[src[c] * p + q];
    Z[d * p + q] = v;
}

// Start of the backward sweep of one level (grid: the level's row blocks x column chunks), tiles
// of RBK rows x RBB columns of G = [M; L21 M]: each panel's accumulator acc = G^T v with
// v = [y_panel; 0; -x_cb] -- the panel's forward result yfw (pivoted order), zero on the rows of the
// front's later panels (their share is subtracted by k_bwd_update once their x is known), and the
// contribution block's x, fixed by the ancestors and read through the front's row list (static,
// read before waiting).  The tile is copied from the packed solve factor to shared memory (16-byte
// cp.async) before waiting for the previous launch.  A panel with one row block writes directly;
// otherwise each block writes its partial sums and the last block of a (panel, column chunk) to
// finish (counted with an atomic, after a fence) adds the partials in a fixed order and re-arms the
// counter.  The accumulator goes to Zs; for the front's last panel it is final and goes to x too.
template <class T, int PB>
__global__ void __launch_bounds__(256) k_bwd_step(const SolveDesc *sdescs, const int32_t *blk_desc, const int64_t *zo,
                                                  const int32_t *nc, const int32_t *sn_start,
                                                  const int64_t *rows_off, const int32_t *rows,
                                                  const SolveBufs<T> *jb, int64_t cnt_off, int p, LaunchTrace *tr) {
    TraceScope trace_scope(tr);
    const T *Gp = jb[blockIdx.z].G, *yfw = jb[blockIdx.z].yfw;
    T *Zs = jb[blockIdx.z].Zs, *P = jb[blockIdx.z].P, *x = jb[blockIdx.z].y;
    unsigned int *cnt = jb[blockIdx.z].cnt + cnt_off;
    constexpr int E = 16 / sizeof(T);
    extern __shared__ __align__(16) unsigned char smraw[];
    T *Gs = reinterpret_cast<T *>(smraw);    // RBB columns x bwd_ldg rows
    T *vs = Gs + RBB * bwd_ldg<T>();         // RBK x PB
    T *red = PB == 8 ? Gs : vs + RBK * PB;  // 8 warps x 8 x RBB partial sums
    __shared__ int s_last;
    const int di = blk_desc[blockIdx.x];
    const SolveDesc d = sdescs[di];
    const int cc = blockIdx.y * RBB;
    if (cc >= d.w) {
        pdl_wait();
        return;
    }
    const int s = d.front, k0 = d.k0, w = d.w, ncs = nc[s], R = w + d.m2, cb0 = ncs - k0;
    const int b = (int)(blockIdx.x - d.offk_l), nb = bwd_start_blocks(R, cb0);
    const int r0 = b == 0 ? 0 : (cb0 & ~3) + (b - 1) * RBK;  // relative to k0
    const int nr = b == 0 ? w : min(RBK, R - r0), nrv = (nr + E - 1) / E;
    const int wc = min(RBB, w - cc);
    const int64_t zb = zo[s] + k0, ld = sg_ld(R);
    bwd_tile_issue(Gs, Gp + d.goff + (int64_t)cc * ld + r0, ld, wc, nrv);
    // thread i loads row i of v: the panel's y, zero on later panels' rows, -x on the contribution block
    static_assert(RBK == 256, "one row of v per thread");
    const int i = threadIdx.x, rr = r0 + i;
    const int kind = i >= nr ? 0 : (b == 0 ? 1 : (rr < cb0 ? 0 : 3));
    const int64_t src = kind == 1 ? ((int64_t)sn_start[s] + k0 + rr) * p
                      : kind == 3 ? (int64_t)rows[rows_off[s] + k0 + rr] * p : 0;
    pdl_wait();
    pdl_trigger();
    {
        T *vr = vs + i * PB;
        if (kind == 0) {
#pragma unroll
            for (int q = 0; q < PB; ++q) vr[q] = T(0);
        } else {
            const T *sp = kind == 1 ? yfw + src : x + src;
            const T sg = kind == 1 ? T(1) : T(-1);
#pragma unroll
            for (int q = 0; q < PB; ++q) vr[q] = q < p ? sg * sp[q] : T(0);
        }
    }
    cp_async_commit_wait();
    __syncthreads();
    const int64_t tile = (int64_t)RBB * PB;
    T *out = P + ((d.offk_l + b) * SUBS + blockIdx.y) * tile;
    T *zsp = Zs + (zb + cc) * p;
    T *xp = k0 + w >= ncs ? x + ((int64_t)sn_start[s] + k0 + cc) * p : nullptr;
#pragma unroll
    for (int q0 = 0; q0 < PB; q0 += 8) {
        T o2[2];
        bwd_tile_product<T, PB>(Gs, vs, red, nrv * E, q0, o2);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int o = threadIdx.x + 256 * h, q = q0 + o / RBB, c = o % RBB;
            if (nb == 1) {
                if (c < wc && q < p) {
                    zsp[c * p + q] = o2[h];
                    if (xp) xp[c * p + q] = o2[h];
                }
            } else {
                out[q * RBB + c] = o2[h];
            }
        }
    }
    if (nb == 1) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int prev = atomicAdd(&cnt[(size_t)di * SUBS + blockIdx.y], 1u);
        s_last = prev == (unsigned int)(nb - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    bwd_finish<T, PB>(P + (d.offk_l * SUBS + blockIdx.y) * tile, (int64_t)SUBS * tile, nb, wc, p, zsp, xp, Gs);
    if (threadIdx.x == 0) cnt[(size_t)di * SUBS + blockIdx.y] = 0u;
}

// ------------------------------------------------------------------------------------------
// Host drivers
// ------------------------------------------------------------------------------------------
template <class T>
static size_t build_m_smem() { return 8 * ((size_t)(SPW + NB) * 33 + (size_t)NB * (NB + 1)); }
template <class T>
static size_t trsm_smem() { return sizeof(T) * (size_t)2 * NB * (NB + 1); }
template <class T>
static size_t apply_m_smem() { return sizeof(T) * ((size_t)RBB * 33 + (size_t)32 * 257); }
template <class T, int PB>
static size_t fwd_step_smem() { return fwd_gtile_bytes<T>() + sizeof(T) * (size_t)SPW * PB; }
template <class T, int PB>
static size_t bwd_step_smem() { return bwd_tile_smem<T, PB>(); }
static int rhs_pad(int p) { return p <= 8 ? 8 : (p <= 16 ? 16 : 32); }

template <class T, int PB>
static void set_step_attrs() {
    smem_limit((const void *)k_fwd_step<T, PB>, fwd_step_smem<T, PB>());
    smem_limit((const void *)k_bwd_step<T, PB>, bwd_step_smem<T, PB>());
    smem_limit((const void *)k_bwd_update<T, PB>, bwd_step_smem<T, PB>());
}

// CTAs of 256 threads of `kern` (dynamic shared memory smem) that the device holds at once: the grid
// of the grid-stride solve kernels.  Cached per device and kernel.
template <class K>
static int64_t resident_grid(K *kern, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int64_t> cache;
    int dev = 0;
    MBL_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, reinterpret_cast<const void *>(kern));
    auto itc = cache.find(key);
    if (itc != cache.end()) return itc->second;
    int occ = 0, sms = 0;
    MBL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem));
    MBL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t g = (int64_t)std::max(1, occ) * sms;
    cache[key] = g;
    return g;
}

template <class T>
static void set_solve_attrs() {
    smem_limit((const void *)k_build_m<T>, build_m_smem<T>());
    smem_limit((const void *)k_apply_m<T>, apply_m_smem<T>());
    set_step_attrs<T, 8>();
    set_step_attrs<T, 16>();
    set_step_attrs<T, 32>();
}

template <class T>
static void factor_impl(Factorization &fz, cudaStream_t st) {
    Plan &p = *fz.plan;
    mbl_sector *sec = fz.sec;
    LeanArena *lean = fz.lean.get();
    T *arena = lean ? reinterpret_cast<T *>(lean->base) : static_cast<T *>(fz.arena.m.p);
    T *Dg = static_cast<T *>(fz.D.m.p);
    T *wscr = static_cast<T *>(fz.wscr.m.p);
    T *Gp = static_cast<T *>(fz.gpk.m.p);
    MBL_CUDA(cudaMemsetAsync(Gp, 0, (size_t)p.sg_elems * sizeof(T), st));  // padding rows of G stay zero
    // G = [M; L21 M] of the solve panels of level l (the panels' M blocks first)
    auto build_g_level = [&](int l) {
        if (p.lvl_nd[l] <= 0) return;
        ProfScope ps_g(fz.ctx, "f_build_g", 0.0, st);
        k_build_m<T><<<dim3((unsigned)p.lvl_nd[l], SPW / 32), 256, build_m_smem<T>(), st>>>(
            p.d_sdescs.data() + p.lvl_d0[l], p.d_sn_fo.data(), p.d_sn_f.data(), p.d_sn_start.data(), arena,
            fz.piv.data(), static_cast<T *>(fz.M.m.p));
        MBL_LAUNCH_CHECK();
        for (int si = p.lvl_sstep_ptr[l]; si < p.lvl_sstep_ptr[l + 1]; ++si) {
            const SolveStep &ss = p.ssteps[si];
            k_apply_m<T><<<dim3((unsigned)ss.nrbb, (SPW + 255) / 256), 256, apply_m_smem<T>(), st>>>(
                p.d_sdescs.data() + ss.d0, ss.nd, p.d_sn_fo.data(), p.d_sn_f.data(), arena,
                static_cast<const T *>(fz.M.m.p), Gp);
            MBL_LAUNCH_CHECK();
        }
    };
    smem_limit((const void *)k_panel_trsm<T>, trsm_smem<T>());
    set_solve_attrs<T>();
    MBL_CUDA(cudaMemsetAsync(fz.counters.data(), 0, 5 * sizeof(unsigned long long), st));
    MBL_CUDA(cudaMemsetAsync(fz.counters.data() + 4, 0x7f, sizeof(unsigned int), st));  // min |d| starts huge
    for (int l = 0; l < p.nlevels; ++l) {
        int na = p.asm_ptr[l + 1] - p.asm_ptr[l];
        if (lean)
            for (size_t r = 0; r < p.regions.size(); ++r)
                if (p.regions[r].level == l) lean->map_region(p, r);
        {
            ProfScope ps_asm(fz.ctx, "f_assemble", 0.0, st);
            k_assemble<T><<<na, 256, 0, st>>>(p.d_asm_items.data() + p.asm_ptr[l], p.d_sn_fo.data(), p.d_sn_f.data(),
                                              p.d_sn_nc.data(), p.d_sn_start.data(), p.d_ch_ptr.data(),
                                              p.d_ch_list.data(), p.d_sn_rel_off.data(), p.d_relind.data(),
                                              p.d_amap_ptr.data(), p.d_amap_src.data(), p.d_amap_row.data(),
                                              sec->val.data(), fz.sigma, arena);
            MBL_LAUNCH_CHECK();
        }
        if (lean) {  // contribution blocks last read by this assembly
            MBL_CUDA(cudaStreamSynchronize(st));
            for (size_t r = 0; r < p.regions.size(); ++r)
                if (p.regions[r].level < l && p.regions[r].release == l) lean->unmap_region(p, r);
        }
        for (int si = p.lvl_step_ptr[l]; si < p.lvl_step_ptr[l + 1]; ++si) {
            const PanelStep &stp = p.steps[si];
            const PanelDesc *dd = p.d_descs.data() + stp.d0;
            unsigned int *cmax = static_cast<unsigned int *>(fz.cmax.m.p);
            {  // pivot search, diagonal block and trsm of the panel
                ProfScope ps_pan(fz.ctx, "f_panel", 0.0, st);
                MBL_CUDA(cudaMemsetAsync(cmax, 0, (size_t)stp.nd * NB * sizeof(unsigned int), st));
                if (stp.n2 > 0) {
                    k_panel_colmax<T><<<(unsigned)stp.n2, PANEL_THREADS, 0, st>>>(dd, stp.nd, p.d_sn_fo.data(), p.d_sn_f.data(), arena,
                                                                       cmax);
                    MBL_LAUNCH_CHECK();
                }
                k_panel_diag<T><<<stp.nd, 128, 0, st>>>(dd, p.d_sn_fo.data(), p.d_sn_f.data(), p.d_sn_start.data(), arena,
                                                        Dg, fz.piv.data(), fz.tiny, fz.counters.data(), cmax);
                MBL_LAUNCH_CHECK();
                if (stp.n2 > 0) {
                    k_panel_trsm<T><<<(unsigned)stp.n2, PANEL_THREADS, trsm_smem<T>(), st>>>(dd, stp.nd, p.d_sn_fo.data(),
                                                                                 p.d_sn_f.data(), p.d_sn_start.data(), arena,
                                                                                 Dg, fz.piv.data(), wscr,
                                                                                 fz.counters.data() + 3,
                                                                                 fz.tma ? fz.pieces.m.p : nullptr,
                                                                                 fz.prow,
                                                                                 fz.tma && sizeof(T) == 4 ? fz.tc_mode : 0);
                    MBL_LAUNCH_CHECK();
                }
            }
            if (stp.n3 > 0) {
                double fl = 0.0;  // algorithmic flops: lower triangle of the trailing block, 2 per entry per k
                for (int q = stp.d0; q < stp.d0 + stp.nd; ++q)
                    fl += (double)p.descs[q].m2 * (p.descs[q].m2 + 1) * p.descs[q].w;
                // the autotuned tile shape of this step's size class (tensor cores unless the tuning found the
                // CUDA-core tiles faster for it)
                const bool tc = sizeof(T) == 4 && fz.tc_mode != 0 &&
                                (!p.tuned[fz.tc_mode] || p.tune_tc[fz.tc_mode][p.step_class[si]]);
                if (tc) {
                    ProfScope ps(fz.ctx, "schur_tc", fl, st);
                    if (fz.tma)
                        launch_schur_tma(stp, dd, p.d_sn_fo.data(), p.d_sn_f.data(), reinterpret_cast<float *>(arena),
                                         fz.tmap, fz.counters.data() + 2, st, fz.tc_mode == 2);
                    else
                        launch_schur_tc(stp, dd, p, reinterpret_cast<float *>(arena),
                                        reinterpret_cast<const float *>(wscr), fz.counters.data() + 2, st,
                                        fz.tc_mode == 2);
                } else {
                    ProfScope ps(fz.ctx, sizeof(T) == 8 ? "schur_fp64" : "schur_fp32", fl, st);
                    k_panel_update<T><<<(unsigned)stp.n3, 256, 0, st>>>(dd, stp.nd, p.d_sn_fo.data(), p.d_sn_f.data(),
                                                                        arena, wscr);
                    MBL_LAUNCH_CHECK();
                }
            }
        }
        if (lean) {  // the level's factor columns move to G; then they, and its root fronts, can go
            build_g_level(l);
            MBL_CUDA(cudaStreamSynchronize(st));
            for (int64_t i = p.lean_prefix_ptr[l]; i < p.lean_prefix_ptr[l + 1]; ++i)
                lean->unmap_chunk(p, (size_t)p.lean_prefix[i].first, (size_t)p.lean_prefix[i].second);
            for (size_t r = 0; r < p.regions.size(); ++r)
                if (p.regions[r].level == l && p.regions[r].release == l) lean->unmap_region(p, r);
        }
    }
    if (lean) return;
    // block operators of the solve panels, then G = [M; L21 M] of each panel into the packed solve factor
    if (!p.sdescs.empty()) {
        ProfScope ps_g(fz.ctx, "f_build_g", 0.0, st);
        dim3 grid((unsigned)p.sdescs.size(), SPW / 32);
        k_build_m<T><<<grid, 256, build_m_smem<T>(), st>>>(p.d_sdescs.data(), p.d_sn_fo.data(), p.d_sn_f.data(),
                                                           p.d_sn_start.data(), arena, fz.piv.data(),
                                                           static_cast<T *>(fz.M.m.p));
        MBL_LAUNCH_CHECK();
        for (const SolveStep &ss : p.ssteps) {
            k_apply_m<T><<<dim3((unsigned)ss.nrbb, (SPW + 255) / 256), 256, apply_m_smem<T>(), st>>>(p.d_sdescs.data() + ss.d0, ss.nd,
                                                                           p.d_sn_fo.data(), p.d_sn_f.data(), arena,
                                                                           static_cast<const T *>(fz.M.m.p), Gp);
            MBL_LAUNCH_CHECK();
        }
    }
}

__global__ void k_fill_hash(float *x, int64_t n, uint32_t seed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    x[i] = (float)(h & 0xFFFFFF) * (1.0f / 16777216.0f) - 0.5f;
}

void tune_schur(Factorization &fz, cudaStream_t st) {
    Plan &p = *fz.plan;
    const int mode = fz.tc_mode;
    if (fz.prec != MBL_PREC_FP32 || mode < 1 || mode > 2 || !fz.tma) return;
    std::lock_guard<std::mutex> lk(p.tune_mu);
    if (p.tuned[mode]) return;
    bool present[TUNE_CLASSES] = {};
    for (int32_t c : p.step_class) present[c] = true;
    unsigned long long *err = fz.counters.data() + 2;
    for (int c = 0; c < TUNE_CLASSES; ++c) {
        p.tune_tc[mode][c] = 1;
        p.tune_us[mode][c][0] = p.tune_us[mode][c][1] = 0.f;
        if (!present[c]) continue;
        // a synthetic front whose one 64-column panel leaves a trailing block in the middle of the class
        const int m2 = (int)(64.0 * (double)(1 << c) * 1.41), f = m2 + NB;
        DVec<float> F, W;
        DVec<char> pc;
        DVec<PanelDesc> dd;
        DVec<int64_t> fo;
        DVec<int32_t> fsz;
        F.alloc(fz.ctx, (size_t)f * f);
        W.alloc(fz.ctx, (size_t)m2 * NB);
        pc.alloc(fz.ctx, (size_t)4 * m2 * NB * (mode == 2 ? 2 : 4));
        dd.alloc(fz.ctx, 1);
        fo.alloc(fz.ctx, 1);
        fsz.alloc(fz.ctx, 1);
        k_fill_hash<<<(unsigned)(((int64_t)f * f + 255) / 256), 256, 0, st>>>(F.data(), (int64_t)f * f, 1u + c);
        MBL_LAUNCH_CHECK();
        k_fill_hash<<<(unsigned)(((int64_t)m2 * NB + 255) / 256), 256, 0, st>>>(W.data(), (int64_t)m2 * NB, 7u + c);
        MBL_LAUNCH_CHECK();
        MBL_CUDA(cudaMemsetAsync(pc.data(), 0, pc.size(), st));
        const PanelDesc d{0, 0, NB, m2, 0, 0, 0, 0};
        const int64_t z = 0;
        MBL_CUDA(cudaMemcpyAsync(dd.data(), &d, sizeof(d), cudaMemcpyHostToDevice, st));
        MBL_CUDA(cudaMemcpyAsync(fo.data(), &z, sizeof(z), cudaMemcpyHostToDevice, st));
        MBL_CUDA(cudaMemcpyAsync(fsz.data(), &f, sizeof(int), cudaMemcpyHostToDevice, st));
        alignas(64) unsigned char map[128];
        if (!encode_pieces_map(map, pc.data(), m2, mode == 2)) continue;
        PanelStep stp{};
        stp.nd = 1;
        const int64_t T64 = (m2 + TB - 1) / TB, T128 = (m2 + 127) / 128;
        stp.n3 = T64 * (T64 + 1) / 2;
        stp.n3t = T128 * (T128 + 1) / 2;
        cudaEvent_t e[3];
        for (auto &x : e) MBL_CUDA(cudaEventCreate(&x));
        float us[2] = {0.f, 0.f};
        for (int v = 0; v < 2; ++v) {
            auto run = [&] {
                if (v == 0)
                    launch_schur_tma(stp, dd.data(), fo.data(), fsz.data(), F.data(), map, err, st, mode == 2);
                else {
                    k_panel_update<float><<<(unsigned)stp.n3, 256, 0, st>>>(dd.data(), 1, fo.data(), fsz.data(),
                                                                            F.data(), W.data());
                    MBL_LAUNCH_CHECK();
                }
            };
            run();  // warm-up (and the kernel load)
            MBL_CUDA(cudaEventRecord(e[0], st));
            for (int r = 0; r < 3; ++r) run();
            MBL_CUDA(cudaEventRecord(e[1], st));
            MBL_CUDA(cudaEventSynchronize(e[1]));
            float ms = 0.f;
            MBL_CUDA(cudaEventElapsedTime(&ms, e[0], e[1]));
            us[v] = 1000.f * ms / 3.f;
        }
        for (auto &x : e) cudaEventDestroy(x);
        p.tune_us[mode][c][0] = us[0];
        p.tune_us[mode][c][1] = us[1];
        p.tune_tc[mode][c] = us[0] <= us[1] ? 1 : 0;
    }
    // the synthetic updates counted no real time-outs: clear the counter the factorization reads
    MBL_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned long long), st));
    MBL_CUDA(cudaStreamSynchronize(st));
    if (fz.lean) trim_device_pool(fz.ctx->device);  // the synthetic fronts' memory back to the device
    p.tuned[mode] = true;
}

void numeric_factor(Factorization &fz, cudaStream_t st) {
    if (fz.prec == MBL_PREC_FP64) factor_impl<double>(fz, st);
    else factor_impl<float>(fz, st);
}

// The level x panel sequence between the permutations for K jobs of one plan (grid z = job):
// jb[k] holds job k's buffers.  trb (optional) receives one launch record per launch.
template <class T, int PB>
static void solve_levels(const Plan &pl, const SolveBufs<T> *jb, unsigned K, int p, LaunchTrace *trb,
                         std::vector<int> *kinds, cudaStream_t st) {
    const size_t fsm = fwd_step_smem<T, PB>(), bsm = bwd_step_smem<T, PB>();
    const int64_t fwd_cap = resident_grid(k_fwd_step<T, PB>, fsm);
    int it = 0;
    auto next_tr = [&](int kind) -> LaunchTrace * {
        if (!trb) return nullptr;
        if (kinds) kinds->push_back(kind);
        return trb + it++;
    };
    for (int l = 0; l < pl.nlevels; ++l) {
        {
            const int64_t f0 = pl.lvl_fg_ptr[l], nrows = pl.lvl_fg_ptr[l + 1] - f0;
            launch_pdl(k_fwd_gather_rows<T>, dim3((unsigned)((nrows * p + 255) / 256), 1, K), dim3(256), 0, st, nrows,
                       pl.d_fg_dst.data() + f0, pl.d_fg_own.data() + f0, pl.d_fg_cptr.data() + f0,
                       (const int64_t *)pl.d_fg_src.data(), jb, p, next_tr(0));
        }
        for (int si = pl.lvl_sstep_ptr[l]; si < pl.lvl_sstep_ptr[l + 1]; ++si) {
            const SolveStep &ss = pl.ssteps[si];
            const SolveDesc *sd = pl.d_sdescs.data() + ss.d0;
            if (ss.maxw <= 32) {
                launch_pdl(k_fwd_narrow<T, PB>, dim3((unsigned)((ss.nrb + 7) / 8), 1, K), dim3(256), 0, st, sd,
                           (const int32_t *)pl.d_fblk_desc.data() + ss.fblk0, (int)ss.nrb, pl.d_sn_zo.data(),
                           pl.d_sn_start.data(), jb, p, next_tr(1));
                continue;
            }
            const int64_t items = ss.nrb * (int64_t)K;
            launch_pdl(k_fwd_step<T, PB>, dim3((unsigned)std::min<int64_t>(items, fwd_cap)), dim3(256), fsm, st, sd,
                       (const int32_t *)pl.d_fblk_desc.data() + ss.fblk0, (int)ss.nrb, (int)K, pl.d_sn_zo.data(),
                       pl.d_sn_start.data(), jb, p, next_tr(1));
        }
    }
    for (int l = pl.nlevels - 1; l >= 0; --l) {
        const SolveDesc *sdl = pl.d_sdescs.data() + pl.lvl_d0[l];
        if (pl.lvl_maxw[l] <= 32 && pl.lvl_maxr[l] <= 512) {  // single narrow, short panels: a warp each
            launch_pdl(k_bwd_narrow<T, PB>, dim3((unsigned)((pl.lvl_nd[l] + 7) / 8), 1, K), dim3(256), 0, st, sdl,
                       pl.lvl_nd[l], pl.d_sn_zo.data(), pl.d_sn_nc.data(), pl.d_sn_start.data(),
                       pl.d_sn_rows_off.data(), pl.d_rows.data(), jb, p, next_tr(2));
        } else {
            launch_pdl(k_bwd_step<T, PB>, dim3((unsigned)pl.lvl_nrbk[l], (pl.lvl_maxw[l] + RBB - 1) / RBB, K),
                       dim3(256), bsm, st, sdl, (const int32_t *)pl.d_lvl_bblk_desc.data() + pl.lvl_bblk0[l],
                       pl.d_sn_zo.data(), pl.d_sn_nc.data(), pl.d_sn_start.data(), pl.d_sn_rows_off.data(),
                       pl.d_rows.data(), jb, (int64_t)pl.lvl_d0[l] * SUBS, p, next_tr(2));
        }
        for (int u = pl.bu_ptr[l]; u < pl.bu_ptr[l + 1]; ++u) {
            const BwdUpd &bu = pl.bupd[u];
            launch_pdl(k_bwd_update<T, PB>, dim3((unsigned)bu.nit, SUBS, K), dim3(256), bsm, st,
                       (const SolveDesc *)pl.d_sdescs.data(), (const int32_t *)pl.d_bu_items.data() + 2 * bu.it0,
                       pl.d_sn_zo.data(), pl.d_sn_start.data(), jb, p, next_tr(3));
        }
    }
}

// The sequence on one factorization's own buffers, with its optional launch trace.
template <class T, int PB>
static void solve_levels_fz(Factorization &fz, int p, cudaStream_t st) {
    Plan &pl = *fz.plan;
    const int ntr = 2 * pl.nlevels + (int)pl.ssteps.size() + (int)pl.bupd.size();
    LaunchTrace *trb = nullptr;
    if (fz.trace_on && fz.trace.size() >= (size_t)ntr) {  // allocated when tracing is switched on
        trb = fz.trace.data();
        k_trace_reset<<<(ntr + 255) / 256, 256, 0, st>>>(trb, ntr);
        MBL_LAUNCH_CHECK();
        fz.trace_kind.clear();
    }
    solve_levels<T, PB>(pl, reinterpret_cast<const SolveBufs<T> *>(fz.dbufs.m.p), 1u, p, trb, &fz.trace_kind, st);
}

template <class T>
static void solve_levels_p(Factorization &fz, int p, cudaStream_t st) {
    switch (rhs_pad(p)) {
        case 8: solve_levels_fz<T, 8>(fz, p, st); break;
        case 16: solve_levels_fz<T, 16>(fz, p, st); break;
        default: solve_levels_fz<T, 32>(fz, p, st); break;
    }
}

// Batched solves: per job k, rows of its right-hand-side block B_k are permuted into its y, the
// level sequence runs over all K jobs (grid z), and the result goes back to X_k.
template <class T>
__global__ void k_perm_in_b(int64_t n, int p, const int32_t *perm, const SolveIO *io, const SolveBufs<T> *jb) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * p) return;
    const int64_t k = idx / p;
    const int q = (int)(idx - k * p);
    const SolveIO &o = io[blockIdx.z];
    jb[blockIdx.z].y[idx] = (T)o.B[(int64_t)perm[k] * o.ldb + q * o.ldbq];
}

template <class T>
__global__ void k_perm_out_b(int64_t n, int p, const int32_t *perm, const SolveIO *io, const SolveBufs<T> *jb) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * p) return;
    const int64_t k = idx / p;
    const int q = (int)(idx - k * p);
    const SolveIO &o = io[blockIdx.z];
    const double v = (double)jb[blockIdx.z].y[idx];
    double *dst = o.X + (int64_t)perm[k] * o.ldx + q * o.ldxq;
    *dst = o.accumulate ? *dst + v : v;
}

template <class T>
static void enqueue_batched_t(const Plan &pl, const void *tab, const SolveIO *io, unsigned K, int p, cudaStream_t st) {
    const SolveBufs<T> *jb = static_cast<const SolveBufs<T> *>(tab);
    const unsigned g = (unsigned)((pl.n * p + 255) / 256);
    k_perm_in_b<T><<<dim3(g, 1, K), 256, 0, st>>>(pl.n, p, pl.d_perm.data(), io, jb);
    MBL_LAUNCH_CHECK();
    switch (rhs_pad(p)) {
        case 8: solve_levels<T, 8>(pl, jb, K, p, nullptr, nullptr, st); break;
        case 16: solve_levels<T, 16>(pl, jb, K, p, nullptr, nullptr, st); break;
        default: solve_levels<T, 32>(pl, jb, K, p, nullptr, nullptr, st); break;
    }
    k_perm_out_b<T><<<dim3(g, 1, K), 256, 0, st>>>(pl.n, p, pl.d_perm.data(), io, jb);
    MBL_LAUNCH_CHECK();
}

void enqueue_batched_solve(const Plan &pl, int prec, const void *tab, const SolveIO *io, unsigned K, int p,
                           cudaStream_t st) {
    if (p < 1 || p > 32 || K < 1 || K > 65535) fail(MBL_ERR_INVALID, "batched solve: bad block width or job count");
    if (prec == MBL_PREC_FP64) enqueue_batched_t<double>(pl, tab, io, K, p, st);
    else enqueue_batched_t<float>(pl, tab, io, K, p, st);
}

template <class T>
static void solve_impl(Factorization &fz, const double *B, int64_t ldb, int64_t ldbq, double *X, int64_t ldx,
                       int64_t ldxq, int p, bool accumulate, cudaStream_t st) {
    Plan &pl = *fz.plan;
    int64_t n = pl.n;
    fz.ensure_solve_work(p);
    set_solve_attrs<T>();
    T *y = static_cast<T *>(fz.ywork.m.p);
    int64_t tot = n * p;
    unsigned g = (unsigned)((tot + 255) / 256);
    ProfScope ps(fz.ctx, sizeof(T) == 8 ? "trisolve_fp64" : "trisolve_fp32",
                 2.0 * (double)(pl.nnz_l + n) * sizeof(T) + 16.0 * (double)n * p, st);
    k_perm_in<T><<<g, 256, 0, st>>>(n, p, pl.d_perm.data(), B, ldb, ldbq, y);
    MBL_LAUNCH_CHECK();
    // the fixed sequence of ~(levels + 4 x solve steps) launches is captured once per block width
    // and replayed as a CUDA graph
    if (fz.graph_p != p) {
        if (fz.graph_exec) {
            cudaGraphExecDestroy(fz.graph_exec);
            fz.graph_exec = nullptr;
        }
        cudaGraph_t graph;
        const long long before = t_launches;
        MBL_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            if (fz.dataflow) solve_dataflow<T>(fz, p, st);
            else solve_levels_p<T>(fz, p, st);
        } catch (...) {
            cudaGraph_t dummy;
            cudaStreamEndCapture(st, &dummy);
            if (dummy) cudaGraphDestroy(dummy);
            throw;
        }
        MBL_CUDA(cudaStreamEndCapture(st, &graph));
        fz.graph_nodes = t_launches - before;
        t_launches = before;
        g_launches.fetch_sub(fz.graph_nodes);  // counted when replayed
        MBL_CUDA(cudaGraphInstantiate(&fz.graph_exec, graph, 0));
        cudaGraphDestroy(graph);
        fz.graph_p = p;
    }
    MBL_CUDA(cudaGraphLaunch(fz.graph_exec, st));
    g_launches.fetch_add(fz.graph_nodes);
    k_perm_out<T><<<g, 256, 0, st>>>(n, p, pl.d_perm.data(), y, X, ldx, ldxq, accumulate ? 1 : 0);
    MBL_LAUNCH_CHECK();
}

void factor_solve_raw(Factorization &fz, const double *B, int64_t ldb, double *X, int64_t ldx, int p, bool accumulate,
                      cudaStream_t st) {
    if (p < 1 || p > 32) fail(MBL_ERR_INVALID, "solve: 1 <= nrhs <= 32 per block");
    if (fz.ctx->batcher && !fz.dataflow && !fz.trace_on) {
        // a serving worker: the solve joins the other workers' solves of the same plan in one launch
        batched_solve(fz.ctx->batcher, fz, B, ldb, X, ldx, p, accumulate, st);
        return;
    }
    if (fz.prec == MBL_PREC_FP64) solve_impl<double>(fz, B, ldb, 1, X, ldx, 1, p, accumulate, st);
    else solve_impl<float>(fz, B, ldb, 1, X, ldx, 1, p, accumulate, st);
}

void factor_solve_colmajor(Factorization &fz, const double *B, double *X, int p, cudaStream_t st) {
    if (p < 1 || p > 32) fail(MBL_ERR_INVALID, "solve: 1 <= nrhs <= 32 per block");
    const int64_t n = fz.plan->n;
    if (fz.prec == MBL_PREC_FP64) solve_impl<double>(fz, B, 1, n, X, 1, n, p, false, st);
    else solve_impl<float>(fz, B, 1, n, X, 1, n, p, false, st);
}

template <class T>
SolveBufs<T> solve_bufs(const Factorization &fz) {
    SolveBufs<T> b;
    b.G = static_cast<const T *>(fz.gpk.m.p);
    b.D = static_cast<const T *>(fz.D.m.p);
    b.Z = static_cast<T *>(fz.zwork.m.p);
    b.Zs = static_cast<T *>(fz.zsolved.m.p);
    b.y = static_cast<T *>(fz.ywork.m.p);
    b.yfw = static_cast<T *>(fz.yfw.m.p);
    b.P = static_cast<T *>(fz.pwork.m.p);
    b.cnt = fz.scnt.data();
    return b;
}
template SolveBufs<float> solve_bufs<float>(const Factorization &);
template SolveBufs<double> solve_bufs<double>(const Factorization &);

template <class T>
static void write_bufs(Factorization &fz) {
    const SolveBufs<T> b = solve_bufs<T>(fz);
    if (fz.dbufs.size() < sizeof(b)) fz.dbufs.alloc(fz.ctx, sizeof(b));
    MBL_CUDA(cudaMemcpyAsync(fz.dbufs.data(), &b, sizeof(b), cudaMemcpyHostToDevice, fz.ctx->stream));
    MBL_CUDA(cudaStreamSynchronize(fz.ctx->stream));
}

void Factorization::ensure_solve_work(int p) {
    if (p <= work_p) return;
    size_t es = elem_size();
    Plan &pl = *plan;
    zwork.alloc(ctx, (size_t)pl.zwork_elems * p * es);
    zsolved.alloc(ctx, (size_t)pl.zwork_elems * p * es);
    ywork.alloc(ctx, (size_t)pl.n * p * es);
    yfw.alloc(ctx, (size_t)pl.n * p * es);
    pwork.alloc(ctx, (size_t)std::max<int64_t>(std::max<int64_t>(pl.max_lvl_nrbk * SUBS, pl.df_pslots), 1) * RBB *
                         rhs_pad(p) * es);
    work_p = p;
    // the device table the level-sequence kernels read (the solve graph is recaptured with it)
    if (prec == MBL_PREC_FP64) write_bufs<double>(*this);
    else write_bufs<float>(*this);
    if (graph_exec) {
        cudaGraphExecDestroy(graph_exec);
        graph_exec = nullptr;
        graph_p = 0;
    }
}

bool arena_is_lean(const Plan &p, int prec, int mode) {
    if (mode == ARENA_LEAN) return true;
    if (mode == ARENA_FULL) return false;
    const double es = prec == MBL_PREC_FP64 ? 8.0 : 4.0;
    return (double)p.arena_elems * es > 8.0 * (double)(1ull << 30);
}

double arena_peak_bytes(const Plan &p, int prec, int mode) {
    const double es = prec == MBL_PREC_FP64 ? 8.0 : 4.0;
    return (arena_is_lean(p, prec, mode) ? (double)p.lean_peak_elems : (double)p.arena_elems) * es;
}

void Factorization::allocate(bool lean_arena) {
    Plan &pl = *plan;
    size_t es = elem_size();
    lean_used = lean_arena;
    if (lean_arena) {
        // the lean arena's chunks come from the device, not the stream-ordered pool: hand the pool's
        // cached free blocks back first
        MBL_CUDA(cudaStreamSynchronize(ctx->stream));
        trim_device_pool(ctx->device);
        lean = std::make_unique<LeanArena>();
        lean->reserve(ctx, pl, es);
    } else {
        arena.alloc(ctx, (size_t)pl.arena_elems * es);
    }
    D.alloc(ctx, (size_t)pl.n * es);
    piv.alloc(ctx, pl.n);
    counters.alloc(ctx, 5);
    wscr.alloc(ctx, (size_t)std::max<int64_t>(pl.wscratch_elems, 1) * es);
    cmax.alloc(ctx, (size_t)std::max<int64_t>(pl.max_desc_per_step, 1) * NB * sizeof(unsigned int));
    M.alloc(ctx, (size_t)std::max<int64_t>(pl.m_elems, 1) * es);
    gpk.alloc(ctx, (size_t)std::max<int64_t>(pl.sg_elems, 1) * es);
    scnt.alloc(ctx, std::max<size_t>(pl.sdescs.size() * SUBS, 1));
    dfcnt.alloc(ctx, (size_t)4 * pl.ns + 2);
    tma = false;
    if (prec == MBL_PREC_FP32 && tc_mode != 0 && pl.wscratch_elems > 0) {
        // operand pieces of the TMA-fed Schur update: 4 arrays of prow rows x NB pieces
        prow = pl.wscratch_elems / NB;
        const size_t eb = tc_mode == 2 ? 2 : 4;
        pieces.alloc(ctx, (size_t)4 * prow * NB * eb);
        tma = encode_pieces_map(tmap, pieces.m.p, prow, tc_mode == 2);
        if (!tma) pieces.release();
    }
    MBL_CUDA(cudaMemset(scnt.data(), 0, std::max<size_t>(pl.sdescs.size() * SUBS, 1) * sizeof(unsigned int)));
}

void reset_solve_counters(Factorization &fz, cudaStream_t st) {
    MBL_CUDA(cudaMemsetAsync(fz.counters.data() + 2, 0, sizeof(unsigned long long), st));
    MBL_CUDA(cudaMemsetAsync(fz.scnt.data(), 0, fz.scnt.size() * sizeof(unsigned int), st));
    MBL_CUDA(cudaStreamSynchronize(st));
}

void Factorization::release_scratch() {
    wscr.release();
    pieces.release();
    cmax.release();
    M.release();      // folded into G = [M; L21 M]
    arena.release();  // the solves read only the packed G and D
    if (lean) {
        MBL_CUDA(cudaStreamSynchronize(ctx->stream));
        lean->release_all(plan.get());
        lean.reset();
    }
}

Factorization::Factorization() = default;

size_t Factorization::held_bytes() const {
    size_t b = 0;
    for (const DevMem *m : {&arena.m, &D.m, &wscr.m, &cmax.m, &M.m, &zwork.m, &zsolved.m, &ywork.m, &yfw.m, &pwork.m,
                            &gpk.m, &piv.m, &scnt.m, &dfcnt.m, &counters.m, &trace.m, &dev_b.m, &dev_x.m, &dbufs.m,
                            &pieces.m})
        b += m->bytes;
    return b;
}

Factorization::~Factorization() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (lean) {
        if (ctx_alive(ctx)) cudaStreamSynchronize(ctx->stream);
        lean->release_all(plan.get());
    }
}

}  // namespace mbl
