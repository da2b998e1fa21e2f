// solve_tile.cuh -- device pieces shared by the level-by-level (factor.cu) and the dataflow
// (solve_df.cu) triangular solves: 16-byte asynchronous copies out of the packed solve factor, the
// product of one backward tile and the final reduction of a backward panel's partial sums.
//
// Backward tile: RBK rows x RBB columns of a solve panel's G = [M; L21 M] (packed column-major,
// every column 16-byte aligned, zero padding rows), times v = [y_panel; -x_below] (RBK x PB).
#pragma once

#include "plan.h"

namespace mbl {

template <class T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static __device__ __forceinline__ float get(const float4 &v, int e) {
        return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
    }
};
template <>
struct Vec16<double> {
    using type = double2;
    static __device__ __forceinline__ double get(const double2 &v, int e) { return e == 0 ? v.x : v.y; }
};

// Column stride of a backward tile in shared memory: RBK rows plus a pad that puts the 16-byte
// reads of eight consecutive columns on distinct bank groups (stride / (16 / sizeof(T)) odd).
template <class T>
__host__ __device__ constexpr int bwd_ldg() {
    return sizeof(T) == 4 ? RBK + 4 : RBK + 2;
}

// Shared memory of a backward step: the G tile, v, and (for more than 8 right-hand sides) the
// cross-warp partial sums, which otherwise reuse the G tile.
template <class T, int PB>
__host__ __device__ constexpr size_t bwd_tile_smem() {
    return sizeof(T) * ((size_t)RBB * bwd_ldg<T>() + (size_t)RBK * PB + (PB == 8 ? 0 : (size_t)64 * RBB));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Issue the copies of a backward tile: columns [0, wc) x 16-byte row groups [0, nrv) of G (column
// stride ld; G and ld 16-byte aligned) into Gs (column stride bwd_ldg<T>()).
template <class T>
__device__ __forceinline__ void bwd_tile_issue(T *Gs, const T *G, int64_t ld, int wc, int nrv) {
    constexpr int E = 16 / sizeof(T), LDG = bwd_ldg<T>();
    for (int idx = threadIdx.x; idx < wc * nrv; idx += blockDim.x) {
        const int c = idx / nrv, v = idx - c * nrv;
        cp_async16(Gs + c * LDG + v * E, G + (int64_t)c * ld + (int64_t)v * E);
    }
}

// Partial products of a backward tile for right-hand sides [q0, q0 + 8): warp j takes rows
// [32 j, 32 j + 32) below nrows (a whole number of 16-byte row groups; the rows of vs past the
// panel are zero), lane l takes columns l and l + 32.  The eight warps' sums meet in red
// (8 x 8 x RBB; it may alias Gs, so the call starts with a barrier) and thread t returns the
// outputs o = t and t + 256 (q = q0 + o / RBB, c = o % RBB) in out[0], out[1].  256 threads.
template <class T, int PB>
__device__ __forceinline__ void bwd_tile_product(const T *Gs, const T *vs, T *red, int nrows, int q0, T out[2]) {
    constexpr int E = 16 / sizeof(T), LDG = bwd_ldg<T>();
    using V = typename Vec16<T>::type;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int i0 = wp * 32, i1 = min(i0 + 32, nrows);
    T a0[8], a1[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a0[q] = a1[q] = T(0);
    for (int i = i0; i < i1; i += E) {
        const V g0 = *reinterpret_cast<const V *>(Gs + lane * LDG + i);
        const V g1 = *reinterpret_cast<const V *>(Gs + (lane + 32) * LDG + i);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const T ga = Vec16<T>::get(g0, e), gb = Vec16<T>::get(g1, e);
            const V *vr = reinterpret_cast<const V *>(vs + (i + e) * PB + q0);
#pragma unroll
            for (int u = 0; u < 8 / E; ++u) {
                const V vv = vr[u];
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const T vk = Vec16<T>::get(vv, k);
                    a0[u * E + k] += ga * vk;
                    a1[u * E + k] += gb * vk;
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        red[(wp * 8 + q) * RBB + lane] = a0[q];
        red[(wp * 8 + q) * RBB + lane + 32] = a1[q];
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int o = threadIdx.x + 256 * h, q = o / RBB, c = o % RBB;
        T v = T(0);
#pragma unroll
        for (int j = 0; j < 8; ++j) v += red[(j * 8 + q) * RBB + c];
        out[h] = v;
    }
}

// Last block of a (panel, column chunk): add the nb partial tiles ([q][c], RBB x PB each, stride
// apart) in a fixed order and write the result -- columns c < wc, right-hand sides q < p -- to
// zs[c p + q] and, unless xo is null, xo[c p + q].  comb: scratch of 2 x RBB x PB in shared memory.
// 256 threads.
template <class T, int PB>
__device__ void bwd_finish(const T *src, int64_t stride, int nb, int wc, int p, T *zs, T *xo, T *comb) {
    constexpr int E = 16 / sizeof(T), NV = RBB * PB / E;
    constexpr int NG = NV >= 256 ? 1 : 256 / NV;  // groups of partial tiles summed separately
    using V = typename Vec16<T>::type;
    const int g = NG > 1 ? (int)threadIdx.x / NV : 0;
    const int v0 = NG > 1 ? (int)threadIdx.x % NV : (int)threadIdx.x, vstep = NG > 1 ? NV : 256;
    for (int vi = v0; vi < NV; vi += vstep) {
        T acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = T(0);
#pragma unroll 8
        for (int bb = g; bb < nb; bb += NG) {
            const V v = __ldcg(reinterpret_cast<const V *>(src + (int64_t)bb * stride) + vi);
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] += Vec16<T>::get(v, e);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int o = vi * E + e;
            if (NG > 1) {
                comb[g * RBB * PB + o] = acc[e];
            } else {
                const int q = o / RBB, c = o % RBB;
                if (c < wc && q < p) {
                    zs[c * p + q] = acc[e];
                    if (xo) xo[c * p + q] = acc[e];
                }
            }
        }
    }
    if (NG > 1) {
        __syncthreads();
        for (int o = threadIdx.x; o < RBB * PB; o += blockDim.x) {
            T v = T(0);
            for (int gg = 0; gg < NG; ++gg) v += comb[gg * RBB * PB + o];
            const int q = o / RBB, c = o % RBB;
            if (c < wc && q < p) {
                zs[c * p + q] = v;
                if (xo) xo[c * p + q] = v;
            }
        }
    }
}

}  // namespace mbl
