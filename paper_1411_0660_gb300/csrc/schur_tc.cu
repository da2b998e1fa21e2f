// schur_tc.cu -- trailing (Schur) update of the frontal matrices on the tcgen05 tensor cores.
//
// The dense contraction of the multifrontal LDL^T (numerical-method section of arXiv:1411.0660,
// through the factorization of H - sigma): C[i][j] -= sum_t L21[i][t] W21[j][t] on the lower
// triangle of the trailing block, K = panel width (<= 64).  FP32 data, FP32 accumulation.  Each
// operand x is split into two pieces x = hi + lo (hi = x rounded to the piece format, lo = x - hi
// rounded too), and three MMAs accumulate hi*hi + hi*lo + lo*hi into a 128 x 128 FP32 tile in
// tensor memory (TMEM).  Two piece formats: TF32 (kind::tf32, 8 k per MMA; about 21 significant bits
// kept) and BF16 (kind::f16 with BF16 operands, 16 k per MMA, twice the tensor rate per operand;
// about 16 bits kept).  One CTA of 256 threads per tile; every memory access that does not depend
// on the MMA is issued first so that their latencies overlap:
//   1. the raw FP32 operand tiles go to shared memory by cp.async, and each thread loads its 64
//      entries of the C tile (row = TMEM lane, half of the columns) into registers;
//   2. the raw tiles are split into hi/lo pieces in the canonical K-major, no-swizzle core-matrix
//      layout (8 rows x 16 bytes per core matrix), then fenced for the tensor core;
//   3. one thread issues 3 MMAs per k step and a tcgen05.commit to an mbarrier;
//   4. all threads wait on the mbarrier (bounded by %globaltimer: on expiry the CTA flags an
//      error, skips its epilogue, frees its TMEM and returns), read the accumulator with
//      tcgen05.ld (warps w and w + 4 share TMEM lanes 32(w mod 4).., each taking 64 columns) and
//      store C - acc, coalesced along the rows.
#include <cuda.h>
#include <mutex>
#include <cuda_bf16.h>

#include "factor.h"

namespace mbl {

namespace {

constexpr int TM = 128, TN = 128, TK = NB;  // tile and maximal K
constexpr uint32_t CORE = 128;               // bytes per core matrix
constexpr uint32_t LBO = CORE;               // next k group
constexpr uint32_t TMEM_COLS = 128;
constexpr int THREADS = 256;

// Piece format: bytes per element, elements per 16-byte k group, k per MMA, instruction descriptor
// (D = F32, A = B = the piece format, both K-major, N = 128, M = 128).
template <bool BF16>
struct Piece {
    static constexpr int EB = BF16 ? 2 : 4;
    static constexpr int EPG = 16 / EB;          // k values per 16-byte group
    static constexpr int KG = TK / EPG;          // 16-byte k groups per row
    static constexpr uint32_t SBO = KG * CORE;   // next 8-row group
    static constexpr uint32_t OPB = TM * TK * EB;  // bytes per operand piece
    static constexpr int KMMA = 2 * EPG;         // k per MMA (two k groups)
    static constexpr uint32_t IDESC = (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) |
                                      ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // fixed 0b001 at bits 46..48; base offset 0, no swizzle
    return d;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// bounded wait on phase `parity` of an mbarrier; returns false on time-out
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint64_t limit_ns) {
    uint64_t t0 = globaltimer();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ int find_desc3t(const PanelDesc *d, int nd, int64_t b) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (d[mid].off3t <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

// hi/lo pieces of 4 (TF32) or 8 (BF16) consecutive k values of one row, packed into 16 bytes
__device__ __forceinline__ void split_group(const float *v, uint4 &hi, uint4 &lo, bool bf16) {
    if (!bf16) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            h[e] = to_tf32(v[e]);
            l[e] = to_tf32(v[e] - __uint_as_float(h[e]));
        }
        hi = make_uint4(h[0], h[1], h[2], h[3]);
        lo = make_uint4(l[0], l[1], l[2], l[3]);
    } else {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * e]), h1 = __float2bfloat16_rn(v[2 * e + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * e] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * e + 1] - __bfloat162float(h1));
            h[e] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            l[e] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        hi = make_uint4(h[0], h[1], h[2], h[3]);
        lo = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

}  // namespace

template <bool BF16>
__global__ void __launch_bounds__(THREADS) k_schur_tc(const PanelDesc *descs, int nd, const int64_t *fo,
                                                      const int32_t *fsz, float *arena, const float *wscr,
                                                      unsigned long long *err) {
    using PC = Piece<BF16>;
    constexpr uint32_t OPB = PC::OPB, SBO = PC::SBO;
    constexpr int KG = PC::KG, EPG = PC::EPG;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    unsigned char *Ahi = sm, *Alo = sm + OPB, *Bhi = sm + 2 * OPB, *Blo = sm + 3 * OPB;
    float *Araw = reinterpret_cast<float *>(sm + 4 * OPB);  // [k][row], TK x TM
    float *Braw = Araw + TK * TM;

    const int di = find_desc3t(descs, nd, blockIdx.x);
    const PanelDesc d = descs[di];
    const int s = d.front, f = fsz[s], k0 = d.k0, w = d.w, m2 = d.m2;
    const int64_t t = (int64_t)blockIdx.x - d.off3t;
    int bi = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(bi + 1) * (bi + 2) / 2 <= t) ++bi;
    while ((int64_t)bi * (bi + 1) / 2 > t) --bi;
    const int bj = (int)(t - (int64_t)bi * (bi + 1) / 2);
    const int base = k0 + w;
    const int i0 = base + bi * TM, j0 = base + bj * TN;
    float *F = arena + fo[s];
    const float *W = wscr + d.woff;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, half = warp >> 2;

    // 1a. raw operands: A = L21 rows i0.. (front columns k0..k0+w), B = W21 rows j0.. (ld m2)
    const int rowsA = min(TM, f - i0), rowsB = min(TN, f - j0);
    for (int idx = threadIdx.x; idx < TK * TM; idx += THREADS) {
        const int k = idx / TM, r = idx % TM;
        float *da = Araw + idx, *db = Braw + idx;
        if (k < w && r < rowsA) cp_async4(da, F + (int64_t)(k0 + k) * f + i0 + r);
        else *da = 0.0f;
        if (k < w && r < rowsB) cp_async4(db, W + (int64_t)k * m2 + (j0 - base) + r);
        else *db = 0.0f;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    // 1b. this thread's part of C: row gi, columns j0 + 64 half + c (lower triangle only)
    const int gi = i0 + quarter * 32 + lane;
    float cv[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) {
        const int gj = j0 + 64 * half + c;
        cv[c] = (gi < f && gj < f && gi >= gj) ? F[(int64_t)gj * f + gi] : 0.0f;
    }
    // TMEM accumulator (one warp allocates) and the completion barrier
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // 2. hi/lo pieces in the canonical layout, one 16-byte core-matrix row per unit
    for (int u = threadIdx.x; u < TM * KG; u += THREADS) {
        const int r = u % TM, c = u / TM;
        const uint32_t off = (uint32_t)(r >> 3) * SBO + (uint32_t)(r & 7) * 16u + (uint32_t)c * CORE;
        float va[EPG], vb[EPG];
#pragma unroll
        for (int e = 0; e < EPG; ++e) {
            va[e] = Araw[(EPG * c + e) * TM + r];
            vb[e] = Braw[(EPG * c + e) * TM + r];
        }
        uint4 hi, lo;
        split_group(va, hi, lo, BF16);
        *reinterpret_cast<uint4 *>(Ahi + off) = hi;
        *reinterpret_cast<uint4 *>(Alo + off) = lo;
        split_group(vb, hi, lo, BF16);
        *reinterpret_cast<uint4 *>(Bhi + off) = hi;
        *reinterpret_cast<uint4 *>(Blo + off) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // 3. the MMAs
    if (threadIdx.x == 0) {
        const int ksteps = (w + PC::KMMA - 1) / PC::KMMA;
        uint32_t acc = 0;
        for (int ks = 0; ks < ksteps; ++ks) {
            const uint32_t koff = (uint32_t)ks * 2u * CORE;  // two k groups per MMA
            const uint64_t ah = sdesc(smem_u32(Ahi) + koff, SBO), al = sdesc(smem_u32(Alo) + koff, SBO);
            const uint64_t bh = sdesc(smem_u32(Bhi) + koff, SBO), bl = sdesc(smem_u32(Blo) + koff, SBO);
            const uint64_t as[3] = {ah, ah, al}, bs[3] = {bh, bl, bh};
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                if (BF16)
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(as[u]), "l"(bs[u]), "r"(PC::IDESC), "r"(acc));
                else
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(as[u]), "l"(bs[u]), "r"(PC::IDESC), "r"(acc));
                acc = 1;
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(&mbar))
                     : "memory");
    }
    // 4. bounded wait, then C - acc for this thread's row and 64 columns
    const bool ok = mbar_wait(smem_u32(&mbar), 0, 2000000000ull);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!ok) {
        if (lane == 0) atomicAdd(err, 1ull);
        mbar_wait(smem_u32(&mbar), 0, 2000000000ull);  // give the in-flight MMAs a second chance
    } else {
#pragma unroll
        for (int jc = 0; jc < 64; jc += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(64 * half + jc), r);
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const int gj = j0 + 64 * half + jc + c;
                if (gi < f && gj < f && gi >= gj) F[(int64_t)gj * f + gi] = cv[jc + c] - __uint_as_float(r[c]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---------------------------------------------------------------------------------------------
// TMA-fed form.  The panel's trsm has written the hi/lo pieces of L21 (pieces 0, 1) and W21 (2, 3)
// row-major, NB pieces per row, rows at the descriptor's woff / NB.  A 4-D tensor map views them as
// (16-byte k group elements, rows, k groups, pieces) with strides (row = NB pieces, k group = 16 bytes,
// piece = the array), so that one cp.async.bulk.tensor per operand (box: a k group x 128 rows x every
// k group x 2 pieces) lands the two pieces of a 128-row tile in the canonical K-major, no-swizzle
// core-matrix layout the MMA reads: k groups 128 x 16 = 2048 bytes apart (LBO), 8-row groups 128 bytes
// apart (SBO).  One thread arms an mbarrier with the expected bytes and issues both copies; meanwhile
// every thread loads its part of C into registers; the MMAs follow as in k_schur_tc.
template <bool BF16>
struct TmaPiece {
    static constexpr int EB = BF16 ? 2 : 4;
    static constexpr int EPG = 16 / EB;              // elements per 16-byte k group
    static constexpr int KG = NB / EPG;              // k groups per row
    static constexpr uint32_t OPB = 128u * NB * EB;  // bytes per piece of a 128-row tile
    static constexpr uint32_t LBO_T = 128u * 16u;    // next k group
    static constexpr uint32_t SBO_T = 128u;          // next 8-row group
    static constexpr int KMMA = 2 * EPG;
};

__device__ __forceinline__ uint64_t sdesc2(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // fixed 0b001 at bits 46..48; base offset 0, no swizzle
    return d;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void *tmap, int c0, int c1, int c2, int c3,
                                            uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}

template <bool BF16>
__global__ void __launch_bounds__(THREADS) k_schur_tma(const __grid_constant__ CUtensorMap pieces,
                                                       const PanelDesc *descs, int nd, const int64_t *fo,
                                                       const int32_t *fsz, float *arena, unsigned long long *err) {
    using PC = TmaPiece<BF16>;
    constexpr uint32_t OPB = PC::OPB;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar_ld, mbar_mma;
    __shared__ uint32_t tmem_slot;
    unsigned char *Apc = sm, *Bpc = sm + 2 * OPB;  // [piece][k group][row][16 bytes]

    const int di = find_desc3t(descs, nd, blockIdx.x);
    const PanelDesc d = descs[di];
    const int s = d.front, f = fsz[s], k0 = d.k0, w = d.w;
    const int64_t t = (int64_t)blockIdx.x - d.off3t;
    int bi = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(bi + 1) * (bi + 2) / 2 <= t) ++bi;
    while ((int64_t)bi * (bi + 1) / 2 > t) --bi;
    const int bj = (int)(t - (int64_t)bi * (bi + 1) / 2);
    const int base = k0 + w;
    const int i0 = base + bi * TM, j0 = base + bj * TN;
    float *F = arena + fo[s];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int row0 = (int)(d.woff / NB);

    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar_ld)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(&mbar_ld)),
                     "r"(4u * OPB)
                     : "memory");
        tma_load_4d(smem_u32(Apc), &pieces, 0, row0 + bi * TM, 0, 0, smem_u32(&mbar_ld));
        tma_load_4d(smem_u32(Bpc), &pieces, 0, row0 + bj * TN, 0, 2, smem_u32(&mbar_ld));
    }
    // this thread's part of C: row gi, columns j0 + 64 half + c (lower triangle only)
    const int gi = i0 + quarter * 32 + lane;
    float cv[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) {
        const int gj = j0 + 64 * half + c;
        cv[c] = (gi < f && gj < f && gi >= gj) ? F[(int64_t)gj * f + gi] : 0.0f;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    // operands landed (bounded wait); then one thread issues the MMAs
    bool ok = mbar_wait(smem_u32(&mbar_ld), 0, 2000000000ull);
    if (threadIdx.x == 0 && ok) {
        const int ksteps = (w + PC::KMMA - 1) / PC::KMMA;
        uint32_t acc = 0;
        for (int ks = 0; ks < ksteps; ++ks) {
            const uint32_t koff = (uint32_t)ks * 2u * PC::LBO_T;  // two k groups per MMA
            const uint64_t ah = sdesc2(smem_u32(Apc) + koff, PC::LBO_T, PC::SBO_T);
            const uint64_t al = sdesc2(smem_u32(Apc) + OPB + koff, PC::LBO_T, PC::SBO_T);
            const uint64_t bh = sdesc2(smem_u32(Bpc) + koff, PC::LBO_T, PC::SBO_T);
            const uint64_t bl = sdesc2(smem_u32(Bpc) + OPB + koff, PC::LBO_T, PC::SBO_T);
            const uint64_t as[3] = {ah, ah, al}, bs[3] = {bh, bl, bh};
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                if (BF16)
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(as[u]), "l"(bs[u]), "r"(Piece<true>::IDESC), "r"(acc));
                else
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(as[u]), "l"(bs[u]), "r"(Piece<false>::IDESC), "r"(acc));
                acc = 1;
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(&mbar_mma))
                     : "memory");
    }
    if (ok) ok = mbar_wait(smem_u32(&mbar_mma), 0, 2000000000ull);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!ok) {
        // a wait expired: flag it, give the copies and MMAs in flight a second bounded wait, skip the
        // epilogue
        if (lane == 0) atomicAdd(err, 1ull);
        mbar_wait(smem_u32(&mbar_ld), 0, 2000000000ull);
        if (threadIdx.x == 0) mbar_wait(smem_u32(&mbar_mma), 0, 2000000000ull);
    } else {
#pragma unroll
        for (int jc = 0; jc < 64; jc += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(64 * half + jc), r);
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const int gj = j0 + 64 * half + jc + c;
                if (gi < f && gj < f && gi >= gj) F[(int64_t)gj * f + gi] = cv[jc + c] - __uint_as_float(r[c]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

size_t schur_tc_smem(bool bf16) {
    return 4 * (size_t)(bf16 ? Piece<true>::OPB : Piece<false>::OPB) + 2 * (size_t)TK * TM * sizeof(float);
}

size_t schur_tma_smem(bool bf16) { return 4 * (size_t)(bf16 ? TmaPiece<true>::OPB : TmaPiece<false>::OPB); }

bool encode_pieces_map(void *map, void *pieces, int64_t prow, bool bf16) {
    using Encode = decltype(&::cuTensorMapEncodeTiled);
    static Encode enc = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        (void)cudaGetLastError();
        return reinterpret_cast<Encode>(fn);
    }();
    if (!enc || !pieces || prow < 1) return false;
    const int eb = bf16 ? 2 : 4, epg = 16 / eb;
    cuuint64_t dims[4] = {(cuuint64_t)epg, (cuuint64_t)prow, (cuuint64_t)(NB / epg), 4};
    cuuint64_t strides[3] = {(cuuint64_t)NB * eb, 16, (cuuint64_t)prow * NB * eb};
    cuuint32_t box[4] = {(cuuint32_t)epg, (cuuint32_t)TM, (cuuint32_t)(NB / epg), 2};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = enc(static_cast<CUtensorMap *>(map),
                           bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, pieces,
                           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

void launch_schur_tma(const PanelStep &stp, const PanelDesc *d_descs, const int64_t *fo, const int32_t *fsz,
                      float *arena, const void *map, unsigned long long *err, cudaStream_t st, bool bf16) {
    static std::mutex mu;
    static bool ready[64] = {};
    int dev = 0;
    MBL_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 0 || dev >= 64 || !ready[dev]) {
            MBL_CUDA(cudaFuncSetAttribute(k_schur_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)schur_tma_smem(false)));
            MBL_CUDA(cudaFuncSetAttribute(k_schur_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)schur_tma_smem(true)));
            if (dev >= 0 && dev < 64) ready[dev] = true;
        }
    }
    const CUtensorMap &m = *static_cast<const CUtensorMap *>(map);
    if (bf16)
        k_schur_tma<true><<<(unsigned)stp.n3t, THREADS, schur_tma_smem(true), st>>>(m, d_descs, stp.nd, fo, fsz, arena,
                                                                                     err);
    else
        k_schur_tma<false><<<(unsigned)stp.n3t, THREADS, schur_tma_smem(false), st>>>(m, d_descs, stp.nd, fo, fsz,
                                                                                       arena, err);
    MBL_LAUNCH_CHECK();
}

void launch_schur_tc(const PanelStep &stp, const PanelDesc *d_descs, const Plan &p, float *arena, const float *wscr,
                     unsigned long long *err, cudaStream_t st, bool bf16) {
    smem_limit((const void *)k_schur_tc<false>, schur_tc_smem(false));
    smem_limit((const void *)k_schur_tc<true>, schur_tc_smem(true));
    if (bf16)
        k_schur_tc<true><<<(unsigned)stp.n3t, THREADS, schur_tc_smem(true), st>>>(
            d_descs, stp.nd, p.d_sn_fo.data(), p.d_sn_f.data(), arena, wscr, err);
    else
        k_schur_tc<false><<<(unsigned)stp.n3t, THREADS, schur_tc_smem(false), st>>>(
            d_descs, stp.nd, p.d_sn_fo.data(), p.d_sn_f.data(), arena, wscr, err);
    MBL_LAUNCH_CHECK();
}

}  // namespace mbl
