// tc_pieces.cuh -- splitting FP32 values into two tensor-core operand pieces, x ~ hi + lo.
//
// The trailing (Schur) update of the FP32 fronts runs on the tcgen05 tensor cores as three products
// of pieces, hi*hi + hi*lo + lo*hi, accumulated in FP32.  Two piece formats: TF32 (19-bit pieces in
// 32-bit containers, rounded to nearest with ties away from zero) and BF16.  The panel's trsm writes
// the pieces of L21 and W21 once per panel, row-major with NB pieces per row (zero past the panel
// width), so that the update loads them with the tensor memory accelerator.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace mbl {

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// TF32 pieces of x: hi and lo as 32-bit containers
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = tf32_bits(x);
    lo = tf32_bits(x - __uint_as_float(hi));
}

// BF16 pieces of x
__device__ __forceinline__ void split_bf16(float x, uint16_t &hi, uint16_t &lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}

}  // namespace mbl
