// Float-float accumulation: a sum kept as an unevaluated pair hi + lo of
// single-precision numbers, built from error-free transformations (Knuth's
// TwoSum for additions, the fused multiply-add residual for products).  It
// carries about twice single precision while running on the FP32 pipe, which
// on this GPU is far faster than the FP64 one; only the final value is
// converted to double.  The explicit _rn intrinsics keep the compiler from
// contracting or reordering the transformations.
#pragma once
#include <cuda_runtime.h>

namespace dnsk {

// (hi, lo) += (bh, bl)
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
    const float s = __fadd_rn(hi, bh);
    const float v = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(bh, v));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, bl));
}

// (hi, lo) += a * b, the product taken exactly as p + fma(a, b, -p)
__device__ __forceinline__ void ff_add_prod(float& hi, float& lo, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    ff_add(hi, lo, p, pe);
}

// (hi, lo) += (a + al) * (b + bl) for operands held as single-precision
// pairs (|al| <= ulp(a) / 2, |bl| <= ulp(b) / 2): the leading product exactly
// as above, the two cross terms into lo (their own rounding is far below
// single precision of the sum); al * bl is dropped
__device__ __forceinline__ void ff_add_prod2(float& hi, float& lo, float a, float b, float al, float bl) {
    ff_add_prod(hi, lo, a, b);
    lo = __fmaf_rn(a, bl, lo);
    lo = __fmaf_rn(al, b, lo);
}

// butterfly over the warp; lane 0's result is used (a fixed order)
__device__ __forceinline__ void ff_warp_sum(float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l = __shfl_xor_sync(0xffffffffu, lo, o);
        ff_add(hi, lo, h, l);
    }
}

// Two CTA-wide float-float sums.  Per-warp partials go through `red` (4 x 32
// floats of shared memory); warp 0 combines them in a fixed order and thread 0
// returns both sums as doubles.  Contains one barrier; every thread calls it.
__device__ __forceinline__ void ff_block_sum2(float h1, float l1, float h2, float l2, float* red,
                                              double* s1, double* s2) {
    ff_warp_sum(h1, l1);
    ff_warp_sum(h2, l2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        red[4 * warp] = h1;
        red[4 * warp + 1] = l1;
        red[4 * warp + 2] = h2;
        red[4 * warp + 3] = l2;
    }
    __syncthreads();
    if (warp == 0) {
        h1 = lane < nw ? red[4 * lane] : 0.f;
        l1 = lane < nw ? red[4 * lane + 1] : 0.f;
        h2 = lane < nw ? red[4 * lane + 2] : 0.f;
        l2 = lane < nw ? red[4 * lane + 3] : 0.f;
        ff_warp_sum(h1, l1);
        ff_warp_sum(h2, l2);
        if (lane == 0) {
            *s1 = (double)h1 + (double)l1;
            *s2 = (double)h2 + (double)l2;
        }
    }
}

}  // namespace dnsk
